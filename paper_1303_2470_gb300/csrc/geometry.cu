// geometry.cu -- node classification of a medium (solid S, fluid F, interfacial I subset of
// F: fluid nodes with at least one solid D3Q19 neighbour; paper Sec. "Algorithm", the three
// node classes of the Boltzmann weights) packed into per-32-node bit words, plus the
// exclusive prefix and the sorted list of interfacial nodes used to address the compact
// adsorbed-population arrays.
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.cuh"

namespace mp {

namespace {

thread_local std::string g_last_error;

// one thread per node; a warp covers one 32-node word
__global__ void k_classify(const uint8_t* __restrict__ solid, int nx, int ny, int nz, int N, int W,
                           uint32_t* __restrict__ fluid_w, uint32_t* __restrict__ iface_w)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    bool fl = false, itf = false;
    if (n < N) {
        fl = solid[n] == 0;
        if (fl) {
            int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                int xs = x + cx(i), ys = y + cy(i), zs = z + cz(i);
                xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
                zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
                itf |= solid[xs + nx * (ys + ny * zs)] != 0;
            }
        }
    }
    unsigned bf = __ballot_sync(0xffffffffu, fl);
    unsigned bi = __ballot_sync(0xffffffffu, itf);
    int w = n >> 5;
    if ((threadIdx.x & 31) == 0 && w < W) {
        fluid_w[w] = bf;
        iface_w[w] = bi;
    }
}

// single block: exclusive prefix of popc(iface_w) into ibase, and the two totals
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
    k_scan(const uint32_t* __restrict__ fluid_w, const uint32_t* __restrict__ iface_w, int W,
           int32_t* __restrict__ ibase, long long* __restrict__ totals)
{
    __shared__ long long s_i[kScanThreads / 32], s_f[kScanThreads / 32];
    int per = (W + kScanThreads - 1) / kScanThreads;
    int lo = threadIdx.x * per;
    int hi = min(W, lo + per);
    long long ci = 0, cf = 0;
    for (int w = lo; w < hi; ++w) {
        ci += __popc(iface_w[w]);
        cf += __popc(fluid_w[w]);
    }
    // inclusive warp scan of ci, warp sum of cf
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = ci, sf = cf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
        sf += __shfl_xor_sync(0xffffffffu, sf, o);
    }
    if (lane == 31) s_i[warp] = inc;
    if (lane == 0) s_f[warp] = sf;
    __syncthreads();
    long long before = 0, tot_i = 0, tot_f = 0;
    for (int k = 0; k < kScanThreads / 32; ++k) {
        if (k < warp) before += s_i[k];
        tot_i += s_i[k];
        tot_f += s_f[k];
    }
    long long excl = before + inc - ci;
    for (int w = lo; w < hi; ++w) {
        ibase[w] = (int32_t)excl;
        excl += __popc(iface_w[w]);
    }
    if (threadIdx.x == 0) {
        totals[0] = tot_f;
        totals[1] = tot_i;
    }
}

__global__ void k_list(const uint32_t* __restrict__ iface_w, const int32_t* __restrict__ ibase, int N,
                       int32_t* __restrict__ ilist)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    uint32_t bits = iface_w[n >> 5];
    int b = n & 31;
    if ((bits >> b) & 1u) ilist[ibase[n >> 5] + __popc(bits & ((1u << b) - 1u))] = n;
}

template <typename T>
int dev_alloc(T** p, size_t count, cudaStream_t s, bool stream_ordered)
{
    cudaError_t e = stream_ordered ? cudaMallocAsync((void**)p, count * sizeof(T), s)
                                   : cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
        return MP_ENOMEM;
    }
    return MP_OK;
}

template <typename T>
void dev_free(T*& p, cudaStream_t s, bool stream_ordered)
{
    if (p) {
        if (stream_ordered)
            cudaFreeAsync(p, s);
        else
            cudaFree(p);
    }
    p = nullptr;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
const char* last_error_text() { return g_last_error.c_str(); }

int cuda_fail(cudaError_t e, const char* what)
{
    set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return MP_ENOMEM;
    return MP_ECUDA;
}

void free_geometry(Geometry* g, cudaStream_t s, bool so)
{
    dev_free(g->fluid, s, so);
    dev_free(g->iface, s, so);
    dev_free(g->ibase, s, so);
    dev_free(g->ilist, s, so);
}

int build_geometry(const mp_geometry* g, cudaStream_t s, bool so, bool want_list, Geometry* out)
{
    if (!g || !g->solid) {
        set_error("geometry or its solid mask is NULL");
        return MP_EINVAL;
    }
    if (g->nx < 3 || g->ny < 3 || g->nz < 3) {
        set_error("every lattice dimension must be >= 3");
        return MP_EINVAL;
    }
    long long N = (long long)g->nx * g->ny * g->nz;
    if (N >= (1LL << 31) - 64) {
        set_error("lattice too large: nx*ny*nz must be < 2^31");
        return MP_EINVAL;
    }
    if (g->location != MP_HOST && g->location != MP_DEVICE) {
        set_error("geometry location must be MP_HOST or MP_DEVICE");
        return MP_EINVAL;
    }
    Geometry G;
    G.nx = g->nx;
    G.ny = g->ny;
    G.nz = g->nz;
    G.N = (int)N;
    G.W = (int)((N + 31) / 32);
    int rc;
    uint8_t* solid_d = nullptr;
    long long* totals = nullptr;
    if ((rc = dev_alloc(&G.fluid, G.W, s, so)) || (rc = dev_alloc(&G.iface, G.W, s, so)) ||
        (rc = dev_alloc(&G.ibase, G.W, s, so)) || (rc = dev_alloc(&totals, 2, s, so))) {
        free_geometry(&G, s, so);
        dev_free(totals, s, so);
        return rc;
    }
    const uint8_t* solid = g->solid;
    if (g->location == MP_HOST) {
        if ((rc = dev_alloc(&solid_d, (size_t)N, s, so))) {
            free_geometry(&G, s, so);
            dev_free(totals, s, so);
            return rc;
        }
        cudaError_t e = cudaMemcpyAsync(solid_d, g->solid, (size_t)N, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            free_geometry(&G, s, so);
            dev_free(totals, s, so);
            dev_free(solid_d, s, so);
            return cuda_fail(e, "cudaMemcpyAsync(solid)");
        }
        solid = solid_d;
    }
    int threads = 256;
    int blocks = (int)(((long long)G.W * 32 + threads - 1) / threads);
    k_classify<<<blocks, threads, 0, s>>>(solid, G.nx, G.ny, G.nz, G.N, G.W, G.fluid, G.iface);
    k_scan<<<1, kScanThreads, 0, s>>>(G.fluid, G.iface, G.W, G.ibase, totals);
    long long h_tot[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_tot, totals, sizeof(h_tot), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(solid_d, s, so);
    dev_free(totals, s, so);
    if (e != cudaSuccess) {
        free_geometry(&G, s, so);
        return cuda_fail(e, "geometry classification");
    }
    G.n_fluid = h_tot[0];
    G.n_iface = h_tot[1];
    if (want_list && G.n_iface > 0) {
        if ((rc = dev_alloc(&G.ilist, (size_t)G.n_iface, s, so))) {
            free_geometry(&G, s, so);
            return rc;
        }
        k_list<<<(G.N + 255) / 256, 256, 0, s>>>(G.iface, G.ibase, G.N, G.ilist);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            free_geometry(&G, s, so);
            return cuda_fail(e, "interface list");
        }
    }
    *out = G;
    return MP_OK;
}

}  // namespace mp
