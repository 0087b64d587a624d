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

// single block: exclusive prefixes of popc(iface_w) into ibase and of popc(fluid_w) into
// fbase, and the two totals
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
    k_scan(const uint32_t* __restrict__ fluid_w, const uint32_t* __restrict__ iface_w, int W,
           int32_t* __restrict__ ibase, int32_t* __restrict__ fbase, long long* __restrict__ totals)
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
    // the same for the fluid bits (second pass over this thread's words)
    __syncthreads();
    long long incf = cf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long v = __shfl_up_sync(0xffffffffu, incf, o);
        if (lane >= o) incf += v;
    }
    if (lane == 31) s_i[warp] = incf;
    __syncthreads();
    long long beforef = 0;
    for (int k = 0; k < warp; ++k) beforef += s_i[k];
    long long exclf = beforef + incf - cf;
    for (int w = lo; w < hi; ++w) {
        fbase[w] = (int32_t)exclf;
        exclf += __popc(fluid_w[w]);
    }
    if (threadIdx.x == 0) {
        totals[0] = tot_f;
        totals[1] = tot_i;
    }
}

__global__ void k_list(const uint32_t* __restrict__ bits_w, const int32_t* __restrict__ base, int N,
                       int32_t* __restrict__ list)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    uint32_t bits = bits_w[n >> 5];
    int b = n & 31;
    if ((bits >> b) & 1u) list[base[n >> 5] + __popc(bits & ((1u << b) - 1u))] = n;
}

// Connected components by monotone min-label propagation: every fluid node starts with its
// own index and repeatedly takes the smallest label among itself, its label's label
// (pointer jumping) and its fluid D3Q19 neighbours. Labels only decrease and always name a
// node of the same cluster, so races between threads only delay convergence; the fixed
// point is the smallest node index of each cluster, whatever the schedule.
__global__ void k_cc_init(const uint32_t* __restrict__ fluid_w, int N, int* __restrict__ label)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N) label[n] = ((fluid_w[n >> 5] >> (n & 31)) & 1u) ? n : 0x7fffffff;
}

__global__ void k_cc_sweep(const uint32_t* __restrict__ fluid_w, int nx, int ny, int nz, int N, int* label,
                           int* __restrict__ changed)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N || !((fluid_w[n >> 5] >> (n & 31)) & 1u)) return;
    volatile int* lab = label;
    int cur = lab[n];
    int l = cur;
    int l2 = lab[l];
    if (l2 < l) l = l2;
    int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        int xs = x + cx(i), ys = y + cy(i), zs = z + cz(i);
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        int m = xs + nx * (ys + ny * zs);
        if ((fluid_w[m >> 5] >> (m & 31)) & 1u) {
            int lm = lab[m];
            if (lm < l) l = lm;
        }
    }
    if (l < cur) {
        atomicMin(label + n, l);
        *changed = 1;
    }
}

__global__ void k_cc_count(const uint32_t* __restrict__ fluid_w, int N, const int* __restrict__ label,
                           int* __restrict__ count)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < N && ((fluid_w[n >> 5] >> (n & 31)) & 1u)) atomicAdd(count + label[n], 1);
}

// key = size << 32 | (0xffffffff - root): the maximum is the largest cluster, ties to the
// smallest root index
__global__ void k_cc_best(const int* __restrict__ count, int N, unsigned long long* __restrict__ best)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = 0ull;
    if (n < N && count[n] > 0) key = ((unsigned long long)count[n] << 32) | (0xffffffffull - (unsigned)n);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, key, o);
        key = v > key ? v : key;
    }
    if ((threadIdx.x & 31) == 0 && key) atomicMax(best, key);
}

__global__ void k_cc_mark(const uint32_t* __restrict__ fluid_w, int N, int W, const int* __restrict__ label,
                          const unsigned long long* __restrict__ best, uint32_t* __restrict__ cluster_w)
{
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int root = (int)(0xffffffffull - (*best & 0xffffffffull));
    bool in = n < N && ((fluid_w[n >> 5] >> (n & 31)) & 1u) && label[n] == root;
    unsigned b = __ballot_sync(0xffffffffu, in);
    if ((threadIdx.x & 31) == 0 && (n >> 5) < W) cluster_w[n >> 5] = b;
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
    dev_free(g->cluster, s, so);
    dev_free(g->fluid, s, so);
    dev_free(g->iface, s, so);
    dev_free(g->ibase, s, so);
    dev_free(g->ilist, s, so);
    dev_free(g->fbase, s, so);
    dev_free(g->flist, s, so);
}

int build_cluster(Geometry* G, cudaStream_t s, bool so)
{
    int* label = nullptr;
    int* count = nullptr;
    int* changed = nullptr;
    unsigned long long* best = nullptr;
    int rc;
    if ((rc = dev_alloc(&G->cluster, G->W, s, so)) || (rc = dev_alloc(&label, G->N, s, so)) ||
        (rc = dev_alloc(&count, G->N, s, so)) || (rc = dev_alloc(&changed, 1, s, so)) ||
        (rc = dev_alloc(&best, 1, s, so))) {
        dev_free(label, s, so);
        dev_free(count, s, so);
        dev_free(changed, s, so);
        dev_free(best, s, so);
        return rc;
    }
    const int threads = 256, blocks = (G->N + threads - 1) / threads;
    const int wblocks = (int)(((long long)G->W * 32 + threads - 1) / threads);
    cudaError_t e = cudaSuccess;
    k_cc_init<<<blocks, threads, 0, s>>>(G->fluid, G->N, label);
    // sweep until a whole pass changes nothing; the flag is read every 8 passes
    for (int pass = 0; e == cudaSuccess; pass += 8) {
        int h_changed = 0;
        e = cudaMemsetAsync(changed, 0, sizeof(int), s);
        for (int k = 0; k < 8 && e == cudaSuccess; ++k) {
            k_cc_sweep<<<blocks, threads, 0, s>>>(G->fluid, G->nx, G->ny, G->nz, G->N, label, changed);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_changed, changed, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || !h_changed) break;
        if (pass > 4 * (G->nx + G->ny + G->nz) + G->N) {  // cannot happen: labels strictly decrease
            e = cudaErrorUnknown;
            break;
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)G->N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(best, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        k_cc_count<<<blocks, threads, 0, s>>>(G->fluid, G->N, label, count);
        k_cc_best<<<blocks, threads, 0, s>>>(count, G->N, best);
        k_cc_mark<<<wblocks, threads, 0, s>>>(G->fluid, G->N, G->W, label, best, G->cluster);
        e = cudaGetLastError();
    }
    unsigned long long h_best = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_best, best, sizeof(h_best), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(label, s, so);
    dev_free(count, s, so);
    dev_free(changed, s, so);
    dev_free(best, s, so);
    if (e != cudaSuccess) return cuda_fail(e, "connected clusters");
    G->n_cluster = (int64_t)(h_best >> 32);
    return MP_OK;
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
    // per-node launches round the node count up to whole 256-thread blocks in int
    // arithmetic, and node indices stay below 2^31
    if (N > (1LL << 31) - 256) {
        set_error("lattice too large: nx*ny*nz must be at most 2^31 - 256");
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
        (rc = dev_alloc(&G.ibase, G.W, s, so)) || (rc = dev_alloc(&G.fbase, G.W, s, so)) ||
        (rc = dev_alloc(&totals, 2, s, so))) {
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
    k_scan<<<1, kScanThreads, 0, s>>>(G.fluid, G.iface, G.W, G.ibase, G.fbase, totals);
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
    if (want_list) {
        if ((G.n_iface > 0 && (rc = dev_alloc(&G.ilist, (size_t)G.n_iface, s, so))) ||
            (G.n_fluid > 0 && (rc = dev_alloc(&G.flist, (size_t)G.n_fluid, s, so)))) {
            free_geometry(&G, s, so);
            return rc;
        }
        if (G.n_iface > 0) k_list<<<(G.N + 255) / 256, 256, 0, s>>>(G.iface, G.ibase, G.N, G.ilist);
        if (G.n_fluid > 0) k_list<<<(G.N + 255) / 256, 256, 0, s>>>(G.fluid, G.fbase, G.N, G.flist);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            free_geometry(&G, s, so);
            return cuda_fail(e, "node lists");
        }
    }
    *out = G;
    return MP_OK;
}

}  // namespace mp

extern "C" int mp_classify(const mp_geometry* g, uint8_t* cls, int64_t* n_fluid, int64_t* n_interface,
                           int64_t* n_cluster, void* stream)
{
    using namespace mp;
    clear_error();
    if (!cls) {
        set_error("mp_classify: cls is NULL");
        return MP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Geometry G;
    int rc = build_geometry(g, s, true, false, &G);
    if (rc == MP_OK) rc = build_cluster(&G, s, true);
    if (rc != MP_OK) {
        free_geometry(&G, s, true);
        cudaStreamSynchronize(s);
        return rc;
    }
    const size_t W = (size_t)G.W;
    uint32_t* h = (uint32_t*)malloc(3 * W * sizeof(uint32_t));
    if (!h) {
        free_geometry(&G, s, true);
        cudaStreamSynchronize(s);
        set_error("host allocation failed");
        return MP_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(h, G.fluid, W * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + W, G.iface, W * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + 2 * W, G.cluster, W * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        for (int n = 0; n < G.N; ++n) {
            const uint32_t b = 1u << (n & 31);
            const size_t w = (size_t)(n >> 5);
            cls[n] = (uint8_t)((h[w] & b ? 1 : 0) + (h[W + w] & b ? 1 : 0) + (h[2 * W + w] & b ? 4 : 0));
        }
        if (n_fluid) *n_fluid = G.n_fluid;
        if (n_interface) *n_interface = G.n_iface;
        if (n_cluster) *n_cluster = G.n_cluster;
    }
    free(h);
    free_geometry(&G, s, true);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_classify");
    return MP_OK;
}

