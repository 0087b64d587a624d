// mp_noalloc.cu -- one moment-propagation + sorption step on caller-owned dense arrays that
// allocates no memory at all, for callers that cannot allocate device memory: code that runs
// inside a host application which owns every device allocation (a fixed memory budget or
// its own pool, where a stray cudaMalloc would fail or break its accounting), or code that
// must not trigger the implicit device synchronisation of cudaMalloc / cudaFree.
//
// The only scratch the step needs -- the per-block partial sums of its FP64 reduction and a
// completion counter -- lives in a file-scope __device__ array of fixed size. Every GPU that
// runs this entry point keeps that array until the library is unloaded.
#include <mutex>

#include "internal.cuh"
#include "link_arith.cuh"

using namespace mp;

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaWarps = kNaThreads / 32;
constexpr int kNaMaxBlocks = 8192;  // one thread per node: at most 2,097,152 nodes per call
constexpr long long kNaMaxNodes = (long long)kNaThreads * kNaMaxBlocks;
constexpr size_t kNaTicketOffset = kNaMaxBlocks * sizeof(double);

// [0, kNaTicketOffset): one FP64 partial sum per block; then the completion counter.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaTicketOffset + 256];

struct NaArgs {
    int nx, ny, nz, N;
    int g;  // direction of the velocity weight of the sum, -1 for the plain sum
    float hl, pa, pd;
};

__device__ __forceinline__ int na_wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Same update as the library's step kernel, read from dense arrays: X(r) + sum of net link
// fluxes, then the sorption exchange on interfacial nodes (paper Sec. "Algorithm",
// Eqs. propagated_quantity, Pads, newP), and sum_r X'(r) u*_g(r) in FP64.
__global__ void __launch_bounds__(kNaThreads)
    k_step_noalloc(const NaArgs a, const uint8_t* __restrict__ solid, const float* __restrict__ u,
                   const float* __restrict__ X, const float* __restrict__ Xa, float* __restrict__ Xn,
                   float* __restrict__ Xan, double* __restrict__ z_out, unsigned char* __restrict__ scratch)
{
    double* partials = reinterpret_cast<double*>(scratch);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kNaTicketOffset);
    const int n = blockIdx.x * kNaThreads + threadIdx.x;
    float zp = 0.0f;
    if (n < a.N) {
        if (solid[n]) {
            Xn[n] = 0.0f;
            Xan[n] = 0.0f;
        } else {
            const int x = n % a.nx, y = (n / a.nx) % a.ny, z = n / (a.nx * a.ny);
            float ux = 0.f, uy = 0.f, uz = 0.f;
            if (u) {
                ux = u[n];
                uy = u[a.N + n];
                uz = u[2 * a.N + n];
            }
            const float ar = rn_mul(-1.5f, rn_add(rn_add(rn_mul(ux, ux), rn_mul(uy, uy)), rn_mul(uz, uz)));
            const float whl_face = rn_mul(weight<float>(1), a.hl), whl_edge = rn_mul(weight<float>(5), a.hl);
            const float xr = X[n];
            float delta = 0.0f, us = 0.0f;
            bool itf = false;
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                const int s = na_wrap(x - cx(i), a.nx) +
                              a.nx * (na_wrap(y - cy(i), a.ny) + a.ny * na_wrap(z - cz(i), a.nz));
                if (solid[s]) {
                    itf = true;
                    continue;
                }
                float sx = 0.f, sy = 0.f, sz = 0.f;
                if (u) {
                    sx = u[s];
                    sy = u[a.N + s];
                    sz = u[2 * a.N + s];
                }
                const float as = rn_mul(-1.5f, rn_add(rn_add(rn_mul(sx, sx), rn_mul(sy, sy)), rn_mul(sz, sz)));
                const float whl = is_face(i) ? whl_face : whl_edge;
                const float pin = rn_fma(weight<float>(i), qlink(edot<float>(i, sx, sy, sz), as), whl);
                const float pout = rn_fma(weight<float>(i), qlink(edot<float>(opposite(i), ux, uy, uz), ar), whl);
                delta = rn_add(delta, rn_sub(rn_mul(pin, X[s]), rn_mul(pout, xr)));
                if (a.g >= 0) {
                    const int c = ci(opposite(i), a.g);
                    if (c != 0) us += float(c) * pout;
                }
            }
            if (itf) {
                const float xa = Xa[n];
                const float js = rn_sub(rn_mul(a.pa, xr), rn_mul(a.pd, xa));
                delta = rn_sub(delta, js);
                Xan[n] = rn_add(xa, js);
            } else {
                Xan[n] = 0.0f;
            }
            const float xn = rn_add(xr, delta);
            Xn[n] = xn;
            zp = a.g >= 0 ? xn * us : xn;
        }
    }
    // FP32 within the warp, FP64 across warps and blocks, in a fixed order
    __shared__ double s_red[kNaWarps];
    __shared__ unsigned int s_last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zp += __shfl_xor_sync(0xffffffffu, zp, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)zp;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNaWarps; ++w) t += s_red[w];
        partials[blockIdx.x] = t;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kNaThreads) v += __ldcg(partials + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNaWarps; ++w) t += s_red[w];
        *z_out = t;
        *ticket = 0u;
    }
}

// Device address of the scratch array. In host code the array's name is only a host-side
// stand-in, so the address is looked up with cudaGetSymbolAddress (with the device current)
// and remembered per device together with the unique id of the context it belongs to. A
// cudaDeviceReset ends that context and the next call runs in a new one, whose module copy
// of the array lives elsewhere: a changed context id triggers a fresh lookup. The driver's
// context queries are resolved through the runtime, so the library needs no link to libcuda.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

std::mutex g_scratch_mu;
struct ScratchSlot {
    unsigned char* ptr = nullptr;
    unsigned long long ctx_id = 0;
};
ScratchSlot g_scratch[128];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// unique id of the calling thread's current context; 0 if none or not available
unsigned long long current_ctx_id()
{
    if (!g_ctx_fns_tried) {
        g_ctx_fns_tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!g_ctx_current || !g_ctx_id || g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

int scratch_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 128) {
        set_error("mp_step_noalloc: device ordinal out of range");
        return MP_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot& slot = g_scratch[dev];
    const unsigned long long id = slot.ptr ? current_ctx_id() : 0;
    if (!slot.ptr || id == 0 || id != slot.ctx_id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also makes the device's context current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        slot.ptr = static_cast<unsigned char*>(p);
        slot.ctx_id = current_ctx_id();
    }
    *out = slot.ptr;
    return MP_OK;
}

// [a, a + na) and [b, b + nb) share a byte (null pointers share nothing)
bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

}  // namespace

extern "C" int mp_step_noalloc(int nx, int ny, int nz, const uint8_t* solid, const float* u, double D_b,
                               double k_a, double k_d, int direction, const float* X, const float* X_ads,
                               float* X_out, float* X_ads_out, double* Z_out, void* stream)
{
    clear_error();
    if (nx < 3 || ny < 3 || nz < 3) {
        set_error("mp_step_noalloc: every lattice dimension must be >= 3");
        return MP_EINVAL;
    }
    const long long N = (long long)nx * ny * nz;
    if (N > kNaMaxNodes) {
        set_error("mp_step_noalloc: " + std::to_string(N) + " nodes exceed the limit of " +
                  std::to_string(kNaMaxNodes) + " set by its fixed reduction scratch");
        return MP_EINVAL;
    }
    if (!solid || !X || !X_ads || !X_out || !X_ads_out || !Z_out) {
        set_error("mp_step_noalloc: solid, X, X_ads, X_out, X_ads_out and Z_out are required");
        return MP_EINVAL;
    }
    {
        // the step reads neighbours of every node while other threads write their results,
        // so no output byte may lie in any input (or in the other output)
        const size_t fb = (size_t)N * sizeof(float);
        const void* in[5] = {X, X_ads, solid, u, Z_out};
        const size_t in_b[5] = {fb, fb, (size_t)N, u ? 3 * fb : 0, sizeof(double)};
        const void* outs[2] = {X_out, X_ads_out};
        bool bad = overlap(X_out, fb, X_ads_out, fb);
        for (int o = 0; o < 2; ++o)
            for (int j = 0; j < 5; ++j) bad = bad || overlap(outs[o], fb, in[j], in_b[j]);
        if (bad) {
            set_error("mp_step_noalloc: the output arrays must not overlap the inputs, Z_out or each other");
            return MP_EINVAL;
        }
    }
    if (!(D_b > 0.0 && D_b <= 0.25) || !(k_a >= 0.0 && k_a <= 1.0) || !(k_d >= 0.0 && k_d <= 1.0) ||
        direction < -1 || direction > 2) {
        set_error("mp_step_noalloc: need 0 < D_b <= 0.25, k_a and k_d in [0, 1], direction in -1..2");
        return MP_EINVAL;
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != MP_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the completion counter must start at zero (the previous call may have been cut short)
    MP_CUDA(cudaMemsetAsync(scratch + kNaTicketOffset, 0, sizeof(unsigned int), s));
    NaArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.N = (int)N;
    a.g = direction;
    a.hl = (float)(6.0 * D_b);  // lambda/2 = 12 D_b / 2
    a.pa = (float)k_a;
    a.pd = (float)k_d;
    const int blocks = (int)((N + kNaThreads - 1) / kNaThreads);
    k_step_noalloc<<<blocks, kNaThreads, 0, s>>>(a, solid, u, X, X_ads, X_out, X_ads_out, Z_out, scratch);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}
