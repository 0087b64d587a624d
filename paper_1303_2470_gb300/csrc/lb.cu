// lb.cu -- steady BGK lattice-Boltzmann flow (paper Eq. lb_evolution) for the velocity
// field that biases the moment propagation. One fused pull step per launch:
//   stream   f_i(r) <- f_i^post(r - c_i), or f_ibar^post(r) when r - c_i is solid
//            (halfway bounce-back, ibar the opposite link);
//   moments  rho = sum f_i, u = (sum f_i c_i + F/2) / rho;
//   collide  f_i^post = f_i - (f_i - f_i^eq(rho,u))/tau
//                       + (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i.u) c_i].F   (Guo force).
// Populations are FP32 deviations g_i = f_i - w_i, which keeps ~9 significant digits of the
// O(u) part that sets the velocity, stored for fluid nodes only, in the order of the sorted
// fluid list: g[i*N_F + k] for fluid node k (structure of arrays). One thread per fluid node;
// the compact index of a neighbour s is prefix[s >> 5] + popc(fluid bits of s's word below
// s), from two bit-sized arrays that stay cache-resident, so a warp's reads and writes cover
// whole sectors of fluid data only. The steady criterion max|u(t) - u(t-1)| is evaluated in
// FP64.
// The body force acts on the largest connected fluid cluster only (sealed pockets stay at
// rest, their steady Stokes velocity). At every failed residual check the state is replaced
// by the mean of the last two iterates: the fixed point is unchanged, an error mode of
// eigenvalue lambda is scaled by (1 + lambda)/2, and the undamped period-2 modes that
// bounce-back sustains at nodes with few open links disappear (without it the residual of a
// porous medium stalls near |F|).
#include <cmath>
#include <cstring>
#include <string>

#include "internal.cuh"
#include "lattice.cuh"

using namespace mp;

namespace {

constexpr int kLbThreads = 256;
// 5 resident blocks per SM (48 registers a thread): with sources located by row (eight
// prefix + popcount lookups a node) the step keeps its 19 gathers and the row centres in
// registers; measured at 8, 6, 5 and 4 blocks (32 registers spill), 5 is fastest
#ifndef MP_LB_MIN_BLOCKS
#define MP_LB_MIN_BLOCKS 5
#endif

struct LbArgs {
    int nx, ny, nz, N, NF;
    Div dx, dxy;  // division by nx and by nx*ny
    const uint32_t* fluid;
    const int32_t* fbase;    // fluid nodes before each 32-node word
    const int32_t* flist;    // lattice node of fluid index k
    const uint32_t* omask;   // open-link mask of fluid index k (bit i-1: r - c_i is fluid)
    const uint2* fw;         // {fluid bits, fluid nodes before the word} per 32-node word
    const uint32_t* forced;  // the force acts on these nodes (the largest fluid cluster)
    float Fx, Fy, Fz;
    float inv_tau;
    float guo;  // 1 - 1/(2 tau)
};

__device__ __forceinline__ bool lb_bit(const uint32_t* __restrict__ w, int n)
{
    return (__ldg(w + (n >> 5)) >> (n & 31)) & 1u;
}

// mode 0: plain step; 1: also store u into u_prev; 2: store u into u_out (and rho into
// rho_out when given), fold max|u - u_prev| (FP64) into *res_bits (non-negative doubles
// order like their bits), then store u into u_prev. u_prev is compact [3][N_F]; u_out and
// rho_out are dense (their solid entries are zeroed once by the host).
__global__ void __launch_bounds__(kLbThreads, MP_LB_MIN_BLOCKS)
    k_lb_step(const LbArgs a, const float* __restrict__ g, float* __restrict__ gn, int mode,
              float* __restrict__ u_prev, float* __restrict__ u_out, float* __restrict__ rho_out,
              unsigned long long* __restrict__ res_bits)
{
    pdl_enter();  // launched with programmatic dependent launch: the previous step's populations
    const int k = blockIdx.x * kLbThreads + threadIdx.x;
    const size_t NF = (size_t)a.NF;
    double res = 0.0;
    if (k < a.NF) {
        const int n = __ldg(a.flist + k);
        const uint32_t mask = __ldg(a.omask + k);
        const Nbr b = nbrs_of(a.nx, a.ny, a.nz, a.dx, a.dxy, n);
        // fluid-list index of each source row's centre; sources in a row are consecutive
        int C[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) C[j] = fluid_index(a.fw, src_of(b, row_centre(j)));
        const bool xlo = b.oxm == -1, xhi = b.oxp == 1;
        float f[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            if (i == 0) {
                f[0] = g[k];
            } else if ((mask >> (i - 1)) & 1u) {
                f[i] = g[(size_t)i * NF + source_index(i, k, C, mask, xlo, xhi, b, a.fw)];
            } else {
                f[i] = g[(size_t)opposite(i) * NF + k];  // halfway bounce-back
            }
        }
        float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            drho += f[i];
            mx += float(cx(i)) * f[i];
            my += float(cy(i)) * f[i];
            mz += float(cz(i)) * f[i];
        }
        const bool on = lb_bit(a.forced, n);
        const float Fx = on ? a.Fx : 0.0f, Fy = on ? a.Fy : 0.0f, Fz = on ? a.Fz : 0.0f;
        const float rho = 1.0f + drho;
        const float inv_rho = 1.0f / rho;
        const float ux = (mx + 0.5f * Fx) * inv_rho;
        const float uy = (my + 0.5f * Fy) * inv_rho;
        const float uz = (mz + 0.5f * Fz) * inv_rho;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const float m15uu = -1.5f * uu;
        const float m3uF = -3.0f * uF;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const float w = weight<float>(i);
            // c_i.u and c_i.F: signed sums of one or two components (zero for the rest link)
            float cu = 0.f, cF = 0.f;
            if (cx(i)) {
                cu += float(cx(i)) * ux;
                cF += float(cx(i)) * Fx;
            }
            if (cy(i)) {
                cu += float(cy(i)) * uy;
                cF += float(cy(i)) * Fy;
            }
            if (cz(i)) {
                cu += float(cz(i)) * uz;
                cF += float(cz(i)) * Fz;
            }
            // f^eq - w = w [(rho - 1) + rho (cu (3 + 4.5 cu) - 1.5 uu)]
            const float geq = w * fmaf(rho, fmaf(cu, fmaf(4.5f, cu, 3.0f), m15uu), drho);
            // Guo: (1 - 1/(2 tau)) w [3 (c_i - u).F + 9 (c_i.u)(c_i.F)] = ... w [3 cF (1 + 3 cu) - 3 u.F]
            const float src = a.guo * w * fmaf(3.0f * cF, fmaf(3.0f, cu, 1.0f), m3uF);
            gn[(size_t)i * NF + k] = fmaf(-a.inv_tau, f[i] - geq, f[i]) + src;
        }
        if (mode == 1) {
            u_prev[k] = ux;
            u_prev[NF + k] = uy;
            u_prev[2 * NF + k] = uz;
        } else if (mode == 2) {
            u_out[n] = ux;
            u_out[(size_t)a.N + n] = uy;
            u_out[2 * (size_t)a.N + n] = uz;
            if (rho_out) rho_out[n] = rho;
            res = fmax(fabs((double)ux - (double)u_prev[k]),
                       fmax(fabs((double)uy - (double)u_prev[NF + k]), fabs((double)uz - (double)u_prev[2 * NF + k])));
            // a non-finite velocity (fmax drops NaN) counts as an infinite residual
            if (!(fabs((double)ux) + fabs((double)uy) + fabs((double)uz) <= 1.0e300)) res = INFINITY;
            // this node's u(t) is the reference of the next check when it is due next step
            u_prev[k] = ux;
            u_prev[NF + k] = uy;
            u_prev[2 * NF + k] = uz;
        }
    }
    if (mode == 2) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
        if ((threadIdx.x & 31) == 0 && res > 0.0) atomicMax(res_bits, (unsigned long long)__double_as_longlong(res));
    }
}

// g0 <- (g0 + g1) / 2 over all populations: the mean of the last two iterates
__global__ void k_lb_mean(float* __restrict__ g0, const float* __restrict__ g1, size_t count)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x)
        g0[k] = 0.5f * (g0[k] + g1[k]);
}

// f = f^eq(rho0, u0) as deviations (u0 = 0 and rho0 = 1 when NULL; both dense); u_prev = u0
__global__ void k_lb_init(const LbArgs a, const float* __restrict__ u0, const float* __restrict__ rho0,
                          float* __restrict__ g, float* __restrict__ u_prev)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.NF) return;
    const size_t NF = (size_t)a.NF;
    const int n = __ldg(a.flist + k);
    float ux = 0.f, uy = 0.f, uz = 0.f, rho = 1.f;
    if (u0) {
        ux = u0[n];
        uy = u0[(size_t)a.N + n];
        uz = u0[2 * (size_t)a.N + n];
    }
    if (rho0) rho = rho0[n];
    const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const float cu = float(cx(i)) * ux + float(cy(i)) * uy + float(cz(i)) * uz;
        // f^eq - w = w [(rho - 1) + rho (3 cu + 4.5 cu^2 - 1.5 uu)]
        g[(size_t)i * NF + k] = weight<float>(i) * ((rho - 1.0f) + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
    }
    u_prev[k] = ux;
    u_prev[NF + k] = uy;
    u_prev[2 * NF + k] = uz;
}

}  // namespace

// Per lb_steady call: the open-link mask of every fluid node and the {fluid bits, prefix}
// words that locate link sources in the fluid list.
__global__ void k_lb_prep(const LbArgs a, int W, uint32_t* __restrict__ omask, uint2* __restrict__ fw)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < W) fw[t] = make_uint2(a.fluid[t], (uint32_t)a.fbase[t]);
    if (t < a.NF) {
        const Nbr b = nbrs_of(a.nx, a.ny, a.nz, a.dx, a.dxy, a.flist[t]);
        uint32_t m = 0;
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            const int s = src_of(b, i);
            if ((a.fluid[s >> 5] >> (s & 31)) & 1u) m |= 1u << (i - 1);
        }
        omask[t] = m;
    }
}

extern "C" int lb_steady(const mp_geometry* geom, const double force[3], double tau, double tol, int64_t max_steps,
                         int64_t check_every, const float* u_init, const float* rho_init, float* u_out,
                         float* rho_out, int64_t* steps_out, double* residual_out, void* stream_ptr)
{
    clear_error();
    if (!force || !u_out || !(tau > 0.5) || max_steps < 1 || check_every < 1 || !(tol >= 0.0)) {
        set_error("lb_steady: need force, u_out, tau > 1/2, tol >= 0, max_steps >= 1, check_every >= 1");
        return MP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream_ptr;
    Geometry G;
    int rc = build_geometry(geom, s, true, true, &G);
    if (rc != MP_OK) return rc;
    // the body force acts on the largest connected fluid cluster: in a sealed pocket a
    // uniform force is balanced by pressure and the steady velocity is zero
    rc = build_cluster(&G, s, true);
    if (rc != MP_OK) {
        free_geometry(&G, s, true);
        cudaStreamSynchronize(s);
        return rc;
    }
    const size_t N = (size_t)G.N;
    const size_t NF = (size_t)(G.n_fluid > 0 ? G.n_fluid : 1);
    float *g0 = nullptr, *g1 = nullptr, *uprev = nullptr;
    uint32_t* omask = nullptr;
    uint2* fw = nullptr;
    unsigned long long* res_d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&g0, sizeof(float) * kQ * NF, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&omask, sizeof(uint32_t) * NF, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&fw, sizeof(uint2) * (size_t)(G.W > 0 ? G.W : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&g1, sizeof(float) * kQ * NF, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&uprev, sizeof(float) * 3 * NF, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&res_d, sizeof(unsigned long long), s);
    // solid entries of the dense outputs stay zero; fluid entries are written at every check
    if (e == cudaSuccess) e = cudaMemsetAsync(u_out, 0, sizeof(float) * 3 * N, s);
    if (e == cudaSuccess && rho_out) e = cudaMemsetAsync(rho_out, 0, sizeof(float) * N, s);
    auto cleanup = [&]() {
        if (g0) cudaFreeAsync(g0, s);
        if (g1) cudaFreeAsync(g1, s);
        if (uprev) cudaFreeAsync(uprev, s);
        if (omask) cudaFreeAsync(omask, s);
        if (fw) cudaFreeAsync(fw, s);
        if (res_d) cudaFreeAsync(res_d, s);
        free_geometry(&G, s, true);
        cudaStreamSynchronize(s);
    };
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "lb_steady allocation");
        cleanup();
        return rc;
    }
    LbArgs a;
    a.nx = G.nx;
    a.ny = G.ny;
    a.nz = G.nz;
    a.N = G.N;
    a.NF = (int)G.n_fluid;
    a.dx = make_div((unsigned)G.nx);
    a.dxy = make_div((unsigned)(G.nx * G.ny));
    a.fluid = G.fluid;
    a.fbase = G.fbase;
    a.flist = G.flist;
    a.omask = omask;
    a.fw = fw;
    a.forced = G.cluster;
    a.Fx = (float)force[0];
    a.Fy = (float)force[1];
    a.Fz = (float)force[2];
    a.inv_tau = (float)(1.0 / tau);
    a.guo = (float)(1.0 - 0.5 / tau);
    // one thread per fluid node (at least one block, so that a medium without fluid still
    // runs its checks: its residual is 0)
    const int blocks = (int)((NF + kLbThreads - 1) / kLbThreads);
    const size_t prep = std::max<size_t>(NF, (size_t)G.W);
    k_lb_prep<<<(unsigned)((prep + 255) / 256), 256, 0, s>>>(a, G.W, omask, fw);
    k_lb_init<<<blocks, kLbThreads, 0, s>>>(a, u_init, rho_init, g0, uprev);
    e = cudaGetLastError();
    int64_t t = 0;
    double res = INFINITY;
    bool converged = false;
    while (e == cudaSuccess && t < max_steps) {
        const int64_t t1 = t + 1;
        int mode = 0;
        if (t1 % check_every == 0 || t1 == max_steps)
            mode = 2;
        else if ((t1 + 1) % check_every == 0 || t1 + 1 == max_steps)
            mode = 1;
        if (mode == 2) e = cudaMemsetAsync(res_d, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess)
            e = launch_pdl(k_lb_step, dim3(blocks), dim3(kLbThreads), s, a, (const float*)g0, g1, mode, uprev, u_out,
                           rho_out, res_d);
        float* tmp = g0;
        g0 = g1;
        g1 = tmp;
        t = t1;
        if (mode == 2 && e == cudaSuccess) {
            unsigned long long bits = 0;
            e = cudaMemcpyAsync(&bits, res_d, sizeof(bits), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            memcpy(&res, &bits, sizeof(res));
            if (res < tol) {
                converged = true;
                break;
            }
            if (std::isinf(res)) break;  // the flow is no longer finite: give up
            // the mean of the last two iterates (g0 = t, g1 = t-1): same fixed point, and the
            // undamped period-2 modes that bounce-back sustains at confined nodes vanish
            if (t < max_steps) {
                k_lb_mean<<<2 * 152 * 4, 256, 0, s>>>(g0, g1, (size_t)kQ * NF);
                e = cudaGetLastError();
            }
        }
    }
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "lb_steady step");
        cleanup();
        return rc;
    }
    cleanup();
    if (steps_out) *steps_out = t;
    if (residual_out) *residual_out = res;
    if (!converged) {
        set_error(std::isinf(res) ? "lb_steady: the velocity became non-finite by step " + std::to_string(t) +
                                        " (unstable: tau, force or initial state)"
                                  : "lb_steady: residual " + std::to_string(res) + " above tol after " +
                                        std::to_string(t) + " steps");
        return MP_ENOTCONVERGED;
    }
    return MP_OK;
}
