// mp.cu -- sorption-modified moment propagation on the GPU (paper Sec. "Algorithm"):
// the initialisation of the density and velocity-moment fields, the fused propagation +
// sorption step with its FP64 VACF / D(t) reduction, and the C-ABI context functions.
//
// Per fluid node r and step (Eq. propagated_quantity, Eqs. Pads and newP):
//   P*(r)      = sum_i X(r - c_i) p_i(r - c_i) + X(r) (1 - sum_i p_i(r) - p_a 1_I(r))
//   Xa(r,t+1)  = p_a X(r) + (1 - p_d) Xa(r)            on interfacial nodes
//   X(r,t+1)   = P*(r) + p_d Xa(r)                      on interfacial nodes
// with p_i(s) = w_i [lambda/2 + 3 c_i.u(s) + 9/2 (c_i.u(s))^2 - 3/2 u(s).u(s)] on links
// whose far end is fluid, zero otherwise; lambda = 12 D_b; p_a = k_a, p_d = k_d.
// The step is evaluated as X + sum of net link fluxes (see k_step), which is the same
// update in exact arithmetic and conserves mass in FP32.
// The VACF of direction g is Z_g(t) = sum_r P_g(r,t) u*_g(r), u*_g(r) = sum_i p_i(r) c_ig.
//
// Work layout: one thread per fluid node of the compact fluid list (no solid lanes). The
// flow is steady, so everything that depends on it alone is prepared once by mp_init: the
// 18-bit open-link mask of every fluid node and, for every node, (u_x, u_y, u_z, -3/2|u|^2)
// packed in one 16-byte vector, so that a neighbour's link probability costs one load and
// three fused multiply-adds. All species sharing the medium reuse the flow-dependent part
// q_i of p_i = w_i (q_i + lambda/2); only lambda/2, p_a and p_d differ per species.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "internal.cuh"
#include "lattice.cuh"
#include "link_arith.cuh"
#include "mp_ctx.cuh"

namespace mp {
const char* last_error_text();
}

using namespace mp;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxF = 4;  // density + up to three velocity moments
constexpr uint32_t kAllLinks = (1u << 18) - 1u;

// ---------------------------------------------------------------------------------------
// Storage type TS of the fields: float or double (the arithmetic type T itself), or IEEE
// binary16 with FP32 arithmetic. A record is widened to T on load and narrowed on store.
// Binary16 rounding is to nearest or stochastic: the magnitude is rounded up with
// probability equal to the dropped fraction of the binary16 spacing, compared against
// random bits from a counter-based hash of (step, element). Stochastic rounding is
// unbiased, so per-step changes below half a spacing still move a field on average.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float widen1(float v) { return v; }
__device__ __forceinline__ double widen1(double v) { return v; }
__device__ __forceinline__ float widen1(__half v) { return __half2float(v); }

// 32-bit integer hash "lowbias32" (C. Wellons, "Prospecting for hash functions", 2018)
__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ __half half_stochastic(float x, uint32_t r)
{
    if (fabsf(x) < 6.103515625e-05f) {
        // below the smallest normal binary16 the spacing is 2^-24: round q = x 2^24 to an
        // integer, up with probability q - floor(q); the result is exact in binary16
        const float q = x * 16777216.0f;
        const float lo = floorf(q);
        const float u = (float)(r >> 8) * 5.9604644775390625e-08f;  // uniform in [0, 1)
        return __float2half_rz((u < q - lo ? lo + 1.0f : lo) * 5.9604644775390625e-08f);
    }
    // normal range: binary16 keeps 10 of the 23 FP32 mantissa bits; adding 13 random bits
    // below the kept ones carries into them with the probability of the dropped fraction
    const uint32_t b = (__float_as_uint(x) + (r & 0x1fffu)) & ~0x1fffu;
    return __float2half_rz(__uint_as_float(b));
}

template <typename TS>
struct Narrow;
template <>
struct Narrow<float> {
    __device__ static float one(float v, uint32_t, bool) { return v; }
};
template <>
struct Narrow<double> {
    __device__ static double one(double v, uint32_t, bool) { return v; }
};
template <>
struct Narrow<__half> {
    __device__ static __half one(float v, uint32_t key, bool stochastic)
    {
        return stochastic ? half_stochastic(v, hash32(key)) : __float2half_rn(v);
    }
};

template <typename T, typename TS, int W>
__device__ __forceinline__ FieldVec<T, W> ld_wide(const FieldVec<TS, W>* p)
{
    if constexpr (std::is_same<T, TS>::value) {
        return ld_rec(p);
    } else {
        const FieldVec<TS, W> h = *p;
        FieldVec<T, W> r;
#pragma unroll
        for (int j = 0; j < W; ++j) r.v[j] = widen1(h.v[j]);
        return r;
    }
}

// key: distinct per stored element and step (see step_body)
template <typename T, typename TS, int W>
__device__ __forceinline__ void st_narrow(FieldVec<TS, W>* p, const FieldVec<T, W>& v, uint32_t key, bool stochastic)
{
    if constexpr (std::is_same<T, TS>::value) {
        st_rec(p, v);
    } else {
        FieldVec<TS, W> h;
#pragma unroll
        for (int j = 0; j < W; ++j) h.v[j] = Narrow<TS>::one(v.v[j], key + (uint32_t)j, stochastic);
        *p = h;
    }
}

template <typename T>
struct Args {
    int nx, ny, nz, N, NF, NI;
    int FP;  // fields per species record, padded: 2 or 4
    int SP;  // species, padded to a whole number of chunks (1 for one species)
    int SC;  // species per chunk (1 for one species, else 8 / FP); element (n, s, f) sits at
             // (((s / SC) * rows + n) * SC + s % SC) * FP + f, rows = N for P, NI for P_ads
    int compact;  // P over the fluid list: row = work item k, rows = NF
    Div dx, dxy;  // division by nx and by nx*ny
    const uint32_t* iface;
    const int32_t* ibase;
    const int32_t* flist;    // fluid node of each work item
    const uint32_t* fmask;   // bit i-1: link i (inflow from r - c_i) is open
    const Flow4<T>* u4;      // dense, zero on solid nodes
    int S, F, M;
    int dir[3];  // direction of velocity moment m (field m+1)
    T hl[MP_MAX_SPECIES];  // lambda/2
    T pa[MP_MAX_SPECIES];
    T pd[MP_MAX_SPECIES];
    T whf[MP_MAX_SPECIES];  // w_face * lambda/2, correctly rounded (the diffusive part of p)
    T whe[MP_MAX_SPECIES];  // w_edge * lambda/2
    double zsc[MP_MAX_SPECIES];  // stored value x zsc = field value (1 unless binary16 storage)
    int stochastic;              // binary16 storage: stochastic rounding (else to nearest)
    double* partials;            // [gridDim.x][K]
    unsigned int* ticket;        // blocks done in the current launch
    double* Z;             // [K_series][cap]
    double* D;
    long long* tdev;  // time index of the last written series entry
    long long cap;
};

struct InitExtra {
    double invZ[MP_MAX_SPECIES];  // 1 / partition function (free weight per fluid node)
    double K[MP_MAX_SPECIES];     // k_a / k_d (0 without sorption)
    double inv_nf;                // 1 / N_fluid
    double sc[MP_MAX_SPECIES];    // storage scale: stored = field value x sc (1 / zsc)
    int uniform;                  // density starts uniform-free
};

__device__ __forceinline__ bool bit_of(const uint32_t* __restrict__ w, int n)
{
    return (__ldg(w + (n >> 5)) >> (n & 31)) & 1u;
}

// element (row, species, field) of a chunk-major field array with `rows` rows
template <typename T>
__device__ __forceinline__ size_t elem(const Args<T>& a, size_t rows, size_t row, int sp, int f)
{
    return ((((size_t)(sp / a.SC)) * rows + row) * a.SC + (size_t)(sp % a.SC)) * a.FP + f;
}

template <typename T>
__device__ __forceinline__ T pick(const T v[3], int g)
{
    return g == 0 ? v[0] : (g == 1 ? v[1] : v[2]);
}

template <typename T>
__device__ __forceinline__ Nbr node_nbrs(const Args<T>& a, int n)
{
    return nbrs_of(a.nx, a.ny, a.nz, a.dx, a.dxy, n);
}

// What a fluid node r needs from its links. Link i is the inflow direction c_i: its source
// is s_i = r - c_i, and the reverse link (opposite(i), from r to s_i) carries the outflow.
// Both are open iff s_i is fluid.
template <typename T>
struct Node {
    T cin[kQ];    // q of link i at s_i (s_i -> r)
    T cout[kQ];   // q of link opposite(i) at r (r -> s_i)
    int src[kQ];  // s_i, or -1 when s_i is solid
    int n;
    bool itf;
    int aidx;  // compact index among interfacial nodes
};

template <typename T>
__device__ __forceinline__ int iface_index(const Args<T>& a, int n)
{
    const uint32_t bits = __ldg(a.iface + (n >> 5));
    return __ldg(a.ibase + (n >> 5)) + __popc(bits & ((1u << (n & 31)) - 1u));
}

template <typename T>
__device__ __forceinline__ void load_node(const Args<T>& a, int k, Node<T>& d)
{
    const int n = __ldg(a.flist + k);
    const uint32_t mask = __ldg(a.fmask + k);
    const Nbr b = node_nbrs(a, n);
    const Flow4<T> ur = a.u4[n];
    d.n = n;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        if ((mask >> (i - 1)) & 1u) {
            const int s = src_of(b, i);
            const Flow4<T> us = a.u4[s];
            d.cin[i] = qlink(edot<T>(i, us.x, us.y, us.z), us.w);
            d.cout[i] = qlink(edot<T>(opposite(i), ur.x, ur.y, ur.z), ur.w);
            d.src[i] = s;
        } else {
            d.cin[i] = d.cout[i] = T(0);
            d.src[i] = -1;
        }
    }
    d.itf = mask != kAllLinks;
    d.aidx = d.itf ? iface_index(a, n) : 0;
}

// link probabilities of one species: p = w q + w lambda/2
template <typename T>
__device__ __forceinline__ void species_probs(const Node<T>& d, T hl, T (&pin)[kQ], T (&pout)[kQ])
{
    const T whl_face = rn_mul(weight<T>(1), hl), whl_edge = rn_mul(weight<T>(5), hl);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const T whl = is_face(i) ? whl_face : whl_edge;
        pin[i] = d.src[i] >= 0 ? rn_fma(weight<T>(i), d.cin[i], whl) : T(0);
        pout[i] = d.src[i] >= 0 ? rn_fma(weight<T>(i), d.cout[i], whl) : T(0);
    }
}

// u*_g(r) = sum over open outgoing links of p c_g, and sum of p c_g^2, for direction g
template <typename T>
__device__ __forceinline__ void mean_step(const T (&pout)[kQ], int g, T& us, T& us2)
{
    us = T(0);
    us2 = T(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const int c = ci(opposite(i), g);
        if (c != 0) {
            us += T(c) * pout[i];
            us2 += pout[i];
        }
    }
}

// Sum `cnt` per-thread values over the block: warp sums in T (FP32 or FP64), then FP64
// across warps in fixed order; thread j < cnt writes the total of value j to out[j].
template <typename T, int kMax>
__device__ __forceinline__ void block_sum_store(const T (&v)[kMax], int cnt, double* out)
{
    __shared__ double s_red[kWarps][2 * kMaxF];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMax; ++j) {
        if (j < cnt) {
            T w = warp_sum(v[j]);
            if (lane == 0) s_red[warp][j] = (double)w;
        }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double tot = 0.0;
        for (int k = 0; k < kWarps; ++k) tot += s_red[k][threadIdx.x];
        out[threadIdx.x] = tot;
    }
    __syncthreads();
}

// Last block of a launch (or of one context's block range in a grouped launch): FP64 sum of
// the per-block partials of each of the K series values, in a fixed order; `emit(k, total)`
// is called by thread 0. Thread j < K must have written partial j of this block.
template <int kB, typename Emit>
__device__ __forceinline__ bool grid_total(double* partials, int K, unsigned int* ticket, int nblk, Emit emit)
{
    __shared__ unsigned int s_last;
    __shared__ double s_red[kB / 32];
    // the threads that wrote this block's partials make them visible before the ticket
    if (threadIdx.x < K) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)nblk - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblk; b += kB) v += __ldcg(partials + (size_t)b * K + k);
        v = warp_sum(v);
        if (lane == 0) s_red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < kB / 32; ++w) tot += s_red[w];
            emit(k, tot);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// ---------------------------------------------------------------------------------------
// Step t -> t+1 of every species and field, fused with Z_g(t+1) and D_g(t+1).
//
// Eq. propagated_quantity is evaluated as X(r) + sum_i J_i with the net flux of link i
//   J_i = fl(p_i(s_i) X(s_i)) - fl(p_opp(i)(r) X(r)),
// every factor and product correctly rounded in a fixed order. The node at the other end
// of the link computes the same two products, so it sees exactly -J_i: the exchange is
// antisymmetric and total mass changes only through the final rounding of each node's
// update, which is unbiased and vanishes for a stationary field (|sum J| below half an
// ulp). The direct form X* = inflow + stay X would instead carry the rounding of the stay
// fraction (about 3e-8 in FP32) into every step. The sorption exchange
// J_s = fl(p_a X) - fl(p_d X_ads) is applied the same way (Eqs. Pads and newP).
//
// All FP fields of a node are one vector, so a neighbour costs one flow load and one
// field load. With one species the link loop consumes each neighbour at once (few live
// registers); with several, the flow-dependent parts of the 18 links are kept in registers
// and reused by every species. Each warp reduces its Z terms with shuffles into shared
// memory; the block combines them after one barrier.
// ---------------------------------------------------------------------------------------
template <typename T, typename TS, int FP, bool kSingle, int kB>
__device__ __forceinline__ void step_body(const Args<T>& a, int blk, int nblk, const TS* __restrict__ P,
                                          TS* __restrict__ Pn, const TS* __restrict__ A, TS* __restrict__ An)
{
    constexpr int kW = kB / 32;
    using V = FieldVec<T, FP>;
    using VS = FieldVec<TS, FP>;
    const VS* __restrict__ Pv = reinterpret_cast<const VS*>(P);
    VS* __restrict__ Pnv = reinterpret_cast<VS*>(Pn);
    const VS* __restrict__ Av = reinterpret_cast<const VS*>(A);
    VS* __restrict__ Anv = reinterpret_cast<VS*>(An);
    // binary16 storage: rounding keys from the new time index, then array and element
    uint32_t tkey = 0;
    if constexpr (!std::is_same<T, TS>::value) tkey = hash32((uint32_t)(*(const volatile long long*)a.tdev + 1));
    const uint32_t akey = tkey ^ 0x68e31da4u;
    __shared__ double s_part[kW][MP_MAX_SPECIES * (kMaxF - 1)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blk * kB + threadIdx.x;
    const bool active = k < a.NF;
    const int K = a.S * a.M;

    if constexpr (kSingle) {
        const T hl = a.hl[0], pa = a.pa[0], pd = a.pd[0];
        T zv[kMaxF - 1] = {T(0), T(0), T(0)};
        if (active) {
            const int n = __ldg(a.flist + k);
            const uint32_t mask = __ldg(a.fmask + k);
            const Nbr b = node_nbrs(a, n);
            const Flow4<T> ur = a.u4[n];
            const V xr = ld_wide<T, TS, FP>(Pv + n);
            const T whl_face = rn_mul(weight<T>(1), hl), whl_edge = rn_mul(weight<T>(5), hl);
            T delta[FP];
#pragma unroll
            for (int f = 0; f < FP; ++f) delta[f] = T(0);
            T us[3] = {T(0), T(0), T(0)};
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                if ((mask >> (i - 1)) & 1u) {
                    const int s = src_of(b, i);
                    const Flow4<T> uf = a.u4[s];
                    const V xs = ld_wide<T, TS, FP>(Pv + s);
                    const T whl = is_face(i) ? whl_face : whl_edge;
                    const T pin = rn_fma(weight<T>(i), qlink(edot<T>(i, uf.x, uf.y, uf.z), uf.w), whl);
                    const T pout = rn_fma(weight<T>(i), qlink(edot<T>(opposite(i), ur.x, ur.y, ur.z), ur.w), whl);
#pragma unroll
                    for (int f = 0; f < FP; ++f)
                        delta[f] = rn_add(delta[f], rn_sub(rn_mul(pin, xs.v[f]), rn_mul(pout, xr.v[f])));
#pragma unroll
                    for (int g = 0; g < 3; ++g)
                        if (ci(opposite(i), g) != 0) us[g] += T(ci(opposite(i), g)) * pout;
                }
            }
            if (mask != kAllLinks) {
                const int ai = iface_index(a, n);
                const V xa = ld_wide<T, TS, FP>(Av + ai);
                V xan;
#pragma unroll
                for (int f = 0; f < FP; ++f) {
                    const T js = rn_sub(rn_mul(pa, xr.v[f]), rn_mul(pd, xa.v[f]));
                    delta[f] = rn_sub(delta[f], js);
                    xan.v[f] = rn_add(xa.v[f], js);
                }
                st_narrow<T, TS, FP>(Anv + ai, xan, akey + (uint32_t)ai * FP, a.stochastic);
            }
            V xn;
#pragma unroll
            for (int f = 0; f < FP; ++f) xn.v[f] = rn_add(xr.v[f], delta[f]);
            st_narrow<T, TS, FP>(Pnv + n, xn, tkey + (uint32_t)n * FP, a.stochastic);
#pragma unroll
            for (int m = 0; m < kMaxF - 1; ++m)
                if (m < a.M && 1 + m < FP) zv[m] = xn.v[(1 + m) < FP ? 1 + m : 0] * pick(us, a.dir[m]);
        }
#pragma unroll
        for (int m = 0; m < kMaxF - 1; ++m) {
            if (m < a.M) {
                const T w = warp_sum(zv[m]);
                if (lane == 0) s_part[warp][m] = (double)w;
            }
        }
    } else {
        // Several species, in 32-byte chunks of kSC species x FP fields stored chunk-major
        // ([chunk][node]): a warp's chunk loads of consecutive fluid nodes are consecutive.
        // A pass covers up to kCP chunks (8 species of density + one moment); inside it the
        // link loop is outermost: the flow-dependent part of the link probability is computed
        // once per link and every neighbour chunk is fetched once, serving all its species.
        constexpr int kSC = 8 / FP;
        constexpr int kCP = 2;
        constexpr int kMaxPass = MP_MAX_SPECIES / (kCP * kSC);
        using VC = FieldVec<T, kSC * FP>;
        using VCS = FieldVec<TS, kSC * FP>;
        // per-species constants staged in shared memory, read with compile-time indices
        __shared__ T s_whf[MP_MAX_SPECIES], s_whe[MP_MAX_SPECIES], s_hl[MP_MAX_SPECIES], s_pa[MP_MAX_SPECIES],
            s_pd[MP_MAX_SPECIES];
        for (int j = threadIdx.x; j < MP_MAX_SPECIES; j += kB) {
            s_whf[j] = a.whf[j];
            s_whe[j] = a.whe[j];
            s_hl[j] = a.hl[j];
            s_pa[j] = a.pa[j];
            s_pd[j] = a.pd[j];
        }
        __syncthreads();
        const VCS* __restrict__ Pc = reinterpret_cast<const VCS*>(P);
        VCS* __restrict__ Pnc = reinterpret_cast<VCS*>(Pn);
        const VCS* __restrict__ Ac = reinterpret_cast<const VCS*>(A);
        VCS* __restrict__ Anc = reinterpret_cast<VCS*>(An);
        const int cpn = a.SP / kSC;  // chunks per node
        int n = 0, aidx = 0;
        uint32_t mask = 0;
        Nbr b{};
        Flow4<T> ur{T(0), T(0), T(0), T(0)};
        if (active) {
            n = __ldg(a.flist + k);
            mask = __ldg(a.fmask + k);
            b = node_nbrs(a, n);
            ur = a.u4[n];
            if (mask != kAllLinks) aidx = iface_index(a, n);
        }
#pragma unroll
        for (int pass = 0; pass < kMaxPass; ++pass) {
            const int c0 = pass * kCP;
            if (c0 >= cpn) break;
            const int nc = cpn - c0 < kCP ? cpn - c0 : kCP;
            VC xr[kCP];
            T delta[kCP][kSC * FP];
            // u*_g of species s is UA_g + lambda_s/2 UW_g, sums over the open outgoing links
            T UA[3] = {T(0), T(0), T(0)}, UW[3] = {T(0), T(0), T(0)};
            if (active) {
#pragma unroll
                for (int cc = 0; cc < kCP; ++cc) {
                    if (cc < nc) xr[cc] = ld_wide<T, TS, kSC * FP>(Pc + (size_t)(c0 + cc) * a.N + n);
#pragma unroll
                    for (int j = 0; j < kSC * FP; ++j) delta[cc][j] = T(0);
                }
#pragma unroll
                for (int i = 1; i < kQ; ++i) {
                    if ((mask >> (i - 1)) & 1u) {
                        const int s = src_of(b, i);
                        const Flow4<T> uf = a.u4[s];
                        const T qin = qlink(edot<T>(i, uf.x, uf.y, uf.z), uf.w);
                        const T qout = qlink(edot<T>(opposite(i), ur.x, ur.y, ur.z), ur.w);
#pragma unroll
                        for (int g = 0; g < 3; ++g) {
                            const int c = ci(opposite(i), g);
                            if (c != 0) {
                                UA[g] += T(c) * weight<T>(i) * qout;
                                UW[g] += T(c) * weight<T>(i);
                            }
                        }
#pragma unroll
                        for (int cc = 0; cc < kCP; ++cc) {
                            if (cc < nc) {
                                const VC xs = ld_wide<T, TS, kSC * FP>(Pc + (size_t)(c0 + cc) * a.N + s);
#pragma unroll
                                for (int q = 0; q < kSC; ++q) {
                                    const int sp = (c0 + cc) * kSC + q;
                                    const T whl = is_face(i) ? s_whf[sp] : s_whe[sp];
                                    const T pin = rn_fma(weight<T>(i), qin, whl);
                                    const T pout = rn_fma(weight<T>(i), qout, whl);
#pragma unroll
                                    for (int f = 0; f < FP; ++f) {
                                        const int j = q * FP + f;
                                        delta[cc][j] = rn_add(delta[cc][j],
                                                              rn_sub(rn_mul(pin, xs.v[j]), rn_mul(pout, xr[cc].v[j])));
                                    }
                                }
                            }
                        }
                    }
                }
            }
            // finish each chunk: sorption, store, Z terms and their warp sums
#pragma unroll
            for (int cc = 0; cc < kCP; ++cc) {
                T zv[kSC][kMaxF - 1];
#pragma unroll
                for (int q = 0; q < kSC; ++q)
#pragma unroll
                    for (int m = 0; m < kMaxF - 1; ++m) zv[q][m] = T(0);
                if (active && cc < nc) {
                    if (mask != kAllLinks) {
                        const size_t ai = (size_t)(c0 + cc) * a.NI + aidx;
                        const VC xa = ld_wide<T, TS, kSC * FP>(Ac + ai);
                        VC xan;
#pragma unroll
                        for (int q = 0; q < kSC; ++q) {
                            const int sp = (c0 + cc) * kSC + q;
                            const T pa = s_pa[sp], pd = s_pd[sp];
#pragma unroll
                            for (int f = 0; f < FP; ++f) {
                                const int j = q * FP + f;
                                const T js = rn_sub(rn_mul(pa, xr[cc].v[j]), rn_mul(pd, xa.v[j]));
                                delta[cc][j] = rn_sub(delta[cc][j], js);
                                xan.v[j] = rn_add(xa.v[j], js);
                            }
                        }
                        st_narrow<T, TS, kSC * FP>(Anc + ai, xan, akey + (uint32_t)ai * (kSC * FP), a.stochastic);
                    }
                    VC xn;
#pragma unroll
                    for (int j = 0; j < kSC * FP; ++j) xn.v[j] = rn_add(xr[cc].v[j], delta[cc][j]);
                    const size_t pi = (size_t)(c0 + cc) * a.N + n;
                    st_narrow<T, TS, kSC * FP>(Pnc + pi, xn, tkey + (uint32_t)pi * (kSC * FP), a.stochastic);
#pragma unroll
                    for (int q = 0; q < kSC; ++q) {
                        const T h = s_hl[(c0 + cc) * kSC + q];
#pragma unroll
                        for (int m = 0; m < kMaxF - 1; ++m) {
                            if (m < a.M && 1 + m < FP) {
                                const int g = a.dir[m];
                                zv[q][m] = xn.v[q * FP + ((1 + m) < FP ? 1 + m : 0)] * (pick(UA, g) + h * pick(UW, g));
                            }
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kSC; ++q) {
                    const int sp = (c0 + cc) * kSC + q;
                    if (sp < a.S) {
#pragma unroll
                        for (int m = 0; m < kMaxF - 1; ++m) {
                            if (m < a.M) {
                                const T w = warp_sum(zv[q][m]);
                                if (lane == 0) s_part[warp][sp * a.M + m] = (double)w;
                            }
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < K; j += kB) {
        double t = 0.0;
        for (int w = 0; w < kW; ++w) t += s_part[w][j];
        a.partials[(size_t)blk * K + j] = t;
    }
    const long long cap = a.cap;
    double* Z = a.Z;
    double* D = a.D;
    long long* tdev = a.tdev;
    __shared__ long long s_t1;
    if (threadIdx.x == 0) s_t1 = *((volatile long long*)tdev) + 1;
    // s_t1 is only read by thread 0 of the last block, after the barriers in grid_total
    bool last = grid_total<kB>(a.partials, K, a.ticket, nblk, [&](int kk, double tot) {
        const long long t1 = s_t1;
        const double z = tot * a.zsc[kk / a.M];  // series kk = species * M + moment
        Z[(size_t)kk * cap + t1] = z;
        D[(size_t)kk * cap + t1] = D[(size_t)kk * cap + t1 - 1] + z;
    });
    if (last && threadIdx.x == 0) *tdev = s_t1;
}

// the multi-species body keeps two 32-byte chunks per link in flight; capping registers so
// that 768 threads stay resident per SM trades some of that load hoisting for occupancy
// (the single-species body fits in 32 registers, i.e. full occupancy at 256 threads)
// (FP32: the single-species body fits in 32 registers, full occupancy at 256 threads;
// FP64 needs twice the registers and is left uncapped)
constexpr int min_blocks(bool single, int block, int elem)
{
    return elem == 8 ? 1 : (single ? 2048 / block : (768 / block > 1 ? 768 / block : 1));
}

template <typename T, typename TS, int FP, bool kSingle>
__global__ void __launch_bounds__(kThreads, min_blocks(kSingle, kThreads, sizeof(T)))
    k_step(const __grid_constant__ Args<T> a, const TS* __restrict__ P, TS* __restrict__ Pn,
           const TS* __restrict__ A, TS* __restrict__ An)
{
    // launched with programmatic dependent launch: wait for the previous step's fields, Z/D
    // entries, partials and ticket before touching any of them
    pdl_enter();
    // __grid_constant__: step_body reads the arguments through a reference, straight from
    // the constant bank (without it the whole structure would be copied per thread)
    step_body<T, TS, FP, kSingle, kThreads>(a, blockIdx.x, gridDim.x, P, Pn, A, An);
}

// ---------------------------------------------------------------------------------------
// Grouped step: one launch advances several contexts (media of different sizes, each with
// its own species). Blocks [bofs[c], bofs[c+1]) work on context c; each context keeps its
// own partials, ticket and series, so the result equals separate launches with the same
// block size. The per-context arguments and the two phases' field pointers live in device
// memory owned by the group.
// ---------------------------------------------------------------------------------------
constexpr int kMaxGroup = 16;

struct GroupPtrs {
    const float* P;
    float* Pn;
    const float* A;
    float* An;
};

struct GroupArgs {
    const Args<float>* args;    // [n]
    const GroupPtrs* ptrs;      // [2][n]: field pointers of step phase 0 and 1
    int bofs[kMaxGroup + 1];    // block prefix
    int n;
};

template <int FP, bool kSingle, int kB>
__global__ void __launch_bounds__(kB, kSingle ? 1536 / kB : min_blocks(false, kB, 4))
    k_step_group(const GroupArgs g, int phase)
{
    // context of this block; constant indices only, so the parameter array stays in the
    // constant bank
    int c = 0, b0 = 0, b1 = g.bofs[1];
#pragma unroll
    for (int j = 1; j < kMaxGroup; ++j) {
        if (j < g.n && (int)blockIdx.x >= g.bofs[j]) {
            c = j;
            b0 = g.bofs[j];
            b1 = g.bofs[j + 1];
        }
    }
    pdl_enter();  // launched with programmatic dependent launch, like k_step
    const GroupPtrs p = g.ptrs[phase * g.n + c];
    step_body<float, float, FP, kSingle, kB>(g.args[c], (int)blockIdx.x - b0, b1 - b0, p.P, p.Pn, p.A, p.An);
}

// ---------------------------------------------------------------------------------------
// Initialisation: density at t = 1 (one step from its t = 0 state), velocity moments at
// t = 1 (P_g(r,1) = sum_i pi(r - c_i) p_i(r - c_i) c_ig, no adsorbed share), Z_g(0), Z_g(1).
// The free Boltzmann weight pi = 1/Z is the same on every fluid node (neutral tracer).
// ---------------------------------------------------------------------------------------
template <typename T, typename TS>
__global__ void __launch_bounds__(kThreads)
    k_init(const Args<T> a, const InitExtra b, TS* __restrict__ P1, TS* __restrict__ A1)
{
    const int k = blockIdx.x * kThreads + threadIdx.x;
    const bool active = k < a.NF;
    Node<T> d;
    if (active) load_node<T>(a, k, d);
    const size_t prows = a.compact ? (size_t)a.NF : (size_t)a.N;
    const size_t prow = a.compact ? (size_t)k : (size_t)d.n;
    const int K2 = 2 * a.S * a.M;
    for (int sp = 0; sp < a.S; ++sp) {
        const T hl = a.hl[sp], pa = a.pa[sp], pd = a.pd[sp];
        const T invZ = (T)b.invZ[sp];
        const T sc = (T)b.sc[sp];  // stored values are field values x sc
        T zp[2 * kMaxF] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        if (active) {
            T pin[kQ], pout[kQ];
            species_probs(d, hl, pin, pout);
            T out = T(0), inw = T(0);
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                out += pout[i];
                inw += pin[i];
            }
            const T stay = T(1) - out - (d.itf ? pa : T(0));
            // density field: X0 uniform over the free fluid (1/N_f or the free weight 1/Z),
            // adsorbed K/Z on the interface for the equilibrium start
            const T x0 = b.uniform ? (T)b.inv_nf : invZ;
            const T xa0 = (b.uniform || !d.itf) ? T(0) : (T)b.K[sp] * invZ;
            T xn = inw * x0 + stay * x0;
            if (d.itf) {
                const size_t ai = elem(a, a.NI, d.aidx, sp, 0);
                xn += pd * xa0;
                A1[ai] = Narrow<TS>::one((pa * x0 + (T(1) - pd) * xa0) * sc, 0u, false);
            }
            P1[elem(a, prows, prow, sp, 0)] = Narrow<TS>::one(xn * sc, 0u, false);
#pragma unroll
            for (int m = 0; m < kMaxF - 1; ++m) {
                if (m < a.M) {
                    const int g = a.dir[m];
                    T pg = T(0);
#pragma unroll
                    for (int i = 1; i < kQ; ++i)
                        if (ci(i, g) != 0) pg += pin[i] * T(ci(i, g));
                    pg *= invZ;
                    P1[elem(a, prows, prow, sp, 1 + m)] = Narrow<TS>::one(pg * sc, 0u, false);
                    if (d.itf) A1[elem(a, a.NI, d.aidx, sp, 1 + m)] = Narrow<TS>::one(T(0), 0u, false);
                    T us, us2;
                    mean_step(pout, g, us, us2);
                    zp[2 * m] = invZ * us2;
                    zp[2 * m + 1] = pg * us;
                }
            }
        }
        block_sum_store<T, 2 * kMaxF>(zp, 2 * a.M, a.partials + (size_t)blockIdx.x * K2 + sp * 2 * a.M);
    }
    const long long cap = a.cap;
    double* Z = a.Z;
    double* D = a.D;
    bool last = grid_total<kThreads>(a.partials, K2, a.ticket, (int)gridDim.x, [&](int kk, double tot) {
        const int series = kk / 2;
        if ((kk & 1) == 0) {
            Z[(size_t)series * cap + 0] = tot;
            D[(size_t)series * cap + 0] = tot / 2.0;
        } else {
            Z[(size_t)series * cap + 1] = tot;
            D[(size_t)series * cap + 1] = D[(size_t)series * cap + 0] + tot;
        }
    });
    if (last && threadIdx.x == 0) *a.tdev = 1;
}

// Count open links with p_i < 0 and nodes with a negative stay fraction, over species.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_negative(const Args<T> a, unsigned long long* __restrict__ counts)
{
    const int k = blockIdx.x * kThreads + threadIdx.x;
    if (k >= a.NF) return;
    Node<T> d;
    load_node<T>(a, k, d);
    for (int sp = 0; sp < a.S; ++sp) {
        T pin[kQ], pout[kQ];
        species_probs(d, a.hl[sp], pin, pout);
        unsigned neg = 0;
        T out = T(0);
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            neg += (d.src[i] >= 0 && pout[i] < T(0)) ? 1u : 0u;
            out += pout[i];
        }
        const T stay = T(1) - out - (d.itf ? a.pa[sp] : T(0));
        if (neg) atomicAdd(&counts[0], (unsigned long long)neg);
        if (stay < T(0)) atomicAdd(&counts[1], 1ull);
    }
}

// FP64 per-block partial sums of the density field of one species: sum_F P, sum_I Gamma,
// sum_I P.
template <typename T, typename TS>
__global__ void __launch_bounds__(kThreads)
    k_mass(const Args<T> a, int sp, const TS* __restrict__ P, const TS* __restrict__ A, double* __restrict__ out)
{
    const int k = blockIdx.x * kThreads + threadIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    if (k < a.NF) {
        const int n = __ldg(a.flist + k);
        v[0] = (double)widen1(P[a.compact ? elem(a, a.NF, k, sp, 0) : elem(a, a.N, n, sp, 0)]);
        const uint32_t bits = __ldg(a.iface + (n >> 5));
        if ((bits >> (n & 31)) & 1u) {
            const int j = __ldg(a.ibase + (n >> 5)) + __popc(bits & ((1u << (n & 31)) - 1u));
            v[1] = (double)widen1(A[elem(a, a.NI, j, sp, 0)]);
            v[2] = v[0];
        }
    }
    __shared__ double s[3][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double w = warp_sum(v[j]);
        if (lane == 0) s[j][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < kWarps; ++q) t += s[threadIdx.x][q];
        out[(size_t)blockIdx.x * 3 + threadIdx.x] = t;
    }
}

// Static flow data: Flow4 of every node (zero on solids) and the open mask of every fluid
// node. -3/2 |u|^2 is computed here once, so both ends of a link read the same value.
template <typename T>
__global__ void k_pack_flow(const float* __restrict__ in, const uint32_t* __restrict__ fluid, int N,
                            Flow4<T>* __restrict__ u4)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    Flow4<T> v{T(0), T(0), T(0), T(0)};
    if (in && bit_of(fluid, n)) {
        v.x = (T)in[n];
        v.y = (T)in[(size_t)N + n];
        v.z = (T)in[2 * (size_t)N + n];
        v.w = rn_mul(T(-1.5), rn_add(rn_add(rn_mul(v.x, v.x), rn_mul(v.y, v.y)), rn_mul(v.z, v.z)));
    }
    u4[n] = v;
}

__global__ void k_open_mask(const int32_t* __restrict__ flist, const uint32_t* __restrict__ fluid, int NF,
                            int nx, int ny, int nz, uint32_t* __restrict__ fmask)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NF) return;
    const int n = flist[k];
    const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    uint32_t m = 0;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        int xs = x - cx(i), ys = y - cy(i), zs = z - cz(i);
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        if (bit_of(fluid, xs + nx * (ys + ny * zs))) m |= 1u << (i - 1);
    }
    fmask[k] = m;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Context and C ABI
// ---------------------------------------------------------------------------------------

namespace {

template <typename T>
Args<T> make_args(const mp_ctx* c)
{
    Args<T> a;
    memset(&a, 0, sizeof(a));
    a.nx = c->geo.nx;
    a.ny = c->geo.ny;
    a.nz = c->geo.nz;
    a.N = c->geo.N;
    a.NF = (int)c->geo.n_fluid;
    a.NI = (int)c->geo.n_iface;
    a.FP = c->FP;
    a.SP = c->SP;
    a.SC = c->SC;
    a.compact = c->compact ? 1 : 0;
    a.dx = make_div((unsigned)c->geo.nx);
    a.dxy = make_div((unsigned)(c->geo.nx * c->geo.ny));
    a.iface = c->geo.iface;
    a.ibase = c->geo.ibase;
    a.flist = c->geo.flist;
    a.fmask = c->fmask;
    a.u4 = (const Flow4<T>*)c->u4;
    a.S = c->S;
    a.F = c->F;
    a.M = c->M;
    for (int m = 0; m < 3; ++m) a.dir[m] = c->dir[m];
    for (int s = 0; s < c->S; ++s) {
        a.hl[s] = (T)(6.0 * c->Db[s]);  // lambda/2 = 12 D_b / 2
        a.whf[s] = (T)((double)weight<T>(1) * (double)a.hl[s]);
        a.whe[s] = (T)((double)weight<T>(5) * (double)a.hl[s]);
        a.pa[s] = (T)c->ka[s];
        a.pd[s] = (T)c->kd[s];
    }
    for (int s = 0; s < c->S; ++s) a.zsc[s] = c->zsc[s];
    a.stochastic = c->stochastic;
    a.partials = c->partials;
    a.ticket = c->ticket;
    a.Z = c->Z;
    a.D = c->D;
    a.tdev = c->tdev;
    a.cap = c->cap;
    return a;
}

void destroy(mp_ctx* c)
{
    if (!c) return;
    direct_free(c);
    for (int b = 0; b < 2; ++b) {
        if (c->exec[b]) cudaGraphExecDestroy(c->exec[b]);
        if (c->graph[b]) cudaGraphDestroy(c->graph[b]);
    }
    free_geometry(&c->geo, nullptr, false);
    cudaFree(c->u4);
    cudaFree(c->fmask);
    for (int b = 0; b < 2; ++b) {
        cudaFree(c->P[b]);
        cudaFree(c->A[b]);
    }
    cudaFree(c->Z);
    cudaFree(c->D);
    cudaFree(c->tdev);
    cudaFree(c->partials);
    cudaFree(c->ticket);
    delete c;
}

template <typename T, typename TS>
int init_typed(mp_ctx* c, const float* u_in, int init_density)
{
    // binary16 storage keeps field values x Z_s (the partition function), so the
    // equilibrium free density is stored as 1; other storage types are unscaled
    double invZ[MP_MAX_SPECIES];
    for (int s = 0; s < c->S; ++s) {
        const double K = c->ka[s] == 0.0 ? 0.0 : c->ka[s] / c->kd[s];
        invZ[s] = 1.0 / ((double)c->geo.n_fluid + K * (double)c->geo.n_iface);
        c->zsc[s] = std::is_same<T, TS>::value ? 1.0 : invZ[s];
    }
    const int N = c->geo.N;
    const size_t NI = (size_t)(c->geo.n_iface > 0 ? c->geo.n_iface : 1);
    c->FP = c->F <= 2 ? 2 : 4;
    const int chunk = 8 / c->FP;  // species per 32-byte chunk of a node record
    c->SP = c->S == 1 ? 1 : (c->S + chunk - 1) / chunk * chunk;
    c->SC = c->S == 1 ? 1 : chunk;
    const size_t fieldN = (size_t)c->SP * (c->compact ? (size_t)c->geo.n_fluid : (size_t)N) * c->FP;
    const size_t fieldA = (size_t)c->SP * NI * c->FP;
    const int Kser = c->S * c->M;
    c->elem = sizeof(TS);
    c->blocks = (int)((c->geo.n_fluid + kThreads - 1) / kThreads);
    MP_CUDA(cudaMalloc(&c->u4, sizeof(Flow4<T>) * (size_t)N));
    MP_CUDA(cudaMalloc(&c->fmask, sizeof(uint32_t) * (size_t)c->geo.n_fluid));
    for (int b = 0; b < 2; ++b) {
        MP_CUDA(cudaMalloc(&c->P[b], sizeof(TS) * fieldN));
        MP_CUDA(cudaMalloc(&c->A[b], sizeof(TS) * fieldA));
        MP_CUDA(cudaMemsetAsync(c->P[b], 0, sizeof(TS) * fieldN, c->stream));
        MP_CUDA(cudaMemsetAsync(c->A[b], 0, sizeof(TS) * fieldA, c->stream));
    }
    MP_CUDA(cudaMalloc(&c->Z, sizeof(double) * (size_t)Kser * c->cap));
    MP_CUDA(cudaMalloc(&c->D, sizeof(double) * (size_t)Kser * c->cap));
    MP_CUDA(cudaMemsetAsync(c->Z, 0, sizeof(double) * (size_t)Kser * c->cap, c->stream));
    MP_CUDA(cudaMemsetAsync(c->D, 0, sizeof(double) * (size_t)Kser * c->cap, c->stream));
    MP_CUDA(cudaMalloc(&c->tdev, sizeof(long long)));
    MP_CUDA(cudaMemsetAsync(c->tdev, 0, sizeof(long long), c->stream));
    // per-block partials: 2 S M values (initialisation) or 3 (mass check), whichever is more
    const size_t per_block = (size_t)(2 * Kser > 3 ? 2 * Kser : 3);
    const size_t max_blocks = (size_t)((c->geo.n_fluid + 127) / 128);  // smallest group block size
    MP_CUDA(cudaMalloc(&c->partials, sizeof(double) * (max_blocks > (size_t)c->blocks ? max_blocks : c->blocks) * per_block));
    MP_CUDA(cudaMalloc(&c->ticket, sizeof(unsigned int)));
    MP_CUDA(cudaMemsetAsync(c->ticket, 0, sizeof(unsigned int), c->stream));
    k_pack_flow<T><<<(N + 255) / 256, 256, 0, c->stream>>>(u_in, c->geo.fluid, N, (Flow4<T>*)c->u4);
    k_open_mask<<<c->blocks, kThreads, 0, c->stream>>>(c->geo.flist, c->geo.fluid, (int)c->geo.n_fluid,
                                                        c->geo.nx, c->geo.ny, c->geo.nz, c->fmask);
    MP_CUDA(cudaGetLastError());

    Args<T> a = make_args<T>(c);
    // negative link probabilities / stay fractions
    unsigned long long* counts = nullptr;
    MP_CUDA(cudaMalloc(&counts, 2 * sizeof(unsigned long long)));
    cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), c->stream);
    k_negative<T><<<c->blocks, kThreads, 0, c->stream>>>(a, counts);
    unsigned long long h_counts[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_counts, counts, sizeof(h_counts), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(counts);
    if (e != cudaSuccess) return cuda_fail(e, "negative-probability check");
    c->n_neg_links = (long long)h_counts[0];
    c->n_neg_stay = (long long)h_counts[1];
    if (c->n_neg_stay > 0) {
        set_error("negative stay fraction 1 - sum_i p_i - p_a at " + std::to_string(c->n_neg_stay) +
                  " node-species (D_b, k_a or |u| too large)");
        return MP_ENEGPROB;
    }

    InitExtra b;
    memset(&b, 0, sizeof(b));
    for (int s = 0; s < c->S; ++s) {
        b.K[s] = c->ka[s] == 0.0 ? 0.0 : c->ka[s] / c->kd[s];
        b.invZ[s] = invZ[s];
        b.sc[s] = 1.0 / c->zsc[s];
    }
    b.inv_nf = 1.0 / (double)c->geo.n_fluid;
    b.uniform = init_density == MP_INIT_UNIFORM;
    k_init<T, TS><<<c->blocks, kThreads, 0, c->stream>>>(a, b, (TS*)c->P[0], (TS*)c->A[0]);
    MP_CUDA(cudaGetLastError());
    c->cur = 0;
    c->t = 1;
    return MP_OK;
}

// Long runs on a context with its own stream replay a CUDA graph of this many steps (even,
// so a replay ends on the buffer it started from); the launches are the same as plain ones.
constexpr int kCtxGraphSteps = 64;

bool capturable(cudaStream_t s)
{
    return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

template <typename T, typename TS>
int step_typed(mp_ctx* c, long long n)
{
    Args<T> a = make_args<T>(c);
    auto kern = c->FP == 2 ? (c->S == 1 ? k_step<T, TS, 2, true> : k_step<T, TS, 2, false>)
                           : (c->S == 1 ? k_step<T, TS, 4, true> : k_step<T, TS, 4, false>);
    cudaError_t le = cudaSuccess;  // first failed launch, if any
    auto launch = [&](long long count) {
        for (long long k = 0; k < count; ++k) {
            const int s = c->cur;
            const cudaError_t e = launch_pdl(kern, dim3(c->blocks), dim3(kThreads), c->stream, a, (const TS*)c->P[s],
                                             (TS*)c->P[1 - s], (const TS*)c->A[s], (TS*)c->A[1 - s]);
            if (e != cudaSuccess && le == cudaSuccess) le = e;
            c->cur = 1 - s;
        }
    };
    if (capturable(c->stream) && n >= 2 * kCtxGraphSteps) {
        const int b = c->cur;
        if (!c->exec[b]) {
            cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                launch(kCtxGraphSteps);
                e = cudaStreamEndCapture(c->stream, &c->graph[b]);
            }
            c->cur = b;
            if (e == cudaSuccess && le != cudaSuccess) e = le;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->exec[b], c->graph[b], 0);
            if (e != cudaSuccess) return cuda_fail(e, "mp_step: graph capture");
        }
        for (; n >= kCtxGraphSteps; n -= kCtxGraphSteps) {
            MP_CUDA(cudaGraphLaunch(c->exec[b], c->stream));
            c->t += kCtxGraphSteps;
        }
    }
    launch(n);
    c->t += n;
    if (le != cudaSuccess) return cuda_fail(le, "mp_step: launch");
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

template <typename T, typename TS>
int mass_typed(mp_ctx* c, int sp, double out[3])
{
    Args<T> a = make_args<T>(c);
    const TS* P = (const TS*)c->P[c->cur];
    const TS* A = (const TS*)c->A[c->cur];
    k_mass<T, TS><<<c->blocks, kThreads, 0, c->stream>>>(a, sp, P, A, c->partials);
    std::vector<double> h((size_t)c->blocks * 3);
    MP_CUDA(cudaGetLastError());
    MP_CUDA(cudaMemcpyAsync(h.data(), c->partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaStreamSynchronize(c->stream));
    out[0] = out[1] = out[2] = 0.0;
    for (int b = 0; b < c->blocks; ++b)
        for (int j = 0; j < 3; ++j) out[j] += h[(size_t)b * 3 + j];
    for (int j = 0; j < 3; ++j) out[j] *= c->zsc[sp];
    return MP_OK;
}

int check_ctx(const mp_ctx* c)
{
    if (!c) {
        set_error("context is NULL");
        return MP_EINVAL;
    }
    return MP_OK;
}

}  // namespace

extern "C" {

void mp_default_options(mp_options* opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->precision = MP_FP32;
    opt->directions = 1;
    opt->init_density = MP_INIT_EQUILIBRIUM;
    opt->allow_negative = 0;
    opt->capacity = 131072;
    opt->stream = nullptr;
    opt->rounding = MP_ROUND_STOCHASTIC;
    opt->scheme = MP_SCHEME_FLUX;
    opt->autotune = 0;
    opt->variant = 0;
}

const char* mp_last_error(void) { return mp::last_error_text(); }

int mp_init_batch(mp_ctx** out, const mp_geometry* g, const float* u, int n_species, const double* D_b,
                  const double* k_a, const double* k_d, const mp_options* opt_in)
{
    clear_error();
    if (!out) {
        set_error("out is NULL");
        return MP_EINVAL;
    }
    mp_options opt;
    mp_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.directions == 0) opt.directions = 1;
    if (opt.capacity == 0) opt.capacity = 131072;
    if (n_species < 1 || n_species > MP_MAX_SPECIES || !D_b || !k_a || !k_d) {
        set_error("n_species must be in 1..MP_MAX_SPECIES with non-NULL parameter arrays");
        return MP_EINVAL;
    }
    if (opt.precision != MP_FP32 && opt.precision != MP_FP64 && opt.precision != MP_FP16) {
        set_error("precision must be MP_FP32, MP_FP64 or MP_FP16");
        return MP_EINVAL;
    }
    if (opt.scheme != MP_SCHEME_FLUX && opt.scheme != MP_SCHEME_DIRECT) {
        set_error("scheme must be MP_SCHEME_FLUX or MP_SCHEME_DIRECT");
        return MP_EINVAL;
    }
    if (opt.variant < 0 || opt.variant > 31 || (opt.variant & 12) == 12) {
        set_error("variant must combine MP_VARIANT_* flags (one block size at most)");
        return MP_EINVAL;
    }
    if (opt.scheme == MP_SCHEME_DIRECT && opt.precision != MP_FP32) {
        set_error("MP_SCHEME_DIRECT needs MP_FP32 storage");
        return MP_EINVAL;
    }
    if (opt.rounding != MP_ROUND_STOCHASTIC && opt.rounding != MP_ROUND_NEAREST) {
        set_error("rounding must be MP_ROUND_STOCHASTIC or MP_ROUND_NEAREST");
        return MP_EINVAL;
    }
    if (opt.directions < 1 || opt.directions > 7) {
        set_error("directions must be a nonzero mask of 1 (x), 2 (y), 4 (z)");
        return MP_EINVAL;
    }
    if (opt.init_density != MP_INIT_EQUILIBRIUM && opt.init_density != MP_INIT_UNIFORM) {
        set_error("init_density must be MP_INIT_EQUILIBRIUM or MP_INIT_UNIFORM");
        return MP_EINVAL;
    }
    if (opt.capacity < 2 || opt.capacity > (1LL << 40)) {
        set_error("capacity must be >= 2");
        return MP_EINVAL;
    }
    for (int s = 0; s < n_species; ++s) {
        if (!(D_b[s] > 0.0 && D_b[s] <= 0.25)) {
            set_error("D_b must be in (0, 0.25] (lambda = 12 D_b <= 3 keeps the bulk stay >= 0)");
            return MP_EINVAL;
        }
        if (!(k_a[s] >= 0.0 && k_a[s] <= 1.0 && k_d[s] >= 0.0 && k_d[s] <= 1.0)) {
            set_error("k_a and k_d must be probabilities per step, in [0, 1]");
            return MP_EINVAL;
        }
        if (k_a[s] > 0.0 && k_d[s] == 0.0) {
            set_error("k_a > 0 with k_d = 0 has no equilibrium (Boltzmann weights need K = k_a/k_d)");
            return MP_EINVAL;
        }
        if (opt.precision == MP_FP16 && k_a[s] > 30000.0 * k_d[s]) {
            set_error("binary16 storage needs K = k_a/k_d <= 30000 (stored adsorbed values reach K)");
            return MP_EINVAL;
        }
    }
    mp_ctx* c = new (std::nothrow) mp_ctx();
    if (!c) {
        set_error("host allocation failed");
        return MP_ENOMEM;
    }
    c->precision = opt.precision;
    c->scheme = opt.scheme;
    c->stochastic = opt.rounding == MP_ROUND_STOCHASTIC;
    c->stream = (cudaStream_t)opt.stream;
    c->cap = opt.capacity;
    c->S = n_species;
    c->M = 0;
    for (int g = 0; g < 3; ++g)
        if (opt.directions & (1 << g)) c->dir[c->M++] = g;
    c->F = 1 + c->M;
    for (int s = 0; s < n_species; ++s) {
        c->Db[s] = D_b[s];
        c->ka[s] = k_a[s];
        c->kd[s] = k_d[s];
    }
    int rc = build_geometry(g, c->stream, false, true, &c->geo);
    if (rc != MP_OK) {
        delete c;
        return rc;
    }
    if (c->geo.n_fluid == 0) {
        set_error("the medium has no fluid node");
        destroy(c);
        return MP_EINVAL;
    }
    if (c->geo.n_iface > 0) {
        c->ilist.resize((size_t)c->geo.n_iface);
        cudaError_t e = cudaMemcpyAsync(c->ilist.data(), c->geo.ilist, sizeof(int32_t) * c->ilist.size(),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "interface list copy");
            destroy(c);
            return rc;
        }
    }
    c->compact = c->scheme == MP_SCHEME_DIRECT && c->S > 1;
    if (c->compact) {
        c->hflist.resize((size_t)c->geo.n_fluid);
        cudaError_t e = cudaMemcpyAsync(c->hflist.data(), c->geo.flist, sizeof(int32_t) * c->hflist.size(),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fluid list copy");
            destroy(c);
            return rc;
        }
    }
    rc = c->precision == MP_FP64   ? init_typed<double, double>(c, u, opt.init_density)
         : c->precision == MP_FP16 ? init_typed<float, __half>(c, u, opt.init_density)
                                   : init_typed<float, float>(c, u, opt.init_density);
    if (rc == MP_OK && c->n_neg_links > 0 && !opt.allow_negative) {
        set_error(std::to_string(c->n_neg_links) +
                  " open links have a negative probability p_i (set allow_negative to accept)");
        rc = MP_ENEGPROB;
    }
    if (rc == MP_OK && c->scheme == MP_SCHEME_DIRECT) rc = direct_setup(c, opt.autotune, opt.variant);
    if (rc != MP_OK) {
        destroy(c);
        return rc;
    }
    *out = c;
    return MP_OK;
}

int mp_init(mp_ctx** out, const mp_geometry* g, const float* u, double D_b, double k_a, double k_d,
            const mp_options* opt)
{
    return mp_init_batch(out, g, u, 1, &D_b, &k_a, &k_d, opt);
}

int mp_step(mp_ctx* c, int64_t n)
{
    clear_error();
    if (int rc = check_ctx(c)) return rc;
    if (n < 0) {
        set_error("n must be >= 0");
        return MP_EINVAL;
    }
    if (c->t + n > c->cap - 1) {
        set_error("the Z/D series is full: capacity " + std::to_string(c->cap) + " time points");
        return MP_EINVAL;
    }
    if (c->owner) {
        set_error("the context belongs to a group: step it with mp_group_step");
        return MP_EINVAL;
    }
    if (c->scheme == MP_SCHEME_DIRECT) return direct_step(c, n);
    return c->precision == MP_FP64   ? step_typed<double, double>(c, n)
           : c->precision == MP_FP16 ? step_typed<float, __half>(c, n)
                                     : step_typed<float, float>(c, n);
}

const char* mp_variant(mp_ctx* c)
{
    if (!c) return "";
    return c->scheme == MP_SCHEME_DIRECT ? direct_state_variant(c->dstate) : "flux";
}

int mp_vacf(mp_ctx* c, int species, int direction, double* Z, double* D, int64_t cap, int64_t* n_out)
{
    clear_error();
    if (int rc = check_ctx(c)) return rc;
    int m = -1;
    for (int k = 0; k < c->M; ++k)
        if (c->dir[k] == direction) m = k;
    if (species < 0 || species >= c->S || m < 0 || cap < 0) {
        set_error("species out of range, direction not propagated, or negative cap");
        return MP_EINVAL;
    }
    if (int rc = direct_check(c)) return rc;
    const long long avail = c->t + 1;
    const long long cnt = cap < avail ? cap : avail;
    const size_t off = (size_t)(species * c->M + m) * c->cap;
    if (cnt > 0 && Z) MP_CUDA(cudaMemcpyAsync(Z, c->Z + off, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
    if (cnt > 0 && D) MP_CUDA(cudaMemcpyAsync(D, c->D + off, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaStreamSynchronize(c->stream));
    if (n_out) *n_out = avail;
    return MP_OK;
}

int mp_mass(mp_ctx* c, int species, double out[3])
{
    clear_error();
    if (int rc = check_ctx(c)) return rc;
    if (species < 0 || species >= c->S || !out) {
        set_error("species out of range or out is NULL");
        return MP_EINVAL;
    }
    if (int rc = direct_check(c)) return rc;
    return c->precision == MP_FP64   ? mass_typed<double, double>(c, species, out)
           : c->precision == MP_FP16 ? mass_typed<float, __half>(c, species, out)
                                     : mass_typed<float, float>(c, species, out);
}

int mp_info(mp_ctx* c, mp_info_t* info)
{
    clear_error();
    if (int rc = check_ctx(c)) return rc;
    if (!info) {
        set_error("info is NULL");
        return MP_EINVAL;
    }
    info->n_nodes = c->geo.N;
    info->n_fluid = c->geo.n_fluid;
    info->n_interface = c->geo.n_iface;
    info->n_negative_links = c->n_neg_links;
    info->t = c->t;
    info->n_species = c->S;
    info->n_fields = c->F;
    info->precision = c->precision;
    return MP_OK;
}

int mp_get_field(mp_ctx* c, int species, int field, double* free_dense, double* ads_dense)
{
    clear_error();
    if (int rc = check_ctx(c)) return rc;
    if (species < 0 || species >= c->S || field < 0 || field >= c->F || !free_dense) {
        set_error("species or field out of range, or free_dense is NULL");
        return MP_EINVAL;
    }
    if (int rc = direct_check(c)) return rc;
    const size_t N = (size_t)c->geo.N;
    const size_t NI = (size_t)(c->geo.n_iface > 0 ? c->geo.n_iface : 1);
    const size_t FP = (size_t)c->FP, SP = (size_t)c->SP, E = c->elem;
    const size_t rowsP = c->compact ? c->hflist.size() : N;
    std::vector<char> buf(rowsP * SP * FP * E), abuf(NI * SP * FP * E);
    MP_CUDA(cudaMemcpyAsync(buf.data(), c->P[c->cur], buf.size(), cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaMemcpyAsync(abuf.data(), c->A[c->cur], abuf.size(), cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaStreamSynchronize(c->stream));
    const size_t SC = (size_t)c->SC;
    const double zsc = c->zsc[species];
    auto at = [&](const std::vector<char>& v, size_t i) {
        const size_t rows = &v == &buf ? rowsP : NI;
        const size_t j = ((((size_t)species / SC) * rows + i) * SC + (size_t)species % SC) * FP + (size_t)field;
        if (E == 8) return ((const double*)v.data())[j];
        if (E == 4) return (double)((const float*)v.data())[j];
        return (double)__half2float(((const __half*)v.data())[j]) * zsc;
    };
    if (c->compact) {
        for (size_t n = 0; n < N; ++n) free_dense[n] = 0.0;
        for (size_t k = 0; k < rowsP; ++k) free_dense[c->hflist[k]] = at(buf, k);
    } else {
        for (size_t n = 0; n < N; ++n) free_dense[n] = at(buf, n);
    }
    if (ads_dense) {
        for (size_t n = 0; n < N; ++n) ads_dense[n] = 0.0;
        for (size_t k = 0; k < c->ilist.size(); ++k) ads_dense[c->ilist[k]] = at(abuf, k);
    }
    return MP_OK;
}

int mp_set_field(mp_ctx* c, int species, int field, const double* free_dense, const double* ads_dense)
{
    clear_error();
    if (int rc = check_ctx(c)) return rc;
    if (species < 0 || species >= c->S || field < 0 || field >= c->F || !free_dense) {
        set_error("species or field out of range, or free_dense is NULL");
        return MP_EINVAL;
    }
    const size_t N = (size_t)c->geo.N;
    const size_t NI = (size_t)(c->geo.n_iface > 0 ? c->geo.n_iface : 1);
    const size_t FP = (size_t)c->FP, SP = (size_t)c->SP, E = c->elem;
    // read the node records, replace one species' field, write them back; solids stay zero
    const size_t rowsP = c->compact ? c->hflist.size() : N;
    std::vector<uint32_t> fl((size_t)c->geo.W);
    std::vector<char> buf(rowsP * SP * FP * E), abuf(NI * SP * FP * E);
    MP_CUDA(cudaMemcpyAsync(fl.data(), c->geo.fluid, fl.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaMemcpyAsync(buf.data(), c->P[c->cur], buf.size(), cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaMemcpyAsync(abuf.data(), c->A[c->cur], abuf.size(), cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(cudaStreamSynchronize(c->stream));
    const size_t SC = (size_t)c->SC;
    const double zsc = c->zsc[species];
    auto put = [&](std::vector<char>& v, size_t i, double x) {
        const size_t rows = &v == &buf ? rowsP : NI;
        const size_t j = ((((size_t)species / SC) * rows + i) * SC + (size_t)species % SC) * FP + (size_t)field;
        if (E == 8)
            ((double*)v.data())[j] = x;
        else if (E == 4)
            ((float*)v.data())[j] = (float)x;
        else
            ((__half*)v.data())[j] = __float2half_rn((float)(x / zsc));
    };
    if (c->compact) {
        for (size_t k = 0; k < rowsP; ++k) put(buf, k, free_dense[c->hflist[k]]);
    } else {
        for (size_t n = 0; n < N; ++n) put(buf, n, ((fl[n >> 5] >> (n & 31)) & 1u) ? free_dense[n] : 0.0);
    }
    for (size_t k = 0; k < c->ilist.size(); ++k) put(abuf, k, ads_dense ? ads_dense[c->ilist[k]] : 0.0);
    MP_CUDA(cudaMemcpyAsync(c->P[c->cur], buf.data(), buf.size(), cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(cudaMemcpyAsync(c->A[c->cur], abuf.data(), abuf.size(), cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(cudaStreamSynchronize(c->stream));
    return MP_OK;
}

void mp_free(mp_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    destroy(c);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Groups: several FP32 contexts advanced by one launch per step (k_step_group), with an
// autotuned block size and CUDA-graph replay of runs of steps.
// ---------------------------------------------------------------------------------------
struct mp_group {
    std::vector<mp_ctx*> ctx;
    int FP = 2;
    bool single = true;
    int block = kThreads;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Args<float>* d_args = nullptr;
    GroupPtrs* d_ptrs = nullptr;
    GroupArgs ga;
    int phase = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_steps = 0;
    mp::DirectState* direct = nullptr;  // a group of MP_SCHEME_DIRECT contexts
};

namespace {

void group_set_block(mp_group* g, int block)
{
    g->block = block;
    g->ga.bofs[0] = 0;
    for (size_t c = 0; c < g->ctx.size(); ++c)
        g->ga.bofs[c + 1] = g->ga.bofs[c] + (int)((g->ctx[c]->geo.n_fluid + block - 1) / block);
}

template <int FP, bool kSingle>
cudaError_t launch_group_fp(mp_group* g)
{
    const int blocks = g->ga.bofs[g->ctx.size()];
    if (g->block == 128)
        return launch_pdl(k_step_group<FP, kSingle, 128>, dim3(blocks), dim3(128), g->stream, g->ga, g->phase);
    if (g->block == 512)
        return launch_pdl(k_step_group<FP, kSingle, 512>, dim3(blocks), dim3(512), g->stream, g->ga, g->phase);
    return launch_pdl(k_step_group<FP, kSingle, 256>, dim3(blocks), dim3(256), g->stream, g->ga, g->phase);
}

// one grouped step: launch, then advance every context's phase, buffer and time
cudaError_t group_launch(mp_group* g, bool advance_ctx)
{
    const cudaError_t e = g->FP == 2 ? (g->single ? launch_group_fp<2, true>(g) : launch_group_fp<2, false>(g))
                                     : (g->single ? launch_group_fp<4, true>(g) : launch_group_fp<4, false>(g));
    g->phase ^= 1;
    if (advance_ctx)
        for (mp_ctx* c : g->ctx) {
            c->cur ^= 1;
            c->t += 1;
        }
    return e;
}

int group_sync_in(mp_group* g)
{
    for (mp_ctx* c : g->ctx) {
        MP_CUDA(cudaEventRecord(g->ev, c->stream));
        MP_CUDA(cudaStreamWaitEvent(g->stream, g->ev, 0));
    }
    return MP_OK;
}

int group_sync_out(mp_group* g)
{
    MP_CUDA(cudaEventRecord(g->ev, g->stream));
    for (mp_ctx* c : g->ctx) MP_CUDA(cudaStreamWaitEvent(c->stream, g->ev, 0));
    return MP_OK;
}

// Time `steps` grouped steps at each candidate block size on the current state, restoring
// fields, adsorbed arrays, buffers, times and series counters after each trial.
int group_autotune(mp_group* g, int steps)
{
    const int cand[3] = {128, 256, 512};
    std::vector<void*> bP(g->ctx.size(), nullptr), bA(g->ctx.size(), nullptr);
    std::vector<size_t> nP(g->ctx.size()), nA(g->ctx.size());
    int rc = MP_OK;
    for (size_t c = 0; c < g->ctx.size() && rc == MP_OK; ++c) {
        mp_ctx* x = g->ctx[c];
        const size_t NI = (size_t)(x->geo.n_iface > 0 ? x->geo.n_iface : 1);
        nP[c] = (size_t)x->SP * x->geo.N * x->FP * sizeof(float);
        nA[c] = (size_t)x->SP * NI * x->FP * sizeof(float);
        if (cudaMalloc(&bP[c], nP[c]) != cudaSuccess || cudaMalloc(&bA[c], nA[c]) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("autotune: no device memory for the state backup");
            rc = MP_ENOMEM;
        }
    }
    std::vector<int> cur0(g->ctx.size());
    std::vector<long long> t0(g->ctx.size());
    for (size_t c = 0; c < g->ctx.size(); ++c) {
        cur0[c] = g->ctx[c]->cur;
        t0[c] = g->ctx[c]->t;
    }
    const int phase0 = g->phase;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == MP_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        set_error("autotune: event creation failed");
        rc = MP_ECUDA;
    }
    float best_ms = 1e30f;
    int best = g->block;
    for (int k = 0; k < 3 && rc == MP_OK; ++k) {
        cudaError_t e = cudaSuccess;
        for (size_t c = 0; c < g->ctx.size() && e == cudaSuccess; ++c) {
            mp_ctx* x = g->ctx[c];
            e = cudaMemcpyAsync(bP[c], x->P[x->cur], nP[c], cudaMemcpyDeviceToDevice, g->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(bA[c], x->A[x->cur], nA[c], cudaMemcpyDeviceToDevice, g->stream);
        }
        group_set_block(g, cand[k]);
        if (e == cudaSuccess) e = group_launch(g, false);  // warm-up launch of this configuration
        if (e == cudaSuccess) e = cudaEventRecord(e0, g->stream);
        for (int s2 = 0; s2 < steps && e == cudaSuccess; ++s2) e = group_launch(g, false);
        if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        // restore the state the trial started from
        g->phase = phase0;
        for (size_t c = 0; c < g->ctx.size() && e == cudaSuccess; ++c) {
            mp_ctx* x = g->ctx[c];
            e = cudaMemcpyAsync(x->P[cur0[c]], bP[c], nP[c], cudaMemcpyDeviceToDevice, g->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(x->A[cur0[c]], bA[c], nA[c], cudaMemcpyDeviceToDevice, g->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(x->tdev, &t0[c], sizeof(long long), cudaMemcpyHostToDevice, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune");
            break;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[k];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (size_t c = 0; c < g->ctx.size(); ++c) {
        cudaFree(bP[c]);
        cudaFree(bA[c]);
    }
    group_set_block(g, best);
    return rc;
}

void group_destroy(mp_group* g)
{
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->direct) direct_state_free(g->direct);
    for (mp_ctx* c : g->ctx) c->owner = nullptr;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->d_args);
    cudaFree(g->d_ptrs);
    if (g->ev) cudaEventDestroy(g->ev);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

}  // namespace

extern "C" {

int mp_group_create(mp_group** out, mp_ctx* const* ctxs, int n, int graph_steps, int autotune)
{
    return mp_group_create_ex(out, ctxs, n, graph_steps, autotune, 0);
}

int mp_group_create_ex(mp_group** out, mp_ctx* const* ctxs, int n, int graph_steps, int autotune, int variant)
{
    clear_error();
    if (!out || !ctxs || n < 1 || n > kMaxGroup || graph_steps < 0 || graph_steps % 2) {
        set_error("mp_group_create: need 1..16 contexts and an even graph_steps >= 0");
        return MP_EINVAL;
    }
    if (variant < 0 || variant > 31 || (variant & 12) == 12) {
        set_error("mp_group_create_ex: variant must combine MP_VARIANT_* flags (one block size at most)");
        return MP_EINVAL;
    }
    for (int c = 0; c < n; ++c) {
        if (!ctxs[c] || ctxs[c]->precision != MP_FP32 || ctxs[c]->owner || ctxs[c]->FP != ctxs[0]->FP ||
            ctxs[c]->scheme != ctxs[0]->scheme) {
            set_error("mp_group_create: contexts must be distinct, FP32, ungrouped, with the same field layout "
                      "and scheme");
            return MP_EINVAL;
        }
        for (int d = 0; d < c; ++d)
            if (ctxs[d] == ctxs[c]) {
                set_error("mp_group_create: a context is listed twice");
                return MP_EINVAL;
            }
    }
    mp_group* g = new (std::nothrow) mp_group();
    if (!g) {
        set_error("host allocation failed");
        return MP_ENOMEM;
    }
    g->ctx.assign(ctxs, ctxs + n);
    g->FP = ctxs[0]->FP;
    g->single = true;
    for (mp_ctx* c : g->ctx) g->single = g->single && c->S == 1;
    g->ga.n = n;
    int rc = MP_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming);
    if (e == cudaSuccess && ctxs[0]->scheme == MP_SCHEME_DIRECT) {
        // a direct group: its own launch state over the contexts, on the group's stream
        rc = group_sync_in(g);
        if (rc == MP_OK) rc = direct_state_create(ctxs, n, g->stream, autotune, variant, &g->direct);
        if (rc != MP_OK) {
            group_destroy(g);
            return rc;
        }
        for (mp_ctx* c : g->ctx) c->owner = g;
        *out = g;
        return MP_OK;
    }
    if (e == cudaSuccess) e = cudaMalloc(&g->d_args, sizeof(Args<float>) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_ptrs, sizeof(GroupPtrs) * 2 * n);
    if (e == cudaSuccess) {
        std::vector<Args<float>> h_args(n);
        std::vector<GroupPtrs> h_ptrs(2 * n);
        for (int c = 0; c < n; ++c) {
            mp_ctx* x = g->ctx[c];
            h_args[c] = make_args<float>(x);
            for (int ph = 0; ph < 2; ++ph) {
                const int in = (x->cur + ph) & 1;
                h_ptrs[ph * n + c] = GroupPtrs{(const float*)x->P[in], (float*)x->P[1 - in], (const float*)x->A[in],
                                               (float*)x->A[1 - in]};
            }
        }
        e = cudaMemcpy(g->d_args, h_args.data(), sizeof(Args<float>) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_ptrs, h_ptrs.data(), sizeof(GroupPtrs) * 2 * n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "mp_group_create");
        group_destroy(g);
        return rc;
    }
    g->ga.args = g->d_args;
    g->ga.ptrs = g->d_ptrs;
    group_set_block(g, kThreads);
    for (mp_ctx* c : g->ctx) c->owner = g;
    if (autotune) {
        long long room = LLONG_MAX;
        for (mp_ctx* c : g->ctx) room = std::min(room, c->cap - 1 - c->t);
        if (room < 1) {
            set_error("mp_group_create: autotune needs free room in every Z/D series");
            group_destroy(g);
            return MP_EINVAL;
        }
        rc = group_sync_in(g);
        if (rc == MP_OK) rc = group_autotune(g, 20);
        if (rc != MP_OK) {
            group_destroy(g);
            return rc;
        }
    }
    if (graph_steps > 0) {
        // graph_steps launches alternating the two phases, starting at phase 0
        const int phase0 = g->phase;
        g->phase = 0;
        e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = cudaSuccess;
            for (int k = 0; k < graph_steps; ++k) {
                const cudaError_t e2 = group_launch(g, false);
                if (le == cudaSuccess) le = e2;
            }
            e = cudaStreamEndCapture(g->stream, &g->graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
        g->phase = phase0;
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "mp_group_create: graph capture");
            group_destroy(g);
            return rc;
        }
        g->graph_steps = graph_steps;
    }
    *out = g;
    return MP_OK;
}

int mp_group_step(mp_group* g, int64_t n)
{
    clear_error();
    if (!g || n < 0) {
        set_error("mp_group_step: group is NULL or n < 0");
        return MP_EINVAL;
    }
    for (mp_ctx* c : g->ctx)
        if (c->t + n > c->cap - 1) {
            set_error("mp_group_step: a context's Z/D series is full");
            return MP_EINVAL;
        }
    if (int rc = group_sync_in(g)) return rc;
    if (g->direct) {
        if (int rc = direct_state_step(g->direct, n)) return rc;
        return group_sync_out(g);
    }
    while (n > 0 && g->graph_steps > 0 && g->phase != 0) {
        MP_CUDA(group_launch(g, true));
        --n;
    }
    while (g->graph_steps > 0 && n >= g->graph_steps) {
        MP_CUDA(cudaGraphLaunch(g->exec, g->stream));
        for (mp_ctx* c : g->ctx) {
            c->cur = (c->cur + g->graph_steps) & 1;
            c->t += g->graph_steps;
        }
        n -= g->graph_steps;
    }
    while (n > 0) {
        MP_CUDA(group_launch(g, true));
        --n;
    }
    MP_CUDA(cudaGetLastError());
    return group_sync_out(g);
}

int mp_group_block_size(mp_group* g)
{
    if (g && g->direct) return direct_state_block(g->direct);
    return g ? g->block : 0;
}

const char* mp_group_variant(mp_group* g)
{
    if (!g) return "";
    return g->direct ? direct_state_variant(g->direct) : "flux";
}

void mp_group_free(mp_group* g) { group_destroy(g); }

}  // extern "C"
