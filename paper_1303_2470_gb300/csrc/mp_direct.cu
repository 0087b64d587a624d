// mp_direct.cu -- the moment-propagation + sorption step in the paper's direct form
// (Sec. "Algorithm", Eq. propagated_quantity with Eqs. Pads and newP, reading R1):
//   X'(r)  = sum_i p_i(r - c_i) X(r - c_i) + X(r) (1 - sum_i p_i(r) - p_a 1_I(r)) + p_d Xa(r)
//   Xa'(r) = p_a X(r) + (1 - p_d) Xa(r)
// evaluated as X' = [inflow - out(r) X(r)] + X(r) (+ p_d Xa), out(r) = sum_i p_i(r) + p_a 1_I.
//
// The flow is steady, so everything that depends on it alone is tabulated once per context:
// for every fluid node the probabilities of its 18 incoming links (one species) or their
// flow-dependent parts q_i (several species: p = w_i q_i + w_i lambda/2, one fused
// multiply-add per species), the outgoing sum out(r) and the mean displacement
// u*_g(r) = sum_i p_i(r) c_ig of the VACF sum Z_g = sum_r P_g(r) u*_g(r). A step then costs,
// per link, one coalesced table load, one gather of the source's field record and one
// fused multiply-add per field. The link values are bitwise those of the flux scheme
// (mp.cu). One species keeps dense fields: links into solid nodes meet zero fields (solid
// entries are never written), so that inflow needs no open-link test. Several species keep
// their fields for the fluid nodes only and locate each open link's source in the fluid list
// (lattice.cuh); closed links are skipped. A variant recomputes q_i from the flow vector of
// the source instead of reading the table (less memory traffic, more arithmetic), and for
// several species a tiled variant stages planes of the medium in shared memory.
//
// Unlike the flux scheme, total mass is not conserved to the last bit: the FP32 rounding
// of out(r) is a fixed relative error per node and step (below 2^-25 of X(r) for out < 1/2),
// of random sign across the nodes of a porous medium.
//
// Launch forms: one launch per step (programmatic dependent launch; CUDA-graph replay on
// streams that can be captured), or one persistent cooperative launch for a run of steps,
// with a device-wide barrier between steps whose waits are bounded in time (a wait that
// gives up sets an error flag that the host reports as MP_ETIMEOUT). Several contexts
// (media of any size, each with its own species) can share one launch: work is cut into
// virtual blocks of `block` fluid nodes, numbered context after context.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"
#include "lattice.cuh"
#include "link_arith.cuh"
#include "mp_ctx.cuh"

namespace mp {

struct DirectTables {
    int32_t* flist = nullptr;   // [NF] the work list of the step (fluid nodes, ascending)
    uint32_t* fmask = nullptr;  // [NF] open-link mask, bit i-1: the source r - c_i is fluid
    int32_t* aidx = nullptr;  // [NF] compact interface index, -1 off the interface
    float* tab = nullptr;     // incoming p_i (one species) or q_i (several), warp-blocked (tab_at)
    float* own = nullptr;     // [NF][OW] per-node record, see k_direct_tables
    int OW = 0;               // floats per node record
    // several species (fields over the fluid list): {fluid bits, fluid nodes before the
    // word} per 32-node word, and the flow vector of every fluid node in list order
    uint2* fw = nullptr;
    uint2* iw = nullptr;  // {interface bits, interfacial nodes before the word} per word
    Flow4<float>* uc = nullptr;
};

namespace {

constexpr int kMaxCtx = 16;
constexpr int kMaxSeries = MP_MAX_SPECIES * 3;
constexpr uint32_t kAll = (1u << 18) - 1u;
constexpr int kGraphSteps = 64;
constexpr int kMaxPersistentSteps = 1 << 20;  // barrier counter stays below 2^32
constexpr long long kWaitNs = 2000000000LL;   // a grid barrier wait gives up after 2 s

// Resident threads per SM that the register budget of the step kernels is set for (64
// registers a thread: measured faster than full occupancy, since a thread then keeps more
// of its independent link loads in flight), and the 32-byte chunks of species per pass of
// the several-species link loop.
#ifndef MP_DIRECT_SINGLE_THREADS
#define MP_DIRECT_SINGLE_THREADS 1024
#endif
#ifndef MP_DIRECT_MULTI_THREADS
#define MP_DIRECT_MULTI_THREADS 1024
#endif
#ifndef MP_DIRECT_CP
#define MP_DIRECT_CP 1
#endif

struct DArgs {
    int nx, ny, nz, N, NF, NI;
    Div dx, dxy;
    int S, M, SP, K;
    int dir[3];
    int in0;  // buffer read at phase 0
    int nvb;  // virtual blocks of this context
    int ntx, nty, tz;  // tiled variant: tiles along x and y, planes per tile
    const int32_t* flist;
    const uint32_t* fmask;  // open-link mask of each fluid node (bit i-1: source r - c_i is fluid)
    const int32_t* aidx;
    const float* tab;
    const float* own;
    const Flow4<float>* u4;
    const uint2* fw;          // several species: fluid bits and prefix per 32-node word
    const uint2* iw;          // several species: interface bits and prefix per 32-node word
    const Flow4<float>* uc;   // several species: flow of each fluid node, list order
    float* P[2];
    float* A[2];
    float whf[MP_MAX_SPECIES], whe[MP_MAX_SPECIES], pa[MP_MAX_SPECIES], pd[MP_MAX_SPECIES];
    double* part;  // [2][slots][K] partial sums of the K = S*M series, by step parity
    double* Z;
    double* D;
    long long* tdev;
    long long cap;
};

struct DLaunch {
    const DArgs* args;          // [n], device
    int vbofs[kMaxCtx + 1];     // virtual-block prefix over the contexts
    int n;
};

// Link table layout: the 18 values of 32 consecutive work items are stored together, link
// by link ([NF/32][18][32]), so a warp reads one 128-byte line per link and a run of work
// items reads one contiguous stretch of memory.
__host__ __device__ __forceinline__ size_t tab_at(int k, int i)
{
    return ((size_t)(k >> 5) * 18 + (size_t)(i - 1)) * 32 + (size_t)(k & 31);
}

// ---- field loads: read-only (non-coherent path) inside a one-step launch; plain loads in
// the persistent kernel, where the fields read in a step were written earlier in the launch
template <bool kCoherent, int W>
__device__ __forceinline__ FieldVec<float, W> ld_field(const FieldVec<float, W>* p)
{
    FieldVec<float, W> r;
    if constexpr (W == 2) {
        if constexpr (kCoherent)
            asm volatile("ld.global.v2.f32 {%0,%1}, [%2];" : "=f"(r.v[0]), "=f"(r.v[1]) : "l"(p) : "memory");
        else
            asm("ld.global.nc.v2.f32 {%0,%1}, [%2];" : "=f"(r.v[0]), "=f"(r.v[1]) : "l"(p));
    } else if constexpr (W == 4) {
        if constexpr (kCoherent)
            asm volatile("ld.global.v4.f32 {%0,%1,%2,%3}, [%4];"
                         : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
                         : "l"(p)
                         : "memory");
        else
            asm("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
                : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
                : "l"(p));
    } else {
        static_assert(W == 8, "records of 2, 4 or 8 floats");
        if constexpr (kCoherent)
            asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]),
                           "=f"(r.v[6]), "=f"(r.v[7])
                         : "l"(p)
                         : "memory");
        else
            asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]),
                  "=f"(r.v[6]), "=f"(r.v[7])
                : "l"(p));
    }
    return r;
}

template <int W>
__device__ __forceinline__ void st_field(FieldVec<float, W>* p, const FieldVec<float, W>& r)
{
    if constexpr (W == 8) {
        st_rec<float, 8>(p, r);
    } else {
        *p = r;
    }
}

__device__ __forceinline__ Flow4<float> ld_flow(const Flow4<float>* p)
{
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return Flow4<float>{v.x, v.y, v.z, v.w};
}

// Block sums of `cnt` series values held by every thread (FP32 within a warp, FP64 across
// warps in a fixed order); thread j < cnt writes the total of series j to out[j].
template <int kB, int kN>
__device__ __forceinline__ void block_partials(double (*s_red)[kMaxSeries], int cnt, const float (&v)[kN])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kN; ++j) {
        if (j < cnt) {
            const float w = warp_sum(v[j]);
            if (lane == 0) s_red[warp][j] = (double)w;
        }
    }
}

// Thread j < cnt adds series j over the warps (FP64, fixed order) and stores it to out[j], or
// adds it to out[j] (a shared accumulator owned by thread j) when `accumulate`.
template <int kB>
__device__ __forceinline__ void block_store(double (*s_red)[kMaxSeries], int cnt, double* out, bool accumulate)
{
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kB) {
        double t = 0.0;
        for (int w = 0; w < kB / 32; ++w) t += s_red[w][j];
        out[j] = accumulate ? out[j] + t : t;
    }
    __syncthreads();
}

// streamed per-node data (read once per step, no reuse): kept out of L1
__device__ __forceinline__ float ld_stream(const float* p)
{
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_stream(const int32_t* p)
{
    int v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p)
{
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

// ---------------------------------------------------------------------------------------
// One virtual block of one context: fluid nodes vb*kB .. vb*kB + kB - 1 of its work list.
// Reads buffer `in`, writes 1 - in. One species: each thread adds its node's Z terms to
// zacc (FP32, reduced over the block by the caller); links into solid nodes are skipped.
// ---------------------------------------------------------------------------------------
template <int FP, bool kTable, bool kCoherent, int kB>
__device__ __forceinline__ void vblock_single(const DArgs& a, int vb, int in, float (&zacc)[3])
{
    using V = FieldVec<float, FP>;
    const V* Pin = reinterpret_cast<const V*>(a.P[in]);
    V* Pout = reinterpret_cast<V*>(a.P[1 - in]);
    const V* Ain = reinterpret_cast<const V*>(a.A[in]);
    V* Aout = reinterpret_cast<V*>(a.A[1 - in]);
    const int k = vb * kB + threadIdx.x;
    const int M = a.M;
    if (k < a.NF) {
        const int n = ld_stream(a.flist + k);
        const uint32_t mask = kTable ? kAll : ld_stream(a.fmask + k);
        const int ai = ld_stream(a.aidx + k);
        float out, us[3];
        if constexpr (FP == 2) {
            const float2 o = ld_stream(reinterpret_cast<const float2*>(a.own) + k);
            out = o.x;
            us[0] = o.y;
            us[1] = us[2] = 0.f;
        } else {
            const float4 o = ld_stream(reinterpret_cast<const float4*>(a.own) + k);
            out = o.x;
            us[0] = o.y;
            us[1] = o.z;
            us[2] = o.w;
        }
        const Nbr b = nbrs_of(a.nx, a.ny, a.nz, a.dx, a.dxy, n);
        const float whf = a.whf[0], whe = a.whe[0];
        float acc[FP];
#pragma unroll
        for (int f = 0; f < FP; ++f) acc[f] = 0.f;
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            // with the table, closed links read p = 0 and a zero field (no dependence on the
            // mask, so all table loads issue at once); recomputing, they are skipped
            if (kTable || ((mask >> (i - 1)) & 1u)) {
                const int s = src_of(b, i);
                float p;
                if constexpr (kTable) {
                    p = ld_stream(a.tab + tab_at(k, i));
                } else {
                    const Flow4<float> uf = ld_flow(a.u4 + s);
                    p = rn_fma(weight<float>(i), qlink(edot<float>(i, uf.x, uf.y, uf.z), uf.w), is_face(i) ? whf : whe);
                }
                const V xs = ld_field<kCoherent, FP>(Pin + s);
#pragma unroll
                for (int f = 0; f < FP; ++f) acc[f] = __fmaf_rn(p, xs.v[f], acc[f]);
            }
        }
        const V xr = ld_field<kCoherent, FP>(Pin + n);
        V xn;
#pragma unroll
        for (int f = 0; f < FP; ++f) xn.v[f] = __fadd_rn(__fmaf_rn(-out, xr.v[f], acc[f]), xr.v[f]);
        if (ai >= 0) {
            const float pa = a.pa[0], pd = a.pd[0];
            const V xa = ld_field<kCoherent, FP>(Ain + ai);
            V xan;
#pragma unroll
            for (int f = 0; f < FP; ++f) {
                xn.v[f] = __fmaf_rn(pd, xa.v[f], xn.v[f]);
                xan.v[f] = __fmaf_rn(pa, xr.v[f], __fmaf_rn(-pd, xa.v[f], xa.v[f]));
            }
            st_field<FP>(Aout + ai, xan);
        }
        st_field<FP>(Pout + n, xn);
#pragma unroll
        for (int m = 0; m < 3; ++m)
            if (m < M && 1 + m < FP) zacc[m] = __fmaf_rn(xn.v[(1 + m) < FP ? 1 + m : 0], us[m], zacc[m]);
    }
}

// block sums of the per-thread single-species Z sums: stored to out[0..M), or added to a
// shared accumulator
template <int kB>
__device__ __forceinline__ void reduce_zacc(double (*s_red)[kMaxSeries], int M, const float (&zacc)[3], double* out,
                                            bool accumulate)
{
    block_partials<kB, 3>(s_red, M, zacc);
    block_store<kB>(s_red, M, out, accumulate);
}

// Several species: fields chunk-major over the fluid list, [chunk][k][8 floats] with 8/FP
// species per chunk (k = index in the sorted fluid list = work item). The link loop is
// outermost within a pass of up to two chunks: q_i is read (or recomputed) once per link and
// serves every species of both chunks. Sources are located in the fluid list by row (above).
template <int FP, bool kTable, bool kCoherent, int kB>
__device__ __forceinline__ void vblock_multi(const DArgs& a, int vb, int in, double* part, bool acc_part,
                                             double (*s_red)[kMaxSeries], const float* s_whf, const float* s_whe,
                                             const float* s_pa, const float* s_pd)
{
    constexpr int kSC = 8 / FP;
    constexpr int kCP = MP_DIRECT_CP;
    constexpr int kMaxPass = MP_MAX_SPECIES / (kCP * kSC);
    constexpr int kOW4 = FP == 2 ? 2 : 4;  // float4s per node record
    using VC = FieldVec<float, 8>;
    const VC* Pin = reinterpret_cast<const VC*>(a.P[in]);
    VC* Pout = reinterpret_cast<VC*>(a.P[1 - in]);
    const VC* Ain = reinterpret_cast<const VC*>(a.A[in]);
    VC* Aout = reinterpret_cast<VC*>(a.A[1 - in]);
    const int k = vb * kB + threadIdx.x;
    const bool active = k < a.NF;
    const int M = a.M, K = a.K;
    const size_t NF = (size_t)a.NF, NI = (size_t)a.NI;
    int ai = -1, n = 0;
    uint32_t mask = 0;
    int C[8];  // fluid-list index of each row centre (or of the first fluid node after it)
    bool xlo = true, xhi = true;  // x - 1 and x + 1 lie in r's row without wrapping
    const float4* o = reinterpret_cast<const float4*>(a.own) + (size_t)(active ? k : 0) * kOW4;
    if (active) {
        n = ld_stream(a.flist + k);
        mask = ld_stream(a.fmask + k);
        ai = ld_stream(a.aidx + k);
        const Nbr b = nbrs_of(a.nx, a.ny, a.nz, a.dx, a.dxy, n);
#pragma unroll
        for (int j = 0; j < 8; ++j) C[j] = fluid_index(a.fw, src_of(b, row_centre(j)));
        xlo = b.oxm == -1;
        xhi = b.oxp == 1;
    }
    // the source of link i where x - 1 or x + 1 wraps around the box (rare): the periodic
    // neighbourhood is rebuilt from n there, so that it is not kept live through the loop
    auto wrapped_source = [&](int i) {
        const Nbr b = nbrs_of(a.nx, a.ny, a.nz, a.dx, a.dxy, n);
        return fluid_index(a.fw, src_of(b, i));
    };
    const int cpn = a.SP / kSC;
#pragma unroll 1
    for (int pass = 0; pass < kMaxPass; ++pass) {
        const int c0 = pass * kCP;
        if (c0 >= cpn) break;
        const int nc = cpn - c0 < kCP ? cpn - c0 : kCP;
        float acc[kCP][8];
#pragma unroll
        for (int cc = 0; cc < kCP; ++cc)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[cc][j] = 0.f;
        if (active) {
#pragma unroll
            for (int i = 1; i < kQ; ++i) {
                if (!((mask >> (i - 1)) & 1u)) continue;
                const int row = row_of(i);
                const int base = row < 0 ? k : C[row < 0 ? 0 : row];
                int s;
                if (cx(i) == 0)
                    s = base;
                else if (cx(i) > 0)
                    s = xlo ? base - 1 : wrapped_source(i);
                else
                    s = xhi ? base + (row < 0 ? 1 : (int)((mask >> (row_centre(row < 0 ? 0 : row) - 1)) & 1u))
                            : wrapped_source(i);
                float q;
                if constexpr (kTable) {
                    q = ld_stream(a.tab + tab_at(k, i));
                } else {
                    const Flow4<float> uf = ld_flow(a.uc + s);
                    q = qlink(edot<float>(i, uf.x, uf.y, uf.z), uf.w);
                }
#pragma unroll
                for (int cc = 0; cc < kCP; ++cc) {
                    if (cc < nc) {
                        const VC xs = ld_field<kCoherent, 8>(Pin + (size_t)(c0 + cc) * NF + s);
#pragma unroll
                        for (int qq = 0; qq < kSC; ++qq) {
                            const int sp = (c0 + cc) * kSC + qq;
                            const float p = rn_fma(weight<float>(i), q, is_face(i) ? s_whf[sp] : s_whe[sp]);
#pragma unroll
                            for (int f = 0; f < FP; ++f)
                                acc[cc][qq * FP + f] = __fmaf_rn(p, xs.v[qq * FP + f], acc[cc][qq * FP + f]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int cc = 0; cc < kCP; ++cc) {
            float zv[kSC * 3];
#pragma unroll
            for (int j = 0; j < kSC * 3; ++j) zv[j] = 0.f;
            if (active && cc < nc) {
                const VC xr = ld_field<kCoherent, 8>(Pin + (size_t)(c0 + cc) * NF + k);
                const float4 o0 = __ldg(o);
                VC xn;
#pragma unroll
                for (int qq = 0; qq < kSC; ++qq) {
                    const int sp = (c0 + cc) * kSC + qq;
                    // out = sum_i (w_i q_i + w_i lambda/2) + p_a 1_I: the flow part A, the open
                    // face and edge link counts times w lambda/2, the interface flag times p_a
                    const float out =
                        __fmaf_rn(o0.w, s_pa[sp], __fmaf_rn(o0.z, s_whe[sp], __fmaf_rn(o0.y, s_whf[sp], o0.x)));
#pragma unroll
                    for (int f = 0; f < FP; ++f) {
                        const int j = qq * FP + f;
                        xn.v[j] = __fadd_rn(__fmaf_rn(-out, xr.v[j], acc[cc][j]), xr.v[j]);
                    }
                }
                if (ai >= 0) {
                    const size_t ia = (size_t)(c0 + cc) * NI + ai;
                    const VC xa = ld_field<kCoherent, 8>(Ain + ia);
                    VC xan;
#pragma unroll
                    for (int qq = 0; qq < kSC; ++qq) {
                        const int sp = (c0 + cc) * kSC + qq;
                        const float pa = s_pa[sp], pd = s_pd[sp];
#pragma unroll
                        for (int f = 0; f < FP; ++f) {
                            const int j = qq * FP + f;
                            const float x0 = xr.v[j];
                            xn.v[j] = __fmaf_rn(pd, xa.v[j], xn.v[j]);
                            xan.v[j] = __fmaf_rn(pa, x0, __fmaf_rn(-pd, xa.v[j], xa.v[j]));
                        }
                    }
                    st_field<8>(Aout + ia, xan);
                }
                st_field<8>(Pout + (size_t)(c0 + cc) * NF + k, xn);
#pragma unroll
                for (int qq = 0; qq < kSC; ++qq) {
                    const int sp = (c0 + cc) * kSC + qq;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (m < M && 1 + m < FP) {
                            // u*_g = UA_g + (face sum of c_g) w_f lambda/2 + (edge sum) w_e lambda/2
                            const float4 om = __ldg(o + 1 + m);
                            const float us = __fmaf_rn(om.z, s_whe[sp], __fmaf_rn(om.y, s_whf[sp], om.x));
                            zv[qq * 3 + m] = xn.v[qq * FP + ((1 + m) < FP ? 1 + m : 0)] * us;
                        }
                    }
                }
            }
            // warp sums of this chunk's series into the block's shared partials
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int qq = 0; qq < kSC; ++qq) {
                const int sp = (c0 + cc) * kSC + qq;
                if (cc < nc && sp < a.S) {
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (m < M) {
                            const float w = warp_sum(zv[qq * 3 + m]);
                            if (lane == 0) s_red[warp][sp * M + m] = (double)w;
                        }
                    }
                }
            }
        }
    }
    block_store<kB>(s_red, K, part, acc_part);
}

// ---------------------------------------------------------------------------------------
// Several species, tiled: a virtual block is a tile of 32 x kRows lattice columns (x, y)
// over a segment of planes z0 .. z1 - 1 (kRows = 2 per warp). The block marches along z with
// a ring of planes (three, or four with MP_TILE_SLOTS 4) of the tile plus a one-node halo in x
// and y in shared memory: per position the 32-byte field chunk and the flow vector of the
// node (zero if solid), its fluid-list index (-1 if solid) and its interface index, filled by
// asynchronous 16-byte copies through L2 (three slots: the copies of plane z + 2 are issued
// once plane z is computed; four: while it is computed). Each warp owns two rows of the tile;
// their fluid nodes are packed onto its lanes, and every link reads its source from shared
// memory (a closed link meets zeros and adds p * 0 = 0). The per-node arithmetic is that of
// vblock_multi (same link order and roundings), so the fields are bitwise the same; the Z
// terms are summed over a warp per plane (FP32) and over the planes in FP64. Several chunks
// of species: one march per chunk.
// ---------------------------------------------------------------------------------------
constexpr int kTileX = 32;
constexpr int kTilePX = kTileX + 2;
// ring slots: 4 = copies of plane z + 2 in flight while plane z is computed; 3 = copies
// issued after plane z is computed (less shared memory, more blocks per SM)
#ifndef MP_TILE_SLOTS
#define MP_TILE_SLOTS 3
#endif
constexpr int kTileSlots = MP_TILE_SLOTS;
static_assert(kTileSlots == 3 || kTileSlots == 4, "ring of 3 or 4 planes");
template <int kB>
__host__ __device__ constexpr int tile_rows()
{
    return 2 * (kB / 32);
}
template <int kB>
__host__ __device__ constexpr int tile_pos()
{
    return kTilePX * (tile_rows<kB>() + 2);
}
// dynamic shared memory of the tiled body: the ring (fields in two 16-byte halves, flow,
// fluid-list and interface indices), the wrapped coordinates of the tile's columns and rows,
// and each warp's lane map
template <int kB>
__host__ __device__ constexpr size_t tile_smem()
{
    return (size_t)kTileSlots * tile_pos<kB>() * (3 * sizeof(float4) + 2 * sizeof(int)) +
           (size_t)(kTilePX + tile_rows<kB>() + 2) * sizeof(int) + (size_t)(kB / 32) * 64;
}

__device__ __forceinline__ int wrap_mod(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ void cp_async_cg16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

template <int FP, bool kCoherent, int kB>
__device__ __forceinline__ void vblock_tiled(const DArgs& a, int vb, int in, double* part, bool acc_part,
                                             double (*s_red)[kMaxSeries], const float* s_whf, const float* s_whe,
                                             const float* s_pa, const float* s_pd, unsigned char* tsm)
{
    constexpr int kSC = 8 / FP;
    constexpr int kOW4 = FP == 2 ? 2 : 4;
    constexpr int kRows = tile_rows<kB>();
    constexpr int kP = tile_pos<kB>();
    constexpr int kPJ = (kP + kB - 1) / kB;  // positions per thread in a plane
    using VC = FieldVec<float, 8>;
    float4* sF0 = reinterpret_cast<float4*>(tsm);  // [slot][position]: fields 0..3 of the chunk
    float4* sF1 = sF0 + kTileSlots * kP;            // fields 4..7
    float4* sU = sF1 + kTileSlots * kP;             // flow vector
    int* sK = reinterpret_cast<int*>(sU + kTileSlots * kP);  // fluid-list index, -1 if solid
    int* sI = sK + kTileSlots * kP;                 // interface index, -1 off the interface
    int* sX = sI + kTileSlots * kP;                 // lattice x of tile column 0..33
    int* sY = sX + kTilePX;                         // lattice y of tile row 0..kRows+1
    unsigned char* sMap = reinterpret_cast<unsigned char*>(sY + kRows + 2);  // [warp][64]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = vb % a.ntx, t1 = vb / a.ntx, ty = t1 % a.nty, tzs = t1 / a.nty;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int x0 = tx * kTileX, y0 = ty * kRows, z0 = tzs * a.tz;
    const int z1 = min(z0 + a.tz, a.nz);
    const int M = a.M, K = a.K;
    const size_t NF = (size_t)a.NF, NI = (size_t)a.NI;
    const float* Pin = a.P[in];
    VC* Pout = reinterpret_cast<VC*>(a.P[1 - in]);
    const VC* Ain = reinterpret_cast<const VC*>(a.A[in]);
    VC* Aout = reinterpret_cast<VC*>(a.A[1 - in]);
    __syncthreads();  // the previous virtual block is done with the shared tables
    if (tid < kTilePX) sX[tid] = wrap_mod(x0 - 1 + tid, a.nx);
    if (tid < kRows + 2) sY[tid] = wrap_mod(y0 - 1 + tid, a.ny);
    for (int j = tid; j < kMaxSeries; j += kB)
        for (int w = 0; w < kB / 32; ++w) s_red[w][j] = 0.0;
    __syncthreads();

    // lattice node of this thread's positions p = tid + kB j within a plane (without z)
    int pxy[kPJ];
#pragma unroll
    for (int j = 0; j < kPJ; ++j) {
        const int p = tid + kB * j;
        const int ly = p / kTilePX, lx = p - ly * kTilePX;
        pxy[j] = p < kP ? sY[ly] * a.nx + sX[lx] : 0;
    }
    // fluid and interface words of this thread's positions of plane z, and the positions' bit
    // in them (fetched before their copies are issued, so that their latency overlaps work)
    uint2 wf[kPJ], wi[kPJ];
    int bj[kPJ];
    auto fetch_words = [&](int z) {
        const long long zoff = (long long)wrap_mod(z, a.nz) * a.ny * a.nx;
#pragma unroll
        for (int j = 0; j < kPJ; ++j) {
            if (tid + kB * j < kP) {
                const int n = (int)(zoff + pxy[j]);
                bj[j] = n & 31;
                wf[j] = __ldg(a.fw + (n >> 5));
                wi[j] = __ldg(a.iw + (n >> 5));
            }
        }
    };

    const int cpn = a.SP / kSC;
#pragma unroll 1
    for (int ch = 0; ch < cpn; ++ch) {
        const float* Pc = Pin + (size_t)ch * NF * 8;
        // copies of plane z (z0 - 1 <= z <= z1) into its ring slot, from the fetched words
        auto issue_plane = [&](int z) {
            const int slot = (z - z0 + 1) % kTileSlots;
#pragma unroll
            for (int j = 0; j < kPJ; ++j) {
                const int p = tid + kB * j;
                if (p < kP) {
                    const int b = bj[j];
                    const uint32_t lt = (1u << b) - 1u;
                    int kk = -1;
                    if ((wf[j].x >> b) & 1u) {
                        kk = (int)wf[j].y + __popc(wf[j].x & lt);
                        const float* src = Pc + (size_t)kk * 8;
                        cp_async_cg16(&sF0[slot * kP + p], src);
                        cp_async_cg16(&sF1[slot * kP + p], src + 4);
                        cp_async_cg16(&sU[slot * kP + p], a.uc + kk);
                    } else {
                        // a solid source: zero fields and flow, so that a closed link adds
                        // p * 0 = 0 and the link loop needs no test
                        sF0[slot * kP + p] = zero4;
                        sF1[slot * kP + p] = zero4;
                        sU[slot * kP + p] = zero4;
                    }
                    sK[slot * kP + p] = kk;
                    sI[slot * kP + p] = ((wi[j].x >> b) & 1u) ? (int)wi[j].y + __popc(wi[j].x & lt) : -1;
                }
            }
        };
        __syncthreads();  // the previous chunk's march is done with the ring
        fetch_words(z0 - 1);
        issue_plane(z0 - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        fetch_words(z0);
        issue_plane(z0);
        asm volatile("cp.async.commit_group;" ::: "memory");
        fetch_words(z0 + 1);
        issue_plane(z0 + 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (kTileSlots == 4 && z0 + 2 <= z1) fetch_words(z0 + 2);
#pragma unroll 1
        for (int z = z0; z < z1; ++z) {
            if constexpr (kTileSlots == 4) {
                // plane z + 2 into the slot of plane z - 2 (free since the last barrier); words
                // of plane z + 3
                if (z + 2 <= z1) issue_plane(z + 2);
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (z + 3 <= z1) fetch_words(z + 3);
                asm volatile("cp.async.wait_group 1;" ::: "memory");  // planes up to z + 1 have landed
            } else {
                if (z + 2 <= z1) fetch_words(z + 2);  // its copies follow this plane's work
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            const int sc = (z - z0 + 1) % kTileSlots;
            const int sm = (z - z0) % kTileSlots, sp = (z - z0 + 2) % kTileSlots;
            // this warp's two rows: fluid nodes inside the lattice, packed onto the lanes
            uint32_t bits[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int ly = 1 + 2 * warp + r;
                const bool fl = y0 + 2 * warp + r < a.ny && x0 + lane < a.nx &&
                                sK[sc * kP + ly * kTilePX + 1 + lane] >= 0;
                bits[r] = __ballot_sync(0xffffffffu, fl);
                if (fl) sMap[warp * 64 + (r ? __popc(bits[0]) : 0) + __popc(bits[r] & ((1u << lane) - 1u))] =
                    (unsigned char)((r << 5) | lane);
            }
            __syncwarp();
            const int ntot = __popc(bits[0]) + __popc(bits[1]);
            float zt[kSC * 3];
#pragma unroll
            for (int j = 0; j < kSC * 3; ++j) zt[j] = 0.f;
            for (int j = lane; j < ntot; j += 32) {
                const int e = sMap[warp * 64 + j];
                const int pos = (1 + 2 * warp + (e >> 5)) * kTilePX + 1 + (e & 31);
                const int kk = sK[sc * kP + pos];
                const int ai = sI[sc * kP + pos];
                // the node's record and adsorbed fields, requested before the link loop
                const float4* o = reinterpret_cast<const float4*>(a.own) + (size_t)kk * kOW4;
                const float4 o0 = __ldg(o);
                float4 om[kOW4 - 1];
#pragma unroll
                for (int m = 0; m < kOW4 - 1; ++m) om[m] = m < M ? __ldg(o + 1 + m) : make_float4(0.f, 0.f, 0.f, 0.f);
                const size_t ia = (size_t)ch * NI + (ai >= 0 ? ai : 0);
                VC xa;
                if (ai >= 0) xa = ld_field<kCoherent, 8>(Ain + ia);
                float acc[8];
#pragma unroll
                for (int f = 0; f < 8; ++f) acc[f] = 0.f;
#pragma unroll
                for (int i = 1; i < kQ; ++i) {
                    const int sl = cz(i) > 0 ? sm : (cz(i) < 0 ? sp : sc);
                    const int q_at = sl * kP + pos - cx(i) - cy(i) * kTilePX;
                    const float4 uf = sU[q_at];
                    const float q = qlink(edot<float>(i, uf.x, uf.y, uf.z), uf.w);
                    const float4 f0 = sF0[q_at], f1 = sF1[q_at];
                    const float xs[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
                    for (int qq = 0; qq < kSC; ++qq) {
                        const int spc = ch * kSC + qq;
                        const float pl = rn_fma(weight<float>(i), q, is_face(i) ? s_whf[spc] : s_whe[spc]);
#pragma unroll
                        for (int f = 0; f < FP; ++f) acc[qq * FP + f] = __fmaf_rn(pl, xs[qq * FP + f], acc[qq * FP + f]);
                    }
                }
                const float4 r0 = sF0[sc * kP + pos], r1 = sF1[sc * kP + pos];
                const float xr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                VC xn;
#pragma unroll
                for (int qq = 0; qq < kSC; ++qq) {
                    const int spc = ch * kSC + qq;
                    const float out =
                        __fmaf_rn(o0.w, s_pa[spc], __fmaf_rn(o0.z, s_whe[spc], __fmaf_rn(o0.y, s_whf[spc], o0.x)));
#pragma unroll
                    for (int f = 0; f < FP; ++f) {
                        const int j2 = qq * FP + f;
                        xn.v[j2] = __fadd_rn(__fmaf_rn(-out, xr[j2], acc[j2]), xr[j2]);
                    }
                }
                if (ai >= 0) {
                    VC xan;
#pragma unroll
                    for (int qq = 0; qq < kSC; ++qq) {
                        const int spc = ch * kSC + qq;
                        const float pa = s_pa[spc], pd = s_pd[spc];
#pragma unroll
                        for (int f = 0; f < FP; ++f) {
                            const int j2 = qq * FP + f;
                            xn.v[j2] = __fmaf_rn(pd, xa.v[j2], xn.v[j2]);
                            xan.v[j2] = __fmaf_rn(pa, xr[j2], __fmaf_rn(-pd, xa.v[j2], xa.v[j2]));
                        }
                    }
                    st_field<8>(Aout + ia, xan);
                }
                st_field<8>(Pout + (size_t)ch * NF + kk, xn);
#pragma unroll
                for (int qq = 0; qq < kSC; ++qq) {
                    const int spc = ch * kSC + qq;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (m < M && 1 + m < FP) {
                            const float us = __fmaf_rn(om[m].z, s_whe[spc], __fmaf_rn(om[m].y, s_whf[spc], om[m].x));
                            zt[qq * 3 + m] += xn.v[qq * FP + ((1 + m) < FP ? 1 + m : 0)] * us;
                        }
                    }
                }
            }
            // this plane's Z terms: warp sums (FP32), added to the warp's FP64 accumulators
#pragma unroll
            for (int qq = 0; qq < kSC; ++qq) {
                const int spc = ch * kSC + qq;
                if (spc < a.S) {
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (m < M) {
                            const float w = warp_sum(zt[qq * 3 + m]);
                            if (lane == 0) s_red[warp][spc * M + m] += (double)w;
                        }
                    }
                }
            }
            __syncthreads();  // before the next copies reuse the slot of plane z - 1 (or z - 2)
            if constexpr (kTileSlots == 3) {
                if (z + 2 <= z1) issue_plane(z + 2);
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    block_store<kB>(s_red, K, part, acc_part);
}

// Several species: stage the per-species constants in shared memory (uniform across the
// block) and run the body; block sums to part[0..K) (stored, or added when acc_part).
template <int FP, bool kTable, bool kCoherent, int kB>
__device__ __forceinline__ void run_multi(const DArgs& a, int vb, int in, double* part, bool acc_part,
                                          double (*s_red)[kMaxSeries], float* s_c)
{
    for (int j = threadIdx.x; j < MP_MAX_SPECIES; j += kB) {
        s_c[j] = a.whf[j];
        s_c[MP_MAX_SPECIES + j] = a.whe[j];
        s_c[2 * MP_MAX_SPECIES + j] = a.pa[j];
        s_c[3 * MP_MAX_SPECIES + j] = a.pd[j];
    }
    __syncthreads();
    vblock_multi<FP, kTable, kCoherent, kB>(a, vb, in, part, acc_part, s_red, s_c, s_c + MP_MAX_SPECIES,
                                            s_c + 2 * MP_MAX_SPECIES, s_c + 3 * MP_MAX_SPECIES);
}

template <int FP, bool kCoherent, int kB>
__device__ __forceinline__ void run_tiled(const DArgs& a, int vb, int in, double* part, bool acc_part,
                                          double (*s_red)[kMaxSeries], float* s_c, unsigned char* tsm)
{
    for (int j = threadIdx.x; j < MP_MAX_SPECIES; j += kB) {
        s_c[j] = a.whf[j];
        s_c[MP_MAX_SPECIES + j] = a.whe[j];
        s_c[2 * MP_MAX_SPECIES + j] = a.pa[j];
        s_c[3 * MP_MAX_SPECIES + j] = a.pd[j];
    }
    vblock_tiled<FP, kCoherent, kB>(a, vb, in, part, acc_part, s_red, s_c, s_c + MP_MAX_SPECIES,
                                            s_c + 2 * MP_MAX_SPECIES, s_c + 3 * MP_MAX_SPECIES, tsm);
}

__device__ __forceinline__ int ctx_of(const DLaunch& L, int v)
{
    int c = 0;
#pragma unroll
    for (int j = 1; j < kMaxCtx; ++j)
        if (j < L.n && v >= L.vbofs[j]) c = j;
    return c;
}

// FP64 total of series j over the context's virtual blocks, in a fixed order (thread 0 gets it)
template <int kB>
__device__ __forceinline__ double ctx_series_total(const double* part, int nvb, int K, int j, double* s_tmp)
{
    // four independent chains of loads, added in a fixed order
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int b = threadIdx.x;
    for (; b + 3 * kB < nvb; b += 4 * kB) {
        v0 += __ldcg(part + (size_t)b * K + j);
        v1 += __ldcg(part + (size_t)(b + kB) * K + j);
        v2 += __ldcg(part + (size_t)(b + 2 * kB) * K + j);
        v3 += __ldcg(part + (size_t)(b + 3 * kB) * K + j);
    }
    for (; b < nvb; b += kB) v0 += __ldcg(part + (size_t)b * K + j);
    double v = (v0 + v1) + (v2 + v3);
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kB / 32; ++w) tot += s_tmp[w];
    __syncthreads();
    return tot;
}

template <int FP, bool kSingle, bool kTiled = false>
constexpr int min_blocks_direct(int block)
{
    // tiled: as many blocks as the shared-memory ring leaves room for (three of 128 threads)
    return kTiled ? 3
                  : (kSingle ? MP_DIRECT_SINGLE_THREADS / block
                             : (MP_DIRECT_MULTI_THREADS / block > 1 ? MP_DIRECT_MULTI_THREADS / block : 1));
}

// Appends Z(t1), D(t1) = D(t1 - 1) + Z(t1) of every series of context a, t1 = t + 1, from
// `slots` partial sums; called by one whole block.
template <int kB>
__device__ __forceinline__ void append_series(const DArgs& a, const double* part, int slots, double* s_tmp)
{
    long long t1 = 0;
    if (threadIdx.x == 0) t1 = *((volatile long long*)a.tdev) + 1;
    for (int j = 0; j < a.K; ++j) {
        const double z = ctx_series_total<kB>(part, slots, a.K, j, s_tmp);
        if (threadIdx.x == 0) {
            a.Z[(size_t)j * a.cap + t1] = z;
            a.D[(size_t)j * a.cap + t1] = a.D[(size_t)j * a.cap + t1 - 1] + z;
        }
    }
    if (threadIdx.x == 0) *a.tdev = t1;
}

// ---------------------------------------------------------------------------------------
// One step of every context in the launch; block partials to the half of the partials array
// of this step's parity (`phase`). The series of the previous step are appended here, by
// block c for context c while the other blocks work (`pending`: the previous launch was a
// step whose partials are not yet added), so no block waits for the others at the end; the
// last step of a run is appended by k_direct_finish.
// ---------------------------------------------------------------------------------------
template <int FP, bool kSingle, bool kTable, int kB, bool kTiled>
__global__ void __launch_bounds__(kB, min_blocks_direct<FP, kSingle, kTiled>(kB))
    k_direct_step(const __grid_constant__ DLaunch L, int phase, int pending)
{
    extern __shared__ __align__(16) unsigned char tsm[];  // tiled variant's ring
    __shared__ double s_red[kB / 32][kMaxSeries];
    __shared__ float s_c[4 * MP_MAX_SPECIES];
    __shared__ double s_tmp[kB / 32];
    const int c = ctx_of(L, (int)blockIdx.x);
    pdl_enter();  // the previous step's fields, partials and series are complete and visible
    if (pending && (int)blockIdx.x < L.n) {
        const DArgs& r = L.args[blockIdx.x];
        append_series<kB>(r, r.part + (size_t)(phase ^ 1) * r.nvb * r.K, r.nvb, s_tmp);
    }
    const DArgs& a = L.args[c];
    const int vb = (int)blockIdx.x - L.vbofs[c];
    const int in = (a.in0 + phase) & 1;
    double* part = a.part + ((size_t)phase * a.nvb + vb) * a.K;
    if (kSingle || a.S == 1) {
        float zacc[3] = {0.f, 0.f, 0.f};
        vblock_single<FP, kTable, false, kB>(a, vb, in, zacc);
        reduce_zacc<kB>(s_red, a.M, zacc, part, false);
    } else if constexpr (kTiled) {
        run_tiled<FP, false, kB>(a, vb, in, part, false, s_red, s_c, tsm);
    } else {
        run_multi<FP, kTable, false, kB>(a, vb, in, part, false, s_red, s_c);
    }
}

// appends the series of the step of parity `phase` (the last step of a run), block c for
// context c
template <int kB>
__global__ void __launch_bounds__(kB) k_direct_finish(const __grid_constant__ DLaunch L, int phase)
{
    __shared__ double s_tmp[kB / 32];
    pdl_enter();
    const DArgs& r = L.args[blockIdx.x];
    append_series<kB>(r, r.part + (size_t)phase * r.nvb * r.K, r.nvb, s_tmp);
}

// ---------------------------------------------------------------------------------------
// Device-wide barrier with a bounded wait. Thread 0 of every block arrives (release), then
// waits (acquire) until `target` arrivals are counted, another block has reported a failure,
// or timeout_ns has passed on the global timer; in the last case it records MP_ETIMEOUT in
// *err. Returns false on failure (the caller leaves its loop). The waiting thread sleeps
// between polls. The counter is cleared by the host before every launch.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_wait(unsigned int* count, unsigned int target, int* err, long long timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned long long t0 = global_ns();
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (*((volatile int*)err) != 0) {
                ok = 0;
                break;
            }
            if ((long long)(global_ns() - t0) > timeout_ns) {
                atomicCAS(err, 0, MP_ETIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// A run of `nsteps` steps of every context in one cooperative launch. The T virtual blocks
// are dealt to the G blocks round-robin (v = b, b + G, ...; kRoundRobin) or in contiguous
// runs ([lo(b), lo(b+1)), lo(b) = floor(b T / G)); either way the same every step, and the
// virtual blocks of one context that a block handles are consecutive in its loop. A block
// adds the partial sums of its virtual blocks of context c (FP64, fixed order) and writes
// them to its slot of c: round-robin, c has min(nvb_c, G) slots and block b writes slot
// (b - vbofs[c]) mod G; contiguous, the owners fb(c)..lb(c) of its first and last virtual
// block write slots b - fb(c). After the barrier that ends step st, block c (c < number of
// contexts) adds context c's slots of that step (kept in the half of the partials array of
// the step's parity, so that the next step can write the other half meanwhile) and appends
// Z, D.
#ifndef MP_DIRECT_RR
#define MP_DIRECT_RR 1
#endif
constexpr bool kRoundRobin = MP_DIRECT_RR != 0;

template <int FP, bool kSingle, bool kTable, int kB, bool kTiled>
__global__ void __launch_bounds__(kB, min_blocks_direct<FP, kSingle, kTiled>(kB))
    k_direct_persistent(const __grid_constant__ DLaunch L, int phase0, int nsteps, unsigned int* bar, int* err,
                        long long timeout_ns)
{
    extern __shared__ __align__(16) unsigned char tsm[];  // tiled variant's ring
    __shared__ double s_red[kB / 32][kMaxSeries];
    __shared__ double s_acc[kMaxSeries];
    __shared__ float s_c[4 * MP_MAX_SPECIES];
    __shared__ double s_tmp[kB / 32];
    const int total = L.vbofs[L.n];
    const int G = (int)gridDim.x;
    float zacc[3] = {0.f, 0.f, 0.f};
    const int v_lo = kRoundRobin ? (int)blockIdx.x : (int)((long long)blockIdx.x * total / G);
    const int v_hi = kRoundRobin ? total : (int)((long long)(blockIdx.x + 1) * total / G);
    const int v_step = kRoundRobin ? G : 1;
    // owner block of virtual block v (contiguous runs)
    auto owner = [&](int v) { return (int)(((long long)(v + 1) * G + total - 1) / total) - 1; };
    // slots of context c, and the slot of this block
    auto slots_of = [&](int c) {
        return kRoundRobin ? min(L.vbofs[c + 1] - L.vbofs[c], G) : owner(L.vbofs[c + 1] - 1) - owner(L.vbofs[c]) + 1;
    };
    // the block's sums of context c for step st into its slot: per-thread sums (one species)
    // or the shared accumulator (several)
    auto flush = [&](int c, int st) {
        const DArgs& a = L.args[c];
        const int slot = kRoundRobin ? (((int)blockIdx.x - L.vbofs[c]) % G + G) % G
                                     : (int)blockIdx.x - owner(L.vbofs[c]);
        double* dst = a.part + ((size_t)(st & 1) * slots_of(c) + slot) * a.K;
        if (kSingle || a.S == 1) {
            reduce_zacc<kB>(s_red, a.M, zacc, s_acc, false);
        }
        for (int j = threadIdx.x; j < a.K; j += kB) {
            dst[j] = s_acc[j];
            __threadfence();
        }
    };
    for (int st = 0; st < nsteps; ++st) {
        const int phase = (phase0 + st) & 1;
        int cur = -1;
        for (int v = v_lo; v < v_hi; v += v_step) {
            const int c = ctx_of(L, v);
            if (c != cur) {
                if (cur >= 0) flush(cur, st);
                for (int j = threadIdx.x; j < kMaxSeries; j += kB) s_acc[j] = 0.0;
                zacc[0] = zacc[1] = zacc[2] = 0.f;
                cur = c;
            }
            const DArgs& a = L.args[c];
            const int in = (a.in0 + phase) & 1;
            if (kSingle || a.S == 1)
                vblock_single<FP, kTable, true, kB>(a, v - L.vbofs[c], in, zacc);
            else if constexpr (kTiled)
                run_tiled<FP, true, kB>(a, v - L.vbofs[c], in, s_acc, true, s_red, s_c, tsm);
            else
                run_multi<FP, kTable, true, kB>(a, v - L.vbofs[c], in, s_acc, true, s_red, s_c);
        }
        if (cur >= 0) flush(cur, st);
        if (!grid_wait(bar, (unsigned int)(st + 1) * G, err, timeout_ns)) return;
        if ((int)blockIdx.x < L.n) {
            const DArgs& a = L.args[blockIdx.x];
            const int slots = slots_of((int)blockIdx.x);
            append_series<kB>(a, a.part + (size_t)(st & 1) * slots * a.K, slots, s_tmp);
        }
    }
}

// Barrier alone, for the self-test entry point: `rounds` barriers; with `unreachable` the
// target counts one block more than the grid has, so every wait must give up.
__global__ void k_grid_wait_selftest(int rounds, int unreachable, unsigned int* bar, int* err, long long timeout_ns)
{
    for (int r = 0; r < rounds; ++r) {
        const unsigned int target = (unsigned int)(r + 1) * gridDim.x + (unreachable ? 1u : 0u);
        if (!grid_wait(bar, target, err, timeout_ns)) return;
    }
}

// Fluid-list addressing of a several-species context (once, at mp_init): {bits, nodes before
// the word} per 32-node word (of the fluid and of the interface), and the flow vectors in
// list order.
__global__ void k_fluid_words(const uint32_t* __restrict__ fluid, const int32_t* __restrict__ fbase, int W,
                              uint2* __restrict__ fw)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W) fw[w] = make_uint2(fluid[w], (uint32_t)fbase[w]);
}
__global__ void k_list_flow(const int32_t* __restrict__ flist, const Flow4<float>* __restrict__ u4, int NF,
                            Flow4<float>* __restrict__ uc)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NF) uc[k] = u4[flist[k]];
}

// ---------------------------------------------------------------------------------------
// Tables of one context (once, at mp_init). Per entry k of the work list:
//  fmask[k]       open-link mask (bit i-1: the source r - c_i is fluid)
//  aidx[k]        compact interface index, -1 off the interface
//  tab[k, i]      one species: p_i(r - c_i) of the incoming link i (0 if closed);
//                 several: q_i(r - c_i), the flow-dependent part (w_i q_i + w_i lambda/2 = p)
//  own[k]         one species: {out, u*_g of each propagated moment}, out = sum of the
//                 outgoing p_j(r) + p_a 1_I (FP64 sums of the FP32 link values, rounded once);
//                 several: {A, n_face, n_edge, 1_I} then per moment {UA_g, cf_g, ce_g, 0},
//                 A = sum_j w_j q_j(r), UA_g = sum_j w_j q_j c_jg, n_face/n_edge the open
//                 outgoing face/edge links and cf_g/ce_g their sums of c_jg.
// The values p_i are formed exactly as in the flux scheme, so both ends agree bitwise.
// ---------------------------------------------------------------------------------------
__global__ void k_direct_tables(const int32_t* __restrict__ flist, const uint32_t* __restrict__ fluid,
                                uint32_t* __restrict__ fmask, const uint32_t* __restrict__ iface,
                                const int32_t* __restrict__ ibase,
                                const Flow4<float>* __restrict__ u4, int NF, int nx, int ny, int nz, Div dx, Div dxy,
                                int single, int M, int d0, int d1, int d2, float whf, float whe, float pa,
                                int32_t* __restrict__ aidx, float* __restrict__ tab, float* __restrict__ own)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NF) return;
    const int n = flist[k];
    const Nbr b = nbrs_of(nx, ny, nz, dx, dxy, n);
    uint32_t mask = 0;
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const int s = src_of(b, i);
        if ((fluid[s >> 5] >> (s & 31)) & 1u) mask |= 1u << (i - 1);
    }
    fmask[k] = mask;
    const Flow4<float> ur = u4[n];
    const bool itf = mask != kAll;
    if (itf) {
        const uint32_t bits = iface[n >> 5];
        aidx[k] = ibase[n >> 5] + __popc(bits & ((1u << (n & 31)) - 1u));
    } else {
        aidx[k] = -1;
    }
    const int dir[3] = {d0, d1, d2};
    double out = 0.0, A = 0.0, nfo = 0.0, neo = 0.0;
    double us[3] = {0.0, 0.0, 0.0}, ua[3] = {0.0, 0.0, 0.0}, cf[3] = {0.0, 0.0, 0.0}, ce[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const bool open = (mask >> (i - 1)) & 1u;
        const int s = src_of(b, i);
        const Flow4<float> uf = u4[s];
        const float qin = qlink(edot<float>(i, uf.x, uf.y, uf.z), uf.w);
        const float whl = is_face(i) ? whf : whe;
        tab[tab_at(k, i)] = open ? (single ? rn_fma(weight<float>(i), qin, whl) : qin) : 0.f;
        if (open) {
            // the outgoing link opposite(i), from r to s_i
            const int j = opposite(i);
            const float qout = qlink(edot<float>(j, ur.x, ur.y, ur.z), ur.w);
            const float pout = rn_fma(weight<float>(j), qout, whl);
            const double wq = (double)weight<float>(j) * (double)qout;
            out += (double)pout;
            A += wq;
            if (is_face(j))
                nfo += 1.0;
            else
                neo += 1.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                if (m < M) {
                    const int c = ci(j, dir[m]);
                    us[m] += (double)c * (double)pout;
                    ua[m] += (double)c * wq;
                    if (is_face(j))
                        cf[m] += (double)c;
                    else
                        ce[m] += (double)c;
                }
            }
        }
    }
    if (single) {
        out += itf ? (double)pa : 0.0;
        if (M == 1) {
            reinterpret_cast<float2*>(own)[k] = make_float2((float)out, (float)us[0]);
        } else {
            reinterpret_cast<float4*>(own)[k] = make_float4((float)out, (float)us[0], (float)us[1], (float)us[2]);
        }
    } else {
        const int ow4 = M == 1 ? 2 : 4;
        float4* o = reinterpret_cast<float4*>(own) + (size_t)k * ow4;
        o[0] = make_float4((float)A, (float)nfo, (float)neo, itf ? 1.f : 0.f);
        for (int m = 0; m < ow4 - 1; ++m)
            o[1 + m] = m < M ? make_float4((float)ua[m], (float)cf[m], (float)ce[m], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

}  // namespace

// Tiles of a several-species context for the tiled variant: 32 x 8 columns, planes per tile
// chosen so that the tiles fill the device about eight times over (at least two planes).
void set_tiles(DArgs& a, int sms)
{
    a.ntx = (a.nx + kTileX - 1) / kTileX;
    a.nty = (a.ny + tile_rows<128>() - 1) / tile_rows<128>();
    const long long cols = (long long)a.ntx * a.nty;
    const long long want = 8LL * 3 * std::max(sms, 1);
    long long tz = (cols * a.nz + want - 1) / want;
    tz = std::max(2LL, std::min<long long>(tz, a.nz));
    a.tz = (int)tz;
}
int tiles_of(const DArgs& a) { return a.ntx * a.nty * ((a.nz + a.tz - 1) / a.tz); }
// virtual blocks of the untiled variants at the smallest block (128), or tiles
size_t part_rows(const DArgs& a)
{
    const size_t rows = (size_t)((a.NF + 127) / 128);
    return a.S > 1 ? std::max(rows, (size_t)tiles_of(a)) : rows;
}

// ---------------------------------------------------------------------------------------
// Launch state over a set of contexts
// ---------------------------------------------------------------------------------------
struct DirectState {
    std::vector<mp_ctx*> ctx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int FP = 2;
    bool single = true;
    int block = 256;
    bool table = true;
    bool persistent = false;
    bool tiled = false;  // several-species contexts by tiles (block 128)
    int phase = 0;
    DArgs* d_args = nullptr;
    std::vector<DArgs> h_args;
    DLaunch L{};
    double* part = nullptr;  // all contexts' partials
    unsigned int* bar = nullptr;
    int* err = nullptr;
    int pgrid = 0;  // blocks of the persistent launch
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::string variant;
};

namespace {

template <bool kTiled, int kB>
constexpr size_t dyn_smem()
{
    return kTiled ? tile_smem<kB>() : 0;
}

template <int FP, bool kSingle, bool kTable, int kB, bool kTiled>
cudaError_t launch_step_t(DirectState* d, int pending)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(d->L.vbofs[d->L.n]);
    cfg.blockDim = dim3(kB);
    cfg.dynamicSmemBytes = dyn_smem<kTiled, kB>();
    cfg.stream = d->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_direct_step<FP, kSingle, kTable, kB, kTiled>, d->L, d->phase, pending);
}

// appends the series of the last step (parity `phase`) of a run of one-step launches
cudaError_t launch_finish(DirectState* d, int phase)
{
    return launch_pdl(k_direct_finish<256>, dim3(d->L.n), dim3(256), d->stream, d->L, phase);
}

template <int FP, bool kSingle, bool kTable, int kB, bool kTiled>
cudaError_t launch_persistent_t(DirectState* d, int nsteps)
{
    cudaError_t e = cudaMemsetAsync(d->bar, 0, sizeof(unsigned int), d->stream);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(d->pgrid);
    cfg.blockDim = dim3(kB);
    cfg.dynamicSmemBytes = dyn_smem<kTiled, kB>();
    cfg.stream = d->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_direct_persistent<FP, kSingle, kTable, kB, kTiled>, d->L, d->phase, nsteps,
                              d->bar, d->err, kWaitNs);
}

// allows the tiled instances their dynamic shared memory; the persistent grid's blocks per SM
template <int FP, bool kSingle, bool kTable, int kB, bool kTiled>
int occupancy_t(int* blocks_per_sm)
{
    if (kTiled) {
        const int bytes = (int)dyn_smem<kTiled, kB>();
        if (cudaFuncSetAttribute(k_direct_step<FP, kSingle, kTable, kB, kTiled>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
            cudaFuncSetAttribute(k_direct_persistent<FP, kSingle, kTable, kB, kTiled>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
            return MP_ECUDA;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                         k_direct_persistent<FP, kSingle, kTable, kB, kTiled>, kB,
                                                         dyn_smem<kTiled, kB>()) == cudaSuccess
               ? MP_OK
               : MP_ECUDA;
}

// dispatch over the compile-time variants: fields per record, one or several species, table or
// recomputed link terms, block size, tiled (several species, block 128)
template <typename Fn>
auto dispatch(const DirectState* d, Fn&& fn)
{
    auto by_block = [&](auto fp, auto single, auto table) {
        if constexpr (!decltype(single)::value && !decltype(table)::value) {
            if (d->tiled) return fn(fp, single, table, std::integral_constant<int, 128>{}, std::true_type{});
        }
        if (d->block == 128) return fn(fp, single, table, std::integral_constant<int, 128>{}, std::false_type{});
        if (d->block == 512) return fn(fp, single, table, std::integral_constant<int, 512>{}, std::false_type{});
        return fn(fp, single, table, std::integral_constant<int, 256>{}, std::false_type{});
    };
    auto by_table = [&](auto fp, auto single) {
        if (d->table) return by_block(fp, single, std::true_type{});
        return by_block(fp, single, std::false_type{});
    };
    auto by_single = [&](auto fp) {
        if (d->single) return by_table(fp, std::true_type{});
        return by_table(fp, std::false_type{});
    };
    if (d->FP == 2) return by_single(std::integral_constant<int, 2>{});
    return by_single(std::integral_constant<int, 4>{});
}

cudaError_t launch_step(DirectState* d, int pending)
{
    return dispatch(d, [&](auto fp, auto single, auto table, auto kb, auto tiled) {
        return launch_step_t<decltype(fp)::value, decltype(single)::value, decltype(table)::value,
                             decltype(kb)::value, decltype(tiled)::value>(d, pending);
    });
}

cudaError_t launch_persistent(DirectState* d, int nsteps)
{
    return dispatch(d, [&](auto fp, auto single, auto table, auto kb, auto tiled) {
        return launch_persistent_t<decltype(fp)::value, decltype(single)::value, decltype(table)::value,
                                   decltype(kb)::value, decltype(tiled)::value>(d, nsteps);
    });
}

int persistent_grid(DirectState* d)
{
    int per_sm = 0;
    int rc = dispatch(d, [&](auto fp, auto single, auto table, auto kb, auto tiled) {
        return occupancy_t<decltype(fp)::value, decltype(single)::value, decltype(table)::value, decltype(kb)::value,
                           decltype(tiled)::value>(&per_sm);
    });
    if (rc != MP_OK) return rc;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MP_ECUDA;
    const int total = d->L.vbofs[d->L.n];
    d->pgrid = std::min(std::max(per_sm, 0) * sms, total);
    if (d->pgrid < (int)d->ctx.size()) d->pgrid = 0;  // needs a block per context for the totals
    return MP_OK;
}

void drop_graphs(DirectState* d)
{
    for (int b = 0; b < 2; ++b)
        if (d->exec[b]) {
            cudaGraphExecDestroy(d->exec[b]);
            d->exec[b] = nullptr;
        }
}

// (re)build the per-context launch arguments for the current block size and variant
int upload_args(DirectState* d)
{
    const int n = (int)d->ctx.size();
    d->L.n = n;
    d->L.vbofs[0] = 0;
    for (int c = 0; c < n; ++c) {
        DArgs& a = d->h_args[c];
        const int blk = d->tiled ? 128 : d->block;  // the launch's block size
        a.nvb = d->tiled && a.S > 1 ? tiles_of(a) : (int)((d->ctx[c]->geo.n_fluid + blk - 1) / blk);
        d->L.vbofs[c + 1] = d->L.vbofs[c] + a.nvb;
    }
    // partials: [2][nvb][K] per context, sized for the most virtual blocks of any variant
    size_t off = 0;
    for (int c = 0; c < n; ++c) {
        DArgs& a = d->h_args[c];
        a.part = d->part + off;
        off += 2 * part_rows(a) * a.K;
    }
    MP_CUDA(cudaMemcpyAsync(d->d_args, d->h_args.data(), sizeof(DArgs) * n, cudaMemcpyHostToDevice, d->stream));
    MP_CUDA(cudaStreamSynchronize(d->stream));
    d->L.args = d->d_args;
    drop_graphs(d);
    int rc = persistent_grid(d);
    if (rc != MP_OK) return cuda_fail(cudaGetLastError(), "occupancy query");
    return MP_OK;
}

void set_variant_name(DirectState* d)
{
    // a persistent variant that found no room for its grid runs one launch per step
    d->variant = std::string(d->persistent && d->pgrid > 0 ? "persistent" : "per-step") +
                 (d->table ? ",table" : ",recompute") +
                 (d->tiled ? ",tiled,block=128" : ",block=" + std::to_string(d->block));
}

// advance the bookkeeping of every context by n steps
void advance(DirectState* d, long long n)
{
    d->phase = (int)((d->phase + n) & 1);
    for (mp_ctx* c : d->ctx) {
        c->cur = (int)((c->cur + n) & 1);
        c->t += n;
    }
}

bool capturable_stream(cudaStream_t s)
{
    return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

// n steps on the state's stream, without touching the contexts' bookkeeping
int run_steps(DirectState* d, long long n)
{
    if (d->persistent && d->pgrid > 0) {
        int ph = d->phase;
        while (n > 0) {
            const int m = (int)std::min<long long>(n, kMaxPersistentSteps);
            const int save = d->phase;
            d->phase = ph;
            const cudaError_t e = launch_persistent(d, m);
            d->phase = save;
            if (e != cudaSuccess) return cuda_fail(e, "mp_step: persistent launch");
            ph = (ph + m) & 1;
            n -= m;
        }
        return MP_OK;
    }
    const int ph0 = d->phase;
    int ph = ph0;
    cudaError_t le = cudaSuccess;
    // `count` one-step launches, then the launch that appends the last step's series
    auto plain = [&](long long count) {
        for (long long k = 0; k < count; ++k) {
            d->phase = ph;
            const cudaError_t e = launch_step(d, k > 0 ? 1 : 0);
            if (e != cudaSuccess && le == cudaSuccess) le = e;
            ph ^= 1;
        }
        if (count > 0) {
            const cudaError_t e = launch_finish(d, ph ^ 1);
            if (e != cudaSuccess && le == cudaSuccess) le = e;
        }
    };
    if (capturable_stream(d->stream) && n >= 2 * kGraphSteps) {
        const int b = ph;
        if (!d->exec[b]) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                plain(kGraphSteps);
                e = cudaStreamEndCapture(d->stream, &g);
            }
            ph = b;
            if (e == cudaSuccess && le != cudaSuccess) e = le;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&d->exec[b], g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                d->phase = ph0;
                return cuda_fail(e, "mp_step: graph capture");
            }
        }
        for (; n >= kGraphSteps; n -= kGraphSteps) {
            const cudaError_t e = cudaGraphLaunch(d->exec[b], d->stream);
            if (e != cudaSuccess) {
                d->phase = ph0;
                return cuda_fail(e, "mp_step: graph launch");
            }
        }
    }
    plain(n);
    d->phase = ph0;
    if (le != cudaSuccess) return cuda_fail(le, "mp_step: launch");
    return MP_OK;
}

// Time `steps` steps of each candidate variant on the current state and keep the fastest;
// the fields, adsorbed arrays and series position of every context are restored after each
// trial (the trials overwrite only series entries past the current time).
int autotune(DirectState* d, int steps)
{
    struct Cand {
        bool table, persistent;
        int block;
        bool tiled;
    };
    std::vector<Cand> cands;
    for (int tb = 1; tb >= 0; --tb)
        for (int ps = 0; ps < 2; ++ps) {
            for (int blk : {128, 256, 512}) cands.push_back({tb != 0, ps != 0, blk, false});
            if (!d->single && tb == 0) cands.push_back({false, ps != 0, 128, true});
        }
    const size_t n = d->ctx.size();
    std::vector<void*> bP(n, nullptr), bA(n, nullptr);
    std::vector<size_t> nP(n), nA(n);
    std::vector<long long> t0(n);
    int rc = MP_OK;
    for (size_t c = 0; c < n && rc == MP_OK; ++c) {
        mp_ctx* x = d->ctx[c];
        const size_t NI = (size_t)(x->geo.n_iface > 0 ? x->geo.n_iface : 1);
        nP[c] = (size_t)x->SP * (x->compact ? (size_t)x->geo.n_fluid : (size_t)x->geo.N) * x->FP * sizeof(float);
        nA[c] = (size_t)x->SP * NI * x->FP * sizeof(float);
        t0[c] = x->t;
        if (cudaMalloc(&bP[c], nP[c]) != cudaSuccess || cudaMalloc(&bA[c], nA[c]) != cudaSuccess) {
            (void)cudaGetLastError();
            set_error("autotune: no device memory for the state backup");
            rc = MP_ENOMEM;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == MP_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        set_error("autotune: event creation failed");
        rc = MP_ECUDA;
    }
    for (size_t c = 0; c < n && rc == MP_OK; ++c) {
        mp_ctx* x = d->ctx[c];
        if (cudaMemcpyAsync(bP[c], x->P[x->cur], nP[c], cudaMemcpyDeviceToDevice, d->stream) != cudaSuccess ||
            cudaMemcpyAsync(bA[c], x->A[x->cur], nA[c], cudaMemcpyDeviceToDevice, d->stream) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "autotune: backup");
    }
    float best_ms = 1e30f;
    Cand best{d->table, d->persistent, d->block, d->tiled};
    for (const Cand& cd : cands) {
        if (rc != MP_OK) break;
        d->table = cd.table;
        d->persistent = cd.persistent;
        d->block = cd.block;
        d->tiled = cd.tiled;
        rc = upload_args(d);
        if (rc != MP_OK) break;
        if (d->persistent && d->pgrid == 0) continue;
        float ms = 0.f;
        rc = run_steps(d, 2);  // warm-up of this variant
        cudaError_t e = rc == MP_OK ? cudaEventRecord(e0, d->stream) : cudaSuccess;
        if (rc == MP_OK && e == cudaSuccess) rc = run_steps(d, steps);
        if (rc == MP_OK && e == cudaSuccess) e = cudaEventRecord(e1, d->stream);
        if (rc == MP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (rc == MP_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        // restore the state the trial started from
        for (size_t c = 0; c < n && e == cudaSuccess && rc == MP_OK; ++c) {
            mp_ctx* x = d->ctx[c];
            e = cudaMemcpyAsync(x->P[x->cur], bP[c], nP[c], cudaMemcpyDeviceToDevice, d->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(x->A[x->cur], bA[c], nA[c], cudaMemcpyDeviceToDevice, d->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(x->tdev, &t0[c], sizeof(long long), cudaMemcpyHostToDevice, d->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (rc == MP_OK && e != cudaSuccess) rc = cuda_fail(e, "autotune");
        if (rc == MP_OK) rc = direct_state_check(d);
        if (rc == MP_OK && ms < best_ms) {
            best_ms = ms;
            best = cd;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (size_t c = 0; c < n; ++c) {
        cudaFree(bP[c]);
        cudaFree(bA[c]);
    }
    d->table = best.table;
    d->persistent = best.persistent;
    d->block = best.block;
    d->tiled = best.tiled;
    const int rc2 = upload_args(d);
    set_variant_name(d);
    return rc != MP_OK ? rc : rc2;
}

DArgs make_dargs(mp_ctx* c)
{
    DArgs a;
    memset(&a, 0, sizeof(a));
    a.nx = c->geo.nx;
    a.ny = c->geo.ny;
    a.nz = c->geo.nz;
    a.N = c->geo.N;
    a.NF = (int)c->geo.n_fluid;
    a.NI = (int)(c->geo.n_iface > 0 ? c->geo.n_iface : 1);
    a.dx = make_div((unsigned)c->geo.nx);
    a.dxy = make_div((unsigned)(c->geo.nx * c->geo.ny));
    a.S = c->S;
    a.M = c->M;
    a.SP = c->SP;
    a.K = c->S * c->M;
    for (int m = 0; m < 3; ++m) a.dir[m] = c->dir[m];
    a.in0 = c->cur;
    a.flist = c->dtab->flist;
    a.fmask = c->dtab->fmask;
    a.aidx = c->dtab->aidx;
    a.tab = c->dtab->tab;
    a.own = c->dtab->own;
    a.u4 = (const Flow4<float>*)c->u4;
    a.fw = c->dtab->fw;
    a.iw = c->dtab->iw;
    a.uc = c->dtab->uc;
    for (int b = 0; b < 2; ++b) {
        a.P[b] = (float*)c->P[b];
        a.A[b] = (float*)c->A[b];
    }
    for (int s = 0; s < c->S; ++s) {
        const float hl = (float)(6.0 * c->Db[s]);  // lambda/2 = 12 D_b / 2
        a.whf[s] = (float)((double)weight<float>(1) * (double)hl);
        a.whe[s] = (float)((double)weight<float>(5) * (double)hl);
        a.pa[s] = (float)c->ka[s];
        a.pd[s] = (float)c->kd[s];
    }
    a.Z = c->Z;
    a.D = c->D;
    a.tdev = c->tdev;
    a.cap = c->cap;
    return a;
}

}  // namespace

int direct_state_create(mp_ctx* const* ctxs, int n, cudaStream_t stream, int tune, int variant, DirectState** out)
{
    if (n < 1 || n > kMaxCtx) {
        set_error("direct scheme: 1..16 contexts per launch");
        return MP_EINVAL;
    }
    DirectState* d = new (std::nothrow) DirectState();
    if (!d) {
        set_error("host allocation failed");
        return MP_ENOMEM;
    }
    d->ctx.assign(ctxs, ctxs + n);
    d->stream = stream;
    d->FP = ctxs[0]->FP;
    d->single = true;
    for (mp_ctx* c : d->ctx) d->single = d->single && c->S == 1;
    d->table = !(variant & MP_VARIANT_RECOMPUTE);
    d->persistent = (variant & MP_VARIANT_PERSISTENT) != 0;
    d->block = (variant & MP_VARIANT_BLOCK128) ? 128 : ((variant & MP_VARIANT_BLOCK512) ? 512 : 256);
    d->tiled = (variant & MP_VARIANT_TILED) != 0 && !d->single;
    if (d->tiled) {
        d->table = false;  // the tiled body recomputes the link terms
        d->block = 128;    // and runs in blocks of 128 (one-species contexts of the launch too)
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete d;
        set_error("direct scheme: device query failed");
        return MP_ECUDA;
    }
    size_t part_elems = 0;
    for (mp_ctx* c : d->ctx) {
        d->h_args.push_back(make_dargs(c));
        set_tiles(d->h_args.back(), sms);
        part_elems += 2 * part_rows(d->h_args.back()) * (size_t)(c->S * c->M);
    }
    cudaError_t e = cudaMalloc(&d->d_args, sizeof(DArgs) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d->part, sizeof(double) * std::max<size_t>(part_elems, 1));
    if (e == cudaSuccess) e = cudaMalloc(&d->bar, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&d->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d->err, 0, sizeof(int), stream);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "direct scheme: state allocation");
        direct_state_free(d);
        return rc;
    }
    int rc = upload_args(d);
    if (rc == MP_OK && tune) {
        long long room = LLONG_MAX;
        for (mp_ctx* c : d->ctx) room = std::min(room, c->cap - 1 - c->t);
        if (room >= 24) rc = autotune(d, 20);  // needs series room for the trial steps
    }
    set_variant_name(d);
    if (rc != MP_OK) {
        direct_state_free(d);
        return rc;
    }
    *out = d;
    return MP_OK;
}

int direct_state_step(DirectState* d, long long n)
{
    if (n <= 0) return MP_OK;
    // the contexts may have been stepped by another launch state since (a group, or their
    // own): find the phase at which each reads its current buffer, and start afresh (phase
    // 0 at the current buffers) when they disagree
    const int ph = (d->ctx[0]->cur - d->h_args[0].in0) & 1;
    bool same = true;
    for (size_t c = 0; c < d->ctx.size(); ++c) same = same && ((d->ctx[c]->cur - d->h_args[c].in0) & 1) == ph;
    if (same) {
        d->phase = ph;
    } else {
        for (size_t c = 0; c < d->ctx.size(); ++c) d->h_args[c].in0 = d->ctx[c]->cur;
        d->phase = 0;
        if (int rc = upload_args(d)) return rc;
    }
    const int rc = run_steps(d, n);
    if (rc != MP_OK) return rc;
    advance(d, n);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int direct_state_check(DirectState* d)
{
    int h = 0;
    MP_CUDA(cudaMemcpyAsync(&h, d->err, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    MP_CUDA(cudaStreamSynchronize(d->stream));
    if (h != 0) {
        MP_CUDA(cudaMemsetAsync(d->err, 0, sizeof(int), d->stream));
        MP_CUDA(cudaStreamSynchronize(d->stream));
        set_error("a device-wide barrier wait of the persistent step gave up (fields and series after it are "
                  "not valid)");
        return MP_ETIMEOUT;
    }
    return MP_OK;
}

void direct_state_free(DirectState* d)
{
    if (!d) return;
    if (d->stream) cudaStreamSynchronize(d->stream);
    drop_graphs(d);
    cudaFree(d->d_args);
    cudaFree(d->part);
    cudaFree(d->bar);
    cudaFree(d->err);
    delete d;
}

const char* direct_state_variant(const DirectState* d) { return d ? d->variant.c_str() : ""; }

int direct_state_block(const DirectState* d) { return d ? d->block : 0; }

int direct_setup(mp_ctx* c, int tune, int variant)
{
    if (c->precision != MP_FP32) {
        set_error("the direct scheme runs FP32 storage only");
        return MP_EINVAL;
    }
    DirectTables* t = new (std::nothrow) DirectTables();
    if (!t) {
        set_error("host allocation failed");
        return MP_ENOMEM;
    }
    c->dtab = t;
    const size_t NF = (size_t)c->geo.n_fluid;
    t->OW = c->S == 1 ? (c->M == 1 ? 2 : 4) : 4 * (c->M == 1 ? 2 : 4);
    // the work list (the context's sorted fluid list) and the open-link masks in its order
    MP_CUDA(cudaMalloc(&t->flist, sizeof(int32_t) * NF));
    MP_CUDA(cudaMalloc(&t->fmask, sizeof(uint32_t) * NF));
    MP_CUDA(cudaMemcpyAsync(t->flist, c->geo.flist, sizeof(int32_t) * NF, cudaMemcpyDeviceToDevice, c->stream));
    MP_CUDA(cudaMalloc(&t->aidx, sizeof(int32_t) * NF));
    MP_CUDA(cudaMalloc(&t->tab, sizeof(float) * 18 * ((NF + 31) / 32 * 32)));
    MP_CUDA(cudaMalloc(&t->own, sizeof(float) * t->OW * NF));
    const float hl = (float)(6.0 * c->Db[0]);
    const float whf = (float)((double)weight<float>(1) * (double)hl);
    const float whe = (float)((double)weight<float>(5) * (double)hl);
    k_direct_tables<<<(unsigned)((NF + 255) / 256), 256, 0, c->stream>>>(
        t->flist, c->geo.fluid, t->fmask, c->geo.iface, c->geo.ibase, (const Flow4<float>*)c->u4, (int)NF, c->geo.nx,
        c->geo.ny, c->geo.nz, make_div((unsigned)c->geo.nx), make_div((unsigned)(c->geo.nx * c->geo.ny)),
        c->S == 1 ? 1 : 0, c->M, c->dir[0], c->dir[1], c->dir[2], whf, whe, (float)c->ka[0], t->aidx, t->tab, t->own);
    MP_CUDA(cudaGetLastError());
    if (c->compact) {
        MP_CUDA(cudaMalloc(&t->fw, sizeof(uint2) * (size_t)c->geo.W));
        MP_CUDA(cudaMalloc(&t->iw, sizeof(uint2) * (size_t)c->geo.W));
        MP_CUDA(cudaMalloc(&t->uc, sizeof(Flow4<float>) * NF));
        k_fluid_words<<<(unsigned)((c->geo.W + 255) / 256), 256, 0, c->stream>>>(c->geo.fluid, c->geo.fbase, c->geo.W,
                                                                                   t->fw);
        k_fluid_words<<<(unsigned)((c->geo.W + 255) / 256), 256, 0, c->stream>>>(c->geo.iface, c->geo.ibase, c->geo.W,
                                                                                   t->iw);
        k_list_flow<<<(unsigned)((NF + 255) / 256), 256, 0, c->stream>>>(t->flist, (const Flow4<float>*)c->u4, (int)NF,
                                                                          t->uc);
        MP_CUDA(cudaGetLastError());
    }
    mp_ctx* one[1] = {c};
    return direct_state_create(one, 1, c->stream, tune, variant, &c->dstate);
}

int direct_step(mp_ctx* c, long long n) { return direct_state_step(c->dstate, n); }

int direct_check(mp_ctx* c) { return c->dstate ? direct_state_check(c->dstate) : MP_OK; }

void direct_free(mp_ctx* c)
{
    if (c->dstate) direct_state_free(c->dstate);
    c->dstate = nullptr;
    if (c->dtab) {
        cudaFree(c->dtab->flist);
        cudaFree(c->dtab->fmask);
        cudaFree(c->dtab->aidx);
        cudaFree(c->dtab->tab);
        cudaFree(c->dtab->own);
        cudaFree(c->dtab->fw);
        cudaFree(c->dtab->iw);
        cudaFree(c->dtab->uc);
        delete c->dtab;
    }
    c->dtab = nullptr;
}

}  // namespace mp

// ---------------------------------------------------------------------------------------
// C ABI: self-test of the bounded device-wide barrier
// ---------------------------------------------------------------------------------------
extern "C" int mp_grid_wait_selftest(int n_blocks, int rounds, int unreachable, int64_t timeout_ns, void* stream)
{
    using namespace mp;
    clear_error();
    if (n_blocks < 1 || rounds < 1 || rounds > 1000000 || timeout_ns < 0 || timeout_ns > 10000000000LL) {
        set_error("mp_grid_wait_selftest: need n_blocks >= 1, 1 <= rounds <= 1e6, 0 <= timeout_ns <= 1e10");
        return MP_EINVAL;
    }
    int dev = 0, sms = 0, per_sm = 0;
    MP_CUDA(cudaGetDevice(&dev));
    MP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_wait_selftest, 32, 0));
    if (n_blocks > sms * per_sm) {
        set_error("mp_grid_wait_selftest: more blocks than can be resident at once");
        return MP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int* bar = nullptr;
    int* err = nullptr;
    MP_CUDA(cudaMalloc(&bar, sizeof(unsigned int)));
    cudaError_t e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n_blocks);
        cfg.blockDim = dim3(32);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_grid_wait_selftest, rounds, unreachable, bar, err, (long long)timeout_ns);
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bar);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "mp_grid_wait_selftest");
    if (h != 0) {
        set_error("mp_grid_wait_selftest: a barrier wait gave up");
        return MP_ETIMEOUT;
    }
    return MP_OK;
}
