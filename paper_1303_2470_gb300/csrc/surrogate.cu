// surrogate.cu -- kernels of the learned warm start for lb_steady (include/surrogate.h): 3x3x3
// periodic convolutions as implicit GEMMs on the tensor cores (forward and input-gradient
// convolutions on the 5th-generation tensor cores, tcgen05.mma with accumulators in tensor
// memory; the weight gradient with mma.sync m16n8k16; BF16 operands, FP32 accumulation),
// pooling, upsampling, the masked loss and the Adam update. Nothing here belongs to the moment-propagation
// method itself; the network's output only seeds lb_steady.
#include <cuda_bf16.h>

#include "../../include/surrogate.h"
#include "internal.cuh"

using namespace mp;

namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// D += A B for one m16n8k16 tile; fragments as the PTX ISA lays them out for .bf16:
// a0..a3 rows (g, g+8) x cols (2t, 2t+1) and (+8); b0, b1 rows (2t, 2t+1) and (+8) of col g.
__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct ConvArgs {
    const bf16* x;
    const bf16* w;
    const float* bias;
    bf16* y;
    float* yf;
    int D, H, W, V, K, N, sign, relu;
};

// ---------------------------------------------------------------------------------------
// Forward (and transposed) convolution on the 5th-generation tensor cores: an implicit GEMM
// with M = 128 voxels per block, N = the block's output channels (up to 256, one MMA wide),
// K = 27 taps x K input channels, flattened tap-major, in stages of 64 consecutive elements
// (four MMAs of K = 16; a stage spans several taps when K < 64). Operands sit in shared
// memory in the K-major layout with 128-byte swizzling:
// each 8-row group is one 1024-byte atom whose row r holds the stage's 64 elements as eight
// 16-byte chunks, chunk j stored at position j ^ (r mod 8); a descriptor with stride offset
// 1024 (next atom) whose start advances by 32 bytes per 16-channel slice describes any
// K = 16 slice. With this layout the eight lanes that copy one voxel row read its 128
// contiguous bytes and write eight distinct bank groups. The accumulators (FP32) live in
// tensor memory; one thread issues the MMAs. A ring of shared-memory stages is filled by
// asynchronous copies (cp.async, L1-cached, zero-filled outside the volume); the MMAs of a
// stage signal an mbarrier when they complete, which frees its buffer for the copies of a
// later stage. The epilogue reads the accumulators back with tcgen05.ld (warp w holds rows
// 32w..32w+31), adds the bias, applies the ReLU and stores. Every wait is bounded; a wait
// that gives up records it in g_sg_tc_fail (read by sg_check), and the block still releases
// its tensor memory.
// ---------------------------------------------------------------------------------------
constexpr int kTM = 128;         // voxels per block (MMA M)
constexpr int kTKC = 64;         // reduction elements per stage: one swizzle atom row (128 bytes)
#ifndef SG_TC_STAGES
#define SG_TC_STAGES 2
#endif
constexpr int kTStages = SG_TC_STAGES;  // shared-memory ring
constexpr int kTThreads = 128;   // four warps: one accumulator row per thread
constexpr int kTMaxN = 256;      // output channels per block (MMA N)
constexpr int kTAtom = 1024;     // one 8-row group: 8 rows x 128 bytes
constexpr int kTABytes = (kTM / 8) * kTAtom;
constexpr int kTPieces = kTM * 8 / kTThreads;  // 16-byte A pieces per thread and stage
constexpr long long kTWaitNs = 1000000000LL;  // a wait gives up after 1 s of the global timer

__device__ int g_sg_tc_fail;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of 16-byte chunk j of row r in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t swz(int r, int j)
{
    return (uint32_t)((r >> 3) * kTAtom + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

// shared-memory matrix descriptor: start address, stride byte offset 1024 (next 8-row atom),
// leading offset unused with swizzling (1), descriptor version 1 (bit 46), 128-byte
// swizzling (mode 2, bits 61-63)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(kTAtom >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

// 16-byte asynchronous copy global -> shared (zero-filled beyond `bytes`), through L1, where
// the tap-shifted tiles of one block overlap
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ unsigned long long tc_now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of parity `parity` of an mbarrier to complete; false after kTWaitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const unsigned long long t0 = tc_now_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.b32 %0, 1, 0, q;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((long long)(tc_now_ns() - t0) > kTWaitNs) return false;
    }
}

// Epilogue of the tensor-core convolutions: warp w reads accumulator rows 32w..32w+31 (its
// lanes' voxels) from tensor memory, adds the bias, applies the ReLU and stores BF16 and/or
// FP32 outputs of voxel v, channels n0..n0+BN-1.
__device__ __forceinline__ void conv_epilogue(const ConvArgs& a, uint32_t tmem, int warp, int b, int v, int n0, int BN)
{
    const bool vok = v < a.V;
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        const uint32_t addr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!vok) continue;
        const size_t o = ((size_t)b * a.V + v) * a.N + n0 + c0;
        float f[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float t = __uint_as_float(r[c]) + (a.bias ? a.bias[n0 + c0 + c] : 0.0f);
            f[c] = a.relu ? fmaxf(t, 0.0f) : t;
        }
        if (a.y) {
            uint32_t h[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const __nv_bfloat162 p2 = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
                h[c] = *reinterpret_cast<const uint32_t*>(&p2);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.y + o);
            dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
            dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
        }
        if (a.yf) {
            float4* dst = reinterpret_cast<float4*>(a.yf + o);
#pragma unroll
            for (int c = 0; c < 4; ++c) dst[c] = make_float4(f[4 * c], f[4 * c + 1], f[4 * c + 2], f[4 * c + 3]);
        }
    }
}

template <int kK>  // input channels, 0: a.K at run time
__global__ void __launch_bounds__(kTThreads) k_conv_tc(const ConvArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t mbar[kTStages];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n0 = blockIdx.y * kTMaxN;
    const int BN = a.N - n0 < kTMaxN ? a.N - n0 : kTMaxN;  // a multiple of 16
    const int BBytes = (BN / 8) * kTAtom;
    // operand atoms must start on 1024-byte boundaries (the swizzle pattern is anchored there)
    unsigned char* tc_smem = tc_smem_raw + ((kTAtom - (smem_u32(tc_smem_raw) & (kTAtom - 1))) & (kTAtom - 1));
    unsigned char* sA = tc_smem;
    unsigned char* sB = tc_smem + kTStages * kTABytes;
    const int b = blockIdx.z;
    const int v = blockIdx.x * kTM + tid;  // this thread's result row
    // A pieces of this thread: piece p = tid + 128 i covers row p / 8, chunk p % 8 (the
    // chunk is the same for every i)
    const int pj = tid & 7;
    // source voxel of every (tap, row) of the block, periodic (-1: the row lies beyond the
    // volume), computed once: thread t fills row t
    __shared__ int s_src[27][kTM];
    {
        int x = 0, y = 0, z = 0;
        if (v < a.V) {
            x = v % a.W;
            y = (v / a.W) % a.H;
            z = v / (a.W * a.H);
        }
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            s_src[tap][tid] = v < a.V ? (wrap(z + a.sign * dz, a.D) * a.H + wrap(y + a.sign * dy, a.H)) * a.W +
                                            wrap(x + a.sign * dx, a.W)
                                      : -1;
        }
    }
    // stages: 64 consecutive elements of the flattened (tap, channel) reduction index (tap
    // major); a 16-byte chunk never straddles two taps since K is a multiple of 16
    const int K = kK ? kK : a.K;
    const int nst = (27 * K + kTKC - 1) / kTKC;
    uint32_t ncols = 32;
    while ((int)ncols < BN) ncols <<= 1;
    if (tid == 0) {
        for (int s = 0; s < kTStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const bf16* xb = a.x + (size_t)b * a.V * a.K;

    // reduction elements of stage st (a multiple of 16), and the tap and channel of chunk j
    auto stage_kc = [&](int st) { return 27 * K - st * kTKC < kTKC ? 27 * K - st * kTKC : kTKC; };
    auto chunk_of = [&](int st, int j, int& tap, int& ch) {
        const int e = st * kTKC + 8 * j;
        tap = e / K;
        ch = e - tap * K;
    };

    // asynchronous copies of stage st into ring buffer buf
    auto load_stage = [&](int st, int buf) {
        const int kc = stage_kc(st);
        const uint32_t abase = smem_u32(sA + buf * kTABytes);
        if (pj < kc / 8) {
            int tap, ch;
            chunk_of(st, pj, tap, ch);
#pragma unroll
            for (int i = 0; i < kTPieces; ++i) {
                const int row = (tid + kTThreads * i) >> 3;
                const int sv = s_src[tap][row];
                // any valid address (zero-filled) when the row lies outside the volume
                const bf16* src = xb + (sv >= 0 ? (size_t)sv * K + ch : 0);
                cp_async16(abase + swz(row, pj), src, sv >= 0 ? 16u : 0u);
            }
        }
        const uint32_t bbase = smem_u32(sB + buf * BBytes);
        for (int p = tid; p < BN * 8; p += kTThreads) {
            const int n = p >> 3, j = p & 7;
            if (j < kc / 8) {
                int tap, ch;
                chunk_of(st, j, tap, ch);
                cp_async16(bbase + swz(n, j), a.w + ((size_t)tap * a.N + n0 + n) * K + ch, 16u);
            }
        }
    };

    bool ok = true;
    for (int s = 0; s < kTStages - 1; ++s) {
        if (s < nst) load_stage(s, s);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int st = 0; st < nst; ++st) {
        const int buf = st % kTStages;
        // refill: stage st + kTStages - 1 goes to the buffer that stage st - 1's MMAs read
        const int nxt = st + kTStages - 1;
        if (nxt < nst) {
            if (st >= 1) ok = mbar_wait(smem_u32(&mbar[(st - 1) % kTStages]), (uint32_t)(((st - 1) / kTStages) & 1));
            if (ok) load_stage(nxt, nxt % kTStages);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(kTStages - 1) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int kc = stage_kc(st);
            const uint32_t abase = smem_u32(sA + buf * kTABytes), bbase = smem_u32(sB + buf * BBytes);
            const uint32_t idesc = tc_idesc(BN);
            for (int kk = 0; kk < kc; kk += 16) {
                const uint64_t ad = tc_desc(abase + kk * 2), bd = tc_desc(bbase + kk * 2);
                const uint32_t accum = (st > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    // the last stage's commit covers every MMA of the block (they complete in order)
    if (ok) ok = mbar_wait(smem_u32(&mbar[(nst - 1) % kTStages]), (uint32_t)(((nst - 1) / kTStages) & 1));
    if (!ok && tid == 0) atomicExch(&g_sg_tc_fail, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_and(ok)) conv_epilogue(a, tmem, warp, b, v, n0, BN);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------------------
// The same convolution where a block's 128 voxels are one stretch of an x-row (W a multiple
// of 128) and K <= 64: the three taps that differ only in dx read the same source row, so a
// stage holds that row once — the 130 voxels x0 - 1 .. x0 + 128 (periodic) of the source
// row (y + s dy, z + s dz), s the sign — and the taps dx = -1, 0, +1 are three groups of MMAs
// whose A descriptors start 0, 1 or 2 rows into it (the 128-byte swizzle is keyed to the
// absolute shared-memory address, so a descriptor may start at any row of an atom). Nine
// stages, one per (dz, dy), in tap order; within a stage the taps in dx order and each tap's
// channels in order, so the accumulation order is that of k_conv_tc and the outputs are
// bitwise the same. Three B tiles (one per dx) per stage.
// ---------------------------------------------------------------------------------------
constexpr int kRRows = 136;                  // staged source row: 130 voxels in 17 atoms
constexpr int kRABytes = (kRRows / 8) * kTAtom;
constexpr int kRMaxN = 64;                   // output channels: the ring stays below 90 KB

template <int kK>
__global__ void __launch_bounds__(kTThreads) k_conv_row(const ConvArgs a)
{
    static_assert(kK == 16 || kK == 32 || kK == 64, "one swizzle atom row per voxel");
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t mbar[kTStages];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n0 = blockIdx.y * kTMaxN;
    const int BN = a.N - n0 < kTMaxN ? a.N - n0 : kTMaxN;  // a multiple of 16
    const int BTile = (BN / 8) * kTAtom;                   // one tap's B tile
    unsigned char* tc_smem = tc_smem_raw + ((kTAtom - (smem_u32(tc_smem_raw) & (kTAtom - 1))) & (kTAtom - 1));
    unsigned char* sA = tc_smem;
    unsigned char* sB = tc_smem + kTStages * kRABytes;
    const int b = blockIdx.z;
    const int v0 = blockIdx.x * kTM, v = v0 + tid;
    const int x0 = v0 % a.W, y = (v0 / a.W) % a.H, z = v0 / (a.W * a.H);
    constexpr int kJ = kK / 8;  // 16-byte chunks of a voxel's channels
    uint32_t ncols = 32;
    while ((int)ncols < BN) ncols <<= 1;
    if (tid == 0) {
        for (int s = 0; s < kTStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const bf16* xb = a.x + (size_t)b * a.V * kK;

    // stage st = 3 (dz + 1) + (dy + 1): the source row and the three taps' weights
    auto load_stage = [&](int st, int buf) {
        const int dz = st / 3 - 1, dy = st % 3 - 1;
        const int ys = wrap(y + a.sign * dy, a.H), zs = wrap(z + a.sign * dz, a.D);
        const bf16* row = xb + (size_t)(zs * a.H + ys) * a.W * kK;
        const uint32_t abase = smem_u32(sA + buf * kRABytes);
        for (int p = tid; p < 130 * kJ; p += kTThreads) {
            const int r = p / kJ, j = p - r * kJ;
            const int x = wrap(x0 - 1 + r, a.W);
            cp_async16(abase + swz(r, j), row + (size_t)x * kK + 8 * j, 16u);
        }
        const uint32_t bbase = smem_u32(sB + buf * 3 * BTile);
        for (int p = tid; p < 3 * BN * kJ; p += kTThreads) {
            const int t = p / (BN * kJ), q = p - t * (BN * kJ);
            const int n = q / kJ, j = q - n * kJ;
            const int tap = 3 * st + t;  // 9 (dz + 1) + 3 (dy + 1) + (dx + 1)
            cp_async16(bbase + t * BTile + swz(n, j), a.w + ((size_t)tap * a.N + n0 + n) * kK + 8 * j, 16u);
        }
    };

    bool ok = true;
    constexpr int nst = 9;
    for (int s = 0; s < kTStages - 1; ++s) {
        load_stage(s, s);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int st = 0; st < nst; ++st) {
        const int buf = st % kTStages;
        const int nxt = st + kTStages - 1;
        if (nxt < nst) {
            if (st >= 1) ok = mbar_wait(smem_u32(&mbar[(st - 1) % kTStages]), (uint32_t)(((st - 1) / kTStages) & 1));
            if (ok) load_stage(nxt, nxt % kTStages);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(kTStages - 1) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t abase = smem_u32(sA + buf * kRABytes), bbase = smem_u32(sB + buf * 3 * BTile);
            const uint32_t idesc = tc_idesc(BN);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                // tap dx = t - 1 reads source voxel x + s dx: row 1 + s dx of the stage
                const uint32_t arow = (uint32_t)(1 + a.sign * (t - 1)) * 128u;
#pragma unroll
                for (int kk = 0; kk < kK; kk += 16) {
                    const uint64_t ad = tc_desc(abase + arow + kk * 2), bd = tc_desc(bbase + t * BTile + kk * 2);
                    const uint32_t accum = (st > 0 || t > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (ok) ok = mbar_wait(smem_u32(&mbar[(nst - 1) % kTStages]), (uint32_t)(((nst - 1) / kTStages) & 1));
    if (!ok && tid == 0) atomicExch(&g_sg_tc_fail, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_and(ok)) conv_epilogue(a, tmem, warp, b, v, n0, BN);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

struct WgradArgs {
    const bf16* x;
    const bf16* dy;
    float* dw;
    int D, H, W, V, Cin, Cout;
    long long total;  // B * V voxels of the reduction
    int chunk;        // voxels per block (a multiple of 32)
    int ci_tiles;     // tiles of 64 input channels
};

// four 8x8 BF16 matrices from shared memory, transposed on the way (lanes 8j..8j+7 give the
// row addresses of matrix j): each lane receives (M[2(l%4)][l/4], M[2(l%4)+1][l/4]) of every
// matrix, which is the m16n8k16 fragment layout for an operand stored K-major
__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const bf16* p)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

constexpr int kWM = 64, kWN = 64, kWS = 32, kWLd = 72, kWThreads = 128;

// Weight gradient of one tap (blockIdx.x % 27) over one chunk of voxels (blockIdx.x / 27) for
// one 64 x 64 tile of (input, output) channels (blockIdx.y): rows = input channels, columns =
// output channels, reduction over voxels in stages of 32. Both operands stay channels-last in
// shared memory ([voxel][channel], 144-byte rows) and the fragments come from transposing
// loads. The next stage is fetched into registers during the current one's products.
__global__ void __launch_bounds__(kWThreads) k_wgrad(const WgradArgs a)
{
    __shared__ __align__(16) bf16 Xs[2][kWS][kWLd];
    __shared__ __align__(16) bf16 Gs[2][kWS][kWLd];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tap = blockIdx.x % 27;
    const long long e0 = (long long)(blockIdx.x / 27) * a.chunk;
    const long long e1 = e0 + a.chunk < a.total ? e0 + a.chunk : a.total;
    const int ci0 = (blockIdx.y % a.ci_tiles) * kWM, co0 = (blockIdx.y / a.ci_tiles) * kWN;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int lr = tid >> 2, lc = (tid & 3) * 16;  // this thread stages voxel row lr, 16 channels from lc
    const int ncols = a.Cout - co0 < kWN ? a.Cout - co0 : kWN;
    uint4 rx0, rx1, rg0, rg1;
    auto fetch = [&](long long e) {
        rx0 = rx1 = rg0 = rg1 = make_uint4(0u, 0u, 0u, 0u);
        const long long ev = e + lr;
        if (ev < e1) {
            const long long bb = ev / a.V;
            const int v = (int)(ev - bb * a.V);
            const int xa = v % a.W, ya = (v / a.W) % a.H, za = v / (a.W * a.H);
            const int xs = wrap(xa + dx, a.W), ys = wrap(ya + dy, a.H), zs = wrap(za + dz, a.D);
            const size_t src = (size_t)bb * a.V + (size_t)((zs * a.H + ys) * a.W + xs);
            if (ci0 + lc < a.Cin) {
                const bf16* p = a.x + src * a.Cin + ci0 + lc;
                rx0 = *reinterpret_cast<const uint4*>(p);
                rx1 = *reinterpret_cast<const uint4*>(p + 8);
            }
            if (co0 + lc < a.Cout) {
                const bf16* p = a.dy + (size_t)ev * a.Cout + co0 + lc;
                rg0 = *reinterpret_cast<const uint4*>(p);
                rg1 = *reinterpret_cast<const uint4*>(p + 8);
            }
        }
    };
    auto stash = [&](int buf) {
        *reinterpret_cast<uint4*>(&Xs[buf][lr][lc]) = rx0;
        *reinterpret_cast<uint4*>(&Xs[buf][lr][lc + 8]) = rx1;
        *reinterpret_cast<uint4*>(&Gs[buf][lr][lc]) = rg0;
        *reinterpret_cast<uint4*>(&Gs[buf][lr][lc + 8]) = rg1;
    };
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;
    const int nst = (int)((e1 - e0 + kWS - 1) / kWS);
    const int r = lane & 7, mat = lane >> 3;
    fetch(e0);
    stash(0);
    __syncthreads();
    for (int st = 0; st < nst; ++st) {
        const int cur = st & 1;
        if (st + 1 < nst) fetch(e0 + (long long)(st + 1) * kWS);
#pragma unroll
        for (int kk = 0; kk < kWS; kk += 16) {
            // A (rows = input channels of this warp): matrices (m0, k0) = (0,0), (8,0), (0,8), (8,8)
            uint32_t a0, a1, a2, a3;
            ldsm_x4_t(a0, a1, a2, a3, &Xs[cur][kk + (mat >> 1) * 8 + r][warp * 16 + (mat & 1) * 8]);
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                if (np * 16 < ncols) {
                    // B for column tiles 2np and 2np+1: matrices (k0, n0) = (0,0), (8,0), (0,8), (8,8)
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_t(b0, b1, b2, b3, &Gs[cur][kk + (mat & 1) * 8 + r][np * 16 + (mat >> 1) * 8]);
                    mma16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
                    if ((2 * np + 1) * 8 < ncols) mma16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
        if (st + 1 < nst) stash(cur ^ 1);
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int co = co0 + nt * 8 + 2 * t;
        if (co >= a.Cout) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ci = ci0 + warp * 16 + g + 8 * h;
            if (ci >= a.Cin) continue;
            float* d = a.dw + ((size_t)tap * a.Cin + ci) * a.Cout + co;
            atomicAdd(d, acc[nt][2 * h]);
            atomicAdd(d + 1, acc[nt][2 * h + 1]);
        }
    }
}

// dbias[c] += sum over voxels of dy[.][c]: block = 256 voxels x one channel group of 32
__global__ void k_bias_grad(const bf16* __restrict__ dy, float* __restrict__ db, long long total, int C)
{
    const int c = blockIdx.y * 32 + (threadIdx.x & 31);
    const int r = threadIdx.x >> 5;  // 8 rows of voxels
    float s = 0.0f;
    if (c < C)
        for (long long e = (long long)blockIdx.x * 256 + r; e < total && e < (long long)(blockIdx.x + 1) * 256; e += 8)
            s += __bfloat162float(dy[(size_t)e * C + c]);
    __shared__ float part[8][32];
    part[r][threadIdx.x & 31] = s;
    __syncthreads();
    if (r == 0 && c < C) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
        atomicAdd(db + c, t);
    }
}

// pooling / upsampling over one BF16 channel pair per thread
__global__ void k_pool2(const bf16* __restrict__ x, bf16* __restrict__ y, int B, int D, int H, int W, int C)
{
    const int d = D / 2, h = H / 2, w = W / 2, C2 = C / 2;
    const long long n = (long long)B * d * h * w * C2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C2) * 2;
    long long r = i / C2;
    const int xo = (int)(r % w), yo = (int)((r / w) % h), zo = (int)((r / ((long long)w * h)) % d);
    const int b = (int)(r / ((long long)w * h * d));
    float s0 = 0.0f, s1 = 0.0f;
    for (int k = 0; k < 8; ++k) {
        const int xs = 2 * xo + (k & 1), ys = 2 * yo + ((k >> 1) & 1), zs = 2 * zo + (k >> 2);
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(
            x + ((((size_t)b * D + zs) * H + ys) * W + xs) * C + c);
        s0 += __low2float(v);
        s1 += __high2float(v);
    }
    *reinterpret_cast<__nv_bfloat162*>(y + (size_t)r * C + c) = __floats2bfloat162_rn(s0 * 0.125f, s1 * 0.125f);
}

// fine-grid pass: every fine voxel reads its coarse parent (pool gradient / upsampling)
template <bool kPoolGrad>
__global__ void k_fine_from_coarse(const bf16* __restrict__ src, bf16* __restrict__ dst, int B, int D, int H, int W,
                                   int C)
{
    // D, H, W: coarse sizes
    const int Df = 2 * D, Hf = 2 * H, Wf = 2 * W, C2 = C / 2;
    const long long n = (long long)B * Df * Hf * Wf * C2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C2) * 2;
    const long long r = i / C2;
    const int xf = (int)(r % Wf), yf = (int)((r / Wf) % Hf), zf = (int)((r / ((long long)Wf * Hf)) % Df);
    const int b = (int)(r / ((long long)Wf * Hf * Df));
    const size_t p = ((((size_t)b * D + zf / 2) * H + yf / 2) * W + xf / 2) * C + c;
    __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(src + p);
    if (kPoolGrad) v = __floats2bfloat162_rn(__low2float(v) * 0.125f, __high2float(v) * 0.125f);
    *reinterpret_cast<__nv_bfloat162*>(dst + (size_t)r * C + c) = v;
}

// coarse-grid pass: sum of the 8 children (upsampling gradient)
__global__ void k_up2_grad(const bf16* __restrict__ dy, bf16* __restrict__ dx, int B, int D, int H, int W, int C)
{
    const int C2 = C / 2;
    const long long n = (long long)B * D * H * W * C2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C2) * 2;
    const long long r = i / C2;
    const int xo = (int)(r % W), yo = (int)((r / W) % H), zo = (int)((r / ((long long)W * H)) % D);
    const int b = (int)(r / ((long long)W * H * D));
    const int Hf = 2 * H, Wf = 2 * W, Df = 2 * D;
    float s0 = 0.0f, s1 = 0.0f;
    for (int k = 0; k < 8; ++k) {
        const int xs = 2 * xo + (k & 1), ys = 2 * yo + ((k >> 1) & 1), zs = 2 * zo + (k >> 2);
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(
            dy + ((((size_t)b * Df + zs) * Hf + ys) * Wf + xs) * C + c);
        s0 += __low2float(v);
        s1 += __high2float(v);
    }
    *reinterpret_cast<__nv_bfloat162*>(dx + (size_t)r * C + c) = __floats2bfloat162_rn(s0, s1);
}

__global__ void k_add(const bf16* __restrict__ a, const bf16* __restrict__ b, bf16* y, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

__global__ void k_relu_grad(const bf16* __restrict__ act, bf16* __restrict__ g, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(__bfloat162float(act[i]) > 0.0f)) g[i] = __float2bfloat16_rn(0.0f);
}

// network coordinates (p, q, r) of lattice node (x, y, z) for a force along `axis`: the
// forced axis comes first, the other two keep their order
__device__ __forceinline__ void to_net(int axis, int x, int y, int z, int& p, int& q, int& r)
{
    if (axis == 0) {
        p = x; q = y; r = z;
    } else if (axis == 1) {
        p = y; q = x; r = z;
    } else {
        p = z; q = x; r = y;
    }
}
__device__ __forceinline__ void net_dims(int axis, int nx, int ny, int nz, int& P, int& Q, int& R)
{
    to_net(axis, nx, ny, nz, P, Q, R);
}
// lattice component of network channel c
__device__ __forceinline__ int lattice_comp(int axis, int c)
{
    if (axis == 0) return c;
    if (axis == 1) return c == 0 ? 1 : (c == 1 ? 0 : 2);
    return c == 0 ? 2 : (c == 1 ? 0 : 1);
}

// network voxel index (x fastest in network order: p fastest) of lattice node n
__device__ __forceinline__ int net_voxel(int axis, int n, int nx, int ny, int nz)
{
    const int x = n % nx, y = (n / nx) % ny, z = n / (nx * ny);
    int p, q, r, P, Q, R;
    to_net(axis, x, y, z, p, q, r);
    net_dims(axis, nx, ny, nz, P, Q, R);
    return (r * Q + q) * P + p;
}

__global__ void k_pack_input(const uint8_t* __restrict__ cls, bf16* __restrict__ x, int nx, int ny, int nz, int axis)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    if (n >= N) return;
    const int v = net_voxel(axis, n, nx, ny, nz);
    const uint8_t c = cls[n];
    bf16* o = x + (size_t)v * 16;
    const bf16 zero = __float2bfloat16_rn(0.0f);
    o[0] = __float2bfloat16_rn((c & 3) != 0 ? 1.0f : 0.0f);
    o[1] = __float2bfloat16_rn((c & 4) != 0 ? 1.0f : 0.0f);
    for (int k = 2; k < 16; ++k) o[k] = zero;
}

// sum and count of y[.][3] over the forced cluster (FP64)
__global__ void k_cluster_mean(const float* __restrict__ y, int ldy, const uint8_t* __restrict__ cls, int nx, int ny,
                               int nz, int axis, double* __restrict__ acc)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    double s = 0.0, c = 0.0;
    if (n < N && (cls[n] & 4)) {
        s = y[(size_t)net_voxel(axis, n, nx, ny, nz) * ldy + 3];
        c = 1.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0 && c > 0.0) {
        atomicAdd(acc, s);
        atomicAdd(acc + 1, c);
    }
}

__global__ void k_unpack_output(const float* __restrict__ y, int ldy, const uint8_t* __restrict__ cls,
                                float* __restrict__ u, float* __restrict__ rho, int nx, int ny, int nz, int axis,
                                float scale_u, float scale_rho, const double* __restrict__ acc)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    if (n >= N || !(cls[n] & 4)) return;
    const int v = net_voxel(axis, n, nx, ny, nz);
    for (int c = 0; c < 3; ++c) u[(size_t)lattice_comp(axis, c) * N + n] += scale_u * y[(size_t)v * ldy + c];
    if (rho) {
        const float m = (float)(acc[0] / acc[1]);
        rho[n] += scale_rho * (y[(size_t)v * ldy + 3] - m);
    }
}

__global__ void k_pack_target(const float* __restrict__ u, const float* __restrict__ rho, float* __restrict__ t,
                              int nx, int ny, int nz, int axis, float scale_u, float scale_rho)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = nx * ny * nz;
    if (n >= N) return;
    const int v = net_voxel(axis, n, nx, ny, nz);
    for (int c = 0; c < 3; ++c) t[(size_t)v * 4 + c] = scale_u * u[(size_t)lattice_comp(axis, c) * N + n];
    t[(size_t)v * 4 + 3] = rho[n] > 0.0f ? scale_rho * (rho[n] - 1.0f) : 0.0f;
}

__global__ void k_mse(const float* __restrict__ y, int ldy, const float* __restrict__ t, int nc,
                      const bf16* __restrict__ x, bf16* __restrict__ dy, double* __restrict__ loss, long long total,
                      double inv)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (e < total) {
        const bool fluid = __bfloat162float(x[(size_t)e * 16]) > 0.5f;
        for (int c = 0; c < ldy; ++c) {
            float gval = 0.0f;
            if (fluid && c < nc) {
                const float d = y[(size_t)e * ldy + c] - t[(size_t)e * nc + c];
                s += (double)d * d;
                gval = (float)(2.0 * inv) * d;
            }
            dy[(size_t)e * ldy + c] = __float2bfloat16_rn(gval);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(loss, s * inv);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2, bf16* __restrict__ wf,
                       bf16* __restrict__ wb, int cin, int cout)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (wf) {
        // master index (tap, ci, co) -> forward copy [tap][co][ci], transposed copy [tap][ci][co]
        const long long per = (long long)cin * cout;
        const int tap = (int)(i / per);
        const int ci = (int)((i % per) / cout), co = (int)(i % cout);
        const bf16 h = __float2bfloat16_rn(pi);
        wf[((size_t)tap * cout + co) * cin + ci] = h;
        wb[i] = h;
    }
}

int grid1(long long n, int block) { return (int)((n + block - 1) / block); }

}  // namespace

extern "C" {

int sg_conv3d(const void* x, const void* w, const float* bias, void* y, float* yf, int B, int D, int H, int W, int K,
              int N, int sign, int relu, void* stream)
{
    clear_error();
    if (!x || !w || (!y && !yf) || B < 1 || D < 1 || H < 1 || W < 1 || K < 16 || N < 16 || K % 16 || N % 16 ||
        (sign != 1 && sign != -1) || (long long)D * H * W > (1LL << 30)) {
        set_error("sg_conv3d: needs x, w, an output, B, D, H, W >= 1, K and N multiples of 16, sign +-1");
        return MP_EINVAL;
    }
    ConvArgs a{(const bf16*)x, (const bf16*)w, bias, (bf16*)y, yf, D, H, W, D * H * W, K, N, sign, relu != 0};
    const int bn = N < kTMaxN ? N : kTMaxN;
    if (W % kTM == 0 && (K == 16 || K == 32 || K == 64) && N <= kRMaxN) {
        // blocks of 128 voxels lie in one x-row: the row-staged kernel
        void (*rkern)(const ConvArgs) = K == 16 ? k_conv_row<16> : K == 32 ? k_conv_row<32> : k_conv_row<64>;
        const size_t rsmem = (size_t)kTStages * (kRABytes + 3 * (size_t)(bn / 8) * kTAtom) + kTAtom;
        MP_CUDA(cudaFuncSetAttribute(rkern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kTStages * (kRABytes + 3 * (kRMaxN / 8) * kTAtom) + kTAtom)));
        dim3 grid(a.V / kTM, (N + kTMaxN - 1) / kTMaxN, B);
        rkern<<<grid, kTThreads, rsmem, (cudaStream_t)stream>>>(a);
        MP_CUDA(cudaGetLastError());
        return MP_OK;
    }
    // the ring plus room to align it to a 1024-byte boundary
    const size_t smem = (size_t)kTStages * (kTABytes + (size_t)(bn / 8) * kTAtom) + kTAtom;
    // instances with the input-channel count fixed at compile time for the network's layers
    void (*kern)(const ConvArgs) = K == 16   ? k_conv_tc<16>
                                   : K == 32 ? k_conv_tc<32>
                                   : K == 64 ? k_conv_tc<64>
                                   : K == 96 ? k_conv_tc<96>
                                   : K == 128 ? k_conv_tc<128>
                                               : k_conv_tc<0>;
    MP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kTStages * (kTABytes + (kTMaxN / 8) * kTAtom) + kTAtom)));
    dim3 grid((a.V + kTM - 1) / kTM, (N + kTMaxN - 1) / kTMaxN, B);
    kern<<<grid, kTThreads, smem, (cudaStream_t)stream>>>(a);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_check(void* stream)
{
    clear_error();
    int h = 0;
    MP_CUDA(cudaMemcpyFromSymbolAsync(&h, g_sg_tc_fail, sizeof(int), 0, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    MP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (h) {
        const int zero = 0;
        MP_CUDA(cudaMemcpyToSymbolAsync(g_sg_tc_fail, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, (cudaStream_t)stream));
        MP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        set_error("sg_check: a bounded wait of the tensor-core convolution gave up (its output is not valid)");
        return MP_ETIMEOUT;
    }
    return MP_OK;
}

int sg_conv3d_wgrad(const void* x, const void* dy, float* dw, float* dbias, int B, int D, int H, int W, int Cin,
                    int Cout, void* stream)
{
    clear_error();
    if (!x || !dy || !dw || B < 1 || D < 1 || H < 1 || W < 1 || Cin < 16 || Cout < 16 || Cin % 16 || Cout % 16) {
        set_error("sg_conv3d_wgrad: needs x, dy, dw, positive sizes, Cin and Cout multiples of 16");
        return MP_EINVAL;
    }
    const int ci_tiles = (Cin + kWM - 1) / kWM, co_tiles = (Cout + kWN - 1) / kWN;
    WgradArgs a{(const bf16*)x, (const bf16*)dy, dw, D, H, W, D * H * W, Cin, Cout, (long long)B * D * H * W, 2048,
                ci_tiles};
    const long long nchunk = (a.total + a.chunk - 1) / a.chunk;
    if (nchunk * 27 > 2147483647LL || ci_tiles * co_tiles > 65535) {
        set_error("sg_conv3d_wgrad: too many voxels or channels");
        return MP_EINVAL;
    }
    dim3 grid((unsigned)(nchunk * 27), (unsigned)(ci_tiles * co_tiles));
    k_wgrad<<<grid, kWThreads, 0, (cudaStream_t)stream>>>(a);
    MP_CUDA(cudaGetLastError());
    if (dbias) {
        dim3 gb(grid1(a.total, 256), (Cout + 31) / 32);
        k_bias_grad<<<gb, 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, dbias, a.total, Cout);
        MP_CUDA(cudaGetLastError());
    }
    return MP_OK;
}

int sg_pool2(const void* x, void* y, int B, int D, int H, int W, int C, void* stream)
{
    clear_error();
    if (!x || !y || B < 1 || D < 2 || H < 2 || W < 2 || (D | H | W) & 1 || C < 2 || C & 1) {
        set_error("sg_pool2: needs even D, H, W and an even channel count");
        return MP_EINVAL;
    }
    const long long n = (long long)B * (D / 2) * (H / 2) * (W / 2) * (C / 2);
    k_pool2<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y, B, D, H, W, C);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_pool2_grad(const void* dy, void* dx, int B, int D, int H, int W, int C, void* stream)
{
    clear_error();
    if (!dy || !dx || B < 1 || D < 2 || H < 2 || W < 2 || (D | H | W) & 1 || C < 2 || C & 1) {
        set_error("sg_pool2_grad: needs even D, H, W and an even channel count");
        return MP_EINVAL;
    }
    const long long n = (long long)B * D * H * W * (C / 2);
    k_fine_from_coarse<true><<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, (bf16*)dx, B, D / 2,
                                                                               H / 2, W / 2, C);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_up2(const void* x, void* y, int B, int D, int H, int W, int C, void* stream)
{
    clear_error();
    if (!x || !y || B < 1 || D < 1 || H < 1 || W < 1 || C < 2 || C & 1) {
        set_error("sg_up2: needs positive sizes and an even channel count");
        return MP_EINVAL;
    }
    const long long n = (long long)B * 8 * D * H * W * (C / 2);
    k_fine_from_coarse<false><<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)x, (bf16*)y, B, D, H, W,
                                                                                C);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_up2_grad(const void* dy, void* dx, int B, int D, int H, int W, int C, void* stream)
{
    clear_error();
    if (!dy || !dx || B < 1 || D < 1 || H < 1 || W < 1 || C < 2 || C & 1) {
        set_error("sg_up2_grad: needs positive sizes and an even channel count");
        return MP_EINVAL;
    }
    const long long n = (long long)B * D * H * W * (C / 2);
    k_up2_grad<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)dy, (bf16*)dx, B, D, H, W, C);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_add(const void* a, const void* b, void* y, int64_t n, void* stream)
{
    clear_error();
    if (!a || !b || !y || n < 0) {
        set_error("sg_add: NULL pointer or negative count");
        return MP_EINVAL;
    }
    if (n == 0) return MP_OK;
    k_add<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)a, (const bf16*)b, (bf16*)y, n);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_relu_grad(const void* act, void* g, int64_t n, void* stream)
{
    clear_error();
    if (!act || !g || n < 0) {
        set_error("sg_relu_grad: NULL pointer or negative count");
        return MP_EINVAL;
    }
    if (n == 0) return MP_OK;
    k_relu_grad<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>((const bf16*)act, (bf16*)g, n);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_pack_input(const uint8_t* cls, void* x, int nx, int ny, int nz, int axis, void* stream)
{
    clear_error();
    if (!cls || !x || nx < 1 || ny < 1 || nz < 1 || axis < 0 || axis > 2) {
        set_error("sg_pack_input: bad arguments");
        return MP_EINVAL;
    }
    const int N = nx * ny * nz;
    k_pack_input<<<grid1(N, 256), 256, 0, (cudaStream_t)stream>>>(cls, (bf16*)x, nx, ny, nz, axis);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_unpack_output(const float* y, int ldy, const uint8_t* cls, float* u, float* rho, int nx, int ny, int nz,
                     int axis, float scale_u, float scale_rho, void* stream)
{
    clear_error();
    if (!y || !cls || !u || ldy < (rho ? 4 : 3) || nx < 1 || ny < 1 || nz < 1 || axis < 0 || axis > 2) {
        set_error("sg_unpack_output: bad arguments");
        return MP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int N = nx * ny * nz;
    double* acc = nullptr;
    if (rho) {
        MP_CUDA(cudaMallocAsync((void**)&acc, 2 * sizeof(double), s));
        cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
        if (e == cudaSuccess) {
            k_cluster_mean<<<grid1(N, 256), 256, 0, s>>>(y, ldy, cls, nx, ny, nz, axis, acc);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            cudaFreeAsync(acc, s);
            return cuda_fail(e, "sg_unpack_output");
        }
    }
    k_unpack_output<<<grid1(N, 256), 256, 0, s>>>(y, ldy, cls, u, rho, nx, ny, nz, axis, scale_u, scale_rho, acc);
    cudaError_t e = cudaGetLastError();
    if (acc) cudaFreeAsync(acc, s);
    if (e != cudaSuccess) return cuda_fail(e, "sg_unpack_output");
    return MP_OK;
}

int sg_pack_target(const float* u, const float* rho, float* t, int nx, int ny, int nz, int axis, float scale_u,
                   float scale_rho, void* stream)
{
    clear_error();
    if (!u || !rho || !t || nx < 1 || ny < 1 || nz < 1 || axis < 0 || axis > 2) {
        set_error("sg_pack_target: bad arguments");
        return MP_EINVAL;
    }
    const int N = nx * ny * nz;
    k_pack_target<<<grid1(N, 256), 256, 0, (cudaStream_t)stream>>>(u, rho, t, nx, ny, nz, axis, scale_u, scale_rho);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_mse(const float* y, int ldy, const float* t, int nc, const void* x, void* dy, double* loss, int B, int V,
           double n_fluid, void* stream)
{
    clear_error();
    if (!y || !t || !x || !dy || !loss || nc < 1 || nc > ldy || B < 1 || V < 1 || !(n_fluid > 0.0)) {
        set_error("sg_mse: bad arguments");
        return MP_EINVAL;
    }
    const long long total = (long long)B * V;
    k_mse<<<grid1(total, 256), 256, 0, (cudaStream_t)stream>>>(y, ldy, t, nc, (const bf16*)x, (bf16*)dy, loss, total,
                                                                1.0 / (nc * n_fluid));
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

int sg_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps, int t,
            void* wf, void* wb, int cin, int cout, void* stream)
{
    clear_error();
    if (!p || !g || !m || !v || n < 0 || t < 1 || ((wf != nullptr) != (wb != nullptr)) ||
        (wf && (cin < 1 || cout < 1 || n != 27LL * cin * cout))) {
        set_error("sg_adam: bad arguments (weights need n = 27 cin cout and both copies)");
        return MP_EINVAL;
    }
    if (n == 0) return MP_OK;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_adam<<<grid1(n, 256), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2, (bf16*)wf,
                                                             (bf16*)wb, cin, cout);
    MP_CUDA(cudaGetLastError());
    return MP_OK;
}

}  // extern "C"
