// surrogate.cu -- kernels of the learned warm start for lb_steady (include/surrogate.h): 3x3x3
// periodic convolutions as implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation), their input and weight gradients, pooling, upsampling,
// the masked loss and the Adam update. Nothing here belongs to the moment-propagation
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

// four 8x8 BF16 matrices from shared memory (lanes 8j..8j+7 give the row addresses of
// matrix j): each lane receives (M[l/4][2(l%4)], M[l/4][2(l%4)+1]) of every matrix, which is
// the m16n8k16 fragment layout of A (row-major) and of B stored as [n][k]
__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3, const bf16* p)
{
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}

// Forward (and transposed) convolution tile: BM = 128 MT voxels x BN = 8 NT output channels
// per block of 8 warps (warp w: voxels 16 MT w .. 16 MT (w + 1) - 1, all NT column tiles),
// reduction over the 27 taps and the input channels in stages of 32 (two m16n8k16 steps).
// Two shapes: 128 x 64 (MT = 1, NT = 8) for N > 32 and 256 x 32 (MT = 2, NT = 4) for
// N <= 32, so that the full-resolution 32-channel layers fill their tiles and each B
// fragment feeds two products. The next stage's operands are loaded into registers while the
// current one is multiplied, then stored to the other shared buffer: one barrier per stage.
// Shared rows hold 40 BF16 (80 bytes), so the eight 16-byte rows of an ldmatrix phase, and
// the staging stores of eight consecutive rows, fall on distinct banks.
constexpr int kCS = 32, kCLd = 40, kCThreads = 256;

template <int MT, int NT>
__device__ __forceinline__ void conv_stage_mma(const bf16 (*As)[kCLd], const bf16 (*Bs)[kCLd],
                                               float (&acc)[MT][NT][4], int ncols)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m0 = warp * 16 * MT;
    // A: matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15), (rows 8-15, k 8-15)
    const int ar = (lane & 7) + ((lane >> 3) & 1) * 8, ac = (lane >> 4) * 8;
    // B ([n][k]): matrices (tile nt, k 0-7), (nt, k 8-15), (nt + 1, k 0-7), (nt + 1, k 8-15)
    const int br = (lane & 7) + (lane >> 4) * 8, bc = ((lane >> 3) & 1) * 8;
#pragma unroll
    for (int kk = 0; kk < kCS; kk += 16) {
        uint32_t af[MT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
            ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &As[m0 + mt * 16 + ar][kk + ac]);
#pragma unroll
        for (int nt = 0; nt < NT; nt += 2) {
            if (nt * 8 < ncols) {  // ncols is a multiple of 16: both tiles of the pair or neither
                uint32_t b0, b1, b2, b3;
                ldsm_x4(b0, b1, b2, b3, &Bs[nt * 8 + br][kk + bc]);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    mma16816(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
                    mma16816(acc[mt][nt + 1], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b2, b3);
                }
            }
        }
    }
}

template <int MT, int NT>
__global__ void __launch_bounds__(kCThreads) k_conv(const ConvArgs a)
{
    constexpr int BM = 128 * MT, BN = 8 * NT;
    constexpr int AP = 2 * BM / kCThreads;  // A pieces (16 channels of one voxel) per thread
    static_assert(AP * kCThreads == 2 * BM && BN * 4 <= kCThreads, "staging shape");
    __shared__ __align__(16) bf16 As[2][BM][kCLd];
    __shared__ __align__(16) bf16 Bs[2][BN][kCLd];
    const int tid = threadIdx.x;
    const int v0 = blockIdx.x * BM, n0 = blockIdx.y * BN, b = blockIdx.z;
    // A piece p = tid + 256 i: voxel row p % BM, channels 16 (p / BM) .. +15 of the stage;
    // B: column row tid % BN, channels 8 (tid / BN) .. +7 (threads below 4 BN)
    int ar[AP], ah[AP], xa[AP], ya[AP], za[AP];
    bool vok[AP];
#pragma unroll
    for (int i = 0; i < AP; ++i) {
        const int p = tid + kCThreads * i;
        ar[i] = p % BM;
        ah[i] = (p / BM) * 16;
        const int va = v0 + ar[i];
        vok[i] = va < a.V;
        xa[i] = ya[i] = za[i] = 0;
        if (vok[i]) {
            xa[i] = va % a.W;
            ya[i] = (va / a.W) % a.H;
            za[i] = va / (a.W * a.H);
        }
    }
    const bool bthr = tid < BN * 4;
    const int br = tid % BN, bq = (tid / BN) * 8;
    const bool nok = bthr && n0 + br < a.N;
    const bf16* xb = a.x + (size_t)b * a.V * a.K;
    const int ncols = a.N - n0 < BN ? a.N - n0 : BN;
    const int cstages = (a.K + kCS - 1) / kCS;  // channel stages per tap (K is a multiple of 16)
    const int nst = 27 * cstages;
    uint4 ra[AP][2], rb;
    // global -> registers for stage st (zero outside the box of channels, voxels, columns)
    auto fetch = [&](int st) {
        const int tap = st / cstages, c0 = (st - tap * cstages) * kCS;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int i = 0; i < AP; ++i) {
            ra[i][0] = ra[i][1] = make_uint4(0u, 0u, 0u, 0u);
            if (vok[i] && c0 + ah[i] < a.K) {
                const int xs = wrap(xa[i] + a.sign * dx, a.W), ys = wrap(ya[i] + a.sign * dy, a.H);
                const int zs = wrap(za[i] + a.sign * dz, a.D);
                const bf16* p = xb + ((size_t)(zs * a.H + ys) * a.W + xs) * a.K + c0 + ah[i];
                ra[i][0] = *reinterpret_cast<const uint4*>(p);
                ra[i][1] = *reinterpret_cast<const uint4*>(p + 8);
            }
        }
        rb = make_uint4(0u, 0u, 0u, 0u);
        if (nok && c0 + bq < a.K) rb = *reinterpret_cast<const uint4*>(a.w + ((size_t)tap * a.N + n0 + br) * a.K + c0 + bq);
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int i = 0; i < AP; ++i) {
            *reinterpret_cast<uint4*>(&As[buf][ar[i]][ah[i]]) = ra[i][0];
            *reinterpret_cast<uint4*>(&As[buf][ar[i]][ah[i] + 8]) = ra[i][1];
        }
        if (bthr) *reinterpret_cast<uint4*>(&Bs[buf][br][bq]) = rb;
    };
    float acc[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int i = 0; i < NT; ++i) acc[mt][i][0] = acc[mt][i][1] = acc[mt][i][2] = acc[mt][i][3] = 0.0f;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int st = 0; st < nst; ++st) {
        const int cur = st & 1;
        if (st + 1 < nst) fetch(st + 1);
        conv_stage_mma<MT, NT>(As[cur], Bs[cur], acc, ncols);
        if (st + 1 < nst) stash(cur ^ 1);
        __syncthreads();
    }
    const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int col = n0 + nt * 8 + 2 * t;
        if (col >= a.N) continue;
        const float b0 = a.bias ? a.bias[col] : 0.0f, b1 = a.bias ? a.bias[col + 1] : 0.0f;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int v = v0 + warp * 16 * MT + mt * 16 + g + 8 * h;
                if (v >= a.V) continue;
                float r0 = acc[mt][nt][2 * h] + b0, r1 = acc[mt][nt][2 * h + 1] + b1;
                if (a.relu) {
                    r0 = fmaxf(r0, 0.0f);
                    r1 = fmaxf(r1, 0.0f);
                }
                const size_t o = ((size_t)b * a.V + v) * a.N + col;
                if (a.y) *reinterpret_cast<__nv_bfloat162*>(a.y + o) = __floats2bfloat162_rn(r0, r1);
                if (a.yf) {
                    a.yf[o] = r0;
                    a.yf[o + 1] = r1;
                }
            }
        }
    }
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
    if (N <= 32) {
        dim3 grid((a.V + 255) / 256, 1, B);
        k_conv<2, 4><<<grid, kCThreads, 0, (cudaStream_t)stream>>>(a);
    } else {
        dim3 grid((a.V + 127) / 128, (N + 63) / 64, B);
        k_conv<1, 8><<<grid, kCThreads, 0, (cudaStream_t)stream>>>(a);
    }
    MP_CUDA(cudaGetLastError());
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
