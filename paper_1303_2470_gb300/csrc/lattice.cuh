// lattice.cuh -- small device helpers shared by the moment-propagation kernels of libmp
// (not part of the C ABI): the packed flow vector, exact division by a lattice extent,
// periodic neighbour offsets, fluid-list indices of link sources, vector records of the
// propagated fields and warp sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace mp {

// (u_x, u_y, u_z, -3/2 |u|^2) of one node, loaded as one vector
template <typename T>
struct alignas(4 * sizeof(T)) Flow4 {
    T x, y, z, w;
};

// exact quotient n / d for 0 <= n < 2^31, 2 <= d < 2^31, with m = floor(2^32 / d): the
// estimate umulhi(n, m) is floor(n/d) or one less
struct Div {
    unsigned d, m;
};
inline Div make_div(unsigned d) { return Div{d, (unsigned)((1ull << 32) / d)}; }
__device__ __forceinline__ unsigned divq(unsigned n, Div v)
{
    unsigned q = __umulhi(n, v.m);
    if (n - q * v.d >= v.d) ++q;
    return q;
}

// all propagated fields of one node and species, stored together (padded to 2 or 4)
template <typename T, int FP>
struct alignas(FP * sizeof(T)) FieldVec {
    T v[FP];
};

// 32-byte records of eight FP32 values move as one 256-bit access (ld/st.global.v8.f32):
// with records scattered over the fluid list, two 16-byte halves would each cost a full
// L1 sector request per lane
template <typename T, int W>
__device__ __forceinline__ FieldVec<T, W> ld_rec(const FieldVec<T, W>* p)
{
    return *p;
}
template <>
__device__ __forceinline__ FieldVec<float, 8> ld_rec<float, 8>(const FieldVec<float, 8>* p)
{
    FieldVec<float, 8> r;
    asm("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
          "=f"(r.v[7])
        : "l"(p));
    return r;
}
template <typename T, int W>
__device__ __forceinline__ void st_rec(FieldVec<T, W>* p, const FieldVec<T, W>& r)
{
    *p = r;
}
template <>
__device__ __forceinline__ void st_rec<float, 8>(FieldVec<float, 8>* p, const FieldVec<float, 8>& r)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(r.v[0]), "f"(r.v[1]), "f"(r.v[2]),
                 "f"(r.v[3]), "f"(r.v[4]), "f"(r.v[5]), "f"(r.v[6]), "f"(r.v[7])
                 : "memory");
}

// Periodic neighbourhood of a node: offsets to x-1, x+1, y-1, y+1, z-1, z+1.
struct Nbr {
    int n, oxm, oxp, oym, oyp, ozm, ozp;
};

// dx, dxy: division by nx and by nx*ny
__device__ __forceinline__ Nbr nbrs_of(int nx, int ny, int nz, Div dx, Div dxy, int n)
{
    Nbr b;
    const int yz = (int)divq((unsigned)n, dx);
    const int x = n - yz * nx;
    const int z = (int)divq((unsigned)n, dxy);
    const int y = yz - z * ny;
    const int nxy = nx * ny;
    b.n = n;
    b.oxm = x == 0 ? nx - 1 : -1;
    b.oxp = x == nx - 1 ? 1 - nx : 1;
    b.oym = y == 0 ? (ny - 1) * nx : -nx;
    b.oyp = y == ny - 1 ? (1 - ny) * nx : nx;
    b.ozm = z == 0 ? (nz - 1) * nxy : -nxy;
    b.ozp = z == nz - 1 ? (1 - nz) * nxy : nxy;
    return b;
}

// s_i = r - c_i
__device__ __forceinline__ int src_of(const Nbr& b, int i)
{
    return b.n + (cx(i) > 0 ? b.oxm : (cx(i) < 0 ? b.oxp : 0)) + (cy(i) > 0 ? b.oym : (cy(i) < 0 ? b.oyp : 0)) +
           (cz(i) > 0 ? b.ozm : (cz(i) < 0 ? b.ozp : 0));
}

// Index of fluid node s in the sorted fluid list: fluid nodes before its 32-node word plus
// those below it within the word.
__device__ __forceinline__ int fluid_index(const uint2* __restrict__ fw, int s)
{
    const uint2 w = __ldg(fw + (s >> 5));
    return (int)w.y + __popc(w.x & ((1u << (s & 31)) - 1u));
}

// The sources r - c_i lie in nine lattice rows (fixed y and z) around r: r's own row
// (links 1, 2) and eight others, row j holding the source of link row_centre(j) (c_x = 0)
// and, for four of them, the sources at x - 1 (link with c_x = +1) and x + 1 (c_x = -1).
// Fluid nodes of a row are consecutive in the fluid list, so one located centre per row
// gives the indices of its x - 1 and x + 1 neighbours.
__host__ __device__ constexpr int row_of(int i)
{
    constexpr int t[kQ] = {-1, -1, -1, 0, 1, 0, 1, 1, 0, 2, 2, 2, 4, 5, 3, 3, 3, 6, 7};
    return t[i];
}
__host__ __device__ constexpr int row_centre(int j)
{
    constexpr int t[8] = {3, 4, 9, 14, 12, 13, 17, 18};
    return t[j];
}

// Fluid-list index of the source r - c_i of an open link i of fluid node r (index k, its
// periodic neighbourhood b, open-link mask `mask`, C[j] = fluid_index of row j's centre,
// xlo / xhi: x - 1 / x + 1 lie in r's row without wrapping): the row's centre, or its x -/+ 1
// neighbour (own row: k -/+ 1); located directly where x - 1 or x + 1 wraps around.
__device__ __forceinline__ int source_index(int i, int k, const int (&C)[8], uint32_t mask, bool xlo, bool xhi,
                                            const Nbr& b, const uint2* __restrict__ fw)
{
    const int row = row_of(i);
    const int base = row < 0 ? k : C[row < 0 ? 0 : row];
    if (cx(i) == 0) return base;
    if (cx(i) > 0) return xlo ? base - 1 : fluid_index(fw, src_of(b, i));
    return xhi ? base + (row < 0 ? 1 : (int)((mask >> (row_centre(row < 0 ? 0 : row) - 1)) & 1u))
               : fluid_index(fw, src_of(b, i));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mp
