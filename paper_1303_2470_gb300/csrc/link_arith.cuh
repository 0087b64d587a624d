// link_arith.cuh -- the correctly rounded link-probability arithmetic shared by the MP
// kernels. A link probability is evaluated at both end nodes of its link; these functions
// fix the sequence of roundings so that both ends obtain the same bits.
#pragma once

#include "internal.cuh"

namespace mp {

// Correctly rounded arithmetic the compiler may not contract or reorder. A link
// probability is evaluated by both end nodes of the link and must come out bitwise equal,
// so that the two ends compute exactly opposite net fluxes.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// e = c_i . u: a signed sum of one or two components, added in x, y, z order
template <typename T>
__device__ __forceinline__ T edot(int i, T ux, T uy, T uz)
{
    T e = T(0);
    bool first = true;
    if (cx(i) != 0) {
        e = cx(i) > 0 ? ux : -ux;
        first = false;
    }
    if (cy(i) != 0) {
        const T v = cy(i) > 0 ? uy : -uy;
        e = first ? v : rn_add(e, v);
        first = false;
    }
    if (cz(i) != 0) {
        const T v = cz(i) > 0 ? uz : -uz;
        e = first ? v : rn_add(e, v);
    }
    return e;
}

// flow-dependent part of p_i / w_i: q = e (3 + 9/2 e) - 3/2 |u|^2 (a = -3/2 |u|^2 stored)
template <typename T>
__device__ __forceinline__ T qlink(T e, T a)
{
    return rn_fma(e, rn_fma(T(4.5), e, T(3)), a);
}

}  // namespace mp
