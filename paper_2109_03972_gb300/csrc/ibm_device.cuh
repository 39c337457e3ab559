// Device helpers shared by the kernels: delta-kernel weights, marker
// positions, reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ibm_internal.h"

#define IBM_PI 3.14159265358979323846

// Three-point regularised delta (Eq. 3pt-stencil).  For a marker with
// fractional position f = xi - floor(xi) in [0, 1), the three cells of its
// stencil, floor(xi) - 1, floor(xi), floor(xi) + 1, sit at offsets
// r = r0 - 1, r0, r0 + 1 with r0 = 1/2 - f, |r0| <= 1/2.  The centre weight
// is phi3(r0) = (1 + s)/3, s = sqrt(1 - 3 r0^2), and partition of unity plus
// the zero first moment of phi3 fix the two outer weights:
//   phi3(r0 - 1) = (2 + 3 r0 - s)/6,  phi3(r0 + 1) = (2 - 3 r0 - s)/6,
// which is what Eq. (3pt-stencil) gives on its outer branch.  One square root
// per axis instead of three.
template <typename T>
__device__ __forceinline__ void phi3_weights(T f, T w[3]) {
    const T r0 = T(0.5) - f;
    const T s = sqrt(T(1) - T(3) * r0 * r0);
    w[1] = (T(1) + s) * T(1.0 / 3.0);
    w[0] = (T(2) + T(3) * r0 - s) * T(1.0 / 6.0);
    w[2] = (T(2) - T(3) * r0 - s) * T(1.0 / 6.0);
}

__device__ __forceinline__ void phi3_weights(float f, float w[3]) {
    const float r0 = 0.5f - f;
    const float s = sqrtf(fmaf(-3.0f * r0, r0, 1.0f));
    w[1] = (1.0f + s) * (1.0f / 3.0f);
    w[0] = (2.0f + 3.0f * r0 - s) * (1.0f / 6.0f);
    w[2] = (2.0f - 3.0f * r0 - s) * (1.0f / 6.0f);
}

// Derivatives of the three weights with respect to the marker position xi
// (grid units), from the same closed form: with r0 = (base + 1/2) - xi,
//   d/dxi phi3(r0)     =  r0 / s
//   d/dxi phi3(r0 - 1) = -(1 + r0/s)/2
//   d/dxi phi3(r0 + 1) =  (1 - r0/s)/2
template <typename T>
__device__ __forceinline__ void phi3_dweights(T f, T dw[3]) {
    const T r0 = T(0.5) - f;
    const T s = sqrt(T(1) - T(3) * r0 * r0);
    const T q = r0 / s;
    dw[1] = q;
    dw[0] = -(T(1) + q) * T(0.5);
    dw[2] = (T(1) - q) * T(0.5);
}

// Four-point regularised delta (Sec. 2.2.3, the |r| form: the first branch
// for |r| <= 1, the second for 1 <= |r| <= 2).  Its stencil starts one cell
// below b = floor(xi - 1/2); with g = (xi - 1/2) - b in [0, 1) the four cells
// sit at r = -1 - g, -g, 1 - g, 2 - g, and the radicands of both branches at
// these offsets are the same number 1 + 4g - 4g^2, so
//   phi4(-1-g) = (3 - 2g - q)/8,  phi4(-g)  = (3 - 2g + q)/8,
//   phi4(1-g)  = (1 + 2g + q)/8,  phi4(2-g) = (1 + 2g - q)/8,
// q = sqrt(1 + 4g - 4g^2): one square root per axis, and the four weights
// sum to 1 by construction.
template <typename T>
__device__ __forceinline__ void phi4_weights(T g, T w[4]) {
    const T q = sqrt(T(1) + T(4) * g - T(4) * g * g);
    w[0] = (T(3) - T(2) * g - q) * T(0.125);
    w[1] = (T(3) - T(2) * g + q) * T(0.125);
    w[2] = (T(1) + T(2) * g + q) * T(0.125);
    w[3] = (T(1) + T(2) * g - q) * T(0.125);
}

__device__ __forceinline__ int wrapi(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

// i modulo n for 0 <= i < 3n, without a division.
__device__ __forceinline__ int wrap_lt3(int i, int n) {
    if (i >= n) i -= n;
    if (i >= n) i -= n;
    return i;
}

// Marker position in grid units, FP64, rounded exactly as
// xi = x_p/h + ((d_p/2)/h) * t  (multiply, then add; no fused multiply-add).
__device__ __forceinline__ double marker_xi64(const PInfo &P, const double *t, int c) {
    return __dadd_rn(P.xi[c], __dmul_rn(P.a, t[c]));
}

// FP32 marker position relative to the particle's base cell.  Returns the base
// cell offset (int) and the fraction in [0,1).  When the FP32 value lies within
// the FP32 error bound of a cell face, the coordinate is recomputed in FP64 so
// that the stencil base cell is exactly floor(xi) of the FP64 position.
__device__ __forceinline__ int marker_split32(const PInfo &P, const float *t32, const double *t64,
                                              int c, float *frac) {
    float s = fmaf(P.af, t32[c], P.fracf[c]);
    float fl = floorf(s);
    float fr = s - fl;
    const float tol = 8.0f * 5.9604645e-8f * (P.af + 2.0f);
    if (fr < tol || fr > 1.0f - tol) {
        double xi = marker_xi64(P, t64, c);
        double fb = floor(xi);
        *frac = (float)(xi - fb);
        return (int)fb;
    }
    *frac = fr;
    return P.base[c] + (int)fl;
}

// FP32 split of xi - 1/2 (the four-point kernel's base and fraction), from
// the three-point split of xi; within the FP32 error bound of a half-integer
// the coordinate is recomputed in FP64, so the base is exactly floor(xi - 1/2)
// of the FP64 position.
__device__ __forceinline__ int marker_split32_half(const PInfo &P, const float *t32, const double *t64, int c,
                                                   float *g) {
    float f;
    const int b = marker_split32(P, t32, t64, c, &f);
    const float tol = 8.0f * 5.9604645e-8f * (P.af + 2.0f);
    if (fabsf(f - 0.5f) < tol) {
        const double xh = marker_xi64(P, t64, c) - 0.5;
        const double fb = floor(xh);
        *g = (float)(xh - fb);
        return (int)fb;
    }
    if (f >= 0.5f) {
        *g = f - 0.5f;
        return b;
    }
    *g = f + 0.5f;
    return b - 1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void set_err(int *err, int bit) { atomicOr(err, bit); }

// atomic max for non-negative doubles (bit pattern is monotone)
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}
