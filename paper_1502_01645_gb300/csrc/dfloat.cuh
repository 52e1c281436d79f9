// Double-float scalars: normalised FP32 pairs for the step scalars of the
// FP32 Alg. 2 kernels, and the same interface over FP64 for the FP64 ones.
#pragma once

#include <cuda_runtime.h>

namespace aln {

// Scalars of the step (γ, κ and their sums) in the FP32 kernel: normalised
// FP32 pairs hi + lo (|lo| ≤ ulp(hi)/2, about 48 significant bits), added
// with TwoSum (Knuth) and renormalised with Fast2Sum (Dekker), in the
// accurate form of double-float addition (Hida, Li and Bailey's QD
// library): GB300's FP64 unit is narrow, and the FP32 pipe forms these in a
// few dependent FP32 adds.  The FP64 kernel keeps FP64 scalars.
struct DF {
    float hi, lo;
};
template <typename T> struct ScT;
template <> struct ScT<float> { using type = DF; };
template <> struct ScT<double> { using type = double; };
template <typename T> using Sc = typename ScT<T>::type;

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| ≥ |b|
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF sc_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    const DF t = df_two_sum(a.lo, b.lo);
    s = df_fast_two_sum(s.hi, s.lo + t.hi);
    return df_fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ double sc_add(double a, double b) { return a + b; }
// A scalar from one value of the iteration type (exact).
__device__ __forceinline__ void sc_set(DF& o, float v) { o = DF{v, 0.0f}; }
__device__ __forceinline__ void sc_set(double& o, float v) { o = (double)v; }
__device__ __forceinline__ void sc_set(double& o, double v) { o = v; }
__device__ __forceinline__ DF sc_shfl_xor(DF a, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ double sc_shfl_xor(double a, int o) {
    return __shfl_xor_sync(0xffffffffu, a, o);
}
// Xor-tree warp sum (every lane gets the same value: the addition is
// commutative in both forms).
template <typename S>
__device__ __forceinline__ S sc_warp_sum(S x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = sc_add(x, sc_shfl_xor(x, o));
    return x;
}
// Comparisons of normalised pairs are lexicographic.
__device__ __forceinline__ bool sc_lt(DF a, DF b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool sc_lt(double a, double b) { return a < b; }
__device__ __forceinline__ bool sc_finite(DF a) { return isfinite(a.hi) && isfinite(a.lo); }
__device__ __forceinline__ bool sc_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool sc_nonpos(DF a) { return a.hi <= 0.0f; }
__device__ __forceinline__ bool sc_nonpos(double a) { return a <= 0.0; }
__device__ __forceinline__ bool sc_zero(DF a) { return a.hi == 0.0f; }
__device__ __forceinline__ bool sc_zero(double a) { return a == 0.0; }
__device__ __forceinline__ double sc_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double sc_double(double a) { return a; }
template <typename S> __device__ __forceinline__ S sc_of_double(double x);
template <> __device__ __forceinline__ DF sc_of_double<DF>(double x) {
    const float h = (float)x;
    return DF{h, isfinite(h) ? (float)(x - (double)h) : 0.0f};
}
template <> __device__ __forceinline__ double sc_of_double<double>(double x) { return x; }
template <typename S> __device__ __forceinline__ S sc_inf();
template <> __device__ __forceinline__ DF sc_inf<DF>() { return DF{__int_as_float(0x7f800000), 0.0f}; }
template <> __device__ __forceinline__ double sc_inf<double>() { return 1.0 / 0.0; }
// Scalars through global memory (8 bytes either way), past L1.
__device__ __forceinline__ void sc_stcg(double* p, DF v) {
    __stcg(reinterpret_cast<float2*>(p), make_float2(v.hi, v.lo));
}
__device__ __forceinline__ void sc_stcg(double* p, double v) { __stcg(p, v); }
template <typename S> __device__ __forceinline__ S sc_ldcg(const double* p);
template <> __device__ __forceinline__ DF sc_ldcg<DF>(const double* p) {
    const float2 f = __ldcg(reinterpret_cast<const float2*>(p));
    return DF{f.x, f.y};
}
template <> __device__ __forceinline__ double sc_ldcg<double>(const double* p) { return __ldcg(p); }

// The step quotient in the kernel's scalar type (FP64: the quotient itself).
__device__ __forceinline__ double sc_quot(double a, double b) { return a / b; }
__device__ __forceinline__ float df_quotient(DF a, DF b);
__device__ __forceinline__ float sc_quot(DF a, DF b) { return df_quotient(a, b); }

// a/b in FP32 from pairs: the quotient of the leading parts, corrected once
// with the residual of the pairs (one Newton step of the division), within
// an FP32 ulp or so of the rounded quotient.
__device__ __forceinline__ float df_quotient(DF a, DF b) {
    const float q = __fdiv_rn(a.hi, b.hi);
    const float r = fmaf(-q, b.hi, a.hi) + fmaf(-q, b.lo, a.lo);
    return q + __fdiv_rn(r, b.hi);
}

}  // namespace aln
