// ls_dfloat.cuh -- double-float arithmetic: FP64-class accuracy on the FP32 pipes.
//
// GB300 runs FP64 at about 1/64 of its FP32 rate, so the FP64 FFT convolutions of the
// mixed-precision solve (its refinement residuals f - H u and the incident right-hand
// sides f = -w^2 G (m u_I), Sec. 2) were bound by the FP64 pipe.  A double-float value
// is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2: about 48
// significant bits, FP32's exponent range.  Its operations are built from the error-free
// transformations of floating-point arithmetic:
//   * TwoSum (Knuth): s = fl(a + b) and the exact error e, a + b = s + e, for any a, b;
//   * Fast2Sum (Dekker): the same in three operations when |a| >= |b|;
//   * TwoProduct by FMA: p = fl(a b), e = fma(a, b, -p) exact, a b = p + e.
// Sums follow Dekker's add (TwoSum of the high parts, the low parts added into the error,
// renormalised by Fast2Sum): its error is a small multiple of u^2 (|a| + |b|), u = 2^-24,
// which is the normwise bound an FFT needs (its error analysis is normwise anyway).
// Products keep hi*hi exactly and the two cross terms, dropping lo*lo (below u^2 |a b|).
// Every FP32 operation is an explicit round-to-nearest intrinsic, which the compiler
// neither contracts into an FMA nor reorders: the transformations are exact only as
// written.
#pragma once

#include "ls_internal.cuh"

struct __align__(8) dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    // from a double: hi its FP32 rounding, lo the rounding of the (exact) remainder.
    // Used for compile-time constants (folded) and on the host.
    __host__ __device__ explicit dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};
struct __align__(16) cdfl {
    dfl x, y;
};

template <> struct cpx<dfl> { using type = cdfl; };
template <> struct real_of<cdfl> { using type = dfl; };
__host__ __device__ __forceinline__ cdfl mkc(dfl a, dfl b) { return cdfl{a, b}; }
template <> __host__ __device__ __forceinline__ cdfl czero<cdfl>() { return cdfl{dfl(0.f, 0.f), dfl(0.f, 0.f)}; }

#ifdef __CUDACC__
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfl(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const dfl s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
// a b + c d with one renormalisation (the complex product's components)
__device__ __forceinline__ dfl df_dot2(dfl a, dfl b, dfl c, dfl d) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float q = __fmul_rn(c.hi, d.hi);
    const dfl s = df_two_sum(p, q);
    float e = __fadd_rn(__fmaf_rn(a.hi, b.hi, -p), __fmaf_rn(c.hi, d.hi, -q));
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(c.hi, d.lo, e);
    e = __fmaf_rn(c.lo, d.hi, e);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, e));
}

__device__ __forceinline__ cdfl operator+(cdfl a, cdfl b) { return cdfl{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdfl operator-(cdfl a, cdfl b) { return cdfl{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdfl operator-(cdfl a) { return cdfl{-a.x, -a.y}; }
__device__ __forceinline__ cdfl operator*(cdfl a, cdfl b) {
    return cdfl{df_dot2(a.x, b.x, -a.y, b.y), df_dot2(a.x, b.y, a.y, b.x)};
}
__device__ __forceinline__ cdfl operator*(dfl s, cdfl a) { return cdfl{s * a.x, s * a.y}; }

// double <-> double-float on the integer pipes (d2f_rn, f2d) plus one FP64 operation:
// the remainder x - hi is exact in FP64, so lo is its FP32 rounding.
__host__ __device__ __forceinline__ dfl dfl_of(double x) {
    const float h = d2f_rn(x);
    return dfl(h, d2f_rn(x - f2d(h)));
}
__host__ __device__ __forceinline__ double dbl_of(dfl a) { return f2d(a.hi) + f2d(a.lo); }

template <> __host__ __device__ __forceinline__ cdfl ccast<cdfl, double2>(double2 a) { return cdfl{dfl_of(a.x), dfl_of(a.y)}; }
template <> __host__ __device__ __forceinline__ double2 ccast<double2, cdfl>(cdfl a) {
    return make_double2(dbl_of(a.x), dbl_of(a.y));
}
template <> __host__ __device__ __forceinline__ cdfl ccast<cdfl, cdfl>(cdfl a) { return a; }

// read-only loads of complex values (one 16-byte load for a double-float complex)
template <typename C> __device__ __forceinline__ C ldg_c(const C* p) { return __ldg(p); }
template <> __device__ __forceinline__ cdfl ldg_c<cdfl>(const cdfl* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return cdfl{dfl(v.x, v.y), dfl(v.z, v.w)};
}
#endif
