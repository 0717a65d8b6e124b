// ls_fft_common.cuh -- pieces shared by the FFT-convolution kernels: the
// in-register DFT of length 2..16, and the pass-1 sources / pass-3 sinks of the
// LS-apply (Sec. 2): D u = m u on the way in, u + (G-term) on the way out.
#pragma once

#include "ls_internal.cuh"

namespace {

// ---------------------------------------------------------------- DFT in registers
template <typename R>
__device__ __forceinline__ R cos16(int i) {  // cos(2 pi i / 16), i in [0, 8]
    return i == 0 ? R(1) : i == 1 ? R(0.92387953251128675613) : i == 2 ? R(0.70710678118654752440)
         : i == 3 ? R(0.38268343236508977173) : i == 4 ? R(0) : i == 5 ? R(-0.38268343236508977173)
         : i == 6 ? R(-0.70710678118654752440) : i == 7 ? R(-0.92387953251128675613) : R(-1);
}

// d * exp(-DIR * 2 pi i idx / 16); idx is a compile-time constant after unrolling.
template <int DIR, typename C>
__device__ __forceinline__ C rot16(C d, int idx) {
    using R = typename real_of<C>::type;
    if (idx == 0) return d;
    if (idx == 4) return DIR > 0 ? mkc(d.y, -d.x) : mkc(-d.y, d.x);
    const R c = cos16<R>(idx);
    const R s = cos16<R>(idx <= 4 ? 4 - idx : idx - 4);  // sin(2 pi idx / 16) for idx in [0, 8)
    if (DIR > 0) return mkc(d.x * c + d.y * s, d.y * c - d.x * s);
    return mkc(d.x * c - d.y * s, d.y * c + d.x * s);
}

template <int R>
__host__ __device__ constexpr int brev(int k) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((k & b) ? 1 : 0);
    return r;
}
template <int R>
__host__ __device__ constexpr int ilog2c() {
    return R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
}

// Natural-order DFT of length R (2, 4, 8, 16): radix-2 decimation in frequency,
// then the bit-reversal permutation.  DIR = +1: exp(-2 pi i nk/R); -1: conjugate.
// HZ: inputs R/2 .. R-1 are known to be zero (a zero-padded transform), so the
// first layer only rotates.
template <int R, int DIR, bool HZ = false, typename C>
__device__ __forceinline__ void dft_reg(C* v) {
#pragma unroll
    for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
        for (int s = 0; s < R; s += 2 * half) {
#pragma unroll
            for (int k = 0; k < half; ++k) {
                if (HZ && half == R / 2) {
                    v[s + k + half] = rot16<DIR>(v[s + k], k * (16 / (2 * half)));
                    continue;
                }
                const C a = v[s + k], b = v[s + k + half];
                v[s + k] = a + b;
                v[s + k + half] = rot16<DIR>(a - b, k * (16 / (2 * half)));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = brev<R>(k);
        if (r > k) {
            const C t = v[k];
            v[k] = v[r];
            v[r] = t;
        }
    }
}

// ---------------------------------------------------------------- pass-1 sources
template <typename T, typename UIn>
struct SrcMU {  // m u  (Sec. 2: D u)
    const T* m;
    const UIn* u;
    int n;
    template <typename C>
    __device__ __forceinline__ C load(int z, int x) const {
        const size_t i = (size_t)z * n + x;
        return m[i] * hw_cast<C>(__ldg(&u[i]));
    }
};

template <typename T>
struct SrcInc {  // m u_I, u_I = exp(i w x cos) exp(i w z sin)  (Sec. 2: D u_I)
    const T* m;
    const double2* ex;
    const double2* ez;
    int n;
    template <typename C>
    __device__ __forceinline__ C load(int z, int x) const {
        const double2 ui = __ldg(&ex[x]) * __ldg(&ez[z]);
        return m[(size_t)z * n + x] * ccast<C>(ui);
    }
};

struct SrcGpad {  // circulant embedding of G_w on the P x P torus (offsets |d| <= n-1)
    const double2* gtab;  // G_w on [-n, n]^2, row-major by dz
    int n, P;
    template <typename C>
    __device__ __forceinline__ C load(int b, int a) const {
        const int at = a < P / 2 ? a : a - P;
        const int bt = b < P / 2 ? b : b - P;
        if (at > n - 1 || at < -(n - 1) || bt > n - 1 || bt < -(n - 1)) return czero<C>();
        return ccast<C>(gtab[(size_t)(bt + n) * (2 * n + 1) + (at + n)]);
    }
};

// ---------------------------------------------------------------- pass-3 sinks
template <typename UIO>
struct DstApply {  // y = u + (G-term)
    const UIO* u;
    UIO* y;
    int n;
    template <typename C>
    __device__ __forceinline__ void store(int z, int x, C v) const {
        const size_t i = (size_t)z * n + x;
        y[i] = u[i] + hw_cast<UIO>(v);
    }
};

struct DstRhs {  // f = -(G-term)
    double2* f;
    int n;
    template <typename C>
    __device__ __forceinline__ void store(int z, int x, C v) const {
        f[(size_t)z * n + x] = -ccast<double2>(v);
    }
};

}  // namespace
