// ls_fft.cu -- zero-padded FFT convolution: the LS-apply y = u + w^2 G (m u).
//
// Sec. 2 of the paper: G is translation invariant on the uniform grid, so the
// dense quadrature matrix is a two-level Toeplitz matrix; embedding it in a
// circulant of size P x P (P >= 2n - 1) turns G v into a cyclic convolution,
// applied by FFT in O(N log N).  With Ghat = (w^2/P^2) FFT2(Gpad):
//     H u = u + IFFT2(Ghat .* FFT2(pad(m u)))[0:n, 0:n]        (unnormalised IFFT)
//
// Three HBM passes (the minimum for a 2-D transform that does not fit on chip):
//   pass 1 (rows)    read u, m; form m u; zero-pad to P; FFT along x; write n x P.
//   pass 2 (columns) for a tile of CW columns kx: FFT along z (input zero-padded,
//                    rows >= n skipped), multiply by Ghat(kx, kz) in registers,
//                    inverse FFT along z, keep rows z < n; write n x P in place.
//   pass 3 (rows)    inverse FFT along x, keep x < n, add u; write y.
// Each transform is a Stockham autosort FFT held in shared memory: a thread
// owns E elements of a transform, every stage loads its radix-R butterflies
// into registers, twiddles them, runs an in-register DFT and stores them back.
// The first stage of a transform reads straight from global memory and the
// last stage writes straight to global memory, so each pass touches HBM once.
// Ghat is even in both indices (G_w is even), so only its (P/2+1)^2 quadrant is
// stored and read.
#include <cmath>
#include <mutex>
#include <type_traits>

#include "ls_fft_common.cuh"
#include "ls_dfloat.cuh"

namespace {

// One Stockham stage on the E/R butterflies a thread owns: twiddle by
// exp(-DIR 2 pi i k r / (Ns R)), k = b mod Ns, then the radix-R DFT.
template <int R, int DIR, int E, typename C>
__device__ __forceinline__ void stage_compute(C (&v)[E], int j, int TPC, int ls, int lp,
                                              const C* __restrict__ tw) {
    constexpr int LR = ilog2c<R>();
#pragma unroll
    for (int e = 0; e < E / R; ++e) {
        if (ls > 0) {
            const int b = j + e * TPC;
            const int k = b & ((1 << ls) - 1);
            const int sh = lp - ls - LR;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = ldg_c(&tw[(k * r) << sh]);
                if (DIR < 0) w.y = -w.y;
                v[e * R + r] = v[e * R + r] * w;
            }
        }
        dft_reg<R, DIR>(&v[e * R]);
    }
}

// Shared-memory slot of element idx: one padding slot every 2^PS elements, so that
// the strided stores of the first Stockham stage (stride = radix) and the unit-
// stride loads of the others both hit distinct banks.
template <int PS>
__device__ __forceinline__ int padx(int idx) { return idx + (idx >> PS); }

// A full transform of length P = plan.P.  On entry v holds the first stage's
// inputs (element j + e*TPC + r*P/R0 in v[e*R0 + r]); on exit v holds the last
// stage's outputs in the same form for the last radix.  buf: the transform in
// shared memory, element idx at slot padx<PS>(idx) (P + P/2^PS slots).
// The inverse (DIR = -1) runs the plan's stages in reverse order.
template <int E, int DIR, int PS, typename C>
__device__ __forceinline__ void fft_core(C (&v)[E], C* buf, const FftPlan& pl, int j, int TPC,
                                         const C* __restrict__ tw) {
    int ls = 0;
    for (int s = 0; s < pl.ns; ++s) {
        const int lr = pl.lr[DIR > 0 ? s : pl.ns - 1 - s];
        if (s > 0) {
#pragma unroll
            for (int qq = 0; qq < E; ++qq) {
                const int e = qq >> lr, r = qq & ((1 << lr) - 1);
                const int idx = j + e * TPC + (r << (pl.lp - lr));
                v[qq] = buf[padx<PS>(idx)];
            }
        }
        switch (lr) {
            case 1: stage_compute<2, DIR>(v, j, TPC, ls, pl.lp, tw); break;
            case 2: stage_compute<4, DIR>(v, j, TPC, ls, pl.lp, tw); break;
            case 3:
                if constexpr (E >= 8) stage_compute<8, DIR>(v, j, TPC, ls, pl.lp, tw);
                break;
            default:
                if constexpr (E >= 16) stage_compute<16, DIR>(v, j, TPC, ls, pl.lp, tw);
                break;
        }
        if (s < pl.ns - 1) {
            __syncthreads();
#pragma unroll
            for (int qq = 0; qq < E; ++qq) {
                const int e = qq >> lr, r = qq & ((1 << lr) - 1);
                const int b = j + e * TPC;
                const int dst = ((b >> ls) << (ls + lr)) + (b & ((1 << ls) - 1)) + (r << ls);
                buf[padx<PS>(dst)] = v[qq];
            }
            __syncthreads();
        }
        ls += lr;
    }
}

// ---------------------------------------------------------------- column-vectorised transform
// The column pass transforms CW adjacent columns together: a thread owns the same
// butterflies of all CW columns, so the butterfly index arithmetic and the
// twiddle loads are paid once per CW elements, and every shared-memory and
// global access moves the CW contiguous values of one row (32 bytes).
template <typename C, int CW>
struct RowVec;  // CW contiguous complex values
template <>
struct RowVec<float2, 4> {
    __device__ __forceinline__ static void load(const float2* p, float2 (&o)[4]) {
        const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
        o[0] = make_float2(a.x, a.y); o[1] = make_float2(a.z, a.w); o[2] = make_float2(b.x, b.y); o[3] = make_float2(b.z, b.w);
    }
    __device__ __forceinline__ static void store(float2* p, const float2 (&o)[4]) {
        reinterpret_cast<float4*>(p)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        reinterpret_cast<float4*>(p)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    }
};
template <>
struct RowVec<double2, 2> {
    __device__ __forceinline__ static void load(const double2* p, double2 (&o)[2]) { o[0] = p[0]; o[1] = p[1]; }
    __device__ __forceinline__ static void store(double2* p, const double2 (&o)[2]) { p[0] = o[0]; p[1] = o[1]; }
};

template <>
struct RowVec<cdfl, 2> {
    __device__ __forceinline__ static void load(const cdfl* p, cdfl (&o)[2]) {
        const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
        o[0] = cdfl{dfl(a.x, a.y), dfl(a.z, a.w)};
        o[1] = cdfl{dfl(b.x, b.y), dfl(b.z, b.w)};
    }
    __device__ __forceinline__ static void store(cdfl* p, const cdfl (&o)[2]) {
        reinterpret_cast<float4*>(p)[0] = make_float4(o[0].x.hi, o[0].x.lo, o[0].y.hi, o[0].y.lo);
        reinterpret_cast<float4*>(p)[1] = make_float4(o[1].x.hi, o[1].x.lo, o[1].y.hi, o[1].y.lo);
    }
};

template <int R, int DIR, int E, int CW, typename C>
__device__ __forceinline__ void stage_compute_vec(C (&v)[CW][E], int j, int TPC, int ls, int lp,
                                                  const C* __restrict__ tw) {
    constexpr int LR = ilog2c<R>();
#pragma unroll
    for (int e = 0; e < E / R; ++e) {
        if (ls > 0) {
            const int b = j + e * TPC;
            const int k = b & ((1 << ls) - 1);
            const int sh = lp - ls - LR;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = ldg_c(&tw[(k * r) << sh]);
                if (DIR < 0) w.y = -w.y;
#pragma unroll
                for (int c = 0; c < CW; ++c) v[c][e * R + r] = v[c][e * R + r] * w;
            }
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) dft_reg<R, DIR>(&v[c][e * R]);
    }
}

// Same contract as fft_core, with v[c][.] holding column c.  Shared memory holds
// each row's CW values as two 16-byte halves in two separate padded arrays
// (half h of element idx at bufh[padx<3>(idx)]), so 128-bit accesses of
// consecutive elements are conflict-free.
template <typename C, int CW>
struct Halves;
template <>
struct Halves<float2, 4> {  // half = 2 columns = float4
    using H = float4;
    __device__ __forceinline__ static void split(const float2 (&r)[4], float4& a, float4& b) {
        a = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
        b = make_float4(r[2].x, r[2].y, r[3].x, r[3].y);
    }
    __device__ __forceinline__ static void join(const float4& a, const float4& b, float2 (&r)[4]) {
        r[0] = make_float2(a.x, a.y); r[1] = make_float2(a.z, a.w); r[2] = make_float2(b.x, b.y); r[3] = make_float2(b.z, b.w);
    }
};
template <>
struct Halves<double2, 2> {  // half = 1 column = double2
    using H = double2;
    __device__ __forceinline__ static void split(const double2 (&r)[2], double2& a, double2& b) { a = r[0]; b = r[1]; }
    __device__ __forceinline__ static void join(const double2& a, const double2& b, double2 (&r)[2]) { r[0] = a; r[1] = b; }
};

template <>
struct Halves<cdfl, 2> {  // half = 1 column = one double-float complex (16 bytes)
    using H = float4;
    __device__ __forceinline__ static void split(const cdfl (&r)[2], float4& a, float4& b) {
        a = make_float4(r[0].x.hi, r[0].x.lo, r[0].y.hi, r[0].y.lo);
        b = make_float4(r[1].x.hi, r[1].x.lo, r[1].y.hi, r[1].y.lo);
    }
    __device__ __forceinline__ static void join(const float4& a, const float4& b, cdfl (&r)[2]) {
        r[0] = cdfl{dfl(a.x, a.y), dfl(a.z, a.w)};
        r[1] = cdfl{dfl(b.x, b.y), dfl(b.z, b.w)};
    }
};

template <int E, int DIR, int CW, typename C>
__device__ __forceinline__ void fft_core_vec(C (&v)[CW][E], typename Halves<C, CW>::H* buf0,
                                             typename Halves<C, CW>::H* buf1, const FftPlan& pl, int j, int TPC,
                                             const C* __restrict__ tw) {
    using HV = Halves<C, CW>;
    int ls = 0;
    for (int s = 0; s < pl.ns; ++s) {
        const int lr = pl.lr[DIR > 0 ? s : pl.ns - 1 - s];
        if (s > 0) {
#pragma unroll
            for (int qq = 0; qq < E; ++qq) {
                const int e = qq >> lr, r = qq & ((1 << lr) - 1);
                const int idx = padx<3>(j + e * TPC + (r << (pl.lp - lr)));
                C row[CW];
                HV::join(buf0[idx], buf1[idx], row);
#pragma unroll
                for (int c = 0; c < CW; ++c) v[c][qq] = row[c];
            }
        }
        switch (lr) {
            case 1: stage_compute_vec<2, DIR>(v, j, TPC, ls, pl.lp, tw); break;
            case 2: stage_compute_vec<4, DIR>(v, j, TPC, ls, pl.lp, tw); break;
            default: stage_compute_vec<8, DIR>(v, j, TPC, ls, pl.lp, tw); break;
        }
        if (s < pl.ns - 1) {
            __syncthreads();
#pragma unroll
            for (int qq = 0; qq < E; ++qq) {
                const int e = qq >> lr, r = qq & ((1 << lr) - 1);
                const int b = j + e * TPC;
                const int dst = ((b >> ls) << (ls + lr)) + (b & ((1 << ls) - 1)) + (r << ls);
                C row[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) row[c] = v[c][qq];
                HV::split(row, buf0[padx<3>(dst)], buf1[padx<3>(dst)]);
            }
            __syncthreads();
        }
        ls += lr;
    }
}

// ---------------------------------------------------------------- kernels
// Row passes: at most 512 threads (P <= 4096, E >= 8).  The double-float ones are held to
// 64 registers so that two CTAs share an SM (their arithmetic is latency-bound at one).
template <typename T> constexpr int rows_min_blocks() { return std::is_same<T, dfl>::value ? 2 : 1; }

template <typename T, int E, class Src>
__global__ void __launch_bounds__(512, rows_min_blocks<T>()) k_rows_fwd(FftPlan pl, int nin, Src src,
                                                                        cpx_t<T>* __restrict__ out,
                                                                        const cpx_t<T>* __restrict__ tw) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int z = blockIdx.x;
    const int j = threadIdx.x, TPC = blockDim.x;
    C v[E];
    const int lr0 = pl.lr[0];
#pragma unroll
    for (int qq = 0; qq < E; ++qq) {
        const int e = qq >> lr0, r = qq & ((1 << lr0) - 1);
        const int x = j + e * TPC + (r << (pl.lp - lr0));
        v[qq] = x < nin ? src.template load<C>(z, x) : czero<C>();
    }
    fft_core<E, +1, (E == 16 ? 4 : 3)>(v, buf, pl, j, TPC, tw);
    const int lrl = pl.lr[pl.ns - 1];
    C* o = out + (size_t)z * pl.P;
#pragma unroll
    for (int qq = 0; qq < E; ++qq) {
        const int e = qq >> lrl, r = qq & ((1 << lrl) - 1);
        o[j + e * TPC + (r << (pl.lp - lrl))] = v[qq];
    }
}

// Column pass with column-vectorised transforms (radix <= 8, EV elements per
// column per thread).  MODE 0: forward z-FFT, times Ghat, inverse z-FFT, rows
// < nout written back in place; MODE 1: forward only, quadrant of qscale * result.
template <typename T, int EV, int CW, int MODE>
__global__ void __launch_bounds__(512) k_cols_vec(FftPlan pl, int nin, int nout, cpx_t<T>* __restrict__ X,
                                                  const cpx_t<T>* __restrict__ ghat, cpx_t<T>* __restrict__ quad,
                                                  T qscale, const cpx_t<T>* __restrict__ tw) {
    using C = cpx_t<T>;
    using H = typename Halves<C, CW>::H;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = pl.P, lp = pl.lp;
    H* buf0 = reinterpret_cast<H*>(smem_raw);
    H* buf1 = buf0 + (P + (P >> 3));
    const int ntile = P / CW;
    const int b = blockIdx.x;
    const int tile = (b & 1) ? (ntile - 1 - (b >> 1)) : (b >> 1);
    const int kx0 = tile * CW;
    const int j = threadIdx.x, TPC = blockDim.x;
    C v[CW][EV];
    const int lr0 = pl.lr[0];
#pragma unroll
    for (int qq = 0; qq < EV; ++qq) {
        const int e = qq >> lr0, r = qq & ((1 << lr0) - 1);
        const int z = j + e * TPC + (r << (lp - lr0));
        C row[CW];
        if (z < nin) RowVec<C, CW>::load(X + (size_t)z * P + kx0, row);
        else {
#pragma unroll
            for (int c = 0; c < CW; ++c) row[c] = czero<C>();
        }
#pragma unroll
        for (int c = 0; c < CW; ++c) v[c][qq] = row[c];
    }
    fft_core_vec<EV, +1, CW>(v, buf0, buf1, pl, j, TPC, tw);
    const int lrl = pl.lr[pl.ns - 1];
    if constexpr (MODE == 0) {
        const C* g[CW];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
            const int kx = kx0 + c;
            g[c] = ghat + (size_t)(kx <= P / 2 ? kx : P - kx) * (P / 2 + 1);
        }
#pragma unroll
        for (int qq = 0; qq < EV; ++qq) {
            const int e = qq >> lrl, r = qq & ((1 << lrl) - 1);
            const int kz = j + e * TPC + (r << (lp - lrl));
            const int kzq = kz <= P / 2 ? kz : P - kz;
#pragma unroll
            for (int c = 0; c < CW; ++c) v[c][qq] = v[c][qq] * ldg_c(&g[c][kzq]);
        }
        fft_core_vec<EV, -1, CW>(v, buf0, buf1, pl, j, TPC, tw);
#pragma unroll
        for (int qq = 0; qq < EV; ++qq) {
            const int e = qq >> lr0, r = qq & ((1 << lr0) - 1);
            const int z = j + e * TPC + (r << (lp - lr0));
            if (z < nout) {
                C row[CW];
#pragma unroll
                for (int c = 0; c < CW; ++c) row[c] = v[c][qq];
                RowVec<C, CW>::store(X + (size_t)z * P + kx0, row);
            }
        }
    } else {
#pragma unroll
        for (int qq = 0; qq < EV; ++qq) {
            const int e = qq >> lrl, r = qq & ((1 << lrl) - 1);
            const int kz = j + e * TPC + (r << (lp - lrl));
            if (kz > P / 2) continue;
#pragma unroll
            for (int c = 0; c < CW; ++c)
                if (kx0 + c <= P / 2) quad[(size_t)(kx0 + c) * (P / 2 + 1) + kz] = qscale * v[c][qq];
        }
    }
}

template <typename T, int E, class Dst>
__global__ void __launch_bounds__(512, rows_min_blocks<T>()) k_rows_inv(FftPlan pl, int n,
                                                                        const cpx_t<T>* __restrict__ X, Dst dst,
                                                                        const cpx_t<T>* __restrict__ tw) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int z = blockIdx.x;
    const int j = threadIdx.x, TPC = blockDim.x;
    C v[E];
    const int lrl = pl.lr[pl.ns - 1];
    const C* xr = X + (size_t)z * pl.P;
#pragma unroll
    for (int qq = 0; qq < E; ++qq) {
        const int e = qq >> lrl, r = qq & ((1 << lrl) - 1);
        v[qq] = xr[j + e * TPC + (r << (pl.lp - lrl))];
    }
    fft_core<E, -1, (E == 16 ? 4 : 3)>(v, buf, pl, j, TPC, tw);
    const int lr0 = pl.lr[0];
#pragma unroll
    for (int qq = 0; qq < E; ++qq) {
        const int e = qq >> lr0, r = qq & ((1 << lr0) - 1);
        const int x = j + e * TPC + (r << (pl.lp - lr0));
        if (x < n) dst.template store<C>(z, x, v[qq]);
    }
}

__global__ void k_twiddles(int P, double2* tw64, float2* tw32) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)P, &s, &c);
    tw64[m] = make_double2(c, -s);
    tw32[m] = make_float2((float)c, (float)-s);
}

__global__ void k_incident_factors(int n, double wh, double cth, double sth, double2* ex, double2* ez) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s, c;
    sincos(wh * (double)(i + 1) * cth, &s, &c);
    ex[i] = make_double2(c, s);
    sincos(wh * (double)(i + 1) * sth, &s, &c);
    ez[i] = make_double2(c, s);
}

// double-float tables (ls_dfloat.cuh): cnt doubles, complex arrays as pairs of reals
__global__ void k_to_dfl(size_t cnt, const double* __restrict__ a, dfl* __restrict__ b) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = dfl_of(a[i]);
}

__global__ void k_incident_factors_df(int n, double wh, double cth, double sth, cdfl* ex, cdfl* ez) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s, c;
    sincos(wh * (double)(i + 1) * cth, &s, &c);
    ex[i] = ccast<cdfl>(make_double2(c, s));
    sincos(wh * (double)(i + 1) * sth, &s, &c);
    ez[i] = ccast<cdfl>(make_double2(c, s));
}

// m u_I in double-float: the incident wave's factors and the medium as double-float tables
struct SrcIncDf {
    const dfl* m;
    const cdfl* ex;
    const cdfl* ez;
    int n;
    template <typename C>
    __device__ __forceinline__ cdfl load(int z, int x) const {
        return m[(size_t)z * n + x] * (ldg_c(&ex[x]) * ldg_c(&ez[z]));
    }
};

__global__ void k_quad_to32(size_t cnt, const double2* a, float2* b) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = ccast<float2>(a[i]);
}

// Elements per thread: row passes FP64 8 / FP32 16; column pass 8 per column of
// its tile.  Column tiles are 2 (FP64) or 4 (FP32) columns: 32-byte row segments.
constexpr int E64 = 8, CW64 = 2;
constexpr int E32 = 16, CW32 = 4;
constexpr int EV = 8;  // column pass: elements per column per thread (radix <= 8)

// shared memory of the padded layouts (one slot every 8 or 16 elements)
constexpr size_t row_smem64(int P) { return sizeof(double2) * (size_t)(P + (P >> 3)); }
constexpr size_t row_smem32(int P) { return sizeof(float2) * (size_t)(P + (P >> 4)); }
constexpr size_t col_smem(int P) { return 2 * 16 * (size_t)(P + (P >> 3)); }

FftPlan make_plan(int lp, int lrmax) {
    FftPlan p{};
    p.P = 1 << lp;
    p.lp = lp;
    int left = lp;
    while (left > 0) {
        const int lr = left >= lrmax ? lrmax : left;
        p.lr[p.ns++] = lr;
        left -= lr;
    }
    return p;
}

template <typename K>
int allow_smem(K kern, size_t bytes) {
    if (bytes > 48 * 1024) LS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return LS_OK;
}

int to_dfl(ls_handle* h, const double* a, dfl* b, size_t cnt) {
    LS_LAUNCH(h, k_to_dfl, (unsigned)((cnt + 255) / 256), 256, 0, cnt, a, b);
    return LS_OK;
}

}  // namespace

int ls_fft_init(ls_handle* h) {
    const int P = h->P;
    h->plan64 = make_plan(h->lp, 3);
    h->plan32 = make_plan(h->lp, 4);
    h->planc64 = make_plan(h->lp, 3);
    h->planc32 = make_plan(h->lp, 3);
    LS_CUDA(cudaMalloc(&h->tw64, sizeof(double2) * P));
    LS_CUDA(cudaMalloc(&h->tw32, sizeof(float2) * P));
    LS_CUDA(cudaMalloc(&h->fftws, sizeof(double2) * (size_t)h->n * P));
    LS_CUDA(cudaMalloc(&h->incx, sizeof(double2) * h->n));
    LS_CUDA(cudaMalloc(&h->incz, sizeof(double2) * h->n));
    LS_LAUNCH(h, k_twiddles, (P + 255) / 256, 256, 0, P, h->tw64, h->tw32);
    const size_t N = (size_t)h->n * h->n;
    LS_CUDA(cudaMalloc(&h->twdf, sizeof(cdfl) * P));
    LS_CUDA(cudaMalloc(&h->mdf, sizeof(dfl) * N));
    LS_CUDA(cudaMalloc(&h->incxdf, sizeof(cdfl) * h->n));
    LS_CUDA(cudaMalloc(&h->inczdf, sizeof(cdfl) * h->n));
    LS_TRY(to_dfl(h, reinterpret_cast<const double*>(h->tw64), reinterpret_cast<dfl*>(h->twdf), 2 * (size_t)P));
    LS_TRY(to_dfl(h, h->m64, h->mdf, N));
    LS_TRY(allow_smem(k_cols_vec<double, EV, CW64, 0>, col_smem(P)));
    LS_TRY(allow_smem(k_cols_vec<double, EV, CW64, 1>, col_smem(P)));
    LS_TRY(allow_smem(k_cols_vec<float, EV, CW32, 0>, col_smem(P)));
    LS_TRY(allow_smem(k_rows_fwd<double, E64, SrcMU<double, double2>>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_fwd<double, E64, SrcInc<double>>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_fwd<double, E64, SrcGpad>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_inv<double, E64, DstApply<double2>>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_inv<double, E64, DstRhs>, row_smem64(P)));
    LS_TRY(allow_smem(k_cols_vec<dfl, EV, CW64, 0>, col_smem(P)));
    LS_TRY(allow_smem(k_rows_fwd<dfl, E64, SrcMU<dfl, double2>>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_fwd<dfl, E64, SrcIncDf>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_inv<dfl, E64, DstApply<double2>>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_inv<dfl, E64, DstRhs>, row_smem64(P)));
    LS_TRY(allow_smem(k_rows_fwd<float, E32, SrcMU<float, float2>>, row_smem32(P)));
    LS_TRY(allow_smem(k_rows_fwd<float, E32, SrcMU<float, double2>>, row_smem32(P)));
    LS_TRY(allow_smem(k_rows_inv<float, E32, DstApply<float2>>, row_smem32(P)));
    LS_TRY(allow_smem(k_rows_inv<float, E32, DstApply<double2>>, row_smem32(P)));
    return ls_fft16_init(h);
}

int ls_spectrum_build(ls_handle* h, const double2* gtab) {
    const int P = h->P, n = h->n;
    const FftPlan& pl = h->plan64;
    double2* work = nullptr;
    const size_t q1 = (size_t)(P / 2 + 1);
    LS_CUDA(cudaMalloc(&work, sizeof(double2) * (size_t)P * P));
    LS_CUDA(cudaMalloc(&h->ghat64, sizeof(double2) * q1 * q1));
    LS_CUDA(cudaMalloc(&h->ghat32, sizeof(float2) * q1 * q1));
    int rc = LS_OK;
    do {
        SrcGpad src{gtab, n, P};
        k_rows_fwd<double, E64, SrcGpad><<<P, P / E64, row_smem64(P), h->stream>>>(pl, P, src, work, h->tw64);
        h->launches++;
        const double qscale = h->omega * h->omega / ((double)P * (double)P);
        k_cols_vec<double, EV, CW64, 1><<<P / CW64, (P / EV), col_smem(P), h->stream>>>(
            h->planc64, P, P, work, nullptr, h->ghat64, qscale, h->tw64);
        h->launches++;
        const size_t cnt = q1 * q1;
        k_quad_to32<<<(unsigned)((cnt + 255) / 256), 256, 0, h->stream>>>(cnt, h->ghat64, h->ghat32);
        h->launches++;
        if (cudaMalloc(&h->ghatdf, sizeof(cdfl) * cnt) != cudaSuccess) {
            rc = LS_ENOMEM;
            break;
        }
        if ((rc = to_dfl(h, reinterpret_cast<const double*>(h->ghat64), reinterpret_cast<dfl*>(h->ghatdf),
                         2 * cnt)) != LS_OK)
            break;
        cudaError_t e = cudaPeekAtLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = ls_cuda_fail(e);
    } while (0);
    cudaFree(work);
    return rc;
}

int ls_apply64(ls_handle* h, const double2* u, double2* y) {
    const int n = h->n, P = h->P;
    const FftPlan& pl = h->plan64;
    double2* X = static_cast<double2*>(h->fftws);
    SrcMU<double, double2> src{h->m64, u, n};
    LS_LAUNCH(h, (k_rows_fwd<double, E64, SrcMU<double, double2>>), n, P / E64, row_smem64(P),
              pl, n, src, X, h->tw64);
    LS_LAUNCH(h, (k_cols_vec<double, EV, CW64, 0>), P / CW64, (P / EV), col_smem(P),
              h->planc64, n, n, X, h->ghat64, (double2*)nullptr, 0.0, h->tw64);
    DstApply<double2> dst{u, y, n};
    LS_LAUNCH(h, (k_rows_inv<double, E64, DstApply<double2>>), n, P / E64, row_smem64(P),
              pl, n, X, dst, h->tw64);
    return LS_OK;
}

// The FP64 apply's three passes in double-float arithmetic (ls_dfloat.cuh): FP64 I/O,
// about 48 significant bits inside, on the FP32 pipes.
int ls_apply_df(ls_handle* h, const double2* u, double2* y) {
    const int n = h->n, P = h->P;
    const FftPlan& pl = h->plan64;
    cdfl* X = static_cast<cdfl*>(h->fftws);
    SrcMU<dfl, double2> src{h->mdf, u, n};
    LS_LAUNCH(h, (k_rows_fwd<dfl, E64, SrcMU<dfl, double2>>), n, P / E64, row_smem64(P), pl, n, src, X, h->twdf);
    LS_LAUNCH(h, (k_cols_vec<dfl, EV, CW64, 0>), P / CW64, (P / EV), col_smem(P), h->planc64, n, n, X, h->ghatdf,
              (cdfl*)nullptr, dfl(0.f, 0.f), h->twdf);
    DstApply<double2> dst{u, y, n};
    LS_LAUNCH(h, (k_rows_inv<dfl, E64, DstApply<double2>>), n, P / E64, row_smem64(P), pl, n, X, dst, h->twdf);
    return LS_OK;
}

int ls_apply32(ls_handle* h, const float2* u, float2* y) {
    if (h->fft_variant != 1 && ls_fft16_supported(h)) return ls_apply32_fft16(h, u, y, h->fft_variant);
    const int n = h->n, P = h->P;
    const FftPlan& pl = h->plan32;
    float2* X = static_cast<float2*>(h->fftws);
    SrcMU<float, float2> src{h->m32, u, n};
    LS_LAUNCH(h, (k_rows_fwd<float, E32, SrcMU<float, float2>>), n, P / E32, row_smem32(P),
              pl, n, src, X, h->tw32);
    LS_LAUNCH(h, (k_cols_vec<float, EV, CW32, 0>), P / CW32, (P / EV), col_smem(P),
              h->planc32, n, n, X, h->ghat32, (float2*)nullptr, 0.0f, h->tw32);
    DstApply<float2> dst{u, y, n};
    LS_LAUNCH(h, (k_rows_inv<float, E32, DstApply<float2>>), n, P / E32, row_smem32(P),
              pl, n, X, dst, h->tw32);
    return LS_OK;
}

int ls_apply_mx(ls_handle* h, const double2* u, double2* y) {
    if (h->fft_variant != 1 && ls_fft16_supported(h)) return ls_apply_mx_fft16(h, u, y, h->fft_variant);
    const int n = h->n, P = h->P;
    const FftPlan& pl = h->plan32;
    float2* X = static_cast<float2*>(h->fftws);
    SrcMU<float, double2> src{h->m32, u, n};
    LS_LAUNCH(h, (k_rows_fwd<float, E32, SrcMU<float, double2>>), n, P / E32, row_smem32(P),
              pl, n, src, X, h->tw32);
    LS_LAUNCH(h, (k_cols_vec<float, EV, CW32, 0>), P / CW32, (P / EV), col_smem(P),
              h->planc32, n, n, X, h->ghat32, (float2*)nullptr, 0.0f, h->tw32);
    DstApply<double2> dst{u, y, n};
    LS_LAUNCH(h, (k_rows_inv<float, E32, DstApply<double2>>), n, P / E32, row_smem32(P),
              pl, n, X, dst, h->tw32);
    return LS_OK;
}

int ls_rhs64(ls_handle* h, double theta, double2* f) {
    const int n = h->n, P = h->P;
    const FftPlan& pl = h->plan64;
    double2* X = static_cast<double2*>(h->fftws);
    LS_LAUNCH(h, k_incident_factors, (n + 255) / 256, 256, 0, n, h->omega * h->h, std::cos(theta),
              std::sin(theta), h->incx, h->incz);
    SrcInc<double> src{h->m64, h->incx, h->incz, n};
    LS_LAUNCH(h, (k_rows_fwd<double, E64, SrcInc<double>>), n, P / E64, row_smem64(P),
              pl, n, src, X, h->tw64);
    LS_LAUNCH(h, (k_cols_vec<double, EV, CW64, 0>), P / CW64, (P / EV), col_smem(P),
              h->planc64, n, n, X, h->ghat64, (double2*)nullptr, 0.0, h->tw64);
    DstRhs dst{f, n};
    LS_LAUNCH(h, (k_rows_inv<double, E64, DstRhs>), n, P / E64, row_smem64(P), pl, n, X, dst, h->tw64);
    return LS_OK;
}

// The incident right-hand side in double-float arithmetic (FP64 output)
int ls_rhs_df(ls_handle* h, double theta, double2* f) {
    const int n = h->n, P = h->P;
    const FftPlan& pl = h->plan64;
    cdfl* X = static_cast<cdfl*>(h->fftws);
    LS_LAUNCH(h, k_incident_factors_df, (n + 255) / 256, 256, 0, n, h->omega * h->h, std::cos(theta),
              std::sin(theta), h->incxdf, h->inczdf);
    SrcIncDf src{h->mdf, h->incxdf, h->inczdf, n};
    LS_LAUNCH(h, (k_rows_fwd<dfl, E64, SrcIncDf>), n, P / E64, row_smem64(P), pl, n, src, X, h->twdf);
    LS_LAUNCH(h, (k_cols_vec<dfl, EV, CW64, 0>), P / CW64, (P / EV), col_smem(P), h->planc64, n, n, X, h->ghatdf,
              (cdfl*)nullptr, dfl(0.f, 0.f), h->twdf);
    DstRhs dst{f, n};
    LS_LAUNCH(h, (k_rows_inv<dfl, E64, DstRhs>), n, P / E64, row_smem64(P), pl, n, X, dst, h->twdf);
    return LS_OK;
}

int ls_rhs(ls_handle* h, double theta, double2* f) {
    return h->dfloat ? ls_rhs_df(h, theta, f) : ls_rhs64(h, theta, f);
}


// ---------------------------------------------------------------- FP32 LS-apply without allocation
// ls_apply_f32_noalloc runs the same three passes as ls_apply32, but its n x P
// scratch and its twiddle tables are file-scope device arrays of fixed size
// instead of memory owned by a handle, so a call allocates nothing.  Those
// arrays exist once per GPU that loads the library and stay until exit; every
// call on a device uses the same scratch.
namespace {

constexpr size_t kNoAllocMaxElems = (size_t)1 << 21;  // n * P <= 2^21 float2 (16 MiB): n <= 1024
constexpr int kNoAllocTwElems = 4096;                  // twiddles of every P = 16..2048, P at offset P - 16
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocMaxElems];
static __device__ __align__(256) float2 g_noalloc_tw[kNoAllocTwElems];

struct NoAllocDevice {
    bool ready = false;
    float2* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    float2* tw = nullptr;       // device address of g_noalloc_tw on this device
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// tw[P - 16 + m] = exp(-2 pi i m / P) for every P = 16, 32, ..., 2048 and m < P
__global__ void k_noalloc_twiddles(float2* tw) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNoAllocTwElems - 16) return;
    int P = 16;
    while (k >= 2 * P - 16) P *= 2;  // segment [P - 16, 2P - 16) belongs to P
    const int m = k - (P - 16);
    double s, c;
    sincospi(2.0 * (double)m / (double)P, &s, &c);
    tw[k] = make_float2((float)c, (float)-s);
}

// First call on a device (that device current): resolve the arrays' device
// addresses, fill the twiddle tables and raise the shared-memory limit of the
// column kernel.  Synchronises `stream` once.
int noalloc_setup(int dev, cudaStream_t stream, NoAllocDevice** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        LS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        d.scratch = static_cast<float2*>(p);
        LS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_tw));
        d.tw = static_cast<float2*>(p);
        k_noalloc_twiddles<<<(kNoAllocTwElems + 255) / 256, 256, 0, stream>>>(d.tw);
        LS_CUDA(cudaPeekAtLastError());
        LS_TRY(allow_smem(k_cols_vec<float, EV, CW32, 0>, col_smem(2048)));
        LS_CUDA(cudaStreamSynchronize(stream));
        d.ready = true;
    }
    *out = &d;
    return LS_OK;
}

}  // namespace

extern "C" int ls_apply_f32_noalloc(int n, const float* m, const ls_c32* ghat, const ls_c32* u, ls_c32* y,
                                    void* stream_) {
    if (n < 8 || !m || !ghat || !u || !y) return LS_EINVAL;
    int lp = 0;
    while ((1 << lp) < 2 * n - 1) ++lp;
    const int P = 1 << lp;
    if ((size_t)n * P > kNoAllocMaxElems || P > 2048) return LS_ETOOBIG;
    int dev = 0;
    LS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return LS_EINVAL;
    // every buffer must be device (or managed) memory of the current device: the
    // scratch used below is this device's, and a launch here cannot read another's
    const void* bufs[4] = {m, ghat, u, y};
    for (const void* b : bufs) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, b) != cudaSuccess) {
            (void)cudaGetLastError();
            return LS_EINVAL;
        }
        if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
            return LS_EINVAL;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    NoAllocDevice* d = nullptr;
    LS_TRY(noalloc_setup(dev, stream, &d));
    const float2* tw = d->tw + (P - 16);
    const FftPlan pr = make_plan(lp, 4), pc = make_plan(lp, 3);
    float2* X = d->scratch;
    SrcMU<float, float2> src{m, reinterpret_cast<const float2*>(u), n};
    k_rows_fwd<float, E32, SrcMU<float, float2>><<<n, P / E32, row_smem32(P), stream>>>(pr, n, src, X, tw);
    LS_CUDA(cudaPeekAtLastError());
    k_cols_vec<float, EV, CW32, 0><<<P / CW32, (P / EV), col_smem(P), stream>>>(
        pc, n, n, X, reinterpret_cast<const float2*>(ghat), (float2*)nullptr, 0.0f, tw);
    LS_CUDA(cudaPeekAtLastError());
    DstApply<float2> dst{reinterpret_cast<const float2*>(u), reinterpret_cast<float2*>(y), n};
    k_rows_inv<float, E32, DstApply<float2>><<<n, P / E32, row_smem32(P), stream>>>(pr, n, X, dst, tw);
    LS_CUDA(cudaPeekAtLastError());
    return LS_OK;
}
