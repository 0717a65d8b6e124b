// ls_internal.cuh -- shared definitions of the GB300 Lippmann-Schwinger library.
//
// Complex helpers, the handle, launch bookkeeping and the declarations that the
// translation units (FFT convolution, stencils, factorisation, sweeps, Krylov,
// C ABI) share.  Everything here is device code or plain host C++; no torch.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "ls.h"

// ------------------------------------------------------------------ complex
template <typename T> struct cpx;
template <> struct cpx<float> { using type = float2; };
template <> struct cpx<double> { using type = double2; };
template <typename T> using cpx_t = typename cpx<T>::type;

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

#define LS_CPX_OPS(C, R)                                                                          \
    __host__ __device__ __forceinline__ C operator+(C a, C b) { return mkc(a.x + b.x, a.y + b.y); } \
    __host__ __device__ __forceinline__ C operator-(C a, C b) { return mkc(a.x - b.x, a.y - b.y); } \
    __host__ __device__ __forceinline__ C operator-(C a) { return mkc(-a.x, -a.y); }               \
    __host__ __device__ __forceinline__ C operator*(C a, C b) {                                    \
        return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                                  \
    }                                                                                              \
    __host__ __device__ __forceinline__ C operator*(R s, C a) { return mkc(s * a.x, s * a.y); }     \
    __host__ __device__ __forceinline__ C conj(C a) { return mkc(a.x, -a.y); }                     \
    __host__ __device__ __forceinline__ R cabs2(C a) { return a.x * a.x + a.y * a.y; }             \
    __host__ __device__ __forceinline__ C cfma(C a, C b, C c) { /* a*b + c */                      \
        return mkc(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));          \
    }                                                                                              \
    __host__ __device__ __forceinline__ C cfms(C a, C b, C c) { /* c - a*b */                      \
        return mkc(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));        \
    }                                                                                              \
    __host__ __device__ __forceinline__ C cconjmul_acc(C a, C b, C c) { /* conj(a)*b + c */        \
        return mkc(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));          \
    }

LS_CPX_OPS(float2, float)
LS_CPX_OPS(double2, double)
#undef LS_CPX_OPS

// FP64 <-> FP32 conversions on the integer pipes.  GB300's FP64 units are few (about
// 1/64 of the FP32 rate) and the hardware conversions run on them, so kernels that move
// FP64 fields into FP32 arithmetic and back (the mixed-precision path) were bound by
// conversions.  These give the same results as the hardware's round-to-nearest-even
// conversion (double -> float) and the exact widening (float -> double), subnormals,
// infinities and NaNs (quieted) included; ls_check_conversions tests them against it.
__host__ __device__ __forceinline__ float d2f_rn(double d) {
#ifdef __CUDA_ARCH__
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return __uint_as_float(sgn | 0x7F800000u | (m ? (0x400000u | (unsigned)(m >> 29)) : 0u));
    int ef = e - 1023 + 127;                       // biased float exponent of a normal result
    if (ef >= 255) return __uint_as_float(sgn | 0x7F800000u);
    const unsigned long long mm = m | (e ? (1ull << 52) : 0ull);   // 53-bit significand
    int sh = 29;                                   // bits dropped for a normal result
    if (ef <= 0) {                                 // subnormal (or zero) float
        sh += 1 - ef;
        ef = 0;
        if (sh > 62) return __uint_as_float(sgn);  // below half the smallest subnormal
    }
    const unsigned long long qv = mm >> sh, rem = mm & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    const unsigned long long r = qv + ((rem > half || (rem == half && (qv & 1ull))) ? 1ull : 0ull);
    // normal: exponent field (ef - 1) plus the significand with its leading 1 (a carry
    // out of the significand bumps the exponent); subnormal: the significand alone
    const unsigned bits = ef > 0 ? ((unsigned)(ef - 1) << 23) + (unsigned)r : (unsigned)r;
    return __uint_as_float(sgn | bits);
#else
    return (float)d;
#endif
}
__host__ __device__ __forceinline__ double f2d(float f) {
#ifdef __CUDA_ARCH__
    const unsigned b = __float_as_uint(f);
    const unsigned long long sgn = (unsigned long long)(b & 0x80000000u) << 32;
    const int e = (int)((b >> 23) & 0xFF);
    const unsigned m = b & 0x7FFFFFu;
    if (e == 0xFF)
        return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull | ((unsigned long long)m << 29) |
                                                (m ? 0x8000000000000ull : 0ull)));
    if (e == 0) {
        if (!m) return __longlong_as_double((long long)sgn);
        const int top = 31 - __clz(m);             // m = 2^top (1.f), value = m 2^-149
        const unsigned long long frac = ((unsigned long long)m << (52 - top)) & 0xFFFFFFFFFFFFFull;
        return __longlong_as_double((long long)(sgn | ((unsigned long long)(top - 149 + 1023) << 52) | frac));
    }
    return __longlong_as_double(
        (long long)(sgn | ((unsigned long long)(e - 127 + 1023) << 52) | ((unsigned long long)m << 29)));
#else
    return (double)f;
#endif
}

template <typename D, typename S> __host__ __device__ __forceinline__ D ccast(S a);
template <> __host__ __device__ __forceinline__ float2 ccast<float2, float2>(float2 a) { return a; }
template <> __host__ __device__ __forceinline__ double2 ccast<double2, double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 ccast<float2, double2>(double2 a) {
    return make_float2(d2f_rn(a.x), d2f_rn(a.y));
}
template <> __host__ __device__ __forceinline__ double2 ccast<double2, float2>(float2 a) {
    return make_double2(f2d(a.x), f2d(a.y));
}
// The same casts by the hardware conversions (FP64 pipe), for kernels whose integer and
// FP32 pipes are the busy ones (the FFT passes of the mixed LS-apply).
template <typename D, typename S> __host__ __device__ __forceinline__ D hw_cast(S a) { return ccast<D>(a); }
template <> __host__ __device__ __forceinline__ float2 hw_cast<float2, double2>(double2 a) {
    return make_float2((float)a.x, (float)a.y);
}
template <> __host__ __device__ __forceinline__ double2 hw_cast<double2, float2>(float2 a) {
    return make_double2((double)a.x, (double)a.y);
}

// ------------------------------------------------------------------ FFT plan
// Stockham stages: log2 radix of each stage in forward order (inverse runs them reversed).
struct FftPlan {
    int P;       // transform length (power of two)
    int lp;      // log2 P
    int ns;      // number of stages
    int lr[8];   // log2 radix per stage
};

// ------------------------------------------------------------------ stencils
// 9 point types x 9 slots; type = (bz+1)*3 + (bx+1), slot = (dz+1)*3 + (dx+1).
struct StencilTables {
    double2 alpha[81];
    double2 wbeta[81];   // w^2 * beta
};

// ------------------------------------------------------------------ CR factors
// Block cyclic reduction of one direction's L strips.  Block tridiagonal along
// the long axis (n blocks of q x q), levels k = 0..K-1 eliminate the odd blocks
// j of level k (global block index i = j << k); level K holds one block.
// All dense matrices are stored column-major (element (r, c) at c*q + r).
struct CrLevel {
    int nk;          // blocks at this level
    int nodd;        // odd blocks: nk / 2
    int neven;       // even blocks: (nk + 1) / 2
    // offsets (in matrices of q*q elements) into the factor pool, per strip
    size_t off_dinv;  // nodd matrices: D^{-1} of odd blocks
    size_t off_p;     // k >= 1: nodd matrices P = D^{-1} W
    size_t off_q;     // k >= 1: nodd matrices Q = D^{-1} E
    size_t off_f;     // k >= 1: neven matrices F = W_j D^{-1}_{j-1} (zero if j == 0)
    size_t off_g;     // k >= 1: neven matrices G = E_j D^{-1}_{j+1} (zero if j+1 == nk)
};

struct DirFactors {
    int K = 0;                    // levels
    std::vector<CrLevel> lev;     // K entries
    size_t off_top = 0;           // D^{-1} of the single block of level K
    size_t mats_per_strip = 0;    // matrices per strip in the pool
    double2* pool64 = nullptr;    // L * mats_per_strip * q*q (FP64; freed in LS_MIXED)
    float2* pool32 = nullptr;     // same layout in FP32 (LS_MIXED)
    // LS_MIXED, tensor-core steps (ls_cr_mma.cu): every matrix as two TF32 planes (re, im)
    // in the tensor cores' 128-byte-swizzled K-major layout (ceil(q/32) atoms of 32
    // K-columns x q rounded up to 8 rows each), so a plane is one contiguous copy
    float* pool_tc = nullptr;
    // LS_MIXED, tensor-core steps: the inverse of the reduced system of level dense_c (the
    // first level with at most 32 blocks), nc = blocks x q unknowns, per strip as TF32
    // planes in blocks of 128 rows x 128 columns (mt row tiles x ks column chunks), so the
    // levels >= dense_c of a local solve are one dense product (ls_cr_dense_apply)
    float* dense_tc = nullptr;
    int dense_c = 0, dense_nc = 0, dense_mt = 0, dense_ks = 0;
    // problem of this direction (the vertical direction is the transposed grid)
    const double* m = nullptr;    // medium of this direction's grid (n x n, long axis fastest)
    StencilTables* tab = nullptr; // device copy of the tables of this direction
    StencilTables host_tab;
    // couplings the solve needs, tabulated in the solve precision (float2 in LS_MIXED):
    //   cw, ce: [l][i][dz+1][r]  west / east neighbour blocks of level 0 (tridiagonal)
    //   cinj:   [l][slot][dx+1][i] trace-injection rows: 0 = row E+t-1 -> E+t, 1 = row E+t -> E+t-1,
    //                              2 = row E -> E-1, 3 = row E-1 -> E
    void* cw = nullptr;
    void* ce = nullptr;
    void* cinj = nullptr;
};

// ------------------------------------------------------------------ handle
constexpr int kMaxBatch = 32;  // right-hand sides per batched Algorithm 2 (ls_bd_cap: the form's own limit)

struct ls_handle {
    int n = 0, L = 0, E = 0, t = 0, q = 0, P = 0, lp = 0, prec = LS_FP64;
    double h = 0, omega = 0;
    ls_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0;
    long long launches = 0;
    bool factored = false;
    bool timing = false;

    double* m64 = nullptr;     // medium, n*n
    float* m32 = nullptr;
    double* mT64 = nullptr;    // transposed medium

    double2 w0{};              // diagonal weight G_w(0)
    double2* ghat64 = nullptr; // spectral quadrant (P/2+1)^2
    float2* ghat32 = nullptr;
    double2* tw64 = nullptr;   // twiddles exp(-2 pi i m / P), m < P
    float2* tw32 = nullptr;
    // double-float copies (ls_dfloat.cuh) of the medium, the spectral quadrant, the
    // twiddles and the incident-wave factors: the FP64-accurate convolutions on the FP32 pipes
    struct dfl* mdf = nullptr;
    struct cdfl* ghatdf = nullptr;
    struct cdfl* twdf = nullptr;
    struct cdfl* incxdf = nullptr;
    struct cdfl* inczdf = nullptr;
    int dfloat = 0;            // 1 (LS_MIXED default): refinement residuals and incident
                               // right-hand sides in double-float arithmetic
    FftPlan plan64{}, plan32{};    // row passes
    FftPlan planc64{}, planc32{};  // column pass
    void* fftws = nullptr;     // n*P complex (FP64 size)
    double2* incx = nullptr;   // incident-wave factors exp(i w h (i+1) cos), exp(i w h (j+1) sin)
    double2* incz = nullptr;

    StencilTables tabs[2];     // host copies: [0] grid, [1] transposed grid
    StencilTables* dtabs = nullptr;  // device copies (2)

    DirFactors fac[2];
    // Sweep workspaces ("lanes"): every lane holds the strip right-hand sides and
    // solutions, traces, transpose scratch, Algorithm 2 staging buffers and its CUDA
    // graphs (one per batch size) for up to nb_cap right-hand sides, so that chunks
    // of a batch can run their Algorithm 2 chains concurrently on different streams.
    struct SweepLane {
        void* srhs = nullptr;      // every strip's right-hand side (n*q each), nb_cap sets
        void* ssol = nullptr;      // every strip's solution
        void* strace = nullptr;    // per layer: row 0 of its down-sweep solution (w^l_0), n each
        void* vtmp = nullptr;      // 4 n*n complex scratch fields (FP64) per right-hand side
        double2* bd_in = nullptr;  // graph staging
        double2* bd_out = nullptr;
        cudaGraph_t graph[kMaxBatch + 1] = {};
        cudaGraphExec_t exec[kMaxBatch + 1] = {};
        long long nodes[kMaxBatch + 1] = {};
        int nb_cap = 0;
        void* cr_part = nullptr;        // partial sums of split reduction steps
        unsigned* cr_cnt = nullptr;     // arrival counters of split reduction steps (kept at 0)
        float2* dense_part = nullptr;   // column-chunk partial products of the reduced inverse
        cudaStream_t stream = nullptr;  // lane 0 runs on the handle's stream
        cudaEvent_t done = nullptr;
    };
    static constexpr int kLanes = 8;
    SweepLane lanes[kLanes];
    int lane = 0;              // lane the sweep functions use (set around concurrent chunks)

    // Krylov workspaces (FP64): the context of ls_krylov.cu and the staging buffers of
    // the host-array entry points, owned by the handle (no library-global state)
    void* krylov = nullptr;
    void* hostbufs = nullptr;
    double* red = nullptr;     // reduction partials
    double* red_host = nullptr;
    size_t red_cap = 0;
    cudaEvent_t ev_fork = nullptr;

    ls_net* net = nullptr;     // learned first step of every outer cycle (ls_unet.cu), or none
    int learned_steps = 0;

    // choices of the autotuner (ls_tune.cu); defaults until ls_autotune runs
    int fft_variant = 2;       // column-pass shape (256 <= P <= 4096): radix 16 with 0 = 1-column tiles,
                               // 3 CTAs/SM; 2 = 2-column tiles; 3 = 1-column tiles, 2 CTAs/SM; radix 8 with
                               // 4 = 1-column tiles; 5 = 2-column tiles.  1: generic radix-8 4-column tiles
    static constexpr int kFftVariants = 9;
    int bd_chunk = 0;          // right-hand sides per Algorithm 2 chain (0: the largest supported)
    int cr_split = 1;          // 1: reduction steps of small levels split blocks over several CTAs
    bool tc_ready = false;     // LS_MIXED: TF32 factor planes and tensor maps built (ls_cr_tc_prepare)
    int tc_sms = 0;            // SMs of the device (tensor-core steps: CTAs per SM by level size)
    int tc_dense = 1;          // tensor-core local solves: levels with <= 32 blocks as one dense product
    int pack_members = 1;      // Algorithm 2 on the members still iterating only, packed (ls_krylov.cu)
    long long sweep_fields = 0;  // fields Algorithm 2 processed during the current solve
    int sweep_hist[LS_MAX_BATCH + 1] = {};  // its applications by batch size, current solve
    int cr_tc = 1;             // FP32 reduction steps on the tensor cores when tc_ready: 0 never,
                               // 1 for batches of 5 or more right-hand sides, 2 always

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double t_apply_ms = 0, t_sweep_ms = 0, t_apply64_ms = 0, t_stencil_ms = 0, t_orth_ms = 0;
    int n_apply = 0, n_sweep = 0, n_apply64 = 0, n_stencil = 0, n_orth = 0;
    // timing without host synchronisation: event pairs recorded during a solve and
    // read once at its end (kind 0: FP32/mixed or FP64 apply, 1: Algorithm 2, 2: FP64 refinement apply)
    std::vector<cudaEvent_t> tev;   // 2 per interval
    std::vector<int> tkind;
    size_t tused = 0;
};

// ------------------------------------------------------------------ errors
#define LS_CUDA(call)                                    \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return ls_cuda_fail(e_);  \
    } while (0)

#define LS_TRY(call)                     \
    do {                                 \
        int rc_ = (call);                \
        if (rc_ != LS_OK) return rc_;    \
    } while (0)

int ls_cuda_fail(cudaError_t e);

// launch + bookkeeping; returns LS_ECUDA from the enclosing function on failure
#define LS_LAUNCH(hdl, kern, grid, block, smem, ...)                                   \
    do {                                                                               \
        kern<<<(grid), (block), (smem), (hdl)->stream>>>(__VA_ARGS__);                 \
        (hdl)->launches++;                                                             \
        cudaError_t e_ = cudaPeekAtLastError();                                        \
        if (e_ != cudaSuccess) return ls_cuda_fail(e_);                                \
    } while (0)

// ------------------------------------------------------------------ internal API
// FFT convolution (ls_fft.cu)
int ls_fft_init(ls_handle* h);                                   // twiddles, plans, workspace
int ls_spectrum_build(ls_handle* h, const double2* gtab);       // Ghat from the G_w table
int ls_apply64(ls_handle* h, const double2* u, double2* y);     // y = H u (FP64)
int ls_apply32(ls_handle* h, const float2* u, float2* y);       // y = H u (FP32)
int ls_apply_mx(ls_handle* h, const double2* u, double2* y);    // FP64 I/O, FP32 arithmetic
int ls_apply_df(ls_handle* h, const double2* u, double2* y);    // FP64 I/O, double-float arithmetic
int ls_rhs_df(ls_handle* h, double theta, double2* f);          // incident right-hand side, double-float
int ls_rhs(ls_handle* h, double theta, double2* f);             // ls_rhs_df if h->dfloat, else ls_rhs64
bool ls_fft16_supported(const ls_handle* h);                     // radix-16 FP32 path: 256 <= P <= 4096
int ls_fft16_init(ls_handle* h);
int ls_apply32_fft16(ls_handle* h, const float2* u, float2* y, int shape);  // shape: fft_variant != 1
int ls_apply_mx_fft16(ls_handle* h, const double2* u, double2* y, int shape);
int ls_rhs64(ls_handle* h, double theta, double2* f);           // f = -w^2 G (m u_I)

// setup (ls_setup_kernels.cu)
int ls_green_table(ls_handle* h, double2** gtab_out);          // G_w on [-n, n]^2 (device)
int ls_stencils_build(ls_handle* h, const double2* gtab);      // alpha, beta for both grids

// stencils + vector kernels (ls_stencil.cu)
int ls_stencil_apply(ls_handle* h, int dir, int withm, const double2* v, const double2* g, double2* y);
int ls_transpose64(ls_handle* h, const double2* a, double2* b);
int ls_transpose64_b(ls_handle* h, const double2* a, double2* b, int nb);
int ls_stencil_apply64(ls_handle* h, int dir, int mode, const double2* v, const double2* g, double2* y);
int ls_stencil_apply_b(ls_handle* h, int dir, int withm, const double2* v, const double2* g, double2* y, int nb);
int ls_stencil_refine_f32(ls_handle* h, int dir, const float2* v, const float2* g, float2* y, int nb);
int ls_stencil_apply_f32(ls_handle* h, int dir, int mode, const float2* v, float2* y);
// Krylov vectors in FP64 (double2) or FP32 (float2); dot products summed in FP64
// One fused pass of a Gram-Schmidt step against nvec directions (ls_stencil.cu) for
// members members[0..cnt) of a lockstep batch in one launch (member m: V and w at
// + m * mstride, coef at + m * cstride, out at + m * ostride):
// mode 0: out = V^H w; 1: w -= V coef, then out = V^H w; 2: w -= V coef, then out[0] = w^H w;
// mode 3: out[0] = w^H w.
int ls_vec_orth_b(ls_handle* h, int mode, int nvec, const double2* V, size_t ld, size_t mstride, const double2* coef,
                  size_t cstride, double2* w, const int* members, int cnt, double2* out, size_t ostride);
int ls_vec_orth_b(ls_handle* h, int mode, int nvec, const float2* V, size_t ld, size_t mstride, const double2* coef,
                  size_t cstride, float2* w, const int* members, int cnt, double2* out, size_t ostride);
// out[m] = ||w + m * mstride|| for the listed members: one pass, one device->host read
int ls_vec_norms_b(ls_handle* h, const double2* w, size_t mstride, const int* members, int cnt, double* out);
int ls_vec_norms_b(ls_handle* h, const float2* w, size_t mstride, const int* members, int cnt, double* out);
int ls_vec_axpby(ls_handle* h, double2 a, const double2* x, double2 b, double2* y);  // y = a x + b y
int ls_vec_axpby(ls_handle* h, double2 a, const float2* x, double2 b, float2* y);
int ls_vec_axpby(ls_handle* h, double2 a, const float2* x, double2 b, double2* y);
int ls_vec_copy(ls_handle* h, const double2* x, double2* y);
int ls_vec_copy(ls_handle* h, const float2* x, float2* y);
int ls_vec_copy(ls_handle* h, const double2* x, float2* y);   // rounded to FP32
int ls_vec_copy(ls_handle* h, const float2* x, double2* y);   // widened
int ls_vec_zero(ls_handle* h, double2* y);
int ls_vec_zero(ls_handle* h, float2* y);
int ls_vec_combine(ls_handle* h, int nvec, const double2* Z, size_t ld, const double2* coef_host, double2* x);
int ls_vec_combine(ls_handle* h, int nvec, const float2* Z, size_t ld, const double2* coef_host, float2* x);

// factorisation (ls_factor.cu)
int ls_factor_all(ls_handle* h);
void ls_factor_free(ls_handle* h);

// sweeps (ls_sweep.cu)
int ls_sweep_alloc(ls_handle* h);
int ls_sweep_dir(ls_handle* h, int dir, const double2* g, double2* v);   // Algorithm 1
int ls_sweep_dir_b(ls_handle* h, int dir, const double2* g, double2* v, int nb);
int ls_sweep_reserve(ls_handle* h, int nb);
int ls_bd_b(ls_handle* h, const double2* g, double2* v, int nb);         // Algorithm 2, nb right-hand sides
int ls_bd_b(ls_handle* h, const float2* g, float2* v, int nb);           // the same on FP32 fields (LS_MIXED)
int ls_bd_lanes(ls_handle* h, const double2* g, double2* v, int nb, int chunk,
                const unsigned char* on = nullptr);
int ls_bd_lanes(ls_handle* h, const float2* g, float2* v, int nb, int chunk,
                const unsigned char* on = nullptr);  // chunks on concurrent lanes, idle chunks skipped
void ls_lanes_free(ls_handle* h);
int ls_bd(ls_handle* h, const double2* g, double2* v);                   // Algorithm 2
int ls_bd_cap(const ls_handle* h);   // right-hand sides one Algorithm 2 pass takes: FP64 4, mixed 8 (32 on tensor cores)
void ls_bd_graph_free(ls_handle* h);
int ls_strip_solve(ls_handle* h, int dir, int layer, const double2* b, double2* x);

// tensor-core reduction steps (ls_cr_mma.cu)
int ls_cr_tc_prepare(ls_handle* h);
void ls_cr_tc_free(ls_handle* h);
int ls_cr_tc_max_nb(const ls_handle* h);
int ls_cr_tc_timeouts(unsigned* count);
int ls_conv_timeouts(unsigned* count);   // tensor-core convolutions of the learned step (ls_unet.cu)
int ls_cr_tc_step(ls_handle* h, int dir, int l, int mode, int k, int nk, unsigned grid, size_t off_a, size_t off_b,
                  size_t off_c, float2* x, size_t SB, int nb, const float2* cw, const float2* ce);
size_t ls_cr_dense_part_elems(const ls_handle* h);   // float2 entries of a lane's dense_part (0: no dense form)
int ls_cr_dense_apply(ls_handle* h, int dir, int l, float2* x, size_t SB, int nb);

// Krylov (ls_krylov.cu)
int ls_inner_gmres(ls_handle* h, const double2* g, double tol, double2* v, int* iters);
int ls_outer_solve(ls_handle* h, const double2* f, double tol, double2* u, int use_x0, ls_stats* st);
int ls_outer_solve_b(ls_handle* h, int nb, const double2* f, double tol, double2* u, int use_x0, ls_stats* st);
int ls_net_apply_field(ls_net* net, cudaStream_t stream, int H, int W, const double2* v, const double* m,
                       double2* z);   // z = s N(v / s, m), one field
