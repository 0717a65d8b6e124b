// ls_stencil.cu -- 9-point stencil applies (Sec. 2) and FP64 vector kernels.
//
//  * (A r)_k = sum_{d in mu(k)} alpha^{t(k)}_d r_{k+d}                   (sparsifying matrix)
//  * (C v)_k = sum_{d in mu(k)} (alpha^{t(k)}_d + w^2 beta^{t(k)}_d m_{k+d}) v_{k+d}
//    (A H kept on the pattern of A, Sec. 2); t(k) is the point type (interior,
//    edge, corner) and mu(k) drops offsets that leave Omega.
//  * e = g - C v is the iterative-refinement residual of Algorithm 2.
// One thread per grid point, x fastest, so neighbour loads along x coalesce and
// the z-neighbours come from L1/L2; the stencil tables sit in shared memory.
//
// Vector kernels for the Krylov levels (Sec. 4) accumulate in FP64 with a fixed
// reduction order (block partials, then one block), so results are reproducible.
#include "ls_internal.cuh"

namespace {

// batch member b = blockIdx.z works on v, g, y at offset b * n * n (m is shared).
// R: arithmetic type of the coefficients and the sum (FP64 I/O either way); FP32 is
// used where the stencil only feeds the preconditioner in mixed precision (on
// GB300 the FP64 form is bound by the FP64 units, the FP32 form by memory).
// A CTA of 32 x 8 threads computes a tile of 32 x 32 points (4 rows per thread): the
// tile's v and m with a one-point halo are staged in shared memory (in the
// arithmetic type) by loads that are all issued before the first store, so every
// value of v and m is read from HBM about once.
constexpr int kStX = 32, kStZ = 32, kStRows = 4;   // tile, rows per thread (threads 32 x 8)
// VF, YF: element types of v and y (double2; float2 for the mixed Algorithm 2's fields,
// which hold FP32 values: v is the FP32 sweep's result, y feeds the FP32 sweep).
template <int MODE, typename R, typename VF = double2, typename YF = double2, typename GF = double2>  // 0: y = A v  1: y = C v  2: y = g - C v
__global__ void __launch_bounds__(256) k_stencil(int n, const StencilTables* __restrict__ tab,
                                                 const double* __restrict__ m, const VF* __restrict__ v,
                                                 const GF* __restrict__ g, YF* __restrict__ y) {
    using CR = cpx_t<R>;
    constexpr int HX = kStX + 2, HZ = kStZ + 2, HN = HX * HZ;
    __shared__ CR sa[81], sb[81];
    __shared__ CR sv[HZ][HX];
    __shared__ R sm[MODE >= 1 ? HZ : 1][MODE >= 1 ? HX : 1];
    {
        const size_t off = (size_t)blockIdx.z * n * n;
        v += off;
        y += off;
        if (MODE == 2) g += off;
    }
    const int tid = threadIdx.y * kStX + threadIdx.x;
    for (int i = tid; i < 81; i += 256) {
        sa[i] = ccast<CR>(tab->alpha[i]);
        sb[i] = ccast<CR>(tab->wbeta[i]);
    }
    const int x0 = blockIdx.x * kStX - 1, z0 = blockIdx.y * kStZ - 1;
    constexpr int PER = (HN + 255) / 256;   // halo tile elements per thread
    const VF vz = {};
    VF vv[PER];
    double mv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = tid + u * 256, hz = e / HX, hx = e % HX, x = x0 + hx, z = z0 + hz;
        const bool in = e < HN && x >= 0 && x < n && z >= 0 && z < n;
        vv[u] = in ? __ldg(&v[(size_t)z * n + x]) : vz;
        if (MODE >= 1) mv[u] = in ? __ldg(&m[(size_t)z * n + x]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = tid + u * 256;
        if (e < HN) {
            sv[e / HX][e % HX] = ccast<CR>(vv[u]);
            if constexpr (MODE >= 1) {
                if constexpr (sizeof(R) == 4) sm[e / HX][e % HX] = d2f_rn(mv[u]);
                else sm[e / HX][e % HX] = mv[u];
            }
        }
    }
    __syncthreads();
    const int i = blockIdx.x * kStX + threadIdx.x;
    if (i >= n) return;
    const int bx = i == 0 ? -1 : (i == n - 1 ? 1 : 0);
#pragma unroll
    for (int rr = 0; rr < kStRows; ++rr) {
        const int lz = threadIdx.y + 8 * rr, j = blockIdx.y * kStZ + lz;
        if (j >= n) break;
        const int bz = j == 0 ? -1 : (j == n - 1 ? 1 : 0);
        const int t = (bz + 1) * 3 + (bx + 1);
        CR acc = czero<CR>();
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            if ((bz == -1 && dz == -1) || (bz == 1 && dz == 1)) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                if ((bx == -1 && dx == -1) || (bx == 1 && dx == 1)) continue;
                const int sl = (dz + 1) * 3 + (dx + 1);
                CR c = sa[t * 9 + sl];
                const int hz = lz + 1 + dz, hx = threadIdx.x + 1 + dx;
                if (MODE >= 1) {
                    const R mm = sm[hz][hx];
                    c = mkc(fma(mm, sb[t * 9 + sl].x, c.x), fma(mm, sb[t * 9 + sl].y, c.y));
                }
                acc = cfma(c, sv[hz][hx], acc);
            }
        }
        const size_t k = (size_t)j * n + i;
        double2 out = ccast<double2>(acc);
        if (MODE == 2) out = ccast<double2>(__ldg(&g[k])) - out;
        y[k] = ccast<YF>(out);
    }
}

__global__ void k_transpose(int n, const double2* __restrict__ a, double2* __restrict__ b) {
    __shared__ double2 tile[32][33];
    a += (size_t)blockIdx.z * n * n;   // batch member blockIdx.z
    b += (size_t)blockIdx.z * n * n;
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int z = z0 + r, x = x0 + threadIdx.x;
        if (z < n && x < n) tile[r][threadIdx.x] = a[(size_t)z * n + x];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int x = x0 + r, z = z0 + threadIdx.x;
        if (z < n && x < n) b[(size_t)x * n + z] = tile[threadIdx.x][r];
    }
}

__global__ void k_transpose_real(int n, const double* __restrict__ a, double* __restrict__ b) {
    __shared__ double tile[32][33];
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int z = z0 + r, x = x0 + threadIdx.x;
        if (z < n && x < n) tile[r][threadIdx.x] = a[(size_t)z * n + x];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int x = x0 + r, z = z0 + threadIdx.x;
        if (z < n && x < n) b[(size_t)x * n + z] = tile[threadIdx.x][r];
    }
}

constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
constexpr int RED_THREADS = 256;

// Vector kernels for FP64 (double2) and FP32 (float2) Krylov vectors.  FP32 vectors are
// combined in FP32 (coefficients rounded once) and their dot products formed in FP32
// per thread and summed in FP64 across threads and blocks, in a fixed order.
template <typename VT> struct Acc;   // the per-thread dot accumulator of a vector type
template <> struct Acc<double2> { using T = double2; };
template <> struct Acc<float2> { using T = float2; };
template <typename VT> __device__ __forceinline__ VT vt_of(double2 c) { return ccast<VT>(c); }

// partial[b * nvec + i] = sum over block b's elements of conj(V_i) w   (i < nvec)
template <typename VT>
__global__ void k_dots(size_t N, int nvec, const VT* __restrict__ V, size_t ld, const VT* __restrict__ w,
                       double2* __restrict__ partial) {
    __shared__ double2 red[RED_THREADS];
    for (int i = 0; i < nvec; ++i) {
        const VT* vi = V + (size_t)i * ld;
        VT acc = czero<VT>();
        for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
            acc = cconjmul_acc(__ldg(&vi[k]), __ldg(&w[k]), acc);
        red[threadIdx.x] = ccast<double2>(acc);
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * nvec + i] = red[0];
        __syncthreads();
    }
}

// out[i] = sum_b partial[b * nvec + i]  (one block, fixed order)
__global__ void k_dots_final(int nblk, int nvec, const double2* __restrict__ partial, double2* __restrict__ out) {
    __shared__ double2 red[RED_THREADS];
    for (int i = 0; i < nvec; ++i) {
        double2 acc = make_double2(0, 0);
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc = acc + partial[(size_t)b * nvec + i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[i] = red[0];
        __syncthreads();
    }
}

// w -= sum_i coef[i] V_i
template <typename VT>
__global__ void k_update(size_t N, int nvec, const VT* __restrict__ V, size_t ld, const double2* __restrict__ coef,
                         VT* __restrict__ w) {
    __shared__ VT sc[128];
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) sc[i] = vt_of<VT>(coef[i]);
    __syncthreads();
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        VT acc = w[k];
        for (int i = 0; i < nvec; ++i) acc = cfms(sc[i], __ldg(&V[(size_t)i * ld + k]), acc);
        w[k] = acc;
    }
}

// Members of a lockstep batch that a batched vector kernel serves: grid row y works on
// member idx[y], whose vectors start idx[y] * mstride after the block's base pointers.
struct MemberList {
    int idx[LS_MAX_BATCH];
};

// One pass of a classical Gram-Schmidt step against nvec <= G directions V_i (stride ld),
// for the members of a batch at once, with everything that is local to an element fused
// into the pass:
//   MODE 0: partial dots V_i^H w;
//   MODE 1: w -= sum_i coef_i V_i, then the partial dots V_i^H w of the updated w;
//   MODE 2: w -= sum_i coef_i V_i, then the partial ||w||^2;
//   MODE 3: the partial ||w||^2 (nvec = 0, w unchanged).
// Grid row y serves member m = ml.idx[y] (its V, w at + m * mstride, its coefficients at
// coef + m * cstride) with gridDim.x blocks; their partial sums go to
// partial[(y * gridDim.x + b) * nout + i].  Per element the operations and their order are
// those of an update followed by a dot pass, so the fused passes give the results of
// separate kernels up to the grouping of the partial sums, while reading each V_i and w
// once.
template <typename VT, int G, int MODE>
__global__ void __launch_bounds__(RED_THREADS) k_orth(size_t N, int nvec, const VT* __restrict__ V, size_t ld,
                                                      size_t mstride, const double2* __restrict__ coef,
                                                      size_t cstride, VT* __restrict__ w, MemberList ml,
                                                      double2* __restrict__ partial) {
    constexpr int NO = MODE >= 2 ? 1 : G;   // sums per thread
    __shared__ VT sc[G];
    __shared__ double2 red[RED_THREADS];
    const size_t mo = (size_t)ml.idx[blockIdx.y] * mstride;
    VT* wm = w + mo;
    if (MODE == 1 || MODE == 2) {
        const double2* cm = coef + (size_t)ml.idx[blockIdx.y] * cstride;
        for (int i = threadIdx.x; i < nvec; i += blockDim.x) sc[i] = vt_of<VT>(cm[i]);
        __syncthreads();
    }
    // per-thread sums in VT over at most kFlush elements, then added into FP64 (with a batch
    // a member gets fewer blocks, so a thread covers more elements than RED_BLOCKS would give)
    constexpr int kFlush = 64;
    VT acc[NO];
    double2 accd[NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        acc[i] = czero<VT>();
        accd[i] = make_double2(0, 0);
    }
    int run = 0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        if (run == kFlush) {
#pragma unroll
            for (int i = 0; i < NO; ++i)
                if (MODE >= 2 || i < nvec) {
                    accd[i] = accd[i] + ccast<double2>(acc[i]);
                    acc[i] = czero<VT>();
                }
            run = 0;
        }
        ++run;
        VT vk[G];
        if (MODE < 3) {
#pragma unroll
            for (int i = 0; i < G; ++i)
                if (i < nvec) vk[i] = __ldg(&V[mo + (size_t)i * ld + k]);
        }
        VT wk = wm[k];
        if (MODE == 1 || MODE == 2) {
#pragma unroll
            for (int i = 0; i < G; ++i)
                if (i < nvec) wk = cfms(sc[i], vk[i], wk);
            wm[k] = wk;
        }
        if (MODE < 2) {
#pragma unroll
            for (int i = 0; i < G; ++i)
                if (i < nvec) acc[i] = cconjmul_acc(vk[i], wk, acc[i]);
        } else {
            acc[0] = cconjmul_acc(wk, wk, acc[0]);
        }
    }
    const int nout = MODE >= 2 ? 1 : nvec;
    double2* pp = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * nout;
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        if (i >= nout) break;
        red[threadIdx.x] = accd[i] + ccast<double2>(acc[i]);
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) pp[i] = red[0];
        __syncthreads();
    }
}

// out[ml.idx[x] * ostride + i] = sum_b partial[(x * bpm + b) * nout + i]: block x sums the
// partials of grid row x of k_orth (fixed order, as k_dots_final).
__global__ void k_orth_final(int bpm, int nout, const double2* __restrict__ partial, MemberList ml,
                             double2* __restrict__ out, size_t ostride) {
    __shared__ double2 red[RED_THREADS];
    const double2* p = partial + (size_t)blockIdx.x * bpm * nout;
    double2* o = out + (size_t)ml.idx[blockIdx.x] * ostride;
    for (int i = 0; i < nout; ++i) {
        double2 acc = make_double2(0, 0);
        for (int b = threadIdx.x; b < bpm; b += blockDim.x) acc = acc + p[(size_t)b * nout + i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) o[i] = red[0];
        __syncthreads();
    }
}

struct Coefs {
    double2 c[64];
};
// x += sum_i c_i Z_i  (Z of type ZT; x of type XT, summed in XT's precision)
template <typename ZT, typename XT>
__global__ void k_combine(size_t N, int nvec, const ZT* __restrict__ Z, size_t ld, Coefs cf, XT* __restrict__ x) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        XT acc = x[k];
        for (int i = 0; i < nvec; ++i) acc = cfma(vt_of<XT>(cf.c[i]), ccast<XT>(__ldg(&Z[(size_t)i * ld + k])), acc);
        x[k] = acc;
    }
}

// y = a x + b y  (x of type XT, y of type YT, arithmetic in YT's precision)
template <typename XT, typename YT>
__global__ void k_axpby(size_t N, double2 a, const XT* __restrict__ x, double2 b, YT* __restrict__ y) {
    const YT aa = vt_of<YT>(a), bb = vt_of<YT>(b);
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
        y[k] = aa * ccast<YT>(x[k]) + bb * y[k];
}

// y = x, converting between the vector types
template <typename XT, typename YT>
__global__ void k_copy(size_t N, const XT* __restrict__ x, YT* __restrict__ y) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
        y[k] = ccast<YT>(x[k]);
}

template <typename VT>
__global__ void k_zero(size_t N, VT* __restrict__ y) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
        y[k] = czero<VT>();
}

// mismatches of the integer-pipe conversions against the hardware ones (NaN: NaN-ness only)
__global__ void k_check_conv(long long n, const double* __restrict__ d, const float* __restrict__ f,
                             unsigned long long* __restrict__ bad) {
    unsigned long long cnt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float a = d2f_rn(d[i]), h = __double2float_rn(d[i]);
        if (isnan(h) ? !isnan(a) : __float_as_uint(a) != __float_as_uint(h)) ++cnt;
        const double a2 = f2d(f[i]), h2 = (double)f[i];
        if (isnan(h2) ? !isnan(a2) : __double_as_longlong(a2) != __double_as_longlong(h2)) ++cnt;
    }
    if (cnt) atomicAdd(bad, cnt);
}

}  // namespace

extern "C" int ls_check_conversions(const double* d, const float* f, long long n, unsigned long long* mismatches) {
    if (!d || !f || !mismatches || n < 0) return LS_EINVAL;
    unsigned long long* dev = nullptr;
    LS_CUDA(cudaMalloc(&dev, sizeof(unsigned long long)));
    int rc = LS_OK;
    if (cudaMemset(dev, 0, sizeof(unsigned long long)) != cudaSuccess) rc = LS_ECUDA;
    if (rc == LS_OK && n > 0) {
        k_check_conv<<<608, 256>>>(n, d, f, dev);
        if (cudaPeekAtLastError() != cudaSuccess) rc = LS_ECUDA;
    }
    if (rc == LS_OK && cudaMemcpy(mismatches, dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = LS_ECUDA;
    cudaFree(dev);
    return rc;
}

template <typename R>
int stencil_launch(ls_handle* h, int dir, int mode, const double2* v, const double2* g, double2* y, int nb) {
    const int n = h->n;
    const size_t N = (size_t)n * n;
    (void)N;
    const dim3 grid((unsigned)((n + kStX - 1) / kStX), (unsigned)((n + kStZ - 1) / kStZ), nb);
    const dim3 block(kStX, 256 / kStX);
    const double* m = dir == 0 ? h->m64 : h->mT64;
    const StencilTables* tab = h->dtabs + dir;
    if (mode == 0) LS_LAUNCH(h, (k_stencil<0, R>), grid, block, 0, n, tab, m, v, g, y);
    else if (mode == 1) LS_LAUNCH(h, (k_stencil<1, R>), grid, block, 0, n, tab, m, v, g, y);
    else LS_LAUNCH(h, (k_stencil<2, R>), grid, block, 0, n, tab, m, v, g, y);
    return LS_OK;
}

// FP64 arithmetic (the operator entry points A and C of the ABI)
int ls_stencil_apply64(ls_handle* h, int dir, int mode, const double2* v, const double2* g, double2* y) {
    return stencil_launch<double>(h, dir, mode, v, g, y, 1);
}

// Inside the solve: FP32 arithmetic in mixed precision (the stencils feed only the
// preconditioner, Algorithm 3 and Algorithm 2), FP64 otherwise.
int ls_stencil_apply_b(ls_handle* h, int dir, int mode, const double2* v, const double2* g, double2* y, int nb) {
    if (h->prec == LS_MIXED) return stencil_launch<float>(h, dir, mode, v, g, y, nb);
    return stencil_launch<double>(h, dir, mode, v, g, y, nb);
}

// Algorithm 2's refinement residual e = g - C u1 in mixed precision, u1 and e in FP32
// storage (their values are FP32 either way); FP32 coefficients and sums.
int ls_stencil_refine_f32(ls_handle* h, int dir, const float2* v, const float2* g, float2* y, int nb) {
    const int n = h->n;
    const dim3 grid((unsigned)((n + kStX - 1) / kStX), (unsigned)((n + kStZ - 1) / kStZ), nb);
    const dim3 block(kStX, 256 / kStX);
    const double* m = dir == 0 ? h->m64 : h->mT64;
    LS_LAUNCH(h, (k_stencil<2, float, float2, float2, float2>), grid, block, 0, n, h->dtabs + dir, m, v, g, y);
    return LS_OK;
}

// y = A v (mode 0) or C v (mode 1) with FP32 vectors and FP32 arithmetic (the mixed
// precision inner solve's operator)
int ls_stencil_apply_f32(ls_handle* h, int dir, int mode, const float2* v, float2* y) {
    const int n = h->n;
    const dim3 grid((unsigned)((n + kStX - 1) / kStX), (unsigned)((n + kStZ - 1) / kStZ), 1);
    const dim3 block(kStX, 256 / kStX);
    const double* m = dir == 0 ? h->m64 : h->mT64;
    const StencilTables* tab = h->dtabs + dir;
    const double2* none = nullptr;
    if (mode == 0) LS_LAUNCH(h, (k_stencil<0, float, float2, float2>), grid, block, 0, n, tab, m, v, none, y);
    else LS_LAUNCH(h, (k_stencil<1, float, float2, float2>), grid, block, 0, n, tab, m, v, none, y);
    return LS_OK;
}

int ls_stencil_apply(ls_handle* h, int dir, int mode, const double2* v, const double2* g, double2* y) {
    return ls_stencil_apply_b(h, dir, mode, v, g, y, 1);
}

int ls_transpose64_b(ls_handle* h, const double2* a, double2* b, int nb) {
    const int n = h->n;
    dim3 grid((n + 31) / 32, (n + 31) / 32, nb), block(32, 8);
    LS_LAUNCH(h, k_transpose, grid, block, 0, n, a, b);
    return LS_OK;
}

int ls_transpose64(ls_handle* h, const double2* a, double2* b) { return ls_transpose64_b(h, a, b, 1); }

int ls_transpose_real(ls_handle* h, const double* a, double* b) {
    const int n = h->n;
    dim3 grid((n + 31) / 32, (n + 31) / 32), block(32, 8);
    LS_LAUNCH(h, k_transpose_real, grid, block, 0, n, a, b);
    return LS_OK;
}

static int red_reserve(ls_handle* h, size_t cnt) {
    if (h->red_cap >= cnt) return LS_OK;
    if (h->red) cudaFree(h->red);
    if (h->red_host) cudaFreeHost(h->red_host);
    h->red = nullptr;
    h->red_host = nullptr;
    LS_CUDA(cudaMalloc(&h->red, cnt * sizeof(double2)));
    LS_CUDA(cudaMallocHost(&h->red_host, cnt * sizeof(double2)));
    h->red_cap = cnt;
    return LS_OK;
}

// dots into device memory out_dev[0..nvec)
template <typename VT>
int vec_dots_dev(ls_handle* h, int nvec, const VT* V, size_t ld, const VT* w, double2* out_dev) {
    const size_t N = (size_t)h->n * h->n;
    LS_TRY(red_reserve(h, (size_t)RED_BLOCKS * 64 + 256));
    double2* partial = reinterpret_cast<double2*>(h->red);
    LS_LAUNCH(h, k_dots<VT>, RED_BLOCKS, RED_THREADS, 0, N, nvec, V, ld, w, partial);
    LS_LAUNCH(h, k_dots_final, 1, RED_THREADS, 0, RED_BLOCKS, nvec, partial, out_dev);
    return LS_OK;
}



template <typename ZT, typename XT>
int vec_combine(ls_handle* h, int nvec, const ZT* Z, size_t ld, const double2* coef_host, XT* x) {
    const size_t N = (size_t)h->n * h->n;
    for (int base = 0; base < nvec; base += 64) {
        Coefs cf;
        const int cnt = nvec - base < 64 ? nvec - base : 64;
        for (int i = 0; i < cnt; ++i) cf.c[i] = coef_host[base + i];
        LS_LAUNCH(h, (k_combine<ZT, XT>), RED_BLOCKS, RED_THREADS, 0, N, cnt, Z + (size_t)base * ld, ld, cf, x);
    }
    return LS_OK;
}

// The fused pass with G the smallest of 2, 4, 8, 16 that holds nvec directions: the
// registers (G values of V and G sums per thread) and so the resident warps that keep
// loads in flight follow the step's own size.
template <typename VT, int G>
int orth_launch(ls_handle* h, int mode, dim3 grid, int nvec, const VT* V, size_t ld, size_t mstride,
                const double2* coef, size_t cstride, VT* w, const MemberList& ml, double2* partial) {
    const size_t N = (size_t)h->n * h->n;
    switch (mode) {
        case 0:
            LS_LAUNCH(h, (k_orth<VT, G, 0>), grid, RED_THREADS, 0, N, nvec, V, ld, mstride, coef, cstride, w, ml, partial);
            break;
        case 1:
            LS_LAUNCH(h, (k_orth<VT, G, 1>), grid, RED_THREADS, 0, N, nvec, V, ld, mstride, coef, cstride, w, ml, partial);
            break;
        case 2:
            LS_LAUNCH(h, (k_orth<VT, G, 2>), grid, RED_THREADS, 0, N, nvec, V, ld, mstride, coef, cstride, w, ml, partial);
            break;
        default:
            LS_LAUNCH(h, (k_orth<VT, G, 3>), grid, RED_THREADS, 0, N, 0, V, ld, mstride, coef, cstride, w, ml, partial);
            break;
    }
    return LS_OK;
}

// The pass of `mode` for members members[0..cnt) of a batch (member m: V + m * mstride,
// w + m * mstride, coef + m * cstride, out + m * ostride); RED_BLOCKS blocks shared out
// among them.  More directions than one pass holds: the separate kernels, member by member.
template <typename VT>
int vec_orth_b(ls_handle* h, int mode, int nvec, const VT* V, size_t ld, size_t mstride, const double2* coef,
               size_t cstride, VT* w, const int* members, int cnt, double2* out, size_t ostride) {
    const size_t N = (size_t)h->n * h->n;
    constexpr int GMAX = sizeof(VT) == 8 ? 16 : 8;
    if (mode < 0 || mode > 3 || cnt < 0 || cnt > LS_MAX_BATCH || (mode < 3 && nvec < 1)) return LS_EINVAL;
    if (cnt == 0) return LS_OK;
    if (mode < 3 && nvec > GMAX) {
        for (int c = 0; c < cnt; ++c) {
            const size_t mo = (size_t)members[c] * mstride;
            double2* o = out + (size_t)members[c] * ostride;
            if (mode == 0) {
                LS_TRY(vec_dots_dev(h, nvec, V + mo, ld, (const VT*)(w + mo), o));
                continue;
            }
            LS_LAUNCH(h, k_update<VT>, RED_BLOCKS, RED_THREADS, 0, N, nvec, V + mo, ld,
                      coef + (size_t)members[c] * cstride, w + mo);
            if (mode == 1) LS_TRY(vec_dots_dev(h, nvec, V + mo, ld, (const VT*)(w + mo), o));
            else LS_TRY(vec_dots_dev(h, 1, (const VT*)(w + mo), 0, (const VT*)(w + mo), o));
        }
        return LS_OK;
    }
    MemberList ml;
    for (int c = 0; c < cnt; ++c) ml.idx[c] = members[c];
    const int bpm = RED_BLOCKS / cnt;   // >= 9: cnt <= LS_MAX_BATCH
    const dim3 grid((unsigned)bpm, (unsigned)cnt);
    LS_TRY(red_reserve(h, (size_t)RED_BLOCKS * 64 + 256));
    double2* partial = reinterpret_cast<double2*>(h->red);
    if (mode == 3 || nvec <= 2) LS_TRY((orth_launch<VT, 2>(h, mode, grid, nvec, V, ld, mstride, coef, cstride, w, ml, partial)));
    else if (nvec <= 4) LS_TRY((orth_launch<VT, 4>(h, mode, grid, nvec, V, ld, mstride, coef, cstride, w, ml, partial)));
    else if (nvec <= 8) LS_TRY((orth_launch<VT, 8>(h, mode, grid, nvec, V, ld, mstride, coef, cstride, w, ml, partial)));
    else if constexpr (GMAX >= 16)
        LS_TRY((orth_launch<VT, 16>(h, mode, grid, nvec, V, ld, mstride, coef, cstride, w, ml, partial)));
    LS_LAUNCH(h, k_orth_final, (unsigned)cnt, RED_THREADS, 0, bpm, mode >= 2 ? 1 : nvec, partial, ml, out, ostride);
    return LS_OK;
}

// ||w_m|| for the members members[0..cnt) (member m at w + m * mstride) into out[m]: one
// pass over all of them and one device->host read.  A NaN or Inf in a member's vector
// gives a non-finite norm.
template <typename VT>
int vec_norms_b(ls_handle* h, const VT* w, size_t mstride, const int* members, int cnt, double* out) {
    if (cnt < 0 || cnt > LS_MAX_BATCH) return LS_EINVAL;
    if (cnt == 0) return LS_OK;
    LS_TRY(red_reserve(h, (size_t)RED_BLOCKS * 64 + 256));
    double2* outd = reinterpret_cast<double2*>(h->red) + (size_t)RED_BLOCKS * 64;
    int top = 0;
    for (int c = 0; c < cnt; ++c) top = members[c] + 1 > top ? members[c] + 1 : top;
    LS_TRY(vec_orth_b(h, 3, 0, (const VT*)nullptr, 0, mstride, nullptr, 0, const_cast<VT*>(w), members, cnt, outd, 1));
    LS_CUDA(cudaMemcpyAsync(h->red_host, outd, sizeof(double2) * top, cudaMemcpyDeviceToHost, h->stream));
    LS_CUDA(cudaStreamSynchronize(h->stream));
    const double2* hr = reinterpret_cast<const double2*>(h->red_host);
    for (int c = 0; c < cnt; ++c) {
        const double d = hr[members[c]].x;
        out[members[c]] = d >= 0 ? sqrt(d) : (d < 0 ? 0.0 : d);
    }
    return LS_OK;
}

int ls_vec_orth_b(ls_handle* h, int mode, int nvec, const double2* V, size_t ld, size_t mstride, const double2* coef,
                  size_t cstride, double2* w, const int* members, int cnt, double2* out, size_t ostride) {
    return vec_orth_b(h, mode, nvec, V, ld, mstride, coef, cstride, w, members, cnt, out, ostride);
}
int ls_vec_orth_b(ls_handle* h, int mode, int nvec, const float2* V, size_t ld, size_t mstride, const double2* coef,
                  size_t cstride, float2* w, const int* members, int cnt, double2* out, size_t ostride) {
    return vec_orth_b(h, mode, nvec, V, ld, mstride, coef, cstride, w, members, cnt, out, ostride);
}
int ls_vec_norms_b(ls_handle* h, const double2* w, size_t mstride, const int* members, int cnt, double* out) {
    return vec_norms_b(h, w, mstride, members, cnt, out);
}
int ls_vec_norms_b(ls_handle* h, const float2* w, size_t mstride, const int* members, int cnt, double* out) {
    return vec_norms_b(h, w, mstride, members, cnt, out);
}

int ls_vec_combine(ls_handle* h, int nvec, const double2* Z, size_t ld, const double2* coef_host, double2* x) {
    return vec_combine(h, nvec, Z, ld, coef_host, x);
}
int ls_vec_combine(ls_handle* h, int nvec, const float2* Z, size_t ld, const double2* coef_host, float2* x) {
    return vec_combine(h, nvec, Z, ld, coef_host, x);
}
int ls_vec_axpby(ls_handle* h, double2 a, const double2* x, double2 b, double2* y) {
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_axpby<double2, double2>), RED_BLOCKS, RED_THREADS, 0, N, a, x, b, y);
    return LS_OK;
}
int ls_vec_axpby(ls_handle* h, double2 a, const float2* x, double2 b, float2* y) {
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_axpby<float2, float2>), RED_BLOCKS, RED_THREADS, 0, N, a, x, b, y);
    return LS_OK;
}
int ls_vec_axpby(ls_handle* h, double2 a, const float2* x, double2 b, double2* y) {   // FP64 y += FP32 x
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_axpby<float2, double2>), RED_BLOCKS, RED_THREADS, 0, N, a, x, b, y);
    return LS_OK;
}
int ls_vec_copy(ls_handle* h, const double2* x, double2* y) {
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_copy<double2, double2>), RED_BLOCKS, RED_THREADS, 0, N, x, y);
    return LS_OK;
}
int ls_vec_copy(ls_handle* h, const float2* x, float2* y) {
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_copy<float2, float2>), RED_BLOCKS, RED_THREADS, 0, N, x, y);
    return LS_OK;
}
int ls_vec_copy(ls_handle* h, const double2* x, float2* y) {   // rounded to FP32
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_copy<double2, float2>), RED_BLOCKS, RED_THREADS, 0, N, x, y);
    return LS_OK;
}
int ls_vec_copy(ls_handle* h, const float2* x, double2* y) {   // widened (exact)
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, (k_copy<float2, double2>), RED_BLOCKS, RED_THREADS, 0, N, x, y);
    return LS_OK;
}
int ls_vec_zero(ls_handle* h, double2* y) {
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, k_zero<double2>, RED_BLOCKS, RED_THREADS, 0, N, y);
    return LS_OK;
}
int ls_vec_zero(ls_handle* h, float2* y) {
    const size_t N = (size_t)h->n * h->n;
    LS_LAUNCH(h, k_zero<float2>, RED_BLOCKS, RED_THREADS, 0, N, y);
    return LS_OK;
}
