// ls_unet.cu -- the learned preconditioner step: a BF16 convolutional U-Net
// trained and applied on the GPU by this library's own kernels.
//
// The paper's outer iteration is flexible GMRES (Sec. 6), whose preconditioner
// may change from step to step; the network is one more right-preconditioner
// stage there (see ls_krylov.cu).  Architecture (fixed; also in the oracle):
//   input (Re r / s, Im r / s, m), s = RMS of r, padded to 16 channels;
//   encoder levels l = 0..L-1 with c_l = c0 2^l channels: two 3x3 conv + ReLU,
//   2x2 average pool between levels; decoder levels l = L-2..0: nearest 2x
//   upsampling, 3x3 conv to c_l + ReLU, concatenation with the encoder's level-l
//   output, two 3x3 conv + ReLU; head: 3x3 conv to 2 channels (padded to 16).
//
// Data: activations NHWC in BF16 (channels innermost, multiples of 16); the
// encoder's level-l output is written straight into the upper half of the
// level-l concatenation buffer, so concatenation costs nothing.  Weights:
// FP32 master copy + Adam moments; BF16 copies [cout][tap][cin] for the forward
// convolution and [cin][8 - tap][cout] for the backward-data convolution.
//
// Convolutions are implicit GEMMs on the tensor cores with FP32 accumulation.
// Forward and backward-data (M = pixels, N = output channels, K = 9 x input
// channels) run on the fifth-generation tensor cores (k_conv_umma): tiles of 128
// pixels, the 3x3 neighbourhood gathered into 128-byte-swizzled shared memory while
// the previous K-slice's tcgen05.mma (kind::f16, BF16 operands) run, the
// accumulator in tensor memory, bias and ReLU applied on its way out.
// Backward-weights (M = output channels, N = 9 x input channels, K = pixels, split
// over pixel chunks and reduced with FP32 atomics) uses WMMA bf16 16x16x16.
#include <mma.h>

#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "ls_internal.cuh"
#include "ls_umma.cuh"

using bf16 = __nv_bfloat16;

namespace {

using namespace nvcuda;

// ------------------------------------------------------------------ kernels
struct View {  // NHWC channel slice: pixel p, channel c at p * stride + off + c
    bf16* p;
    int stride, off, c;
};

struct ConvArgs {
    const bf16* x;
    int xs, xo, cin;    // input view
    const bf16* w;      // [cout][9][cin]
    const float* bias;  // [cout] or null
    bf16* y;
    int ys, yo, cout;   // output view
    int H, W, M;        // M = nb * H * W (multiple of 64)
    int relu;
};

constexpr int kConvThreads = 128;

// y[p][n] = act(bias[n] + sum_{tap, c} w[n][tap][c] x[p + shift(tap)][c])
template <int BN>
__global__ void __launch_bounds__(kConvThreads) k_conv_fwd(ConvArgs a) {
    constexpr int BM = 64, BK = 32, LDA = BK + 8, LDB = BK + 8, LDC = BN + 4;
    __shared__ __align__(32) bf16 As[BM * LDA];
    __shared__ __align__(32) bf16 Bs[BN * LDB];
    __shared__ __align__(32) float Cs[BM * LDC];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int warp = threadIdx.x >> 5;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[BN / 16];
#pragma unroll
    for (int f = 0; f < BN / 16; ++f) wmma::fill_fragment(acc[f], 0.0f);
    const int K = 9 * a.cin, HW = a.H * a.W;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int v = threadIdx.x; v < BM * BK / 8; v += kConvThreads) {
            const int mm = v / (BK / 8), kv = v % (BK / 8);
            const int k = k0 + kv * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (k < K) {
                const int tap = k / a.cin, ci = k % a.cin;
                const int p = m0 + mm;
                const int b = p / HW, rem = p % HW, yy = rem / a.W, xx = rem % a.W;
                const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
                if (sy >= 0 && sy < a.H && sx >= 0 && sx < a.W)
                    val = *reinterpret_cast<const uint4*>(a.x + (size_t)(b * HW + sy * a.W + sx) * a.xs + a.xo + ci);
            }
            *reinterpret_cast<uint4*>(&As[mm * LDA + kv * 8]) = val;
        }
        for (int v = threadIdx.x; v < BN * BK / 8; v += kConvThreads) {
            const int nn = v / (BK / 8), kv = v % (BK / 8);
            uint4 val = make_uint4(0, 0, 0, 0);
            if (k0 + kv * 8 < K) val = *reinterpret_cast<const uint4*>(a.w + (size_t)(n0 + nn) * K + k0 + kv * 8);
            *reinterpret_cast<uint4*>(&Bs[nn * LDB + kv * 8]) = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> fa;
            wmma::load_matrix_sync(fa, As + warp * 16 * LDA + kk, LDA);
#pragma unroll
            for (int f = 0; f < BN / 16; ++f) {
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::col_major> fb;
                wmma::load_matrix_sync(fb, Bs + f * 16 * LDB + kk, LDB);
                wmma::mma_sync(acc[f], fa, fb, acc[f]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int f = 0; f < BN / 16; ++f)
        wmma::store_matrix_sync(Cs + warp * 16 * LDC + f * 16, acc[f], LDC, wmma::mem_row_major);
    __syncthreads();
    for (int e = threadIdx.x; e < BM * BN; e += kConvThreads) {
        const int mm = e / BN, nn = e % BN;
        float v = Cs[mm * LDC + nn] + (a.bias ? a.bias[n0 + nn] : 0.0f);
        if (a.relu) v = fmaxf(v, 0.0f);
        a.y[(size_t)(m0 + mm) * a.ys + a.yo + n0 + nn] = __float2bfloat16(v);
    }
}

// The same convolution on the fifth-generation tensor cores: a CTA of 128 threads
// computes 128 pixels x BN output channels (BN = cout <= 256).  K = 9 cin runs in
// atoms of 64 (one 128-byte swizzled row per pixel or channel).  Each atom's A (the
// gathered 3x3 neighbourhoods, 16-byte chunks of 8 channels) and B (weights
// [cout][tap][cin], K-major) go straight from global to one of kCvStages shared-memory
// stages by asynchronous 16-byte copies (cp.async, zero-filled outside the image),
// kCvStages - 1 atoms ahead of the tensor cores; once an atom has landed, thread 0
// issues its four K = 16 MMAs (kind::f16, BF16 operands) and commits them to the
// stage's barrier, which the copies into that stage wait on.  A thread always moves
// chunk (tid mod 8) of its 8 pixels, so their coordinates are computed once.  Waits
// are bounded (1 s); on expiry the tile is written as NaN and the device counter
// ls_device_timeouts counts it.
__device__ unsigned g_conv_timeouts;
constexpr int kCvThreads = 128, kCvStages = 4;
template <int BN>
constexpr size_t conv_umma_smem() {
    return 1024 + (size_t)kCvStages * (128 * 128 + BN * 128) + 8 * (kCvStages + 1) + 16;
}
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool valid) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}
template <int BN>
__global__ void __launch_bounds__(kCvThreads) k_conv_umma(ConvArgs a) {
    using namespace umma;
    constexpr unsigned ABYTES = 128 * 128, BBYTES = BN * 128, STAGE = ABYTES + BBYTES;
    constexpr int TCOLS = BN < 32 ? 32 : BN;
    constexpr int S = kCvStages;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    auto* sbar = reinterpret_cast<unsigned long long*>(base + S * STAGE);
    auto* done = sbar + S;
    unsigned* tslot = reinterpret_cast<unsigned*>(done + 1);
    int* failed = reinterpret_cast<int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int K = 9 * a.cin, HW = a.H * a.W, NK = (K + 63) / 64;
    // this thread's 8 pixels (rows tid/8 + 16u, u < 8: the 128 rows of the tile, each once
    // per chunk) and chunk c = tid % 8 of every atom
    constexpr int RPT = 128 * 8 / kCvThreads;   // chunks (= rows) per thread: 8
    static_assert(RPT * 16 == 128, "rows tid / 8 + 16 u cover the tile once per chunk");
    const int c = tid & 7;
    int pb[RPT], py[RPT], px[RPT];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int p = m0 + (tid >> 3) + 16 * u;
        const int bb = p / HW, rem = p - bb * HW;
        pb[u] = p < a.M ? bb : -1;
        py[u] = rem / a.W;
        px[u] = rem - py[u] * a.W;
    }
    if (tid == 0) {
        *failed = 0;
        for (int i = 0; i < S; ++i) bar_init(&sbar[i], 1);
        bar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, TCOLS);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = *tslot;
    constexpr unsigned ID = idesc(1u, 128, BN);
    auto issue = [&](int ka) {   // asynchronous copies of atom ka into stage ka % S
        unsigned char* As = base + (size_t)(ka % S) * STAGE;
        unsigned char* Bs = As + ABYTES;
        const int k = ka * 64 + c * 8;
        const bool kin = k < K;
        const int tap = kin ? k / a.cin : 0, ci = kin ? k - tap * a.cin : 0;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
            const int row = (tid >> 3) + 16 * u;
            const int sy = py[u] + dy, sx = px[u] + dx;
            const bool ok = kin && pb[u] >= 0 && sy >= 0 && sy < a.H && sx >= 0 && sx < a.W;
            const bf16* src = ok ? a.x + (size_t)(pb[u] * HW + sy * a.W + sx) * a.xs + a.xo + ci : a.x;
            cp_async16_zfill(As + swz16(row, c), src, ok);
        }
        for (int v = tid; v < BN * 8; v += kCvThreads) {
            const int row = v >> 3, cc = v & 7, kk = ka * 64 + cc * 8;
            const bool ok = kk < K;
            cp_async16_zfill(Bs + swz16(row, cc), ok ? a.w + (size_t)(n0 + row) * K + kk : a.w, ok);
        }
    };
#pragma unroll 1
    for (int ka = 0; ka < S - 1 && ka < NK; ++ka) {
        issue(ka);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
#pragma unroll 1
    for (int ka = 0; ka < NK; ++ka) {
        // atom ka has landed once at most S - 2 newer groups are still pending
        asm volatile("cp.async.wait_group %0;\n" ::"n"(S - 2) : "memory");
        fence_async_smem();
        __syncthreads();
        if (*failed) break;
        if (tid == 0) {
            fence_after();
            const unsigned aa = su32(base + (size_t)(ka % S) * STAGE), bb = aa + ABYTES;
#pragma unroll
            for (int k16 = 0; k16 < 4; ++k16)
                if (ka * 64 + k16 * 16 < K)
                    mma_bf16(tmem, sdesc(aa + 32u * k16), sdesc(bb + 32u * k16), ID, (ka | k16) ? 1u : 0u);
            mma_commit(&sbar[ka % S]);
        }
        // refill the stage that atom ka - 1 used, once its MMAs are done
        const int kn = ka + S - 1;
        if (kn < NK) {
            if (ka >= 1 && !bar_wait(&sbar[(ka - 1) % S], (unsigned)((ka - 1) / S) & 1u)) atomicOr(failed, 1);
            issue(kn);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");   // (possibly empty) group per step
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (tid == 0) mma_commit(done);
    if (!bar_wait(done, 0)) atomicOr(failed, 2);
    fence_after();
    __syncthreads();
    const bool bad = *failed != 0;
    if (bad && tid == 0) atomicAdd(&g_conv_timeouts, 1u);
    // epilogue: warp w holds pixels m0 + 32 w + lane (TMEM lanes 32 w ..)
    const int r = 32 * warp + lane, p = m0 + r;
    const unsigned lrow = tmem + ((unsigned)(32 * warp) << 16);
#pragma unroll 1
    for (int cc = 0; cc < BN; cc += 8) {
        float v[8];
        tmem_ld8(lrow + (unsigned)cc, v);
        if (p < a.M) {
            __align__(16) bf16 o[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float t = bad ? __int_as_float(0x7fc00000) : v[e] + (a.bias ? a.bias[n0 + cc + e] : 0.0f);
                if (a.relu) t = fmaxf(t, 0.0f);
                o[e] = __float2bfloat16(t);
            }
            *reinterpret_cast<uint4*>(a.y + (size_t)p * a.ys + a.yo + n0 + cc) = *reinterpret_cast<const uint4*>(o);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

struct WgradArgs {
    const bf16* dy;
    int ds, dof, cout;  // dL/d(pre-activation) view
    const bf16* x;
    int xs, xo, cin;    // layer input view
    float* dw;          // [cout][9][cin], accumulated
    int H, W, M, chunk; // pixel chunk per CTA (multiple of 32)
};

// dw[m][n] += sum_{p in chunk} dy[p][m] * x[p + shift(tap(n))][ci(n)],  n = tap * cin + ci
template <int BM>
__global__ void __launch_bounds__(kConvThreads) k_conv_wgrad(WgradArgs a) {
    constexpr int BN = 64, BK = 32, LDA = BM + 8, LDB = BN + 8, LDC = BN + 4;
    constexpr int FR = BM / 16;             // fragment rows
    constexpr int FPW = FR * (BN / 16) / 4; // fragments per warp
    __shared__ __align__(32) bf16 As[BK * LDA];   // As[k][m]: column-major A
    __shared__ __align__(32) bf16 Bs[BK * LDB];   // Bs[k][n]: row-major B
    __shared__ __align__(32) float Cs[BM * LDC];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int pbeg = blockIdx.z * a.chunk, pend = min(a.M, pbeg + a.chunk);
    const int warp = threadIdx.x >> 5;
    const int K9 = 9 * a.cin, HW = a.H * a.W;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[FPW];
#pragma unroll
    for (int f = 0; f < FPW; ++f) wmma::fill_fragment(acc[f], 0.0f);
    for (int p0 = pbeg; p0 < pend; p0 += BK) {
        for (int v = threadIdx.x; v < BK * BM / 8; v += kConvThreads) {
            const int kp = v / (BM / 8), mv = v % (BM / 8);
            const int p = p0 + kp;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (p < pend) val = *reinterpret_cast<const uint4*>(a.dy + (size_t)p * a.ds + a.dof + m0 + mv * 8);
            *reinterpret_cast<uint4*>(&As[kp * LDA + mv * 8]) = val;
        }
        for (int v = threadIdx.x; v < BK * BN / 8; v += kConvThreads) {
            const int kp = v / (BN / 8), nv = v % (BN / 8);
            const int p = p0 + kp, n = n0 + nv * 8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (p < pend && n < K9) {
                const int tap = n / a.cin, ci = n % a.cin;
                const int b = p / HW, rem = p % HW, yy = rem / a.W, xx = rem % a.W;
                const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
                if (sy >= 0 && sy < a.H && sx >= 0 && sx < a.W)
                    val = *reinterpret_cast<const uint4*>(a.x + (size_t)(b * HW + sy * a.W + sx) * a.xs + a.xo + ci);
            }
            *reinterpret_cast<uint4*>(&Bs[kp * LDB + nv * 8]) = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
#pragma unroll
            for (int f = 0; f < FPW; ++f) {
                const int fid = warp * FPW + f;
                const int fr = fid % FR, fc = fid / FR;
                wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> fa;
                wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb;
                wmma::load_matrix_sync(fa, As + kk * LDA + fr * 16, LDA);
                wmma::load_matrix_sync(fb, Bs + kk * LDB + fc * 16, LDB);
                wmma::mma_sync(acc[f], fa, fb, acc[f]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int f = 0; f < FPW; ++f) {
        const int fid = warp * FPW + f;
        const int fr = fid % FR, fc = fid / FR;
        wmma::store_matrix_sync(Cs + fr * 16 * LDC + fc * 16, acc[f], LDC, wmma::mem_row_major);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BM * BN; e += kConvThreads) {
        const int mm = e / BN, nn = e % BN;
        if (n0 + nn < K9) atomicAdd(&a.dw[(size_t)(m0 + mm) * K9 + n0 + nn], Cs[mm * LDC + nn]);
    }
}

// db[c] += sum over a pixel chunk of dy[p][c]
__global__ void k_bias_grad(const bf16* __restrict__ dy, int ds, int dof, int cout, int M, int chunk,
                            float* __restrict__ db) {
    const int c = threadIdx.x;
    if (c >= cout) return;
    const int pbeg = blockIdx.x * chunk, pend = min(M, pbeg + chunk);
    float s = 0.0f;
    for (int p = pbeg; p < pend; ++p) s += __bfloat162float(dy[(size_t)p * ds + dof + c]);
    atomicAdd(&db[c], s);
}

// out = (y > 0) ? g : 0 on matching views (out dense, c channels)
__global__ void k_relu_mask(size_t M, int c, const bf16* __restrict__ g, int gs, int go, const bf16* __restrict__ y,
                            int ys, int yo, bf16* __restrict__ out) {
    const size_t n = M * c;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / c;
        const int k = (int)(i % c);
        const float yv = __bfloat162float(y[p * ys + yo + k]);
        out[i] = yv > 0.0f ? g[p * gs + go + k] : __float2bfloat16(0.0f);
    }
}

// 2x2 average pool: in (nb, H, W) view -> out dense (nb, H/2, W/2, c)
__global__ void k_pool(int nb, int H, int W, int c, const bf16* __restrict__ x, int xs, int xo, bf16* __restrict__ y) {
    const int H2 = H / 2, W2 = W / 2;
    const size_t n = (size_t)nb * H2 * W2 * c;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % c);
        const size_t q = i / c;
        const int xx = (int)(q % W2), yy = (int)((q / W2) % H2), b = (int)(q / ((size_t)W2 * H2));
        float s = 0.0f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                s += __bfloat162float(x[((size_t)b * H * W + (size_t)(2 * yy + dy) * W + 2 * xx + dx) * xs + xo + k]);
        y[i] = __float2bfloat16(0.25f * s);
    }
}

// gradient through the pool, plus the skip gradient: out (nb, H, W, c) dense =
// skip view + g2[p / 2] / 4
__global__ void k_pool_bwd_add(int nb, int H, int W, int c, const bf16* __restrict__ g2, const bf16* __restrict__ sk,
                               int ss, int so, bf16* __restrict__ out) {
    const size_t n = (size_t)nb * H * W * c;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % c);
        const size_t q = i / c;
        const int xx = (int)(q % W), yy = (int)((q / W) % H), b = (int)(q / ((size_t)W * H));
        const size_t q2 = (size_t)b * (H / 2) * (W / 2) + (size_t)(yy / 2) * (W / 2) + xx / 2;
        float v = 0.25f * __bfloat162float(g2[q2 * c + k]);
        if (sk) v += __bfloat162float(sk[q * ss + so + k]);
        out[i] = __float2bfloat16(v);
    }
}

// nearest 2x upsampling: in (nb, H/2, W/2) view -> out dense (nb, H, W, c)
__global__ void k_up(int nb, int H, int W, int c, const bf16* __restrict__ x, int xs, int xo, bf16* __restrict__ y) {
    const size_t n = (size_t)nb * H * W * c;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % c);
        const size_t q = i / c;
        const int xx = (int)(q % W), yy = (int)((q / W) % H), b = (int)(q / ((size_t)W * H));
        const size_t q2 = (size_t)b * (H / 2) * (W / 2) + (size_t)(yy / 2) * (W / 2) + xx / 2;
        y[i] = x[q2 * xs + xo + k];
    }
}

// gradient of the upsampling: out (nb, H/2, W/2, c) dense = sum of the 4 children of g (dense, H x W)
__global__ void k_up_bwd(int nb, int H, int W, int c, const bf16* __restrict__ g, bf16* __restrict__ out) {
    const int H2 = H / 2, W2 = W / 2;
    const size_t n = (size_t)nb * H2 * W2 * c;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % c);
        const size_t q = i / c;
        const int xx = (int)(q % W2), yy = (int)((q / W2) % H2), b = (int)(q / ((size_t)W2 * H2));
        float s = 0.0f;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                s += __bfloat162float(g[((size_t)b * H * W + (size_t)(2 * yy + dy) * W + 2 * xx + dx) * c + k]);
        out[i] = __float2bfloat16(s);
    }
}

// sum_b |r_b|^2 per sample (FP64); sums zeroed by the caller
__global__ void k_sumsq(size_t HW, const double2* __restrict__ r, double* __restrict__ sums) {
    __shared__ double red[256];
    const int b = blockIdx.y;
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = r[(size_t)b * HW + i];
        acc += v.x * v.x + v.y * v.y;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&sums[b], red[0]);
}

// x[p] = (Re r / s, Im r / s, m, 0 ...) with 16 channels; s_b = sqrt(sums_b / HW) (1 if 0)
__global__ void k_net_input(size_t HW, int nb, const double2* __restrict__ r, const double* __restrict__ m,
                            const double* __restrict__ sums, bf16* __restrict__ x) {
    const size_t n = HW * nb;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / HW);
        double s = sqrt(sums[b] / (double)HW);
        if (!(s > 0.0)) s = 1.0;
        const double2 v = r[i];
        bf16* o = x + i * 16;
        o[0] = __float2bfloat16((float)(v.x / s));
        o[1] = __float2bfloat16((float)(v.y / s));
        o[2] = __float2bfloat16((float)m[i]);
#pragma unroll
        for (int k = 3; k < 16; ++k) o[k] = __float2bfloat16(0.0f);
    }
}

// loss 0.5 mean((y - e/s)^2) over 2 channels; g = dL/dy (16 channels, zero beyond 2)
__global__ void k_head_loss(size_t HW, int nb, const bf16* __restrict__ y, const double2* __restrict__ e,
                            const double* __restrict__ sums, bf16* __restrict__ g, double* __restrict__ loss) {
    __shared__ double red[256];
    const size_t n = HW * nb;
    const double cnt = 2.0 * (double)n;
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / HW);
        double s = sqrt(sums[b] / (double)HW);
        if (!(s > 0.0)) s = 1.0;
        const double2 t = e[i];
        const double d0 = (double)__bfloat162float(y[i * 16 + 0]) - t.x / s;
        const double d1 = (double)__bfloat162float(y[i * 16 + 1]) - t.y / s;
        acc += 0.5 * (d0 * d0 + d1 * d1);
        bf16* o = g + i * 16;
        o[0] = __float2bfloat16((float)(d0 / cnt));
        o[1] = __float2bfloat16((float)(d1 / cnt));
#pragma unroll
        for (int k = 2; k < 16; ++k) o[k] = __float2bfloat16(0.0f);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / cnt);
}

// z = s (y0 + i y1)
__global__ void k_net_output(size_t HW, int nb, const bf16* __restrict__ y, const double* __restrict__ sums,
                             double2* __restrict__ z) {
    const size_t n = HW * nb;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / HW);
        double s = sqrt(sums[b] / (double)HW);
        if (!(s > 0.0)) s = 1.0;
        z[i] = make_double2(s * __bfloat162float(y[i * 16]), s * __bfloat162float(y[i * 16 + 1]));
    }
}

// Adam on the FP32 master parameters
__global__ void k_adam(size_t n, float* __restrict__ w, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ g, float lr, float b1, float b2, float c1, float c2, float eps) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

// BF16 copies of a layer's weights: wf [cout][9][cin] and the backward-data
// weights wt [cin][8 - tap][cout]
__global__ void k_wcopy(int cout, int cin, const float* __restrict__ w, bf16* __restrict__ wf, bf16* __restrict__ wt) {
    const size_t n = (size_t)cout * 9 * cin;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % cin), tap = (int)((i / cin) % 9), co = (int)(i / ((size_t)9 * cin));
        const bf16 v = __float2bfloat16(w[i]);
        wf[i] = v;
        wt[((size_t)ci * 9 + (8 - tap)) * cout + co] = v;
    }
}

__global__ void k_fzero(size_t n, float* p) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0.0f;
}

unsigned grid_for(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

// ------------------------------------------------------------------ executor
struct ls_net {
    struct Layer {
        int cin, cout;       // padded to multiples of 16
        int cin_real, cout_real;
        size_t woff, boff;   // into the FP32 parameter arrays
    };
    int L = 0, c0 = 0, nbmax = 0, Hmax = 0, Wmax = 0, train = 0;
    size_t pix = 0;          // level-0 pixel capacity
    cudaStream_t stream = nullptr;
    long long launches = 0;
    std::vector<Layer> layers;
    size_t nparam = 0, nweights = 0;
    float *w = nullptr, *m1 = nullptr, *m2 = nullptr, *g = nullptr;
    bf16 *wf = nullptr, *wt = nullptr;
    int step = 0;
    int umma = 1;            // 1: forward / backward-data convolutions on tcgen05; 0: WMMA
    // activations (level l has pix >> 2l pixels)
    bf16* in0 = nullptr;
    std::vector<bf16*> pool, ea, cat, up, da, dbo;
    bf16 *bott = nullptr, *head = nullptr;
    // gradients
    bf16 *g_head = nullptr, *tmp = nullptr, *g_bott = nullptr;
    std::vector<bf16*> g_dbo, g_da, g_cat, g_up, g_ea, g_pool, g_eb;
    double* sums = nullptr;
    double* loss = nullptr;
    std::vector<void*> allocs;
    int ch(int l) const { return c0 << l; }
};

namespace {

#define NET_LAUNCH(net, kern, grid, block, smem, ...)                   \
    do {                                                                \
        kern<<<(grid), (block), (smem), (net)->stream>>>(__VA_ARGS__);  \
        (net)->launches++;                                              \
        cudaError_t e_ = cudaPeekAtLastError();                         \
        if (e_ != cudaSuccess) return ls_cuda_fail(e_);                 \
    } while (0)

template <typename T>
int net_alloc(ls_net* n, T** p, size_t count) {
    void* q = nullptr;
    LS_CUDA(cudaMalloc(&q, sizeof(T) * (count ? count : 1)));
    n->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return LS_OK;
}

// layer indices in the oracle's order
int li_enc(int l, int s) { return 2 * l + s; }
int li_dec(const ls_net* n, int l, int s) { return 2 * n->L + 3 * (n->L - 2 - l) + s; }  // s: 0 up, 1 a, 2 b
int li_head(const ls_net* n) { return 2 * n->L + 3 * (n->L - 1); }

int conv(ls_net* n, int li, View x, View y, int H, int W, int M, bool relu, bool backward_data) {
    const ls_net::Layer& Ly = n->layers[li];
    ConvArgs a;
    a.x = x.p; a.xs = x.stride; a.xo = x.off;
    a.y = y.p; a.ys = y.stride; a.yo = y.off;
    a.H = H; a.W = W; a.M = M;
    if (!backward_data) {
        a.cin = Ly.cin; a.cout = Ly.cout;
        a.w = n->wf + Ly.woff;
        a.bias = n->w + Ly.boff;
        a.relu = relu ? 1 : 0;
    } else {
        a.cin = Ly.cout; a.cout = Ly.cin;
        a.w = n->wt + Ly.woff;
        a.bias = nullptr;
        a.relu = 0;
    }
    if (n->umma) {   // tensor cores, fifth generation: one CTA per 128 pixels x all output channels
        const dim3 grid((unsigned)((M + 127) / 128), 1);
        switch (a.cout) {
            case 16: NET_LAUNCH(n, k_conv_umma<16>, grid, kCvThreads, conv_umma_smem<16>(), a); return LS_OK;
            case 32: NET_LAUNCH(n, k_conv_umma<32>, grid, kCvThreads, conv_umma_smem<32>(), a); return LS_OK;
            case 64: NET_LAUNCH(n, k_conv_umma<64>, grid, kCvThreads, conv_umma_smem<64>(), a); return LS_OK;
            case 128: NET_LAUNCH(n, k_conv_umma<128>, grid, kCvThreads, conv_umma_smem<128>(), a); return LS_OK;
            case 256: NET_LAUNCH(n, k_conv_umma<256>, grid, kCvThreads, conv_umma_smem<256>(), a); return LS_OK;
            default: break;   // other widths: the WMMA form below
        }
    }
    const int BN = a.cout >= 64 ? 64 : a.cout;
    const dim3 grid((unsigned)(M / 64), (unsigned)(a.cout / BN));
    if (BN == 64) NET_LAUNCH(n, k_conv_fwd<64>, grid, kConvThreads, 0, a);
    else if (BN == 32) NET_LAUNCH(n, k_conv_fwd<32>, grid, kConvThreads, 0, a);
    else NET_LAUNCH(n, k_conv_fwd<16>, grid, kConvThreads, 0, a);
    return LS_OK;
}

// weight and bias gradients of layer li: dy dense (cout channels), x its input view
int wgrad(ls_net* n, int li, const bf16* dy, View x, int H, int W, int M) {
    const ls_net::Layer& Ly = n->layers[li];
    WgradArgs a;
    a.dy = dy; a.ds = Ly.cout; a.dof = 0; a.cout = Ly.cout;
    a.x = x.p; a.xs = x.stride; a.xo = x.off; a.cin = Ly.cin;
    a.dw = n->g + Ly.woff;
    a.H = H; a.W = W; a.M = M;
    a.chunk = 4096;
    const int BM = Ly.cout >= 64 ? 64 : Ly.cout;
    const int K9 = 9 * Ly.cin;
    const dim3 grid((unsigned)((K9 + 63) / 64), (unsigned)(Ly.cout / BM), (unsigned)((M + a.chunk - 1) / a.chunk));
    if (BM == 64) NET_LAUNCH(n, k_conv_wgrad<64>, grid, kConvThreads, 0, a);
    else if (BM == 32) NET_LAUNCH(n, k_conv_wgrad<32>, grid, kConvThreads, 0, a);
    else NET_LAUNCH(n, k_conv_wgrad<16>, grid, kConvThreads, 0, a);
    const int bchunk = 1024;
    NET_LAUNCH(n, k_bias_grad, (unsigned)((M + bchunk - 1) / bchunk), Ly.cout, 0, dy, Ly.cout, 0, Ly.cout, M, bchunk,
               n->g + Ly.boff);
    return LS_OK;
}

int mask(ls_net* n, size_t M, int c, View g, View y) {
    NET_LAUNCH(n, k_relu_mask, grid_for(M * c), 256, 0, M, c, g.p, g.stride, g.off, y.p, y.stride, y.off, n->tmp);
    return LS_OK;
}

int refresh_weights(ls_net* n) {
    for (const auto& Ly : n->layers)
        NET_LAUNCH(n, k_wcopy, grid_for((size_t)Ly.cout * 9 * Ly.cin), 256, 0, Ly.cout, Ly.cin, n->w + Ly.woff,
                   n->wf + Ly.woff, n->wt + Ly.woff);
    return LS_OK;
}

int check_shape(const ls_net* n, int nb, int H, int W) {
    const int q = 8 << (n->L - 1);  // the bottom level keeps >= 8 x 8 pixels per sample
    if (nb < 1 || H < q || W < q || H % q || W % q) return LS_EINVAL;
    if ((size_t)nb * H * W > n->pix) return LS_ETOOBIG;
    return LS_OK;
}

int forward(ls_net* n, int nb, int H, int W, const double2* r, const double* m) {
    const size_t HW = (size_t)H * W;
    LS_CUDA(cudaMemsetAsync(n->sums, 0, sizeof(double) * nb, n->stream));
    NET_LAUNCH(n, k_sumsq, dim3(64, nb), 256, 0, HW, r, n->sums);
    NET_LAUNCH(n, k_net_input, grid_for(HW * nb), 256, 0, HW, nb, r, m, n->sums, n->in0);
    View h{n->in0, 16, 0, 16};
    for (int l = 0; l < n->L; ++l) {
        const int Hl = H >> l, Wl = W >> l, M = nb * Hl * Wl, c = n->ch(l);
        if (l > 0) {
            NET_LAUNCH(n, k_pool, grid_for((size_t)M * h.c), 256, 0, nb, 2 * Hl, 2 * Wl, h.c, h.p, h.stride, h.off,
                       n->pool[l]);
            h = View{n->pool[l], h.c, 0, h.c};
        }
        View ea{n->ea[l], c, 0, c};
        LS_TRY(conv(n, li_enc(l, 0), h, ea, Hl, Wl, M, true, false));
        View out = l < n->L - 1 ? View{n->cat[l], 2 * c, c, c} : View{n->bott, c, 0, c};
        LS_TRY(conv(n, li_enc(l, 1), ea, out, Hl, Wl, M, true, false));
        h = out;
    }
    for (int l = n->L - 2; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l, M = nb * Hl * Wl, c = n->ch(l);
        NET_LAUNCH(n, k_up, grid_for((size_t)M * h.c), 256, 0, nb, Hl, Wl, h.c, h.p, h.stride, h.off, n->up[l]);
        View up{n->up[l], 2 * c, 0, 2 * c};
        LS_TRY(conv(n, li_dec(n, l, 0), up, View{n->cat[l], 2 * c, 0, c}, Hl, Wl, M, true, false));
        LS_TRY(conv(n, li_dec(n, l, 1), View{n->cat[l], 2 * c, 0, 2 * c}, View{n->da[l], c, 0, c}, Hl, Wl, M, true,
                    false));
        LS_TRY(conv(n, li_dec(n, l, 2), View{n->da[l], c, 0, c}, View{n->dbo[l], c, 0, c}, Hl, Wl, M, true, false));
        h = View{n->dbo[l], c, 0, c};
    }
    LS_TRY(conv(n, li_head(n), h, View{n->head, 16, 0, 16}, H, W, nb * H * W, false, false));
    return LS_OK;
}

int backward(ls_net* n, int nb, int H, int W) {
    const int L = n->L;
    LS_TRY(wgrad(n, li_head(n), n->g_head, View{n->dbo[0], n->c0, 0, n->c0}, H, W, nb * H * W));
    LS_TRY(conv(n, li_head(n), View{n->g_head, 16, 0, 16}, View{n->g_dbo[0], n->c0, 0, n->c0}, H, W, nb * H * W,
                false, true));
    for (int l = 0; l <= L - 2; ++l) {
        const int Hl = H >> l, Wl = W >> l, M = nb * Hl * Wl, c = n->ch(l);
        // dec_b
        LS_TRY(mask(n, M, c, View{n->g_dbo[l], c, 0, c}, View{n->dbo[l], c, 0, c}));
        LS_TRY(wgrad(n, li_dec(n, l, 2), n->tmp, View{n->da[l], c, 0, c}, Hl, Wl, M));
        LS_TRY(conv(n, li_dec(n, l, 2), View{n->tmp, c, 0, c}, View{n->g_da[l], c, 0, c}, Hl, Wl, M, false, true));
        // dec_a
        LS_TRY(mask(n, M, c, View{n->g_da[l], c, 0, c}, View{n->da[l], c, 0, c}));
        LS_TRY(wgrad(n, li_dec(n, l, 1), n->tmp, View{n->cat[l], 2 * c, 0, 2 * c}, Hl, Wl, M));
        LS_TRY(conv(n, li_dec(n, l, 1), View{n->tmp, c, 0, c}, View{n->g_cat[l], 2 * c, 0, 2 * c}, Hl, Wl, M, false,
                    true));
        // dec_up (its output is the lower half of the concatenation)
        LS_TRY(mask(n, M, c, View{n->g_cat[l], 2 * c, 0, c}, View{n->cat[l], 2 * c, 0, c}));
        LS_TRY(wgrad(n, li_dec(n, l, 0), n->tmp, View{n->up[l], 2 * c, 0, 2 * c}, Hl, Wl, M));
        LS_TRY(conv(n, li_dec(n, l, 0), View{n->tmp, c, 0, c}, View{n->g_up[l], 2 * c, 0, 2 * c}, Hl, Wl, M, false,
                    true));
        // through the upsampling into the output of level l + 1
        bf16* dst = l + 1 <= L - 2 ? n->g_dbo[l + 1] : n->g_bott;
        NET_LAUNCH(n, k_up_bwd, grid_for((size_t)(M / 4) * 2 * c), 256, 0, nb, Hl, Wl, 2 * c, n->g_up[l], dst);
    }
    for (int l = L - 1; l >= 0; --l) {
        const int Hl = H >> l, Wl = W >> l, M = nb * Hl * Wl, c = n->ch(l);
        View out = l < L - 1 ? View{n->cat[l], 2 * c, c, c} : View{n->bott, c, 0, c};
        bf16* gout = n->g_bott;
        if (l < L - 1) {  // skip gradient + the gradient through the pool of level l + 1
            NET_LAUNCH(n, k_pool_bwd_add, grid_for((size_t)M * c), 256, 0, nb, Hl, Wl, c, n->g_pool[l + 1],
                       n->g_cat[l], 2 * c, c, n->g_eb[l]);
            gout = n->g_eb[l];
        }
        LS_TRY(mask(n, M, c, View{gout, c, 0, c}, out));
        LS_TRY(wgrad(n, li_enc(l, 1), n->tmp, View{n->ea[l], c, 0, c}, Hl, Wl, M));
        LS_TRY(conv(n, li_enc(l, 1), View{n->tmp, c, 0, c}, View{n->g_ea[l], c, 0, c}, Hl, Wl, M, false, true));
        LS_TRY(mask(n, M, c, View{n->g_ea[l], c, 0, c}, View{n->ea[l], c, 0, c}));
        const int cin = l > 0 ? n->ch(l - 1) : 16;
        View xin = l > 0 ? View{n->pool[l], cin, 0, cin} : View{n->in0, 16, 0, 16};
        LS_TRY(wgrad(n, li_enc(l, 0), n->tmp, xin, Hl, Wl, M));
        if (l > 0)
            LS_TRY(conv(n, li_enc(l, 0), View{n->tmp, c, 0, c}, View{n->g_pool[l], cin, 0, cin}, Hl, Wl, M, false,
                        true));
    }
    return LS_OK;
}

}  // namespace

int ls_conv_timeouts(unsigned* count) {
    LS_CUDA(cudaMemcpyFromSymbol(count, g_conv_timeouts, sizeof(unsigned)));
    return LS_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int ls_net_set_tensor_cores(ls_net* n, int on) {
    if (!n || (on != 0 && on != 1)) return LS_EINVAL;
    n->umma = on;
    return LS_OK;
}

int ls_net_create(int levels, int c0, int max_batch, int H, int W, int train, unsigned long long seed, void* stream,
                  ls_net** out) {
    if (!out || levels < 2 || levels > 6 || c0 < 16 || c0 % 16 || max_batch < 1) return LS_EINVAL;
    const int q = 8 << (levels - 1);
    if (H < q || W < q || H % q || W % q) return LS_EINVAL;
    {   // the tensor-core convolutions take more than the default 48 KB of shared memory
        const cudaError_t e = [] {
            cudaError_t r = cudaFuncSetAttribute(k_conv_umma<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)conv_umma_smem<16>());
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_conv_umma<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)conv_umma_smem<32>());
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_conv_umma<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)conv_umma_smem<64>());
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_conv_umma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)conv_umma_smem<128>());
            if (r == cudaSuccess) r = cudaFuncSetAttribute(k_conv_umma<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)conv_umma_smem<256>());
            return r;
        }();
        if (e != cudaSuccess) return ls_cuda_fail(e);
    }
    ls_net* n = new (std::nothrow) ls_net();
    if (!n) return LS_ENOMEM;
    n->L = levels;
    n->c0 = c0;
    n->nbmax = max_batch;
    n->Hmax = H;
    n->Wmax = W;
    n->train = train ? 1 : 0;
    n->pix = (size_t)max_batch * H * W;
    n->stream = static_cast<cudaStream_t>(stream);
    // layers in the oracle's order
    auto add = [&](int cout_real, int cin_real) {
        ls_net::Layer Ly;
        Ly.cin_real = cin_real;
        Ly.cout_real = cout_real;
        Ly.cin = (cin_real + 15) / 16 * 16;
        Ly.cout = (cout_real + 15) / 16 * 16;
        Ly.woff = n->nparam;
        n->nparam += (size_t)Ly.cout * 9 * Ly.cin;
        n->layers.push_back(Ly);
    };
    int prev = 3;
    for (int l = 0; l < levels; ++l) {
        add(n->ch(l), prev);
        add(n->ch(l), n->ch(l));
        prev = n->ch(l);
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(n->ch(l), n->ch(l + 1));
        add(n->ch(l), 2 * n->ch(l));
        add(n->ch(l), n->ch(l));
    }
    add(2, n->ch(0));
    n->nweights = n->nparam;
    for (auto& Ly : n->layers) {
        Ly.boff = n->nparam;
        n->nparam += Ly.cout;
    }
    int rc = LS_OK;
    do {
        if ((rc = net_alloc(n, &n->w, n->nparam))) break;
        if ((rc = net_alloc(n, &n->m1, n->nparam))) break;
        if ((rc = net_alloc(n, &n->m2, n->nparam))) break;
        if ((rc = net_alloc(n, &n->g, n->nparam))) break;
        if ((rc = net_alloc(n, &n->wf, n->nweights))) break;
        if ((rc = net_alloc(n, &n->wt, n->nweights))) break;
        if ((rc = net_alloc(n, &n->sums, (size_t)max_batch))) break;
        if ((rc = net_alloc(n, &n->loss, 1))) break;
        const size_t P = n->pix;
        n->pool.assign(levels, nullptr);
        n->ea.assign(levels, nullptr);
        n->cat.assign(levels, nullptr);
        n->up.assign(levels, nullptr);
        n->da.assign(levels, nullptr);
        n->dbo.assign(levels, nullptr);
        n->g_dbo.assign(levels, nullptr);
        n->g_da.assign(levels, nullptr);
        n->g_cat.assign(levels, nullptr);
        n->g_up.assign(levels, nullptr);
        n->g_ea.assign(levels, nullptr);
        n->g_pool.assign(levels, nullptr);
        n->g_eb.assign(levels, nullptr);
        if ((rc = net_alloc(n, &n->in0, P * 16))) break;
        if ((rc = net_alloc(n, &n->head, P * 16))) break;
        for (int l = 0; l < levels && rc == LS_OK; ++l) {
            const size_t Pl = P >> (2 * l);
            const int c = n->ch(l);
            if (l > 0) rc = net_alloc(n, &n->pool[l], Pl * n->ch(l - 1));
            if (!rc) rc = net_alloc(n, &n->ea[l], Pl * c);
            if (l < levels - 1) {
                if (!rc) rc = net_alloc(n, &n->cat[l], Pl * 2 * c);
                if (!rc) rc = net_alloc(n, &n->up[l], Pl * 2 * c);
                if (!rc) rc = net_alloc(n, &n->da[l], Pl * c);
                if (!rc) rc = net_alloc(n, &n->dbo[l], Pl * c);
            } else if (!rc) {
                rc = net_alloc(n, &n->bott, Pl * c);
            }
            if (!n->train || rc) continue;
            if (l > 0) rc = net_alloc(n, &n->g_pool[l], Pl * n->ch(l - 1));
            if (!rc) rc = net_alloc(n, &n->g_ea[l], Pl * c);
            if (l < levels - 1) {
                if (!rc) rc = net_alloc(n, &n->g_cat[l], Pl * 2 * c);
                if (!rc) rc = net_alloc(n, &n->g_up[l], Pl * 2 * c);
                if (!rc) rc = net_alloc(n, &n->g_da[l], Pl * c);
                if (!rc) rc = net_alloc(n, &n->g_dbo[l], Pl * c);
                if (!rc) rc = net_alloc(n, &n->g_eb[l], Pl * c);
            } else if (!rc) {
                rc = net_alloc(n, &n->g_bott, Pl * c);
            }
        }
        if (rc) break;
        if (n->train) {
            if ((rc = net_alloc(n, &n->g_head, P * 16))) break;
            if ((rc = net_alloc(n, &n->tmp, P * n->c0))) break;
        }
        // He-normal initial weights (host, seeded), zero biases; the head starts small
        std::vector<float> hw(n->nparam, 0.0f);
        std::mt19937_64 gen(seed);
        std::normal_distribution<float> nd(0.0f, 1.0f);
        for (size_t i = 0; i < n->layers.size(); ++i) {
            const auto& Ly = n->layers[i];
            float sd = std::sqrt(2.0f / (9.0f * Ly.cin_real));
            if (i + 1 == n->layers.size()) sd *= 0.1f;
            for (int o = 0; o < Ly.cout_real; ++o)
                for (int t = 0; t < 9; ++t)
                    for (int c = 0; c < Ly.cin_real; ++c) hw[Ly.woff + ((size_t)o * 9 + t) * Ly.cin + c] = sd * nd(gen);
        }
        if (cudaMemcpyAsync(n->w, hw.data(), sizeof(float) * n->nparam, cudaMemcpyHostToDevice, n->stream) !=
                cudaSuccess ||
            cudaMemsetAsync(n->m1, 0, sizeof(float) * n->nparam, n->stream) != cudaSuccess ||
            cudaMemsetAsync(n->m2, 0, sizeof(float) * n->nparam, n->stream) != cudaSuccess) {
            rc = ls_cuda_fail(cudaGetLastError());
            break;
        }
        if ((rc = refresh_weights(n))) break;
        if (cudaStreamSynchronize(n->stream) != cudaSuccess) rc = ls_cuda_fail(cudaGetLastError());
    } while (0);
    if (rc != LS_OK) {
        for (void* p : n->allocs) cudaFree(p);
        delete n;
        return rc;
    }
    *out = n;
    return LS_OK;
}

void ls_net_destroy(ls_net* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (void* p : n->allocs) cudaFree(p);
    delete n;
}

size_t ls_net_param_count(const ls_net* n) {
    if (!n) return 0;
    size_t c = 0;
    for (const auto& Ly : n->layers) c += (size_t)Ly.cout_real * Ly.cin_real * 9 + Ly.cout_real;
    return c;
}

// host <-> device parameter transfer in the oracle's layout: per layer (oracle
// order) w[o][c][a][b] then b[o]
static int params_io(ls_net* n, float* host, const float* src_host, bool get, const float* dev) {
    std::vector<float> hw(n->nparam);
    if (get || !src_host) {
        LS_CUDA(cudaMemcpyAsync(hw.data(), dev, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, n->stream));
        LS_CUDA(cudaStreamSynchronize(n->stream));
    }
    size_t k = 0;
    for (const auto& Ly : n->layers) {
        for (int o = 0; o < Ly.cout_real; ++o)
            for (int c = 0; c < Ly.cin_real; ++c)
                for (int t = 0; t < 9; ++t, ++k) {
                    float& v = hw[Ly.woff + ((size_t)o * 9 + t) * Ly.cin + c];
                    if (get) host[k] = v;
                    else v = src_host[k];
                }
        for (int o = 0; o < Ly.cout_real; ++o, ++k) {
            float& v = hw[Ly.boff + o];
            if (get) host[k] = v;
            else v = src_host[k];
        }
    }
    if (!get) {
        LS_CUDA(cudaMemcpyAsync(n->w, hw.data(), sizeof(float) * n->nparam, cudaMemcpyHostToDevice, n->stream));
        LS_TRY(refresh_weights(n));
        LS_CUDA(cudaStreamSynchronize(n->stream));
    }
    return LS_OK;
}

int ls_net_get_params(ls_net* n, float* host, size_t count) {
    if (!n || !host || count != ls_net_param_count(n)) return LS_EINVAL;
    return params_io(n, host, nullptr, true, n->w);
}

int ls_net_set_params(ls_net* n, const float* host, size_t count) {
    if (!n || !host || count != ls_net_param_count(n)) return LS_EINVAL;
    LS_TRY(params_io(n, nullptr, host, false, nullptr));
    n->step = 0;
    LS_CUDA(cudaMemsetAsync(n->m1, 0, sizeof(float) * n->nparam, n->stream));
    LS_CUDA(cudaMemsetAsync(n->m2, 0, sizeof(float) * n->nparam, n->stream));
    return LS_OK;
}

int ls_net_get_grads(ls_net* n, float* host, size_t count) {
    if (!n || !host || count != ls_net_param_count(n) || !n->train) return LS_EINVAL;
    return params_io(n, host, nullptr, true, n->g);
}

int ls_net_forward(ls_net* n, int nb, int H, int W, const ls_c64* r, const double* m, ls_c64* z) {
    if (!n || !r || !m || !z) return LS_EINVAL;
    LS_TRY(check_shape(n, nb, H, W));
    LS_TRY(forward(n, nb, H, W, reinterpret_cast<const double2*>(r), m));
    const size_t HW = (size_t)H * W;
    NET_LAUNCH(n, k_net_output, grid_for(HW * nb), 256, 0, HW, nb, n->head, n->sums, reinterpret_cast<double2*>(z));
    return LS_OK;
}

int ls_net_train_step(ls_net* n, int nb, int H, int W, const ls_c64* r, const double* m, const ls_c64* e, float lr,
                      double* loss_out) {
    if (!n || !r || !m || !e || !n->train || !(lr >= 0.0f)) return LS_EINVAL;
    LS_TRY(check_shape(n, nb, H, W));
    LS_TRY(forward(n, nb, H, W, reinterpret_cast<const double2*>(r), m));
    const size_t HW = (size_t)H * W;
    LS_CUDA(cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
    NET_LAUNCH(n, k_head_loss, grid_for(HW * nb), 256, 0, HW, nb, n->head, reinterpret_cast<const double2*>(e),
               n->sums, n->g_head, n->loss);
    NET_LAUNCH(n, k_fzero, grid_for(n->nparam), 256, 0, n->nparam, n->g);
    LS_TRY(backward(n, nb, H, W));
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
    NET_LAUNCH(n, k_adam, grid_for(n->nparam), 256, 0, n->nparam, n->w, n->m1, n->m2, n->g, lr, b1, b2, c1, c2, 1e-8f);
    LS_TRY(refresh_weights(n));
    if (loss_out) {
        LS_CUDA(cudaMemcpyAsync(loss_out, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        LS_CUDA(cudaStreamSynchronize(n->stream));
    }
    return LS_OK;
}

long long ls_net_kernel_count(const ls_net* n) { return n ? n->launches : 0; }

}  // extern "C"

// z = N(v) for one field of the handle's grid (used inside flexible GMRES)
int ls_net_apply_field(ls_net* n, cudaStream_t stream, int H, int W, const double2* v, const double* m, double2* z) {
    cudaStream_t saved = n->stream;
    n->stream = stream;
    int rc = check_shape(n, 1, H, W);
    if (rc == LS_OK) rc = forward(n, 1, H, W, v, m);
    if (rc == LS_OK) {
        const size_t HW = (size_t)H * W;
        k_net_output<<<grid_for(HW), 256, 0, stream>>>(HW, 1, n->head, n->sums, z);
        n->launches++;
        const cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) rc = ls_cuda_fail(e);
    }
    n->stream = saved;
    return rc;
}
