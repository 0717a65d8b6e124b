// ls_fft16.cu -- the FP32 LS-apply (Sec. 2) with transforms specialised on the
// padded length P = 2^LP (256 <= P <= 4096) and on the radix a thread owns.
//
// Same three HBM passes as the generic path (rows forward, columns forward x
// Ghat x inverse, rows inverse), with everything a transform does fixed at
// compile time:
//   * Stockham stages of radix E = 2^LE (16 or 8; the last forward / first
//     inverse stage takes the remaining radix): P = 4096 needs two
//     shared-memory exchanges per transform at radix 16, three at radix 8;
//   * a thread owns one radix-E butterfly per stage (E elements; in the column
//     pass, E elements of each of its CW columns), all index arithmetic is
//     constant-folded and the stage loop is fully unrolled;
//   * twiddles W^r, r = 1..E-1, come from log2 E table loads (W, W^2, W^4, W^8)
//     and products instead of E - 1 loads;
//   * the zero padding is pruned: the first forward stage sees only its lower
//     E/2 inputs (z, x < n <= P/2), so its first butterfly layer only rotates.
// Radix 16 halves the exchanges, radix 8 halves the registers a thread needs
// (more resident warps to hide latency); the autotuner picks per problem.
// Small P groups several transforms per CTA of at least 256 threads.
//
// The column pass reads and writes 16-byte row segments (2 columns) of the
// row-major n x P slab, one per row at a stride of 8P bytes.  Through the LSU each
// such warp access touches 32 separate lines; the TMA shapes (6, 7, 8) move the
// tile instead with cp.async.bulk.tensor in boxes of up to 256 rows into shared
// memory and back, completion tracked by an mbarrier (a wait bounded in time:
// on expiry the tile is written as NaN and a device counter is raised, so the
// solver's residual checks see it).  Shape 8 also keeps the two columns of a
// tile in packed FP32x2 registers, one instruction per operation on both.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "ls_fft_common.cuh"

namespace {

// Geometry of a transform of P = 2^LP points, E = 2^LE elements per thread.
template <int LP, int LE>
struct Geo {
    static constexpr int P = 1 << LP;
    static constexpr int E = 1 << LE;
    static constexpr int T = P / E;                      // threads per transform
    static constexpr int THREADS = T >= 256 ? T : 256;   // CTA size
    static constexpr int G = THREADS / T;                // transforms per CTA
    static constexpr int NS = (LP + LE - 1) / LE;        // stages
    static constexpr int LRL = LP - LE * (NS - 1);       // log2 radix of the last forward stage
    static constexpr int SLOTS = P + (P >> 4);           // padded shared-memory slots per transform
};

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Asynchronous global -> shared copies (sm_80+ cp.async): the data lands in shared
// memory without passing through registers, while the thread carries on.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <typename V>
__device__ __forceinline__ void cp_async_el(V* smem, const V* gmem) {
    if constexpr (sizeof(V) == 16) cp_async16(smem, gmem);
    else cp_async8(smem, gmem);
}

template <int DIR>
__device__ __forceinline__ float2 ld_tw(const float2* __restrict__ tw, int m) {
    float2 w = __ldg(&tw[m]);
    if (DIR < 0) w.y = -w.y;
    return w;
}

// v[c][e R + r] *= W^(k r), W = exp(-DIR 2 pi i / 2^(LS+LR)), r = 1..R-1.
// tw[m] = exp(-2 pi i m / P), so W^s = tw[s << (LP - LS - LR)].
template <int LR, int LS, int DIR, int LP, int CW, int E, typename V>
__device__ __forceinline__ void twiddle(V (&v)[CW][E], int e, int k, const float2* __restrict__ tw) {
    constexpr int R = 1 << LR;
    constexpr int SH = LP - LS - LR;
    float2 w[16];
    w[1] = ld_tw<DIR>(tw, k << SH);
    if (R > 2) w[2] = ld_tw<DIR>(tw, (2 * k) << SH);
    if (R > 4) w[4] = ld_tw<DIR>(tw, (4 * k) << SH);
    if (R > 8) w[8] = ld_tw<DIR>(tw, (8 * k) << SH);
    if (R > 2) w[3] = w[2] * w[1];
    if (R > 4) {
        w[5] = w[4] * w[1];
        w[6] = w[4] * w[2];
        w[7] = w[4] * w[3];
    }
    if (R > 8) {
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = w[8] * w[r - 8];
    }
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int r = 1; r < R; ++r) v[c][e * R + r] = v[c][e * R + r] * w[r];
}

// One Stockham stage: radix 2^LR, Ns = 2^LS.  Butterfly b = j + e T (e < E/R)
// holds inputs b + r P/R in v[.][e R + r]; twiddle by W^((b mod Ns) r), DFT.
template <int LR, int LS, int DIR, int LP, int LE, bool HZ, int CW, int E, typename V>
__device__ __forceinline__ void stage(V (&v)[CW][E], int j, const float2* __restrict__ tw) {
    constexpr int R = 1 << LR, T = Geo<LP, LE>::T;
#pragma unroll
    for (int e = 0; e < E / R; ++e) {
        if constexpr (LS > 0) twiddle<LR, LS, DIR, LP>(v, e, (j + e * T) & ((1 << LS) - 1), tw);
#pragma unroll
        for (int c = 0; c < CW; ++c) dft_reg<R, DIR, HZ>(&v[c][e * R]);
    }
}

// ------------------------------------------------- two columns per FP32x2 instruction
// The column pass applies identical operations to the two columns of a tile, so a
// pair of values (column 0, column 1) can travel in one 64-bit register and be
// added, multiplied and fused-multiply-added by the packed FP32 instructions of
// sm_100+ (add/sub/mul/fma .rn.f32x2: two IEEE single-precision operations, each
// rounded to nearest, in one instruction).  CP holds a complex value of both
// columns: x = (re0, re1), y = (im0, im1).
struct F2 {
    unsigned long long r;
};
__device__ __forceinline__ F2 f2(float lo, float hi) {
    F2 o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(lo), "f"(hi));
    return o;
}
__device__ __forceinline__ F2 f2s(float a) { return f2(a, a); }
__device__ __forceinline__ void f2split(F2 a, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.r));
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 o;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 o;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 o;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {  // a b + c
    F2 o;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(o.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return o;
}
__device__ __forceinline__ F2 neg2(F2 a) {  // flips both sign bits
    F2 o;
    asm("xor.b64 %0, %1, 0x8000000080000000;" : "=l"(o.r) : "l"(a.r));
    return o;
}

struct CP {
    F2 x, y;
};
__device__ __forceinline__ CP operator+(CP a, CP b) { return CP{add2(a.x, b.x), add2(a.y, b.y)}; }
__device__ __forceinline__ CP operator-(CP a, CP b) { return CP{sub2(a.x, b.x), sub2(a.y, b.y)}; }
// the same twiddle w for both columns
__device__ __forceinline__ CP operator*(CP a, float2 w) {
    const F2 wx = f2s(w.x), wy = f2s(w.y), nwy = f2s(-w.y);
    return CP{fma2(a.y, nwy, mul2(a.x, wx)), fma2(a.y, wx, mul2(a.x, wy))};
}
// a different factor per column: g = (g0, g1)
__device__ __forceinline__ CP cmul2(CP a, float2 g0, float2 g1) {
    const F2 gx = f2(g0.x, g1.x), gy = f2(g0.y, g1.y), ngy = f2(-g0.y, -g1.y);
    return CP{fma2(a.y, ngy, mul2(a.x, gx)), fma2(a.y, gx, mul2(a.x, gy))};
}
// the constant rotations of the in-register DFT (found by argument-dependent lookup)
template <int DIR>
__device__ __forceinline__ CP rot16(CP d, int idx) {
    if (idx == 0) return d;
    if (idx == 4) return DIR > 0 ? CP{d.y, neg2(d.x)} : CP{neg2(d.y), d.x};
    const float c = cos16<float>(idx);
    const float s = cos16<float>(idx <= 4 ? 4 - idx : idx - 4);
    if (DIR > 0) return CP{fma2(d.y, f2s(s), mul2(d.x, f2s(c))), fma2(d.x, f2s(-s), mul2(d.y, f2s(c)))};
    return CP{fma2(d.y, f2s(-s), mul2(d.x, f2s(c))), fma2(d.x, f2s(s), mul2(d.y, f2s(c)))};
}
// a row of a 2-column tile as stored in the slab: (re0, im0, re1, im1)
__device__ __forceinline__ CP cp_of(float4 a) { return CP{f2(a.x, a.z), f2(a.y, a.w)}; }
__device__ __forceinline__ float4 f4_of(CP a) {
    float4 o;
    f2split(a.x, o.x, o.z);
    f2split(a.y, o.y, o.w);
    return o;
}

// Shared-memory element: one complex (CW = 1) or the two complex values of a row of
// a 2-column tile (CW = 2).
template <int CW, typename V = float2>
struct Elem;
template <>
struct Elem<1> {
    using T = float2;
    template <int E>
    __device__ __forceinline__ static T pack(const float2 (&v)[1][E], int q) { return v[0][q]; }
    template <int E>
    __device__ __forceinline__ static void unpack(T a, float2 (&v)[1][E], int q) { v[0][q] = a; }
};
template <>
struct Elem<2> {
    using T = float4;
    template <int E>
    __device__ __forceinline__ static T pack(const float2 (&v)[2][E], int q) {
        return make_float4(v[0][q].x, v[0][q].y, v[1][q].x, v[1][q].y);
    }
    template <int E>
    __device__ __forceinline__ static void unpack(T a, float2 (&v)[2][E], int q) {
        v[0][q] = make_float2(a.x, a.y);
        v[1][q] = make_float2(a.z, a.w);
    }
};

template <>
struct Elem<1, CP> {  // in shared memory as (re0, re1, im0, im1)
    using T = ulonglong2;
    template <int E>
    __device__ __forceinline__ static T pack(const CP (&v)[1][E], int q) { return make_ulonglong2(v[0][q].x.r, v[0][q].y.r); }
    template <int E>
    __device__ __forceinline__ static void unpack(T a, CP (&v)[1][E], int q) { v[0][q] = CP{F2{a.x}, F2{a.y}}; }
};

// Outputs of a stage (radix 2^LR, Ns = 2^LS: output (b / Ns) Ns R + b mod Ns + r Ns)
// through shared memory into the inputs of the next stage (radix 2^LRN).
// FIRST: the buffer has not been read since the CTA started, no barrier before
// the stores.
template <int LR, int LS, int LRN, int LP, int LE, bool FIRST, int CW, int E, typename V>
__device__ __forceinline__ void exchange(V (&v)[CW][E], typename Elem<CW, V>::T* buf, int j) {
    constexpr int R = 1 << LR, RN = 1 << LRN, T = Geo<LP, LE>::T, P = Geo<LP, LE>::P;
    if (!FIRST) __syncthreads();
#pragma unroll
    for (int e = 0; e < E / R; ++e) {
        const int b = j + e * T;
        const int base = ((b >> LS) << (LS + LR)) + (b & ((1 << LS) - 1));
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16(base + (r << LS))] = Elem<CW, V>::pack(v, e * R + r);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E / RN; ++e) {
        const int b = j + e * T;
#pragma unroll
        for (int r = 0; r < RN; ++r) Elem<CW, V>::unpack(buf[pad16(b + r * (P / RN))], v, e * RN + r);
    }
}

// Forward stages S.. (stage S: radix E except the last, 2^LRL; Ns = E^S).
// In at S = 0: v[.][t] = x[j + t T], x[j + t T] = 0 for t >= E/2.
// Out: v[.][e R + r] = X[b + r P/R], b = j + e T, R = 2^LRL.
template <int LP, int LE, int S, bool FIRST, int CW, int E, typename V>
__device__ __forceinline__ void fwd_stages(V (&v)[CW][E], typename Elem<CW, V>::T* buf, int j,
                                           const float2* __restrict__ tw) {
    using Gm = Geo<LP, LE>;
    constexpr int LR = S < Gm::NS - 1 ? LE : Gm::LRL;
    if constexpr (S > 0) exchange<LE, LE * (S - 1), LR, LP, LE, FIRST && S == 1>(v, buf, j);
    stage<LR, LE * S, +1, LP, LE, S == 0>(v, j, tw);
    if constexpr (S + 1 < Gm::NS) fwd_stages<LP, LE, S + 1, FIRST>(v, buf, j, tw);
}

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Inverse (unnormalised) stages S..: the forward radices in reverse order (2^LRL
// first).  In at S = 0: the layout fwd_stages leaves.  Out: v[.][t] = x[j + t T].
// before_last runs after the last exchange, before the last stage (the exchange
// buffer is then free once every thread has passed a barrier).
template <int LP, int LE, int S, bool FIRST, int CW, int E, typename V, typename Hook = NoHook>
__device__ __forceinline__ void inv_stages(V (&v)[CW][E], typename Elem<CW, V>::T* buf, int j,
                                           const float2* __restrict__ tw, const Hook& before_last = Hook{}) {
    using Gm = Geo<LP, LE>;
    constexpr int LRL = Gm::LRL;
    constexpr int LR = S == 0 ? LRL : LE;
    constexpr int LS = S == 0 ? 0 : LRL + LE * (S - 1);
    if constexpr (S > 0) {
        constexpr int LRP = S == 1 ? LRL : LE;
        constexpr int LSP = S == 1 ? 0 : LRL + LE * (S - 2);
        exchange<LRP, LSP, LR, LP, LE, FIRST && S == 1>(v, buf, j);
    }
    if constexpr (S + 1 == Gm::NS) before_last();
    stage<LR, LS, -1, LP, LE, false>(v, j, tw);
    if constexpr (S + 1 < Gm::NS) inv_stages<LP, LE, S + 1, FIRST>(v, buf, j, tw, before_last);
}

// Pass 1: X[z, :] = FFT_x(pad(m u)[z, :]) for rows z < nrows (radix 16).
template <int LP, class Src>
__global__ void __launch_bounds__(Geo<LP, 4>::THREADS) k_rows16_fwd(int nrows, int nin, Src src,
                                                                    float2* __restrict__ X,
                                                                    const float2* __restrict__ tw) {
    using Gm = Geo<LP, 4>;
    constexpr int P = Gm::P, T = Gm::T, E = Gm::E, R = 1 << Gm::LRL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / T, j = threadIdx.x % T;
    float2* buf = reinterpret_cast<float2*>(smem_raw) + grp * Gm::SLOTS;
    const int z = blockIdx.x * Gm::G + grp;
    const bool live = z < nrows;
    float2 v[1][E];
#pragma unroll
    for (int t = 0; t < E / 2; ++t) {
        const int x = j + t * T;
        v[0][t] = (live && x < nin) ? src.template load<float2>(z, x) : make_float2(0.f, 0.f);
    }
    fwd_stages<LP, 4, 0, true>(v, buf, j, tw);
    if (!live) return;
    float2* o = X + (size_t)z * P;
#pragma unroll
    for (int e = 0; e < E / R; ++e)
#pragma unroll
        for (int r = 0; r < R; ++r) o[j + e * T + r * (P / R)] = v[0][e * R + r];
}

// Pass 2: for a tile of CW adjacent columns (1 or 2): forward z-FFT (rows >= nin
// are zero), times Ghat, inverse z-FFT; rows z < nout written back in place.
// The tile's Ghat quadrant rows are copied to shared memory asynchronously at
// the start, behind the forward transform.  Tiles are ordered so that kx and
// P - kx (the same quadrant row) run close together and share it in L2.
// LE: log2 of the radix a thread owns; MINB: CTAs per SM the register
// allocation must allow.
template <int LP, int LE, int CW, int MINB>
__global__ void __launch_bounds__(Geo<LP, LE>::THREADS, MINB) k_cols16(int nin, int nout, float2* __restrict__ X,
                                                                       const float2* __restrict__ ghat,
                                                                       const float2* __restrict__ tw) {
    using Gm = Geo<LP, LE>;
    using EL = typename Elem<CW>::T;
    constexpr int P = Gm::P, T = Gm::T, E = Gm::E, R = 1 << Gm::LRL, Q = P / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / T, j = threadIdx.x % T;
    EL* buf = reinterpret_cast<EL*>(smem_raw) + grp * Gm::SLOTS;
    float2* gs = reinterpret_cast<float2*>(smem_raw + sizeof(EL) * Gm::G * Gm::SLOTS) + grp * CW * Q;
    constexpr int ntile = P / CW;
    const int lin = blockIdx.x * Gm::G + grp;
    const int tile = (lin & 1) ? (ntile - 1 - (lin >> 1)) : (lin >> 1);
    const int kx0 = CW * tile;
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int kx = kx0 + c;
        const float2* g = ghat + (size_t)(kx <= P / 2 ? kx : P - kx) * Q;
        for (int i = j; i < Q; i += T) cp_async8(gs + c * Q + i, g + i);
    }
    cp_async_commit();
    float2 v[CW][E];
#pragma unroll
    for (int t = 0; t < E / 2; ++t) {
        const int z = j + t * T;
        EL a{};
        if (z < nin) a = *reinterpret_cast<const EL*>(X + (size_t)z * P + kx0);
        Elem<CW>::unpack(a, v, t);
    }
    fwd_stages<LP, LE, 0, true>(v, buf, j, tw);
    cp_async_wait_all();
    __syncthreads();  // every thread's share of the Ghat rows has landed
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int e = 0; e < E / R; ++e)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kz = j + e * T + r * (P / R);
                v[c][e * R + r] = v[c][e * R + r] * gs[c * Q + (kz <= P / 2 ? kz : P - kz)];
            }
    inv_stages<LP, LE, 0, false>(v, buf, j, tw);
#pragma unroll
    for (int t = 0; t < E; ++t) {
        const int z = j + t * T;
        if (z < nout) *reinterpret_cast<EL*>(X + (size_t)z * P + kx0) = Elem<CW>::pack(v, t);
    }
}

// ------------------------------------------------------------- TMA column tiles
__device__ unsigned int g_tma_timeouts;  // CTAs whose TMA loads did not arrive in time
unsigned g_tma_shortfall = 0;            // host side: see ls_test_tma_shortfall

constexpr unsigned long long kTmaWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Box (4 floats = one row of a 2-column tile) x BR rows at (x, y) -> shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// true once the barrier's phase `parity` has completed; false after kTmaWaitNs.  The
// global timer (slow to read) is read only after a first failed test, then every 32 tests.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i) {
            if (mbar_test(bar, parity)) return true;
            __nanosleep(64);
        }
        if (global_ns() - t0 > kTmaWaitNs) return false;
    }
}

// Pass 2 on 2-column tiles moved by TMA.  Same transforms, Ghat product and
// arithmetic as k_cols16<LP, LE, 2, MINB>; the tile's rows land densely (16 B per
// row) in the front of the exchange buffer, which the first exchange then
// overwrites (after a barrier), and leave the same way.  BR rows per box.
// shortfall: bytes the barrier expects beyond what the boxes deliver (0; a test sets
// it to make the wait run out with no copy left in flight).
template <int LP, int LE, int MINB>
__global__ void __launch_bounds__(Geo<LP, LE>::THREADS, MINB) k_cols16_tma(const __grid_constant__ CUtensorMap map,
                                                                           int n, float2* __restrict__ X,
                                                                           const float2* __restrict__ ghat,
                                                                           const float2* __restrict__ tw,
                                                                           unsigned shortfall) {
    using Gm = Geo<LP, LE>;
    constexpr int CW = 2;
    using EL = float4;
    constexpr int P = Gm::P, T = Gm::T, E = Gm::E, R = 1 << Gm::LRL, Q = P / 2 + 1, G = Gm::G;
    constexpr int BR = P / 2 < 256 ? P / 2 : 256;
    constexpr int ntile = P / CW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int grp = threadIdx.x / T, j = threadIdx.x % T;
    EL* buf = reinterpret_cast<EL*>(smem_raw) + grp * Gm::SLOTS;
    float2* gs = reinterpret_cast<float2*>(smem_raw + sizeof(EL) * G * Gm::SLOTS) + grp * CW * Q;
    auto* bar = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(EL) * G * Gm::SLOTS +
                                                      sizeof(float2) * G * CW * Q);
    int& failed = *reinterpret_cast<int*>(bar + 1);
    auto tile_of = [&](int g) {
        const int lin = blockIdx.x * G + g;
        return (lin & 1) ? (ntile - 1 - (lin >> 1)) : (lin >> 1);
    };
    const int kx0 = CW * tile_of(grp);
    const int nbox = (n + BR - 1) / BR;
    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(G * nbox * BR * sizeof(EL)) + shortfall;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                     : "memory");
        for (int g = 0; g < G; ++g) {
            EL* stg = reinterpret_cast<EL*>(smem_raw) + g * Gm::SLOTS;
            const int x = 2 * CW * tile_of(g);   // in floats: 16-byte aligned
            for (int k = 0; k < nbox; ++k) tma_load_2d(stg + k * BR, &map, x, k * BR, bar);
        }
    }
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int kx = kx0 + c;
        const float2* g = ghat + (size_t)(kx <= P / 2 ? kx : P - kx) * Q;
        for (int i = j; i < Q; i += T) cp_async8(gs + c * Q + i, g + i);
    }
    cp_async_commit();
    if (!mbar_wait(bar, 0)) atomicOr(&failed, 1);
    __syncthreads();
    if (failed) {  // rows of this CTA's tiles become NaN: visible to every residual check
        if (threadIdx.x == 0) atomicAdd(&g_tma_timeouts, 1u);
        const float nan = __int_as_float(0x7fc00000);
        for (int z = j; z < n; z += T)
            *reinterpret_cast<EL*>(X + (size_t)z * P + kx0) = make_float4(nan, nan, nan, nan);
        cp_async_wait_all();
        return;
    }
    float2 v[CW][E];
#pragma unroll
    for (int t = 0; t < E / 2; ++t) {
        const int z = j + t * T;
        Elem<CW>::unpack(z < n ? buf[z] : EL{}, v, t);
    }
    fwd_stages<LP, LE, 0, false>(v, buf, j, tw);  // its first exchange waits for every staging read
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
        for (int e = 0; e < E / R; ++e)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kz = j + e * T + r * (P / R);
                v[c][e * R + r] = v[c][e * R + r] * gs[c * Q + (kz <= P / 2 ? kz : P - kz)];
            }
    inv_stages<LP, LE, 0, false>(v, buf, j, tw);
    __syncthreads();  // every thread is done with the exchange buffer
#pragma unroll
    for (int t = 0; t < E; ++t) {
        const int z = j + t * T;
        if (z < nbox * BR) buf[z] = Elem<CW>::pack(v, t);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int g = 0; g < G; ++g) {
            const EL* stg = reinterpret_cast<const EL*>(smem_raw) + g * Gm::SLOTS;
            const int x = 2 * CW * tile_of(g);
            for (int k = 0; k < nbox; ++k) tma_store_2d(&map, x, k * BR, stg + k * BR);  // rows >= n are clipped
        }
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");  // shared memory stays until read
    }
}

// k_cols16_tma with the two columns of a tile in packed FP32x2 registers (CP): every
// butterfly, rotation, twiddle and Ghat product acts on both columns at once.  Same
// transforms and summation order as the scalar form; the products are contracted
// to fused multiply-adds in a fixed pattern (results agree to FP32 rounding).
template <int LP, int LE, int MINB>
__global__ void __launch_bounds__(Geo<LP, LE>::THREADS, MINB) k_cols16_tma2(const __grid_constant__ CUtensorMap map,
                                                                            int n, float2* __restrict__ X,
                                                                            const float2* __restrict__ ghat,
                                                                            const float2* __restrict__ tw,
                                                                            unsigned shortfall) {
    using Gm = Geo<LP, LE>;
    constexpr int CW = 2;
    using EL = typename Elem<1, CP>::T;
    constexpr int P = Gm::P, T = Gm::T, E = Gm::E, R = 1 << Gm::LRL, Q = P / 2 + 1, G = Gm::G;
    constexpr int BR = P / 2 < 256 ? P / 2 : 256;
    constexpr int ntile = P / CW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int grp = threadIdx.x / T, j = threadIdx.x % T;
    EL* buf = reinterpret_cast<EL*>(smem_raw) + grp * Gm::SLOTS;
    float4* stg = reinterpret_cast<float4*>(buf);  // the tile's rows as the slab stores them
    float2* gs = reinterpret_cast<float2*>(smem_raw + sizeof(EL) * G * Gm::SLOTS) + grp * CW * Q;
    auto* bar = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(EL) * G * Gm::SLOTS +
                                                      sizeof(float2) * G * CW * Q);
    int& failed = *reinterpret_cast<int*>(bar + 1);
    auto tile_of = [&](int g) {
        const int lin = blockIdx.x * G + g;
        return (lin & 1) ? (ntile - 1 - (lin >> 1)) : (lin >> 1);
    };
    const int kx0 = CW * tile_of(grp);
    const int nbox = (n + BR - 1) / BR;
    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)(G * nbox * BR * sizeof(EL)) + shortfall;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                     : "memory");
        for (int g = 0; g < G; ++g) {
            EL* dst = reinterpret_cast<EL*>(smem_raw) + g * Gm::SLOTS;
            const int x = 2 * CW * tile_of(g);
            for (int k = 0; k < nbox; ++k) tma_load_2d(dst + k * BR, &map, x, k * BR, bar);
        }
    }
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const int kx = kx0 + c;
        const float2* g = ghat + (size_t)(kx <= P / 2 ? kx : P - kx) * Q;
        for (int i = j; i < Q; i += T) cp_async8(gs + c * Q + i, g + i);
    }
    cp_async_commit();
    if (!mbar_wait(bar, 0)) atomicOr(&failed, 1);
    __syncthreads();
    if (failed) {
        if (threadIdx.x == 0) atomicAdd(&g_tma_timeouts, 1u);
        const float nan = __int_as_float(0x7fc00000);
        for (int z = j; z < n; z += T)
            *reinterpret_cast<float4*>(X + (size_t)z * P + kx0) = make_float4(nan, nan, nan, nan);
        cp_async_wait_all();
        return;
    }
    CP v[1][E];
    const CP zero{F2{0ull}, F2{0ull}};
#pragma unroll
    for (int t = 0; t < E / 2; ++t) {
        const int z = j + t * T;
        v[0][t] = z < n ? cp_of(stg[z]) : zero;
    }
    fwd_stages<LP, LE, 0, false>(v, buf, j, tw);
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E / R; ++e)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int kz = j + e * T + r * (P / R);
            const int kq = kz <= P / 2 ? kz : P - kz;
            v[0][e * R + r] = cmul2(v[0][e * R + r], gs[kq], gs[Q + kq]);
        }
    inv_stages<LP, LE, 0, false>(v, buf, j, tw);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < E; ++t) {
        const int z = j + t * T;
        if (z < nbox * BR) stg[z] = f4_of(v[0][t]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int g = 0; g < G; ++g) {
            const EL* src = reinterpret_cast<const EL*>(smem_raw) + g * Gm::SLOTS;
            const int x = 2 * CW * tile_of(g);
            for (int k = 0; k < nbox; ++k) tma_store_2d(&map, x, k * BR, src + k * BR);
        }
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
    }
}

// Pass 3: y[z, x] = u[z, x] + IFFT_x(X[z, :])[x] for x < n (radix 16).  The row of u
// is copied asynchronously into the exchange buffer once the last exchange is done
// (each thread fetches the elements it will write), so its latency hides behind the
// last stage, and the CTA needs no shared memory beyond the exchange buffer.
template <int LP, typename UIO>
__global__ void __launch_bounds__(Geo<LP, 4>::THREADS, 4) k_rows16_inv(int nrows, int n, const float2* __restrict__ X,
                                                                    const UIO* __restrict__ u, UIO* __restrict__ y,
                                                                    const float2* __restrict__ tw) {
    using Gm = Geo<LP, 4>;
    constexpr int P = Gm::P, T = Gm::T, E = Gm::E, R = 1 << Gm::LRL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / T, j = threadIdx.x % T;
    float2* buf = reinterpret_cast<float2*>(smem_raw) + grp * Gm::SLOTS;
    UIO* us = reinterpret_cast<UIO*>(buf);  // the row of u, once the exchanges are done
    const int z = blockIdx.x * Gm::G + grp;
    const bool live = z < nrows;
    float2 v[1][E];
    const float2* xr = X + (size_t)(live ? z : 0) * P;
#pragma unroll
    for (int e = 0; e < E / R; ++e)
#pragma unroll
        for (int r = 0; r < R; ++r) v[0][e * R + r] = xr[j + e * T + r * (P / R)];
    auto prefetch_u = [&]() {
        __syncthreads();  // every thread has read its last exchange
        if (live) {
#pragma unroll
            for (int t = 0; t < E / 2; ++t) {
                const int x = j + t * T;
                if (x < n) cp_async_el(us + x, u + (size_t)z * n + x);
            }
        }
        cp_async_commit();
    };
    inv_stages<LP, 4, 0, true>(v, buf, j, tw, prefetch_u);
    cp_async_wait_all();  // this thread's own copies: no barrier needed
    if (!live) return;
#pragma unroll
    for (int t = 0; t < E / 2; ++t) {
        const int x = j + t * T;
        if (x < n) y[(size_t)z * n + x] = us[x] + hw_cast<UIO>(v[0][t]);
    }
}

// Shared memory: G transforms of P elements, padded (one slot per 16), plus, in the
// column pass, the prefetched Ghat rows (G * CW * (P/2 + 1)).
template <int LP, typename UIO>
constexpr size_t rinv_smem() {  // the row of u (P/2 elements) reuses the exchange buffer
    using Gm = Geo<LP, 4>;
    static_assert(sizeof(UIO) * (Gm::P / 2) <= sizeof(float2) * Gm::SLOTS, "u row must fit");
    return sizeof(float2) * Gm::G * Gm::SLOTS;
}
template <int LP, int LE, int CW>
constexpr size_t cols_smem() {
    using Gm = Geo<LP, LE>;
    return sizeof(float2) * CW * Gm::G * Gm::SLOTS + sizeof(float2) * Gm::G * CW * (Gm::P / 2 + 1);
}
template <int LP, int LE>
constexpr size_t cols_tma_smem() {
    return cols_smem<LP, LE, 2>() + 16;  // + the mbarrier and the CTA's failure flag
}
template <int LP>
constexpr size_t row_smem16() {
    return sizeof(float2) * Geo<LP, 4>::G * Geo<LP, 4>::SLOTS;
}

// Column-pass tile shapes (ls_handle::fft_variant): 0 = radix 16, 1 column, 3 CTAs/SM;
// 2 = radix 16, 2 columns, 2 CTAs/SM; 3 = radix 16, 1 column, 2 CTAs/SM;
// 4 = radix 8, 1 column, 2 CTAs/SM (of up to 512 threads); 5 = radix 8, 2 columns, 1 CTA/SM;
// 6, 7 = shapes 2, 5 with the tiles moved by TMA; 8 = shape 6 in packed FP32x2 arithmetic.
template <int LP, int LE, int CW, int MINB>
int cols_launch(ls_handle* h, int n, float2* X, const float2* gh, const float2* tw) {
    using Gm = Geo<LP, LE>;
    LS_LAUNCH(h, (k_cols16<LP, LE, CW, MINB>), (unsigned)(Gm::P / CW / Gm::G), Gm::THREADS,
              (cols_smem<LP, LE, CW>()), n, n, X, gh, tw);
    return LS_OK;
}

// Tensor map of the n x P slab for the TMA shapes: FP32 elements, rows of 2P, boxes
// of 4 (one row of a 2-column tile, 16 bytes) x BR rows; rows beyond n read as 0.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <int LP, int LE, int MINB, bool PACKED = false>
int cols_launch_tma(ls_handle* h, int n, float2* X, const float2* gh, const float2* tw) {
    using Gm = Geo<LP, LE>;
    constexpr int P = Gm::P, BR = P / 2 < 256 ? P / 2 : 256;
    auto enc = tensor_map_encoder();
    if (!enc) return LS_ECUDA;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * P, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)P * sizeof(float2)};
    const cuuint32_t box[2] = {4, (cuuint32_t)BR};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, X, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return LS_ECUDA;
    if constexpr (PACKED)
        LS_LAUNCH(h, (k_cols16_tma2<LP, LE, MINB>), (unsigned)(P / 2 / Gm::G), Gm::THREADS, (cols_tma_smem<LP, LE>()),
                  map, n, X, gh, tw, g_tma_shortfall);
    else
        LS_LAUNCH(h, (k_cols16_tma<LP, LE, MINB>), (unsigned)(P / 2 / Gm::G), Gm::THREADS, (cols_tma_smem<LP, LE>()),
                  map, n, X, gh, tw, g_tma_shortfall);
    return LS_OK;
}

template <int LP, typename UIO>
int apply_lp(ls_handle* h, const UIO* u, UIO* y, float2* X, int shape) {
    using Gm = Geo<LP, 4>;
    const int n = h->n;
    const float2* tw = static_cast<const float2*>(h->tw32);
    const float2* gh = static_cast<const float2*>(h->ghat32);
    const unsigned rows_grid = (unsigned)((n + Gm::G - 1) / Gm::G);
    SrcMU<float, UIO> src{h->m32, u, n};
    LS_LAUNCH(h, (k_rows16_fwd<LP, SrcMU<float, UIO>>), rows_grid, Gm::THREADS, row_smem16<LP>(), n, n, src, X, tw);
    switch (shape) {
        case 2: LS_TRY((cols_launch<LP, 4, 2, 2>(h, n, X, gh, tw))); break;
        case 3: LS_TRY((cols_launch<LP, 4, 1, 2>(h, n, X, gh, tw))); break;
        case 4: LS_TRY((cols_launch<LP, 3, 1, 2>(h, n, X, gh, tw))); break;
        case 5: LS_TRY((cols_launch<LP, 3, 2, 1>(h, n, X, gh, tw))); break;
        case 6: LS_TRY((cols_launch_tma<LP, 4, 2>(h, n, X, gh, tw))); break;
        case 7: LS_TRY((cols_launch_tma<LP, 3, 1>(h, n, X, gh, tw))); break;
        case 8: LS_TRY((cols_launch_tma<LP, 4, 2, true>(h, n, X, gh, tw))); break;
        default: LS_TRY((cols_launch<LP, 4, 1, 3>(h, n, X, gh, tw))); break;
    }
    LS_LAUNCH(h, (k_rows16_inv<LP, UIO>), rows_grid, Gm::THREADS, (rinv_smem<LP, UIO>()), n, n, X, u, y, tw);
    return LS_OK;
}

template <typename UIO>
int apply_any(ls_handle* h, const UIO* u, UIO* y, int shape) {
    float2* X = static_cast<float2*>(h->fftws);
    switch (h->lp) {
        case 8: return apply_lp<8>(h, u, y, X, shape);
        case 9: return apply_lp<9>(h, u, y, X, shape);
        case 10: return apply_lp<10>(h, u, y, X, shape);
        case 11: return apply_lp<11>(h, u, y, X, shape);
        case 12: return apply_lp<12>(h, u, y, X, shape);
        default: return LS_EINVAL;
    }
}

template <typename K>
int optin(K kern, size_t bytes) {
    if (bytes > 48 * 1024) LS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return LS_OK;
}

template <int LP>
int optin_lp() {
    LS_TRY(optin(k_cols16<LP, 4, 1, 3>, cols_smem<LP, 4, 1>()));
    LS_TRY(optin(k_cols16<LP, 4, 1, 2>, cols_smem<LP, 4, 1>()));
    LS_TRY(optin(k_cols16<LP, 4, 2, 2>, cols_smem<LP, 4, 2>()));
    LS_TRY(optin(k_cols16<LP, 3, 1, 2>, cols_smem<LP, 3, 1>()));
    LS_TRY(optin(k_cols16<LP, 3, 2, 1>, cols_smem<LP, 3, 2>()));
    LS_TRY(optin(k_cols16_tma<LP, 4, 2>, cols_tma_smem<LP, 4>()));
    LS_TRY(optin(k_cols16_tma<LP, 3, 1>, cols_tma_smem<LP, 3>()));
    LS_TRY(optin(k_cols16_tma2<LP, 4, 2>, cols_tma_smem<LP, 4>()));
    LS_TRY(optin(k_rows16_inv<LP, float2>, rinv_smem<LP, float2>()));
    return optin(k_rows16_inv<LP, double2>, rinv_smem<LP, double2>());
}

}  // namespace

bool ls_fft16_supported(const ls_handle* h) { return h->lp >= 8 && h->lp <= 12; }

int ls_fft16_init(ls_handle* h) {
    if (!ls_fft16_supported(h)) return LS_OK;
    LS_TRY(optin_lp<8>());
    LS_TRY(optin_lp<9>());
    LS_TRY(optin_lp<10>());
    LS_TRY(optin_lp<11>());
    return optin_lp<12>();
}

// shape: column-pass tile shape (see apply_lp)
int ls_apply32_fft16(ls_handle* h, const float2* u, float2* y, int shape) { return apply_any(h, u, y, shape); }

int ls_apply_mx_fft16(ls_handle* h, const double2* u, double2* y, int shape) {
    return apply_any(h, u, y, shape);
}

extern "C" int ls_test_tma_shortfall(unsigned bytes) {
    if (bytes % 16 || bytes > 4096) return LS_EINVAL;
    g_tma_shortfall = bytes;
    return LS_OK;
}

extern "C" int ls_device_timeouts(unsigned* count) {
    if (!count) return LS_EINVAL;
    unsigned cols = 0, steps = 0, convs = 0;
    LS_CUDA(cudaMemcpyFromSymbol(&cols, g_tma_timeouts, sizeof(unsigned)));
    LS_TRY(ls_cr_tc_timeouts(&steps));
    LS_TRY(ls_conv_timeouts(&convs));
    *count = cols + steps + convs;
    return LS_OK;
}
