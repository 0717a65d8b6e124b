// ls_cr_mma.cu -- the block cyclic reduction steps of the local solves (Sec. 3.4-3.5,
// Algorithm 1's (C^l)^{-1} g^l) on the fifth-generation tensor cores, for batches of
// up to 32 right-hand sides in FP32 (mixed precision).
//
// One reduction step for block j of a level applies up to three q x q complex
// factor matrices to the batch's vectors at the neighbouring blocks:
//   MODE 0 (level 0, odd j)       x_j = D^{-1} x_j
//   MODE 1 (level k >= 1, even j) x_j = x_j + F (-x_{j-1}) + G (-x_{j+1})
//   MODE 2 (level k >= 1, odd j)  x_j = D^{-1} x_j + P (-x_{j-1}) + Q (-x_{j+1})
//   MODE 3 (top block)            x_0 = D^{-1} x_0
//   MODE 4 (level 0 back, odd j)  x_j = x_j + D^{-1} t,  t = -(W x_{j-1} + E x_{j+1})
//                                 (W, E: the tridiagonal couplings of level 0)
// With NB right-hand sides this is a complex (q x q) . (q x NB) product per matrix:
// a dense contraction, done as two real GEMMs with M = 128 rows (q <= 112 real ones),
// N = 2 NB, K = q per matrix, into two accumulators:
//   acc0 += M_re [X_re | X_im],  acc1 += M_im [X_re | X_im],
//   D_re = acc0[:, :NB] - acc1[:, NB:],  D_im = acc0[:, NB:] + acc1[:, :NB].
// Operand A is a factor matrix: each plane (re, im) stored in TF32 (rounded to
// nearest once, when factored) already in the tensor cores' 128-byte-swizzled
// K-major layout -- ceil(q/32) atoms of 32 K-columns x (q rounded up to 8) rows --
// so a plane is one contiguous bulk copy (cp.async.bulk) from HBM into a ring of
// plane-sized shared-memory stages; each matrix byte is read once per step for the
// whole batch.  Operand B is built by the CTA's threads from the vectors (the
// sign of the step folded in, rounded to TF32): per vector 2NB rows [X_re; X_im].
// One thread issues tcgen05.mma (kind::tf32, K = 8 per instruction; K slices past q,
// all zero, skipped) into the TMEM accumulators (128 lanes x 2 x 2NB FP32 columns); the
// epilogue reads them back with tcgen05.ld and writes (or adds to) x_j.
// Roles in a CTA of 256 threads: thread 0 loads A planes (bulk copies), thread 32 issues
// the MMAs, everyone builds B and runs the epilogue.  Every wait is bounded (1 s
// on %globaltimer); on expiry the step's outputs become NaN and a device counter
// (ls_device_timeouts) is raised, so every residual check rejects the result.
#include <mutex>

#include "ls_internal.cuh"
#include "ls_umma.cuh"

namespace {

__device__ unsigned g_cr_timeouts;   // steps whose copies or MMAs did not complete in time

constexpr int kThreads = 256;

using namespace umma;

__device__ __forceinline__ float tf32_rna(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__host__ __device__ __forceinline__ unsigned swz(int row, int kc) {   // byte offset of TF32 kc in a swizzled atom
    return swz16(row, kc >> 2) + (unsigned)(kc & 3) * 4u;
}
__host__ __device__ constexpr unsigned idesc_tf32(int M, int N) { return idesc(2u, M, N); }

template <int MODE> struct ModeOf {
    static constexpr int NV = MODE == 1 ? 2 : (MODE == 2 ? 3 : 1);   // vectors (= matrices) per step
    static constexpr bool ADD = MODE == 1 || MODE == 4;              // x_j += D instead of x_j = D
};

// Shared memory of one CTA: A ring (S stages of one factor plane each: KA atoms of
// BR x 128 bytes) | B (NV vectors x KA atoms x 2NB rows x 128 B) | barriers (full[S],
// empty[S], done) | TMEM address | failure flag | slack.  The MMA reads 128 rows from
// an atom's start: rows past an atom land on the next atom, on B or on the slack
// (garbage rows of D that are never read); the slack makes the ring's last atom plus
// 128 rows end inside the allocation.  S: as many stages as the step's planes (at most
// kMaxStages) within the budget: 113 KB when two CTAs share an SM (every one-matrix
// step, and the steps of levels with more blocks than SMs), 227 KB otherwise.
constexpr int kMaxStages = 6;
constexpr int kSmemTwo = 113 * 1024, kSmemOne = 227 * 1024;
template <int MODE, int NB, int KA>
struct Cfg {
    static constexpr int NV = ModeOf<MODE>::NV;
    static constexpr int BBYTES = NV * KA * 2 * NB * 128;
    static constexpr int NP = 2 * NV;   // planes per step
    static constexpr int FIXED = 1024 + 8 * (2 * kMaxStages + 1) + 16;   // alignment, barriers, slot, flags
    static int plane_bytes(int q) { return KA * ((q + 7) / 8 * 8) * 128; }
    static int slack(int q) {
        const int over = (128 - (q + 7) / 8 * 8) * 128 - BBYTES - (FIXED - 1024);
        return over > 0 ? over : 0;
    }
    static int stages(int q, bool two) {
        const int fit = ((two ? kSmemTwo : kSmemOne) - FIXED - BBYTES - slack(q)) / plane_bytes(q);
        const int cap = NP < kMaxStages ? NP : kMaxStages;
        return fit < cap ? fit : cap;
    }
    static size_t smem(int q, int stages) { return (size_t)FIXED + (size_t)stages * plane_bytes(q) + BBYTES + slack(q); }
    static constexpr size_t kMaxSmem = kSmemOne;   // bound of smem() for every q and budget
};

struct StepArgs {
    int q, k, nk;             // strip height, level, blocks at this level
    size_t mat0;              // first matrix of this strip in the direction's pool (matrix index)
    size_t off_a, off_b, off_c;  // level offsets (matrices) of the step's 1st, 2nd, 3rd matrix
    const float* pool;        // TF32 planes, pre-swizzled: [matrix][plane][KA atoms][BR rows][32]
    int stages;               // A ring stages (Cfg::stages(q))
    float2* x;                // strip vectors of batch member 0 (block layout); member b at + b * SB
    size_t SB;
    int nb;                   // members present (<= NB)
    const float2* cw;         // MODE 4: level-0 couplings of this strip [i][dz+1][r]
    const float2* ce;
};

// Block j of the step's level that CTA `idx` takes, and its vector slots t: present?,
// block (in the strip), sign, factor matrix (index in the pool).
struct StepGeom {
    size_t s;        // 2^k: blocks between neighbours at this level
    int j;
    bool hw, he;     // west / east neighbour present
    bool pres[3];
    long long blk[3];
    float sgn[3];
    size_t mat[3];
    int npl;         // factor planes to stream: present vectors x 2
};
template <int MODE>
__device__ __forceinline__ StepGeom step_geom(const StepArgs& a, int idx) {
    StepGeom g{};
    const size_t s = (size_t)1 << a.k;
    const int j = (MODE == 1) ? 2 * idx : (MODE == 3 ? 0 : 2 * idx + 1);
    const bool hw = j >= 1, he = j + 1 < a.nk;
    g.s = s;
    g.j = j;
    g.hw = hw;
    g.he = he;
    bool* pres = g.pres;
    long long* blk = g.blk;
    float* sgn = g.sgn;
    size_t* mat = g.mat;
    if (MODE == 0 || MODE == 3 || MODE == 4) {
        pres[0] = true; blk[0] = (long long)j * s; sgn[0] = 1.f; mat[0] = a.mat0 + a.off_a + idx;
    }
    if (MODE == 1) {
        pres[0] = hw; blk[0] = (long long)(j - 1) * (long long)s; sgn[0] = -1.f; mat[0] = a.mat0 + a.off_b + idx;
        pres[1] = he; blk[1] = (long long)(j + 1) * s; sgn[1] = -1.f; mat[1] = a.mat0 + a.off_c + idx;
    }
    if (MODE == 2) {
        pres[0] = true; blk[0] = (long long)j * s; sgn[0] = 1.f; mat[0] = a.mat0 + a.off_a + idx;
        pres[1] = true; blk[1] = (long long)(j - 1) * (long long)s; sgn[1] = -1.f; mat[1] = a.mat0 + a.off_b + idx;
        pres[2] = he; blk[2] = (long long)(j + 1) * s; sgn[2] = -1.f; mat[2] = a.mat0 + a.off_c + idx;
    }
    g.npl = 0;
#pragma unroll
    for (int t = 0; t < ModeOf<MODE>::NV; ++t) g.npl += pres[t] ? 2 : 0;
    return g;
}

// Operand B of the step for the geometry gm: per vector t, atom at, rows [0,NB) = X_re,
// [NB,2NB) = X_im (TF32, the step's sign folded in), built by the kThreads threads tid.
template <int MODE, int NB, int KA>
__device__ __forceinline__ void build_b(const StepArgs& a, const StepGeom& gm, unsigned char* Bs, int tid) {
    constexpr int NV = ModeOf<MODE>::NV;
    constexpr int KP = 32 * KA;
    constexpr unsigned BATOM = 2 * NB * 128;
    const int q = a.q, warp = tid >> 5, lane = tid & 31;
    const int j = gm.j;
    const bool he = gm.he;
    const size_t s = gm.s;
    const bool* pres = gm.pres;
    const long long* blk = gm.blk;
    const float* sgn = gm.sgn;
    // Every load is issued (at a clamped, valid address) before any value is used, so their
    // latencies overlap; absent vectors, members and padding rows are zeroed afterwards.
    const int nbc = a.nb < 1 ? 0 : a.nb - 1;
    if constexpr (MODE == 4) {
        // t = -(W x_{j-1} + E x_{j+1}) with the tridiagonal couplings of level 0.  Warp w
        // takes members b = w + 8 m (m < NB / 8) and rows kk = 32 c + lane (c < KA): the
        // rows kk -+ 1 of a member are in the same warp (the neighbour lane, or lane 31 / 0
        // of the neighbouring chunk), and the couplings of row kk serve all its members.
        constexpr int MW = NB / 8;
        const float2 z2 = make_float2(0.f, 0.f);
        const float2* wj = a.cw + (size_t)j * 3 * q;
        const float2* ej = a.ce + (size_t)j * 3 * q;
        float2 cwr[KA][3], cer[KA][3];
#pragma unroll
        for (int c = 0; c < KA; ++c) {
            const int kk = 32 * c + lane, kc = kk < q ? kk : q - 1;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                cwr[c][d] = __ldg(&wj[(size_t)d * q + kc]);
                cer[c][d] = __ldg(&ej[(size_t)d * q + kc]);
            }
        }
        const size_t om = (size_t)(j - 1) * q, op = (size_t)(he ? j + 1 : j - 1) * q;
        float2 xm[MW][KA], xp[MW][KA];
#pragma unroll
        for (int m = 0; m < MW; ++m)
#pragma unroll
            for (int c = 0; c < KA; ++c) {
                const int b = warp + 8 * m, kk = 32 * c + lane, kc = kk < q ? kk : q - 1;
                const float2* xb = a.x + (size_t)(b < a.nb ? b : nbc) * a.SB;
                xm[m][c] = xb[om + kc];
                xp[m][c] = xb[op + kc];
            }
#pragma unroll
        for (int m = 0; m < MW; ++m)
#pragma unroll
            for (int c = 0; c < KA; ++c)
                if (32 * c + lane >= q) {   // rows outside the strip hold zero
                    xm[m][c] = z2;
                    xp[m][c] = z2;
                }
        auto shf = [](float2 v, int src) {
            return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
        };
        auto up1 = [](float2 v) {
            return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
        };
        auto dn1 = [](float2 v) {
            return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
        };
#pragma unroll
        for (int m = 0; m < MW; ++m) {
            const int b = warp + 8 * m;
#pragma unroll
            for (int c = 0; c < KA; ++c) {
                float2 ml = up1(xm[m][c]), pl = up1(xp[m][c]), mr = dn1(xm[m][c]), pr = dn1(xp[m][c]);
                const float2 mlc = c > 0 ? shf(xm[m][c > 0 ? c - 1 : 0], 31) : z2;
                const float2 plc = c > 0 ? shf(xp[m][c > 0 ? c - 1 : 0], 31) : z2;
                const float2 mrc = c + 1 < KA ? shf(xm[m][c + 1 < KA ? c + 1 : c], 0) : z2;
                const float2 prc = c + 1 < KA ? shf(xp[m][c + 1 < KA ? c + 1 : c], 0) : z2;
                if (lane == 0) { ml = mlc; pl = plc; }
                if (lane == 31) { mr = mrc; pr = prc; }
                float2 acc = cfma(cwr[c][0], ml, z2);
                acc = cfma(cwr[c][1], xm[m][c], acc);
                acc = cfma(cwr[c][2], mr, acc);
                if (he) {
                    acc = cfma(cer[c][0], pl, acc);
                    acc = cfma(cer[c][1], xp[m][c], acc);
                    acc = cfma(cer[c][2], pr, acc);
                }
                const bool live = b < a.nb && 32 * c + lane < q;
                const float re = live ? tf32_rna(-acc.x) : 0.f, im = live ? tf32_rna(-acc.y) : 0.f;
                // rows b and NB + b share (row & 7) (NB is a multiple of 8): NB * 128 bytes apart
                unsigned char* atom = Bs + (size_t)c * BATOM;
                const unsigned off = (unsigned)(b >> 3) * 1024u + (unsigned)(b & 7) * 128u +
                                     (unsigned)(((lane >> 2) ^ (b & 7)) << 4) + (unsigned)(lane & 3) * 4u;
                *reinterpret_cast<float*>(atom + off) = re;
                *reinterpret_cast<float*>(atom + off + NB * 128u) = im;
            }
        }
    } else {
        // Groups of 4 consecutive rows of one member: one 16-byte chunk of a swizzled atom
        // row, so each of the two B rows takes one 16-byte store.
        constexpr int KG = KP / 4, NG = NB * KG, PERG = (NG + kThreads - 1) / kThreads;
        size_t ob[NV];   // absent vectors read the step's own block (a valid address), then zeroed
#pragma unroll
        for (int t = 0; t < NV; ++t) ob[t] = (size_t)(pres[t] ? blk[t] : (long long)j * (long long)s) * q;
        float2 xv[NV][PERG][4];
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int g = 0; g < PERG; ++g) {
                const int o4 = tid + g * kThreads, b = o4 / KG, k0 = 4 * (o4 % KG);
                const float2* xb = a.x + (size_t)(o4 < NG && b < a.nb ? b : nbc) * a.SB + ob[t];
#pragma unroll
                for (int e = 0; e < 4; ++e) xv[t][g][e] = xb[k0 + e < q ? k0 + e : q - 1];
            }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            unsigned char* Bt = Bs + (size_t)t * KA * BATOM;
#pragma unroll
            for (int g = 0; g < PERG; ++g) {
                const int o4 = tid + g * kThreads, b = o4 / KG, c4 = o4 % KG, k0 = 4 * c4;
                if (o4 >= NG) continue;
                float re[4], im[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const bool live = pres[t] && b < a.nb && k0 + e < q;
                    re[e] = live ? tf32_rna(sgn[t] * xv[t][g][e].x) : 0.f;
                    im[e] = live ? tf32_rna(sgn[t] * xv[t][g][e].y) : 0.f;
                }
                const int ch = c4 & 7;   // 16-byte chunk of the 128-byte row in atom c4 / 8
                unsigned char* row = Bt + (size_t)(c4 >> 3) * BATOM + (size_t)(b >> 3) * 1024u + (size_t)(b & 7) * 128u +
                                     (size_t)((ch ^ (b & 7)) << 4);
                *reinterpret_cast<float4*>(row) = make_float4(re[0], re[1], re[2], re[3]);
                *reinterpret_cast<float4*>(row + NB * 128u) = make_float4(im[0], im[1], im[2], im[3]);
            }
        }
    }
}

// x_j before the step, for the steps that add (MODE 1, 4): rows r = 32 (warp % 4) + lane,
// members half * NB/2 .. of warp half = warp / 4 (the epilogue's mapping)
template <int MODE, int NB>
__device__ __forceinline__ void load_old(const StepArgs& a, const StepGeom& gm, int warp, int lane, float2* old) {
    constexpr int HB = NB / 2;
    const int r = 32 * (warp & 3) + lane, half = warp >> 2;
#pragma unroll
    for (int c = 0; c < HB; ++c) {
        const int b = half * HB + c;
        old[c] = (ModeOf<MODE>::ADD && r < a.q && b < a.nb) ? a.x[(size_t)b * a.SB + (size_t)gm.j * gm.s * a.q + r]
                                                            : make_float2(0.f, 0.f);
    }
}

// Epilogue of a step: the two accumulators (tensor memory at tmem) -> x_j (+ old for the
// steps that add), NaN if the step failed.  Warps 0-7: warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (rows r), its half w / 4 of the members.
template <int MODE, int NB>
__device__ __forceinline__ void store_step(const StepArgs& a, const StepGeom& gm, unsigned tmem, bool bad,
                                           const float2* old, int warp, int lane) {
    using MO = ModeOf<MODE>;
    constexpr int NCOL = 2 * NB, HB = NB / 2;
    const int q = a.q, j = gm.j;
    const size_t s = gm.s;
    const int r = 32 * (warp & 3) + lane;
    const int half = warp >> 2;
    // D_re = M_re X_re - M_im X_im = acc0[:, b] - acc1[:, NB + b],
    // D_im = M_re X_im + M_im X_re = acc0[:, NB + b] + acc1[:, b]
    float dre[HB], dim[HB];
    const unsigned tl = tmem + ((unsigned)(32 * (warp & 3)) << 16);
    if constexpr (HB % 8 == 0) {
#pragma unroll
        for (int c = 0; c < HB; c += 8) {
            float rr[8], ri[8], ir[8], ii[8];
            const unsigned col = (unsigned)(half * HB + c);
            tmem_ld8(tl + col, rr);
            tmem_ld8(tl + (unsigned)NB + col, ri);
            tmem_ld8(tl + (unsigned)NCOL + col, ir);
            tmem_ld8(tl + (unsigned)(NCOL + NB) + col, ii);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                dre[c + e] = rr[e] - ii[e];
                dim[c + e] = ri[e] + ir[e];
            }
        }
    } else {   // NB = 8: each half takes 4 members; read 8 and keep its 4
        float rr[8], ri[8], ir[8], ii[8];
        tmem_ld8(tl, rr);
        tmem_ld8(tl + (unsigned)NB, ri);
        tmem_ld8(tl + (unsigned)NCOL, ir);
        tmem_ld8(tl + (unsigned)(NCOL + NB), ii);
#pragma unroll
        for (int c = 0; c < HB; ++c) {
            dre[c] = rr[half * HB + c] - ii[half * HB + c];
            dim[c] = ri[half * HB + c] + ir[half * HB + c];
        }
    }
    if (r < q) {
#pragma unroll
        for (int c = 0; c < HB; ++c) {
            const int b = half * HB + c;
            if (b >= a.nb) continue;
            float2* xj = a.x + (size_t)b * a.SB + (size_t)j * s * q + r;
            float2 v = bad ? make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000))
                           : make_float2(dre[c], dim[c]);
            if (MO::ADD && !bad) v = make_float2(old[c].x + v.x, old[c].y + v.y);
            *xj = v;
        }
    }
}

template <int MODE, int NB, int KA>
__global__ void __launch_bounds__(kThreads, 2) k_cr_mma(StepArgs a) {
    using MO = ModeOf<MODE>;
    constexpr int NV = MO::NV;
    constexpr int BROWS = 2 * NB;                 // rows of one vector's B atom: [X_re; X_im]
    constexpr unsigned BATOM = BROWS * 128;       // bytes of one vector's B atom
    constexpr int NCOL = 2 * NB;                  // columns of one accumulator
    constexpr int TCOLS = 2 * NCOL;               // two accumulators: M_re B, M_im B (32, 64 or 128)
    const int q = a.q;
    const int BR = (q + 7) / 8 * 8;
    const int kStages = a.stages;
    const unsigned kPlane = (unsigned)KA * (unsigned)BR * 128u;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* As = base;
    unsigned char* Bs = As + (size_t)kStages * kPlane;
    auto* full = reinterpret_cast<unsigned long long*>(Bs + (size_t)NV * KA * BATOM);
    auto* empty = full + kMaxStages;
    auto* done = empty + kMaxStages;
    unsigned* tslot = reinterpret_cast<unsigned*>(done + 1);
    int* failed = reinterpret_cast<int*>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int idx = blockIdx.x;
    // The next step may be scheduled now (programmatic dependent launch): its CTAs set up
    // and start streaming their factor planes, which no step writes, while this one runs.
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const StepGeom g = step_geom<MODE>(a, idx);
    const bool* pres = g.pres;
    const size_t* mat = g.mat;
    const int npl = g.npl;

    if (tid == 0) {
        *failed = 0;
        for (int i = 0; i < kStages; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        bar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) {   // TMEM accumulator: 128 lanes x TCOLS columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const unsigned tmem = *tslot;

    // producer: the first min(npl, kStages) planes start streaming before B is built
    auto plane_src = [&](int i) {   // i-th present plane: (vector slot, re/im)
        int t = 0, r = i;
        while (!pres[t] || r >= 2) {
            if (pres[t]) r -= 2;
            ++t;
        }
        return a.pool + (2 * mat[t] + r) * (size_t)KA * BR * 32;
    };
    if (tid == 0) {
        for (int i = 0; i < npl && i < kStages; ++i) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(&full[i])), "r"(kPlane)
                         : "memory");
            bulk_load(As + (size_t)i * kPlane, plane_src(i), kPlane, &full[i]);
        }
    }

    // Vectors are read and written only after the previous kernel of the stream has
    // completed and its writes are visible.
    asm volatile("griddepcontrol.wait;\n" ::: "memory");

    build_b<MODE, NB, KA>(a, g, Bs, tid);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // B visible to the tensor cores
    __syncthreads();

    if (tid == 32) {   // MMA issuer
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        constexpr unsigned ID = idesc_tf32(128, NCOL);
        int i = 0, issued[2] = {0, 0};   // MMAs into each accumulator so far
        bool ok = true;
        for (int t = 0; t < NV && ok; ++t) {
            if (!pres[t]) continue;
            const unsigned bt = su32(Bs + (size_t)t * KA * BATOM);
            for (int p = 0; p < 2; ++p, ++i) {
                const int st = i % kStages;
                if (!bar_wait(&full[st], (unsigned)(i / kStages) & 1u)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                // descriptors built once per plane; a K slice of 8 TF32 (32 bytes) advances the
                // start-address field (address / 16) by 2, an atom by its size / 16
                const unsigned long long ad0 = sdesc(su32(As + (size_t)st * kPlane));
                // plane re into accumulator 0 (M_re [X_re | X_im]), plane im into accumulator 1
                const unsigned long long bd0 = sdesc(bt);
                const unsigned dacc = tmem + (unsigned)(p * NCOL);
                int& iss = issued[p];
#pragma unroll
                for (int at = 0; at < KA; ++at) {
                    const unsigned long long ad = ad0 + (unsigned long long)((unsigned)at * (unsigned)BR * 8u);
                    const unsigned long long bd = bd0 + (unsigned long long)((unsigned)at * (BATOM >> 4));
                    const int kleft = q - 32 * at;   // K slices of 8 beyond q are zero: skipped
                    if (kleft >= 32) {
#pragma unroll
                        for (int k8 = 0; k8 < 4; ++k8, ++iss)
                            mma_tf32(dacc, ad + 2ull * k8, bd + 2ull * k8, ID, iss ? 1u : 0u);
                    } else {
                        const int nk8 = (kleft + 7) / 8;
                        for (int k8 = 0; k8 < nk8; ++k8, ++iss)
                            mma_tf32(dacc, ad + 2ull * k8, bd + 2ull * k8, ID, iss ? 1u : 0u);
                    }
                }
                mma_commit(&empty[st]);   // the stage is free once these MMAs have read it
            }
        }
        if (!ok) atomicOr(failed, 1);
        mma_commit(done);   // every MMA issued above has completed
    }
    if (tid == 0) {   // producer: refill each stage once the MMAs of its previous use are done
        for (int i = kStages; i < npl; ++i) {
            const int st = i % kStages;
            if (!bar_wait(&empty[st], (unsigned)(i / kStages - 1) & 1u)) {
                atomicOr(failed, 2);
                break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(&full[st])),
                         "r"(kPlane)
                         : "memory");
            bulk_load(As + (size_t)st * kPlane, plane_src(i), kPlane, &full[st]);
        }
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows r), columns split between w and w + 4
    float2 old[NB / 2];   // x_j before the step (the steps that add), read while the products run
    load_old<MODE, NB>(a, g, warp, lane, old);
    const bool fin = bar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    const bool bad = !fin || *failed;
    store_step<MODE, NB>(a, g, tmem, bad, old, warp, lane);
    if (bad && tid == 0) atomicAdd(&g_cr_timeouts, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS) : "memory");
}

// column-major complex q x q (FP32) -> two TF32 planes per matrix in the 128-byte-swizzled
// K-major layout of the tensor cores: [plane][KA atoms][BR rows][32 K-columns], zeros
// beyond q (rows and K)
__global__ void k_pack_tc(size_t nmat, int q, int KA, int BR, const float2* __restrict__ src, float* __restrict__ dst) {
    const size_t per = (size_t)2 * KA * BR * 32;   // floats per matrix
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nmat * per; e += (size_t)gridDim.x * blockDim.x) {
        const size_t mi = e / per;
        size_t rem = e % per;
        const int pl = (int)(rem / ((size_t)KA * BR * 32));
        rem %= (size_t)KA * BR * 32;
        const int at = (int)(rem / ((size_t)BR * 32));
        rem %= (size_t)BR * 32;
        const int row = (int)(rem / 32), kc = (int)(rem % 32);
        const int c = 32 * at + kc;   // K index = column of M
        float v = 0.f;
        if (row < q && c < q) {
            const float2 m = src[mi * (size_t)q * q + (size_t)c * q + row];
            v = tf32_rna(pl == 0 ? m.x : m.y);
        }
        float* atom = dst + mi * per + ((size_t)pl * KA + at) * BR * 32;   // (row, kc) at its swizzled offset
        atom[swz(row, kc) / 4] = v;
    }
}

// ------------------------------------------------------------------ reduced-system inverse
// The steps of levels k >= c of a local solve -- the even-block reductions of levels c..K-1,
// the top block and the back substitution down to level c (Sec. 3.4 local solves, factors
// of Sec. 4.1) -- touch only the level-c blocks (strip blocks j 2^c) and map the values
// there linearly to the solution there: x_c = S_c^{-1} b_c, S_c the reduced block-
// tridiagonal system of level c, nc = blocks x q unknowns.  For the first level with at
// most kDenseBlocks blocks that inverse is precomputed (the same steps run on the columns of
// the identity) and stored as TF32 planes in blocks of 128 rows x 128 columns,
// [strip][row tile mt][column chunk kc][plane re, im][4 atoms][128 rows][32], each block
// already in the swizzled K-major layout of the MMA operand A.  A local solve then applies
// it as one product: one CTA per (column chunk, row tile) multiplies its block by the
// batch's values at its 128 columns and writes a partial product; a second kernel adds the
// chunks' partials in the fixed order kc = 0, 1, ... and writes the level-c blocks.
constexpr int kDenseBlocks = 32, kDenseKC = 128, kDenseAtoms = kDenseKC / 32;
constexpr unsigned kDensePlane = kDenseAtoms * 128u * 128u;   // bytes of one plane of a block

struct DenseArgs {
    const float* A;      // this strip's blocks
    int nc, ks, q, c;    // unknowns, column chunks, block height, level
    const float2* x;     // strip vectors, member b at + b * SB (level-c block j at (j << c) * q)
    size_t SB;
    int nb;              // members present
    float2* part;        // [kc][NB][rows] partial products
    int rows;            // row tiles x 128
};

template <int NB>
constexpr size_t dense_smem() {   // ring of 2 atom stages (re and im: 2 x 16 KB) | B | barriers
    return 1024 + 2 * 2 * 16384 + (size_t)kDenseAtoms * 2 * NB * 128 + 8 * 5 + 16;
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 2) k_dense_mma(DenseArgs a) {
    constexpr int NCOL = 2 * NB, TCOLS = 2 * NCOL;
    constexpr unsigned BATOM = 2 * NB * 128;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // A: a ring of two stages, each one K atom of the block (its re and im parts, 16 KB each),
    // so that two CTAs fit on an SM; B: 4 atoms x 2NB rows [X_re; X_im]
    constexpr unsigned kAtom = 128u * 128u, kStage = 2 * kAtom;
    unsigned char* As = base;
    unsigned char* Bs = As + 2 * kStage;
    auto* full = reinterpret_cast<unsigned long long*>(Bs + kDenseAtoms * BATOM);
    auto* empty = full + 2;
    auto* done = empty + 2;
    unsigned* tslot = reinterpret_cast<unsigned*>(done + 1);
    int* failed = reinterpret_cast<int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kc = blockIdx.x, mt = blockIdx.y;
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    if (tid == 0) {
        *failed = 0;
        for (int i = 0; i < 2; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        bar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, TCOLS);
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = *tslot;
    // atom at of the block: re part at src + at * 16 KB, im part one plane further
    const float* src = a.A + ((size_t)mt * a.ks + kc) * 2 * (kDensePlane / 4);
    auto load_atom = [&](int at) {
        const int st = at & 1;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(&full[st])), "r"(kStage)
                     : "memory");
        bulk_load(As + (size_t)st * kStage, src + (size_t)at * (kAtom / 4), kAtom, &full[st]);
        bulk_load(As + (size_t)st * kStage + kAtom, src + kDensePlane / 4 + (size_t)at * (kAtom / 4), kAtom, &full[st]);
    };
    if (tid == 0) {   // the first two atoms (constant data: before the predecessor completes)
        load_atom(0);
        load_atom(1);
    }
    asm volatile("griddepcontrol.wait;\n" ::: "memory");

    // B: column col = 128 kc + kk is unknown (block col / q, row col % q) of level c
    constexpr int PER = NB * kDenseKC / kThreads;
    const int nbc = a.nb < 1 ? 0 : a.nb - 1;
    float2 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int o = tid + u * kThreads, b = o / kDenseKC, kk = o % kDenseKC;
        int col = kc * kDenseKC + kk;
        col = col < a.nc ? col : a.nc - 1;
        const int jb = col / a.q, r = col - jb * a.q;
        v[u] = a.x[(size_t)(b < a.nb ? b : nbc) * a.SB + ((size_t)jb << a.c) * a.q + r];
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int o = tid + u * kThreads, b = o / kDenseKC, kk = o % kDenseKC;
        const bool live = b < a.nb && kc * kDenseKC + kk < a.nc;
        const float re = live ? tf32_rna(v[u].x) : 0.f, im = live ? tf32_rna(v[u].y) : 0.f;
        const int k32 = kk & 31;
        unsigned char* atom = Bs + (size_t)(kk >> 5) * BATOM;
        const unsigned off = (unsigned)(b >> 3) * 1024u + (unsigned)(b & 7) * 128u +
                             (unsigned)(((k32 >> 2) ^ (b & 7)) << 4) + (unsigned)(k32 & 3) * 4u;
        *reinterpret_cast<float*>(atom + off) = re;
        *reinterpret_cast<float*>(atom + off + NB * 128u) = im;
    }
    fence_async_smem();
    __syncthreads();

    if (tid == 32) {   // MMA issuer: plane re into accumulator 0, plane im into accumulator 1
        fence_after();
        constexpr unsigned ID = idesc_tf32(128, NCOL);
        bool ok = true;
        const unsigned long long bd0 = sdesc(su32(Bs));
        for (int at = 0; at < kDenseAtoms && ok; ++at) {
            const int st = at & 1;
            if (!bar_wait(&full[st], (unsigned)(at >> 1) & 1u)) {
                ok = false;
                break;
            }
            fence_after();
#pragma unroll
            for (int p = 0; p < 2; ++p) {   // re part into accumulator 0, im part into accumulator 1
                const unsigned long long ad0 = sdesc(su32(As + (size_t)st * kStage + (size_t)p * kAtom));
                const unsigned dacc = tmem + (unsigned)(p * NCOL);
#pragma unroll
                for (int k8 = 0; k8 < 4; ++k8)
                    mma_tf32(dacc, ad0 + 2ull * k8, bd0 + (unsigned long long)(at * (BATOM >> 4) + 2 * k8), ID,
                             (at | k8) ? 1u : 0u);
            }
            mma_commit(&empty[st]);   // the stage is free once these MMAs have read it
        }
        if (!ok) atomicOr(failed, 1);
        mma_commit(done);
    }
    if (tid == 0) {   // refill: atoms 2 and 3 once the MMAs of atoms 0 and 1 are done
        for (int at = 2; at < kDenseAtoms; ++at) {
            if (!bar_wait(&empty[at & 1], 0u)) {
                atomicOr(failed, 2);
                break;
            }
            load_atom(at);
        }
    }
    const int r = 32 * (warp & 3) + lane;
    const int half = warp >> 2;
    constexpr int HB = NB / 2;
    const bool fin = bar_wait(done, 0);
    fence_after();
    __syncthreads();
    const bool bad = !fin || *failed;
    float dre[HB], dim[HB];
    const unsigned tl = tmem + ((unsigned)(32 * (warp & 3)) << 16);
    if constexpr (HB % 8 == 0) {
#pragma unroll
        for (int c = 0; c < HB; c += 8) {
            float rr[8], ri[8], ir[8], ii[8];
            const unsigned col = (unsigned)(half * HB + c);
            tmem_ld8(tl + col, rr);
            tmem_ld8(tl + (unsigned)NB + col, ri);
            tmem_ld8(tl + (unsigned)NCOL + col, ir);
            tmem_ld8(tl + (unsigned)(NCOL + NB) + col, ii);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                dre[c + e] = rr[e] - ii[e];
                dim[c + e] = ri[e] + ir[e];
            }
        }
    } else {
        float rr[8], ri[8], ir[8], ii[8];
        tmem_ld8(tl, rr);
        tmem_ld8(tl + (unsigned)NB, ri);
        tmem_ld8(tl + (unsigned)NCOL, ir);
        tmem_ld8(tl + (unsigned)(NCOL + NB), ii);
#pragma unroll
        for (int c = 0; c < HB; ++c) {
            dre[c] = rr[half * HB + c] - ii[half * HB + c];
            dim[c] = ri[half * HB + c] + ir[half * HB + c];
        }
    }
    const int row = mt * 128 + r;
    if (row < a.nc) {
        float2* pp = a.part + (size_t)kc * NB * a.rows + row;
        const float2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
#pragma unroll
        for (int c = 0; c < HB; ++c) {
            const int b = half * HB + c;
            if (b < a.nb) pp[(size_t)b * a.rows] = bad ? nan2 : make_float2(dre[c], dim[c]);
        }
    }
    if (bad && tid == 0) atomicAdd(&g_cr_timeouts, 1u);
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// x at the level-c blocks = the sum of the column chunks' partial products (fixed order)
__global__ void k_dense_sum(const float2* __restrict__ part, int ks, int nbt, int rows, int nc, int q, int c,
                            float2* __restrict__ x, size_t SB) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (row >= nc) return;
    // the chunks in groups of 8: the group's loads are issued together, then added in order
    float2 sum = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < ks; k0 += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = k0 + u < ks ? part[((size_t)(k0 + u) * nbt + b) * rows + row] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (k0 + u < ks) sum = make_float2(sum.x + v[u].x, sum.y + v[u].y);
    }
    const int jb = row / q, r = row - jb * q;
    x[(size_t)b * SB + ((size_t)jb << c) * q + r] = sum;
}

// set-up: member b of the batch = column col0 + b of the identity (level-c unknowns)
__global__ void k_dense_identity(float2* x, size_t SB, int q, int c, int nc, int col0, int nbm) {
    const int b = threadIdx.x, col = col0 + b;
    if (b >= nbm || col >= nc) return;
    const int jb = col / q, r = col - jb * q;
    x[(size_t)b * SB + ((size_t)jb << c) * q + r] = make_float2(1.f, 0.f);
}

// set-up: the solutions of the identity columns -> columns col0.. of the inverse, as TF32
// planes in the block layout (rows and columns past nc stay zero)
__global__ void k_dense_pack(const float2* __restrict__ x, size_t SB, int q, int c, int nc, int col0, int nbm, int ks,
                             float* __restrict__ A) {
    const size_t total = (size_t)nbm * nc;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / nc), row = (int)(e % nc), col = col0 + b;
        if (col >= nc) continue;
        const int jb = row / q, r = row - jb * q;
        const float2 v = x[(size_t)b * SB + ((size_t)jb << c) * q + r];
        const int mt = row >> 7, rr = row & 127, kc = col >> 7, kk = col & 127;
        float* blk = A + ((size_t)mt * ks + kc) * 2 * (kDensePlane / 4);
        const size_t off = (size_t)(kk >> 5) * (128 * 32) + swz(rr, kk & 31) / 4;
        blk[off] = tf32_rna(v.x);
        blk[kDensePlane / 4 + off] = tf32_rna(v.y);
    }
}

template <int MODE, int NB, int KA>
int set_smem() {
    const size_t sz = Cfg<MODE, NB, KA>::kMaxSmem;
    LS_CUDA(cudaFuncSetAttribute(k_cr_mma<MODE, NB, KA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz));
    return LS_OK;
}

template <int NB>
int set_smem_dense() {
    LS_CUDA(cudaFuncSetAttribute(k_dense_mma<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem<NB>()));
    return LS_OK;
}

template <int NB, int KA>
int set_smem_all() {
    LS_TRY((set_smem<0, NB, KA>()));
    LS_TRY((set_smem<1, NB, KA>()));
    LS_TRY((set_smem<2, NB, KA>()));
    LS_TRY((set_smem<3, NB, KA>()));
    LS_TRY((set_smem<4, NB, KA>()));
    return LS_OK;
}

template <int MODE, int NB, int KA>
int launch(ls_handle* h, unsigned grid, StepArgs a) {
    using CF = Cfg<MODE, NB, KA>;
    // two CTAs per SM for one-matrix steps and for levels with more blocks than SMs (one
    // CTA's operand build and epilogue overlap the other's copies and products); one CTA
    // with every plane in flight for the small levels
    const bool two = CF::NV == 1 || (int)grid > h->tc_sms;
    a.stages = CF::stages(a.q, two);
    if (a.stages < 1) a.stages = CF::stages(a.q, false);
    if (a.stages < 1) return LS_EINVAL;
    // programmatic stream serialization: the kernel waits (griddepcontrol.wait) for its
    // predecessor before it touches the vectors
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = CF::smem(a.q, a.stages);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_cr_mma<MODE, NB, KA>, a);
    h->launches++;
    if (e != cudaSuccess) return ls_cuda_fail(e);
    return LS_OK;
}

template <int NB, int KA>
int launch_mode(ls_handle* h, int mode, unsigned grid, const StepArgs& a) {
    switch (mode) {
        case 0: return launch<0, NB, KA>(h, grid, a);
        case 1: return launch<1, NB, KA>(h, grid, a);
        case 2: return launch<2, NB, KA>(h, grid, a);
        case 3: return launch<3, NB, KA>(h, grid, a);
        default: return launch<4, NB, KA>(h, grid, a);
    }
}

template <int NB>
int launch_ka(ls_handle* h, int mode, unsigned grid, const StepArgs& a) {
    switch ((a.q + 31) / 32) {
        case 1: return launch_mode<NB, 1>(h, mode, grid, a);
        case 2: return launch_mode<NB, 2>(h, mode, grid, a);
        case 3: return launch_mode<NB, 3>(h, mode, grid, a);
        default: return launch_mode<NB, 4>(h, mode, grid, a);
    }
}

}  // namespace

// The inverse of each strip's reduced system at the first level with at most
// kDenseBlocks blocks, from the tensor-core steps of the levels above it applied to the
// identity's columns, 32 at a time (called once the TF32 planes exist).
static int dense_prepare(ls_handle* h) {
    const int q = h->q, n = h->n;
    const size_t SB = (size_t)n * q;
    float2* xt = nullptr;
    for (int d = 0; d < 2; ++d) {
        DirFactors& F = h->fac[d];
        cudaFree(F.dense_tc);
        F.dense_tc = nullptr;
        F.dense_nc = 0;
        int c = 0;
        for (int k = 1; k < F.K; ++k)
            if (F.lev[k].nk <= kDenseBlocks) {
                c = k;
                break;
            }
        if (!c) continue;   // no level small enough (or a single level): the steps stay
        const int nc = F.lev[c].nk * q, mt = (nc + 127) / 128, ks = (nc + kDenseKC - 1) / kDenseKC;
        const size_t per_strip = (size_t)mt * ks * 2 * (kDensePlane / 4);   // floats
        LS_CUDA(cudaMalloc(&F.dense_tc, sizeof(float) * per_strip * h->L));
        LS_CUDA(cudaMemsetAsync(F.dense_tc, 0, sizeof(float) * per_strip * h->L, h->stream));
        if (!xt) LS_CUDA(cudaMalloc(&xt, sizeof(float2) * SB * 32));
        for (int l = 0; l < h->L; ++l) {
            const float2* cw = static_cast<const float2*>(F.cw) + (size_t)l * n * 3 * q;
            const float2* ce = static_cast<const float2*>(F.ce) + (size_t)l * n * 3 * q;
            for (int col0 = 0; col0 < nc; col0 += 32) {
                const int nbm = nc - col0 < 32 ? nc - col0 : 32;
                LS_CUDA(cudaMemsetAsync(xt, 0, sizeof(float2) * SB * nbm, h->stream));
                LS_LAUNCH(h, k_dense_identity, 1, 32, 0, xt, SB, q, c, nc, col0, nbm);
                for (int k = c; k < F.K; ++k) {
                    const CrLevel& lv = F.lev[k];
                    LS_TRY(ls_cr_tc_step(h, d, l, 1, k, lv.nk, (unsigned)lv.neven, 0, lv.off_f, lv.off_g, xt, SB, nbm,
                                         cw, ce));
                }
                LS_TRY(ls_cr_tc_step(h, d, l, 3, 0, 1, 1u, F.off_top, 0, 0, xt, SB, nbm, cw, ce));
                for (int k = F.K - 1; k >= c; --k) {
                    const CrLevel& lv = F.lev[k];
                    if (!lv.nodd) continue;
                    LS_TRY(ls_cr_tc_step(h, d, l, 2, k, lv.nk, (unsigned)lv.nodd, lv.off_dinv, lv.off_p, lv.off_q, xt,
                                         SB, nbm, cw, ce));
                }
                LS_LAUNCH(h, k_dense_pack, 304, 256, 0, xt, SB, q, c, nc, col0, nbm, ks,
                          F.dense_tc + per_strip * l);
            }
        }
        F.dense_c = c;
        F.dense_nc = nc;
        F.dense_mt = mt;
        F.dense_ks = ks;
    }
    LS_CUDA(cudaStreamSynchronize(h->stream));
    cudaFree(xt);
    // every lane's buffer of partial products (the lanes run Algorithm 2 chunks concurrently)
    const size_t e = ls_cr_dense_part_elems(h);
    for (auto& W : h->lanes) {
        cudaFree(W.dense_part);
        W.dense_part = nullptr;
        if (e) LS_CUDA(cudaMalloc(&W.dense_part, sizeof(float2) * e));
    }
    return LS_OK;
}

// The TF32 planes of both directions' factors (after ls_factor, LS_MIXED): per matrix
// two planes of KA = ceil(q/32) atoms of BR = q rounded up to 8 rows x 32 K-columns,
// already in the tensor cores' swizzled layout.
int ls_cr_tc_prepare(ls_handle* h) {
    if (h->prec != LS_MIXED || h->q > 112) return LS_OK;
    const int q = h->q, KA = (q + 31) / 32, BR = (q + 7) / 8 * 8;
    for (int d = 0; d < 2; ++d) {
        DirFactors& F = h->fac[d];
        if (!F.pool32) return LS_ESTATE;
        const size_t nmat = F.mats_per_strip * (size_t)h->L;
        cudaFree(F.pool_tc);
        F.pool_tc = nullptr;
        LS_CUDA(cudaMalloc(&F.pool_tc, sizeof(float) * 2 * (size_t)KA * BR * 32 * nmat));
        LS_LAUNCH(h, k_pack_tc, 1216, 256, 0, nmat, q, KA, BR, F.pool32, F.pool_tc);
    }
    static std::once_flag once;
    static int rc = LS_OK;
    std::call_once(once, [] {
        int r = LS_OK;
        auto all = [&](auto f) { if (r == LS_OK) r = f(); };
        all([] { return set_smem_all<8, 1>(); });  all([] { return set_smem_all<8, 2>(); });
        all([] { return set_smem_all<8, 3>(); });  all([] { return set_smem_all<8, 4>(); });
        all([] { return set_smem_all<16, 1>(); }); all([] { return set_smem_all<16, 2>(); });
        all([] { return set_smem_all<16, 3>(); }); all([] { return set_smem_all<16, 4>(); });
        all([] { return set_smem_all<32, 1>(); }); all([] { return set_smem_all<32, 2>(); });
        all([] { return set_smem_all<32, 3>(); }); all([] { return set_smem_all<32, 4>(); });
        all([] { return set_smem_dense<8>(); });   all([] { return set_smem_dense<16>(); });
        all([] { return set_smem_dense<32>(); });
        rc = r;
    });
    LS_CUDA(cudaStreamSynchronize(h->stream));
    if (rc != LS_OK) return rc;
    int dev = 0;
    LS_CUDA(cudaGetDevice(&dev));
    LS_CUDA(cudaDeviceGetAttribute(&h->tc_sms, cudaDevAttrMultiProcessorCount, dev));
    h->tc_ready = true;
    return dense_prepare(h);
}

void ls_cr_tc_free(ls_handle* h) {
    for (int d = 0; d < 2; ++d) {
        cudaFree(h->fac[d].pool_tc);
        h->fac[d].pool_tc = nullptr;
        cudaFree(h->fac[d].dense_tc);
        h->fac[d].dense_tc = nullptr;
        h->fac[d].dense_nc = 0;
    }
    h->tc_ready = false;
}

// Largest batch one tensor-core step takes (the B operand of 32 right-hand sides and
// three vectors takes a third of the shared memory).
int ls_cr_tc_max_nb(const ls_handle*) { return 32; }

int ls_cr_tc_timeouts(unsigned* count) {
    LS_CUDA(cudaMemcpyFromSymbol(count, g_cr_timeouts, sizeof(unsigned)));
    return LS_OK;
}

// One reduction step on the tensor cores: `mode` as in k_cr_mma, `grid` blocks of the
// level (one CTA each), strip l of direction dir, nb <= ls_cr_tc_max_nb members.
int ls_cr_tc_step(ls_handle* h, int dir, int l, int mode, int k, int nk, unsigned grid, size_t off_a, size_t off_b,
                  size_t off_c, float2* x, size_t SB, int nb, const float2* cw, const float2* ce) {
    const DirFactors& F = h->fac[dir];
    StepArgs a{h->q, k, nk, (size_t)l * F.mats_per_strip, off_a, off_b, off_c, F.pool_tc, 0, x, SB, nb, cw, ce};
    if (nb <= 8) return launch_ka<8>(h, mode, grid, a);
    if (nb <= 16) return launch_ka<16>(h, mode, grid, a);
    if (nb <= 32) return launch_ka<32>(h, mode, grid, a);
    return LS_EINVAL;
}

// float2 entries of a lane's partial-product buffer for the reduced inverse (0: not built)
size_t ls_cr_dense_part_elems(const ls_handle* h) {
    size_t e = 0;
    for (int d = 0; d < 2; ++d) {
        const DirFactors& F = h->fac[d];
        if (!F.dense_nc) continue;
        const size_t need = (size_t)F.dense_ks * 32 * F.dense_mt * 128;
        e = need > e ? need : e;
    }
    return e;
}

// Levels >= c of the local solve of strip l as one product with the reduced inverse: the
// values at the level-c blocks of x (nb <= 32 members) are replaced by the solution there.
int ls_cr_dense_apply(ls_handle* h, int dir, int l, float2* x, size_t SB, int nb) {
    const DirFactors& F = h->fac[dir];
    const ls_handle::SweepLane& W = h->lanes[h->lane];
    if (!F.dense_nc || !W.dense_part || nb < 1 || nb > 32) return LS_ESTATE;
    const size_t per_strip = (size_t)F.dense_mt * F.dense_ks * 2 * (kDensePlane / 4);
    DenseArgs a{F.dense_tc + per_strip * l, F.dense_nc, F.dense_ks, h->q, F.dense_c, x, SB, nb, W.dense_part,
                F.dense_mt * 128};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)F.dense_ks, (unsigned)F.dense_mt);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    int nbt;
    if (nb <= 8) {
        cfg.dynamicSmemBytes = dense_smem<8>();
        e = cudaLaunchKernelEx(&cfg, k_dense_mma<8>, a);
        nbt = 8;
    } else if (nb <= 16) {
        cfg.dynamicSmemBytes = dense_smem<16>();
        e = cudaLaunchKernelEx(&cfg, k_dense_mma<16>, a);
        nbt = 16;
    } else {
        cfg.dynamicSmemBytes = dense_smem<32>();
        e = cudaLaunchKernelEx(&cfg, k_dense_mma<32>, a);
        nbt = 32;
    }
    h->launches++;
    if (e != cudaSuccess) return ls_cuda_fail(e);
    LS_LAUNCH(h, k_dense_sum, dim3((unsigned)((F.dense_nc + 255) / 256), (unsigned)nb), 256, 0, W.dense_part,
              F.dense_ks, nbt, F.dense_mt * 128, F.dense_nc, h->q, F.dense_c, x, SB);
    return LS_OK;
}
