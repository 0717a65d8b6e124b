// ls_sweep.cu -- local solves, trace injection, Algorithms 1 and 2 (Sec. 3.4-3.5).
//
// Strip data layout: the extended layer l of a direction is stored block by
// block along the long axis: element (r, i) (local row r, column i) at i*q + r,
// so one column of the strip -- one block of the block-tridiagonal C^l -- is q
// contiguous values.  Every strip keeps its right-hand side and its solution, so
// the traces a neighbour needs (two rows next to the interface) are read in place.
//
// Algorithm 1 (Gauss-Seidel preconditioner), with the index reading of the
// oracle (layers l = 0..L-1 from small z up; local row "1" = r = E, row "n^l" =
// r = E + t - 1):
//   downward, l = L-1..0:  g^l = chi g;  if l < L-1:
//        g^l[n]   -= C^l_{n,n+1} w^{l+1}_1,   g^l[n+1] += C^l_{n+1,n} w^{l+1}_0   (eq. pde_GRF_down)
//        w^l = (C^l)^{-1} g^l
//   upward, l = 1..L-1 (keeping g^l), with the up-going traces of the layer below:
//        g^l[1] -= C^l_{1,0} (v^{l-1}_n - w^l_0),  g^l[0] += C^l_{0,1} v^{l-1}_{n+1};  v^l = (C^l)^{-1} g^l
//   (the top injection of layer l-1 reproduces the down-going wave in its row n but
//   cancels it in its extension row n+1; w^l_0, the continuation of layer l's own
//   down-sweep solution below it, is that wave, so the injected pair is the
//   up-going field in both rows.  v^0 = w^0: layer 0 receives nothing upward.)
//   v = rows 1..n of every v^l.
// Algorithm 2: u1 = Alg. 1 on horizontal layers; e = g - C u1; u2 = Alg. 1 on
// vertical layers (the transposed grid); v = u1 + u2.
//
// Local solve (C^l)^{-1} b by the block cyclic reduction factors of ls_factor.cu:
//   forward  level 0:  y_j = D_j^{-1} b_j (odd j);  b_j -= W_j y_{j-1} + E_j y_{j+1} (even j)
//            level k:  b_j -= F_j b_{j-1} + G_j b_{j+1} (even j of level k)
//   top:     x_0 = D^{-1} b_0
//   backward level k:  x_j = D_j^{-1} b_j - P_j x_{j-1} - Q_j x_{j+1} (odd j)
//            level 0:  x_j = y_j - D_j^{-1} (W_j x_{j-1} + E_j x_{j+1}) (odd j)
// Each kernel is one launch per level over all blocks of that level; a block of
// 256 threads handles one block's mat-vecs, its warps splitting the columns of
// the column-major matrices (coalesced reads, all loads independent).
#include "ls_internal.cuh"
#include "ls_strip.cuh"

namespace {

template <typename T>
struct Pool {
    const cpx_t<T>* base;  // strip l's first matrix
    size_t qq;
    __device__ __forceinline__ const cpx_t<T>* mat(size_t off) const { return base + off * qq; }
};

// Mat-vecs spread over a whole block of kMvThreads threads: warp w takes columns
// w, w + kMvWarps, ...; lane l takes rows l, l + 32, ... (RPT rows, q <= 32 RPT).
// Every thread issues its loads independently of the others (column-major
// matrices, so a warp reads 32 consecutive entries of a column), and the
// per-warp partial sums are reduced through shared memory.  A thread-per-row
// loop instead walks all q columns of a matrix one load at a time.
constexpr int kMvWarps = 8;
constexpr int kMvThreads = 32 * kMvWarps;

template <typename T, int RPT>
__device__ __forceinline__ void mv_accumulate(const cpx_t<T>* __restrict__ M, const cpx_t<T>* vs, int q,
                                              cpx_t<T> (&part)[RPT]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 4
    for (int c = warp; c < q; c += kMvWarps) {
        const cpx_t<T> vc = vs[c];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = lane + 32 * k;
            if (r < q) part[k] = cfma(__ldg(&M[(size_t)c * q + r]), vc, part[k]);
        }
    }
}

// The same for NM matrices at once: the loads of all of them for a column are
// issued before any multiply, so one pass over the columns has NM times more
// loads in flight.  Absent terms pass a valid matrix and a zero vector.
template <typename T, int RPT, int NM>
__device__ __forceinline__ void mv_accumulate_n(const cpx_t<T>* const (&M)[NM], const cpx_t<T>* const (&vs)[NM], int q,
                                                cpx_t<T> (&part)[RPT]) {
    using C = cpx_t<T>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 2
    for (int c = warp; c < q; c += kMvWarps) {
        C a[NM][RPT];
#pragma unroll
        for (int t = 0; t < NM; ++t)
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int r = lane + 32 * k;
                a[t][k] = r < q ? __ldg(&M[t][(size_t)c * q + r]) : czero<C>();
            }
#pragma unroll
        for (int t = 0; t < NM; ++t) {
            const C vc = vs[t][c];
#pragma unroll
            for (int k = 0; k < RPT; ++k) part[k] = cfma(a[t][k], vc, part[k]);
        }
    }
}

// red: kMvWarps * q entries of shared memory; returns the full sum for row threadIdx.x (< q)
template <typename T, int RPT>
__device__ __forceinline__ cpx_t<T> mv_reduce(cpx_t<T> (&part)[RPT], cpx_t<T>* red, int q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        const int r = lane + 32 * k;
        if (r < q) red[warp * q + r] = part[k];
    }
    __syncthreads();
    cpx_t<T> s = czero<cpx_t<T>>();
    if ((int)threadIdx.x < q)
        for (int w = 0; w < kMvWarps; ++w) s = s + red[w * q + threadIdx.x];
    return s;
}

// One step of the reduction for one block: out = base + sum_t M_t v_t, where the
// vectors are staged in shared memory with their signs applied.  MODE:
//   0 (level 0 odd):      x_j = D^{-1} x_j
//   1 (forward, level k): x_j = x_j - F x_{j-1} - G x_{j+1}            (even j)
//   2 (backward, level k): x_j = D^{-1} x_j - P x_{j-1} - Q x_{j+1}     (odd j)
//   3 (top block):         x_0 = D^{-1} x_0
template <typename T, int RPT, int MODE>
__global__ void __launch_bounds__(kMvThreads) k_cr_step(int q, int k, int nk, Pool<T> pool, size_t off_a,
                                                       size_t off_b, size_t off_c, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* v0 = reinterpret_cast<C*>(smem_raw);
    C* v1 = v0 + q;
    C* v2 = v1 + q;
    C* red = v2 + q;
    const int idx = blockIdx.x;
    const size_t s = (size_t)1 << k;
    const int j = MODE == 1 ? 2 * idx : (MODE == 3 ? 0 : 2 * idx + 1);
    const bool hw = j >= 1, he = j + 1 < nk;
    const int r = threadIdx.x;
    C* xj = x + ((size_t)j * s) * q;
    if (r < q) {
        if (MODE == 0 || MODE == 3) v0[r] = xj[r];
        if (MODE == 1) {
            v1[r] = hw ? -x[((size_t)(j - 1) * s) * q + r] : czero<C>();
            v2[r] = he ? -x[((size_t)(j + 1) * s) * q + r] : czero<C>();
        }
        if (MODE == 2) {
            v0[r] = xj[r];
            v1[r] = -x[((size_t)(j - 1) * s) * q + r];
            v2[r] = he ? -x[((size_t)(j + 1) * s) * q + r] : czero<C>();
        }
    }
    __syncthreads();
    C part[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) part[i] = czero<C>();
    if (MODE == 0 || MODE == 3) mv_accumulate<T, RPT>(pool.mat(off_a + idx), v0, q, part);
    if (MODE == 1) {  // a missing neighbour has a zero vector; its matrix slot reuses the other one
        const C* F = pool.mat(off_b + idx);
        const C* G = pool.mat(off_c + idx);
        const C* const Ms[2] = {hw ? F : G, he ? G : F};
        const C* const Vs[2] = {v1, v2};
        mv_accumulate_n<T, RPT, 2>(Ms, Vs, q, part);
    }
    if (MODE == 2) {
        const C* Dm = pool.mat(off_a + idx);
        const C* const Ms[3] = {Dm, pool.mat(off_b + idx), he ? pool.mat(off_c + idx) : Dm};
        const C* const Vs[3] = {v0, v1, v2};
        mv_accumulate_n<T, RPT, 3>(Ms, Vs, q, part);
    }
    const C sum = mv_reduce<T, RPT>(part, red, q);
    if (r < q) xj[r] = MODE == 1 ? xj[r] + sum : sum;
}

// level 0 backward, odd blocks: x_j = y_j - D^{-1} (W_j x_{j-1} + E_j x_{j+1})
template <typename T, int RPT>
__global__ void __launch_bounds__(kMvThreads) k_cr_l0_back(int q, int nb, const cpx_t<T>* __restrict__ cw,
                                                          const cpx_t<T>* __restrict__ ce, Pool<T> pool,
                                                          size_t off_dinv, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vt = reinterpret_cast<C*>(smem_raw);
    C* red = vt + q;
    const int o = blockIdx.x;
    const int j = 2 * o + 1;
    const int r = threadIdx.x;
    if (r < q) {
        C acc = czero<C>();
        const C* wj = cw + (size_t)j * 3 * q;
        const C* ej = ce + (size_t)j * 3 * q;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int rr = r + dz;
            if (rr < 0 || rr >= q) continue;
            acc = cfma(wj[(dz + 1) * q + r], x[(size_t)(j - 1) * q + rr], acc);
            if (j + 1 < nb) acc = cfma(ej[(dz + 1) * q + r], x[(size_t)(j + 1) * q + rr], acc);
        }
        vt[r] = -acc;
    }
    __syncthreads();
    C part[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) part[i] = czero<C>();
    mv_accumulate<T, RPT>(pool.mat(off_dinv + o), vt, q, part);
    const C sum = mv_reduce<T, RPT>(part, red, q);
    if (r < q) x[(size_t)j * q + r] = x[(size_t)j * q + r] + sum;
}

// level 0, even blocks: b_j -= W_j y_{j-1} + E_j y_{j+1} (W, E tridiagonal from the stencil)
template <typename T>
__global__ void k_l0_even(int q, int nb, const cpx_t<T>* __restrict__ cw, const cpx_t<T>* __restrict__ ce,
                          cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    const int j = 2 * blockIdx.x;
    const int r = threadIdx.x;
    if (r >= q) return;
    C acc = x[(size_t)j * q + r];
    const C* wj = cw + (size_t)j * 3 * q;
    const C* ej = ce + (size_t)j * 3 * q;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int rr = r + dz;
        if (rr < 0 || rr >= q) continue;
        if (j >= 1) acc = cfms(wj[(dz + 1) * q + r], x[(size_t)(j - 1) * q + rr], acc);
        if (j + 1 < nb) acc = cfms(ej[(dz + 1) * q + r], x[(size_t)(j + 1) * q + rr], acc);
    }
    x[(size_t)j * q + r] = acc;
}

// g^l = chi_{Omega^l} g (+ injection from the layer above), copied to the solution buffer
template <typename T>
__global__ void k_gather(StripGeom g, const cpx_t<T>* __restrict__ inj, int l,
                         const double2* __restrict__ gf, cpx_t<T>* __restrict__ rhs, cpx_t<T>* __restrict__ sol,
                         const cpx_t<T>* __restrict__ above, cpx_t<T>* __restrict__ trace_above) {
    using C = cpx_t<T>;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = g.q, n = g.n, E = g.E, t = g.t;
    if (e >= (size_t)n * q) return;
    const int i = (int)(e / q), r = (int)(e % q);
    if (above && r == 0) trace_above[i] = above[(size_t)i * q + E - 1];  // w^{l+1}_0, kept for the upward sweep
    double2 val = make_double2(0, 0);
    if (r >= E && r < E + t) val = gf[(size_t)(l * t - E + r) * n + i];
    if (above) {
        const cpx_t<T>* c0 = inj + (size_t)l * 12 * n;  // slots 0, 1 of layer l: [slot][dx+1][i]
        if (r == E + t - 1) {  // -C^l_{n,n+1} w^{l+1}_1 ; w^{l+1}_1 = row E of layer l+1
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx >= n) continue;
                val = cfms(ccast<double2>(c0[(size_t)(0 * 3 + dx + 1) * n + i]),
                           ccast<double2>(above[(size_t)(i + dx) * q + E]), val);
            }
        } else if (r == E + t) {  // +C^l_{n+1,n} w^{l+1}_0 ; w^{l+1}_0 = row E-1 of layer l+1
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx >= n) continue;
                val = cfma(ccast<double2>(c0[(size_t)(1 * 3 + dx + 1) * n + i]),
                           ccast<double2>(above[(size_t)(i + dx) * q + E - 1]), val);
            }
        }
    }
    const C cv = ccast<C>(val);
    rhs[e] = cv;
    sol[e] = cv;
}

// sol = g^l + injection from the layer below (upward sweep)
template <typename T>
__global__ void k_inject_up(StripGeom g, const cpx_t<T>* __restrict__ inj, int l,
                            const cpx_t<T>* __restrict__ rhs, cpx_t<T>* __restrict__ sol,
                            const cpx_t<T>* __restrict__ below, const cpx_t<T>* __restrict__ trace_self) {
    using C = cpx_t<T>;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = g.q, n = g.n, E = g.E, t = g.t;
    if (e >= (size_t)n * q) return;
    const int i = (int)(e / q), r = (int)(e % q);
    if (r != E && r != E - 1) {
        sol[e] = rhs[e];
        return;
    }
    double2 val = ccast<double2>(rhs[e]);
    const cpx_t<T>* c0 = inj + (size_t)l * 12 * n;  // slots 2, 3 of layer l: [slot][dx+1][i]
    if (r == E) {  // -C^l_{1,0} (v^{l-1}_n - w^l_0) ; v^{l-1}_n = row E+t-1 of layer l-1
        for (int dx = -1; dx <= 1; ++dx) {
            if (i + dx < 0 || i + dx >= n) continue;
            const double2 p0 = ccast<double2>(below[(size_t)(i + dx) * q + E + t - 1]) - ccast<double2>(trace_self[i + dx]);
            val = cfms(ccast<double2>(c0[(size_t)(2 * 3 + dx + 1) * n + i]), p0, val);
        }
    } else {  // +C^l_{0,1} v^{l-1}_{n+1} ; v^{l-1}_{n+1} = row E+t of layer l-1
        for (int dx = -1; dx <= 1; ++dx) {
            if (i + dx < 0 || i + dx >= n) continue;
            val = cfma(ccast<double2>(c0[(size_t)(3 * 3 + dx + 1) * n + i]),
                       ccast<double2>(below[(size_t)(i + dx) * q + E + t]), val);
        }
    }
    sol[e] = ccast<C>(val);
}

// v = rows 1..n of every layer's solution (concatenation)
template <typename T>
__global__ void k_scatter(StripGeom g, const cpx_t<T>* __restrict__ sol, size_t strip_stride, double2* __restrict__ v) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n;
    if (e >= (size_t)n * n) return;
    const int z = (int)(e / n), i = (int)(e % n);
    const int l = z / g.t, r = z - l * g.t + g.E;
    v[e] = ccast<double2>(sol[(size_t)l * strip_stride + (size_t)i * g.q + r]);
}

// natural strip layout (q rows x n, x fastest) <-> block layout (i*q + r)
template <typename T>
__global__ void k_strip_in(int n, int q, const double2* __restrict__ b, cpx_t<T>* __restrict__ x) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * q) return;
    const int i = (int)(e / q), r = (int)(e % q);
    x[e] = ccast<cpx_t<T>>(b[(size_t)r * n + i]);
}
template <typename T>
__global__ void k_strip_out(int n, int q, const cpx_t<T>* __restrict__ x, double2* __restrict__ b) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * q) return;
    const int r = (int)(e / n), i = (int)(e % n);
    b[e] = ccast<double2>(x[(size_t)i * q + r]);
}

__global__ void k_add(size_t N, const double2* __restrict__ a, double2* __restrict__ b) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x)
        b[k] = b[k] + a[k];
}

StripGeom geom_of(const ls_handle* h) { return StripGeom{h->n, h->t, h->E, h->q, h->opts.shift / h->omega}; }

template <typename T, int RPT>
int cr_solve_rpt(ls_handle* h, int dir, int l, cpx_t<T>* x) {
    using C = cpx_t<T>;
    const DirFactors& F = h->fac[dir];
    const int q = h->q, n = h->n;
    const size_t qq = (size_t)q * q;
    const cpx_t<T>* base;
    if constexpr (sizeof(T) == 4) base = F.pool32;
    else base = F.pool64;
    Pool<T> pool{base + (size_t)l * F.mats_per_strip * qq, qq};
    const int thr = (q + 31) / 32 * 32;
    const size_t sm_step = (3 + kMvWarps) * sizeof(C) * q;
    const size_t sm_back = (1 + kMvWarps) * sizeof(C) * q;
    const CrLevel& l0 = F.lev[0];
    if (l0.nodd)
        LS_LAUNCH(h, (k_cr_step<T, RPT, 0>), l0.nodd, kMvThreads, sm_step, q, 0, l0.nk, pool, l0.off_dinv,
                  (size_t)0, (size_t)0, x);
    const C* cw = static_cast<const C*>(F.cw) + (size_t)l * n * 3 * q;
    const C* ce = static_cast<const C*>(F.ce) + (size_t)l * n * 3 * q;
    LS_LAUNCH(h, k_l0_even<T>, l0.neven, thr, 0, q, n, cw, ce, x);
    for (int k = 1; k < F.K; ++k) {
        const CrLevel& lv = F.lev[k];
        LS_LAUNCH(h, (k_cr_step<T, RPT, 1>), lv.neven, kMvThreads, sm_step, q, k, lv.nk, pool, (size_t)0, lv.off_f,
                  lv.off_g, x);
    }
    LS_LAUNCH(h, (k_cr_step<T, RPT, 3>), 1, kMvThreads, sm_step, q, 0, 1, pool, F.off_top, (size_t)0, (size_t)0, x);
    for (int k = F.K - 1; k >= 1; --k) {
        const CrLevel& lv = F.lev[k];
        if (lv.nodd)
            LS_LAUNCH(h, (k_cr_step<T, RPT, 2>), lv.nodd, kMvThreads, sm_step, q, k, lv.nk, pool, lv.off_dinv,
                      lv.off_p, lv.off_q, x);
    }
    if (l0.nodd)
        LS_LAUNCH(h, (k_cr_l0_back<T, RPT>), l0.nodd, kMvThreads, sm_back, q, n, cw, ce, pool, l0.off_dinv, x);
    return LS_OK;
}

template <typename T>
int cr_solve(ls_handle* h, int dir, int l, cpx_t<T>* x) {
    const int rpt = (h->q + 31) / 32;
    switch (rpt) {
        case 1: return cr_solve_rpt<T, 1>(h, dir, l, x);
        case 2: return cr_solve_rpt<T, 2>(h, dir, l, x);
        case 3: return cr_solve_rpt<T, 3>(h, dir, l, x);
        default: return cr_solve_rpt<T, 4>(h, dir, l, x);
    }
}

template <typename T>
int sweep_impl(ls_handle* h, int dir, const double2* g, double2* v) {
    using C = cpx_t<T>;
    const int n = h->n, q = h->q, L = h->L;
    const size_t sstride = (size_t)n * q;
    C* rhs = static_cast<C*>(h->srhs);
    C* sol = static_cast<C*>(h->ssol);
    C* trc = static_cast<C*>(h->strace);
    const DirFactors& F = h->fac[dir];
    const StripGeom geo = geom_of(h);
    const unsigned nbs = (unsigned)((sstride + 255) / 256);
    for (int l = L - 1; l >= 0; --l) {  // downward sweep
        LS_LAUNCH(h, k_gather<T>, nbs, 256, 0, geo, static_cast<const C*>(F.cinj), l, g, rhs + l * sstride, sol + l * sstride,
                  l < L - 1 ? sol + (l + 1) * sstride : (const C*)nullptr,
                  l < L - 1 ? trc + (size_t)(l + 1) * n : (C*)nullptr);
        LS_TRY(cr_solve<T>(h, dir, l, sol + l * sstride));
    }
    for (int l = 1; l < L; ++l) {  // upward sweep
        LS_LAUNCH(h, k_inject_up<T>, nbs, 256, 0, geo, static_cast<const C*>(F.cinj), l, rhs + l * sstride, sol + l * sstride,
                  sol + (l - 1) * sstride, trc + (size_t)l * n);
        LS_TRY(cr_solve<T>(h, dir, l, sol + l * sstride));
    }
    const size_t N = (size_t)n * n;
    LS_LAUNCH(h, k_scatter<T>, (unsigned)((N + 255) / 256), 256, 0, geo, sol, sstride, v);
    return LS_OK;
}

}  // namespace

int ls_sweep_alloc(ls_handle* h) {
    const size_t cnt = (size_t)h->L * h->n * h->q;
    const size_t es = h->prec == LS_MIXED ? sizeof(float2) : sizeof(double2);
    LS_CUDA(cudaMalloc(&h->srhs, es * cnt));
    LS_CUDA(cudaMalloc(&h->ssol, es * cnt));
    LS_CUDA(cudaMalloc(&h->strace, es * (size_t)h->L * h->n));
    const size_t N = (size_t)h->n * h->n;
    LS_CUDA(cudaMalloc(&h->vtmp, sizeof(double2) * N * 4));
    LS_CUDA(cudaMalloc(&h->bd_in, sizeof(double2) * N));
    LS_CUDA(cudaMalloc(&h->bd_out, sizeof(double2) * N));
    return LS_OK;
}

// Algorithm 1 on direction dir (0: horizontal layers; 1: vertical layers).
int ls_sweep_dir(ls_handle* h, int dir, const double2* g, double2* v) {
    const size_t N = (size_t)h->n * h->n;
    double2* t0 = static_cast<double2*>(h->vtmp);
    double2* t1 = t0 + N;
    if (dir == 0) {
        if (h->prec == LS_MIXED) return sweep_impl<float>(h, 0, g, v);
        return sweep_impl<double>(h, 0, g, v);
    }
    LS_TRY(ls_transpose64(h, g, t0));
    if (h->prec == LS_MIXED) LS_TRY(sweep_impl<float>(h, 1, t0, t1));
    else LS_TRY(sweep_impl<double>(h, 1, t0, t1));
    return ls_transpose64(h, t1, v);
}

// Algorithm 2: v = u1 + u2, u1 = Alg. 1 horizontal (g), u2 = Alg. 1 vertical (g - C u1).
static int bd_direct(ls_handle* h, const double2* g, double2* v) {
    const size_t N = (size_t)h->n * h->n;
    double2* u1 = static_cast<double2*>(h->vtmp) + 2 * N;
    double2* e = u1 + N;
    LS_TRY(ls_sweep_dir(h, 0, g, u1));
    LS_TRY(ls_stencil_apply(h, 0, 2, u1, g, e));   // e = g - C u1
    LS_TRY(ls_sweep_dir(h, 1, e, v));
    LS_LAUNCH(h, k_add, 608, 256, 0, N, u1, v);
    return LS_OK;
}

void ls_bd_graph_free(ls_handle* h) {
    if (h->bd_exec) cudaGraphExecDestroy(h->bd_exec);
    if (h->bd_graph) cudaGraphDestroy(h->bd_graph);
    h->bd_exec = nullptr;
    h->bd_graph = nullptr;
    h->bd_nodes = 0;
}

// Capture Algorithm 2 on the staging buffers once (the sequence of launches and all
// pointers are fixed after ls_factor), then replay it.
static int bd_capture(ls_handle* h) {
    cudaStream_t cap = nullptr;
    LS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = h->stream;
    const long long l0 = h->launches;
    h->stream = cap;
    int rc = LS_OK;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = bd_direct(h, h->bd_in, h->bd_out);
        e = cudaStreamEndCapture(cap, &graph);
    }
    h->stream = saved;
    const long long nodes = h->launches - l0;
    h->launches = l0;
    cudaStreamDestroy(cap);
    if (rc != LS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return ls_cuda_fail(e);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return ls_cuda_fail(e);
    }
    h->bd_graph = graph;
    h->bd_exec = exec;
    h->bd_nodes = nodes;
    return LS_OK;
}

int ls_bd(ls_handle* h, const double2* g, double2* v) {
    if (!h->opts.use_graphs) return bd_direct(h, g, v);
    if (!h->bd_exec) LS_TRY(bd_capture(h));
    const size_t N = (size_t)h->n * h->n;
    LS_CUDA(cudaMemcpyAsync(h->bd_in, g, sizeof(double2) * N, cudaMemcpyDeviceToDevice, h->stream));
    LS_CUDA(cudaGraphLaunch(h->bd_exec, h->stream));
    h->launches += h->bd_nodes;
    LS_CUDA(cudaMemcpyAsync(v, h->bd_out, sizeof(double2) * N, cudaMemcpyDeviceToDevice, h->stream));
    return LS_OK;
}

int ls_strip_solve(ls_handle* h, int dir, int layer, const double2* b, double2* x) {
    const int n = h->n, q = h->q;
    const size_t cnt = (size_t)n * q;
    const unsigned nb = (unsigned)((cnt + 255) / 256);
    if (h->prec == LS_MIXED) {
        float2* s = static_cast<float2*>(h->ssol);
        LS_LAUNCH(h, k_strip_in<float>, nb, 256, 0, n, q, b, s);
        LS_TRY(cr_solve<float>(h, dir, layer, s));
        LS_LAUNCH(h, k_strip_out<float>, nb, 256, 0, n, q, s, x);
    } else {
        double2* s = static_cast<double2*>(h->ssol);
        LS_LAUNCH(h, k_strip_in<double>, nb, 256, 0, n, q, b, s);
        LS_TRY(cr_solve<double>(h, dir, layer, s));
        LS_LAUNCH(h, k_strip_out<double>, nb, 256, 0, n, q, s, x);
    }
    return LS_OK;
}
