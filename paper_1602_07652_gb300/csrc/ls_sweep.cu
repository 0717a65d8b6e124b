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
// threads handles one q x q mat-vec set with one thread per row, reading the
// column-major matrices coalesced.
#include "ls_internal.cuh"
#include "ls_strip.cuh"

namespace {

template <typename T>
struct Pool {
    const cpx_t<T>* base;  // strip l's first matrix
    size_t qq;
    __device__ __forceinline__ const cpx_t<T>* mat(size_t off) const { return base + off * qq; }
};

// acc -= M v (or +=), thread `r` = row; M column-major q x q, v in shared memory
template <typename T>
__device__ __forceinline__ cpx_t<T> matvec_row(const cpx_t<T>* __restrict__ M, const cpx_t<T>* v, int q, int r,
                                               cpx_t<T> acc, bool subtract) {
    if (subtract) {
#pragma unroll 4
        for (int c = 0; c < q; ++c) acc = cfms(__ldg(&M[(size_t)c * q + r]), v[c], acc);
    } else {
#pragma unroll 4
        for (int c = 0; c < q; ++c) acc = cfma(__ldg(&M[(size_t)c * q + r]), v[c], acc);
    }
    return acc;
}

// level 0, odd blocks: y_j = Dinv_j b_j
template <typename T>
__global__ void k_l0_odd(int q, Pool<T> pool, size_t off_dinv, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vb = reinterpret_cast<C*>(smem_raw);
    const int j = 2 * blockIdx.x + 1;
    const int r = threadIdx.x;
    C* xb = x + (size_t)j * q;
    if (r < q) vb[r] = xb[r];
    __syncthreads();
    if (r < q) xb[r] = matvec_row<T>(pool.mat(off_dinv + blockIdx.x), vb, q, r, czero<C>(), false);
}

// level 0, even blocks: b_j -= W_j y_{j-1} + E_j y_{j+1} (W, E tridiagonal from the stencil)
template <typename T>
__global__ void k_l0_even(StripGeom g, const StencilTables* __restrict__ tab, const double* __restrict__ m, int l,
                          int nb, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    const int j = 2 * blockIdx.x;
    const int r = threadIdx.x, q = g.q;
    if (r >= q) return;
    double2 acc = ccast<double2>(x[(size_t)j * q + r]);
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int rr = r + dz;
        if (rr < 0 || rr >= q) continue;
        if (j >= 1) acc = cfms(strip_coef(g, tab, m, l, r, j, -1, dz), ccast<double2>(x[(size_t)(j - 1) * q + rr]), acc);
        if (j + 1 < nb) acc = cfms(strip_coef(g, tab, m, l, r, j, 1, dz), ccast<double2>(x[(size_t)(j + 1) * q + rr]), acc);
    }
    x[(size_t)j * q + r] = ccast<C>(acc);
}

// level k >= 1 forward, even blocks j of level k (global block j << k):
// b_j -= F_j b_{j-1} + G_j b_{j+1}
template <typename T>
__global__ void k_fwd(int q, int k, int nk, Pool<T> pool, size_t off_f, size_t off_g, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vw = reinterpret_cast<C*>(smem_raw);
    C* ve = vw + q;
    const int e = blockIdx.x;  // even index / 2
    const int j = 2 * e;
    const int r = threadIdx.x;
    const bool hw = j >= 1, he = j + 1 < nk;
    const size_t s = (size_t)1 << k;
    if (r < q) {
        if (hw) vw[r] = x[((size_t)(j - 1) * s) * q + r];
        if (he) ve[r] = x[((size_t)(j + 1) * s) * q + r];
    }
    __syncthreads();
    if (r >= q) return;
    C acc = x[((size_t)j * s) * q + r];
    if (hw) acc = matvec_row<T>(pool.mat(off_f + e), vw, q, r, acc, true);
    if (he) acc = matvec_row<T>(pool.mat(off_g + e), ve, q, r, acc, true);
    x[((size_t)j * s) * q + r] = acc;
}

// top: x_0 = Dinv b_0
template <typename T>
__global__ void k_top(int q, Pool<T> pool, size_t off_top, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vb = reinterpret_cast<C*>(smem_raw);
    const int r = threadIdx.x;
    if (r < q) vb[r] = x[r];
    __syncthreads();
    if (r < q) x[r] = matvec_row<T>(pool.mat(off_top), vb, q, r, czero<C>(), false);
}

// The last levels of the reduction (at most kTopBlocks blocks) in one block of
// threads: forward levels k0..K-1, the top block, backward levels K-1..k0, with
// block barriers between levels instead of separate launches.  Thread group g
// (of kGroups, 128 threads each) handles blocks g, g + kGroups, ...; global
// memory written before a __syncthreads is visible to the whole block after it.
constexpr int kGroups = 4;
constexpr int kTopBlocks = 2 * kGroups;

struct TopLevels {
    int k0, K;
    int nk[16];
    size_t off_dinv[16], off_p[16], off_q[16], off_f[16], off_g[16];
    size_t off_top;
};

template <typename T>
__global__ void __launch_bounds__(128 * kGroups) k_top_levels(int q, TopLevels tl, Pool<T> pool, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / 128, r = threadIdx.x % 128;
    C* v0 = reinterpret_cast<C*>(smem_raw) + (size_t)grp * 3 * q;
    C* v1 = v0 + q;
    C* v2 = v1 + q;
    for (int k = tl.k0; k < tl.K; ++k) {  // forward: even blocks
        const int nk = tl.nk[k];
        const size_t s = (size_t)1 << k;
        const int neven = (nk + 1) / 2;
        for (int base = 0; base < neven; base += kGroups) {
            const int e = base + grp;
            const int j = 2 * e;
            const bool act = e < neven, hw = act && j >= 1, he = act && j + 1 < nk;
            if (r < q) {
                if (hw) v0[r] = x[((size_t)(j - 1) * s) * q + r];
                if (he) v1[r] = x[((size_t)(j + 1) * s) * q + r];
            }
            __syncthreads();
            if (act && r < q) {
                C acc = x[((size_t)j * s) * q + r];
                if (hw) acc = matvec_row<T>(pool.mat(tl.off_f[k] + e), v0, q, r, acc, true);
                if (he) acc = matvec_row<T>(pool.mat(tl.off_g[k] + e), v1, q, r, acc, true);
                x[((size_t)j * s) * q + r] = acc;
            }
            __syncthreads();
        }
    }
    if (grp == 0 && r < q) v0[r] = x[r];  // top block
    __syncthreads();
    if (grp == 0 && r < q) x[r] = matvec_row<T>(pool.mat(tl.off_top), v0, q, r, czero<C>(), false);
    __syncthreads();
    for (int k = tl.K - 1; k >= tl.k0; --k) {  // backward: odd blocks
        const int nk = tl.nk[k];
        const size_t s = (size_t)1 << k;
        const int nodd = nk / 2;
        for (int base = 0; base < nodd; base += kGroups) {
            const int o = base + grp;
            const int j = 2 * o + 1;
            const bool act = o < nodd, he = act && j + 1 < nk;
            if (act && r < q) {
                v0[r] = x[((size_t)j * s) * q + r];
                v1[r] = x[((size_t)(j - 1) * s) * q + r];
                if (he) v2[r] = x[((size_t)(j + 1) * s) * q + r];
            }
            __syncthreads();
            if (act && r < q) {
                C acc = matvec_row<T>(pool.mat(tl.off_dinv[k] + o), v0, q, r, czero<C>(), false);
                acc = matvec_row<T>(pool.mat(tl.off_p[k] + o), v1, q, r, acc, true);
                if (he) acc = matvec_row<T>(pool.mat(tl.off_q[k] + o), v2, q, r, acc, true);
                x[((size_t)j * s) * q + r] = acc;
            }
            __syncthreads();
        }
    }
}

// level k >= 1 backward, odd blocks: x_j = Dinv_j b_j - P_j x_{j-1} - Q_j x_{j+1}
template <typename T>
__global__ void k_bwd(int q, int k, int nk, Pool<T> pool, size_t off_dinv, size_t off_p, size_t off_q,
                      cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vb = reinterpret_cast<C*>(smem_raw);
    C* vw = vb + q;
    C* ve = vw + q;
    const int o = blockIdx.x;  // odd index
    const int j = 2 * o + 1;
    const int r = threadIdx.x;
    const bool he = j + 1 < nk;
    const size_t s = (size_t)1 << k;
    if (r < q) {
        vb[r] = x[((size_t)j * s) * q + r];
        vw[r] = x[((size_t)(j - 1) * s) * q + r];
        if (he) ve[r] = x[((size_t)(j + 1) * s) * q + r];
    }
    __syncthreads();
    if (r >= q) return;
    C acc = matvec_row<T>(pool.mat(off_dinv + o), vb, q, r, czero<C>(), false);
    acc = matvec_row<T>(pool.mat(off_p + o), vw, q, r, acc, true);
    if (he) acc = matvec_row<T>(pool.mat(off_q + o), ve, q, r, acc, true);
    x[((size_t)j * s) * q + r] = acc;
}

// level 0 backward, odd blocks: x_j = y_j - Dinv_j (W_j x_{j-1} + E_j x_{j+1})
template <typename T>
__global__ void k_l0_back(StripGeom g, const StencilTables* __restrict__ tab, const double* __restrict__ m, int l,
                          int nb, Pool<T> pool, size_t off_dinv, cpx_t<T>* __restrict__ x) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vt = reinterpret_cast<C*>(smem_raw);
    const int o = blockIdx.x;
    const int j = 2 * o + 1;
    const int r = threadIdx.x, q = g.q;
    if (r < q) {
        double2 acc = make_double2(0, 0);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int rr = r + dz;
            if (rr < 0 || rr >= q) continue;
            acc = cfma(strip_coef(g, tab, m, l, r, j, -1, dz), ccast<double2>(x[(size_t)(j - 1) * q + rr]), acc);
            if (j + 1 < nb) acc = cfma(strip_coef(g, tab, m, l, r, j, 1, dz), ccast<double2>(x[(size_t)(j + 1) * q + rr]), acc);
        }
        vt[r] = ccast<C>(acc);
    }
    __syncthreads();
    if (r >= q) return;
    C* xb = x + (size_t)j * q;
    xb[r] = matvec_row<T>(pool.mat(off_dinv + o), vt, q, r, xb[r], true);
}

// g^l = chi_{Omega^l} g (+ injection from the layer above), copied to the solution buffer
template <typename T>
__global__ void k_gather(StripGeom g, const StencilTables* __restrict__ tab, const double* __restrict__ m, int l,
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
        if (r == E + t - 1) {  // -C^l_{n,n+1} w^{l+1}_1 ; w^{l+1}_1 = row E of layer l+1
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx >= n) continue;
                val = cfms(strip_coef(g, tab, m, l, r, i, dx, 1), ccast<double2>(above[(size_t)(i + dx) * q + E]), val);
            }
        } else if (r == E + t) {  // +C^l_{n+1,n} w^{l+1}_0 ; w^{l+1}_0 = row E-1 of layer l+1
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx >= n) continue;
                val = cfma(strip_coef(g, tab, m, l, r, i, dx, -1), ccast<double2>(above[(size_t)(i + dx) * q + E - 1]), val);
            }
        }
    }
    const C cv = ccast<C>(val);
    rhs[e] = cv;
    sol[e] = cv;
}

// sol = g^l + injection from the layer below (upward sweep)
template <typename T>
__global__ void k_inject_up(StripGeom g, const StencilTables* __restrict__ tab, const double* __restrict__ m, int l,
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
    if (r == E) {  // -C^l_{1,0} (v^{l-1}_n - w^l_0) ; v^{l-1}_n = row E+t-1 of layer l-1
        for (int dx = -1; dx <= 1; ++dx) {
            if (i + dx < 0 || i + dx >= n) continue;
            const double2 p0 = ccast<double2>(below[(size_t)(i + dx) * q + E + t - 1]) - ccast<double2>(trace_self[i + dx]);
            val = cfms(strip_coef(g, tab, m, l, r, i, dx, -1), p0, val);
        }
    } else {  // +C^l_{0,1} v^{l-1}_{n+1} ; v^{l-1}_{n+1} = row E+t of layer l-1
        for (int dx = -1; dx <= 1; ++dx) {
            if (i + dx < 0 || i + dx >= n) continue;
            val = cfma(strip_coef(g, tab, m, l, r, i, dx, 1), ccast<double2>(below[(size_t)(i + dx) * q + E + t]), val);
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

template <typename T>
int cr_solve(ls_handle* h, int dir, int l, cpx_t<T>* x) {
    using C = cpx_t<T>;
    const DirFactors& F = h->fac[dir];
    const int q = h->q, n = h->n;
    const size_t qq = (size_t)q * q;
    const cpx_t<T>* base;
    if constexpr (sizeof(T) == 4) base = F.pool32;
    else base = F.pool64;
    Pool<T> pool{base + (size_t)l * F.mats_per_strip * qq, qq};
    const StripGeom g = geom_of(h);
    const int thr = (q + 31) / 32 * 32;
    const CrLevel& l0 = F.lev[0];
    if (l0.nodd) LS_LAUNCH(h, k_l0_odd<T>, l0.nodd, thr, sizeof(C) * q, q, pool, l0.off_dinv, x);
    LS_LAUNCH(h, k_l0_even<T>, l0.neven, thr, 0, g, F.tab, F.m, l, n, x);
    // levels >= 1 with more than kTopBlocks blocks get one launch each; the rest
    // (and the top block) run in one single-block launch
    int k0 = 1;
    while (k0 < F.K && F.lev[k0].nk > kTopBlocks) ++k0;
    for (int k = 1; k < k0; ++k) {
        const CrLevel& lv = F.lev[k];
        LS_LAUNCH(h, k_fwd<T>, lv.neven, thr, 2 * sizeof(C) * q, q, k, lv.nk, pool, lv.off_f, lv.off_g, x);
    }
    if (F.K > 16) return LS_EINVAL;
    TopLevels tl{};
    tl.k0 = k0;
    tl.K = F.K;
    for (int k = k0; k < F.K; ++k) {
        tl.nk[k] = F.lev[k].nk;
        tl.off_dinv[k] = F.lev[k].off_dinv;
        tl.off_p[k] = F.lev[k].off_p;
        tl.off_q[k] = F.lev[k].off_q;
        tl.off_f[k] = F.lev[k].off_f;
        tl.off_g[k] = F.lev[k].off_g;
    }
    tl.off_top = F.off_top;
    LS_LAUNCH(h, k_top_levels<T>, 1, 128 * kGroups, 3 * kGroups * sizeof(C) * q, q, tl, pool, x);
    for (int k = k0 - 1; k >= 1; --k) {
        const CrLevel& lv = F.lev[k];
        if (lv.nodd)
            LS_LAUNCH(h, k_bwd<T>, lv.nodd, thr, 3 * sizeof(C) * q, q, k, lv.nk, pool, lv.off_dinv, lv.off_p,
                      lv.off_q, x);
    }
    if (l0.nodd) LS_LAUNCH(h, k_l0_back<T>, l0.nodd, thr, sizeof(C) * q, g, F.tab, F.m, l, n, pool, l0.off_dinv, x);
    return LS_OK;
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
        LS_LAUNCH(h, k_gather<T>, nbs, 256, 0, geo, F.tab, F.m, l, g, rhs + l * sstride, sol + l * sstride,
                  l < L - 1 ? sol + (l + 1) * sstride : (const C*)nullptr,
                  l < L - 1 ? trc + (size_t)(l + 1) * n : (C*)nullptr);
        LS_TRY(cr_solve<T>(h, dir, l, sol + l * sstride));
    }
    for (int l = 1; l < L; ++l) {  // upward sweep
        LS_LAUNCH(h, k_inject_up<T>, nbs, 256, 0, geo, F.tab, F.m, l, rhs + l * sstride, sol + l * sstride,
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
