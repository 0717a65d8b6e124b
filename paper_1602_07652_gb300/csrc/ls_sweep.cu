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
//
// Batches: every kernel takes nb right-hand sides at once (batch member b's
// strips at offset b * SB, its grid vectors at offset b * N).  A reduction step
// loads each factor matrix once and applies it to all nb vectors, so a batch
// shares both the factor traffic and the chain of dependent launches.
#include <vector>

#include "ls_internal.cuh"
#include "ls_strip.cuh"

namespace {

template <typename T>
struct Pool {
    const cpx_t<T>* base;  // strip l's first matrix
    size_t qq;
    __device__ __forceinline__ const cpx_t<T>* mat(size_t off) const { return base + off * qq; }
};

constexpr int kMvWarps = 8;
constexpr int kMvThreads = 32 * kMvWarps;

// One reduction step for one block j and NB (>= nb) batch members:
//   out_b = base_b + sum_t M_t v_{t,b}
// Warp w takes columns w, w + 8, ...; lane l takes rows l, l + 32, ... (RPT rows);
// each matrix entry is loaded once and used for every batch member; the
// vectors (signs applied) sit in shared memory, partial sums are reduced there.
//   MODE 0 (level 0 odd):    x_j = D^{-1} x_j
//   MODE 1 (forward):        x_j = x_j - F x_{j-1} - G x_{j+1}          (even j)
//   MODE 2 (backward):       x_j = D^{-1} x_j - P x_{j-1} - Q x_{j+1}   (odd j)
//   MODE 3 (top block):      x_0 = D^{-1} x_0
//
// Split levels (S > 1, for levels with fewer blocks than the GPU has SMs): S CTAs
// share a block, CTA p taking the columns [p q / S, (p+1) q / S) of its matrices.
// Each writes its partial sums to `partial`, and the CTA that arrives last at the
// block's counter (an atomic increment; nobody waits) adds the S partials in the
// fixed order p = 0..S-1, writes the block's result and resets the counter.  The
// result does not depend on which CTA arrives last, and x_j is overwritten only
// after every CTA of the block has read it.
template <typename T, int RPT, int MODE, int NB>
__global__ void __launch_bounds__(kMvThreads, NB >= 4 ? 2 : 1) k_cr_step(int q, int k, int nk, Pool<T> pool, size_t off_a,
                                                       size_t off_b, size_t off_c, cpx_t<T>* __restrict__ x,
                                                       size_t SB, int nb, int S, cpx_t<T>* __restrict__ partial,
                                                       unsigned* __restrict__ counter) {
    using C = cpx_t<T>;
    constexpr int NM = MODE == 1 ? 2 : (MODE == 2 ? 3 : 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int last;
    C* vin = reinterpret_cast<C*>(smem_raw);     // [NM][NB][q]
    C* red = vin + (size_t)NM * NB * q;          // [kMvWarps][NB][q]
    const int idx = blockIdx.x / S, sp = blockIdx.x - idx * S;
    const int cbeg = q * sp / S, cend = q * (sp + 1) / S;
    const size_t s = (size_t)1 << k;
    const int j = MODE == 1 ? 2 * idx : (MODE == 3 ? 0 : 2 * idx + 1);
    const bool hw = j >= 1, he = j + 1 < nk;
    for (int o = threadIdx.x; o < NM * NB * q; o += kMvThreads) {
        const int t = o / (NB * q), b = (o / q) % NB, r = o % q;
        C val = czero<C>();
        if (b < nb) {
            const C* xb = x + (size_t)b * SB;
            if (MODE == 0 || MODE == 3) val = xb[((size_t)j * s) * q + r];
            if (MODE == 1) {
                if (t == 0 && hw) val = -xb[((size_t)(j - 1) * s) * q + r];
                if (t == 1 && he) val = -xb[((size_t)(j + 1) * s) * q + r];
            }
            if (MODE == 2) {
                if (t == 0) val = xb[((size_t)j * s) * q + r];
                if (t == 1) val = -xb[((size_t)(j - 1) * s) * q + r];
                if (t == 2 && he) val = -xb[((size_t)(j + 1) * s) * q + r];
            }
        }
        vin[o] = val;
    }
    __syncthreads();
    const C* Ms[NM];
    if (MODE == 0 || MODE == 3) Ms[0] = pool.mat(off_a + idx);
    if (MODE == 1) {  // a missing neighbour has zero vectors; its matrix slot reuses the other one
        const C* F = pool.mat(off_b + idx);
        const C* G = pool.mat(off_c + idx);
        Ms[0] = hw ? F : G;
        Ms[NM - 1] = he ? G : F;
    }
    if (MODE == 2) {
        const C* Dm = pool.mat(off_a + idx);
        Ms[0] = Dm;
        Ms[1] = pool.mat(off_b + idx);
        Ms[NM - 1] = he ? pool.mat(off_c + idx) : Dm;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C part[RPT][NB];
#pragma unroll
    for (int kk = 0; kk < RPT; ++kk)
#pragma unroll
        for (int b = 0; b < NB; ++b) part[kk][b] = czero<C>();
#pragma unroll 2
    for (int c = cbeg + warp; c < cend; c += kMvWarps) {
        C a[NM][RPT];
#pragma unroll
        for (int t = 0; t < NM; ++t)
#pragma unroll
            for (int kk = 0; kk < RPT; ++kk) {
                const int r = lane + 32 * kk;
                a[t][kk] = r < q ? __ldg(&Ms[t][(size_t)c * q + r]) : czero<C>();
            }
#pragma unroll
        for (int t = 0; t < NM; ++t)
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const C vc = vin[((size_t)t * NB + b) * q + c];
#pragma unroll
                for (int kk = 0; kk < RPT; ++kk) part[kk][b] = cfma(a[t][kk], vc, part[kk][b]);
            }
    }
#pragma unroll
    for (int kk = 0; kk < RPT; ++kk) {
        const int r = lane + 32 * kk;
        if (r < q)
#pragma unroll
            for (int b = 0; b < NB; ++b) red[((size_t)warp * NB + b) * q + r] = part[kk][b];
    }
    __syncthreads();
    if (S == 1) {
        for (int o = threadIdx.x; o < nb * q; o += kMvThreads) {
            const int b = o / q, r = o % q;
            C sum = czero<C>();
            for (int w = 0; w < kMvWarps; ++w) sum = sum + red[((size_t)w * NB + b) * q + r];
            C* xj = x + (size_t)b * SB + ((size_t)j * s) * q;
            xj[r] = MODE == 1 ? xj[r] + sum : sum;
        }
        return;
    }
    C* mine = partial + ((size_t)idx * S + sp) * NB * q;
    for (int o = threadIdx.x; o < nb * q; o += kMvThreads) {
        const int b = o / q, r = o % q;
        C sum = czero<C>();
        for (int w = 0; w < kMvWarps; ++w) sum = sum + red[((size_t)w * NB + b) * q + r];
        mine[(size_t)b * q + r] = sum;
    }
    __threadfence();   // the partial is visible before the counter says so
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&counter[idx], 1u) == (unsigned)(S - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int o = threadIdx.x; o < nb * q; o += kMvThreads) {
        const int b = o / q, r = o % q;
        C tot = czero<C>();
        for (int p = 0; p < S; ++p) tot = tot + __ldcg(&partial[(((size_t)idx * S + p) * NB + b) * q + r]);
        C* xj = x + (size_t)b * SB + ((size_t)j * s) * q;
        xj[r] = MODE == 1 ? xj[r] + tot : tot;
    }
    if (threadIdx.x == 0) counter[idx] = 0u;
}

// level 0 backward, odd blocks: x_j = y_j - D^{-1} (W_j x_{j-1} + E_j x_{j+1})
template <typename T, int RPT, int NB>
__global__ void __launch_bounds__(kMvThreads, NB >= 4 ? 2 : 1) k_cr_l0_back(int q, int nblk, const cpx_t<T>* __restrict__ cw,
                                                          const cpx_t<T>* __restrict__ ce, Pool<T> pool,
                                                          size_t off_dinv, cpx_t<T>* __restrict__ x, size_t SB,
                                                          int nb) {
    using C = cpx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* vt = reinterpret_cast<C*>(smem_raw);   // [NB][q]
    C* red = vt + (size_t)NB * q;             // [kMvWarps][NB][q]
    const int o = blockIdx.x;
    const int j = 2 * o + 1;
    const C* wj = cw + (size_t)j * 3 * q;
    const C* ej = ce + (size_t)j * 3 * q;
    for (int e = threadIdx.x; e < NB * q; e += kMvThreads) {
        const int b = e / q, r = e % q;
        C acc = czero<C>();
        if (b < nb) {
            const C* xb = x + (size_t)b * SB;
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz) {
                const int rr = r + dz;
                if (rr < 0 || rr >= q) continue;
                acc = cfma(wj[(dz + 1) * q + r], xb[(size_t)(j - 1) * q + rr], acc);
                if (j + 1 < nblk) acc = cfma(ej[(dz + 1) * q + r], xb[(size_t)(j + 1) * q + rr], acc);
            }
        }
        vt[e] = -acc;
    }
    __syncthreads();
    const C* M = pool.mat(off_dinv + o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C part[RPT][NB];
#pragma unroll
    for (int kk = 0; kk < RPT; ++kk)
#pragma unroll
        for (int b = 0; b < NB; ++b) part[kk][b] = czero<C>();
#pragma unroll 4
    for (int c = warp; c < q; c += kMvWarps) {
        C a[RPT];
#pragma unroll
        for (int kk = 0; kk < RPT; ++kk) {
            const int r = lane + 32 * kk;
            a[kk] = r < q ? __ldg(&M[(size_t)c * q + r]) : czero<C>();
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const C vc = vt[(size_t)b * q + c];
#pragma unroll
            for (int kk = 0; kk < RPT; ++kk) part[kk][b] = cfma(a[kk], vc, part[kk][b]);
        }
    }
#pragma unroll
    for (int kk = 0; kk < RPT; ++kk) {
        const int r = lane + 32 * kk;
        if (r < q)
#pragma unroll
            for (int b = 0; b < NB; ++b) red[((size_t)warp * NB + b) * q + r] = part[kk][b];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * q; e += kMvThreads) {
        const int b = e / q, r = e % q;
        C sum = czero<C>();
        for (int w = 0; w < kMvWarps; ++w) sum = sum + red[((size_t)w * NB + b) * q + r];
        C* xj = x + (size_t)b * SB + (size_t)j * q;
        xj[r] = xj[r] + sum;
    }
}

// level 0, even blocks: b_j -= W_j y_{j-1} + E_j y_{j+1} (tabulated tridiagonal couplings)
template <typename T>
__global__ void k_l0_even(int q, int nblk, const cpx_t<T>* __restrict__ cw, const cpx_t<T>* __restrict__ ce,
                          cpx_t<T>* __restrict__ x, size_t SB) {
    using C = cpx_t<T>;
    const int j = 2 * blockIdx.x;
    const int r = threadIdx.x;
    if (r >= q) return;
    C* xb = x + (size_t)blockIdx.y * SB;
    C acc = xb[(size_t)j * q + r];
    const C* wj = cw + (size_t)j * 3 * q;
    const C* ej = ce + (size_t)j * 3 * q;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int rr = r + dz;
        if (rr < 0 || rr >= q) continue;
        if (j >= 1) acc = cfms(wj[(dz + 1) * q + r], xb[(size_t)(j - 1) * q + rr], acc);
        if (j + 1 < nblk) acc = cfms(ej[(dz + 1) * q + r], xb[(size_t)(j + 1) * q + rr], acc);
    }
    xb[(size_t)j * q + r] = acc;
}

// g^l = chi_{Omega^l} g (+ injection from the layer above), copied to the solution buffer.
// Batch member b = blockIdx.z: strips at + b * SB, traces at + b * TB, grid vector at + b * N.
// A tiled transpose: a CTA of 32 x 8 threads takes 32 strip rows r x 32 columns i; it
// reads the rows of g that fall in Omega^l along x (coalesced) into shared memory and
// writes the strip's block layout (column i = q contiguous values) along r (coalesced).
// The injected rows (eq. pde_GRF_down) are computed in the strip's precision.
// TR: g is the field of the other direction (the vertical layers' grid is the transpose
// of the field's): strip row r, column i is g[i][l t - E + r], contiguous along r, so the
// reads go straight to the strip layout without the shared-memory tile.
constexpr int kGatherTile = 32;
template <typename T, bool TR, typename GF = double2>
__global__ void __launch_bounds__(256) k_gather(StripGeom g, const cpx_t<T>* __restrict__ inj, int l,
                                                const GF* __restrict__ gf, cpx_t<T>* __restrict__ rhs,
                                                cpx_t<T>* __restrict__ sol, const cpx_t<T>* __restrict__ above,
                                                cpx_t<T>* __restrict__ trace_above, size_t SB, size_t TB) {
    using C = cpx_t<T>;
    __shared__ C tile[kGatherTile][kGatherTile + 1];   // [r - r0][i - i0]
    const int q = g.q, n = g.n, E = g.E, t = g.t;
    const size_t b = blockIdx.z;
    const int i0 = blockIdx.x * kGatherTile, r0 = blockIdx.y * kGatherTile;
    gf += b * (size_t)n * n;
    rhs += b * SB;
    sol += b * SB;
    if (above) {
        above += b * SB;
        trace_above += b * TB;
    }
    const int tx = threadIdx.x, ty = threadIdx.y;
    const GF z0 = {};
    GF v[kGatherTile / 8];
    if constexpr (TR) {
#pragma unroll
        for (int u = 0; u < kGatherTile / 8; ++u) {   // rows of Omega^l (E <= r < E + t), along r
            const int i = i0 + ty + 8 * u, r = r0 + tx;
            v[u] = (r >= E && r < E + t && i < n) ? __ldg(&gf[(size_t)i * n + (l * t - E + r)]) : z0;
        }
    } else {
#pragma unroll
        for (int u = 0; u < kGatherTile / 8; ++u) {   // rows of Omega^l (E <= r < E + t), along x
            const int r = r0 + ty + 8 * u, i = i0 + tx;
            v[u] = (r >= E && r < E + t && i < n) ? __ldg(&gf[(size_t)(l * t - E + r) * n + i]) : z0;
        }
#pragma unroll
        for (int u = 0; u < kGatherTile / 8; ++u) tile[ty + 8 * u][tx] = ccast<C>(v[u]);
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kGatherTile / 8; ++u) {   // strip columns, along r
        const int i = i0 + ty + 8 * u, r = r0 + tx;
        if (i >= n || r >= q) continue;
        const size_t e = (size_t)i * q + r;
        C cv = TR ? ccast<C>(v[u]) : tile[tx][ty + 8 * u];
        if (above) {
            if (r == 0) trace_above[i] = above[(size_t)i * q + E - 1];  // w^{l+1}_0, kept for the upward sweep
            const C* c0 = inj + (size_t)l * 12 * n;  // slots 0, 1 of layer l: [slot][dx+1][i]
            if (r == E + t - 1) {  // -C^l_{n,n+1} w^{l+1}_1 ; w^{l+1}_1 = row E of layer l+1
                for (int dx = -1; dx <= 1; ++dx)
                    if (i + dx >= 0 && i + dx < n)
                        cv = cfms(c0[(size_t)(0 * 3 + dx + 1) * n + i], above[(size_t)(i + dx) * q + E], cv);
            } else if (r == E + t) {  // +C^l_{n+1,n} w^{l+1}_0 ; w^{l+1}_0 = row E-1 of layer l+1
                for (int dx = -1; dx <= 1; ++dx)
                    if (i + dx >= 0 && i + dx < n)
                        cv = cfma(c0[(size_t)(1 * 3 + dx + 1) * n + i], above[(size_t)(i + dx) * q + E - 1], cv);
            }
        }
        rhs[e] = cv;
        sol[e] = cv;
    }
}

// Upward sweep: sol = g^l (a device copy of rhs made just before) plus the injection
// from the layer below, which touches only the two rows E - 1 and E; one thread per
// (column i, row) of those, batch member b = blockIdx.y.
template <typename T>
__global__ void k_inject_up(StripGeom g, const cpx_t<T>* __restrict__ inj, int l, const cpx_t<T>* __restrict__ rhs,
                            cpx_t<T>* __restrict__ sol, const cpx_t<T>* __restrict__ below,
                            const cpx_t<T>* __restrict__ trace_self, size_t SB, size_t TB) {
    using C = cpx_t<T>;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = g.q, n = g.n, E = g.E, t = g.t;
    if (o >= 2 * n) return;
    const size_t b = blockIdx.y;
    rhs += b * SB;
    sol += b * SB;
    below += b * SB;
    trace_self += b * TB;
    const int i = o >> 1, r = (o & 1) ? E : E - 1;
    const size_t e = (size_t)i * q + r;
    C val = rhs[e];   // the injection in the strip's precision
    const C* c0 = inj + (size_t)l * 12 * n;  // slots 2, 3 of layer l: [slot][dx+1][i]
    if (r == E) {  // -C^l_{1,0} (v^{l-1}_n - w^l_0) ; v^{l-1}_n = row E+t-1 of layer l-1
        for (int dx = -1; dx <= 1; ++dx) {
            if (i + dx < 0 || i + dx >= n) continue;
            const C p0 = below[(size_t)(i + dx) * q + E + t - 1] - trace_self[i + dx];
            val = cfms(c0[(size_t)(2 * 3 + dx + 1) * n + i], p0, val);
        }
    } else {  // +C^l_{0,1} v^{l-1}_{n+1} ; v^{l-1}_{n+1} = row E+t of layer l-1
        for (int dx = -1; dx <= 1; ++dx) {
            if (i + dx < 0 || i + dx >= n) continue;
            val = cfma(c0[(size_t)(3 * 3 + dx + 1) * n + i], below[(size_t)(i + dx) * q + E + t], val);
        }
    }
    sol[e] = val;
}

// v = rows 1..n of every layer's solution (concatenation); batch member b = blockIdx.y
template <typename T, typename OF = double2>
__global__ void k_scatter(StripGeom g, const cpx_t<T>* __restrict__ sol, size_t strip_stride, size_t SB,
                          OF* __restrict__ v) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n;
    if (e >= (size_t)n * n) return;
    const size_t b = blockIdx.y;
    const int z = (int)(e / n), i = (int)(e % n);
    const int l = z / g.t, r = z - l * g.t + g.E;
    v[b * (size_t)n * n + e] = ccast<OF>(sol[b * SB + (size_t)l * strip_stride + (size_t)i * g.q + r]);
}

// The same for the other direction's field, added to a field of this one:
// v[i][z] = u[i][z] + (row z of the layers' solutions)[i]  (the vertical sweep's result
// transposed back and added to the horizontal one, Algorithm 2); along z, coalesced.
template <typename T, typename AF = double2, typename OF = double2>
__global__ void k_scatter_tadd(StripGeom g, const cpx_t<T>* __restrict__ sol, size_t strip_stride, size_t SB,
                               const AF* __restrict__ u, OF* __restrict__ v) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n;
    if (e >= (size_t)n * n) return;
    const size_t b = blockIdx.y;
    const int i = (int)(e / n), z = (int)(e % n);
    const int l = z / g.t, r = z - l * g.t + g.E;
    const size_t o = b * (size_t)n * n + e;
    v[o] = ccast<OF>(ccast<double2>(u[o]) + ccast<double2>(sol[b * SB + (size_t)l * strip_stride + (size_t)i * g.q + r]));
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


StripGeom geom_of(const ls_handle* h) { return StripGeom{h->n, h->t, h->E, h->q, h->opts.shift / h->omega}; }

// CTAs per block of a reduction step: levels with fewer blocks than about two per SM
// split each block's columns over up to kCrSplitMax CTAs (at most kCrSplitCtas CTAs in all).
// The handle's cr_split switches it off (1 CTA per block everywhere).
constexpr int kCrSplitCtas = 304, kCrSplitMax = 8;
int cr_split_of(const ls_handle* h, int nblk) {
    if (!h->cr_split) return 1;
    int S = kCrSplitCtas / (nblk > 0 ? nblk : 1);
    return S < 1 ? 1 : (S > kCrSplitMax ? kCrSplitMax : S);
}

template <typename T, int RPT, int NB>
int cr_solve_rpt(ls_handle* h, int dir, int l, cpx_t<T>* x, size_t SB, int nb) {
    using C = cpx_t<T>;
    const DirFactors& F = h->fac[dir];
    const int q = h->q, n = h->n;
    const size_t qq = (size_t)q * q;
    const C* base;
    if constexpr (sizeof(T) == 4) base = F.pool32;
    else base = F.pool64;
    Pool<T> pool{base + (size_t)l * F.mats_per_strip * qq, qq};
    const int thr = (q + 31) / 32 * 32;
    const size_t sm_step = (size_t)(3 + kMvWarps) * NB * sizeof(C) * q;
    const size_t sm_back = (size_t)(1 + kMvWarps) * NB * sizeof(C) * q;
    const CrLevel& l0 = F.lev[0];
    const C* cw = static_cast<const C*>(F.cw) + (size_t)l * n * 3 * q;
    const C* ce = static_cast<const C*>(F.ce) + (size_t)l * n * 3 * q;
    const ls_handle::SweepLane& W = h->lanes[h->lane];
    C* part = static_cast<C*>(W.cr_part);
    unsigned* cnt = W.cr_cnt;
    if (l0.nodd) {
        const int S = cr_split_of(h, l0.nodd);
        LS_LAUNCH(h, (k_cr_step<T, RPT, 0, NB>), l0.nodd * S, kMvThreads, sm_step, q, 0, l0.nk, pool, l0.off_dinv,
                  (size_t)0, (size_t)0, x, SB, nb, S, part, cnt);
    }
    LS_LAUNCH(h, k_l0_even<T>, dim3(l0.neven, nb), thr, 0, q, n, cw, ce, x, SB);
    for (int k = 1; k < F.K; ++k) {
        const CrLevel& lv = F.lev[k];
        const int S = cr_split_of(h, lv.neven);
        LS_LAUNCH(h, (k_cr_step<T, RPT, 1, NB>), lv.neven * S, kMvThreads, sm_step, q, k, lv.nk, pool, (size_t)0,
                  lv.off_f, lv.off_g, x, SB, nb, S, part, cnt);
    }
    {
        const int S = cr_split_of(h, 1);
        LS_LAUNCH(h, (k_cr_step<T, RPT, 3, NB>), S, kMvThreads, sm_step, q, 0, 1, pool, F.off_top, (size_t)0,
                  (size_t)0, x, SB, nb, S, part, cnt);
    }
    for (int k = F.K - 1; k >= 1; --k) {
        const CrLevel& lv = F.lev[k];
        if (!lv.nodd) continue;
        const int S = cr_split_of(h, lv.nodd);
        LS_LAUNCH(h, (k_cr_step<T, RPT, 2, NB>), lv.nodd * S, kMvThreads, sm_step, q, k, lv.nk, pool, lv.off_dinv,
                  lv.off_p, lv.off_q, x, SB, nb, S, part, cnt);
    }
    if (l0.nodd)
        LS_LAUNCH(h, (k_cr_l0_back<T, RPT, NB>), l0.nodd, kMvThreads, sm_back, q, n, cw, ce, pool, l0.off_dinv, x,
                  SB, nb);
    return LS_OK;
}

template <typename T, int NB>
int cr_solve_nb(ls_handle* h, int dir, int l, cpx_t<T>* x, size_t SB, int nb) {
    switch ((h->q + 31) / 32) {
        case 1: return cr_solve_rpt<T, 1, NB>(h, dir, l, x, SB, nb);
        case 2: return cr_solve_rpt<T, 2, NB>(h, dir, l, x, SB, nb);
        case 3: return cr_solve_rpt<T, 3, NB>(h, dir, l, x, SB, nb);
        default: return cr_solve_rpt<T, 4, NB>(h, dir, l, x, SB, nb);
    }
}

// The same local solve with the reduction steps on the tensor cores (ls_cr_mma.cu):
// every step a TF32 GEMM over the whole batch (up to 32 right-hand sides), the
// level-0 even update on the CUDA cores as above.
int cr_solve_tc(ls_handle* h, int dir, int l, float2* x, size_t SB, int nb) {
    const DirFactors& F = h->fac[dir];
    const int q = h->q, n = h->n;
    const CrLevel& l0 = F.lev[0];
    const float2* cw = static_cast<const float2*>(F.cw) + (size_t)l * n * 3 * q;
    const float2* ce = static_cast<const float2*>(F.ce) + (size_t)l * n * 3 * q;
    const int thr = (q + 31) / 32 * 32;
    // levels >= dense_c as one product with the reduced system's inverse, where it is built
    const bool dense = h->tc_dense && F.dense_nc && h->lanes[h->lane].dense_part;
    const int ktop = dense ? F.dense_c : F.K;
    if (l0.nodd) LS_TRY(ls_cr_tc_step(h, dir, l, 0, 0, l0.nk, (unsigned)l0.nodd, l0.off_dinv, 0, 0, x, SB, nb, cw, ce));
    LS_LAUNCH(h, k_l0_even<float>, dim3(l0.neven, nb), thr, 0, q, n, cw, ce, x, SB);
    for (int k = 1; k < ktop; ++k) {
        const CrLevel& lv = F.lev[k];
        LS_TRY(ls_cr_tc_step(h, dir, l, 1, k, lv.nk, (unsigned)lv.neven, 0, lv.off_f, lv.off_g, x, SB, nb, cw, ce));
    }
    if (dense) LS_TRY(ls_cr_dense_apply(h, dir, l, x, SB, nb));
    else LS_TRY(ls_cr_tc_step(h, dir, l, 3, 0, 1, 1u, F.off_top, 0, 0, x, SB, nb, cw, ce));
    for (int k = ktop - 1; k >= 1; --k) {
        const CrLevel& lv = F.lev[k];
        if (!lv.nodd) continue;
        LS_TRY(ls_cr_tc_step(h, dir, l, 2, k, lv.nk, (unsigned)lv.nodd, lv.off_dinv, lv.off_p, lv.off_q, x, SB, nb, cw,
                             ce));
    }
    if (l0.nodd) LS_TRY(ls_cr_tc_step(h, dir, l, 4, 0, l0.nk, (unsigned)l0.nodd, l0.off_dinv, 0, 0, x, SB, nb, cw, ce));
    return LS_OK;
}

// The batch template is the smallest supported NB >= nb (FP64 keeps NB <= 4 for registers).
template <typename T>
int cr_solve(ls_handle* h, int dir, int l, cpx_t<T>* x, size_t SB, int nb) {
    if constexpr (sizeof(T) == 4) {
        // tensor cores: always (cr_tc 2), or for batches past the CUDA-core steps' sweet spot
        // (cr_tc 1: at least 5 right-hand sides; a one-matrix product per step does not fill them)
        if (h->tc_ready && (h->cr_tc == 2 || (h->cr_tc == 1 && nb >= 5))) return cr_solve_tc(h, dir, l, x, SB, nb);
    }
    if (nb <= 1) return cr_solve_nb<T, 1>(h, dir, l, x, SB, nb);
    if (nb <= 2) return cr_solve_nb<T, 2>(h, dir, l, x, SB, nb);
    if (nb <= 4) return cr_solve_nb<T, 4>(h, dir, l, x, SB, nb);
    if constexpr (sizeof(T) == 4) return cr_solve_nb<T, 8>(h, dir, l, x, SB, nb);
    return LS_EINVAL;
}

// tr: g and v are fields of the other direction's grid (read and written transposed);
// add: v = add + the result (tr only).  GF, OF, AF: element types of g, v and add
// (double2; float2 for the mixed Algorithm 2's intermediate fields, which hold FP32
// values either way).
template <typename T, typename GF = double2, typename OF = double2, typename AF = double2>
int sweep_impl(ls_handle* h, int dir, const GF* g, OF* v, int nb, bool tr = false, const AF* add = nullptr) {
    using C = cpx_t<T>;
    const int n = h->n, q = h->q, L = h->L;
    const size_t sstride = (size_t)n * q;
    const size_t SB = (size_t)L * sstride, TB = (size_t)L * n;
    const ls_handle::SweepLane& W = h->lanes[h->lane];
    C* rhs = static_cast<C*>(W.srhs);
    C* sol = static_cast<C*>(W.ssol);
    C* trc = static_cast<C*>(W.strace);
    const DirFactors& F = h->fac[dir];
    const StripGeom geo = geom_of(h);
    const dim3 gg((unsigned)((n + kGatherTile - 1) / kGatherTile), (unsigned)((q + kGatherTile - 1) / kGatherTile), nb);
    const dim3 gb(kGatherTile, 8);
    for (int l = L - 1; l >= 0; --l) {  // downward sweep
        if (tr)
            LS_LAUNCH(h, (k_gather<T, true, GF>), gg, gb, 0, geo, static_cast<const C*>(F.cinj), l, g, rhs + l * sstride,
                      sol + l * sstride, l < L - 1 ? sol + (l + 1) * sstride : (const C*)nullptr,
                      l < L - 1 ? trc + (size_t)(l + 1) * n : (C*)nullptr, SB, TB);
        else
            LS_LAUNCH(h, (k_gather<T, false, GF>), gg, gb, 0, geo, static_cast<const C*>(F.cinj), l, g, rhs + l * sstride,
                      sol + l * sstride, l < L - 1 ? sol + (l + 1) * sstride : (const C*)nullptr,
                      l < L - 1 ? trc + (size_t)(l + 1) * n : (C*)nullptr, SB, TB);
        LS_TRY(cr_solve<T>(h, dir, l, sol + l * sstride, SB, nb));
    }
    const dim3 gi((unsigned)((2 * n + 255) / 256), nb);
    for (int l = 1; l < L; ++l) {  // upward sweep: sol = rhs, then the two injected rows
        LS_CUDA(cudaMemcpy2DAsync(sol + l * sstride, sizeof(C) * SB, rhs + l * sstride, sizeof(C) * SB,
                                  sizeof(C) * sstride, nb, cudaMemcpyDeviceToDevice, h->stream));
        LS_LAUNCH(h, k_inject_up<T>, gi, 256, 0, geo, static_cast<const C*>(F.cinj), l, rhs + l * sstride,
                  sol + l * sstride, sol + (l - 1) * sstride, trc + (size_t)l * n, SB, TB);
        LS_TRY(cr_solve<T>(h, dir, l, sol + l * sstride, SB, nb));
    }
    const size_t N = (size_t)n * n;
    if (tr && add) {
        LS_LAUNCH(h, (k_scatter_tadd<T, AF, OF>), dim3((unsigned)((N + 255) / 256), nb), 256, 0, geo, sol, sstride, SB,
                  add, v);
        return LS_OK;
    }
    LS_LAUNCH(h, (k_scatter<T, OF>), dim3((unsigned)((N + 255) / 256), nb), 256, 0, geo, sol, sstride, SB, v);
    return LS_OK;
}

template <typename T>
int smem_optin(int q) {
    using C = cpx_t<T>;
    const int rpt = (q + 31) / 32;
    const size_t s8 = (size_t)(3 + kMvWarps) * 8 * sizeof(C) * q, s4 = (size_t)(3 + kMvWarps) * 4 * sizeof(C) * q;
    const size_t big = sizeof(T) == 4 ? s8 : s4;
    if (big <= 48 * 1024) return LS_OK;
#define LS_OPTIN(R, NB)                                                                                           \
    do {                                                                                                          \
        const size_t sz = (size_t)(3 + kMvWarps) * NB * sizeof(C) * q;                                            \
        LS_CUDA(cudaFuncSetAttribute(k_cr_step<T, R, 0, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz)); \
        LS_CUDA(cudaFuncSetAttribute(k_cr_step<T, R, 1, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz)); \
        LS_CUDA(cudaFuncSetAttribute(k_cr_step<T, R, 2, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz)); \
        LS_CUDA(cudaFuncSetAttribute(k_cr_step<T, R, 3, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz)); \
        LS_CUDA(cudaFuncSetAttribute(k_cr_l0_back<T, R, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sz)); \
    } while (0)
#define LS_OPTIN_R(NB)                  \
    switch (rpt) {                      \
        case 1: LS_OPTIN(1, NB); break; \
        case 2: LS_OPTIN(2, NB); break; \
        case 3: LS_OPTIN(3, NB); break; \
        default: LS_OPTIN(4, NB); break; \
    }
    LS_OPTIN_R(2);
    LS_OPTIN_R(4);
    if constexpr (sizeof(T) == 4) LS_OPTIN_R(8);
#undef LS_OPTIN_R
#undef LS_OPTIN
    return LS_OK;
}

}  // namespace

// Workspace of the current lane for batches of up to nb right-hand sides (grown on
// demand; the lane's graphs, made for smaller buffers, are dropped).
static void lane_graphs_free(ls_handle::SweepLane& W) {
    for (int b = 0; b <= kMaxBatch; ++b) {
        if (W.exec[b]) cudaGraphExecDestroy(W.exec[b]);
        if (W.graph[b]) cudaGraphDestroy(W.graph[b]);
        W.exec[b] = nullptr;
        W.graph[b] = nullptr;
        W.nodes[b] = 0;
    }
}

int ls_sweep_reserve(ls_handle* h, int nb) {
    ls_handle::SweepLane& W = h->lanes[h->lane];
    if (nb <= W.nb_cap) return LS_OK;
    lane_graphs_free(W);
    const size_t cnt = (size_t)h->L * h->n * h->q * nb;
    const size_t es = h->prec == LS_MIXED ? sizeof(float2) : sizeof(double2);
    const size_t N = (size_t)h->n * h->n;
    void* ptrs[] = {W.srhs, W.ssol, W.strace, W.vtmp, W.bd_in, W.bd_out};
    for (void* p : ptrs) cudaFree(p);
    W.srhs = W.ssol = W.strace = W.vtmp = nullptr;
    W.bd_in = W.bd_out = nullptr;
    W.nb_cap = 0;
    LS_CUDA(cudaMalloc(&W.srhs, es * cnt));
    LS_CUDA(cudaMalloc(&W.ssol, es * cnt));
    LS_CUDA(cudaMalloc(&W.strace, es * (size_t)h->L * h->n * nb));
    LS_CUDA(cudaMalloc(&W.vtmp, sizeof(double2) * N * 4 * nb));
    LS_CUDA(cudaMalloc(&W.bd_in, sizeof(double2) * N * nb));
    LS_CUDA(cudaMalloc(&W.bd_out, sizeof(double2) * N * nb));
    if (!W.cr_part) {  // split-level partial sums (kCrSplitCtas CTAs x 8 vectors x q) and counters
        LS_CUDA(cudaMalloc(&W.cr_part, sizeof(double2) * kCrSplitCtas * 8 * h->q));
        LS_CUDA(cudaMalloc(&W.cr_cnt, sizeof(unsigned) * kCrSplitCtas));
        LS_CUDA(cudaMemset(W.cr_cnt, 0, sizeof(unsigned) * kCrSplitCtas));
    }
    W.nb_cap = nb;
    return LS_OK;
}

void ls_lanes_free(ls_handle* h) {
    for (auto& W : h->lanes) {
        lane_graphs_free(W);
        void* ptrs[] = {W.srhs, W.ssol, W.strace, W.vtmp, W.bd_in, W.bd_out, W.cr_part, W.cr_cnt, W.dense_part};
        for (void* p : ptrs) cudaFree(p);
        if (W.stream) cudaStreamDestroy(W.stream);
        if (W.done) cudaEventDestroy(W.done);
        W = ls_handle::SweepLane{};
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    h->ev_fork = nullptr;
}

int ls_sweep_alloc(ls_handle* h) {
    if (h->prec == LS_MIXED) LS_TRY(smem_optin<float>(h->q));
    else LS_TRY(smem_optin<double>(h->q));
    for (int k = 1; k < ls_handle::kLanes; ++k) {
        LS_CUDA(cudaStreamCreateWithFlags(&h->lanes[k].stream, cudaStreamNonBlocking));
        LS_CUDA(cudaEventCreateWithFlags(&h->lanes[k].done, cudaEventDisableTiming));
    }
    LS_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    h->lane = 0;
    return ls_sweep_reserve(h, 1);
}

// Algorithm 1 on direction dir (0: horizontal layers; 1: vertical layers) for nb
// right-hand sides g (nb x N, contiguous) into v.
int ls_sweep_dir_b(ls_handle* h, int dir, const double2* g, double2* v, int nb) {
    if (nb < 1 || nb > ls_bd_cap(h)) return LS_EINVAL;
    LS_TRY(ls_sweep_reserve(h, nb));  // no-op when called inside a capture (reserved beforehand)
    const size_t N = (size_t)h->n * h->n;
    double2* t0 = static_cast<double2*>(h->lanes[h->lane].vtmp);
    double2* t1 = t0 + N * nb;
    if (dir == 0) {
        if (h->prec == LS_MIXED) return sweep_impl<float>(h, 0, g, v, nb);
        return sweep_impl<double>(h, 0, g, v, nb);
    }
    LS_TRY(ls_transpose64_b(h, g, t0, nb));
    if (h->prec == LS_MIXED) LS_TRY(sweep_impl<float>(h, 1, t0, t1, nb));
    else LS_TRY(sweep_impl<double>(h, 1, t0, t1, nb));
    return ls_transpose64_b(h, t1, v, nb);
}

int ls_sweep_dir(ls_handle* h, int dir, const double2* g, double2* v) { return ls_sweep_dir_b(h, dir, g, v, 1); }

// Algorithm 2 for nb right-hand sides: v = u1 + u2, u1 = Alg. 1 horizontal (g),
// u2 = Alg. 1 vertical (g - C u1).
// Mixed precision: the fields g, v and the intermediate u1, e are FP32 (the values the FP32
// sweeps read and produce), half the traffic of FP64 fields.
static int bd_direct_mixed(ls_handle* h, const float2* g, float2* v, int nb) {
    const size_t N = (size_t)h->n * h->n;
    float2* u1f = reinterpret_cast<float2*>(static_cast<double2*>(h->lanes[h->lane].vtmp) + 2 * N * nb);
    float2* ef = u1f + N * nb;
    LS_TRY((sweep_impl<float, float2, float2, float2>(h, 0, g, u1f, nb)));
    LS_TRY(ls_stencil_refine_f32(h, 0, u1f, g, ef, nb));   // e = g - C u1
    // vertical layers on e as it is stored (their grid is its transpose): the gather reads
    // it transposed, and the scatter writes v = u1 + the result, transposed back
    return sweep_impl<float, float2, float2, float2>(h, 1, ef, v, nb, true, u1f);
}

static int bd_direct(ls_handle* h, const double2* g, double2* v, int nb) {
    const size_t N = (size_t)h->n * h->n;
    double2* u1 = static_cast<double2*>(h->lanes[h->lane].vtmp) + 2 * N * nb;
    double2* e = u1 + N * nb;
    LS_TRY(ls_sweep_dir_b(h, 0, g, u1, nb));
    LS_TRY(ls_stencil_apply_b(h, 0, 2, u1, g, e, nb));   // e = g - C u1
    // vertical layers on e as it is stored (their grid is its transpose): the gather reads
    // it transposed, and the scatter writes v = u1 + the result, transposed back
    return sweep_impl<double>(h, 1, e, v, nb, true, u1);
}

void ls_bd_graph_free(ls_handle* h) {
    for (auto& W : h->lanes) lane_graphs_free(W);
}

// Capture Algorithm 2 for nb right-hand sides on the staging buffers once (the
// sequence of launches and all pointers are fixed after ls_factor), then replay it.
static int bd_capture(ls_handle* h, int nb) {
    cudaStream_t cap = nullptr;
    LS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaStream_t saved = h->stream;
    const long long l0 = h->launches;
    h->stream = cap;
    int rc = LS_OK;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (h->prec == LS_MIXED)
            rc = bd_direct_mixed(h, reinterpret_cast<const float2*>(h->lanes[h->lane].bd_in),
                                 reinterpret_cast<float2*>(h->lanes[h->lane].bd_out), nb);
        else
            rc = bd_direct(h, h->lanes[h->lane].bd_in, h->lanes[h->lane].bd_out, nb);
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
    ls_handle::SweepLane& W = h->lanes[h->lane];
    W.graph[nb] = graph;
    W.exec[nb] = exec;
    W.nodes[nb] = nodes;
    return LS_OK;
}

// Algorithm 2 on FP32 fields (mixed precision): the captured graph reads and writes the
// lane's staging buffers as FP32.
int ls_bd_b(ls_handle* h, const float2* g, float2* v, int nb) {
    if (h->prec != LS_MIXED) return LS_ESTATE;
    if (nb < 1 || nb > ls_bd_cap(h)) return LS_EINVAL;
    LS_TRY(ls_sweep_reserve(h, nb));
    if (!h->opts.use_graphs) return bd_direct_mixed(h, g, v, nb);
    ls_handle::SweepLane& W = h->lanes[h->lane];
    if (!W.exec[nb]) LS_TRY(bd_capture(h, nb));
    const size_t N = (size_t)h->n * h->n;
    LS_CUDA(cudaMemcpyAsync(W.bd_in, g, sizeof(float2) * N * nb, cudaMemcpyDeviceToDevice, h->stream));
    LS_CUDA(cudaGraphLaunch(W.exec[nb], h->stream));
    h->launches += W.nodes[nb];
    LS_CUDA(cudaMemcpyAsync(v, W.bd_out, sizeof(float2) * N * nb, cudaMemcpyDeviceToDevice, h->stream));
    return LS_OK;
}

int ls_bd_b(ls_handle* h, const double2* g, double2* v, int nb) {
    if (nb < 1 || nb > ls_bd_cap(h)) return LS_EINVAL;
    LS_TRY(ls_sweep_reserve(h, nb));
    ls_handle::SweepLane& W = h->lanes[h->lane];
    const size_t N = (size_t)h->n * h->n;
    if (h->prec == LS_MIXED) {   // through FP32 copies in the lane's staging buffers
        float2* in = reinterpret_cast<float2*>(W.bd_in);
        float2* out = reinterpret_cast<float2*>(W.bd_out);
        for (int b = 0; b < nb; ++b) LS_TRY(ls_vec_copy(h, g + b * N, in + b * N));
        if (!h->opts.use_graphs) {
            LS_TRY(bd_direct_mixed(h, in, out, nb));
        } else {
            if (!W.exec[nb]) LS_TRY(bd_capture(h, nb));
            LS_CUDA(cudaGraphLaunch(W.exec[nb], h->stream));
            h->launches += W.nodes[nb];
        }
        for (int b = 0; b < nb; ++b) LS_TRY(ls_vec_copy(h, out + b * N, v + b * N));
        return LS_OK;
    }
    if (!h->opts.use_graphs) return bd_direct(h, g, v, nb);
    if (!W.exec[nb]) LS_TRY(bd_capture(h, nb));
    LS_CUDA(cudaMemcpyAsync(W.bd_in, g, sizeof(double2) * N * nb, cudaMemcpyDeviceToDevice, h->stream));
    LS_CUDA(cudaGraphLaunch(W.exec[nb], h->stream));
    h->launches += W.nodes[nb];
    LS_CUDA(cudaMemcpyAsync(v, W.bd_out, sizeof(double2) * N * nb, cudaMemcpyDeviceToDevice, h->stream));
    return LS_OK;
}

template <typename FT>
static int bd_lanes(ls_handle* h, const FT* g, FT* v, int nb, int chunk, const unsigned char* on) {
    if (chunk < 1) return LS_EINVAL;
    const size_t N = (size_t)h->n * h->n;
    const int nchunks = (nb + chunk - 1) / chunk;
    std::vector<int> run;
    for (int c = 0; c < nchunks; ++c) {
        bool any = !on;
        for (int b = c * chunk; b < nb && b < (c + 1) * chunk && !any; ++b) any = on[b] != 0;
        if (any) run.push_back(c);
    }
    if (run.empty()) return LS_OK;
    if (run.size() == 1) {
        const int b0 = run[0] * chunk, cnt = nb - b0 < chunk ? nb - b0 : chunk;
        return ls_bd_b(h, g + b0 * N, v + b0 * N, cnt);
    }
    cudaStream_t main = h->stream;
    LS_CUDA(cudaEventRecord(h->ev_fork, main));
    bool used[ls_handle::kLanes] = {};
    int rc = LS_OK;
    for (size_t ci = 0; ci < run.size() && rc == LS_OK; ++ci) {
        const int c = run[ci];
        const int k = (int)(ci % ls_handle::kLanes);
        const int b0 = c * chunk, cnt = nb - b0 < chunk ? nb - b0 : chunk;
        ls_handle::SweepLane& W = h->lanes[k];
        if (k > 0 && !used[k]) {
            const cudaError_t e = cudaStreamWaitEvent(W.stream, h->ev_fork, 0);
            if (e != cudaSuccess) {
                rc = ls_cuda_fail(e);
                break;
            }
        }
        used[k] = true;
        h->stream = k > 0 ? W.stream : main;
        h->lane = k;
        rc = ls_bd_b(h, g + b0 * N, v + b0 * N, cnt);
        h->stream = main;
        h->lane = 0;
    }
    for (int k = 1; k < ls_handle::kLanes; ++k) {  // join, also after a failure
        if (!used[k]) continue;
        cudaEventRecord(h->lanes[k].done, h->lanes[k].stream);
        cudaStreamWaitEvent(main, h->lanes[k].done, 0);
    }
    return rc;
}

int ls_bd_lanes(ls_handle* h, const double2* g, double2* v, int nb, int chunk, const unsigned char* on) {
    return bd_lanes(h, g, v, nb, chunk, on);
}
int ls_bd_lanes(ls_handle* h, const float2* g, float2* v, int nb, int chunk, const unsigned char* on) {
    return bd_lanes(h, g, v, nb, chunk, on);
}

int ls_bd(ls_handle* h, const double2* g, double2* v) { return ls_bd_b(h, g, v, 1); }

int ls_bd_cap(const ls_handle* h) {
    if (h->prec != LS_MIXED) return 4;
    return h->tc_ready && h->cr_tc ? ls_cr_tc_max_nb(h) : 8;
}

int ls_strip_solve(ls_handle* h, int dir, int layer, const double2* b, double2* x) {
    const int n = h->n, q = h->q;
    const size_t cnt = (size_t)n * q;
    const unsigned nblk = (unsigned)((cnt + 255) / 256);
    const size_t SB = (size_t)h->L * cnt;
    if (h->prec == LS_MIXED) {
        float2* s = static_cast<float2*>(h->lanes[0].ssol);
        LS_LAUNCH(h, k_strip_in<float>, nblk, 256, 0, n, q, b, s);
        LS_TRY(cr_solve<float>(h, dir, layer, s, SB, 1));
        LS_LAUNCH(h, k_strip_out<float>, nblk, 256, 0, n, q, s, x);
    } else {
        double2* s = static_cast<double2*>(h->lanes[0].ssol);
        LS_LAUNCH(h, k_strip_in<double>, nblk, 256, 0, n, q, b, s);
        LS_TRY(cr_solve<double>(h, dir, layer, s, SB, 1));
        LS_LAUNCH(h, k_strip_out<double>, nblk, 256, 0, n, q, s, x);
    }
    return LS_OK;
}
