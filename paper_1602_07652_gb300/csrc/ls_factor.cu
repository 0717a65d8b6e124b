// ls_factor.cu -- off-line factorisation of the local matrices C^l (Sec. 4.1).
//
// Ordering the unknowns of an extended layer by columns along the layer (the
// long axis) makes C^l block tridiagonal: n blocks of q x q (q = t + 2E), each
// block a column of the strip, coupled to its two neighbours by the 9-point
// stencil (Sec. 3.2 writes C in the same block form along the other axis).
// The paper factors each C^l with a sparse direct solver in O(n) (Sec. 4.1).
// Here every strip is factored by block cyclic reduction (odd-even reduction),
// all strips of a direction in parallel, in FP64:
//   level k eliminates the odd blocks j of the level-k system
//       W_j x_{j-1} + D_j x_j + E_j x_{j+1} = b_j
//   giving the level-(k+1) system on the even blocks with
//       D'_j = D_j - F_j E_{j-1} - G_j W_{j+1},  W'_j = -F_j W_{j-1},  E'_j = -G_j E_{j+1},
//       F_j = W_j D_{j-1}^{-1},  G_j = E_j D_{j+1}^{-1}.
// Stored for the solve: level 0 -- D^{-1} of odd blocks (W, E stay tridiagonal
// and are recomputed from the stencil); levels >= 1 -- D^{-1}, P = D^{-1} W,
// Q = D^{-1} E for odd blocks and F, G for even blocks; the inverse of the last
// block.  A solve then takes 2 log2(n) dependent steps instead of 2n.
// Dense blocks are column-major (element (r, c) at c*q + r) so that a thread per
// row reads a matrix coalesced in the solve's mat-vec.
#include <cmath>
#include <vector>

#include "ls_internal.cuh"
#include "ls_strip.cuh"

namespace {

constexpr int kMaxQ = 112;

// Dense q x q block of level 0: kind 0 = D (dx = 0), 1 = W (dx = -1), 2 = E (dx = +1).
__device__ __forceinline__ double2 level0_entry(const StripGeom& g, const StencilTables* tab, const double* m,
                                                int l, int i, int kind, int r, int c) {
    const int dz = c - r;
    if (dz < -1 || dz > 1) return make_double2(0, 0);
    const int dx = kind == 0 ? 0 : (kind == 1 ? -1 : 1);
    return strip_coef(g, tab, m, l, r, i, dx, dz);
}

// In-place Gauss-Jordan inversion with partial pivoting of a q x q column-major
// matrix held in shared memory (fcol: q scratch entries).  Returns false on a
// zero pivot.  Row interchanges are undone as column interchanges at the end.
__device__ bool gj_invert(double2* M, int q, double2* fcol, int* piv, double* redv, int* redi) {
    const int tid = threadIdx.x, nt = blockDim.x;
    bool ok = true;
    for (int k = 0; k < q; ++k) {
        // pivot search in column k, rows >= k
        double best = -1.0;
        int bi = k;
        for (int r = k + tid; r < q; r += nt) {
            const double a = cabs2(M[k * q + r]);
            if (a > best) { best = a; bi = r; }
        }
        redv[tid] = best;
        redi[tid] = bi;
        __syncthreads();
        for (int s = nt / 2; s > 0; s >>= 1) {
            if (tid < s && redv[tid + s] > redv[tid]) { redv[tid] = redv[tid + s]; redi[tid] = redi[tid + s]; }
            __syncthreads();
        }
        const int p = redi[0];
        const double pbest = redv[0];
        __syncthreads();
        if (tid == 0) piv[k] = p;
        if (!(pbest > 0.0)) ok = false;
        if (p != k)
            for (int c = tid; c < q; c += nt) {
                const double2 tmp = M[c * q + k];
                M[c * q + k] = M[c * q + p];
                M[c * q + p] = tmp;
            }
        __syncthreads();
        const double2 pv = M[k * q + k];
        const double d = cabs2(pv);
        const double2 inv = d > 0 ? make_double2(pv.x / d, -pv.y / d) : make_double2(0, 0);
        // scale row k (its pivot entry becomes 1/pivot); keep the old column k
        for (int c = tid; c < q; c += nt) M[c * q + k] = (c == k) ? inv : M[c * q + k] * inv;
        for (int r = tid; r < q; r += nt) fcol[r] = M[k * q + r];
        __syncthreads();
        // eliminate column k from the other rows
        for (int e = tid; e < q * q; e += nt) {
            const int c = e / q, r = e % q;
            if (r == k) continue;
            const double2 f = fcol[r];
            if (c == k) M[c * q + r] = -1.0 * (f * inv);
            else M[c * q + r] = cfms(f, M[c * q + k], M[c * q + r]);
        }
        __syncthreads();
    }
    for (int k = q - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int r = tid; r < q; r += nt) {
                const double2 tmp = M[k * q + r];
                M[k * q + r] = M[p * q + r];
                M[p * q + r] = tmp;
            }
        __syncthreads();
    }
    return ok;
}

struct InvTask {
    const double2* src;  // dense source (column-major) or null for a level-0 D block
    double2* dst;
    int l, i;            // strip and global block index (level-0 source)
};

__global__ void k_invert(int ntask, const InvTask* __restrict__ tasks, StripGeom g, const StencilTables* tab,
                         const double* m, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int q = g.q;
    double2* M = reinterpret_cast<double2*>(smem_raw);
    double2* fcol = M + q * q;
    double* redv = reinterpret_cast<double*>(fcol + kMaxQ);
    int* redi = reinterpret_cast<int*>(redv + blockDim.x);
    int* piv = redi + blockDim.x;
    const InvTask tk = tasks[blockIdx.x];
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        const int c = e / q, r = e % q;
        M[e] = tk.src ? tk.src[e] : level0_entry(g, tab, m, tk.l, tk.i, 0, r, c);
    }
    __syncthreads();
    const bool ok = gj_invert(M, q, fcol, piv, redv, redi);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) tk.dst[e] = M[e];
}

// Level-0 reduction for an even block j (global block i = j): from the tridiagonal
// W, D, E and the dense inverses of the odd neighbours, form the dense level-1
// blocks D', W', E'.  One thread per output entry (r, c).
struct Red0Task {
    const double2* dinv_w;  // D^{-1}_{j-1} or null
    const double2* dinv_e;  // D^{-1}_{j+1} or null
    double2* D1;
    double2* W1;            // null if j - 1 has no west neighbour
    double2* E1;            // null if j + 1 has no east neighbour
    int l, i;
};

__global__ void k_reduce0(const Red0Task* __restrict__ tasks, StripGeom g, const StencilTables* tab,
                          const double* m) {
    const Red0Task tk = tasks[blockIdx.x];
    const int q = g.q;
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int c = e / q, r = e % q;
    const int l = tk.l, i = tk.i;
    double2 d = level0_entry(g, tab, m, l, i, 0, r, c);
    double2 w1 = make_double2(0, 0), e1 = make_double2(0, 0);
    // F = W_i Dinv_{i-1}: F(r, c') = sum_{r'} W_i(r, r') Dinv(r', c'), W_i tridiagonal
    if (tk.dinv_w) {
        for (int cc = c - 1; cc <= c + 1; ++cc) {
            if (cc < 0 || cc >= q) continue;
            double2 f = make_double2(0, 0);
            for (int rr = r - 1; rr <= r + 1; ++rr) {
                if (rr < 0 || rr >= q) continue;
                f = cfma(level0_entry(g, tab, m, l, i, 1, r, rr), tk.dinv_w[cc * q + rr], f);
            }
            // D' -= F E_{i-1};  W' = -F W_{i-1}
            d = cfms(f, level0_entry(g, tab, m, l, i - 1, 2, cc, c), d);
            if (tk.W1) w1 = cfms(f, level0_entry(g, tab, m, l, i - 1, 1, cc, c), w1);
        }
    }
    if (tk.dinv_e) {
        for (int cc = c - 1; cc <= c + 1; ++cc) {
            if (cc < 0 || cc >= q) continue;
            double2 gg = make_double2(0, 0);
            for (int rr = r - 1; rr <= r + 1; ++rr) {
                if (rr < 0 || rr >= q) continue;
                gg = cfma(level0_entry(g, tab, m, l, i, 2, r, rr), tk.dinv_e[cc * q + rr], gg);
            }
            d = cfms(gg, level0_entry(g, tab, m, l, i + 1, 1, cc, c), d);
            if (tk.E1) e1 = cfms(gg, level0_entry(g, tab, m, l, i + 1, 2, cc, c), e1);
        }
    }
    tk.D1[e] = d;
    if (tk.W1) tk.W1[e] = w1;
    if (tk.E1) tk.E1[e] = e1;
    }
}

// Batched complex GEMM: C = C0 + a1 A1 B1 + a2 A2 B2 (any term may be absent),
// column-major q x q, one 32 x 32 output tile per block.
struct GemmTask {
    const double2* C0;
    const double2* A1;
    const double2* B1;
    const double2* A2;
    const double2* B2;
    double2* C;
    double a1, a2;  // real scalars (the reductions only need -1, +1)
};

__global__ void __launch_bounds__(256) k_gemm(const GemmTask* __restrict__ tasks, int q) {
    __shared__ double2 As[16][33];
    __shared__ double2 Bs[32][17];
    const GemmTask tk = tasks[blockIdx.x];
    const int tiles = (q + 31) / 32;
    const int tr = blockIdx.y / tiles, tc = blockIdx.y % tiles;
    const int r0 = tr * 32, c0 = tc * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    double2 acc[4];
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
        const int r = r0 + ty + 8 * mm, c = c0 + tx;
        acc[mm] = (tk.C0 && r < q && c < q) ? tk.C0[c * q + r] : make_double2(0, 0);
    }
    for (int term = 0; term < 2; ++term) {
        const double2* A = term == 0 ? tk.A1 : tk.A2;
        const double2* B = term == 0 ? tk.B1 : tk.B2;
        const double al = term == 0 ? tk.a1 : tk.a2;
        if (!A) continue;
        double2 part[4];
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) part[mm] = make_double2(0, 0);
        for (int k0 = 0; k0 < q; k0 += 16) {
            // As[kk][rr] = A(r0+rr, k0+kk);  Bs[cc][kk] = B(k0+kk, c0+cc)
            for (int e = threadIdx.x; e < 16 * 32; e += 256) {
                const int kk = e / 32, rr = e % 32;
                const int r = r0 + rr, k = k0 + kk;
                As[kk][rr] = (r < q && k < q) ? A[k * q + r] : make_double2(0, 0);
            }
            for (int e = threadIdx.x; e < 16 * 32; e += 256) {
                const int cc = e / 16, kk = e % 16;
                const int c = c0 + cc, k = k0 + kk;
                Bs[cc][kk] = (c < q && k < q) ? B[c * q + k] : make_double2(0, 0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                const double2 b = Bs[tx][kk];
#pragma unroll
                for (int mm = 0; mm < 4; ++mm) part[mm] = cfma(As[kk][ty + 8 * mm], b, part[mm]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) acc[mm] = acc[mm] + al * part[mm];
    }
#pragma unroll
    for (int mm = 0; mm < 4; ++mm) {
        const int r = r0 + ty + 8 * mm, c = c0 + tx;
        if (r < q && c < q) tk.C[c * q + r] = acc[mm];
    }
}

// Couplings the local solves read (so the solve path never evaluates the FP64
// stencil coefficients): level-0 west/east blocks and the four injection rows.
template <typename C>
__global__ void k_coef_tables(StripGeom g, const StencilTables* tab, const double* m, int L, C* cw, C* ce, C* cinj) {
    const int n = g.n, q = g.q, E = g.E, t = g.t;
    const size_t total = (size_t)L * n * 3 * q;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % q);
        const int dzi = (int)((e / q) % 3);
        const int i = (int)((e / ((size_t)3 * q)) % n);
        const int l = (int)(e / ((size_t)3 * q * n));
        cw[e] = ccast<C>(strip_coef(g, tab, m, l, r, i, -1, dzi - 1));
        ce[e] = ccast<C>(strip_coef(g, tab, m, l, r, i, 1, dzi - 1));
        if (r == 0) {  // one thread per (l, i, dx) fills the four injection rows
            const int dx = dzi - 1;
            const int rows[4] = {E + t - 1, E + t, E, E - 1};
            const int dzs[4] = {1, -1, -1, 1};
            for (int sl = 0; sl < 4; ++sl)
                cinj[(((size_t)l * 4 + sl) * 3 + dzi) * n + i] = ccast<C>(strip_coef(g, tab, m, l, rows[sl], i, dx, dzs[sl]));
        }
    }
}

__global__ void k_to32(size_t cnt, const double2* __restrict__ a, float2* __restrict__ b) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x)
        b[i] = ccast<float2>(a[i]);
}

template <typename T>
int upload(ls_handle* h, const std::vector<T>& v, T** dptr, size_t* cap) {
    if (v.empty()) return LS_OK;
    if (*cap < v.size()) {
        if (*dptr) cudaFree(*dptr);
        *dptr = nullptr;
        LS_CUDA(cudaMalloc(dptr, sizeof(T) * v.size()));
        *cap = v.size();
    }
    LS_CUDA(cudaMemcpyAsync(*dptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->stream));
    return LS_OK;
}

struct Scratch {
    InvTask* inv = nullptr;
    size_t inv_cap = 0;
    Red0Task* red = nullptr;
    size_t red_cap = 0;
    GemmTask* gem = nullptr;
    size_t gem_cap = 0;
    double2* work[2] = {nullptr, nullptr};  // ping-pong level arrays: [D | W | E] x L x nk
    int* err = nullptr;
    ~Scratch() {
        cudaFree(inv);
        cudaFree(red);
        cudaFree(gem);
        cudaFree(work[0]);
        cudaFree(work[1]);
        cudaFree(err);
    }
};

int factor_direction(ls_handle* h, int dir, Scratch& S) {
    DirFactors& F = h->fac[dir];
    const int n = h->n, L = h->L, q = h->q;
    const size_t qq = (size_t)q * q;
    StripGeom g{n, h->t, h->E, q, h->opts.shift / h->omega};
    const StencilTables* tab = h->dtabs + dir;
    const double* m = dir == 0 ? h->m64 : h->mT64;
    F.m = m;
    F.tab = h->dtabs + dir;
    // level bookkeeping
    F.lev.clear();
    size_t off = 0;
    int nk = n;
    while (nk > 1) {
        CrLevel lv{};
        lv.nk = nk;
        lv.nodd = nk / 2;
        lv.neven = (nk + 1) / 2;
        lv.off_dinv = off;
        off += lv.nodd;
        if (!F.lev.empty()) {
            lv.off_p = off;
            off += lv.nodd;
            lv.off_q = off;
            off += lv.nodd;
            lv.off_f = off;
            off += lv.neven;
            lv.off_g = off;
            off += lv.neven;
        }
        F.lev.push_back(lv);
        nk = (nk + 1) / 2;
    }
    F.K = (int)F.lev.size();
    F.off_top = off++;
    F.mats_per_strip = off;
    LS_CUDA(cudaMalloc(&F.pool64, sizeof(double2) * qq * off * L));
    auto mat = [&](int l, size_t o) { return F.pool64 + ((size_t)l * F.mats_per_strip + o) * qq; };
    const int n1 = (n + 1) / 2;
    // working arrays for level-k dense blocks (k >= 1): [kind][l][j]
    auto wk = [&](int buf, int kind, int l, int j, int nkk) {
        return S.work[buf] + (((size_t)kind * L + l) * nkk + j) * qq;
    };
    if (!S.work[0]) {
        LS_CUDA(cudaMalloc(&S.work[0], sizeof(double2) * qq * 3 * (size_t)L * n1));
        LS_CUDA(cudaMalloc(&S.work[1], sizeof(double2) * qq * 3 * (size_t)L * ((n1 + 1) / 2 + 1)));
        LS_CUDA(cudaMalloc(&S.err, sizeof(int)));
    }
    LS_CUDA(cudaMemsetAsync(S.err, 0, sizeof(int), h->stream));
    const size_t inv_smem = (qq + kMaxQ) * sizeof(double2) + 256 * (sizeof(double) + sizeof(int)) + kMaxQ * sizeof(int);
    LS_CUDA(cudaFuncSetAttribute(k_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_smem));
    int cur = 0;
    for (int k = 0; k < F.K; ++k) {
        const CrLevel& lv = F.lev[k];
        const int nkk = lv.nk, nnext = (nkk + 1) / 2;
        // 1) invert odd blocks
        std::vector<InvTask> it;
        it.reserve((size_t)L * lv.nodd);
        for (int l = 0; l < L; ++l)
            for (int j = 1; j < nkk; j += 2) {
                InvTask t{};
                t.src = k == 0 ? nullptr : wk(cur, 0, l, j, nkk);
                t.dst = mat(l, lv.off_dinv + (j - 1) / 2);
                t.l = l;
                t.i = j;  // level 0: global block index = j
                it.push_back(t);
            }
        LS_TRY(upload(h, it, &S.inv, &S.inv_cap));
        if (!it.empty()) LS_LAUNCH(h, k_invert, (unsigned)it.size(), 256, inv_smem, (int)it.size(), S.inv, g, tab, m, S.err);
        const int nxt = 1 - cur;
        if (k == 0) {
            // 2) level-0 reduction of even blocks into level-1 dense blocks
            std::vector<Red0Task> rt;
            rt.reserve((size_t)L * lv.neven);
            for (int l = 0; l < L; ++l)
                for (int j = 0; j < nkk; j += 2) {
                    Red0Task t{};
                    // odd block o sits at index (o - 1) / 2 of the level's D^{-1} list
                    t.dinv_w = j >= 1 ? mat(l, lv.off_dinv + (j - 2) / 2) : nullptr;
                    t.dinv_e = j + 1 < nkk ? mat(l, lv.off_dinv + j / 2) : nullptr;
                    t.D1 = wk(cur, 0, l, j / 2, n1);
                    t.W1 = j >= 2 ? wk(cur, 1, l, j / 2, n1) : nullptr;
                    t.E1 = j + 2 < nkk ? wk(cur, 2, l, j / 2, n1) : nullptr;
                    t.l = l;
                    t.i = j;
                    rt.push_back(t);
                }
            LS_TRY(upload(h, rt, &S.red, &S.red_cap));
            LS_LAUNCH(h, k_reduce0, (unsigned)rt.size(), 256, 0, S.red, g, tab, m);
            // level-1 blocks live in work[cur]; the next level reads them there
            continue;
        }
        // levels >= 1: blocks of this level are in work[cur] with nkk entries per strip
        std::vector<GemmTask> gt;
        gt.reserve((size_t)L * nkk * 2);
        for (int l = 0; l < L; ++l) {
            for (int j = 1; j < nkk; j += 2) {  // odd: P = Dinv W, Q = Dinv E
                const double2* dinv = mat(l, lv.off_dinv + (j - 1) / 2);
                GemmTask t{};
                t.A1 = dinv;
                t.B1 = wk(cur, 1, l, j, nkk);
                t.a1 = 1.0;
                t.C = mat(l, lv.off_p + (j - 1) / 2);
                gt.push_back(t);
                if (j + 1 < nkk) {
                    GemmTask u{};
                    u.A1 = dinv;
                    u.B1 = wk(cur, 2, l, j, nkk);
                    u.a1 = 1.0;
                    u.C = mat(l, lv.off_q + (j - 1) / 2);
                    gt.push_back(u);
                }
            }
            for (int j = 0; j < nkk; j += 2) {  // even: F = W Dinv_{j-1}, G = E Dinv_{j+1}
                if (j >= 1) {
                    GemmTask t{};
                    t.A1 = wk(cur, 1, l, j, nkk);
                    t.B1 = mat(l, lv.off_dinv + (j - 1) / 2);
                    t.a1 = 1.0;
                    t.C = mat(l, lv.off_f + j / 2);
                    gt.push_back(t);
                }
                if (j + 1 < nkk) {
                    GemmTask t{};
                    t.A1 = wk(cur, 2, l, j, nkk);
                    t.B1 = mat(l, lv.off_dinv + j / 2);
                    t.a1 = 1.0;
                    t.C = mat(l, lv.off_g + j / 2);
                    gt.push_back(t);
                }
            }
        }
        const int tiles = (q + 31) / 32;
        LS_TRY(upload(h, gt, &S.gem, &S.gem_cap));
        if (!gt.empty()) LS_LAUNCH(h, k_gemm, dim3((unsigned)gt.size(), tiles * tiles), 256, 0, S.gem, q);
        // 3) reduced blocks for level k+1 into work[nxt]
        std::vector<GemmTask> rt;
        rt.reserve((size_t)L * nnext * 3);
        for (int l = 0; l < L; ++l)
            for (int j = 0; j < nkk; j += 2) {
                const double2* Fm = j >= 1 ? mat(l, lv.off_f + j / 2) : nullptr;
                const double2* Gm = j + 1 < nkk ? mat(l, lv.off_g + j / 2) : nullptr;
                GemmTask d{};
                d.C0 = wk(cur, 0, l, j, nkk);
                if (Fm) { d.A1 = Fm; d.B1 = wk(cur, 2, l, j - 1, nkk); d.a1 = -1.0; }
                if (Gm) { d.A2 = Gm; d.B2 = wk(cur, 1, l, j + 1, nkk); d.a2 = -1.0; }
                d.C = wk(nxt, 0, l, j / 2, nnext);
                rt.push_back(d);
                if (Fm && j >= 2) {
                    GemmTask w{};
                    w.A1 = Fm;
                    w.B1 = wk(cur, 1, l, j - 1, nkk);
                    w.a1 = -1.0;
                    w.C = wk(nxt, 1, l, j / 2, nnext);
                    rt.push_back(w);
                }
                if (Gm && j + 2 < nkk) {
                    GemmTask e{};
                    e.A1 = Gm;
                    e.B1 = wk(cur, 2, l, j + 1, nkk);
                    e.a1 = -1.0;
                    e.C = wk(nxt, 2, l, j / 2, nnext);
                    rt.push_back(e);
                }
            }
        LS_TRY(upload(h, rt, &S.gem, &S.gem_cap));
        if (!rt.empty()) LS_LAUNCH(h, k_gemm, dim3((unsigned)rt.size(), tiles * tiles), 256, 0, S.gem, q);
        cur = nxt;
    }
    // top block: the single block of level K (level 0 if n == 1 is excluded by n >= 8)
    {
        std::vector<InvTask> it;
        for (int l = 0; l < L; ++l) {
            InvTask t{};
            t.src = wk(cur, 0, l, 0, F.K == 1 ? n1 : (F.lev.back().nk + 1) / 2);
            t.dst = mat(l, F.off_top);
            t.l = l;
            t.i = 0;
            it.push_back(t);
        }
        LS_TRY(upload(h, it, &S.inv, &S.inv_cap));
        LS_LAUNCH(h, k_invert, (unsigned)it.size(), 256, inv_smem, (int)it.size(), S.inv, g, tab, m, S.err);
    }
    {  // coupling tables for the solve
        const size_t cnt = (size_t)L * n * 3 * q, ci = (size_t)L * 4 * 3 * n;
        if (h->prec == LS_MIXED) {
            LS_CUDA(cudaMalloc(&F.cw, sizeof(float2) * cnt));
            LS_CUDA(cudaMalloc(&F.ce, sizeof(float2) * cnt));
            LS_CUDA(cudaMalloc(&F.cinj, sizeof(float2) * ci));
            LS_LAUNCH(h, k_coef_tables<float2>, 1216, 256, 0, g, tab, m, L, static_cast<float2*>(F.cw),
                      static_cast<float2*>(F.ce), static_cast<float2*>(F.cinj));
        } else {
            LS_CUDA(cudaMalloc(&F.cw, sizeof(double2) * cnt));
            LS_CUDA(cudaMalloc(&F.ce, sizeof(double2) * cnt));
            LS_CUDA(cudaMalloc(&F.cinj, sizeof(double2) * ci));
            LS_LAUNCH(h, k_coef_tables<double2>, 1216, 256, 0, g, tab, m, L, static_cast<double2*>(F.cw),
                      static_cast<double2*>(F.ce), static_cast<double2*>(F.cinj));
        }
    }
    int herr = 0;
    LS_CUDA(cudaMemcpyAsync(&herr, S.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LS_CUDA(cudaStreamSynchronize(h->stream));
    if (herr) return LS_ESINGULAR;
    if (h->prec == LS_MIXED) {
        const size_t cnt = qq * F.mats_per_strip * L;
        LS_CUDA(cudaMalloc(&F.pool32, sizeof(float2) * cnt));
        LS_LAUNCH(h, k_to32, 1216, 256, 0, cnt, F.pool64, F.pool32);
        LS_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(F.pool64);
        F.pool64 = nullptr;
    }
    return LS_OK;
}

}  // namespace

int ls_factor_all(ls_handle* h) {
    if (h->q > kMaxQ) return LS_EINVAL;
    Scratch S;
    for (int dir = 0; dir < 2; ++dir) LS_TRY(factor_direction(h, dir, S));
    return LS_OK;
}

void ls_factor_free(ls_handle* h) {
    ls_bd_graph_free(h);
    ls_cr_tc_free(h);
    for (int d = 0; d < 2; ++d) {
        DirFactors& F = h->fac[d];
        cudaFree(F.pool64);
        cudaFree(F.pool32);
        cudaFree(F.cw);
        cudaFree(F.ce);
        cudaFree(F.cinj);
        F.pool64 = nullptr;
        F.pool32 = nullptr;
        F.cw = F.ce = F.cinj = nullptr;
    }
}
