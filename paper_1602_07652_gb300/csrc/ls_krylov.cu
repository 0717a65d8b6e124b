// ls_krylov.cu -- the two Krylov levels of Sec. 4 on the device.
//
//  * inner level (Algorithm 3): GMRES on C v = A r, right-preconditioned by
//    Algorithm 2, from v = 0, to the relative tolerance inner_tol (1e-3);
//  * outer level: GMRES on H u = f preconditioned by Algorithm 3.  Algorithm 3
//    stops at a tolerance, so it is not a fixed linear map; the outer level is
//    flexible GMRES (Sec. 6 names it), which stores the preconditioned
//    directions Z.  The inner level uses the same code (with a fixed linear
//    preconditioner flexible GMRES is right-preconditioned GMRES).
//  * LS_MIXED: the outer iteration runs with the FP32 FFT convolution inside an
//    FP64 iterative refinement loop (r = f - H u with the FP64 apply, solve
//    H d = r, u += d) until the FP64 residual meets the tolerance.
// Arnoldi: classical Gram-Schmidt applied twice (CGS2), dot products and norms
// accumulated in FP64 on the device; the small Hessenberg least-squares problem
// (Givens rotations) is solved on the host, with one device->host copy per step.
//
// Batches: nb right-hand sides iterate in lockstep, each with its own Krylov
// space, Hessenberg matrix and stopping test; a step applies the preconditioner
// to the whole block of current directions at once, so every Algorithm 2
// application (the dominant cost) serves all members still iterating.  A
// member that has converged leaves the cycle; its slot in the block is zeroed.
// With nb = 1 this is exactly the single right-hand-side iteration.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "ls_internal.cuh"

int ls_timing_begin(ls_handle* h);
int ls_timing_end(ls_handle* h, int kind);

namespace {

using cd = std::complex<double>;

enum Op { OP_H64, OP_HMIX, OP_C };
enum Pc { PC_NONE, PC_BD, PC_LS, PC_NET };

// Vectors of a Krylov space for up to nbcap members: direction j of member b is
// V + (j * nbcap + b) * N, so the members' j-th directions form one contiguous
// block (what the batched preconditioner reads and writes).
// VT: double2 (LS_FP64) or float2 (LS_MIXED: the FP32 correction solve and Algorithm 3).
template <typename VT>
struct KrylovSpace {
    VT* V = nullptr;          // (m+1) blocks
    VT* Z = nullptr;          // m blocks (preconditioned directions)
    VT* w = nullptr;          // one block of work vectors
    VT* r = nullptr;          // one block of residuals
    double2* hdev = nullptr;  // per member: 2 (m+1) + 2 coefficients
    int m = 0;
};

struct Ctx {
    ls_handle* h;
    KrylovSpace<double2> outer, inner;      // LS_FP64
    KrylovSpace<float2> outer32, inner32;   // LS_MIXED
    double2* tmpA = nullptr;    // A r for Algorithm 3, one block (LS_FP64)
    float2* tmpA32 = nullptr;   // the same in FP32 (LS_MIXED)
    double2* dref = nullptr;    // LS_MIXED: the FP64 refinement residuals, one block
    double2* stage64 = nullptr; // LS_MIXED: two FP64 fields (the learned step's input and output)
    int nbcap = 0;
};
template <typename VT> KrylovSpace<VT>& inner_space(Ctx* c);
template <> KrylovSpace<double2>& inner_space<double2>(Ctx* c) { return c->inner; }
template <> KrylovSpace<float2>& inner_space<float2>(Ctx* c) { return c->inner32; }
double2* tmpA_of(Ctx* c, double2*) { return c->tmpA; }
float2* tmpA_of(Ctx* c, float2*) { return c->tmpA32; }

Ctx* ctx_of(ls_handle* h);

size_t hstride(int m) { return 2 * (size_t)(m + 1) + 2; }

template <typename VT>
int alloc_space(ls_handle* h, KrylovSpace<VT>& S, int m, int nbcap) {
    const size_t N = (size_t)h->n * h->n;
    S.m = m;
    LS_CUDA(cudaMalloc(&S.V, sizeof(VT) * N * (m + 1) * nbcap));
    LS_CUDA(cudaMalloc(&S.Z, sizeof(VT) * N * m * nbcap));
    LS_CUDA(cudaMalloc(&S.w, sizeof(VT) * N * nbcap));
    LS_CUDA(cudaMalloc(&S.r, sizeof(VT) * N * nbcap));
    LS_CUDA(cudaMalloc(&S.hdev, sizeof(double2) * hstride(m) * nbcap));
    return LS_OK;
}

// FP32 vectors (LS_MIXED): H with the FP32-I/O convolution, C with the FP32 stencil
int apply_op(ls_handle* h, Op op, const float2* x, float2* y) {
    if (op == OP_HMIX) {
        LS_TRY(ls_timing_begin(h));
        LS_TRY(ls_apply32(h, x, y));
        return ls_timing_end(h, 0);
    }
    if (op == OP_C) {
        LS_TRY(ls_timing_begin(h));
        LS_TRY(ls_stencil_apply_f32(h, 0, 1, x, y));
        return ls_timing_end(h, 3);
    }
    return LS_EINVAL;   // the FP64 apply takes FP64 vectors
}

int apply_op(ls_handle* h, Op op, const double2* x, double2* y) {
    switch (op) {
        case OP_H64: {
            LS_TRY(ls_timing_begin(h));
            LS_TRY(ls_apply64(h, x, y));
            return ls_timing_end(h, 0);
        }
        case OP_HMIX: {
            LS_TRY(ls_timing_begin(h));
            LS_TRY(ls_apply_mx(h, x, y));
            return ls_timing_end(h, 0);
        }
        default: {
            LS_TRY(ls_timing_begin(h));
            LS_TRY(ls_stencil_apply(h, 0, 1, x, nullptr, y));
            return ls_timing_end(h, 3);
        }
    }
}

struct Result {
    int iters = 0;
    double relres = 0;
    bool converged = false;
};

template <typename VT>
int fgmres_b(ls_handle* h, Ctx* c, KrylovSpace<VT>& S, Op op, Pc pc, const VT* b, VT* x, bool x0,
             const double* tol, int maxit, int nb, const unsigned char* live, Result* res, ls_stats* st);

// Right-hand sides per batched Algorithm 2 call: the autotuner's choice, else the
// largest the sweep kernels take (FP64: 4).
int bd_chunk(const ls_handle* h) {
    const int cap = ls_bd_cap(h);
    return h->bd_chunk > 0 && h->bd_chunk < cap ? h->bd_chunk : cap;
}

// z_b = M v_b for the members with on[b]; v and z are blocks of nb vectors.
// Members that are off have their slot of v zeroed (their z is not used).
// The learned step on a member's field (the network takes FP64 fields): FP32 vectors go
// through the two FP64 staging fields of the context.
int net_apply(ls_handle* h, const double2* v, double2* z) {
    return ls_net_apply_field(h->net, h->stream, h->n, h->n, v, h->m64, z);
}
int net_apply(ls_handle* h, const float2* v, float2* z) {
    Ctx* c = ctx_of(h);
    const size_t N = (size_t)h->n * h->n;
    LS_TRY(ls_vec_copy(h, v, c->stage64));
    LS_TRY(ls_net_apply_field(h->net, h->stream, h->n, h->n, c->stage64, h->m64, c->stage64 + N));
    return ls_vec_copy(h, c->stage64 + N, z);
}
// Algorithm 1 (the Gauss-Seidel preconditioner option) on a chunk of members: FP64 fields
// directly, FP32 ones through the upper half of the lane's FP64 scratch fields (the
// horizontal sweep does not use them).
int gs_chunk(ls_handle* h, const double2* v, double2* z, int cnt) { return ls_sweep_dir_b(h, 0, v, z, cnt); }
int gs_chunk(ls_handle* h, const float2* v, float2* z, int cnt) {
    const size_t N = (size_t)h->n * h->n;
    LS_TRY(ls_sweep_reserve(h, cnt));
    double2* in = static_cast<double2*>(h->lanes[h->lane].vtmp) + 2 * N * cnt;
    double2* out = in + N * cnt;
    for (int b = 0; b < cnt; ++b) LS_TRY(ls_vec_copy(h, v + b * N, in + b * N));
    LS_TRY(ls_sweep_dir_b(h, 0, in, out, cnt));
    for (int b = 0; b < cnt; ++b) LS_TRY(ls_vec_copy(h, out + b * N, z + b * N));
    return LS_OK;
}
int stencil_A(ls_handle* h, const double2* v, double2* y) { return ls_stencil_apply(h, 0, 0, v, nullptr, y); }
int stencil_A(ls_handle* h, const float2* v, float2* y) { return ls_stencil_apply_f32(h, 0, 0, v, y); }

template <typename VT>
int apply_pc_b(ls_handle* h, Pc pc, VT* v, VT* z, int nb, const unsigned char* on, ls_stats* st) {
    const size_t N = (size_t)h->n * h->n;
    int top = 0;
    for (int b = 0; b < nb; ++b)
        if (on[b]) top = b + 1;
    if (pc == PC_NONE) {
        for (int b = 0; b < top; ++b)
            if (on[b]) LS_TRY(ls_vec_copy(h, v + b * N, z + b * N));
        return LS_OK;
    }
    if (pc == PC_NET) {  // the learned step: z = s N(v / s, m)
        for (int b = 0; b < top; ++b)
            if (on[b]) {
                LS_TRY(net_apply(h, v + b * N, z + b * N));
                h->learned_steps++;
            }
        return LS_OK;
    }
    if (pc == PC_BD) {
        const int ch = bd_chunk(h);
        if (h->opts.inner_precond == LS_PC_GS) {
            for (int b = 0; b < top; ++b)
                if (!on[b]) LS_TRY(ls_vec_zero(h, v + b * N));
            LS_TRY(ls_timing_begin(h));
            for (int b0 = 0; b0 < top; b0 += ch) {
                const int cnt = top - b0 < ch ? top - b0 : ch;
                LS_TRY(gs_chunk(h, v + b0 * N, z + b0 * N, cnt));
            }
            h->sweep_fields += top;
            h->sweep_hist[top < LS_MAX_BATCH ? top : LS_MAX_BATCH]++;
            return ls_timing_end(h, 1);
        }
        // Algorithm 2 costs what the batch it runs costs, whether a slot's member is still
        // iterating or not: the members that are on move into the leading slots first.
        // Slot k takes member act[k] >= k in increasing k (a slot is overwritten only
        // after its own member has moved out), and the moves are undone in decreasing k,
        // which restores every member's direction and puts its result in its own slot.
        std::vector<int> act;
        for (int b = 0; b < top; ++b)
            if (on[b]) act.push_back(b);
        const int cnt = h->pack_members ? (int)act.size() : top;
        if (h->pack_members) {
            for (int k = 0; k < cnt; ++k)
                if (act[k] != k) LS_TRY(ls_vec_copy(h, (const VT*)(v + act[k] * N), v + k * N));
        } else {
            for (int b = 0; b < top; ++b)
                if (!on[b]) LS_TRY(ls_vec_zero(h, v + b * N));
        }
        std::vector<unsigned char> all(cnt, 1);
        LS_TRY(ls_timing_begin(h));
        // chunks run concurrently; idle ones are skipped
        LS_TRY(ls_bd_lanes(h, v, z, cnt, ch, h->pack_members ? all.data() : on));
        LS_TRY(ls_timing_end(h, 1));
        h->sweep_fields += cnt;
        h->sweep_hist[cnt < LS_MAX_BATCH ? cnt : LS_MAX_BATCH]++;
        if (h->pack_members)
            for (int k = cnt - 1; k >= 0; --k)
                if (act[k] != k) {
                    LS_TRY(ls_vec_copy(h, (const VT*)(v + k * N), v + act[k] * N));
                    LS_TRY(ls_vec_copy(h, (const VT*)(z + k * N), z + act[k] * N));
                }
        return LS_OK;
    }
    // Algorithm 3: z = GMRES(C, A v, Algorithm 2, inner_tol), all members at once
    Ctx* c = ctx_of(h);
    VT* tA = tmpA_of(c, (VT*)nullptr);
    for (int b = 0; b < top; ++b)
        if (on[b]) {
            LS_TRY(ls_timing_begin(h));
            LS_TRY(stencil_A(h, v + b * N, tA + b * N));
            LS_TRY(ls_timing_end(h, 3));
        }
    std::vector<double> tl(nb, h->opts.inner_tol);
    std::vector<Result> r(nb);
    LS_TRY(fgmres_b(h, c, inner_space<VT>(c), OP_C, PC_BD, (const VT*)tA, z, false, tl.data(), h->opts.inner_maxit,
                    top, on, r.data(), nullptr));
    if (st)
        for (int b = 0; b < top; ++b)
            if (on[b]) {
                st->inner_iters_total += r[b].iters;
                st->inner_calls += 1;
            }
    return LS_OK;
}

struct Member {
    double nb = 0, beta = 0, relres = 0;
    double cyc0 = 0;      // true relative residual when the current cycle started
    int total = 0, k = 0;
    bool active = false;  // still iterating (not converged, under maxit)
    bool cyc = false;     // taking part in the current Arnoldi cycle
    std::vector<cd> H, cs, sn, gv, y;
};

// Flexible GMRES for members b < nb with live[b]: S.V, S.Z hold the members'
// spaces; b, x are blocks of nb vectors (stride N).
template <typename VT>
int fgmres_b(ls_handle* h, Ctx* c, KrylovSpace<VT>& S, Op op, Pc pc, const VT* b, VT* x, bool x0,
             const double* tol, int maxit, int nb, const unsigned char* live, Result* res, ls_stats* st) {
    const size_t N = (size_t)h->n * h->n;
    const size_t ldv = N * c->nbcap;  // distance between directions j and j+1 of a member
    const int m = S.m;
    const size_t HS = hstride(m);
    auto V = [&](int j, int mb) { return S.V + (size_t)j * ldv + mb * N; };
    auto Zb = [&](int j) { return S.Z + (size_t)j * ldv; };
    std::vector<Member> M(nb);
    std::vector<double> nrm(nb, 0.0);   // norms of the members' vectors, by member
    std::vector<int> lv, nz;            // live members; live members with b != 0
    for (int i = 0; i < nb; ++i) {
        res[i] = Result{};
        if (live[i]) lv.push_back(i);
    }
    LS_TRY(ls_vec_norms_b(h, b, N, lv.data(), (int)lv.size(), nrm.data()));
    for (int i : lv) {
        Member& e = M[i];
        const VT* bi = b + i * N;
        VT* xi = x + i * N;
        VT* ri = S.r + i * N;
        e.nb = nrm[i];
        if (!std::isfinite(e.nb)) return LS_ENAN;
        if (e.nb == 0.0) {
            LS_TRY(ls_vec_zero(h, xi));
            res[i].converged = true;
            continue;
        }
        nz.push_back(i);
        if (x0) {
            LS_TRY(apply_op(h, op, xi, ri));
            LS_TRY(ls_vec_axpby(h, make_double2(1, 0), bi, make_double2(-1, 0), ri));  // r = b - A x
        } else {
            LS_TRY(ls_vec_zero(h, xi));
            LS_TRY(ls_vec_copy(h, bi, ri));
        }
    }
    LS_TRY(ls_vec_norms_b(h, (const VT*)S.r, N, nz.data(), (int)nz.size(), nrm.data()));
    for (int i : nz) {
        Member& e = M[i];
        e.beta = nrm[i];
        e.relres = e.beta / e.nb;
        if (!std::isfinite(e.relres)) return LS_ENAN;
        e.active = e.relres > tol[i] && e.total < maxit;
        e.H.assign((size_t)(m + 1) * m, cd(0));
        e.cs.assign(m, cd(0));
        e.sn.assign(m, cd(0));
        e.gv.assign(m + 1, cd(0));
        e.y.assign(m, cd(0));
    }
    std::vector<double2> hh_all(HS * nb);  // host copy of the members' coefficients
    std::vector<unsigned char> on(nb);
    for (;;) {
        bool any = false;
        for (int i = 0; i < nb; ++i) {
            Member& e = M[i];
            e.cyc = e.active;
            if (!e.active) continue;
            any = true;
            LS_TRY(ls_vec_axpby(h, make_double2(1.0 / e.beta, 0), S.r + i * N, make_double2(0, 0), V(0, i)));
            std::fill(e.gv.begin(), e.gv.end(), cd(0));
            std::fill(e.H.begin(), e.H.end(), cd(0));
            e.gv[0] = e.beta;
            e.cyc0 = e.relres;
            e.k = 0;
        }
        if (!any) break;
        for (int j = 0; j < m; ++j) {
            bool inc = false;
            for (int i = 0; i < nb; ++i) {
                on[i] = M[i].cyc;
                inc = inc || M[i].cyc;
            }
            if (!inc) break;
            // with a network attached, the outer cycle's first direction is the learned step
            const Pc pcj = (pc == PC_LS && j == 0 && h->net) ? PC_NET : pc;
            LS_TRY(apply_pc_b(h, pcj, V(j, 0), Zb(j), nb, on.data(), st));
            std::vector<int> ons;
            for (int i = 0; i < nb; ++i)
                if (on[i]) {
                    ons.push_back(i);
                    LS_TRY(apply_op(h, op, Zb(j) + i * N, V(j + 1, i)));
                }
            // CGS2 against V_0..V_j in three fused passes (dots; update and dots; update and
            // norm), each one launch for all members; coefficients stay on the device
            const int cnt = (int)ons.size();
            LS_TRY(ls_timing_begin(h));
            LS_TRY(ls_vec_orth_b(h, 0, j + 1, S.V, ldv, N, nullptr, 0, V(j + 1, 0), ons.data(), cnt, S.hdev, HS));
            LS_TRY(ls_vec_orth_b(h, 1, j + 1, S.V, ldv, N, S.hdev, HS, V(j + 1, 0), ons.data(), cnt,
                                 S.hdev + (m + 1), HS));
            LS_TRY(ls_vec_orth_b(h, 2, j + 1, S.V, ldv, N, S.hdev + (m + 1), HS, V(j + 1, 0), ons.data(), cnt,
                                 S.hdev + 2 * (m + 1), HS));
            LS_TRY(ls_timing_end(h, 4));
            LS_CUDA(cudaMemcpyAsync(hh_all.data(), S.hdev, sizeof(double2) * HS * nb, cudaMemcpyDeviceToHost,
                                    h->stream));
            LS_CUDA(cudaStreamSynchronize(h->stream));
            for (int i = 0; i < nb; ++i) {
                if (!on[i]) continue;
                Member& e = M[i];
                const double2* hh = hh_all.data() + i * HS;
                std::vector<cd>& H = e.H;
                for (int r = 0; r <= j; ++r)
                    H[(size_t)r * m + j] = cd(hh[r].x + hh[m + 1 + r].x, hh[r].y + hh[m + 1 + r].y);
                const double hn = std::sqrt(std::max(hh[2 * (m + 1)].x, 0.0));
                if (!std::isfinite(hn)) return LS_ENAN;
                H[(size_t)(j + 1) * m + j] = hn;
                for (int r = 0; r < j; ++r) {  // previous rotations
                    const cd t = e.cs[r] * H[(size_t)r * m + j] + e.sn[r] * H[(size_t)(r + 1) * m + j];
                    H[(size_t)(r + 1) * m + j] =
                        -std::conj(e.sn[r]) * H[(size_t)r * m + j] + e.cs[r] * H[(size_t)(r + 1) * m + j];
                    H[(size_t)r * m + j] = t;
                }
                const cd a = H[(size_t)j * m + j], cc = H[(size_t)(j + 1) * m + j];
                const double den = std::sqrt(std::norm(a) + std::norm(cc));
                if (den == 0.0) {
                    e.cs[j] = 1.0;
                    e.sn[j] = 0.0;
                } else if (std::abs(a) == 0.0) {
                    e.cs[j] = 0.0;
                    e.sn[j] = 1.0;
                } else {
                    e.cs[j] = std::abs(a) / den;
                    e.sn[j] = (a / std::abs(a)) * std::conj(cc) / den;
                }
                H[(size_t)j * m + j] = e.cs[j] * a + e.sn[j] * cc;
                H[(size_t)(j + 1) * m + j] = 0.0;
                e.gv[j + 1] = -std::conj(e.sn[j]) * e.gv[j];
                e.gv[j] = e.cs[j] * e.gv[j];
                ++e.total;
                e.k = j + 1;
                e.relres = std::abs(e.gv[j + 1]) / e.nb;
                if (e.relres <= tol[i] || e.total >= maxit || hn == 0.0) {
                    e.cyc = false;
                    continue;
                }
                VT* vn = V(j + 1, i);
                LS_TRY(ls_vec_axpby(h, make_double2(1.0 / hn, 0), vn, make_double2(0, 0), vn));
            }
        }
        // end of the cycle: x += Z y for every member that iterated, then its true residual
        std::vector<int> done;
        for (int i = 0; i < nb; ++i) {
            Member& e = M[i];
            if (!e.active) continue;
            done.push_back(i);
            const int k = e.k;
            for (int r = k - 1; r >= 0; --r) {
                cd s = e.gv[r];
                for (int l = r + 1; l < k; ++l) s -= e.H[(size_t)r * m + l] * e.y[l];
                e.y[r] = s / e.H[(size_t)r * m + r];
            }
            std::vector<double2> yc(k);
            for (int r = 0; r < k; ++r) yc[r] = make_double2(e.y[r].real(), e.y[r].imag());
            VT* xi = x + i * N;
            VT* ri = S.r + i * N;
            LS_TRY(ls_vec_combine(h, k, Zb(0) + i * N, ldv, yc.data(), xi));
            LS_TRY(apply_op(h, op, xi, ri));
            LS_TRY(ls_vec_axpby(h, make_double2(1, 0), b + i * N, make_double2(-1, 0), ri));
        }
        LS_TRY(ls_vec_norms_b(h, (const VT*)S.r, N, done.data(), (int)done.size(), nrm.data()));
        for (int i : done) {
            Member& e = M[i];
            e.beta = nrm[i];
            e.relres = e.beta / e.nb;
            if (!std::isfinite(e.relres)) return LS_ENAN;
            e.active = e.relres > tol[i] && e.total < maxit;
            // the FP32 correction of a mixed solve stops where FP32 stops gaining (a cycle
            // that did not halve its true residual): the FP64 refinement takes it from there
            if (op == OP_HMIX && e.relres > 0.5 * e.cyc0) e.active = false;
        }
    }
    for (int i = 0; i < nb; ++i) {
        if (!live[i] || M[i].nb == 0.0) continue;
        res[i].iters = M[i].total;
        res[i].relres = M[i].relres;
        res[i].converged = M[i].relres <= tol[i];
    }
    return LS_OK;
}

}  // namespace

// per-handle Krylov context
namespace {
Ctx* ctx_of(ls_handle* h) { return static_cast<Ctx*>(h->krylov); }
template <typename VT>
void free_space(KrylovSpace<VT>& S) {
    cudaFree(S.V);
    cudaFree(S.Z);
    cudaFree(S.w);
    cudaFree(S.r);
    cudaFree(S.hdev);
    S = KrylovSpace<VT>{};
}
void free_all(Ctx* c) {
    free_space(c->outer);
    free_space(c->inner);
    free_space(c->outer32);
    free_space(c->inner32);
    cudaFree(c->tmpA);
    cudaFree(c->tmpA32);
    cudaFree(c->dref);
    cudaFree(c->stage64);
    c->tmpA = nullptr;
    c->tmpA32 = nullptr;
    c->dref = nullptr;
    c->stage64 = nullptr;
    c->nbcap = 0;
}
// Krylov spaces for nb members (grown on demand, never shrunk): FP64 vectors for
// LS_FP64, FP32 ones (plus the FP64 refinement residuals) for LS_MIXED.
int ctx_ensure(ls_handle* h, int nb) {
    Ctx* c = ctx_of(h);
    if (c && c->nbcap >= nb) return LS_OK;
    if (!c) {
        c = new Ctx();
        c->h = h;
        h->krylov = c;
    }
    free_all(c);
    const size_t N = (size_t)h->n * h->n;
    if (h->prec == LS_FP64) {
        LS_TRY(alloc_space(h, c->outer, h->opts.outer_restart, nb));
        LS_TRY(alloc_space(h, c->inner, h->opts.inner_restart, nb));
        LS_CUDA(cudaMalloc(&c->tmpA, sizeof(double2) * N * nb));
    } else {
        LS_TRY(alloc_space(h, c->outer32, h->opts.outer_restart, nb));
        LS_TRY(alloc_space(h, c->inner32, h->opts.inner_restart, nb));
        LS_CUDA(cudaMalloc(&c->tmpA32, sizeof(float2) * N * nb));
        LS_CUDA(cudaMalloc(&c->dref, sizeof(double2) * N * nb));
        LS_CUDA(cudaMalloc(&c->stage64, sizeof(double2) * N * 2));
    }
    c->nbcap = nb;
    return LS_OK;
}
}  // namespace

void ls_krylov_free(ls_handle* h) {
    Ctx* c = ctx_of(h);
    if (!c) return;
    free_all(c);
    delete c;
    h->krylov = nullptr;
}

int ls_inner_gmres(ls_handle* h, const double2* g, double tol, double2* v, int* iters) {
    LS_TRY(ctx_ensure(h, 1));
    Ctx* c = ctx_of(h);
    Result r;
    const unsigned char live = 1;
    if (h->prec == LS_FP64) {
        LS_TRY(fgmres_b(h, c, c->inner, OP_C, PC_BD, g, v, false, &tol, h->opts.inner_maxit, 1, &live, &r,
                        nullptr));
    } else {  // FP32 vectors: g rounded into the outer space's work block, the result widened into v
        float2* g32 = c->outer32.w;
        float2* v32 = c->inner32.w;
        LS_TRY(ls_vec_copy(h, g, g32));
        LS_TRY(fgmres_b(h, c, c->inner32, OP_C, PC_BD, (const float2*)g32, v32, false, &tol, h->opts.inner_maxit,
                        1, &live, &r, nullptr));
        LS_TRY(ls_vec_copy(h, (const float2*)v32, v));
    }
    if (iters) *iters = r.iters;
    return r.converged ? LS_OK : LS_ENOCONV;
}

// Solve H u_b = f_b for nb right-hand sides (blocks of nb vectors) in lockstep.
// Statistics: iteration counts summed over the members, refinement steps and
// the true relative residual the largest over the members.
int ls_outer_solve_b(ls_handle* h, int nb, const double2* f, double tol, double2* u, int use_x0, ls_stats* st) {
    LS_TRY(ctx_ensure(h, nb));
    Ctx* c = ctx_of(h);
    const size_t N = (size_t)h->n * h->n;
    std::vector<double> nf(nb), relres(nb, 0.0), stol(nb);
    std::vector<unsigned char> live(nb, 0);
    std::vector<Result> r(nb);
    int nlive = 0;
    std::vector<int> all(nb);
    for (int i = 0; i < nb; ++i) all[i] = i;
    LS_TRY(ls_vec_norms_b(h, f, N, all.data(), nb, nf.data()));
    for (int i = 0; i < nb; ++i) {
        if (!std::isfinite(nf[i])) return LS_ENAN;
        if (nf[i] == 0.0) LS_TRY(ls_vec_zero(h, u + i * N));
        else {
            live[i] = 1;
            ++nlive;
        }
    }
    double worst = 0.0;
    bool all_conv = true;
    if (nlive == 0) {
        if (st) st->true_rel_residual = 0.0;
        return LS_OK;
    }
    if (h->prec == LS_FP64) {
        std::vector<double> tl(nb, tol);
        LS_TRY(fgmres_b(h, c, c->outer, OP_H64, PC_LS, f, u, use_x0 != 0, tl.data(), h->opts.outer_maxit, nb,
                        live.data(), r.data(), st));
        for (int i = 0; i < nb; ++i) {
            if (!live[i]) continue;
            if (st) st->outer_iters += r[i].iters;
            worst = std::max(worst, r[i].relres);
            all_conv = all_conv && r[i].converged;
        }
        if (st) {
            st->refine_steps = 1;
            st->true_rel_residual = worst;
        }
        return all_conv ? LS_OK : LS_ENOCONV;
    }
    // LS_MIXED: FP64 iterative refinement around the FP32 outer iteration. dref holds
    // the FP64 residuals; outer32.w their FP32 roundings (the correction's right-hand
    // sides) and inner32.w the FP32 corrections. Flexible GMRES itself never touches
    // the w blocks of the space it runs in.
    double2* d = c->dref;
    float2* d32 = c->outer32.w;
    float2* corr = c->inner32.w;
    if (!use_x0)
        for (int i = 0; i < nb; ++i)
            if (live[i]) LS_TRY(ls_vec_zero(h, u + i * N));
    std::vector<unsigned char> act(live);
    std::vector<int> steps(nb, 0);
    std::vector<double> nr(nb, 0.0);
    for (;;) {
        bool any = false;
        std::vector<int> cur;
        for (int i = 0; i < nb; ++i) {
            if (!act[i]) continue;
            cur.push_back(i);
            double2* di = d + i * N;
            if (steps[i] == 0 && !use_x0) {  // u = 0: the residual is f itself
                LS_TRY(ls_vec_copy(h, f + i * N, di));
            } else {
                LS_TRY(ls_timing_begin(h));
                // d = H u: FP64-accurate (double-float arithmetic by default, else FP64)
                LS_TRY(h->dfloat ? ls_apply_df(h, u + i * N, di) : ls_apply64(h, u + i * N, di));
                LS_TRY(ls_timing_end(h, 2));
                LS_TRY(ls_vec_axpby(h, make_double2(1, 0), f + i * N, make_double2(-1, 0), di));  // d = f - H u
            }
        }
        LS_TRY(ls_vec_norms_b(h, (const double2*)d, N, cur.data(), (int)cur.size(), nr.data()));
        for (int i : cur) {
            relres[i] = nr[i] / nf[i];
            if (!std::isfinite(relres[i])) return LS_ENAN;
            if (relres[i] <= tol || steps[i] >= h->opts.refine_maxit) {
                act[i] = 0;
                continue;
            }
            any = true;
            // ask the FP32 correction for what is still missing, never below what FP32 can deliver
            double s = 0.3 * tol / relres[i];
            if (s < h->opts.refine_inner_tol) s = h->opts.refine_inner_tol;
            if (s > 0.5) s = 0.5;
            stol[i] = s;
        }
        if (!any) break;
        for (int i = 0; i < nb; ++i)
            if (act[i]) LS_TRY(ls_vec_copy(h, (const double2*)(d + i * N), d32 + i * N));
        LS_TRY(fgmres_b(h, c, c->outer32, OP_HMIX, PC_LS, (const float2*)d32, corr, false, stol.data(),
                        h->opts.outer_maxit, nb, act.data(), r.data(), st));
        for (int i = 0; i < nb; ++i) {
            if (!act[i]) continue;
            if (st) st->outer_iters += r[i].iters;
            LS_TRY(ls_vec_axpby(h, make_double2(1, 0), (const float2*)(corr + i * N), make_double2(1, 0),
                                u + i * N));  // u += corr
            ++steps[i];
        }
    }
    int smax = 0;
    for (int i = 0; i < nb; ++i) {
        if (!live[i]) continue;
        worst = std::max(worst, relres[i]);
        all_conv = all_conv && relres[i] <= tol;
        smax = std::max(smax, steps[i]);
    }
    if (st) {
        st->refine_steps = smax;
        st->true_rel_residual = worst;
    }
    return all_conv ? LS_OK : LS_ENOCONV;
}

int ls_outer_solve(ls_handle* h, const double2* f, double tol, double2* u, int use_x0, ls_stats* st) {
    return ls_outer_solve_b(h, 1, f, tol, u, use_x0, st);
}
