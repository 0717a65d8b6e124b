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
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "ls_internal.cuh"

int ls_vec_dots_dev(ls_handle* h, int nvec, const double2* V, size_t ld, const double2* w, double2* out_dev);
int ls_timing_begin(ls_handle* h);
int ls_timing_end(ls_handle* h, int kind);

namespace {

using cd = std::complex<double>;

enum Op { OP_H64, OP_HMIX, OP_C };
enum Pc { PC_NONE, PC_BD, PC_LS };

struct KrylovSpace {
    double2* V = nullptr;   // (m+1) vectors
    double2* Z = nullptr;   // m vectors
    double2* w = nullptr;   // work vectors
    double2* r = nullptr;
    double2* hdev = nullptr;  // 2 * (m+1) + 1 coefficients on the device
    int m = 0;
};

struct Ctx {
    ls_handle* h;
    KrylovSpace outer, inner;
    double2* tmpA = nullptr;  // A r for Algorithm 3
    bool ready = false;
};

Ctx* ctx_of(ls_handle* h);

int alloc_space(ls_handle* h, KrylovSpace& S, int m) {
    const size_t N = (size_t)h->n * h->n;
    S.m = m;
    LS_CUDA(cudaMalloc(&S.V, sizeof(double2) * N * (m + 1)));
    LS_CUDA(cudaMalloc(&S.Z, sizeof(double2) * N * m));
    LS_CUDA(cudaMalloc(&S.w, sizeof(double2) * N));
    LS_CUDA(cudaMalloc(&S.r, sizeof(double2) * N));
    LS_CUDA(cudaMalloc(&S.hdev, sizeof(double2) * (2 * (m + 1) + 2)));
    return LS_OK;
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
            LS_TRY(ls_apply_mixed(h, x, y));
            return ls_timing_end(h, 0);
        }
        default: return ls_stencil_apply(h, 0, 1, x, nullptr, y);
    }
}

struct Result {
    int iters = 0;
    double relres = 0;
    bool converged = false;
};

int fgmres(ls_handle* h, KrylovSpace& S, Op op, Pc pc, const double2* b, double2* x, bool x0, double tol,
           int maxit, Result& res, ls_stats* st);

int apply_pc(ls_handle* h, Pc pc, const double2* v, double2* z, ls_stats* st) {
    if (pc == PC_NONE) return ls_vec_copy(h, v, z);
    if (pc == PC_BD) {
        LS_TRY(ls_timing_begin(h));
        LS_TRY(ls_bd(h, v, z));
        return ls_timing_end(h, 1);
    }
    // Algorithm 3: z = GMRES(C, A v, Algorithm 2, inner_tol)
    Ctx* c = ctx_of(h);
    LS_TRY(ls_stencil_apply(h, 0, 0, v, nullptr, c->tmpA));
    Result r;
    LS_TRY(fgmres(h, c->inner, OP_C, PC_BD, c->tmpA, z, false, h->opts.inner_tol, h->opts.inner_maxit, r, nullptr));
    if (st) {
        st->inner_iters_total += r.iters;
        st->inner_calls += 1;
    }
    return LS_OK;
}

int fgmres(ls_handle* h, KrylovSpace& S, Op op, Pc pc, const double2* b, double2* x, bool x0, double tol,
           int maxit, Result& res, ls_stats* st) {
    const size_t N = (size_t)h->n * h->n;
    const int m = S.m;
    double nb;
    LS_TRY(ls_vec_norm(h, b, &nb));
    if (!std::isfinite(nb)) return LS_ENAN;
    res = Result{};
    if (nb == 0.0) {
        LS_TRY(ls_vec_zero(h, x));
        res.converged = true;
        return LS_OK;
    }
    if (x0) {
        LS_TRY(apply_op(h, op, x, S.r));
        LS_TRY(ls_vec_axpby(h, make_double2(1, 0), b, make_double2(-1, 0), S.r));  // r = b - A x
    } else {
        LS_TRY(ls_vec_zero(h, x));
        LS_TRY(ls_vec_copy(h, b, S.r));
    }
    double beta;
    LS_TRY(ls_vec_norm(h, S.r, &beta));
    double relres = beta / nb;
    std::vector<cd> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
    std::vector<double2> hh(2 * (m + 1) + 2);
    int total = 0;
    while (relres > tol && total < maxit) {
        if (!std::isfinite(relres)) return LS_ENAN;
        LS_TRY(ls_vec_axpby(h, make_double2(1.0 / beta, 0), S.r, make_double2(0, 0), S.V));  // V0 = r / beta
        std::fill(gv.begin(), gv.end(), cd(0));
        std::fill(H.begin(), H.end(), cd(0));
        gv[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double2* vj = S.V + (size_t)j * N;
            double2* zj = S.Z + (size_t)j * N;
            double2* vn = S.V + (size_t)(j + 1) * N;
            LS_TRY(apply_pc(h, pc, vj, zj, st));
            LS_TRY(apply_op(h, op, zj, vn));
            // CGS2 against V_0..V_j; coefficients stay on the device between the passes
            LS_TRY(ls_vec_dots_dev(h, j + 1, S.V, N, vn, S.hdev));
            LS_TRY(ls_vec_update(h, j + 1, S.V, N, S.hdev, vn));
            LS_TRY(ls_vec_dots_dev(h, j + 1, S.V, N, vn, S.hdev + (m + 1)));
            LS_TRY(ls_vec_update(h, j + 1, S.V, N, S.hdev + (m + 1), vn));
            LS_TRY(ls_vec_dots_dev(h, 1, vn, 0, vn, S.hdev + 2 * (m + 1)));
            LS_CUDA(cudaMemcpyAsync(hh.data(), S.hdev, sizeof(double2) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost,
                                    h->stream));
            LS_CUDA(cudaStreamSynchronize(h->stream));
            for (int i = 0; i <= j; ++i)
                H[(size_t)i * m + j] = cd(hh[i].x + hh[m + 1 + i].x, hh[i].y + hh[m + 1 + i].y);
            const double hn = std::sqrt(std::max(hh[2 * (m + 1)].x, 0.0));
            if (!std::isfinite(hn)) return LS_ENAN;
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {  // previous rotations
                const cd t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
                H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = t;
            }
            const cd a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
            const double den = std::sqrt(std::norm(a) + std::norm(c));
            if (den == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else if (std::abs(a) == 0.0) {
                cs[j] = 0.0;
                sn[j] = 1.0;
            } else {
                cs[j] = std::abs(a) / den;
                sn[j] = (a / std::abs(a)) * std::conj(c) / den;
            }
            H[(size_t)j * m + j] = cs[j] * a + sn[j] * c;
            H[(size_t)(j + 1) * m + j] = 0.0;
            gv[j + 1] = -std::conj(sn[j]) * gv[j];
            gv[j] = cs[j] * gv[j];
            ++total;
            k = j + 1;
            relres = std::abs(gv[j + 1]) / nb;
            if (relres <= tol || total >= maxit || hn == 0.0) break;
            LS_TRY(ls_vec_axpby(h, make_double2(1.0 / hn, 0), vn, make_double2(0, 0), vn));
        }
        for (int i = k - 1; i >= 0; --i) {
            cd s = gv[i];
            for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
            y[i] = s / H[(size_t)i * m + i];
        }
        std::vector<double2> yc(k);
        for (int i = 0; i < k; ++i) yc[i] = make_double2(y[i].real(), y[i].imag());
        LS_TRY(ls_vec_combine(h, k, S.Z, N, yc.data(), x));
        // true residual
        LS_TRY(apply_op(h, op, x, S.r));
        LS_TRY(ls_vec_axpby(h, make_double2(1, 0), b, make_double2(-1, 0), S.r));
        LS_TRY(ls_vec_norm(h, S.r, &beta));
        relres = beta / nb;
        if (!std::isfinite(relres)) return LS_ENAN;
    }
    res.iters = total;
    res.relres = relres;
    res.converged = relres <= tol;
    return LS_OK;
}

}  // namespace

// per-handle Krylov context
namespace {
struct CtxStore {
    ls_handle* h;
    Ctx* c;
};
std::vector<CtxStore>& ctx_list() {
    static std::vector<CtxStore> v;
    return v;
}
Ctx* ctx_of(ls_handle* h) {
    for (auto& e : ctx_list())
        if (e.h == h) return e.c;
    return nullptr;
}
int ctx_ensure(ls_handle* h) {
    Ctx* c = ctx_of(h);
    if (c && c->ready) return LS_OK;
    if (!c) {
        c = new Ctx();
        c->h = h;
        ctx_list().push_back({h, c});
    }
    const size_t N = (size_t)h->n * h->n;
    LS_TRY(alloc_space(h, c->outer, h->opts.outer_restart));
    LS_TRY(alloc_space(h, c->inner, h->opts.inner_restart));
    LS_CUDA(cudaMalloc(&c->tmpA, sizeof(double2) * N));
    c->ready = true;
    return LS_OK;
}
void free_space(KrylovSpace& S) {
    cudaFree(S.V);
    cudaFree(S.Z);
    cudaFree(S.w);
    cudaFree(S.r);
    cudaFree(S.hdev);
    S = KrylovSpace{};
}
}  // namespace

void ls_krylov_free(ls_handle* h) {
    auto& L = ctx_list();
    for (size_t i = 0; i < L.size(); ++i)
        if (L[i].h == h) {
            free_space(L[i].c->outer);
            free_space(L[i].c->inner);
            cudaFree(L[i].c->tmpA);
            delete L[i].c;
            L.erase(L.begin() + i);
            return;
        }
}

int ls_inner_gmres(ls_handle* h, const double2* g, double tol, double2* v, int* iters) {
    LS_TRY(ctx_ensure(h));
    Ctx* c = ctx_of(h);
    Result r;
    LS_TRY(fgmres(h, c->inner, OP_C, PC_BD, g, v, false, tol, h->opts.inner_maxit, r, nullptr));
    if (iters) *iters = r.iters;
    return r.converged ? LS_OK : LS_ENOCONV;
}

int ls_outer_solve(ls_handle* h, const double2* f, double tol, double2* u, int use_x0, ls_stats* st) {
    LS_TRY(ctx_ensure(h));
    Ctx* c = ctx_of(h);
    double nf;
    LS_TRY(ls_vec_norm(h, f, &nf));
    if (!std::isfinite(nf)) return LS_ENAN;
    if (nf == 0.0) {
        LS_TRY(ls_vec_zero(h, u));
        if (st) st->true_rel_residual = 0.0;
        return LS_OK;
    }
    if (h->prec == LS_FP64) {
        Result r;
        LS_TRY(fgmres(h, c->outer, OP_H64, PC_LS, f, u, use_x0 != 0, tol, h->opts.outer_maxit, r, st));
        if (st) {
            st->outer_iters += r.iters;
            st->refine_steps = 1;
            st->true_rel_residual = r.relres;
        }
        return r.converged ? LS_OK : LS_ENOCONV;
    }
    // LS_MIXED: FP64 iterative refinement around the FP32-apply outer iteration.
    // Buffers: outer.w holds the refinement right-hand side and inner.w the
    // correction; flexible GMRES itself never touches either.
    double2* d = c->outer.w;
    double2* corr = c->inner.w;
    if (!use_x0) LS_TRY(ls_vec_zero(h, u));
    double relres = 1.0;
    int steps = 0;
    for (;;) {
        LS_TRY(ls_timing_begin(h));
        LS_TRY(ls_apply64(h, u, d));  // d = H u (FP64)
        LS_TRY(ls_timing_end(h, 2));
        LS_TRY(ls_vec_axpby(h, make_double2(1, 0), f, make_double2(-1, 0), d));  // d = f - H u
        double nr;
        LS_TRY(ls_vec_norm(h, d, &nr));
        relres = nr / nf;
        if (!std::isfinite(relres)) return LS_ENAN;
        if (relres <= tol || steps >= h->opts.refine_maxit) break;
        // ask the FP32 correction for what is still missing, never below what FP32 can deliver
        double stol = 0.3 * tol / relres;
        if (stol < h->opts.refine_inner_tol) stol = h->opts.refine_inner_tol;
        if (stol > 0.5) stol = 0.5;
        Result r;
        LS_TRY(fgmres(h, c->outer, OP_HMIX, PC_LS, d, corr, false, stol, h->opts.outer_maxit, r, st));
        if (st) st->outer_iters += r.iters;
        LS_TRY(ls_vec_axpby(h, make_double2(1, 0), corr, make_double2(1, 0), u));  // u += correction
        ++steps;
    }
    if (st) {
        st->refine_steps = steps;
        st->true_rel_residual = relres;
    }
    return relres <= tol ? LS_OK : LS_ENOCONV;
}
