// ls_api.cu -- the C ABI declared in include/ls.h: handle lifetime, argument
// checks, status codes, timing and the host-buffer entry point.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "ls_internal.cuh"

int ls_transpose_real(ls_handle* h, const double* a, double* b);
void ls_krylov_free(ls_handle* h);

namespace {

thread_local char g_last_cuda[256] = "";

__global__ void k_real_to32(size_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

struct HostBufs {
    ls_handle* h = nullptr;
    double2* f = nullptr;  // device staging for host right-hand sides / plane-wave sources
    double2* u = nullptr;  // device staging for host solutions
    int cap = 0;           // fields each buffer holds
};
HostBufs* host_bufs(ls_handle* h, bool create) {
    if (!h->hostbufs && create) {
        HostBufs* b = new HostBufs();
        b->h = h;
        h->hostbufs = b;
    }
    return static_cast<HostBufs*>(h->hostbufs);
}

// Staging buffers for nb fields (grown on demand).
int host_reserve(ls_handle* h, int nb, HostBufs** out) {
    HostBufs* b = host_bufs(h, true);
    if (!b) return LS_ENOMEM;
    if (b->cap < nb) {
        cudaFree(b->f);
        cudaFree(b->u);
        b->f = b->u = nullptr;
        b->cap = 0;
        const size_t bytes = sizeof(double2) * (size_t)h->n * h->n * nb;
        LS_CUDA(cudaMalloc(&b->f, bytes));
        LS_CUDA(cudaMalloc(&b->u, bytes));
        b->cap = nb;
    }
    *out = b;
    return LS_OK;
}

void release(ls_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    ls_krylov_free(h);
    ls_factor_free(h);
    ls_lanes_free(h);
    if (HostBufs* b = host_bufs(h, false)) {
        cudaFree(b->f);
        cudaFree(b->u);
        delete b;
        h->hostbufs = nullptr;
    }
    void* ptrs[] = {h->m64, h->m32, h->mT64, h->ghat64, h->ghat32, h->tw64, h->tw32, h->fftws, h->incx,
                    h->incz, h->dtabs, h->red, h->mdf, h->ghatdf, h->twdf, h->incxdf, h->inczdf};
    for (void* p : ptrs) cudaFree(p);
    if (h->red_host) cudaFreeHost(h->red_host);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    delete h;
}

int next_pow2_log(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

int ls_cuda_fail(cudaError_t e) {
    std::snprintf(g_last_cuda, sizeof(g_last_cuda), "%s", cudaGetErrorString(e));
    cudaGetLastError();  // clear a non-sticky error
    return LS_ECUDA;
}

// Timed intervals are pairs of events recorded on the handle's stream; nothing
// waits on them until ls_timing_collect, so timing adds no host synchronisation.
int ls_timing_begin(ls_handle* h) {
    if (!h->timing) return LS_OK;
    if (2 * h->tused + 2 > h->tev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            LS_CUDA(cudaEventCreate(&e));
            h->tev.push_back(e);
        }
        h->tkind.resize(h->tev.size() / 2);
    }
    LS_CUDA(cudaEventRecord(h->tev[2 * h->tused], h->stream));
    return LS_OK;
}

int ls_timing_end(ls_handle* h, int kind) {
    if (!h->timing) return LS_OK;
    LS_CUDA(cudaEventRecord(h->tev[2 * h->tused + 1], h->stream));
    h->tkind[h->tused] = kind;
    h->tused++;
    return LS_OK;
}

// Wait for the recorded intervals and add them to the per-kind totals.
int ls_timing_collect(ls_handle* h) {
    if (h->tused) LS_CUDA(cudaEventSynchronize(h->tev[2 * h->tused - 1]));
    for (size_t k = 0; k < h->tused; ++k) {
        float ms = 0;
        LS_CUDA(cudaEventElapsedTime(&ms, h->tev[2 * k], h->tev[2 * k + 1]));
        if (h->tkind[k] == 0) {
            h->t_apply_ms += ms;
            h->n_apply++;
        } else if (h->tkind[k] == 2) {
            h->t_apply64_ms += ms;
            h->n_apply64++;
        } else if (h->tkind[k] == 3) {
            h->t_stencil_ms += ms;
            h->n_stencil++;
        } else if (h->tkind[k] == 4) {
            h->t_orth_ms += ms;
            h->n_orth++;
        } else {
            h->t_sweep_ms += ms;
            h->n_sweep++;
        }
    }
    h->tused = 0;
    return LS_OK;
}

extern "C" {

void ls_default_opts(ls_opts* o) {
    if (!o) return;
    o->inner_tol = 1e-3;
    o->inner_restart = 30;
    o->inner_maxit = 200;
    o->outer_restart = 40;
    o->outer_maxit = 200;
    o->shift = 10.0;
    o->refine_maxit = 6;
    o->refine_inner_tol = 1e-4;
    o->use_graphs = 1;
    o->inner_precond = LS_PC_BD;
}

const char* ls_strerror(int code) {
    switch (code) {
        case LS_OK: return "ok";
        case LS_EINVAL: return "invalid argument (size, option or null pointer)";
        case LS_ENOMEM: return "out of memory";
        case LS_ECUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
        case LS_ESINGULAR: return "zero pivot in a local factorisation";
        case LS_ENOCONV: return "iteration limit reached before the tolerance";
        case LS_ENAN: return "NaN or Inf in an input or a residual";
        case LS_ETIMEOUT: return "a bounded device wait ran out";
        case LS_ESTATE: return "call out of order (ls_factor required first)";
        case LS_ETOOBIG: return "size exceeds the fixed scratch of ls_apply_f32_noalloc (n <= 1024)";
        default: return "unknown status";
    }
}

int ls_setup(const ls_grid* grid, double hstep, double omega, const double* m, const ls_opts* opts, void* stream,
             ls_handle** out) {
    if (!out) return LS_EINVAL;
    *out = nullptr;
    if (!grid || !m) return LS_EINVAL;
    const int n = grid->nx;
    if (grid->nx != grid->nz || n < 8 || grid->layers < 1 || grid->nz % grid->layers != 0 || grid->ext < 1)
        return LS_EINVAL;
    if (grid->precision != LS_FP64 && grid->precision != LS_MIXED) return LS_EINVAL;
    if (!(hstep > 0) || !(omega > 0)) return LS_EINVAL;
    const int lp = next_pow2_log(2 * n - 1);
    if (lp > 12) return LS_EINVAL;  // FFT kernels are sized for P <= 4096 (n <= 2048)
    const int t = n / grid->layers, q = t + 2 * grid->ext;
    if (q > 112) return LS_EINVAL;  // local blocks are inverted in shared memory
    ls_handle* h = new (std::nothrow) ls_handle();
    if (!h) return LS_ENOMEM;
    h->n = n;
    h->L = grid->layers;
    h->E = grid->ext;
    h->t = t;
    h->q = q;
    h->lp = lp;
    h->P = 1 << lp;
    h->prec = grid->precision;
    h->dfloat = grid->precision == LS_MIXED ? 1 : 0;
    h->h = hstep;
    h->omega = omega;
    ls_default_opts(&h->opts);
    if (opts) h->opts = *opts;
    if (h->opts.outer_restart < 1 || h->opts.outer_restart > 63 || h->opts.inner_restart < 1 ||
        h->opts.inner_restart > 63 || (h->opts.inner_precond != LS_PC_BD && h->opts.inner_precond != LS_PC_GS)) {
        delete h;
        return LS_EINVAL;
    }
    h->stream = static_cast<cudaStream_t>(stream);
    int rc = LS_OK;
    do {
        if (cudaGetDevice(&h->device) != cudaSuccess) { rc = LS_ECUDA; break; }
        const size_t N = (size_t)n * n;
        if (cudaMalloc(&h->m64, sizeof(double) * N) != cudaSuccess ||
            cudaMalloc(&h->m32, sizeof(float) * N) != cudaSuccess ||
            cudaMalloc(&h->mT64, sizeof(double) * N) != cudaSuccess) {
            rc = LS_ENOMEM;
            break;
        }
        if (cudaMemcpyAsync(h->m64, m, sizeof(double) * N, cudaMemcpyDefault, h->stream) != cudaSuccess) {
            rc = LS_ECUDA;
            break;
        }
        k_real_to32<<<608, 256, 0, h->stream>>>(N, h->m64, h->m32);
        h->launches++;
        if ((rc = ls_transpose_real(h, h->m64, h->mT64)) != LS_OK) break;
        if ((rc = ls_fft_init(h)) != LS_OK) break;
        double2* gtab = nullptr;
        if ((rc = ls_green_table(h, &gtab)) != LS_OK) break;
        rc = ls_spectrum_build(h, gtab);
        if (rc == LS_OK) rc = ls_stencils_build(h, gtab);
        cudaFree(gtab);
        if (rc != LS_OK) break;
        if ((rc = ls_sweep_alloc(h)) != LS_OK) break;
        if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
            rc = LS_ECUDA;
            break;
        }
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) { rc = LS_ECUDA; break; }
    } while (0);
    if (rc != LS_OK) {
        release(h);
        return rc;
    }
    *out = h;
    return LS_OK;
}

int ls_factor(ls_handle* h) {
    if (!h) return LS_EINVAL;
    ls_factor_free(h);
    h->factored = false;
    int rc = ls_factor_all(h);
    if (rc == LS_OK) rc = ls_cr_tc_prepare(h);   // LS_MIXED: TF32 planes for the tensor-core steps
    if (rc != LS_OK) {
        ls_factor_free(h);
        return rc;
    }
    h->factored = true;
    return LS_OK;
}

int ls_apply(ls_handle* h, const ls_c64* u, ls_c64* y) {
    if (!h || !u || !y) return LS_EINVAL;
    return ls_apply64(h, reinterpret_cast<const double2*>(u), reinterpret_cast<double2*>(y));
}

int ls_axpby(ls_handle* h, double a_re, double a_im, const ls_c64* x, double b_re, double b_im, ls_c64* y) {
    if (!h || !x || !y) return LS_EINVAL;
    return ls_vec_axpby(h, make_double2(a_re, a_im), reinterpret_cast<const double2*>(x), make_double2(b_re, b_im),
                        reinterpret_cast<double2*>(y));
}

int ls_apply_f32(ls_handle* h, const ls_c32* u, ls_c32* y) {
    if (!h || !u || !y) return LS_EINVAL;
    return ls_apply32(h, reinterpret_cast<const float2*>(u), reinterpret_cast<float2*>(y));
}

int ls_apply_mixed(ls_handle* h, const ls_c64* u, ls_c64* y) {
    if (!h || !u || !y) return LS_EINVAL;
    return ls_apply_mx(h, reinterpret_cast<const double2*>(u), reinterpret_cast<double2*>(y));
}

int ls_incident_rhs(ls_handle* h, double theta, ls_c64* f) {
    if (!h || !f || !std::isfinite(theta)) return LS_EINVAL;
    return ls_rhs(h, theta, reinterpret_cast<double2*>(f));
}

int ls_host_alloc(size_t bytes, void** out) {
    if (!out) return LS_EINVAL;
    *out = nullptr;
    if (bytes == 0) return LS_EINVAL;
    if (cudaHostAlloc(out, bytes, cudaHostAllocPortable) != cudaSuccess) {
        *out = nullptr;
        cudaGetLastError();   // the failure is reported by the return code
        return LS_ENOMEM;
    }
    return LS_OK;
}

int ls_host_free(void* p) {
    if (!p) return LS_OK;
    return cudaFreeHost(p) == cudaSuccess ? LS_OK : LS_ECUDA;
}

int ls_get_sweep_histogram(ls_handle* h, int* counts, int len) {
    if (!h || !counts || len < 1) return LS_EINVAL;
    for (int k = 0; k < len; ++k) counts[k] = k <= LS_MAX_BATCH ? h->sweep_hist[k] : 0;
    return LS_OK;
}

int ls_apply_double_float(ls_handle* h, const ls_c64* u, ls_c64* y) {
    if (!h || !u || !y) return LS_EINVAL;
    return ls_apply_df(h, reinterpret_cast<const double2*>(u), reinterpret_cast<double2*>(y));
}

int ls_solve_batch(ls_handle* h, int nrhs, const ls_c64* f, double tol, ls_c64* u, int use_x0, ls_stats* st) {
    if (!h || !f || !u || !(tol > 0) || nrhs < 1 || nrhs > LS_MAX_BATCH) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    ls_stats local{};
    ls_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    h->t_apply_ms = h->t_sweep_ms = h->t_apply64_ms = h->t_stencil_ms = h->t_orth_ms = 0;
    h->n_apply = h->n_sweep = h->n_apply64 = h->n_stencil = h->n_orth = 0;
    h->learned_steps = 0;
    h->sweep_fields = 0;
    std::memset(h->sweep_hist, 0, sizeof(h->sweep_hist));
    const long long l0 = h->launches;
    const auto t0 = std::chrono::steady_clock::now();
    h->tused = 0;
    int rc = ls_outer_solve_b(h, nrhs, reinterpret_cast<const double2*>(f), tol, reinterpret_cast<double2*>(u),
                              use_x0, s);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && rc == LS_OK) rc = ls_cuda_fail(cudaGetLastError());
    const int rct = ls_timing_collect(h);
    if (rc == LS_OK) rc = rct;
    s->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    s->t_apply_ms = h->t_apply_ms;
    s->n_apply = h->n_apply;
    s->t_apply64_ms = h->t_apply64_ms;
    s->n_apply64 = h->n_apply64;
    s->t_sweep_ms = h->t_sweep_ms;
    s->n_sweep = h->n_sweep;
    s->kernel_launches = h->launches - l0;
    s->learned_steps = h->learned_steps;
    s->t_stencil_ms = h->t_stencil_ms;
    s->n_stencil = h->n_stencil;
    s->t_orth_ms = h->t_orth_ms;
    s->n_orth = h->n_orth;
    s->sweep_fields = h->sweep_fields;
    return rc;
}

int ls_set_learned(ls_handle* h, ls_net* net) {
    if (!h) return LS_EINVAL;
    h->net = net;
    return LS_OK;
}

int ls_solve(ls_handle* h, const ls_c64* f, double tol, ls_c64* u, int use_x0, ls_stats* st) {
    return ls_solve_batch(h, 1, f, tol, u, use_x0, st);
}

int ls_solve_plane_wave(ls_handle* h, double theta, double tol, ls_c64* u, ls_stats* st) {
    if (!h || !u) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    HostBufs* b = nullptr;
    LS_TRY(host_reserve(h, 1, &b));
    const long long l0 = h->launches;
    LS_TRY(ls_rhs(h, theta, b->f));
    const long long extra = h->launches - l0;
    const int rc = ls_solve(h, reinterpret_cast<const ls_c64*>(b->f), tol, u, 0, st);
    if (st) st->kernel_launches += extra;
    return rc;
}

int ls_solve_batch_host(ls_handle* h, int nrhs, const ls_c64* f_host, double tol, ls_c64* u_host, ls_stats* st) {
    if (!h || !f_host || !u_host || nrhs < 1 || nrhs > LS_MAX_BATCH) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    HostBufs* b = nullptr;
    LS_TRY(host_reserve(h, nrhs, &b));
    const size_t bytes = sizeof(double2) * (size_t)h->n * h->n * nrhs;
    LS_CUDA(cudaMemcpyAsync(b->f, f_host, bytes, cudaMemcpyHostToDevice, h->stream));
    const int rc = ls_solve_batch(h, nrhs, reinterpret_cast<const ls_c64*>(b->f), tol,
                                  reinterpret_cast<ls_c64*>(b->u), 0, st);
    if (rc != LS_OK && rc != LS_ENOCONV) return rc;
    LS_CUDA(cudaMemcpyAsync(u_host, b->u, bytes, cudaMemcpyDeviceToHost, h->stream));
    LS_CUDA(cudaStreamSynchronize(h->stream));
    return rc;
}

// Independent problems solved concurrently: a pool of host workers takes the
// problems in turn; each solve runs on its own handle's stream, so the GPU
// overlaps the problems' kernels (small grids leave most SMs idle on their own).
int ls_solve_group(int nprob, ls_handle* const* hs, const ls_c64* const* f, double tol, ls_c64* const* u,
                   ls_stats* stats, int* status) {
    if (nprob < 1 || !hs || !f || !u || !(tol > 0)) return LS_EINVAL;
    for (int i = 0; i < nprob; ++i) {
        if (!hs[i] || !f[i] || !u[i]) return LS_EINVAL;
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return LS_EINVAL;  // a handle serves one thread at a time
    }
    for (int i = 0; i < nprob; ++i)
        if (!hs[i]->factored) return LS_ESTATE;
    std::vector<int> rc(nprob, LS_OK);
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nprob) return;
            if (cudaSetDevice(hs[i]->device) != cudaSuccess) {
                rc[i] = LS_ECUDA;
                continue;
            }
            rc[i] = ls_solve(hs[i], f[i], tol, u[i], 0, stats ? &stats[i] : nullptr);
        }
    };
    const int nw = std::min(nprob, (int)LS_GROUP_WORKERS);
    std::vector<std::thread> pool;
    pool.reserve(nw);
    for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    int out = LS_OK;
    for (int i = 0; i < nprob; ++i) {
        if (status) status[i] = rc[i];
        if (out == LS_OK && rc[i] != LS_OK) out = rc[i];
    }
    return out;
}

int ls_solve_host(ls_handle* h, const ls_c64* f_host, double tol, ls_c64* u_host, ls_stats* st) {
    return ls_solve_batch_host(h, 1, f_host, tol, u_host, st);
}

int ls_apply_A(ls_handle* h, const ls_c64* r, ls_c64* y) {
    if (!h || !r || !y) return LS_EINVAL;
    return ls_stencil_apply64(h, 0, 0, reinterpret_cast<const double2*>(r), nullptr, reinterpret_cast<double2*>(y));
}

int ls_apply_C(ls_handle* h, const ls_c64* v, ls_c64* y) {
    if (!h || !v || !y) return LS_EINVAL;
    return ls_stencil_apply64(h, 0, 1, reinterpret_cast<const double2*>(v), nullptr, reinterpret_cast<double2*>(y));
}

int ls_sweep(ls_handle* h, int dir, const ls_c64* g, ls_c64* v) {
    if (!h || !g || !v || (dir != 0 && dir != 1)) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    return ls_sweep_dir(h, dir, reinterpret_cast<const double2*>(g), reinterpret_cast<double2*>(v));
}

int ls_precond_bd(ls_handle* h, const ls_c64* g, ls_c64* v) {
    if (!h || !g || !v) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    return ls_bd(h, reinterpret_cast<const double2*>(g), reinterpret_cast<double2*>(v));
}

int ls_precond_bd_batch(ls_handle* h, int nrhs, const ls_c64* g, ls_c64* v) {
    if (!h || !g || !v || nrhs < 1) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    if (nrhs > ls_bd_cap(h)) return LS_EINVAL;
    return ls_bd_b(h, reinterpret_cast<const double2*>(g), reinterpret_cast<double2*>(v), nrhs);
}

int ls_inner_solve(ls_handle* h, const ls_c64* g, double tol, ls_c64* v, int* iters) {
    if (!h || !g || !v || !(tol > 0)) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    const int rc = ls_inner_gmres(h, reinterpret_cast<const double2*>(g), tol, reinterpret_cast<double2*>(v), iters);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && rc == LS_OK) return ls_cuda_fail(cudaGetLastError());
    return rc;
}

int ls_local_solve(ls_handle* h, int dir, int layer, const ls_c64* b, ls_c64* x) {
    if (!h || !b || !x || (dir != 0 && dir != 1) || layer < 0 || layer >= h->L) return LS_EINVAL;
    if (!h->factored) return LS_ESTATE;
    return ls_strip_solve(h, dir, layer, reinterpret_cast<const double2*>(b), reinterpret_cast<double2*>(x));
}

int ls_get_stencils(ls_handle* h, ls_c64* alpha, ls_c64* beta) {
    if (!h) return LS_EINVAL;
    const double w2 = h->omega * h->omega;
    for (int i = 0; i < 81; ++i) {
        if (alpha) alpha[i] = ls_c64{h->tabs[0].alpha[i].x, h->tabs[0].alpha[i].y};
        if (beta) beta[i] = ls_c64{h->tabs[0].wbeta[i].x / w2, h->tabs[0].wbeta[i].y / w2};
    }
    return LS_OK;
}

int ls_get_spectrum(ls_handle* h, ls_c64* ghat, int* P_out) {
    if (!h) return LS_EINVAL;
    if (P_out) *P_out = h->P;
    if (ghat) {
        const size_t q1 = (size_t)(h->P / 2 + 1);
        LS_CUDA(cudaMemcpyAsync(ghat, h->ghat64, sizeof(double2) * q1 * q1, cudaMemcpyDeviceToDevice, h->stream));
    }
    return LS_OK;
}

int ls_get_diag_weight(ls_handle* h, ls_c64* w0) {
    if (!h || !w0) return LS_EINVAL;
    *w0 = ls_c64{h->w0.x, h->w0.y};
    return LS_OK;
}

int ls_get_layout(ls_handle* h, int* t, int* q) {
    if (!h) return LS_EINVAL;
    if (t) *t = h->t;
    if (q) *q = h->q;
    return LS_OK;
}

int ls_set_timing(ls_handle* h, int on) {
    if (!h) return LS_EINVAL;
    h->timing = on != 0;
    return LS_OK;
}

long long ls_kernel_count(ls_handle* h) { return h ? h->launches : -1; }

void ls_destroy(ls_handle* h) { release(h); }

}  // extern "C"
