// ls_tune.cu -- a small autotuner for the two shape choices of the on-line path.
//
//  * FFT tile shape of the FP32 / mixed LS-apply: radix-16 transforms with
//    1-column tiles (3 or 2 CTAs per SM) or 2-column tiles (ls_fft16.cu), or
//    radix-8 transforms on 4-column tiles (generic path of ls_fft.cu);
//  * band-block batching of Algorithm 2: how many right-hand sides share one
//    pass over the local-solve factors (1, 2, 4 or 8; FP64 up to 4).
// Each candidate runs once to warm up and is then timed with CUDA events on the
// handle's stream over `reps` calls; the fastest is kept in the handle and used
// by every later apply and batched solve.  The inputs are incident-wave
// right-hand sides of the handle's own problem, so the timings see the real
// sizes and value ranges.
#include "ls_internal.cuh"

namespace {

int time_ms(ls_handle* h, int reps, float* ms, int (*fn)(ls_handle*, void*), void* arg) {
    LS_TRY(fn(h, arg));  // warm-up (also captures graphs, allocates buffers)
    LS_CUDA(cudaEventRecord(h->ev0, h->stream));
    for (int r = 0; r < reps; ++r) LS_TRY(fn(h, arg));
    LS_CUDA(cudaEventRecord(h->ev1, h->stream));
    LS_CUDA(cudaEventSynchronize(h->ev1));
    LS_CUDA(cudaEventElapsedTime(ms, h->ev0, h->ev1));
    *ms /= reps;
    return LS_OK;
}

struct ApplyArg {
    double2* x;
    double2* y;
};
int run_apply(ls_handle* h, void* a) {
    auto* p = static_cast<ApplyArg*>(a);
    return ls_apply_mx(h, p->x, p->y);
}

struct BdArg {
    double2* g;
    double2* v;
    int nrhs, chunk;
};
int run_bd(ls_handle* h, void* a) {  // as the batched solve runs it: chunks on concurrent lanes
    auto* p = static_cast<BdArg*>(a);
    return ls_bd_lanes(h, p->g, p->v, p->nrhs, p->chunk);
}

}  // namespace

extern "C" int ls_autotune(ls_handle* h, int nrhs, int reps, ls_tuning* out) {
    if (!h || nrhs < 1 || nrhs > LS_MAX_BATCH || reps < 1) return LS_EINVAL;
    ls_tuning t{};
    const size_t N = (size_t)h->n * h->n;
    double2* buf = nullptr;
    LS_CUDA(cudaMalloc(&buf, sizeof(double2) * N * 2 * nrhs));
    int rc = LS_OK;
    do {
        for (int b = 0; b < nrhs && rc == LS_OK; ++b) rc = ls_rhs(h, 0.7 + 0.9 * b, buf + b * N);
        if (rc != LS_OK) break;
        // FFT tile shape (the variant the solve's FP32 / mixed apply uses)
        ApplyArg aa{buf, buf + nrhs * N};
        float best = 0;
        int pick = 0;
        for (int v = 0; v < ls_handle::kFftVariants && rc == LS_OK; ++v) {
            if (v != 1 && !ls_fft16_supported(h)) {
                t.fft_ms[v] = -1;
                continue;
            }
            h->fft_variant = v;
            float ms = 0;
            rc = time_ms(h, reps, &ms, run_apply, &aa);
            t.fft_ms[v] = ms;
            if (rc == LS_OK && (best == 0 || ms < best)) {
                best = ms;
                pick = v;
            }
        }
        if (rc != LS_OK) break;
        h->fft_variant = pick;
        t.fft_variant = pick;
        // band-block batching of Algorithm 2 for nrhs right-hand sides (needs the factors):
        // reduction steps on the CUDA cores (chunks 1, 2, 4, 8, blocks of small levels split
        // over several CTAs or not) and, when built, on the tensor cores (chunks 1, 8, 16, 32)
        if (!h->factored) break;
        best = 0;
        int chunk = 1, split = 1, tc = 0;
        const int tc_avail = h->tc_ready && h->cr_tc ? 1 : 0;   // switched off by ls_set_tensor_steps: not tried
        const int tc_user = h->cr_tc;
        for (int form = tc_avail ? 2 : 1; form >= 0 && rc == LS_OK; --form) {  // 2: tensor cores, 1: split, 0: unsplit
            const int want_tc = form == 2, sp = form == 2 ? h->cr_split : form;
            if (h->cr_split != sp || h->cr_tc != 2 * want_tc) {
                h->cr_split = sp;
                h->cr_tc = 2 * want_tc;   // measured in the pure forms
                ls_bd_graph_free(h);  // the captured launches bake the grid shapes in
            }
            const int cap = ls_bd_cap(h);
            const int tc_chunks[4] = {1, 8, 16, 32};
            for (int k = 0; k < 4 && rc == LS_OK; ++k) {
                const int c = want_tc ? tc_chunks[k] : (1 << k);
                if (c > cap || (c > nrhs && c > 1)) break;
                BdArg ba{buf, buf + nrhs * N, nrhs, c};
                float ms = 0;
                rc = time_ms(h, reps, &ms, run_bd, &ba);
                (want_tc ? t.bd_ms_tc : (sp ? t.bd_ms : t.bd_ms_nosplit))[k] = ms / nrhs;
                if (rc == LS_OK && (best == 0 || ms < best)) {
                    best = ms;
                    chunk = c;
                    split = sp;
                    tc = want_tc;
                }
            }
        }
        if (rc != LS_OK) {
            h->cr_tc = tc_user;
            break;
        }
        if (h->cr_split != split || h->cr_tc != 2 * tc) {
            h->cr_split = split;
            h->cr_tc = 2 * tc;
            ls_bd_graph_free(h);
        }
        h->bd_chunk = chunk;
        t.bd_chunk = chunk;
        t.cr_split = split;
        t.tensor_steps = tc;
    } while (0);
    cudaStreamSynchronize(h->stream);
    cudaFree(buf);
    if (rc == LS_OK && out) *out = t;
    return rc;
}

extern "C" int ls_set_shapes(ls_handle* h, int fft_variant, int bd_chunk) {
    if (!h || fft_variant < 0 || fft_variant >= ls_handle::kFftVariants) return LS_EINVAL;
    const int cap = ls_bd_cap(h);
    if (bd_chunk < 0 || bd_chunk > cap) return LS_EINVAL;
    h->fft_variant = fft_variant;
    h->bd_chunk = bd_chunk;
    return LS_OK;
}

extern "C" int ls_set_reduction(ls_handle* h, int cr_split) {
    if (!h || (cr_split != 0 && cr_split != 1)) return LS_EINVAL;
    if (h->cr_split != cr_split) {
        LS_CUDA(cudaStreamSynchronize(h->stream));
        h->cr_split = cr_split;
        ls_bd_graph_free(h);
    }
    return LS_OK;
}

extern "C" int ls_set_tensor_steps(ls_handle* h, int on) {
    if (!h || on < 0 || on > 2) return LS_EINVAL;
    if (on && !h->tc_ready) return LS_ESTATE;
    if (h->cr_tc != on) {
        LS_CUDA(cudaStreamSynchronize(h->stream));
        h->cr_tc = on;
        if (h->bd_chunk > ls_bd_cap(h)) h->bd_chunk = 0;
        ls_bd_graph_free(h);
    }
    return LS_OK;
}

extern "C" int ls_set_pack_members(ls_handle* h, int on) {
    if (!h || on < 0 || on > 1) return LS_EINVAL;
    h->pack_members = on;
    return LS_OK;
}

extern "C" int ls_set_double_float(ls_handle* h, int on) {
    if (!h || on < 0 || on > 1) return LS_EINVAL;
    h->dfloat = on;
    return LS_OK;
}

extern "C" int ls_set_reduced_inverse(ls_handle* h, int on) {
    if (!h || on < 0 || on > 1) return LS_EINVAL;
    if (h->tc_dense != on) {
        LS_CUDA(cudaStreamSynchronize(h->stream));
        h->tc_dense = on;
        ls_bd_graph_free(h);
    }
    return LS_OK;
}
