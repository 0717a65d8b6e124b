/*
 * ls.h -- C ABI of the GB300 (sm_103a) two-level Lippmann-Schwinger solver.
 *
 * Method: Zepeda-Nunez & Zhao, "Fast alternating bi-directional preconditioner
 * for the 2D high-frequency Lippmann-Schwinger equation".  Sections, equations
 * and algorithms below refer to that paper.
 *
 * Conventions shared by every entry point
 *   - Grid (Sec. 2): nodes x_{i,j} = (h i, h j), 1 <= i <= nx, 1 <= j <= nz.
 *     A field is an array of nz*nx elements, x fastest: element (i, j) sits at
 *     index (j-1)*nx + (i-1) (eq. global_ordering / eq. trace_ordering).
 *   - Complex fields are interleaved (re, im): ls_c64 = two doubles,
 *     ls_c32 = two floats.
 *   - Unless an entry point says otherwise, every field pointer is a DEVICE
 *     pointer on the handle's device; the caller owns it and must keep it
 *     alive until the call's work on the handle's stream has finished.
 *     Calls are stream-ordered on the stream given to ls_setup; the functions
 *     that return iteration counts or residuals synchronise that stream.
 *   - Return value: LS_OK (0) or a negative LS_E* code; ls_strerror() names it.
 *     No entry point aborts the process, and none falls back to the CPU.
 *   - A handle is used by one host thread at a time.
 */
#ifndef LS_H
#define LS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } ls_c64;
typedef struct { float re, im; } ls_c32;

enum {
    LS_OK = 0,
    LS_EINVAL = -1,     /* bad size, option or null pointer                         */
    LS_ENOMEM = -2,     /* device or host allocation failed                         */
    LS_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed              */
    LS_ESINGULAR = -4,  /* zero pivot in a local factorisation                      */
    LS_ENOCONV = -5,    /* iteration limit reached; output holds the best iterate   */
    LS_ENAN = -6,       /* NaN or Inf in an input or a residual                     */
    LS_ETIMEOUT = -7,   /* a bounded device-side wait ran out                       */
    LS_ESTATE = -8,     /* call out of order (e.g. solve before ls_factor)          */
    LS_ETOOBIG = -9     /* size beyond the fixed scratch of ls_apply_f32_noalloc    */
};

enum { LS_FP64 = 0, LS_MIXED = 1 };

/* Right-hand sides per batched call: ls_solve_batch takes up to LS_MAX_BATCH;
 * ls_precond_bd_batch takes up to LS_MAX_BD_BATCH (LS_MIXED with the reduction steps
 * on the tensor cores), 8 (LS_MIXED on the CUDA cores) or 4 (LS_FP64). */
enum { LS_MAX_BATCH = 64, LS_MAX_BD_BATCH = 32 };

typedef struct {
    int nx, nz;       /* grid points per direction (this build requires nx == nz >= 8)      */
    int layers;       /* L, number of layers per direction (Sec. 3.1); must divide nz       */
    int ext;          /* extension rows on each side of a layer (Sec. 5: 10); >= 1          */
    int precision;    /* LS_FP64: all FP64.  LS_MIXED: FP32 FFT convolution and local
                         solves inside FP64 refinement; FP64 factorisation and Arnoldi     */
} ls_grid;

typedef struct {
    double inner_tol;      /* Algorithm 3 inner GMRES tolerance (Sec. 4: 1e-3)             */
    int inner_restart;     /* inner GMRES restart length (default 30)                       */
    int inner_maxit;       /* inner GMRES iteration cap (default 200)                       */
    int outer_restart;     /* outer flexible GMRES restart length (default 40)              */
    int outer_maxit;       /* outer iteration cap (default 200)                             */
    double shift;          /* complex-shift constant c: the cut-off region adds i c w to
                              the w^2-weighted coefficient (Sec. 3.3; default 10)            */
    int refine_maxit;      /* LS_MIXED: refinement steps cap (default 6)                    */
    double refine_inner_tol; /* LS_MIXED: floor of the relative tolerance of each FP32
                                correction solve (default 1e-4: the last correction then
                                over-solves, and at tol 1e-6 the field stays within 1e-6 of
                                the converged one; 1e-6 usually needs one correction only,
                                faster, with the field as close as a 1e-6 residual allows);
                                a correction whose restart cycle does not halve its true
                                residual stops there and the FP64 refinement takes another
                                step                                                        */
    int use_graphs;        /* 1 (default): replay Algorithm 2 as a captured CUDA graph;
                              0: launch its kernels one by one (same arithmetic)            */
    int inner_precond;     /* preconditioner of the inner GMRES: LS_PC_BD (default,
                              Algorithm 2) or LS_PC_GS (Algorithm 1 on horizontal layers
                              only, the one-directional polarized-traces sweep that
                              Table 1 compares against)                                      */
} ls_opts;

enum { LS_PC_BD = 0, LS_PC_GS = 1 };

typedef struct {
    int outer_iters;         /* outer (flexible) GMRES iterations, all refinement steps     */
    int inner_iters_total;   /* inner GMRES iterations summed over all preconditioner calls */
    int inner_calls;         /* Algorithm 3 applications                                     */
    int refine_steps;        /* LS_MIXED refinement steps (1 = no correction needed)         */
    double true_rel_residual;/* ||f - H u|| / ||f|| with an FP64-accurate apply of H (LS_MIXED:
                                the double-float one unless ls_set_double_float(h, 0))     */
    double t_solve_s;        /* wall time of the call                                        */
    double t_apply_ms;       /* device time of FP32-arithmetic LS-applies (LS_MIXED) or of all
                                FP64 LS-applies (LS_FP64), if timing is enabled            */
    int n_apply;             /* LS-applies counted in t_apply_ms                             */
    double t_apply64_ms;     /* LS_MIXED: device time of the refinement-residual applies
                                (double-float or FP64, ls_set_double_float)                */
    int n_apply64;           /* LS-applies counted in t_apply64_ms                           */
    double t_sweep_ms;       /* total device time of Algorithm 2 applications (if timing)   */
    int n_sweep;             /* Algorithm 2 applications counted in t_sweep_ms               */
    long long kernel_launches; /* kernels this library launched during the call            */
    int learned_steps;     /* outer steps that used the attached network (ls_set_learned)   */
    double t_stencil_ms;     /* device time of the 9-point stencil applies A v, C v of the inner
                                solve (Algorithm 3), if timing                              */
    int n_stencil;           /* stencil applies counted in t_stencil_ms                      */
    double t_orth_ms;        /* device time of the Arnoldi orthogonalisations (CGS2 dots and
                                updates, both Krylov levels), if timing                     */
    int n_orth;              /* Arnoldi steps counted in t_orth_ms                           */
    long long sweep_fields;  /* fields the Algorithm 2 applications processed, summed: the
                                members still iterating (ls_set_pack_members), else the
                                batch up to the last one still iterating                    */
} ls_stats;

typedef struct ls_handle ls_handle;

/* Defaults of ls_opts (the paper's values where it gives them). */
void ls_default_opts(ls_opts* opts);

/* ls_setup -- create a handle for the discrete problem of Sec. 2.
 *   grid: sizes and precision (see ls_grid).  h: mesh step; omega: frequency.
 *   m: DEVICE array nz*nx of the contrast m(x_{i,j}) (1/c^2 = 1 + m, Sec. 1);
 *      copied, the caller keeps ownership.
 *   opts: NULL for defaults.  stream: cudaStream_t (NULL = legacy default stream).
 * Allocates the handle's device memory (medium, spectrum, stencil tables,
 * workspaces).  Computes the quadrature weights G_w (Sec. 2), the spectrum of
 * the circulant embedding, and the sparsifying stencils alpha, beta (Sec. 2).
 * Errors: LS_EINVAL (sizes, L not dividing nz, null pointers), LS_ENOMEM, LS_ECUDA.
 * On error *out is NULL and nothing is leaked. */
int ls_setup(const ls_grid* grid, double h, double omega, const double* m,
             const ls_opts* opts, void* stream, ls_handle** out);

/* ls_factor -- off-line stage (Sec. 4.1): assemble the local matrices C^l of
 * the L horizontal and the L vertical layers (Sec. 3.1, 3.3) and factor each
 * by block cyclic reduction in FP64.  LS_ESINGULAR on a zero pivot. */
int ls_factor(ls_handle* h);

/* ls_apply -- y = H u = u + w^2 G (m u) (Sec. 2, eq. discrete_Lipmann-Schwinger),
 * FP64, by the zero-padded FFT convolution.  u, y: device, nz*nx; may alias. */
int ls_apply(ls_handle* h, const ls_c64* u, ls_c64* y);

/* ls_apply_f32 -- the same operator with FP32 complex arithmetic and FP32 I/O. */
int ls_apply_f32(ls_handle* h, const ls_c32* u, ls_c32* y);

/* ls_apply_mixed -- the same operator with FP64 input/output and FP32 complex arithmetic
 * (the apply LS_MIXED uses inside its refinement loop).  u, y: device, nz*nx; may alias. */
int ls_apply_mixed(ls_handle* h, const ls_c64* u, ls_c64* y);

/* ls_apply_double_float -- the same operator with FP64 input/output and double-float
 * arithmetic inside (each real a pair hi + lo of FP32 numbers, about 48 significant bits,
 * on the FP32 pipes; relative error a few 1e-13 against ls_apply).  LS_MIXED solves compute
 * their refinement residuals f - H u this way (ls_set_double_float).  u, y: device, nz*nx;
 * may alias. */
int ls_apply_double_float(ls_handle* h, const ls_c64* u, ls_c64* y);

/* ls_axpby -- y = a x + b y over the nz*nx grid (a = a_re + i a_im, b likewise), on
 * the handle's stream: the residual r = f - H u (ls_apply, then a = 1, b = -1 with
 * y = H u) and corrections e = u* - u of the outer iteration (Sec. 4) without
 * leaving the device.  x, y: device, nz*nx; may alias. */
int ls_axpby(ls_handle* h, double a_re, double a_im, const ls_c64* x, double b_re, double b_im, ls_c64* y);

/* ls_incident_rhs -- f = -w^2 G (m u_I) with u_I = exp(i w (x cos theta + z sin theta))
 * generated on the device (Sec. 2, f = -w^2 G D u_I).  FP64 output; the convolution runs
 * in double-float arithmetic when ls_set_double_float is on (the LS_MIXED default), else
 * in FP64.  f: device, nz*nx. */
int ls_incident_rhs(ls_handle* h, double theta, ls_c64* f);

/* ls_solve -- solve H u = f (Sec. 4): outer flexible GMRES preconditioned by
 * Algorithm 3 (inner GMRES on C v = A r preconditioned by Algorithm 2).
 *   tol: relative residual target ||f - H u|| / ||f||, checked with FP64 H.
 *   u: in: initial guess if use_x0 != 0, else ignored; out: solution.
 *   stats: may be NULL.
 * Requires ls_factor.  LS_ENOCONV if the caps are reached (u = best iterate,
 * stats filled); LS_ENAN on NaN/Inf in f or a residual.  f = 0 gives u = 0. */
int ls_solve(ls_handle* h, const ls_c64* f, double tol, ls_c64* u, int use_x0, ls_stats* stats);

/* ls_solve_host -- ls_solve with HOST arrays f and u (pageable or pinned); the
 * host<->device copies run on the handle's stream inside the call. */
int ls_solve_host(ls_handle* h, const ls_c64* f_host, double tol, ls_c64* u_host, ls_stats* stats);

/* ls_solve_plane_wave -- f = ls_incident_rhs(theta) followed by ls_solve. */
int ls_solve_plane_wave(ls_handle* h, double theta, double tol, ls_c64* u, ls_stats* stats);

/* ls_solve_batch -- nrhs independent solves H u_b = f_b (1 <= nrhs <= LS_MAX_BATCH)
 * in one call: f and u hold nrhs fields back to back (field b at offset b*nz*nx).
 * The same H serves every right-hand side (Sec. 5 solves one scatterer for 64
 * incident waves); the members iterate in lockstep, each with its own Krylov
 * spaces and stopping test, and share every application of Algorithm 2 (its
 * factor traffic and its chain of launches): the batch is cut into chunks of
 * up to 8 (ls_autotune / ls_set_shapes pick the size) whose Algorithm 2 chains
 * run concurrently on up to 8 streams of the handle; chunks whose members have
 * all converged are skipped.  Each u_b is what ls_solve would
 * return for f_b up to rounding.  stats: iteration counts summed over the
 * members; refine_steps and true_rel_residual the largest over the members.
 * Device memory: the Krylov spaces grow to nrhs * (2 (outer_restart +
 * inner_restart) + 7) fields (LS_ENOMEM if they do not fit): at 2048^2 and the
 * default restarts 40 / 30, 9.9 GB per right-hand side.  Return codes as
 * ls_solve; LS_ENOCONV if any member misses the tolerance. */
int ls_solve_batch(ls_handle* h, int nrhs, const ls_c64* f, double tol, ls_c64* u, int use_x0,
                   ls_stats* stats);

/* ls_solve_batch_host -- ls_solve_batch with HOST arrays f and u of nrhs fields
 * (pinned or pageable); the host<->device copies run on the handle's stream
 * inside the call. */
int ls_solve_batch_host(ls_handle* h, int nrhs, const ls_c64* f_host, double tol, ls_c64* u_host,
                        ls_stats* stats);

/* ls_solve_group -- nprob INDEPENDENT problems (distinct handles, each set up and
 * factored for its own medium and grid size), one right-hand side each, solved
 * concurrently: up to LS_GROUP_WORKERS host threads take the problems in turn
 * and run ls_solve(hs[i], f[i], tol, u[i]) on handle i's stream.  For the GPU
 * to overlap the problems the handles must have been set up on distinct
 * streams (on one shared stream the solves serialise, with the same results).
 * Each u[i] is exactly what ls_solve gives for that handle.
 *   hs, f, u: arrays of nprob pointers (f[i], u[i] device fields of hs[i]'s size);
 *   stats, status: NULL or arrays of nprob entries (per-problem statistics and
 *   return codes).
 * Returns LS_OK, LS_EINVAL (a null pointer, a handle given twice), LS_ESTATE
 * (a handle not factored; nothing is solved), else the first failing problem's code. */
enum { LS_GROUP_WORKERS = 32 };
int ls_solve_group(int nprob, ls_handle* const* hs, const ls_c64* const* f, double tol, ls_c64* const* u,
                   ls_stats* stats, int* status);

/* ls_autotune -- pick the two shape choices of the on-line path by timing them on
 * this handle with incident-wave right-hand sides of its own problem:
 *   - the FFT tile shape of the FP32 / mixed LS-apply (column pass): fft_variant
 *     0 = radix-16 transforms on 1-column tiles, 3 CTAs per SM; 2 = radix-16 on
 *     2-column tiles (the default); 3 = radix-16 on 1-column tiles, 2 CTAs per SM;
 *     4 = radix-8 per thread on 1-column tiles; 5 = radix-8 per thread on
 *     2-column tiles; 6, 7 = shapes 2 and 5 with the column tiles moved between
 *     HBM and shared memory by TMA; 8 = shape 6 with the two columns of a tile in
 *     packed FP32x2 instructions (0 and 2..8 need 256 <= P <= 4096); 1 = the
 *     generic radix-8 transforms on 4-column tiles;
 *   - the band-block batching of Algorithm 2 for nrhs right-hand sides: bd_chunk
 *     = right-hand sides per pass over the local-solve factors (1, 2, 4, 8;
 *     FP64 up to 4), chunks running concurrently on separate streams, and
 *     cr_split = whether the block-cyclic-reduction steps of levels with few
 *     blocks split each block over several CTAs (partial sums combined in a
 *     fixed order, so results are reproducible for a given choice).
 * Each candidate runs once, then reps times under CUDA events; the fastest is
 * kept by the handle for later applies and batched solves (results agree up to
 * rounding whichever is chosen).  Before ls_factor only the FFT shape is tuned
 * (bd_chunk = 0 in out).  Allocates 2 * nrhs fields of scratch for the call;
 * synchronises the stream.  out: may be NULL. */
typedef struct {
    int fft_variant;    /* chosen FFT tile shape                                       */
    int bd_chunk;       /* chosen right-hand sides per Algorithm 2 pass                */
    double fft_ms[9];   /* LS-apply (FP64 I/O, FP32 arithmetic) per variant; -1: n/a   */
    double bd_ms[4];    /* Algorithm 2 ms per right-hand side, chunks 1, 2, 4, 8 (0: not tried) */
    double bd_ms_nosplit[4]; /* the same without splitting the blocks of small levels        */
    int cr_split;       /* 1: the reduction steps of levels with fewer blocks than SMs split
                           each block's columns over several CTAs; 0: one CTA per block     */
    double bd_ms_tc[4]; /* LS_MIXED: the same with the reduction steps on the tensor cores,
                           chunks 1, 8, 16, 32 (0: not tried; tried only while that form
                           is switched on, see ls_set_tensor_steps)                        */
    int tensor_steps;   /* 1: the tensor-core steps were chosen (the handle keeps on = 2)   */
} ls_tuning;
int ls_autotune(ls_handle* h, int nrhs, int reps, ls_tuning* out);

/* ls_set_shapes -- pin the two shape choices (e.g. from an earlier ls_autotune):
 * fft_variant 0..8 as above (a radix-16/8 shape on a P outside 256..4096 falls back
 * to the generic one), bd_chunk 1..32 with the tensor-core steps, 1..8 on the CUDA
 * cores (FP64: 1..4), or 0 for the largest.  LS_EINVAL otherwise.  Results agree up to
 * rounding whichever shapes are set. */
int ls_set_shapes(ls_handle* h, int fft_variant, int bd_chunk);

/* ls_set_tensor_steps -- LS_MIXED: where the block-cyclic-reduction steps of the local
 * solves (Algorithm 1's (C^l)^{-1}, Sec. 3.4; factors of Sec. 4.1) run: on the tensor
 * cores (each step one TF32 matrix product over the whole batch, factor planes copied
 * in bulk, accumulators in tensor memory) or on the CUDA cores in FP32.  on = 0: CUDA
 * cores; 1 (the default after ls_factor): tensor cores for passes of 5 or more
 * right-hand sides, CUDA cores below; 2: tensor cores always.  ls_autotune leaves the
 * measured choice (0 or 2).  The tensor-core form rounds the factors and vectors to
 * TF32 (about 3 decimal digits): it changes the preconditioner by that much, never the
 * converged solution, which the FP64 residual judges.  Synchronises the stream and
 * drops the captured sweep graphs on a change.  LS_ESTATE when on > 0 and the form is
 * not built (LS_FP64, before ls_factor, or q > 112); LS_EINVAL for other values. */
int ls_set_tensor_steps(ls_handle* h, int on);

/* ls_host_alloc -- bytes of page-locked host memory for the host-array entry points
 * (ls_solve_host, ls_solve_batch_host), allocated by this library's CUDA runtime as
 * portable pinned memory, so that their copies run as direct transfers.  On GB300 the
 * host-array batched solve ran about 8 per cent faster end to end from such buffers than
 * from buffers pinned by another runtime in the same process.  *out: the block, or NULL
 * with LS_ENOMEM when the allocation fails; LS_EINVAL for a null out or bytes = 0.
 * Release with ls_host_free (a null pointer is accepted). */
int ls_host_alloc(size_t bytes, void** out);
int ls_host_free(void* p);

/* ls_get_sweep_histogram -- counts[k] = how many batched Algorithm 2 applications of the
 * last solve ran on k fields (k = 0 .. len - 1; entries past LS_MAX_BATCH are 0).
 * LS_EINVAL for a null pointer or len < 1. */
int ls_get_sweep_histogram(ls_handle* h, int* counts, int len);

/* ls_set_pack_members -- on = 1 (default): before each batched Algorithm 2 application
 * (Sec. 3.5) inside a lockstep batch, the members still iterating are moved into the
 * leading slots and Algorithm 2 runs on that many fields only (the results are moved
 * back); the members that have converged cost nothing.  on = 0: it runs on the batch up
 * to the last member still iterating, the others' slots zeroed.  Results agree up to the
 * rounding of the form the smaller batch takes (batches below 5 run the local solves on
 * the CUDA cores in FP32 instead of TF32 on the tensor cores).  LS_EINVAL for other
 * values of on. */
int ls_set_pack_members(ls_handle* h, int on);

/* ls_set_double_float -- on = 1: the FP64-accurate convolutions of a solve, the
 * refinement residuals f - H u of LS_MIXED (Sec. 4's outer iteration around the FP32
 * correction) and ls_incident_rhs, run in double-float arithmetic (ls_apply_double_float):
 * GB300's FP64 pipe is about 1/64 of its FP32 rate, and a residual correct to a few 1e-13
 * is far below any solve tolerance.  on = 0: FP64.  Default 1 for LS_MIXED handles, 0 for
 * LS_FP64 ones.  ls_apply stays FP64 either way.  LS_EINVAL for other values of on. */
int ls_set_double_float(ls_handle* h, int on);

/* ls_set_reduced_inverse -- LS_MIXED, tensor-core local solves (Sec. 3.4; factors of
 * Sec. 4.1): the block-cyclic-reduction steps of the levels at and above the first level
 * with at most 32 blocks (its even-block reductions, the top block and the back
 * substitution down to it) form one linear map, the inverse of that level's reduced
 * system.  ls_factor precomputes it per strip (those steps applied to the identity's
 * columns, stored as TF32 planes: (32 q)^2 complex values per strip) and on = 1 (the
 * default) applies it as one tensor-core product instead of those steps; on = 0 runs the
 * steps.  Both round to TF32; they differ by that rounding (the inverse is rounded once
 * more).  Synchronises the stream and drops the captured sweep graphs on a change.
 * LS_EINVAL for other values of on. */
int ls_set_reduced_inverse(ls_handle* h, int on);

/* ls_set_reduction -- pin the form of the block-cyclic-reduction local solves of
 * Algorithm 1 (Sec. 3.4): cr_split 1 lets the steps of levels with fewer blocks
 * than SMs split each block's columns over several CTAs, 0 keeps one CTA per block
 * (as in ls_tuning).  Synchronises the handle's stream and drops the captured sweep
 * graphs when the form changes.  LS_EINVAL for other values.  Results agree up to
 * rounding in either form. */
int ls_set_reduction(ls_handle* h, int cr_split);

/* ls_device_timeouts -- health counter of the kernels fed by TMA (the paper has no
 * counterpart of this counter): *count = how many CTAs found their copies or their
 * tensor-core products not complete within one second since the library was loaded --
 * CTAs of the LS-apply's TMA column tile shapes (6, 7, 8; Sec. 2), of the tensor-core
 * reduction steps of the local solves (Sec. 3.4-3.5) and of the learned step's
 * tensor-core convolutions; 0 in a healthy run.
 * Such a CTA writes its outputs as NaN (so the solver's residual checks reject the
 * result) and returns instead of waiting on.  Synchronous read of device counters.
 * LS_EINVAL if count is NULL. */
int ls_device_timeouts(unsigned* count);

/* ls_test_tma_shortfall -- test hook for the timeout path above (no counterpart in the
 * paper): every later launch of the TMA column pass (any handle) makes its barrier
 * expect `bytes` more than its boxes deliver, so each of its waits runs out after one
 * second with every copy already landed.  0 (the default) restores normal operation.
 * bytes: a multiple of 16, at most 4096, else LS_EINVAL.  Not thread-safe against
 * concurrent applies. */
int ls_test_tma_shortfall(unsigned bytes);

/* ---- learned preconditioner step (an addition: the paper has no network) ----
 * A BF16 convolutional U-Net N, trained and applied by this library's own
 * kernels (tensor-core convolutions, FP32 accumulation).  The paper's outer
 * iteration is flexible GMRES (Sec. 6), which admits a different
 * preconditioner at every step; with a network attached, the first direction
 * of every outer cycle is z = s N(v / s, m) (s = RMS of v) and the others come
 * from Algorithm 3 as before, so the plain preconditioner stays in the loop and
 * the FP64 residual of the refinement decides convergence.
 * Architecture: `levels` levels, c0 * 2^l channels at level l (c0 a multiple of
 * 16), 3x3 convolutions, 2x2 average pooling, nearest 2x upsampling, skip
 * concatenation; input (Re v / s, Im v / s, m), output 2 channels.  Fields are
 * nb samples of H x W (x fastest), H and W multiples of 8 * 2^(levels-1).
 * Parameters (host FP32) are in the layer order: encoder l = 0..L-1 (a, b),
 * decoder l = L-2..0 (up, a, b), head; per layer w[o][c][3][3] then b[o]. */
typedef struct ls_net ls_net;
int ls_net_create(int levels, int c0, int max_batch, int H, int W, int train, unsigned long long seed,
                  void* stream, ls_net** out);      /* max_batch * H * W pixels of buffers      */
size_t ls_net_param_count(const ls_net* net);
int ls_net_get_params(ls_net* net, float* host, size_t count);
int ls_net_set_params(ls_net* net, const float* host, size_t count);   /* resets Adam          */
/* z_b = s_b N(r_b / s_b, m_b): r, z DEVICE complex fields, m DEVICE real fields (nb each) */
int ls_net_forward(ls_net* net, int nb, int H, int W, const ls_c64* r, const double* m, ls_c64* z);
/* one Adam step (lr; betas 0.9, 0.999) on 0.5 mean((N(r/s, m) - e/s)^2); *loss (host) may be NULL */
int ls_net_train_step(ls_net* net, int nb, int H, int W, const ls_c64* r, const double* m, const ls_c64* e,
                      float lr, double* loss);
int ls_net_get_grads(ls_net* net, float* host, size_t count);   /* of the last training step */
long long ls_net_kernel_count(const ls_net* net);
void ls_net_destroy(ls_net* net);
/* ls_net_set_tensor_cores -- where the network's forward and backward-data convolutions
 * run (no counterpart in the paper; the network is the learned step of Sec. 6's
 * flexible outer iteration): on = 1 (the default) on the fifth-generation tensor cores
 * (tcgen05.mma kind::f16 on BF16 operands, FP32 accumulation in tensor memory), 0 on the
 * WMMA path; both accumulate in FP32, so results agree to BF16 rounding of the outputs.
 * The weight gradients use WMMA either way.  LS_EINVAL for a NULL net or other values. */
int ls_net_set_tensor_cores(ls_net* net, int on);

/* attach (net != NULL) or detach the learned step of handle h's outer iteration; the
 * network must accept the handle's n x n grid (batch 1) and outlive the attachment. */
int ls_set_learned(ls_handle* h, ls_net* net);

/* ---- operators of the inner level (Sec. 2-3), exposed for checking and reuse ---- */

/* y = A r: sparsifying stencil (Sec. 2), 9-point with boundary types.  FP64. */
int ls_apply_A(ls_handle* h, const ls_c64* r, ls_c64* y);

/* y = C v: sparsified matrix C = A H kept on the 9-point pattern (Sec. 2). FP64. */
int ls_apply_C(ls_handle* h, const ls_c64* v, ls_c64* y);

/* v = Algorithm 1 (Gauss-Seidel polarized-traces preconditioner, Sec. 3.4) applied
 * to g, on horizontal layers (dir = 0) or vertical layers (dir = 1).  Requires
 * ls_factor.  Local solves in the handle's precision. */
int ls_sweep(ls_handle* h, int dir, const ls_c64* g, ls_c64* v);

/* v = Algorithm 2 (bi-directional preconditioner, Sec. 3.5) applied to g. */
int ls_precond_bd(ls_handle* h, const ls_c64* g, ls_c64* v);

/* Algorithm 2 applied to nrhs fields g_b at once (back to back, as in
 * ls_solve_batch): v_b equals ls_precond_bd(g_b) up to rounding.  1 <= nrhs <=
 * LS_MAX_BD_BATCH for LS_MIXED, <= 4 for LS_FP64 (else LS_EINVAL). */
int ls_precond_bd_batch(ls_handle* h, int nrhs, const ls_c64* g, ls_c64* v);

/* Inner level of Algorithm 3: GMRES on C v = g preconditioned by Algorithm 2,
 * from v = 0, to relative tolerance tol.  *iters receives the iteration count. */
int ls_inner_solve(ls_handle* h, const ls_c64* g, double tol, ls_c64* v, int* iters);

/* Local solve x = (C^l)^{-1} b on layer l of direction dir (Sec. 3.1): b and x are
 * DEVICE arrays of q*nx elements, q = t + 2*ext rows of the extended layer,
 * local row r <-> global row l*t - ext + r (rows outside Omega are identity
 * rows), x fastest.  Uses the factors of ls_factor in the handle's precision. */
int ls_local_solve(ls_handle* h, int dir, int layer, const ls_c64* b, ls_c64* x);

/* ls_apply_f32_noalloc -- the FP32 LS-apply y = u + IFFT2(Ghat .* FFT2(pad(m u)))[0:n, 0:n]
 * of ls_apply_f32, for callers that must not allocate device memory when they call it:
 * code that runs under a memory manager which owns the whole device budget and forbids
 * driver allocations after start-up, or a latency-critical loop that cannot afford the
 * device synchronisation an allocation may cause.  It needs no handle and allocates
 * nothing: its n x P scratch and its twiddle tables are fixed file-scope device arrays
 * (16 MiB + 32 KiB, held by every GPU that loads the library until the process exits).
 * The paper has no counterpart.
 *   n: grid points per direction, 8 <= n <= 1024 (n * P <= 2^21, P = smallest power of
 *      two >= 2n - 1); larger n returns LS_ETOOBIG and does nothing.
 *   m: DEVICE float[n*n], the contrast (x fastest).
 *   ghat: DEVICE ls_c32[(P/2+1)^2], the spectral quadrant of ls_get_spectrum rounded to
 *      FP32 (index kx*(P/2+1) + kz).
 *   u, y: DEVICE ls_c32[n*n]; may alias.  stream: cudaStream_t (NULL = legacy stream).
 *   m, ghat, u and y must be memory of the CURRENT device (device or managed
 *   allocations); a buffer on another device, or host memory, returns LS_EINVAL.
 * The first call on a device (with that device current) sets up the arrays for that
 * device -- resolves their addresses, fills the twiddle tables, synchronises `stream`
 * once -- so it should come before any stream capture.  The scratch needs no clearing
 * (pass 1 writes every element the later passes read), but all calls on a device share
 * it: calls that overlap on the GPU (other streams, other host threads) race. */
int ls_apply_f32_noalloc(int n, const float* m, const ls_c32* ghat, const ls_c32* u, ls_c32* y, void* stream);

/* ls_check_conversions -- self-check of the FP64 <-> FP32 conversions the mixed-
 * precision kernels use (integer-pipe routines: GB300's FP64 units, which the
 * hardware conversions occupy, are few; the paper has no counterpart): for
 * i < n compares the library's double -> float (round to nearest even) of d[i] and
 * float -> double of f[i] with the hardware's, bit for bit (NaN inputs: NaN-ness
 * only).  d, f: DEVICE arrays of n elements; *mismatches (host) = the number of
 * differing results, 0 when the routines are exact.  Runs on the legacy stream and
 * synchronises; allocates 8 bytes of device memory for the call.  LS_EINVAL on NULL
 * pointers or n < 0. */
int ls_check_conversions(const double* d, const float* f, long long n, unsigned long long* mismatches);

/* ---- introspection (host copies of small tables) ---- */

/* alpha, beta: host arrays of 81 ls_c64 each, index [type*9 + slot] with
 * type = (bz+1)*3 + (bx+1) and slot = (dz+1)*3 + (dx+1) (Sec. 2 stencils;
 * beta_d = sum_e alpha_e G_w(e - d)). Either may be NULL. */
int ls_get_stencils(ls_handle* h, ls_c64* alpha, ls_c64* beta);

/* Quadrant of the spectral factor Ghat = (w^2/P^2) FFT2(circulant embedding of G),
 * (P/2+1)^2 elements, index [kx*(P/2+1) + kz] (the quadrant is symmetric, G being
 * radial).  P = smallest power of two >= 2*nx - 1.  ghat: DEVICE array. *P_out = P. */
int ls_get_spectrum(ls_handle* h, ls_c64* ghat, int* P_out);

/* Diagonal quadrature weight G_w(0) (Sec. 2) as used by the handle. */
int ls_get_diag_weight(ls_handle* h, ls_c64* w0);

/* Local strip height q = t + 2*ext and t = nz / layers. */
int ls_get_layout(ls_handle* h, int* t, int* q);

/* Turn per-call CUDA-event timing of LS-apply and Algorithm 2 on (1) or off (0). */
int ls_set_timing(ls_handle* h, int on);

/* Number of kernels the library has launched on this handle since setup. */
long long ls_kernel_count(ls_handle* h);

void ls_destroy(ls_handle* h);
const char* ls_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LS_H */
