/*
 * esi.h -- C ABI of libesi: the GB300 (sm_103a) hot path of time-domain extended-source
 * waveform inversion (ESI), after P. Yang & W. Zhou, "Algorithmic analysis towards
 * time-domain extended source waveform inversion" (arXiv 2211.06300).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Grid      : nz x ny x nx cells (ny = 1 in 2D), spacing dx on every axis, x fastest.
 *              Cell (iz, iy, ix) sits at (x, y, z) = (ix dx, iy dx, iz dx).  The grid
 *              includes the absorbing sponge of nb cells on every side.  N = nz*ny*nx.
 *  Physics   : (1/v^2) u_tt - Lap u = q  (Eq. "wave"), discretised O(dt^2, dx^8) with a
 *              damping sponge (Numerical tests section).  Step n (0 <= n < nt) consumes
 *              the source q_n (time n dt) and produces u_{n+1}; u_0 = u_{-1} = 0.
 *  Sampling  : R (Eq. "fwi") uses bilinear (2D) / trilinear (3D) weights; trace sample n
 *              is R u_{n+1}.  A point source injects f_n * w / dx^d at the same nodes.
 *  Traces    : "seismogram" buffers are CSR-packed per shot, time-major:
 *              shot s occupies nt * nrec(s) values starting at nt * rec_offset[s],
 *              element (s, n, r) at nt * rec_offset[s] + n * nrec(s) + r.
 *  Fields    : space-time buffers (extended sources, adjoint outputs, CG solutions) are
 *              [shot][n][iz][iy][ix], dense, element type = the context precision.
 *  Precision : ESI_F32 (float) or ESI_F64 (double) for fields and traces; CG scalars,
 *              dot products and misfits are always accumulated in double.
 *  Memory    : every *_dev pointer is CUDA device memory owned by the caller (the Python
 *              binding passes PyTorch tensors); host pointers are plain host memory.  The
 *              library never frees caller memory.  The context owns its scratch (wave
 *              states, checkpoints, CG work vectors), allocated on first use and released
 *              by esi_destroy.
 *  Streams   : all work is enqueued on the stream given to esi_create (or
 *              esi_set_stream).  Calls return after enqueueing, except where stated
 *              (esi_cg_solve, esi_gradient's misfit, esi_dft_extract's scales), which
 *              synchronise the stream to read a few scalars back.
 *  Errors    : every call returns an esi_status; nothing is thrown across the ABI.  On
 *              failure esi_last_error(ctx) gives a message.  A context whose call failed
 *              with ESI_ERR_CUDA should be destroyed.
 */
#ifndef ESI_H
#define ESI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ESI_API __attribute__((visibility("default")))
#else
#define ESI_API
#endif

typedef enum esi_status {
    ESI_OK = 0,
    ESI_ERR_ARG = 1,            /* invalid argument (NULL, size, point outside the grid) */
    ESI_ERR_CFL = 2,            /* v_max dt / dx above the stability limit of the scheme */
    ESI_ERR_OOM = 3,            /* device allocation failed */
    ESI_ERR_CUDA = 4,           /* a CUDA call failed (message in esi_last_error) */
    ESI_ERR_BREAKDOWN = 5,      /* CG: p^T A p <= 0 or a non-finite scalar */
    ESI_ERR_TIMEOUT = 6,        /* a bounded device wait expired */
    ESI_ERR_NOT_CONVERGED = 7,  /* CG stopped at max_iter above tol (outputs valid) */
    ESI_ERR_UNSUPPORTED = 8     /* option combination not implemented */
} esi_status;

typedef enum esi_dtype { ESI_F32 = 0, ESI_F64 = 1 } esi_dtype;

typedef struct esi_ctx esi_ctx;

typedef struct esi_grid {
    int ndim;            /* 2 or 3 */
    int nz, ny, nx;      /* cells; ny must be 1 when ndim == 2 */
    double dx;           /* metres */
    int nb;              /* sponge width in cells on every side (0 = rigid edges) */
    double sponge_R;     /* target reflection coefficient of the sponge, e.g. 1e-3 */
    double sponge_vref;  /* velocity used in the damping profile (> 0, m/s) */
    int dtype;           /* esi_dtype */
} esi_grid;

typedef struct esi_geometry {
    int ns;                        /* number of shots */
    const double *src_xyz;         /* host [ns][3]: source (x, y, z) in metres */
    const long long *rec_offset;   /* host [ns + 1]: CSR offsets into rec_xyz */
    const double *rec_xyz;         /* host [rec_offset[ns]][3]: receivers, metres */
} esi_geometry;

/*
 * esi_create -- set up the discrete wave operator A(m) on a velocity model
 * (Eq. "wave": constant-density acoustic, m = v) with the shots' sampling operators R
 * (Eq. "fwi") and source positions.
 *   out          : receives the new context
 *   grid         : grid description (copied)
 *   geom         : acquisition (copied)
 *   velocity_dev : device [nz][ny][nx] velocity in m/s, element type = grid->dtype
 *   dt           : time step in seconds;  nt : number of steps (>= 1)
 *   stream       : cudaStream_t (NULL = legacy default stream)
 * Rejects a time step above the stability limit with ESI_ERR_CFL:
 *   v_max dt / dx <= sqrt(4 / (ndim * 6.5015873...)), the Nyquist symbol of the 8th-order
 *   Laplacian.  Points outside the grid give ESI_ERR_ARG.  Synchronises the stream once.
 */
ESI_API esi_status esi_create(esi_ctx **out, const esi_grid *grid, const esi_geometry *geom,
                              const void *velocity_dev, double dt, int nt, void *stream);

ESI_API void esi_destroy(esi_ctx *ctx);

/* Replace the context's stream (cudaStream_t). */
ESI_API esi_status esi_set_stream(esi_ctx *ctx, void *stream);

/* Replace the velocity model (same grid, same sponge reference); device pointer.  Shot
 * groups (esi_set_shot_groups) follow it. */
ESI_API esi_status esi_set_velocity(esi_ctx *ctx, const void *velocity_dev);

/*
 * esi_set_shot_groups -- run the context's shots as `groups` concurrent groups.  The paper's
 * shots are independent systems (one extended source q and one normal equation per shot),
 * so the batch can be split: the context makes child contexts over contiguous shot ranges
 * (shot s in group k when k ns / groups <= s < (k + 1) ns / groups), each with a stream of
 * its own, and esi_forward, esi_adjoint, esi_normal_apply, esi_cg_solve (plain or diagonal
 * preconditioner), esi_wri_solve, esi_dscg_solve, esi_fdcg_solve, esi_gradient and
 * esi_dft_extract then run every group in a host thread of its own: their launches, host
 * synchronisations and the partly filled last wave of each step launch overlap.  Per-shot
 * outputs are those of the ungrouped context (each group writes its shots' slices); the
 * gradient, a sum over shots, is the groups' partial sums added in group order by a
 * kernel, and the misfit likewise.  A CG report gives per-shot iterations and residual
 * histories as before; its phase times are the longest group's.  esi_invert's evaluations
 * (inner solve, objective and gradient) go through these calls and so run on the groups;
 * esi_forward_noalloc (whose fixed scratch the groups would share) and the learned
 * preconditioner run on the context itself.  Each call's groups start after the
 * work already queued on the context stream, which then waits for all of them.
 * esi_set_profiling, esi_get_profile (entries merged by name, times summed over the groups'
 * streams) and esi_launch_count include the groups.
 *   groups       : 1 .. ns (1 removes the groups)
 *   velocity_dev : the current velocity model, as for esi_create (device pointer)
 * The groups own their scratch (per shot, as the context would).  Synchronises the context
 * stream.  Errors: ESI_ERR_ARG (groups outside 1 .. ns, no velocity), those of esi_create.
 */
ESI_API esi_status esi_set_shot_groups(esi_ctx *ctx, int groups, const void *velocity_dev);

/*
 * esi_forward -- forward modelling d = R A^{-1} q for every shot (Eq. "fwi", "wave").
 *   wavelet_dev : device [ns][nt] point-source time functions f_n, or NULL
 *   ext_src_dev : device [ns][nt][N] extended source q (Eq. "newq2"), or NULL
 *                 (both may be given; they add)
 *   traces_dev  : device seismogram buffer (CSR layout above), written
 */
ESI_API esi_status esi_forward(esi_ctx *ctx, const void *wavelet_dev, const void *ext_src_dev,
                               void *traces_dev);

/*
 * esi_forward_noalloc -- the same forward modelling as esi_forward, for callers that must
 * not allocate device memory: a host framework that owns every byte of device memory
 * through its own pool (a side cudaMalloc would fail or break its accounting), or a
 * latency-bound loop that cannot pay for the device-wide synchronisation cudaMalloc and
 * cudaFree imply.  esi_forward allocates the two wave states on its first call; this
 * entry point instead keeps them in a fixed 32 MiB device array compiled into the
 * library (every GPU that loads the library holds it until the process exits) and calls
 * no allocator.  The paper has no counterpart: this is a deployment variant.
 *   Limit     : 2 * ns * nz * ny * round_up(nx, 32) * sizeof(element) <= 32 MiB, else
 *               ESI_ERR_ARG with a message (nothing is enqueued).
 *   Set-up    : the first call on a device looks up the array's device address with that
 *               device current; make that first call before any stream capture.
 *   Sharing   : all calls in the process share the one array per device.  It is cleared
 *               at the start of every call, so results do not depend on earlier calls,
 *               but calls whose work overlaps on the GPU (other streams, other threads,
 *               other contexts on the same device) race on it: serialise them.
 *   Launches  : the step kernels of esi_forward, issued one by one (no CUDA graph, since
 *               instantiating one may take device memory), every step after the first a
 *               programmatic dependent launch; recorded by esi_get_profile like esi_forward.
 *   Arguments : as esi_forward; traces_dev must not be NULL.
 */
ESI_API esi_status esi_forward_noalloc(esi_ctx *ctx, const void *wavelet_dev,
                                       const void *ext_src_dev, void *traces_dev);

/*
 * esi_adjoint -- exact discrete adjoint S^T e = A^{-T} R^T e (Eq. "FWI_lambda"; the
 * right-hand side b = S^H d of the CG section), the transpose of esi_forward's map from
 * the extended source to the traces.
 *   traces_dev  : device seismogram-layout adjoint data e
 *   ext_out_dev : device [ns][nt][N] receives (S^T e), or NULL
 *   wavelet_out_dev : device [ns][nt] receives the adjoint of the point-source injection
 *                 (the transpose of esi_forward's wavelet -> traces map), or NULL
 */
ESI_API esi_status esi_adjoint(esi_ctx *ctx, const void *traces_dev, void *ext_out_dev,
                               void *wavelet_out_dev);

typedef enum esi_grad_mode {
    ESI_GRAD_ADJOINT_STATE = 0,  /* back-propagate a data residual (Eq. "gradient") */
    ESI_GRAD_SADDLE_POINT = 1,   /* Algorithm 2: lambda = beta B^H B q, no adjoint run */
    ESI_GRAD_WRI_SADDLE = 2      /* WRI (Eq. "gradient2"): u = A^{-1}(f + q), lambda = beta q */
} esi_grad_mode;

typedef enum esi_param { ESI_PARAM_C = 0, ESI_PARAM_V = 1, ESI_PARAM_M = 2 } esi_param;

/* Compressed kinds store u_n and the difference u_n - u_{n-1} of each checkpoint, each with
 * its own per-shot scale; u_{n-1} is rebuilt as decoded u_n minus decoded difference. */
typedef enum esi_ckpt_kind {
    ESI_CKPT_F32 = 0,            /* checkpoints stored in the field precision */
    ESI_CKPT_F16 = 1,            /* IEEE half with a per-snapshot scale */
    ESI_CKPT_BF16 = 2            /* bfloat16 with a per-snapshot scale */
} esi_ckpt_kind;

typedef struct esi_grad_opts {
    int mode;          /* esi_grad_mode */
    int param;         /* esi_param: c = v^2 dt^2, v, or m = 1/v^2 */
    int ckpt_every;    /* checkpoint interval in steps (>= 1) */
    int ckpt_kind;     /* esi_ckpt_kind */
    double beta;       /* penalty weight (saddle-point mode) */
    double eps;        /* annihilator offset in metres (<= 0: dx) */
} esi_grad_opts;

/*
 * esi_gradient -- zero-lag cross-correlation gradient (Eq. "gradient", "gradewi").
 * Adjoint-state mode: u = A^{-1}(wavelet, ext_src); the adjoint field of the data
 *   residual e is correlated with Lap u_n + q_n over all steps.  e is adj_src_dev when
 *   given (a vector-Jacobian product, J = <e, d>), otherwise e = R u - dobs and
 *   *misfit = 1/2 ||e||^2 (Eq. "fwi").  The forward states are recomputed per segment of
 *   ckpt_every steps from stored (optionally compressed) checkpoints.
 * Saddle-point mode (Algorithm 2): ext_src is the ESI solution q, the
 *   adjoint field is lambda = beta B^H B q with B = ||x - x_s|| + eps; one forward run.
 * WRI saddle mode (Eq. "newadj2", "gradient2"): ext_src is the WRI solution q and
 *   wavelet_dev the point sources f; u = A^{-1}(f + q), lambda = beta q (B = I); one
 *   forward run.
 *   With dobs_dev in either saddle mode the same forward run also samples R u and
 *   *misfit receives the objective at (m, q): Eq. "esi", 1/2 ||R u - d||^2 +
 *   beta/2 ||B q||^2 (WRI: Eq. "wrimisfit", B = 1), summed over shots; the call then
 *   synchronises.
 *   grad_dev    : device [N], written (sum over all shots) in the chosen parameter
 *   misfit      : host double, written with dobs (may be NULL)
 */
ESI_API esi_status esi_gradient(esi_ctx *ctx, const void *wavelet_dev, const void *ext_src_dev,
                                const void *dobs_dev, const void *adj_src_dev,
                                const esi_grad_opts *opts, void *grad_dev, double *misfit);

/*
 * esi_invert -- the outer loop, Algorithm "nestedloop" (variable projection between m and
 * q): per outer iteration i, the inner CG solve for q at the penalty beta_i = beta0 growth^i
 * (ESI: Eq. "normalewi" with the chosen preconditioner; WRI: Eq. "normalwri"), the objective
 * (Eq. "esi" / "wrimisfit") and the saddle-point gradient in the velocity (Eq. "gradewi" /
 * "gradient2") from one forward run, an L-BFGS direction (two-loop recursion over the newest
 * `memory` pairs, initial matrix (s^T y / y^T y) I; a pair is kept when s^T y > 1e-12 |s| |y|;
 * a non-descent direction clears the memory and takes -g) and a projected backtracking line
 * search (trial v_t = clamp(v + alpha d, vmin, vmax); accepted when J(v_t) <= J(v) +
 * c1 g^T (v_t - v); alpha halved up to max_ls times; first trial alpha = 1 with pairs, else
 * the step moving the fastest cell by step_frac max|v|).  A new penalty re-evaluates J and g
 * and clears the memory.  The sponge keeps the reference velocity fixed at creation.
 *   wavelet_dev  : point sources f (WRI only; else NULL)
 *   dobs_dev     : device seismogram-layout observed data
 *   velocity_dev : device [N] velocity: the start model in, the last accepted model out;
 *                  the context's model is left at it
 *   grad_dev     : device [N] caller scratch: each evaluation's gradient is written here
 *                  before `reduce` sees it; on return, the gradient at the output model
 *   reduce       : (opts) NULL on one rank; for shots sharded over ranks, a callback that
 *                  sums J (host) and grad_dev (device, n values, stream synchronised) over
 *                  the ranks in place and returns 0
 * The context owns the scratch (the inner solution q, [ns][nt][N], and 6 + 2 memory model
 * vectors).  A failed line search ends the loop with ESI_OK and stop_reason 1.  Errors:
 * ESI_ERR_ARG (options, a reduce failure), ESI_ERR_CFL (vmax violates the stability limit),
 * and those of esi_cg_solve and esi_gradient.
 */
typedef int (*esi_reduce_fn)(void *user, double *J, void *grad_dev, long long n);

typedef struct esi_invert_opts {
    int mode;              /* ESI_GRAD_SADDLE_POINT (ESI) or ESI_GRAD_WRI_SADDLE (WRI) */
    int n_outer;           /* outer iterations (>= 0) */
    int n_cg;              /* inner CG iterations (cap, >= 1) */
    double cg_tol;         /* inner relative tolerance; 0 runs n_cg iterations */
    int precond;           /* ESI inner solve: esi_precond */
    double beta0, growth;  /* penalty schedule beta_i = beta0 growth^i (> 0) */
    int memory;            /* L-BFGS pairs, 1 .. 64 */
    double c1;             /* Armijo constant, (0, 1) */
    double step_frac;      /* first-trial scale without pairs (> 0) */
    int max_ls;            /* line-search trials (>= 1) */
    double vmin, vmax;     /* velocity bounds, 0 < vmin < vmax */
    double eps;            /* annihilator offset in metres (<= 0: dx) */
    esi_reduce_fn reduce;  /* cross-rank sum, or NULL */
    void *reduce_user;
} esi_invert_opts;

typedef struct esi_invert_report {
    int max_iters;         /* capacity of the host arrays below (>= n_outer) */
    double *J_start;       /* per iteration: J at its start and after its step (its penalty) */
    double *J_end;
    double *alpha;         /* accepted step */
    double *beta;          /* penalty */
    int *trials;           /* line-search trials */
    int iters_done;        /* accepted steps */
    int evaluations;       /* objective + gradient evaluations */
    int cg_iters_total;    /* inner iterations summed over evaluations (max over shots) */
    int stop_reason;       /* 0 all iterations, 1 line search failed, 2 zero gradient */
    double ms_total;       /* host wall clock */
} esi_invert_report;

ESI_API esi_status esi_invert(esi_ctx *ctx, const esi_invert_opts *opts, const void *wavelet_dev,
                              const void *dobs_dev, void *velocity_dev, void *grad_dev,
                              esi_invert_report *report);

typedef enum esi_dft_out { ESI_DFT_C64 = 0, ESI_DFT_C32_HALF = 1 } esi_dft_out;

/*
 * esi_dft_extract -- forward modelling with the on-the-fly DTFT of the wavefield
 * (Eq. "dtft"): U_m(x) = sum_{n=0}^{nt-1} u_{n+1}(x) exp(+j 2 pi f_m (n+1) dt).
 *   freqs_hz    : host [nf] frequencies
 *   out_dev     : device [ns][nf][N] complex: float2/double2 pairs (ESI_DFT_C64 means
 *                 the context precision) or __half2 pairs (ESI_DFT_C32_HALF, each
 *                 frequency scaled by 1/scales[s*nf+m])
 *   scales_host : host [ns*nf] decode scales for the half output (may be NULL otherwise)
 *   traces_dev  : optional seismogram output of the same run (may be NULL)
 */
ESI_API esi_status esi_dft_extract(esi_ctx *ctx, const void *wavelet_dev, const void *ext_src_dev,
                                   const double *freqs_hz, int nf, void *out_dev, int out_kind,
                                   float *scales_host, void *traces_dev);

typedef enum esi_precond { ESI_PC_NONE = 0, ESI_PC_DIAG = 1, ESI_PC_LEARNED = 2 } esi_precond;

typedef struct esi_cg_report {
    int iters_max;           /* largest iteration count over shots */
    int converged;           /* 1 when every shot met tol */
    int max_hist;            /* capacity of rel_res (entries per shot), set by caller */
    int *iters;              /* host [ns] iterations per shot (may be NULL) */
    double *rel_res;         /* host [ns][max_hist] ||r_{k+1}|| / ||r_0|| (may be NULL) */
    /* per-phase device time (CUDA events on the context stream), summed over iterations:
     * the product S^T S p + lambda B^2 p, the vector updates and reductions, the learned
     * preconditioner; ms_total is the host wall clock of the whole call (set-up, S^T d) */
    double ms_matvec, ms_vector, ms_precond, ms_total;
} esi_cg_report;

/*
 * esi_cg_solve -- Algorithm 1 (CG) on the ESI normal equation (Eq. "normalewi"):
 *   (S^T S + lambda B^T B) q = S^T d,   B = ||x - x_s|| + eps  (per shot),
 * with lambda naming the paper's penalty beta.  Every matrix-vector
 * product is one forward modelling with p as the extended source and one adjoint
 * modelling of its traces (CG section, second bullet), plus lambda B^2 p.  Shots are
 * independent systems, each with its own scalars; a shot stops at
 * ||r_{k+1}|| < tol ||r_0|| or after max_iter iterations.
 *   dobs_dev  : device seismogram-layout observed data d
 *   q_out_dev : device [ns][nt][N] receives the solution x = q
 *   precond   : esi_precond; ESI_PC_DIAG uses z = r / (lambda B^2) in standard PCG
 *               (beta_k = <r_{k+1}, z_{k+1}> / <r_k, z_k>), ESI_PC_LEARNED the network
 *               loaded by esi_pc_load in flexible (Polak-Ribiere) CG
 *   eps       : annihilator offset in metres (<= 0: dx)
 *   report    : may be NULL
 * Synchronises every iteration (reads 8 bytes per shot).  Returns ESI_ERR_NOT_CONVERGED
 * (q valid) when some shot did not reach tol.
 */
ESI_API esi_status esi_cg_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                const void *dobs_dev, void *q_out_dev, int precond, double eps,
                                esi_cg_report *report);

/*
 * esi_fdcg_solve -- frequency-domain ESI by time-domain modelling (the section "Frequency
 * domain inversion by time domain modelling"; Eq. "dtft", "idtft", "normaldtft"): Algorithm 1
 * on the Hermitian positive definite system
 *   F (S^T S + lambda B^T B) F^H qbar / nt = F S^T d,   F[m][n] = exp(+j 2 pi f_m n dt),
 * (the inverse DTFT being the adjoint of F scaled by 1/nt) for the extended source at nf
 * frequencies, qbar: per shot nf complex fields.  The observed data enter as the time series
 * d.  CG runs in the real representation with Re <x, y> as inner product.  Each product
 * synthesises the real and the imaginary part of F^H qbar / nt block by block into a
 * K-step source stash (K = 16, 32 or 64 steps, the longest whose stash fits in 1/16 of the
 * device memory) during two forward modellings, folds the two adjoint modellings of
 * their traces block by block into the frequency slices, and adds lambda B^2 (F F^H / nt)
 * qbar per cell; no space-time vector is stored (the CG vectors hold 2 nf values per cell).
 *   dobs_dev     : device seismogram-layout observed data d
 *   freqs_hz     : host [nf] frequencies, 1 <= nf <= 8
 *   precond      : ESI_PC_NONE, or ESI_PC_DIAG: z = r / (lambda B^2) per cell at every
 *                  frequency (the inverse of the penalty term on the DFT grid, where
 *                  F F^H / nt = I); ESI_PC_LEARNED gives ESI_ERR_UNSUPPORTED
 *   qbar_out_dev : device [ns][nf][N][2] (re, im) receives the solution
 *   eps, report  : as esi_cg_solve (ms_matvec: the products, ms_vector: the vector work)
 * Per-shot stopping, errors and frozen shots as esi_cg_solve; lambda must be > 0.  The
 * time-domain source is q = F^H qbar / nt (its real part for a real source).
 */
ESI_API esi_status esi_fdcg_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                  const void *dobs_dev, const double *freqs_hz, int nf,
                                  int precond, void *qbar_out_dev, double eps,
                                  esi_cg_report *report);

/*
 * esi_dscg_solve -- the ESI normal equation solved in data space (the section "Switching
 * from the wavefield to data space"; Eq. "wd", "q"): Algorithm 1 on
 *   (I + K) w = K d,   K = S (lambda B^2)^{-1} S^T,   B = ||x - x_s|| + eps,
 * for the synthetic data w, then q = (lambda B^2)^{-1} S^T (d - w).  Each product K p is
 * one adjoint modelling of p, whose space-time field is kept in context scratch (one
 * pitched [ns][nt][N] vector), and one forward modelling with that field times
 * 1/(lambda B^2) as the extended source; the CG vectors are traces-layout data vectors.
 * Per shot, stopping and frozen shots as in esi_cg_solve (the residual is the data-space
 * one).  q_out_dev: device [ns][nt][N]; w_out_dev: device traces layout (may be NULL).
 * Errors and report as esi_cg_solve (ms_matvec: the products, ms_vector: the data-space
 * vector work).
 */
ESI_API esi_status esi_dscg_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                  const void *dobs_dev, void *q_out_dev, void *w_out_dev,
                                  double eps, esi_cg_report *report);

/*
 * esi_wri_solve -- WRI by the same CG (the CG section: B = I and WRI's own right-hand
 * side; Eq. "normalwri"):
 *   (S^T S + lambda I) q = S^T (d - S f),
 * f the point sources (wavelet_dev [ns][nt], as in esi_forward) and d the observed traces.
 * One forward modelling with f gives the data residual d - S f (kept in context scratch);
 * then Algorithm 1 exactly as in esi_cg_solve (no preconditioner: with B = I the diagonal
 * one is a constant).  The wavefield is u = A^{-1}(f + q); the WRI gradient is
 * esi_gradient in ESI_GRAD_WRI_SADDLE mode.  q_out_dev: device [ns][nt][N].  Errors and
 * report as esi_cg_solve.
 */
ESI_API esi_status esi_wri_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                 const void *wavelet_dev, const void *dobs_dev, void *q_out_dev,
                                 esi_cg_report *report);

/*
 * esi_normal_apply -- the ESI normal operator (Eq. "normalewi"; the matrix-vector product
 * bullet of the CG section): out = S^T S p + lambda B^2 p, B = ||x - x_s|| + eps (eps <= 0:
 * dx), one forward and one adjoint modelling.  p_dev, out_dev: device [ns][nt][N] dense.
 */
ESI_API esi_status esi_normal_apply(esi_ctx *ctx, double lambda, double eps, const void *p_dev,
                                    void *out_dev);

/*
 * Learned CG preconditioner (the paper's conclusion: an efficient preconditioner to cut
 * the inner CG iterations).  For a residual r of one shot:
 *     s = r / (lambda B^2),   z = s + up2(U(pack(s)))
 * where pack() averages 2 x 2 cells and groups 16 consecutive time samples as the 16
 * channels of an image (time padded with zeros to a multiple of 16), U is a 4-level U-Net
 * with 32 channels (3 x 3 convolutions with zero padding and ReLU, 2 x 2 average pooling
 * with zero fill at odd edges, nearest upsampling with skip additions; the last layer is
 * linear with 16 outputs) and up2() repeats each coarse cell over its 2 x 2 block.  Images
 * are BF16 [img][h][w][16] (h = ceil(nz/2), w = ceil(nx/2)); U computes in BF16 with FP32
 * accumulation on the tensor cores.  Parameters: esi_pc_param_count() FP32 values, per
 * layer (enc1 16->32, enc2, enc3, bott, dec3, dec2 32->32, dec1 32->16) the weights
 * W[3][3][cin][cout] followed by the biases b[cout].  Each image is divided by its RMS
 * before U and the output multiplied by it (y = rms U(x / rms), so the preconditioner is
 * positively homogeneous).  The network is a learned object: its only judge is the CG
 * residual.  In the solver the correction enters per shot as z = s + theta up2(y): theta = 1
 * while <z, r> >= <s, r> / 2 (s the diagonal preconditioner's output) on every active shot;
 * the first time that fails on any shot the solve drops the network (theta = 0 to its end)
 * and every shot restarts its directions from the diagonal preconditioner.
 */
typedef struct esi_pc esi_pc;

ESI_API size_t esi_pc_param_count(void);

/* Load trained parameters (device FP32, esi_pc_param_count() values) into a 2D FP32 context;
 * esi_cg_solve(..., ESI_PC_LEARNED, ...) then uses flexible (Polak-Ribiere) CG with z above. */
ESI_API esi_status esi_pc_load(esi_ctx *ctx, const void *weights_dev, size_t bytes);

/* How many learned solves of this context dropped the network and restarted diagonally. */
ESI_API long long esi_pc_fallbacks(const esi_ctx *ctx);

/* Pack a field (scaled by 1 / (lambda B^2) when scale != 0) into the network's BF16 images
 * [ns * ceil(nt/16)][h][w][16] (2D FP32 contexts).  pitched == 0: the field is dense
 * [ns][nt][nz][nx]; otherwise it has the CG vectors' layout [ns][nt][nz][px], px = nx rounded
 * up to a multiple of 32, pad columns zero (the form the learned CG packs its residuals in). */
ESI_API esi_status esi_pc_pack(esi_ctx *ctx, const void *field_dev, double lambda, double eps,
                               int scale, int pitched, void *img_dev);

/* A stand-alone network for h x w images, batches of up to max_batch, on a stream. */
ESI_API esi_status esi_pc_create(esi_pc **out, int h, int w, int max_batch, void *stream);
ESI_API void esi_pc_destroy(esi_pc *pc);
ESI_API const char *esi_pc_last_error(const esi_pc *pc);
/* Parameters in and out (device FP32, layout above); setting them resets the Adam state. */
ESI_API esi_status esi_pc_set_params(esi_pc *pc, const float *params_dev);
ESI_API esi_status esi_pc_get_params(esi_pc *pc, float *params_dev);
/* y = rms(x) U(x / rms(x)) for n images: x BF16 [n][h][w][16], y FP32 [n][h][w][16]. */
ESI_API esi_status esi_pc_apply(esi_pc *pc, const void *in_dev, int n, float *y_dev);
/* Training objective on n pairs (x = packed scaled residual, e = packed CG error):
 * loss = mean_i (1 - <x_i + y_i, e_i>^2 / (|x_i + y_i|^2 |e_i|^2)), y as in esi_pc_apply.  Writes the
 * parameter gradient (device FP32, may be NULL) and the loss (host, may be NULL). */
ESI_API esi_status esi_pc_grad(esi_pc *pc, const void *in_dev, const void *target_dev, int n,
                               float *grad_dev, double *loss);
/* Vector-Jacobian product of the network: grad_dev (FP32, esi_pc_param_count() values,
 * overwritten) = d<gy, y(in)>/d(parameters) for the output gradient gy_dev (device FP32,
 * the layout of esi_pc_apply's y) of the n images in_dev.  Lets a caller train the network
 * on an objective the library does not compute itself (the preconditioner section of the
 * conclusion leaves the objective open). */
ESI_API esi_status esi_pc_vjp(esi_pc *pc, const void *in_dev, const float *gy_dev, int n,
                              float *grad_dev);
/* esi_pc_grad followed by one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at rate lr. */
ESI_API esi_status esi_pc_train_step(esi_pc *pc, const void *in_dev, const void *target_dev,
                                     int n, double lr, double *loss);

/* Static string for a status code. */
ESI_API const char *esi_status_string(esi_status s);

/* Last error message of a context ("" when none); valid until the next call. */
ESI_API const char *esi_last_error(const esi_ctx *ctx);

/* Number of kernels this context has launched since creation (for accounting). */
ESI_API long long esi_launch_count(const esi_ctx *ctx);

/*
 * Kernel timing (tracing).  When enabled, every run of consecutive launches of one
 * kernel variant (a propagation loop, a CG vector pass) is bracketed by CUDA events on
 * the context stream and accumulated per variant.  esi_get_profile synchronises the
 * stream, fills up to max entries and returns the number of variants seen; the
 * counters reset when profiling is (re-)enabled.
 */
typedef struct esi_kernel_stat {
    char name[48];       /* e.g. "fd2_step[CGP|SMP]" */
    long long launches;  /* kernel launches */
    long long cells;     /* cell updates (or vector elements) processed */
    double bytes_per_cell;  /* algorithmic HBM bytes per cell update / element */
    double ms;           /* accumulated device time between the bracketing events */
} esi_kernel_stat;

ESI_API esi_status esi_set_profiling(esi_ctx *ctx, int on);
ESI_API int esi_get_profile(esi_ctx *ctx, esi_kernel_stat *out, int max);

#ifdef __cplusplus
}
#endif
#endif /* ESI_H */
