/*
 * ppe.h -- C ABI of the GB300 pressure-Poisson (PPE) hot path.
 *
 * The library solves the pressure Poisson equation of a fractional-step
 * immersed-boundary flow solver,
 *
 *     M dp = S                                   (Sec. 2.1 Eq. 6; Sec. 2.2 Eq. 10)
 *
 * on a 2-D tensor-product, cell-centred, non-uniform Cartesian grid with
 * homogeneous Neumann walls.  M is the variable-spacing 5-point Laplacian
 * D*G: the face gradient is (p[i+1]-p[i]) / ((dx[i]+dx[i+1])/2) and the
 * divergence divides the net face flux by the cell width.  Internally the
 * symmetric positive semidefinite form A = -V*M, b = -V*S (V = dx[i]*dy[j])
 * is solved, with the constant null space projected out.
 *
 * Solvers (Sec. 2.2, Sec. 2.5):
 *   PPE_MODE_PCG     Jacobi-preconditioned conjugate gradient.
 *   PPE_MODE_HYBRID  HyDEA: up to num_cg CG-type iterations alternate with up
 *                    to num_dlsm deep-learning line-search (DLSM) steps
 *                    e = NN(r), alpha = r.e / e.(A e), x += alpha e
 *                    (Eqs. 11-12), until the residual criterion holds.
 *
 * Conventions for every call:
 *   - Fields are row-major [ny][nx] (x index contiguous), FP64 unless stated.
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     "host" pointers are ordinary host memory.
 *   - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *     default stream).
 *   - Every call returns a ppe_status and never aborts the process.  On
 *     failure ppe_last_error() returns a message for the calling thread.
 *   - Handles are not thread-safe; distinct handles may be used concurrently
 *     on distinct streams.
 */
#ifndef PPE_GB300_H
#define PPE_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PPE_API __attribute__((visibility("default")))
#else
#define PPE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PPE_OK = 0,
    PPE_ERR_ARG = 1,               /* invalid argument (null, size, layout)            */
    PPE_ERR_CUDA = 2,              /* a CUDA runtime/driver call failed                */
    PPE_ERR_NOMEM = 3,             /* device or host allocation failed                 */
    PPE_ERR_INCOMPATIBLE_RHS = 4,  /* |sum V*S| > 1e-6 * sum |V*S|: no Neumann solution */
    PPE_ERR_NOT_CONVERGED = 5,     /* iteration cap reached; x holds the best iterate   */
    PPE_ERR_TIMEOUT = 6,           /* a bounded device-side wait expired               */
    PPE_ERR_NAN = 7,               /* non-finite value met inside the solve            */
    PPE_ERR_NO_NET = 8,            /* hybrid mode requested without a network          */
    PPE_ERR_FORMAT = 9             /* malformed weights file                           */
} ppe_status;

typedef enum { PPE_BC_NEUMANN = 0 } ppe_bc;          /* dp: zero normal flux on all walls */
typedef enum { PPE_MODE_PCG = 0, PPE_MODE_HYBRID = 1 } ppe_mode;
typedef enum {
    PPE_PREC_FP64 = 0,   /* every inner vector and operation in FP64                        */
    PPE_PREC_MIXED = 1   /* FP32 inner iterations, FP64 true residual + iterative refinement */
} ppe_precision;

typedef struct ppe_grid ppe_grid;
typedef struct ppe_net ppe_net;

/* Per-solve report.  Iteration counts follow the paper's convention: a
 * CG-type iteration or a DLSM step each count as one iteration. */
typedef struct {
    int32_t status;         /* ppe_status of the solve                                  */
    int32_t iters_pcg;      /* CG-type iterations                                        */
    int32_t iters_dlsm;     /* DLSM steps applied                                        */
    int32_t dlsm_skipped;   /* DLSM directions rejected by the curvature guard           */
    int32_t refinements;    /* FP64 true-residual evaluations                            */
    int32_t fell_back;      /* 1 if hybrid mode exhausted its budget and finished as PCG */
    int32_t net_calls;      /* network inferences run                                    */
    int32_t launches;       /* solver-kernel launches                                    */
    double rel_res_true;    /* ||P(b - A x)|| / ||P b|| in FP64 at exit                  */
    double incompat;        /* |sum b| / sum |b| before projection                       */
    double ms_total;        /* wall time of the call on its stream (ms)                  */
    double ms_net;          /* device time from each segment that asked for a DLSM
                               direction to the segment that used it: the network
                               inference and the direction's mean removal (ms)         */
    double ms_pcg;          /* device time of the CG-type passes (Sec. 2.2; ms)          */
    double ms_dlsm;         /* device time of the DLSM passes: r.e, e.Ae and the update
                               of Eqs. 11-12 (ms)                                        */
    double ms_refine;       /* device time of the FP64 passes: statistics of b, true
                               residuals (iterative refinement), finalisation (ms)       */
    int32_t drive;          /* 0: the solve ran as one CUDA graph launch whose device-side
                               loop alternated solver segments and network branches
                               (no host round-trip per hybrid cycle); 1: the host
                               launched each segment and direction                       */
    int32_t precision_fallback; /* 1: the mixed solve's FP32 inner iteration stalled (three
                               refinements in a row failed to halve the true residual, as
                               happens once the system's conditioning exceeds what FP32
                               resolves) and the solve was continued in FP64 from there; the
                               counts and times include both parts                      */
} ppe_solve_info;

/* Solver options; ppe_default_options() fills the defaults shown. */
typedef struct {
    int32_t max_iters;      /* cap on CG-type + DLSM iterations per solve (200000)            */
    int32_t num_cg;         /* Num_CG-type: CG iterations per hybrid cycle (3; Sec. 2.2)      */
    int32_t num_dlsm;       /* Num_DLSM: DLSM steps per hybrid cycle (2; Sec. 2.2)            */
    int32_t hybrid_budget;  /* iterations after which hybrid mode continues as plain PCG      */
    double inner_rtol;      /* MIXED: FP32 residual drop that triggers an FP64 residual
                               replacement (0.3: measured on GB300, 3,660 iterations on the
                               512^2 refined-box grid against 4,338 at 0.1)                 */
    double dlsm_guard;      /* skip a DLSM step if e.Ae <= guard * e.e * max(diag A) (1e-10)   */
    int32_t blocks_per_sm;  /* cap on persistent-kernel CTAs per SM (2; 0 = as many as fit;
                               the solver kernels fit one)                                    */
    int32_t keep_dir_after_dlsm; /* 0: every CG-type phase restarts with p = z (Sec. 2.2 workflow,
                               as a fresh KSPSolve); 1: CG directions continue across DLSM steps */
    int32_t iter_pass;      /* MIXED precision only: 0 = the autotuned choice if there is one
                               (ppe_autotune), else by size (default); 1 = tiles of 128 cells
                               by 16 or 8 rows (tile_rows) shared by a whole CTA; 2 = streaming (each warp marches
                               down a 120-wide strip; for grids far larger than the number of
                               CTAs).  Same arithmetic, same results up to rounding order.     */
    int32_t dlsm_stall_limit; /* hybrid: continue as plain PCG after this many unprofitable DLSM
                               steps in a row (6; 0 = never).  A step is unprofitable when it
                               removes less of the error's A-norm energy, (r.e)^2 / (e.Ae),
                               than dlsm_cost_iters iterations of the CG phase before it
                               remove at their mean (alpha r.u each).  Not in the paper: a
                               guard against a network that does not pay for its inference. */
    int32_t dlsm_cost_iters;  /* a DLSM step's cost in CG iterations for that test (16)        */
    int32_t spin_limit_ms;  /* bound on every device-side wait of the solver kernel, in ms (2000).
                               On expiry the kernel returns and the solve reports PPE_ERR_TIMEOUT. */
    int32_t host_loop;      /* 0: one graph launch with device-side alternation (default);
                               1: the host launches each solver segment and network direction
                               (always so for a grid with a direction source)                 */
    int32_t debug_skip_block; /* test hook, 0 = off: block debug_skip_block - 1 of the solver
                               kernel withholds its partial sums at its second step, so the
                               other blocks' bounded waits expire (PPE_ERR_TIMEOUT)           */
    int32_t preconditioner; /* CG-type partner of PPE_MODE_PCG (Sec. 2.6): 0 = Jacobi (default);
                               1 = multigrid (the paper's MGPCG analogue on the tensor grid): CG
                               preconditioned by one V-cycle per iteration -- cells merged
                               pairwise per axis, the operator re-discretised on every level,
                               linear prolongation with restriction its transpose, damped
                               alternating line-Jacobi smoothing, pseudo-inverse on a coarsest
                               level of at most 256 cells.  Runs FP32 inner iterations with
                               FP64 refinement (PPE_PREC_MIXED); single systems only
                               (ppe_solve; PPE_ERR_ARG for hybrid mode, FP64 precision or a
                               batch).  The hierarchy is built on the grid's first multigrid
                               solve (allocates; later solves reuse it).                     */
    int32_t debug_force_stall; /* test hook, 0 = off: a mixed-precision solve counts every
                               refinement after the first as one that failed to halve the
                               true residual, so its stall rule ends the FP32 iteration and
                               the solve continues in FP64 from the iterate
                               (ppe_solve_info.precision_fallback = 1)                      */
    int32_t tile_rows;      /* rows of a tile-cooperative tile: 0 = by size (default: a small
                               grid takes 8 or 4 rows, spreading over two or four times the
                               CTAs, while the tiles fit one per SM; else 16); 4, 8 or 16 to
                               choose.  Any precision; same arithmetic, same results up to
                               rounding order.  Ignored by the streaming pass (16).          */
    int32_t reserved[2];
} ppe_solve_opts;

PPE_API void ppe_default_options(ppe_solve_opts *opts);

/*
 * Create a grid handle.
 *   nx, ny   cell counts (>= 1 each; nx*ny < 2^31)
 *   dx, dy   host arrays of nx / ny positive, finite cell widths (copied)
 *   bc       PPE_BC_NEUMANN
 *   mask     nullable host array [ny][nx] of 0/1 body flags (copied).  The
 *            operator never depends on it (Sec. 2.6: the PPE matrix of the
 *            decoupled IB projection method is body-independent); it is kept
 *            for the network's optional use and for reporting.
 *   out      receives the handle.  The handle owns its device workspaces
 *            (allocated here, on the current device) until ppe_destroy_grid.
 */
PPE_API ppe_status ppe_create_grid(int nx, int ny, const double *dx, const double *dy,
                           ppe_bc bc, const uint8_t *mask, ppe_grid **out);
PPE_API void ppe_destroy_grid(ppe_grid *grid);
PPE_API ppe_status ppe_grid_shape(const ppe_grid *grid, int *nx, int *ny);
PPE_API ppe_status ppe_set_options(ppe_grid *grid, const ppe_solve_opts *opts);

/*
 * y = A x with A = -V*M the volume-scaled operator (Sec. 2.1 Eq. 6, scaled
 * by -V to make it symmetric), FP64.  x, y: device [ny][nx]; may not alias.
 */
PPE_API ppe_status ppe_apply(ppe_grid *grid, const double *x_dev, double *y_dev, void *stream);
/* r = -V*S - A x (FP64, no projection): the residual of the scaled system for
 * source S and iterate x.  All device [ny][nx]; r may not alias S or x. */
PPE_API ppe_status ppe_residual(ppe_grid *grid, const double *S_dev, const double *x_dev, double *r_dev,
                                void *stream);

/*
 * The projection step around the PPE (Sec. 2.1 Eqs. 6-8) on the staggered
 * grid: u device [ny][nx+1] (x faces; face i of row j lies between cells i-1
 * and i), v device [ny+1][nx] (y faces), FP64.  The wall faces hold the
 * prescribed normal velocity.
 *   ppe_source:  S = (D u* - bc2) / dt, the PPE source of Eq. 6 (device
 *                [ny][nx]): the whole divergence of u* over dt, the wall faces'
 *                prescribed normal velocity (the bc2 part) included.  It is
 *                compatible when the net flux through the walls vanishes.
 *   ppe_project: u <- u - dt G dp, v <- v - dt G dp on the interior faces
 *                (Eq. 7) and, if p is not NULL, p <- p + dp (Eq. 8).  The wall
 *                faces are not changed.
 * D G equals the operator M that ppe_solve inverts, so after ppe_solve on S
 * and ppe_project the interior divergence of (u, v) vanishes to the solve's
 * tolerance.  Kernels on `stream`; no synchronisation.  dt > 0.
 */
PPE_API ppe_status ppe_source(ppe_grid *grid, const double *u_dev, const double *v_dev, double dt, double *S_dev,
                              void *stream);
PPE_API ppe_status ppe_project(ppe_grid *grid, const double *dp_dev, double dt, double *u_dev, double *v_dev,
                               double *p_dev, void *stream);

/*
 * Solve M x = S (Eq. 10) to ||P(b - A x)|| <= tol_rel * ||P b||.
 *   rhs_dev  device [ny][nx]: the source S (e.g. (D u* - bc2) / dt).  Must be
 *            compatible: |sum V*S| <= 1e-6 * sum |V*S|; smaller defects are
 *            projected out and reported in info->incompat.
 *   x_dev    device [ny][nx]: in: initial guess (warm start), out: the
 *            solution with zero volume-weighted mean.  On
 *            PPE_ERR_NOT_CONVERGED it holds the best iterate.
 *   tol_rel  relative residual target (> 0), e.g. 1e-8.
 *   mode     PPE_MODE_PCG or PPE_MODE_HYBRID (needs net attached to grid).
 *   precision PPE_PREC_FP64 or PPE_PREC_MIXED.
 *   net      nullable for PCG; for HYBRID a network attached with net_attach.
 *   stream   cudaStream_t as void*.  The call synchronises that stream
 *            before it returns (the report is read back).
 *   info     nullable; receives the report.
 */
PPE_API ppe_status ppe_solve(ppe_grid *grid, const double *rhs_dev, double *x_dev,
                     double tol_rel, ppe_mode mode, ppe_precision precision,
                     ppe_net *net, void *stream, ppe_solve_info *info);

/*
 * Solve n independent systems in one persistent launch (Sec. 2.2 applied to
 * a batch).  grids[i], rhs_dev[i], x_dev[i] as in ppe_solve.  Systems retire
 * independently when converged.  info: nullable array of n reports.
 */
PPE_API ppe_status ppe_solve_batch(int n, ppe_grid *const *grids, const double *const *rhs_dev,
                           double *const *x_dev, double tol_rel, ppe_mode mode,
                           ppe_precision precision, ppe_net *net, void *stream,
                           ppe_solve_info *info);

/*
 * Direction source for the DLSM steps in place of the network (validation
 * with known directions, or a user's own predictor).  When set on a grid,
 * hybrid solves on it call fn instead of the network: fn receives the
 * normalised residual r_hat = (r - mean r) / ||r - mean r|| (device FP32
 * [ny][nx], valid during the call) and must write the direction e (device
 * FP32 [ny][nx]) in stream order on `stream` before returning.  fn = NULL
 * removes the source.  The grid owns the two FP32 staging buffers.
 */
typedef void (*ppe_direction_fn)(void *user, const float *r_hat_dev, float *e_dev, int nx, int ny, void *stream);
PPE_API ppe_status ppe_set_direction_source(ppe_grid *grid, ppe_direction_fn fn, void *user);

/*
 * Allocation-free plain-PCG solve.  The paper has no counterpart: this entry
 * point serves callers that cannot allocate device memory -- a host whose
 * device memory is reserved up front by its own pool allocator, a loop that
 * must not allocate after initialisation, a plugin whose host forbids device
 * allocations.  It runs the same persistent solver kernel as ppe_solve but
 * takes all scratch from one fixed-size __device__ array inside the library
 * (about 3.3 MB, held by every GPU that loads the library until exit), and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   nx, ny    1 <= nx, ny <= 4096 and nx*ny <= 65536; larger grids return
 *             PPE_ERR_ARG with a message naming the limit.
 *   dx, dy    host arrays of the cell widths (copied into the array).
 *   rhs_dev, x_dev, tol_rel, precision, stream, info: as in ppe_solve
 *             (mode is PPE_MODE_PCG).
 * Every call shares the array and it keeps the last call's contents; each
 * call clears what must start at zero.  Calls whose work overlaps on the GPU
 * (different streams, or different host threads) race: serialise them.  The
 * first call on a device looks the array's address up with that device
 * current; make it before any stream capture.  The call synchronises stream.
 */
PPE_API ppe_status ppe_solve_noalloc(int nx, int ny, const double *dx, const double *dy, const double *rhs_dev,
                                     double *x_dev, double tol_rel, ppe_precision precision, void *stream,
                                     ppe_solve_info *info);

/*
 * Autotuner of the persistent kernel's launch configuration (the paper has no
 * counterpart).  In MIXED precision it times, on this grid, the iteration-pass
 * variants of ppe_solve_opts.iter_pass (tile-cooperative on tiles of 16, 8
 * and 4 rows, and streaming) by capped solves of a smooth synthetic source,
 * and keeps the fastest: on the grid (used by ppe_solve when
 * opts.iter_pass, and for the height opts.tile_rows, are 0) and in a
 * process-wide table keyed by (nx, ny) that later grids of the same shape
 * use.  If the environment variable PPE_TUNE_CACHE names a file, the table
 * is read from it on first use and each new entry is appended (one JSON
 * object per line).  The call allocates two temporary device fields of
 * nx*ny doubles, runs about thirty solves of at most 40 iterations and
 * synchronises `stream`.
 */
typedef struct {
    int32_t iter_pass;       /* chosen variant: 1 tile-cooperative, 2 streaming          */
    int32_t blocks_per_sm;   /* chosen CTAs per SM (0: as many as fit)                    */
    double us_per_iter[3];   /* measured: tile-cooperative (its fastest height),
                                (unused), streaming                                      */
    int32_t tile_rows;       /* fastest tile-cooperative height: 16, 8 or 4 rows          */
    int32_t reserved[3];
} ppe_tune_report;
PPE_API ppe_status ppe_autotune(ppe_grid *grid, void *stream, ppe_tune_report *report);

/* Message describing the last failure on the calling thread ("" if none). */
PPE_API const char *ppe_last_error(void);
/* Library build identification, e.g. "ppe-gb300 sm_103a". */
PPE_API const char *ppe_version(void);

/* ------------------------------------------------------------------------
 * Grid-spacing-aware DeepONet (Sec. 2.4): U-Net branch of Mesh-Convs whose
 * inputs are scaled by eta = exp(-Phi(Delta)^2) (Eqs. 16-17), Delta being the
 * level-K map of distances to the four neighbours; coordinate trunk; output
 * sum_c branch_c * trunk_c + bias.
 * ------------------------------------------------------------------------ */
#define PPE_NET_MAX_LEVELS 6
typedef struct {
    int32_t levels;                          /* U-Net levels (2..6)                         */
    int32_t widths[PPE_NET_MAX_LEVELS];      /* channels per level (multiples of 16)        */
    int32_t c_last;                          /* branch / trunk feature count                 */
    int32_t trunk_hidden[2];                 /* trunk MLP hidden widths (2 -> h0 -> h1 -> c_last) */
    int32_t phi_hidden;                      /* hidden width of each Mesh-Conv weight network (1..16) */
    int32_t mesh_conv;                       /* 1: Mesh-Conv; 0: standard convolution (eta = 1) */
    int32_t reserved[4];
} ppe_net_config;

/* Defaults: 4 levels, widths 32/64/128/256, c_last 100, trunk 100/200,
 * phi_hidden 16, mesh_conv 1. */
PPE_API void net_default_config(ppe_net_config *cfg);
/* Create a network with seeded initial parameters (host-side generator). */
PPE_API ppe_status net_create(const ppe_net_config *cfg, uint64_t seed, ppe_net **out);
PPE_API void net_destroy(ppe_net *net);
/* Number of FP32 parameters; the flat order is: for every Mesh-Conv in
 * execution order (enc0a, enc0b, ..., up{L-2}, dec{L-2}a, dec{L-2}b, ..., dec0b)
 * w[Cout][Cin][3][3], b[Cout], phi1.w[H][4], phi1.b[H], phi2.w[H], phi2.b[1];
 * then head.w[c_last][w0], head.b[c_last]; trunk0.w[h0][2], trunk0.b[h0],
 * trunk1.w[h1][h0], trunk1.b[h1], trunk2.w[c_last][h1], trunk2.b[c_last];
 * out.b[1]. */
PPE_API ppe_status net_param_count(const ppe_net *net, int64_t *count);
PPE_API ppe_status net_get_config(const ppe_net *net, ppe_net_config *cfg);
/* Copy parameters in/out (host FP32 arrays of net_param_count entries). */
PPE_API ppe_status net_set_params(ppe_net *net, const float *params, int64_t count);
PPE_API ppe_status net_get_params(const ppe_net *net, float *params, int64_t count);
/* Binary weights file: magic "PPENET01", version, flags (bit 0: Adam moments
 * present), config, parameter count, step, parameters, [Adam m, v], CRC32.
 * net_save writes the moments (to resume training), net_save_params only the
 * parameters (for inference).  net_load reads either and returns
 * PPE_ERR_FORMAT for a malformed or corrupted file.  A file with moments
 * resumes at its saved step; one without them starts a fresh optimiser at
 * step 0 (zero moments, the cosine schedule from lr0). */
PPE_API ppe_status net_save(const ppe_net *net, const char *path);
PPE_API ppe_status net_save_params(const ppe_net *net, const char *path);
PPE_API ppe_status net_load(const char *path, ppe_net **out);
/* Build the per-grid caches (distance maps, eta per layer, trunk features)
 * for this grid; required before net_infer / hybrid solves on it. */
PPE_API ppe_status net_attach(ppe_net *net, ppe_grid *grid);
/* e = NN(r) on the grid (Sec. 2.2 Eq. 11's e^NN).  r_dev, e_dev: device FP32
 * [ny][nx].  The network sees r exactly as given (the solver feeds r/||r||). */
PPE_API ppe_status net_infer(ppe_net *net, ppe_grid *grid, const float *r_dev, float *e_dev, void *stream);
/* Same for a batch of `batch` inputs stored back to back ([batch][ny][nx]). */
PPE_API ppe_status net_infer_batch(ppe_net *net, ppe_grid *grid, int batch, const float *r_dev, float *e_dev,
                                   void *stream);

/* Training hyper-parameters (Sec. 2.4: Adam with SAM, cosine decay). */
typedef struct {
    double lr0;            /* initial learning rate (2e-4)                               */
    int64_t total_steps;   /* length of the cosine schedule (steps)                      */
    double rho;            /* SAM perturbation radius (2e-4); 0 disables SAM             */
    double beta1, beta2;   /* Adam moment decay (0.9, 0.999)                             */
    double eps;            /* Adam epsilon (1e-8)                                        */
    int32_t reserved[8];
} ppe_train_hparams;

PPE_API void net_default_hparams(ppe_train_hparams *hp);
/*
 * One training step on a batch of `batch` right-hand sides R (device FP32
 * [batch][ny][nx], each R made unit-norm by the caller, Eq. 14) on one grid:
 * loss L = mean over the batch and the nx*ny cells of (R - A NN(R))^2 with
 * A = -V M the volume-scaled operator (Eq. 18); gradient by the network's
 * backward kernels; SAM perturbation w + rho g / ||g|| and a second
 * gradient there; Adam update with learning rate
 * 0.5 lr0 (1 + cos(pi t / total_steps)).  loss_out (host, nullable)
 * receives L at the unperturbed weights; the call synchronises `stream`.
 * The network must be attached to the grid.
 */
PPE_API ppe_status net_train_step(ppe_net *net, ppe_grid *grid, int batch, const float *R_dev,
                                  const ppe_train_hparams *hp, void *stream, double *loss_out);
/* Test hook: loss (Eq. 18) and its gradient at the current parameters
 * (grad_host: nullable host FP32 array of net_param_count entries). */
PPE_API ppe_status net_loss_grad(ppe_net *net, ppe_grid *grid, int batch, const float *R_dev, void *stream,
                                 double *loss_out, float *grad_host);
/* Number of optimiser steps taken (the t of the schedule). */
PPE_API ppe_status net_get_step(const ppe_net *net, int64_t *step);

/* Test hook: one V-cycle of the multigrid partner (see ppe_solve_opts.preconditioner)
 * applied to r (device FP32 [ny][nx], zero sum); z (device FP32 [ny][nx]) receives it.
 * Builds the grid's hierarchy on first use. */
PPE_API ppe_status ppe_debug_mg_vcycle(ppe_grid *grid, const float *r_dev, float *z_dev, void *stream);

/* Test hook: one 3x3 convolution (zero padding 1, no activation) of a BF16
 * NHWC input in_bf16 [B][H][W][cin] with packed BF16 weights
 * w_bf16 [cout][9][cin] (tap = 3*ky + kx) and FP32 bias [cout] (nullable);
 * FP32 output out [B][H][W][cout].  impl 0: tensor-core (tcgen05) kernel,
 * 1: CUDA-core kernel.  All pointers are device pointers. */
PPE_API ppe_status ppe_debug_conv3x3(const void *in_bf16, const void *w_bf16, const float *bias, int B, int H, int W,
                                     int cin, int cout, float *out, int impl, void *stream);

/* Test hook: the weight gradient of one 3x3 convolution (Sec. 2.4, the
 * training step's backward), added into dW [cout][cin][9] (FP32, tap =
 * 3*ky + kx): dW[co][ci][t] += sum over pixels of dZ[p][co] * X[p + t][ci],
 * X zero outside the image.  dZ_bf16 [B][H][W][cout] and X_bf16
 * [B][H][W][cin] are BF16 NHWC.  impl 0: tensor-core (tcgen05) kernel
 * (PPE_ERR_ARG for channel counts it does not take), 1: CUDA-core kernel.
 * All pointers are device pointers. */
PPE_API ppe_status ppe_debug_wgrad(const void *dZ_bf16, const void *X_bf16, int B, int H, int W, int cin, int cout,
                                   float *dW, int impl, void *stream);

/* Test hook: one GEMM of the DeepONet trunk (Sec. 2.4; the trunk's layers
 * and their backward), FP32 in and out:
 *   C[m][n] = act(sum_k A(m, k) B(k, n) + bias[m]) (+ C[m][n] if accumulate)
 * with A(m, k) = transA ? A[k*lda + m] : A[m*lda + k], B(k, n) = transB ?
 * B[n*ldb + k] : B[k*ldb + n], C[m*ldc + n], act 0 (identity) or 1 (tanh),
 * bias nullable [M].  impl 0: the tensor-core (tcgen05, TF32 operands) form
 * when the shape is one of the trunk's (N >= 1024 pixels with M, K <= 256
 * and !transB; or K >= 4096 pixels, !transA, transB, 16 <= N <= 256, no bias
 * and act 0), the thin forms on the CUDA cores where they apply (3: N <= 4
 * with K >= 1024, !transA, no bias, act 0; 4: K <= 4 with N >= 1024,
 * !transB), else the general CUDA-core kernel; 1: always the general
 * CUDA-core kernel.  *form (nullable) receives the form used (1-4, 0 the
 * general kernel).  All array pointers are device pointers. */
/* Test hook: the solver's choice of iteration pass and tile height for a
 * solve (no CUDA calls): precision PPE_PREC_FP64 or PPE_PREC_MIXED,
 * ppe_solve_opts.iter_pass (0-2) and tile_rows (0, 4, 8, 16), the grid's
 * count of 128x16 tiles and the device's SM count.  *pass_out receives 1
 * (tile-cooperative) or 2 (streaming), *rows_out the tile height (16 for
 * the streaming pass).  PPE_ERR_ARG for arguments out of range. */
PPE_API ppe_status ppe_debug_pick_variant(int precision, int iter_pass, int ntiles, int tile_rows, int sms,
                                          int *pass_out, int *rows_out);

/* Test hook: the tile-range planner of the persistent solver kernel (the
 * host and the device's batch re-planning run the same function; no CUDA
 * calls).  ntiles[n]: tiles of each system (0: none); max_blocks: blocks of
 * the launch; max_ranges: capacity of `ranges` (four int32 per range: first
 * tile, end tile, first system, last system).  Writes tile0[n] (prefix
 * sums), blk0[n] and nparts[n] (the ranges whose tiles include the system),
 * part0[n] (its first record slot), the ranges, *nranges (-1 if more than
 * max_ranges would be needed) and *nslots (record slots).  A range holds
 * tiles of at most 8 systems. */
PPE_API ppe_status ppe_debug_plan_ranges(int n, const int32_t *ntiles, int max_blocks, int max_ranges,
                                         int32_t *tile0, int32_t *blk0, int32_t *nparts, int32_t *part0,
                                         int32_t *ranges, int *nranges, int *nslots);

PPE_API ppe_status ppe_debug_gemm(int M, int N, int K, const float *A, int lda, int transA, const float *B, int ldb,
                                  int transB, float *C, int ldc, const float *bias, int act, int accumulate, int impl,
                                  int *form, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PPE_GB300_H */
