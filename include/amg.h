/*
 * amg.h -- C ABI of the GB300 (sm_103a) PCG + aggregation-AMG solver.
 *
 * The library solves A x = b (Eq. linearsystem, Sec. 2.1) for a sparse
 * symmetric positive-definite A by the conjugate gradient method (Sec. 3,
 * flexible CG) preconditioned by one V(1,1) cycle of aggregation-based
 * algebraic multigrid (Eq. amg, Sec. 2.3).  The hierarchy is built on the GPU:
 * pairwise aggregation by weighted matching (Sec. 2.3, "Coupled Aggregation
 * Based on Compatible Weighted Matching"), the Galerkin product
 * A_{l+1} = P_l^T A_l P_l (Sec. 2.3) and the l1-Jacobi smoother (Sec. 2.3,
 * "GPU enabled smoothers"); the coarsest level is solved by dense Cholesky.
 *
 * Conventions shared by every entry point:
 *  - Pointers documented "device" point to GPU global memory of the current
 *    device; "host" pointers to CPU memory.  The caller owns every buffer it
 *    passes; the library never frees or retains caller buffers after a call
 *    returns (amg_setup copies the matrix).
 *  - A handle owns all internal device memory (hierarchy, work vectors,
 *    captured CUDA graphs) until amg_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls documented "synchronous" wait for it.
 *  - Every function returns an int status: 0 success, >0 a soft condition
 *    (AMG_NOT_CONVERGED), <0 an error (the AMG_ERR_* codes below), mirroring
 *    the `info` argument of the paper's library calls (Sec. 2.1).  After an
 *    error the handle stays valid unless the status is AMG_ERR_CUDA.
 *  - Matrices are CSR with int64 row pointers, int32 column indices sorted
 *    ascending within each row, float64 values, zero-based.  A must be
 *    symmetric bit for bit (a_ij == a_ji), have a positive diagonal entry
 *    stored in every row, and be SPD.
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* amg_stream_t; /* same object as cudaStream_t */

/* ------------------------------------------------------------ status codes */
#define AMG_OK 0
#define AMG_NOT_CONVERGED 1      /* PCG hit maxit before reaching tol */
#define AMG_ERR_ARG (-1)         /* bad size, null pointer or option */
#define AMG_ERR_NOT_SPD (-2)     /* coarse Cholesky pivot <= 0 */
#define AMG_ERR_BREAKDOWN (-3)   /* PCG: p^T A p <= 0 */
#define AMG_ERR_NAN (-4)         /* NaN/Inf in a PCG scalar */
#define AMG_ERR_CUDA (-5)        /* a CUDA runtime call or launch failed */
#define AMG_ERR_OOM (-6)         /* device allocation failed */
#define AMG_ERR_DEVICE_CHECK (-7) /* a kernel's own bounds/limit check fired */
#define AMG_ERR_UNSUPPORTED (-8) /* input outside the implemented limits */

/* Value precision of the stored hierarchy and of the V-cycle arithmetic. */
#define AMG_PREC_F64 0
#define AMG_PREC_F32 1

/* Flexible-CG beta choice (Sec. 3; flexible CG with truncation 1). */
#define PCG_BETA_AUTO (-1)     /* FR for an F64 hierarchy, flexible otherwise */
#define PCG_BETA_FR 0          /* beta = (r+, z+) / (r, z) */
#define PCG_BETA_FLEXIBLE 1    /* beta = -(z+, q) / (p, q), q = A p */

typedef struct amg_handle amg_handle;

/* A sparse matrix in CSR (device pointers, see conventions above). */
typedef struct amg_csr {
  int64_t n;              /* rows = columns */
  int64_t nnz;            /* stored entries, == rowptr[n] - rowptr[0] */
  const int64_t* rowptr;  /* device, n + 1 */
  const int32_t* col;     /* device, nnz */
  const double* val;      /* device, nnz */
} amg_csr;

/* Hierarchy options (Sec. 2.3 prec%set keys in brackets). */
typedef struct amg_options {
  int sweeps;            /* matching sweeps per level; aggregates <= 2^sweeps
                            [aggr_size]; 1..3, default 2 */
  int max_levels;        /* level cap, default 30 */
  int64_t max_coarse;    /* stop once a level has <= max_coarse rows, default 200 */
  double stall_ratio;    /* stop when n_{l+1} > stall_ratio * n_l, default 0.9 */
  int64_t max_dense;     /* largest coarsest block (system) factored densely,
                            default 8192, at most 16384 */
  int precision;         /* AMG_PREC_F64 (default) or AMG_PREC_F32 */
  int bf16_from_level;   /* with F32: levels >= this keep BF16 values; 0 = off */
  int slice_height;      /* sliced-ELL rows per slice 1/2/4/8/16/32/64; 0 =
                            default: 32 / threads_per_row (one slice per warp).
                            Any other height decouples the slices from the
                            warps (a warp covers 32 / threads_per_row rows of
                            one or several slices); not for batched systems,
                            which always use 32 / threads_per_row */
  int threads_per_row;   /* 1/2/4/8/16/32 threads per row; 0 = default: 32 /
                            slice_height if that is set, else 1, more on levels
                            whose rows average 64 entries or more (about one
                            thread per 16) */
  int autotune;          /* 1: choose slice height and threads per row per level
                            by timing the level's kernels at setup: threads per
                            row 1/2/4/8 (16, 32 on wide rows) x slice heights
                            8/16/32/64 and 32 / threads per row (batched systems:
                            the latter only); choices are kept for the process,
                            keyed by rows, entries per row and value type */
  int64_t tail_rows;     /* levels (other than level 0) with at most this many
                            rows, and the coarsest solve, run as one persistent
                            launch instead of one launch per step: one CTA when
                            the largest of them has at most 16384 rows (and the
                            coarsest level is one block), else a cooperative
                            grid with bounded grid barriers.  Same results bit
                            for bit.  0 = off; default 1024 */
  int smooth_sweeps;     /* l1-Jacobi sweeps nu_0 before and after the coarse
                            correction on level 0, 1..8; default 1 (V(1,1)) */
  int variable_cycle;    /* 1: nu_l = nu_0 * 2^l sweeps on level l, the variable
                            V-cycle of Sec. 3 (VMATCH); 0 (default): nu_0 on
                            every level */
  int coarse_solver;     /* 0 (default): dense Cholesky of the coarsest level;
                            1: PCG preconditioned by its l1-Jacobi scaling
                            (Sec. 3, VBM/VMATCH coarsest solver), one CUDA block,
                            FP64; not for batched systems */
  int coarse_maxit;      /* PCG coarsest solve: iteration cap, default 40 */
  double coarse_tol;     /* PCG coarsest solve: stop at ||r|| <= tol ||b||,
                            default 1e-4 (0: run coarse_maxit iterations) */
  int compress_columns;  /* 1: store 2-byte column offsets where every slice
                            allows (see amg_level_layout); 0 (default): plain
                            4-byte indices.  Same results bit for bit; fewer
                            bytes, but slower on GB300 (more load instructions
                            for fewer bytes each) */
  int smooth_prolongator; /* 1: smoothed prolongators P = (I - w D^-1 A) P_hat,
                            w = 1 / ||D^-1 A||_inf, coarse matrices P^T (A P)
                            (Sec. 2.3, SMATCH); restriction by P^T, prolongation
                            by P.  Not with batched systems, several
                            right-hand sides, the two-grid loss or the
                            autotuner; tail_rows is ignored.  0 (default):
                            P_hat, the 0/1 aggregate map */
  int aggregation;       /* 0 (default): `sweeps` pairwise matching sweeps
                            (Sec. 2.3, coupled aggregation by compatible
                            weighted matching); 1: decoupled Vanek-Mandel-Brezina
                            aggregation (Sec. 2.3, VBM) with strength threshold
                            vbm_theta (`sweeps` is then unused) */
  double vbm_theta;      /* VBM strength threshold theta in [0, 1): j is a strong
                            neighbour of i when |a_ij| >= theta sqrt(a_ii a_jj);
                            default 0.01 */
  double prolongator_filter; /* with smooth_prolongator: > 0 smooths P with the
                            filtered matrix A_F (entries with |a_ij| < this x
                            sqrt(a_ii a_jj) dropped and added to the diagonal,
                            row sums kept): P = P_hat - w D^-1 A_F P_hat, D and
                            w from A; 0 (default): with A, the paper's formula.
                            In [0, 1) */
  int stream_ring;       /* 1 (default): the level kernels with FP64 or FP32
                            operator values of a one-system hierarchy with one
                            thread per row (pre- and post-smoother; the FP64
                            PCG product) stream each slice into a
                            shared-memory ring by bulk copies (cp.async.bulk,
                            mbarrier completion), with the library's number of
                            stages per warp; 2..4: with that many stages;
                            0: every lane loads its own entries.  Same rows bit
                            for bit; dot products may round differently
                            (another summation order) */
} amg_options;

/* PCG controls (Sec. 3, psb_krylov arguments). */
typedef struct pcg_options {
  double tol;            /* stop when ||r_k||_2 / ||b||_2 <= tol (recursive r) */
  int maxit;             /* iteration cap */
  int beta_form;         /* PCG_BETA_* */
  double* res_history;   /* host, maxit + 1 entries or NULL: relative residuals */
  double* x_history;     /* device, (maxit + 1) * n entries or NULL: iterates */
  int use_graph;         /* 1 (default via pcg_default_options): all iterations
                            as one captured CUDA graph whose conditional while
                            node runs the stopping test on the device (one host
                            wait per solve; without histories), else one graph
                            per iteration; 2: one graph per iteration, the host
                            testing after each; 0: plain launches.  Same
                            results in every mode */
} pcg_options;

/* Result of a solve. */
typedef struct pcg_stats {
  int iterations;        /* SpMV + update steps taken */
  int status;            /* same as the return value */
  double rel_residual;   /* recursive ||r|| / ||b|| at exit */
  double true_rel_residual; /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
  double solve_ms;       /* device time of the solve (CUDA events) */
} pcg_stats;

/* Fills `opt` with the defaults documented above. Never fails. */
int amg_default_options(amg_options* opt);
int pcg_default_options(pcg_options* opt);

/* Text for a status code (static storage). */
const char* amg_status_string(int status);

/*
 * Builds the AMG hierarchy of A on the GPU (Sec. 2.3 hierarchy build and
 * smoother build).  A: device CSR (see conventions).  opt: host, may be NULL
 * for defaults.  On success *H receives a new handle.  Synchronous.
 * Errors: AMG_ERR_ARG (n <= 0, nnz mismatch, bad option), AMG_ERR_NOT_SPD
 * (coarsest matrix not SPD), AMG_ERR_UNSUPPORTED (coarsening stalled above
 * max_dense rows, or a Galerkin row above the kernel's staging limit),
 * AMG_ERR_OOM, AMG_ERR_CUDA.  *H is NULL on error.
 */
int amg_setup(const amg_csr* A, const amg_options* opt, amg_stream_t stream, amg_handle** H);

/* Releases everything the handle owns. NULL is accepted. */
int amg_destroy(amg_handle* H);

/*
 * New coefficient values for the matrix H was built from, with the same
 * sparsity (Sec. 2.2: coefficients of a matrix whose structure is preserved
 * are updated in place, and the hierarchy is rebuilt on the assembled one).
 * Keeps H's aggregates and layout on every level (no matching); recomputes
 * the Galerkin values, l1-Jacobi scales (damping weights reset to 1), the
 * V-cycle operators and the coarsest factor.  A: device CSR with H's n, nnz,
 * row pointers and columns (checked by a fingerprint of the pattern).
 * Synchronous; H keeps its address, previously captured graphs are dropped.
 * Errors: AMG_ERR_ARG (NULL, other sizes or pattern), AMG_ERR_UNSUPPORTED
 * (batched handles), AMG_ERR_NOT_SPD, AMG_ERR_OOM, AMG_ERR_CUDA; on error H
 * is unchanged.
 */
int amg_update_values(amg_handle* H, const amg_csr* A, amg_stream_t stream);

/*
 * Replaces the level-0 smoother damping weights: s_i = omega_i * (1 / d_i)
 * with d_i the l1 row sum (Sec. 2.3, l1-Jacobi).  omega: device float32[n0],
 * each in (0, 2) (every such omega keeps the smoother A-convergent and the
 * V-cycle SPD; see mlp_set_omega_max), or NULL to restore omega == 1.
 * Levels >= 1 keep plain l1-Jacobi.  Asynchronous.
 */
int amg_set_smoother_weights(amg_handle* H, const float* omega, amg_stream_t stream);

/*
 * z = B r: one V(1,1) cycle with zero initial guess (Eq. amg).  r, z: device
 * float64[n0], distinct.  Asynchronous.
 */
int amg_vcycle_apply(const amg_handle* H, const double* r, double* z, amg_stream_t stream);

/*
 * y = alpha * A_l x + beta * y with the level-l matrix in FP64 (level 0 = the
 * input A).  x, y: device float64[n_l], distinct.  beta == 0 ignores y's
 * contents.  Asynchronous.
 */
int amg_spmv(const amg_handle* H, int level, double alpha, const double* x, double beta,
             double* y, amg_stream_t stream);

/*
 * Preconditioned CG for A x = b (Sec. 3; psb_krylov('FCG', ...)).
 * b: device float64[n0]; x: device float64[n0], initial guess in, solution
 * out.  o: host, NULL for defaults; st: host, may be NULL.  Synchronous.
 * Returns AMG_OK, AMG_NOT_CONVERGED, AMG_ERR_BREAKDOWN, AMG_ERR_NAN or an
 * error code.
 */
int pcg_solve(amg_handle* H, const double* b, double* x, const pcg_options* o, pcg_stats* st,
              amg_stream_t stream);

/* ----------------------------------------------------------- multiple right-hand sides */

/*
 * Z = B R for nrhs right-hand sides at once (Eq. amg applied column by
 * column).  R, Z: device float64, row-major n0 x nrhs (row i's nrhs values
 * contiguous), distinct.  1 <= nrhs <= 64.  Every column equals what
 * amg_vcycle_apply returns for it, bit for bit; each matrix entry is read
 * once for all columns.  The first call for a given nrhs allocates the
 * handle's multi-RHS workspace.  Needs a hierarchy of at least two levels
 * built by amg_setup (AMG_ERR_UNSUPPORTED otherwise).  Asynchronous.
 */
int amg_vcycle_apply_multi(amg_handle* H, int nrhs, const double* R, double* Z,
                           amg_stream_t stream);

/*
 * nrhs independent PCG solves of A X = B sharing every matrix read (blocked
 * SpMM; Sec. 3's method per column).  B, X: device float64 row-major
 * n0 x nrhs; X holds the initial guesses and receives the solutions.  Each
 * column has its own alpha, beta and stopping test; converged columns are
 * frozen.  st: host array of nrhs stats or NULL.  o->res_history and
 * o->x_history must be NULL.  Synchronous.  Returns the worst column status.
 */
int pcg_solve_multi(amg_handle* H, int nrhs, const double* B, double* X, const pcg_options* o,
                    pcg_stats* st, amg_stream_t stream);

/* ----------------------------------------------------------- batched systems */

/*
 * Builds one hierarchy for nsys independent SPD systems of uneven sizes (the
 * paper solves one system per call, Sec. 3; this batches many small ones).
 * A: host array of nsys CSR descriptors (device pointers, conventions above).
 * The systems are concatenated into one block-diagonal matrix; its hierarchy
 * is block diagonal, so each system gets exactly the V-cycle it would get
 * alone except that coarsening continues until the whole batch has at most
 * max_coarse rows.  Every level is sliced so that no slice holds rows of two
 * systems.  Synchronous.  Errors as amg_setup.
 */
int amg_setup_batch(int nsys, const amg_csr* A, const amg_options* opt, amg_stream_t stream,
                    amg_handle** H);

/* nsys (host) and, if row_offsets is not NULL, the first row of every system
 * in the concatenated vectors (host int64[nsys + 1]). */
int amg_batch_info(const amg_handle* H, int* nsys, int64_t* row_offsets);

/*
 * Independent PCG solves of all systems of a batched handle at once: each
 * system has its own alpha, beta, residual norm and stopping test; converged
 * systems are frozen while the others iterate.  b, x: device float64, the
 * systems' vectors concatenated in order (amg_batch_info offsets); x holds the
 * initial guesses and receives the solutions.  st: host array of nsys stats
 * (or NULL).  o->res_history and o->x_history must be NULL.  Synchronous.
 * Returns the worst status over the systems.
 */
int pcg_solve_batch(amg_handle* H, const double* b, double* x, const pcg_options* o,
                    pcg_stats* st, amg_stream_t stream);

/* ----------------------------------------------------------- learned smoother weights */
/*
 * A 9 -> 32 -> 32 -> 1 MLP (GELU hidden layers, output
 * omega = max(omega_max * sigmoid(z), 1e-3), omega_max = 1 unless set) maps
 * each row's stencil features to the l1-Jacobi damping weight omega_i, so
 * s_i = omega_i / d_i stays an A-convergent smoother and the V-cycle stays
 * SPD (Sec. 2.3, l1-Jacobi; the network itself is not in the paper).  Weights are FP32 on the device; 1409 parameters laid out as
 * W1[32][9], b1[32], W2[32][32], b2[32], W3[32], b3.
 */
typedef struct mlp_handle mlp_handle;

/* Number of parameters (1409). */
int mlp_num_params(void);

/* New network with N(0, 1/fan_in) weights from splitmix64 stream `seed`,
 * zero biases and output bias 4 (omega ~ 0.98).  Synchronous. */
int mlp_create(uint64_t seed, mlp_handle** M);
int mlp_destroy(mlp_handle* M);

/* Copy the parameters to / from host float[1409] (set also resets the Adam
 * state and the accumulated gradient).  Synchronous. */
int mlp_get_params(const mlp_handle* M, float* host);
int mlp_set_params(mlp_handle* M, const float* host);

/*
 * Output cap omega_max in [1, 2) (default 1: omega in (0, 1], the plain
 * smoother's step at most).  Above 1 the network may over-relax; any
 * omega_i < 2 keeps 2 diag(d / omega) - A = (2/omega - 1) diag(d) +
 * (diag(d) - A) positive definite (diag(d) - A is diagonally dominant for the
 * l1 row sums d), so the smoother stays A-convergent and the V-cycle SPD.
 * Not in the paper.  Errors: AMG_ERR_ARG (M NULL, omega_max outside [1, 2)).
 */
int mlp_set_omega_max(mlp_handle* M, double omega_max);

/* Accumulated gradient (host double[1409]).  Synchronous. */
int mlp_get_grad(const mlp_handle* M, double* host);

/*
 * Nine features per row of a 7-point operator on an nx x ny x nz grid with
 * lexicographic rows (x fastest): a_ij / a_ii towards -x, +x, -y, +y, -z, +z
 * (0 where absent), sum_{j!=i} |a_ij| / a_ii, log(max |a_ij| / min |a_ij|)
 * over present neighbours, and the neighbour count / 6.  A: device CSR with
 * A->n == nx*ny*nz.  feat: device float[n][9].  Asynchronous.
 */
int mlp_features(const amg_csr* A, int64_t nx, int64_t ny, int64_t nz, float* feat,
                 amg_stream_t stream);

/*
 * omega[i] = network(feat[i]) for n rows (device float arrays).  By default
 * the two hidden layers run on the tensor cores (FP16 operands, FP32
 * accumulation; omega within about 1e-3 of the FP32 pass); after
 * mlp_set_exact_forward(M, 1), in FP32 on the CUDA cores.  Asynchronous.
 */
int mlp_forward(const mlp_handle* M, int64_t n, const float* feat, float* omega,
                amg_stream_t stream);

/* Forward pass in FP32 on the CUDA cores (exact = 1) or on the tensor cores
 * (0, default).  Not in the paper.  Errors: AMG_ERR_ARG. */
int mlp_set_exact_forward(mlp_handle* M, int exact);

/*
 * Gradient of sum_i domega[i] * omega[i] with respect to the parameters
 * (device float feat[n][9], domega[n]); added to the accumulated gradient if
 * accumulate != 0, else replaces it.  Summed in FP64 in a fixed order
 * (reproducible).  Asynchronous.
 */
int mlp_backward(mlp_handle* M, int64_t n, const float* feat, const float* domega,
                 int accumulate, amg_stream_t stream);

/* One Adam step (Kingma & Ba) on grad_scale * accumulated gradient, then
 * clears the gradient.  Asynchronous. */
int mlp_adam_step(mlp_handle* M, double lr, double beta1, double beta2, double eps,
                  double grad_scale, amg_stream_t stream);

/*
 * Two-grid loss of the level-0 smoother weights currently set on H and its
 * gradient: L = mean_j log(||E^K e0_j||_A / ||e0_j||_A) / K with
 * E = S (I - P A_1^-1 P^T A) S, S = I - diag(s) A (Eq. amg with two levels).
 * A_1^-1 is applied by PCG-AMG on levels >= 1 to 1e-12 (exactly when level 1
 * is the coarsest).  e0: device float64[nsamples][n0] initial errors.
 * loss: host.  domega: device float[n0] receiving dL/domega, or NULL.  Needs
 * >= 2 levels (AMG_ERR_UNSUPPORTED otherwise).  The first call builds the
 * inner solver.  Synchronous.
 */
int amg_twogrid_loss(amg_handle* H, int nsamples, int ncycles, const double* e0, double* loss,
                     float* domega, amg_stream_t stream);

/* ----------------------------------------------------------- inspection */

/* One V-cycle kernel launch timed by amg_vcycle_profile. */
typedef struct amg_kernel_time {
  int level;     /* hierarchy level */
  int kind;      /* 0 pre-smooth+residual, 1 restriction (sums over aggregates, or
                    the product with P^T for smoothed prolongators),
                    2 prolongation+post-smooth, 3 coarsest-level solve, 4 the
                    persistent launch of levels >= `level` (all their steps and
                    the coarsest solve), 5 a further smoothing sweep
                    (smooth_sweeps > 1) */
  double bytes;  /* algorithmic bytes: each matrix entry (value + column index:
                    4 bytes, or 2 plus a share of the slice column's base when
                    compressed) and each vector entry read or written once */
  double ms;     /* device time between CUDA events around the launch */
} amg_kernel_time;

/*
 * z = B r like amg_vcycle_apply, with a CUDA event pair around every kernel
 * (the paper reports time per iteration; this splits it per kernel).  The
 * kernels are the ones a PCG iteration runs: the level-0 post-smoother also
 * forms the dot products PCG fuses into it ((r, z), and (z, q) with an FP32
 * hierarchy, q being internal scratch), and an FP32 hierarchy first copies r
 * to FP32 (untimed) as the CG update does.
 * out: host array of max_out records; *count receives the number of kernels
 * launched (records beyond max_out are dropped).  Synchronous.
 */
int amg_vcycle_profile(const amg_handle* H, const double* r, double* z, amg_kernel_time* out,
                       int max_out, int* count, amg_stream_t stream);

/* Number of levels (>= 1). */
int amg_num_levels(const amg_handle* H, int* levels);

/* Rows and stored entries of level l. */
int amg_level_info(const amg_handle* H, int level, int64_t* n, int64_t* nnz);

/*
 * Storage of level l's matrix A in the kernels (sliced ELL, Sec. 2.2):
 * slice height C, threads per row, stored slots (entries plus padding), and
 * whether column indices are compressed: slot e of ELL column k of a slice
 * then holds a 2-byte offset from a 4-byte base shared by the C slots of that
 * column (else a plain 4-byte index).  Compression is used whenever every
 * slice's offsets fit 16 bits; results are identical either way.  `ap`
 * picks the operator: 0 A, 1 A P (the post-smoother's operator), and with
 * smoothed prolongators 2 P and 3 R = P^T (restriction).  No counterpart in
 * the paper.  Errors: AMG_ERR_ARG (bad level, NULL out, ap outside 0..3,
 * ap > 0 on the coarsest level, ap >= 2 without smoothed prolongators).
 */
typedef struct amg_layout {
  int slice_height;
  int threads_per_row;
  int64_t slots;
  int compressed;
} amg_layout;
int amg_level_layout(const amg_handle* H, int level, int ap, amg_layout* out);

/*
 * Copies level-l data into caller device buffers (each may be NULL):
 * rowptr int64[n+1], col int32[nnz], val float64[nnz] (levels >= 1 only;
 * level 0 is the caller's own matrix), agg int32[n] (row -> aggregate on
 * level l+1; not for the coarsest level), sscale float64[n] (smoother
 * scale s_i = omega_i / d_i).  Asynchronous.
 */
int amg_level_export(const amg_handle* H, int level, int64_t* rowptr, int32_t* col,
                     double* val, int32_t* agg, double* sscale, amg_stream_t stream);

/*
 * The smoothed prolongator of level l (option smooth_prolongator; Sec. 2.3):
 * P = (I - w D^-1 A_l) P_hat, n_l x n_{l+1}, columns ascending in every row,
 * copied into caller device buffers (each may be NULL): rowptr int64[n_l+1],
 * col int32[nnz], val float64[nnz].  nnz and w (the damping
 * 1 / max_i sum_j |a_ij| / a_ii): host, may be NULL.  Asynchronous.
 * Errors: AMG_ERR_ARG (coarsest or bad level, handle without smoothed
 * prolongators).
 */
int amg_level_prolongator(const amg_handle* H, int level, int64_t* rowptr, int32_t* col,
                          double* val, int64_t* nnz, double* w, amg_stream_t stream);

/*
 * Pairwise locally-dominant weighted matching of the graph of A (Sec. 2.3;
 * the first sweep of one coarsening step), as a standalone call.  A: device
 * CSR.  mate: device int32[n], receives the partner of each row or -1.
 * rounds: host, may be NULL, receives the number of pointer rounds.
 * Errors: AMG_ERR_ARG (NULL pointers, n <= 0, nnz < n), AMG_ERR_UNSUPPORTED
 * (n beyond int32), AMG_ERR_DEVICE_CHECK (the rounds did not end),
 * AMG_ERR_OOM / AMG_ERR_CUDA.  Synchronous.
 */
int amg_pairwise_match(const amg_csr* A, int32_t* mate, int* rounds, amg_stream_t stream);

/* Largest matrix (rows) that amg_pairwise_match_noalloc accepts. */
#define AMG_NOALLOC_MAX_ROWS 262144

/*
 * amg_pairwise_match without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc, such as
 * applications whose device memory is owned by a pool or framework that
 * forbids outside allocations, and real-time loops that must not allocate
 * after start-up.
 * Same arguments and result as amg_pairwise_match (bit-identical mate and
 * rounds).  Its scratch is one fixed device array of 24 bytes per row for
 * AMG_NOALLOC_MAX_ROWS rows (6 MiB), held by every GPU that loads the library
 * until the process exits; larger matrices return AMG_ERR_UNSUPPORTED.  The
 * first call on a device looks up that array's address (a one-time set-up,
 * kept until the process exits; a device reset invalidates it, so do not call
 * this on a device reset by cudaDeviceReset); make that first call before any
 * stream capture.  All calls share the array, so calls that overlap on the
 * GPU (other streams or host threads) race and must be serialised by the
 * caller.  Errors: as amg_pairwise_match (never AMG_ERR_OOM), and
 * AMG_ERR_UNSUPPORTED for more than AMG_NOALLOC_MAX_ROWS rows.  Synchronous.
 */
int amg_pairwise_match_noalloc(const amg_csr* A, int32_t* mate, int* rounds,
                               amg_stream_t stream);

/* ----------------------------------------------------------- test hooks */

/*
 * Host-side fault injection: the `count`-th device allocation made by the
 * library from now on (0 = the next one) fails with AMG_ERR_OOM before any
 * GPU memory is touched; -1 disarms.  No counterpart in the paper (its
 * routines report failures through `info`, Sec. 2.1); used to test error
 * paths without faulting a GPU.
 */
int amg_debug_fail_alloc_after(long count);

/*
 * Barrier-timeout injection for the persistent small-level launch (the
 * `tail_rows` option): while `on` is 1, that launch's grid barrier waits for
 * one arrival that never comes, every CTA gives up after 10 ms, and the
 * next pcg_solve / pcg_solve_batch returns AMG_ERR_DEVICE_CHECK (clearing
 * the failure state).  No GPU fault is involved: the waits are bounded and
 * the kernel returns.  No counterpart in the paper; used to test the
 * timeout path.  Errors: AMG_ERR_ARG (H NULL).
 */
int amg_debug_tail_timeout(amg_handle* H, int on);

/*
 * out[i] = GELU(u[i]) as the tensor-core MLP forward pass evaluates it (erf
 * by Abramowitz & Stegun 7.1.26), for n device floats, so tests can bound
 * its error against the exact GELU.  No counterpart in the paper.  Errors:
 * AMG_ERR_ARG.  Asynchronous.
 */
int mlp_debug_gelu(const float* u, float* out, int64_t n, amg_stream_t stream);

/*
 * The V-cycle kernels' precision conversions on n device elements:
 * out32[i] = in64[i] rounded to binary32 (nearest, ties to even) and
 * out64[i] = in32[i] widened to binary64, both by the integer-pipe routines
 * the FP32 hierarchies' kernels use, so tests can compare them bit for bit
 * with the hardware conversions.  Either pair may be NULL.  No counterpart in
 * the paper (its FP32 runs are not mixed-precision).  Errors: AMG_ERR_ARG
 * (n < 0, or one pointer of a pair NULL).  Asynchronous.
 */
int amg_debug_convert(const double* in64, float* out32, const float* in32, double* out64,
                      int64_t n, amg_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* AMG_GB300_H */
