/*
 * airg.h -- C ABI of libairg.so: AIRG reduction multigrid (approximate ideal restriction with
 * GMRES polynomials) as a preconditioner for GMRES, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Dargaville, Smedley-Stevenson, Smith & Pain, "Coarsening and parallelism with reduction
 * multigrids for hyperbolic Boltzmann transport", arXiv 2408.08262:
 *   - Section "CF splitting": strength of connection (eq. soc), PMISR (Algorithm 1) and the
 *     diagonal-dominance cleanup DDC (Algorithm 2);
 *   - Section "AIRG": per-level setup steps 1-11, the GMRES polynomial (eq. gmres_poly) with
 *     first-order fixed sparsity (eq. fixed_sparsity), approximate ideal restriction
 *     Z = -A_cf Ainv_ff (eq. prolong), one-point prolongation, A_c = R A P;
 *   - Section "Results": V-cycle with up F-point smoothing only; Section "Timing results for
 *     parallel optimisations": GMRES-polynomial coarse-grid solver.
 *
 * Conventions shared by every entry point
 *   - Matrices are square CSR with int32 row pointers and column indices, columns sorted and
 *     unique within each row, every diagonal entry stored and nonzero, FP64 values.
 *   - Pointers named "device" must be CUDA device (or managed) memory on the current device;
 *     pointers named "host" are ordinary host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All GPU work of a call is issued
 *     on that stream; calls that must report sizes or convergence synchronise it.
 *   - The caller owns every pointer it passes; the library never keeps a caller pointer after a
 *     call returns (airg_setup copies the matrix).  A hierarchy owns all of its device memory.
 *   - Return value: AIRG_OK (0), a negative AIRG_ERR_* code, or AIRG_NOT_CONVERGED (1).  The
 *     library never aborts, traps or exits.  airg_status_string() names every code.
 *   - Not thread-safe per hierarchy: one hierarchy must not be used by two calls at once.
 */
#ifndef AIRG_H
#define AIRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* airg_stream_t; /* same object as cudaStream_t */

enum {
  AIRG_OK = 0,
  AIRG_NOT_CONVERGED = 1,   /* solve hit max_it; x and info are still filled */
  AIRG_ERR_ARG = -1,        /* null pointer, negative size, bad option value */
  AIRG_ERR_CSR = -2,        /* row pointers not monotone, column out of range/unsorted/duplicate */
  AIRG_ERR_ZERO_DIAG = -3,  /* a diagonal entry is missing or zero */
  AIRG_ERR_NAN = -4,        /* NaN/Inf met in a norm during the solve */
  AIRG_ERR_OOM = -5,        /* device allocation failed */
  AIRG_ERR_CUDA = -6,       /* any other CUDA runtime error */
  AIRG_ERR_UNSUPPORTED = -7, /* a product row exceeded the library's working-set limit */
  AIRG_ERR_SCRATCH = -8      /* input too large for airg_cf_split_noalloc's fixed scratch array */
};

enum { AIRG_FP64 = 0, AIRG_FP32 = 1, AIRG_BF16_VALUES = 2 };
enum { AIRG_OUTER_FGMRES = 0, AIRG_OUTER_RICHARDSON = 1 };

/* Square CSR matrix in device memory. */
typedef struct {
  int32_t n;              /* rows = columns */
  int32_t nnz;            /* rowptr[n] */
  const int32_t* rowptr;  /* device, n+1 */
  const int32_t* col;     /* device, nnz, sorted unique per row */
  const double* val;      /* device, nnz */
} airg_csr;

/* Setup parameters.  Defaults (airg_params_default) follow the paper's parallel settings
 * (Section "Parallel results"): strength 0.5, n_loops^max = 3, DDC fraction 10 %, drop 0.01 on Z
 * and 0.001 on the coarse matrices, 6th-order polynomials (m = 7) with first-order fixed sparsity; two up F-smooths (Section "Results"); the coarse solve uses
 * three iterations of a 12th-order fixed-sparsity polynomial (Section "Timing results"), with the
 * hierarchy truncated automatically at clamp(n_top / 16, 64, 60000) unknowns (the paper truncates
 * at ~300k on CPU ranks; on one GB300, setup plus solve time averaged over seeds is lowest near 60k
 * for the 1.57M- and 6.29M-DOF systems, and smaller systems keep a multilevel hierarchy). */
typedef struct {
  double strong_threshold;  /* alpha in eq. soc, in [0, 1] */
  double ddc_fraction;      /* fraction of F-points DDC converts, in [0, 1] */
  int pmisr_max_loops;      /* n_loops^max of Algorithm 1; <= 0 means no cap */
  int poly_order;           /* degree d of the GMRES polynomial on A_ff (m = d+1 coefficients), <= 14 */
  int coarse_poly_order;    /* degree of the coarsest-level polynomial */
  int coarse_iters;         /* iterations of the coarsest-level polynomial solve (>= 1) */
  int coarse_size;          /* a level with n <= coarse_size is the coarsest; <= 0: automatic,
                               clamp(n_top / 16, 64, 60000) */
  int max_levels;           /* hierarchy depth cap (>= 1) */
  double drop_R;            /* relative row-wise inf-norm drop on Z */
  double drop_Ac;           /* relative row-wise inf-norm drop on A_c (diagonal always kept) */
  int n_smooth_up;          /* up F-point smooths per level */
  int precision;            /* AIRG_FP64; or the mixed-precision form: AIRG_FP32 (V-cycle operators and
                               vectors in FP32, FP32 accumulation) or AIRG_BF16_VALUES (operator values
                               stored as bf16, vectors and accumulation FP32).  Setup (coefficient fits
                               included), the outer residual, Arnoldi and the Hessenberg least squares
                               stay FP64 in every mode. */
  int keep_setup;           /* 1: keep natural-numbering setup operators for airg_export_level */
  uint64_t seed;            /* seeds PMISR weights and the Box-Muller right-hand sides */
  int sparsity_order;       /* fixed sparsity of the A_ff polynomials (Section "AIRG"): 1 = pattern of
                               A_ff (default), 2 = pattern of A_ff^2; the coarsest-level polynomial
                               always uses first order */
  int matrix_free;          /* 1: the solve applies every polynomial matrix-free, q(A_ff) r by Horner's
                               rule with m - 1 products by A_ff (q(A) r with the coarsest matrix), in
                               place of the assembled fixed-sparsity inverse (Section "AIRG" names this
                               alternative); setup still assembles Ainv for Z.  FP64 only; 0 (default):
                               assembled */
  int ideal_prolong;        /* 1: approximate ideal prolongator P = [W; I], W = -Ainv A_fc (eq. prolong)
                               with drop_R's relative drop, in place of the one-point operator (setup
                               step 10's alternative); FP64 only; 0 (default): one-point */
} airg_params;

typedef struct airg_hierarchy airg_hierarchy; /* opaque, library-owned */

typedef struct {
  int outer;    /* AIRG_OUTER_FGMRES (right-preconditioned, CGS2) or AIRG_OUTER_RICHARDSON */
  int restart;  /* FGMRES restart length, 1..32 */
  int max_it;   /* maximum preconditioner applications */
  double rtol;  /* stop when ||b - A x||_2 <= rtol ||b||_2 */
  int x0_zero;  /* 1: ignore x on entry and start from zero */
} airg_solve_opts;

typedef struct {
  int iters;      /* preconditioner applications (V-cycles) */
  double relres;  /* true relative residual ||b - A x|| / ||b|| at exit */
  int status;     /* same code as the return value */
  int levels;     /* hierarchy levels */
} airg_solve_info;

/* Fills *p with the defaults above (seed 240808262). */
void airg_params_default(airg_params* p);

/* Builds the AIRG hierarchy of A (setup steps 1-11 of Section "AIRG" on every level, the
 * coarsest-level polynomial, and the permuted solve-phase operators).  A's arrays are read on
 * `stream` and copied; *out receives a new hierarchy, freed with airg_free.  Synchronises the
 * stream several times per level (sizes of products).  Errors: AIRG_ERR_ARG, AIRG_ERR_CSR,
 * AIRG_ERR_ZERO_DIAG, AIRG_ERR_OOM, AIRG_ERR_CUDA, AIRG_ERR_UNSUPPORTED; *out is NULL then. */
int airg_setup(const airg_csr* A, const airg_params* p, airg_stream_t stream, airg_hierarchy** out);

/* The same as airg_setup with A's three arrays in HOST memory (pinned memory lets the copies run
 * at full speed; pageable memory works too): the library copies them to the device on `stream`
 * inside the call and does not keep the host pointers.  With airg_solve_host, a caller whose data
 * lives on the host sets up and solves through the C ABI alone. */
int airg_setup_host(const airg_csr* A_host, const airg_params* p, airg_stream_t stream, airg_hierarchy** out);

/* Setups of many independent systems (the batched form), run concurrently: `nthreads` host
 * threads (<= 0: 8), each with a stream of its own, take the systems in turn and build their
 * hierarchies as airg_setup does (same parameters for all; As: nsys device CSR descriptors).
 * Small systems leave most of the GPU idle, and each setup waits on the host for its sizes, so
 * running several at once fills the GPU.  Each hierarchy is bitwise the one airg_setup builds.
 * Synchronises `stream` first (the inputs may be produced on it); returns once every hierarchy is
 * built, each then belonging to `stream`.  outs: host array of nsys handles, each freed with
 * airg_free.  On any error every handle is freed, set to NULL, and the first error returned. */
int airg_setup_many(const airg_csr* As, int nsys, const airg_params* p, int nthreads, airg_stream_t stream,
                    airg_hierarchy** outs);

/* Setup re-use (Sections "Strong tolerances" and "Conclusions" name re-using the CF splitting
 * across the many solves of a Boltzmann problem).  Builds the hierarchy of A as airg_setup does,
 * except that the CF splittings of the first `levels` levels (levels <= 0: every non-coarsest level
 * of T) are taken from the template hierarchy T instead of computed (no strength graph transpose,
 * PMISR or DDC there).  Intended for a matrix with T's sparsity pattern and new values (another
 * energy group, cross section or time step of the same mesh and direction).  With strength
 * threshold 0 the level-0 splitting depends on the pattern only, so re-using it reproduces a fresh
 * setup exactly; deeper levels (whose patterns depend on the drops) get a valid, not identical,
 * splitting.  T is only read and must stay alive during the call; A->n must equal T's size, else
 * AIRG_ERR_ARG.  Same parameters, errors and ownership as airg_setup otherwise. */
int airg_setup_reuse(const airg_csr* A, const airg_params* p, const airg_hierarchy* T, int levels,
                     airg_stream_t stream, airg_hierarchy** out);

/* Solves A x = b with the hierarchy as preconditioner.  b, x: device, n FP64.  x holds the initial
 * guess on entry (unless opts->x0_zero) and the solution on exit.  Synchronises the stream once per
 * iteration.  Returns AIRG_OK, AIRG_NOT_CONVERGED, or an error (x undefined on error). */
int airg_solve(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* opts,
               airg_solve_info* info, airg_stream_t stream);

/* Same as airg_solve with b and x in HOST memory: copies b (and x) to the device, solves, copies
 * x back; the copies run on `stream`. */
int airg_solve_host(airg_hierarchy* H, const double* b_host, double* x_host, const airg_solve_opts* opts,
                    airg_solve_info* info, airg_stream_t stream);

/* Adjoint form.  Builds the AIRG hierarchy of A^T (a separate setup: A^T has its own strong
 * connections) for the adjoint solve A^T lambda = g.  A is transposed on the device (deterministic:
 * rows of A^T sorted by column) and passed to airg_setup; same parameters, errors and ownership. */
int airg_setup_transpose(const airg_csr* A, const airg_params* p, airg_stream_t stream, airg_hierarchy** out);

/* A^T in CSR into caller-owned DEVICE arrays: rowptr_out (n+1), col_out (nnz), val_out (nnz);
 * columns sorted within each row.  Synchronises the stream. */
int airg_transpose(const airg_csr* A, int32_t* rowptr_out, int32_t* col_out, double* val_out, airg_stream_t stream);

/* Sampled dense-dense product on a sparsity pattern: out_val[k] = (scale * lam[i]) * x[col[k]] for
 * every stored entry k = (i, col[k]) of `pattern` (its values are not read).  With lam the adjoint
 * solution of A^T lam = dJ/dx and scale = -1 this is dJ/dA = -lam x^T restricted to A's pattern.
 * lam, x: device, n; out_val: device, nnz.  Does not synchronise. */
int airg_sddmm(const airg_csr* pattern, const double* lam, const double* x, double scale, double* out_val,
               airg_stream_t stream);

/* Batched form: many independent systems, each with its own (FP64) hierarchy, solved together.
 * airg_batch_create concatenates, for every hierarchy depth, the level operators of all systems
 * into grouped CSR matrices (columns relabelled to positions in one concatenated vector, rows
 * mapped to their positions), so every V-cycle step is one launch over all systems; the batched
 * V-cycle is captured once as a CUDA graph.  The hierarchies must outlive the batch and share
 * coarse_iters and n_smooth_up, and use assembled polynomials and one-point prolongators
 * (matrix_free = ideal_prolong = 0; else AIRG_ERR_ARG).
 * airg_solve_batched runs right-preconditioned FGMRES on every system
 * in lockstep, with per-system (segmented) reductions and per-system convergence: b[q], x[q] are
 * device pointers of system q's size (x holds the initial guess unless opts->x0_zero), infos has
 * nsys entries.  Returns the worst status (a negative error if any system failed). */
typedef struct airg_batch airg_batch;
int airg_batch_create(airg_hierarchy* const* Hs, int nsys, airg_stream_t stream, airg_batch** out);
int airg_solve_batched(airg_batch* B, const double* const* b, double* const* x, const airg_solve_opts* opts,
                       airg_solve_info* infos, airg_stream_t stream);
void airg_batch_free(airg_batch* B);

/* The batched form's SpMV autotuner.  airg_batch_create times the row-length rule's lanes per row
 * and its two neighbours (half and twice as many, within 1..32) on each grouped operator with at
 * least 16384 rows and keeps the fastest;
 * smaller groups keep the row-length rule.  Setting the environment variable AIRG_NO_AUTOTUNE=1
 * keeps the rule everywhere.  The variants sum a row in different orders, so the chosen variants
 * can change results in the last bits.  airg_batch_tuned writes, for the first `cap` tuned groups,
 * the rule's lanes and the chosen lanes (host arrays; either may be NULL) and returns the number of
 * tuned groups. */
int airg_batch_tuned(const airg_batch* B, int* rule_lanes, int* chosen_lanes, int cap);

/* One V-cycle from a zero guess, x = M b (b, x: device, n).  For tests and diagnostics. */
int airg_vcycle(airg_hierarchy* H, const double* b, double* x, airg_stream_t stream);

/* The two-pass CF splitting alone (eq. soc, Algorithm 1, Algorithm 2) of one matrix, as done on
 * level `level` of a setup (the level index salts the PMISR weight stream).  cf_out: device, n
 * int8; 1 = F-point, 2 = C-point.  Synchronises the stream. */
int airg_cf_split(const airg_csr* A, const airg_params* p, int level, int8_t* cf_out, airg_stream_t stream);

/* The CF splitting of airg_cf_split, computed without allocating any device memory.  The paper
 * has no counterpart: this entry point exists for callers that cannot call cudaMalloc (or any
 * allocating routine) at the point they need the splitting -- for example a program that reserves
 * all device memory at start-up and allocates nothing afterwards, or a latency-critical loop in
 * which an allocation, and the synchronisation it may trigger, is not acceptable.
 * All temporaries live in one fixed 32 MiB device array.  The input needs about 5 bytes per
 * nonzero plus 34 bytes per row; larger inputs return AIRG_ERR_SCRATCH before any GPU work.  The
 * result is identical to airg_cf_split's (same kernels, same arithmetic), and so are the argument
 * checks (AIRG_ERR_ARG) and the cf_out encoding.
 *   - The first call on a device is the set-up: CUDA loads the library's modules lazily, so that
 *     call loads the kernels the splitting launches and the array itself (allocated then, and held
 *     until the process exits), and looks up the array's device address (cudaGetSymbolAddress).
 *     It allocates device memory: make it at start-up, before reserving the rest of the device,
 *     and outside any stream capture.  Later calls allocate nothing.  After a device reset
 *     (cudaDeviceReset) the next call on that device is a first call again.
 *   - Every call shares the one array.  Calls that can overlap on the GPU (other streams, other
 *     host threads) race on it and must be serialised by the caller.  Each call clears what it
 *     needs; the array otherwise keeps the last call's contents.
 *   - Synchronises the stream. */
int airg_cf_split_noalloc(const airg_csr* A, const airg_params* p, int level, int8_t* cf_out,
                          airg_stream_t stream);

/* Diagnostic (the diagonal-dominance ratios behind DDC, Algorithm 2 and Section "CF splitting"):
 * theta_i = sum_{j in F, j != i} |a_ij| / |a_ii| over the F-points of the splitting cf (device, n
 * int8, 1 = F, 2 = C), 0 for C-points and for F rows with no F neighbour.  theta: device, n FP64.
 * Sums run over the row in storage order.  The splitting before DDC is the one airg_cf_split gives
 * with ddc_fraction = 0.  Synchronises the stream.  Errors: AIRG_ERR_ARG, AIRG_ERR_CSR,
 * AIRG_ERR_ZERO_DIAG, AIRG_ERR_CUDA. */
int airg_ddc_theta(const airg_csr* A, const int8_t* cf, double* theta, airg_stream_t stream);

/* Frees a hierarchy and everything it owns (NULL is allowed).  Synchronises the stream the
 * hierarchy was built on. */
void airg_free(airg_hierarchy* H);

/* Number of levels (>= 1), or a negative error. */
int airg_num_levels(const airg_hierarchy* H);

/* Per-level sizes into info[0..17] (host, 18 entries): n, nnz(A), n_f, n_c, nnz(A_ff), nnz(A_fc), nnz(Ainv),
 * nnz(Z), coarsest flag, nnz(A_cf), fitted polynomial coefficients, nnz(AF solve operator), and the
 * level's setup time in microseconds split as in the paper's per-component setup figure:
 * [12] CF splitting + extraction, [13] GMRES polynomial (steps 3-8), [14] restrictor product,
 * [15] prolongator + coarse matrix; [16] nnz(W) of the approximate ideal prolongator (0 for one-point);
 * [17] which solve operators the SpMVs read in sliced ELL form (bits: 1 [A_ff A_fc], 2 Ainv, 4 Z,
 * 8 coarsest A, 16 A_ff of the matrix-free form, 32 W); the others are read as CSR.
 * Level -1 gives totals: [0] levels, [1] grid complexity x1e6, [2] operator complexity x1e6,
 * [3] storage complexity x1e6 (eq. mat_store), [4] setup wall ms x1e3, [5..9] summed microseconds of
 * the five phases (CF splitting, extraction, polynomial, restrictor, prolongator + coarse matrix),
 * [10] microseconds spent building the solve-phase layout (sliced ELL copies included), [11] 1 if the
 * top-level operator is read in sliced ELL form. */
int airg_level_info(const airg_hierarchy* H, int level, int64_t* info);

/* Copies a level operator to HOST arrays (sizes from airg_level_info).
 * Natural numbering of the level (needs params.keep_setup = 1, else AIRG_ERR_ARG):
 *   which 0 A, 1 A_ff, 2 A_fc, 3 A_cf, 5 Ainv, 6 Z (rows: C-points in ascending order, columns:
 *   F-points in ascending order).
 * Solve-phase layout (always available): 7 [A_ff A_fc] rows of the F-points with columns in the
 *   level's F-then-C numbering (nnz = info[11]), 8 Z with rows in the next level's F-then-C
 *   numbering, 9 the top-level matrix permuted to level 0's F-then-C numbering (n0 x n0, nnz of
 *   the input), 10 Ainv as used by the solve, 11 coarsest-level matrix, 13 W with columns in the
 *   next level's F-then-C numbering (ideal_prolong only).
 * 12: W in natural numbering (rows F-points, columns C-points, ascending; needs keep_setup and
 *   ideal_prolong).
 * Any of rowptr/col/val may be NULL. */
int airg_export_csr(const airg_hierarchy* H, int level, int which, int32_t* rowptr, int32_t* col, double* val);

/* Copies level vectors to HOST arrays: cf (n int8, 1 F / 2 C; NULL on the coarsest level),
 * w (n_f int32: C index of each F-point's one-point interpolation source, -1 for none), alpha
 * (fitted polynomial coefficients, poly_order+1 or coarse_poly_order+1 doubles).  Needs
 * keep_setup for cf and w. */
int airg_export_vectors(const airg_hierarchy* H, int level, int8_t* cf, int32_t* w, double* alpha);

/* Copies the solve-phase numbering of a level to HOST arrays: pos (n entries; natural index of
 * the level -> nested position: F-points first in ascending order, then the C-points in the next
 * level's nested numbering; identity on the coarsest level) and
 * w_solve (n_f entries; one-point source of each F-point in the next level's solve numbering,
 * -1 for none).  Either may be NULL. */
int airg_export_layout(const airg_hierarchy* H, int level, int32_t* pos, int32_t* w_solve);

/* Kernel timing for roofline reports.  `enable` is a bit mask of kernel classes (bit c = class c;
 * 0 disables, -1 times every class).  Every launch of a selected class is bracketed by CUDA events
 * on its stream; airg_kernel_times() returns, per kernel
 * class (0: smoother residual A_F*, 1: smoother update Ainv, 2: restriction Z, 3: top-level
 * operator, 4: coarsest level, 5: prolongation gather, 6: Gram-Schmidt passes, 7: whole V-cycle
 * applications, each timed by one event pair outside the cycle, with the summed algorithmic bytes
 * of all of the cycle's SpMVs), the launch count, the summed milliseconds and the summed
 * algorithmic bytes (CSR arrays + vectors read/written once).  Every call of airg_profile_enable
 * resets the sums. */
int airg_profile_enable(airg_hierarchy* H, int enable);
int airg_kernel_times(airg_hierarchy* H, int64_t* launches, double* ms, double* bytes, int nclasses);
/* The same sums restricted to the launches that worked on hierarchy level `level` (classes 3 and 6
 * are counted on level 0). */
int airg_kernel_times_level(airg_hierarchy* H, int level, int64_t* launches, double* ms, double* bytes, int nclasses);

/* Total number of CUDA kernel launches this library has issued in the process (all hierarchies,
 * all calls).  Used to count the GPU work of a timed region. */
int64_t airg_launch_count(void);

/* Human-readable name of a status code. */
const char* airg_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* AIRG_H */
