/*
 * nlfeti -- one-level FETI for finite element discretizations of nonlocal diffusion
 * (integrable and fractional kernels) and bond-based peridynamics, on one GPU.
 *
 * C ABI.  All entry points return an nlfeti_status and never throw.  On error the
 * outputs are left untouched and nlfeti_last_error(ctx) describes the failure.
 *
 * Problem statement (the calls follow it): given a P1 mesh of the unit domain and
 * its Dirichlet collar, a kernel with horizon delta, and a local decomposition into
 * K parts, solve A u = f - B g (Sec. 2.3.3, eq. weak_nonloc-h) with the one-level
 * FETI method (Algorithm 1) on the nonlocal subdivision built from the local parts
 * (Sec. 5.1).  Outputs are nodal values.
 *
 * Memory: the caller owns every host array and every device array it passes; the
 * library copies what it needs before a call returns (except *_device calls, which
 * read and write the caller's device buffers on the context's stream).  Device
 * memory of the library comes from the dev_alloc/dev_free callbacks given to
 * nlfeti_create (or cudaMalloc/cudaFree when they are NULL).
 *
 * Threads: a context and its problems are not thread-safe; a server is (one
 * submit/wait mutex; its slots are worker threads with their own streams).
 */
#ifndef NLFETI_H
#define NLFETI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nlfeti_ctx nlfeti_ctx;
typedef struct nlfeti_problem nlfeti_problem;
typedef struct nlfeti_server nlfeti_server;
typedef uint64_t nlfeti_ticket;

typedef enum {
    NLFETI_OK = 0,
    NLFETI_E_INVALID = -1,        /* malformed input (sizes, indices, decomposition) */
    NLFETI_E_NOMEM = -2,          /* device allocation failed / over the HBM budget */
    NLFETI_E_NOT_SPD = -3,        /* a pivot block was not positive definite */
    NLFETI_E_NOT_CONVERGED = -4,  /* PCG or refinement hit its iteration limit */
    NLFETI_E_TIMEOUT = -5,        /* a wait ran out of time */
    NLFETI_E_CUDA = -6,           /* a CUDA call failed */
    NLFETI_E_BUSY = -7            /* no free server slot */
} nlfeti_status;

/* Kernel types (Sec. 6.1). */
enum {
    NLFETI_K_CONST_LINF = 0,      /* constant, l-infinity ball (1-D: the interval |x-y|<=delta); eq. constantkernel */
    NLFETI_K_CONST_L2 = 1,        /* constant, l2 ball approximated by the nocaps polygon (Fig. approximate-ball e) */
    NLFETI_K_FRACTIONAL = 2,      /* c |x-y|^-(d+2s), l2 ball, nocaps; eq. fractionalkernel */
    NLFETI_K_PERIDYNAMIC = 3      /* c (x-y)(x-y)^T/|x-y|^3, l2 ball, nocaps, 2 dofs per node; eq. peridynamics */
};

/* Mesh (Sec. 2.3.1): P1 simplices covering the domain and its Dirichlet collar.
 * xy: dim*n_nodes doubles, node-major.  elems: (dim+1)*n_elems int32 node ids
 * (triangles counter-clockwise).  node_is_dirichlet: 1 for nodes in the closed
 * collar Gamma^D_h.  elem_is_dirichlet: 1 for elements of the collar. */
typedef struct {
    int dim;
    int64_t n_nodes;
    const double *xy;
    int64_t n_elems;
    const int32_t *elems;
    const int8_t *node_is_dirichlet;
    const int8_t *elem_is_dirichlet;
} nlfeti_mesh;

/* Kernel: type, horizon delta, fractional order s (type 2 only) and constant c
 * (scale > 0 required; the library does not pick a default).
 * ball: the approximate interaction ball of the 2-D l2 kernels (types 1-3; Sec. 2.3,
 * Fig. approximate-ball): 0 = "nocaps" (E' clipped to the polygon of its vertices in the
 * closed disc and the edge/circle crossings); whole elements E' selected when
 * 1 = its barycenter, 2 = at least one vertex ("123vertices"), 3 = at least two vertices
 * ("23vertices") lie in the closed disc about the outer quadrature point; 4 = "approxcaps"
 * (Fig. approximate-ball f): the nocaps polygon with each circular cap it leaves out
 * replaced by the triangle on the cap's chord and the midpoint of its arc (requires
 * 2 delta > the longest element edge, else NLFETI_E_INVALID).  Must be 0 for the
 * l-infinity constant kernel (type 0, exact square) and in 1-D (exact interval). */
typedef struct {
    int type;
    double delta;
    double s;
    double scale;
    int ball;
} nlfeti_kernel;

/* Local decomposition (Sec. 5.1): K parts, one label in [0, K) per non-Dirichlet
 * element (labels of collar elements are ignored).  1 <= K <= 4096. */
typedef struct {
    int32_t K;
    const int32_t *elem_subdomain;
} nlfeti_decomp;

/* Solver options.
 * precision: 0 = FP64 operators throughout ("plain"); 1 = FP32 subdomain operators
 *            with FP64 PCG vectors, coarse problem and iterative refinement ("mixed").
 * tol: PCG stop when ||P r||_2 <= tol ||P d||_2 per right-hand side (FP64 path);
 *      the mixed path uses inner_tol per refinement sweep and stops refining a
 *      right-hand side when its relative nodal correction, or the remaining error that
 *      correction predicts from the observed contraction, is within refine_tol.
 * batched: 1 = one launch per stage over all subdomains (graph-captured loop);
 *          0 = one launch per subdomain per stage, no graphs (baseline).
 * graph_loop (batched only): 1 = each PCG loop runs on the device as one graph with a
 *          WHILE node (no host round trips); 0 = graphs of 4 iterations with a host check
 *          of convergence in between (for profilers that cannot look inside conditional
 *          graphs).  Profiling (nlfeti_set_profiling) always uses the second form.
 * precond_fp16 (mixed path): the scaled Dirichlet preconditioner applies S_k from an FP16
 *          copy scaled by one power of two (half the bytes of the preconditioner apply; the
 *          preconditioner only steers the PCG, the accuracy reached is set by F and the FP64
 *          refinement).  1 = on the FP32 pipes (x in FP32; the default); 2 = on the tensor
 *          cores (x in FP16, scaled per column by a power of two from its norm; FP32
 *          accumulation) for at most 64 right-hand sides, else as 1; 0 = the FP32 S_k.
 *          nlfeti_apply ops 0-4 always use the FP32 S_k.
 * factor_tc (FP32 operators): the rank-64 updates of the factorization sweeps on the tensor
 *          cores (tcgen05 kind::tf32, each FP32 panel entry split into three TF32 terms) --
 *          1 = in both sweeps (the Omega sweep of A^k and the sweep of the pinned S_k), 2 = in the
 *          Omega sweep only (the default), 0 = on the FP32 pipes only.  The tensor cores
 *          accumulate with truncation: in the sweep of the pinned S_k (the pseudo-inverse S_k^+)
 *          that error costs the mixed path's refinement an extra sweep on some problems, in the
 *          Omega sweep it does not; all settings meet the same tolerances.  Read by nlfeti_factor.
 * residual_format (mixed path): how the FP32 factorization keeps A^k for the FP64-accurate
 *          refinement residual (double-single arithmetic either way) -- 0 = chosen from the
 *          sparsity of A^k (the default): a CSR when at most an eighth of the dense entries are
 *          nonzero (kernels of compact support with a horizon of a few mesh sizes), else dense
 *          pairs streamed in tiles; 1 = dense; 2 = CSR.  Read by nlfeti_factor. */
typedef struct {
    int precision;
    double tol;
    int max_it;
    int max_refine;
    double inner_tol;
    double refine_tol;
    int batched;
    size_t hbm_budget;
    int graph_loop;
    int precond_fp16;
    int factor_tc;
    int residual_format;
} nlfeti_options;

typedef struct {
    int iterations;            /* PCG iterations summed over refinement sweeps (max over RHS) */
    int refine_sweeps;
    double final_rel_residual; /* last ||P r|| / ||P d|| (max over RHS) */
    double rel_correction;     /* last relative nodal correction (mixed path) */
    double ms_setup, ms_factor, ms_solve;
    double ms_queue;           /* server requests: time from nlfeti_submit until a slot took the
                                  request (ms_solve then runs to its result on the host side) */
} nlfeti_stats;

/* Sizes of a created problem.  residual_nnz: nonzeros of A^k (all subdomains) when the FP32
 * factorization keeps it as a CSR for the refinement residual (options.residual_format), else
 * 0 (dense, or the FP32 operators not factored). */
typedef struct {
    int32_t K, ncomp, n_floating, n_coarse;
    int64_t n_lambda, n_u, sum_nk, sum_nk2, sum_ngamma2;
    int32_t max_nk, max_ngamma;
    int64_t residual_nnz;
} nlfeti_info;

/* Default options: FP64 plain, tol 1e-10, max_it 1000, at most 10 refinement sweeps,
 * inner_tol 1e-3 (each sweep's contraction is limited by the FP32 operators to ~1e-4
 * anyway), refine_tol 1e-9, batched, graph_loop 1. */
void nlfeti_default_options(nlfeti_options *opt);

/* Context on the given CUDA stream (cudaStream_t, NULL = the legacy stream).
 * dev_alloc(size, user) / dev_free(ptr, user): optional device allocator. */
nlfeti_status nlfeti_create(nlfeti_ctx **out, const nlfeti_options *opt, void *cuda_stream,
                            void *(*dev_alloc)(size_t, void *), void (*dev_free)(void *, void *), void *alloc_user);
void nlfeti_destroy(nlfeti_ctx *ctx);
const char *nlfeti_last_error(const nlfeti_ctx *ctx);

/* Build the nonlocal subdivision (Sec. 5.1: delta/2 extension of each local part,
 * Gamma^D_k within delta, zeta, Omega_k / Gamma_k dofs, B, B_D, Z) on the host,
 * upload it, and assemble every subdomain matrix A^k on the GPU (eq.
 * bilinear-multi1, kernel weighted by 1/zeta).  Setup is synchronous. */
nlfeti_status nlfeti_problem_create(nlfeti_ctx *ctx, const nlfeti_mesh *mesh, const nlfeti_kernel *kernel,
                                    const nlfeti_decomp *decomp, nlfeti_problem **out);
void nlfeti_problem_destroy(nlfeti_problem *p);
nlfeti_status nlfeti_problem_info(const nlfeti_problem *p, nlfeti_info *info);
/* Replace the problem's options (copied).  NLFETI_E_INVALID for a precision other than 0/1
 * or precond_fp16 outside 0..2.  Selecting precond_fp16 = 2 once the FP32 operators are
 * factored builds the tiled FP16 copy of S_k the tensor-core apply reads (synchronous). */
nlfeti_status nlfeti_problem_set_options(nlfeti_problem *p, const nlfeti_options *opt);

/* Factor the subdomain operators (eq. splittingBlockCholesky, eq. subSchurComplement,
 * Sec. 5.3): per subdomain A_OO^-1, A_GO A_OO^-1 and the Schur complement S_k, the
 * pseudo-inverse S_k^+ (pinning + projection on ker Z_k^T), and (G^T G)^-1.
 * precision_mask: bit 0 = FP64 operators, bit 1 = FP32 operators. */
nlfeti_status nlfeti_factor(nlfeti_problem *p, int precision_mask);

/* Solve for nrhs right-hand sides (host arrays).  rhs: n_nodes*ncomp x nrhs,
 * column-major; rhs_kind 0 = nodal values of f (P1 interpolant integrated against
 * the basis), 1 = load vector.  g: Dirichlet data, same shape, or NULL for zero.
 * u_out: n_nodes*ncomp x nrhs; Dirichlet entries are set to g (or 0). */
nlfeti_status nlfeti_solve(nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs, const double *g,
                           double *u_out, nlfeti_stats *stats);
/* Same with device arrays (already resident; the call is asynchronous on the
 * context stream except for a few scalar reads of convergence flags). */
nlfeti_status nlfeti_solve_device(nlfeti_problem *p, int nrhs, int rhs_kind, const double *d_rhs,
                                  const double *d_g, double *d_u_out, nlfeti_stats *stats);

/* The paper's baseline solver (section "Considered solver strategies"): conjugate gradients
 * with the diagonal preconditioner on the single-domain system A u = F - A_D g, FP64, on the
 * same mesh, kernel, loads and Dirichlet data as nlfeti_solve, for comparing the two solvers
 * on one GPU.  A is assembled once per problem as CSR over the global dofs from the subdomain
 * matrices (which sum to A through the zeta weights; Dirichlet dofs get identity rows):
 * nlfeti_cg_prepare does it explicitly (host work and a device upload, synchronous),
 * otherwise the first CG solve does.  The CG stops per right-hand side at
 * ||r||_2 <= opt.tol ||b||_2 or after opt.max_it iterations (NLFETI_E_NOT_CONVERGED, output
 * still written); stats.iterations is the largest count over the right-hand sides and
 * stats.final_rel_residual the largest ||r|| / ||b||.  At most 32 right-hand sides per call
 * (NLFETI_E_INVALID beyond).  Arguments, layouts and stream behaviour as nlfeti_solve /
 * nlfeti_solve_device.  The options precision, precond_fp16 and refinement fields do not
 * apply; batched = 0 runs the loop without graphs. */
nlfeti_status nlfeti_cg_prepare(nlfeti_problem *p);
nlfeti_status nlfeti_solve_cg(nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs, const double *g,
                              double *u_out, nlfeti_stats *stats);
nlfeti_status nlfeti_solve_cg_device(nlfeti_problem *p, int nrhs, int rhs_kind, const double *d_rhs,
                                     const double *d_g, double *d_u_out, nlfeti_stats *stats);

/* Introspection for bit-exact tests (host arrays, caller-sized from nlfeti_info):
 * n_k[K], n_gamma[K], node lists (sum n_k / ncomp node ids, Omega first then
 * Gamma per subdomain), B rows as U indices (n_lambda each), floating[K]. */
nlfeti_status nlfeti_get_decomposition(const nlfeti_problem *p, int32_t *n_k, int32_t *n_gamma, int32_t *node_lists,
                                       int64_t *B_plus, int64_t *B_minus, int8_t *floating);

/* Replace the assembled matrix A^k of subdomain k (n_k x n_k, row-major FP64 host array in
 * the subdomain's dof order, Omega_k dofs first, as nlfeti_get_operator which 0 returns) with
 * the caller's own, e.g. a matrix assembled by other quadrature (eq. bilinear-multi1 defines
 * what it stands for; the Dirichlet coupling and the loads are unchanged).  Copied before the
 * call returns.  The factorizations and the single-domain CG matrix of the problem are
 * dropped: nlfeti_factor must run again before the next solve (solves return
 * NLFETI_E_INVALID until then).  A matrix whose Omega block or pinned Neumann block is not
 * positive definite makes that nlfeti_factor return NLFETI_E_NOT_SPD, after which the problem
 * stays usable (set a valid matrix and factor again).  NLFETI_E_INVALID for k out of range or
 * a non-finite entry. */
nlfeti_status nlfeti_problem_set_matrix(nlfeti_problem *p, int k, const double *A);

/* Autotuner of the batched interface apply (the persistent bulk-copy pipeline that applies
 * S_k^+ and S_k in every PCG iteration; the paper has no counterpart, its subdomain solves run
 * on CPUs).  Its shape for nrhs right-hand sides: rc, the right-hand sides per streamed pass
 * over the operator (1, 2, 4, 8 or 16, at most nrhs; 8 for FP64: fewer passes read the operator
 * fewer times but hold more accumulators), ctas_per_sm (1 or 2) of its persistent grid, and
 * rows_per_warp (4, or 8 for the FP32 and FP16 operators with rc >= 4: half the consumer warps,
 * each shared-memory load of x serving twice the rows).
 * nlfeti_autotune times every candidate with CUDA events on the problem's factored operators
 * for each operator kind it has -- 0 FP32 S_k^+ and S_k, 1 the FP16 copy of S_k the mixed
 * path's preconditioner applies, 2 FP64 -- and keeps the fastest in the problem: later solves
 * and applies with nrhs right-hand sides use it.  cache_path (nullable): a JSON file of earlier
 * choices keyed by the device, the subdomain operator shapes, the kind and nrhs; a choice found
 * there is used without timing (from_cache = 1), new ones are added (the file is rewritten).
 * For kind 1 the candidates also include the tensor-core apply of the FP16 copy (tcgen05 kind::f16
 * with x in FP16 scaled per column, as precond_fp16 = 2 selects; nrhs <= 64), reported as
 * rc = -1; it builds the tiled FP16 copy of S_k when chosen.
 * out: up to 3 entries (one per kind), *n_out their number.  Every shape of the bulk-copy apply
 * gives bitwise the same results (each column is summed in the same order whatever the pass
 * width and schedule); the tensor-core preconditioner rounds differently (it only steers the
 * PCG: the iteration count may change, not the accuracy reached).
 * nlfeti_set_apply_choice pins a shape (rc 0 clears it, back to the default: the widest block
 * up to nrhs, two CTAs per SM, 4 rows per warp; rc -1 selects the tensor-core apply for kind 1;
 * rows_per_warp 0 means 4);
 * NLFETI_E_INVALID for shapes outside the lists above. */
typedef struct {
    int32_t kind, nrhs, rc, ctas_per_sm;
    double us;              /* mean time per apply launch of the chosen shape */
    int32_t from_cache;
    int32_t rows_per_warp;  /* 4 or 8 */
} nlfeti_tune_entry;
nlfeti_status nlfeti_autotune(nlfeti_problem *p, int nrhs, const char *cache_path, nlfeti_tune_entry *out,
                              int *n_out);
nlfeti_status nlfeti_set_apply_choice(nlfeti_problem *p, int kind, int nrhs, int rc, int ctas_per_sm,
                                      int rows_per_warp);

/* Fault injection for tests of the bounded device waits (not for production use; the paper has
 * no counterpart).  The batched interface apply (a persistent bulk-copy pipeline) bounds every
 * mbarrier wait: a wait that runs out sets the workspace's error word, the CTA lets the copies
 * it issued land and returns, and the solve returns NLFETI_E_TIMEOUT with the context usable.
 * wait_tries: polls of a stage barrier before the apply's consumers give up (0 = the default,
 * 2^24 polls, seconds); withhold_copies = 1: the apply's producer issues no copies, so that the
 * consumers' first wait runs out with nothing in flight.  Applies to the solves that follow
 * (the batched path; the per-subdomain baseline has no waits).  NLFETI_E_INVALID for negative
 * tries or withhold_copies outside 0/1. */
nlfeti_status nlfeti_debug_apply_waits(nlfeti_problem *p, long long wait_tries, int withhold_copies);

/* Copy one subdomain operator to the host (row-major, FP64):
 * which 0 = assembled A^k (n_k x n_k), 1 = S_k (n_g x n_g), 2 = S_k^+ (n_g x n_g);
 * precision 0 = FP64 operators, 1 = FP32 operators (widened). */
nlfeti_status nlfeti_get_operator(const nlfeti_problem *p, int k, int which, int precision, double *out);

/* Apply one FETI operator to host vectors (nrhs columns, column-major):
 * op 0 = F = B S^+ B^T (Lambda -> Lambda), 1 = M^-1 = B_D S B_D^T, 2 = P (eq. P),
 * 3 = S^+ (U -> U), 4 = S (U -> U), 5 = S (U -> U) through the copy the preconditioner of
 * the mixed path applies (precision 1 and the options' precond_fp16: FP16 on the FP32 pipes,
 * FP16 on the tensor cores with x scaled per column by a power of two from its largest
 * entry, or FP32; precision 0: the FP64 S). */
nlfeti_status nlfeti_apply(nlfeti_problem *p, int op, int precision, int nrhs, const double *in, double *out);

/* No-allocation interface apply (the paper has no counterpart: an integration entry point).
 * d_out = blockdiag_k(M_k) d_in with M_k = S_k^+ (which 0) or S_k (which 1), the operators of
 * the given precision (0 FP64, 1 FP32; factored before).  d_in, d_out: device arrays,
 * column-major n_u x nrhs (FP64), U ordered as in nlfeti_apply; d_out is written, d_in only
 * read.  For callers that must not allocate device memory during the call (a fixed memory
 * plan frozen after warm-up, a framework that forbids allocations between its own, an
 * allocator that would synchronise the device): the call makes no cudaMalloc, cudaFree or
 * allocator-callback call.  It stages its input in a scratch array that is part of the
 * library's device image, NLFETI_NOALLOC_SCRATCH_BYTES per device; it needs
 * n_up * nrhs * (8 for precision 0, 4 for precision 1) bytes of it, n_up being the sum over
 * subdomains of n_gamma rounded up to a multiple of 8.  Larger requests return
 * NLFETI_E_INVALID (nothing launched; nlfeti_last_error gives the sizes).  All calls on a
 * device share that scratch: calls that can overlap in time (other threads, other streams)
 * race, so the caller serialises them.  Nothing in it has to start at zero.  The first call
 * on a device resolves the scratch address with that device current (once); a caller that
 * captures streams makes that first call before capturing.  The call must be made with the
 * device of the problem's context current (NLFETI_E_INVALID otherwise).  Asynchronous on the context
 * stream, ordered after the caller's stream and before its later work (as
 * nlfeti_solve_device). */
#define NLFETI_NOALLOC_SCRATCH_BYTES (8u << 20)
nlfeti_status nlfeti_apply_schur_noalloc(nlfeti_problem *p, int which, int precision, int nrhs, const double *d_in,
                                         double *d_out);

/* Kernel accounting of a problem's solves (for roofline reporting).  With profiling on,
 * every launch of the dense interface apply (the per-iteration products with S_k^+ and
 * S_k) is bracketed by CUDA events on the library stream, also inside captured graphs.
 * kernel_launches counts every kernel of the library launched by solves (graph kernel
 * nodes included).  apply_*: launches, milliseconds and bytes read (operator entries plus
 * x and y per launch) of the applies with the operators in their stored precision;
 * half_apply_*: the same for the preconditioner's applies of the FP16 copy of S_k (mixed
 * path with precond_fp16).  Reading resets the counters. */
typedef struct {
    int64_t kernel_launches;
    int64_t apply_launches;
    double apply_ms;
    double apply_bytes;
    int64_t half_apply_launches;
    double half_apply_ms;
    double half_apply_bytes;
} nlfeti_profile;
nlfeti_status nlfeti_set_profiling(nlfeti_problem *p, int on);
nlfeti_status nlfeti_get_profile(nlfeti_problem *p, nlfeti_profile *out);

/* Serving (the paper's setup amortized over repeated solves, Sec. 6.4): a server takes solve
 * requests as they arrive and runs them on max_slots slots, each a worker thread with its own
 * CUDA stream, so the kernels of the batches in flight overlap on the device.  Continuous
 * batching: when a slot starts the oldest admissible request it also takes the other queued
 * requests on the same problem with the same rhs_kind (up to 64 right-hand sides in all) and
 * runs them as one batched solve whose launches serve all of them; a request that arrives while
 * a batch of its problem runs joins the next one.  Every column of a batched solve is computed
 * in an order that does not depend on the other columns, so each request's result is bitwise
 * the one it gets alone.  Right-hand-side counts are rounded up to buckets (zero columns) so
 * that workspaces and their captured PCG loops are reused.
 * Admission by device footprint: the server counts the bytes it holds -- its solve workspaces
 * (in use or kept for reuse) and the problems it created for nlfeti_submit_mesh requests --
 * against hbm_budget (0 = no limit), evicting idle ones least recently used first; a batch
 * that does not fit waits.  Problems created by the caller (nlfeti_submit) are the caller's
 * memory and are not counted.  The caller must not use the context or the problems passed to
 * nlfeti_submit from other threads while the server runs requests on them.
 * nlfeti_submit: a request on a factored problem (copies rhs and g: n_dofs x nrhs, column-major;
 * 1 <= nrhs <= 64); NLFETI_E_NOMEM when the request alone exceeds the budget.
 * nlfeti_submit_mesh: a request on the problem given by its inputs (as nlfeti_problem_create,
 * with the options opt or the defaults; all copied): factorization cache keyed by a hash of
 * the mesh, kernel, decomposition and options -- the first request of a key creates, assembles
 * and factors the problem (stats ms_setup / ms_factor), later ones reuse it while it stays
 * cached; invalid inputs fail the request with NLFETI_E_INVALID at nlfeti_wait.
 * nlfeti_wait: the result (u_out as nlfeti_solve) and stats (ms_queue: submission to start,
 * ms_solve: start to result); NLFETI_E_TIMEOUT if not done within timeout_ms (< 0: no limit),
 * the request stays pending.  Submission never blocks on the GPU. */
nlfeti_status nlfeti_server_create(nlfeti_ctx *ctx, size_t hbm_budget, int max_slots, nlfeti_server **out);
nlfeti_status nlfeti_submit(nlfeti_server *s, nlfeti_problem *p, int nrhs, int rhs_kind, const double *rhs,
                            const double *g, nlfeti_ticket *out);
nlfeti_status nlfeti_submit_mesh(nlfeti_server *s, const nlfeti_mesh *mesh, const nlfeti_kernel *kernel,
                                 const nlfeti_decomp *decomp, const nlfeti_options *opt, int nrhs, int rhs_kind,
                                 const double *rhs, const double *g, nlfeti_ticket *out);
nlfeti_status nlfeti_wait(nlfeti_server *s, nlfeti_ticket t, int timeout_ms, double *u_out, nlfeti_stats *stats);

/* Server counters: finished requests, batches run, requests that ran in a batch with others,
 * factorization-cache hits / misses / evictions and problems cached, the most slots busy at
 * once, requests queued, and the device bytes the server holds now and at most so far. */
typedef struct {
    int64_t requests_done, batches, merged_requests;
    int64_t problem_hits, problem_misses, problems_evicted;
    int32_t problems_cached, peak_active, queued;
    size_t bytes_in_use, peak_bytes;
} nlfeti_server_info;
nlfeti_status nlfeti_server_get_info(nlfeti_server *s, nlfeti_server_info *out);
void nlfeti_server_destroy(nlfeti_server *s);

#ifdef __cplusplus
}
#endif
#endif
