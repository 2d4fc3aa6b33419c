/*
 * hs.h -- C ABI of the GB300 hierarchical sparse solver.
 *
 * The method is the hierarchical solver of arXiv 1611.03189 (Yang, Pouransari,
 * Darve, "Sparse Hierarchical Solvers with Guaranteed Convergence"): the
 * LoRaSp factorization (Sec. 3) and its GC enrichment (Sec. 6), applied as a
 * preconditioner (Appendix A, Algorithm 2) inside conjugate gradients.
 *
 * Conventions for every entry point:
 *   - Return value is an hs_status code; HS_OK is 0.  On failure a message is
 *     available from hs_last_error() (thread-local, valid until the next call
 *     on the same thread).  No C++ exception ever crosses this boundary.
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     calls that take a factorization handle must run with the device it
 *     was created on current (HS_ERR_INVALID otherwise);
 *     "host" pointers are ordinary CPU memory.  Arguments are borrowed for the
 *     duration of the call only; the library keeps no reference to them.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; calls that must read results back synchronise it.
 *   - There is no CPU fallback: without a CUDA device every compute call
 *     returns HS_ERR_CUDA.
 *   - Dense vectors with several right-hand sides are column-major: column j
 *     (right-hand side j) starts at ptr + j*ld, ld >= n.
 */
#ifndef HS_H
#define HS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HS_OK = 0,
  HS_ERR_INVALID = 1,         /* bad argument, CSR, clustering or option          */
  HS_ERR_NOT_SPD = 2,         /* a pivot block (A_ss, S or the root) lost
                                 positive definiteness; see hs_last_error()      */
  HS_ERR_CAPACITY = 3,        /* a size exceeded a fixed library limit             */
  HS_ERR_OOM = 4,             /* device or host allocation failed                  */
  HS_ERR_NO_CONVERGENCE = 5,  /* hs_pcg hit maxit; x, iters, relres still filled   */
  HS_ERR_TIMEOUT = 6,         /* a bounded device wait ran out                     */
  HS_ERR_CUDA = 7             /* CUDA runtime error or no device                   */
} hs_status;

/* Compression variants (Sec. 3.2 and Sec. 6). */
enum {
  HS_LORASP = 0,       /* truncated SVD of A_sw only (Sec. 3.2)                  */
  HS_GC_CONSTANT = 1,  /* GC: also preserve the constant vector (Sec. 6, Sec. 7) */
  HS_GC_USER = 2,      /* GC: preserve caller-supplied vectors phi (Sec. 6)      */
  HS_GC_PROJ = 3       /* Appendix B, first-order one-sided projection: U_1 from
                          the truncated SVD of [X_s, A_sw X_w] at eps1, then GC */
};

/* Elimination order of the super nodes of a level (hs_opts.order_mode). */
enum { HS_ORDER_WAVES = 0, HS_ORDER_SEQUENTIAL = 1 };

/* Most preserved vectors per problem (n_phi) for HS_GC_USER and HS_GC_PROJ. */
#define HS_MAX_PHI 4

/* Arithmetic of the factorization (the PCG is always FP64).  The mixed
 * precisions keep blocks and factor records in FP32 and run the dense
 * contractions of the elimination (Sec. 3.2 eqs. extended_rearranged and
 * eliminated: L^-1 U and its CholQR, L^-1 A_sN, M_ss, P_ss, A_Nr, A_rr, the
 * Schur update; the blocked Cholesky's panel and trailing updates) on the
 * tensor cores; the outer FP64 PCG wins the accuracy back. */
enum {
  HS_PREC_F64 = 0,     /* every factor step in FP64                              */
  HS_PREC_F32 = 1,     /* blocks, Gram, eigen-solves and factor records in FP32
                          (CUDA cores); the rank is decided on the FP32
                          eigenvalues of the Gram matrix (an FP64 Sturm count
                          and threshold comparison on the FP32 tridiagonal),
                          or entirely in FP64 with hs_opts.rank_f64          */
  HS_PREC_TF32 = 2,    /* contractions on tensor cores with TF32 operands and
                          FP32 accumulation; blocks, records and the
                          truncation as HS_PREC_F32 (hs_opts.rank_f64 moves
                          the truncation to FP64)                           */
  HS_PREC_BF16 = 3,    /* as HS_PREC_TF32 with BF16 operands                    */
  HS_PREC_TF32X3 = 4   /* contractions on tensor cores with each FP32 operand
                          split into TF32 high and low parts, a b taken as
                          a_hi b_hi + a_hi b_lo + a_lo b_hi (near-FP32
                          accuracy), FP32 accumulation; truncation as
                          HS_PREC_F32                                          */
};

/* Sparse SPD matrix A in CSR form (Sec. 2: A symmetric positive definite).
 * rowptr[n+1], col[nnz], val[nnz]: DEVICE pointers, int32 / int32 / float64.
 * The pattern must be structurally symmetric with a full diagonal; columns
 * within a row may come in any order. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t *rowptr;
  const int32_t *col;
  const double *val;
} hs_csr;

/* Leaf clustering (Sec. 3: 2N = 2^L red nodes; "recursively bisecting").
 * HOST pointers.  perm[p] = original index of the p-th unknown in cluster
 * order (a permutation of 0..n-1).  Leaf i holds cluster-order unknowns
 * leaf_ptr[i] .. leaf_ptr[i+1]-1; nleaf must be a power of two, leaves must be
 * non-empty and in sibling order (leaves 2j and 2j+1 are merged first).
 * nbr_dist: the neighbour rule (Sec. 3.1).  0 or 1: two nodes of a level are
 * neighbours when their leaf sets are joined by an edge of the original
 * graph, the paper's algebraic rule; every other block is well separated and
 * compressed.  2: also the nodes of a level that share a neighbour, an
 * algebraic stand-in for the geometric rule of the paper's experiments
 * (Sec. 7: well separated when the distance exceeds the cluster size), which
 * compresses less.  Other values are HS_ERR_INVALID. */
typedef struct {
  const int32_t *perm;
  const int32_t *leaf_ptr;
  int32_t nleaf;
  int32_t nbr_dist;
} hs_clustering;

/* Device-memory hook (hs_opts.allocator).  The paper has no counterpart:
 * this is how a caller that manages device memory itself -- a serving loop
 * that admits work against a fixed budget, or a framework with its own
 * caching allocator (PyTorch's) -- makes the handle take every block of
 * device memory it holds from that allocator, so that the caller's count of
 * the bytes in use is exact.
 *   alloc(bytes, device, stream, ctx): returns a DEVICE pointer to `bytes`
 *     bytes on `device`, 256-byte aligned, that work enqueued on `stream` may
 *     use at once (stream-ordered, as the PyTorch caching allocator and
 *     cudaMallocAsync give), or NULL when it cannot; the library then fails
 *     the call with HS_ERR_OOM.  A failed hs_factor_create (or batch create)
 *     returns every block it took; a handle whose refactor or solve ran out
 *     keeps what it holds until a later call succeeds or hs_factor_destroy.
 *     A misaligned pointer is handed back through free and the call fails
 *     with HS_ERR_INVALID.
 *   free(ptr, device, stream, ctx): takes back a pointer alloc returned.  The
 *     library first synchronises `stream`, the stream of the call that gives
 *     the block back (hs_factor_destroy: the stream of the last
 *     factorization; a solve that grows its workspaces: its own), so no work
 *     the library enqueued there still uses the block.  It does not
 *     synchronise the whole device (that would break CUDA graph captures
 *     under way in other threads), so work of the handle that the caller
 *     enqueued on other streams must have completed by then, and the stream
 *     of the last factorization must still exist when hs_factor_destroy
 *     runs: the same rules as for any stream-ordered allocator.
 *   ctx: passed through unchanged.
 * Both are called on the calling thread, inside library calls on the handle
 * (creation, refactor, the solves, which grow their workspaces on first use
 * of a larger right-hand-side count, and destroy), never concurrently for one
 * handle.  The hook covers the device memory a handle owns: its copies of the
 * CSR, blocks and factor records, the factorization's scratch and task
 * descriptors, and the solve workspaces.  Pinned host staging buffers, the
 * per-device autotuner table and hs_gemm_tc's buffers are not handle memory
 * and use the CUDA runtime.  The struct is copied at creation; the functions
 * and ctx must stay valid until hs_factor_destroy returns. */
typedef void *(*hs_alloc_fn)(uint64_t bytes, int32_t device, void *stream, void *ctx);
typedef void (*hs_free_fn)(void *ptr, int32_t device, void *stream, void *ctx);
typedef struct {
  hs_alloc_fn alloc;
  hs_free_fn free;
  void *ctx;
} hs_allocator;

/* Factorization options.
 * eps: truncation tolerance (Sec. 3.2, "compression threshold"); a singular
 *   value is kept when sigma_i > eps * ||A_sw||_2.  eps == 0 disables
 *   truncation (every red node keeps a complete basis; the factorization is
 *   then exact).  0 < eps < 1e-6 is rejected (HS_ERR_INVALID): the Gram-matrix
 *   eigen-solve cannot resolve singular values that small.
 * variant: HS_LORASP, HS_GC_CONSTANT, HS_GC_USER or HS_GC_PROJ.
 * phi: HOST pointer, n_phi vectors of n doubles each (vector j at phi + j*n),
 *   in the ORIGINAL ordering; used by HS_GC_USER (vectors preserved exactly,
 *   Sec. 6) and HS_GC_PROJ (the scaled vectors X of Appendix B, e.g.
 *   e_i / lambda_i, kept approximately).  Required by both.
 * factor_prec: HS_PREC_F64, HS_PREC_F32, HS_PREC_TF32, HS_PREC_BF16 or
 *   HS_PREC_TF32X3.
 * eps_level: NULL, or a HOST array of tolerances per level for the adaptive
 *   choice of Sec. 7 (Table 3).  Entry j replaces eps for the super nodes j
 *   levels above the leaves (j = 0: the pairs of leaves); a problem with 2^L
 *   leaves reads entries 0 .. L-2, and n_eps_level must cover them.  Each
 *   entry obeys the rules of eps.  The same list serves problems of different
 *   depth in hs_factor_create_batch.
 * n_phi: number of vectors in phi, 1 .. HS_MAX_PHI (0 reads as 1); must be
 *   1 or 0 for HS_LORASP and HS_GC_CONSTANT.
 * eps1: HS_GC_PROJ's first tolerance (Appendix B, eps_1 <= eps_2 = eps): U_1
 *   keeps the left singular vectors of [X_s, A_sw X_w] with
 *   sigma_i > max(eps1, 1e-12) * sigma_1.  Finite and >= 0; ignored by the
 *   other variants.
 * scale: 0, or 1 to factor the symmetrically scaled D^-1/2 A D^-1/2 (D =
 *   diag A) instead of A and apply A_H^-1 = D^-1/2 A'_H^-1 D^-1/2.  The paper
 *   does not mention scaling; it keeps every row of A_sw on one scale, which
 *   GC-constant needs to stay definite at high coefficient contrast.  With
 *   scaling, GC-constant preserves the constant vector of the scaled system
 *   and HS_GC_USER / HS_GC_PROJ vectors phi are mapped to D^1/2 phi, so they
 *   stay preserved for A.  hs_pcg and hs_gmres still solve A x = b.  A
 *   diagonal entry <= 0 is HS_ERR_NOT_SPD.
 * timeout_cycles: bound, in SM clock cycles, of each wait inside the
 *   handle's kernels: the tensor-core GEMM of HS_PREC_TF32 / HS_PREC_BF16 /
 *   HS_PREC_TF32X3 (its mbarriers) and the grid barriers of the opt-in
 *   persistent apply (HS_APPLY_PERSISTENT=1); 0 means the default, 2e9
 *   cycles (about one second).  A wait that runs out makes the call fail
 *   with HS_ERR_TIMEOUT (the factorization, or hs_pcg / hs_gmres for the
 *   apply); the device stays usable (the GEMM waits for its own tensor-core
 *   work with the default bound before it frees its tensor memory and
 *   returns).  A bound far below a real wait (a few microseconds) fails
 *   correct work.  >= 0.
 * order_mode: the elimination order of a level's super nodes, "a given
 *   ordering" in Sec. 3.2.  HS_ORDER_WAVES (0, the default): canonical waves
 *   (see the planner below), each wave one batch of independent
 *   eliminations.  HS_ORDER_SEQUENTIAL (1): one super node at a time in
 *   ascending index, the paper's sequential reading; the same method, one
 *   launch group per super node (slow; for comparison).
 * max_rank_ratio: 0 (no cap), or in (0, 1]: every truncation with eps > 0
 *   keeps at most max(floor(max_rank_ratio * m), 1) columns -- the leading
 *   singular vectors (GC: the basis U_1 whole, then the leading ones of the
 *   projected block) -- bounding the red nodes' sizes and so the factor's
 *   memory.  Not in the paper; a cap that binds trades preconditioner
 *   quality for memory, and a harsh one can cost GC-constant its
 *   definiteness (HS_ERR_NOT_SPD).
 * allocator: NULL (the CUDA runtime: cudaMalloc / cudaFree), or a device-
 *   memory hook (hs_allocator above) with both functions set; the handle
 *   takes all its device memory from it.  hs_factor_create_batch gives every
 *   handle of the batch the same hook.
 * rank_f64: 0, or 1 to keep the truncation of the FP32 / TF32 / BF16 /
 *   3xTF32 factors in FP64: the Gram matrix A_sw A_sw^T (and A_sw phi_w) is
 *   formed in FP64 from FP64 copies of the FP32 blocks, eigen-decomposed in
 *   FP64, the rank decided in FP64 (Sec. 3.2 threshold; Sec. 6 for GC), and
 *   the basis U rounded to FP32 for the elimination, which stays in the
 *   factor precision.  The rank then answers for the FP32 blocks themselves
 *   rather than for an FP32 eigen-solve of their Gram matrix.  It costs the
 *   FP64 eigen-solves (GB300's FP64 rate is a small fraction of its FP32
 *   rate).  Ignored by HS_PREC_F64, which decides in FP64 anyway. */
typedef struct {
  double eps;
  int32_t variant;
  int32_t factor_prec;
  const double *phi;
  const double *eps_level;
  int32_t n_eps_level;
  int32_t n_phi;
  double eps1;
  int32_t scale;
  int64_t timeout_cycles;
  int32_t order_mode;
  double max_rank_ratio;
  const hs_allocator *allocator;
  int32_t rank_f64;
} hs_opts;

/* Sizes and counters of a factorization (all host values). */
typedef struct {
  int64_t n;
  int32_t levels;            /* L = log2(nleaf)                                   */
  int32_t waves;             /* total number of elimination waves                 */
  int32_t super_nodes;       /* super nodes eliminated (root excluded)            */
  int32_t root_size;         /* size of the dense root block (0 if none)          */
  int32_t max_rank;          /* largest red-node size k                           */
  int32_t max_super;         /* largest super-node size m                         */
  int64_t device_bytes;      /* device memory held by the handle                  */
  int64_t factor_bytes;      /* bytes one hs_apply reads from the factor records  */
  double factor_flops;       /* flops the factorization's GEMM and Cholesky
                                kernels execute (2MNK per product, m^3/3 per
                                Cholesky); see alg_flops for the algorithmic count */
  double eig_flops;          /* nominal eigen-solve flops, reported apart: per
                                truncated node 4/3 m^3 + 2 m^2 k                  */
  double factor_ms;          /* device time of the last factorization             */
  double trunc_big_ms;       /* device time of the large-node truncation launches
                                (tridiagonal eigen path), CUDA events             */
  double trunc_big_flops;    /* nominal eigen-solve flops of those nodes          */
  int32_t trunc_big_launches;/* waves that ran the large-node truncation (one
                                launch per thread-count class in each)            */
  double host_ms;            /* host wall time of the factorization call          */
  double wait_ms;            /* of which waiting for the device (rank reads)      */
  double phase_ms[16];       /* with hs_profile_phases(1): device time of the
                                factor's launch groups -- 0 merge, 1 gather of
                                A_sN/A_sW, 2 Cholesky of A_ss, 3 Gram, 4 small
                                truncation, 5 large truncation, 6 CholQR of the
                                large-path U, 7 extension GEMMs and CholQR, 8
                                Schur scatter, 9 root; within 5, the multi-CTA
                                path: 10 prepare, 11 tridiagonal steps, 12 Q^T Z,
                                13 eigenvectors of T, 14 Q Y; 15 unused;
                                otherwise zeros                                 */
  double alg_flops;          /* algorithmic flops of the factorization, counted
                                per super node from its sizes (m, rank k,
                                well-separated width w, neighbour width d_N):
                                Gram 2m^2 w, R^T 2mkw, Cholesky m^3/3, Y 2m^2 k,
                                S 2mk^2 + k^3/3, G 2m^2 d_N, H 2mk d_N, Schur
                                2(m+k) d_N^2, M_ss and P_ss 2m^2 k; root m^3/3.
                                factor_flops counts what the kernels execute.  */
  double tc_flops;           /* flops executed by the tensor-core GEMM          */
  double tc_ms;              /* device time of its launches (CUDA event pairs)  */
  int64_t tc_launches;       /* its launches in the last factorization          */
} hs_info;

typedef struct hs_factor_s *hs_factor;

/* hs_factor_create: hierarchical factorization of A (Algorithm 1; Sec. 3.2 and
 * Sec. 6 for the compression).  A is borrowed; the handle keeps its own copy of
 * what the solves need.  On success *out owns device memory until
 * hs_factor_destroy.  Errors: HS_ERR_INVALID, HS_ERR_NOT_SPD (message names the
 * level and super node), HS_ERR_OOM, HS_ERR_CUDA. */
int hs_factor_create(const hs_csr *A, const hs_clustering *cl, const hs_opts *opts,
                     void *stream, hs_factor *out);

/* hs_factor_refactor: factor new values of the same matrix pattern with the
 * same clustering and options (Algorithm 1 again; the symbolic plan is reused).
 * val: DEVICE, nnz doubles in the order of the CSR given to hs_factor_create.
 * The previous factorization is released.  On error the handle holds no valid
 * factorization until the next successful refactor. */
int hs_factor_refactor(hs_factor f, const double *val, void *stream);

/* hs_factor_create_batch: `count` independent systems factored together.
 * The paper factors one matrix; this batched form has no counterpart there.
 * Each problem follows Algorithm 1 exactly as hs_factor_create would do it
 * alone.  The problems advance in lock step: at every step (a level counted
 * from the leaves, then a wave of that level) the work of every problem that
 * has the step runs in the same kernel launches, with one read of the new
 * ranks for all of them.
 *   A, cl: arrays of `count` problems (the same layout and ownership as in
 *     hs_factor_create).
 *   opts: one set for all problems (eps, variant, factor_prec).  opts->phi is
 *     ignored.
 *   phi: per-problem preserved vectors (HOST, opts->n_phi vectors of n_p
 *     doubles each, laid out as opts->phi) for HS_GC_USER and HS_GC_PROJ;
 *     otherwise it may be NULL.
 *   out: `count` handles, each used and destroyed like one from
 *     hs_factor_create.
 *   status: NULL, or `count` ints that receive each problem's own result.
 * Results are those of factoring each problem alone, bit for bit.
 * Errors:
 *   - A problem whose pivot block is not positive definite leaves the lock
 *     step: status[p] = HS_ERR_NOT_SPD and out[p] = NULL.  The others are
 *     finished and returned.  The call then returns HS_ERR_NOT_SPD with the
 *     first failed problem named in hs_last_error.
 *   - Any other error fails the whole call and returns no handle. */
int hs_factor_create_batch(int32_t count, const hs_csr *A, const hs_clustering *cl,
                           const hs_opts *opts, const double *const *phi, void *stream,
                           hs_factor *out, int32_t *status);

/* hs_factor_refactor_batch: hs_factor_refactor of `count` distinct handles in
 * lock step, as in hs_factor_create_batch.  val[p] are DEVICE values of
 * handle f[p]'s pattern.  status: as in hs_factor_create_batch.  A handle
 * whose refactor failed holds no valid factorization until its next
 * successful refactor. */
int hs_factor_refactor_batch(int32_t count, hs_factor *f, const double *const *val, void *stream,
                             int32_t *status);

/* hs_apply: z = A_H^{-1} r (Appendix A, Algorithm 2: forward substitution,
 * restriction, parent solve, prolongation, backward substitution).
 * r, z: DEVICE, n x nrhs column-major with leading dimension ld >= n;
 * r and z may alias.  1 <= nrhs <= 64. */
int hs_apply(hs_factor f, const double *r, double *z, int32_t nrhs, int64_t ld, void *stream);

/* hs_apply_static: the same z = A_H^{-1} r as hs_apply, for callers that must
 * not allocate device memory while they solve -- for instance a service whose
 * device memory is fixed at start-up, or code that runs where a cudaMalloc
 * could block behind other work or is not permitted.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: the apply workspace is one 16 MiB
 * static device array inside this library, which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart; this
 * is a property of this library's interface only.
 *   - Needs (ws_unknowns x nrhs + 2 x scratch_unknowns x nrhs) elements of the
 *     factor precision; larger requests fail with HS_ERR_CAPACITY and a
 *     message giving the bytes needed.  r, z, nrhs, ld as for hs_apply.
 *   - The device the factorization was created on must be current
 *     (HS_ERR_INVALID otherwise).
 *   - Each call outside a stream capture looks up the array's device address
 *     (with that device current) and keeps it for calls made while a stream
 *     capture is in progress, which cannot look it up; so the first call on a
 *     device must come before any stream capture.
 *   - All calls on a device share the array and leave the last call's
 *     contents in it (the parts that must start at zero are cleared by each
 *     call).  Calls that overlap on the GPU -- on different streams or
 *     threads -- race on it: serialise them. */
int hs_apply_static(hs_factor f, const double *r, double *z, int32_t nrhs, int64_t ld, void *stream);

/* hs_pcg: solve A x = b by conjugate gradients preconditioned with A_H^{-1},
 * x_0 = 0, stopping when ||r_k||_2 <= rtol ||b||_2 for each right-hand side
 * (Sec. 7: relative residual 1e-10).  A is the matrix of the last successful
 * hs_factor_create / hs_factor_refactor.  b, x: DEVICE, n x nrhs column-major, leading dimension
 * ld.  iters, relres: HOST arrays of nrhs; iters[j] = completed CG updates of
 * column j, relres[j] = ||b_j - A x_j|| / ||b_j|| recomputed at the end.
 * Returns HS_ERR_NO_CONVERGENCE (with x, iters, relres filled) if some column
 * needs more than maxit iterations. */
int hs_pcg(hs_factor f, const double *b, double *x, int32_t nrhs, int64_t ld, double rtol,
           int32_t maxit, int32_t *iters, double *relres, void *stream);

/* hs_gmres: solve A x = b by GMRES right-preconditioned with A_H^{-1}, the
 * outer solver of the paper's experiments (Sec. 7, Tables 2-5), x_0 = 0, one
 * right-hand side, FP64.  Stops when the Arnoldi least-squares residual falls
 * below rtol ||b||_2 (Sec. 7: relative residual 1e-10), restarting every
 * `restart` steps (0: no restart).  A is the matrix of the last successful
 * hs_factor_create / hs_factor_refactor.  b, x: DEVICE, n doubles (original
 * ordering).  iters, relres: HOST; *iters = Arnoldi steps over all cycles,
 * *relres = ||b - A x|| / ||b|| recomputed at the end.  Flexible form: the
 * preconditioned vectors are kept and x is updated from them, so an FP32
 * factor (whose applications round differently) still reaches rtol on the
 * true residual.  The handle keeps the Krylov basis, (2 m + 6) n doubles of
 * device memory with m = restart, or maxit when restart is 0; m must be
 * <= 1000 (HS_ERR_INVALID otherwise).  Returns
 * HS_ERR_NO_CONVERGENCE (with x, iters, relres filled) after maxit steps. */
int hs_gmres(hs_factor f, const double *b, double *x, double rtol, int32_t maxit, int32_t restart,
             int32_t *iters, double *relres, void *stream);

/* hs_factor_info: sizes and counters of a factorization. */
int hs_factor_info(hs_factor f, hs_info *info);

/* hs_factor_ranks: red-node sizes k of one level (level = L .. 2, the level at
 * which the super node was eliminated).  ranks[i] = k of super node i, or -1 if
 * super node i had no well-separated block (no red node) or did not exist.
 * `cap` is the capacity of ranks; the number of super nodes of the level
 * (2^(level-1)) is returned in *count.  HOST arrays. */
int hs_factor_ranks(hs_factor f, int32_t level, int32_t *ranks, int32_t cap, int32_t *count);

/* hs_factor_destroy: release the handle and its device memory (NULL is OK). */
int hs_factor_destroy(hs_factor f);

/* hs_profile_phases: on != 0 makes later factorizations (all handles, all
 * threads) time their launch groups with CUDA events into hs_info.phase_ms;
 * 0 turns it off (the default).  A measurement aid; the paper has no
 * counterpart.  Returns HS_OK. */
int hs_profile_phases(int32_t on);

/* hs_gemm_tc: one C = alpha op(A) op(B) + beta C through the tensor-core GEMM
 * that the mixed factorizations use for their contractions (tcgen05, operands
 * rounded to TF32 or BF16, FP32 accumulation), exported so that the kernel can
 * be checked and measured on its own.  The paper has no counterpart.
 *   prec: HS_PREC_TF32, HS_PREC_BF16 or HS_PREC_TF32X3.  A, B, C: DEVICE,
 *   FP32, row-major;
 *   op(A) is M x K (A[i lda + k], or A[k lda + i] when ta), op(B) is K x N
 *   (B[k ldb + j], or B[j ldb + k] when tb), C is M x N with leading
 *   dimension ldc.  C must not overlap A or B.  M, N >= 1, K >= 0.
 *   bn: tile width, 64 or 128 (0: the library's choice).
 * The call synchronises `stream`.  HS_ERR_TIMEOUT if a bounded wait inside
 * the kernel ran out (C is then not fully written). */
int hs_gemm_tc(int32_t prec, int32_t M, int32_t N, int32_t K, float alpha, const float *A, int64_t lda,
               int32_t ta, const float *B, int64_t ldb, int32_t tb, float beta, float *C, int64_t ldc,
               int32_t bn, void *stream);

/* hs_gemm_tune_report: the table of the GEMM autotuner for operand
 * precision `prec` (HS_PREC_TF32, HS_PREC_BF16 or HS_PREC_TF32X3) on the
 * current device,
 * building it first if needed (that synchronises the device).  For each class
 * of task shapes c (max(M, N) bucket 0..4 = up to 32, 64, 128, 256, more; K
 * bucket 0..3 = up to 32, 128, 512, more; c = 4 * mn + k): ms[3c .. 3c+2] =
 * measured times of the CUDA-core kernel and of the tensor-core kernel with
 * 64- and 128-wide tiles on a synthetic batch of that class, route[c] = the
 * choice (0 CUDA cores, 64 or 128).  HOST arrays of 3 cap floats and cap ints.
 * Returns the number of classes (20), or a negative hs_status on error.  The
 * paper has no counterpart. */
int hs_gemm_tune_report(int32_t prec, float *ms, int32_t *route, int32_t cap);

/* hs_test_wait_probe: on != 0 makes every later tensor-core GEMM launch and
 * every later persistent apply launch (HS_APPLY_PERSISTENT=1; all handles, all
 * threads) first wait, with the handle's bound (hs_opts.timeout_cycles), on a
 * barrier that nothing completes, so that the wait runs out: the
 * factorization fails with HS_ERR_TIMEOUT before any tensor-core work is
 * issued, and hs_pcg / hs_gmres fail with HS_ERR_TIMEOUT (the time-out is
 * reported once; the handle stays usable).  0 turns it off (the default).  A
 * test of the time-out paths, which no GPU fault can exercise on a shared
 * machine; the paper has no counterpart.  The persistent apply's switch is a
 * device variable of the CURRENT device, read at run time (so recorded solve
 * graphs follow it).  Returns HS_OK, or an error when no CUDA device is
 * present. */
int hs_test_wait_probe(int32_t on);

/* hs_last_error: message of the last failing call on this thread. */
const char *hs_last_error(void);

/* hs_launch_count: number of CUDA kernels this library has launched in the
 * process so far (all handles, all threads). */
int64_t hs_launch_count(void);

/* hs_abi_sizes: sizeof of the ABI structs as this library was compiled --
 * sizes[0] hs_csr, [1] hs_clustering, [2] hs_opts, [3] hs_info,
 * [4] hs_allocator -- so that a binding can check its own struct layouts (no
 * device needed).  Writes min(cap, 5) entries and returns the number of
 * structs (5).  A build check; the paper has no counterpart. */
int hs_abi_sizes(int64_t *sizes, int32_t cap);

/* ---------------------------------------------------------------------------
 * Symbolic planner (host only; no device needed).  The elimination order is
 * "a given ordering" of super nodes (Sec. 3.2); this library uses canonical
 * waves: within a level, repeatedly take, in ascending super-node index, a
 * maximal set of super nodes no two of which share a block, and eliminate it.
 * Blocks and well-separatedness follow Sec. 3.1 (adjacency in the original
 * graph; fill-in creates blocks, never adjacency).
 * ------------------------------------------------------------------------- */
typedef struct hs_plan_s *hs_plan;

/* hs_plan_create: plan from the HOST CSR pattern (rowptr[n+1], col[nnz]) and
 * the clustering.  Errors: HS_ERR_INVALID, HS_ERR_OOM. */
int hs_plan_create(int64_t n, const int32_t *rowptr, const int32_t *col,
                   const hs_clustering *cl, hs_plan *out);

/* hs_plan_level_waves: for level `level` (L .. 2), writes wave_of[i] = wave
 * index of super node i (or -1 if the super node does not exist) for
 * i < 2^(level-1) <= cap, and *nwaves.  HOST arrays. */
int hs_plan_level_waves(hs_plan p, int32_t level, int32_t *wave_of, int32_t cap,
                        int32_t *nwaves);

/* hs_plan_super_lists: neighbour set N(s) and well-separated set W(s) of super
 * node s at `level`, as node keys (super j -> j, red node made from super j ->
 * 2^(level-1) + j), ascending.  Writes at most cap entries into each array;
 * *nn and *nw receive the full counts. */
int hs_plan_super_lists(hs_plan p, int32_t level, int32_t s, int32_t *nbrs, int32_t *wsep,
                        int32_t cap, int32_t *nn, int32_t *nw);

int hs_plan_destroy(hs_plan p);

#ifdef __cplusplus
}
#endif

#endif /* HS_H */
