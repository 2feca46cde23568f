/*
 * dmrg_heff.h -- C ABI of the GB300 (sm_103a) two-site DMRG effective-Hamiltonian
 * library: H_eff*psi and the Davidson eigensolver that calls it.
 *
 * The operation (paper: Numerical procedure, Eq. 2 and the Lanczos/Davidson step
 * after it, which takes ~80% of the run time and scales as O(D^3)): the local
 * two-site eigenproblem of DMRG with the effective Hamiltonian in symmetry-sector
 * form
 *
 *     H_eff = sum_t c_t (A_t (x) B_t) P_t ,
 *
 * A_t acting on the left enlarged block and shifting its (n, 2S_z) sector by
 * Delta_t, B_t acting on the right block and shifting it by -Delta_t, and
 * P_t = (-1)^{n_L} on the *input* left sector for terms with the parity flag
 * (odd Delta_n: fermionic operators that pass the left block), identity otherwise.
 * Block-wise, every term and every wave-function block q = (q_L, q_R) gives
 *
 *     y[q_L+Delta, q_R-Delta] += c_t s_t A_t[q_L+Delta <- q_L] x[q] B_t[q_R-Delta <- q_R]^T .
 *
 * Layouts
 *   sector tables   int32 (nsec x 3) rows (n, two_sz, dim), strictly ascending in
 *                   (n, two_sz), dim >= 1.
 *   wave function   blocks (q_L, q_R) with q_L + q_R = target, ascending in the
 *                   left sector, each row-major dim(q_L) x dim(q_R), concatenated;
 *                   nvec vectors are stored one after another (stride = dim).
 *   operator blocks A_t[p <- q] is row-major dim(p) x dim(q) at op_data[a_off[t*nl+q]],
 *                   p = q + Delta_t;  B_t[p <- q] is row-major dim(p) x dim(q) at
 *                   op_data[b_off[t*nr+q]], p = q - Delta_t.  Offset -1 = absent.
 *
 * Ownership: dmrg_heff_create copies every host array it is given; the handle owns
 * its device memory.  x, y, diag and x_inout of the device entry points are caller
 * owned device pointers.  A handle is not thread-safe; distinct handles are.
 * Errors: every entry point returns DMRG_OK (0) or a negative DMRG_ERR_* code; no
 * exception crosses the ABI.  dmrg_strerror gives a message, dmrg_last_error the
 * detail of the last failure on the calling thread.
 */
#ifndef DMRG_HEFF_H
#define DMRG_HEFF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DMRG_OK                   0
#define DMRG_ERR_INVALID_ARG     -1  /* null pointer, bad size, unsorted table, bad offset */
#define DMRG_ERR_SECTOR_MISMATCH -2  /* a block present for a shift whose sector is absent */
#define DMRG_ERR_OOM             -3  /* device or host allocation failed */
#define DMRG_ERR_CUDA            -4  /* a CUDA runtime call failed */
#define DMRG_ERR_DEVICE_TIMEOUT  -5  /* a bounded device-side wait gave up */
#define DMRG_ERR_NOT_CONVERGED   -6  /* Davidson stopped before reaching tol */
#define DMRG_ERR_BOUNDS          -7  /* bounds-checked build saw an out-of-range access */
#define DMRG_ERR_UNSUPPORTED     -8  /* option or size the library does not support  */

/* Arithmetic of the contractions. */
#define DMRG_PREC_FP64        0  /* FP64 DMMA tensor-core tiles (mma.sync m16n8k16 f64) */
#define DMRG_PREC_SPLIT_BF16  1  /* Ozaki split: FP64 operands as BF16 digit slices on
                                    tcgen05 tensor cores, exact FP32 partial sums,
                                    recombined in FP64 */

typedef struct dmrg_heff* dmrg_heff_t;

typedef struct {
    int32_t precision;  /* DMRG_PREC_*                                               */
    int32_t n_slices;   /* split path: digit slices per operand, 0 or 6 (the only
                           count built; others give DMRG_ERR_UNSUPPORTED)            */
    int32_t max_nvec;   /* largest nvec passed to apply (sizes the scratch), >= 1   */
    int32_t flags;      /* DMRG_FLAG_* bits                                           */
    int64_t split_mid_bytes;  /* split path: device bytes of stage-2 intermediate
                           slices per output chunk (0 = 64 GiB).  An apply takes the
                           output blocks in chunks whose intermediates fit under it and
                           reuses one buffer for them; results do not depend on it.  */
} dmrg_heff_opts;

/* Build only the host-side plan: no device memory is touched, so the handle works
 * without a GPU; only dmrg_heff_dim, _flops, _memory, _plan_dump and _destroy may be
 * called. */
#define DMRG_FLAG_PLAN_ONLY 1
/* Launch every apply kernel directly instead of replaying a CUDA graph.  By default
 * each apply is captured once per (x, y, nvec) into a graph (up to 64 per handle) and
 * replayed; per-kernel timing (dmrg_heff_profile) also launches directly. */
#define DMRG_FLAG_NO_GRAPH 2

typedef struct {
    /* outputs */
    int32_t iters;       /* Rayleigh-Ritz steps taken                                */
    int32_t matvecs;     /* vectors multiplied by H_eff                              */
    int32_t converged;   /* 1 if every wanted residual norm <= tol                   */
    int32_t restarts;    /* thick restarts taken                                     */
    double  resid_max;   /* largest residual norm of the wanted pairs at exit        */
    double  seconds;     /* wall time inside dmrg_davidson                           */
    /* optional inputs: per-step history (host arrays of hist_cap entries, or NULL)  */
    double* hist_theta;  /* lowest Ritz value after step i                           */
    double* hist_time;   /* seconds since the call started, at the end of step i     */
    int32_t hist_cap;
    int32_t pad;
} dmrg_davidson_info;

/* Build a handle: validate the tables, index the wave-function blocks, plan every
 * (term, block) contraction (cheaper of (A x)B^T and A(x B^T) by exact integer flop
 * count, A-first on a tie), lay the operator blocks out on the device and build the
 * grouped-GEMM work lists.  All pointers are host pointers; all arrays are copied.
 *   left, right : sector tables (nl x 3, nr x 3)
 *   target_*    : quantum numbers of the two-site wave function
 *   coef (T), delta (T x 2: dn, d2sz), parity (T: 0 or 1)
 *   a_off (T x nl), b_off (T x nr): block offsets into op_data (-1 = absent)
 *   op_data (op_len doubles), opts (NULL = FP64, max_nvec 1)
 * Returns DMRG_ERR_INVALID_ARG / _SECTOR_MISMATCH for malformed input, _OOM, _CUDA. */
int dmrg_heff_create(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
                     int32_t target_n, int32_t target_2sz,
                     const double* coef, const int32_t* delta, const int32_t* parity,
                     const int64_t* a_off, const int64_t* b_off, int64_t n_terms,
                     const double* op_data, int64_t op_len,
                     const dmrg_heff_opts* opts, dmrg_heff_t* out);

/*
 * Spin-adapted (SU(2)) H_eff (paper: the DMRG is spin-adapted, Introduction and
 * Numerical procedure).  Sectors are (n, 2S) multiplets: tables (n, two_s, dim) with
 * dim = number of multiplets, 0 <= two_s <= 40, strictly ascending in (n, two_s).
 * Term t is c_t sum_mu (-1)^{k-mu} T_mu U_-mu (times (-1)^{n_L(input)} if parity[t]),
 * T and U rank-k tensors (rank2[t] = 2k <= 40) shifting n by +dn[t] (left) and -dn[t]
 * (right), given by reduced blocks in the Clebsch-Gordan-normalised Wigner-Eckart
 * convention <S' m'| T_mu |S m> = <S m; k mu | S' m'> A[S' <- S].
 *   a_blocks (n_a x 4), b_blocks (n_b x 4): rows (term, in sector, out sector, offset of
 *       the row-major dim(out) x dim(in) block in op_data), any order, each at most once;
 *       out n = in n + dn (A) or in n - dn (B), (S_in, k, S_out) a triangle.
 * The reduced wave function of (target_n, target_2s) holds one block per sector pair
 * with n_L + n_R = target_n and (S_L, S_R, S) a triangle, in (left, right) order
 * (dmrg_heff_psi_blocks lists them); every (term, A block, B block) between two such
 * blocks contributes c_t s_t W A x B^T with W the recoupling coefficient of
 * dmrg_su2_recoupling.  The plan dump, apply, diagonal, Davidson, Lanczos and truncation
 * entry points work as for dmrg_heff_create.
 * Returns DMRG_ERR_INVALID_ARG / _SECTOR_MISMATCH for malformed input, _OOM, _CUDA. */
int dmrg_heff_create_su2(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
                         int32_t target_n, int32_t target_2s,
                         const double* coef, const int32_t* rank2, const int32_t* dn,
                         const int32_t* parity, int64_t n_terms,
                         const int64_t* a_blocks, int64_t n_a, const int64_t* b_blocks, int64_t n_b,
                         const double* op_data, int64_t op_len,
                         const dmrg_heff_opts* opts, dmrg_heff_t* out);

/* Recoupling coefficient of the spin-adapted terms (host only, all arguments twice the
 * spins): W = <(S_L' S_R') S M | sum_mu (-1)^{k-mu} T_mu U_-mu | (S_L S_R) S M> for unit
 * reduced blocks, computed as (-1)^{S_L+S_R'+k+S} sqrt((2S_L'+1)(2S_R'+1))
 * {S_L' S_L k; S_R S_R' S} (Racah's 6j sum); 0 unless every triangle holds.
 * DMRG_ERR_INVALID_ARG for a spin outside [0, 20] (total spin [0, 40]) or w NULL. */
int dmrg_su2_recoupling(int32_t two_sl_out, int32_t two_sr_out, int32_t two_sl_in, int32_t two_sr_in,
                        int32_t two_k, int32_t two_s, double* w);

/* Number of wave-function entries |psi| (0 for an empty target sector). */
int64_t dmrg_heff_dim(dmrg_heff_t h);

/* Algorithmic flops of one H_eff*psi for one vector: the sum over the plan of the
 * cheaper order's 2abc + 2acd or 2bcd + 2abd. */
int dmrg_heff_flops(dmrg_heff_t h, int64_t* flops);

/* Device memory of a handle, in bytes (for a plan-only handle: what a full handle with
 * the same options would hold).
 *   operators        the FP64 operator copy in the grouped layout (FP64 handles; a split
 *                    handle keeps none after set-up)
 *   operator_slices  split handles: the operators' digit slices, exponents and row sums
 *   apply_buffers    per-apply buffers for max_nvec vectors: FP64 stage-1 scratch and
 *                    split-K partials, or the split path's psi and intermediate slices,
 *                    exponents and stage-2 sums
 *   setup_peak       the largest transient buffer of set-up (split: the operator staging
 *                    buffer the FP64 operators are streamed through, block by block)
 *   total            operators + operator_slices + apply_buffers */
typedef struct {
    int64_t operators, operator_slices, apply_buffers, setup_peak, total;
} dmrg_memory;
int dmrg_heff_memory(dmrg_heff_t h, dmrg_memory* m);

/* Canonical plan: rows (out_block, term, in_block, order 0=A-first 1=B-first, flops),
 * int64, sorted by (out_block, term, in_block).  Call with buf = NULL to get *n_rows;
 * otherwise buf must hold *n_rows * 5 values. */
int dmrg_heff_plan_dump(dmrg_heff_t h, int64_t* buf, int64_t* n_rows);

/* y = H_eff x for nvec vectors (1 <= nvec <= max_nvec); x, y device pointers of
 * nvec*dim doubles, x and y must not overlap; runs asynchronously on `stream`
 * (a cudaStream_t, NULL = legacy default stream) as one CUDA-graph launch (the graph is
 * captured at the first call with these x, y, nvec; see DMRG_FLAG_NO_GRAPH). */
int dmrg_heff_apply(dmrg_heff_t h, const double* x, double* y, int32_t nvec, void* stream);

/* Same as dmrg_heff_apply with host x and y: copies x in, applies, copies y out and
 * waits for the result (pinned host memory gives the fastest copies). */
int dmrg_heff_apply_host(dmrg_heff_t h, const double* x, double* y, int32_t nvec);

/* diag (device, dim doubles) = diagonal of H_eff: sum over Delta = 0 terms of
 * c_t s_t A_t[l,l] B_t[r,r]. */
int dmrg_heff_diagonal(dmrg_heff_t h, double* diag, void* stream);

/* Lowest k_eig eigenpairs by block Davidson with FP64 CGS2 orthogonalisation,
 * Rayleigh-Ritz by cyclic Jacobi on the device, diagonal preconditioner and thick
 * restart; the steps are those of the library's documented Davidson variant.
 *   block      : vectors added per step (1 <= block <= min(8, max_nvec)); the basis
 *                holds max(8 block, 24) vectors and must fit k_eig + 2 block
 *   tol        : residual-norm target ||H x - theta x|| for unit x
 *   max_iter   : Rayleigh-Ritz steps allowed
 *   n_iter     : > 0 runs exactly this many steps (no convergence test), else 0
 *   x_inout    : device, max(block, k_eig)*dim doubles: the first `block` rows are the
 *                start block (need not be orthonormal); on return the first k_eig rows
 *                hold the Ritz vectors
 *   evals      : host, k_eig doubles; info: host, may be NULL.
 * Returns DMRG_ERR_NOT_CONVERGED (results still written) when tol was not met. */
int dmrg_davidson(dmrg_heff_t h, int32_t k_eig, double tol, int32_t max_iter, int32_t block,
                  int32_t n_iter, double* x_inout, double* evals, dmrg_davidson_info* info);

/* Lowest eigenpair by restarted Lanczos (paper: Numerical procedure, the Lanczos
 * alternative to Davidson named after Eq. 2): per step one H_eff product, the
 * three-term recurrence, full FP64 reorthogonalisation against the basis (two
 * Gram-Schmidt passes) and Rayleigh-Ritz on the tridiagonal matrix for its lowest
 * pair on the device (multisection on Sturm counts, then inverse iteration); explicit
 * restart from the Ritz vector when the basis holds m_max vectors.  Converged when the residual estimate beta_j |s_j| <= tol, or when the
 * Krylov space becomes invariant.
 *   max_iter : steps allowed (each one product);  m_max : 2 .. 63
 *   x_inout  : device, dim doubles: the start vector (any norm); on return the unit
 *              Ritz vector
 *   eval     : host, 1 double; info: host, may be NULL (resid_max is the explicit
 *              residual ||H x - theta x|| of the returned vector).
 * Returns DMRG_ERR_NOT_CONVERGED (results still written) when tol was not met. */
int dmrg_lanczos(dmrg_heff_t h, double tol, int32_t max_iter, int32_t m_max, double* x_inout, double* eval,
                 dmrg_davidson_info* info);

/* Size of the fixed device array used by dmrg_heff_apply_noalloc (32 MiB per GPU). */
#define DMRG_NOALLOC_SCRATCH_BYTES (32 * 1024 * 1024)

/* y = H_eff x for one vector, allocating no GPU memory.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory themselves,
 * e.g. code whose GPU memory is owned and budgeted by a host framework's allocator, or
 * a plugin that only receives device buffers from its host application.
 *   left .. b_off, n_terms : host arrays, exactly as for dmrg_heff_create
 *   op_data (op_len doubles), x, y (dim doubles each): device pointers owned by the
 *   caller, in the layouts of this header; y is fully overwritten and must not overlap
 *   x (DMRG_ERR_INVALID_ARG otherwise).
 * Everything else lives in one file-scope device array of DMRG_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library keeps until the process exits: the term tables (staged
 * from the host arrays, which the call has finished reading when it returns) and one
 * intermediate block of max(dim L) x max(dim R) doubles per CTA.  Problems with more than
 * 512 sectors per block, or whose tables plus one such block exceed the array, are
 * rejected with DMRG_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Each call waits for earlier work on `stream` and for its staged tables to
 * land (a stream synchronisation), then queues the kernel and returns; on a stream that
 * is capturing it returns DMRG_ERR_UNSUPPORTED without touching the stream.  All calls
 * share the array: calls from several host threads are serialised per device from the
 * staging of the tables to the kernel launch, but calls whose kernels overlap on the GPU
 * (e.g. on two streams without ordering) race and give wrong results.  Arithmetic: FP64,
 * terms summed in order per output block. */
int dmrg_heff_apply_noalloc(const int32_t* left, int32_t nl, const int32_t* right, int32_t nr,
                            int32_t target_n, int32_t target_2sz,
                            const double* coef, const int32_t* delta, const int32_t* parity,
                            const int64_t* a_off, const int64_t* b_off, int64_t n_terms,
                            const double* op_data, int64_t op_len,
                            const double* x, double* y, void* stream);

/*
 * Schedule of the grouped GEMMs (batching step of the method; the paper's own
 * scheduler assigns tasks to CPU and GPUs and has no counterpart of these fields).
 * It fixes only how the planned GEMMs are cut into work items and launched: every
 * schedule computes the same H_eff*psi (the split path bit for bit, the FP64 path up
 * to the order of its split-K sums).  Stage-2 GEMMs fall into three shape classes by
 * contraction length K: [0] K <= 2048, [1] K <= 16384, [2] longer.
 *   fp64_kchunk[c]    K per FP64 stage-2 work item of class c: 0 (whole K, no split)
 *                     or a positive multiple of 16.  Default 512, 512, 2048.
 *   fp64_ctas_per_sm  resident CTAs of the FP64 tile kernel per SM, 0..64; 0 (default)
 *                     and values above the occupancy limit mean that limit.
 *   split_kchunk[c]   K tiles (of 32) per split stage-2 work item of class c: 0
 *                     (default: adaptive, the longest that leaves >= 4 items per SM)
 *                     or a multiple of 8 up to 256.
 *   per_gemm          0 (default): each stage is one persistent launch over all its
 *                     GEMMs; 1: one launch per grouped GEMM (for comparison).
 *   fp64_tile         output tile of the FP64 tile kernel: 0 (default) 32 x 32 (4
 *                     warps), 1 64 x 32, 2 32 x 64 (8 warps); each element's sum runs
 *                     in the same order whatever the tile.  The split path's slice GEMM
 *                     tile is fixed at 128 x 96 (five accumulators of 96 columns fill
 *                     480 of the 512 tensor-memory columns).
 */
typedef struct {
    int32_t fp64_kchunk[3];
    int32_t fp64_ctas_per_sm;
    int32_t split_kchunk[3];
    int32_t per_gemm;
    int32_t fp64_tile;
} dmrg_schedule;

/* Current schedule of the handle. */
int dmrg_heff_schedule_get(dmrg_heff_t h, dmrg_schedule* s);

/* Replace the schedule: rebuilds and uploads the work lists (plan-only handles:
 * builds and checks them on the host), synchronises the device first and drops the
 * captured graphs.  DMRG_ERR_INVALID_ARG for a field out of range, leaving the
 * schedule unchanged. */
int dmrg_heff_schedule_set(dmrg_heff_t h, const dmrg_schedule* s);

/* Outcome of dmrg_heff_autotune: applies timed, median ms per apply of the schedule
 * the handle had on entry and of the one chosen, and the output tile (rows x columns)
 * of the GEMM kernel under the chosen schedule. */
typedef struct {
    int32_t trials, nvec;
    double default_ms, best_ms;
    dmrg_schedule best;
    int32_t tile_m, tile_n;
} dmrg_tune_report;

/*
 * Autotuner: times candidate schedules on this handle's plan with nvec vectors
 * (deterministic internal test vectors; `reps` timed applies per candidate, 1..100,
 * median) by coordinate descent over the stage-2 K extent of every shape class that
 * has GEMMs (and, FP64, the output tile and the CTAs per SM), and leaves the fastest
 * schedule in place.
 * Allocates two nvec x dim device vectors for the duration and synchronises the
 * device.  Not for plan-only handles.
 */
int dmrg_heff_autotune(dmrg_heff_t h, int32_t nvec, int32_t reps, dmrg_tune_report* report);

/* Number of grouped GEMMs of the plan for nvec vectors: counts[0] in stage 1 (one per
 * term group), counts[1] in stage 2 (per output block and contraction order); with
 * per_gemm set, an apply launches counts[0] + counts[1] GEMM kernels. */
int dmrg_heff_gemm_count(dmrg_heff_t h, int32_t nvec, int64_t counts[2]);

/*
 * Operator renormalisation (paper: the renormalisation of the block operators in the
 * new, truncated basis that follows each local update, Numerical procedure):
 *     O'[p <- q] = U_p^T O[p <- q] U_q   for every listed block,
 * with per-sector bases U_q (d_q x d'_q, normally orthonormal columns).  No handle.
 *   nsec, dims, dims_new : sector count, old dims d_q, new dims d'_q (1 <= d'_q <= d_q)
 *   U        : device, the bases row-major one after another in sector order
 *              (sum_q d_q d'_q doubles)
 *   blocks   : host, n_blocks rows (q, p, offset): input sector, output sector and the
 *              offset of the row-major d_p x d_q block in op
 *   op       : device, op_len doubles;  out: device, out_len doubles >= sum d'_p d'_q
 *   out_off  : host, n_blocks offsets of the d'_p x d'_q results in out (block order)
 * Runs on `stream` and returns when the results are written; it allocates and frees
 * its scratch (dmrg_renorm_create / _run below keep it across calls).
 * DMRG_ERR_INVALID_ARG for out-of-range sectors, dims or offsets, checked on the host
 * before any device work. */
int dmrg_renormalise(int32_t nsec, const int32_t* dims, const int32_t* dims_new, const double* U,
                     const int64_t* blocks, int64_t n_blocks, const double* op, int64_t op_len, double* out,
                     int64_t out_len, int64_t* out_off, void* stream);

/* The same renormalisation split into set-up and run, for a block list that is
 * renormalised repeatedly (every sweep step with the same sector structure):
 * dmrg_renorm_create validates the arguments like dmrg_renormalise (same meaning; op_len
 * and out_len are the sizes the runs will pass), fills out_off, builds the GEMM lists and
 * allocates and uploads every device buffer the runs need, on the current device.
 * dmrg_renorm_run copies the bases, then launches the two GEMM stages on `stream` and
 * returns without synchronising; it allocates nothing.  A plan's scratch is shared by its
 * runs: runs of one plan that overlap on the GPU (several streams) race.  U, op, out:
 * device, as above.  dmrg_renorm_destroy frees the plan (after its runs have finished). */
typedef struct dmrg_renorm* dmrg_renorm_t;
int dmrg_renorm_create(int32_t nsec, const int32_t* dims, const int32_t* dims_new, const int64_t* blocks,
                       int64_t n_blocks, int64_t op_len, int64_t out_len, int64_t* out_off, dmrg_renorm_t* plan);
int dmrg_renorm_run(dmrg_renorm_t plan, const double* U, const double* op, double* out, void* stream);
void dmrg_renorm_destroy(dmrg_renorm_t plan);

/* Layout of the wave function: n_blocks rows (left sector, right sector, rows, cols,
 * offset) in storage order; with buf NULL only *n_blocks is set, otherwise buf holds
 * *n_blocks * 5 values. */
int dmrg_heff_psi_blocks(dmrg_heff_t h, int64_t* buf, int64_t* n_blocks);

/*
 * Two-site decomposition and truncation (paper: the matrix factorisation of the two-site
 * wave function after each local update, Numerical procedure).  One matrix per left
 * sector present in psi: its wave-function blocks side by side in block order (rows = dim
 * of the left sector, cols = the sum of their right dims).  A U(1) handle has one block per
 * left sector; a spin-adapted one has one per right spin coupling to the target, and the
 * squared singular values are then the multiplet weights of the left block's density
 * matrix summed over the magnetic sublevels.  Per matrix the singular values and left
 * singular vectors (one-sided Jacobi in FP64 on the device: one CTA per matrix up to
 * 64 KB, an 8-CTA cluster per larger matrix; up to 8192 columns), then the D largest singular values over all matrices are kept (values below
 * 1e-13 of the largest are zero and never kept; ties go to the earlier matrix, then
 * position).  Matrices are indexed in the order of their left sectors.
 *   psi       : device, dim doubles
 *   sv        : host, sum_m min(rows_m, cols_m) doubles: each matrix's singular values,
 *               descending, in matrix order
 *   kept      : host, one per matrix: kept values (a prefix of its sv)
 *   U, u_len  : device: the kept left vectors of matrix m, row-major rows_m x kept_m at
 *               u_off[m] (host, one per matrix); u_len must hold sum rows_m kept_m (U may
 *               be NULL when nothing is kept)
 *   discarded : host: the sum of the squares of the singular values not kept.
 * Synchronises the device; allocates and frees its scratch. */
int dmrg_svd_truncate(dmrg_heff_t h, const double* psi, int32_t D, double* sv, int32_t* kept, double* U, int64_t u_len,
                      int64_t* u_off, double* discarded);

/* Release the handle and its device memory (NULL is ignored). */
void dmrg_heff_destroy(dmrg_heff_t h);

/* Static message for a DMRG_* code. */
const char* dmrg_strerror(int code);

/* Detail of the last failure on the calling thread ("" if none). */
const char* dmrg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DMRG_HEFF_H */
