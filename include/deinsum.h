/*
 * deinsum.h -- C ABI of the GB300 (sm_103a) MTTKRP / TTMc library.
 *
 * The library computes, on one GPU, the local Einstein-summation contractions
 * of Deinsum's two multilinear kernel classes (arXiv 2206.08301):
 *
 *   MTTKRP, mode n (Sec. III-B; Table IV rows MTTKRP-O3-M*, MTTKRP-O5-M*):
 *     i_0..i_{N-1}, i_0 r, .., i_{n-1} r, i_{n+1} r, .., i_{N-1} r -> i_n r
 *     M[i_n, r] = sum_{i_m, m != n} X[i_0..i_{N-1}] prod_{m != n} U^m[i_m, r]
 *
 *   TTMc, keep mode n (Sec. III-B; Table IV row TTMc-O5-M0):
 *     i_0..i_{N-1}, i_m r_m (m != n) -> r_0 .. r_{n-1} i_n r_{n+1} .. r_{N-1}
 *     Y = X x_0 U^0 .. x_{n-1} U^{n-1} x_{n+1} U^{n+1} .. x_{N-1} U^{N-1}
 *
 * Conventions shared by every entry point
 *   - Tensors are dense and row-major (last index fastest), as in the NumPy
 *     listings of Sec. II-A; indices are 0-based (Sec. III).
 *   - A factor U^m is I_m x R (row-major) and is contracted on its first index,
 *     the einsum term "i_m r".
 *   - Every tensor pointer passed to an execute call is a DEVICE pointer owned
 *     by the caller; the library never frees it.  Pointers to float32 data must
 *     be 4-byte aligned, to float64 data 8-byte aligned; X is loaded by tiled
 *     tensor-memory copies when X and its rows are 16-byte aligned, otherwise
 *     (split-BF16) by four copies per tile, one per class of rows congruent
 *     mod 4, or by per-thread loads; every path gives the same bits.
 *   - Outputs are overwritten (beta = 0): Listing 1 accumulates into a zeroed
 *     output, which is the same value.
 *   - Calls return a status and never throw or abort.  Execute calls are
 *     asynchronous on the given stream; a failure detected on the device (a
 *     bounded wait that gave up) is recorded in a device word and reported by
 *     deinsum_last_device_status() after the stream has been synchronised.
 *   - A plan may be executed on one stream at a time; concurrent executions
 *     need separate plans.  Plans are not tied to a device until their first
 *     execute, which allocates the plan's workspace on the current device
 *     (so make that first call before any stream capture).
 *   - There is no CPU fallback: without a usable sm_103a device every execute
 *     returns DEINSUM_ERR_CUDA.
 */
#ifndef DEINSUM_H
#define DEINSUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DEINSUM_OK = 0,
    DEINSUM_ERR_PARSE = 1,        /* malformed einsum string */
    DEINSUM_ERR_UNSUPPORTED = 2,  /* well-formed but not an MTTKRP / TTMc pattern */
    DEINSUM_ERR_SHAPE = 3,        /* bad extent count or value */
    DEINSUM_ERR_DTYPE = 4,        /* dtype / precision combination not offered */
    DEINSUM_ERR_ALIGN = 5,        /* pointer not aligned to its element size */
    DEINSUM_ERR_OOM = 6,          /* device allocation failed */
    DEINSUM_ERR_CUDA = 7,         /* CUDA runtime error (no device, launch failure, ...) */
    DEINSUM_ERR_TIMEOUT = 8,      /* a device-side bounded wait gave up */
    DEINSUM_ERR_INVALID = 9       /* NULL plan / pointer, wrong operand count, ... */
} deinsum_status;

typedef enum {
    DEINSUM_F32 = 0,              /* IEEE binary32 tensors */
    DEINSUM_F64 = 1               /* IEEE binary64 tensors (plain precision only) */
} deinsum_dtype;

typedef enum {
    /* CUDA-core arithmetic in the tensor dtype (FP32 FMA or FP64 FMA). */
    DEINSUM_PREC_PLAIN = 0,
    /* F32 tensors only.  Each F32 operand x is split into x_hi = bf16_rn(x) and
       x_lo = bf16_rn(x - x_hi); the four products hi*hi, hi*lo, lo*hi, lo*lo are
       formed on the tcgen05 tensor cores with FP32 accumulation in tensor
       memory, which recovers FP32 accuracy (about 2^-16 relative per term). */
    DEINSUM_PREC_SPLIT_BF16 = 1
} deinsum_prec;

typedef enum {
    DEINSUM_KIND_MTTKRP = 0,
    DEINSUM_KIND_TTMC = 1
} deinsum_kind;

typedef struct deinsum_plan_s *deinsum_plan_t;

/* A cudaStream_t passed as an opaque pointer; NULL is the legacy default stream. */
typedef void *deinsum_stream_t;

/* Plan summary (host data, filled by deinsum_plan_info). */
typedef struct {
    int kind;                 /* deinsum_kind */
    int order;                /* N, the order of X (2..8) */
    int mode;                 /* MTTKRP output mode n / TTMc kept mode n */
    int dtype;                /* deinsum_dtype */
    int prec;                 /* deinsum_prec */
    int64_t dims[8];          /* I_0..I_{N-1} */
    int64_t ranks[8];         /* R (MTTKRP: same in every mode) or R_m (TTMc); ranks[n] = I_n */
    int64_t out_elems;        /* elements of the output */
    double alg_bytes;         /* |X| + factor bytes + output bytes (compulsory traffic) */
    double alg_flops;         /* 2 x multiply-adds of the FLOP-minimal binary chain */
    int64_t n_units;          /* work units of the main kernel (0 before the first execute) */
    int64_t mm_cols;          /* MTTKRP followed by a matrix product: L (columns of C); else 0 */
    /* MTTKRP: the row view the kernels run (zero for TTMc) */
    int view_merged;          /* the inner mode is merged with its neighbour (split-BF16) */
    int view_packed;          /* tiles hold several outer indices (rows of at most 64) */
    int64_t view_groups;      /* leading indices (or packed outer indices) per 128-row tile */
    int view_aligned_rows;    /* rows are 16-byte aligned when X is: one tensor map */
    int view_row_classes;     /* otherwise the four row-class maps serve them (split-BF16 F32) */
    /* MTTKRP: the I/O lower bound of Sec. IV-E (deinsum_mttkrp_io_bound) for the row view
       (P, I_n, Q), an order-3 MTTKRP, with S = one SM's shared plus tensor memory in FP32
       words; zero for TTMc */
    double io_fast_mem_words; /* S */
    double io_rho;            /* S^(2/3) / 3 */
    double io_bound_bytes;    /* 4 x |X| R / min(rho, R): the least HBM traffic of the X stream */
} deinsum_plan_info_t;

/*
 * deinsum_plan -- parse and classify an einsum, fix the kernel and its schedule.
 *
 *   einsum     NUL-terminated "in,in,..->out" string with explicit output, e.g.
 *              "ijk,ja,ka->ia" (MTTKRP-O3-M0) or "ijkl,jb,kc,ld->ibcd" (TTMc).
 *              The first operand is X (N distinct letters); every other operand
 *              is a factor "<X letter><rank letter>".  MTTKRP: N-1 factors sharing
 *              one rank letter, output "<kept letter><rank letter>".  TTMc: N-1
 *              factors with distinct rank letters, output = X's letters with each
 *              contracted letter replaced by its rank letter in place.
 *              MTTKRP (order >= 3) followed by a matrix product (the running
 *              example of Sec. II-A, "ijk,ja,ka,al->il"): the MTTKRP operands, then one
 *              more operand "<rank letter><new letter>" (C, R x L), output
 *              "<kept letter><new letter>"; the product with C is applied in the
 *              final reduction, so the I_n x R MTTKRP result never reaches HBM.
 *              Anything else returns DEINSUM_ERR_UNSUPPORTED (paper Sec. III-A
 *              semantics: repeated letters are summed, output letters kept).
 *              TTMc with SPLIT_BF16 is the fused kernel of the last two modes,
 *              then the chain over the others: it needs the kept mode below N-2
 *              and R_{N-2}, R_{N-1} <= 32 (else DEINSUM_ERR_UNSUPPORTED).  Rows
 *              of I_{N-1} words that are not 16-byte aligned (I_{N-1} not a
 *              multiple of 4, or X offset from a 16-byte boundary) take the
 *              row-class maps; those need at least 4 rows in all
 *              (I_0 ... I_{N-2}) and extents within 32-bit coordinates (else
 *              DEINSUM_ERR_UNSUPPORTED at plan time for I_{N-1} mod 4 != 0,
 *              DEINSUM_ERR_ALIGN at execute time for an offset X).
 *   extents    one positive extent per distinct letter, in order of first
 *              appearance in `einsum` (host array of n_extents values).
 *   dtype      tensor element type.
 *   prec       arithmetic (see deinsum_prec); SPLIT_BF16 needs F32 and R <= 64.
 *   out        receives the plan (host object; free with deinsum_destroy).
 * Host only: makes no CUDA call.
 */
deinsum_status deinsum_plan(const char *einsum, const int64_t *extents, int n_extents,
                            deinsum_dtype dtype, deinsum_prec prec, deinsum_plan_t *out);

/*
 * deinsum_execute -- run the planned contraction on `stream` (asynchronous).
 *
 *   inputs     n_inputs DEVICE pointers, one per einsum operand in string order
 *              (inputs[0] = X, then the factors), each dense row-major in the
 *              plan's dtype.
 *   output     DEVICE pointer to the dense row-major output (overwritten):
 *              MTTKRP I_n x R; TTMc with the extents of the output letters.
 * The first call on a device allocates the plan's workspace there (cudaMalloc);
 * later calls allocate nothing.  Returns DEINSUM_ERR_INVALID for NULL pointers
 * or a wrong operand count, DEINSUM_ERR_ALIGN for a pointer not aligned to its
 * element size, DEINSUM_ERR_CUDA when a launch fails.
 */
deinsum_status deinsum_execute(deinsum_plan_t plan, const void *const *inputs, int n_inputs,
                               void *output, deinsum_stream_t stream);

/* Bytes of device workspace the plan owns once executed (partial sums, split
 * factor tiles, schedule table, status word).  Host only. */
deinsum_status deinsum_workspace_size(deinsum_plan_t plan, size_t *bytes);

/* Caller-provided workspace (for runtimes that manage device memory
 * themselves, e.g. the serving loop below).  deinsum_plan_workspace_bytes
 * fixes the plan's device (the current one) and schedule and returns the
 * bytes its workspace needs; deinsum_plan_bind_workspace hands it a DEVICE
 * buffer of at least that size (1024-byte aligned; DEINSUM_ERR_ALIGN
 * otherwise, DEINSUM_ERR_SHAPE if too small), uploading the schedule on
 * `stream`.  A bound workspace stays owned by the caller (deinsum_destroy does
 * not free it) and must outlive the plan's executions.  Binding is refused
 * (DEINSUM_ERR_INVALID) once the plan has a workspace. */
deinsum_status deinsum_plan_workspace_bytes(deinsum_plan_t plan, size_t *bytes);
deinsum_status deinsum_plan_bind_workspace(deinsum_plan_t plan, void *workspace, size_t bytes,
                                           deinsum_stream_t stream);

/* Fill *info with the plan summary.  Host only. */
deinsum_status deinsum_plan_info(deinsum_plan_t plan, deinsum_plan_info_t *info);

/*
 * deinsum_mttkrp_io_bound -- the tight MTTKRP I/O lower bound and its tiling (Sec. IV-E).
 *
 * For u[i, l] = sum_{j,k} T[i, j, k] v[j, l] w[k, l] and a fast memory of S elements,
 * a set of X multiply-adds that touches I, J, K, L distinct values of i, j, k, l needs
 * I J K + J L + K L + I L <= X elements of T, v, w and u in fast memory.  The tiles that
 * maximise I J K L under that constraint are I = J = K = (2X/5)^(1/3) and
 * L = X^(2/3) / (2^(1/3) 5^(2/3)); the computation size that maximises the I/O cost (the
 * least intensity I J K L / (X - S)) is X0 = 5S/2, which gives
 *     I = J = K = S^(1/3),  L = S^(2/3) / 2,  rho = S^(2/3) / 3,
 * and any schedule moves at least Q >= |V| / rho elements, |V| = N_i N_j N_k N_l.  The paper
 * prints the constraint without the output term I L; its tiles and X0 satisfy the constraint
 * with that term (and use only 4/5 of X without it), which is the reading taken here.
 * When the rank R (the extent of l) is below L, the rank is not tiled and one element of T
 * takes part in at most R multiply-adds: the intensity is min(rho, R) and the bound
 * |V| / min(rho, R), i.e. for R <= rho reading T once.  Any order-N MTTKRP is this form on
 * its row view (j over the modes before n, i = i_n, k over the modes after n).
 *   S        fast-memory elements (> 0).
 *   t_elems  elements of T (|V| = t_elems x R).
 *   R        the rank (>= 1).
 * Host only.  DEINSUM_ERR_INVALID for a NULL `out` or non-positive arguments.
 */
typedef struct {
    double X0;          /* 5S/2 */
    double I, J, K, L;  /* S^(1/3), S^(1/3), S^(1/3), S^(2/3)/2 */
    double rho;         /* S^(2/3)/3 */
    double rho_rank;    /* min(rho, R) */
    double q_min;       /* t_elems x R / rho_rank elements */
} deinsum_io_bound_t;
deinsum_status deinsum_mttkrp_io_bound(double S, double t_elems, int64_t R, deinsum_io_bound_t *out);

/* Device-side status of the plan's executes since the workspace was attached or
 * since the previous call: DEINSUM_OK, or DEINSUM_ERR_TIMEOUT when a bounded
 * wait inside a kernel gave up (that execute's output is then incomplete; the
 * kernel stopped every role, let its own copies and MMAs finish and returned).
 * Reads one word from the device and, if it was set, clears it (synchronous);
 * call after synchronising the stream. */
deinsum_status deinsum_last_device_status(deinsum_plan_t plan);

/* Limit, in nanoseconds, of every bounded wait inside the tensor-core kernels
 * launched from now on (process-wide; 0 restores the default of 2 s).  The
 * waits exist so that a stalled pipeline ends with DEINSUM_ERR_TIMEOUT instead of
 * hanging the device; a very short limit makes a normal execute give up, which
 * is how the failure path is tested.  Batched executes take the limit in force
 * when their graph is captured.  Host only. */
void deinsum_set_wait_limit_ns(uint64_t ns);

/* Number of device (cudaMalloc) and pinned host (cudaMallocHost) allocations
 * the library has made in this process (all entry points, all devices). */
int64_t deinsum_alloc_count(void);

/* Free the plan and its workspace.  NULL is ignored.  The device must not be
 * running an execute of this plan. */
void deinsum_destroy(deinsum_plan_t plan);

/* Static, human-readable name of a status code. */
const char *deinsum_status_string(deinsum_status status);

/* Number of kernels the library has launched in this process (all entry
 * points, all devices) -- a counter for benchmarks and tests. */
int64_t deinsum_kernel_launch_count(void);

/*
 * Benchmark support.  With timing enabled, every execute of the plan records a
 * pair of CUDA events on its stream around the plan's main kernel (the MTTKRP
 * contraction kernel; for TTMc the first, largest TTM).  deinsum_kernel_time
 * waits for the recorded events, returns the summed device time (ms) and the
 * number of recorded launches, and clears the record.  Events are created on
 * first use and kept by the plan.  Disabled by default.
 */
deinsum_status deinsum_set_kernel_timing(deinsum_plan_t plan, int enable);
deinsum_status deinsum_kernel_time(deinsum_plan_t plan, double *total_ms, int64_t *launches);

/*
 * Batched MTTKRP: `n` instances (each an MTTKRP einsum with its own extents
 * and rank <= 64, float32) computed together.  With DEINSUM_PREC_SPLIT_BF16
 * they run in one persistent tensor-core launch (plus factor-split, weight-table
 * and reduction launches) replayed from a CUDA graph captured on the first
 * execute with a given set of pointers.  Every instance's rows are cut into work
 * units of about total / (SMs x unit_div) bytes of X; the units form one list,
 * grouped by how an instance loads X (tensor map when its rows are 16-byte
 * aligned, row-class tensor maps otherwise; K-major or MN-major operand) and
 * largest first within a group, which the CTAs take in order from a device
 * ticket counter.  With DEINSUM_PREC_PLAIN every instance runs as its own plain
 * launch.  Results are deterministic (each unit writes its own partial block and
 * the reduction order is fixed) and within the split-BF16 tolerance of the
 * single-instance split path (which may regroup a short inner mode).
 */
typedef struct deinsum_batch_s *deinsum_batch_t;

/* Host only.  einsums[i], extents[i] (n_extents[i] values) as for deinsum_plan.
 * The unit granularity comes from the autotune cache when the batch signature
 * (count, size, rank mix) is known, else unit_div = 4. */
deinsum_status deinsum_plan_batched(int n, const char *const *einsums, const int64_t *const *extents,
                                    const int *n_extents, deinsum_dtype dtype, deinsum_prec prec,
                                    deinsum_batch_t *out);

/* inputs[i]: HOST array of DEVICE pointers of instance i's operands (string
 * order); outputs[i]: DEVICE pointer of its output.  Asynchronous on `stream`;
 * the first call with a new set of pointers uploads the instance tables,
 * launches once and captures the graph (so it must not run under an outer
 * stream capture); later calls with the same pointers replay the graph. */
deinsum_status deinsum_execute_batched(deinsum_batch_t b, const void *const *const *inputs, void *const *outputs,
                                       deinsum_stream_t stream);

/* Time the split-BF16 batch on the device and keep the fastest schedule: first the unit
 * size of the whole batch (units of about total / (SMs x unit_div) bytes of X, unit_div in
 * {1, 2, 4, 8, 16, 32, 64}), then, for each kind of instance present (tensor-map or
 * row-class loads, K-major or MN-major operand), twice or half as many units for that kind
 * while that is faster.  If DEINSUM_AUTOTUNE_CACHE names a file the result is appended there
 * for later batches with the same signature.  Synchronous. */
deinsum_status deinsum_batched_autotune(deinsum_batch_t b, const void *const *const *inputs,
                                        void *const *outputs, deinsum_stream_t stream, double *best_ms);

/* Units, grid (CTAs of the persistent launch), unit divisor and algorithmic
 * bytes (sum over the instances). */
deinsum_status deinsum_batched_info(deinsum_batch_t b, int64_t *n_units, int *grid, int *unit_div,
                                    double *alg_bytes);

/* After synchronising: DEINSUM_OK or DEINSUM_ERR_TIMEOUT (a bounded wait gave up
 * in an execute since the previous call; the call clears the word). */
deinsum_status deinsum_batched_status(deinsum_batch_t b);

void deinsum_batched_destroy(deinsum_batch_t b);

/*
 * CP-ALS on the device.  The paper names CP decomposition as the computation
 * MTTKRP serves (Sec. I); the ALS steps follow Kolda & Bader (SIAM Review
 * 2009, Sec. 3.4).  Per sweep, for n = 0..N-1 (Gauss-Seidel): M = MTTKRP_n
 * (this library, `prec`), V = Hadamard of the Grams U_m^T U_m (m != n), U_n
 * solves U_n V = M by Cholesky, columns normalised to unit 2-norm (norms into
 * lambda; a zero column keeps lambda = 0), G_n = U_n^T U_n; after the sweep
 * fit = 1 - ||X - [[lambda; U]]|| / ||X|| from ||X||^2 + ||Xhat||^2 - 2<X, Xhat>.
 * Grams, Hadamard products, Cholesky, solves, norms and the fit are FP64.
 *
 * Dimension tree (order 3, SPLIT_BF16, rank <= 32, I_2 a multiple of 4, X
 * 16-byte aligned; on by default): modes 0 and 1 of a sweep share
 * T = X x_2 U_2 (I_0 x I_1 x rank, computed once on the tensor cores), so X is
 * read twice per sweep instead of three times; the handle's workspace grows by T.
 */
typedef struct deinsum_cpals_s *deinsum_cpals_t;

/* Host only: plans the N MTTKRPs of an order-`order` tensor with extents
 * dims[0..order-1] (host array) and rank `rank` (1..64). */
deinsum_status deinsum_cpals_create(int order, const int64_t *dims, int rank, deinsum_prec prec,
                                    deinsum_cpals_t *out);

/* Run `sweeps` ALS sweeps on `stream` (asynchronous).
 *   X        DEVICE float32 tensor (read only).
 *   factors  HOST array of `order` DEVICE float32 I_m x rank matrices: the
 *            initial factors on entry, the (column-normalised) result on exit.
 *   lambda   DEVICE float64[rank]: the column norms after the last update.
 *   fits     DEVICE float64[sweeps]: the fit after every sweep, from the expansion
 *            above; its FP32-level MTTKRP input makes it cancel once the residual is
 *            small (~1e-3 absolute as the fit approaches 1).  So when the last sweep's
 *            residual^2 is below 1e-2 ||X||^2, the last fit is computed from the
 *            residual ||X - Xhat|| directly instead (FP32 reconstruction, FP64 sum:
 *            ~1e-7); above that the expansion is within ~5e-5 and is kept.
 * The first call allocates the handle's workspace (one cudaMalloc). */
deinsum_status deinsum_cpals_run(deinsum_cpals_t h, const float *X, float *const *factors, double *lambda,
                                 int sweeps, double *fits, deinsum_stream_t stream);

/* Caller-provided workspace for the handle and its plans (same rules as
 * deinsum_plan_bind_workspace); without it the first run allocates one. */
deinsum_status deinsum_cpals_workspace_bytes(deinsum_cpals_t h, size_t *bytes);
deinsum_status deinsum_cpals_bind_workspace(deinsum_cpals_t h, void *workspace, size_t bytes,
                                            deinsum_stream_t stream);

/* Enable (default) or disable the dimension tree for later runs; and whether runs
 * use it (1 when the shape allows it and it is enabled). */
deinsum_status deinsum_cpals_set_dimension_tree(deinsum_cpals_t h, int enable);
int deinsum_cpals_uses_dimension_tree(deinsum_cpals_t h);

/* After synchronising the stream: DEINSUM_OK, DEINSUM_ERR_TIMEOUT if a bounded
 * wait of an MTTKRP or of the dimension-tree kernel gave up, DEINSUM_ERR_INVALID
 * if a Gram-Hadamard matrix was not positive definite to FP64 precision (its
 * pivot was floored).  Covers the handle's latest run. */
deinsum_status deinsum_cpals_status(deinsum_cpals_t h);

/* Free the handle, its plans and its workspace.  NULL is ignored. */
void deinsum_cpals_destroy(deinsum_cpals_t h);

/*
 * Serving: CP-ALS requests with continuous batching under an HBM budget.
 * The server owns one device arena of `hbm_budget_bytes` (one cudaMalloc at
 * creation) and `slots` CUDA streams.  A request waits in a FIFO until a slot
 * is free and the arena can place its footprint (X, factors, generating
 * factors, lambda, fits, CP-ALS workspace); on admission its X is generated on
 * the device from its seed (deinsum_gen_cp_f32), its sweeps are enqueued on the
 * slot's stream and an event marks the end.  Requests admitted while others
 * run overlap with them on the device.  deinsum_server_poll retires finished
 * requests and admits waiting ones; it never waits for running work.  Results
 * depend only on the request (deterministic kernels), not on what else ran.
 * The server is not thread-safe; use it from one host thread.
 */
typedef struct deinsum_server_s *deinsum_server_t;

typedef struct {
    int order;                          /* 2..8 */
    int64_t dims[8];                    /* extents of X */
    int rank;                           /* CP-ALS rank, 1..64 */
    int sweeps;                         /* ALS sweeps, 1..4096 */
    uint64_t seed;                      /* seed of the noise of X */
    int cp_rank;                        /* rank of the generating CP tensor */
    double noise;                       /* sigma of the additive noise */
    const float *const *cp_factors;     /* HOST: `order` float32 I_m x cp_rank generating factors */
    const float *const *init_factors;   /* HOST: `order` float32 I_m x rank initial factors */
    double arrival_s;                   /* arrival time on deinsum_server_clock() */
    int want_factors;                   /* keep the final factors for deinsum_server_take */
} deinsum_request_t;

typedef struct {
    int64_t id;
    int status;                         /* deinsum_status of the request */
    double arrival_s, admit_s, done_s;  /* deinsum_server_clock() times */
    double gen_ms;                      /* device time of generating X */
    int sweeps;
    double fit;                         /* fit after the last sweep */
} deinsum_result_t;

/* Steady clock (seconds) the server stamps admission and completion with. */
double deinsum_server_clock(void);

deinsum_status deinsum_server_create(size_t hbm_budget_bytes, int slots, deinsum_prec prec,
                                     deinsum_server_t *out);

/* Queue a request (host data is copied); *id identifies it.  Shape errors are
 * refused here; a request larger than the whole budget finishes with
 * DEINSUM_ERR_OOM when it reaches the head of the queue. */
deinsum_status deinsum_server_submit(deinsum_server_t s, const deinsum_request_t *req, int64_t *id);

/* Retire finished requests and admit waiting ones; reports the number of
 * running and waiting requests. */
deinsum_status deinsum_server_poll(deinsum_server_t s, int *n_active, int *n_waiting);

/* Copy a finished request's result (and, if non-NULL, its fits[sweeps],
 * lambda[rank] and -- if it asked for them -- the factors concatenated by mode)
 * into host buffers and forget it.  DEINSUM_ERR_INVALID if it is unknown or
 * not finished yet. */
deinsum_status deinsum_server_take(deinsum_server_t s, int64_t id, deinsum_result_t *res, double *fits,
                                   double *lambda, float *factors);

/* Wait for running work, free the arena, streams and every request. */
void deinsum_server_destroy(deinsum_server_t s);

/*
 * deinsum_mttkrp_noalloc -- split-BF16 MTTKRP that allocates no device memory.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc: code whose device memory is owned by another
 * allocator (a framework's caching allocator that has reserved the HBM
 * budget), or latency-critical loops that cannot accept the implicit device
 * synchronisation of cudaMalloc / cudaFree.  It computes the same mode-`mode`
 * MTTKRP as deinsum_plan + deinsum_execute with DEINSUM_PREC_SPLIT_BF16 and
 * the same kernels, but keeps its scratch (schedule, per-unit partial sums,
 * split factor tiles, weight tables, status word) in one fixed device array of about 13 MiB
 * inside the library, which every GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *   order, dims  N (2..8) and the extents I_0..I_{N-1} of X (host array).
 *   mode         the output mode n.
 *   rank         R, 1..64.
 *   X            DEVICE pointer, dense row-major float32 tensor.
 *   factors      HOST array of `order` DEVICE pointers; factors[m] is the
 *                I_m x R row-major float32 factor (factors[mode] is ignored).
 *   out          DEVICE pointer to the I_n x R row-major float32 output (overwritten).
 * Limits of the fixed scratch: I_n <= 32768 (at most 256 blocks of 128 output
 * rows); the mode contracted on the tensor cores (I_{N-1}, or I_{N-2} when
 * n = N-1) at most 16384 for R <= 16, 8192 for R <= 32, 4096 for R <= 64;
 * the weight tables, (P' + O') x R_pad floats, at most 2^20 floats, where
 * P' = I_0 ... I_{n-1} when 0 < n < N-1 (else 0), O' = I_{n+1} ... I_{N-2}
 * when n < N-2, I_0 ... I_{N-3} when n = N-1 and N > 2 (else 0), and R_pad is
 * R rounded up to 16, 32 or 64.
 * Larger problems return DEINSUM_ERR_SHAPE without launching anything.
 * Returns DEINSUM_ERR_INVALID for NULL pointers or a bad order / mode,
 * DEINSUM_ERR_ALIGN for pointers not 4-byte aligned, DEINSUM_ERR_CUDA when a
 * launch fails.  The first call on a device looks up that device's address of
 * the scratch array (with the device current); make that first call before
 * any stream capture.  Every call shares the one array and leaves its
 * contents behind (each call clears what must start at zero), so calls that
 * overlap on the GPU -- on different streams, or from different threads --
 * race; serialise them.
 */
deinsum_status deinsum_mttkrp_noalloc(int order, const int64_t *dims, int mode, int rank,
                                      const float *X, const float *const *factors, float *out,
                                      deinsum_stream_t stream);

/* Device-side status of the latest deinsum_mttkrp_noalloc call on the current
 * device: DEINSUM_OK, or DEINSUM_ERR_TIMEOUT when a bounded wait inside its
 * kernel gave up (the output is then incomplete).  Copies the status word out
 * of the fixed array (synchronous, allocates nothing); call after synchronising
 * the stream of that call.  DEINSUM_ERR_CUDA if the copy fails. */
deinsum_status deinsum_mttkrp_noalloc_status(void);

/*
 * Seeded synthetic inputs on the device.  These implement, bit for bit, the
 * counter-based generator of the project's input module (SplitMix64 by
 * S. Vigna: state0 = mix64(seed + stream_id * 0x9E3779B97F4A7C15), element i is
 * mix64(state0 + (i + 1) * 0x9E3779B97F4A7C15)); they hold none of the
 * contraction arithmetic.  `out` is a DEVICE pointer to n elements.
 */

/* out[i] = (raw_i >> 40) * 2^-23 - 1, uniform on [-1, 1) in float32. */
deinsum_status deinsum_gen_uniform_f32(uint64_t seed, uint64_t stream_id, int64_t n,
                                       float *out, deinsum_stream_t stream);

/* out[i] = (raw_i >> 11) * 2^-52 - 1, uniform on [-1, 1) in float64. */
deinsum_status deinsum_gen_uniform_f64(uint64_t seed, uint64_t stream_id, int64_t n,
                                       double *out, deinsum_stream_t stream);

/*
 * Rank-`rank` CP tensor plus noise, float32, row-major with extents dims[0..order-1]:
 *   out[idx] = sum_{s<rank} prod_{m<order} A_m[i_m, s] + f32(sigma) * f32(z(idx))
 * evaluated in float32 with every multiply and add rounded to nearest (product
 * over m left to right, sum over s left to right, no fused multiply-add);
 * z(idx) = (sum of the four 16-bit lanes of raw(idx) - 2^17) * (sqrt(3) * 2^-16),
 * in float64, on stream 2 under `seed`.  `factors` is a HOST array of `order`
 * DEVICE pointers to float32 I_m x rank matrices.  order <= 8.
 */
deinsum_status deinsum_gen_cp_f32(uint64_t seed, int order, const int64_t *dims, int rank,
                                  const float *const *factors, double sigma, float *out,
                                  deinsum_stream_t stream);

/*
 * Block distribution and redistribution (paper Sec. II-C/D, Sec. V), host only.
 *
 * An iteration space of extents N_0..N_{D-1} is distributed over a Cartesian grid
 * of P_0 x .. x P_{D-1} processes, one block per process (Eqs. (12)-(13)): along
 * dimension j the block size is B_j = ceil(N_j / P_j) and process coordinate p_j
 * holds indices [p_j B_j, min((p_j + 1) B_j, N_j)).  Ranks number the grid
 * row-major (the last dimension fastest, as MPI_Cart_create without reordering).
 * A tensor on the grid uses some of its dimensions (`dims[t]` = the grid
 * dimension of tensor mode t); its blocks are replicated over the sub-grids of
 * the unused dimensions (the MPI_Cart_sub view of the paper's listing).
 */
typedef struct {
    int ndim;              /* D, 1..8 */
    int64_t extent[8];     /* N_j >= 1 */
    int procs[8];          /* P_j >= 1 */
} deinsum_grid_t;

/* B_j = ceil(N_j / P_j) (0 on bad arguments). */
int64_t deinsum_grid_block(const deinsum_grid_t *g, int j);
/* Coordinates of `rank` (HOST array of ndim ints) / rank of `coords` (-1 if out of range). */
deinsum_status deinsum_grid_coords(const deinsum_grid_t *g, int64_t rank, int *coords);
int64_t deinsum_grid_rank(const deinsum_grid_t *g, const int *coords);
/* The block of `rank`: [lo[j], hi[j]) per dimension (HOST arrays of ndim values). */
deinsum_status deinsum_grid_block_range(const deinsum_grid_t *g, int64_t rank, int64_t *lo, int64_t *hi);
/* MPI_Cart_sub semantics: the sub-grid keeping the dimensions with remain[j] != 0.
 * `color` numbers the sub-grid (row-major over the dropped coordinates), `key` is
 * the rank inside it (row-major over the kept coordinates). */
deinsum_status deinsum_grid_sub(const deinsum_grid_t *g, const int *remain, int64_t rank, int64_t *color,
                                int64_t *key);

/* One dimension of a redistribution from block size Bx to By (Eqs. (20)-(24)):
 * with p^(y) B^(y) = xi B^(x) + lambda, the offsets o^(y) of y-block py fall into
 * k = ceil((By + lambda) / Bx) runs; run m, o^(y) in [oy_lo, oy_hi), comes from
 * x-process px = xi + m at offsets [ox_lo, ox_hi). */
typedef struct {
    int64_t px;
    int64_t oy_lo, oy_hi;
    int64_t ox_lo, ox_hi;
} deinsum_dim_part_t;
/* Fills parts[0..k) and returns k (-1 on bad arguments or k > max_parts).  Blocks
 * are taken as full (B^(y) offsets); clip against the extent for a last block. */
int deinsum_redist_dim_partitions(int64_t Bx, int64_t By, int64_t py, deinsum_dim_part_t *parts, int max_parts);
/* Message matching (Eq. (25)): the y-process coordinates [*py_lo, *py_hi) whose
 * blocks meet x-block px (before clipping to the grid). */
void deinsum_redist_match(int64_t Bx, int64_t By, int64_t px, int64_t *py_lo, int64_t *py_hi);

/* One message of a redistribution: the peer rank and the box [lo, hi) of global
 * tensor coordinates (one entry per tensor mode). */
typedef struct {
    int64_t peer;
    int64_t lo[8], hi[8];
} deinsum_msg_t;
/* The messages `rank` sends (sending != 0, rank on gx) or receives (rank on gy)
 * when a tensor of `order` modes moves from its block distribution on gx
 * (modes on grid dimensions xdims) to the one on gy (ydims); extents must agree.
 * A block replicated on gx is sent once, by its replica with zero coordinates in
 * the unused dimensions; every replica on gy receives its part.  Between two
 * ranks there is at most one message (the intersection of two blocks is one box).
 * Writes up to max_msgs entries to msgs (may be NULL to count) and returns the
 * number of messages, or -1 on bad arguments or when max_msgs is too small. */
int deinsum_redist_plan(const deinsum_grid_t *gx, const int *xdims, const deinsum_grid_t *gy, const int *ydims,
                        int order, int64_t rank, int sending, deinsum_msg_t *msgs, int max_msgs);

#ifdef __cplusplus
}
#endif

#endif /* DEINSUM_H */
