/*
 * phisplit.h -- C ABI of the GB300 (sm_103a) direction-split phi-function library.
 *
 * The library computes the PHISPLIT approximation of Caliari & Cassini,
 * "Direction splitting of phi-functions in exponential integrators for
 * d-dimensional problems in Kronecker form" (arXiv 2304.02327):
 *
 *   phi_l(tau K) v  ~  vec( ((l!)^(d-1) V) x_1 phi_l(tau A_1) x_2 ... x_d phi_l(tau A_d) )
 *
 * for a Kronecker sum K = A_d (+) ... (+) A_1 (Section 1, eq. (1b); Section 3,
 * Theorem 1 / eq. (14) and the definition of P_l^(2) after it), and the
 * exponential integrators built on it (Section 3.2, eq. (17)-(20)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Layout.  An order-d tensor of sizes n_1 x ... x n_d is a contiguous device
 *   array of N = n_1 * ... * n_d doubles, index i_1 fastest (the column-stacking
 *   vec of Section 1).  Small matrices are n x n, column-major (entry (i, j) at
 *   i + n*j).  A_1 acts on i_1.
 * - Pointers.  Every array argument is a DEVICE pointer unless its comment says
 *   host.  The caller owns every buffer it passes; the plan owns the phi
 *   matrices it forms and frees them in phi_plan_destroy.
 * - Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  All calls are stream-ordered and return without synchronising,
 *   except phi_plan_create, phi_plan_status and the *_info queries, which say so.
 * - Errors.  Every call returns MM_OK (0) or a negative MM_ERR_* code and leaves
 *   its outputs unspecified on error.  Argument and shape errors are detected on
 *   the host before any launch.  Device-side conditions (a non-finite value
 *   written by an integrator step, a bounded wait that ran out) are OR-ed into a
 *   per-plan status word that phi_plan_status reads.
 * - Precision.  MM_FP64: every product and sum in double (the plain form).
 *   MM_TF32X3 / MM_BF16X3: the mu-mode products run on tcgen05 tensor cores with
 *   split operands accumulated in FP32 (TF32x3: operand in two TF32 parts, phi in
 *   three, 4 products; BF16x3: both in three BF16 parts, 6 products); the phi
 *   matrices are formed in FP64 and the state update u + tau*y is FP64, while
 *   K u + g and the Tucker intermediates are FP32.  The tensor cores' FP32
 *   accumulation truncates toward zero; the main product of every K-block
 *   therefore goes to a fresh accumulator that is summed in FP32 registers (round
 *   to nearest).  Accuracy, relative to the FP64 result: one mumode_phi_apply
 *   within 4e-6 of max|P| (the split operands carry 2^-22 (TF32x3) or ~2^-25
 *   (BF16x3) of each value, the intermediates FP32); an integration (expint_step)
 *   within 1e-6 in the infinity and Frobenius norms, since the error lands on the
 *   increment tau*y, not on u (measured: 5.6e-7 after the 100 ETD2RK steps of 3D
 *   advection-diffusion-reaction at n = 320).
 *   Dense (non-tridiagonal) A_mu: d = 2 only in the mixed forms, the band of A_mu
 *   as an FP32 stencil and the remainder on the tensor cores.
 */
#ifndef PHISPLIT_H
#define PHISPLIT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MM_API __attribute__((visibility("default")))
#else
#define MM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MM_OK               0
#define MM_ERR_ARG         -1   /* null pointer, bad enum, bad scalar          */
#define MM_ERR_SHAPE       -2   /* sizes out of range or inconsistent          */
#define MM_ERR_UNSUPPORTED -3   /* valid request this build does not implement */
#define MM_ERR_CUDA        -4   /* a CUDA runtime call failed                  */
#define MM_ERR_TIMEOUT     -5   /* a bounded device wait ran out               */
#define MM_ERR_NONFINITE   -6   /* a step produced inf/nan                     */
#define MM_ERR_NOMEM       -7   /* device allocation failed (plan creation)    */
#define MM_ERR_WORKSPACE   -8   /* workspace missing or too small              */

/* Device status-word bits (phi_plan_status). */
#define MM_STATUS_NONFINITE 1u
#define MM_STATUS_TIMEOUT   2u

/* ---- precision forms ------------------------------------------------- */
#define MM_FP64    0
#define MM_TF32X3  1
#define MM_BF16X3  2

/* ---- time-stepping schemes (Section 2 and Section 3.2) ----------------- */
#define MM_EXPEULER     0   /* eq. (11) / tensor form eq. (19)               */
#define MM_ETD2RK       1   /* eq. (12) / tensor form eq. (20)               */
#define MM_LAWSON_EULER 2   /* eq. (9)  / tensor form eq. (17)               */
#define MM_LAWSON2B     3   /* eq. (10) / tensor form eq. (18)               */
#define MM_EXPROSEULER  4   /* eq. (13) / tensor form eq. (21): Riccati G, FP64 */
#define MM_EXPEULER_ALT 5   /* exp. Euler, alternative form (Section 3.2), FP64 */

/* ---- nonlinearity g(t, u) (eq. (1a)) ----------------------------------- */
#define MM_G_NONE            0  /* g = 0                                         */
#define MM_G_CUBIC           1  /* g = c0 + c1 u + c2 u^2 + c3 u^3, pointwise    */
#define MM_G_RICCATI         2  /* G(U) = C + U B U, d = 2 (eq. (2)-(3))         */
#define MM_G_ADR_MANUFACTURED 3 /* g = 1/(1+u^2) + e^t a - 1/(1 + e^{2t} b^2),   */
                                /* the paper's ADR test (Section 4.2, eq. (25))  */

typedef struct mm_nonlin {
    int kind;              /* MM_G_*                                              */
    double c[4];           /* MM_G_CUBIC coefficients c0..c3                      */
    const double* B;       /* MM_G_RICCATI: n_2 x n_1, column-major (device)      */
    const double* C;       /* MM_G_RICCATI: n_1 x n_2, column-major (device)      */
    const double* psi_a;   /* MM_G_ADR_MANUFACTURED: N doubles, tensor layout     */
    const double* psi_b;   /* MM_G_ADR_MANUFACTURED: N doubles, tensor layout     */
} mm_nonlin;

/* Opaque, immutable after creation (apart from its status word and its cache of
 * captured CUDA graphs).  One plan may be used from one host thread at a time. */
typedef struct mm_plan_s* mm_plan;

/*
 * phi_plan_create -- form phi_l(tau A_mu), l = 0..ell_max, for every direction
 * (Section 3.1: scaling so that ||tau A / 2^s||_1 <= 1, a truncated Taylor
 * series of phi_ell_max at the scaled matrix, phi_{l-1}(X) = X phi_l(X) + I/(l-1)!,
 * then s applications of the squaring recurrence eq. (16)), all in FP64 on the
 * GPU.  Directions whose A_mu are bitwise equal share one set of phi matrices.
 * If every A_mu is tridiagonal, K u is evaluated later as a 3-point stencil;
 * otherwise as dense mu-mode products.
 *
 *   out     host pointer receiving the plan handle.
 *   d       number of directions, 1 <= d <= 8.
 *   n       host array of d sizes, 1 <= n_mu <= 8192, N = prod n_mu < 2^40.
 *   A       host array of d device pointers; A[mu] is n_mu x n_mu column-major.
 *           Read during the call only.
 *   tau     time step (finite).  tau = 0 is allowed (phi_l = I / l!).
 *   ell_max highest phi index needed, 0..3 (ETD2RK needs 2).
 *   prec    MM_FP64, MM_TF32X3 or MM_BF16X3 (the mixed forms also split the phi
 *           matrices into their operand parts, and the remainders A_mu - band for
 *           dense A_mu when d = 2).
 *   stream  ordering stream for the set-up kernels.
 * Synchronises `stream` (it reads norms and band widths back).  Allocates the
 * plan's device memory with cudaMalloc.  Errors: MM_ERR_ARG, MM_ERR_SHAPE,
 * MM_ERR_NOMEM, MM_ERR_CUDA; *out is NULL on error.
 */
MM_API int phi_plan_create(mm_plan* out, int d, const int64_t* n, const double* const* A,
                    double tau, int ell_max, int prec, void* stream);

/* Frees the plan and everything it owns (synchronises the device).  NULL is OK. */
MM_API int phi_plan_destroy(mm_plan p);

/*
 * phi_plan_info -- host query of a plan.  Any output pointer may be NULL.
 *   d (1), n (d entries), ell_max (1), prec (1), squarings (d entries: the s used
 *   for direction mu), tridiagonal (1: 1 if K u runs as a stencil).
 */
MM_API int phi_plan_info(mm_plan p, int* d, int64_t* n, int* ell_max, int* prec,
                  int* squarings, int* tridiagonal);

/*
 * phi_plan_get_phi -- copy phi_ell(tau A_mu) (mu = 1..d, FP64, n_mu x n_mu,
 * column-major) into the device buffer dst.  Stream-ordered.
 * Errors: MM_ERR_ARG (ell > ell_max, mu out of range, dst NULL), MM_ERR_CUDA.
 */
MM_API int phi_plan_get_phi(mm_plan p, int ell, int mu, double* dst, void* stream);

/*
 * phi_plan_status -- synchronises `stream`, returns the OR of MM_STATUS_* bits
 * raised on the device since the last reset (>= 0), or a negative MM_ERR_*.
 * reset != 0 clears the word afterwards.
 */
MM_API int phi_plan_status(mm_plan p, int reset, void* stream);

/* Workspace bytes mumode_phi_apply needs (N doubles when d >= 2, else 0). */
MM_API size_t mumode_workspace_bytes(mm_plan p);

/*
 * mumode_phi_apply -- P = alpha * (ell!)^(d-1) * V x_1 phi_ell(tau A_1) ... x_d
 * phi_ell(tau A_d), the tensor formulation P_l^(2) of Section 3 (Theorem 1);
 * for ell = 0 this is the exact e^{tau K} v of eq. (5)-(6).
 *
 *   V   N doubles (input, not modified).  P: N doubles (output).  V and P must
 *       not overlap.  ws: workspace of >= mumode_workspace_bytes(p) bytes,
 *       8-byte aligned (16 for the split-precision forms), overlapping neither V
 *       nor P.
 * Accuracy: FP64 form ~1e-15 of max|P|; TF32x3 / BF16x3 within 4e-6 of max|P|.
 * Errors: MM_ERR_ARG (ell > ell_max, null pointers, overlap), MM_ERR_WORKSPACE,
 * MM_ERR_CUDA (launch failure).
 */
MM_API int mumode_phi_apply(mm_plan p, int ell, const double* V, double* P, double alpha,
                     void* ws, size_t ws_bytes, void* stream);

/* Workspace bytes expint_step needs for `scheme` and nonlinearity `g`. */
MM_API size_t expint_workspace_bytes(mm_plan p, int scheme, const mm_nonlin* g);

/*
 * expint_step -- advance U in place by nsteps steps of size tau (the plan's)
 * with the PHISPLIT form of `scheme` (Section 3.2):
 *   MM_EXPEULER     U+ = U + tau P_1^(2)(K U + G(t, U))                   eq. (19)
 *   MM_ETD2RK       U2 = U + tau P_1^(2)(K U + G(t, U))
 *                   U+ = U2 + tau P_2^(2)(G(t + tau, U2) - G(t, U))       eq. (20)
 *   MM_LAWSON_EULER U+ = (U + tau G(t, U)) x_mu e^{tau A_mu}              eq. (17)
 *   MM_LAWSON2B     eq. (18)
 *   MM_EXPEULER_ALT U+ = U x_mu e^{tau A_mu} + tau P_1^(2)(G(U)): the alternative
 *                   form of Section 3.2, exact for linear autonomous problems (plan
 *                   form MM_FP64 only: a mixed form would keep the whole new state, not
 *                   an increment, at the split precision; pointwise g only)
 *   MM_EXPROSEULER  U+ = U + tau (K U + G(U)) x_1 phi_1(tau J_1) x_2 phi_1(tau J_2),
 *                   J_1 = A_1 + U B, J_2 = A_2 + (B U)^T: the Riccati term's
 *                   Jacobian at U (Section 4.1, eq. (21)), phi_1 formed on the GPU
 *                   every step in FP64 (plan form MM_FP64 only; the scaling is chosen
 *                   on the host, so each step synchronises `stream` and the steps are
 *                   launched directly, never replayed from a graph)
 * P_l^(2) carries the (l!)^(d-1) factor of Theorem 1 (so the phi_2 stage of
 * ETD2RK is scaled by 2^(d-1)), and tau multiplies both K U and G in the first
 * stage, as the vector forms eq. (11)-(12) require.
 *
 *   g       host pointer to the nonlinearity descriptor (device arrays inside).
 *           MM_G_RICCATI requires d = 2; MM_G_ADR_MANUFACTURED requires psi_a,
 *           psi_b of N doubles.
 *   U       N doubles, in/out.
 *   t0      time of the first step (used by time-dependent g only).
 *   nsteps  >= 0.
 *   ws      >= expint_workspace_bytes(p, scheme, g) bytes, 8-byte aligned, not
 *           overlapping U or g's arrays.
 * The ell_max of the plan must cover the scheme (ETD2RK: 2, exp. Euler: 1,
 * Lawson: 0).  A non-finite value in the updated state raises
 * MM_STATUS_NONFINITE in the plan's status word.
 * Graphs: unless turned off (phi_plan_set_graphs), the first call with a given
 * (scheme, g's contents, U, ws, nsteps[, t0 for a time-dependent g]) captures the
 * nsteps steps into a CUDA graph on a stream of the plan, and every call with the
 * same arguments replays it on `stream` (one launch of host work).  A graph holds
 * at most 32 steps: longer calls replay a 32-step graph (and one for the rest), or
 * launch directly when g depends on t.  The plan keeps the eight most recent
 * graphs.  Calls made while `stream` is being captured, or while event tracing is
 * on (mm_trace_enable(1)), launch the kernels directly.
 * Errors: MM_ERR_ARG, MM_ERR_UNSUPPORTED, MM_ERR_WORKSPACE, MM_ERR_CUDA.
 */
MM_API int expint_step(mm_plan p, int scheme, const mm_nonlin* g, double* U, double t0,
                int nsteps, void* ws, size_t ws_bytes, void* stream);

/* Turn the graph capture and replay of expint_step on (default) or off.  Host only. */
MM_API int phi_plan_set_graphs(mm_plan p, int on);

/* ---- allocation-free Tucker chain ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory when they need the split
 * action: code embedded in a host application that owns every byte of device
 * memory through its own pool and forbids side allocations, loops with latency
 * budgets that cannot afford cudaMalloc/cudaFree (both may synchronise the
 * device), and plug-ins whose process does not let them call the CUDA allocator.
 *
 * tucker_apply_noalloc computes, in FP64,
 *     P = alpha * V x_1 M_1 x_2 M_2 ... x_d M_d
 * (the same contraction chain as mumode_phi_apply; pass M_mu = phi_l(tau A_mu),
 * for instance from phi_plan_get_phi, and alpha = alpha' * (l!)^(d-1) to get
 * P_l^(2)).  Its intermediate tensor lives in one fixed array of
 * MM_NOALLOC_MAX_ELEMS doubles (16 MiB) compiled into the library, which every
 * GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 *   d      1..8;  n: host array of d sizes, 1..8192 each.
 *   M      host array of d device pointers, M[mu] n_mu x n_mu column-major.
 *   V, P   device tensors of N = prod n_mu doubles (i_1 fastest); must not
 *          overlap.  N > MM_NOALLOC_MAX_ELEMS is rejected with MM_ERR_SHAPE
 *          before any device work.
 *   stream cudaStream_t as void*; stream-ordered, no synchronisation.
 * The first call on a device (with that device current) looks up the array's
 * device address once (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls on a device share the one array and it keeps the
 * last call's contents (every element is written before it is read, so nothing
 * needs clearing): calls whose execution overlaps on the GPU -- on different
 * streams, or from different host threads -- race on it and must be ordered by
 * the caller.  Errors: MM_ERR_ARG, MM_ERR_SHAPE, MM_ERR_UNSUPPORTED (device
 * ordinal >= 64), MM_ERR_CUDA. */
#define MM_NOALLOC_MAX_ELEMS (1LL << 21)
MM_API int tucker_apply_noalloc(int d, const int64_t* n, const double* const* M,
                                const double* V, double* P, double alpha, void* stream);

/* ---- batches of independent problems ------------------------------------
 * Many independent 2D problems of uneven size (exponential Euler, eq. (19)),
 * advanced together in a mixed form: instances of equal (n1, n2) share packed
 * operand buffers, and each step is four launches for the whole batch (the
 * K u + g prepass, one persistent tensor-core launch per direction over the tiles
 * of every instance, the FP64 update), captured once in a CUDA graph.
 *
 * mm_tune: autotune = 1 picks the tile widths at creation by timing the batch's own
 * Tucker launches: every candidate nc in {160, 128, 96, 64} for all size classes at
 * once, then each class alone at every candidate, and keeps the per-class choices
 * if they beat the best uniform width (expint_batch_schedule reports the result);
 * nc_cap = 16..160 (a multiple of 16) fixes the width instead (0: autotune or 160);
 * graph = 1 makes
 * expint_batch_run replay a captured graph of its nsteps steps (0: plain launches).
 * A NULL mm_tune means {autotune 0, nc_cap 0, graph 1}. */
typedef struct mm_tune {
    int autotune;
    int nc_cap;
    int graph;
} mm_tune;

typedef struct mm_batch_s* mm_batch;

/*
 * expint_batch_create -- prepare `count` instances for batched stepping.
 *   plans  host array of count plans: all d = 2, the same mixed precision
 *          (MM_TF32X3 or MM_BF16X3), tridiagonal A_mu, ell_max >= 1; each plan's
 *          own tau is used for its instance.  The plans must outlive the batch.
 *   g      host array of count descriptors (MM_G_NONE or MM_G_CUBIC), or NULL.
 *   U      host array of count device pointers, n1 x n2 doubles each (i_1
 *          fastest), 8-byte aligned; the batch updates them in place.  When
 *          every n1 is even and every U 16-byte aligned the prepass takes two
 *          columns per thread (same results, fewer instructions).
 *   scheme MM_EXPEULER (others: MM_ERR_UNSUPPORTED).
 * Allocates the batch's device memory (packed operands: the two directions' split
 * inputs, 6 bytes per element each for BF16x3, 8 for TF32x3, and 4 bytes of FP32
 * result per element; each instance's phi_1 parts; and a second
 * FP64 state of every instance, 8 bytes per element, for the fused passes of
 * expint_batch_run), copies the instances' phi_1 parts, builds the tile lists
 * (and autotunes), then synchronises `stream`.  Errors: MM_ERR_ARG,
 * MM_ERR_UNSUPPORTED, MM_ERR_SHAPE (an instance with 2^31 elements or more),
 * MM_ERR_NOMEM, MM_ERR_CUDA; *out is NULL on error.
 */
MM_API int expint_batch_create(mm_batch* out, int count, const mm_plan* plans, const mm_nonlin* g,
                               double* const* U, int scheme, const mm_tune* tune, void* stream);

/* nsteps steps of every instance (Section 3.2, eq. (19)), stream-ordered, no
 * synchronisation.  Within a run the update u + tau y of one step and the prepass
 * K u + g of the next are one pass: it reads the state from one buffer and writes
 * the updated state to the other (the caller's U, the batch's second set, the
 * caller's U, ...), so that neighbouring tiles never see each other's new values;
 * the last step's update writes the caller's U.  Every value is bit for bit what
 * separate passes produce, so a run of k steps equals k runs of one step.  With the
 * graph option the first run with a given nsteps captures the steps (on a stream
 * of the batch) and every run replays the graph on `stream`.  t0 is the time of
 * the first step (the supported g are autonomous).  Errors: MM_ERR_ARG,
 * MM_ERR_CUDA. */
MM_API int expint_batch_run(mm_batch b, double t0, int nsteps, void* stream);

/* Synchronises `stream`; OR of MM_STATUS_* raised by the batch (>= 0). */
MM_API int expint_batch_status(mm_batch b, int reset, void* stream);

/* Host query: number of size classes, the tile width of class 0 (of every class
 * unless the autotuner kept per-class widths), mode-1 tiles per step, total degrees
 * of freedom.  Any pointer may be NULL. */
MM_API int expint_batch_info(mm_batch b, int* nclasses, int* nc_cap, int64_t* tiles_mode1,
                             int64_t* total_dof);

/* Host query of the autotuner's outcome: the tile width of every size class (into
 * nc_per_class, max_classes entries, or NULL), the number of classes, and the Tucker
 * time of one step (both directions, ms) with the best uniform width and with the
 * widths in use (0 without autotuning).  Returns 1 if per-class widths were kept,
 * 0 if one width serves every class, or MM_ERR_ARG (b NULL, max_classes too small). */
MM_API int expint_batch_schedule(mm_batch b, int32_t* nc_per_class, int max_classes, int* nclasses,
                                 float* ms_uniform, float* ms_chosen);

/* Host query: the tile order the grouped launches use: 0 = decreasing cost, taken
 * round-robin by the CTAs; 1 = the same with every other round of tiles reversed (the
 * autotuner keeps it when it times faster).  Errors: MM_ERR_ARG. */
MM_API int expint_batch_tile_order(mm_batch b);

/* Host setting: expint_batch_run replays a captured graph (on != 0, the default of
 * mm_tune) or launches the kernels directly (on = 0: each launch then carries its
 * own trace events, see mm_trace_enable).  Errors: MM_ERR_ARG. */
MM_API int expint_batch_set_graph(mm_batch b, int on);

/* Frees the batch (synchronises the device).  NULL is OK. */
MM_API int expint_batch_destroy(mm_batch b);

/* One-shot: create, run nsteps, synchronise, destroy. */
MM_API int expint_batched(int count, const mm_plan* plans, const mm_nonlin* g, double* const* U,
                          int scheme, double t0, int nsteps, const mm_tune* tune, void* stream);

/* Host-only (no device work): the tile list a batch of these sizes uses for one
 * direction (mode 1 or 2) at tile width nc_cap, tiles of decreasing cost.  Each
 * tile is 4 ints {instance, row tile, column split, size class}; pass tiles =
 * NULL to get the count only.  Errors: MM_ERR_ARG, MM_ERR_SHAPE,
 * MM_ERR_UNSUPPORTED (more than 32 size classes). */
MM_API int mm_batch_tile_plan(int count, const int64_t* n1, const int64_t* n2, int prec, int nc_cap,
                              int mode, int32_t* tiles, int64_t max_tiles, int64_t* ntiles);

/* ---- launch tracing --------------------------------------------------
 * Kernel classes counted by the library.  Counting is always on; with tracing
 * enabled every launch is also bracketed by a pair of CUDA events recorded on
 * the stream it is launched on (not while that stream is being captured).   */
#define MM_KC_CONTRACT_FP64 0   /* FP64 mu-mode / plain contraction kernel     */
#define MM_KC_CONTRACT_TF32 1   /* TF32x3 tcgen05 mu-mode contraction kernel   */
#define MM_KC_PREPASS       2   /* K u + g stencil / pointwise prepass         */
#define MM_KC_SPLIT         3   /* FP64 -> TF32 hi/lo operand split            */
#define MM_KC_COUNT         4

/* Start a new window: zero the counters; on != 0 also records event pairs.
 * Host-only, never fails. */
MM_API int mm_trace_enable(int on);

/* Launches of class `cls` in the current window and, if ms != NULL, their summed
 * device time in milliseconds (synchronises on the recorded events; 0 if
 * tracing is off).  launches is a host pointer to a long long.
 * Errors: MM_ERR_ARG (cls out of range), MM_ERR_CUDA. */
MM_API int mm_trace_read(int cls, long long* launches, double* ms);

/* Human-readable name of a status code (static string). */
MM_API const char* mm_status_str(int code);

/* Library version, major*10000 + minor*100 + patch. */
MM_API int mm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PHISPLIT_H */
