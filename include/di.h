/*
 * di.h -- C ABI of libdi.so, a single-GPU (sm_103a) D-Iteration solver.
 *
 * D-Iteration (Hong, Huynh, Mathieu, arXiv:1501.06350) solves the PageRank
 * equation x = d P x + (1 - d) Z (Section 2.1, Eq. pagerank-pf) by fluid
 * diffusion: a fluid vector F starts at (1 - d) Z, a history vector H at 0,
 * and diffusing a node i moves F(i) into H(i) and sends d F(i) P e_i to its
 * out-neighbours (Section 3.1, Eq. defF).  |x - H|_1 <= |F|_1 / (1 - d) at
 * every step (Theorem 1, Eq. SL), which is the stopping rule used here.
 *
 * Conventions shared by every entry point
 *  - Node ids are int32 in [0, n); n >= 1.  Link counts are int64.
 *  - The library copies every input it keeps; the caller keeps ownership of
 *    all buffers it passes.  Outputs go to caller-owned buffers.
 *  - A buffer argument lives in host memory or in device memory as the
 *    call's `mem` argument says (DI_MEM_HOST / DI_MEM_DEVICE).  Device
 *    buffers must be on the device the graph was created on.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *    of a call is ordered on that stream and the call returns only after it
 *    has completed, so the returned status is final and host outputs are
 *    valid on return.
 *  - Every call returns a di_status; on an error the handles stay valid and
 *    unchanged unless the description says otherwise.  DI_ERR_CUDA means a
 *    CUDA runtime call failed (di_last_cuda_error() gives its code).
 *  - Handles are not thread-safe: one host thread per handle at a time.
 *  - Device scratch comes from the device's default stream-ordered memory
 *    pool (cudaMallocAsync).  The first di_graph_create on a device sets that
 *    pool's release threshold to 16 GiB, so up to 16 GiB of freed scratch and
 *    replaced link arrays stays mapped for reuse by later calls instead of
 *    being unmapped at every synchronisation; it is an attribute of this
 *    process's pool only.  The
 *    allocation-free entry point di_residual_l1_noalloc allocates nothing.
 */
#ifndef DI_H
#define DI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct di_graph_s *di_graph_t;
typedef struct di_state_s *di_state_t;

typedef enum {
    DI_OK = 0,
    DI_ERR_INVALID_ARG = 1,    /* a scalar argument or a pointer is invalid        */
    DI_ERR_BAD_GRAPH = 2,      /* link structure or weights fail validation        */
    DI_ERR_OOM = 3,            /* device or host allocation failed                 */
    DI_ERR_NOT_CONVERGED = 4,  /* sweep cap reached; outputs hold the best state   */
    DI_ERR_CUDA = 5,           /* a CUDA runtime call failed                       */
    DI_ERR_DEVICE_TIMEOUT = 6  /* reserved: no kernel of this library waits on
                                  another, so no call returns it                  */
} di_status;

enum { DI_LAYOUT_CSR = 0, DI_LAYOUT_CSC = 1 };
enum { DI_W_NONE = 0, DI_W_F32 = 1, DI_W_F64 = 2 };
enum { DI_MEM_HOST = 0, DI_MEM_DEVICE = 1 };
enum { DI_PREC_F64 = 0, DI_PREC_F32 = 1 };

/* Solver options.  Always start from di_opts_default(). */
typedef struct {
    double theta_factor;   /* c in the frontier threshold theta_t = c |F|_1 / n; the
                              DI-argmax scheduler of Section 3.4 is c = 1.  0 < c <= 1
                              (then the largest fluid always qualifies).             */
    int64_t max_sweeps;    /* cap on frontier sweeps; reaching it returns
                              DI_ERR_NOT_CONVERGED with the state kept.  >= 1.       */
    int32_t check_every;   /* loop without CUDA graph: poll the stop flag every k
                              sweeps.  >= 1.                                         */
    int32_t use_graph;     /* 1: run the sweep loop as one CUDA graph with a device-
                              side while-condition (no host round trip per sweep).   */
    int32_t normalize;     /* 1: H_out = (1-d)/(1-d-d l) H, the solution for P
                              completed on dangling columns by Z (Section 3.3).      */
    int32_t profile;       /* 1: time every push launch with CUDA events (implies the
                              loop without CUDA graph); fills the push_* fields.     */
    int32_t precision;     /* arithmetic of the fluid F moved by the sweeps:
                              DI_PREC_F64: F is FP64 throughout.
                              DI_PREC_F32: iterative refinement.  The sweeps move an
                              FP32 copy of F and add every taken fluid, exactly, to an
                              FP64 accumulator D (the history gained in this cycle).
                              A cycle ends once the FP32 |F|_1 bound falls below
                              refine_ratio times its starting value (or below tol/2
                              of the stop test); then H += D and the FP64 fluid is
                              replaced by the exact residual F + d P D - D, which
                              equals (1-d) Z + d P H - H by Eq. HnFn.  The stop test
                              is applied to that FP64 residual only, so the returned
                              bound is certified in FP64 whatever the FP32 rounding. */
    double refine_ratio;   /* DI_PREC_F32 only: 0 < refine_ratio < 1.               */
    int32_t hub_deg;       /* degree-bin threshold: rows with more links than this are
                              taken by the plan kernel and pushed as pieces by many
                              warps; shorter rows are pushed by the warp that owns
                              their 128-node unit.  32 <= hub_deg <= 65536.            */
    int32_t piece;         /* links per hub piece (tile of the hub push), 128 <= piece
                              <= 65536.                                               */
} di_opts;

/* Solver report. */
typedef struct {
    double resid_l1;         /* |F|_1 of the returned state, exact FP64 sum in a fixed order */
    double l_dangling;       /* l = sum of H over dangling nodes (Section 3.3)              */
    double bound;            /* resid_l1 / (1 - d): certified |x - H|_1 bound (Eq. SL)      */
    double bound_completed;  /* resid_l1 / (1 - d - d l): distance of the normalised H to
                                the completed-P solution (Section 3.3)                     */
    int64_t sweeps;          /* frontier sweeps run by this call                            */
    int64_t diffusions;      /* elementary diffusions (nodes taken) by this call            */
    int64_t edge_pushes;     /* links pushed by this call (sum of out-degrees taken)        */
    double time_ms;          /* device time of the call's solve loop (CUDA events)          */
    double push_ms;          /* profile: summed duration of the push launches               */
    int64_t push_launches;   /* profile: number of push launches timed                      */
    int64_t push_edges;      /* profile: links pushed by those launches                     */
    int64_t push_entries;    /* profile: frontier entries read by those launches            */
    int64_t refinements;     /* DI_PREC_F32: FP64 refinement passes run by this call         */
    int64_t refine_links;    /* DI_PREC_F32: links pushed by those passes                    */
    double resid_inf;        /* max_i |F_i| of the returned state (FP64)                     */
    int64_t push_hot_links;  /* profile: links of the timed pushes whose target is a hot page
                                (summed in shared memory, not by a global atomic)           */
} di_info;

/* Fill *o with the defaults: theta_factor 1, max_sweeps 100000, check_every 8,
   use_graph 1, normalize 0, profile 0, precision DI_PREC_F64, refine_ratio 1e-5,
   hub_deg 256, piece 1024. */
void di_opts_default(di_opts *o);

/* Human-readable name of a status code (static storage). */
const char *di_status_str(di_status s);

/* cudaError_t code of the last failing CUDA call seen by this library on the
   calling thread (0 if none). */
int di_last_cuda_error(void);

/* Number of CUDA kernels this library has launched in the process so far
   (kernels run by the solver's CUDA-graph loop included).  Diagnostics only. */
int64_t di_kernel_launches(void);

/* Measured throughput, in 1e9 operations per second, of FP64 atomic additions
   at random slots of a 32 MB (L2-resident) vector on `device`: 32M additions
   per launch, a multiplicative hash of the operation index as the slot, best
   of three timed launches (CUDA events on `stream`) after a warm-up launch.
   Not a step of the method: every pushed link whose target is not summed in
   shared memory costs one such addition, so this is the push's roofline.
   Allocates and frees 32 MB of scratch; returns after the timing. */
di_status di_probe_atomic_adds(int device, double *gops, void *stream);

/* ---------------------------------------------------------------------------
 * Graph (Section 2.1, Eq. def-p).  P[i][j] = w(j,i) / sum_k w(j,k) for a link
 * j -> i, so column j of P is the out-link row of j; a node without out-link
 * (dangling) has a zero column.  Unweighted graphs have P[i][j] = 1/out(j).
 *
 * di_graph_create builds the canonical structure on the current CUDA device:
 * rows sorted by target, duplicate links merged (weights summed in input
 * order), self-links kept.  Input:
 *   n       nodes (1 <= n < 2^31)
 *   nnz     links in the input (0 <= nnz < 2^32)
 *   ptr     int64[n+1], ptr[0] = 0, non-decreasing, ptr[n] = nnz
 *   idx     int32[nnz], each in [0, n)
 *   w       weights (NULL = unweighted), float32 or float64 per w_dtype, each
 *           finite and > 0 (Section 2.1 requires w > 0)
 *   layout  DI_LAYOUT_CSR: rows of ptr are sources, idx holds targets;
 *           DI_LAYOUT_CSC: rows are targets, idx holds sources.
 *   mem     where ptr/idx/w live.
 * Returns DI_ERR_BAD_GRAPH when validation fails (nothing is created).
 * ------------------------------------------------------------------------- */
di_status di_graph_create(int64_t n, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                          const void *w, int w_dtype, int layout, int mem, void *stream,
                          di_graph_t *out);
di_status di_graph_destroy(di_graph_t g);

/* Sizes of the canonical graph: nodes, merged links, dangling nodes, weighted. */
di_status di_graph_info(di_graph_t g, int64_t *n, int64_t *nnz, int64_t *n_dangling,
                        int *weighted);

/* Copy the canonical out-link CSR: ptr int64[n+1], idx int32[nnz], w float64[nnz]
   (w may be NULL; for unweighted graphs it receives 1.0 per link). */
di_status di_graph_export_csr(di_graph_t g, int64_t *ptr, int32_t *idx, double *w, int mem,
                              void *stream);

/* Copy the in-link structure: for each target i, its sources in ascending
   order (ptr int64[n+1], idx int32[nnz], w float64[nnz] or NULL).  Built on
   the device on first use and kept with the graph. */
di_status di_graph_export_csc(di_graph_t g, int64_t *ptr, int32_t *idx, double *w, int mem,
                              void *stream);

/* ---------------------------------------------------------------------------
 * Solver state: the fluid F and history H (Section 3.1) of one problem on
 * one graph, kept on the device, plus the solver's working buffers.
 * ------------------------------------------------------------------------- */
di_status di_state_create(di_graph_t g, di_state_t *out);
di_status di_state_destroy(di_state_t s);

/* Solve x = d P x + (1 - d) Z from scratch (F = (1-d) Z, H = 0) until
 * |F|_1 / (1 - d) <= tol (Theorem 1, Eq. SL).
 *   d      damping, 0 < d < 1 (Section 2.1)
 *   Z      float64[n] in `mem`, any finite values (need not be a distribution);
 *          NULL = uniform 1/n
 *   tol    > 0
 *   opts   NULL = defaults
 *   H_out  float64[n] in `mem` receiving H (or its normalised form); may be NULL
 *   info   may be NULL
 * DI_ERR_NOT_CONVERGED: sweep cap reached; H_out/info hold the reached state. */
di_status di_solve(di_graph_t g, di_state_t s, double d, const double *Z, double tol,
                   const di_opts *opts, double *H_out, di_info *info, int mem, void *stream);

/* Continue from the state's current (H, F) until |F|_1 / (1 - d) <= tol, with
 * the damping of the last di_solve.  Used after di_update_edges (Theorem
 * update) or to tighten a tolerance.  Same outputs as di_solve. */
di_status di_resume(di_graph_t g, di_state_t s, double tol, const di_opts *opts,
                    double *H_out, di_info *info, int mem, void *stream);

/* Dynamic update (Section 3.5, Theorem update).  Applies m link changes in
 * batch order: op[k] = +1 makes src[k] -> dst[k] present (weight w[k], or 1
 * for unweighted graphs; an existing link gets the new weight), op[k] = -1
 * makes it absent (no-op if absent).  For every source j whose column of P
 * changes, the correction fluid d (P' - P) H is injected into F, H is kept,
 * and the graph becomes P'.  F may turn negative (Section 3.5 remark).  Call
 * di_resume next.  The state must belong to g and hold a solved or resumed
 * problem.  w: float64[m] or NULL (required iff the graph is weighted). */
di_status di_update_edges(di_graph_t g, di_state_t s, int64_t m, const int32_t *src,
                          const int32_t *dst, const double *w, const int8_t *op, int mem,
                          void *stream);

/* Read the state: H and F float64[n] (either may be NULL) and l (may be NULL). */
di_status di_state_export(di_state_t s, double *H, double *F, double *l, int mem, void *stream);

/* Overwrite the state's (H, F) with caller values (checkpoint resume), with
 * damping d for later di_resume calls.  Both float64[n], finite. */
di_status di_state_import(di_state_t s, const double *H, const double *F, double d, int mem,
                          void *stream);

/* ---------------------------------------------------------------------------
 * Autotuner (not in the paper).  Times from-scratch solves of g (uniform
 * teleport vector, damping d, tolerance tol, fluid precision `precision`) and
 * returns in *out the options that were fastest: one pass of coordinate search
 * over the threshold factor c (Section 3.4), the degree-bin threshold hub_deg,
 * the hub piece size and (DI_PREC_F32) the refinement ratio, starting from
 * di_opts_default; each candidate is the best of two solves (device time).
 *   budget      maximum number of candidates timed (>= 1; 20 covers the pass)
 *   cache_path  NULL, or a text file: a line for this graph shape, d, tol and
 *               precision is reused without timing anything; a new result is
 *               appended (one line per tuned problem).
 *   out         receives di_opts_default with the tuned fields
 *   best_ms, default_ms   time of the tuned and of the default options (may be NULL)
 *   trials      candidates timed by this call (0 when taken from the cache; may be NULL)
 * The graph itself is not changed; a private solver state is used. */
di_status di_autotune(di_graph_t g, double d, double tol, int32_t precision, int32_t budget, const char *cache_path,
                      di_opts *out, double *best_ms, double *default_ms, int32_t *trials, void *stream);

/* ---------------------------------------------------------------------------
 * Batched personalised solves: B teleport vectors on one graph (topic-
 * sensitive PageRank, Section 2.1; DI of Section 3.1 for each column).
 *
 * Solves x_c = d P x_c + (1 - d) Z_c for c = 0 .. B-1 together.  The fluid of
 * all columns of a node is stored contiguously, so one read of a node's links
 * serves every column and one link adds B contiguous values.  Each column has
 * its own DI-argmax threshold (Section 3.4) and stop test
 * |F_c|_1 / (1 - d) <= tol (Theorem 1); a node is diffused (all its columns)
 * when one of its unconverged columns passes its threshold.  Arithmetic as
 * DI_PREC_F32 of di_solve: FP32 fluid in the sweeps, FP64 accumulation of the
 * taken fluid, and cycles ended by an FP64 refinement R = R + d P D - D
 * (Eq. HnFn, computed by a pull over the in-links) on which the stop test is
 * applied, so every column's bound is certified in FP64.
 *   B        1 <= B <= 64 (fewer than 64 columns are padded internally)
 *   d        0 < d < 1
 *   Z        float64[n][B] in `mem`, node-major (Z[i*B + c]); finite; NULL = every
 *            column uniform 1/n
 *   tol      > 0, for every column
 *   opts     NULL = defaults; theta_factor, max_sweeps, use_graph, check_every and
 *            refine_ratio apply; precision is ignored; profile = 1 runs the loop
 *            one sweep at a time and fills push_ms / push_launches / push_edges
 *   H_out    float64[n][B] in `mem` (node-major) or NULL
 *   resid_out float64[B] in `mem` or NULL: |F_c|_1 of each column's returned
 *            state (exact FP64 sum in a fixed order)
 *   info     may be NULL; resid_l1 / bound are those of the worst column
 * Temporary device memory: about n x 64 x 36 bytes plus the graph's reverse
 * structure (kept with the graph).  DI_ERR_NOT_CONVERGED: sweep cap reached. */
di_status di_solve_batch(di_graph_t g, int32_t B, double d, const double *Z, double tol, const di_opts *opts,
                         double *H_out, double *resid_out, di_info *info, int mem, void *stream);

/* ---------------------------------------------------------------------------
 * Adjoint (backward pass of the solve; the paper has no counterpart).
 *
 * For a loss L = g . x with x = (1 - d)(I - d P)^-1 Z (Section 2.1,
 * Eq. pagerank-pf), the adjoint lambda solves (I - d P)^T lambda = g.  It is
 * computed by the fluid diffusion of Section 3.1 on the reverse graph (node i
 * sends d F_i P[i][j] to every j with a link j -> i), with the same sweep
 * kernels as di_solve: fluid F_0 = g, history H_0 = 0.  Rows of P^T sum to at
 * most 1, so the stop test is on the infinity norm:
 * |lambda - H|_inf <= |F|_inf / (1 - d) <= tol, and the frontier threshold is
 * capped at (1 - d)/2 max |F_i| (max |F| then shrinks every sweep).
 *   d        damping, 0 < d < 1
 *   gvec     float64[n] in `mem`: dL/dx, finite
 *   x        float64[n] in `mem`: the forward solution (e.g. H_out of di_solve);
 *            required when grad_w_out is given, else may be NULL
 *   tol      > 0, bound on |lambda - lambda_out|_inf
 *   opts     NULL = defaults; precision must be DI_PREC_F64; theta_factor,
 *            max_sweeps, use_graph, check_every, profile as for di_solve
 *   lambda_out  float64[n] or NULL: lambda
 *   grad_Z_out  float64[n] or NULL: dL/dZ = (1 - d) lambda
 *   grad_w_out  float64[nnz] or NULL: dL/dw per link of the canonical out-CSR
 *            (the order of di_graph_export_csr): for a link j -> k with
 *            P[k][j] = w(j,k) / W_j (unweighted graphs: all w = 1),
 *            dL/dw(j,k) = d x_j / W_j (lambda_k - (P^T lambda)_j)
 *   info     may be NULL; bound = |F|_inf / (1 - d), resid_inf = |F|_inf
 * The reverse graph and its solver state are built on the first call for the
 * graph's current link set and kept with the graph (about the size of the
 * graph plus one solver state).  DI_ERR_NOT_CONVERGED: sweep cap reached; the
 * outputs hold the reached state. */
di_status di_adjoint(di_graph_t g, double d, const double *gvec, const double *x, double tol,
                     const di_opts *opts, double *lambda_out, double *grad_Z_out, double *grad_w_out,
                     di_info *info, int mem, void *stream);

/* ---------------------------------------------------------------------------
 * Single steps of the sweep, exposed for verification.
 * ------------------------------------------------------------------------- */

/* Frontier selection alone (the DI-argmax test of Section 3.4 applied to a
 * fluid snapshot): writes the ascending ids i with |F_i| >= theta and F_i != 0
 * to ids (int32[n] capacity) and their number to *count.  F (float64[n]) and
 * ids live in `mem`; nothing in the graph or any state changes. */
di_status di_frontier_select(di_graph_t g, const double *F, double theta, int32_t *ids,
                             int64_t *count, int mem, void *stream);

/* |v|_1 of a float64[n] vector, summed on the device in a fixed order (the
 * result does not depend on launch timing). */
di_status di_residual_l1(di_graph_t g, const double *v, double *out, int mem, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free variant (no counterpart in the paper).
 *
 * di_residual_l1_noalloc computes exactly what di_residual_l1 computes (same
 * kernel, same fixed summation order, same result bit for bit) without
 * allocating any memory.  It is meant for callers that must not allocate on
 * the device: a serving loop whose device memory is entirely reserved by its
 * own pool, or a caller that cannot afford the implicit device-wide
 * synchronisation that cudaMalloc / cudaFree may cause.
 *   v       float64[n] in DEVICE (or managed) memory of the graph's device;
 *           anything else, host memory included, returns DI_ERR_INVALID_ARG
 *           before any work is queued (staging a host vector would need an
 *           allocation)
 *   out     host double receiving |v|_1
 * Scratch: one static device array of about 256 KiB (256 bytes of control
 * block and two float64 partials per 8,192-node tile) in libdi.so, present on
 * every device that loads the library until the process exits; it limits the
 * graph to n <= 2^16 * 2048 = 134,217,728 nodes (larger graphs return
 * DI_ERR_INVALID_ARG).  The first call made on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture on the device.  Every call clears the
 * part of the array it relies on, but all calls share the one array: calls
 * whose GPU work overlaps (other streams, other host threads) race and must
 * be serialised by the caller.  Returns after the result is on the host. */
di_status di_residual_l1_noalloc(di_graph_t g, const double *v, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DI_H */
