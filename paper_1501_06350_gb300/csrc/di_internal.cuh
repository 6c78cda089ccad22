// Internal declarations shared by the translation units of libdi.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/di.h"

namespace di {

// ---------------------------------------------------------------- errors
struct Err {
    di_status st;
};

di_status note_cuda(cudaError_t e);          // records e for di_last_cuda_error()
#define DI_CUDA(call)                                                      \
    do {                                                                   \
        cudaError_t _e = (call);                                           \
        if (_e != cudaSuccess) return ::di::note_cuda(_e);                 \
    } while (0)
#define DI_TRY(call)                                                       \
    do {                                                                   \
        di_status _s = (call);                                             \
        if (_s != DI_OK) return _s;                                        \
    } while (0)

// Stream-ordered device allocation; returns DI_ERR_OOM on failure.
di_status dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
void pool_keep(int device);
// tab[q] = row of link q << KEY_BUCKET_SHIFT for q < ceil(nnz / 2^KEY_BUCKET_SHIFT);
// tab[that count] = n - 1.  tab holds that count + 1 entries; nnz >= 1.
di_status row_bucket_table(const uint32_t *rp, int64_t n, int64_t nnz, uint32_t *tab, cudaStream_t s);   // keep freed scratch in the default pool (once per device)

template <typename T>
di_status dalloc_t(T **p, size_t count, cudaStream_t s)
{
    return dalloc(reinterpret_cast<void **>(p), count * sizeof(T) + 16, s);
}

// RAII holder for temporaries of one call (freed stream-ordered).
struct Temps {
    cudaStream_t s;
    void *p[64];
    int k = 0;
    explicit Temps(cudaStream_t st) : s(st) {}
    template <typename T>
    di_status get(T **out, size_t count)
    {
        if (k >= 64) return DI_ERR_OOM;
        di_status r = dalloc_t(out, count, s);
        if (r == DI_OK) p[k++] = *out;
        return r;
    }
    ~Temps()
    {
        for (int i = 0; i < k; i++) dfree(p[i], s);
    }
};

// ---------------------------------------------------------------- primitives
// Exclusive prefix sum of n values (uint8/uint32/uint64 input) into uint64 out;
// *total_dev receives the sum (device pointer, may be null).  Deterministic.
template <typename T>
di_status scan_exclusive(const T *in, uint64_t *out, int64_t n, uint64_t *total_dev,
                         cudaStream_t s);

// Stable LSD radix sort of (key, val) pairs over the listed bit ranges (each
// range <= 8 bits, applied in order).  Result ends up in (*keys, *vals); the
// alternate buffers are swapped in as needed.
di_status radix_sort_pairs(uint64_t **keys, uint32_t **vals, uint64_t **keys_alt,
                           uint32_t **vals_alt, int64_t n, const int *bit_lo,
                           const int *bit_cnt, int npass, cudaStream_t s);

// Bits needed to represent values in [0, n).
inline int bits_for(int64_t n)
{
    int b = 0;
    while (b < 63 && (int64_t(1) << b) < n) b++;
    return b;
}

int sm_count(int device);

// Kernel launches issued by the library (process-wide counter).
void count_launches(int64_t k);
int64_t launches();

}  // namespace di

// ---------------------------------------------------------------- handles
struct di_graph_s {
    int device = 0;
    int64_t n = 0;
    int64_t nnz = 0;
    int64_t n_dangling = 0;
    bool weighted = false;
    bool off64 = false;       // reserved: offsets are uint32 (nnz < 2^32)
    int64_t version = 0;      // bumped by every structural update
    void *rp = nullptr;       // out-CSR row pointers, uint32 or uint64 [n+1]
    int32_t *col = nullptr;   // targets [nnz]
    double *w = nullptr;      // link weights [nnz] (weighted only)
    double *wsum = nullptr;   // W_j = sum of row j's weights, left to right [n]
    // push copy of col: links into the HOT_K most linked-to pages carry
    // 0x80000000 | slot instead of the page id (built on demand per version)
    int32_t *pcol = nullptr;  // [nnz]
    float *w32 = nullptr;     // [nnz] FP32 copy of w for the FP32-fluid push (weighted only)
    unsigned *indeg = nullptr;    // [n] in-links per page, kept current by updates
    int32_t *hot_node = nullptr;  // [HOT_K] page of each hot slot
    int *slot_of = nullptr;       // [n] hot slot of each page, -1 if none (kept across link updates)
    int nhot = 0;
    int64_t pcol_version = -1;
    // reverse graph (links i -> j for every j -> i, weight P[i][j]) and the
    // solver state of the adjoint, built on demand per version
    struct di_graph_s *rev = nullptr;
    struct di_state_s *rev_state = nullptr;
    int64_t rev_version = -1;
    // in-link structure, built on demand
    int64_t *cp = nullptr;    // [n+1]
    int32_t *crow = nullptr;  // [nnz]
    double *cw = nullptr;     // [nnz] (weighted only)
};

// Device-side control block of the sweep loop (one per state).
struct DevCtl {
    double theta;          // threshold used by the next selection
    double l1;             // |F|_1 at the start of the last sweep
    double stop_l1;        // (1 - d) tol
    double d;
    double theta_factor;
    double final_l1;       // |F|_1 of the final state (FP64, fixed order)
    double final_l;        // sum of H over dangling nodes (final reduction)
    double sweep_stop;     // the sweep loop ends when its |F|_1 bound is at most this
    double refine_ratio;   // FP32 fluid: each cycle ends at refine_ratio x its starting |F|_1
    double inf_cap;        // inf_norm: the threshold never exceeds inf_cap x max |F_i|
    double final_max;      // max |F_i| of the final state (FP64)
    double hot_scale;      // bound on what one sweep adds into one page: sets the push's fixed point
    unsigned long long diffusions;
    unsigned long long edge_pushes;
    unsigned long long sweep;         // pushes performed by this call
    unsigned long long max_sweeps;
    unsigned long long npieces;       // hub pieces cut by the plan (read by the push)
    unsigned long long sweep_links;   // links pushed by the running push
    unsigned long long sweep_hot;     // ... of which into hot pages (summed in shared memory)
    unsigned long long nent;          // frontier nodes of the last selection (mask bits)
    int inf_norm;              // 1: stop test and threshold cap on max |F_i| (adjoint)
    unsigned int done;         // 0 running, 1 converged, 2 sweep cap
    unsigned int ticket2;      // last-block ticket of the reductions
    unsigned int err;          // unused (keeps the layout of the block)
    unsigned int push_ready;   // 1: the mask/pieces describe a frontier not yet pushed
    unsigned int pad1;
};

// The buffers of a graph and a state that move when the graph is updated or
// the degree bins change.  The sweep kernels read them from this block (one
// copy per state in device memory, rewritten before every solve), so a
// captured sweep loop stays valid across updates.
struct GraphPtrs {
    const uint32_t *rp;
    const int32_t *pcol;
    const double *w;
    const float *w32;
    unsigned *hub_list;
    uint64_t hub_cap;         // entries of hub_list
    uint32_t *pc_row;
    uint32_t *pc_len;
    double *pc_val;
    int nhot;
    uint32_t piece;
};

struct di_state_s {
    di_graph_t g = nullptr;
    int device = 0;
    int64_t ntiles = 0;
    int64_t max_items = 0;         // capacity of the hub-piece queue
    double d = 0.85;
    bool have_problem = false;
    int64_t prep_version = 0;      // graph version the derived buffers were built for
    int64_t problem_version = -1;  // graph version (H, F) belongs to
    double *F = nullptr;
    double *H = nullptr;
    // FP32-fluid form: the working fluid, the FP64 sum of the fluid taken at
    // each node during the current cycle, and the control block of the
    // refinement pass (allocated on the first FP32 solve)
    float *F32 = nullptr;
    double *D = nullptr;
    DevCtl *rctl = nullptr;
    DevCtl *host_rctl = nullptr;
    double *dscale = nullptr;      // d / W_j (or d / out(j)) per node, 0 if dangling
    double *dtab = nullptr;        // d / k for k <= DTAB_MAX (fills dscale without FP64 divisions)
    double dscale_d = -1.0;        // damping dscale was built for
    // frontier of the last selection: one bit per selected node that is not a
    // hub; selected hubs (more than hub_deg links) go to hub_list
    unsigned int *mask = nullptr;      // [slots / 32]
    unsigned int *hubbits = nullptr;   // [slots / 32] static: node has more than hub_deg links
    int hub_deg = 256;                 // degree-bin threshold the hub bits were built for
    int piece = 1024;                  // links per hub piece
    unsigned int *hub_list = nullptr;  // [nhub_cap]
    int64_t nhub_cap = 0;
    // hub pieces (rows longer than hub_deg, cut into `piece` links)
    unsigned int *pc_row = nullptr;
    unsigned int *pc_len = nullptr;
    double *pc_val = nullptr;
    // per-tile partials
    unsigned int *tile_cnt = nullptr;
    unsigned int *tile_hub = nullptr;        // selected hubs of each tile (listed from hub_base[tile] on)
    uint64_t *hub_base = nullptr;            // first hub-list slot of each tile (its hub nodes before it)
    unsigned int *tile_diff = nullptr;
    float *tile_l1f = nullptr;               // |F|_1 partial, FP32 rounded upward
    unsigned *tile_maxf = nullptr;           // max |F_i|, FP32 bits rounded downward
    unsigned *tile_maxu = nullptr;           // max |F_i|, FP32 bits rounded upward
    double *tile_max = nullptr;              // FP64 max partials of the reductions
    double *tile_l1 = nullptr;               // FP64 partials of the reductions
    double *tile_l = nullptr;
    DevCtl *ctl = nullptr;
    DevCtl *host_ctl = nullptr;    // pinned mirror
    GraphPtrs *gp = nullptr;       // device copy of the moving buffers
    GraphPtrs *host_gp = nullptr;  // pinned mirror
    // CUDA graph of the sweep loop
    cudaGraphExec_t gexec = nullptr;     // FP64 fluid sweep loop
    cudaGraphExec_t gexec32 = nullptr;   // FP32 fluid sweep loop
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // per-sweep frontier statistics (links, entries) written by the selection
    unsigned long long *stats = nullptr;
    cudaEvent_t *pev = nullptr;    // profile: event pairs around push launches
    int npev = 0;
};

namespace di {
constexpr int SEL_THREADS = 512;
constexpr int SEL_PER_THREAD = 16;
constexpr int TILE = SEL_THREADS * SEL_PER_THREAD;   // nodes per selection tile
// Row-pointer arrays read by the push carry RP_PAD zeroed entries past rp[n]:
// the push stages the 129 row pointers of a whole 128-page unit, which reaches
// rp[n + 127] for the unit that holds page n - 1.
constexpr int RP_PAD = 128;
// Links per bucket of the row lookup table (row_bucket_table).
constexpr int KEY_BUCKET_SHIFT = 8;
constexpr int PUSH_THREADS = 256;
constexpr int HUB_DEG = 256;                         // default degree-bin threshold (di_opts.hub_deg)
constexpr int DTAB_MAX = 65536;                      // out-degrees with a tabulated d / out(j)
constexpr int PIECE = 1024;                          // default links per hub piece (di_opts.piece)
constexpr int RED_THREADS = 256;
constexpr int STAT_CAP = 4096;                       // sweeps with recorded statistics
constexpr int PLAN_CTAS = 64;                        // CTAs of the per-sweep plan kernel
constexpr int HOT_K = 2048;                          // pages accumulated in shared memory by the push
constexpr unsigned HOT_MIN_INDEG = 64;               // ... if they have at least this many in-links

di_status graph_build_csc(di_graph_s *g, cudaStream_t s);
di_status graph_build_push_targets(di_graph_s *g, cudaStream_t s);
di_status graph_create(int64_t n, int64_t nnz, const int64_t *ptr, const int32_t *idx, const void *w,
                       int wdt, int layout, int mem, cudaStream_t s, di_graph_s *g);
di_status graph_export(di_graph_s *g, bool csc, int64_t *ptr, int32_t *idx, double *w, int mem,
                       cudaStream_t s);
void graph_release(di_graph_s *g);
int last_cuda();
di_status copy_out_H(di_state_s *st, double *H_out, bool normalize, double l, int mem, cudaStream_t s);
di_status state_l(di_graph_s *g, di_state_s *st, double *l, cudaStream_t s);
di_status check_finite(const double *v, int64_t n, bool *ok, cudaStream_t s);
di_status state_alloc(di_state_s *st, cudaStream_t s);
di_status state_prepare_graph(di_graph_s *g, di_state_s *st, cudaStream_t s);
di_status state_set_bins(di_graph_s *g, di_state_s *st, int hub_deg, int piece, cudaStream_t s);
di_status state_sync_ptrs(di_graph_s *g, di_state_s *st, cudaStream_t s);
di_status autotune(di_graph_s *g, double d, double tol, int precision, int budget, const char *cache,
                   di_opts *best, double *best_ms, double *default_ms, int *trials, int *from_cache,
                   cudaStream_t s);
di_status state_free(di_state_s *st);
di_status solve_loop(di_graph_s *g, di_state_s *st, double tol, const di_opts *o, di_info *info,
                     cudaStream_t s, bool fresh, const double *Z_dev, bool inf_norm = false);
di_status graph_build_reverse(di_graph_s *g, cudaStream_t s);
void reverse_release(di_graph_s *g);
di_status solve_batch(di_graph_s *g, int B, double d, const double *Z, double tol, const di_opts *o, double *H_out,
                      double *resid_out, di_info *info, int mem, cudaStream_t s);
di_status adjoint(di_graph_s *g, double d, const double *gvec, const double *x, double tol, const di_opts *o,
                  double *lambda, double *grad_Z, double *grad_w, di_info *info, cudaStream_t s);
di_status l1_device(di_graph_s *g, const double *v, double *out_host, cudaStream_t s);
di_status l1_device_into(di_graph_s *g, const double *v, double *part_l1, double *part_l, DevCtl *ctl,
                         double *out_host, cudaStream_t s);
di_status select_only(di_graph_s *g, const double *F, double theta, int32_t *ids, int64_t *count,
                      cudaStream_t s);
di_status update_edges(di_graph_s *g, di_state_s *st, int64_t m, const int32_t *src,
                       const int32_t *dst, const double *w, const int8_t *op, cudaStream_t s);
}  // namespace di
