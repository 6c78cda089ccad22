// Dynamic update (Section 3.5, Theorem update): apply a batch of link
// insertions/deletions to the canonical graph and inject the correction fluid
// d (P' - P) H into F, keeping H.
//
// Only the batch is sorted (stable radix sort of source << 32 | target, so the
// last operation on a link decides).  Each distinct batch link is looked up
// in its (sorted) old row and classified: inserted, deleted, re-weighted or
// no-op.  Rows without an effective change are moved as they are (a warp per
// 32 rows, coalesced); in the changed rows every kept old link and every
// inserted link computes its own position from prefix counts (no serial merge).
// A source j is "touched" when its set of out-links or a weight changes, i.e.
// when column j of P changes; only those columns contribute to d (P' - P) H,
// and for them the whole old column is withdrawn and the whole new column
// injected (every entry changes when out(j) or W_j changes).
#include <cuda_runtime.h>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;
constexpr unsigned FULL = 0xffffffffu;

enum : unsigned char { EFF_NOP = 0, EFF_INS = 1, EFF_DEL = 2, EFF_UPD = 3 };

__global__ void k_check_batch(const int32_t *src, const int32_t *dst, const double *w, const int8_t *op,
                              int64_t m, int64_t n, unsigned *err)
{
    unsigned e = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (src[k] < 0 || src[k] >= n || dst[k] < 0 || dst[k] >= n) e |= 1u;
        if (op[k] != 1 && op[k] != -1) e |= 2u;
        if (w && op[k] == 1 && !(isfinite(w[k]) && w[k] > 0.0)) e |= 4u;
    }
    if (e) atomicOr(err, e);
}

__global__ void k_batch_keys(const int32_t *src, const int32_t *dst, int64_t m, uint64_t *keys,
                             uint32_t *vals)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        keys[k] = ((uint64_t)(uint32_t)src[k] << 32) | (uint32_t)dst[k];
        vals[k] = (uint32_t)k;
    }
}

// The last entry of each run of equal keys is the last operation on that link.
__global__ void k_run_ends(const uint64_t *keys, int64_t m, uint8_t *keep)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        keep[e] = (e == m - 1 || keys[e + 1] != keys[e]) ? 1 : 0;
}

__global__ void k_unique(const uint64_t *keys, const uint32_t *vals, const uint8_t *keep, const uint64_t *pos,
                         int64_t m, const int8_t *op, const double *wb, uint64_t *ukey, int8_t *uop, double *uw)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[e]) continue;
        const int64_t k = (int64_t)pos[e];
        const uint32_t b = vals[e];
        ukey[k] = keys[e];
        uop[k] = op[b];
        uw[k] = wb ? wb[b] : 1.0;
    }
}

// Classify each distinct batch link against its old row (binary search);
// count the row's degree change, flag the row, keep in-degrees current.
__global__ void k_classify(const uint64_t *ukey, const int8_t *uop, const double *uw, const uint64_t *nu_dev,
                           const Off *rp, const int32_t *col, const double *w, uint8_t *eff, int *delta,
                           uint8_t *touched, unsigned *indeg)
{
    const int64_t nu = (int64_t)*nu_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nu;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t sr = (uint32_t)(ukey[k] >> 32);
        const int32_t tg = (int32_t)(uint32_t)ukey[k];
        const Off end = rp[sr + 1];
        Off lo = rp[sr], hi = end;
        while (lo < hi) {
            const Off mid = lo + ((hi - lo) >> 1);
            if (col[mid] < tg) lo = mid + 1;
            else hi = mid;
        }
        const bool present = lo < end && col[lo] == tg;
        const bool keep = uop[k] == 1;
        unsigned char e = EFF_NOP;
        int dl = 0;
        if (present && !keep) {
            e = EFF_DEL;
            dl = -1;
        } else if (!present && keep) {
            e = EFF_INS;
            dl = 1;
        } else if (present && keep && w && uw[k] != w[lo]) {
            e = EFF_UPD;
        }
        eff[k] = e;
        if (e != EFF_NOP) {
            if (dl) atomicAdd(delta + sr, dl);
            touched[sr] = 1;
            if (indeg && dl) atomicAdd(indeg + tg, (unsigned)dl);
        }
    }
}

__global__ void k_new_degree(const Off *rp, const int *delta, int64_t n, uint32_t *deg)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        deg[j] = (uint32_t)((int64_t)(rp[j + 1] - rp[j]) + delta[j]);
}

__global__ void k_rp_from_scan(const uint64_t *ex, const uint64_t *total, int64_t n, Off *nrp)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n;
         j += (int64_t)gridDim.x * blockDim.x)
        nrp[j] = (Off)(j < n ? ex[j] : *total);
}

// Rows without an effective change keep their links; a warp moves the links
// of 32 consecutive rows (lane l owns row 32g + l) to their new offsets.
__global__ void k_copy_rows(const Off *rp, const Off *nrp, const int32_t *col, const double *w,
                            const int32_t *pcol, const uint8_t *touched, int64_t n, int32_t *ncol, double *nw,
                            int32_t *npcol)
{
    const int lane = threadIdx.x & 31;
    const int64_t ngroups = (n + 31) / 32;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < ngroups; gi += nwarp) {
        const int64_t r = gi * 32 + lane;
        Off a = 0, na = 0, len = 0;
        if (r < n) {
            a = rp[r];
            na = nrp[r];
            if (!touched[r]) len = rp[r + 1] - a;
        }
        Off incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Off y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const Off total = __shfl_sync(FULL, incl, 31);
        const Off excl = incl - len;
        // 4 x 32 links in flight per warp: positions first, then the loads,
        // then the stores
        for (Off base = 0; base < total; base += 128) {
            Off from[4], to[4];
#pragma unroll
            for (int g = 0; g < 4; g++) {
                const Off e = base + (Off)(32 * g + lane);
                const Off eq = e < total ? e : total - 1;
                int j = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const Off ex = __shfl_sync(FULL, excl, j + step);
                    if (ex <= eq) j += step;
                }
                const Off o = eq - __shfl_sync(FULL, excl, j);
                from[g] = __shfl_sync(FULL, a, j) + o;
                to[g] = __shfl_sync(FULL, na, j) + o;
            }
            int32_t c[4], pc[4];
            double wv[4];
#pragma unroll
            for (int g = 0; g < 4; g++) {
                const bool ok = base + (Off)(32 * g + lane) < total;
                c[g] = ok ? col[from[g]] : 0;
                pc[g] = (ok && npcol) ? pcol[from[g]] : 0;
                wv[g] = (ok && w) ? w[from[g]] : 0.0;
            }
#pragma unroll
            for (int g = 0; g < 4; g++) {
                if (base + (Off)(32 * g + lane) >= total) continue;
                ncol[to[g]] = c[g];
                if (w) nw[to[g]] = wv[g];
                if (npcol) npcol[to[g]] = pc[g];
            }
        }
    }
}

__global__ void k_list(const uint8_t *flag, const uint64_t *pos, int64_t n, uint32_t *list)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) list[pos[i]] = (uint32_t)i;
}

// Range [qs, qe) of the distinct batch entries of each changed row (the
// entries are sorted by source, and every changed row has at least one).
__global__ void k_row_ranges(const uint64_t *ukey, const uint64_t *nu_dev, const uint8_t *touched,
                             const uint64_t *tpos, uint32_t *qs, uint32_t *qe)
{
    const int64_t nu = (int64_t)*nu_dev;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nu;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(ukey[e] >> 32);
        if (!touched[j]) continue;
        if (e == 0 || (uint32_t)(ukey[e - 1] >> 32) != j) qs[tpos[j]] = (uint32_t)e;
        if (e == nu - 1 || (uint32_t)(ukey[e + 1] >> 32) != j) qe[tpos[j]] = (uint32_t)(e + 1);
    }
}

// Changed rows are cut into chunks of CH old links (a row without old links
// is one chunk), so that a long row is merged and injected by many threads.
constexpr Off CH = 256;

// (Rows of at most `short_max` links get no chunk: k_merge_short handles them.)
__global__ void k_chunk_counts(const uint32_t *tlist, const uint64_t *nt_dev, const Off *rp, uint32_t *cnt,
                               Off short_max)
{
    const int64_t nt = (int64_t)*nt_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = tlist[k];
        const Off deg = rp[j + 1] - rp[j];
        if (short_max && deg <= short_max) cnt[k] = 0u;
        else cnt[k] = deg == 0 ? 1u : (uint32_t)((deg + CH - 1) / CH);
    }
}

__global__ void k_chunk_fill(const uint32_t *cnt, const uint64_t *cpos, const uint64_t *nt_dev, uint32_t *ch_row,
                             uint32_t *ch_idx)
{
    const int64_t nt = (int64_t)*nt_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t base = cpos[k];
        for (uint32_t c = 0; c < cnt[k]; c++) {
            ch_row[base + c] = (uint32_t)k;
            ch_idx[base + c] = c;
        }
    }
}

// The two coefficients of changed row j's column of d (P' - P) H (Theorem
// update), one thread per changed row: d H_j (1/out'(j) - 1/out(j)) for a kept
// link and -d H_j / out(j) for a deleted one.  (Computed once per row with
// every lane busy: FP64 division is slow on this part, and a per-chunk
// computation by one lane kept the FP64 pipe busy for the whole merge.)
__global__ void k_row_coef(const uint32_t *tlist, const uint64_t *nt_dev, const Off *rp, const Off *nrp,
                           const double *H, double d, double2 *coef)
{
    const int64_t nt = (int64_t)*nt_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = tlist[k];
        const Off deg = rp[j + 1] - rp[j], dn = nrp[j + 1] - nrp[j];
        double c_keep = 0.0, c_del = 0.0;
        if (deg) {
            const double h = d * H[j];
            c_del = -(h / (double)deg);
            c_keep = (dn ? h / (double)dn : 0.0) + c_del;
        }
        coef[k] = make_double2(c_keep, c_del);
    }
}

// First batch entry of row j whose target is >= key's, inside [q, qe).
__device__ __forceinline__ int64_t lower_target(const uint64_t *ukey, int64_t q, int64_t qe, uint64_t key)
{
    while (q < qe) {
        const int64_t mid = (q + qe) >> 1;
        if (ukey[mid] < key) q = mid + 1;
        else qe = mid;
    }
    return q;
}

// The merged row j of the new CSR holds, in target order, the old links not
// deleted and the inserted ones.  An old link at position i (target c) lands
// at nrp[j] + (i - rp[j]) - (deletions with target < c) + (insertions with
// target < c); the batch entries of the row are sorted by target, so both
// counts are prefix differences (ins_pre / del_pre: exclusive counts over the
// sorted batch) at the row's first entry with target >= c.  One warp per
// chunk of CH old links, one lane per link.
//
// With F given (unweighted graphs), the correction fluid of Theorem update is
// added here too: column j of d (P' - P) H is d H_j (1/out'(j) - 1/out(j)) at
// a link kept in the row, -d H_j / out(j) at a deleted one and d H_j / out'(j)
// at an inserted one (k_merge_ins), one add per link instead of a withdrawal
// of the old column plus an injection of the new one.
__global__ void k_merge_old(const uint32_t *ch_row, const uint32_t *ch_idx, const uint64_t *nch_dev,
                            const uint32_t *tlist, const uint32_t *qs, const uint32_t *qes, const Off *rp,
                            const int32_t *col, const double *w, const int32_t *pcol, const Off *nrp,
                            const uint64_t *ukey, const uint8_t *eff, const double *uw, const uint64_t *ins_pre,
                            const uint64_t *del_pre, int32_t *ncol, double *nw, int32_t *npcol, const double2 *coef,
                            double *F)
{
    const int64_t nch = (int64_t)*nch_dev;
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nch; t += nwarp) {
        const uint32_t r = ch_row[t];
        const uint32_t j = tlist[r];
        const Off a = rp[j], b = rp[j + 1];
        const Off i0 = a + ch_idx[t] * CH;
        const Off i1 = (b > i0 && b - i0 > CH) ? i0 + CH : b;
        const int64_t q = qs[r], qe = qes[r];
        const uint64_t rowkey = (uint64_t)j << 32;
        const Off out0 = nrp[j] - a;
        double c_keep = 0.0, c_del = 0.0;
        if (F && i0 < i1) {
            const double2 cf = coef[r];
            c_keep = cf.x;
            c_del = cf.y;
        }
        // the batch entries whose targets fall inside this chunk's target range
        // (all of the row's when it has few): two searches per chunk, by two lanes
        int64_t klo = q, khi = qe;
        if (qe - q > 32 && i0 < i1) {
            int64_t kk = 0;
            if (lane < 2) {
                const uint32_t c = (uint32_t)col[lane ? i1 - 1 : i0];
                kk = lower_target(ukey, q, qe, (rowkey | c) + (uint64_t)lane);
            }
            klo = __shfl_sync(FULL, kk, 0);
            khi = __shfl_sync(FULL, kk, 1);
        }
        const int64_t nb = khi - klo;
        if (nb <= 32) {
            // those few entries sit in the lanes' registers (lane k: entry
            // klo + k, ascending targets); a link finds how many have a smaller
            // target by a search over the lanes, and counts the deletions and
            // insertions among them from two ballots, on top of the row's
            // counts before the window
            const Off dl0 = klo > q ? (Off)(del_pre[klo] - del_pre[q]) : 0;
            const Off in0 = klo > q ? (Off)(ins_pre[klo] - ins_pre[q]) : 0;
            uint32_t tgt = 0;
            unsigned char ef = EFF_NOP;
            if (lane < nb) {
                tgt = (uint32_t)ukey[klo + lane];
                ef = eff[klo + lane];
            }
            const unsigned dmask = __ballot_sync(FULL, lane < nb && ef == EFF_DEL);
            const unsigned imask = __ballot_sync(FULL, lane < nb && ef == EFF_INS);
            for (Off base = i0; base < i1; base += 32) {
                const Off i = base + lane;
                const bool live = i < i1;
                const uint32_t c = live ? (uint32_t)col[i] : 0u;
                int kk = 0;   // entries with target < c
#pragma unroll
                for (int step = 32; step > 0; step >>= 1) {
                    const uint32_t tk = __shfl_sync(FULL, tgt, (kk + step - 1) & 31);
                    if (kk + step <= (int)nb && tk < c) kk += step;
                }
                const uint32_t tm = __shfl_sync(FULL, tgt, kk & 31);
                const unsigned char ek = (unsigned char)__shfl_sync(FULL, (unsigned)ef, kk & 31);
                const bool match = kk < (int)nb && tm == c;
                const unsigned char em = match ? ek : EFF_NOP;
                const unsigned below = kk >= 32 ? 0xffffffffu : (1u << kk) - 1u;
                if (!live) continue;
                if (F) atomicAdd(F + c, em == EFF_DEL ? c_del : c_keep);
                if (em == EFF_DEL) continue;
                const Off out = out0 + i - (dl0 + (Off)__popc(dmask & below)) + (in0 + (Off)__popc(imask & below));
                ncol[out] = (int32_t)c;
                if (nw) nw[out] = em == EFF_UPD ? uw[klo + kk] : w[i];
                if (npcol) npcol[out] = pcol[i];
            }
        } else {
            for (Off i = i0 + lane; i < i1; i += 32) {
                const int32_t c = col[i];
                const int64_t k = lower_target(ukey, q, qe, rowkey | (uint32_t)c);
                unsigned char e = EFF_NOP;
                if (k < qe && (uint32_t)ukey[k] == (uint32_t)c) e = eff[k];
                if (F) atomicAdd(F + c, e == EFF_DEL ? c_del : c_keep);
                if (e == EFF_DEL) continue;
                const Off out = out0 + i - (Off)(del_pre[k] - del_pre[q]) + (Off)(ins_pre[k] - ins_pre[q]);
                ncol[out] = c;
                if (nw) nw[out] = e == EFF_UPD ? uw[k] : w[i];
                if (npcol) npcol[out] = pcol[i];
            }
        }
    }
}

// The changed rows of at most CH old links (unweighted graphs), 32 rows per
// warp: lane l reads row tlist[32g + l] (its bounds, batch range and
// coefficients) and the links of the 32 rows are dealt to the lanes 32 at a
// time, so that the chain of dependent loads that starts a row is paid once
// per 32 rows rather than once per row.  A link's place and correction fluid
// are those of k_merge_old (its row's batch entries searched in global memory:
// a short row has few).
__global__ void k_merge_short(const uint32_t *tlist, const uint64_t *nt_dev, const uint32_t *qs,
                              const uint32_t *qes, const Off *rp, const int32_t *col, const int32_t *pcol,
                              const Off *nrp, const uint64_t *ukey, const uint8_t *eff, const uint64_t *ins_pre,
                              const uint64_t *del_pre, int32_t *ncol, int32_t *npcol, const double2 *coef,
                              double *F)
{
    const int64_t nt = (int64_t)*nt_dev;
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi * 32 < nt; gi += nwarp) {
        const int64_t k = gi * 32 + lane;
        uint32_t j = 0, q = 0, qe = 0;
        Off a = 0, len = 0, out0 = 0;
        double c_keep = 0.0, c_del = 0.0;
        if (k < nt) {
            j = tlist[k];
            a = rp[j];
            const Off b = rp[j + 1];
            if (b - a <= CH) {
                len = b - a;
                q = qs[k];
                qe = qes[k];
                out0 = nrp[j] - a;
                if (F && len) {
                    const double2 cf = coef[k];
                    c_keep = cf.x;
                    c_del = cf.y;
                }
            }
        }
        Off incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Off y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const Off total = __shfl_sync(FULL, incl, 31);
        const Off excl = incl - len;
        for (Off base = 0; base < total; base += 32) {
            const Off e = base + lane;
            const Off eq = e < total ? e : total - 1;
            int r = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const Off ex = __shfl_sync(FULL, excl, r + step);
                if (ex <= eq) r += step;
            }
            const Off i = __shfl_sync(FULL, a, r) + (eq - __shfl_sync(FULL, excl, r));
            const uint32_t jr = __shfl_sync(FULL, j, r);
            const uint32_t qr = __shfl_sync(FULL, q, r), qer = __shfl_sync(FULL, qe, r);
            const Off o0 = __shfl_sync(FULL, out0, r);
            const double ck = __shfl_sync(FULL, c_keep, r), cd = __shfl_sync(FULL, c_del, r);
            if (e >= total) continue;
            const int32_t c = col[i];
            const int64_t kq = lower_target(ukey, qr, qer, ((uint64_t)jr << 32) | (uint32_t)c);
            unsigned char em = EFF_NOP;
            if (kq < (int64_t)qer && (uint32_t)ukey[kq] == (uint32_t)c) em = eff[kq];
            if (F) atomicAdd(F + c, em == EFF_DEL ? cd : ck);
            if (em == EFF_DEL) continue;
            const Off out = o0 + i - (Off)(del_pre[kq] - del_pre[qr]) + (Off)(ins_pre[kq] - ins_pre[qr]);
            ncol[out] = c;
            if (npcol) npcol[out] = pcol[i];
        }
    }
}

// First position in the old row [a, b) whose target is >= c.
__device__ __forceinline__ Off lower_col(const int32_t *col, Off a, Off b, int32_t c)
{
    while (a < b) {
        const Off mid = a + ((b - a) >> 1);
        if (col[mid] < c) a = mid + 1;
        else b = mid;
    }
    return a;
}

// An inserted link (batch entry k of row j, target c) lands at nrp[j] + (old
// links with target < c) - (deletions before it) + (insertions before it).
// One thread per distinct batch entry.
__global__ void k_merge_ins(const uint64_t *ukey, const uint64_t *nu_dev, const uint8_t *eff, const double *uw,
                            const uint64_t *ins_pre, const uint64_t *del_pre, const uint64_t *tpos, const uint32_t *qs,
                            const Off *rp, const int32_t *col, const int *slot_of, const Off *nrp, int32_t *ncol,
                            double *nw, int32_t *npcol, const double *H, double d, double *F)
{
    const int64_t nu = (int64_t)*nu_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nu;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (eff[k] != EFF_INS) continue;
        const uint32_t j = (uint32_t)(ukey[k] >> 32);
        const int32_t c = (int32_t)(uint32_t)ukey[k];
        const int64_t q = qs[tpos[j]];
        const Off a = rp[j];
        const Off ob = lower_col(col, a, rp[j + 1], c);
        const Off out = nrp[j] + (ob - a) - (Off)(del_pre[k] - del_pre[q]) + (Off)(ins_pre[k] - ins_pre[q]);
        ncol[out] = c;
        if (nw) nw[out] = uw[k];
        if (npcol) {
            const int sl = slot_of[c];
            npcol[out] = sl >= 0 ? (int32_t)(0x80000000u | (unsigned)sl) : c;
        }
        if (F) atomicAdd(F + c, d * H[j] / (double)(nrp[j + 1] - nrp[j]));
    }
}

// Per changed row: W_j of the new row (left to right, as at creation) and the
// change in the number of dangling nodes.
__global__ void k_row_finish(const uint32_t *tlist, const uint64_t *nt_dev, const Off *rp, const Off *nrp,
                             const double *nw, double *nwsum, long long *ddang)
{
    const int64_t nt = (int64_t)*nt_dev;
    long long dd = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nt;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = tlist[k];
        if (nwsum) {
            double ws = 0.0;
            for (Off e = nrp[j]; e < nrp[j + 1]; e++) ws = e == nrp[j] ? nw[e] : ws + nw[e];
            nwsum[j] = ws;
        }
        const bool was = rp[j + 1] == rp[j], now = nrp[j + 1] == nrp[j];
        dd += (long long)now - (long long)was;
    }
    if (dd) atomicAdd((unsigned long long *)ddang, (unsigned long long)dd);
}

__global__ void k_flags(const uint8_t *eff, const uint64_t *nu_dev, uint8_t *ins, uint8_t *del)
{
    const int64_t nu = (int64_t)*nu_dev;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nu;
         k += (int64_t)gridDim.x * blockDim.x) {
        ins[k] = eff[k] == EFF_INS;
        del[k] = eff[k] == EFF_DEL;
    }
}

// F += sign * d H_j P[:, j] for the listed columns (chunks of at most CH
// links), one warp per chunk: lane 0 computes the column's share (one FP64
// division per chunk), and the lanes add it along the chunk's links, four
// links each in flight (their targets loaded before the adds).
__global__ void k_inject_chunks(const uint32_t *ch_row, const uint32_t *ch_idx, const uint64_t *nch_dev,
                                const uint32_t *tlist, const Off *rp, const int32_t *col, const double *w,
                                const double *wsum, const double *H, double sd, double *F)
{
    const int64_t nch = (int64_t)*nch_dev;
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nch; t += nwarp) {
        const uint32_t j = tlist[ch_row[t]];
        const Off a = rp[j], b = rp[j + 1];
        const Off i0 = a + ch_idx[t] * CH;
        if (i0 >= b) continue;
        const Off i1 = (b - i0 > CH) ? i0 + CH : b;
        double unit = 0.0;
        if (lane == 0) {
            const double h = sd * H[j];
            unit = w ? h / wsum[j] : h / (double)(b - a);
        }
        unit = __shfl_sync(FULL, unit, 0);
        for (Off base = i0; base < i1; base += 128) {
            int32_t c[4];
            double v[4];
#pragma unroll
            for (int g = 0; g < 4; g++) {
                const Off e = base + g * 32 + lane;
                c[g] = e < i1 ? col[e] : -1;
                v[g] = (e < i1 && w) ? unit * w[e] : unit;
            }
#pragma unroll
            for (int g = 0; g < 4; g++)
                if (c[g] >= 0) atomicAdd(F + c[g], v[g]);
        }
    }
}

static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

di_status update_edges(di_graph_s *g, di_state_s *st, int64_t m, const int32_t *src, const int32_t *dst,
                       const double *wb, const int8_t *op, cudaStream_t s)
{
    const int64_t n = g->n, nnz = g->nnz;
    if (nnz + m >= (int64_t(1) << 32)) return DI_ERR_INVALID_ARG;
    Temps t(s);
    unsigned *err;
    DI_TRY(t.get(&err, 1));
    DI_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    k_check_batch<<<grid_for(m, 256), 256, 0, s>>>(src, dst, g->weighted ? wb : nullptr, op, m, n, err);
    count_launches(1);
    unsigned herr = 0;
    DI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if (herr) return DI_ERR_INVALID_ARG;
    if (m == 0) return DI_OK;

    // 1. the batch alone, sorted by (source, target), batch order kept for ties
    uint64_t *keys, *keys2, *pos, *total;
    uint32_t *vals, *vals2;
    uint8_t *keep;
    DI_TRY(t.get(&keys, m));
    DI_TRY(t.get(&keys2, m));
    DI_TRY(t.get(&vals, m));
    DI_TRY(t.get(&vals2, m));
    DI_TRY(t.get(&keep, m));
    DI_TRY(t.get(&pos, m));
    DI_TRY(t.get(&total, 1));
    k_batch_keys<<<grid_for(m, 256), 256, 0, s>>>(src, dst, m, keys, vals);
    count_launches(1);
    const int bb = bits_for(n);
    int lo[16], cnt[16], np = 0;
    for (int x = 0; x < bb; x += 8) { lo[np] = x; cnt[np] = bb - x < 8 ? bb - x : 8; np++; }
    for (int x = 0; x < bb; x += 8) { lo[np] = 32 + x; cnt[np] = bb - x < 8 ? bb - x : 8; np++; }
    DI_TRY(radix_sort_pairs(&keys, &vals, &keys2, &vals2, m, lo, cnt, np, s));
    // 2. one entry per distinct link: the last operation on it.  Counts that
    // only the device knows (distinct links nu, changed rows nt, chunks) stay
    // on the device: the arrays are sized by their bounds and the kernels
    // that depend on a count read it there, so the whole update runs without
    // a host round trip until the new link count is read at the end.
    // grids of the count-driven kernels: one full wave (2048 threads per SM)
    const unsigned pgrid = (unsigned)(8 * sm_count(g->device));    // 256-thread blocks
    const unsigned pgrid128 = 2 * pgrid;                           // 128-thread blocks
    uint64_t *nu_dev, *mnew_dev, *nt_dev, *och_dev, *nch_dev;
    DI_TRY(t.get(&nu_dev, 1));
    DI_TRY(t.get(&mnew_dev, 1));
    DI_TRY(t.get(&nt_dev, 1));
    DI_TRY(t.get(&och_dev, 1));
    DI_TRY(t.get(&nch_dev, 1));
    k_run_ends<<<grid_for(m, 256), 256, 0, s>>>(keys, m, keep);
    count_launches(1);
    DI_TRY(scan_exclusive<uint8_t>(keep, pos, m, nu_dev, s));
    uint64_t *ukey;
    int8_t *uop;
    double *uw;
    uint8_t *eff, *touched;
    int *delta;
    DI_TRY(t.get(&ukey, m));
    DI_TRY(t.get(&uop, m));
    DI_TRY(t.get(&uw, m));
    DI_TRY(t.get(&eff, m));
    DI_TRY(t.get(&touched, n));
    DI_TRY(t.get(&delta, n));
    DI_CUDA(cudaMemsetAsync(touched, 0, n, s));
    DI_CUDA(cudaMemsetAsync(delta, 0, sizeof(int) * n, s));
    k_unique<<<grid_for(m, 256), 256, 0, s>>>(keys, vals, keep, pos, m, op, g->weighted ? wb : nullptr, ukey, uop,
                                              uw);
    count_launches(1);
    // 3. classify against the old rows
    const Off *rp = static_cast<const Off *>(g->rp);
    k_classify<<<pgrid, 256, 0, s>>>(ukey, uop, uw, nu_dev, rp, g->col, g->w, eff, delta, touched, g->indeg);
    count_launches(1);
    // 4. new row pointers (at most m links more than before)
    uint32_t *deg;
    uint64_t *ex;
    DI_TRY(t.get(&deg, n));
    DI_TRY(t.get(&ex, n));
    k_new_degree<<<grid_for(n, 256), 256, 0, s>>>(rp, delta, n, deg);
    count_launches(1);
    DI_TRY(scan_exclusive<uint32_t>(deg, ex, n, mnew_dev, s));
    const int64_t cap = nnz + m;
    // the tagged push copy of the links is carried over (same hot pages) for
    // unweighted graphs; a weighted graph rebuilds it with its FP32 weights
    const bool carry_pcol = !g->weighted && g->pcol && g->slot_of && g->pcol_version == g->version;
    int32_t *ncol = nullptr, *npcol = nullptr;
    double *nwv = nullptr, *nwsum = nullptr;
    Off *nrp = nullptr;
    DI_TRY(dalloc_t(&ncol, cap, s));
    if (carry_pcol) DI_TRY(dalloc_t(&npcol, cap, s));
    DI_TRY(dalloc_t(&nrp, n + 1 + RP_PAD, s));
    DI_CUDA(cudaMemsetAsync(nrp + n + 1, 0, sizeof(Off) * RP_PAD, s));
    if (g->weighted) {
        DI_TRY(dalloc_t(&nwv, cap, s));
        DI_TRY(dalloc_t(&nwsum, n, s));
        DI_CUDA(cudaMemcpyAsync(nwsum, g->wsum, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    k_rp_from_scan<<<grid_for(n + 1, 256), 256, 0, s>>>(ex, mnew_dev, n, nrp);
    count_launches(1);
    // 5. unchanged rows move, changed rows are merged
    k_copy_rows<<<grid_for(n, 256), 256, 0, s>>>(rp, nrp, g->col, g->w, g->pcol, touched, n, ncol, nwv, npcol);
    count_launches(1);
    const int64_t tcap = (n < m ? n : m) + 1;   // changed rows: at most one per distinct batch link
    uint64_t *tpos;
    DI_TRY(t.get(&tpos, n));
    DI_TRY(scan_exclusive<uint8_t>(touched, tpos, n, nt_dev, s));
    uint32_t *tlist, *qs, *qe;
    long long *ddang;
    DI_TRY(t.get(&tlist, tcap));
    DI_TRY(t.get(&qs, tcap));
    DI_TRY(t.get(&qe, tcap));
    DI_TRY(t.get(&ddang, 1));
    DI_CUDA(cudaMemsetAsync(ddang, 0, sizeof(long long), s));
    k_list<<<grid_for(n, 256), 256, 0, s>>>(touched, tpos, n, tlist);
    k_row_ranges<<<pgrid, 256, 0, s>>>(ukey, nu_dev, touched, tpos, qs, qe);
    count_launches(2);
    // insertions / deletions before each batch entry (exclusive counts; the
    // flags past the last distinct entry stay 0)
    uint8_t *fins, *fdel;
    uint64_t *ins_pre, *del_pre;
    DI_TRY(t.get(&fins, m + 1));
    DI_TRY(t.get(&fdel, m + 1));
    DI_TRY(t.get(&ins_pre, m + 1));
    DI_TRY(t.get(&del_pre, m + 1));
    DI_CUDA(cudaMemsetAsync(fins, 0, m + 1, s));
    DI_CUDA(cudaMemsetAsync(fdel, 0, m + 1, s));
    k_flags<<<pgrid, 256, 0, s>>>(eff, nu_dev, fins, fdel);
    count_launches(1);
    DI_TRY(scan_exclusive<uint8_t>(fins, ins_pre, m + 1, nullptr, s));
    DI_TRY(scan_exclusive<uint8_t>(fdel, del_pre, m + 1, nullptr, s));
    // chunks of the changed rows, old and new (counts past nt stay 0)
    uint32_t *ocnt, *ncnt;
    uint64_t *ocpos, *ncpos;
    DI_TRY(t.get(&ocnt, tcap));
    DI_TRY(t.get(&ncnt, tcap));
    DI_TRY(t.get(&ocpos, tcap));
    DI_TRY(t.get(&ncpos, tcap));
    DI_CUDA(cudaMemsetAsync(ocnt, 0, sizeof(uint32_t) * tcap, s));
    DI_CUDA(cudaMemsetAsync(ncnt, 0, sizeof(uint32_t) * tcap, s));
    // (the new rows' chunks serve only the separate injection of weighted graphs)
    const bool new_chunks = st && g->weighted;
    // unweighted graphs: rows of at most CH old links are merged 32 to a warp
    // (k_merge_short); weighted graphs chunk every row (the old columns are
    // also withdrawn per chunk)
    const Off short_max = g->weighted ? 0 : CH;
    k_chunk_counts<<<pgrid, 256, 0, s>>>(tlist, nt_dev, rp, ocnt, short_max);
    count_launches(1);
    DI_TRY(scan_exclusive<uint32_t>(ocnt, ocpos, tcap, och_dev, s));
    if (new_chunks) {
        k_chunk_counts<<<pgrid, 256, 0, s>>>(tlist, nt_dev, nrp, ncnt, 0);
        count_launches(1);
        DI_TRY(scan_exclusive<uint32_t>(ncnt, ncpos, tcap, nch_dev, s));
    }
    // a row of d links has ceil(d / CH) chunks (1 if empty)
    const int64_t ocap = nnz / CH + tcap + 1, ncap = cap / CH + tcap + 1;
    uint32_t *och_row, *och_idx, *nch_row = nullptr, *nch_idx = nullptr;
    DI_TRY(t.get(&och_row, ocap));
    DI_TRY(t.get(&och_idx, ocap));
    k_chunk_fill<<<pgrid, 256, 0, s>>>(ocnt, ocpos, nt_dev, och_row, och_idx);
    count_launches(1);
    if (new_chunks) {
        DI_TRY(t.get(&nch_row, ncap));
        DI_TRY(t.get(&nch_idx, ncap));
        k_chunk_fill<<<pgrid, 256, 0, s>>>(ncnt, ncpos, nt_dev, nch_row, nch_idx);
        count_launches(1);
    }
    // 6. F += d (P' - P) H.  Unweighted: during the merge, one add per link of
    // a changed column.  Weighted (W'_j is summed after the merge): the old
    // columns withdrawn and the new ones injected afterwards.
    double *fuse_F = (st && !g->weighted) ? st->F : nullptr;
    const double *fuse_H = st ? st->H : nullptr;
    const double dd = st ? st->d : 0.0;
    double2 *coef = nullptr;
    if (fuse_F) {
        DI_TRY(t.get(&coef, tcap));
        k_row_coef<<<pgrid, 256, 0, s>>>(tlist, nt_dev, rp, nrp, fuse_H, dd, coef);
        count_launches(1);
    }
    if (short_max) {
        k_merge_short<<<pgrid, 256, 0, s>>>(tlist, nt_dev, qs, qe, rp, g->col, g->pcol, nrp, ukey, eff, ins_pre, del_pre,
                                            ncol, npcol, coef, fuse_F);
        count_launches(1);
    }
    k_merge_old<<<pgrid, 256, 0, s>>>(och_row, och_idx, och_dev, tlist, qs, qe, rp, g->col, g->w, g->pcol, nrp, ukey,
                                      eff, uw, ins_pre, del_pre, ncol, nwv, npcol, coef, fuse_F);
    k_merge_ins<<<pgrid, 256, 0, s>>>(ukey, nu_dev, eff, uw, ins_pre, del_pre, tpos, qs, rp, g->col, g->slot_of, nrp,
                                      ncol, nwv, npcol, fuse_H, dd, fuse_F);
    count_launches(2);
    k_row_finish<<<pgrid128, 128, 0, s>>>(tlist, nt_dev, rp, nrp, nwv, nwsum, ddang);
    count_launches(1);
    if (st && g->weighted) {
        k_inject_chunks<<<pgrid, 256, 0, s>>>(och_row, och_idx, och_dev, tlist, rp, g->col, g->w, g->wsum, st->H,
                                             -st->d, st->F);
        k_inject_chunks<<<pgrid, 256, 0, s>>>(nch_row, nch_idx, nch_dev, tlist, nrp, ncol, nwv, nwsum, st->H, st->d,
                                             st->F);
        count_launches(2);
    }
    DI_CUDA(cudaGetLastError());
    long long hd = 0;
    uint64_t mnew = 0;
    DI_CUDA(cudaMemcpyAsync(&hd, ddang, sizeof(hd), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaMemcpyAsync(&mnew, mnew_dev, sizeof(mnew), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));

    // install P'
    dfree(g->rp, s);
    dfree(g->col, s);
    dfree(g->w, s);
    dfree(g->wsum, s);
    dfree(g->cp, s);
    dfree(g->crow, s);
    dfree(g->cw, s);
    g->rp = nrp;
    g->col = ncol;
    g->w = nwv;
    g->wsum = nwsum;
    if (carry_pcol) {
        // the caller bumps the version after a successful update
        dfree(g->pcol, s);
        g->pcol = npcol;
        g->pcol_version = g->version + 1;
    }
    g->cp = nullptr;
    g->crow = nullptr;
    g->cw = nullptr;
    g->nnz = (int64_t)mnew;
    g->n_dangling += hd;
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

}  // namespace di
