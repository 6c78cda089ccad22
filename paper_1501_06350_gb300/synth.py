"""Seeded synthetic inputs for the D-Iteration solver and its oracle.

This module only draws graphs, teleport vectors and edge-change batches. It holds
none of the method's arithmetic (no diffusion matrix, no fluid, no history), so
that the CUDA path and the CPU oracle can both be fed from it without sharing
any code that computes a result.

The paper's measurements use a crawl of the .uk web domain (Section 4: 133 M
pages, 5.5 B links). That dataset is not available here; the generators below
stand in for it with the structure that matters to a push-diffusion solver:

* ``pa_graph``   -- out-degrees drawn from a truncated Zipf law, targets chosen
  by sequential preferential attachment on in-degree, a fraction of dangling
  pages (no out-links).  Small graphs (about 10^4 nodes).
* ``web_graph``  -- pages grouped into hosts of lognormal size, most links
  internal to the host (the locality noted in Section 2.5), power-law
  in-degree through Chung-Lu attractiveness with a Pareto tail, Zipf
  out-degrees with a wide clip (hub pages), dangling pages.

All graphs are returned as a raw out-CSR ``(ptr int64[n+1], idx int32[nnz])``
whose rows are *not* sorted and may contain duplicate links, exactly what a
crawler would hand over; building the canonical diffusion structure out of it
is the solver's job (and the oracle's, independently).
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import math
import os

import numpy as np

#: Base of every seed used by the test-suite and the benchmark.
SEED_BASE = 150106350


@dataclasses.dataclass
class RawGraph:
    n: int
    ptr: np.ndarray          # int64 [n+1]
    idx: np.ndarray          # int32 [nnz]
    w: np.ndarray | None     # float32/float64 [nnz] or None (unweighted)
    meta: dict

    @property
    def nnz(self) -> int:
        return int(self.ptr[-1])


def rng_for(seed_offset: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(seed_offset)))


def zipf_degrees(rng: np.random.Generator, count: int, alpha: float, lo: int, hi: int,
                 target_sum: int | None) -> np.ndarray:
    """Draw ``count`` degrees with P(k) proportional to k^-alpha on [lo, hi].

    When ``target_sum`` is given, every draw is scaled by one common factor with
    stochastic rounding and clipped back to [lo, hi]; the factor is found by
    bisection so that the realised sum lands within 1% of the target.
    """
    if count == 0:
        return np.zeros(0, dtype=np.int64)
    k = np.arange(lo, hi + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-alpha))
    cdf /= cdf[-1]
    raw = k[np.minimum(np.searchsorted(cdf, rng.random(count), side="right"), len(k) - 1)]
    if target_sum is None:
        return raw.astype(np.int64)
    u = rng.random(count)

    def realise(s: float) -> np.ndarray:
        return np.clip(np.floor(raw * s + u), lo, hi).astype(np.int64)

    a, b = 1e-3, 1e4
    for _ in range(80):
        m = math.sqrt(a * b)
        if realise(m).sum() < target_sum:
            a = m
        else:
            b = m
    return realise(b)


def pa_graph(n: int = 10_000, m_target: int = 100_000, dangling_frac: float = 0.10,
             alpha: float = 2.1, deg_hi: int = 1000, seed_offset: int = 1) -> RawGraph:
    """Preferential-attachment graph: Zipf out-degrees, targets by a Polya urn.

    Each link picks its target with probability proportional to (in-degree + 1)
    at the moment it is drawn (links are drawn source by source, in id order).
    Self-links are redrawn; duplicate links are kept (the builders merge them).
    """
    rng = rng_for(seed_offset)
    n_dang = int(round(dangling_frac * n))
    dang = np.zeros(n, dtype=bool)
    dang[rng.permutation(n)[:n_dang]] = True
    deg = np.zeros(n, dtype=np.int64)
    deg[~dang] = zipf_degrees(rng, int((~dang).sum()), alpha, 1, min(deg_hi, max(n - 1, 1)),
                              m_target)
    if n == 1:
        deg[:] = 0
    m = int(deg.sum())
    urn = np.empty(n + m, dtype=np.int64)
    urn[:n] = np.arange(n)
    ulen = n
    idx = np.empty(m, dtype=np.int32)
    draws = rng.random(4 * m + 16)
    di = 0
    e = 0
    for src in range(n):
        for _ in range(int(deg[src])):
            while True:
                if di >= len(draws):
                    draws = rng.random(4 * m + 16)
                    di = 0
                t = int(urn[int(draws[di] * ulen)])
                di += 1
                if t != src:
                    break
            idx[e] = t
            e += 1
            urn[ulen] = t
            ulen += 1
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=ptr[1:])
    return RawGraph(n, ptr, idx, None,
                    dict(kind="pa", n=n, raw_nnz=m, dangling=n_dang, alpha=alpha, deg_hi=deg_hi,
                         seed=SEED_BASE + seed_offset))


def web_graph(n: int = 4_000_000, m_target: int = 40_000_000, dangling_frac: float = 0.15,
              host_mean: float = 100.0, host_sigma: float = 1.0, intra: float = 0.80,
              in_tail: float = 1.1, alpha: float = 2.1, deg_hi: int = 50_000,
              weighted: str | None = None, seed_offset: int = 2) -> RawGraph:
    """Host-structured web-like graph (Chung-Lu targets within and across hosts).

    * host sizes ~ lognormal with the given mean and log-sd, consecutive ids;
    * attractiveness a_v ~ Pareto(x_min=1, tail ``in_tail``), which gives an
      in-degree power law with exponent 1 + in_tail;
    * a fraction ``intra`` of links picks its target inside the source's host
      with probability proportional to a_v, the rest over the whole graph;
    * ``dangling_frac`` of the pages have no out-link; the others draw Zipf
      out-degrees on [1, deg_hi] rescaled to hit ``m_target`` links;
    * ``weighted``: None, "lognormal32" (lognormal(0,1) in float32) or
      "lognormal64".
    """
    rng = rng_for(seed_offset)
    mu = math.log(host_mean) - 0.5 * host_sigma ** 2
    sizes = []
    tot = 0
    while tot < n:
        s = np.maximum(1, np.round(rng.lognormal(mu, host_sigma, size=max(16, n // 50))))
        s = s.astype(np.int64)
        sizes.append(s)
        tot += int(s.sum())
    sizes = np.concatenate(sizes)
    csz = np.cumsum(sizes)
    nh = int(np.searchsorted(csz, n, side="left")) + 1
    sizes = sizes[:nh].copy()
    sizes[-1] -= int(csz[nh - 1] - n)
    hstart = np.zeros(nh + 1, dtype=np.int64)
    np.cumsum(sizes, out=hstart[1:])
    host_of = np.repeat(np.arange(nh, dtype=np.int64), sizes)

    attract = (1.0 - rng.random(n)) ** (-1.0 / in_tail)
    cum = np.zeros(n + 1, dtype=np.float64)
    np.cumsum(attract, out=cum[1:])

    n_dang = int(round(dangling_frac * n))
    dang = np.zeros(n, dtype=bool)
    dang[rng.permutation(n)[:n_dang]] = True
    deg = np.zeros(n, dtype=np.int64)
    # rows must be drawable without repeats: clip at half the page count
    deg[~dang] = zipf_degrees(rng, int((~dang).sum()), alpha, 1, min(deg_hi, max((n - 1) // 2, 1)),
                              m_target)
    if n == 1:
        deg[:] = 0
    m = int(deg.sum())
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    h = host_of[src]
    lo = cum[hstart[h]]
    hi = cum[hstart[h + 1]]
    single = sizes[h] <= 1
    is_intra = (rng.random(m) < intra) & ~single
    u = rng.random(m)
    val = np.where(is_intra, lo + u * (hi - lo), u * cum[n])
    tgt = np.searchsorted(cum, val, side="right") - 1
    tgt = np.clip(tgt, 0, n - 1)
    # A page links to distinct pages: redraw self-links and repeated links of a
    # row (inside the host for the first rounds, then across the graph, and
    # finally uniformly, which always terminates).
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=rowptr[1:])
    sub = np.arange(m, dtype=np.int64)          # links whose rows are re-checked
    for it in range(40):
        key = src[sub] * n + tgt[sub]
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(len(sub), dtype=bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        bad = sub[np.nonzero(dup | (tgt[sub] == src[sub]))[0]]
        if len(bad) == 0:
            break
        uu = rng.random(len(bad))
        if it < 4:
            vv = np.where(is_intra[bad], lo[bad] + uu * (hi[bad] - lo[bad]), uu * cum[n])
            tgt[bad] = np.clip(np.searchsorted(cum, vv, side="right") - 1, 0, n - 1)
        elif it < 12:
            tgt[bad] = np.clip(np.searchsorted(cum, uu * cum[n], side="right") - 1, 0, n - 1)
        else:
            tgt[bad] = rng.integers(0, n, size=len(bad))
        rows = np.unique(src[bad])
        lens = rowptr[rows + 1] - rowptr[rows]
        starts = np.repeat(rowptr[rows] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
        sub = starts + np.arange(int(lens.sum()), dtype=np.int64)
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=ptr[1:])
    w = None
    if weighted == "lognormal32":
        w = rng.lognormal(0.0, 1.0, size=m).astype(np.float32)
    elif weighted == "lognormal64":
        w = rng.lognormal(0.0, 1.0, size=m).astype(np.float64)
    elif weighted is not None:
        raise ValueError(weighted)
    return RawGraph(n, ptr, tgt.astype(np.int32), w,
                    dict(kind="web", n=n, raw_nnz=m, hosts=nh, dangling=n_dang, intra=intra,
                         in_tail=in_tail, alpha=alpha, deg_hi=deg_hi, weighted=weighted,
                         seed=SEED_BASE + seed_offset))


def small_graph(n: int, m: int, seed_offset: int, dangling_frac: float = 0.1,
                self_loops: bool = False, weighted: bool = False) -> RawGraph:
    """Uniform random multigraph for unit tests (optional self-links and weights)."""
    rng = rng_for(1000 + seed_offset)
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    if n > 1 and dangling_frac > 0:
        dang = rng.random(n) < dangling_frac
        keep = ~dang[src]
        src, dst = src[keep], dst[keep]
    if not self_loops and n > 1:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, src + 1, 1)
    ptr = np.cumsum(ptr)
    w = rng.lognormal(0.0, 1.0, size=len(dst)) if weighted else None
    return RawGraph(n, ptr, dst.astype(np.int32), w, dict(kind="small", n=n))


def with_in_hubs(g: RawGraph, n_hubs: int, frac: float, seed_offset: int) -> RawGraph:
    """The same links plus ``n_hubs`` heavy in-hubs: each page that already has
    out-links gets, with probability ``frac``, one extra link to a hub chosen
    uniformly (hubs are the pages 0 .. n_hubs-1).  Rows keep input order with
    the extra link appended, so duplicates and self-links may appear."""
    rng = rng_for(8000 + seed_offset)
    deg = np.diff(g.ptr)
    extra = (rng.random(g.n) < frac) & (deg > 0)
    hub = rng.integers(0, n_hubs, size=g.n)
    ptr = np.zeros(g.n + 1, dtype=np.int64)
    ptr[1:] = np.cumsum(deg + extra)
    idx = np.empty(int(ptr[-1]), dtype=np.int32)
    w = None if g.w is None else np.empty(int(ptr[-1]), dtype=g.w.dtype)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    pos = ptr[src] + (np.arange(g.nnz, dtype=np.int64) - g.ptr[src])
    idx[pos] = g.idx
    rows = np.nonzero(extra)[0]
    idx[ptr[rows + 1] - 1] = hub[rows]
    if w is not None:
        w[pos] = g.w
        w[ptr[rows + 1] - 1] = rng.lognormal(0.0, 1.0, size=len(rows)).astype(g.w.dtype)
    return RawGraph(g.n, ptr, idx, w, dict(g.meta, in_hubs=n_hubs, hub_frac=frac))


def edges_from_csr(g: RawGraph) -> tuple[np.ndarray, np.ndarray]:
    """Expand a CSR into (src, dst) arrays in input order."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.ptr))
    return src, g.idx.astype(np.int64)


def to_csc(g: RawGraph) -> RawGraph:
    """Re-express the same link multiset as an in-edge CSR (ptr over targets).

    Within each target row the sources keep input order; this is a pure
    re-indexing of the input and is used to feed the CSC entry of the builders.
    """
    src, dst = edges_from_csr(g)
    order = np.argsort(dst, kind="stable")
    ptr = np.zeros(g.n + 1, dtype=np.int64)
    np.add.at(ptr, dst + 1, 1)
    ptr = np.cumsum(ptr)
    w = None if g.w is None else g.w[order]
    return RawGraph(g.n, ptr, src[order].astype(np.int32), w, dict(g.meta, layout="csc"))


def uniform_z(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n, dtype=np.float64)


def random_z(n: int, seed_offset: int, signed: bool = False) -> np.ndarray:
    rng = rng_for(2000 + seed_offset)
    z = rng.random(n)
    if signed:
        z = z - 0.3
    return z / np.abs(z).sum()


def seed_set_z(n: int, n_seeds: int, seed_offset: int) -> np.ndarray:
    """Personalised teleport vector: uniform over ``n_seeds`` random seed pages."""
    rng = rng_for(3000 + seed_offset)
    z = np.zeros(n, dtype=np.float64)
    z[rng.choice(n, size=min(n_seeds, n), replace=False)] = 1.0 / min(n_seeds, n)
    return z


def seed_set_batch(n: int, B: int, seed_offset: int, max_seeds: int = 1000) -> np.ndarray:
    """B personalised teleport vectors as an n x B node-major matrix: column c is
    uniform over a random set of 1 .. max_seeds seed pages."""
    rng = rng_for(3500 + seed_offset)
    Z = np.zeros((n, B), dtype=np.float64)
    for c in range(B):
        k = int(rng.integers(1, max_seeds + 1))
        k = min(k, n)
        Z[rng.choice(n, size=k, replace=False), c] = 1.0 / k
    return Z


def small_web_graphs(count: int, n_lo: int, n_hi: int, avg_deg: float, seed_offset: int) -> list:
    """``count`` independent host-structured graphs with sizes uniform in
    [n_lo, n_hi] and about ``avg_deg`` links per page."""
    rng = rng_for(5000 + seed_offset)
    out = []
    for k in range(count):
        nk = int(rng.integers(n_lo, n_hi + 1))
        out.append(web_graph(n=nk, m_target=int(avg_deg * nk), seed_offset=6000 + seed_offset * 1000 + k,
                             deg_hi=min(50_000, nk - 1)))
    return out


def union(graphs: list) -> tuple:
    """Block-diagonal union of independent graphs (node ids offset graph by
    graph) and the node offsets; the teleport vector that is uniform on each
    component (1/n_k on graph k)."""
    offs = np.zeros(len(graphs) + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        offs[k + 1] = offs[k] + g.n
    n = int(offs[-1])
    ptr = np.zeros(n + 1, dtype=np.int64)
    idx_parts = []
    for k, g in enumerate(graphs):
        ptr[offs[k] + 1:offs[k + 1] + 1] = np.diff(g.ptr)
        idx_parts.append(g.idx.astype(np.int64) + offs[k])
    ptr = np.cumsum(ptr)
    idx = np.concatenate(idx_parts).astype(np.int32) if idx_parts else np.zeros(0, np.int32)
    Z = np.concatenate([np.full(g.n, 1.0 / g.n) for g in graphs])
    return RawGraph(n, ptr, idx, None, {"components": len(graphs)}), offs, Z


def edge_batch(g_canon_ptr: np.ndarray, g_canon_idx: np.ndarray, n: int, frac: float,
               seed_offset: int, insert_share: float = 0.5) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Random link changes: ``frac`` of the current links, half deletions of existing
    links and half insertions of new (src, dst) pairs, src != dst.

    Returns (src int32, dst int32, op int8) with op = +1 insert, -1 delete, in
    random order.  Insertions may hit links that already exist and deletions
    are drawn from existing links, so both the no-op and the effective cases
    occur.
    """
    rng = rng_for(4000 + seed_offset)
    nnz = int(g_canon_ptr[-1])
    m = max(1, int(round(frac * max(nnz, 1))))
    n_ins = int(round(insert_share * m))
    n_del = m - n_ins if nnz > 0 else 0
    src_e = np.repeat(np.arange(n, dtype=np.int64), np.diff(g_canon_ptr))
    pick = rng.integers(0, max(nnz, 1), size=n_del)
    ds, dd = src_e[pick], g_canon_idx[pick].astype(np.int64)
    is_ = rng.integers(0, n, size=n_ins)
    id_ = rng.integers(0, n, size=n_ins)
    if n > 1:
        same = is_ == id_
        id_[same] = (id_[same] + 1) % n
    src = np.concatenate([ds, is_])
    dst = np.concatenate([dd, id_])
    op = np.concatenate([-np.ones(n_del, np.int8), np.ones(n_ins, np.int8)])
    perm = rng.permutation(len(src))
    return src[perm].astype(np.int32), dst[perm].astype(np.int32), op[perm]


def cached(fn, **kw) -> RawGraph:
    """Memoise a generator on disk (``$DI_SYNTH_CACHE``, default /tmp/di_synth_cache),
    keyed by the generator name and its arguments."""
    root = os.environ.get("DI_SYNTH_CACHE", "/tmp/di_synth_cache")
    key = hashlib.sha1(json.dumps([fn.__name__, sorted(kw.items())], default=str).encode()).hexdigest()[:16]
    path = os.path.join(root, f"{fn.__name__}_{key}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        meta = json.loads(str(z["meta"]))
        return RawGraph(int(z["n"]), z["ptr"], z["idx"], z["w"] if "w" in z.files else None, meta)
    g = fn(**kw)
    os.makedirs(root, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    arrs = dict(n=np.int64(g.n), ptr=g.ptr, idx=g.idx, meta=np.array(json.dumps(g.meta, default=str)))
    if g.w is not None:
        arrs["w"] = g.w
    np.savez(tmp, **arrs)
    os.replace(tmp, path)
    return g


def exact_batch(ptr: np.ndarray, idx: np.ndarray, n: int, frac: float, seed_offset: int):
    """Link changes whose exact inverse is known: ``frac``/2 of the existing links
    are deleted (distinct) and as many new distinct links (absent, no
    self-link) are inserted.  Returns (src, dst, op) of the forward batch;
    the inverse batch is the same pairs with op negated."""
    rng = rng_for(5000 + seed_offset)
    nnz = int(ptr[-1])
    k = max(1, int(round(frac * nnz / 2)))
    src_e = np.repeat(np.arange(n, dtype=np.int64), np.diff(ptr))
    keys = src_e * n + idx.astype(np.int64)          # ascending for a canonical CSR
    dpos = rng.choice(nnz, size=min(k, nnz), replace=False)
    ds, dd = src_e[dpos], idx[dpos].astype(np.int64)
    ins_s = np.zeros(0, np.int64)
    ins_d = np.zeros(0, np.int64)
    seen = set()
    while len(ins_s) < k:
        cs = rng.integers(0, n, size=2 * k)
        cd = rng.integers(0, n, size=2 * k)
        ck = cs * n + cd
        pos = np.searchsorted(keys, ck)
        exists = (pos < nnz) & (keys[np.minimum(pos, nnz - 1)] == ck) if nnz else np.zeros(len(ck), bool)
        ok = (~exists) & (cs != cd)
        _, first = np.unique(ck, return_index=True)
        uniq = np.zeros(len(ck), bool)
        uniq[first] = True
        ok &= uniq
        cand = [(a, b) for a, b in zip(cs[ok], cd[ok]) if (a * n + b) not in seen]
        for a, b in cand:
            seen.add(a * n + b)
        if cand:
            arr = np.array(cand, dtype=np.int64)
            ins_s = np.concatenate([ins_s, arr[:, 0]])
            ins_d = np.concatenate([ins_d, arr[:, 1]])
    ins_s, ins_d = ins_s[:k], ins_d[:k]
    src = np.concatenate([ds, ins_s]).astype(np.int32)
    dst = np.concatenate([dd, ins_d]).astype(np.int32)
    op = np.concatenate([-np.ones(len(ds), np.int8), np.ones(k, np.int8)])
    perm = rng.permutation(len(src))
    return src[perm], dst[perm], op[perm]


def web_graph_device(n: int, m_target: int, dangling_frac: float = 0.15, host_mean: float = 100.0,
                     host_sigma: float = 1.0, intra: float = 0.80, alpha: float = 2.1, deg_hi: int = 50_000,
                     in_tail: float = 1.1, seed_offset: int = 50, device: str = "cuda"):
    """Host-structured web-like graph drawn on the GPU with torch, for sizes whose
    NumPy generation would take many minutes (tens of millions of pages).

    Same recipe as ``web_graph`` (hosts of lognormal size with consecutive ids,
    ``intra`` of the links inside the host, ``dangling_frac`` pages without
    links, Zipf(alpha) out-degrees on [1, deg_hi] scaled to ``m_target``), with
    two simplifications: a link's target is drawn by inverse-CDF sampling of a
    power law over the page ranks of its host (intra-host) or of the whole
    graph (the rest), P(rank k) ~ k^(-1/in_tail) (an in-degree tail of exponent
    1 + in_tail), so low ids inside a host and overall are the popular pages;
    and repeated links are left to the builders' merge.
    Returns (ptr int64 [n+1], idx int32 [links]) as device tensors."""
    import torch
    gen = torch.Generator(device=device).manual_seed(150106350 + seed_offset)
    # hosts: consecutive id ranges of lognormal size
    mu = np.log(host_mean) - 0.5 * host_sigma ** 2
    est = int(1.3 * n / host_mean) + 16
    sizes = torch.exp(mu + host_sigma * torch.randn(est, generator=gen, device=device, dtype=torch.float64))
    sizes = torch.clamp(torch.round(sizes), min=1).to(torch.int64)
    ends = torch.cumsum(sizes, 0)
    nh = int(torch.searchsorted(ends, torch.tensor([n], device=device)).item()) + 1
    ends = ends[:nh].clone()
    ends[-1] = n
    starts = torch.cat([torch.zeros(1, dtype=torch.int64, device=device), ends[:-1]])
    # out-degrees: Zipf(alpha) on [1, deg_hi] by inverse CDF, dangling pages 0, scaled to m_target
    u = torch.rand(n, generator=gen, device=device, dtype=torch.float64)
    a1 = 1.0 - alpha
    lo, hi = 1.0, float(deg_hi) + 1.0
    deg = torch.floor((lo ** a1 + u * (hi ** a1 - lo ** a1)) ** (1.0 / a1))
    dang = torch.rand(n, generator=gen, device=device) < dangling_frac
    deg = torch.where(dang, torch.zeros_like(deg), deg)
    deg = deg * (m_target / float(deg.sum().item()))
    deg = torch.floor(deg + torch.rand(n, generator=gen, device=device, dtype=torch.float64))
    deg = torch.where(dang, torch.zeros_like(deg), torch.clamp(deg, min=1, max=deg_hi)).to(torch.int64)
    ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    ptr[1:] = torch.cumsum(deg, 0)
    m = int(ptr[-1].item())
    src_all = torch.repeat_interleave(torch.arange(n, device=device), deg, output_size=m)
    hsize = ends - starts
    one_s = 1.0 - 1.0 / in_tail
    big = torch.pow(torch.tensor(n + 1.0, device=device, dtype=torch.float64), one_s) - 1.0
    out = torch.empty(m, dtype=torch.int32, device=device)
    chunk = 1 << 27                              # links per chunk: bounds the temporaries
    for c0 in range(0, m, chunk):
        src = src_all[c0:c0 + chunk]
        k = src.numel()
        host = torch.searchsorted(ends, src, right=True)
        h0, hs = starts[host], hsize[host]
        del host
        # rank k (1-based) with P(k) ~ k^-s, s = 1/in_tail, by the inverse CDF of the
        # continuous law on [1, N + 1): k = (1 + u ((N+1)^(1-s) - 1))^(1/(1-s))
        v = torch.rand(k, generator=gen, device=device, dtype=torch.float64)
        inside = torch.rand(k, generator=gen, device=device) < intra
        span = torch.pow(hs.to(torch.float64) + 1.0, one_s) - 1.0
        r_in = torch.pow(1.0 + v * span, 1.0 / one_s).to(torch.int64) - 1
        del span
        tgt = h0 + torch.minimum(torch.clamp(r_in, min=0), hs - 1)
        del r_in
        r_out = torch.clamp(torch.pow(1.0 + v * big, 1.0 / one_s).to(torch.int64) - 1, min=0, max=n - 1)
        tgt = torch.where(inside, tgt, r_out)
        del r_out, v
        # no self-links: move to the next page of the host (or of the graph)
        same = tgt == src
        tgt = torch.where(same & inside, h0 + torch.remainder(tgt - h0 + 1, hs), tgt)
        tgt = torch.where(same & ~inside, torch.remainder(tgt + 1, n), tgt)
        out[c0:c0 + k] = tgt.to(torch.int32)
        del same, tgt, h0, hs, inside, src
    del src_all
    return ptr, out


def edge_batch_device(ptr, idx, n: int, frac: float, seed_offset: int):
    """``frac`` of the links changed, half deletions of existing links and half
    insertions of random new pairs (no self-link), drawn on the GPU; returns
    (src, dst, op) device tensors in random order."""
    import torch
    gen = torch.Generator(device=idx.device).manual_seed(4500 + seed_offset)
    m = int(ptr[-1].item())
    k = max(1, int(round(frac * m)))
    nd = k // 2
    ni = k - nd
    pick = torch.randint(0, m, (nd,), generator=gen, device=idx.device)
    ds = torch.searchsorted(ptr, pick, right=True) - 1
    dd = idx[pick].to(torch.int64)
    is_ = torch.randint(0, n, (ni,), generator=gen, device=idx.device)
    id_ = torch.randint(0, n, (ni,), generator=gen, device=idx.device)
    id_ = torch.where(is_ == id_, torch.remainder(id_ + 1, n), id_)
    src = torch.cat([ds, is_])
    dst = torch.cat([dd, id_])
    op = torch.cat([-torch.ones(nd, dtype=torch.int8, device=idx.device),
                    torch.ones(ni, dtype=torch.int8, device=idx.device)])
    perm = torch.randperm(k, generator=gen, device=idx.device)
    return src[perm].to(torch.int32), dst[perm].to(torch.int32), op[perm]
