#!/usr/bin/env python
"""Benchmark of the D-Iteration hot path on one GB300 (or N replicas under torchrun).

Workload: the host-structured web-like graph (4,000,000 pages, 40,000,000 links,
hosts of lognormal size with mean 100, 80% intra-host links, Pareto(1.1)
attractiveness, 15% dangling pages, Zipf(2.1) out-degrees clipped to
[1, 50000]), d = 0.85, uniform Z, tol = 1e-9 on |F|_1 / (1 - d).

One step = the whole hot path on that graph: a from-scratch solve to tol
(init, frontier sweeps, stop test), then a 1% link-change batch (half
deletions, half insertions) applied by correction-fluid injection and
re-converged, then the inverse batch applied and re-converged, which leaves
the graph as it started.  The metric is edge pushes per second over the step
(links pushed by all three solves / step time); the from-scratch time to tol
is reported beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(sequential FP64 DI-argmax) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1501_06350_gb300 import synth  # noqa: E402

D = 0.85
TOL = 1e-9
BATCH_FRAC = 0.01
METRIC = "edge-pushes/s"
WORKLOAD = ("web-like graph: 4,000,000 pages, 40,000,000 links, hosts lognormal(mean 100), "
            "80% intra-host links, Pareto(1.1) attractiveness, 15% dangling, Zipf(2.1) out-degree "
            "in [1,50000]; d=0.85, uniform Z, solve to |F|_1/(1-d) <= 1e-9 (fluid arithmetic: config "
            "'precision'), then a 1% link-update round trip (inject + re-converge, twice)")
GEN_KW = dict(n=4_000_000, m_target=40_000_000)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_workload(small: bool):
    kw = dict(n=200_000, m_target=2_000_000) if small else GEN_KW
    t = time.time()
    g = synth.cached(synth.web_graph, **kw)
    log(f"[bench] workload n={g.n} raw links={g.nnz} ready in {time.time() - t:.1f}s")
    return g


# ---------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"di_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first
        # sample so that the samples cover the timed region
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ reference arm
def run_reference(args, g):
    import oracle
    oracle.build()
    cp, ci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
    rounds = 3  # one round = n elementary diffusions (Section 4.2)
    cap = rounds * g.n
    times, pushes = [], []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        _, _, info, _ = oracle.di_solve(g.n, cp, ci, None, D, None, tol=TOL, max_diffusions=cap)
        dt = time.perf_counter() - t
        if k >= args.warmup:
            times.append(dt)
            pushes.append(info["edge_pushes"])
    val = sum(pushes) / sum(times)
    sample = (f"sequential FP64 DI-argmax oracle, first {rounds} rounds ({cap} diffusions) of the "
              f"from-scratch solve per step, 1 thread")
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config_dict(g, {"nnz": int(cp[-1]), "n_dangling": int((np.diff(cp) == 0).sum())}),
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def atomic_ceiling(torch):
    """Throughput of FP64 atomic additions at random slots of an L2-resident
    32 MB vector (the push adds into its 32 MB fluid at random pages), measured
    live by the library's probe (di_probe_atomic_adds): the ceiling of an
    atomic-bound scatter on this GPU."""
    from paper_1501_06350_gb300 import _lib
    g = ctypes.c_double(0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(_lib.lib().di_probe_atomic_adds(torch.cuda.current_device(), ctypes.byref(g), stream),
               "di_probe_atomic_adds")
    return g.value


def update_bytes(cp, n, src, op):
    """Algorithmic bytes of one link batch applied by Section 3.5 (Theorem
    update): the batch read (source, target, op: 9 B per change), the CSR
    rewritten (old link targets and row pointers read, new ones written: 4 B
    per link and per row each way), and for every changed column j the
    correction fluid d (P' - P) H: H_j read (8 B) and, per link of the old and
    of the new row, the 4 B target read and the 8 B add into F."""
    deg_old = np.diff(cp).astype(np.int64)
    delta = np.zeros(n, dtype=np.int64)
    np.add.at(delta, src.astype(np.int64), op.astype(np.int64))
    touched = np.unique(src.astype(np.int64))
    deg_new = deg_old + delta
    nnz_old, nnz_new = int(deg_old.sum()), int(deg_new.sum())
    csr = 4 * nnz_old + 4 * (n + 1) + 4 * nnz_new + 4 * (n + 1)
    inject = 8 * len(touched) + 12 * int(deg_old[touched].sum()) + 12 * int(deg_new[touched].sum())
    return {"batch": 9 * len(src), "csr": csr, "inject": inject, "total": 9 * len(src) + csr + inject,
            "changed_columns": int(len(touched)),
            "injected_links": int(deg_old[touched].sum() + deg_new[touched].sum())}


def update_roofline(cp, n, src, op, ms, peak):
    """The update step against the HBM roofline: the algorithmic bytes of
    update_bytes (for an exact batch of distinct insertions and deletions the
    inverse batch moves the same bytes) over the CUDA-event time of one
    di_update_edges call (median over the timed steps and both directions)."""
    b = update_bytes(cp, n, src, op)
    achieved = b["total"] / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "bytes": b, "ms": ms, "traffic": None}


def config_dict(g, gi, precision="f64"):
    c = {"workload": WORKLOAD, "n": g.n, "links": gi["nnz"] if gi else None, "d": D, "tol": TOL,
         "precision": precision,
         "z": "uniform", "batch_frac": BATCH_FRAC, "parallelism": "replicas (one independent solve per GPU)",
         "l2": "inputs larger than L2 (160 MB of link targets); L2 flushed (256 MB write) between steps"}
    if gi:
        c["dangling"] = gi["n_dangling"]
    return c


def cpu_baseline(g, cp, ci):
    import oracle
    oracle.build()
    t = time.perf_counter()
    H, F, info, _ = oracle.di_solve(g.n, cp, ci, None, D, None, tol=TOL)
    dt = time.perf_counter() - t
    return {"value": info["edge_pushes"] / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": ("one full from-scratch solve of the same graph to |F|_1/(1-d) <= 1e-9 by the "
                       "sequential FP64 DI-argmax oracle (no update round trip)"),
            "time_to_tol_s": dt, "edge_pushes": info["edge_pushes"], "diffusions": info["diffusions"]}, (H, F)


def adjoint_leg(torch, di, reps=4):
    """Backward pass on the weighted 2M-page / 20M-link web graph (lognormal(0,1)
    FP32 weights): forward solve to tol, then lambda with |lambda - H|_inf <= tol,
    dL/dZ and dL/dw for L = g . x, g ~ N(0,1).  Device times (CUDA events)."""
    ga = synth.cached(synth.web_graph, n=2_000_000, m_target=20_000_000, weighted="lognormal32",
                      seed_offset=4)
    G = di.Graph(ga.n, ga.ptr, ga.idx, ga.w)
    gv = torch.from_numpy(synth.rng_for(41).standard_normal(ga.n)).cuda()
    x, xi, st = di.solve(G, D, tol=TOL)
    fwd, bwd, info = [], [], None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for k in range(reps + 1):
        ev[0].record()
        x, xi = st.solve(D, tol=TOL)
        ev[1].record()
        lam, gz, gw, info = di.adjoint(G, D, gv, x, tol=TOL)
        ev[2].record()
        torch.cuda.synchronize()
        if k:
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[1].elapsed_time(ev[2]))
    gi = G.info()
    out = {"workload": "web-like graph, 2,000,000 pages, 20,000,000 links, lognormal(0,1) FP32 weights, "
                       "d=0.85; L = g.x with g ~ N(0,1)",
           "links": gi["nnz"], "forward_ms": statistics.median(fwd), "backward_ms": statistics.median(bwd),
           "backward_includes": "adjoint diffusion to |lambda-H|_inf <= 1e-9, dL/dZ, dL/dw (all links)",
           "adjoint_sweeps": info["sweeps"], "adjoint_edge_pushes": info["edge_pushes"],
           "adjoint_edge_pushes_per_s": info["edge_pushes"] / (info["time_ms"] / 1e3),
           "adjoint_solve_ms": info["time_ms"], "bound_inf": info["bound"]}
    st.close()
    G.close()
    return out


def update50m_leg(torch, di, reps=2):
    """The dynamic update at scale: a host-structured graph of 50,000,000 pages
    and about 600,000,000 links drawn on the GPU (synth.web_graph_device, 1.05e9
    draws merged), d = 0.85, uniform Z, tol 1e-9.  From-scratch solves in both
    forms, then a 1% link batch (half deletions of existing links, half new
    random links) injected (Section 3.5) and re-converged in the FP32 form, against
    a from-scratch FP32 solve of the new graph.  Device times (CUDA events)."""
    t0 = time.time()
    ptr, idx = synth.web_graph_device(50_000_000, 1_050_000_000)
    G = di.Graph(50_000_000, ptr, idx)
    del ptr, idx
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    gi = G.info()
    st = di.State(G)
    out = {"workload": "host-structured web graph drawn on the GPU: 50,000,000 pages, %d links (int32 CSR), "
                       "d=0.85, uniform Z, tol 1e-9; 1%% link changes (half deletions, half insertions)" % gi["nnz"],
           "pages": gi["n"], "links": gi["nnz"], "dangling": gi["n_dangling"], "generate_and_build_s": setup_s}
    for name, kw in (("f64", {}), ("f32_refined", {"precision": 1})):
        ts, info = [], None
        for _ in range(reps):
            _, info = st.solve(D, tol=TOL, **kw)
            ts.append(info["time_ms"])
        out["from_scratch_" + name] = {"time_to_tol_ms": min(ts), "sweeps": info["sweeps"],
                                       "edge_pushes": info["edge_pushes"],
                                       "edge_pushes_per_s": info["edge_pushes"] / (min(ts) / 1e3)}
    cp, ci, _ = G.export_csr(device=True, weights=False)
    src, dst, op = synth.edge_batch_device(cp, ci, gi["n"], 0.01, 5)
    cp_h = cp.cpu().numpy()
    del cp, ci
    st.solve(D, tol=TOL, precision=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the update alone as an NVTX range, so that a profiler can list its launches
    torch.cuda.nvtx.range_push("update")
    e0.record()
    st.update_edges(src, dst, op)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    _, ri = st.resume(tol=TOL, precision=1)
    st2 = di.State(G)
    _, si = st2.solve(D, tol=TOL, precision=1)
    out["update"] = {"batch_links": int(src.numel()), "inject_and_patch_ms": e0.elapsed_time(e1),
                     "reconverge_ms": ri["time_ms"], "reconverge_pushes": ri["edge_pushes"],
                     "from_scratch_new_graph_ms": si["time_to_tol_ms"] if "time_to_tol_ms" in si else si["time_ms"],
                     "from_scratch_new_graph_pushes": si["edge_pushes"],
                     "update_vs_scratch_time": (e0.elapsed_time(e1) + ri["time_ms"]) / si["time_ms"]}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(pk_path)).get("hbm_gbs", 6800.0) if os.path.exists(pk_path) else 6800.0
    out["update"]["roofline"] = update_roofline(cp_h, gi["n"], src.cpu().numpy(), op.cpu().numpy(),
                                                e0.elapsed_time(e1), peak)
    st.close()
    st2.close()
    G.close()
    return out


def batch_leg(torch, di, peak, reps=3, union=True):
    """Batched personalised solves and uneven independent graphs.

    (a) 64 teleport vectors, each uniform over 1 to 1000 random seed pages, on
    the host-structured 1M-page / 10M-link graph, in one batched solve
    (di_solve_batch: FP32 fluid, FP64 refinement, tol 1e-9 per column), against
    64 single FP64 solves of the same vectors.  (b) 256 independent graphs of
    1,000 to 50,000 pages (8 links per page on average) as one block-diagonal
    union in one FP32 solve, against 256 separate solves.  Device times (the
    library's CUDA events)."""
    from paper_1501_06350_gb300 import _lib
    g = synth.cached(synth.web_graph, n=1_000_000, m_target=10_000_000, seed_offset=3)
    G = di.Graph(g.n, g.ptr, g.idx)
    Z = torch.from_numpy(synth.seed_set_batch(g.n, 64, 8)).cuda()
    ts, info = [], None
    for k in range(reps + 1):
        H, res, info = di.solve_batch(G, Z, D, tol=TOL)
        if k:
            ts.append(info["time_ms"])
    _, _, prof = di.solve_batch(G, Z, D, tol=TOL, profile=1)
    links_per_launch = prof["push_edges"] / max(prof["push_launches"], 1)
    push_s = prof["push_ms"] / 1e3 / max(prof["push_launches"], 1)
    # per pushed link: 4 B target + 64 x 4 B fluid added at the target
    achieved = 260.0 * links_per_launch / push_s / 1e9
    st = di.State(G)
    single = []
    for c in range(64):
        _, i1 = st.solve(D, Z=Z[:, c].contiguous(), tol=TOL)
        single.append(i1["time_ms"])
    st.close()
    G.close()
    batch_ms = statistics.median(ts)
    out = {"workload": "host-structured web graph, 1,000,000 pages, 10,000,000 links; 64 teleport vectors, "
                       "each uniform over 1-1000 random seed pages; d=0.85, tol 1e-9 per column",
           "columns": 64, "time_to_tol_ms": batch_ms, "sweeps": info["sweeps"], "refinements": info["refinements"],
           "link_pushes": info["edge_pushes"], "column_link_pushes_per_s": 64 * info["edge_pushes"] / (batch_ms / 1e3),
           "worst_resid_l1": info["resid_l1"], "single_f64_total_ms": sum(single),
           "speedup_vs_single_f64": sum(single) / batch_ms,
           "k_bpush": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "traffic": traffic_for("bpush_web1m_traffic.json"),
                       "bytes_per_link": 260.0, "links_per_launch": links_per_launch,
                       "push_ms_avg": 1e3 * push_s, "launches": prof["push_launches"]}}
    if not union:
        return out
    # (b) uneven graphs
    gs = [synth.cached(synth.web_graph, n=nk, m_target=8 * nk, seed_offset=7000 + k, deg_hi=min(50_000, nk - 1))
          for k, nk in enumerate(synth.rng_for(77).integers(1_000, 50_001, size=256).tolist())]
    u, offs, Zu = synth.union(gs)
    Gu = di.Graph(u.n, u.ptr, u.idx)
    su = di.State(Gu)
    tu, iu = [], None
    for k in range(reps + 1):
        _, iu = su.solve(D, Z=Zu, tol=TOL, precision=_lib.DI_PREC_F32)
        if k:
            tu.append(iu["time_ms"])
    su.close()
    Gu.close()
    sep = 0.0
    for gk in gs:
        Gk = di.Graph(gk.n, gk.ptr, gk.idx)
        _, ik, sk = di.solve(Gk, D, tol=TOL)
        sep += ik["time_ms"]
        sk.close()
        Gk.close()
    um = statistics.median(tu)
    out["union"] = {"graphs": len(gs), "pages": u.n, "links": int(u.ptr[-1]), "time_to_tol_ms": um,
                    "precision": "f32 fluid / f64 refinement", "sweeps": iu["sweeps"],
                    "separate_f64_total_ms": sep, "speedup_vs_separate": sep / um,
                    "stop": "|F|_1/(1-d) <= 1e-9 over the union, which bounds every component"}
    return out


def aggregate_ranks(t_local: float, units: float, world: int, dist=None, device: str = "cuda"):
    """Whole-job throughput over the ranks of a replicated run: the units all
    ranks processed divided by the slowest rank's time.  Returns (value,
    max time, total units)."""
    if world <= 1:
        return units / t_local, t_local, units
    import torch
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(uu)
    t_max, total = float(tt.item()), float(uu.item())
    return total / t_max, t_max, total


ORACLE_TOL = 1e-14


def oracle_x(g, cp, ci, state=None):
    """The oracle's x to |F|_1/(1-d) <= 1e-14 (resumed from the state of its
    timed solve when given), to state each form's error: its own error on any
    page is then at most 1e-14, below 3e-7 of the smallest x_i = (1-d)/n on this
    graph, so a per-page relative error near 1e-6 is measurable."""
    import oracle
    if state is None:
        H, _, _, _ = oracle.di_solve(g.n, cp, ci, None, D, None, tol=ORACLE_TOL)
    else:
        H, _, _, _ = oracle.di_solve(g.n, cp, ci, None, D, None, tol=ORACLE_TOL, H=state[0], F=state[1])
    return H


def error_vs_oracle(H, x_ref):
    """L1 error and largest per-page relative error of H against the oracle's x."""
    h = H.cpu().numpy() if hasattr(H, "cpu") else np.asarray(H)
    diff = np.abs(h - x_ref)
    return {"err_l1_vs_oracle": float(diff.sum()), "max_rel_err_vs_oracle": float((diff / np.abs(x_ref)).max()),
            "oracle_tol": ORACLE_TOL}


def traffic_for(record: str, opts: dict | None = None):
    """DRAM traffic per launch from a committed ncu record (profiles/<record>),
    if the kernel's source section is still the one the counters were taken on
    and the record's solver options match `opts` (else None)."""
    path = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    src = open(os.path.join(ROOT, rec["source_file"])).read()
    a, b = rec["source_section"]
    if a not in src or b not in src:
        return None
    h = hashlib.sha1(src[src.index(a):src.index(b)].encode()).hexdigest()
    if rec.get("source_sha1") != h:
        return None
    if opts is not None:
        taken = rec.get("options", {})
        for k in ("theta_factor", "hub_deg", "piece"):
            if k in opts and abs(float(taken.get(k, -1)) - float(opts[k])) > 1e-12:
                return None
    return rec.get("dram_bytes_per_launch")


def forms(st, G, g, torch, x_ref, di, reps=5):
    """Time to tol of a from-scratch solve in each form (L2 flushed before each
    run, CUDA events inside the library), with the L1 error and the largest
    per-page relative error of the returned H against the FP64 oracle's x when
    it is available; each form at the library defaults and at the options the
    autotuner picks for its precision, and both forms at tol 1e-12, where the
    per-page relative error is also held to 1e-6."""
    from paper_1501_06350_gb300 import _lib
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {}
    runs = [("f64", {}, TOL), ("f32_refined", {"precision": _lib.DI_PREC_F32}, TOL)]
    for name, prec in (("f64_tuned", _lib.DI_PREC_F64), ("f32_refined_tuned", _lib.DI_PREC_F32)):
        tuned, _ = di.autotune(G, D, TOL, prec, 20)
        runs.append((name, dict(tuned), TOL))
    runs += [("f64_tol1e-12", {}, 1e-12), ("f32_refined_tol1e-12", {"precision": _lib.DI_PREC_F32}, 1e-12)]
    for name, kw, tol in runs:
        ts, info, H = [], None, None
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            H, info = st.solve(D, tol=tol, **kw)
            ts.append(info["time_ms"])
        rec = {"tol": tol, "time_to_tol_ms": statistics.median(ts), "min_ms": min(ts), "sweeps": info["sweeps"],
               "edge_pushes": info["edge_pushes"], "refinements": info["refinements"],
               "refine_links": info["refine_links"], "resid_l1": info["resid_l1"], "bound": info["bound"]}
        if x_ref is not None:
            rec.update(error_vs_oracle(H, x_ref))
            rec["meets_1e-9_l1"] = rec["err_l1_vs_oracle"] <= 1e-9
            rec["meets_1e-6_rel"] = rec["max_rel_err_vs_oracle"] <= 1e-6
        if name.endswith("_tuned"):
            rec["options"] = {k: kw[k] for k in ("theta_factor", "hub_deg", "piece", "refine_ratio") if k in kw}
        out[name] = rec
    out["f32_speedup"] = out["f64"]["time_to_tol_ms"] / out["f32_refined"]["time_to_tol_ms"]
    out["f32_speedup_tuned"] = out["f64_tuned"]["time_to_tol_ms"] / out["f32_refined_tuned"]["time_to_tol_ms"]
    return out


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--small", action="store_true", help="200k-page graph (quick check)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--theta", type=float, default=None,
                    help="frontier threshold factor c (default: the library default)")
    ap.add_argument("--eager", action="store_true",
                    help="launch the sweep kernels one by one instead of the CUDA-graph loop")
    ap.add_argument("--precision", choices=["f64", "f32"], default="f64",
                    help="fluid arithmetic of the timed step: plain FP64, or FP32 fluid with FP64 "
                         "history and FP64 residual refinement")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the side-by-side time to tol of both forms")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the backward-pass timing on the 2M-page weighted graph")
    ap.add_argument("--no-tune", action="store_true",
                    help="time the step with the library defaults instead of the autotuned options")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched personalised solve and the union of 256 small graphs")
    ap.add_argument("--no-union", action="store_true", help="batched leg without the union of 256 graphs")
    ap.add_argument("--update50m", action="store_true",
                    help="run only the dynamic update on the 50M-page / ~600M-link graph and print it")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched leg (for profiling) and print it as the JSON line")
    ap.add_argument("--profile-solve", action="store_true",
                    help="profiling aid: one warm from-scratch solve, then one eager solve inside the NVTX "
                         "range 'profiled' (options from --theta/--hub-deg/--piece/--precision); prints the "
                         "push statistics of that solve")
    ap.add_argument("--hub-deg", type=int, default=None, help="degree-bin threshold (default: library default)")
    ap.add_argument("--piece", type=int, default=None, help="links per hub piece (default: library default)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.small:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        g = load_workload(args.small)
        print(json.dumps(run_reference(args, g)), flush=True)
        return 0

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if args.update50m:
        from paper_1501_06350_gb300 import di as di_mod
        print(json.dumps({"update50m": update50m_leg(torch, di_mod)}), flush=True)
        return 0
    if args.profile_solve:
        return profile_solve(args, torch)
    if args.batch_only:
        from paper_1501_06350_gb300 import di as di_mod
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        print(json.dumps({"batch": batch_leg(torch, di_mod, pk.get("hbm_gbs", 6800.0), union=not args.no_union)}),
              flush=True)
        return 0
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1501_06350_gb300 import _lib, di

    g = load_workload(args.small)
    G = di.Graph(g.n, g.ptr, g.idx)
    gi = G.info()
    cp, ci, _ = G.export_csr()
    src, dst, op = synth.exact_batch(cp, ci, g.n, BATCH_FRAC, 1)
    bs, bd, bo = (torch.from_numpy(x).cuda() for x in (src, dst, op))
    bo_inv = -bo
    st = di.State(G)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    L = _lib.lib()

    ug = 0 if args.eager else 1
    sopt = {}
    tuning = None
    if args.precision == "f32":
        sopt["precision"] = _lib.DI_PREC_F32
    if not args.no_tune:
        # one-time tuning of the launch shape on this graph (outside the timed region)
        tuned, trep = di.autotune(G, D, TOL, sopt.get("precision", 0), 20)
        sopt.update({k: tuned[k] for k in ("theta_factor", "hub_deg", "piece")})
        if args.precision == "f32":
            sopt["refine_ratio"] = tuned["refine_ratio"]
        tuning = {"options": {k: sopt[k] for k in sopt}, "tuned_ms": trep["best_ms"],
                  "default_ms": trep["default_ms"], "trials": trep["trials"]}
    if args.theta is not None:
        sopt["theta_factor"] = args.theta
    if args.hub_deg is not None:
        sopt["hub_deg"] = args.hub_deg
    if args.piece is not None:
        sopt["piece"] = args.piece

    def step():
        H, i1 = st.solve(D, tol=TOL, use_graph=ug, **sopt)
        st.update_edges(bs, bd, bo)
        H, i2 = st.resume(tol=TOL, use_graph=ug, **sopt)
        st.update_edges(bs, bd, bo_inv)
        H, i3 = st.resume(tol=TOL, use_graph=ug, **sopt)
        assert i1["converged"] and i2["converged"] and i3["converged"], (i1, i2, i3)
        return i1, i2, i3

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    # events: start, solved, first batch applied, re-converged, inverse applied, end
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(6)) for _ in range(args.steps)]
    launches0 = L.di_kernel_launches()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    infos = []
    # the timed steps as one NVTX range, so that a profiler can list their launches alone
    torch.cuda.nvtx.range_push("timed")
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        _, i1 = st.solve(D, tol=TOL, use_graph=ug, **sopt)
        ev[k][1].record()
        st.update_edges(bs, bd, bo)
        ev[k][2].record()
        _, i2 = st.resume(tol=TOL, use_graph=ug, **sopt)
        ev[k][3].record()
        st.update_edges(bs, bd, bo_inv)
        ev[k][4].record()
        _, i3 = st.resume(tol=TOL, use_graph=ug, **sopt)
        ev[k][5].record()
        infos.append((i1, i2, i3))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    torch.cuda.nvtx.range_pop()
    launches = L.di_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[5]) for e in ev]
    solve_ms = [e[0].elapsed_time(e[1]) for e in ev]
    # inject + patch of each link batch (Section 3.5), both directions
    patch_ms = [x for e in ev for x in (e[1].elapsed_time(e[2]), e[3].elapsed_time(e[4]))]
    pushes = sum(i1["edge_pushes"] + i2["edge_pushes"] + i3["edge_pushes"] for i1, i2, i3 in infos)
    t_local = sum(step_ms) / 1e3
    value, t_max, pushes_all = aggregate_ranks(t_local, pushes, world, dist, "cuda")

    # roofline of the dominant kernel (push), CUDA events around each launch
    _, prof = st.solve(D, tol=TOL, profile=1, **sopt)
    per_launch_links = prof["push_edges"] / max(prof["push_launches"], 1)
    push_avg_s = prof["push_ms"] / 1e3 / max(prof["push_launches"], 1)
    # algorithmic bytes per launch: per pushed link the 4 B target and the fluid
    # word added at the target; per diffused node 8 B of row pointers, the
    # fluid word taken (read + write), 16 B history read + write (FP64 H, or
    # the FP64 cycle accumulator), 8 B d/W_j and 4 B of frontier
    link_bytes = 8.0 if args.precision == "f32" else 12.0
    node_bytes = 36.0 if args.precision == "f32" else 44.0
    per_launch_nodes = prof["push_entries"] / max(prof["push_launches"], 1)
    alg_bytes = link_bytes * per_launch_links + node_bytes * per_launch_nodes
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = alg_bytes / push_avg_s / 1e9
    run_opts = {"theta_factor": sopt.get("theta_factor", 1.0), "hub_deg": sopt.get("hub_deg", 256),
                "piece": sopt.get("piece", 1024)}
    traffic = traffic_for(f"push_web4m_{args.precision}_c{run_opts['theta_factor']:g}_h{run_opts['hub_deg']}"
                          f"_p{run_opts['piece']}_traffic.json", run_opts)
    # the push's binding limit on this GPU is the L2's throughput of atomic
    # additions, not HBM: per launch, one exchange and one history add per
    # taken node and one add per link whose target is not a hot page (hot
    # pages are summed in shared memory; their one add per CTA is not counted)
    hot_per_launch = prof.get("push_hot_links", 0) / max(prof["push_launches"], 1)
    atomic_ops = per_launch_links - hot_per_launch + 2.0 * per_launch_nodes
    ceiling = atomic_ceiling(torch)
    atomics = {"bound": "l2_atomics", "achieved": atomic_ops / push_avg_s / 1e9, "peak": ceiling,
               "unit": "G atomic ops/s", "frac": atomic_ops / push_avg_s / 1e9 / ceiling,
               "ops_per_launch": atomic_ops, "hot_link_share": hot_per_launch / max(per_launch_links, 1.0),
               "peak_source": "measured live: di_probe_atomic_adds, 32M FP64 atomic adds at random slots of a 32 MB vector"}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "l2_atomics": atomics,
                "kernel": "k_push<float>" if args.precision == "f32" else "k_push<double>",
                "bytes_per_link": link_bytes, "bytes_per_node": node_bytes,
                "nodes_per_launch": per_launch_nodes,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_launch": alg_bytes, "links_per_launch": per_launch_links,
                "launches": prof["push_launches"], "push_ms_avg": 1e3 * push_avg_s,
                "push_share_of_solve": prof["push_ms"] / prof["time_ms"] if prof["time_ms"] else None}

    solve_pushes = statistics.median([i1["edge_pushes"] for i1, _, _ in infos])
    out = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 fluid / f64 history" if args.precision == "f32" else "f64", "data": "synthetic",
           "config": dict(config_dict(g, gi, args.precision), tuning=tuning),
           "time_to_tol_ms": statistics.median(solve_ms),
           "solve": {"edge_pushes": solve_pushes, "sweeps": statistics.median([i1["sweeps"] for i1, _, _ in infos]),
                     "edge_pushes_per_s": solve_pushes / (statistics.median(solve_ms) / 1e3),
                     "rounds_equiv": solve_pushes / gi["nnz"]},
           "update": {"ms": statistics.median([s - v for s, v in zip(step_ms, solve_ms)]),
                      "batch_links": int(len(src)),
                      "inject_patch_ms": statistics.median(patch_ms),
                      "reconverge_pushes": statistics.median([i2["edge_pushes"] + i3["edge_pushes"] for _, i2, i3 in infos]),
                      "roofline": update_roofline(cp, g.n, src, op, statistics.median(patch_ms), peak)},
           "wall_s": wall, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline}

    if rank == 0 and world == 1 and not args.no_e2e:
        out["e2e"] = e2e(args, g, src, dst, op, di, torch, sopt)
    x_ref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        # the oracle works on its own canonical build of the generator's links
        ocp, oci, _ = oracle.canonical_csr(g.n, g.ptr, g.idx)
        out["cpu_baseline"], ostate = cpu_baseline(g, ocp, oci)
        x_ref = oracle_x(g, ocp, oci, ostate)
    if rank == 0 and not args.no_forms:
        out["forms"] = forms(st, G, g, torch, x_ref, di)
    if rank == 0 and (not args.no_adjoint or not args.no_batch):
        st.close()
        G.close()
    if rank == 0 and not args.no_adjoint:
        out["adjoint"] = adjoint_leg(torch, di)
    if rank == 0 and not args.no_batch:
        out["batch"] = batch_leg(torch, di, peak, union=not args.no_union)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def profile_solve(args, torch):
    """The solve a DRAM-traffic record of the push is taken on: the same
    workload, the given options, one warm solve and then the eager solve
    inside the NVTX range 'profiled'.  Prints the push statistics (links,
    frontier nodes and hot-page links per launch) of that solve."""
    from paper_1501_06350_gb300 import _lib, di
    g = load_workload(args.small)
    G = di.Graph(g.n, g.ptr, g.idx)
    st = di.State(G)
    opts = {}
    if args.theta is not None:
        opts["theta_factor"] = args.theta
    if args.hub_deg is not None:
        opts["hub_deg"] = args.hub_deg
    if args.piece is not None:
        opts["piece"] = args.piece
    if args.precision == "f32":
        opts["precision"] = _lib.DI_PREC_F32
    st.solve(D, tol=TOL, **opts)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("profiled")
    _, p = st.solve(D, tol=TOL, profile=1, **opts)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    nl = max(p["push_launches"], 1)
    print(json.dumps({"profile_solve": {"options": opts, "push_launches": p["push_launches"],
                                        "links_per_launch": p["push_edges"] / nl,
                                        "nodes_per_launch": p["push_entries"] / nl,
                                        "hot_links_per_launch": p["push_hot_links"] / nl,
                                        "sweeps": p["sweeps"]}}), flush=True)
    return 0


def e2e(args, g, src, dst, op, di, torch, sopt):
    """Same step through the public API with host buffers: graph upload from
    pinned host memory, host Z in, host H out after every solve (with the
    solver options of the device-timed step)."""
    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t.numpy()
    ptr, idx = pinned(g.ptr), pinned(g.idx)
    Z = pinned(np.full(g.n, 1.0 / g.n))
    s, d_, o, oi = pinned(src), pinned(dst), pinned(op), pinned(-op)
    Hh = pinned(np.zeros(g.n))
    times, pushes = [], []
    for k in range(2 + max(1, min(args.steps, 3))):
        t = time.perf_counter()
        G = di.Graph(g.n, ptr, idx)
        st = di.State(G)
        _, i1 = st.solve(D, Z=Z, tol=TOL, out=Hh, device=False, **sopt)
        st.update_edges(s, d_, o)
        _, i2 = st.resume(tol=TOL, out=Hh, device=False, **sopt)
        st.update_edges(s, d_, oi)
        _, i3 = st.resume(tol=TOL, out=Hh, device=False, **sopt)
        dt = time.perf_counter() - t
        st.close()
        G.close()
        if k >= 2:
            times.append(dt)
            pushes.append(i1["edge_pushes"] + i2["edge_pushes"] + i3["edge_pushes"])
    h2d = ptr.nbytes + idx.nbytes + Z.nbytes + 2 * (s.nbytes + d_.nbytes + o.nbytes)
    d2h = 3 * Hh.nbytes
    return {"value": sum(pushes) / sum(times), "unit": METRIC, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * sum(times) / len(times),
            "includes": "graph build from pinned host CSR, state setup, 3 solves with host Z/H, 2 updates",
            "options": dict(sopt)}


if __name__ == "__main__":
    sys.exit(main())
