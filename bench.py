"""Benchmark: Matlab-compatible sparse assembly on the 3D P1 tetrahedral cube.

One step = one full assembly S = sparse(i,j,s,m,n) of the 100^3-vertex Kuhn
cube (93,148,704 triplets, no plan reuse) followed by 50 numeric-only
re-assemblies of the same pattern with fresh values (rotating 4 value
buffers), as in a time-dependent nonlinear PDE solve.  The metric is
G triplets/s over the whole job (51 assemblies of L triplets per step);
the JSON line also reports the full and numeric-only phases separately,
the HBM roofline of the dominant kernel (the numeric fold), the batched vs
plain comparison on 256 uneven instances, the other configurations and
the paper's own three data sets (with the paper's method timed on the host
cores beside them), an end-to-end figure through host buffers, clocks,
and the CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun, one rank per GPU) every rank assembles its own
replica (independent problems, no collective on the data path); the
timing is the max over ranks and the value is the total over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1406_1066_gb300 import inputs  # noqa: E402

WORKLOAD = "mesh3d_100"
NUMERIC_STEPS = 50
VALUE_SEEDS = (1409, 1410, 1411, 1412)
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal; the measured copy peak is the denominator


def workload_desc(t) -> str:
    N, dim = t.meta.get("N"), t.meta.get("dim")
    tail = (f"L={t.L} int32 1-based triplets, FP64 values; full assembly then {NUMERIC_STEPS} "
            f"numeric re-assemblies")
    if dim == 3:
        return (f"{t.name}: 3D P1 Kuhn-tetrahedral cube, {N}^3 vertices (m=n={t.m}), "
                f"{(N - 1) ** 3 * 6} tets, element order, U(-1,1) values, {tail}")
    if dim == 2:
        return (f"{t.name}: 2D P1 triangulated square, {N}^2 vertices (m=n={t.m}), "
                f"{(N - 1) ** 2 * 2} triangles, element order, U(-1,1) values, {tail}")
    return f"{t.name}: m={t.m}, n={t.n}, {tail}"


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(*files) -> str:
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1406_1066_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(summary: str, src_hash: str):
    """DRAM bytes per launch from a committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        kv = {}
        for line in open(path):
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha1") != src_hash:
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", self.gpu], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.tmp.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity when world == 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- CPU oracle leg
def oracle_job(t, frac_den: int, numeric_steps: int):
    """Run the oracle on the first L/frac_den triplets (element order); return (seconds, L_s)."""
    import oracle
    Ls = (t.L // frac_den) // 16 * 16
    ii, jj, s = t.ii[:Ls].copy(), t.jj[:Ls].copy(), t.s[:Ls].copy()
    vals = [inputs.mesh_values(Ls, 9000 + k) for k in range(4)]
    t0 = time.perf_counter()
    r = oracle.assemble(ii, jj, s, t.m, t.n)
    for k in range(numeric_steps):
        oracle.numeric(r.irank, vals[k % 4], r.nnz)
    return time.perf_counter() - t0, Ls


def paper_method_job(t, frac_den: int, reps: int = 2):
    """The paper's own CPU method (§2.3, in the threaded form of §3; "serial"
    is that routine on one thread): full assembly of
    the first L/frac_den triplets, best of `reps` runs of each variant (the
    first run of each also pays for faulting in its tables)."""
    from oracle import paper_method
    Ls = (t.L // frac_den) // 16 * 16
    ii, jj, s = t.ii[:Ls].copy(), t.jj[:Ls].copy(), t.s[:Ls].copy()
    what = "the whole workload" if frac_den == 1 else f"first {Ls} triplets (1/{frac_den} of the workload)"
    out = {"unit": "G triplets/s (full assembly)", "kind": "paper method (§2.3 in the threaded form of §3; serial = one thread)",
           "openmp": None, "sample": f"{what}, element order, best of {reps} runs"}

    def best(threads):
        sec, used = 1e30, 1
        for _ in range(reps):
            t0 = time.perf_counter()
            res = paper_method.assemble(ii, jj, s, t.m, t.n, threads=threads, want_irank=False)
            sec = min(sec, time.perf_counter() - t0)
            if threads is not None:
                used = res[1]
        return sec, used

    sec, _ = best(None)
    out["serial"] = {"value": Ls / sec / 1e9, "seconds": sec, "cores": 1}
    sec, used = best(0)
    out["threaded"] = {"value": Ls / sec / 1e9, "seconds": sec, "cores": used}
    out["openmp"] = bool(paper_method.openmp)
    return out


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    t = inputs.workload(args.workload)
    den = 16 if t.L > 10**7 else 1
    for _ in range(args.warmup):
        oracle_job(t, den, NUMERIC_STEPS)
    times = []
    Ls = 0
    for _ in range(args.steps):
        sec, Ls = oracle_job(t, den, NUMERIC_STEPS)
        times.append(sec)
    per = statistics.mean(times)
    value = Ls * (1 + NUMERIC_STEPS) / per / 1e9
    sample = (f"first {Ls} triplets (1/{den} of the cube in element order): one oracle assembly "
              f"+ {NUMERIC_STEPS} oracle numeric passes per step, single thread")
    line = {"impl": "reference", "metric": "G triplets/s (full assembly + 50 numeric re-assemblies)",
            "value": value, "unit": "G triplets/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(t), "workload_name": t.name,
                       "numeric_steps": NUMERIC_STEPS, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "G triplets/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "G triplets/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
def append_timing(torch, fsparse, ii_d, jj_d, t, full_ms, reps: int = 5):
    """Delayed assembly: the last part of the workload (half, and 1%) appended
    to a plan of the rest, against one full assembly of everything."""
    out = {"full_assembly_ms": full_ms,
           "note": "the last part appended to a plan of the rest (symbolic of the new part + merge); "
                   "full_assembly_ms assembles all triplets from scratch"}
    for name, cut in (("half", t.L // 2), ("one_percent", t.L - t.L // 100)):
        base = fsparse.symbolic(ii_d[:cut], jj_d[:cut], t.m, t.n)
        ms = []
        for r in range(reps + 2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p2 = fsparse.append(base, ii_d[cut:], jj_d[cut:])
            e1.record()
            torch.cuda.synchronize()
            if r >= 2:
                ms.append(e0.elapsed_time(e1))
            p2.close()
        base.close()
        sym = []   # the appended part's own symbolic pass, for the split of the time
        for r in range(reps + 2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p3 = fsparse.symbolic(ii_d[cut:], jj_d[cut:], t.m, t.n)
            e1.record()
            torch.cuda.synchronize()
            if r >= 2:
                sym.append(e0.elapsed_time(e1))
            p3.close()
        a_ms = statistics.median(ms)
        out[name] = {"ms": a_ms, "appended_triplets": t.L - cut, "plan_triplets": cut,
                     "gtps_appended": (t.L - cut) / a_ms / 1e6, "vs_full_assembly": full_ms / a_ms,
                     "new_part_symbolic_ms": statistics.median(sym)}
    return out


def adjoint_timing(torch, fsparse, ii_d, jj_d, s_d, t, peak, reps: int = 20):
    """The adjoint ds[k] = dprS[irank[k]] (the backward of the numeric
    assembly) on the benchmark's own plan; irank is derived once, before the
    timed launches, which run back to back between two events."""
    jcS, irS, pr, plan = fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n)
    nnz = plan.nnz
    dprS = pr[:nnz].clone()
    ds = torch.empty(t.L, dtype=torch.float64, device=s_d.device)
    for _ in range(3):
        fsparse.numeric_adjoint(plan, dprS, ds)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fsparse.numeric_adjoint(plan, dprS, ds)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    plan.close()
    B = 12 * t.L + 8 * nnz
    return {"ms": ms, "gtps": t.L / ms / 1e6, "algorithmic_bytes": B,
            "hbm_frac": B / (ms / 1e3) / 1e9 / peak,
            "note": "irank read 4L + ds written 8L + dprS read 8nnz per launch; inputs larger than L2"}


def batched_vs_plain(torch, fsparse, to_dev, peak, steps: int = 100):
    """256 uneven mesh instances, 100 re-assembly steps rotating two value
    buffers: the batched numeric (one launch per step) against per-instance
    launches, both graph-captured and not; plus one batched symbolic pass
    against 256 per-instance symbolic calls.  Every timed loop only replays
    or launches: value buffers are bound at capture (one graph per buffer),
    so no copy sits inside the timed region."""
    b = inputs.batch(256, 1416)
    insts = b.instances
    ii_cat = to_dev(np.concatenate([t.ii for t in insts]))
    jj_cat = to_dev(np.concatenate([t.jj for t in insts]))
    off = [0] + np.cumsum([t.L for t in insts]).tolist()
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, reps):
        torch.cuda.synchronize()
        e0, e1 = mk(), mk()
        e0.record()
        for r in range(reps):
            fn(r)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # symbolic: one batched pass vs one call per instance (each synchronises)
    views_i = [ii_cat[off[i]:off[i + 1]] for i in range(len(insts))]
    views_j = [jj_cat[off[i]:off[i + 1]] for i in range(len(insts))]
    for _ in range(2):
        fsparse.batch_symbolic(ii_cat, jj_cat, off, [t.m for t in insts], [t.n for t in insts]).close()
    sym_b = timed(lambda r: fsparse.batch_symbolic(ii_cat, jj_cat, off, [t.m for t in insts],
                                                   [t.n for t in insts]).close(), 3)
    plans = [fsparse.symbolic(views_i[i], views_j[i], t.m, t.n) for i, t in enumerate(insts)]
    for p in plans:
        p.close()
    t0 = time.perf_counter()
    plans = [fsparse.symbolic(views_i[i], views_j[i], t.m, t.n) for i, t in enumerate(insts)]
    torch.cuda.synchronize()
    sym_p = (time.perf_counter() - t0) * 1e3

    bt = fsparse.batch_symbolic(ii_cat, jj_cat, off, [t.m for t in insts], [t.n for t in insts])
    total, total_nnz = bt.len_off[-1], bt.nnz_off[-1]
    vals = [torch.from_numpy(inputs.mesh_values(total, 1416 + k)).to("cuda") for k in range(2)]
    out_b = [torch.empty(total_nnz, dtype=torch.float64, device="cuda") for _ in range(2)]
    outs_p = [[torch.empty(p.cap, dtype=torch.float64, device="cuda") for p in plans] for _ in range(2)]
    vviews = [[vals[k][off[i]:off[i + 1]] for i in range(len(plans))] for k in range(2)]

    def plain_step(k):
        for p, v, o in zip(plans, vviews[k], outs_p[k]):
            fsparse.numeric(p, v, o)

    def capture(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    # the batch's numeric tile: every supported tile, each on its own batch
    tiles = {}
    for tile in (1024, 2048, 4096):
        fsparse.fsparse_set_config({"strategy": 0, "radix_bits": 0, "sweep_items": 0, "sweep_threads": 0,
                                    "bucket_target": 0, "numeric_tile": tile})
        bt_t = fsparse.Batch(plans)
        fsparse.fsparse_set_config(None)
        gs = [capture(lambda k=k: bt_t.numeric(vals[k], out_b[k])) for k in range(2)]
        tiles[tile] = timed(lambda r: gs[r & 1].replay(), steps)
        del gs
        bt_t.close()
    best_tile = min(tiles, key=tiles.get)
    graphs_b = [capture(lambda k=k: bt.numeric(vals[k], out_b[k])) for k in range(2)]
    batched_ms = timed(lambda r: graphs_b[r & 1].replay(), steps)
    graphs_p = [capture(lambda k=k: plain_step(k)) for k in range(2)]
    plain_graph_ms = timed(lambda r: graphs_p[r & 1].replay(), steps)
    n0 = fsparse.fsparse_kernel_launches()
    plain_ms = timed(lambda r: plain_step(r & 1), steps)
    plain_launches = (fsparse.fsparse_kernel_launches() - n0) // steps
    torch.cuda.synchronize()
    same = all(torch.equal(out_b[k][bt.nnz_off[i]:bt.nnz_off[i + 1]], outs_p[k][i][: plans[i].nnz])
               for k in range(2) for i in range(len(plans)))
    B = 12 * total + 8 * total_nnz
    res = {"instances": len(plans), "total_triplets": total, "total_nnz": total_nnz, "steps": steps,
           "batched_kernel_ms": batched_ms, "batched_gtps": total / batched_ms / 1e6,
           "hbm_frac": B / (batched_ms / 1e3) / 1e9 / peak, "algorithmic_bytes": B,
           "tile_sweep_ms": tiles, "best_tile": best_tile,
           "plain_graph_ms": plain_graph_ms, "plain_ms": plain_ms, "plain_launches_per_step": plain_launches,
           "speedup_vs_plain": plain_ms / batched_ms, "speedup_vs_plain_graph": plain_graph_ms / batched_ms,
           "identical": bool(same),
           "symbolic": {"batched_ms": sym_b, "per_instance_ms": sym_p, "speedup": sym_p / sym_b,
                        "note": "one fsparse_batch_symbolic pass vs 256 fsparse_symbolic calls (host clock, "
                                "each call synchronises)"},
           "note": "batched = one fsparse_batch_numeric launch per step (graph replay); plain = 256 "
                   "fsparse_numeric launches per step, captured in one graph (plain_graph_ms) or launched "
                   "(plain_ms); value buffers bound at capture, no copies timed; the batch of the "
                   "batched leg comes from fsparse_batch_symbolic, the tile sweep from fsparse_batch_create"}
    del graphs_b, graphs_p
    bt.close()
    for p in plans:
        p.close()
    return res


PER_CONFIG = ("mesh2d_64", "uniform_1e6", "pooled_2e4", "mesh3d_60")


def full_and_numeric(torch, fsparse, ii_d, jj_d, s_d, s2, t, reps: int):
    """Full assembly (median of `reps` calls, no plan reuse) and numeric
    re-assembly (mean of `reps` launches, alternating two value arrays);
    returns (full ms, nnz, numeric ms)."""
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    prS = torch.empty(t.L, dtype=torch.float64, device=s_d.device)
    out_n = torch.empty(t.L, dtype=torch.float64, device=s_d.device)
    for _ in range(3):
        fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n, prS=prS)[3].close()
    full = []
    for _ in range(reps):
        e0, e1 = mk(), mk()
        e0.record()
        _, _, _, plan = fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n, prS=prS)
        e1.record()
        torch.cuda.synchronize()
        full.append(e0.elapsed_time(e1))
        nnz = plan.nnz
        plan.close()
    _, _, _, plan = fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n, prS=prS)
    for _ in range(3):
        fsparse.numeric(plan, s2, out_n)
    torch.cuda.synchronize()
    e0, e1 = mk(), mk()
    e0.record()
    for r in range(reps):
        fsparse.numeric(plan, s2 if r & 1 else s_d, out_n)
    e1.record()
    torch.cuda.synchronize()
    num_ms = e0.elapsed_time(e1) / reps
    plan.close()
    return statistics.median(full), nnz, num_ms


def per_config(torch, fsparse, to_dev, peak, reps: int = 10, tune: bool = True):
    """Configs other than the benchmark's own, one line each: full assembly
    (median of `reps`, no plan reuse) and numeric re-assembly (mean of
    `reps` launches), with their fractions of the measured copy bandwidth."""
    out = {}
    for name in PER_CONFIG:
        t = inputs.workload(name)
        ii_d, jj_d, s_d = to_dev(t.ii), to_dev(t.jj), to_dev(t.s)
        s2 = to_dev(inputs.mesh_values(t.L, 77))
        if tune:
            fsparse.autotune(ii_d, jj_d, s_d, t.m, t.n, reps=2)
        prS = torch.empty(t.L, dtype=torch.float64, device=s_d.device)
        fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n, prS=prS)[3].close()
        phases = full_phases(torch, fsparse, ii_d, jj_d, s_d, t, prS, reps=3)
        f_ms, nnz, num_ms = full_and_numeric(torch, fsparse, ii_d, jj_d, s_d, s2, t, reps)
        B_full = 16 * t.L + 12 * nnz + 4 * (t.n + 1)
        B_num = 12 * t.L + 8 * nnz
        out[name] = {"L": t.L, "nnz": nnz, "m": t.m, "n": t.n,
                     "full_ms": f_ms, "full_gtps": t.L / f_ms / 1e6,
                     "full_hbm_frac": B_full / (f_ms / 1e3) / 1e9 / peak,
                     "numeric_ms": num_ms, "numeric_gtps": t.L / num_ms / 1e6,
                     "numeric_hbm_frac": B_num / (num_ms / 1e3) / 1e9 / peak,
                     "full_phases_ms": phases, "launch": fsparse.fsparse_get_config(t.L, t.m, t.n),
                     "inputs_vs_l2": "inside L2 (fractions not meaningful)" if 16 * t.L < 64e6
                     else "inputs larger than L2"}
        del ii_d, jj_d, s_d, s2, prS
        torch.cuda.empty_cache()
    return out


# The paper's own benchmark sets (§4.2, ransparse(siz, nnz_row, nrep): every
# row nnz_row times, uniform columns, every pair nrep times, shuffled, values
# one; 25,000,000 triplets each) and the paper's times for them in seconds,
# serial and parallel fsparse on its 6-core (C1) and 16-core (C2) hosts (§4.3,
# table of overall speedups).  Those hosts are other machines: context only.
PAPER_DATA = {
    "data1": ((10_000, 50, 50), {"C1": {"serial_s": 1.51, "parallel_s": 0.65},
                                 "C2": {"serial_s": 1.61, "parallel_s": 0.33}}),
    "data2": ((50_000, 50, 10), {"C1": {"serial_s": 1.87, "parallel_s": 0.83},
                                 "C2": {"serial_s": 2.95, "parallel_s": 0.46}}),
    "data3": ((50_000, 10, 50), {"C1": {"serial_s": 1.67, "parallel_s": 0.76},
                                 "C2": {"serial_s": 1.78, "parallel_s": 0.43}}),
}


def paper_data(torch, fsparse, to_dev, peak, cpu: bool, reps: int = 10):
    """Full assembly and numeric re-assembly of the paper's three data sets on
    the GPU, with their device phases, and (with `cpu`) the paper's own method
    on the host cores on the same sets, beside the times the paper prints."""
    out = {}
    for name, ((siz, nnz_row, nrep), published) in PAPER_DATA.items():
        t = inputs.ransparse(siz, nnz_row, nrep, seed=1100 + int(name[-1]))
        ii_d, jj_d, s_d = to_dev(t.ii), to_dev(t.jj), to_dev(t.s)
        s2 = to_dev(inputs.mesh_values(t.L, 78))
        prS = torch.empty(t.L, dtype=torch.float64, device=s_d.device)
        fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n, prS=prS)[3].close()
        phases = full_phases(torch, fsparse, ii_d, jj_d, s_d, t, prS, reps=3)
        f_ms, nnz, num_ms = full_and_numeric(torch, fsparse, ii_d, jj_d, s_d, s2, t, reps)
        B_full = 16 * t.L + 12 * nnz + 4 * (t.n + 1)
        B_num = 12 * t.L + 8 * nnz
        row = {"siz": siz, "nnz_row": nnz_row, "nrep": nrep, "L": t.L, "nnz": nnz,
               "full_ms": f_ms, "full_gtps": t.L / f_ms / 1e6,
               "full_hbm_frac": B_full / (f_ms / 1e3) / 1e9 / peak,
               "numeric_ms": num_ms, "numeric_gtps": t.L / num_ms / 1e6,
               "numeric_hbm_frac": B_num / (num_ms / 1e3) / 1e9 / peak,
               "full_phases_ms": phases, "launch": fsparse.fsparse_get_config(t.L, t.m, t.n),
               "paper_published": published}
        if cpu:
            row["paper_method_on_host"] = paper_method_job(t, 1)
        out[name] = row
        del ii_d, jj_d, s_d, s2, prS
        torch.cuda.empty_cache()
    return out


def full_phases(torch, fsparse, ii_d, jj_d, s_d, t, prS, reps: int = 5):
    """Device time of every phase of one full assembly (FSPARSE_TIMING=1,
    CUDA events between the phases; median of `reps` calls)."""
    os.environ["FSPARSE_TIMING"] = "1"
    runs = []
    try:
        for _ in range(reps):
            fsparse.assemble(ii_d, jj_d, s_d, t.m, t.n, prS=prS)[3].close()
            runs.append(fsparse.fsparse_last_timings())
    finally:
        os.environ.pop("FSPARSE_TIMING", None)
    names = [n for n, _ in runs[-1]]
    return {n: statistics.median([dict(r).get(n, 0.0) for r in runs]) for n in names}


def gpu_arm(args):
    import torch

    from paper_1406_1066_gb300 import fsparse

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    t = inputs.workload(args.workload) if args.workload != WORKLOAD else inputs.workload(WORKLOAD)
    L = t.L
    ii_d, jj_d = to_dev(t.ii), to_dev(t.jj)
    vals = [to_dev(t.s)] + [to_dev(inputs.mesh_values(L, sd)) for sd in VALUE_SEEDS[1:]]
    prS = torch.empty(L, dtype=torch.float64, device=dev)
    out = torch.empty(L, dtype=torch.float64, device=dev)
    # The library's autotuner picks the launch configuration for this size
    # class (sort strategy and shape by symbolic time, then the numeric tile
    # by repeated folds); it runs before, and outside, the timed region.
    default_cfg = fsparse.fsparse_get_config(L, t.m, t.n)
    tune_s = None
    if not args.no_tune:
        t0 = time.perf_counter()
        fsparse.autotune(ii_d, jj_d, vals[0], t.m, t.n, reps=2)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
    cfg = fsparse.fsparse_get_config(L, t.m, t.n)

    def step(timing=None):
        if timing is not None:
            timing["a0"].record()
        jcS, irS, pr, plan = fsparse.assemble(ii_d, jj_d, vals[0], t.m, t.n, prS=prS)
        if timing is not None:
            timing["a1"].record()
        for r in range(NUMERIC_STEPS):
            if timing is not None:
                timing["n"][r][0].record()
            fsparse.numeric(plan, vals[(r + 1) % 4], out)
            if timing is not None:
                timing["n"][r][1].record()
        nnz = plan.nnz
        plan.close()
        return nnz

    for _ in range(args.warmup):
        nnz = step()
    torch.cuda.synchronize()

    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] if world == 1 else str(local)
    sampler = ClockSampler(gpu_index)
    mk = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    timings = [{"a0": mk(), "a1": mk(), "n": [(mk(), mk()) for _ in range(NUMERIC_STEPS)]}
               for _ in range(args.steps)]
    ev0, ev1 = mk(), mk()
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    n_launch0 = fsparse.fsparse_kernel_launches()
    ev0.record()
    for k in range(args.steps):
        nnz = step(timings[k])
    ev1.record()
    torch.cuda.synchronize()
    launches = fsparse.fsparse_kernel_launches() - n_launch0
    barrier(world)
    clocks = sampler.stop()
    local_ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(local_ms, world, dev)
    full_ms = statistics.median([tm["a0"].elapsed_time(tm["a1"]) for tm in timings])
    num_ms = [a.elapsed_time(b) for tm in timings for (a, b) in tm["n"]]
    num_avg = statistics.mean(num_ms)

    peak, peak_kind = hbm_peak()
    props = torch.cuda.get_device_properties(dev)
    B_num = 12 * L + 8 * nnz
    B_full = 16 * L + 12 * nnz + 4 * (t.n + 1)
    achieved = B_num / (num_avg / 1e3) / 1e9
    src_hash = kernel_source_hash("numeric.cu", "common.cuh")
    traffic = profiled_traffic(f"numeric_kernel_{args.workload}.md", src_hash)
    value = world * L * (1 + NUMERIC_STEPS) / (ms / 1e3) / 1e9

    # ---- end to end through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_ii = torch.from_numpy(t.ii).pin_memory()
        h_jj = torch.from_numpy(t.jj).pin_memory()
        h_vals = [torch.from_numpy(t.s).pin_memory()] + \
                 [torch.from_numpy(inputs.mesh_values(L, sd)).pin_memory() for sd in VALUE_SEEDS[1:]]
        h_out = torch.empty(L, dtype=torch.float64).pin_memory()
        h_jc = torch.empty(t.n + 1, dtype=torch.int32).pin_memory()
        h_ir = torch.empty(L, dtype=torch.int32).pin_memory()
        d_s = torch.empty(L, dtype=torch.float64, device=dev)
        # Host link: uploads of the next values overlap the current fold and
        # the download of the previous result (one stream per direction).
        vbuf = [torch.empty(L, dtype=torch.float64, device=dev) for _ in range(2)]
        obuf = [torch.empty(L, dtype=torch.float64, device=dev) for _ in range(2)]
        up_s, down_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

        def e2e_step():
            cur = torch.cuda.current_stream()
            up_done = [torch.cuda.Event() for _ in range(NUMERIC_STEPS)]
            fold_done = [torch.cuda.Event() for _ in range(NUMERIC_STEPS)]
            down_done = [torch.cuda.Event() for _ in range(NUMERIC_STEPS)]

            def upload(r):
                if r >= 2:
                    up_s.wait_event(fold_done[r - 2])     # vbuf[r % 2] is free again
                with torch.cuda.stream(up_s):
                    vbuf[r % 2].copy_(h_vals[(r + 1) % 4], non_blocking=True)
                up_done[r].record(up_s)

            upload(0)                                     # overlaps the assembly below
            ii_d.copy_(h_ii, non_blocking=True)
            jj_d.copy_(h_jj, non_blocking=True)
            d_s.copy_(h_vals[0], non_blocking=True)
            jcS, irS, pr, plan = fsparse.assemble(ii_d, jj_d, d_s, t.m, t.n, prS=prS)
            nz = plan.nnz
            ev = torch.cuda.Event()
            ev.record(cur)
            down_s.wait_event(ev)
            with torch.cuda.stream(down_s):
                h_jc.copy_(jcS, non_blocking=True)
                h_ir[:nz].copy_(irS[:nz], non_blocking=True)
                h_out[:nz].copy_(pr[:nz], non_blocking=True)
            for r in range(NUMERIC_STEPS):
                if r + 1 < NUMERIC_STEPS:
                    upload(r + 1)
                cur.wait_event(up_done[r])
                if r >= 2:
                    cur.wait_event(down_done[r - 2])      # obuf[r % 2] has been read back
                fsparse.numeric(plan, vbuf[r % 2], obuf[r % 2])
                fold_done[r].record(cur)
                down_s.wait_event(fold_done[r])
                with torch.cuda.stream(down_s):
                    h_out[:nz].copy_(obuf[r % 2][:nz], non_blocking=True)
                down_done[r].record(down_s)
            torch.cuda.synchronize()
            plan.close()
            return nz

        e2e_step()
        e_steps = max(3, args.steps // 3)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = mk(), mk()
        e0.record()
        for _ in range(e_steps):
            nz = e2e_step()
        e1.record()
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1) / e_steps, world, dev)
        h2d = 8 * L + 8 * L * (1 + NUMERIC_STEPS)
        d2h = 4 * (t.n + 1) + 12 * nz + 8 * nz * NUMERIC_STEPS
        e2e = {"value": world * L * (1 + NUMERIC_STEPS) / (e_ms / 1e3) / 1e9, "unit": "G triplets/s",
               "ms_per_step": e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": e_steps}

    extra = {}
    if rank == 0 and world == 1:
        extra["full_phases_ms"] = full_phases(torch, fsparse, ii_d, jj_d, vals[0], t, prS)
        extra["append"] = append_timing(torch, fsparse, ii_d, jj_d, t, full_ms)
        extra["adjoint"] = adjoint_timing(torch, fsparse, ii_d, jj_d, vals[0], t, peak)
    if rank == 0 and world == 1 and not args.no_batch:
        del vals, prS, out
        torch.cuda.empty_cache()
        extra["batched_vs_plain"] = batched_vs_plain(torch, fsparse, to_dev, peak)
    if rank == 0 and world == 1 and not args.no_configs:
        extra["per_config"] = per_config(torch, fsparse, to_dev, peak, tune=not args.no_tune)
        extra["paper_data"] = paper_data(torch, fsparse, to_dev, peak, cpu=not args.no_cpu)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # one whole step of the workload (about 10 s on the machine's host cores)
        sec, Ls = oracle_job(t, 1, NUMERIC_STEPS)
        cpu = {"value": Ls * (1 + NUMERIC_STEPS) / sec / 1e9, "unit": "G triplets/s", "cores": 1,
               "kind": "oracle", "seconds": sec,
               "sample": f"one step of the whole workload ({Ls} triplets): one oracle assembly "
                         f"+ {NUMERIC_STEPS} oracle numeric passes, single thread"}

    paper_cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        paper_cpu = paper_method_job(t, 1)

    if rank == 0:
        line = {
            "metric": "G triplets/s (full assembly + 50 numeric re-assemblies)",
            "value": value, "unit": "G triplets/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(t), "workload_name": t.name,
                       "numeric_steps": NUMERIC_STEPS,
                       "nnz": nnz, "l2": "inputs larger than L2 (1.49 GB of triplets per assembly)",
                       "l2_bytes": getattr(props, "L2_cache_size", None), "sm_count": props.multi_processor_count,
                       "device": props.name,
                       "launch": cfg, "launch_default": default_cfg, "autotune_s": tune_s,
                       "parallelism": f"replicas{world}"},
            "full": {"ms": full_ms, "gtps": L / full_ms / 1e6,
                     "algorithmic_bytes": B_full, "hbm_frac": B_full / (full_ms / 1e3) / 1e9 / peak,
                     "hbm_frac_nominal": B_full / (full_ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
                     "algorithmic_bytes_with_irank": B_full + 4 * L,
                     "hbm_frac_with_irank": (B_full + 4 * L) / (full_ms / 1e3) / 1e9 / peak},
            "numeric": {"ms": num_avg, "gtps": L / num_avg / 1e6, "algorithmic_bytes": B_num,
                        "hbm_frac": achieved / peak, "hbm_frac_nominal": achieved / NOMINAL_HBM_GBS},
            "roofline": {"kernel": "numeric_kernel", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_launch": B_num, "kernel_source_sha1": src_hash},
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "cpu_paper_method": paper_cpu,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configs' lines and the paper's data sets")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="mesh3d_100 (default), or mesh3d_<N> for a smaller cube (profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
