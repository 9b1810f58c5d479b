"""Benchmark of the Javelin hot path on GB300.

One step = one pass of the whole hot path over the 7-point 128^3 Laplacian
(n = 2,097,152, nnz = 14,581,760, FP64, diagonal shift 1e-3): ILU(0) factor,
L solve, U solve and spmv, with the analysis done once beforehand (the paper
does not time setup, Sec. V).  ``value`` is the whole-job throughput in GB/s
of algorithmic (compulsory) bytes: every matrix value and index read once,
every vector read / written once --

    factor  nnz (2v + 4) + 12 n          (read vals, write LU, indices)
    L solve nnzL (v + 4) + 8 n + 2 v n + 4 n
    U solve (nnzU + n)(v + 4) + 8 n + 2 v n + 4 n
    spmv    nnz (v + 4) + 4 (n + 1) + 2 v n         (v = 8 for FP64)

divided by the device time of the step (CUDA events on the library's
stream, L2 flushed before every step).  ``e2e`` is the same metric through
the public API from pinned host buffers: values and right-hand side copied
in, factor + solves + spmv, both results copied out, every step.

``--impl reference`` times the serial CPU oracle (the only reference this
method has) on the same workload and prints the same line.

Multi-GPU: the path does not shard (every row depends on earlier rows across
any partition), so N GPUs run N independent replicas; rank 0 prints the
aggregate over the max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ILU(0) factor + stri + spmv GB/s (% HBM peak)"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20

# ncu DRAM traffic (read + write bytes) per launch of the dominant kernel on
# this workload, with the hash of the kernel source it was captured from; a
# changed source makes the number stale and it is reported as null.
TRAFFIC = {}


def _src_hash(fname):
    p = os.path.join(ROOT, "paper_1812_06160_gb300", "csrc", fname)
    with open(p, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def byte_model(n, nnz, nnzl, nnzu, v, nrhs=1):
    return {
        "factor": nnz * (2 * v + 4) + 12 * n,
        "lsolve": nnzl * (v + 4) + 8 * n + 2 * v * n * nrhs + 4 * n,
        "usolve": (nnzu + n) * (v + 4) + 8 * n + 2 * v * n * nrhs + 4 * n,
        "spmv": nnz * (v + 4) + 4 * (n + 1) + 2 * v * n,
    }


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"jv_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(gpus):
    rank, world = 0, 1
    if gpus > 1 or "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if world > 1:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
    return rank, world


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------- CPU oracle
def run_oracle(c, budget_s):
    import oracle as O
    rp, ci, v, b = c["rowptr"], c["colidx"], c["vals"], c["b"]
    diag = O.diag_ptr(rp, ci)
    times = []
    t_end = time.perf_counter() + budget_s
    while time.perf_counter() < t_end or len(times) < 1:
        t0 = time.perf_counter()
        lu, _, _ = O.ilu0(rp, ci, v, diag)
        y = O.lsolve(rp, ci, diag, lu, b)
        z = O.usolve(rp, ci, diag, lu, y)
        O.spmv(rp, ci, v, z)
        times.append(time.perf_counter() - t0)
    return times


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="syncfree", choices=["syncfree", "level"])
    ap.add_argument("--reorder", action="store_true")
    ap.add_argument("--scale", type=int, default=None, help="smaller grid (testing only)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-krylov", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    a = ap.parse_args()
    assert a.warmup >= 3 or a.scale, "at least 3 warm-up steps"

    rank, world = dist_setup(a.gpus)
    c = W.config("c2", scale=a.scale)
    n = len(c["rowptr"]) - 1
    nnz = len(c["colidx"])
    rows =np.repeat(np.arange(n), np.diff(c["rowptr"]))
    nnzl = int((c["colidx"] < rows).sum())
    nnzu = nnz - n - nnzl
    model = byte_model(n, nnz, nnzl, nnzu, 8)
    step_bytes = sum(model.values())
    workload = f"{c['name']} natural-order" + (" level-reordered" if a.reorder else "")
    config = {"workload": workload, "n": n, "nnz": nnz, "mode": a.mode, "reorder": a.reorder,
              "step": "ilu0_factor + lsolve + usolve + spmv", "l2": "flushed before every step",
              "parallelism": f"replicas x{world}"}

    if a.impl == "reference":
        if rank != 0:
            return
        times = run_oracle(c, max(a.cpu_budget, 1.0) if a.steps else 1.0)
        med = statistics.median(times)
        val = step_bytes / med / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": a.gpus,
                "steps": len(times), "warmup": 0, "ms_per_step": med * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config,
                "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": f"{len(times)} full steps of the workload, median"},
                "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_1812_06160_gb300 as jv
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rp = torch.tensor(c["rowptr"], device=dev)
    ci = torch.tensor(c["colidx"], device=dev)
    h = jv.jv_analyze(rp, ci, mode=a.mode, reorder=a.reorder, check=False)
    vals = torch.tensor(c["vals"], device=dev)
    b = torch.tensor(c["b"], device=dev)
    if a.reorder:
        vals = jv.jv_permute_values(h, vals)
        b = jv.jv_permute_vector(h, b)
    lu = torch.empty_like(vals)
    y = torch.empty_like(b)
    z = torch.empty_like(b)
    s = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    kernels = ["factor", "lsolve", "usolve", "spmv"]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        jv.jv_ilu0_factor(h, vals, lu)
        if ev is not None:
            ev[1].record(stream)
        jv.jv_lsolve(h, lu, b, y)
        if ev is not None:
            ev[2].record(stream)
        jv.jv_usolve(h, lu, y, z)
        if ev is not None:
            ev[3].record(stream)
        jv.jv_spmv(h, vals, z, s)
        if ev is not None:
            ev[4].record(stream)

    for _ in range(a.warmup):
        flush.zero_()
        step()
    st, row = jv.jv_status_sync(h)
    if st != 0:
        raise SystemExit(f"device status {st} ({jv.jv_status_string(st)}) at row {row}")
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(a.steps)]
    launches0 = jv.jv_launch_count()
    with Clocks(local) as clk:
        torch.cuda.synchronize(dev)
        barrier(world)
        for k in range(a.steps):
            flush.zero_()
            step(evs[k])
        torch.cuda.synchronize(dev)
        barrier(world)
    launches = jv.jv_launch_count() - launches0
    st, row = jv.jv_status_sync(h)
    if st != 0:
        raise SystemExit(f"device status {st} ({jv.jv_status_string(st)}) at row {row}")
    per = {k: [] for k in kernels}
    tot = []
    for e in evs:
        for i, k in enumerate(kernels):
            per[k].append(e[i].elapsed_time(e[i + 1]))
        tot.append(e[0].elapsed_time(e[4]))
    ms_local = sum(tot) / len(tot)
    ms = reduce_max(ms_local, world)
    value = world * step_bytes / (ms * 1e-3) / 1e9
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    dom = max(avg, key=avg.get)
    peak, peak_kind = measured_peaks()
    achieved = model[dom] / (avg[dom] * 1e-3) / 1e9
    tr = TRAFFIC.get((dom, a.mode, a.reorder))
    traffic = tr[0] if tr and tr[1] == _src_hash(tr[2]) else None
    kern = {k: {"ms": avg[k], "bytes": model[k], "gbs": model[k] / (avg[k] * 1e-3) / 1e9,
                "frac_of_peak": model[k] / (avg[k] * 1e-3) / 1e9 / peak} for k in kernels}

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                         "peak_source": peak_kind},
            "kernels": kern, "gpu_launches": launches, "clocks": clk.summary()}

    if not a.no_e2e:
        hv = torch.tensor(c["vals"]).pin_memory()
        hb = torch.tensor(c["b"]).pin_memory()
        hz = torch.empty(n, dtype=torch.float64).pin_memory()
        hs = torch.empty(n, dtype=torch.float64).pin_memory()
        dv = torch.empty_like(vals)
        db = torch.empty_like(b)

        def e2e_step():
            dv.copy_(hv, non_blocking=True)
            db.copy_(hb, non_blocking=True)
            src_v, src_b = dv, db
            if a.reorder:
                src_v = jv.jv_permute_values(h, dv)
                src_b = jv.jv_permute_vector(h, db)
            jv.jv_ilu0_factor(h, src_v, lu)
            jv.jv_lsolve(h, lu, src_b, y)
            jv.jv_usolve(h, lu, y, z)
            jv.jv_spmv(h, src_v, z, s)
            hz.copy_(z, non_blocking=True)
            hs.copy_(s, non_blocking=True)

        for _ in range(max(2, a.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k2 = max(3, a.steps // 2)
        barrier(world)
        e0.record(stream)
        for _ in range(k2):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = reduce_max(e0.elapsed_time(e1) / k2, world)
        line["e2e"] = {"value": world * step_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
                       "ms_per_step": e2e_ms, "h2d_bytes_per_step": 8 * nnz + 8 * n,
                       "d2h_bytes_per_step": 16 * n}

    if not a.no_krylov:
        kry = {}
        bvec = b
        for name, ldt in (("fp64", torch.float64), ("fp32_prec", torch.float32)):
            x = torch.zeros_like(bvec)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            lu_k = jv.jv_ilu0_factor(h, vals, lu_dtype=ldt)
            x, info = jv.jv_pcg(h, vals, lu_k, bvec, x, tol=1e-8)
            torch.cuda.synchronize(dev)
            kry[name] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": info["iters"],
                         "true_relres": info["true_relres"], "converged": info["converged"]}
        line["krylov_pcg_time_to_1e-8"] = kry

    if rank == 0 and not a.no_cpu and world == 1:
        budget = a.cpu_budget
        times = run_oracle(c, budget)
        med = statistics.median(times)
        line["cpu_baseline"] = {"value": step_bytes / med / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(times)} full oracle steps of the same workload "
                                          f"(~{budget:.0f} s budget), median"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
