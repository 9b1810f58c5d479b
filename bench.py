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

# ncu DRAM traffic (read + write bytes) per launch of the dominant kernel,
# keyed by (config, dtype, kernel, mode, reorder), with a hash of the kernel
# sources it was captured from; a changed source makes the number stale and
# it is reported as null.
KERNEL_SOURCES = {"factor": ("factor.cu", "jv_internal.cuh"),
                  "lsolve": ("trisolve.cu", "jv_internal.cuh"),
                  "usolve": ("trisolve.cu", "jv_internal.cuh")}
TRAFFIC = {
    ("c2", "f64", "factor", "syncfree", False): (463_433_216, "935fc88ac78b"),
    ("c2", "f64", "lsolve", "syncfree", False): (265_663_232, "1cd43ef4689d"),
    ("c2", "f64", "usolve", "syncfree", False): (268_394_496, "1cd43ef4689d"),
}


def _src_hash(fnames):
    h = hashlib.sha1()
    for fname in fnames:
        with open(os.path.join(ROOT, "paper_1812_06160_gb300", "csrc", fname), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def byte_model(n, nnz, nnzl, nnzu, v, nrhs=1, adjoint=False):
    """Compulsory bytes per kernel (v = value size; i32 indices; nnzu
    excludes the diagonal).  The solves read their level's row list (4 n)
    and two row-pointer arrays (8 n); the transposed solves also read the
    CSC-to-CSR value map (4 per entry); the masked outer products read both
    n x nrhs operands once and write the gradient on the pattern."""
    r = nrhs
    m = {
        "factor": nnz * (2 * v + 4) + 12 * n,
        "lsolve": nnzl * (v + 4) + 8 * n + 2 * v * n * r + 4 * n,
        "usolve": (nnzu + n) * (v + 4) + 8 * n + 2 * v * n * r + 4 * n,
    }
    if adjoint:
        m["usolve_t"] = (nnzu + n) * (v + 8) + 8 * n + 2 * v * n * r + 4 * n
        m["lsolve_t"] = nnzl * (v + 8) + 8 * n + 2 * v * n * r + 4 * n
        m["outer"] = nnz * (v + 4) + 8 * n + 4 * v * n * r
    else:
        m["spmv"] = nnz * (v + 4) + 4 * (n + 1) + 2 * v * n
    return m


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
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # nvidia-smi takes a while to start: let its first sample land before
        # the timed region begins, so the samples cover that region
        t_end = time.time() + 5.0
        while self.proc and self.proc.poll() is None and time.time() < t_end:
            if os.path.exists(self.path) and os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
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
        if world > 1 and not dist.is_initialized():
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


# ---------------------------------------------------------------- workloads
# Kernels of one step; c5 (32 right-hand sides) runs the preconditioner
# apply and its adjoint instead of the spmv.
SOLVE_STEP = ["factor", "lsolve", "usolve", "spmv"]
ADJOINT_STEP = ["factor", "lsolve", "usolve", "usolve_t", "lsolve_t", "outer"]
# level structure each kernel walks (index into jv_info.nlev: L, U, U^T, L^T)
DAG_OF = {"factor": 0, "lsolve": 0, "usolve": 1, "usolve_t": 2, "lsolve_t": 3}


def load_workload(name, scale, dtype):
    return workload_meta(W.config(name, scale=scale), dtype)


def workload_meta(c, dtype):
    n = len(c["rowptr"]) - 1
    nnz = len(c["colidx"])
    rows = np.repeat(np.arange(n), np.diff(c["rowptr"]))
    nnzl = int((c["colidx"] < rows).sum())
    nnzu = nnz - n - nnzl
    nrhs = 1 if c["b"].ndim == 1 else c["b"].shape[1]
    adjoint = "g" in c
    v = 8 if dtype == "f64" else 4
    meta = dict(n=n, nnz=nnz, nnzl=nnzl, nnzu=nnzu, nrhs=nrhs, adjoint=adjoint, v=v,
                kernels=ADJOINT_STEP if adjoint else SOLVE_STEP)
    return c, meta, byte_model(n, nnz, nnzl, nnzu, v, nrhs, adjoint)


# --------------------------------------------------------------- CPU oracle
def run_oracle(c, meta, dtype, budget_s, milu=False):
    """The serial oracle on the same step (the factor in the step's
    precision, the solves in FP64); returns the seconds of every step run
    within the budget (at least one)."""
    import oracle as O
    rp, ci, v, b = c["rowptr"], c["colidx"], c["vals"], c["b"]
    diag = O.diag_ptr(rp, ci)
    odt = np.float32 if dtype == "f32" else np.float64
    times = []
    t_end = time.perf_counter() + budget_s
    while time.perf_counter() < t_end or not times:
        t0 = time.perf_counter()
        lu, _, _ = O.ilu0(rp, ci, v, diag, dtype=odt, milu=milu)
        y = O.lsolve(rp, ci, diag, lu, b)
        z = O.usolve(rp, ci, diag, lu, y)
        if meta["adjoint"]:
            gy = O.usolve_t(rp, ci, diag, lu, c["g"])
            gr = O.lsolve_t(rp, ci, diag, lu, gy)
            O.masked_outer(rp, ci, diag, 0, gr, y, alpha=-1.0)
            O.masked_outer(rp, ci, diag, 1, gy, z, alpha=-1.0)
        else:
            O.spmv(rp, ci, v, z)
        times.append(time.perf_counter() - t0)
    return times


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "c4n"],
                    help="workload (default: the 7-point 128^3 Laplacian)")
    ap.add_argument("--dtype", default=None, choices=["f64", "f32"],
                    help="factor / solve precision (default f64; f32 for c5)")
    ap.add_argument("--mode", default="syncfree", choices=["syncfree", "level", "hybrid"],
                    help="hybrid: two-stage split, wide levels one launch each")
    ap.add_argument("--er-corner", action="store_true",
                    help="Even-Rows corner: the thin tail of the factor in one CTA (needs --reorder "
                         "unless the tail is already the last rows)")
    ap.add_argument("--stage-min-rows", type=int, default=0,
                    help="stage test: levels with fewer rows are second-stage (0: 1024)")
    ap.add_argument("--reorder", action="store_true")
    ap.add_argument("--band-rows", type=int, default=0, help="sync-free band size (0: none)")
    ap.add_argument("--milu", action="store_true", help="modified ILU(0) factor")
    ap.add_argument("--exact", action="store_true",
                    help="every FP64 result bit for bit the serial algorithm's (divisions, "
                         "serial sums of long rows)")
    ap.add_argument("--sym-levels", action="store_true", help="levels of lower(A + A^T)")
    ap.add_argument("--fill-level", type=int, default=0,
                    help="ILU(k): factor on the level-k fill pattern (symbolic phase timed apart)")
    ap.add_argument("--scale", type=int, default=None, help="smaller grid (testing only)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-krylov", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    a = ap.parse_args(argv)
    if a.dtype is None:
        a.dtype = "f32" if a.config == "c5" else "f64"
    return a


def main(argv=None):
    a = parse_args(argv)
    assert a.warmup >= 3 or a.scale, "at least 3 warm-up steps"

    rank, world = dist_setup(a.gpus)
    c, meta, model = load_workload(a.config, a.scale, a.dtype)
    symbolic_ms = None
    if a.fill_level:
        # ILU(k): the step runs on the filled pattern, A's values scattered on
        # it (zeros on the fill); the symbolic phase is setup, timed apart
        if a.impl == "reference":
            import oracle as O
            frp, fci, _ = O.iluk_pattern(c["rowptr"], c["colidx"], a.fill_level)
            fv = O.scatter_values(c["rowptr"], c["colidx"], c["vals"], frp, fci)
        else:
            import torch
            import paper_1812_06160_gb300 as jv
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            rp0 = torch.tensor(c["rowptr"], device="cuda")
            ci0 = torch.tensor(c["colidx"], device="cuda")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            frp_d, fci_d = jv.jv_iluk_symbolic(rp0, ci0, a.fill_level)
            e1.record()
            torch.cuda.synchronize()
            symbolic_ms = e0.elapsed_time(e1)
            fv = jv.jv_scatter_values(rp0, ci0, torch.tensor(c["vals"], device="cuda"), frp_d,
                                      fci_d).cpu().numpy()
            frp, fci = frp_d.cpu().numpy(), fci_d.cpu().numpy()
        c = dict(c, rowptr=frp, colidx=fci, vals=fv, name=f"{c['name']} ILU({a.fill_level})")
        c, meta, model = workload_meta(c, a.dtype)
    n, nnz, nrhs, kernels = meta["n"], meta["nnz"], meta["nrhs"], meta["kernels"]
    step_bytes = sum(model.values())
    workload = f"{c['name']} natural-order" + (" level-reordered" if a.reorder else "")
    config = {"workload": workload, "n": n, "nnz": nnz, "nrhs": nrhs, "mode": a.mode,
              "reorder": a.reorder, "step": " + ".join(kernels),
              "l2": "flushed before every step", "parallelism": f"replicas x{world}"}
    if a.band_rows:
        config["band_rows"] = a.band_rows
    if a.milu:
        config["factor"] = "MILU(0)"
    if a.exact:
        config["arithmetic"] = "exact (serial order, divisions)"
    if a.sym_levels:
        config["levels"] = "lower(A+A^T)"
    if a.er_corner:
        config["factor_second_stage"] = "Even-Rows corner"
    if a.stage_min_rows:
        config["stage_min_rows"] = a.stage_min_rows
    if a.fill_level:
        config["fill_level"] = a.fill_level
        if symbolic_ms is not None:
            config["iluk_symbolic_ms"] = symbolic_ms

    if a.impl == "reference":
        if rank != 0:
            return
        times = run_oracle(c, meta, a.dtype, max(a.cpu_budget, 1.0) if a.steps else 1.0, a.milu)
        med = statistics.median(times)
        val = step_bytes / med / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": a.gpus,
                "steps": len(times), "warmup": 0, "ms_per_step": med * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": a.dtype,
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
    dt = torch.float64 if a.dtype == "f64" else torch.float32
    rp = torch.tensor(c["rowptr"], device=dev)
    ci = torch.tensor(c["colidx"], device=dev)
    h = jv.jv_analyze(rp, ci, mode=a.mode, reorder=a.reorder, check=False,
                      band_rows=a.band_rows, milu=a.milu, sym_levels=a.sym_levels,
                      er_corner=a.er_corner, stage_min_rows=a.stage_min_rows, exact=a.exact)
    info = jv.jv_get_info(h)
    # level statistics of the factor's DAG and of the U solve's
    for which in ("L", "U"):
        nl, lptr, _, _ = jv.jv_get_levels(h, which)
        w = np.diff(lptr.cpu().numpy())
        config[f"levels_{which}"] = {"n": int(nl), "narrowest": int(w.min()), "widest": int(w.max()),
                                     "median": float(np.median(w))}
    if a.er_corner:
        t = 0 if a.dtype == "f64" else 1
        config["corner_rows"] = info["corner_rows"][t]
        config["corner_levels"] = info["corner_levels"][t]
    if a.mode == "hybrid":
        config["hybrid_launches"] = {"factor": info["hybrid_launches_factor"],
                                     "solves": info["hybrid_launches"]}

    # device buffers of one step; `inputs` are what the e2e run copies in,
    # `outputs` what it copies back
    vals = torch.tensor(c["vals"], device=dev).to(dt)
    rhs = torch.tensor(c["b"], device=dev).to(dt)
    g_in = torch.tensor(c["g"], device=dev).to(dt) if meta["adjoint"] else None
    if a.reorder:
        vals = jv.jv_permute_values(h, vals)
        rhs = jv.jv_permute_vector(h, rhs)
        if g_in is not None:
            g_in = jv.jv_permute_vector(h, g_in)
    lu = torch.empty_like(vals)
    y = torch.empty_like(rhs)
    z = torch.empty_like(rhs)
    # one set of step buffers: the inputs the e2e run copies in, the outputs it
    # copies back, and the intermediates (shared by the sets: the kernels run
    # in order on one stream)
    if meta["adjoint"]:
        gy = torch.empty_like(rhs)
        B0 = {"lu": lu, "y": y, "z": z, "gy": gy, "vals": vals, "rhs": rhs, "g_in": g_in,
              "gr": torch.empty_like(rhs), "glu": torch.zeros_like(vals)}
        in_names, out_names = ["vals", "rhs", "g_in"], ["gr", "glu"]
    else:
        B0 = {"lu": lu, "y": y, "vals": vals, "rhs": rhs, "z": z,
              "s": torch.empty(n, dtype=dt, device=dev)}
        in_names, out_names = ["vals", "rhs"], ["z", "s"]
    inputs = [B0[k] for k in in_names]
    outputs = [B0[k] for k in out_names]

    def run_kernel(k, B=B0):
        if k == "factor":
            jv.jv_ilu0_factor(h, B["vals"], B["lu"])
        elif k == "lsolve":
            jv.jv_lsolve(h, B["lu"], B["rhs"], B["y"])
        elif k == "usolve":
            jv.jv_usolve(h, B["lu"], B["y"], B["z"])
        elif k == "spmv":
            jv.jv_spmv(h, B["vals"], B["z"], B["s"])
        elif k == "usolve_t":
            jv.jv_usolve_t(h, B["lu"], B["g_in"], B["gy"])
        elif k == "lsolve_t":
            jv.jv_lsolve_t(h, B["lu"], B["gy"], B["gr"])
        else:  # outer
            jv.jv_masked_outer(h, 0, B["gr"], B["y"], alpha=-1.0, g=B["glu"])
            jv.jv_masked_outer(h, 1, B["gy"], B["z"], alpha=-1.0, g=B["glu"])

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None, B=B0):
        for i, k in enumerate(kernels):
            if ev is not None:
                ev[i].record(stream)
            run_kernel(k, B)
        if ev is not None:
            ev[len(kernels)].record(stream)

    def check_status():
        st, row = jv.jv_status_sync(h)
        if st != 0:
            raise SystemExit(f"device status {st} ({jv.jv_status_string(st)}) at row {row}")

    for _ in range(a.warmup):
        flush.zero_()
        step()
    check_status()
    nk = len(kernels)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nk + 1)] for _ in range(a.steps)]
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
    check_status()
    per = {k: [] for k in kernels}
    tot = []
    for e in evs:
        for i, k in enumerate(kernels):
            per[k].append(e[i].elapsed_time(e[i + 1]))
        tot.append(e[0].elapsed_time(e[nk]))
    ms_local = sum(tot) / len(tot)
    ms = reduce_max(ms_local, world)
    value = world * step_bytes / (ms * 1e-3) / 1e9
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    dom = max(avg, key=avg.get)
    peak, peak_kind = measured_peaks()
    achieved = model[dom] / (avg[dom] * 1e-3) / 1e9
    # the captured variant only: the default factor at full size (no MILU,
    # fill, corner, band, symmetric levels, stage option or exact division)
    plain = not (a.milu or a.fill_level or a.er_corner or a.sym_levels or a.exact or
                 a.band_rows or a.scale or a.stage_min_rows)
    tr = TRAFFIC.get((a.config, a.dtype, dom, a.mode, a.reorder)) if plain else None
    traffic = tr[0] if tr and dom in KERNEL_SOURCES and tr[1] == _src_hash(KERNEL_SOURCES[dom]) \
        else None
    kern = {}
    for k in kernels:
        gbs = model[k] / (avg[k] * 1e-3) / 1e9
        kern[k] = {"ms": avg[k], "bytes": model[k], "gbs": gbs, "frac_of_peak": gbs / peak}
        if k in DAG_OF:
            nlev = info["nlev"][DAG_OF[k]]
            kern[k]["levels"] = nlev
            kern[k]["us_per_level"] = avg[k] * 1e3 / nlev

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": a.dtype, "data": "synthetic", "config": config,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                         "peak_source": peak_kind},
            "kernels": kern, "gpu_launches": launches, "clocks": clk.summary()}
    if dom in DAG_OF:
        # the second bound: one dependency hop per level on the critical path
        hop = jv.jv_hop_latency()
        nlev = info["nlev"][DAG_OF[dom]]
        line["roofline"]["critical_path"] = {
            "levels": nlev, "hop_us": hop, "floor_ms": nlev * hop * 1e-3,
            "frac": nlev * hop * 1e-3 / avg[dom]}

    if not a.no_e2e:
        host_in = [t.cpu().pin_memory() for t in inputs]
        host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outputs]

        def e2e_step():
            for d, hsrc in zip(inputs, host_in):
                d.copy_(hsrc, non_blocking=True)
            step()
            for hdst, d in zip(host_out, outputs):
                hdst.copy_(d, non_blocking=True)

        def timed(fn, k2):
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            barrier(world)
            e0.record(stream)
            fn(k2)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            check_status()
            return reduce_max(e0.elapsed_time(e1) / k2, world)

        # serial: every step copies its inputs in, runs, copies its results out
        def serial(k2):
            for _ in range(k2):
                e2e_step()

        # pipelined: while step i runs, the copy engines bring step i+1's inputs
        # in and take step i-1's results out (two input and output buffer sets;
        # every step still copies all of its inputs and results)
        B1 = dict(B0)
        for k in in_names + out_names:
            B1[k] = torch.empty_like(B0[k])
        sets = [B0, B1]
        cs_in, cs_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def pipelined(k2):
            ev = lambda: torch.cuda.Event()
            in_ready, done, out_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
            start = ev()
            start.record(stream)

            def copy_in(i):
                with torch.cuda.stream(cs_in):
                    cs_in.wait_event(start)
                    if i >= 2:
                        cs_in.wait_event(done[i % 2])     # step i-2 has read this set
                    for name, hsrc in zip(in_names, host_in):
                        sets[i % 2][name].copy_(hsrc, non_blocking=True)
                    in_ready[i % 2].record(cs_in)

            copy_in(0)
            for i in range(k2):
                if i + 1 < k2:
                    copy_in(i + 1)
                stream.wait_event(in_ready[i % 2])
                if i >= 2:
                    stream.wait_event(out_done[i % 2])     # step i-2's results are out
                step(B=sets[i % 2])
                done[i % 2].record(stream)
                with torch.cuda.stream(cs_out):
                    cs_out.wait_event(done[i % 2])
                    for hdst, name in zip(host_out, out_names):
                        hdst.copy_(sets[i % 2][name], non_blocking=True)
                    out_done[i % 2].record(cs_out)
            stream.wait_event(out_done[(k2 - 1) % 2])

        k2 = max(3, a.steps // 2)
        serial(max(2, a.warmup // 2))
        serial_ms = timed(serial, k2)
        pipelined(max(2, a.warmup // 2))
        e2e_ms = timed(pipelined, k2)
        line["e2e"] = {"value": world * step_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s",
                       "ms_per_step": e2e_ms, "pipelined": True,
                       "serial": {"value": world * step_bytes / (serial_ms * 1e-3) / 1e9,
                                  "ms_per_step": serial_ms},
                       "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in host_in),
                       "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in host_out)}

    if not a.no_krylov and not meta["adjoint"]:
        # time to a 1e-8 relative residual from b on the device, factor
        # included: all-FP64 vs FP32 factors inside the FP64 iteration
        kry = {}
        vals64 = torch.tensor(c["vals"], device=dev)
        b64 = torch.tensor(c["b"], device=dev)
        if a.reorder:
            vals64 = jv.jv_permute_values(h, vals64)
            b64 = jv.jv_permute_vector(h, b64)
        pcg = a.config in ("c1", "c2")
        for name, ldt in (("fp64", torch.float64), ("fp32_prec", torch.float32)):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            lu_k = jv.jv_ilu0_factor(h, vals64, lu_dtype=ldt)
            if pcg:
                _, kinfo = jv.jv_pcg(h, vals64, lu_k, b64, tol=1e-8)
            else:
                _, kinfo = jv.jv_fgmres(h, vals64, lu_k, b64, tol=1e-8, restart=30)
            torch.cuda.synchronize(dev)
            kry[name] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": kinfo["iters"],
                         "true_relres": kinfo["true_relres"], "converged": kinfo["converged"]}
        line["krylov_time_to_1e-8"] = {"method": "pcg" if pcg else "fgmres(30)", **kry}

    if not meta["adjoint"]:
        # FP32 factor and solves against the FP64 path (itself bit-exact with
        # the FP64 oracle in the tests): largest entrywise relative error over
        # entries above 1e-6 of the largest magnitude, and the normwise error
        import torch as _t
        vals64 = torch.tensor(c["vals"], device=dev)
        b64 = torch.tensor(c["b"], device=dev)
        if a.reorder:
            vals64 = jv.jv_permute_values(h, vals64)
            b64 = jv.jv_permute_vector(h, b64)

        def rel(x32, x64):
            x32 = x32.to(_t.float64)
            big = x64.abs() > 1e-6 * x64.abs().max()
            ent = ((x32 - x64).abs()[big] / x64.abs()[big]).max().item()
            return {"max_entry_rel": ent,
                    "normwise_rel": ((x32 - x64).abs().max() / x64.abs().max()).item()}
        l64 = jv.jv_ilu0_factor(h, vals64)
        l32 = jv.jv_ilu0_factor(h, vals64, lu_dtype=_t.float32)
        y64 = jv.jv_lsolve(h, l64, b64)
        y32 = jv.jv_lsolve(h, l32, b64.float())
        z64 = jv.jv_usolve(h, l64, y64)
        z32 = jv.jv_usolve(h, l32, y32)
        line["fp32_vs_fp64"] = {"factor": rel(l32, l64), "lsolve": rel(y32, y64),
                                "usolve": rel(z32, z64)}

    if rank == 0 and not a.no_cpu and world == 1:
        budget = a.cpu_budget
        times = run_oracle(c, meta, a.dtype, budget, a.milu)
        med = statistics.median(times)
        line["cpu_baseline"] = {"value": step_bytes / med / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(times)} full oracle steps of the same workload "
                                          f"(~{budget:.0f} s budget), median"}
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
    if "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
