"""Host-side logic of bench.py, on the CPU: the compulsory-byte model against
the closed-form sizes of the 7-point 128^3 workload, the reference arm (the
serial oracle) on a small grid, and the multi-rank plumbing (max over ranks,
barrier, rank 0 alone prints) with two gloo ranks."""
import contextlib
import io
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def test_byte_model_closed_forms():
    m = 128
    n = m ** 3
    nnz = 7 * n - 6 * m * m                   # 7-point stencil, Dirichlet
    nnzl = (nnz - n) // 2
    b = bench.byte_model(n, nnz, nnzl, nnzl, 8)
    assert nnz == 14_581_760 and nnzl == 6_242_304
    assert round(b["spmv"] / 1e6, 1) == 216.9
    assert round(b["lsolve"] / 1e6, 1) == 133.6
    assert round(b["usolve"] / 1e6, 1) == 158.8
    assert round(b["factor"] / 1e6, 1) == 316.8
    b32 = bench.byte_model(n, nnz, nnzl, nnzl, 4)
    assert b32["factor"] == nnz * 12 + 12 * n and round(b32["spmv"] / 1e6, 1) == 141.8
    # 32 right-hand sides of the 1024^2 anisotropic 5-point problem, FP32
    m = 1024
    n = m * m
    nnz = 5 * n - 4 * m
    nnzl = (nnz - n) // 2
    b5 = bench.byte_model(n, nnz, nnzl, nnzl, 4, nrhs=32, adjoint=True)
    assert round(b5["lsolve"] / 1e6, 1) == 297.8 and round(b5["usolve"] / 1e6, 1) == 306.2
    assert set(b5) == {"factor", "lsolve", "usolve", "usolve_t", "lsolve_t", "outer"}


def _run_main(argv):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.main(argv)
    out = buf.getvalue().strip()
    return json.loads(out.splitlines()[-1]) if out else None


def test_reference_arm_small_grid():
    line = _run_main(["--impl", "reference", "--scale", "8", "--cpu-budget", "0.2"])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["n"] == 512
    line5 = _run_main(["--impl", "reference", "--config", "c5", "--scale", "16",
                       "--cpu-budget", "0.2"])
    assert line5["dtype"] == "f32" and line5["config"]["nrhs"] == 32
    assert "usolve_t" in line5["config"]["step"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    r, w = bench.dist_setup(world)
    got = bench.reduce_max(1.5 + r, w)
    bench.barrier(w)
    # the reference arm: rank 0 alone runs and prints
    line = _run_main(["--impl", "reference", "--scale", "6", "--cpu-budget", "0.1",
                      "--gpus", str(world)])
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, got, line is not None))


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert res == [(0, 2, 2.5, True), (1, 2, 2.5, False)]


if __name__ == "__main__":
    pytest.main([__file__, "-q"])
