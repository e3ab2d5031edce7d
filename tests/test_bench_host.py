"""Host-side logic of bench.py: rank aggregation over gloo (2 processes on CPU)
and the reference arm (the CPU oracle) on a small cube."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.max_over_ranks(10.0 + 5.0 * rank, world)   # per-rank step times
    out.put((rank, got))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 15.0, 1: 15.0}   # every rank sees the slowest rank's time


def test_reference_arm_small_cube():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "3", "--workload", "mesh3d_10"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    # non-zero ranks print nothing and exit 0
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_committed_fold_profile_matches_the_kernel_source():
    """bench.py reports the fold's DRAM traffic from the committed ncu summary
    only while its recorded source hash names the current numeric.cu and
    common.cuh; the summary in the repository must be the current one."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    h = bench.kernel_source_hash("numeric.cu", "common.cuh")
    traffic = bench.profiled_traffic("numeric_kernel_mesh3d_100.md", h)
    assert traffic is not None, f"profiles/numeric_kernel_mesh3d_100.md does not name source hash {h}"
    # DRAM bytes of one launch near the algorithmic 12L + 8nnz of the cube
    algorithmic = 12 * 93_148_704 + 8 * 14_761_198
    assert 0.9 * algorithmic < traffic < 1.5 * algorithmic


def test_paper_data_sets_match_the_paper_table():
    """The benchmark's copy of the paper's data sets (§4.2): 25,000,000
    triplets each, the same parameters as the parity tests, and the paper's
    printed serial/parallel seconds (§4.3), parallel faster on every host."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import test_gpu_paper_data as pd
    assert set(bench.PAPER_DATA) == set(pd.DATA)
    for name, ((siz, nnz_row, nrep), published) in bench.PAPER_DATA.items():
        assert (siz, nnz_row, nrep) == pd.DATA[name]
        assert siz * nnz_row * nrep == 25_000_000
        assert set(published) == {"C1", "C2"}
        for host in published.values():
            assert 0 < host["parallel_s"] < host["serial_s"]
