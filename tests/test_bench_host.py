"""Host logic of bench.py (no GPU): the replica aggregation across ranks
(world_size 2, gloo) and the CPU reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    v = bench.whole_job_step_time(times[rank], world, "cpu")
    out.put((rank, v))
    dist.destroy_process_group()


def test_replica_step_time_is_slowest_rank_over_world():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.010, 0.014]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == pytest.approx(0.014 / 2)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_step_time(0.02, 1, "cpu") == 0.02


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "2d32",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "s/time step" and line["value"] > 0 and line["higher_is_better"] is False
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["steps"] == 2 and line["warmup"] == 1


def test_reference_arm_config_matches_ours():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2108_02054_gb300 import inputs as I
    w = I.WORKLOADS["3d192"]
    warm, timed = bench.step_indices(w, 3, 20)
    assert warm == [1, 2, 3] and timed == list(range(4, 24))
    assert bench.sampled_steps(w.T, 5, max(timed)) == [0, 1, 2, 10, 20]
    assert bench.sampled_steps(10, 9, 9) == [0, 1, 2]
    # the default oracle leg: sampled steps on the large grids, every step on the small ones
    assert bench.oracle_steps(w, -1, max(timed)) == [0, 1, 2, 10, 20]
    w64 = I.WORKLOADS["3d64"]
    assert bench.oracle_steps(w64, -1, 23) == list(range(24))
    assert bench.oracle_steps(w64, 3, 23) == [0, 1, 2]
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "2d32",
                          "--steps", "3", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    w2 = I.WORKLOADS["2d32"]
    assert line["config"] == bench.bench_config("2d32", w2, bench.step_indices(w2, 1, 3)[1])
    cb = line["cpu_baseline"]
    assert cb["os_cpu_count"] >= cb["affinity_cores"] >= 1 and cb["processes"] >= 1


def test_oracle_sample_worker_pinned_and_bounded():
    """The oracle leg's worker (spawned, pinned to one core) returns u of the
    sampled step and, per coarse level, values with their absolute-term bound."""
    sys.path.insert(0, ROOT)
    import tempfile

    import numpy as np

    import bench
    import oracle as O
    from paper_2108_02054_gb300 import inputs as I
    d = tempfile.mkdtemp()
    pool = bench._core_pool(2)
    try:
        res = pool.map(bench._oracle_sample, [("2d32", 3, d), ("2d32", 0, d)], chunksize=1)
    finally:
        pool.close()
        pool.join()
    w = I.WORKLOADS["2d32"]
    ncpu, aff = bench.cpu_cores()
    for r in res:
        assert r["status"] == 0 and r["rel_resid"] <= 1e-8
        assert (r["core"] in aff) and (len(aff) == 1 or r["core"] != aff[0])
        z = np.load(r["file"])
        ptr, col, v = O.poisson_assemble(w.dim, w.N, I.density(w.dim, w.N, r["k"], w.T))
        import scipy.sparse as sp
        A = sp.csr_matrix((v, col, ptr), shape=(w.n, w.n))
        assert np.linalg.norm(I.rhs(w.n) - A @ z["u"]) <= 1.01e-8 * np.linalg.norm(I.rhs(w.n))
        for l in range(1, r["nlevels"]):
            assert np.all(z[f"bound{l}"] >= np.abs(z[f"val{l}"]) * (1 - 1e-12))
        z.close()
        os.unlink(r["file"])
    assert res[0]["t_rebuild_s"] is not None and res[1]["t_rebuild_s"] is None
    os.rmdir(d)
