"""The multi-rank (replica) host logic of the benchmark, run as two gloo ranks on the CPU:
the job's time is the slowest rank's, and the job's throughput counts every rank's units.
Each rank processes its own independent lattices, so there is no data-path collective to
test; only the timing reduction crosses ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        local_ms = [120.0, 95.5][rank]
        slowest = bench.max_over_ranks(local_ms, ws)
        dist.barrier()
        rate = bench.job_rate(1000.0, ws, slowest * 1e-3)
        q.put((rank, env, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, slowest, rate in out:
        assert env == (2, rank, rank)
        assert slowest == 120.0
        assert rate == pytest.approx(2 * 1000.0 / 0.120)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_json_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and prints one JSON
    line with the GPU arm's metric, unit and config, impl = reference, a cpu_baseline of kind
    oracle and an e2e object without host-device copies (no GPU needed)."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, OMP_NUM_THREADS="4")
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-seconds", "0.3"], capture_output=True, text=True, timeout=600,
                         cwd=root, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "MLUPS"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("spinodal decomposition, 4096x4096")
    # ms_per_step is the measured oracle sample of a timed step (about --ref-seconds), the
    # full-workload figure only an extrapolation beside it
    assert 0 < d["ms_per_step"] < 60_000
    assert d["ms_per_step_extrapolated_full_workload"] > d["ms_per_step"]


def test_reference_arm_does_not_load_the_product_library():
    """The oracle leg of the benchmark takes every parameter (temperature, coexistence densities,
    sigma^Li, relaxation times) from the oracle package: after it has run, no liblbm.so is mapped
    into the process."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import bench, sys\n"
            "v, cores, sample, sec = bench.oracle_mlups(64, 0.05, crop=32)\n"
            "assert v > 0 and sec > 0\n"
            "maps = open('/proc/self/maps').read()\n"
            "assert 'liblbm_oracle.so' in maps\n"
            "sys.exit(3 if 'liblbm.so' in maps else 0)\n")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=root,
                         env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert out.returncode == 0, (out.returncode, out.stderr[-2000:])
