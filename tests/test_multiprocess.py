"""Multi-process host logic of bench.py on the CPU (gloo, world size 2): the
job time is the slowest rank's, the whole-job rate counts every rank's
replica, and the reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [10.0, 12.5][rank]
    dist.barrier()
    worst = bench.max_over_ranks(ms, world)
    rate = bench.whole_job_rate(world, 100, worst)
    if rank == 0:
        with open(out_path, "w") as fh:
            json.dump({"worst": worst, "rate": rate}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "r.json"
    mp.spawn(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    r = json.loads(out.read_text())
    assert r["worst"] == 12.5
    assert r["rate"] == pytest.approx(2 * 100 / 0.0125)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.25, 1) == 7.25
    assert bench.whole_job_rate(1, 50, 500.0) == pytest.approx(100.0)


def _run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT="29555")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "16",
                           "--steps", "1", "--warmup", "0", "--gpus", str(world)],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)


def test_reference_arm_rank0_only():
    r1 = _run_reference(1, 2)
    assert r1.returncode == 0, r1.stderr
    assert r1.stdout.strip() == ""
    r0 = _run_reference(0, 2)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"


def _fake_sampler(lines, window):
    import bench
    s = bench.ClockSampler(0)

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class _Thread:
        def join(self, timeout=None):
            pass

    s.proc, s.t, s.lines = _Proc(), _Thread(), lines
    s.mark(*window)
    return s


CLOCK_LINES = [
    (0.5, "0, 1500, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
    (1.0, "0, 2070, 2070, 1000.0, 0x4, Not Active, Not Active, Not Active, Active"),
    (1.5, "0, 2060, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
    (3.0, "0, 900, 2070, 300.0, 0x8, Active, Not Active, Not Active, Not Active"),
]


def test_clock_summary_uses_only_the_timed_window():
    """The clocks line reports the median SM clock and the throttle reasons seen
    inside the timed region only (samples before and after it are dropped)."""
    out = _fake_sampler(CLOCK_LINES, (0.9, 2.0)).stop()
    assert out == {"sm_mhz": 2065.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}


def test_clock_summary_short_region_takes_next_sample():
    out = _fake_sampler(CLOCK_LINES, (1.01, 1.02)).stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2060.0 and out["reasons"] == []
