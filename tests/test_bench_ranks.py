"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2, launched like the GPU run:
torch.distributed.run on 127.0.0.1): every rank gets the slowest rank's time, the value
counts the units of all ranks, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slowest_rank_sets_the_job_time(tmp_path):
    pytest.importorskip("torch.distributed")
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import json, sys
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo")
        rank, world, _ = bench._dist_env()
        local_ms = [120.0, 200.0][rank]          # rank 1 is the slow one
        t = bench.max_over_ranks(local_ms, world)
        rate = bench.whole_job_rate(world, 1000, 4, t)
        with open({str(tmp_path)!r} + f"/rank{{rank}}.json", "w") as fh:
            json.dump({{"rank": rank, "world": world, "t": t, "rate": rate}}, fh)
        dist.destroy_process_group()
    """))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node",
           "2", "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(script)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    rows = [json.loads((tmp_path / f"rank{r}.json").read_text()) for r in range(2)]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["world"] == 2
        assert r["t"] == 200.0
        # 2 ranks x 1000 units x 4 steps in the slowest rank's 0.2 s
        assert r["rate"] == pytest.approx(2 * 1000 * 4 / 0.2)


def test_one_rank_is_the_plain_rate():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 294912, 20, 80.0) == pytest.approx(294912 * 20 / 0.08)


def test_reference_arm_runs_on_rank_zero_only():
    """A non-zero rank of `bench.py --impl reference` exits 0 at once and prints nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2"], capture_output=True, text=True, timeout=120, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_contraction_rates():
    """Executed MMA flops of the split forms (three products) over the stage time, against
    the measured BF16 peak scaled by the nominal TF32 : BF16 ratio."""
    sys.path.insert(0, ROOT)
    import bench

    peaks = {"bf16_tflops": 1934.0, "bf16_tflops_sustained": 1746.0}
    r = bench.contraction_rates(7.45e9, 0.559, "tf32x3", peaks)
    assert r["executed_mma_tflop"] == pytest.approx(3 * 7.45e9 / 1e12)
    assert r["mma_tflops"] == pytest.approx(3 * 7.45e9 / 0.559e-3 / 1e12)
    assert r["mma_peak_tflops"] == pytest.approx(1746.0 * 1.1 / 2.25)
    assert r["mma_frac"] == pytest.approx(r["mma_tflops"] / r["mma_peak_tflops"])
    b = bench.contraction_rates(7.45e9, 0.489, "bf16x3", {"bf16_tflops": 1900.0})
    assert b["mma_peak_tflops"] == pytest.approx(1900.0)
    assert bench.contraction_rates(7.45e9, 20.0, "fp64", peaks) == {"mma_tflops": None}
    assert bench.contraction_rates(7.45e9, 0.0, "tf32x3", peaks) == {"mma_tflops": None}


def test_walk_bandwidth():
    sys.path.insert(0, ROOT)
    import bench

    r = bench.walk_bandwidth(527e6, 749e6, 1.15, {"hbm_gbs": 6657.6})
    assert r["table_gbs"] == pytest.approx(527e6 / 1.15e-3 / 1e9)
    assert r["traffic_gbs"] == pytest.approx(749e6 / 1.15e-3 / 1e9)
    assert r["traffic_frac"] == pytest.approx(r["traffic_gbs"] / 6657.6)
    assert "traffic_gbs" not in bench.walk_bandwidth(527e6, None, 1.15, {"hbm_gbs": 6800.0})
    assert bench.walk_bandwidth(527e6, 749e6, 0.0, {"hbm_gbs": 6800.0}) == {"table_gbs": None}
