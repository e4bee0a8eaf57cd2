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


def test_kernel_rooflines():
    """Each kernel class's achieved rate is its algorithmic work over its summed event time:
    160 B per walked segment for the walk, n^3/3 flops for the factor, the split-product MMA
    flops for the tensor-core contraction (and the ratio to the counted algorithmic flops),
    4 double-float multiply-adds per table element and vector for the apply."""
    sys.path.insert(0, ROOT)
    import bench

    peaks = {"hbm_gbs": 6757.9, "bf16_tflops": 1894.9}
    kms = {"walk_tables": (6.0, 1), "split": (1.0, 3), "contract": (1.2, 3), "factor": (26.8, 1),
           "chain": (6.0, 12), "apply": (24.0, 9)}
    cnt = {"segments": 82_230_391, "table_bytes": 16 * 134_000_000, "contract_flops": 64.9e9,
           "algorithmic_flops": 9.0e9, "apply_vectors": 51, "apply_passes": 9}
    r = bench.kernel_rooflines(kms, cnt, 12167, "bf16x3", peaks, "parallelepiped24")
    w = r["walk_tables"]
    assert w["achieved"] == pytest.approx(160 * 82_230_391 / 6.0e-3 / 1e9)
    assert w["frac"] == pytest.approx(w["achieved"] / 6757.9)
    assert w["fp64_tflops"] == pytest.approx(25 * 82_230_391 / 6.0e-3 / 1e12)
    f = r["factor"]   # blocked tensor-core factorisation at this order: TF32 split products
    assert f["bound"] == "tensor"
    assert f["achieved"] == pytest.approx(3 * 12167 ** 3 / 3 / 26.8e-3 / 1e12)
    assert f["peak"] == pytest.approx(1894.9 * 1.1 / 2.25)
    f2 = bench.kernel_rooflines(kms, cnt, 3375, "bf16x3", peaks, "cube16_jitter")["factor"]
    assert f2["bound"] == "alu"
    assert f2["achieved"] == pytest.approx(3375 ** 3 / 3 / 26.8e-3 / 1e12)
    assert f2["peak"] == pytest.approx(152 * 128 * 2 * 2.070 / 1e3)
    c = r["contract"]
    assert c["achieved"] == pytest.approx(3 * 64.9e9 / 1.2e-3 / 1e12)
    assert c["peak"] == pytest.approx(1894.9)
    assert c["executed_over_algorithmic"] == pytest.approx(3 * 64.9e9 / 9.0e9)
    a = r["apply"]
    assert a["achieved"] == pytest.approx(4 * 13 * 134e6 * 51 / 24.0e-3 / 1e12)
    assert a["peak"] == pytest.approx(152 * 128 * 2.070 / 1e3)
    # with the tables' nonzeros counted: 2 multiply-adds per nonzero of L or R and vector
    nz = bench.kernel_rooflines(kms, dict(cnt, table_nnz=150_000_000), 12167, "bf16x3", peaks,
                                "parallelepiped24")["apply"]
    assert nz["achieved"] == pytest.approx(2 * 13 * 150e6 * 51 / 24.0e-3 / 1e12)
    assert nz["nonzero_fraction_of_bin_tables"] == pytest.approx(150e6 / (2 * 134e6))
    # split: 16 B read + BF16 operands (8 B) per element, then the dense W R pair (8 B) or the
    # two list layouts (2 x 10 B per nonzero)
    assert r["split"]["achieved"] == pytest.approx((16 + 8 + 8) * 134e6 / 1.0e-3 / 1e9)
    sl = bench.kernel_rooflines(kms, dict(cnt, table_nnz=150_000_000, apply_lists=True), 12167,
                                "bf16x3", peaks, "parallelepiped24")["split"]
    assert sl["achieved"] == pytest.approx(((16 + 8) * 134e6 + 20 * 150e6) / 1.0e-3 / 1e9)
    sd = bench.kernel_rooflines(kms, dict(cnt, table_nnz=150_000_000, apply_lists=False), 12167,
                                "tf32x3", peaks, "parallelepiped24")["split"]
    assert sd["achieved"] == pytest.approx((16 + 16 + 8) * 134e6 / 1.0e-3 / 1e9)
    assert r["chain"]["launch_ms"] == pytest.approx(0.5)
    t = bench.kernel_rooflines(kms, cnt, 12167, "tf32x3", peaks, "parallelepiped24")
    assert t["contract"]["peak"] == pytest.approx(1894.9 * 1.1 / 2.25)
    s64 = bench.kernel_rooflines({"contract": (150.0, 3)}, cnt, 12167, "fp64", peaks, "x")
    assert s64["contract"]["bound"] == "alu" and s64["contract"]["peak"] == pytest.approx(
        152 * 128 * 2 * 2.070 / 1e3 / 64)


def test_measured_traffic_scales_and_expires(monkeypatch):
    """ncu traffic is scaled to the launch's units and dropped once the source changed."""
    sys.path.insert(0, ROOT)
    import bench

    sha = bench._source_sha("walk.cu")
    monkeypatch.setitem(bench.TRAFFIC, "k_walk_tables",
                        {"source": "walk.cu", "sha256": sha, "bytes": 1.0e9, "units": 1.0e7})
    assert bench.measured_traffic("k_walk_tables", 2.0e7) == pytest.approx(2.0e9)
    monkeypatch.setitem(bench.TRAFFIC, "k_walk_tables",
                        {"source": "walk.cu", "sha256": "0" * 64, "bytes": 1.0e9, "units": 1.0e7})
    assert bench.measured_traffic("k_walk_tables", 2.0e7) is None
    assert bench.measured_traffic("k_other", 1.0) is None


def test_cpu_baseline_all_core_leg(monkeypatch):
    """The all-core leg times the same sample's element sum on threads and keeps every other
    term of the one-core estimate (mesh build, load, factor, solve), on a 4^3 cube."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1811_03339_gb300 import inputs

    mesh = inputs.cube_mesh(4, 0.2, 3)
    F = inputs.random_rhs(mesh.n_nodes, 2, 5)
    r = bench.oracle_sample("cube16_jitter", mesh, F, gp_stride=2, n_chol=64, threads=2)
    n_gp = 4 * mesh.n_tets
    scale = n_gp / len(range(0, n_gp, 2))
    assert r["paths"] == 3 * n_gp
    assert r["lines_s"] > 0 and r["lines_all_s"] > 0
    assert (r["est_step_all_s"] - r["lines_all_s"] * scale
            == pytest.approx(r["est_step_s"] - r["lines_s"] * scale))
    real = bench.oracle_sample
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda w, m, f, gp_stride, n_chol, threads=0: real(w, m, f, 2, 64, threads))
    monkeypatch.setattr(bench, "_oracle_threads", lambda: 2)
    out = bench.cpu_baseline("cube16_jitter", mesh, F)
    assert out["cores"] == 1 and out["kind"] == "oracle" and out["value"] > 0
    assert out["all_cores"]["cores"] == 2 and out["all_cores"]["value"] > 0
    monkeypatch.setattr(bench, "_oracle_threads", lambda: 1)
    assert "all_cores" not in bench.cpu_baseline("cube16_jitter", mesh, F)


def test_profile_commands_parse():
    """Every bench command that a summary under profiles/ gives (the plain run and the one under
    ncu) is accepted by bench.py's own argument parser: the summaries name runnable commands."""
    import glob
    import re
    import shlex

    sys.path.insert(0, ROOT)
    import bench

    found = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read().replace("\\\n", " ")
        for m in re.finditer(r"python bench\.py([^\n`]*)", text):
            args = shlex.split(m.group(1))
            if args and args[0].startswith("`"):
                continue
            bench.build_parser().parse_args(args)
            found += 1
    assert found >= 8, found
