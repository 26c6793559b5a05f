"""Host-side helpers of bench.py: the algorithmic byte counts behind the
roofline, the FP64 instruction count behind the FP64 roof, and the JSON-lines
export of the per-check metrics.  No GPU needed."""

import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import lpgen  # noqa: E402
from paper_2311_12180_gb300 import pdlp as P  # noqa: E402


def test_algorithmic_bytes_count_each_array_once():
    """k_primal: K' row starts, indices and values, the gathered y, and the
    eight n-vectors it reads or writes; k_dual: K's, the gathered x', and its
    seven m-vectors; FP32 values save 4 bytes per nonzero."""
    lp = lpgen.tiny_lp(0)
    m, n, z = lp.m, lp.n, lp.nnz
    assert bench.algorithmic_bytes(lp, "k_primal") == 4 * (n + 1) + 12 * z + 8 * m + 64 * n
    assert bench.algorithmic_bytes(lp, "k_dual") == 4 * (m + 1) + 12 * z + 8 * n + 56 * m
    assert bench.algorithmic_bytes(lp, "k_dual", 4) == bench.algorithmic_bytes(lp, "k_dual") - 4 * z
    assert bench.algorithmic_bytes(lp, "k_primal_reuse_g") == 72 * n


def test_fp64_instruction_count_follows_the_layout():
    """One FMA per stored entry (32 per warp instruction), one epilogue per
    slice (8 FP64 operations per row in k_dual, 5 in k_primal) and, per 32
    long rows, a 31-addition butterfly plus one epilogue."""
    lay = {"K_stored": 6400, "K_slices": 10, "K_long_rows": 33, "KT_stored": 3200, "KT_slices": 100,
           "KT_long_rows": 0}
    assert bench.fp64_warp_instructions(lay, "k_dual") == 6400 / 32 + 8 * 10 + (31 + 8) * 2
    assert bench.fp64_warp_instructions(lay, "k_primal") == 3200 / 32 + 5 * 100


def test_trace_export_writes_one_json_line_per_check(tmp_path):
    tr = np.zeros(3, dtype=P.CHECK_DTYPE)
    tr["k"] = [64, 128, 192]
    tr["restart"] = [4, 0, 1]
    tr["rel_gap"] = [1e-2, 5e-3, 1e-3]
    path = tmp_path / "checks.jsonl"
    bench.write_trace(str(path), tr, 1e-4, 3)
    bench.write_trace(str(path), tr[:1], 1e-6, 1)
    lines = [json.loads(s) for s in path.read_text().splitlines()]
    assert len(lines) == 4
    assert [r["k"] for r in lines] == [64, 128, 192, 64]
    assert lines[0]["restart"] == 4 and lines[2]["rel_gap"] == 1e-3
    assert lines[3]["tol"] == 1e-6 and lines[3]["checks_recorded"] == 1
    assert set(lines[0]) == {"tol", "checks_recorded", *P.CHECK_DTYPE.names}


def test_qp_workload_counts_the_diagonal_of_q():
    """The QP workload is the default LP with a diagonal quadratic objective:
    its primal step reads one more n-vector (Q's diagonal) and issues an FMA
    and a division more per row; its objective adds x'Qx/2, zero error at
    the planted optimum."""
    lp, desc = bench.make_workload("qp", seed=1, scale=0.002)
    base, _ = bench.make_workload("large", seed=1, scale=0.002)
    assert lp.qdiag is not None and lp.qdiag.shape == (lp.n,) and "QP" in desc
    assert np.array_equal(lp.val, base.val) and not np.array_equal(lp.c, base.c)
    assert bench.algorithmic_bytes(lp, "k_primal") == bench.algorithmic_bytes(base, "k_primal") + 8 * lp.n
    assert bench.algorithmic_bytes(lp, "k_dual") == bench.algorithmic_bytes(base, "k_dual")
    lay = {"KT_stored": 3200, "KT_slices": 100, "KT_long_rows": 0}
    assert bench.fp64_warp_instructions(lay, "k_primal", qp=True) == 3200 / 32 + 7 * 100
    assert bench.objective(lp, lp.x_star) == lp.obj_star
    assert bench.objective(base, base.x_star) == float(np.dot(base.c, base.x_star))


def test_clock_summary_reads_the_sampled_csv(tmp_path):
    """The clocks record of a bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active in any sample;
    malformed lines are skipped."""
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "garbage line\n"
                    "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c = bench.Clocks(0)
    c.path = str(path)
    c.proc = object()  # as if nvidia-smi had run
    s = c.summary()
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.proc = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_mlp_step_flops():
    """Six FLOPs per weight and batch row (forward product, the two backward
    products): 23.9 GFLOP for the 16-256-256-60500 network at batch 256."""
    assert bench.mlp_step_flops(16, 256, 60500, 256) == 6 * 256 * (16 * 256 + 256 * 256 + 256 * 60500)
    assert abs(bench.mlp_step_flops(16, 256, 60500, 256) / 1e9 - 23.9) < 0.01


def test_mlp_workload_line(monkeypatch, capsys):
    """The mlp workload's glue on the host, with the network replaced by a
    stand-in: 5 untimed steps, then the timed ones, and one JSON line with
    the step rate and the TFLOP/s it implies."""
    import types

    from paper_2311_12180_gb300 import _build

    calls = []

    class _Net:
        def __init__(self, din, hid, dout, max_batch):
            calls.append(("create", din, hid, dout, max_batch))

        def __enter__(self):
            return self

        def __exit__(self, *a):
            pass

        def set_params(self, p):
            calls.append(("params", p.size))

        def set_data(self, X, T):
            calls.append(("data", X.shape, T.shape))

        def train(self, idx):
            calls.append(("train", idx.shape))
            return np.linspace(1.0, 0.5, len(idx))

    monkeypatch.setattr(P, "Mlp", _Net)
    monkeypatch.setattr(_build, "build", lambda: None)
    bench.run_mlp(types.SimpleNamespace(mlp_steps=7), 0, 1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert calls[0] == ("create", 16, 256, 60500, 256) and calls[2] == ("data", (2048, 16), (2048, 60500))
    assert calls[3] == ("train", (5, 256)) and calls[4] == ("train", (7, 256))
    assert line["steps"] == 7 and line["unit"] == "steps/s" and line["value"] > 0
    assert line["tflops"] == pytest.approx(line["value"] * bench.mlp_step_flops(16, 256, 60500, 256) / 1e12)
    assert line["loss_first_last"] == [1.0, 0.5]
    bench.run_mlp(types.SimpleNamespace(mlp_steps=7), 1, 2)  # other ranks print nothing
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the contract's keys, its own metric, and e2e and
    cpu_baseline describing the same run."""
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_two_ranks_prints_once():
    """Launched as two ranks (torch.distributed.run, loopback), the reference
    arm runs on rank 0 only: one JSON line, and every rank exits 0."""
    import socket
    import subprocess

    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        port = s_.getsockname()[1]
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                          "--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["impl"] == "reference"
