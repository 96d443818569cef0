"""Host-side logic of bench.py, without a GPU: the reference arm's JSON line (with the oracle sample
timing stubbed out), the algorithmic-byte count (shared data columns counted once, FP32 copies in
mixed precision), the naming and byte accounting of the step's evaluation kernel, the whole-job
rate of a weak-scaling run, and the format of the committed ncu counters the roofline reads."""
import contextlib
import io
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2608_16265_gb300.ir import Model  # noqa: E402


def test_reference_arm_json_line(monkeypatch):
    calls = []

    def fake_sample(wls, pts, budget_s=15.0, nnz_only=False):
        calls.append(budget_s)
        return 1.0e6, 0.5, [0, 1], 500_000  # rate, seconds, members used, nonzeros

    monkeypatch.setattr(bench, "oracle_sample_rate", fake_sample)
    monkeypatch.setattr(bench, "make_batch", lambda rank, n: ([None] * n, [None] * n))
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "2", "--warmup", "3", "--members", "4"])
    assert rc == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] == pytest.approx(1.0e6)  # all nonzeros over all seconds of the timed steps
    assert line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert len(calls) == 5 and max(calls) <= 20.0  # 3 warm-up samples and 2 timed ones, bounded


def test_algorithmic_bytes_counts_each_column_once():
    m = Model()
    x = m.add_var(6)
    n = 4
    data = dict(a=np.array([0, 1, 2, 3], np.int32), w=np.linspace(0.5, 1.5, n))
    m.add_obj(lambda d: d.w * x[d.a] ** 2, data=data)
    m.add_con(lambda d: d.w * x[d.a] + x[d.a + 1], data=data)  # the same two columns again
    fl = m.flat()
    nvar, ncon, nnzj, nnzh = 6, 4, 8, 4
    cols = data["a"].nbytes + data["w"].nbytes
    want = 8 * nvar + 8 * ncon + cols + 8 * (nnzj + nnzh) + 8 * ncon + 8 * 0 + 8 * n
    assert bench.algorithmic_bytes([fl], nnzj, nnzh, nvar, ncon, 0, n) == want
    # mixed precision: the f64 column counts at 4 bytes per value (its FP32 copy)
    want_mixed = want - data["w"].nbytes // 2
    assert bench.algorithmic_bytes([fl], nnzj, nnzh, nvar, ncon, 0, n, mixed=True) == want_mixed
    assert bench.pattern_counts([fl]) == (0, n)


class _FakeModel:
    def __init__(self, kind, nnzhc=0, direct=0, fused=0, nnzj=10, nnzj_csc=10, nnzh=20, nnzh_csc=12):
        self.s = {"eval_kernel_kind": kind, "nnzh_compressed": nnzhc, "csc_direct": direct,
                  "eval_fused_step": fused}
        self.nnzj, self.nnzj_csc, self.nnzh, self.nnzh_csc = nnzj, nnzj_csc, nnzh, nnzh_csc

    def stat(self, key):
        return self.s[key]


def test_step_kernel_names_and_bytes():
    assert bench.step_kernel(_FakeModel(0), 1000) == ("exa_all", 1000)
    assert bench.step_kernel(_FakeModel(1, nnzhc=7), 1000) == ("exa_all_b", 1000 + 56)
    assert bench.step_kernel(_FakeModel(3, nnzhc=7), 1000) == ("exa_first+exa_hess_b", 1000 + 56)
    # a duplicate-free Jacobian CSC scattered by the kernel: its writes count (the Hessian has
    # duplicates here, so it is not scattered)
    assert bench.step_kernel(_FakeModel(0, direct=1), 1000) == ("exa_all with CSC scatter", 1000 + 80)
    # the fused step moves the whole step's bytes
    assert bench.step_kernel(_FakeModel(1, nnzhc=7, fused=1), 1000, 5000) == ("exa_step_b (fused step)", 5000)


def test_whole_job_rate_is_weak_scaling():
    assert bench.whole_job_rate(1_000_000, 4, 2.0) == pytest.approx(4 * 1_000_000 / 2e-3)
    assert bench.reduce_max(3.5, None, None) == 3.5


def test_committed_counters_format():
    with open(os.path.join(ROOT, "profiles", "eval_kernel_counters.json")) as fh:
        d = json.load(fh)
    assert d
    for key, e in d.items():
        prec, kern = key.split(":")
        assert prec in ("fp64", "mixed") and kern in bench.KERNEL_KINDS.values()
        assert len(e["csrc_sha256"]) == 64 and e["nnz"] > 0
        assert 0 < e["fp64_inst_per_nnz"] < 10 and 0 < e["dram_bytes_per_nnz"] < 100
        assert "--clock-control none" in e["command"] and " -c 1 " in e["command"]
    assert bench.read_counters("fp64", "no_such_kernel") is None
