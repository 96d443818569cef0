"""Benchmark: full derivative evaluation of the batched polar-ACOPF workload on GB300.

One step = one `exa_eval_all` call over the whole batch: objective, dense gradient, constraints,
Jacobian and Lagrangian-Hessian values in COO and their duplicate sums in CSC (every row of the
hot path except the products, which are timed separately and reported under "extras").
Metric: Jacobian + Hessian COO nonzeros produced per second (whole job, all ranks).

Workload: 256 synthetic ACOPF instances of uneven size (buses log-uniform in [200, 20000],
branches 1.5x buses, generators buses/6, per-instance load multiplier U[0.8, 1.2]), evaluated at a
flat start plus 0.05 N(0,1), y ~ N(0,1), sigma = 1.  Inputs and outputs (about 2 GB) exceed the
129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl exa|reference] [--precision fp64|mixed]

--impl reference times the CPU oracle (the reference arm: a plain single-threaded FP64 evaluator)
on a bounded sample of the same workload.  Under torchrun each rank evaluates its own batch
(weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Jac+Hess nonzeros/sec and % of HBM roofline; FP64 vs FP32-mixed vs batched"
UNIT = "nnz/s"
WORKLOAD = "acopf_batch_256"


# ------------------------------------------------------------------ helpers shared by both arms
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def batch_seed(rank: int) -> int:
    """Each rank evaluates its own batch; rank 0's is the reference configuration."""
    return 7 + 1000 * rank


def make_batch(rank: int, n_inst: int = 256):
    import synth
    wls = synth.acopf_batch(n_inst, seed=batch_seed(rank))
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    return wls, pts


def algorithmic_bytes(flats, nnzj, nnzh, nvar, ncon, naug, nnzg, mixed=False):
    """Bytes one evaluation of every pattern must move at least: x and y read once, every data
    column read once (columns shared by several patterns count once), every COO slot, constraint
    value, augmentation term and gradient slot written once.  In mixed precision the f64 data
    columns count at 4 bytes per value (the kernel may read FP32 copies of them)."""
    data = 0
    for fl in flats:
        seen = set()
        for p in fl.patterns:
            for f in p.fields:
                key = f.__array_interface__["data"][0]
                if key not in seen:
                    seen.add(key)
                    data += f.nbytes // 2 if (mixed and f.dtype == np.float64) else f.nbytes
    return 8 * nvar + 8 * ncon + data + 8 * (nnzj + nnzh) + 8 * ncon + 8 * naug + 8 * nnzg


def reduce_max(v: float, pg, device) -> float:
    """Max over ranks (the only collective of a multi-rank run: timing, not data)."""
    if pg is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nnz_per_rank: int, world_size: int, ms_max: float) -> float:
    """Weak scaling: every rank evaluates its own batch; all ranks' nonzeros over the slowest rank."""
    return world_size * nnz_per_rank / (ms_max * 1e-3)


_T0 = time.perf_counter()


def phase(msg: str):
    """Progress of the run on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def measure_fp64_peak(B, local: int):
    """Measured FP64 FMA rate of the device (the DFMA probe of include/exa_probe.h), with the SM
    clock sampled while it runs.  DMUL and DADD issue on the same pipe at the same rate, so the
    rate bounds FP64 instructions of every kind."""
    clk = ClockSampler(local)
    clk.start()
    r = B.exa_probe_fp64_fma(local, 400.0)
    clocks = clk.stop()
    return {"g_inst_per_s": r["dfma_per_s"] / 1e9, "ms": r["ms"], "sms": r["sms"], "clocks": clocks,
            "derived_g_inst_per_s": 2 * r["sms"] * (clocks.get("sm_max_mhz") or 2070.0) / 1e3}


def csrc_digest() -> str:
    """sha256 over the sources that generate the evaluation kernels (the code generator and the
    descriptor layout): ncu counters recorded for other generated kernels are stale."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2608_16265_gb300", "csrc")
    for f in ("exa_internal.h", "exa_lower.cpp", "exa_fp64_sincos.inc"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def read_counters(precision: str, kernel: str):
    """Per-nonzero DRAM bytes and FP64 instructions of the evaluation kernel(s) `kernel` (e.g.
    "exa_all_b") from the committed ncu capture (profiles/eval_kernel_counters.json, key
    "<precision>:<kernel>"), or None when there is none or the sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "eval_kernel_counters.json")) as fh:
            d = json.load(fh)
        e = d[f"{precision}:{kernel}"]
        if e.get("csrc_sha256") != csrc_digest():
            return None
        return e
    except Exception:
        return None


# the generated kernel(s) an exa_eval_all step with every output runs (exa_stat "eval_kernel_kind")
KERNEL_KINDS = {0: "exa_all", 1: "exa_all_b", 2: "exa_first+exa_hess", 3: "exa_first+exa_hess_b"}


def step_kernel(m, nbytes, step_bytes=None):
    """Name and algorithmic bytes of the evaluation kernel(s) of the model's full step: the COO
    kernel's bytes plus, when the step forms the compressed Hessian sums, their writes, and when it
    scatters a duplicate-free CSC from the kernel (EXA_FLAG_CSC_SCATTER), those writes.  A fused
    step (EXA_FLAG_FUSED_STEP: evaluation and reductions in one kernel) moves the whole step's
    algorithmic bytes, `step_bytes`."""
    kind = int(m.stat("eval_kernel_kind"))
    if m.stat("eval_fused_step") and kind in (0, 1) and step_bytes is not None:
        return ("exa_step_b" if kind == 1 else "exa_step") + " (fused step)", step_bytes
    name, extra = KERNEL_KINDS[kind], 8 * int(m.stat("nnzh_compressed")) if kind in (1, 3) else 0
    if m.stat("csc_direct"):
        scat = [n for n, n_csc in ((m.nnzj, m.nnzj_csc), (m.nnzh, m.nnzh_csc)) if n == n_csc]
        if scat:
            extra += 8 * sum(scat)
            name += " with CSC scatter"
    return name, nbytes + extra


def live_kernel_ms(m, step, n):
    """The step's evaluation kernel(s) timed live: the library records CUDA events on the model
    stream right before and after them in every exa_eval_all step (inside its cached graph); the
    mean over n steps, each read after its step."""
    v = []
    for _ in range(n):
        step()
        t = m.stat("eval_kernel_ms")
        if t > 0:
            v.append(t)
    return float(np.mean(v)) if v else float("nan")


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        """Starts sampling and waits until the first sample has arrived."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return float("nan")

        sm = np.array([num(r[1]) for r in rows])
        smax = np.nanmax([num(r[2]) for r in rows])
        pw = np.array([num(r[3]) for r in rows])
        loaded = pw >= np.nanmedian(pw) if len(pw) > 2 else np.ones(len(pw), bool)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for j, n in enumerate(names) if any(r[5 + j].strip() == "Active" for r in rows)]
        return {"sm_mhz": float(np.nanmedian(sm[loaded])), "sm_max_mhz": float(smax), "reasons": reasons,
                "samples": len(rows), "power_w_max": float(np.nanmax(pw))}


def oracle_sample_rate(wls, pts, budget_s: float = 15.0, nnz_only: bool = False):
    """Times the CPU oracle on a bounded sample of the workload: members in a fixed seeded order
    until about budget_s of work.  Each member does what one GPU step does for it."""
    import oracle
    order = np.random.default_rng(0).permutation(len(wls))
    nnz = 0
    t_total = 0.0
    used = []
    for i in order:
        o = oracle.Oracle(wls[i].flat)
        x, y, s = pts[i]
        t0 = time.perf_counter()
        if not nnz_only:
            o.obj(x); o.grad(x); o.cons(x)
        jac = o.jac_coord(x)
        hess = o.hess_coord(x, y, s)
        if not nnz_only:
            o.jac_csc(x); o.hess_csc(x, y, s)
        t_total += time.perf_counter() - t0
        nnz += o.nnzj + o.nnzh
        used.append(int(i))
        if t_total >= budget_s:
            break
    return nnz / t_total, t_total, used, nnz


# ------------------------------------------------------------------ reference arm (CPU oracle)
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    wls, pts = make_batch(0, args.members)
    steps, warm = (args.steps if args.steps > 0 else 5), args.warmup
    # bounded per-step sample so the whole run stays within a few minutes
    per_step = max(1.0, min(20.0, 150.0 / max(1, steps + warm)))
    for _ in range(warm):
        oracle_sample_rate(wls, pts, budget_s=per_step * 0.2)
    rates, times, nnzs = [], [], []
    for _ in range(steps):
        r, t, used, nnz = oracle_sample_rate(wls, pts, budget_s=per_step)
        rates.append(r); times.append(t); nnzs.append(nnz)
    value = float(sum(nnzs) / sum(times))
    total_nnz = None
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.members == 256 else f"acopf_batch_{args.members}",
                   "members": args.members, "sample": "bounded"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step: batch members in seeded order until {per_step:.1f} s of "
                                   f"single-thread oracle work (obj, grad, cons, jac, hess, jac_csc, hess_csc)",
                         "cpu": platform.processor() or platform.machine(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ GPU arm
def pattern_counts(flats):
    """Augmentation terms and objective gradient slots are written once per instance of those
    pattern kinds (their sizes enter the algorithmic bytes)."""
    naug = sum(p.n_inst for fl in flats for p in fl.patterns if p.kind == 2)
    nobj = sum(p.n_inst for fl in flats for p in fl.patterns if p.kind == 0)
    return naug, nobj


def make_timer(torch):
    def timed(fn, k):
        """Milliseconds per call of fn over k calls, CUDA events on torch's current stream (the
        stream the binding points the library at), synchronized on both sides."""
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k
    return timed


def calls_for(timed, fn, target_ms=200.0, lo=5, hi=2000):
    """Calls that take about target_ms, from a short probe."""
    probe = timed(fn, 3)
    return int(min(hi, max(lo, target_ms / max(probe, 1e-3))))


FAMILIES = (
    # name, generator, point function, number of points (the configurations of the benchmark
    # workload family table: Rosenbrock-type at 10 points, ACOPF 500 and 30000 buses, PDE 1000^2)
    ("rosenbrock_n1000", lambda s: s.rosenbrock(1000), "rosenbrock_point", 10),
    ("acopf_b500_l700_g100", lambda s: s.acopf(500, 700, 100, seed=1), "acopf_point", 1),
    ("acopf_b30000_l45000_g5000", lambda s: s.acopf(30000, 45000, 5000, seed=2), "acopf_point", 1),
    ("pde_n1000", lambda s: s.pde(1000), "pde_point", 1),
)

SWEEP = (
    # larger members of the same families, whose working sets exceed the 129 MB L2 many times over
    ("pde_n2000", lambda s: s.pde(2000), "pde_point"),
    ("pde_n3000", lambda s: s.pde(3000), "pde_point"),
    ("pde_n4000", lambda s: s.pde(4000), "pde_point"),
    ("acopf_b100000_l150000_g16666", lambda s: s.acopf(100000, 150000, 16666, seed=3), "acopf_point"),
    ("acopf_b300000_l450000_g50000", lambda s: s.acopf(300000, 450000, 50000, seed=4), "acopf_point"),
)

L2_BYTES = 129e6


def normwise(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def measure_model(B, torch, timed, flat, pts, precision, local, peak_hbm, ref=None):
    """One model of one family in one precision: full step (every output: f, g, c, COO, CSC), the
    evaluation kernel alone (J and H COO), the paper's two callbacks (jac_coord + hess_coord), the
    kernel's algorithmic bytes and HBM fraction; with `ref` (oracle outputs at point 0), the
    normwise error of every output."""
    dev = torch.device(f"cuda:{local}")
    t0 = time.perf_counter()
    m = B.exa_create(flat, precision=precision, device=local)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    E = lambda n: torch.empty(max(int(n), 1), dtype=torch.float64, device=dev)
    outs = dict(f=E(1), g=E(m.nvar), c=E(m.ncon), jac=E(m.nnzj), hess=E(m.nnzh), jac_csc=E(m.nnzj_csc),
                hess_csc=E(m.nnzh_csc))
    xb, yb = E(m.nvar), E(m.ncon)
    step_ms, kern_ms, coo_ms, jh_ms, errs = [], [], [], [], None
    for i, (x, y, s) in enumerate(pts):  # the same buffers for every point: one cached graph each
        xb.copy_(torch.as_tensor(x))
        if len(y):
            yb.copy_(torch.as_tensor(y))
        step = lambda: m.exa_eval_all(xb, yb, s, **outs)
        kern = lambda: m.exa_eval_all(xb, yb, s, jac=outs["jac"], hess=outs["hess"])
        jh = lambda: (m.exa_jac_coord(xb, outs["jac"]), m.exa_hess_coord(xb, yb, s, outs["hess"]))
        step()
        if i == 0 and ref is not None:
            torch.cuda.synchronize()
            got = {k: v.cpu().numpy()[:n] for (k, v), n in
                   zip(outs.items(), (1, m.nvar, m.ncon, m.nnzj, m.nnzh, m.nnzj_csc, m.nnzh_csc))}
            errs = {k: (abs(float(got["f"][0]) - ref["f"]) / max(abs(ref["f"]), 1e-300) if k == "f"
                        else normwise(got[k], ref[k])) for k in got}
        step_ms.append(timed(step, calls_for(timed, step)))
        kern_ms.append(live_kernel_ms(m, step, 20))
        kern()
        coo_ms.append(timed(kern, calls_for(timed, kern)))
        jh_ms.append(timed(jh, calls_for(timed, jh)))
    naug, nobj = pattern_counts([flat])
    nbytes = algorithmic_bytes([flat], m.nnzj, m.nnzh, m.nvar, m.ncon, naug, nobj,
                               mixed=precision == B.EXA_MIXED_FP32)
    nnz = m.nnzj + m.nnzh
    kname, kbytes = step_kernel(m, nbytes)
    st, kt, jt = float(np.mean(step_ms)), float(np.mean(kern_ms)), float(np.mean(jh_ms))
    ct = float(np.mean(coo_ms))
    rec = {"nnz": nnz, "step_ms": st, "step_nnz_per_s": nnz / (st * 1e-3), "kernel": kname, "kernel_ms": kt,
           "kernel_nnz_per_s": nnz / (kt * 1e-3), "jac_plus_hess_coord_ms": jt,
           "algorithmic_bytes": kbytes, "kernel_gbs": kbytes / (kt * 1e-3) / 1e9,
           "kernel_hbm_frac": kbytes / (kt * 1e-3) / 1e9 / peak_hbm,
           "coo_kernel_ms": ct, "coo_kernel_hbm_frac": nbytes / (ct * 1e-3) / 1e9 / peak_hbm,
           "l2_resident": nbytes < L2_BYTES, "create_s": create_s, "tuned_options": m.tuned_options(),
           "eval_regs": m.stat("eval_regs")}
    if errs is not None:
        rec["rel_err_vs_oracle"] = errs
    m.destroy()
    return rec


def family_configs(B, torch, timed, local, peak_hbm, cpu_budget, sweep=False):
    """The benchmark workload families at 1 GPU, each in FP64 and mixed precision, with the
    single-thread CPU oracle timed on the same inputs (a bounded number of points)."""
    import oracle
    import synth
    res = {}
    for name, mk, ptf, npts in FAMILIES:
        phase(f"config {name}")
        wl = mk(synth)
        pts = [getattr(synth, ptf)(wl, s) for s in range(npts)]
        o = oracle.Oracle(wl.flat)
        t, n, ref = 0.0, 0, None
        while True:  # one step's callbacks per point, points in turn, until the budget
            x, y, s = pts[n % npts]
            t0 = time.perf_counter()
            r = dict(f=o.obj(x), g=o.grad(x), c=o.cons(x), jac=o.jac_coord(x), hess=o.hess_coord(x, y, s),
                     jac_csc=o.jac_csc(x), hess_csc=o.hess_csc(x, y, s))
            t += time.perf_counter() - t0
            ref = ref or r
            n += 1
            if t >= cpu_budget or n >= 1000:
                break
        nnz = o.nnzj + o.nnzh
        rec = {"nvar": o.nvar, "ncon": o.ncon, "nnzj": o.nnzj, "nnzh": o.nnzh, "nnzj_csc": o.nnzj_csc,
               "nnzh_csc": o.nnzh_csc, "points": npts,
               "oracle": {"nnz_per_s": nnz * n / t, "ms_per_step": 1e3 * t / n, "steps": n, "cores": 1,
                          "kind": "oracle"}}
        del o
        for tag, prec in (("fp64", B.EXA_FP64), ("mixed", B.EXA_MIXED_FP32)):
            rec[tag] = measure_model(B, torch, timed, wl.flat, pts, prec, local, peak_hbm, ref)
            rec[tag]["vs_oracle"] = rec[tag]["step_nnz_per_s"] / rec["oracle"]["nnz_per_s"]
        rec["note"] = ("working set below the 129 MB L2: the step is L2-resident and bound by launch "
                       "latency, not HBM" if rec["fp64"]["l2_resident"] else "working set exceeds the L2")
        res[name] = rec
    sw = {}
    if sweep:
        for name, mk, ptf in SWEEP:
            phase(f"sweep {name}")
            wl = mk(synth)
            pts = [getattr(synth, ptf)(wl, 0)]
            sw[name] = {tag: measure_model(B, torch, timed, wl.flat, pts, prec, local, peak_hbm)
                        for tag, prec in (("fp64", B.EXA_FP64), ("mixed", B.EXA_MIXED_FP32))}
            del wl
    return res, sw


def compile_sweep(args):
    """Code generation + NVRTC time and model-creation time against the number of patterns and the
    size of their trees (the analogue of the paper's experiment in its section on model compilation time): P
    constraint patterns over one variable array, pattern p a sum of K terms
    c_pj sin(x[k+j] + p) x[k+j+1]^2 + exp(x[k+j] / (p+2)) with its own constants, so every pattern
    is distinct code.  Creation is timed without the autotuner and with an empty module cache for
    the first model of each size (the second creation of the same model reuses the compiled
    module)."""
    from paper_2608_16265_gb300 import binding as B
    from paper_2608_16265_gb300.ir import Model, sin, exp
    import torch
    rows = []
    for K in (4, 16):
        for P in (1, 2, 4, 8, 16):
            mod = Model()
            n = 100000
            xv = mod.add_var(n + K + 1)
            for pidx in range(P):
                coef = [1.0 + 0.01 * (pidx * 31 + j) for j in range(K)]

                def pat(d, pidx=pidx, coef=coef):
                    e = 0
                    for j in range(K):
                        e = e + coef[j] * sin(xv[d.k + j] + pidx) * xv[d.k + j + 1] ** 2 + exp(xv[d.k + j] / (pidx + 2))
                    return e
                mod.add_con(pat, n=n)
            flat = mod.flat()
            nodes = sum(len(pp.vop) for pp in flat.patterns)
            rec = {"patterns": P, "terms_per_pattern": K, "tree_nodes_total": nodes}
            for prec, tag in ((B.EXA_FP64, "fp64"), (B.EXA_MIXED_FP32, "mixed")):
                t0 = time.perf_counter()
                B.exa_compile_check(flat, precision=prec, block=128)
                rec[f"{tag}_generate_and_nvrtc_s"] = time.perf_counter() - t0
            t0 = time.perf_counter()
            m = B.exa_create(flat, flags=B.EXA_FLAG_NO_TUNE, block=128)
            torch.cuda.synchronize()
            rec["create_s"] = time.perf_counter() - t0
            rec["create_nvrtc_ms"] = m.stat("nvrtc_ms")
            m.destroy()
            t0 = time.perf_counter()
            m = B.exa_create(flat, flags=B.EXA_FLAG_NO_TUNE, block=128)
            torch.cuda.synchronize()
            rec["create_cached_s"] = time.perf_counter() - t0
            m.destroy()
            rows.append(rec)
            phase(f"compile sweep {rec}")
    print(json.dumps({"compile_sweep": rows, "cpu": platform.processor() or platform.machine(),
                      "nproc": os.cpu_count()}))
    return 0


def run_exa(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2608_16265_gb300 import binding as B

    phase("generate batch")
    prec = B.EXA_MIXED_FP32 if args.precision == "mixed" else B.EXA_FP64
    t0 = time.perf_counter()
    if args.workload != "batch":  # profiling modes only: one model of a workload family
        import synth
        spec = {n: (mk, ptf) for n, mk, ptf, *_ in FAMILIES + SWEEP}[args.workload]
        wl = spec[0](synth)
        wls, pts = [wl], [getattr(synth, spec[1])(wl, 0)]
    else:
        wls, pts = make_batch(rank, args.members)
    flats = [w.flat for w in wls]
    t_gen = time.perf_counter() - t0
    phase("create batch model")
    t0 = time.perf_counter()
    pin = {}
    if args.pin:
        vals = [int(v) for v in args.pin.split(",")]
        b_, mb_, gf_, fl_ = vals[:4]
        pin = dict(block=b_, min_blocks=mb_, grid_factor=gf_, flags=fl_ | B.EXA_FLAG_NO_TUNE,
                   chunks=vals[4] if len(vals) > 4 else 1, wave_pct=vals[5] if len(vals) > 5 else 0)
    m = B.exa_create_batch(flats, precision=prec, device=local, **pin)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    dev = torch.device(f"cuda:{local}")
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    sigma = 1.0
    xt = torch.as_tensor(x, device=dev)
    yt = torch.as_tensor(y, device=dev)
    E = lambda n: torch.empty(n, dtype=torch.float64, device=dev)
    f, g, c = E(1), E(m.nvar), E(m.ncon)
    jac, hess, jcsc, hcsc = E(m.nnzj), E(m.nnzh), E(m.nnzj_csc), E(m.nnzh_csc)
    timed = make_timer(torch)

    def step():
        m.exa_eval_all(xt, yt, sigma, f=f, g=g, c=c, jac=jac, hess=hess, jac_csc=jcsc, hess_csc=hcsc)

    def barrier():
        if pg is not None:
            pg.barrier()

    if args.steps_only:
        # profiling mode: one untimed step, then steps_only timed steps (the launch list of a step)
        step()
        sms = timed(step, args.steps_only)
        if rank == 0:
            print(json.dumps({"profile": "steps_only", "nnz_per_rank": m.nnzj + m.nnzh, "steps": args.steps_only,
                              "ms_per_step": sms, "precision": args.precision, "members": args.members,
                              "tuned_options": ",".join(str(v) for v in m.tuned_options().values())}))
        return
    if args.kernel_only:
        # profiling mode: only the dominant call (the evaluation kernel writing J and H COO), one
        # untimed call and then kernel_only timed calls; one JSON line with the sizes
        kcall = lambda: m.exa_eval_all(xt, yt, sigma, jac=jac, hess=hess)
        kcall()
        kms = timed(kcall, args.kernel_only)
        if rank == 0:
            print(json.dumps({"profile": "kernel_only", "nnz_per_rank": m.nnzj + m.nnzh, "calls": args.kernel_only,
                              "kernel_ms": kms, "precision": args.precision, "members": args.members,
                              "tuned_options": ",".join(str(v) for v in m.tuned_options().values())}))
        return
    phase("warm-up")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.steps <= 0:  # auto: about two seconds of timed work
        probe = timed(step, 3)
        args.steps = int(min(5000, max(20, 2000.0 / max(probe, 1e-3))))
        args.steps = int(reduce_max(args.steps, pg, dev))
    phase(f"timed region: {args.steps} steps")
    barrier()
    clk = ClockSampler(local)
    clk.start()
    ms = timed(step, args.steps)
    clocks = clk.stop()
    # kernels per step: counted by the library in the captured graph of the step's exa_eval_all call
    launches_per_step = int(m.stat("graph_kernels"))
    barrier()
    ms = reduce_max(ms, pg, dev)
    nnz_rank = m.nnzj + m.nnzh
    value = whole_job_rate(nnz_rank, ws, ms)

    phase("dominant kernel and callbacks")
    # the dominant kernel, live: the step's evaluation kernel(s) between the CUDA events the library
    # records around them in every step (the last timed step's pair, then more steps read one by one)
    last_ms = m.stat("eval_kernel_ms")
    kern_ms = live_kernel_ms(m, step, max(5, min(args.steps, 100)))
    if last_ms > 0:
        kern_ms = (kern_ms * max(5, min(args.steps, 100)) + last_ms) / (max(5, min(args.steps, 100)) + 1)
    # the COO-only variant alone (exa_eval_all writing J and H, no compressed sums, no reductions)
    coo_ms = timed(lambda: m.exa_eval_all(xt, yt, sigma, jac=jac, hess=hess), max(5, min(args.steps, 200)))
    # Jacobian + Hessian callbacks alone (exa_jac_coord + exa_hess_coord)
    jh_ms = timed(lambda: (m.exa_jac_coord(xt, jac), m.exa_hess_coord(xt, yt, sigma, hess)), max(5, min(args.steps, 200)))
    naug, nobj = pattern_counts(flats)
    nbytes = algorithmic_bytes(flats, m.nnzj, m.nnzh, m.nvar, m.ncon, naug, nobj, mixed=prec == B.EXA_MIXED_FP32)
    # bytes of the whole step's outputs beyond the kernel's: the dense gradient, the CSC values
    # (each written once) and the objective
    step_bytes = nbytes + 8 * (m.nvar + m.nnzj_csc + m.nnzh_csc + 1)
    peak, peak_kind = read_peaks()
    kname, kbytes = step_kernel(m, nbytes, step_bytes)
    achieved = kbytes / (kern_ms * 1e-3) / 1e9
    ctr = read_counters(args.precision, kname)
    traffic = int(ctr["dram_bytes_per_nnz"] * nnz_rank) if ctr else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "kernel": f"{kname} (generated evaluation kernel of the step)", "algorithmic_bytes": kbytes,
                "kernel_ms": kern_ms, "kernel_timing": "CUDA events around the kernel inside the step's graph",
                "step_algorithmic_bytes": step_bytes,
                "step_hbm_frac": step_bytes / (ms * 1e-3) / 1e9 / peak,
                "coo_only_kernel_ms": coo_ms, "coo_only_algorithmic_bytes": nbytes,
                "coo_only_hbm_frac": nbytes / (coo_ms * 1e-3) / 1e9 / peak}
    phase("FP64 peak probe")
    fp64 = measure_fp64_peak(B, local)
    # write-only HBM rate (the evaluation kernels' traffic is mostly writes): a 4 GiB memset
    wbuf = torch.empty(1 << 29, dtype=torch.float64, device=dev)
    wbuf.zero_()
    hbm_write_gbs = wbuf.numel() * 8 / (timed(lambda: wbuf.zero_(), 5) * 1e-3) / 1e9
    del wbuf
    if ctr and ctr.get("fp64_inst_per_nnz"):
        # the FP64 pipe bounds this kernel when its FP64 instruction rate is the larger fraction of
        # its peak (DMUL and DADD take a pipe slot like DFMA, so instructions, not flops, are counted)
        pk = fp64["g_inst_per_s"]
        ginst = ctr["fp64_inst_per_nnz"] * nnz_rank / (kern_ms * 1e-3) / 1e9
        gflops = ctr["fp64_flops_per_nnz"] * nnz_rank / (kern_ms * 1e-3) / 1e9
        alu = {"bound": "alu", "achieved": ginst, "peak": pk, "unit": "G FP64 instructions/s",
               "frac": ginst / pk, "traffic": traffic,
               "peak_source": "measured: DFMA probe (include/exa_probe.h) in this run",
               "kernel": roofline["kernel"], "fp64_inst": int(ctr["fp64_inst_per_nnz"] * nnz_rank),
               "fp64_gflops": gflops, "fp64_gflops_frac": gflops / (2 * pk),
               "kernel_ms": kern_ms, "kernel_timing": roofline["kernel_timing"], "hbm_frac": roofline["frac"],
               "hbm_achieved_gbs": roofline["achieved"], "algorithmic_bytes": kbytes,
               "step_algorithmic_bytes": step_bytes, "step_hbm_frac": roofline["step_hbm_frac"],
               "coo_only_kernel_ms": coo_ms, "coo_only_algorithmic_bytes": nbytes,
               "coo_only_hbm_frac": roofline["coo_only_hbm_frac"]}
        if alu["frac"] > roofline["frac"]:
            roofline = alu

    extras = {"jac_plus_hess_coord_nnz_per_s": nnz_rank / (jh_ms * 1e-3), "jac_plus_hess_ms": jh_ms,
              "nnzj": m.nnzj, "nnzh": m.nnzh, "nnzj_csc": m.nnzj_csc, "nnzh_csc": m.nnzh_csc,
              "nvar": m.nvar, "ncon": m.ncon, "create_s": t_create, "generate_s": t_gen,
              "eval_regs": m.stat("eval_regs"), "eval_block": m.stat("eval_block"),
              "eval_persist": m.stat("eval_persist"), "eval_grid": m.stat("eval_grid"), "eval_tiles": m.stat("eval_tiles"),
              "eval_min_blocks": m.stat("eval_min_blocks"), "eval_split": m.stat("eval_split"),
              "csc_direct": m.stat("csc_direct"), "hess_compressed": m.stat("hess_compressed"),
              "eval_chunks": m.stat("eval_chunks"),
              "nnzh_compressed": m.stat("nnzh_compressed"), "grad_compact": m.stat("grad_compact"),
              "tuned_options": ",".join(str(v) for v in m.tuned_options().values()),
              "device_bytes": m.stat("device_bytes"), "fp64_peak": fp64,
              "hbm_write_only_gbs": hbm_write_gbs}
    if not args.no_extras:
        phase("extras: products")
        v = torch.randn(m.nvar, dtype=torch.float64, device=dev)
        w = torch.randn(m.ncon, dtype=torch.float64, device=dev)
        out_c, out_v = E(m.ncon), E(m.nvar)
        extras["jprod_ms"] = timed(lambda: m.exa_jprod(xt, v, out_c), 5)
        extras["jtprod_ms"] = timed(lambda: m.exa_jtprod(xt, w, out_v), 5)
        extras["hprod_ms"] = timed(lambda: m.exa_hprod(xt, yt, sigma, v, out_v), 5)
        # 256 per-instance models launched one after another (the unbatched form)
        # (each with the batch's tuned launch shape, fixed, so that 256 creations stay quick)
        phase("extras: per-instance models")
        tuned = m.tuned_options()
        # each single model inlines its own index constants, so each is its own NVRTC compile:
        # created from a pool of host threads (the library call releases the interpreter lock)
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
            singles = list(ex.map(lambda fl: B.exa_create(fl, precision=prec, device=local, **tuned), flats))
        xs = [torch.as_tensor(p[0], device=dev) for p in pts]
        ys = [torch.as_tensor(p[1], device=dev) for p in pts]
        outs = [(E(s.nnzj), E(s.nnzh)) for s in singles]

        def seq():
            for s_, xi, yi, (jo, ho) in zip(singles, xs, ys, outs):
                s_.exa_jac_coord(xi, jo)
                s_.exa_hess_coord(xi, yi, sigma, ho)
        seq()
        seq_ms = timed(seq, 3)
        extras["sequential_per_instance_jac_hess_ms"] = seq_ms
        extras["sequential_per_instance_nnz_per_s"] = nnz_rank / (seq_ms * 1e-3)
        for s_ in singles:
            s_.destroy()
        del singles, outs
        # the same batch in the other precision mode, timed the same way
        phase("extras: other precision")
        other = B.EXA_FP64 if prec == B.EXA_MIXED_FP32 else B.EXA_MIXED_FP32
        m2 = B.exa_create_batch(flats, precision=other, device=local)
        step2 = lambda: m2.exa_eval_all(xt, yt, sigma, f=f, g=g, c=c, jac=jac, hess=hess, jac_csc=jcsc, hess_csc=hcsc)
        step2()
        ms2 = timed(step2, max(5, min(args.steps, 200)))
        k2 = live_kernel_ms(m2, step2, max(5, min(args.steps, 100)))
        k2coo = timed(lambda: m2.exa_eval_all(xt, yt, sigma, jac=jac, hess=hess), max(5, min(args.steps, 200)))
        tag = "mixed" if other == B.EXA_MIXED_FP32 else "fp64"
        # error of the mixed outputs against the FP64 outputs on the whole batch (every member of
        # both is checked against the CPU oracle in the parity tests)
        outs = {}
        for mm in (m, m2):
            r = {k: E(n) for k, n in (("f", 1), ("g", m.nvar), ("c", m.ncon), ("jac", m.nnzj), ("hess", m.nnzh),
                                       ("jac_csc", m.nnzj_csc), ("hess_csc", m.nnzh_csc))}
            mm.exa_eval_all(xt, yt, sigma, **r)
            outs[mm is m] = r
        ref, mix = (outs[True], outs[False]) if tag == "mixed" else (outs[False], outs[True])
        extras["mixed_rel_err_vs_fp64"] = {
            k: float(torch.linalg.vector_norm(mix[k] - ref[k]) / torch.linalg.vector_norm(ref[k])) for k in ref}
        del outs, ref, mix
        extras[f"{tag}_step_ms"] = ms2
        extras[f"{tag}_nnz_per_s"] = nnz_rank / (ms2 * 1e-3)
        nbytes2 = algorithmic_bytes(flats, m.nnzj, m.nnzh, m.nvar, m.ncon, naug, nobj, mixed=tag == "mixed")
        kname2, kbytes2 = step_kernel(m2, nbytes2)
        extras[f"{tag}_kernel"] = kname2
        extras[f"{tag}_kernel_ms"] = k2
        extras[f"{tag}_kernel_hbm_frac"] = kbytes2 / (k2 * 1e-3) / 1e9 / peak
        extras[f"{tag}_algorithmic_bytes"] = kbytes2
        extras[f"{tag}_coo_kernel_ms"] = k2coo
        extras[f"{tag}_coo_kernel_hbm_frac"] = nbytes2 / (k2coo * 1e-3) / 1e9 / peak
        extras[f"{tag}_eval_regs"] = m2.stat("eval_regs")
        extras[f"{tag}_tuned_options"] = ",".join(str(v) for v in m2.tuned_options().values())
        m2.destroy()
        # two-stage stochastic ACOPF (shared generator dispatch, 256 load scenarios of a 1000-bus
        # network): the scenario axis as one more data dimension, full step in both precisions
        phase("extras: two-stage")
        import synth
        ts = synth.two_stage_acopf(1000, 1500, 166, 256, seed=11)
        tx, ty, tsig = synth.two_stage_point(ts, 0)
        txt, tyt = torch.as_tensor(tx, device=dev), torch.as_tensor(ty, device=dev)
        two = {"workload": ts.name}
        for tname, tprec in (("fp64", B.EXA_FP64), ("mixed", B.EXA_MIXED_FP32)):
            mt = B.exa_create(ts.flat, precision=tprec, device=local)
            to = {k: E(n) for k, n in (("f", 1), ("g", mt.nvar), ("c", mt.ncon), ("jac", mt.nnzj), ("hess", mt.nnzh),
                                        ("jac_csc", mt.nnzj_csc), ("hess_csc", mt.nnzh_csc))}
            tstep = lambda: mt.exa_eval_all(txt, tyt, tsig, **to)
            tstep()
            tms = timed(tstep, 50)
            two[f"{tname}_step_ms"] = tms
            two[f"{tname}_nnz_per_s"] = (mt.nnzj + mt.nnzh) / (tms * 1e-3)
            two["nnz"] = mt.nnzj + mt.nnzh
            mt.destroy()
        extras["two_stage"] = two
        # the workload families one by one (Rosenbrock-type, ACOPF 500 and 30000 buses, PDE 1000^2),
        # FP64 and mixed, the CPU oracle on the same inputs beside each
        if rank == 0:
            extras["configs"], sweep = family_configs(B, torch, timed, local, peak, args.config_cpu_budget,
                                                      sweep=args.sweep)
            if sweep:
                extras["sweep"] = sweep

    # End to end through the C ABI with host buffers (exa_eval_all_host), every step: x and y from
    # pinned host memory in, every output of the step (f, g, c, Jacobian and Hessian COO and CSC
    # values) back to pinned host memory; the call returns when they are there.
    phase("end to end")
    xh = torch.as_tensor(x).pin_memory()
    yh = torch.as_tensor(y).pin_memory()
    PH = lambda n: torch.empty(n, dtype=torch.float64).pin_memory()
    host = dict(f=PH(1), g=PH(m.nvar), c=PH(m.ncon), jac=PH(m.nnzj), hess=PH(m.nnzh), jac_csc=PH(m.nnzj_csc),
                hess_csc=PH(m.nnzh_csc))

    def e2e_step():
        m.exa_eval_all_host(xh, yh, sigma, **host)

    for _ in range(2):
        e2e_step()
    e2e_ms = timed(e2e_step, max(3, min(args.steps // 2, 100)))
    e2e_ms = reduce_max(e2e_ms, pg, dev)
    d2h = sum(t.numel() for t in host.values()) * 8
    h2d = int(xh.numel() * 8 + yh.numel() * 8)
    # the same host buffers filled by plain copies from the device outputs, one at a time: the
    # rate the host link gives into these very buffers (their pages may sit on either host node)
    srcs = dict(f=f, g=g, c=c, jac=jac, hess=hess, jac_csc=jcsc, hess_csc=hcsc)
    buf_gbs = {k: host[k].numel() * 8 / (timed(lambda k=k: host[k].copy_(srcs[k], non_blocking=True), 3) * 1e-3) / 1e9
               for k in ("jac", "hess", "jac_csc")}
    numa = sorted(n for n in os.listdir("/sys/devices/system/node") if n.startswith("node")) \
        if os.path.isdir("/sys/devices/system/node") else []
    e2e_diag = {"d2h_gbs_into_e2e_buffers": buf_gbs, "buffers_pinned": all(t.is_pinned() for t in host.values()),
                "cpu_affinity": len(os.sched_getaffinity(0)), "numa_nodes": numa}
    # the host link that bounds this step, measured (include/exa_probe.h)
    link = B.exa_probe_host_link(local, 1 << 30)
    link_ms = 1e3 * (h2d / link["h2d_bytes_per_s"] + d2h / link["d2h_bytes_per_s"])
    # the same call with only f, g and c coming back (the derivative arrays left on the device)
    fgc = dict(f=host["f"], g=host["g"], c=host["c"])
    e2e_fgc = lambda: m.exa_eval_all_host(xh, yh, sigma, jac=jac, hess=hess, jac_csc=jcsc, hess_csc=hcsc, **fgc)
    e2e_fgc()
    extras["e2e_derivatives_on_device_ms"] = timed(e2e_fgc, max(3, min(args.steps // 2, 100)))
    # the same step without the member-chunk pipeline of exa_eval_all_host (all inputs in, the
    # graph, then all outputs back), on a model created with the same launch configuration
    opts = m.tuned_options()
    opts["flags"] |= B.EXA_FLAG_HOST_SERIAL
    ms_serial = B.exa_create_batch(flats, precision=prec, device=local, **opts)
    e2e_serial = lambda: ms_serial.exa_eval_all_host(xh, yh, sigma, **host)
    e2e_serial()
    extras["e2e_serial_ms"] = timed(e2e_serial, max(3, min(args.steps // 2, 100)))
    ms_serial.destroy()
    del host

    cpu = None
    if rank == 0 and not args.no_cpu:
        phase("CPU baseline")
        rate, secs, used, _ = oracle_sample_rate(wls, pts, budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(used)} of 256 batch members in seeded order, {secs:.1f} s of single-thread "
                         f"oracle work doing one step's callbacks each",
               "cpu": platform.processor() or platform.machine(), "nproc": os.cpu_count()}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == B.EXA_FP64 else "f32+f64",
        "data": "synthetic (seeded generator; paper's suites not available)",
        "config": {"workload": WORKLOAD if args.members == 256 else f"acopf_batch_{args.members}", "members": args.members, "buses": "log-uniform 200-20000",
                   "nnz_per_rank": nnz_rank, "precision": args.precision, "parallelism": f"replicas{ws}",
                   "l2": "inputs+outputs ~2 GB per step > 129 MB L2 (no flush needed)",
                   "e2e": "x, y in and every output (f, g, c, J and H in COO and CSC) out, pinned host memory"},
        "e2e": {"value": whole_job_rate(nnz_rank, ws, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
                "link": {"h2d_gbs": link["h2d_bytes_per_s"] / 1e9, "d2h_gbs": link["d2h_bytes_per_s"] / 1e9,
                         "copy_ms": link_ms, "copy_frac_of_step": link_ms / e2e_ms,
                         "h2d_ms": 1e3 * h2d / link["h2d_bytes_per_s"], "d2h_ms": 1e3 * d2h / link["d2h_bytes_per_s"],
                         "how": "exa_probe_host_link: 1 GiB page-locked cudaMemcpyAsync each way, best of 3"},
                "diagnostics": e2e_diag},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "extras": extras,
    }
    phase("done")
    if rank == 0:
        print(json.dumps(out))
    m.destroy()
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: about two seconds of work)")
    ap.add_argument("--members", type=int, default=256, help="batch members (256 is the benchmark workload)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["exa", "reference"], default="exa")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--config-cpu-budget", type=float, default=1.5,
                    help="seconds of single-thread oracle work per workload family in extras.configs")
    ap.add_argument("--sweep", action="store_true", help="also measure the larger family members of the "
                    "supplemental roofline sweep (PDE 2000^2-4000^2, ACOPF 100k and 300k buses)")
    ap.add_argument("--steps-only", type=int, default=0, help="profiling mode: one untimed step, then this many "
                    "steps, print the step time, exit (no extras, no CPU baseline)")
    ap.add_argument("--kernel-only", type=int, default=0, help="profiling mode: run only the evaluation-kernel "
                    "call (J and H COO) this many times after one untimed call, print its sizes, exit")
    ap.add_argument("--compile-sweep", action="store_true", help="time code generation, NVRTC and model "
                    "creation against the number of patterns and their tree size; print one JSON line and exit")
    ap.add_argument("--workload", default="batch", help="profiling modes only (--steps-only, --kernel-only): "
                    "'batch' (the benchmark workload) or one model of a workload family, e.g. pde_n2000")
    ap.add_argument("--pin", default="", help="block,min_blocks,grid_factor,flags[,chunks[,wave_pct]]: fixed launch configuration "
                    "(extras.tuned_options of an earlier run) instead of autotuning, for profiling runs")
    args = ap.parse_args(argv)
    if args.workload != "batch" and not (args.steps_only or args.kernel_only):
        ap.error("--workload applies to the profiling modes (--steps-only, --kernel-only)")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.compile_sweep:
        return compile_sweep(args)
    return run_exa(args)


if __name__ == "__main__":
    sys.exit(main())
