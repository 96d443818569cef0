"""Mixed FP32/FP64 mode (EXA_MIXED_FP32) against the FP64 oracle.

Pattern arithmetic runs in FP32; x, y and data are loaded in FP64, trig/exp arguments are formed
and reduced in FP64, all cross-instance sums and the outputs are FP64.  Target: 1e-6 relative,
normwise per output; the objective scalar too, whose terms are evaluated in FP64 (terms of opposite
sign cancel in the sum, so FP32 terms would leave it far less accurate than each term).
The errors each case reaches are printed (pytest -s)."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import all_ops_model, all_ops_point, flow_collision_model, flow_collision_point, more_ops_model, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TARGET = 1e-6


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda")


CASES = {
    "all_ops": lambda: (all_ops_model().flat(), all_ops_point()),
    "flow_collisions": lambda: (flow_collision_model().flat(), flow_collision_point()),
    "more_ops": lambda: (more_ops_model().flat(), (np.random.default_rng(2).uniform(0.2, 0.9, 6),
                                                   np.random.default_rng(3).standard_normal(10), 1.3)),
    "rosenbrock_1000": lambda: (lambda w: (w.flat, synth.rosenbrock_point(w, 0)))(synth.rosenbrock(1000)),
    "acopf_small": lambda: (lambda w: (w.flat, synth.acopf_point(w, 0)))(synth.acopf(500, 700, 100, seed=1)),
    "pde_41": lambda: (lambda w: (w.flat, synth.pde_point(w, 2)))(synth.pde(41)),
    "goddard_2000": lambda: (lambda w: (w.flat, synth.goddard_point(w, 2)))(synth.goddard(2000)),
    "two_stage_acopf": lambda: (lambda w: (w.flat, synth.two_stage_point(w, 2)))(synth.two_stage_acopf(120, 180, 20, 8, seed=4)),
}


@pytest.mark.parametrize("variant", ["tuned", "lanes2", "lazy", "stage"])
@pytest.mark.parametrize("name", list(CASES))
def test_mixed_parity(name, variant):
    from paper_2608_16265_gb300 import binding as B
    flat, (x, y, s) = CASES[name]()
    o = oracle.Oracle(flat)
    extra = {"tuned": {}, "lanes2": dict(flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_LANES2, block=128),
             "lazy": dict(flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_LAZY_LOADS, block=128, min_blocks=8),
             "stage": dict(flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_STAGE_SMEM | B.EXA_FLAG_LAZY_LOADS, block=64,
                           grid_factor=2)}[variant]
    m = B.exa_create(flat, precision=B.EXA_MIXED_FP32, **extra)
    out = m.eval_all(_t(x), _t(y if len(y) else np.zeros(1)), s, csc=True)
    ref = dict(g=o.grad(x), c=o.cons(x), jac=o.jac_coord(x), hess=o.hess_coord(x, y, s),
               jac_csc=o.jac_csc(x), hess_csc=o.hess_csc(x, y, s))
    errs = {k: normwise(out[k].cpu().numpy(), v) for k, v in ref.items()}
    fo = o.obj(x)
    errs["f"] = abs(float(out["f"].item()) - fo) / max(abs(fo), 1e-300)
    print(name, {k: float(f"{v:.2e}") for k, v in errs.items()})
    # structures are the same as in FP64 mode
    r, c = m.jac_structure()
    ro, co = o.jac_structure()
    assert np.array_equal(r.cpu().numpy(), ro) and np.array_equal(c.cpu().numpy(), co)
    bad = {k: v for k, v in errs.items() if not v <= TARGET}
    assert not bad, bad


def test_mixed_conversions_are_exact():
    """c_k = x_k in mixed mode is the FP64 -> FP32 -> FP64 round trip of x_k; it must equal numpy's
    IEEE round-to-nearest-even conversion bit for bit, ties and special values included."""
    from paper_2608_16265_gb300 import binding as B
    from paper_2608_16265_gb300.ir import Model
    rng = np.random.default_rng(3)
    one = 1.0
    specials = [0.0, -0.0, one, -one, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24, 1 + 2.0 ** -23 + 2.0 ** -24,
                float(np.finfo(np.float32).max), 3.4028235677973366e38, 1e39, -1e39, 1e300, 1e-300,
                1.1754943508222875e-38, 1e-39, -1e-40, 1e-45, 7e-46, np.inf, -np.inf, 2.0 ** 127, 2.0 ** -126]
    vals = np.concatenate([np.array(specials), rng.standard_normal(2000) * 10.0 ** rng.uniform(-30, 30, 2000),
                           rng.uniform(-1, 1, 2000)])
    n = len(vals)
    m = Model()
    xv = m.add_var(n)
    m.add_con(lambda d: xv[d.k], n=n)
    mod = B.exa_create(m.flat(), precision=B.EXA_MIXED_FP32)
    with np.errstate(over="ignore", under="ignore"):
        want = vals.astype(np.float32).astype(np.float64)
    got = mod.cons(_t(vals)).cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), \
        [(v, g, w) for v, g, w in zip(vals, got, want) if g.tobytes() != w.tobytes()][:5]


FULL = {
    "acopf_30k": lambda: (lambda w: (w.flat, synth.acopf_point(w, 0)))(synth.acopf(30000, 45000, 5000, seed=2)),
    "pde_1000": lambda: (lambda w: (w.flat, synth.pde_point(w, 0)))(synth.pde(1000)),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", list(FULL))
def test_mixed_full_size(name):
    """The full-size configurations in mixed precision (ACOPF 30k buses / 45k branches / 5k
    generators; PDE on a 1000 x 1000 grid): every output against the FP64 oracle, each error
    printed, all within 1e-6."""
    from paper_2608_16265_gb300 import binding as B
    flat, (x, y, s) = FULL[name]()
    o = oracle.Oracle(flat)
    m = B.exa_create(flat, precision=B.EXA_MIXED_FP32)
    out = m.eval_all(_t(x), _t(y), s, csc=True)
    ref = dict(g=o.grad(x), c=o.cons(x), jac=o.jac_coord(x), hess=o.hess_coord(x, y, s),
               jac_csc=o.jac_csc(x), hess_csc=o.hess_csc(x, y, s))
    errs = {k: normwise(out[k].cpu().numpy(), v) for k, v in ref.items()}
    fo = o.obj(x)
    errs["f"] = abs(float(out["f"].item()) - fo) / max(abs(fo), 1e-300)
    print(name, "mixed vs oracle", {k: float(f"{v:.2e}") for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if not v <= TARGET}
    assert not bad, bad
