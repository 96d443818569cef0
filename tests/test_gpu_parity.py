"""GPU path (through the C ABI) against the CPU oracle on identical seeded inputs.

Bar: structures and CSC maps bit-exact; FP64 values within 1e-12 relative, normwise per output
array.  Sizes span several tiles with ragged tails; full-size configurations (ACOPF 30k buses,
PDE 1000^2, the 256-member batch) are compared whole, every output of every batch member."""
import copy

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import all_ops_model, all_ops_point, flow_collision_model, flow_collision_point, more_ops_model, normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _B():
    from paper_2608_16265_gb300 import binding
    return binding


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def check_model(flat, x, y, s, block=0, tol=TOL, o=None, flags=0, precision=0, grid_factor=0, min_blocks=0,
                wave_pct=0):
    B = _B()
    o = o or oracle.Oracle(flat)
    m = B.exa_create(flat, block=block, flags=flags, precision=precision, grid_factor=grid_factor,
                     min_blocks=min_blocks, wave_pct=wave_pct)
    assert (m.nvar, m.ncon, m.nnzj, m.nnzh, m.nnzj_csc, m.nnzh_csc) == \
        (o.nvar, o.ncon, o.nnzj, o.nnzh, o.nnzj_csc, o.nnzh_csc)
    # structures: bit-exact
    for got, want in ((m.jac_structure(), o.jac_structure()), (m.hess_structure(), o.hess_structure())):
        assert np.array_equal(_np(got[0]), want[0]) and np.array_equal(_np(got[1]), want[1])
    for got, want in ((m.jac_csc_structure(), o.jac_csc_structure()),
                      (m.hess_csc_structure(), o.hess_csc_structure())):
        for g_, w_ in zip(got, want):
            assert np.array_equal(_np(g_), w_)
    xt, yt = _t(x), _t(y if len(y) else np.zeros(1))
    f = float(_np(m.obj(xt))[0])
    fo = o.obj(x)
    assert abs(f - fo) <= tol * max(abs(fo), 1e-300) or f == fo
    errs = {}
    errs["grad"] = normwise(_np(m.grad(xt)), o.grad(x))
    errs["cons"] = normwise(_np(m.cons(xt)), o.cons(x))
    errs["jac"] = normwise(_np(m.jac_coord(xt)), o.jac_coord(x))
    errs["hess"] = normwise(_np(m.hess_coord(xt, yt, s)), o.hess_coord(x, y, s))
    errs["jac_csc"] = normwise(_np(m.jac_csc(xt)), o.jac_csc(x))
    errs["hess_csc"] = normwise(_np(m.hess_csc(xt, yt, s)), o.hess_csc(x, y, s))
    rng = np.random.default_rng(5)
    v = rng.standard_normal(o.nvar)
    w = rng.standard_normal(o.ncon)
    errs["jprod"] = normwise(_np(m.jprod(xt, _t(v))), o.jprod(x, v))
    errs["jtprod"] = normwise(_np(m.jtprod(xt, _t(w if len(w) else np.zeros(1)))), o.jtprod(x, w))
    errs["hprod"] = normwise(_np(m.hprod(xt, yt, s, _t(v))), o.hprod(x, y, s, v))
    allv = m.eval_all(xt, yt, s, csc=True)
    errs["all_f"] = abs(float(_np(allv["f"])[0]) - fo) / max(abs(fo), 1e-300)
    errs["all_g"] = normwise(_np(allv["g"]), o.grad(x))
    errs["all_c"] = normwise(_np(allv["c"]), o.cons(x))
    errs["all_jac"] = normwise(_np(allv["jac"]), o.jac_coord(x))
    errs["all_hess"] = normwise(_np(allv["hess"]), o.hess_coord(x, y, s))
    errs["all_jac_csc"] = normwise(_np(allv["jac_csc"]), o.jac_csc(x))
    errs["all_hess_csc"] = normwise(_np(allv["hess_csc"]), o.hess_csc(x, y, s))
    m.exa_check_status()
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad
    return m, errs


CASES = {
    "all_ops": lambda: (all_ops_model().flat(), all_ops_point()),
    "flow_collisions": lambda: (flow_collision_model().flat(), flow_collision_point()),
    "more_ops": lambda: (more_ops_model().flat(), (np.random.default_rng(2).uniform(0.2, 0.9, 6),
                                                   np.random.default_rng(3).standard_normal(10), 1.3)),
    "rosenbrock_1000": lambda: (lambda w: (w.flat, synth.rosenbrock_point(w, 0)))(synth.rosenbrock(1000)),
    "acopf_small": lambda: (lambda w: (w.flat, synth.acopf_point(w, 0)))(synth.acopf(500, 700, 100, seed=1)),
    "acopf_shunts": lambda: (lambda w: (w.flat, synth.acopf_point(w, 3)))(synth.acopf(37, 61, 9, seed=4, shunts=True)),
    "pde_41": lambda: (lambda w: (w.flat, synth.pde_point(w, 2)))(synth.pde(41)),
    "goddard_2000": lambda: (lambda w: (w.flat, synth.goddard_point(w, 2)))(synth.goddard(2000)),
    "two_stage_acopf": lambda: (lambda w: (w.flat, synth.two_stage_point(w, 2)))(synth.two_stage_acopf(120, 180, 20, 8, seed=4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_parity_small(name):
    flat, (x, y, s) = CASES[name]()
    check_model(flat, x, y, s)


@pytest.mark.parametrize("name", ["all_ops", "acopf_shunts", "pde_41"])
def test_parity_unfused(name):
    """Every pattern in its own thread (no fused groups) gives the same results."""
    flat, (x, y, s) = CASES[name]()
    check_model(flat, x, y, s, flags=_B().EXA_FLAG_NO_FUSE)


@pytest.mark.parametrize("grid_factor,pf,wave", [(1, 0, 0), (2, 0, 0), (1, 1, 0), (1, 2, 0), (-1, 2, 0), (2, 2, 0),
                                                 (1, 0, 50), (1, 2, 75)])
def test_parity_persistent_grid(grid_factor, pf, wave):
    """A persistent grid (CTAs loop over the tile list) gives the same results, with and without
    the L2 prefetch of later tiles' data columns (pf 1) and gather lines (pf 2); one CTA per tile
    (grid_factor -1) prefetches one wave of resident CTAs ahead; a grid of part of one wave
    (wave_pct) leaves room on the SMs."""
    B = _B()
    flags = {0: 0, 1: B.EXA_FLAG_PF_COLUMNS, 2: B.EXA_FLAG_PF_GATHERS}[pf]
    wl = synth.pde(600)  # ~5600 tiles of 128: more than two waves of resident CTAs
    x, y, s = synth.pde_point(wl, 1)
    m, _ = check_model(wl.flat, x, y, s, grid_factor=grid_factor, flags=flags, wave_pct=wave)
    assert m.stat("eval_prefetch") == pf and m.stat("eval_wave_pct") == wave
    if wave:
        assert m.stat("eval_grid") < m.stat("eval_tiles")
    elif grid_factor > 0:
        assert m.stat("eval_persist") == grid_factor and m.stat("eval_grid") < m.stat("eval_tiles")
    else:
        assert m.stat("eval_grid") == m.stat("eval_tiles")


def test_autotuned_model():
    """Default creation tunes block size and grid shape on models large enough to fill the GPU."""
    wl = synth.pde(300)
    x, y, s = synth.pde_point(wl, 3)
    m, _ = check_model(wl.flat, x, y, s)
    assert m.stat("eval_block") in (64, 128, 256) and m.stat("tune_ms") > 0


@pytest.mark.parametrize("choice", ["split", "scatter", "no_hcomp", "upfront", "split+scatter+no_hcomp+upfront",
                                    "lanes2", "lanes2+split+no_hcomp", "stage", "stage+split+no_hcomp+upfront"])
def test_pinned_launch_choices(choice):
    """Every choice the tuner makes, fixed through the creation options instead, gives the same
    results: first/second order split, the Jacobian CSC scattered by the evaluation kernel, the
    Hessian CSC summed from the COO slots, the up-front emission order, two warp sets per instance,
    inputs staged in shared memory, and a register cap through min_blocks."""
    B = _B()
    flags = B.EXA_FLAG_NO_TUNE
    flags |= B.EXA_FLAG_SPLIT if "split" in choice else 0
    flags |= B.EXA_FLAG_CSC_SCATTER if "scatter" in choice else 0
    flags |= B.EXA_FLAG_NO_HCOMP if "no_hcomp" in choice else 0
    flags |= B.EXA_FLAG_UPFRONT if "upfront" in choice else 0
    flags |= B.EXA_FLAG_LANES2 if "lanes2" in choice else 0
    flags |= B.EXA_FLAG_STAGE_SMEM if "stage" in choice else 0
    wl = synth.acopf(200, 300, 40, seed=8)
    x, y, s = synth.acopf_point(wl, 2)
    m, _ = check_model(wl.flat, x, y, s, flags=flags, block=64, min_blocks=12)
    assert m.stat("eval_split") == ("split" in choice)
    assert m.stat("csc_direct") == ("scatter" in choice)
    assert m.stat("hess_compressed") == ("no_hcomp" not in choice)
    assert m.stat("eval_min_blocks") == 12 and m.stat("eval_block") == 64
    assert m.stat("eval_upfront") == ("upfront" in choice)
    assert m.stat("eval_lanes") == (2 if "lanes2" in choice else 1)
    assert m.stat("eval_stage") == ("stage" in choice)


@pytest.mark.parametrize("name", ["all_ops", "flow_collisions", "more_ops", "acopf_shunts", "pde_41", "goddard_2000", "two_stage_acopf"])
def test_parity_lazy_loads(name):
    """Each pattern's inputs loaded one pattern ahead instead of at the top of the fused group (the
    third emission order the tuner searches) on every workload kind, with a register cap."""
    B = _B()
    flat, (x, y, s) = CASES[name]()
    m, _ = check_model(flat, x, y, s, flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_LAZY_LOADS, block=64, min_blocks=12)
    assert m.stat("eval_lazy") == 1


@pytest.mark.parametrize("name", ["all_ops", "flow_collisions", "more_ops", "acopf_shunts", "pde_41", "goddard_2000", "two_stage_acopf"])
def test_parity_two_warp_sets(name):
    """Two warp sets per instance (each a contiguous subset of a fused group's patterns) on every
    workload kind in FP64 (the mixed-precision tests cover the other precision), with a persistent
    grid."""
    B = _B()
    flat, (x, y, s) = CASES[name]()
    check_model(flat, x, y, s, flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_LANES2, block=128, grid_factor=1)


@pytest.mark.parametrize("name", ["all_ops", "flow_collisions", "more_ops", "acopf_shunts", "pde_41", "goddard_2000", "two_stage_acopf"])
@pytest.mark.parametrize("order", ["eager", "lazy"])
def test_parity_smem_staging(name, order):
    """The next tile's inputs staged in shared memory by cp.async (double-buffered persistent tile
    loop) on every workload kind, with the gathers loaded eagerly or one pattern ahead; a persistent
    grid of two waves so that every CTA runs several tiles, with a ragged last tile per pattern."""
    B = _B()
    flat, (x, y, s) = CASES[name]()
    flags = B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_STAGE_SMEM | (B.EXA_FLAG_LAZY_LOADS if order == "lazy" else 0)
    m, _ = check_model(flat, x, y, s, flags=flags, block=64, grid_factor=2)
    assert m.stat("eval_stage") == 1 and m.stat("eval_dsmem") > 0


@pytest.mark.parametrize("name", ["all_ops", "flow_collisions", "more_ops", "acopf_shunts", "pde_41", "goddard_2000",
                                  "two_stage_acopf"])
def test_parity_fused_step(name):
    """The fused step (one persistent kernel taking evaluation tiles and the step's reductions from
    one work queue) on every workload kind; a single model's reductions all wait for its tiles."""
    B = _B()
    flat, (x, y, s) = CASES[name]()
    m, _ = check_model(flat, x, y, s, flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_FUSED_STEP, block=64)
    assert m.stat("eval_fused_step") == 1


@pytest.mark.parametrize("extra", ["", "no_hcomp", "scatter", "lazy"])
def test_fused_step_batch(extra):
    """The fused step on a batch, whose members' reductions are queued between later members' tiles
    and wait for their own: every member against the oracle, and every output bit for bit against
    the same configuration without the fused step (the objective, whose per-CTA partials differ,
    within 1e-12); no wait may time out."""
    B = _B()
    wls = synth.acopf_batch(11, seed=5, bmin=20, bmax=300)
    flats = [w.flat for w in wls]
    flags = B.EXA_FLAG_NO_TUNE | {"": 0, "no_hcomp": B.EXA_FLAG_NO_HCOMP, "scatter": B.EXA_FLAG_CSC_SCATTER,
                                  "lazy": B.EXA_FLAG_LAZY_LOADS}[extra]
    prec = B.EXA_FP64
    ref = B.exa_create_batch(flats, block=64, flags=flags, precision=prec)
    fused = B.exa_create_batch(flats, block=64, flags=flags | B.EXA_FLAG_FUSED_STEP, precision=prec)
    assert fused.stat("eval_fused_step") == 1
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    a = ref.eval_all(_t(x), _t(y), 1.0, csc=True)
    for _ in range(2):  # the second call replays the cached graph
        b = fused.eval_all(_t(x), _t(y), 1.0, csc=True)
        fused.exa_check_status()
        for k in a:
            if k == "f":
                fa, fb = float(_np(a["f"])[0]), float(_np(b["f"])[0])
                assert abs(fa - fb) <= 1e-12 * abs(fa), (fa, fb)
            else:
                assert np.array_equal(_np(a[k]).view(np.uint64), _np(b[k]).view(np.uint64)), k
    compare_batch_members(fused, wls, pts, b, range(len(wls)), TOL)


def test_fused_step_wait_times_out_and_recovers():
    """The fused step's bounded wait, made to run out from the host: one member's tile counter
    starts one short (exa_debug_hold_step), its reductions give up after their bound, the kernel
    still finishes, exa_check_status reports EXA_E_TIMEOUT; the next call is normal and matches the
    oracle.  No fault, no hang: the wait has a poll limit."""
    B = _B()
    wls = synth.acopf_batch(4, seed=9, bmin=20, bmax=120)
    flats = [w.flat for w in wls]
    m = B.exa_create_batch(flats, block=64, flags=B.EXA_FLAG_NO_TUNE | B.EXA_FLAG_FUSED_STEP)
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    x = _t(np.concatenate([p[0] for p in pts]))
    y = _t(np.concatenate([p[1] for p in pts]))
    m.eval_all(x, y, 1.0, csc=True)
    m.exa_check_status()
    m.exa_debug_hold_step(2)
    m.eval_all(x, y, 1.0, csc=True)
    with pytest.raises(B.ExaError) as e:
        m.exa_check_status()
    assert e.value.status == B.EXA_E_TIMEOUT
    out = m.eval_all(x, y, 1.0, csc=True)
    m.exa_check_status()
    compare_batch_members(m, wls, pts, out, range(len(wls)), TOL)
    with pytest.raises(B.ExaError):
        m.exa_debug_hold_step(7)  # no such member
    single = B.exa_create(wls[0].flat, flags=B.EXA_FLAG_NO_TUNE)
    with pytest.raises(B.ExaError):
        single.exa_debug_hold_step(0)  # not a fused-step model


def test_option_conflicts_are_rejected():
    B = _B()
    flat, _ = CASES["all_ops"]()
    for kw in (dict(block=32, flags=B.EXA_FLAG_LANES2), dict(block=64, flags=B.EXA_FLAG_LANES2 | B.EXA_FLAG_PF_COLUMNS),
               dict(block=64, flags=B.EXA_FLAG_LAZY_LOADS | B.EXA_FLAG_UPFRONT),
               dict(block=64, flags=B.EXA_FLAG_STAGE_SMEM | B.EXA_FLAG_LANES2),
               dict(block=64, flags=B.EXA_FLAG_STAGE_SMEM | B.EXA_FLAG_PF_GATHERS),
               dict(block=64, flags=B.EXA_FLAG_FUSED_STEP | B.EXA_FLAG_STAGE_SMEM),
               dict(block=64, flags=B.EXA_FLAG_FUSED_STEP | B.EXA_FLAG_LANES2),
               dict(block=64, flags=B.EXA_FLAG_FUSED_STEP, precision=B.EXA_MIXED_FP32)):
        with pytest.raises(B.ExaError) as e:
            B.exa_create(flat, **kw)
        assert e.value.status == B.EXA_E_INVALID


def test_tuned_options_reproduce_the_model():
    """tuned_options() recreates the tuner's configuration without tuning; the kernels and their
    launch shapes are the same, so every output is the same bit for bit."""
    B = _B()
    wl = synth.pde(300)
    x, y, s = synth.pde_point(wl, 2)
    m1 = B.exa_create(wl.flat)
    opts = m1.tuned_options()
    m2 = B.exa_create(wl.flat, **opts)
    for key in ("eval_block", "eval_min_blocks", "eval_persist", "eval_grid", "eval_split", "csc_direct",
                "hess_compressed", "eval_regs"):
        assert m1.stat(key) == m2.stat(key), key
    xt, yt = _t(x), _t(y)
    a1, a2 = m1.eval_all(xt, yt, s, csc=True), m2.eval_all(xt, yt, s, csc=True)
    for k in a1:
        assert np.array_equal(_np(a1[k]).view(np.uint64), _np(a2[k]).view(np.uint64)), k


@pytest.mark.parametrize("block", [32, 64, 256])
def test_parity_block_sizes(block):
    wl = synth.acopf(200, 300, 40, seed=8)
    x, y, s = synth.acopf_point(wl, 1)
    check_model(wl.flat, x, y, s, block=block)


def test_rosenbrock_ten_points():
    wl = synth.rosenbrock(1000)
    o = oracle.Oracle(wl.flat)
    for seed in range(10):
        x, y, s = synth.rosenbrock_point(wl, seed)
        check_model(wl.flat, x, y, s, o=o)


def test_bounds_checked_kernels():
    """With EXA_FLAG_BOUNDS_CHECK every gather index is checked on the device; valid models give the
    same results and a clean status."""
    B = _B()
    flat, (x, y, s) = CASES["acopf_shunts"]()
    m, _ = check_model(flat, x, y, s, flags=B.EXA_FLAG_BOUNDS_CHECK)
    m.exa_check_status()


def test_acopf_ten_points():
    wl = synth.acopf(500, 700, 100, seed=1)
    o = oracle.Oracle(wl.flat)
    for seed in range(10):
        x, y, s = synth.acopf_point(wl, seed)
        check_model(wl.flat, x, y, s, o=o)


def test_empty_and_degenerate_patterns():
    from paper_2608_16265_gb300.ir import Model
    m = Model()
    x = m.add_var(5)
    m.add_obj(lambda d: x[d.k] ** 2, n=0)                       # empty objective pattern
    blk = m.add_con(lambda d: x[d.k] * x[d.k + 1], n=4)
    m.add_con_aug(blk, lambda d: (d.r, x[d.k]), data=dict(r=np.zeros(0, np.int32)))  # empty aug
    m.add_con_aug(blk, lambda d: (d.r, 3.0 * x[4]), data=dict(r=np.array([1, 1, 3], np.int32)))
    m.add_obj(lambda d: x[d.a] * x[d.b], data=dict(a=np.array([0, 2], np.int32), b=np.array([0, 3], np.int32)))
    x0 = np.array([0.5, -1.0, 2.0, 0.25, 1.5])
    check_model(m.flat(), x0, np.array([1.0, -2.0, 0.5, 3.0]), 0.7)


def test_no_constraints_and_no_objective():
    from paper_2608_16265_gb300.ir import Model, exp
    m = Model()
    x = m.add_var(300)
    m.add_obj(lambda d: exp(x[d.k]) * x[d.k + 1], n=299)
    check_model(m.flat(), np.linspace(-1, 1, 300), np.zeros(0), 1.3)
    m = Model()
    x = m.add_var(300)
    m.add_con(lambda d: exp(x[d.k]) * x[d.k + 1], n=299)
    check_model(m.flat(), np.linspace(-1, 1, 300), np.linspace(1, 2, 299), 1.0)


def test_determinism():
    wl = synth.acopf(500, 700, 100, seed=1)
    x, y, s = synth.acopf_point(wl, 0)
    m = _B().exa_create(wl.flat)
    a = m.eval_all(_t(x), _t(y), s, csc=True)
    b = m.eval_all(_t(x), _t(y), s, csc=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_create_errors():
    from paper_2608_16265_gb300.ir import Model
    B = _B()
    m = Model()
    x = m.add_var(3)
    m.add_obj(lambda d: x[d.i] ** 2, data=dict(i=np.array([0, 3], np.int32)))
    with pytest.raises(B.ExaError) as e:
        B.exa_create(m.flat())
    assert e.value.status == B.EXA_E_BOUNDS
    m = Model()
    x = m.add_var(3)
    b = m.add_con(lambda d: x[d.k], n=2)
    m.add_con_aug(b, lambda d: (d.r, x[0]), data=dict(r=np.array([2], np.int32)))
    with pytest.raises(B.ExaError) as e:
        B.exa_create(m.flat())
    assert e.value.status == B.EXA_E_BOUNDS


# ------------------------------------------------------------------ batch
def _csc_slice(colptr, rowval, vals, c0, c1, roff):
    """Columns [c0, c1) of a block-diagonal batch CSC as a stand-alone CSC (rows shifted by -roff)."""
    p0, p1 = int(colptr[c0]), int(colptr[c1])
    return colptr[c0:c1 + 1] - p0, rowval[p0:p1] - roff, vals[p0:p1], p0


def compare_batch_members(mb, wls, pts, out, members, tol, structures=True, log=None):
    """Every output of a batch evaluation against the oracle of each listed member, on that member's
    slice: COO values, constraint values, gradient, and both CSC value arrays with (when
    `structures`) their colptr/rowval/coo2csc bit-exact.  A member's variables, rows, COO slots and
    CSC columns are contiguous ranges of the batch's (members are block-diagonal).  Returns the
    worst normwise error per output."""
    worst = {}
    jcp, jrv, jmap = (_np(t) for t in mb.jac_csc_structure())
    hcp, hrv, hmap = (_np(t) for t in mb.hess_csc_structure())
    res = {k: _np(v) for k, v in out.items()}
    for i in members:
        w, (xi, yi, si) = wls[i], pts[i]
        o = oracle.Oracle(w.flat)
        xs, cs = slice(mb.xoff[i], mb.xoff[i + 1]), slice(mb.coff[i], mb.coff[i + 1])
        js, hs = slice(mb.joff[i], mb.joff[i + 1]), slice(mb.hoff[i], mb.hoff[i + 1])
        errs = {"jac": normwise(res["jac"][js], o.jac_coord(xi)),
                "hess": normwise(res["hess"][hs], o.hess_coord(xi, yi, si)),
                "c": normwise(res["c"][cs], o.cons(xi)), "g": normwise(res["g"][xs], o.grad(xi))}
        jc = _csc_slice(jcp, jrv, res["jac_csc"], mb.xoff[i], mb.xoff[i + 1], mb.coff[i])
        hc = _csc_slice(hcp, hrv, res["hess_csc"], mb.xoff[i], mb.xoff[i + 1], mb.xoff[i])
        errs["jac_csc"] = normwise(jc[2], o.jac_csc(xi))
        errs["hess_csc"] = normwise(hc[2], o.hess_csc(xi, yi, si))
        if structures:
            for (cp, rv, _, p0), (ocp, orv, omap), gmap, sl in ((jc, o.jac_csc_structure(), jmap, js),
                                                               (hc, o.hess_csc_structure(), hmap, hs)):
                assert np.array_equal(cp, ocp) and np.array_equal(rv, orv), f"member {i}: CSC structure"
                assert np.array_equal(gmap[sl] - p0, omap), f"member {i}: COO->CSC map"
        for k, e in errs.items():
            worst[k] = max(worst.get(k, 0.0), e)
        bad = {k: e for k, e in errs.items() if not e <= tol}
        assert not bad, (i, bad)
    if log is not None:
        log.update(worst)
    return worst


def batch_objective(wls, pts):
    """The batch objective from the members' oracle objectives (exactly rounded sum of them)."""
    import math
    return math.fsum(oracle.Oracle(w.flat).obj(p[0]) for w, p in zip(wls, pts))


BATCH_OPTIONS = {
    "untuned": dict(flags=2),
    # the launch configuration the benchmark's autotuner picks for the 256-member batch
    # (block 128, 8 CTAs per SM register cap, one CTA per tile, up-front emission, compressed
    # Hessian sums gathered into the CSC, one member chunk)
    "bench_tuned": dict(block=128, min_blocks=8, grid_factor=-1, flags=2 | 128, chunks=1),
    "split_scatter": dict(flags=2 | 16 | 32),
    "no_hcomp_chunks": dict(flags=2 | 64, chunks=3),
    "chunks_partial_wave_prefetch": dict(flags=2 | 512, chunks=4, wave_pct=50, block=32),
    "two_warp_sets_split": dict(flags=2 | 1024 | 16, block=128, chunks=2),
    "smem_staging_lazy_chunks": dict(flags=2 | 4096 | 2048, block=64, grid_factor=2, chunks=3),
}


@pytest.mark.parametrize("opts", list(BATCH_OPTIONS))
def test_batch_matches_members(opts):
    """Batch outputs, member by member, against the oracle: COO, CSC (values, structure, maps),
    c, g and f, in the launch configurations the tuner can pick."""
    B = _B()
    wls = synth.acopf_batch(6, seed=3, bmin=20, bmax=400)
    flats = [w.flat for w in wls]
    mb = B.exa_create_batch(flats, **BATCH_OPTIONS[opts])
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    out = mb.eval_all(_t(x), _t(y), 1.0, csc=True)
    compare_batch_members(mb, wls, pts, out, range(len(wls)), TOL)
    fo = batch_objective(wls, pts)
    assert abs(float(_np(out["f"])[0]) - fo) <= TOL * abs(fo)
    # single callbacks agree with the fused evaluation's slices
    xt, yt = _t(x), _t(y)
    for name, got in (("jac", mb.jac_coord(xt)), ("hess", mb.hess_coord(xt, yt, 1.0)), ("c", mb.cons(xt)),
                      ("g", mb.grad(xt)), ("jac_csc", mb.jac_csc(xt)), ("hess_csc", mb.hess_csc(xt, yt, 1.0))):
        assert normwise(_np(got), _np(out[name])) <= TOL, name
    assert abs(float(_np(mb.obj(xt))[0]) - fo) <= TOL * abs(fo)
    # the member alone gives bitwise the same COO values as its batch slice
    jb, hb = _np(out["jac"]), _np(out["hess"])
    for i, (w, (xi, yi, si)) in enumerate(zip(wls, pts)):
        mi = B.exa_create(w.flat, **BATCH_OPTIONS[opts])
        assert np.array_equal(_np(mi.jac_coord(_t(xi))), _np(mb.jac_coord(xt))[mb.joff[i]:mb.joff[i + 1]])
        assert np.array_equal(_np(mi.hess_coord(_t(xi), _t(yi), si)),
                              _np(mb.hess_coord(xt, yt, si))[mb.hoff[i]:mb.hoff[i + 1]])
    del jb, hb


@pytest.mark.parametrize("chunks,extra", [(2, 0), (3, 0), (5, "split"), (4, "scatter"), (4, "no_hcomp"), (11, 0)])
def test_member_chunks_match_one_pass(chunks, extra):
    """exa_eval_all over member chunks (reductions of one chunk overlapping the evaluation of the
    next) gives every output bit for bit as one pass over all members, in every kernel variant,
    through device and host buffers; and the oracle's values."""
    B = _B()
    wls = synth.acopf_batch(11, seed=5, bmin=20, bmax=600)
    flats = [w.flat for w in wls]
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    flags = B.EXA_FLAG_NO_TUNE
    flags |= {"split": B.EXA_FLAG_SPLIT, "scatter": B.EXA_FLAG_CSC_SCATTER, "no_hcomp": B.EXA_FLAG_NO_HCOMP}.get(extra, 0)
    m1 = B.exa_create_batch(flats, flags=flags, chunks=1)
    mc = B.exa_create_batch(flats, flags=flags, chunks=chunks)
    assert mc.stat("eval_chunks") == chunks
    a = m1.eval_all(_t(x), _t(y), 0.8, csc=True)
    b = mc.eval_all(_t(x), _t(y), 0.8, csc=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    host = {k: torch.empty(v.numel(), dtype=torch.float64).pin_memory() for k, v in a.items()}
    mc.exa_eval_all_host(torch.as_tensor(x).pin_memory(), torch.as_tensor(y).pin_memory(), 0.8, **host)
    for k in a:
        assert torch.equal(host[k], a[k].cpu()), k
    for i, (w, (xi, yi, si)) in enumerate(zip(wls, pts)):
        o = oracle.Oracle(w.flat)
        cs = slice(mc.coff[i], mc.coff[i + 1])
        xs = slice(mc.xoff[i], mc.xoff[i + 1])
        assert normwise(_np(b["c"])[cs], o.cons(xi)) <= TOL and normwise(_np(b["g"])[xs], o.grad(xi)) <= TOL


# ------------------------------------------------------------------ full-size configurations
@pytest.mark.slow
def test_full_acopf_large():
    wl = synth.acopf(30000, 45000, 5000, seed=2)
    x, y, s = synth.acopf_point(wl, 0)
    check_model(wl.flat, x, y, s)


@pytest.mark.slow
def test_full_pde():
    wl = synth.pde(1000)
    x, y, s = synth.pde_point(wl, 0)
    check_model(wl.flat, x, y, s)


def _full_batch(precision):
    B = _B()
    wls = synth.acopf_batch(256)
    mb = B.exa_create_batch([w.flat for w in wls], precision=precision)  # autotuned, as in the benchmark
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    out = mb.eval_all(_t(x), _t(y), 1.0, csc=True)
    torch.cuda.synchronize()
    return mb, wls, pts, out


@pytest.mark.slow
def test_full_batch_every_member():
    """The 256-member benchmark batch exactly as the benchmark creates it (autotuned launch shape):
    every output of every member against the oracle, CSC structures and maps bit-exact."""
    mb, wls, pts, out = _full_batch(0)
    worst = compare_batch_members(mb, wls, pts, out, range(len(wls)), TOL)
    fo = batch_objective(wls, pts)
    worst["f"] = abs(float(_np(out["f"])[0]) - fo) / abs(fo)
    print("fp64 batch", mb.tuned_options(), {k: float(f"{v:.2e}") for k, v in worst.items()})
    assert worst["f"] <= TOL


@pytest.mark.slow
def test_full_batch_mixed_every_member():
    """The benchmark batch in mixed precision: every output of every member against the FP64
    oracle within 1e-6 (the structures are those of the FP64 model)."""
    mb, wls, pts, out = _full_batch(_B().EXA_MIXED_FP32)
    worst = compare_batch_members(mb, wls, pts, out, range(len(wls)), 1e-6, structures=False)
    fo = batch_objective(wls, pts)
    worst["f"] = abs(float(_np(out["f"])[0]) - fo) / abs(fo)
    print("mixed batch", mb.tuned_options(), {k: float(f"{v:.2e}") for k, v in worst.items()})
    assert worst["f"] <= 1e-6


def test_eval_all_graph_replay_matches_direct_launches():
    """exa_eval_all replays a cached CUDA graph; results equal those of direct launches, also
    after switching between argument tuples and after changing x in place."""
    B = _B()
    wl = synth.acopf(200, 300, 40, seed=8)
    x, y, s = synth.acopf_point(wl, 1)
    mg = B.exa_create(wl.flat)
    md = B.exa_create(wl.flat, flags=B.EXA_FLAG_NO_GRAPH)
    xt, yt = _t(x), _t(y)
    outs = {}
    for name, m in (("graph", mg), ("direct", md)):
        res = []
        for sigma in (1.0, 0.5, 1.0):
            o = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k, n in
                 (("f", 1), ("g", m.nvar), ("c", m.ncon), ("jac", m.nnzj), ("hess", m.nnzh),
                  ("jac_csc", m.nnzj_csc), ("hess_csc", m.nnzh_csc))}
            m.exa_eval_all(xt, yt, sigma, **o)
            m.exa_eval_all(xt, yt, sigma, **o)  # second call with the same tuple replays
            res.append({k: v.clone() for k, v in o.items()})
        xt.mul_(1.01)
        m.exa_eval_all(xt, yt, 1.0, **o)
        res.append({k: v.clone() for k, v in o.items()})
        xt.copy_(_t(x))
        outs[name] = res
    for a, b in zip(outs["graph"], outs["direct"]):
        for k in a:
            assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("pinned", [True, False])
def test_eval_all_host_buffers(pinned):
    """exa_eval_all_host (host x, y in; host outputs) equals exa_eval_all on device buffers bit for
    bit, with page-locked and with pageable host memory, with host and device arguments mixed, and
    leaves unrequested outputs alone."""
    B = _B()
    wl = synth.acopf(200, 300, 40, seed=8)
    x, y, s = synth.acopf_point(wl, 3)
    m = B.exa_create(wl.flat)
    sizes = (("f", 1), ("g", m.nvar), ("c", m.ncon), ("jac", m.nnzj), ("hess", m.nnzh),
             ("jac_csc", m.nnzj_csc), ("hess_csc", m.nnzh_csc))
    dev = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k, n in sizes}
    m.exa_eval_all(_t(x), _t(y), s, **dev)
    pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
    host = {k: pin(torch.full((n,), -7.0, dtype=torch.float64)) for k, n in sizes}
    xh, yh = pin(torch.as_tensor(x)), pin(torch.as_tensor(y))
    for _ in range(2):  # the second call replays the cached graph
        m.exa_eval_all_host(xh, yh, s, **host)
        for k in host:
            assert torch.equal(host[k], dev[k].cpu()), k
    # a subset of the outputs: the same kernels as the device call with that subset (a different
    # output set may select another kernel variant, whose FMA contraction can differ in the last bit)
    part = {k: pin(torch.full((n,), -7.0, dtype=torch.float64)) for k, n in sizes}
    m.exa_eval_all_host(xh, yh, s, g=part["g"], hess_csc=part["hess_csc"])
    devp = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k, n in sizes if k in ("g", "hess_csc")}
    m.exa_eval_all(_t(x), _t(y), s, **devp)
    assert torch.equal(part["g"], devp["g"].cpu()) and torch.equal(part["hess_csc"], devp["hess_csc"].cpu())
    assert bool((part["c"] == -7.0).all()) and bool((part["jac"] == -7.0).all())
    # host and device arguments mixed: device arrays are used in place
    mix = {"g": pin(torch.full((m.nvar,), -7.0, dtype=torch.float64)),
           "hess": torch.full((m.nnzh,), -7.0, dtype=torch.float64, device="cuda")}
    m.exa_eval_all_host(_t(x), yh, s, **mix)
    devm = {"g": torch.empty(m.nvar, dtype=torch.float64, device="cuda"),
            "hess": torch.empty(m.nnzh, dtype=torch.float64, device="cuda")}
    m.exa_eval_all(_t(x), _t(y), s, **devm)
    assert torch.equal(mix["g"], devm["g"].cpu()) and torch.equal(mix["hess"], devm["hess"])


@pytest.mark.parametrize("opts", ["untuned", "bench_tuned", "two_warp_sets_split", "no_hcomp_chunks"])
def test_eval_all_host_batch_pipeline(opts):
    """exa_eval_all_host on a batch (the member-chunk pipeline: inputs copied in per chunk, each
    chunk evaluated once its inputs are in, its outputs copied back after its reductions) against
    the oracle member by member, and bit for bit against exa_eval_all on device buffers for every
    output except the objective, whose per-chunk partial sums are added in another order (1e-12);
    EXA_FLAG_HOST_SERIAL gives the graph path's results bit for bit.  Pageable inputs, a host/device
    mix and an output subset go through the pipeline too."""
    B = _B()
    wls = synth.acopf_batch(11, seed=5, bmin=20, bmax=300)
    flats = [w.flat for w in wls]
    kw = BATCH_OPTIONS[opts]
    mb = B.exa_create_batch(flats, **kw)
    pts = [synth.acopf_point(w, i) for i, w in enumerate(wls)]
    x = np.concatenate([p[0] for p in pts])
    y = np.concatenate([p[1] for p in pts])
    sizes = (("f", 1), ("g", mb.nvar), ("c", mb.ncon), ("jac", mb.nnzj), ("hess", mb.nnzh),
             ("jac_csc", mb.nnzj_csc), ("hess_csc", mb.nnzh_csc))
    dev = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k, n in sizes}
    mb.exa_eval_all(_t(x), _t(y), 1.0, **dev)
    host = {k: torch.full((n,), -7.0, dtype=torch.float64).pin_memory() for k, n in sizes}
    xh, yh = torch.as_tensor(x).pin_memory(), torch.as_tensor(y).pin_memory()
    for _ in range(2):
        mb.exa_eval_all_host(xh, yh, 1.0, **host)
        for k in host:
            if k == "f":
                assert abs(float(host["f"][0]) - float(dev["f"][0])) <= 1e-12 * abs(float(dev["f"][0]))
            else:
                assert torch.equal(host[k], dev[k].cpu()), k
    out = {k: v.cuda() for k, v in host.items()}
    compare_batch_members(mb, wls, pts, out, range(len(wls)), TOL)
    fo = batch_objective(wls, pts)
    assert abs(float(host["f"][0]) - fo) <= TOL * abs(fo)
    # the serial path (all inputs, graph, all outputs) equals the device call bit for bit
    kw_s = dict(kw)
    kw_s["flags"] = kw.get("flags", 0) | B.EXA_FLAG_HOST_SERIAL
    ms = B.exa_create_batch(flats, **kw_s)
    ser = {k: torch.full((n,), -7.0, dtype=torch.float64).pin_memory() for k, n in sizes}
    ms.exa_eval_all_host(xh, yh, 1.0, **ser)
    for k in ser:
        assert torch.equal(ser[k], dev[k].cpu()), k
    # pageable inputs, x on the device, and a subset of host outputs (the rest untouched)
    part = {"g": torch.full((mb.nvar,), -7.0, dtype=torch.float64),
            "hess_csc": torch.full((mb.nnzh_csc,), -7.0, dtype=torch.float64),
            "jac": torch.full((mb.nnzj,), -7.0, dtype=torch.float64, device="cuda")}
    mb.exa_eval_all_host(_t(x), torch.as_tensor(y), 1.0, **part)
    devp = {k: torch.empty(v.numel(), dtype=torch.float64, device="cuda") for k, v in part.items()}
    mb.exa_eval_all(_t(x), _t(y), 1.0, **devp)
    for k in part:
        assert torch.equal(part[k].cpu(), devp[k].cpu()), k


def test_two_stage_scenario_parameters():
    """Replacing one scenario's loads with exa_set_theta (the builder's single-scenario accessor)
    gives the results of a model created with those loads, bit for bit."""
    B = _B()
    wl = synth.two_stage_acopf(60, 90, 12, 6, seed=9)
    x, y, s = synth.two_stage_point(wl, 1)
    m = B.exa_create(wl.flat)
    pd = wl.meta["pd"]
    new = wl.model.scenario_theta(wl.flat.theta, pd, 3, np.linspace(0.1, 1.0, 60))
    m.exa_set_theta(new)
    flat2 = copy.copy(wl.flat)
    flat2.theta = new
    m2 = B.exa_create(flat2)
    a, b = m.eval_all(_t(x), _t(y), s, csc=True), m2.eval_all(_t(x), _t(y), s, csc=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    o = oracle.Oracle(flat2)
    assert normwise(_np(a["c"]), o.cons(x)) <= TOL


def test_set_theta():
    """Changing the parameters of a created model gives the results of a model built with them."""
    B = _B()
    flat, (x, y, s) = CASES["all_ops"]()
    m = B.exa_create(flat)
    new_theta = np.array([-0.4, 2.5])
    m.exa_set_theta(new_theta)
    flat.theta = new_theta
    o = oracle.Oracle(flat)
    xt, yt = _t(x), _t(y)
    assert abs(float(m.obj(xt).item()) - o.obj(x)) <= TOL * abs(o.obj(x))
    assert normwise(_np(m.cons(xt)), o.cons(x)) <= TOL
    assert normwise(_np(m.hess_coord(xt, yt, s)), o.hess_coord(x, y, s)) <= TOL
    with pytest.raises(B.ExaError):
        m.exa_set_theta(np.zeros(3))


def test_invalid_arguments_are_reported():
    """NULL arrays and wrong sizes come back as EXA_E_INVALID with a message; nothing is launched."""
    B = _B()
    flat, (x, y, s) = CASES["all_ops"]()
    m = B.exa_create(flat)
    xt = _t(x)
    for call in (lambda: m.exa_jac_coord(xt, None), lambda: m.exa_hess_coord(xt, None, 1.0, _t(np.zeros(m.nnzh))),
                 lambda: m.exa_obj(None, _t(np.zeros(1))), lambda: m.exa_eval_all(None, None, 1.0)):
        with pytest.raises(B.ExaError) as e:
            call()
        assert e.value.status == B.EXA_E_INVALID and "NULL" in str(e.value)
    m.exa_check_status()


def test_fp64_sin_cos_accuracy():
    """FP64 sin and cos of the generated code (Cody-Waite reduction, minimax polynomials) against
    the host C library over a sweep that includes arguments next to multiples of pi/2, signed
    zeros, tiny and large arguments (the library path beyond 2^20): within 3 ulp of the host
    values (6.7e-16 relative)."""
    from paper_2608_16265_gb300 import ir
    from paper_2608_16265_gb300.ir import Model
    B = _B()
    rng = np.random.default_rng(11)
    k = np.arange(-2000, 2001)
    near = np.concatenate([k * (np.pi / 2) + d for d in (0.0, 1e-9, -1e-12, 3e-7)])
    vals = np.concatenate([near, rng.uniform(-4, 4, 4000), rng.uniform(-1e5, 1e5, 4000),
                           10.0 ** rng.uniform(-30, 0, 500), -10.0 ** rng.uniform(-30, 0, 500),
                           rng.uniform(-3e6, 3e6, 200), [0.0, -0.0, 1048575.9, 1048576.0, 2.0 ** 30]])
    n = len(vals)
    m = Model()
    xv = m.add_var(n)
    m.add_con(lambda d: ir.sin(xv[d.k]), n=n)
    m.add_con(lambda d: ir.cos(xv[d.k]), n=n)
    mod = B.exa_create(m.flat())
    c = _np(mod.cons(_t(vals)))
    for got, want in ((c[:n], np.sin(vals)), (c[n:], np.cos(vals))):
        err = np.abs(got - want)
        ok = err <= 6.7e-16 * np.abs(want)
        assert ok.all(), [(v, g, w) for v, g, w in zip(vals[~ok], got[~ok], want[~ok])][:5]
    assert np.signbit(c[n - 4]) and not np.signbit(c[n - 5])  # sin(-0) = -0, sin(+0) = +0
    # derivatives come from the same pair: d sin = cos, d cos = -sin
    jac = _np(mod.jac_coord(_t(vals)))
    assert np.array_equal(jac[:n], c[n:]) and np.array_equal(jac[n:], -c[:n])


def test_exact_integer_pipe_negation_and_doubling():
    """FP64 negation and multiplication by 2 are done on the integer pipe in the generated code;
    they must equal IEEE -x and 2 x bit for bit: signed zeros, subnormals (including ones whose
    double is normal), the largest binade (overflow to infinity), infinities and NaN."""
    from paper_2608_16265_gb300.ir import Model
    B = _B()
    rng = np.random.default_rng(12)
    tiny = np.finfo(np.float64).tiny
    specials = [0.0, -0.0, 5e-324, -5e-324, 1e-310, -2.2e-308, tiny, -tiny, tiny / 2, tiny * (1 - 2 ** -52),
                1.0, -1.0, 8.98846567431158e307, -8.98846567431158e307, 1.7976931348623157e308,
                4.49423283715579e307, np.inf, -np.inf, np.nan]
    vals = np.concatenate([np.array(specials), rng.standard_normal(1000) * 10.0 ** rng.uniform(-300, 300, 1000)])
    n = len(vals)
    m = Model()
    xv = m.add_var(n)
    m.add_con(lambda d: 2 * xv[d.k], n=n)
    m.add_con(lambda d: -xv[d.k], n=n)
    mod = B.exa_create(m.flat())
    c = _np(mod.cons(_t(vals)))
    with np.errstate(over="ignore"):
        want2, wantn = 2.0 * vals, -vals
    for got, want in ((c[:n], want2), (c[n:], wantn)):
        same = (got.view(np.uint64) == want.view(np.uint64)) | (np.isnan(got) & np.isnan(want))
        assert same.all(), [(v, g, w) for v, g, w in zip(vals[~same], got[~same], want[~same])][:5]
