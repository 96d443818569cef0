"""Two-stage models (Sec. 8.1, Eq. (extensions) with one batch instance): the builder's scenario
replication, stage tags and single-scenario parameter accessor, pinned on the section's own example
(root x[1:2], per-scenario z[1:3, s] and theta[1:3, s], objective x1^2 + x2^2 + sum (z - theta)^2,
constraints z[j, s] + x2), whose derivatives have closed forms, and on invariants of the two-stage
ACOPF."""
import numpy as np

import oracle
import synth
from paper_2608_16265_gb300.ir import TwoStageModel
from tests.helpers import dense_hess, dense_jac

S = 4


def paper_example(theta):
    m = TwoStageModel(S)
    x = m.add_var(2)
    z = m.add_var(3, scenario=True)
    th = m.add_par(theta, scenario=True)
    idx = dict(j=np.arange(3, dtype=np.int32))
    m.add_obj(lambda d: x[0] ** 2 + x[1] ** 2, n=1)
    m.add_obj(lambda d: (z[d.j, d.s] - th[d.j, d.s]) ** 2, data=idx, scenario=True)
    m.add_con(lambda d: z[d.j, d.s] + x[1], data=idx, scenario=True)
    return m, x, z, th


def test_paper_example_closed_forms():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal((3, S))
    m, xb, zb, thb = paper_example(theta)
    flat = m.flat()
    assert (flat.nvar, flat.ncon) == (2 + 3 * S, 3 * S)
    # layout: root first, then z scenario-major (z[j, s] at 2 + 3 s + j); theta likewise
    assert np.array_equal(m.var_stage(), np.r_[[0, 0], np.repeat(np.arange(1, S + 1), 3)])
    assert np.array_equal(m.con_stage(), np.repeat(np.arange(1, S + 1), 3))
    assert np.array_equal(flat.theta, theta.T.ravel())
    o = oracle.Oracle(flat)
    v = rng.standard_normal(flat.nvar)
    y = rng.standard_normal(flat.ncon)
    sig = 0.7
    X, Z = v[:2], v[2:].reshape(S, 3)
    T = theta.T
    assert abs(o.obj(v) - (X @ X + ((Z - T) ** 2).sum())) <= 1e-14 * (1 + abs(o.obj(v)))
    assert np.allclose(o.grad(v), np.r_[2 * X, (2 * (Z - T)).ravel()], rtol=0, atol=1e-15)
    assert np.allclose(o.cons(v), (Z + X[1]).ravel(), rtol=0, atol=1e-15)
    J = dense_jac(o.ncon, o.nvar, *o.jac_structure(), o.jac_coord(v))
    Jw = np.zeros((3 * S, 2 + 3 * S))
    Jw[:, 1] = 1.0
    Jw[:, 2:] = np.eye(3 * S)
    assert np.array_equal(J, Jw)
    H = dense_hess(o.nvar, *o.hess_structure(), o.hess_coord(v, y, sig))
    assert np.array_equal(H, 2 * sig * np.eye(2 + 3 * S))
    # the root variable x2 couples every scenario: its Jacobian column holds one entry per row
    colptr, rowval, _ = o.jac_csc_structure()
    assert colptr[2] - colptr[1] == 3 * S and colptr[1] - colptr[0] == 0


def test_scenario_theta_accessor_touches_one_scenario():
    rng = np.random.default_rng(1)
    theta = rng.standard_normal((3, S))
    m, xb, zb, thb = paper_example(theta)
    flat = m.flat()
    new = m.scenario_theta(flat.theta, thb, 2, [5.0, 6.0, 7.0])
    changed = np.nonzero(new != flat.theta)[0]
    assert np.array_equal(changed, np.arange(thb.offset + 2 * 3, thb.offset + 3 * 3))
    v = rng.standard_normal(flat.nvar)
    g0 = oracle.Oracle(flat).grad(v)
    flat.theta = new
    g1 = oracle.Oracle(flat).grad(v)
    diff = np.nonzero(g1 != g0)[0]
    assert set(m.var_stage()[diff].tolist()) == {3}  # scenario 2 is stage 3


def test_two_stage_acopf_counts_and_stages():
    B, L, G = 30, 45, 6
    wl = synth.two_stage_acopf(B, L, G, S, seed=2)
    m, flat = wl.model, wl.flat
    o = oracle.Oracle(flat)
    assert flat.nvar == G + S * (2 * B + G + 4 * L) and flat.ncon == S * (1 + 7 * L + 2 * B)
    # per scenario: reference 1, flows 4 x 5, angle 2, thermal 2 x 2, generator and arc terms
    assert o.nnzj == S * (1 + 30 * L + 2 * G)
    # root cost G, per scenario: reactive cost G, flows 4 x 9, thermal 2 x 2
    assert o.nnzh == G + S * (G + 40 * L)
    vs, cs = m.var_stage(), m.con_stage()
    assert (vs[:G] == 0).all() and np.array_equal(np.bincount(vs[G:]), np.r_[0, [2 * B + G + 4 * L] * S])
    assert np.array_equal(np.bincount(cs), np.r_[0, [1 + 7 * L + 2 * B] * S])
    # every Jacobian entry couples a row with a variable of its own scenario or the root
    r, c = o.jac_structure()
    assert ((vs[c] == 0) | (vs[c] == cs[r])).all()
    # every root generator appears in each scenario's P balance
    colptr, rowval, _ = o.jac_csc_structure()
    assert np.array_equal(np.diff(colptr)[:G], np.full(G, S))


def test_identical_scenarios_give_identical_blocks():
    """With no load spread and the same scenario variables in every scenario, every scenario's
    constraint values, Jacobian entries and multiplier-weighted Hessian entries are the same."""
    B, L, G = 12, 18, 3
    wl = synth.two_stage_acopf(B, L, G, S, seed=5, spread=0.0)
    m, flat = wl.model, wl.flat
    o = oracle.Oracle(flat)
    vs, cs = m.var_stage(), m.con_stage()
    rng = np.random.default_rng(3)
    x = rng.standard_normal(flat.nvar)
    y = rng.standard_normal(flat.ncon)
    for s in range(2, S + 1):  # scenario copies in the same (block, position) order
        x[vs == s] = x[vs == 1]
        y[cs == s] = y[cs == 1]
    c = o.cons(x)
    assert all(np.array_equal(c[cs == 1], c[cs == s]) for s in range(2, S + 1))
    jr, jc = o.jac_structure()
    jv = o.jac_coord(x)
    for s in range(2, S + 1):
        assert np.array_equal(jv[cs[jr] == 1], jv[cs[jr] == s])
    hr, hc = o.hess_structure()
    hv = o.hess_coord(x, y, 1.0)
    for s in range(2, S + 1):
        assert np.array_equal(hv[vs[hr] == 1], hv[vs[hr] == s])


def test_builder_rejects_misuse():
    import pytest
    m = TwoStageModel(3)
    x = m.add_var(2)
    with pytest.raises(ValueError):
        m.add_par(np.zeros((2, 4)), scenario=True)  # last axis must be the scenario count
    with pytest.raises(ValueError):
        m.add_con(lambda d: x[0] + d.s, data=dict(s=np.zeros(2, np.int32)), scenario=True)  # reserved name
    root = m.add_con(lambda d: x[d.k], n=2)
    with pytest.raises(ValueError):
        m.add_con_aug(root, lambda d: (0, x[1]), n=1, scenario=True)  # per-scenario term into a root block
    with pytest.raises(ValueError):
        TwoStageModel(0)
    z = m.add_var(2, scenario=True)
    with pytest.raises(IndexError):
        z[0]  # the scenario index is required


def test_root_and_scenario_augmentations_land_in_the_right_rows():
    """A per-scenario augmentation term goes to its own scenario's row of a per-scenario block; the
    oracle's constraint values show it row by row."""
    m = TwoStageModel(3)
    x = m.add_var(1)
    z = m.add_var(2, scenario=True)
    blk = m.add_con(lambda d: z[d.i, d.s], data=dict(i=np.arange(2, dtype=np.int32)), scenario=True)
    m.add_con_aug(blk, lambda d: (1, 10.0 * x[0]), n=1, scenario=True)
    flat = m.flat()
    v = np.array([2.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0])  # x, then z[:, 0], z[:, 1], z[:, 2]
    c = oracle.Oracle(flat).cons(v)
    assert np.array_equal(c, [1.0, 22.0, 3.0, 24.0, 5.0, 26.0])
