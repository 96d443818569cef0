"""Pins of the CPU oracle against values the paper prints, closed forms, complex-step and
finite-difference derivatives, brute force on tiny models, and library routines (scipy.sparse).
None of these reuse the oracle's own formulas."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from paper_2608_16265_gb300.ir import Model, exp, sin
from tests.helpers import all_ops_model, all_ops_point, flow_collision_model, flow_collision_point, dense_hess, dense_jac, more_ops_model, normwise

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_pins.json")))


def paper_rosenbrock_model(i_one_based):
    """The paper's pattern 100 (x[i-1]^2 - x[i])^2 + (x[i-1] - 1)^2 over data points i."""
    m = Model()
    x = m.add_var(3)
    i0 = np.asarray(i_one_based, np.int32) - 1  # 0-based position of x[i]
    m.add_obj(lambda d: 100 * (x[d.i - 1] ** 2 - x[d.i]) ** 2 + (x[d.i - 1] - 1) ** 2,
              data=dict(i=i0))
    return oracle.Oracle(m.flat())


# ------------------------------------------------------------------ the paper's printed values
def test_paper_rosenbrock_values():
    g = GOLD["rosenbrock_term_value"]
    for i, v in zip(g["i_one_based"], g["value"]):
        assert paper_rosenbrock_model([i]).obj(g["x"]) == v


def test_paper_rosenbrock_gradient():
    g = GOLD["rosenbrock_term_gradient"]
    o = paper_rosenbrock_model([g["i_one_based"]])
    gr = o.grad(g["x"])
    assert gr[0] == g["gradient"][0] and gr[1] == g["gradient"][1] and gr[2] == 0.0
    c = g["leaf_contributions"]
    assert c[0] + c[2] == g["gradient"][0] and c[1] == g["gradient"][1]


def test_paper_product_example():
    g = GOLD["product_example"]
    m = Model()
    x = m.add_var(2)
    m.add_obj(lambda d: x[0] ** 2 * x[1], n=1)
    o = oracle.Oracle(m.flat())
    assert o.obj(g["x"]) == g["value"]
    assert o.grad(g["x"]).tolist() == g["gradient"]


def test_paper_compressors():
    g = GOLD["rosenbrock_compressors"]
    o = paper_rosenbrock_model([2])
    info = o.pattern_info(0)
    c1, c2 = o.compressors(0)
    assert list(c1) == g["comp1"] and info["o1step"] == g["o1step"]
    assert list(c2) == g["comp2"] and info["o2step"] == g["o2step"]


def test_rosenbrock_term_hessian_closed_form():
    """H11 = 1200 u^2 - 400 v + 2, H21 = -400 u, H22 = 200 (u = x_{i-1}, v = x_i) at (2, 3)."""
    o = paper_rosenbrock_model([2])
    r, c = o.hess_structure()
    H = dense_hess(3, r, c, o.hess_coord([2.0, 3.0, 5.0], np.zeros(0), 1.0))
    assert H[0, 0] == 1200 * 4 - 400 * 3 + 2 == 3602
    assert H[1, 0] == -800 and H[0, 1] == -800
    assert H[1, 1] == 200 and H[2, 2] == 0


# ------------------------------------------------------------------ closed forms on the workloads
def test_rosenbrock_closed_forms():
    wl = synth.rosenbrock(12)
    o = oracle.Oracle(wl.flat)
    x, y, s = synth.rosenbrock_point(wl, 3)
    n = 12
    f = sum(100 * (x[i + 1] - x[i] ** 2) ** 2 + (1 - x[i]) ** 2 for i in range(n - 1))
    assert abs(o.obj(x) - f) <= 1e-13 * abs(f)
    g = np.zeros(n)
    for i in range(n - 1):
        g[i] += -400 * x[i] * (x[i + 1] - x[i] ** 2) - 2 * (1 - x[i])
        g[i + 1] += 200 * (x[i + 1] - x[i] ** 2)
    assert normwise(o.grad(x), g) < 1e-14
    # constraint i uses a = x_i, b = x_{i+1}, c = x_{i+2}
    J = np.zeros((n - 2, n))
    Hc = np.zeros((n, n))
    cval = np.zeros(n - 2)
    for i in range(n - 2):
        a, b, c = x[i], x[i + 1], x[i + 2]
        cval[i] = (3 * b ** 3 + 2 * c - 5 + np.sin(b - c) * np.sin(b + c) + 4 * b
                   - a * np.exp(a - b) - 3)
        e = np.exp(a - b)
        J[i, i] = -e - a * e
        J[i, i + 1] = 9 * b ** 2 + np.cos(b - c) * np.sin(b + c) + np.sin(b - c) * np.cos(b + c) + 4 + a * e
        J[i, i + 2] = 2 - np.cos(b - c) * np.sin(b + c) + np.sin(b - c) * np.cos(b + c)
        # second derivatives; sin(b-c) sin(b+c) = (cos 2c - cos 2b)/2
        Haa, Hab = -2 * e - a * e, e + a * e
        Hbb = 18 * b + 2 * np.cos(2 * b) - a * e
        Hcc = -2 * np.cos(2 * c)
        idx = [i, i + 1, i + 2]
        loc = np.array([[Haa, Hab, 0], [Hab, Hbb, 0], [0, 0, Hcc]])
        Hc[np.ix_(idx, idx)] += y[i] * loc
    assert normwise(o.cons(x), cval) < 1e-14
    jr, jc = o.jac_structure()
    assert normwise(dense_jac(n - 2, n, jr, jc, o.jac_coord(x)), J) < 1e-14
    Hf = np.zeros((n, n))
    for i in range(n - 1):
        Hf[i, i] += 1200 * x[i] ** 2 - 400 * x[i + 1] + 2
        Hf[i + 1, i] += -400 * x[i]
        Hf[i, i + 1] += -400 * x[i]
        Hf[i + 1, i + 1] += 200
    hr, hc = o.hess_structure()
    H = dense_hess(n, hr, hc, o.hess_coord(x, y, s))
    assert normwise(H, s * Hf + Hc) < 1e-14


def test_pde_closed_forms():
    N = 7
    wl = synth.pde(N)
    o = oracle.Oracle(wl.flat)
    x, y, s = synth.pde_point(wl, 4)
    h = 1.0 / (N - 1)
    U = x[:N * N].reshape(N, N)
    nI = (N - 2) ** 2
    nu = N * N
    J = np.zeros((nI, nu + nI))
    Hd = np.zeros(nu + nI)
    Hd[:nu] = s * 1.0
    Hd[nu:] = s * 1e-4
    r = 0
    for i in range(1, N - 1):
        for j in range(1, N - 1):
            J[r, i * N + j] = 4 / h ** 2 + 3 * U[i, j] ** 2
            for (a, b) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                J[r, a * N + b] = -1 / h ** 2
            J[r, nu + r] = -1
            Hd[i * N + j] += 6 * U[i, j] * y[r]
            r += 1
    jr, jc = o.jac_structure()
    assert normwise(dense_jac(nI, nu + nI, jr, jc, o.jac_coord(x)), J) < 1e-14
    hr, hc = o.hess_structure()
    assert np.all(hr == hc)
    H = dense_hess(nu + nI, hr, hc, o.hess_coord(x, y, s))
    assert normwise(H, np.diag(Hd)) < 1e-14
    assert o.nnzh_csc == nu + nI


def test_acopf_flow_partials_textbook():
    """dp_f/dvm_f = 2 g_ff vm_f + vm_t (g_ft cos th + b_ft sin th);
    dp_f/dth = vm_f vm_t (-g_ft sin th + b_ft cos th), th = va_f - va_t (polar power flow)."""
    wl = synth.acopf(6, 9, 2, seed=5)
    o = oracle.Oracle(wl.flat)
    x, y, s = synth.acopf_point(wl, 2)
    B, L = 6, 9
    pf = wl.flat.patterns[2]
    assert pf.name == "p_from"
    f, t = pf.fields[0], pf.fields[1]
    gff, gft, bft = pf.fields[2], pf.fields[4], pf.fields[5]
    va, vm = x[:B], x[B:2 * B]
    J = dense_jac(o.ncon, o.nvar, *o.jac_structure(), o.jac_coord(x))
    for l in range(L):
        th = va[f[l]] - va[t[l]]
        row = 1 + l  # after the reference-angle row
        dvmf = 2 * gff[l] * vm[f[l]] + vm[t[l]] * (gft[l] * np.cos(th) + bft[l] * np.sin(th))
        dth = vm[f[l]] * vm[t[l]] * (-gft[l] * np.sin(th) + bft[l] * np.cos(th))
        # constraint is p - p_f(...), so partials carry a minus sign
        assert abs(J[row, B + f[l]] + dvmf) <= 1e-14 * max(1, abs(dvmf))
        assert abs(J[row, f[l]] + dth) <= 1e-14 * max(1, abs(dth))
        assert abs(J[row, t[l]] - dth) <= 1e-14 * max(1, abs(dth))
        assert J[row, 2 * B + 2 * 2 + l] == 1.0


# ------------------------------------------------------------------ complex step / FD / brute force
def _cs_jacobian(o, x, h=1e-30):
    n = o.nvar
    Jc = np.zeros((o.ncon, n))
    g = np.zeros(n)
    for j in range(n):
        xi = np.zeros(n); xi[j] = h
        Jc[:, j] = o.cons_complex(x, xi).imag / h
        g[j] = o.obj_complex(x, xi).imag / h
    return g, Jc


def _cs_hessian(o, x, y, s, h=1e-30):
    n = o.nvar
    H = np.zeros((n, n))
    for j in range(n):
        xi = np.zeros(n); xi[j] = h
        H[:, j] = o.lag_grad_complex(x, xi, y, s).imag / h
    return H


CASES = [
    ("all_ops", lambda: (all_ops_model().flat(), all_ops_point())),
    ("flow_collisions", lambda: (flow_collision_model().flat(), flow_collision_point())),
    ("more_ops", lambda: (more_ops_model().flat(), (np.random.default_rng(2).uniform(0.2, 0.9, 6),
                                                     np.random.default_rng(3).standard_normal(10), 1.3))),
    ("rosenbrock", lambda: (lambda w: (w.flat, synth.rosenbrock_point(w, 1)))(synth.rosenbrock(7))),
    ("acopf", lambda: (lambda w: (w.flat, synth.acopf_point(w, 1)))(synth.acopf(5, 7, 2, seed=3, shunts=True))),
    ("pde", lambda: (lambda w: (w.flat, synth.pde_point(w, 1)))(synth.pde(5))),
    ("goddard", lambda: (lambda w: (w.flat, synth.goddard_point(w, 1)))(synth.goddard(6))),
    ("two_stage", lambda: (lambda w: (w.flat, synth.two_stage_point(w, 1)))(synth.two_stage_acopf(5, 7, 2, 3, seed=3))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_complex_step_first_order(name, make):
    flat, (x, y, s) = make()
    o = oracle.Oracle(flat)
    g, Jc = _cs_jacobian(o, x)
    assert normwise(o.grad(x), g) < 1e-14
    J = dense_jac(o.ncon, o.nvar, *o.jac_structure(), o.jac_coord(x))
    assert normwise(J, Jc) < 1e-14
    xr = np.asarray(x, float)
    assert abs(o.obj_complex(xr, np.zeros_like(xr)).real - o.obj(x)) <= 1e-13 * max(1, abs(o.obj(x)))
    assert normwise(o.cons_complex(xr, np.zeros_like(xr)).real, o.cons(x)) < 1e-14


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_complex_step_hessian(name, make):
    """Complex step on a first-order AD gradient uses no second-derivative rule."""
    flat, (x, y, s) = make()
    o = oracle.Oracle(flat)
    Hcs = _cs_hessian(o, x, y, s)
    assert normwise(Hcs, Hcs.T) < 1e-13
    hr, hc = o.hess_structure()
    H = dense_hess(o.nvar, hr, hc, o.hess_coord(x, y, s))
    assert normwise(H, Hcs) < 1e-13
    # the structure covers every nonzero of the true Hessian
    nz = np.argwhere(np.abs(np.tril(Hcs)) > 1e-12 * np.abs(Hcs).max())
    have = set(zip(hr.tolist(), hc.tolist()))
    for r, c in nz.tolist():
        assert (r, c) in have


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_finite_differences(name, make):
    flat, (x, y, s) = make()
    o = oracle.Oracle(flat)
    x = np.asarray(x, float)
    n, hstep = o.nvar, 1e-6
    J = dense_jac(o.ncon, n, *o.jac_structure(), o.jac_coord(x))
    g = o.grad(x)
    for j in range(n):
        e = np.zeros(n); e[j] = hstep
        fd_c = (o.cons(x + e) - o.cons(x - e)) / (2 * hstep)
        fd_f = (o.obj(x + e) - o.obj(x - e)) / (2 * hstep)
        assert np.allclose(J[:, j], fd_c, rtol=1e-6, atol=1e-6 * max(1, np.abs(J).max()))
        assert abs(g[j] - fd_f) <= 1e-6 * max(1, np.abs(g).max())


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_products_consistent(name, make):
    """J v against a complex-step directional derivative of c; H v against a complex-step
    directional derivative of the AD gradient of the Lagrangian; J^T w against w^T J (dense)."""
    flat, (x, y, s) = make()
    o = oracle.Oracle(flat)
    x = np.asarray(x, float)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(o.nvar)
    w = rng.standard_normal(o.ncon)
    h = 1e-30
    jv_cs = o.cons_complex(x, h * v).imag / h
    assert normwise(o.jprod(x, v), jv_cs) < 1e-14
    hv_cs = o.lag_grad_complex(x, h * v, y, s).imag / h
    assert normwise(o.hprod(x, y, s, v), hv_cs) < 1e-13
    J = dense_jac(o.ncon, o.nvar, *o.jac_structure(), o.jac_coord(x))
    assert normwise(o.jtprod(x, w), J.T @ w) < 1e-14


def test_repeated_symbol_on_diagonal_doubles():
    """x[a] * x[b] with a == b at run time must give d2/dx^2 (x^2) = 2 on the diagonal."""
    m = Model()
    x = m.add_var(3)
    m.add_obj(lambda d: x[d.a] * x[d.b], data=dict(a=np.array([0, 1], np.int32), b=np.array([0, 2], np.int32)))
    o = oracle.Oracle(m.flat())
    hr, hc = o.hess_structure()
    H = dense_hess(3, hr, hc, o.hess_coord([0.3, 0.4, 0.5], np.zeros(0), 1.0))
    assert H.tolist() == [[2.0, 0, 0], [0, 0, 1.0], [0, 1.0, 0]]


# ------------------------------------------------------------------ CSC against scipy.sparse
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_csc_against_scipy(name, make):
    flat, (x, y, s) = make()
    o = oracle.Oracle(flat)
    for (r, c), coo, (cp, rv, m), csc, nrow in (
            (o.jac_structure(), o.jac_coord(x), o.jac_csc_structure(), o.jac_csc(x), o.ncon),
            (o.hess_structure(), o.hess_coord(x, y, s), o.hess_csc_structure(), o.hess_csc(x, y, s), o.nvar)):
        # structural CSC: pattern of all entries, explicit zeros included
        ones = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(nrow, o.nvar)).tocsc()
        ones.sum_duplicates()
        ones.sort_indices()
        assert np.array_equal(ones.indptr, cp) and np.array_equal(ones.indices, rv)
        A = sp.coo_matrix((coo, (r, c)), shape=(nrow, o.nvar)).tocsc()
        A.sum_duplicates()
        dense_ref = A.toarray()
        dense_csc = sp.csc_matrix((csc, rv, cp), shape=(nrow, o.nvar)).toarray()
        assert normwise(dense_csc, dense_ref) < 1e-15
        # coo2csc sends every COO entry to the CSC slot of its own (row, col)
        for q in range(len(r)):
            p = m[q]
            assert rv[p] == r[q] and cp[c[q]] <= p < cp[c[q] + 1]


# ------------------------------------------------------------------ structure counts
def test_structure_counts_acopf():
    B, L, G = 40, 60, 7
    o = oracle.Oracle(synth.acopf(B, L, G, seed=9).flat)
    assert o.nvar == 2 * B + 2 * G + 4 * L
    assert o.ncon == 1 + 7 * L + 2 * B
    assert o.nnzj == 1 + 30 * L + 2 * B + 2 * G
    assert o.nnzh == G + 40 * L + 2 * B


def test_structure_counts_rosenbrock_pde():
    o = oracle.Oracle(synth.rosenbrock(1000).flat)
    assert (o.nnzj, o.nnzh) == (2994, 7987)
    N = 9
    o = oracle.Oracle(synth.pde(N).flat)
    nI = (N - 2) ** 2
    assert (o.nvar, o.ncon, o.nnzj, o.nnzh, o.nnzh_csc) == (N * N + nI, nI, 6 * nI, N * N + 2 * nI, N * N + nI)


def test_validation_errors():
    m = Model()
    x = m.add_var(3)
    m.add_obj(lambda d: x[d.i] ** 2, data=dict(i=np.array([0, 3], np.int32)))
    with pytest.raises(oracle.OracleError, match="variable index out of range"):
        oracle.Oracle(m.flat())
    m = Model()
    x = m.add_var(3)
    b = m.add_con(lambda d: x[d.k], n=2)
    m.add_con_aug(b, lambda d: (d.r, x[0]), data=dict(r=np.array([2], np.int32)))
    with pytest.raises(oracle.OracleError, match="augmentation row"):
        oracle.Oracle(m.flat())


def test_empty_patterns():
    m = Model()
    x = m.add_var(4)
    m.add_obj(lambda d: x[d.k] ** 2, n=0)
    blk = m.add_con(lambda d: x[d.k] * x[d.k + 1], n=3)
    m.add_con_aug(blk, lambda d: (d.r, x[d.k]), data=dict(r=np.zeros(0, np.int32)))
    o = oracle.Oracle(m.flat())
    x0 = np.array([1.0, 2.0, 3.0, 4.0])
    assert o.obj(x0) == 0.0 and np.all(o.grad(x0) == 0)
    assert o.cons(x0).tolist() == [2.0, 6.0, 12.0]
    assert o.nnzj == 6 and o.nnzh == 3


def test_first_order_slot_order_left_to_right():
    """The probe visits leaves in the order the reverse pass does: left operand before right
    (Sec. 5.2.1: the first two visits come from the left term 100(x_{i-1}^2 - x_i)^2).  An
    asymmetric tree pins the order: x[2]*x[0] + x[1] -> slots x2, x0, x1."""
    m = Model()
    x = m.add_var(3)
    m.add_con(lambda d: x[2] * x[0] + x[1], n=1)
    o = oracle.Oracle(m.flat())
    assert o.jac_structure()[1].tolist() == [2, 0, 1]


def test_second_order_slot_order():
    """Reading of Sec. 5.2.2 ("two diagonal entries and one off-diagonal", comp2 = (1,2,3,1)):
    a binary node emits its children's entries first, then the cross pairs."""
    o = paper_rosenbrock_model([2])
    r, c = o.hess_structure()
    assert list(zip(r.tolist(), c.tolist())) == [(0, 0), (1, 1), (1, 0)]
    m = Model()
    x = m.add_var(4)
    m.add_obj(lambda d: sin(x[3] * x[1]) + x[2] * exp(x[0]), n=1)
    o = oracle.Oracle(m.flat())
    r, c = o.hess_structure()
    # sin(x3 x1): diag x3, diag x1, cross (x3, x1); then x2 * exp(x0): diag x0, cross (x2, x0)
    assert list(zip(r.tolist(), c.tolist())) == [(3, 3), (1, 1), (3, 1), (0, 0), (2, 0)]
