"""The pattern builder: construction-time simplification (Sec. 7.1.3), literal powers, index
canonicalisation, and serialisation."""
import numpy as np
import pytest

from paper_2608_16265_gb300 import ir
from paper_2608_16265_gb300.ir import Const, Model, Un, Var


def _x():
    m = Model()
    return m.add_var(4)[1]


def test_simplification_table():
    """x+0 -> x, x*1 -> x, x/1 -> x, x^0 -> 1, x^1 -> x, x^2 -> abs2(x), x^-1 -> inv(x),
    0*x -> 0, 0/x -> 0 (the identity table of Sec. 7.1.3)."""
    x = _x()
    assert (x + 0) is x and (0 + x) is x
    assert (x * 1) is x and (1 * x) is x
    assert (x / 1) is x
    assert isinstance(x ** 0, Const) and (x ** 0).v == 1.0
    assert (x ** 1) is x
    assert isinstance(x ** 2, Un) and (x ** 2).op == ir.V_ABS2
    assert isinstance(x ** -1, Un) and (x ** -1).op == ir.V_INV
    assert isinstance(0 * x, Const) and (0 * x).v == 0.0
    assert isinstance(x * 0, Const)
    assert isinstance(0 / x, Const) and (0 / x).v == 0.0


def test_literal_powers_and_folding():
    x = _x()
    p = x ** 3
    assert isinstance(p, Un) and p.op == ir.V_POWI and p.n == 3
    assert (x ** 2.5).op == ir.V_POW
    assert isinstance(ir.sin(Const(0.5)), Const)
    assert (Const(2.0) * 3).v == 6.0


def test_index_canonicalisation():
    m = Model()
    x = m.add_var(10)
    d = ir.DataView(["i"], [ir.F_I32])
    a, b = x[d.i - 1], x[(d.i + 2) - 3]
    fa, fb = ir.flatten_pattern(ir.Pattern(ir.K_OBJ, 1, [np.zeros(1, np.int32)], ["i"], a)), \
        ir.flatten_pattern(ir.Pattern(ir.K_OBJ, 1, [np.zeros(1, np.int32)], ["i"], b))
    assert fa.iop.tolist() == fb.iop.tolist() and fa.ii.tolist() == fb.ii.tolist()


def test_flatten_postorder():
    m = Model()
    x = m.add_var(3)
    m.add_obj(lambda d: x[d.k] * ir.sin(x[d.k + 1]) + 2.0, n=2)
    p = m.flat().patterns[0]
    # children precede parents; the root is last
    for n, (op, a, b) in enumerate(zip(p.vop, p.va, p.vb)):
        if op >= 10:
            assert a < n
        if op >= 40:
            assert b < n
    assert p.vop[-1] == ir.V_ADD


def test_augmentation_needs_block():
    m = Model()
    x = m.add_var(3)
    blk = m.add_con(lambda d: x[d.k], n=3)
    m.add_con_aug(blk, lambda d: (d.r, x[d.k]), data=dict(r=np.array([2, 0], np.int32)))
    f = m.flat()
    assert f.ncon == 3 and f.patterns[1].kind == ir.K_AUG and f.patterns[1].row_limit == 3
    assert f.patterns[1].row_root >= 0


def test_bad_data_lengths():
    m = Model()
    x = m.add_var(3)
    with pytest.raises(ValueError):
        m.add_obj(lambda d: x[d.a], data=dict(a=np.zeros(2, np.int32), b=np.zeros(3)))
