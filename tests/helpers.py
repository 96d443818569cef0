"""Shared test helpers: dense assembly of COO output and small hand-written models."""
import numpy as np

from paper_2608_16265_gb300.ir import (Model, sin, cos, exp, log, sqrt, tan, tanh, atan, inv, sinh, cosh,
                                       asin, acos, log1p, expm1, log2, log10, exp2, atan2, hypot)


def dense_jac(nrow, ncol, rows, cols, vals):
    J = np.zeros((nrow, ncol))
    np.add.at(J, (rows, cols), vals)
    return J


def dense_hess(n, rows, cols, vals):
    """Symmetric expansion of a lower-triangle COO with duplicates."""
    H = np.zeros((n, n))
    np.add.at(H, (rows, cols), vals)
    off = rows != cols
    np.add.at(H, (cols[off], rows[off]), vals[off])
    return H


def normwise(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def all_ops_model(seed=0):
    """Tiny model touching every opcode, a parameter, an augmentation and a repeated symbol."""
    rng = np.random.default_rng(seed)
    m = Model()
    x = m.add_var(6)
    th = m.add_par([0.7, -1.3])
    n = 4
    data = dict(a=np.array([0, 1, 2, 3], np.int32), b=np.array([1, 2, 3, 4], np.int32),
                w=rng.uniform(0.5, 1.5, n))
    m.add_obj(lambda d: d.w * exp(x[d.a]) * x[d.b] + th[0] * x[d.a] ** 3 + x[d.b] / (2 + x[d.a] ** 2),
              data=data)
    m.add_obj(lambda d: sqrt(3 + x[d.a] ** 2) * log(2 + x[d.b] ** 2) + atan(x[d.a] * x[d.b]), data=data)
    blk = m.add_con(lambda d: sin(x[d.a]) * cos(x[d.b]) + tan(0.3 * x[d.a]) - tanh(x[d.b] - x[d.a])
                    + inv(2 + x[d.b] ** 2) + x[d.a] ** -3 + (1.5 + x[d.b] ** 2) ** (0.5 + 0.1 * x[d.a]),
                    data=data)
    m.add_con(lambda d: th[1] * x[d.a] * x[d.a] - x[d.b] * x[d.b] * x[d.b], data=data)
    m.add_con_aug(blk, lambda d: (d.r, x[d.s] * x[d.t] - d.w),
                  data=dict(r=np.array([0, 0, 3, 1], np.int32), s=np.array([5, 4, 5, 0], np.int32),
                            t=np.array([4, 4, 2, 5], np.int32), w=rng.uniform(-1, 1, 4)))
    return m


def flow_collision_model(seed=0):
    """The four polar branch-flow patterns of ACOPF on one data array (one fused group, so the
    Hessian CSC can come from per-branch compressed sums) on a network with self-loops (from bus =
    to bus) and a parallel branch: Hessian slots over two different symbols that resolve to one
    variable, and compressed sums whose terms agree up to sign (h(tf,tf) = h(tt,tt) = -h(tf,tt))."""
    rng = np.random.default_rng(seed)
    nb = 5
    m = Model()
    va = m.add_var(nb)
    vm = m.add_var(nb)
    f = np.array([0, 1, 2, 2, 3, 4, 4, 0], np.int32)
    t = np.array([1, 2, 2, 3, 0, 4, 1, 1], np.int32)  # self-loops at buses 2 and 4; 0-1 twice
    nl = len(f)
    br = dict(f=f, t=t, g=rng.uniform(0.5, 2.0, nl), b=rng.uniform(-3.0, -1.0, nl), gs=rng.uniform(0.0, 0.1, nl))
    m.add_con(lambda d: d.gs * vm[d.f] ** 2 + vm[d.f] * vm[d.t] * (
        d.g * cos(va[d.f] - va[d.t]) + d.b * sin(va[d.f] - va[d.t])), data=br)
    m.add_con(lambda d: -d.gs * vm[d.f] ** 2 - vm[d.f] * vm[d.t] * (
        d.b * cos(va[d.f] - va[d.t]) - d.g * sin(va[d.f] - va[d.t])), data=br)
    m.add_con(lambda d: d.gs * vm[d.t] ** 2 + vm[d.t] * vm[d.f] * (
        d.g * cos(va[d.t] - va[d.f]) + d.b * sin(va[d.t] - va[d.f])), data=br)
    m.add_con(lambda d: -d.gs * vm[d.t] ** 2 - vm[d.t] * vm[d.f] * (
        d.b * cos(va[d.t] - va[d.f]) - d.g * sin(va[d.t] - va[d.f])), data=br)
    m.add_obj(lambda d: (vm[d.k] - 1.0) ** 2, n=nb)
    return m


def flow_collision_point(seed=1):
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.uniform(-0.3, 0.3, 5), rng.uniform(0.9, 1.1, 5)])
    y = rng.standard_normal(32)
    return x, y, 0.5


def all_ops_point(seed=1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 0.9, 6)
    y = rng.standard_normal(8)
    return x, y, 0.75


def more_ops_model(seed=0):
    """The functions beyond the basic set (Sec. 7.1.4 registry): sinh, cosh, asin, acos, log1p,
    expm1, log2, log10, exp2, atan2, hypot."""
    rng = np.random.default_rng(seed)
    m = Model()
    x = m.add_var(6)
    data = dict(a=np.array([0, 1, 2, 3, 4], np.int32), b=np.array([1, 2, 3, 4, 5], np.int32),
                w=rng.uniform(0.5, 1.5, 5))
    m.add_obj(lambda d: sinh(x[d.a]) * cosh(x[d.b]) + asin(0.5 * x[d.a]) * acos(0.3 * x[d.b])
              + d.w * log1p(x[d.a] * x[d.b]), data=data)
    m.add_con(lambda d: expm1(x[d.a] - x[d.b]) + log2(1 + x[d.a] ** 2) * log10(2 + x[d.b])
              + exp2(x[d.a] * x[d.b]) + atan2(x[d.a], 1 + x[d.b]) + hypot(x[d.a], x[d.b] + 0.5), data=data)
    m.add_con(lambda d: atan2(x[d.b] - 0.1, x[d.a]) * hypot(x[d.a] * x[d.b], 1.0) - sinh(x[d.a] * x[d.b]),
              data=data)
    return m
