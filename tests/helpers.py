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
