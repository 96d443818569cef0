"""Pattern IR: the modeling front end that turns repeated algebraic patterns into flat arrays.

A model is the SIMD form of the problem (Sec. 2.2, Eq. (simd)): an objective made of objective
patterns, each evaluated over its own data array, and constraint blocks made of one base pattern
(one row per data item) plus augmentation patterns that add one term to a data-selected row of
a block (Sec. 3.3, ConstraintAugmentation).  A pattern is one expression tree built by operator
overloading on variable, parameter and data sources (Sec. 4.1), with the paper's construction-time
algebraic simplifications applied as nodes are built (Sec. 7.1.3) and integer literal powers
lowered to dedicated nodes.

This module only builds trees and serialises them; it computes no derivatives.  The flat layout
(one postorder array of value nodes and one postorder array of integer index nodes per pattern) is
what `exa_create` in `include/exa.h` accepts.

Index expressions are 0-based integer expressions over the pattern's int32 data fields, the
instance number k (0-based) and integer constants.  Two `Var` leaves of one pattern are the same
symbol exactly when their serialised index subtrees are identical, so the builder canonicalises
index expressions (constant folding, `a - c` written as `a + (-c)`, nested constant offsets merged).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Union

import numpy as np

# ---------------------------------------------------------------- opcodes (mirrors include/exa.h)
V_CONST, V_DATA, V_VAR, V_PARAM = 0, 1, 2, 3
V_NEG, V_ABS2, V_INV, V_EXP, V_LOG, V_SIN, V_COS, V_SQRT, V_TAN, V_TANH, V_ATAN, V_POWI = range(10, 22)
V_SINH, V_COSH, V_ASIN, V_ACOS, V_LOG1P, V_EXPM1, V_LOG2, V_LOG10, V_EXP2 = range(22, 31)
V_ADD, V_SUB, V_MUL, V_DIV, V_POW, V_ATAN2, V_HYPOT = range(40, 47)
I_CONST, I_FIELD, I_INST = 0, 1, 2
I_ADD, I_SUB, I_MUL = 10, 11, 12

K_OBJ, K_CON, K_AUG = 0, 1, 2
F_I32, F_F64 = 0, 1

UNARY_NAMES = {V_NEG: "neg", V_ABS2: "abs2", V_INV: "inv", V_EXP: "exp", V_LOG: "log",
               V_SIN: "sin", V_COS: "cos", V_SQRT: "sqrt", V_TAN: "tan", V_TANH: "tanh",
               V_ATAN: "atan", V_POWI: "powi", V_SINH: "sinh", V_COSH: "cosh", V_ASIN: "asin",
               V_ACOS: "acos", V_LOG1P: "log1p", V_EXPM1: "expm1", V_LOG2: "log2", V_LOG10: "log10",
               V_EXP2: "exp2"}
BINARY_NAMES = {V_ADD: "+", V_SUB: "-", V_MUL: "*", V_DIV: "/", V_POW: "^", V_ATAN2: "atan2",
                V_HYPOT: "hypot"}


# ---------------------------------------------------------------- integer index expressions
class IExpr:
    """Integer index expression (0-based).  Supports +, -, * with ints and other IExprs."""

    def _key(self):
        raise NotImplementedError

    def __add__(self, o):
        return _iadd(self, _ilift(o))

    def __radd__(self, o):
        return _iadd(_ilift(o), self)

    def __sub__(self, o):
        o = _ilift(o)
        if isinstance(o, IConst):
            return _iadd(self, IConst(-o.v))
        return _ibin(I_SUB, self, o)

    def __rsub__(self, o):
        return _ilift(o) - self

    def __mul__(self, o):
        return _imul(self, _ilift(o))

    def __rmul__(self, o):
        return _imul(_ilift(o), self)


@dataclass(frozen=True, eq=False)
class IConst(IExpr):
    v: int


@dataclass(frozen=True, eq=False)
class IField(IExpr):
    f: int  # field number within the pattern's data table


@dataclass(frozen=True, eq=False)
class IInst(IExpr):
    pass


@dataclass(frozen=True, eq=False)
class IBin(IExpr):
    op: int
    a: IExpr
    b: IExpr


def _ilift(o) -> IExpr:
    if isinstance(o, IExpr):
        return o
    if isinstance(o, (int, np.integer)) and not isinstance(o, bool):
        return IConst(int(o))
    raise TypeError(f"index expressions take ints, got {type(o).__name__}")


def _ibin(op, a, b):
    if isinstance(a, IConst) and isinstance(b, IConst):
        return IConst({I_ADD: a.v + b.v, I_SUB: a.v - b.v, I_MUL: a.v * b.v}[op])
    return IBin(op, a, b)


def _iadd(a: IExpr, b: IExpr) -> IExpr:
    if isinstance(a, IConst) and a.v == 0:
        return b
    if isinstance(b, IConst) and b.v == 0:
        return a
    if isinstance(a, IConst) and not isinstance(b, IConst):  # constant offsets go right
        a, b = b, a
    if isinstance(b, IConst) and isinstance(a, IBin) and a.op == I_ADD and isinstance(a.b, IConst):
        return _iadd(a.a, IConst(a.b.v + b.v))
    return _ibin(I_ADD, a, b)


def _imul(a: IExpr, b: IExpr) -> IExpr:
    if isinstance(a, IConst) and a.v == 1:
        return b
    if isinstance(b, IConst) and b.v == 1:
        return a
    if isinstance(a, IConst) and a.v == 0 or isinstance(b, IConst) and b.v == 0:
        return IConst(0)
    return _ibin(I_MUL, a, b)


# ---------------------------------------------------------------- value expressions
class Expr:
    """Node of a parameterized expression tree (Sec. 4.2)."""

    def __add__(self, o):
        return add(self, o)

    def __radd__(self, o):
        return add(o, self)

    def __sub__(self, o):
        return sub(self, o)

    def __rsub__(self, o):
        return sub(o, self)

    def __mul__(self, o):
        return mul(self, o)

    def __rmul__(self, o):
        return mul(o, self)

    def __truediv__(self, o):
        return div(self, o)

    def __rtruediv__(self, o):
        return div(o, self)

    def __pow__(self, o):
        return power(self, o)

    def __rpow__(self, o):
        return power(o, self)

    def __neg__(self):
        return neg(self)

    def __pos__(self):
        return self


@dataclass(frozen=True, eq=False)
class Const(Expr):
    v: float


@dataclass(frozen=True, eq=False)
class Data(Expr):
    f: int


@dataclass(frozen=True, eq=False)
class Var(Expr):
    idx: IExpr


@dataclass(frozen=True, eq=False)
class Param(Expr):
    idx: IExpr


@dataclass(frozen=True, eq=False)
class Un(Expr):
    op: int
    a: Expr
    n: int = 0  # exponent of V_POWI


@dataclass(frozen=True, eq=False)
class Bin(Expr):
    op: int
    a: Expr
    b: Expr


def lift(o) -> Expr:
    if isinstance(o, Expr):
        return o
    if isinstance(o, IField):  # an int32 data field used as a value
        return Data(o.f)
    if isinstance(o, (int, float, np.integer, np.floating)) and not isinstance(o, bool):
        return Const(float(o))
    raise TypeError(f"cannot use {type(o).__name__} in an expression")


def _is(c: Expr, v: float) -> bool:
    return isinstance(c, Const) and c.v == v


# Construction-time simplification (Sec. 7.1.3): x+0, x*1, x/1, x^0, x^1, x^2, x^-1, 0*x, 0/x,
# plus folding of operations whose operands are all constants.
def add(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(a.v + b.v)
    if _is(b, 0.0):
        return a
    if _is(a, 0.0):
        return b
    return Bin(V_ADD, a, b)


def sub(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(a.v - b.v)
    return Bin(V_SUB, a, b)


def mul(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(a.v * b.v)
    if _is(a, 0.0) or _is(b, 0.0):
        return Const(0.0)
    if _is(b, 1.0):
        return a
    if _is(a, 1.0):
        return b
    return Bin(V_MUL, a, b)


def div(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(a.v / b.v)
    if _is(b, 1.0):
        return a
    if _is(a, 0.0):
        return Const(0.0)
    return Bin(V_DIV, a, b)


def power(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(a.v ** b.v)
    if isinstance(b, Const) and float(b.v).is_integer():
        n = int(b.v)
        if n == 0:
            return Const(1.0)
        if n == 1:
            return a
        if n == 2:
            return Un(V_ABS2, a)
        if n == -1:
            return Un(V_INV, a)
        return Un(V_POWI, a, n)
    return Bin(V_POW, a, b)


def _unary(op, fn):
    def f(a):
        a = lift(a)
        if isinstance(a, Const):
            return Const(fn(a.v))
        return Un(op, a)
    f.__name__ = UNARY_NAMES[op]
    return f


neg = _unary(V_NEG, lambda v: -v)
abs2 = _unary(V_ABS2, lambda v: v * v)
inv = _unary(V_INV, lambda v: 1.0 / v)
exp = _unary(V_EXP, math.exp)
log = _unary(V_LOG, math.log)
sin = _unary(V_SIN, math.sin)
cos = _unary(V_COS, math.cos)
sqrt = _unary(V_SQRT, math.sqrt)
tan = _unary(V_TAN, math.tan)
tanh = _unary(V_TANH, math.tanh)
atan = _unary(V_ATAN, math.atan)
sinh = _unary(V_SINH, math.sinh)
cosh = _unary(V_COSH, math.cosh)
asin = _unary(V_ASIN, math.asin)
acos = _unary(V_ACOS, math.acos)
log1p = _unary(V_LOG1P, math.log1p)
expm1 = _unary(V_EXPM1, math.expm1)
log2 = _unary(V_LOG2, math.log2)
log10 = _unary(V_LOG10, math.log10)
exp2 = _unary(V_EXP2, lambda v: 2.0 ** v)


def atan2(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(math.atan2(a.v, b.v))
    return Bin(V_ATAN2, a, b)


def hypot(a, b):
    a, b = lift(a), lift(b)
    if isinstance(a, Const) and isinstance(b, Const):
        return Const(math.hypot(a.v, b.v))
    return Bin(V_HYPOT, a, b)


# ---------------------------------------------------------------- model containers
class DataView:
    """Symbolic view of one data item: `d.name` is an IExpr (int32 field) or Data (f64 field),
    `d.k` the instance number."""

    def __init__(self, names: Sequence[str], types: Sequence[int]):
        object.__setattr__(self, "_map", {n: (i, t) for i, (n, t) in enumerate(zip(names, types))})

    @property
    def k(self) -> IExpr:
        return IInst()

    def __getattr__(self, name):
        try:
            i, t = self._map[name]
        except KeyError:
            raise AttributeError(name) from None
        return IField(i) if t == F_I32 else Data(i)

    def __getitem__(self, name):
        return self.__getattr__(name)


class VarBlock:
    """A block of variables `x[offset : offset + prod(shape)]`, row-major."""

    def __init__(self, offset: int, shape: tuple):
        self.offset, self.shape = offset, shape
        self.size = int(np.prod(shape)) if shape else 1

    def _flat(self, idx):
        if not isinstance(idx, tuple):
            idx = (idx,)
        if len(idx) != len(self.shape):
            raise IndexError(f"block has {len(self.shape)} dimensions, got {len(idx)} indices")
        flat = IConst(0)
        for d, i in enumerate(idx):
            flat = flat * self.shape[d] + _ilift(i) if d else _ilift(i)
        return flat

    def __getitem__(self, idx):
        return Var(self._flat(idx) + self.offset)

    def at(self, flat_idx):
        """Variable by row-major flat position within the block."""
        return Var(_ilift(flat_idx) + self.offset)


class ParBlock(VarBlock):
    def __getitem__(self, idx):
        return Param(self._flat(idx) + self.offset)


@dataclass
class Pattern:
    kind: int
    n_inst: int
    fields: List[np.ndarray]
    field_names: List[str]
    root: Expr
    row_base: int = -1
    row_limit: int = 0
    row_expr: Optional[IExpr] = None
    name: str = ""


@dataclass
class ConBlock:
    row_base: int
    n_rows: int
    pattern_index: int


class Model:
    """Host-side model builder (the ExaCore analog, Sec. 3.1).

    add_var / add_par declare blocks; add_obj / add_con / add_con_aug append patterns in
    declaration order, which fixes the order of the COO blocks (Sec. 5.3)."""

    def __init__(self):
        self.nvar = 0
        self.ncon = 0
        self.theta: List[float] = []
        self.patterns: List[Pattern] = []
        self.x0: List[np.ndarray] = []

    def add_var(self, *shape) -> VarBlock:
        b = VarBlock(self.nvar, tuple(int(s) for s in shape))
        self.nvar += b.size
        return b

    def add_par(self, values) -> ParBlock:
        values = np.asarray(values, dtype=np.float64)
        b = ParBlock(len(self.theta), values.shape)
        self.theta.extend(values.ravel().tolist())
        return b

    @staticmethod
    def _table(data: Dict[str, np.ndarray], n: Optional[int]):
        names, arrs, types = [], [], []
        for k, v in data.items():
            v = np.asarray(v)
            if v.dtype.kind in "iub":
                v = np.ascontiguousarray(v, dtype=np.int32)
                types.append(F_I32)
            else:
                v = np.ascontiguousarray(v, dtype=np.float64)
                types.append(F_F64)
            names.append(k)
            arrs.append(v)
        lens = {len(a) for a in arrs}
        if n is None:
            if len(lens) != 1:
                raise ValueError("data columns must have one common length (or pass n)")
            n = lens.pop()
        elif lens and lens != {n}:
            raise ValueError("data columns must all have length n")
        return names, arrs, types, int(n)

    def add_obj(self, fn: Callable[[DataView], Expr], data: Dict[str, np.ndarray] = None,
                n: Optional[int] = None, name: str = "") -> int:
        names, arrs, types, n = self._table(data or {}, n)
        root = lift(fn(DataView(names, types)))
        self.patterns.append(Pattern(K_OBJ, n, arrs, names, root, name=name))
        return len(self.patterns) - 1

    def add_con(self, fn: Callable[[DataView], Expr], data: Dict[str, np.ndarray] = None,
                n: Optional[int] = None, name: str = "") -> ConBlock:
        names, arrs, types, n = self._table(data or {}, n)
        root = lift(fn(DataView(names, types)))
        p = Pattern(K_CON, n, arrs, names, root, row_base=self.ncon, row_limit=n, name=name)
        self.patterns.append(p)
        blk = ConBlock(self.ncon, n, len(self.patterns) - 1)
        self.ncon += n
        return blk

    def add_con_aug(self, block: ConBlock, fn: Callable[[DataView], tuple],
                    data: Dict[str, np.ndarray] = None, n: Optional[int] = None,
                    name: str = "") -> int:
        """Augmentation `idx => value` (Sec. 3.3): fn returns (row index within block, term)."""
        names, arrs, types, n = self._table(data or {}, n)
        idx, val = fn(DataView(names, types))
        p = Pattern(K_AUG, n, arrs, names, lift(val), row_base=block.row_base,
                    row_limit=block.n_rows, row_expr=_ilift(idx), name=name)
        self.patterns.append(p)
        return len(self.patterns) - 1

    # -------------------------------------------------------------- serialisation
    def flat(self) -> "FlatModel":
        return FlatModel(self.nvar, self.ncon, np.asarray(self.theta, dtype=np.float64),
                         [flatten_pattern(p) for p in self.patterns])



# ---------------------------------------------------------------- two-stage models
class ScenarioBlock(VarBlock):
    """A block declared once per scenario: `z[j..., s]` with the scenario index last (Sec. 8.1.2,
    the EachScenario marker).  Storage is scenario-major, `offset + s * size + rowmajor(j)`, so every
    scenario's copy is one contiguous range."""

    def __init__(self, offset: int, shape: tuple, nscen: int):
        super().__init__(offset, shape)
        self.nscen = nscen

    def _flat_s(self, idx):
        if not isinstance(idx, tuple):
            idx = (idx,)
        if len(idx) != len(self.shape) + 1:
            raise IndexError(f"block has {len(self.shape)} dimensions plus the scenario, got {len(idx)} indices")
        inner = self._flat(idx[:-1]) if self.shape else IConst(0)
        return _ilift(idx[-1]) * self.size + inner + self.offset

    def __getitem__(self, idx):
        return Var(self._flat_s(idx))

    def scenario_range(self, s: int) -> slice:
        """Positions of scenario s's copy in x (or theta)."""
        return slice(self.offset + s * self.size, self.offset + (s + 1) * self.size)


class ScenarioParBlock(ScenarioBlock):
    def __getitem__(self, idx):
        return Param(self._flat_s(idx))


@dataclass
class ScenarioConBlock(ConBlock):
    n_per: int = 0  # rows per scenario; scenario s owns rows [s * n_per, (s + 1) * n_per) of the block


class TwoStageModel(Model):
    """Two-stage builder (Sec. 8.1, Eq. (extensions) with B = 1; the TwoStageExaCore analog).

    Declarations with `scenario=True` are replicated once per scenario s = 0 .. S-1 (the paper's
    scenarios 1 .. S; the root is stage 0): variable and parameter blocks gain the scenario as last
    index, constraint and objective patterns run over their data once per scenario, with the data
    columns repeated and an int32 field `s` holding the scenario.  Every replicated pattern is still
    one pattern, so it is generated and compiled once and evaluated across all scenarios in one
    launch.  Root declarations are those of `Model`.  Stage tags: `var_stage()` / `con_stage()` give
    0 for the root and s + 1 for scenario s."""

    def __init__(self, nscen: int):
        super().__init__()
        if nscen < 1:
            raise ValueError("a two-stage model needs at least one scenario")
        self.nscen = int(nscen)
        self._vstage: List[tuple] = []  # (start, count, stage) ranges
        self._cstage: List[tuple] = []

    def add_var(self, *shape, scenario: bool = False) -> VarBlock:
        if not scenario:
            b = super().add_var(*shape)
            self._vstage.append((b.offset, b.size, 0))
            return b
        b = ScenarioBlock(self.nvar, tuple(int(v) for v in shape), self.nscen)
        for s in range(self.nscen):
            self._vstage.append((b.offset + s * b.size, b.size, s + 1))
        self.nvar += b.size * self.nscen
        return b

    def add_par(self, values, scenario: bool = False) -> ParBlock:
        """With scenario=True, `values` has the scenario as its last axis."""
        if not scenario:
            return super().add_par(values)
        values = np.asarray(values, dtype=np.float64)
        if values.ndim < 1 or values.shape[-1] != self.nscen:
            raise ValueError("scenario parameter values need the scenario as last axis of length nscen")
        b = ScenarioParBlock(len(self.theta), values.shape[:-1], self.nscen)
        self.theta.extend(np.moveaxis(values, -1, 0).ravel().tolist())
        return b

    def _replicate(self, data: Dict[str, np.ndarray], n: Optional[int]):
        data = dict(data or {})
        if "s" in data:
            raise ValueError("the data field name 's' is reserved for the scenario index")
        names, arrs, types, n = self._table(data, n)
        rep = {k: np.tile(a, self.nscen) for k, a in zip(names, arrs)}
        rep["s"] = np.repeat(np.arange(self.nscen, dtype=np.int32), n)
        return rep, n

    def add_obj(self, fn, data=None, n=None, name: str = "", scenario: bool = False) -> int:
        if not scenario:
            return super().add_obj(fn, data, n, name)
        rep, n = self._replicate(data, n)
        return super().add_obj(fn, rep, n * self.nscen, name)

    def add_con(self, fn, data=None, n=None, name: str = "", scenario: bool = False) -> ConBlock:
        if not scenario:
            blk = super().add_con(fn, data, n, name)
            self._cstage.append((blk.row_base, blk.n_rows, 0))
            return blk
        rep, n = self._replicate(data, n)
        blk = super().add_con(fn, rep, n * self.nscen, name)
        for s in range(self.nscen):
            self._cstage.append((blk.row_base + s * n, n, s + 1))
        return ScenarioConBlock(blk.row_base, blk.n_rows, blk.pattern_index, n_per=n)

    def add_con_aug(self, block: ConBlock, fn, data=None, n=None, name: str = "",
                    scenario: bool = False) -> int:
        """With scenario=True the pattern runs once per scenario and its row index (within one
        scenario's rows of a scenario block) is moved to scenario s's rows."""
        if not scenario:
            return super().add_con_aug(block, fn, data, n, name)
        if not isinstance(block, ScenarioConBlock):
            raise ValueError("a per-scenario augmentation needs a per-scenario constraint block")
        rep, n = self._replicate(data, n)

        def shifted(d):
            idx, val = fn(d)
            return _ilift(idx) + d.s * block.n_per, val
        return super().add_con_aug(block, shifted, rep, n * self.nscen, name)

    def var_stage(self) -> np.ndarray:
        out = np.zeros(self.nvar, dtype=np.int32)
        for a, c, st in self._vstage:
            out[a:a + c] = st
        return out

    def con_stage(self) -> np.ndarray:
        out = np.zeros(self.ncon, dtype=np.int32)
        for a, c, st in self._cstage:
            out[a:a + c] = st
        return out

    def scenario_theta(self, theta: np.ndarray, block: ScenarioParBlock, s: int, values) -> np.ndarray:
        """A copy of `theta` with scenario s's values of a per-scenario parameter block replaced
        (the single-scenario accessor; pass the result to exa_set_theta)."""
        out = np.array(theta, dtype=np.float64, copy=True)
        out[block.scenario_range(s)] = np.asarray(values, dtype=np.float64).ravel()
        return out

@dataclass
class FlatPattern:
    kind: int
    n_inst: int
    row_base: int
    row_limit: int
    row_root: int
    vop: np.ndarray
    va: np.ndarray
    vb: np.ndarray
    vi: np.ndarray
    vf: np.ndarray
    iop: np.ndarray
    ia: np.ndarray
    ib: np.ndarray
    ii: np.ndarray
    ftype: np.ndarray
    fields: List[np.ndarray]
    name: str = ""


@dataclass
class FlatModel:
    nvar: int
    ncon: int
    theta: np.ndarray
    patterns: List[FlatPattern]

    def same_ir(self, other: "FlatModel") -> bool:
        """True when both models have identical pattern trees (batch members)."""
        if len(self.patterns) != len(other.patterns):
            return False
        for p, q in zip(self.patterns, other.patterns):
            if p.kind != q.kind or p.row_root != q.row_root:
                return False
            for a in ("vop", "va", "vb", "vi", "vf", "iop", "ia", "ib", "ii", "ftype"):
                if not np.array_equal(getattr(p, a), getattr(q, a)):
                    return False
        return True


def flatten_pattern(p: Pattern) -> FlatPattern:
    vop, va, vb, vi, vf = [], [], [], [], []
    iop, ia, ib, ii = [], [], [], []

    def emit_i(e: IExpr) -> int:
        if isinstance(e, IConst):
            op, a, b, v = I_CONST, -1, -1, e.v
        elif isinstance(e, IField):
            op, a, b, v = I_FIELD, -1, -1, e.f
        elif isinstance(e, IInst):
            op, a, b, v = I_INST, -1, -1, 0
        else:
            a = emit_i(e.a)
            b = emit_i(e.b)
            op, v = e.op, 0
        iop.append(op); ia.append(a); ib.append(b); ii.append(v)
        return len(iop) - 1

    def emit_v(e: Expr) -> int:
        a = b = -1
        iv, fv = 0, 0.0
        if isinstance(e, Const):
            op, fv = V_CONST, e.v
        elif isinstance(e, Data):
            op, iv = V_DATA, e.f
        elif isinstance(e, Var):
            op, a = V_VAR, emit_i(e.idx)
        elif isinstance(e, Param):
            op, a = V_PARAM, emit_i(e.idx)
        elif isinstance(e, Un):
            a = emit_v(e.a)
            op, iv = e.op, e.n
        elif isinstance(e, Bin):
            a = emit_v(e.a)
            b = emit_v(e.b)
            op = e.op
        else:
            raise TypeError(type(e))
        vop.append(op); va.append(a); vb.append(b); vi.append(iv); vf.append(fv)
        return len(vop) - 1

    emit_v(p.root)
    row_root = emit_i(p.row_expr) if p.kind == K_AUG else -1
    ftype = np.array([F_I32 if f.dtype == np.int32 else F_F64 for f in p.fields], dtype=np.int32)
    return FlatPattern(
        p.kind, p.n_inst, p.row_base, p.row_limit, row_root,
        np.array(vop, np.int32), np.array(va, np.int32), np.array(vb, np.int32),
        np.array(vi, np.int64), np.array(vf, np.float64),
        np.array(iop, np.int32), np.array(ia, np.int32), np.array(ib, np.int32),
        np.array(ii, np.int64), ftype, list(p.fields), p.name)
