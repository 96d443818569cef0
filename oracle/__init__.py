"""CPU FP64 oracle for the derivative-evaluation path (test infrastructure).

Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may use this
package.  The GPU library never imports or links it.  It wraps `exa_oracle.c`, a plain
single-threaded C99 evaluator with its own IR reader, structure rule and tape-based AD; see the
header of that file for what each function follows in the paper.

Every function is pinned (tests/test_oracle_pins.py): values printed in the paper, closed forms,
complex-step and finite-difference derivatives, brute force on tiny models and scipy.sparse.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exa_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libexa_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + libm; -O2, no fast-math)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.orc_new.restype = vp
        lib.orc_new.argtypes = [C.c_int64, C.c_int64, C.c_int64, _f64p]
        lib.orc_error.restype = C.c_char_p
        lib.orc_error.argtypes = [vp]
        lib.orc_add_pattern.restype = C.c_int
        lib.orc_add_pattern.argtypes = [vp, C.c_int, C.c_int64, C.c_int64, C.c_int64, C.c_int,
                                        C.c_int, _i32p, _i32p, _i32p, _i64p, _f64p,
                                        C.c_int, _i32p, _i32p, _i32p, _i64p,
                                        C.c_int, _i32p, C.POINTER(C.c_void_p)]
        lib.orc_finalize.restype = C.c_int
        lib.orc_finalize.argtypes = [vp]
        lib.orc_dims.argtypes = [vp, _i64p]
        lib.orc_pattern_info.argtypes = [vp, C.c_int, _i64p]
        lib.orc_pattern_comp.argtypes = [vp, C.c_int, _i32p, _i32p]
        for n in ("orc_jac_structure", "orc_hess_structure"):
            getattr(lib, n).argtypes = [vp, _i32p, _i32p]
        for n in ("orc_jac_csc_structure", "orc_hess_csc_structure"):
            getattr(lib, n).argtypes = [vp, _i32p, _i32p, _i32p]
        lib.orc_obj.argtypes = [vp, _f64p, _f64p]
        lib.orc_cons.argtypes = [vp, _f64p, _f64p]
        lib.orc_grad.argtypes = [vp, _f64p, _f64p]
        lib.orc_grad_coo.argtypes = [vp, _f64p, _f64p, _i32p]
        lib.orc_jac_coord.argtypes = [vp, _f64p, _f64p]
        lib.orc_hess_coord.argtypes = [vp, _f64p, _f64p, C.c_double, _f64p]
        lib.orc_jac_csc.argtypes = [vp, _f64p, _f64p]
        lib.orc_hess_csc.argtypes = [vp, _f64p, _f64p, C.c_double, _f64p]
        lib.orc_jprod.argtypes = [vp, _f64p, _f64p, _f64p]
        lib.orc_jtprod.argtypes = [vp, _f64p, _f64p, _f64p]
        lib.orc_hprod.argtypes = [vp, _f64p, _f64p, C.c_double, _f64p, _f64p]
        lib.orc_obj_complex.argtypes = [vp, _f64p, _f64p, _f64p, _f64p]
        lib.orc_cons_complex.argtypes = [vp, _f64p, _f64p, _f64p, _f64p]
        lib.orc_lag_grad_complex.argtypes = [vp, _f64p, _f64p, _f64p, C.c_double, _f64p, _f64p]
        for n in ("orc_obj", "orc_cons", "orc_grad", "orc_grad_coo", "orc_jac_coord",
                  "orc_hess_coord", "orc_jac_csc", "orc_hess_csc", "orc_jprod", "orc_jtprod",
                  "orc_hprod", "orc_obj_complex", "orc_cons_complex", "orc_lag_grad_complex"):
            getattr(lib, n).restype = C.c_int
        lib.orc_free.argtypes = [vp]
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """The oracle for one model given as flat IR (`paper_2608_16265_gb300.ir.FlatModel`)."""

    def __init__(self, flat):
        lib = _load()
        self._lib = lib
        self._keep = []
        theta = _f64(flat.theta if len(flat.theta) else np.zeros(1))
        self._keep.append(theta)
        self._m = lib.orc_new(flat.nvar, flat.ncon, len(flat.theta), theta)
        for p in flat.patterns:
            ptrs = (C.c_void_p * max(1, len(p.fields)))()
            for i, f in enumerate(p.fields):
                ptrs[i] = f.ctypes.data
            self._keep.extend(p.fields)
            self._keep.append(ptrs)
            rc = lib.orc_add_pattern(self._m, p.kind, p.n_inst, p.row_base, p.row_limit, p.row_root,
                                     len(p.vop), p.vop, p.va, p.vb, p.vi, p.vf,
                                     len(p.iop), p.iop, p.ia, p.ib, p.ii,
                                     len(p.fields), np.ascontiguousarray(p.ftype, np.int32), ptrs)
            self._check(rc)
        self._check(lib.orc_finalize(self._m))
        d = np.zeros(7, np.int64)
        lib.orc_dims(self._m, d)
        (self.nvar, self.ncon, self.nnzj, self.nnzh, self.nnzj_csc, self.nnzh_csc,
         self.nnzg) = (int(v) for v in d)
        self.npat = len(flat.patterns)

    def _check(self, rc):
        if rc != 0:
            raise OracleError(f"oracle error {rc}: {self._lib.orc_error(self._m).decode()}")

    def __del__(self):
        m = getattr(self, "_m", None)
        if m:
            self._lib.orc_free(m)
            self._m = None

    # structure
    def pattern_info(self, i):
        out = np.zeros(5, np.int64)
        self._lib.orc_pattern_info(self._m, i, out)
        return dict(nsym=int(out[0]), o1step=int(out[1]), o2step=int(out[2]),
                    nraw1=int(out[3]), nraw2=int(out[4]))

    def compressors(self, i):
        info = self.pattern_info(i)
        c1 = np.zeros(max(1, info["nraw1"]), np.int32)
        c2 = np.zeros(max(1, info["nraw2"]), np.int32)
        self._lib.orc_pattern_comp(self._m, i, c1, c2)
        return tuple(c1[:info["nraw1"]].tolist()), tuple(c2[:info["nraw2"]].tolist())

    def jac_structure(self):
        r = np.zeros(max(1, self.nnzj), np.int32); c = np.zeros_like(r)
        self._lib.orc_jac_structure(self._m, r, c)
        return r[:self.nnzj], c[:self.nnzj]

    def hess_structure(self):
        r = np.zeros(max(1, self.nnzh), np.int32); c = np.zeros_like(r)
        self._lib.orc_hess_structure(self._m, r, c)
        return r[:self.nnzh], c[:self.nnzh]

    def jac_csc_structure(self):
        cp = np.zeros(self.nvar + 1, np.int32)
        rv = np.zeros(max(1, self.nnzj_csc), np.int32)
        m = np.zeros(max(1, self.nnzj), np.int32)
        self._lib.orc_jac_csc_structure(self._m, cp, rv, m)
        return cp, rv[:self.nnzj_csc], m[:self.nnzj]

    def hess_csc_structure(self):
        cp = np.zeros(self.nvar + 1, np.int32)
        rv = np.zeros(max(1, self.nnzh_csc), np.int32)
        m = np.zeros(max(1, self.nnzh), np.int32)
        self._lib.orc_hess_csc_structure(self._m, cp, rv, m)
        return cp, rv[:self.nnzh_csc], m[:self.nnzh]

    # values
    def _x(self, x):
        x = _f64(x)
        if x.shape != (self.nvar,):
            raise ValueError("x has the wrong length")
        return x

    def _y(self, y):
        y = _f64(y if self.ncon else np.zeros(1))
        return y

    def obj(self, x) -> float:
        f = np.zeros(1)
        self._check(self._lib.orc_obj(self._m, self._x(x), f))
        return float(f[0])

    def grad(self, x):
        g = np.zeros(max(1, self.nvar))
        self._check(self._lib.orc_grad(self._m, self._x(x), g))
        return g[:self.nvar]

    def grad_coo(self, x):
        b = np.zeros(max(1, self.nnzg)); v = np.zeros(max(1, self.nnzg), np.int32)
        self._check(self._lib.orc_grad_coo(self._m, self._x(x), b, v))
        return b[:self.nnzg], v[:self.nnzg]

    def cons(self, x):
        c = np.zeros(max(1, self.ncon))
        self._check(self._lib.orc_cons(self._m, self._x(x), c))
        return c[:self.ncon]

    def jac_coord(self, x):
        v = np.zeros(max(1, self.nnzj))
        self._check(self._lib.orc_jac_coord(self._m, self._x(x), v))
        return v[:self.nnzj]

    def hess_coord(self, x, y, sigma=1.0):
        v = np.zeros(max(1, self.nnzh))
        self._check(self._lib.orc_hess_coord(self._m, self._x(x), self._y(y), float(sigma), v))
        return v[:self.nnzh]

    def jac_csc(self, x):
        v = np.zeros(max(1, self.nnzj_csc))
        self._check(self._lib.orc_jac_csc(self._m, self._x(x), v))
        return v[:self.nnzj_csc]

    def hess_csc(self, x, y, sigma=1.0):
        v = np.zeros(max(1, self.nnzh_csc))
        self._check(self._lib.orc_hess_csc(self._m, self._x(x), self._y(y), float(sigma), v))
        return v[:self.nnzh_csc]

    def jprod(self, x, v):
        out = np.zeros(max(1, self.ncon))
        self._check(self._lib.orc_jprod(self._m, self._x(x), _f64(v), out))
        return out[:self.ncon]

    def jtprod(self, x, w):
        out = np.zeros(max(1, self.nvar))
        self._check(self._lib.orc_jtprod(self._m, self._x(x), self._y(w), out))
        return out[:self.nvar]

    def hprod(self, x, y, sigma, v):
        out = np.zeros(max(1, self.nvar))
        self._check(self._lib.orc_hprod(self._m, self._x(x), self._y(y), float(sigma), _f64(v), out))
        return out[:self.nvar]

    # complex-step helpers
    def obj_complex(self, xr, xi):
        fr = np.zeros(1); fi = np.zeros(1)
        self._check(self._lib.orc_obj_complex(self._m, self._x(xr), self._x(xi), fr, fi))
        return complex(fr[0], fi[0])

    def cons_complex(self, xr, xi):
        cr = np.zeros(max(1, self.ncon)); ci = np.zeros_like(cr)
        self._check(self._lib.orc_cons_complex(self._m, self._x(xr), self._x(xi), cr, ci))
        return cr[:self.ncon] + 1j * ci[:self.ncon]

    def lag_grad_complex(self, xr, xi, y, sigma):
        gr = np.zeros(max(1, self.nvar)); gi = np.zeros_like(gr)
        self._check(self._lib.orc_lag_grad_complex(self._m, self._x(xr), self._x(xi), self._y(y),
                                                   float(sigma), gr, gi))
        return gr[:self.nvar] + 1j * gi[:self.nvar]
