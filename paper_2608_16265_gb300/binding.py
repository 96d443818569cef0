"""Thin ctypes binding to libexa.so (include/exa.h).  Argument marshalling only: every step of the
evaluation runs in the library's CUDA kernels.

Module-level functions carry the C names (`exa_create`, `exa_obj`, ...) and take torch CUDA tensors
for device arrays; each call first points the model at torch's current CUDA stream so library work
is ordered with the caller's PyTorch work (and is captured by torch.cuda.graph).  The `Model` class
is a convenience wrapper that allocates outputs.

There is no CPU fallback: if the library cannot be built or loaded, or no sm_103 device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import threading
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build
from . import ir

EXA_OK, EXA_E_INVALID, EXA_E_OOM, EXA_E_NVRTC, EXA_E_CUDA, EXA_E_BOUNDS, EXA_E_TIMEOUT, \
    EXA_E_UNSUPPORTED, EXA_E_INTERNAL = range(9)
EXA_FP64, EXA_MIXED_FP32 = 0, 1
EXA_FLAG_BOUNDS_CHECK, EXA_FLAG_NO_TUNE, EXA_FLAG_NO_FUSE, EXA_FLAG_NO_GRAPH = 1, 2, 4, 8
EXA_FLAG_SPLIT, EXA_FLAG_CSC_SCATTER, EXA_FLAG_NO_HCOMP, EXA_FLAG_UPFRONT = 16, 32, 64, 128
EXA_FLAG_PF_COLUMNS, EXA_FLAG_PF_GATHERS, EXA_FLAG_LANES2, EXA_FLAG_LAZY_LOADS = 256, 512, 1024, 2048
EXA_FLAG_STAGE_SMEM, EXA_FLAG_HOST_SERIAL, EXA_FLAG_FUSED_STEP = 4096, 8192, 16384
STATUS_NAMES = ["EXA_OK", "EXA_E_INVALID", "EXA_E_OOM", "EXA_E_NVRTC", "EXA_E_CUDA", "EXA_E_BOUNDS",
                "EXA_E_TIMEOUT", "EXA_E_UNSUPPORTED", "EXA_E_INTERNAL"]

# Every function include/exa.h declares.
EXPORTS = ["exa_create", "exa_create_batch", "exa_destroy", "exa_last_error", "exa_create_error",
           "exa_dims", "exa_batch_offsets", "exa_set_theta", "exa_set_stream", "exa_obj", "exa_obj_noalloc", "exa_grad", "exa_cons",
           "exa_jac_structure", "exa_jac_coord", "exa_hess_structure", "exa_hess_coord",
           "exa_jac_csc_structure", "exa_hess_csc_structure", "exa_jac_csc", "exa_hess_csc",
           "exa_eval_all", "exa_eval_all_host", "exa_jprod", "exa_jtprod", "exa_hprod", "exa_check_status",
           "exa_debug_hold_step", "exa_compile_check", "exa_stat"]
# Every function include/exa_probe.h declares (measurement, not part of the evaluation path).
PROBE_EXPORTS = ["exa_probe_fp64_fma", "exa_probe_host_link"]


class exa_vnode(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("pad", C.c_int32),
                ("ival", C.c_int64), ("fval", C.c_double)]


class exa_inode(C.Structure):
    _fields_ = [("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32), ("pad", C.c_int32),
                ("ival", C.c_int64)]


class exa_field(C.Structure):
    _fields_ = [("type", C.c_int32), ("pad", C.c_int32), ("data", C.c_void_p)]


class exa_pattern_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_fields", C.c_int32), ("n_inst", C.c_int64),
                ("row_base", C.c_int64), ("row_limit", C.c_int64), ("row_root", C.c_int32),
                ("n_vnodes", C.c_int32), ("n_inodes", C.c_int32), ("pad", C.c_int32),
                ("vnodes", C.POINTER(exa_vnode)), ("inodes", C.POINTER(exa_inode)),
                ("fields", C.POINTER(exa_field))]


class exa_model_desc(C.Structure):
    _fields_ = [("nvar", C.c_int64), ("ncon", C.c_int64), ("npar", C.c_int64),
                ("theta", C.POINTER(C.c_double)), ("n_patterns", C.c_int32), ("pad", C.c_int32),
                ("patterns", C.POINTER(exa_pattern_desc))]


class exa_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("device", C.c_int32), ("block_threads", C.c_int32),
                ("flags", C.c_int32), ("grid_factor", C.c_int32), ("min_blocks", C.c_int32),
                ("chunks", C.c_int32), ("wave_pct", C.c_int32)]


_lib = None
_lock = threading.Lock()


def load():
    """Builds (if stale) and loads libexa.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(_build.build())
        vp, i64p, i32p, dp = C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p
        sig = {
            "exa_create": [C.POINTER(exa_model_desc), C.POINTER(exa_options), C.POINTER(vp)],
            "exa_create_batch": [C.POINTER(C.POINTER(exa_model_desc)), C.c_int32, C.POINTER(exa_options),
                                 C.POINTER(vp)],
            "exa_destroy": [vp],
            "exa_last_error": [vp],
            "exa_create_error": [],
            "exa_dims": [vp, i64p, i64p, i64p, i64p, i64p, i64p],
            "exa_batch_offsets": [vp, C.POINTER(C.c_int32), i64p, i64p, i64p, i64p],
            "exa_set_stream": [vp, vp],
            "exa_set_theta": [vp, C.POINTER(C.c_double), C.c_int64],
            "exa_obj": [vp, dp, dp],
            "exa_obj_noalloc": [vp, dp, dp],
            "exa_grad": [vp, dp, dp],
            "exa_cons": [vp, dp, dp],
            "exa_jac_structure": [vp, i32p, i32p],
            "exa_jac_coord": [vp, dp, dp],
            "exa_hess_structure": [vp, i32p, i32p],
            "exa_hess_coord": [vp, dp, dp, C.c_double, dp],
            "exa_jac_csc_structure": [vp, i32p, i32p, i32p],
            "exa_hess_csc_structure": [vp, i32p, i32p, i32p],
            "exa_jac_csc": [vp, dp, dp],
            "exa_hess_csc": [vp, dp, dp, C.c_double, dp],
            "exa_eval_all": [vp, dp, dp, C.c_double, dp, dp, dp, dp, dp, dp, dp],
            "exa_eval_all_host": [vp, dp, dp, C.c_double, dp, dp, dp, dp, dp, dp, dp],
            "exa_jprod": [vp, dp, dp, dp],
            "exa_jtprod": [vp, dp, dp, dp],
            "exa_hprod": [vp, dp, dp, C.c_double, dp, dp],
            "exa_check_status": [vp],
            "exa_debug_hold_step": [vp, C.c_int32],
            "exa_compile_check": [C.POINTER(exa_model_desc), C.POINTER(exa_options), C.c_char_p, C.c_size_t],
            "exa_stat": [vp, C.c_char_p, C.POINTER(C.c_double)],
            "exa_probe_fp64_fma": [C.c_int32, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int32)],
            "exa_probe_host_link": [C.c_int32, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.exa_destroy.restype = None
        lib.exa_last_error.restype = C.c_char_p
        lib.exa_create_error.restype = C.c_char_p
        _lib = lib
        return lib


class ExaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {msg}")
        self.status = status


# ------------------------------------------------------------------ descriptor marshalling
class _Desc:
    """Keeps the ctypes descriptor of one flat model (and every buffer it points to) alive."""

    def __init__(self, flat: ir.FlatModel):
        self.keep = []
        pats = (exa_pattern_desc * max(1, len(flat.patterns)))()
        for i, p in enumerate(flat.patterns):
            nv, ni = len(p.vop), len(p.iop)
            vn = (exa_vnode * max(1, nv))()
            for j in range(nv):
                vn[j] = exa_vnode(int(p.vop[j]), int(p.va[j]), int(p.vb[j]), 0, int(p.vi[j]), float(p.vf[j]))
            inn = (exa_inode * max(1, ni))()
            for j in range(ni):
                inn[j] = exa_inode(int(p.iop[j]), int(p.ia[j]), int(p.ib[j]), 0, int(p.ii[j]))
            fl = (exa_field * max(1, len(p.fields)))()
            for j, f in enumerate(p.fields):
                f = np.ascontiguousarray(f)
                self.keep.append(f)
                fl[j] = exa_field(int(p.ftype[j]), 0, f.ctypes.data)
            self.keep += [vn, inn, fl]
            pats[i] = exa_pattern_desc(p.kind, len(p.fields), p.n_inst, p.row_base, p.row_limit, p.row_root,
                                       nv, ni, 0, vn, inn, fl)
        theta = np.ascontiguousarray(flat.theta if len(flat.theta) else np.zeros(1), dtype=np.float64)
        self.keep += [pats, theta]
        self.desc = exa_model_desc(flat.nvar, flat.ncon, len(flat.theta),
                                   theta.ctypes.data_as(C.POINTER(C.c_double)), len(flat.patterns), 0, pats)


def _opts(precision, block, flags, device, grid_factor=0, min_blocks=0, chunks=0, wave_pct=0):
    return exa_options(precision, device, block, flags, grid_factor, min_blocks, chunks, wave_pct)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------ ABI-named functions
def exa_create(flat: ir.FlatModel, precision: int = EXA_FP64, block: int = 0, flags: int = 0,
               device: int = 0, grid_factor: int = 0, min_blocks: int = 0, chunks: int = 0,
               wave_pct: int = 0) -> "Model":
    return exa_create_batch([flat], precision, block, flags, device, grid_factor, min_blocks, chunks, wave_pct)


def exa_create_batch(flats: Sequence[ir.FlatModel], precision: int = EXA_FP64, block: int = 0,
                     flags: int = 0, device: int = 0, grid_factor: int = 0, min_blocks: int = 0,
                     chunks: int = 0, wave_pct: int = 0) -> "Model":
    lib = load()
    descs = [_Desc(f) for f in flats]
    arr = (C.POINTER(exa_model_desc) * len(descs))(*[C.pointer(d.desc) for d in descs])
    h = C.c_void_p()
    opt = _opts(precision, block, flags, device, grid_factor, min_blocks, chunks, wave_pct)
    rc = lib.exa_create_batch(arr, len(descs), C.byref(opt), C.byref(h))
    if rc != EXA_OK:
        raise ExaError(rc, lib.exa_create_error().decode())
    return Model(h, len(descs), device)


def exa_compile_check(flat: ir.FlatModel, precision: int = EXA_FP64, block: int = 0, flags: int = 0,
                      min_blocks: int = 0) -> None:
    lib = load()
    d = _Desc(flat)
    buf = C.create_string_buffer(8192)
    rc = lib.exa_compile_check(C.byref(d.desc), C.byref(_opts(precision, block, flags, 0, 0, min_blocks)), buf, 8192)
    if rc != EXA_OK:
        raise ExaError(rc, buf.value.decode(errors="replace"))


def exa_probe_fp64_fma(device: int = 0, target_ms: float = 300.0) -> dict:
    """Measured FP64 FMA rate of the device (include/exa_probe.h): DFMA instructions per second,
    the timed kernel's milliseconds and the SM count."""
    lib = load()
    r, t, n = C.c_double(), C.c_double(), C.c_int32()
    rc = lib.exa_probe_fp64_fma(device, float(target_ms), C.byref(r), C.byref(t), C.byref(n))
    if rc != EXA_OK:
        raise ExaError(rc, "FP64 FMA probe failed")
    return {"dfma_per_s": r.value, "ms": t.value, "sms": n.value}


def exa_probe_host_link(device: int = 0, nbytes: int = 1 << 30) -> dict:
    """Measured host link of the device (include/exa_probe.h): page-locked host <-> device copy
    rates in bytes per second."""
    lib = load()
    h2d, d2h = C.c_double(), C.c_double()
    rc = lib.exa_probe_host_link(device, int(nbytes), C.byref(h2d), C.byref(d2h))
    if rc != EXA_OK:
        raise ExaError(rc, "host link probe failed")
    return {"h2d_bytes_per_s": h2d.value, "d2h_bytes_per_s": d2h.value}


class Model:
    """A created model (opaque handle) with pythonic callbacks over torch CUDA tensors."""

    def __init__(self, handle, nb, device):
        self._h = handle
        self._lib = load()
        self.device = device
        v = [C.c_int64() for _ in range(6)]
        self._call("exa_dims", *[C.byref(t) for t in v], set_stream=False)
        (self.nvar, self.ncon, self.nnzj, self.nnzh, self.nnzj_csc, self.nnzh_csc) = (t.value for t in v)
        nbv = C.c_int32()
        offs = [(C.c_int64 * (nb + 1))() for _ in range(4)]
        self._call("exa_batch_offsets", C.byref(nbv), *offs, set_stream=False)
        self.nb = nbv.value
        self.xoff, self.coff, self.joff, self.hoff = (list(o) for o in offs)

    def _call(self, name, *args, set_stream=True):
        if self._h is None:
            raise ExaError(EXA_E_INVALID, "model destroyed")
        if set_stream:
            self._lib.exa_set_stream(self._h, _stream())
        rc = getattr(self._lib, name)(self._h, *args)
        if rc != EXA_OK:
            raise ExaError(rc, self._lib.exa_last_error(self._h).decode(errors="replace"))

    def destroy(self):
        if self._h is not None:
            self._lib.exa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def tuned_options(self) -> dict:
        """Creation options that reproduce this model's launch configuration without tuning."""
        flags = EXA_FLAG_NO_TUNE
        flags |= EXA_FLAG_SPLIT if self.stat("eval_split") else 0
        flags |= EXA_FLAG_CSC_SCATTER if self.stat("csc_direct") else 0
        flags |= EXA_FLAG_NO_HCOMP if not self.stat("hess_compressed") else 0
        flags |= EXA_FLAG_UPFRONT if self.stat("eval_upfront") else 0
        pf = int(self.stat("eval_prefetch"))
        flags |= EXA_FLAG_PF_GATHERS if pf == 2 else EXA_FLAG_PF_COLUMNS if pf == 1 else 0
        flags |= EXA_FLAG_LANES2 if self.stat("eval_lanes") == 2 else 0
        flags |= EXA_FLAG_LAZY_LOADS if self.stat("eval_lazy") else 0
        flags |= EXA_FLAG_STAGE_SMEM if self.stat("eval_stage") else 0
        flags |= EXA_FLAG_FUSED_STEP if self.stat("eval_fused_step") else 0
        persist = int(self.stat("eval_persist"))
        return dict(block=int(self.stat("eval_block")), min_blocks=int(self.stat("eval_min_blocks")),
                    grid_factor=persist if persist > 0 else -1, flags=flags, chunks=int(self.stat("eval_chunks")),
                    wave_pct=int(self.stat("eval_wave_pct")))

    def stat(self, key: str) -> float:
        v = C.c_double()
        self._call("exa_stat", key.encode(), C.byref(v), set_stream=False)
        return v.value

    # ---- raw calls (outputs preallocated by the caller)
    def exa_obj(self, x, f): self._call("exa_obj", _ptr(x), _ptr(f))
    def exa_obj_noalloc(self, x, f): self._call("exa_obj_noalloc", _ptr(x), _ptr(f))
    def exa_grad(self, x, g): self._call("exa_grad", _ptr(x), _ptr(g))
    def exa_cons(self, x, c): self._call("exa_cons", _ptr(x), _ptr(c))
    def exa_jac_structure(self, r, c): self._call("exa_jac_structure", _ptr(r), _ptr(c))
    def exa_hess_structure(self, r, c): self._call("exa_hess_structure", _ptr(r), _ptr(c))
    def exa_jac_coord(self, x, v): self._call("exa_jac_coord", _ptr(x), _ptr(v))
    def exa_hess_coord(self, x, y, s, v): self._call("exa_hess_coord", _ptr(x), _ptr(y), float(s), _ptr(v))
    def exa_jac_csc_structure(self, cp, rv, m): self._call("exa_jac_csc_structure", _ptr(cp), _ptr(rv), _ptr(m))
    def exa_hess_csc_structure(self, cp, rv, m): self._call("exa_hess_csc_structure", _ptr(cp), _ptr(rv), _ptr(m))
    def exa_jac_csc(self, x, v): self._call("exa_jac_csc", _ptr(x), _ptr(v))
    def exa_hess_csc(self, x, y, s, v): self._call("exa_hess_csc", _ptr(x), _ptr(y), float(s), _ptr(v))

    def exa_eval_all(self, x, y, s, f=None, g=None, c=None, jac=None, hess=None, jac_csc=None, hess_csc=None):
        self._call("exa_eval_all", _ptr(x), _ptr(y), float(s), _ptr(f), _ptr(g), _ptr(c), _ptr(jac),
                   _ptr(hess), _ptr(jac_csc), _ptr(hess_csc))

    def exa_eval_all_host(self, x, y, s, f=None, g=None, c=None, jac=None, hess=None, jac_csc=None, hess_csc=None):
        """exa_eval_all with arrays in host memory (CPU tensors, preferably pinned) or on the device;
        returns when the host outputs are filled."""
        for t in (x, y, f, g, c, jac, hess, jac_csc, hess_csc):
            if t is not None and not t.is_contiguous():
                raise ValueError("exa_eval_all_host takes contiguous tensors")
        self._call("exa_eval_all_host", _ptr(x), _ptr(y), float(s), _ptr(f), _ptr(g), _ptr(c), _ptr(jac),
                   _ptr(hess), _ptr(jac_csc), _ptr(hess_csc))

    def exa_jprod(self, x, v, out): self._call("exa_jprod", _ptr(x), _ptr(v), _ptr(out))
    def exa_jtprod(self, x, w, out): self._call("exa_jtprod", _ptr(x), _ptr(w), _ptr(out))
    def exa_hprod(self, x, y, s, v, out): self._call("exa_hprod", _ptr(x), _ptr(y), float(s), _ptr(v), _ptr(out))
    def exa_check_status(self): self._call("exa_check_status")
    def exa_debug_hold_step(self, member): self._call("exa_debug_hold_step", int(member))

    def exa_set_theta(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float64)
        self._call("exa_set_theta", t.ctypes.data_as(C.POINTER(C.c_double)), len(t))

    # ---- allocating conveniences
    def _empty(self, n, dtype=None):
        import torch
        return torch.empty(max(int(n), 0), dtype=dtype or torch.float64, device=f"cuda:{self.device}")

    def obj(self, x):
        f = self._empty(1)
        self.exa_obj(x, f)
        return f

    def grad(self, x):
        g = self._empty(self.nvar)
        self.exa_grad(x, g)
        return g

    def cons(self, x):
        c = self._empty(self.ncon)
        self.exa_cons(x, c)
        return c

    def jac_structure(self):
        import torch
        r, c = self._empty(self.nnzj, torch.int32), self._empty(self.nnzj, torch.int32)
        self.exa_jac_structure(r, c)
        return r, c

    def hess_structure(self):
        import torch
        r, c = self._empty(self.nnzh, torch.int32), self._empty(self.nnzh, torch.int32)
        self.exa_hess_structure(r, c)
        return r, c

    def jac_coord(self, x):
        v = self._empty(self.nnzj)
        self.exa_jac_coord(x, v)
        return v

    def hess_coord(self, x, y, sigma=1.0):
        v = self._empty(self.nnzh)
        self.exa_hess_coord(x, y, sigma, v)
        return v

    def jac_csc_structure(self):
        import torch
        cp = self._empty(self.nvar + 1, torch.int32)
        rv = self._empty(self.nnzj_csc, torch.int32)
        m = self._empty(self.nnzj, torch.int32)
        self.exa_jac_csc_structure(cp, rv, m)
        return cp, rv, m

    def hess_csc_structure(self):
        import torch
        cp = self._empty(self.nvar + 1, torch.int32)
        rv = self._empty(self.nnzh_csc, torch.int32)
        m = self._empty(self.nnzh, torch.int32)
        self.exa_hess_csc_structure(cp, rv, m)
        return cp, rv, m

    def jac_csc(self, x):
        v = self._empty(self.nnzj_csc)
        self.exa_jac_csc(x, v)
        return v

    def hess_csc(self, x, y, sigma=1.0):
        v = self._empty(self.nnzh_csc)
        self.exa_hess_csc(x, y, sigma, v)
        return v

    def jprod(self, x, v):
        out = self._empty(self.ncon)
        self.exa_jprod(x, v, out)
        return out

    def jtprod(self, x, w):
        out = self._empty(self.nvar)
        self.exa_jtprod(x, w, out)
        return out

    def hprod(self, x, y, sigma, v):
        out = self._empty(self.nvar)
        self.exa_hprod(x, y, sigma, v, out)
        return out

    def eval_all(self, x, y, sigma=1.0, csc=False):
        out = dict(f=self._empty(1), g=self._empty(self.nvar), c=self._empty(self.ncon),
                   jac=self._empty(self.nnzj), hess=self._empty(self.nnzh))
        if csc:
            out.update(jac_csc=self._empty(self.nnzj_csc), hess_csc=self._empty(self.nnzh_csc))
        self.exa_eval_all(x, y, sigma, **out)
        return out
