"""Python binding of the GB300 temporally blocked stencil library (``libgirih.so``).

Thin ctypes marshalling over the C ABI declared in ``include/girih.h``: every step of a sweep
runs in the library's CUDA kernels; PyTorch only provides device memory and streams.  There is
no CPU fallback: if the library has not been built, importing works but every call raises.

    import paper_1510_04995_gb300 as girih
    p = girih.plan(girih.S7C, 512, 512, 512, dtype="f64", T=64)
    girih.run(p, u, u_prev)              # u, u_prev: CUDA tensors of shape p.shape
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgirih.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "girih.h")

S7C, S7V, S25C, S25V, S25CG, S27B, S7RB = 0, 1, 2, 3, 4, 5, 6
F64, F32 = 0, 1
NAIVE, MWD = 0, 1
FED, RELAXED, FED_BULK, FED_ELEM, RELAXED_ELEM, FED_PERSISTENT, RELAXED_PERSISTENT, OVERLAP_PERSISTENT = (
    0, 1, 2, 3, 4, 5, 6, 7)
RADIUS = {0: 1, 1: 1, 2: 4, 3: 4, 4: 4, 5: 1, 6: 1}
NCOEF = {0: 0, 1: 7, 2: 0, 3: 13, 4: 1, 5: 0, 6: 0}
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EKERNEL", 5: "ETIMEOUT", 6: "ENOTIMPL"}
MLP_FEATURES = 16
MLP_HIDDEN = 64
MLP_STATIC_MAX_ROWS = 4096


class GirihError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("dw", ctypes.c_int32), ("nf", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("threads", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("zseg", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def __repr__(self):
        return "Config(%s)" % ", ".join(f"{k}={v}" for k, v in self.as_dict().items())


class Params(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 5), ("force_cfg", ctypes.c_int32), ("cfg", Config)]


class TuneRow(ctypes.Structure):
    _fields_ = [("cfg", Config), ("glups", ctypes.c_double), ("seconds", ctypes.c_double),
                ("steps", ctypes.c_int64), ("smem", ctypes.c_int64), ("tune_seconds", ctypes.c_double)]


def config(algo=MWD, dw=8, nf=1, cluster=1, threads=256, variant=FED, zseg=0) -> Config:
    return Config(algo, dw, nf, cluster, threads, variant, zseg)


def config_array(cfgs):
    """(ctypes array, count) of configurations for the tuner calls; (None, 0) for all candidates."""
    if cfgs is None:
        return None, 0
    arr = (Config * len(cfgs))(*cfgs)
    return arr, len(cfgs)


_lib = None
_VP, _I32, _I64, _F32, _F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
_SIGS = {
    "girih_plan": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _I64, _I64, _I64, _I64, _I32, _I64]),
    "girih_plan_destroy": (ctypes.c_int, [_VP]),
    "girih_plan_get_config": (ctypes.c_int, [_VP, ctypes.POINTER(Config)]),
    "girih_plan_set_config": (ctypes.c_int, [_VP, ctypes.POINTER(Config)]),
    "girih_config_check": (ctypes.c_int, [_VP, ctypes.POINTER(Config), ctypes.POINTER(_I64)]),
    "girih_run": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(Params), _VP]),
    "girih_run_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(Params), _VP]),
    "girih_status": (ctypes.c_int, [_VP, _VP]),
    "girih_plan_layout": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "girih_plan_launch_count": (ctypes.c_int, [_VP, ctypes.POINTER(Config), ctypes.POINTER(_I64)]),
    "girih_last_error": (ctypes.c_char_p, []),
    "girih_model_cache_block": (_F64, [_F64, _I32, _I32, _I32, _I32]),
    "girih_model_code_balance": (_F64, [_I32, _I32, _I32, _I32]),
    "girih_check_bounded_wait": (ctypes.c_int, [_VP, _I64, _VP]),
    "girih_measure_fma_rate": (ctypes.c_int, [_I32, ctypes.POINTER(_F64), ctypes.POINTER(_F64), _VP]),
    "girih_tune_candidates": (ctypes.c_int, [_VP, ctypes.POINTER(Config), _I32, ctypes.POINTER(_I32)]),
    "girih_tune_measure": (ctypes.c_int, [_VP, ctypes.POINTER(Config), _F64, _I64, ctypes.POINTER(TuneRow)]),
    "girih_tune_exhaustive": (ctypes.c_int, [_VP, ctypes.POINTER(Config), _I32, _F64, _I64, ctypes.c_char_p,
                                             ctypes.POINTER(TuneRow), ctypes.POINTER(_I32)]),
    "girih_mlp_features": (ctypes.c_int, [_I32, _I32, _I64, _I64, _I64, ctypes.POINTER(Config), _VP]),
    "girih_mlp_num_params": (_I64, [_I32]),
    "girih_mlp_workspace_floats": (_I64, [_I32]),
    "girih_mlp_forward": (ctypes.c_int, [_VP, _VP, _I32, _I32, _VP, _VP, _VP]),
    "girih_mlp_backward": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _VP, _VP, _VP, _VP]),
    "girih_mlp_backward_static": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _VP, _VP, _VP]),
    "girih_mlp_sgd": (ctypes.c_int, [_VP, _VP, _I64, _F32, _VP]),
    "girih_mlp_adam": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _I64, _F32, _F32, _F32, _F32, _VP]),
    "girih_tune_learned": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(Config), _I32, _I32, _F64, _I64,
                                          ctypes.POINTER(TuneRow), ctypes.POINTER(_I32)]),
}


def lib():
    """Load libgirih.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1510_04995_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols():
    """Names of every function the public header declares."""
    with open(HEADER) as f:
        return re.findall(r"GIRIH_API\s+[\w\s\*]+?\b(girih_\w+)\s*\(", f.read())


def last_error() -> str:
    return (lib().girih_last_error() or b"").decode()


def check(rc: int):
    if rc != 0:
        raise GirihError(rc, last_error())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


_DT = {"f64": F64, "float64": F64, F64: F64, "f32": F32, "float32": F32, F32: F32}


class Plan:
    """Owns a girih_plan_t: the problem (stencil, sizes, dtype, T) and the chosen configuration."""

    def __init__(self, stencil, nx, ny, nz, dtype="f64", T=1, ldx=0):
        self.stencil, self.nx, self.ny, self.nz, self.T = int(stencil), int(nx), int(ny), int(nz), int(T)
        self.dtype = _DT[dtype]
        self._h = ctypes.c_void_p()
        check(lib().girih_plan(ctypes.byref(self._h), self.stencil, self.nx, self.ny, self.nz, int(ldx),
                               self.dtype, self.T))
        n, r, ld = _I64(), _I32(), _I64()
        check(lib().girih_plan_layout(self._h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(ld)))
        self.elems, self.R, self.ldx = n.value, r.value, ld.value
        self.shape = (self.nz + 2 * self.R, self.ny + 2 * self.R, self.ldx)

    @property
    def handle(self):
        return self._h

    @property
    def config(self) -> Config:
        c = Config()
        check(lib().girih_plan_get_config(self._h, ctypes.byref(c)))
        return c

    def set_config(self, cfg: Config):
        check(lib().girih_plan_set_config(self._h, ctypes.byref(cfg)))

    def check_config(self, cfg: Config):
        """Shared memory bytes per block if feasible, else raise GirihError."""
        s = _I64()
        check(lib().girih_config_check(self._h, ctypes.byref(cfg), ctypes.byref(s)))
        return s.value

    def feasible(self, cfg: Config) -> bool:
        return lib().girih_config_check(self._h, ctypes.byref(cfg), None) == 0

    def candidates(self) -> list:
        """The tuner's candidate configurations for this plan (girih_tune_candidates)."""
        n = _I32()
        check(lib().girih_tune_candidates(self._h, None, 0, ctypes.byref(n)))
        arr = (Config * max(n.value, 1))()
        check(lib().girih_tune_candidates(self._h, arr, n.value, ctypes.byref(n)))
        return list(arr[:n.value])

    def launch_count(self, cfg: Config | None = None) -> int:
        n = _I64()
        check(lib().girih_plan_launch_count(self._h, ctypes.byref(cfg) if cfg is not None else None,
                                            ctypes.byref(n)))
        return n.value

    def close(self):
        if self._h:
            lib().girih_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan(stencil, nx, ny, nz, dtype="f64", T=1, ldx=0) -> Plan:
    return Plan(stencil, nx, ny, nz, dtype, T, ldx)


def _params(c, cfg):
    p = Params()
    if c is not None:
        for i, v in enumerate(c):
            p.c[i] = float(v)
    if cfg is not None:
        p.force_cfg = 1
        p.cfg = cfg
    return p


def _default_c(stencil):
    return (0.4, 0.1) if stencil == S7C else ((-0.9, 0.05, 0.025, 0.0125, 0.00625) if stencil == S25C else ())


def run(p: Plan, u, u_prev, coeffs=None, c=None, cfg: Config | None = None, stream=None):
    """Advance CUDA tensors u, u_prev (shape p.shape) by p.T steps; coeffs [ncoef, *p.shape]."""
    import torch
    want = torch.float64 if p.dtype == F64 else torch.float32
    for name, t in (("u", u), ("u_prev", u_prev)) + ((("coeffs", coeffs),) if coeffs is not None else ()):
        if not t.is_cuda or t.dtype != want or not t.is_contiguous():
            raise GirihError(1, f"{name} must be a contiguous CUDA tensor of dtype {want}")
    if tuple(u.shape) != p.shape or tuple(u_prev.shape) != p.shape:
        raise GirihError(1, f"u and u_prev must have shape {p.shape}")
    if NCOEF[p.stencil]:
        if coeffs is None or tuple(coeffs.shape) != (NCOEF[p.stencil],) + p.shape:
            raise GirihError(1, f"coeffs must have shape {(NCOEF[p.stencil],) + p.shape}")
    prm = _params(c if c is not None else _default_c(p.stencil), cfg)
    check(lib().girih_run(p.handle, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u_prev.data_ptr()),
                          ctypes.c_void_p(coeffs.data_ptr()) if coeffs is not None else None,
                          ctypes.byref(prm), _stream_handle(stream)))


def status(p: Plan, stream=None):
    """Synchronise and raise GirihError if a device-side wait of a previous run ran out."""
    check(lib().girih_status(p.handle, _stream_handle(stream)))


def run_host(p: Plan, u, u_prev, coeffs=None, c=None, cfg: Config | None = None, stream=None):
    """Same as run() for host arrays (numpy or CPU tensors, pinned or not); synchronises."""
    def ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr())
        return a.ctypes.data_as(ctypes.c_void_p)
    prm = _params(c if c is not None else _default_c(p.stencil), cfg)
    check(lib().girih_run_host(p.handle, ptr(u), ptr(u_prev), ptr(coeffs), ctypes.byref(prm),
                               _stream_handle(stream)))


def measure_fma_rate(dtype="f64", stream=None):
    """(FMA instructions per second, seconds of the timed launch) of the current GPU in dtype."""
    rate, secs = _F64(), _F64()
    check(lib().girih_measure_fma_rate(_DT[dtype], ctypes.byref(rate), ctypes.byref(secs), _stream_handle(stream)))
    return rate.value, secs.value


def model_cache_block(n_xb, dw, nf, r, nd) -> float:
    """C_S of Eq. 3 in bytes."""
    return lib().girih_model_cache_block(float(n_xb), int(dw), int(nf), int(r), int(nd))


def model_code_balance(dw, r, nd, elem_bytes=8) -> float:
    """B_C of Eq. 5 in bytes per LUP."""
    return lib().girih_model_code_balance(int(dw), int(r), int(nd), int(elem_bytes))
