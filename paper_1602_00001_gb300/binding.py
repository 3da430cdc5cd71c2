"""Thin Python binding of libpide (include/pide.h): argument marshalling only.

Every step of the computation runs in the CUDA library; torch is used for
device memory, streams and autograd plumbing.  There is no CPU fallback: if
the library is missing or the GPU is not a GB300, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from contextlib import contextmanager

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpide.so")

PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "fp8": 3, "fp8x2": 4, "bf16_fp8": 5, "fp16": 6,
              "fp16_fp8": 7, "auto": 8}
SWEEPS_AUTO = -1          # PIDE_SWEEPS_AUTO: the sweep count pide_setup_auto measured
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ETIMEOUT",
          6: "EUNSUPPORTED"}


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("h", ctypes.c_double)]


class Grid3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("h", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("contraction", ctypes.c_double), ("ms", ctypes.c_double)]


class HandleInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("ld", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("num_sms", ctypes.c_int32), ("store_bytes", ctypes.c_size_t),
                ("setup_ms", ctypes.c_double), ("dims", ctypes.c_int32),
                ("sweeps_hint", ctypes.c_int32)]


class AutoCandidate(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("corr_mask", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("error", ctypes.c_double),
                ("contraction", ctypes.c_double), ("cost", ctypes.c_double)]


class AutoReport(ctypes.Structure):
    _fields_ = [("target", ctypes.c_double), ("nprobe", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("ncand", ctypes.c_int32),
                ("chosen", ctypes.c_int32), ("cand", AutoCandidate * 6)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nprob", ctypes.c_int32), ("simt_items", ctypes.c_int32),
                ("tc_items", ctypes.c_int32), ("tc_items_bn", ctypes.c_int32 * 3),
                ("simt_problems_tn", ctypes.c_int32 * 3), ("tf32_problems", ctypes.c_int32),
                ("apply_launches", ctypes.c_int32)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32 * 5), ("ms", ctypes.c_double * 5)]


class PideError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_LIB = None

_P = ctypes.c_void_p
_I = ctypes.c_int32
_D = ctypes.c_double
_SIGS = {
    "pide_setup": (_I, [ctypes.POINTER(Grid), _P, _I, _P, ctypes.POINTER(_P)]),
    "pide_setup_3d": (_I, [ctypes.POINTER(Grid3), _P, _I, _P, ctypes.POINTER(_P)]),
    "pide_setup_auto": (_I, [ctypes.POINTER(Grid), _P, _D, _P, _I, _I, _P, ctypes.POINTER(_P)]),
    "pide_get_auto_report": (_I, [_P, ctypes.POINTER(AutoReport)]),
    "pide_destroy": (None, [_P]),
    "pide_apply": (_I, [_P, _P, _P, _I, _I, _D, _P, _P, ctypes.POINTER(Info)]),
    "pide_apply_host": (_I, [_P, _P, _P, _I, _I, _D, _P, ctypes.POINTER(Info)]),
    "pide_residual": (_I, [_P, _P, _P, _P, _I, _P]),
    "pide_rhs_from_charge": (_I, [_P, _P, _P, _I, _P]),
    "pide_apply_backward": (_I, [_P, _P, _P, _P, _P, _P, _I, _I, _P]),
    "pide_apply_batched": (_I, [_P, _I, _P, _P, _P, _I, _P]),
    "pide_batch_create": (_I, [_P, _I, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "pide_batch_run": (_I, [_P, _I, _I, _P]),
    "pide_batch_destroy": (None, [_P]),
    "pide_batch_get_info": (_I, [_P, ctypes.POINTER(BatchInfo)]),
    "pide_reserve": (_I, [_P, _I]),
    "pide_apply_noalloc": (_I, [_P, _P, _P, _I, _I, _P]),
    "pide_save": (_I, [_P, ctypes.c_char_p]),
    "pide_load": (_I, [ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "pide_get_handle_info": (_I, [_P, ctypes.POINTER(HandleInfo)]),
    "pide_profile_begin": (_I, [_P]),
    "pide_profile_end": (_I, [_P, ctypes.POINTER(Profile)]),
    "pide_get_inverse_row": (_I, [_P, _I, _P]),
    "pide_set_tuning": (_I, [_P, _I, _I]),
    "pide_get_tuning": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "pide_selftest_wait_timeout": (_I, [ctypes.c_int64, _P]),
    "pide_selftest_convert": (_I, [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P]),
    "pide_selftest_residual_df": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "pide_solve_stream": (_I, [_P, _P, _P, ctypes.c_int64, _I, _I, _I, _P]),
    "pide_round_inverse_decimal": (_I, [_P, _I, _P]),
    "pide_status_string": (ctypes.c_char_p, [_I]),
    "pide_last_error": (ctypes.c_char_p, []),
    "pide_version": (_I, []),
}


_PREC_NAMES = {v: k for k, v in PRECISIONS.items()}


def load_library(path: str = LIB_PATH):
    """Load libpide.so (build it first with ``build.build()``)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libpide.so not found at {path}: run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        msg = _LIB.pide_last_error().decode(errors="replace")
        raise PideError(status, f"{what}: {msg}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _as_dev(x, device):
    import torch
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    x = x.to(device=device, dtype=torch.float64)
    return x.contiguous()


class Solver:
    """One operator (grid + node permittivity) with its stored inverse.

    ``precision``: 'fp64' (plain FP64 inverse and apply), 'fp32', 'bf16',
    'fp8' or 'fp8x2' (low-precision inverse, FP64 refinement), 'fp16' (FP16
    inverse and right-hand sides with power-of-two row / column scales), or
    'bf16_fp8' / 'fp16_fp8' (the BF16 / FP16 inverse plus an e4m3 correction
    term added in the applies that the 'corr_mask' tuning key selects), or
    'auto' (the store measured cheapest for a 0.5e-6 error: pide_setup with
    PIDE_AUTO; ``Solver.auto`` sets the target and the probe).  ``precision``
    then names the store the handle holds.
    """

    def __init__(self, nx: int, ny: int, h: float, eps=None, precision: str = "bf16",
                 stream=None, _handle=None):
        import torch
        self.lib = load_library()
        self.nx, self.ny, self.h = int(nx), int(ny), float(h)
        self.n = (self.nx - 2) * (self.ny - 2)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        if _handle is not None:
            self.handle = _handle
        else:
            g = Grid(self.nx, self.ny, self.h)
            eps_p = None
            self._eps_keep = None
            if eps is not None:
                e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(self.ny, self.nx))
                self._eps_keep = e
                eps_p = e.ctypes.data_as(ctypes.c_void_p)
            h_out = ctypes.c_void_p()
            _check(self.lib.pide_setup(ctypes.byref(g), eps_p, PRECISIONS[precision],
                                       _stream(stream), ctypes.byref(h_out)), "pide_setup")
            self.handle = h_out
        self.eps = None if eps is None else np.asarray(eps, dtype=np.float64).reshape(self.ny, self.nx)
        if self.precision == "auto":
            self.precision = _PREC_NAMES[self.info().precision]

    @classmethod
    def auto(cls, nx: int, ny: int, h: float, eps=None, target: float = 0.5e-6, probe=None,
             nprobe: int = 16, max_sweeps: int = 8, stream=None) -> "Solver":
        """pide_setup_auto: the stored format chosen by the measured refinement
        on ``probe`` ([nprobe][n] float64 right-hand sides on the host; None =
        the library's built-in probes)."""
        lib = load_library()
        g = Grid(int(nx), int(ny), float(h))
        eps_p, keep = None, None
        if eps is not None:
            keep = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(int(ny), int(nx)))
            eps_p = keep.ctypes.data_as(ctypes.c_void_p)
        probe_p = None
        if probe is not None:
            probe = np.ascontiguousarray(np.asarray(probe, dtype=np.float64)).reshape(
                -1, (int(nx) - 2) * (int(ny) - 2))
            nprobe = probe.shape[0]
            probe_p = probe.ctypes.data_as(ctypes.c_void_p)
        h_out = ctypes.c_void_p()
        _check(lib.pide_setup_auto(ctypes.byref(g), eps_p, float(target), probe_p, int(nprobe),
                                   int(max_sweeps), _stream(stream), ctypes.byref(h_out)),
               "pide_setup_auto")
        hi = HandleInfo()
        _check(lib.pide_get_handle_info(h_out, ctypes.byref(hi)), "pide_get_handle_info")
        obj = cls(nx, ny, h, None, _PREC_NAMES[hi.precision], _handle=h_out)
        obj.eps = None if eps is None else keep
        return obj

    def auto_report(self) -> dict:
        """What pide_setup_auto measured: target, probe size, and per candidate
        store its sweeps to the target, error, contraction and modelled cost."""
        r = AutoReport()
        _check(self.lib.pide_get_auto_report(self.handle, ctypes.byref(r)), "pide_get_auto_report")
        cands = [{"precision": _PREC_NAMES[c.precision], "corr_mask": c.corr_mask,
                  "sweeps": c.sweeps, "error": c.error, "contraction": c.contraction,
                  "cost": c.cost} for c in r.cand[:r.ncand]]
        return {"target": r.target, "nprobe": r.nprobe, "max_sweeps": r.max_sweeps,
                "chosen": cands[r.chosen]["precision"], "sweeps": cands[r.chosen]["sweeps"],
                "candidates": cands}

    # -- life cycle
    def close(self):
        if getattr(self, "handle", None):
            self.lib.pide_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> HandleInfo:
        out = HandleInfo()
        _check(self.lib.pide_get_handle_info(self.handle, ctypes.byref(out)), "pide_get_handle_info")
        return out

    # -- step 3 with refinement
    def apply(self, b, u=None, sweeps: int = 0, tol: float = 0.0, g=None, stream=None,
              want_info: bool = False):
        import torch
        b = _as_dev(b, self.device)
        b2 = b.reshape(-1, self.n)
        B = b2.shape[0]
        if u is None:
            u = torch.empty_like(b2)
        gd = _as_dev(g, self.device) if g is not None else None
        info = Info()
        _check(self.lib.pide_apply(self.handle, _ptr(b2), _ptr(u), B, int(sweeps), float(tol),
                                   _ptr(gd), _stream(stream),
                                   ctypes.byref(info) if want_info else None), "pide_apply")
        return (u, info) if want_info else u

    def apply_host(self, b_host: np.ndarray, u_host: np.ndarray | None = None, sweeps: int = 0,
                   tol: float = 0.0, stream=None, want_info: bool = False):
        """Host buffers in and out (numpy float64 [B][n], or pinned torch CPU tensors)."""
        import torch
        if isinstance(b_host, torch.Tensor):
            bptr, B = b_host.data_ptr(), b_host.reshape(-1, self.n).shape[0]
            if u_host is None:
                u_host = torch.empty_like(b_host)
            uptr = u_host.data_ptr()
        else:
            b_host = np.ascontiguousarray(b_host, dtype=np.float64).reshape(-1, self.n)
            B = b_host.shape[0]
            if u_host is None:
                u_host = np.empty_like(b_host)
            bptr, uptr = b_host.ctypes.data, u_host.ctypes.data
        info = Info()
        _check(self.lib.pide_apply_host(self.handle, ctypes.c_void_p(bptr), ctypes.c_void_p(uptr),
                                        B, int(sweeps), float(tol), _stream(stream),
                                        ctypes.byref(info) if want_info else None),
               "pide_apply_host")
        return (u_host, info) if want_info else u_host

    def solve_stream(self, in_host, u_host=None, chunk: int = 1024, sweeps: int = 0,
                     charge: bool = False, stream=None):
        """pide_solve_stream: T right-hand sides (or charge densities) in host
        memory, [T][n] float64 (numpy or pinned torch CPU tensor), solved in
        chunks with the copies overlapping the solves; returns u on the host."""
        import torch
        if isinstance(in_host, torch.Tensor):
            T = in_host.reshape(-1, self.n).shape[0]
            if u_host is None:
                u_host = torch.empty_like(in_host)
            iptr, uptr = in_host.data_ptr(), u_host.data_ptr()
        else:
            in_host = np.ascontiguousarray(in_host, dtype=np.float64).reshape(-1, self.n)
            T = in_host.shape[0]
            if u_host is None:
                u_host = np.empty_like(in_host)
            iptr, uptr = in_host.ctypes.data, u_host.ctypes.data
        _check(self.lib.pide_solve_stream(self.handle, ctypes.c_void_p(iptr), ctypes.c_void_p(uptr),
                                          T, int(chunk), int(sweeps), 1 if charge else 0,
                                          _stream(stream)), "pide_solve_stream")
        return u_host

    def residual(self, b, u, stream=None):
        import torch
        b = _as_dev(b, self.device).reshape(-1, self.n)
        u = _as_dev(u, self.device).reshape(-1, self.n)
        r = torch.empty_like(b)
        _check(self.lib.pide_residual(self.handle, _ptr(b), _ptr(u), _ptr(r), b.shape[0],
                                      _stream(stream)), "pide_residual")
        return r

    def residual_df(self, b, u, g=None, stream=None):
        """The refinement's double-float residual as FP32 (test hook; see pide.h)."""
        import torch
        b = _as_dev(b, self.device).reshape(-1, self.n)
        u = _as_dev(u, self.device).reshape(-1, self.n)
        gp = None
        if g is not None:
            g = _as_dev(g, self.device).reshape(-1)
            gp = _ptr(g)
        r = torch.empty(b.shape, dtype=torch.float32, device=b.device)
        _check(self.lib.pide_selftest_residual_df(self.handle, _ptr(b), _ptr(u), gp, _ptr(r),
                                                  b.shape[0], _stream(stream)),
               "pide_selftest_residual_df")
        return r

    def rhs_from_charge(self, rho, stream=None):
        import torch
        rho = _as_dev(rho, self.device).reshape(-1, self.n)
        b = torch.empty_like(rho)
        _check(self.lib.pide_rhs_from_charge(self.handle, _ptr(rho), _ptr(b), rho.shape[0],
                                             _stream(stream)), "pide_rhs_from_charge")
        return b

    def backward(self, gout, u, b, sweeps: int = 4, stream=None, want_deps: bool = True):
        """(dLoss/db, dLoss/deps) for u = L(eps)^-1 b given gout = dLoss/du
        (deps is None when want_deps is False)."""
        import torch
        gout = _as_dev(gout, self.device).reshape(-1, self.n)
        u = _as_dev(u, self.device).reshape(-1, self.n)
        b = _as_dev(b, self.device).reshape(-1, self.n)
        db = torch.empty_like(gout)
        deps = None
        if want_deps:
            shape = (self.ny, self.nx) if not hasattr(self, "nz") else (self.nz, self.ny, self.nx)
            deps = torch.zeros(shape, dtype=torch.float64, device=self.device)
        _check(self.lib.pide_apply_backward(self.handle, _ptr(gout), _ptr(u), _ptr(b), _ptr(db),
                                            _ptr(deps) if deps is not None else None,
                                            gout.shape[0], int(sweeps), _stream(stream)),
               "pide_apply_backward")
        return db, deps

    TUNE_KEYS = {"gemv_threads": 0, "gemv_unroll": 1, "gemv_max_b": 2, "gemm_bn": 3,
                 "gemm_streamk": 4, "overlap": 5, "resid_ctas": 6, "symv": 7,
                 "resid_emul": 8, "resid_shape": 9,
                 "gemm_2cta": 10, "gemm_a_hint": 11,
                 "resid_prefetch": 12, "corr_mask": 13,
                 "gemm_u_hint": 14, "batch_tc": 15, "batch_bn": 16, "batch_tn": 17,
                 "prep_cluster": 18}

    def set_tuning(self, **kv):
        for k, v in kv.items():
            _check(self.lib.pide_set_tuning(self.handle, self.TUNE_KEYS[k], int(v)),
                   "pide_set_tuning")

    def get_tuning(self) -> dict:
        out = {}
        for k, key in self.TUNE_KEYS.items():
            v = ctypes.c_int32()
            _check(self.lib.pide_get_tuning(self.handle, key, ctypes.byref(v)), "pide_get_tuning")
            out[k] = v.value
        return out

    def reserve(self, Bmax: int):
        _check(self.lib.pide_reserve(self.handle, int(Bmax)), "pide_reserve")

    def round_inverse_decimal(self, digits: int, stream=None):
        """Table 1: round the stored FP64 inverse to `digits` decimals, in place."""
        _check(self.lib.pide_round_inverse_decimal(self.handle, int(digits), _stream(stream)),
               "pide_round_inverse_decimal")

    def inverse_row(self, p: int) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        _check(self.lib.pide_get_inverse_row(self.handle, int(p),
                                             out.ctypes.data_as(ctypes.c_void_p)),
               "pide_get_inverse_row")
        return out

    def save(self, path: str):
        _check(self.lib.pide_save(self.handle, path.encode()), "pide_save")

    @classmethod
    def load(cls, path: str, stream=None) -> "Solver":
        lib = load_library()
        h_out = ctypes.c_void_p()
        _check(lib.pide_load(path.encode(), _stream(stream), ctypes.byref(h_out)), "pide_load")
        hi = HandleInfo()
        _check(lib.pide_get_handle_info(h_out, ctypes.byref(hi)), "pide_get_handle_info")
        inv = {v: k for k, v in PRECISIONS.items()}
        # grid shape is in the file header; read it back from the header bytes
        import struct
        with open(path, "rb") as f:
            head = f.read(56 + 8)
        _, version, nx, ny, prec, n, ld = struct.unpack("<8s6i", head[:32])
        (h,) = struct.unpack("<d", head[32:40])
        if version == 2:                          # 3-D: nz follows the 56-byte header
            (nz, _dims) = struct.unpack("<2i", head[56:64])
            obj = Solver3D.__new__(Solver3D)
            import torch
            obj.lib = lib
            obj.nx, obj.ny, obj.nz, obj.h = nx, ny, nz, h
            obj.n = (nx - 2) * (ny - 2) * (nz - 2)
            obj.precision = inv[hi.precision]
            obj.device = torch.device("cuda", torch.cuda.current_device())
            obj.handle = h_out
            obj.eps = None
            obj._eps_keep = None
            return obj
        return cls(nx, ny, h, None, inv[hi.precision], _handle=h_out)

    @contextmanager
    def profile(self):
        """Event-time every kernel launched inside the block; yields a dict
        filled at exit: {'apply': (launches, ms), 'residual': ..., 'prep': ..., 'other': ...,
        'reduce': ...} ('reduce': the sums of a tensor-core apply's K-split last round)."""
        out: dict = {}
        _check(self.lib.pide_profile_begin(self.handle), "pide_profile_begin")
        try:
            yield out
        finally:
            p = Profile()
            _check(self.lib.pide_profile_end(self.handle, ctypes.byref(p)), "pide_profile_end")
            for i, name in enumerate(["apply", "residual", "prep", "other", "reduce"]):
                out[name] = (int(p.launches[i]), float(p.ms[i]))


class Solver3D(Solver):
    """The same on an nx x ny x nz node grid (pide_setup_3d): eps is
    [nz][ny][nx]; right-hand sides and solutions are [B][(nx-2)(ny-2)(nz-2)],
    x fastest; boundary values g are [nz][ny][nx]."""

    def __init__(self, nx: int, ny: int, nz: int, h: float, eps=None, precision: str = "bf16",
                 stream=None):
        import torch
        self.lib = load_library()
        self.nx, self.ny, self.nz, self.h = int(nx), int(ny), int(nz), float(h)
        self.n = (self.nx - 2) * (self.ny - 2) * (self.nz - 2)
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device())
        g = Grid3(self.nx, self.ny, self.nz, self.h)
        eps_p = None
        self._eps_keep = None
        if eps is not None:
            e = np.ascontiguousarray(
                np.asarray(eps, dtype=np.float64).reshape(self.nz, self.ny, self.nx))
            self._eps_keep = e
            eps_p = e.ctypes.data_as(ctypes.c_void_p)
        h_out = ctypes.c_void_p()
        _check(self.lib.pide_setup_3d(ctypes.byref(g), eps_p, PRECISIONS[precision],
                                      _stream(stream), ctypes.byref(h_out)), "pide_setup_3d")
        self.handle = h_out
        self.eps = None if eps is None else self._eps_keep
        if self.precision == "auto":
            self.precision = _PREC_NAMES[self.info().precision]


def apply_batched(solvers, bs, us, sweeps: int = 2, stream=None):
    """pide_apply_batched over several solvers (uneven grids, ragged B)."""
    lib = load_library()
    k = len(solvers)
    hs = (ctypes.c_void_p * k)(*[s.handle.value for s in solvers])
    bp = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
    up = (ctypes.c_void_p * k)(*[u.data_ptr() for u in us])
    Bs = (ctypes.c_int32 * k)(*[b.reshape(-1, s.n).shape[0] for b, s in zip(bs, solvers)])
    _check(lib.pide_apply_batched(hs, k, bp, up, Bs, int(sweeps), _stream(stream)),
           "pide_apply_batched")


class BatchPlan:
    """pide_batch_create / run / destroy: the uneven-grid batched apply with
    optional CUDA-graph replay (buffers are fixed in the plan)."""

    def __init__(self, solvers, bs, us, sweeps_per_problem=None, tune_cache=None):
        """tune_cache: an autotune.TuneCache whose batched-plan entries are set
        on each solver (by precision, n and B bucket) before the plan is built."""
        self.lib = load_library()
        k = len(solvers)
        if tune_cache is not None:
            from . import autotune
            for s, b in zip(solvers, bs):
                autotune.apply_cached_batch(s, b.reshape(-1, s.n).shape[0], cache=tune_cache)
        self._keep = (solvers, bs, us)
        sk = None
        if sweeps_per_problem is not None:
            sk = (ctypes.c_int32 * k)(*[int(x) for x in sweeps_per_problem])
        hs = (ctypes.c_void_p * k)(*[s.handle.value for s in solvers])
        bp = (ctypes.c_void_p * k)(*[b.data_ptr() for b in bs])
        up = (ctypes.c_void_p * k)(*[u.data_ptr() for u in us])
        Bs = (ctypes.c_int32 * k)(*[b.reshape(-1, s.n).shape[0] for b, s in zip(bs, solvers)])
        out = ctypes.c_void_p()
        _check(self.lib.pide_batch_create(hs, k, bp, up, Bs, sk, ctypes.byref(out)),
               "pide_batch_create")
        self.plan = out

    def info(self) -> dict:
        """The shapes the plan launches (pide_batch_get_info)."""
        bi = BatchInfo()
        _check(self.lib.pide_batch_get_info(self.plan, ctypes.byref(bi)), "pide_batch_get_info")
        return {"nprob": bi.nprob, "simt_items": bi.simt_items, "tc_items": bi.tc_items,
                "tc_items_bn": {32: bi.tc_items_bn[0], 64: bi.tc_items_bn[1],
                                128: bi.tc_items_bn[2]},
                "simt_problems_tn": {16: bi.simt_problems_tn[0], 32: bi.simt_problems_tn[1],
                                     64: bi.simt_problems_tn[2]},
                "tf32_problems": bi.tf32_problems, "apply_launches": bi.apply_launches}

    def run(self, sweeps: int = 2, use_graph: bool = True, stream=None):
        _check(self.lib.pide_batch_run(self.plan, int(sweeps), 1 if use_graph else 0,
                                       _stream(stream)), "pide_batch_run")

    def close(self):
        if getattr(self, "plan", None):
            self.lib.pide_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def header_symbols(header: str | None = None):
    """Names of the functions include/pide.h declares."""
    import re
    header = header or os.path.join(HERE, "..", "include", "pide.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(pide_[a-z_0-9]+)\s*\(", text)))


def _autograd():
    import torch

    class PideApply(torch.autograd.Function):
        """u = L(eps)^-1 b with the refined apply; backward through the adjoint
        kernels (dLoss/db = D mu, dLoss/deps via the face gradient)."""

        @staticmethod
        def forward(ctx, b, eps, solver, sweeps):
            u = solver.apply(b, sweeps=sweeps)
            ctx.solver, ctx.sweeps = solver, sweeps
            ctx.save_for_backward(b, u)
            return u.reshape(b.shape)

        @staticmethod
        def backward(ctx, gout):
            b, u = ctx.saved_tensors
            db, deps = ctx.solver.backward(gout.contiguous(), u, b, sweeps=ctx.sweeps)
            return db.reshape(b.shape), deps, None, None

    return PideApply


_PIDE_APPLY = None


def pide_apply_autograd(b, eps_t, solver: Solver, sweeps: int = 4):
    """Differentiable apply: gradients flow to b and to the node permittivity
    tensor eps_t ([ny][nx], the values the solver was built with)."""
    global _PIDE_APPLY
    if _PIDE_APPLY is None:
        _PIDE_APPLY = _autograd()
    return _PIDE_APPLY.apply(b, eps_t, solver, sweeps)
