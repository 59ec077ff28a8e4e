"""Thin Python binding of the C ABI in include/cpm.h (argument marshalling only).

Every computation runs in the CUDA library ``libcpm_gb300.so``; this module
only converts arguments.  Device buffers are torch CUDA tensors (float64,
contiguous); streams are torch streams.  There is no CPU fallback: without the
built library, ``load_library`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcpm_gb300.so")

STATUS = {0: "CPM_OK", 1: "CPM_E_ARG", 2: "CPM_E_OOM", 3: "CPM_E_BUDGET", 4: "CPM_E_NOT_SPD", 5: "CPM_E_STATE",
          6: "CPM_E_CUDA", 7: "CPM_E_TIMEOUT", 8: "CPM_E_NONFINITE"}
BOUNDARY = {"3d": 0, "slab": 1, "wire": 2, "ew2d": 3}
PRECISION = {"fp64": 0, "fp32": 1, "bf16x3": 2, "f16x2": 3}
MATRIX = {"A": 0, "S": 1, "SG": 2, "u": 3}
CHOL = {"fp64": 0, "fp32_ir": 1}


class CPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class cpm_tp_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("tau", ctypes.c_double), ("T", ctypes.c_double), ("dv0", ctypes.c_double)]


class cpm_params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("boundary", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("rcut", ctypes.c_double), ("kcut", ctypes.c_double), ("symm", ctypes.c_int32),
                ("s_prec", ctypes.c_int32), ("k_prec", ctypes.c_int32), ("hbm_budget", ctypes.c_size_t),
                ("chol", ctypes.c_int32), ("kspace", ctypes.c_int32), ("p3m_order", ctypes.c_int32),
                ("p3m_mesh", ctypes.c_int32 * 3), ("p3m_matrix", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIGS = {
    "cpm_create": ([ctypes.POINTER(cpm_params), _P, ctypes.POINTER(_P)], _I32),
    "cpm_destroy": ([_P], None),
    "cpm_assemble": ([_P, _I64, _P, _P, _P, _I32], _I32),
    "cpm_invert": ([_P], _I32),
    "cpm_prepare": ([_P, _I64, _P, _P, _P, _I32], _I32),
    "cpm_release_assembly": ([_P], _I32),
    "cpm_export": ([_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "cpm_import": ([_P, _P, ctypes.c_size_t], _I32),
    "cpm_bvec": ([_P, _I32, _I64, _P, _P, _P], _I32),
    "cpm_update": ([_P, _I32, _P, _P, _P, _P], _I32),
    "cpm_step_host": ([_P, _I32, _I64, _P, _P, _P, _P, _P], _I32),
    "cpm_update_ccm": ([_P, _I32, _P, _P, _P, _P, _P], _I32),
    "cpm_update_tp": ([_P, _I32, ctypes.POINTER(cpm_tp_params), _P, _P, _P, _P, _P, _P], _I32),
    "cpm_update_ffield": ([_P, _I32, _P, _P, _P, _P], _I32),
    "cpm_step_graph": ([_P, _I32, _I64, _P, _P, _P, _P, _P, _P], _I32),
    "cpm_sync": ([_P], _I32),
    "cpm_selftest_timeout": ([_P, _D], _I32),
    "cpm_last_error": ([_P], ctypes.c_char_p),
    "cpm_get_matrix": ([_P, _I32, _P], _I32),
    "cpm_capacitance": ([_P, _P], _I32),
    "cpm_kvectors": ([_P, _P, _I64, ctypes.POINTER(_I64)], _I32),
    "cpm_capacitance_ir": ([_P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_D)], _I32),
    "cpm_save": ([_P, ctypes.c_char_p], _I32),
    "cpm_load": ([_P, ctypes.c_char_p], _I32),
    "cpm_device_bytes": ([_P], ctypes.c_size_t),
    "cpm_launch_count": ([_P], _I64),
    "cpm_bvec_noalloc": ([ctypes.POINTER(cpm_params), _I64, _P, _P, _I64, _P, _P, _P, _P], _I32),
    "cpm_gemm_plan": ([_P, _I32, _P, ctypes.POINTER(_D)], _I32),
    "cpm_gemm_set_plan": ([_P, _I32, _P], _I32),
    "cpm_set_s_prec": ([_P, _I32], _I32),
    "cpm_inversion_info": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_D)], _I32),
    "cpm_profile": ([_P, _I32], _I32),
    "cpm_profile_read": ([_P, _I32, ctypes.POINTER(_D), ctypes.POINTER(_I64), _I32], _I32),
}
KERNELS = ["stats", "cells", "real", "phases", "sf", "sfred", "site", "combine", "gemv", "neutral", "col0", "tcgemm",
           "p3m"]


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load the CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CPM CUDA library not built: {p} is missing (run python -m paper_2203_15461_gb300.build)")
    lib = ctypes.CDLL(p)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None and not torch.cuda.is_available():
        return 0   # the library itself reports that no device is usable
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_noalloc_args(site_xyz, site_eta, xyz, Q, b_out) -> None:
    """Sizes, types and devices of cpm_bvec_noalloc's arguments.

    The C entry point receives bare device pointers and cannot see how long the buffers are, so a
    short or mistyped tensor would be read or written past its end on the GPU; everything is
    checked here, before anything is launched (TypeError for a type or device, ValueError for a
    shape)."""
    import torch
    named = {"site_xyz": site_xyz, "site_eta": site_eta, "b_out": b_out}
    if xyz is not None or Q is not None:
        named.update(xyz=xyz, Q=Q)
    for name, t in named.items():
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name}: expected a torch tensor, got {type(t).__name__}")
        if t.dtype != torch.float64:
            raise TypeError(f"{name}: expected float64, got {t.dtype}")
    n = int(site_xyz.shape[0]) if site_xyz.dim() == 2 else -1
    if site_xyz.dim() != 2 or site_xyz.shape[1] != 3 or n < 1:
        raise ValueError(f"site_xyz: expected shape (n, 3) with n >= 1, got {tuple(site_xyz.shape)}")
    if site_eta.numel() != n:
        raise ValueError(f"site_eta: expected {n} values, got {site_eta.numel()}")
    if b_out.numel() < n:
        raise ValueError(f"b_out: expected at least {n} values, got {b_out.numel()}")
    if "xyz" in named:
        if xyz is None or Q is None:
            raise ValueError("xyz and Q: give both or neither")
        if xyz.dim() != 2 or xyz.shape[1] != 3:
            raise ValueError(f"xyz: expected shape (n_e, 3), got {tuple(xyz.shape)}")
        if Q.numel() != xyz.shape[0]:
            raise ValueError(f"Q: expected {xyz.shape[0]} values, got {Q.numel()}")
    devs = {t.device for t in named.values()}
    if len(devs) != 1 or not next(iter(devs)).type == "cuda":
        raise TypeError(f"all tensors must be on one CUDA device, got {sorted(map(str, devs))}")
    if next(iter(devs)).index not in (None, torch.cuda.current_device()):
        raise TypeError(f"tensors are on {next(iter(devs))}, the current device is cuda:{torch.cuda.current_device()}")
    for name, t in named.items():
        if not t.is_contiguous():
            raise TypeError(f"{name}: expected a contiguous tensor")


def cpm_bvec_noalloc(params: cpm_params, site_xyz, site_eta, xyz, Q, b_out, stream=None) -> None:
    """b for one electrolyte configuration without any device allocation (see include/cpm.h).

    For callers that cannot allocate device memory: the library's fixed 4 MiB scratch
    array holds the reciprocal-space grid, shared by all calls (serialise overlapping calls).
    """
    _check_noalloc_args(site_xyz, site_eta, xyz, Q, b_out)
    lib = load_library()
    n_e = int(xyz.shape[0]) if xyz is not None else 0
    st = lib.cpm_bvec_noalloc(ctypes.byref(params), int(site_xyz.shape[0]), _ptr(site_xyz), _ptr(site_eta), n_e,
                              _ptr(xyz) if n_e else None, _ptr(Q) if n_e else None, _ptr(b_out),
                              _P(_stream_handle(stream)))
    if st != 0:
        raise CPMError(st, "cpm_bvec_noalloc failed")


class CPM:
    """One CPM context: one electrode geometry on the current CUDA device and one stream."""

    def __init__(self, box, boundary: str, alpha: float, rcut: float, kcut: float, symm: bool = True,
                 s_prec: str = "fp64", k_prec: str = "fp64", hbm_budget: int = 0, stream=None, chol: str = "fp64",
                 p3m=None, p3m_matrix: bool = False):
        self.lib = load_library()
        p = cpm_params()
        p.box[:] = [float(b) for b in box]
        p.boundary = BOUNDARY[boundary]
        p.alpha, p.rcut, p.kcut = float(alpha), float(rcut), float(kcut)
        p.symm = 1 if symm else 0
        p.s_prec, p.k_prec = PRECISION[s_prec], PRECISION[k_prec]
        p.hbm_budget = int(hbm_budget)
        p.chol = CHOL[chol]
        if p3m is not None:   # (mesh (Kx, Ky, Kz), order): the reciprocal part of b by P3M
            mesh, order = p3m
            p.kspace, p.p3m_order = 1, int(order)
            p.p3m_mesh[:] = [int(v) for v in mesh]
        p.p3m_matrix = 1 if p3m_matrix else 0
        self.params = p
        self.stream = stream
        h = _P()
        st = self.lib.cpm_create(ctypes.byref(p), _P(_stream_handle(stream)), ctypes.byref(h))
        if st != 0:
            raise CPMError(st, "cpm_create failed")
        self.handle = h
        self.n = 0
        self.n_groups = 0

    @classmethod
    def for_electrodes(cls, el, **kw):
        """A context for the electrodes' cell and splitting; P3M when they carry a mesh and an order."""
        if getattr(el, "p3m_order", 0) and "p3m" not in kw:
            kw["p3m"] = (tuple(el.p3m_mesh), el.p3m_order)
            kw.setdefault("p3m_matrix", bool(getattr(el, "p3m_matrix", False)))
        return cls(el.box, el.boundary, el.alpha, el.rcut, el.kcut, **kw)

    # -- plumbing
    def _check(self, st: int):
        if st != 0:
            msg = self.lib.cpm_last_error(self.handle)
            raise CPMError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.cpm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI
    def cpm_assemble(self, xyz, eta, group, n_groups: int):
        self.n, self.n_groups = int(xyz.shape[0]), int(n_groups)
        self._check(self.lib.cpm_assemble(self.handle, self.n, _ptr(xyz), _ptr(eta), _ptr(group), self.n_groups))

    def cpm_invert(self):
        self._check(self.lib.cpm_invert(self.handle))

    def cpm_prepare(self, xyz, eta, group, n_groups: int):
        self.n, self.n_groups = int(xyz.shape[0]), int(n_groups)
        self._check(self.lib.cpm_prepare(self.handle, self.n, _ptr(xyz), _ptr(eta), _ptr(group), self.n_groups))

    def cpm_release_assembly(self):
        self._check(self.lib.cpm_release_assembly(self.handle))

    def cpm_export(self, buf=None):
        """Checkpoint of S, SG and u into ``buf`` (a host tensor or array of uint8; allocated pinned when None)."""
        need = ctypes.c_size_t(0)
        self._check(self.lib.cpm_export(self.handle, None, 0, ctypes.byref(need)))
        if buf is None:
            import torch
            buf = torch.empty(need.value, dtype=torch.uint8, pin_memory=torch.cuda.is_available())
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
        nbytes = buf.numel() if hasattr(buf, "numel") else buf.nbytes
        self._check(self.lib.cpm_export(self.handle, _P(ptr), nbytes, ctypes.byref(need)))
        return buf

    def cpm_import(self, buf):
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else buf.ctypes.data
        nbytes = buf.numel() if hasattr(buf, "numel") else buf.nbytes
        self._check(self.lib.cpm_import(self.handle, _P(ptr), nbytes))

    def cpm_bvec(self, m: int, n_e: int, xyz, Q, b_out):
        self._check(self.lib.cpm_bvec(self.handle, int(m), int(n_e), _ptr(xyz) if n_e else None,
                                      _ptr(Q) if n_e else None, _ptr(b_out)))

    def cpm_update(self, m: int, psi, b, q_out, qtot_out=None):
        self._check(self.lib.cpm_update(self.handle, int(m), _ptr(psi), _ptr(b), _ptr(q_out),
                                        _ptr(qtot_out) if qtot_out is not None else None))

    def cpm_update_ccm(self, m: int, qtilde, b, q_out, qtot_out=None, vtilde_out=None):
        self._check(self.lib.cpm_update_ccm(self.handle, int(m), _ptr(qtilde), _ptr(b), _ptr(q_out),
                                            _ptr(qtot_out) if qtot_out is not None else None,
                                            _ptr(vtilde_out) if vtilde_out is not None else None))

    def cpm_update_tp(self, m: int, dt: float, tau: float, T: float, dv0: float, qcap, X, b, q_out, qcap_out,
                      dv_out=None):
        tp = cpm_tp_params(float(dt), float(tau), float(T), float(dv0))
        self._check(self.lib.cpm_update_tp(self.handle, int(m), ctypes.byref(tp), _ptr(qcap), _ptr(X), _ptr(b),
                                           _ptr(q_out), _ptr(qcap_out), _ptr(dv_out) if dv_out is not None else None))

    def cpm_update_ffield(self, m: int, dv0, b, q_out, qtot_out=None):
        self._check(self.lib.cpm_update_ffield(self.handle, int(m), _ptr(dv0), _ptr(b), _ptr(q_out),
                                               _ptr(qtot_out) if qtot_out is not None else None))

    def cpm_step_host(self, m: int, n_e: int, xyz: np.ndarray, Q: np.ndarray, psi: np.ndarray, q_out: np.ndarray,
                      qtot_out: np.ndarray | None = None):
        def hp(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return a.data_ptr()
            assert a.dtype == np.float64 and a.flags.c_contiguous
            return a.ctypes.data
        self._check(self.lib.cpm_step_host(self.handle, int(m), int(n_e), hp(xyz) if n_e else None,
                                           hp(Q) if n_e else None, hp(psi), hp(q_out), hp(qtot_out)))

    def cpm_step_graph(self, m: int, n_e: int, xyz, Q, psi, b_out, q_out, qtot_out=None):
        self._check(self.lib.cpm_step_graph(self.handle, int(m), int(n_e), _ptr(xyz) if n_e else None,
                                            _ptr(Q) if n_e else None, _ptr(psi), _ptr(b_out), _ptr(q_out),
                                            _ptr(qtot_out) if qtot_out is not None else None))

    def cpm_selftest_timeout(self, wait_ms: float = 50.0) -> str:
        """Run the bounded-wait self test; returns the status name (CPM_E_TIMEOUT when it works)."""
        return STATUS[self.lib.cpm_selftest_timeout(self.handle, float(wait_ms))]

    def cpm_gemm_plan(self, m: int) -> dict:
        """Tile plan of the tensor-core S product for m replicas (tuned on first use; see include/cpm.h)."""
        plan = np.zeros(5, dtype=np.int32)
        ms = _D(0.0)
        self._check(self.lib.cpm_gemm_plan(self.handle, int(m), plan.ctypes.data, ctypes.byref(ms)))
        return {"BN": int(plan[0]), "stages": int(plan[1]), "splits": int(plan[2]), "ctas": int(plan[3]),
                "candidates": int(plan[4]), "ms": float(ms.value)}

    def cpm_inversion_info(self):
        """(refinement sweeps, final residual) of the last FP32-factor inversion."""
        it, res = _I32(0), _D(0.0)
        self._check(self.lib.cpm_inversion_info(self.handle, ctypes.byref(it), ctypes.byref(res)))
        return int(it.value), float(res.value)

    def cpm_set_s_prec(self, s_prec: str):
        self._check(self.lib.cpm_set_s_prec(self.handle, PRECISION[s_prec]))
        self.params.s_prec = PRECISION[s_prec]

    def cpm_gemm_set_plan(self, m: int, BN: int, stages: int, splits: int, ctas: int = 152):
        plan = np.array([BN, stages, splits, ctas], dtype=np.int32)
        self._check(self.lib.cpm_gemm_set_plan(self.handle, int(m), plan.ctypes.data))

    def cpm_sync(self):
        self._check(self.lib.cpm_sync(self.handle))

    def cpm_get_matrix(self, which: str):
        import torch
        shape = {"A": (self.n, self.n), "S": (self.n, self.n), "SG": (self.n, self.n_groups), "u": (self.n,)}[which]
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        self._check(self.lib.cpm_get_matrix(self.handle, MATRIX[which], _ptr(out)))
        return out

    def cpm_capacitance(self) -> np.ndarray:
        C = np.zeros((self.n_groups, self.n_groups))
        self._check(self.lib.cpm_capacitance(self.handle, C.ctypes.data))
        return C

    def cpm_capacitance_ir(self):
        """(C~, refinement sweeps, final residual) from the FP32 factor with FP64 refinement."""
        C = np.zeros((self.n_groups, self.n_groups))
        it, res = _I32(0), _D(0.0)
        self._check(self.lib.cpm_capacitance_ir(self.handle, C.ctypes.data, ctypes.byref(it), ctypes.byref(res)))
        return C, int(it.value), float(res.value)

    def cpm_kvectors(self) -> np.ndarray:
        nk = _I64(0)
        self._check(self.lib.cpm_kvectors(self.handle, None, 0, ctypes.byref(nk)))
        out = np.zeros((max(nk.value, 1), 3), dtype=np.int32)
        self._check(self.lib.cpm_kvectors(self.handle, out.ctypes.data, nk.value, ctypes.byref(nk)))
        return out[:nk.value]

    def cpm_save(self, path: str):
        self._check(self.lib.cpm_save(self.handle, path.encode()))

    def cpm_load(self, path: str):
        self._check(self.lib.cpm_load(self.handle, path.encode()))

    def cpm_launch_count(self) -> int:
        return int(self.lib.cpm_launch_count(self.handle))

    def cpm_device_bytes(self) -> int:
        return int(self.lib.cpm_device_bytes(self.handle))

    def cpm_profile(self, enable: bool):
        self._check(self.lib.cpm_profile(self.handle, 1 if enable else 0))

    def cpm_profile_read(self, reset: bool = False) -> dict:
        """{kernel name: (total ms, launches)} since the last reset."""
        out = {}
        for k, name in enumerate(KERNELS):
            ms, cnt = _D(0.0), _I64(0)
            last = reset and k == len(KERNELS) - 1
            self._check(self.lib.cpm_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(cnt), 1 if last else 0))
            out[name] = (ms.value, cnt.value)
        return out

    # -- conveniences over the same calls
    def setup(self, el):
        """cpm_assemble + cpm_invert for an ``systems.Electrodes`` geometry (inputs copied to the device)."""
        import torch
        dev = "cuda"
        xyz = torch.as_tensor(np.ascontiguousarray(el.xyz, dtype=np.float64), device=dev)
        eta = torch.as_tensor(np.ascontiguousarray(el.eta, dtype=np.float64), device=dev)
        grp = torch.as_tensor(np.ascontiguousarray(el.group, dtype=np.int32), device=dev)
        torch.cuda.synchronize()
        self.cpm_assemble(xyz, eta, grp, el.n_groups)
        self.cpm_invert()
        return self
