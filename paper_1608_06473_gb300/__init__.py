"""GB300 two-scale HHG multigrid: Python binding of libhhg.so.

Argument marshalling only.  Every step of the method (setup of the shell
hierarchy, the LSQP surrogate fit, operator application, smoothing, residual,
transfers and the V-cycle) runs in the CUDA library whose C ABI is declared in
include/hhg.h; the functions below carry the same names and arguments.
Vectors are torch CUDA tensors (device pointers) or NumPy arrays (host
pointers, copied by the library); `stream` defaults to torch's current CUDA
stream.  There is no fallback: without libhhg.so every call raises.

Method: Bauer et al., "A two-scale approach for efficient on-the-fly operator
assembly in massively parallel high performance multigrid codes"
(arXiv:1608.06473).
"""
from __future__ import annotations

import ctypes
import os
from enum import IntEnum

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhhg.so")

HHG_OK, HHG_EINVAL, HHG_ENOMEM, HHG_ECUDA, HHG_ENOTFIT, HHG_ENOCONV, HHG_EDIVERGED, HHG_ETIMEOUT = \
    0, -1, -2, -3, -4, -5, -6, -7
HHG_OP_IFEM, HHG_OP_LSQP, HHG_OP_DD = 0, 1, 2
HHG_F64, HHG_F32 = 0, 1


class Status(IntEnum):
    OK = 0
    EINVAL = -1
    ENOMEM = -2
    ECUDA = -3
    ENOTFIT = -4
    ENOCONV = -5
    EDIVERGED = -6
    ETIMEOUT = -7


class HHGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{Status(status).name}: {msg}")
        self.status = Status(status)


class hhg_shell_desc(ctypes.Structure):
    _fields_ = [("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double), ("tang_refine", ctypes.c_int),
                ("radial_layers", ctypes.c_int), ("fine_log2_intervals", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("unprojected", ctypes.c_int)]


class hhg_server_desc(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int), ("q", ctypes.c_int),
                ("j", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("rtol", ctypes.c_double), ("dtype", ctypes.c_int), ("max_batch_rhs", ctypes.c_int)]


class hhg_problem(ctypes.Structure):
    _fields_ = [("r_inner", ctypes.c_double), ("r_outer", ctypes.c_double), ("tang_refine", ctypes.c_int),
                ("radial_layers", ctypes.c_int), ("L", ctypes.c_int)]


class hhg_request_info(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_end", ctypes.c_double),
                ("cycles", ctypes.c_int), ("reused", ctypes.c_int), ("status", ctypes.c_int),
                ("batch_rhs", ctypes.c_int)]


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "hhg_setup_shell": [ctypes.POINTER(hhg_shell_desc), _P, ctypes.POINTER(_P)],
    "hhg_destroy": [_P],
    "hhg_setup_shells": [ctypes.POINTER(hhg_shell_desc), _I, _P, ctypes.POINTER(_P)],
    "hhg_shell_part": [_P, _I, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "hhg_num_nodes": [_P, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "hhg_node_coords": [_P, _I, _P],
    "hhg_fit_surrogate": [_P, _I, _I, _P],
    "hhg_fit_ipoly": [_P, _P],
    "hhg_fit_cons": [_P, _I, _I, _P],
    "hhg_fit_ipoly_degree": [_P, _I, _P],
    "hhg_load_vector": [_P, _I, _P, _P, _P],
    "hhg_apply": [_P, _I, _I, _I, _P, _P, _I, _P],
    "hhg_residual": [_P, _I, _I, _I, _P, _P, _P, _I, _P, _P],
    "hhg_smooth": [_P, _I, _I, _I, _P, _P, _I, _I, _P],
    "hhg_vcycle": [_P, _I, _I, _P, _P, _I, _I, _I, ctypes.c_double, _I, _P, _P, _P],
    "hhg_residual_noalloc": [_P, _I, _I, _P, _P, _P, _P, _P],
    "hhg_problem_nodes": [ctypes.POINTER(hhg_problem), ctypes.POINTER(ctypes.c_int64),
                          ctypes.POINTER(ctypes.c_int64)],
    "hhg_server_create": [ctypes.POINTER(hhg_server_desc), ctypes.POINTER(_P)],
    "hhg_server_submit": [_P, ctypes.POINTER(hhg_problem), _P, _I, ctypes.POINTER(ctypes.c_int64)],
    "hhg_server_wait": [_P, ctypes.c_int64, _P, _P, ctypes.POINTER(hhg_request_info)],
    "hhg_server_stats": [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "hhg_server_destroy": [_P],
    "hhg_timing": [_P, _I],
    "hhg_tuning": [_P, _I, ctypes.POINTER(ctypes.c_int), _P],
    "hhg_set_tuning": [_P, _I, _I],
    "hhg_set_fp64_kernel": [_P, _I],
    "hhg_fp64_kernel": [_P, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "hhg_run_lists": [_I, _P, ctypes.c_int64, _P, _P, ctypes.POINTER(ctypes.c_int64)],
    "hhg_slab_planes": [_I, _I, _P],
    "hhg_set_graphs": [_P, _I],
    "hhg_timing_read": [_P, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
    "hhg_peak_rate": [_I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P],
    "hhg_check_arith": [_I, _P, _P, _P, ctypes.c_int64, _P],
}


def lib() -> ctypes.CDLL:
    """The loaded libhhg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1608_06473_gb300._build` "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.hhg_last_error.argtypes = []
        L.hhg_last_error.restype = ctypes.c_char_p
        L.hhg_launch_count.argtypes = []
        L.hhg_launch_count.restype = ctypes.c_int64
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS) + ["hhg_last_error", "hhg_launch_count"]


HHG_T_CELL_SMOOTH, HHG_T_CELL_RESIDUAL, HHG_T_CELL_APPLY = 0, 1, 2
HHG_T_COARSE, HHG_T_FIT, HHG_T_SMOOTH, HHG_T_RESIDUAL, HHG_T_TRANSFER = 3, 4, 5, 6, 7
TIMERS = {"cell_smooth_finest": 0, "cell_residual_finest": 1, "cell_apply_finest": 2, "coarse_solve": 3, "fit": 4,
          "smooth_all_levels": 5, "residual_all_levels": 6, "transfers": 7}


def hhg_launch_count() -> int:
    return lib().hhg_launch_count()


def hhg_timing(shell: int, enable: bool):
    _check(lib().hhg_timing(shell, int(bool(enable))))


def hhg_timing_read(shell: int, which: int):
    """(total device ms, launches) of one timed kernel class."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().hhg_timing_read(shell, which, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


PEAK_FP64_FMA, PEAK_FP32_FMA, PEAK_INT32_IMAD = 0, 1, 2


def hhg_peak_rate(kind: int, stream=None):
    """(multiply-adds per second, ms of the best timed run) of one arithmetic
    pipe on the current device (kind: PEAK_FP64_FMA, PEAK_FP32_FMA,
    PEAK_INT32_IMAD)."""
    r, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().hhg_peak_rate(kind, ctypes.byref(r), ctypes.byref(ms), _stream(stream)))
    return r.value, ms.value


def hhg_check_arith(which: int, a, b, out, n: int, stream=None):
    """The kernels' hand-written arithmetic helpers applied elementwise
    (which 0: FP32 divide, 1: 2^E / W on the integer pipe, 2: W 2^-E on the
    integer pipe; W int64, E int32); device tensors."""
    _check(lib().hhg_check_arith(which, _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)))


def hhg_tuning(shell: int, L: int):
    """(chosen FP32 smoother configuration, per-candidate ms) of level L."""
    cfg = ctypes.c_int()
    ms = np.zeros(10)
    _check(lib().hhg_tuning(shell, L, ctypes.byref(cfg), ms.ctypes.data))
    return cfg.value, ms


def hhg_set_graphs(shell: int, enable: bool):
    _check(lib().hhg_set_graphs(shell, int(bool(enable))))


def hhg_set_tuning(shell: int, L: int, cfg: int):
    _check(lib().hhg_set_tuning(shell, L, cfg))


FP64_NODES, FP64_RUNS, FP64_RESIDENT = 0, 1, 2


def hhg_set_fp64_kernel(shell: int, variant: int):
    _check(lib().hhg_set_fp64_kernel(shell, variant))


def hhg_run_lists(N: int):
    """(items as an (n, 2) uint32 array, off6, kidx as a (4, N + 1, 2) array) of a cell at N (host only)."""
    n = ctypes.c_int64()
    off = np.zeros(6, dtype=np.int32)
    _check(lib().hhg_run_lists(N, None, 0, off.ctypes.data, None, ctypes.byref(n)))
    items = np.zeros((n.value, 2), dtype=np.uint32)
    kidx = np.zeros((4, N + 1, 2), dtype=np.int32)
    _check(lib().hhg_run_lists(N, items.ctypes.data, n.value, off.ctypes.data, kidx.ctypes.data, ctypes.byref(n)))
    return items, off, kidx


def hhg_slab_planes(N: int, cluster: int):
    """Plane bounds (cluster + 1 values) of the cell-resident sweep's slabs (host only)."""
    kb = np.zeros(cluster + 1, dtype=np.int32)
    _check(lib().hhg_slab_planes(N, cluster, kb.ctypes.data))
    return kb


def hhg_fp64_kernel(shell: int, L: int):
    """(FP64 kernel variant, CTAs per cluster of the resident sweep on level L; 0 = per-colour launches)."""
    v, cs = ctypes.c_int(), ctypes.c_int()
    _check(lib().hhg_fp64_kernel(shell, L, ctypes.byref(v), ctypes.byref(cs)))
    return v.value, cs.value


def hhg_last_error() -> str:
    return lib().hhg_last_error().decode()


def _check(st: int):
    if st != HHG_OK:
        raise HHGError(st, hhg_last_error())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("host vectors must be C-contiguous float64 arrays")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported vector type {type(x)}")


def _vec(x, n, what, f32=False, device_only=False) -> int:
    """_ptr(x) after checking that x (a NumPy array or a torch tensor) holds
    at least n values of the type the call reads: float64, or float32 when
    f32 (tensors only; host vectors are always float64).  The C side cannot
    check lengths, so a short or mistyped vector would be read or written
    out of bounds.  Raw integer addresses are passed through unchecked."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if isinstance(x, np.ndarray):
        if device_only:
            raise ValueError(f"{what}: this call takes device vectors only")
        if x.size < n:
            raise ValueError(f"{what}: {x.size} values, the call needs {n}")
        return _ptr(x)
    if hasattr(x, "data_ptr"):
        import torch
        want = torch.float32 if f32 else torch.float64
        if x.dtype != want:
            raise ValueError(f"{what}: dtype {x.dtype}, the call needs {want}")
        if device_only and not x.is_cuda:
            raise ValueError(f"{what}: this call takes device vectors only")
        if x.numel() < n:
            raise ValueError(f"{what}: {x.numel()} values, the call needs {n}")
        return _ptr(x)
    return _ptr(x)


def _n(shell: int, L: int) -> int:
    return hhg_num_nodes(shell, L)[0]


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def hhg_setup_shell(r_inner=0.55, r_outer=1.0, tang_refine=0, radial_layers=1, fine_log2_intervals=4,
                    hbm_budget_bytes=0, stream=None, unprojected=False) -> int:
    d = hhg_shell_desc(r_inner, r_outer, tang_refine, radial_layers, fine_log2_intervals, hbm_budget_bytes,
                       int(bool(unprojected)))
    h = ctypes.c_void_p()
    _check(lib().hhg_setup_shell(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
    return h.value


def hhg_setup_shells(radii, tang_refine=0, radial_layers=1, fine_log2_intervals=4, hbm_budget_bytes=0,
                     stream=None) -> int:
    """One hierarchy over several shells (radii: list of (r_inner, r_outer))."""
    arr = (hhg_shell_desc * len(radii))(*[hhg_shell_desc(a, b, tang_refine, radial_layers, fine_log2_intervals,
                                                         hbm_budget_bytes) for a, b in radii])
    h = ctypes.c_void_p()
    _check(lib().hhg_setup_shells(arr, len(radii), _stream(stream), ctypes.byref(h)))
    return h.value


def hhg_shell_part(shell: int, L: int, k: int):
    """[(start, count)] of shell k's vertex, edge, face and cell nodes on level L."""
    st, ct = (ctypes.c_int64 * 4)(), (ctypes.c_int64 * 4)()
    _check(lib().hhg_shell_part(shell, L, k, st, ct))
    return [(st[t], ct[t]) for t in range(4)]


def hhg_destroy(shell: int):
    _check(lib().hhg_destroy(shell))


def hhg_num_nodes(shell: int, L: int):
    nt, nf = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().hhg_num_nodes(shell, L, ctypes.byref(nt), ctypes.byref(nf)))
    return nt.value, nf.value


def hhg_node_coords(shell: int, L: int) -> np.ndarray:
    nt, _ = hhg_num_nodes(shell, L)
    out = np.empty((nt, 3), dtype=np.float64)
    _check(lib().hhg_node_coords(shell, L, out.ctypes.data))
    return out


def hhg_fit_surrogate(shell: int, q: int = 2, j: int = 2, stream=None):
    _check(lib().hhg_fit_surrogate(shell, q, j, _stream(stream)))


def hhg_fit_ipoly(shell: int, stream=None):
    _check(lib().hhg_fit_ipoly(shell, _stream(stream)))


def hhg_fit_ipoly_degree(shell: int, q: int = 2, stream=None):
    _check(lib().hhg_fit_ipoly_degree(shell, q, _stream(stream)))


def hhg_fit_cons(shell: int, q: int = 2, j: int = 2, stream=None):
    _check(lib().hhg_fit_cons(shell, q, j, _stream(stream)))


def hhg_load_vector(shell: int, L: int, f, b, stream=None):
    n = _n(shell, L)
    _check(lib().hhg_load_vector(shell, L, _vec(f, n, "f"), _vec(b, n, "b"), _stream(stream)))


def hhg_apply(shell: int, L: int, op: int, dtype: int, u, y, nrhs: int = 1, stream=None):
    n, f32 = _n(shell, L) * nrhs, dtype == HHG_F32
    _check(lib().hhg_apply(shell, L, op, dtype, _vec(u, n, "u", f32), _vec(y, n, "y", f32), nrhs, _stream(stream)))


def hhg_residual(shell: int, L: int, op: int, dtype: int, u, f, r, nrhs: int = 1, want_norms: bool = True,
                 stream=None):
    norms = np.zeros(nrhs) if want_norms else None
    n, f32 = _n(shell, L) * nrhs, dtype == HHG_F32
    _check(lib().hhg_residual(shell, L, op, dtype, _vec(u, n, "u", f32), _vec(f, n, "f", f32), _vec(r, n, "r", f32),
                              nrhs,
                              norms.ctypes.data if want_norms else None, _stream(stream)))
    return norms


def hhg_smooth(shell: int, L: int, op: int, dtype: int, f, u, sweeps: int = 1, nrhs: int = 1, stream=None):
    n, f32 = _n(shell, L) * nrhs, dtype == HHG_F32
    _check(lib().hhg_smooth(shell, L, op, dtype, _vec(f, n, "f", f32), _vec(u, n, "u", f32), sweeps, nrhs,
                            _stream(stream)))


def hhg_vcycle(shell: int, op: int, dtype: int, f, u, nu1: int = 3, nu2: int = 3, max_cycles: int = 50,
               rtol: float = 1e-8, nrhs: int = 1, stream=None, raise_on_noconv: bool = True, L=None):
    """Returns (relres per right-hand side, cycles run, status).  f and u are
    FP64 in both precisions; with L (the finest level) their lengths are
    checked."""
    rel = np.zeros(nrhs)
    cyc = ctypes.c_int()
    n = _n(shell, L) * nrhs if L is not None else 0
    st = lib().hhg_vcycle(shell, op, dtype, _vec(f, n, "f"), _vec(u, n, "u"), nu1, nu2, max_cycles, rtol, nrhs,
                          rel.ctypes.data,
                          ctypes.byref(cyc), _stream(stream))
    if st != HHG_OK and (st != HHG_ENOCONV or raise_on_noconv):
        raise HHGError(st, hhg_last_error())
    return rel, cyc.value, st


HHG_NOALLOC_SCRATCH = 16384


def hhg_residual_noalloc(shell: int, L: int, op: int, u, f, r, norm2_dev, stream=None):
    """r = f - L u and ||r||^2 into the device double norm2_dev, allocating
    nothing (device pointers only; see include/hhg.h).  Tensors are checked
    for type, device and length here (u, f, r: CUDA float64 with at least
    n_total values; norm2_dev: CUDA float64 with at least one), because the
    C side cannot see lengths; raw integer addresses are passed unchecked."""
    n = _n(shell, L)
    _check(lib().hhg_residual_noalloc(shell, L, op, _vec(u, n, "u", device_only=True),
                                      _vec(f, n, "f", device_only=True), _vec(r, n, "r", device_only=True),
                                      _vec(norm2_dev, 1, "norm2_dev", device_only=True), _stream(stream)))


class Shell:
    """Owning handle around hhg_setup_shell / hhg_destroy."""

    def __init__(self, r_inner=0.55, r_outer=1.0, tang_refine=0, radial_layers=1, fine_log2_intervals=4,
                 hbm_budget_bytes=0, stream=None, unprojected=False):
        self.handle = hhg_setup_shell(r_inner, r_outer, tang_refine, radial_layers, fine_log2_intervals,
                                      hbm_budget_bytes, stream, unprojected)
        self.L = fine_log2_intervals

    @classmethod
    def group(cls, radii, tang_refine=0, radial_layers=1, fine_log2_intervals=4, hbm_budget_bytes=0, stream=None):
        """Several shells of the same macro topology and level, differing in
        radii, as one hierarchy (every kernel launch spans all of them)."""
        obj = cls.__new__(cls)
        obj.handle = hhg_setup_shells(radii, tang_refine, radial_layers, fine_log2_intervals, hbm_budget_bytes,
                                      stream)
        obj.L = fine_log2_intervals
        obj.n_parts = len(radii)
        return obj

    def part_index(self, k, L=None):
        """Indices of shell k's nodes in the group's canonical vector, in the
        order of that shell's own canonical vector."""
        rng = hhg_shell_part(self.handle, self.L if L is None else L, k)
        return np.concatenate([np.arange(s, s + c) for s, c in rng])

    def close(self):
        if self.handle:
            hhg_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_nodes(self, L=None):
        return hhg_num_nodes(self.handle, self.L if L is None else L)

    def node_coords(self, L=None):
        return hhg_node_coords(self.handle, self.L if L is None else L)

    def fit(self, q=2, j=2, stream=None):
        hhg_fit_surrogate(self.handle, q, j, stream)

    def fit_ipoly(self, q=2, stream=None):
        if q == 2:
            hhg_fit_ipoly(self.handle, stream)
        else:
            hhg_fit_ipoly_degree(self.handle, q, stream)

    def fit_cons(self, q=2, j=2, stream=None):
        hhg_fit_cons(self.handle, q, j, stream)

    def load_vector(self, f, b, L=None, stream=None):
        hhg_load_vector(self.handle, self.L if L is None else L, f, b, stream)

    def apply(self, u, y, L=None, op=HHG_OP_LSQP, dtype=HHG_F64, nrhs=1, stream=None):
        hhg_apply(self.handle, self.L if L is None else L, op, dtype, u, y, nrhs, stream)

    def residual(self, u, f, r, L=None, op=HHG_OP_LSQP, dtype=HHG_F64, nrhs=1, stream=None):
        return hhg_residual(self.handle, self.L if L is None else L, op, dtype, u, f, r, nrhs, True, stream)

    def smooth(self, f, u, sweeps=1, L=None, op=HHG_OP_LSQP, dtype=HHG_F64, nrhs=1, stream=None):
        hhg_smooth(self.handle, self.L if L is None else L, op, dtype, f, u, sweeps, nrhs, stream)

    def vcycle(self, f, u, nu1=3, nu2=3, max_cycles=50, rtol=1e-8, op=HHG_OP_LSQP, dtype=HHG_F64, nrhs=1,
               stream=None, raise_on_noconv=True):
        return hhg_vcycle(self.handle, op, dtype, f, u, nu1, nu2, max_cycles, rtol, nrhs, stream, raise_on_noconv,
                          L=self.L)


def hhg_problem_nodes(r_inner, r_outer, tang_refine, radial_layers, L):
    """(n_total, n_free) of a shell problem (no GPU work)."""
    p = hhg_problem(r_inner, r_outer, tang_refine, radial_layers, L)
    nt, nf = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().hhg_problem_nodes(ctypes.byref(p), ctypes.byref(nt), ctypes.byref(nf)))
    return nt.value, nf.value


class Server:
    """Solve service over resident hierarchies (hhg_server_* of include/hhg.h):
    submit() queues a shell problem with its right-hand sides (host arrays,
    copied), wait() returns (u, relres, info) once it is solved."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=4, q=2, j=2, nu1=3, nu2=3, max_cycles=60, rtol=1e-8,
                 dtype=HHG_F32, max_batch_rhs=0):
        d = hhg_server_desc(hbm_budget_bytes, max_inflight, q, j, nu1, nu2, max_cycles, rtol, dtype, max_batch_rhs)
        h = ctypes.c_void_p()
        _check(lib().hhg_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h.value
        self._shapes = {}

    def submit(self, f, r_inner=0.55, r_outer=1.0, tang_refine=0, radial_layers=1, L=4) -> int:
        f = np.ascontiguousarray(f, dtype=np.float64)
        nrhs = 1 if f.ndim == 1 else f.shape[0]
        p = hhg_problem(r_inner, r_outer, tang_refine, radial_layers, L)
        t = ctypes.c_int64()
        _check(lib().hhg_server_submit(self.handle, ctypes.byref(p), f.ctypes.data, nrhs, ctypes.byref(t)))
        self._shapes[t.value] = (nrhs, f.shape[-1])
        return t.value

    def wait(self, ticket, raise_on_error=True):
        nrhs, n = self._shapes.pop(ticket)
        u = np.empty((nrhs, n))
        rel = np.empty(nrhs)
        info = hhg_request_info()
        st = lib().hhg_server_wait(self.handle, ticket, u.ctypes.data, rel.ctypes.data, ctypes.byref(info))
        if st != HHG_OK and raise_on_error:
            raise HHGError(st, hhg_last_error())
        return u, rel, {"t_submit": info.t_submit, "t_start": info.t_start, "t_end": info.t_end,
                        "cycles": info.cycles, "reused": bool(info.reused), "status": info.status,
                        "batch_rhs": info.batch_rhs}

    def stats(self):
        n, b, built, ev = ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().hhg_server_stats(self.handle, ctypes.byref(n), ctypes.byref(b), ctypes.byref(built),
                                      ctypes.byref(ev)))
        return {"resident": n.value, "bytes": b.value, "built": built.value, "evicted": ev.value}

    def close(self):
        if self.handle:
            _check(lib().hhg_server_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
