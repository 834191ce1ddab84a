"""Python binding of libpdmk.so (periodic DMK lattice sums on B300).

Argument marshalling only: every step of an evaluation runs in the library's CUDA
kernels (and cuFFT).  PyTorch supplies device memory and the current stream.  If the
compiled library is missing the import of ``lib()`` raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdmk.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "pdmk.h")

PDMK_HOST, PDMK_DEVICE = 0, 1
PDMK_FP64, PDMK_MIXED = 0, 1


class PdmkError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {code} ({_strerror(code)})")


class Opts(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("n_s", ctypes.c_int), ("precision", ctypes.c_int),
                ("window_w", ctypes.c_int), ("n_proxy", ctypes.c_int), ("n_pw", ctypes.c_int),
                ("max_depth", ctypes.c_int), ("neutrality", ctypes.c_int), ("profile", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("wait_test", ctypes.c_int), ("autotune", ctypes.c_int),
                ("root_mode", ctypes.c_int), ("build_mode", ctypes.c_int), ("tensor_cores", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("eps", ctypes.c_double), ("c", ctypes.c_double),
                ("rc", ctypes.c_double), ("V", ctypes.c_double), ("kappa", ctypes.c_double),
                ("n_s", ctypes.c_int), ("window_w", ctypes.c_int), ("n_proxy", ctypes.c_int),
                ("n_pw", ctypes.c_int), ("precision", ctypes.c_int), ("M", ctypes.c_int * 3),
                ("nroot", ctypes.c_int * 3), ("n", ctypes.c_int64), ("n_images", ctypes.c_int64),
                ("nboxes", ctypes.c_int), ("nleaves", ctypes.c_int), ("depth", ctypes.c_int),
                ("ntarget_leaves", ctypes.c_int), ("n_pw_boxes_out", ctypes.c_int),
                ("n_pw_boxes_in", ctypes.c_int), ("near_pairs", ctypes.c_int64), ("near_pairs_in", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("launches", ctypes.c_int),
                ("pw_moment_sources", ctypes.c_int64), ("pw_merge_parents", ctypes.c_int),
                ("pw_down_parents", ctypes.c_int), ("pw_eval_targets", ctypes.c_int64),
                ("spread_subproblems", ctypes.c_int), ("n_targets", ctypes.c_int64)]


_lib = None


def lib():
    """Load libpdmk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2606_28608_b300/build.py (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        L.pdmk_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.pdmk_default_opts.restype = None
        L.pdmk_plan_create.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.POINTER(Opts), ctypes.POINTER(P)]
        L.pdmk_plan_create.restype = ctypes.c_int
        L.pdmk_set_sources.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int]
        L.pdmk_set_sources.restype = ctypes.c_int
        L.pdmk_set_sources_targets.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int64, P, ctypes.c_int]
        L.pdmk_set_sources_targets.restype = ctypes.c_int
        L.pdmk_set_charges.argtypes = [P, P, ctypes.c_int]
        L.pdmk_set_charges.restype = ctypes.c_int
        L.pdmk_eval.argtypes = [P, P, P, ctypes.c_int]
        L.pdmk_eval.restype = ctypes.c_int
        L.pdmk_eval_bloch.argtypes = [P, P, P, P, ctypes.c_int]
        L.pdmk_eval_bloch.restype = ctypes.c_int
        L.pdmk_eval_targets.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int]
        L.pdmk_eval_targets.restype = ctypes.c_int
        L.pdmk_eval_noalloc.argtypes = [P, P, P]
        L.pdmk_eval_noalloc.restype = ctypes.c_int
        L.pdmk_eval_adjoint.argtypes = [P, P, P, P, P, P, ctypes.c_int]
        L.pdmk_eval_adjoint.restype = ctypes.c_int
        L.pdmk_batch_create.argtypes = [ctypes.c_int, P, P, P, ctypes.POINTER(Opts), ctypes.POINTER(P)]
        L.pdmk_batch_create.restype = ctypes.c_int
        L.pdmk_batch_set_sources.argtypes = [P, P, P, P, ctypes.c_int]
        L.pdmk_batch_set_sources.restype = ctypes.c_int
        L.pdmk_batch_eval.argtypes = [P, P, P, ctypes.c_int]
        L.pdmk_batch_eval.restype = ctypes.c_int
        L.pdmk_batch_plan.argtypes = [P, ctypes.c_int]
        L.pdmk_batch_plan.restype = P
        L.pdmk_batch_destroy.argtypes = [P]
        L.pdmk_batch_destroy.restype = None
        L.pdmk_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.pdmk_stage_times.restype = ctypes.c_int
        L.pdmk_setup_times.argtypes = [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.pdmk_setup_times.restype = ctypes.c_int
        L.pdmk_get_info.argtypes = [P, ctypes.POINTER(Info)]
        L.pdmk_get_info.restype = ctypes.c_int
        L.pdmk_plan_destroy.argtypes = [P]
        L.pdmk_plan_destroy.restype = None
        L.pdmk_plan_message.argtypes = [P]
        L.pdmk_plan_message.restype = ctypes.c_char_p
        L.pdmk_strerror.argtypes = [ctypes.c_int]
        L.pdmk_strerror.restype = ctypes.c_char_p
        L.pdmk_cell_work.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.POINTER(Opts), ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_double)]
        L.pdmk_cell_work.restype = ctypes.c_int
        L.pdmk_partition_cells.argtypes = [ctypes.c_int, P, ctypes.c_int, P]
        L.pdmk_partition_cells.restype = ctypes.c_int
        L.pdmk_kernel_table_eval.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double)]
        L.pdmk_kernel_table_eval.restype = ctypes.c_int
        _lib = L
    return _lib


def _strerror(code):
    try:
        return lib().pdmk_strerror(code).decode()
    except Exception:  # noqa: BLE001
        return "?"


def header_functions(path: str = HEADER):
    """Names of the functions declared by include/pdmk.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pdmk_[a-z_0-9]+)\s*\(", txt)))


def kernel_table(d: int, eps: float, kind: int, x: float = 0.0) -> float:
    """FP64 kernel-table query (host only): see pdmk_kernel_table_eval in include/pdmk.h."""
    v = ctypes.c_double()
    rc = lib().pdmk_kernel_table_eval(int(d), float(eps), int(kind), float(x), ctypes.byref(v))
    if rc != 0:
        raise PdmkError(rc, "pdmk_kernel_table_eval")
    return v.value


def cell_work(L, eps: float, n: int) -> float:
    """Estimated flops of one evaluation of a cell (pdmk_cell_work; host only)."""
    L = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
    Lc = np.ascontiguousarray(L.T)
    v = ctypes.c_double()
    rc = lib().pdmk_cell_work(L.shape[0], Lc.ctypes.data, float(eps), None, int(n), ctypes.byref(v))
    if rc != 0:
        raise PdmkError(rc, "pdmk_cell_work")
    return v.value


def partition_cells(work, nranks: int):
    """Rank of every cell (pdmk_partition_cells: decreasing work to the least-loaded rank)."""
    w = np.ascontiguousarray(np.asarray(work, dtype=np.float64))
    out = np.empty(len(w), dtype=np.int32)
    rc = lib().pdmk_partition_cells(len(w), w.ctypes.data, int(nranks), out.ctypes.data)
    if rc != 0:
        raise PdmkError(rc, "pdmk_partition_cells")
    return out


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:
        return False


class Plan:
    """A periodic DMK plan for lattice L (columns = lattice vectors) and precision eps."""

    def __init__(self, L, eps: float, *, precision: str = "fp64", kappa: float = 0.0, n_s: int = 0,
                 window_w: int = 0, n_proxy: int = 0, n_pw: int = 0, max_depth: int = -1,
                 neutrality: int = 1, profile: bool = False, stream=None, wait_test: int = 0,
                 autotune: bool = False, root_mode: int = 0, build: str = "auto", tensor_cores: bool = True):
        L = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
        self.d = L.shape[0]
        self._L = L
        o = Opts()
        lib().pdmk_default_opts(ctypes.byref(o))
        o.kappa = kappa
        o.n_s = n_s
        o.precision = PDMK_MIXED if precision == "mixed" else PDMK_FP64
        o.window_w = window_w
        o.n_proxy = n_proxy
        o.n_pw = n_pw
        o.max_depth = max_depth
        o.neutrality = neutrality
        o.profile = 1 if profile else 0
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        o.stream = stream or None
        o.wait_test = int(wait_test)
        o.autotune = 1 if autotune else 0
        o.root_mode = int(root_mode)
        o.build_mode = {"auto": 0, "host": 1, "device": 2, "compare": 3}[build]
        o.tensor_cores = 0 if tensor_cores else 1
        self.opts = o
        Lc = np.ascontiguousarray(L.T)  # column-major
        h = ctypes.c_void_p()
        rc = lib().pdmk_plan_create(self.d, Lc.ctypes.data, float(eps), ctypes.byref(o), ctypes.byref(h))
        if rc != 0:
            raise PdmkError(rc, "pdmk_plan_create")
        self._h = h
        self.n = 0
        self.m = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().pdmk_plan_destroy(h)
            except Exception:  # noqa: BLE001
                pass
            self._h = None

    def close(self):
        self.__del__()

    def set_sources(self, y, q, x=None):
        """Sources y (n x d) with charges q (n); optional separate targets x (m x d), else the
        evaluation is at the sources.  numpy arrays (host) or CUDA tensors (device)."""
        dev = _is_torch(y)
        if dev:
            assert y.is_cuda and y.dtype.is_floating_point
            yy = y.contiguous().double()
            qq = q.contiguous().double()
            xx = x.contiguous().double() if x is not None else None
            n, ptr = yy.shape[0], (lambda a: a.data_ptr())
        else:
            yy = np.ascontiguousarray(np.asarray(y, dtype=np.float64).reshape(-1, self.d))
            qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
            xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, self.d)) if x is not None else None
            n, ptr = yy.shape[0], (lambda a: a.ctypes.data)
        where = PDMK_DEVICE if dev else PDMK_HOST
        if xx is None:
            rc = lib().pdmk_set_sources(self._h, n, ptr(yy), ptr(qq), where)
            m = n
        else:
            m = xx.shape[0]
            rc = lib().pdmk_set_sources_targets(self._h, n, ptr(yy), ptr(qq), m, ptr(xx), where)
        if rc != 0:
            raise PdmkError(rc, "pdmk_set_sources: " + self.message())
        self.n = n
        self.m = m
        self.separate_targets = xx is not None

    def set_charges(self, q):
        if _is_torch(q):
            qq = q.contiguous().double()
            rc = lib().pdmk_set_charges(self._h, qq.data_ptr(), PDMK_DEVICE)
        else:
            qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
            rc = lib().pdmk_set_charges(self._h, qq.ctypes.data, PDMK_HOST)
        if rc != 0:
            raise PdmkError(rc, "pdmk_set_charges")

    def eval(self, grad: bool = True, out=None):
        """Host evaluation: returns numpy (pot, grad or None).  out=(pot, grad) writes into
        caller arrays instead (C-contiguous float64 of shapes (n,) and (n, d); page-locked host
        memory, e.g. a pinned torch tensor's .numpy(), makes the device-to-host copy a DMA)."""
        if out is not None:
            pot, g = out
            ok = (isinstance(pot, np.ndarray) and pot.dtype == np.float64 and pot.shape == (self.m,)
                  and pot.flags.c_contiguous)
            if grad:
                ok = ok and (isinstance(g, np.ndarray) and g.dtype == np.float64 and g.shape == (self.m, self.d)
                             and g.flags.c_contiguous)
            if not ok:
                raise ValueError("out must be C-contiguous float64 arrays of shapes (m,) and (m, d)")
        else:
            pot = np.empty(self.m, dtype=np.float64)
            g = np.empty((self.m, self.d), dtype=np.float64) if grad else None
        rc = lib().pdmk_eval(self._h, pot.ctypes.data, g.ctypes.data if grad else None, PDMK_HOST)
        if rc != 0:
            raise PdmkError(rc, "pdmk_eval")
        return pot, g

    def eval_device(self, pot, grad=None):
        """Device evaluation into torch CUDA tensors (float64), asynchronous on the stream."""
        rc = lib().pdmk_eval(self._h, pot.data_ptr(), grad.data_ptr() if grad is not None else None, PDMK_DEVICE)
        if rc != 0:
            raise PdmkError(rc, "pdmk_eval")

    def eval_targets(self, x, grad: bool = True, out=None):
        """Potential (and gradient) of the plan's sources at targets x (m x d), evaluated per call
        against the existing source tree (pdmk_eval_targets).  x: numpy array (host results as
        numpy) or CUDA tensor (results written into out=(pot, grad) CUDA tensors, or new ones)."""
        if _is_torch(x):
            import torch
            xx = x.contiguous().double()
            m = xx.shape[0]
            if out is None:
                pot = torch.empty(m, dtype=torch.float64, device=xx.device)
                g = torch.empty((m, self.d), dtype=torch.float64, device=xx.device) if grad else None
            else:
                pot, g = out
            rc = lib().pdmk_eval_targets(self._h, m, xx.data_ptr(), pot.data_ptr(),
                                         g.data_ptr() if g is not None else None, PDMK_DEVICE)
        else:
            xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, self.d))
            m = xx.shape[0]
            pot = np.empty(m, dtype=np.float64)
            g = np.empty((m, self.d), dtype=np.float64) if grad else None
            rc = lib().pdmk_eval_targets(self._h, m, xx.ctypes.data, pot.ctypes.data,
                                         g.ctypes.data if g is not None else None, PDMK_HOST)
        if rc != 0:
            raise PdmkError(rc, "pdmk_eval_targets")
        return pot, g

    def eval_bloch(self, beta, grad: bool = True):
        """Quasi-periodic potential (and gradient) at the plan's points for the Bloch wave vector
        beta (pdmk_eval_bloch): complex numpy arrays of shapes (m,) and (m, d)."""
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(self.d))
        pot = np.empty(2 * self.m, dtype=np.float64)
        g = np.empty(2 * self.m * self.d, dtype=np.float64) if grad else None
        rc = lib().pdmk_eval_bloch(self._h, b.ctypes.data, pot.ctypes.data, g.ctypes.data if grad else None,
                                   PDMK_HOST)
        if rc != 0:
            raise PdmkError(rc, "pdmk_eval_bloch: " + lib().pdmk_plan_message(self._h).decode())
        pc = pot[0::2] + 1j * pot[1::2]
        gc = (g[0::2] + 1j * g[1::2]).reshape(self.m, self.d) if grad else None
        return pc, gc

    def eval_noalloc(self, pot, grad=None):
        """Device evaluation into caller-owned torch CUDA tensors (float64) without any device
        allocation in the call: the spreading scratch is the library's fixed 16 MiB static
        array (see pdmk_eval_noalloc in include/pdmk.h).  Raises PdmkError (TOO_LARGE) if the
        plan's spreading scratch does not fit."""
        rc = lib().pdmk_eval_noalloc(self._h, pot.data_ptr(), grad.data_ptr() if grad is not None else None)
        if rc != 0:
            raise PdmkError(rc, "pdmk_eval_noalloc")

    def eval_adjoint(self, g_pot, want_q: bool = True, want_y: bool = True, want_x: bool = None):
        """Vector-Jacobian product of the evaluation (pdmk_eval_adjoint): for the upstream
        gradient g_pot = dLoss/dPhi (one value per evaluated point) returns (dLoss/dq, dLoss/dy)
        and, with separate targets, (dLoss/dq, dLoss/dy, dLoss/dx); numpy arrays for numpy
        input, CUDA float64 tensors for a CUDA tensor input (None where not wanted)."""
        sep = getattr(self, "separate_targets", False)
        if want_x is None:
            want_x = sep
        if want_x and not sep:
            raise ValueError("without separate targets the target derivative is part of dLoss/dy")
        if _is_torch(g_pot):
            import torch
            g = g_pot.contiguous().to(torch.float64)
            mk = lambda *s: torch.empty(s, dtype=torch.float64, device=g.device)  # noqa: E731
            ptr, where = (lambda a: a.data_ptr()), PDMK_DEVICE
        else:
            g = np.ascontiguousarray(np.asarray(g_pot, dtype=np.float64).reshape(-1))
            mk = lambda *s: np.empty(s, dtype=np.float64)  # noqa: E731
            ptr, where = (lambda a: a.ctypes.data), PDMK_HOST
        if g.shape[0] != self.m:
            raise ValueError("g_pot must have one value per evaluated point")
        gq = mk(self.n) if want_q else None
        gy = mk(self.n, self.d) if want_y else None
        gx = mk(self.m, self.d) if want_x else None
        rc = lib().pdmk_eval_adjoint(self._h, ptr(g), None, ptr(gq) if want_q else None,
                                     ptr(gy) if want_y else None, ptr(gx) if want_x else None, where)
        if rc != 0:
            raise PdmkError(rc, "pdmk_eval_adjoint")
        return (gq, gy, gx) if sep else (gq, gy)

    def info(self) -> dict:
        inf = Info()
        rc = lib().pdmk_get_info(self._h, ctypes.byref(inf))
        if rc != 0:
            raise PdmkError(rc, "pdmk_get_info")
        out = {}
        for name, _ in Info._fields_:
            v = getattr(inf, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out

    def stage_times(self) -> dict:
        names = (ctypes.c_char_p * 32)()
        ms = (ctypes.c_double * 32)()
        n = lib().pdmk_stage_times(self._h, names, ms, 32)
        return {names[i].decode(): ms[i] for i in range(max(n, 0))}

    def message(self) -> str:
        """Detail of the plan's last error or check (pdmk_plan_message)."""
        m = lib().pdmk_plan_message(self._h)
        return m.decode() if m else ""

    def setup_times(self) -> dict:
        """Host wall-clock ms of the phases of the last set_sources (pdmk_setup_times)."""
        names = (ctypes.c_char_p * 32)()
        ms = (ctypes.c_double * 32)()
        n = lib().pdmk_setup_times(self._h, names, ms, 32)
        return {names[i].decode(): ms[i] for i in range(max(min(n, 32), 0))}


class Batch:
    """Many independent cells evaluated together (pdmk_batch_*): one plan per cell, one CUDA
    graph per evaluation of all cells.  cells: list of (L, eps); every cell shares the options."""

    def __init__(self, cells, *, precision: str = "fp64", kappa: float = 0.0, n_s: int = 0,
                 neutrality: int = 1, stream=None):
        Ls = [np.ascontiguousarray(np.asarray(L, dtype=np.float64)) for L, _ in cells]
        self.dims = [L.shape[0] for L in Ls]
        o = Opts()
        lib().pdmk_default_opts(ctypes.byref(o))
        o.kappa = kappa
        o.n_s = n_s
        o.precision = PDMK_MIXED if precision == "mixed" else PDMK_FP64
        o.neutrality = neutrality
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        o.stream = stream or None
        dd = np.asarray(self.dims, dtype=np.int32)
        Lp = np.ascontiguousarray(np.concatenate([L.T.reshape(-1) for L in Ls]))  # column-major each
        ee = np.asarray([float(e) for _, e in cells], dtype=np.float64)
        h = ctypes.c_void_p()
        rc = lib().pdmk_batch_create(len(cells), dd.ctypes.data, Lp.ctypes.data, ee.ctypes.data, ctypes.byref(o),
                                     ctypes.byref(h))
        if rc != 0:
            raise PdmkError(rc, "pdmk_batch_create")
        self._h = h
        self.counts = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().pdmk_batch_destroy(h)
            except Exception:  # noqa: BLE001
                pass
            self._h = None

    def close(self):
        self.__del__()

    def set_sources(self, ys, qs):
        """ys, qs: per-cell lists of host arrays (n_c x d_c positions, n_c charges)."""
        self.counts = [len(q) for q in qs]
        off = np.zeros(len(qs) + 1, dtype=np.int64)
        off[1:] = np.cumsum(self.counts)
        y = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in ys]))
        q = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in qs]))
        rc = lib().pdmk_batch_set_sources(self._h, off.ctypes.data, y.ctypes.data, q.ctypes.data, PDMK_HOST)
        if rc != 0:
            raise PdmkError(rc, "pdmk_batch_set_sources")
        self._off = off

    def eval(self):
        """Host evaluation: per-cell lists of potentials and gradients."""
        ntot = int(self._off[-1])
        ytot = sum(c * d for c, d in zip(self.counts, self.dims))
        pot = np.empty(ntot)
        grad = np.empty(ytot)
        rc = lib().pdmk_batch_eval(self._h, pot.ctypes.data, grad.ctypes.data, PDMK_HOST)
        if rc != 0:
            raise PdmkError(rc, "pdmk_batch_eval")
        pots, grads, yo = [], [], 0
        for c, (n, d) in enumerate(zip(self.counts, self.dims)):
            pots.append(pot[self._off[c]:self._off[c + 1]])
            grads.append(grad[yo:yo + n * d].reshape(n, d))
            yo += n * d
        return pots, grads

    def eval_device(self, pot, grad=None):
        """Device evaluation into packed float64 CUDA tensors (offsets / row layouts)."""
        rc = lib().pdmk_batch_eval(self._h, pot.data_ptr(), grad.data_ptr() if grad is not None else None,
                                   PDMK_DEVICE)
        if rc != 0:
            raise PdmkError(rc, "pdmk_batch_eval")
