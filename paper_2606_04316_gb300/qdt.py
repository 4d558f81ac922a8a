"""Thin Python binding of libqdt (include/qdt.h): argument marshalling only.

Every step of a transformation runs in the library's CUDA kernels; PyTorch is
used for device memory and streams.  There is no CPU fallback: if the
extension is missing the import of the library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

COULOMB, GAUNT, GAUGE = 1, 2, 4
FP64, SPLIT = 0, 1
BLOCK_BITS = {"coulomb": COULOMB, "gaunt": GAUNT, "gauge": GAUGE}
ERRORS = {-1: "QDT_ERR_ARG", -2: "QDT_ERR_OOM", -3: "QDT_ERR_CUDA", -4: "QDT_ERR_STATE",
          -5: "QDT_ERR_UNIMPLEMENTED", -6: "QDT_ERR_TIMEOUT", -7: "QDT_ERR_ADMISSION"}

EXPORTS = ["qdt_create", "qdt_destroy", "qdt_set_basis", "qdt_num_functions", "qdt_set_coefficients",
           "qdt_packed_size", "qdt_transform", "qdt_unpack", "qdt_last_error", "qdt_version",
           "qdt_footprint", "qdt_server_create", "qdt_server_destroy", "qdt_submit", "qdt_poll", "qdt_wait",
           "qdt_second_half_noalloc", "qdt_transform_batch", "qdt_graph_counts",
           "qdt_set_spinor_coefficients", "qdt_set_rkb_coefficients", "qdt_set_route",
           "qdt_check_bounded_wait", "qdt_f32_error_ratio", "qdt_alu_peak"]
BATCH_GRAPH = 1


class QdtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "QDT_ERR"), code, msg))
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_density", ctypes.c_double),
                ("ms_screen", ctypes.c_double), ("ms_eri", ctypes.c_double),
                ("ms_half1", ctypes.c_double), ("ms_half2", ctypes.c_double),
                ("ms_pack", ctypes.c_double), ("flops_half1", ctypes.c_double),
                ("flops_half2", ctypes.c_double), ("quartets_total", ctypes.c_longlong * 3),
                ("quartets_kept", ctypes.c_longlong * 3), ("eri_values", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_int), ("precision", ctypes.c_int),
                ("slices", ctypes.c_int), ("flops_eri", ctypes.c_double),
                ("quartets_f32", ctypes.c_longlong * 3), ("f32_bound", ctypes.c_double),
                ("flops_eri_f32", ctypes.c_double)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class Request(ctypes.Structure):
    _fields_ = [("n_centers", ctypes.c_int), ("xyz", ctypes.c_void_p), ("n_shells", ctypes.c_int),
                ("shell_center", ctypes.c_void_p), ("shell_l", ctypes.c_void_p), ("shell_nprim", ctypes.c_void_p),
                ("exps", ctypes.c_void_p), ("coefs", ctypes.c_void_p), ("nK", ctypes.c_int),
                ("CL", ctypes.c_void_p), ("CS", ctypes.c_void_p), ("blocks", ctypes.c_uint),
                ("k_begin", ctypes.c_int), ("k_end", ctypes.c_int), ("schwarz_tau", ctypes.c_double),
                ("precision", ctypes.c_int), ("out", ctypes.c_void_p), ("out_bytes", ctypes.c_size_t)]


class BatchItem(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("blocks", ctypes.c_uint), ("k_begin", ctypes.c_int),
                ("k_end", ctypes.c_int), ("schwarz_tau", ctypes.c_double), ("precision", ctypes.c_int),
                ("out", ctypes.c_void_p), ("out_bytes", ctypes.c_size_t), ("stats", ctypes.c_void_p),
                ("status", ctypes.c_int)]


_LIB = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libqdt.so (building it in-tree with nvcc if absent)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError("libqdt.so is not built: run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.qdt_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
    L.qdt_destroy.argtypes = [vp]
    L.qdt_destroy.restype = None
    L.qdt_set_basis.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp, vp]
    L.qdt_num_functions.argtypes = [vp]
    L.qdt_set_coefficients.argtypes = [vp, ctypes.c_int, vp, vp]
    L.qdt_set_spinor_coefficients.argtypes = [vp, ctypes.c_int, vp, vp]
    L.qdt_set_rkb_coefficients.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_int]
    L.qdt_set_route.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.qdt_check_bounded_wait.argtypes = [vp, ctypes.c_double]
    L.qdt_f32_error_ratio.argtypes = [vp, ctypes.c_uint, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp]
    L.qdt_packed_size.argtypes = [vp, ctypes.c_uint, ctypes.c_int, ctypes.c_int]
    L.qdt_packed_size.restype = ctypes.c_size_t
    L.qdt_transform.argtypes = [vp, ctypes.c_uint, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_int, vp, ctypes.c_size_t, ctypes.POINTER(Stats)]
    L.qdt_unpack.argtypes = [vp, vp, ctypes.c_int, ctypes.c_uint, vp]
    L.qdt_last_error.argtypes = [vp]
    L.qdt_last_error.restype = ctypes.c_char_p
    L.qdt_version.restype = ctypes.c_char_p
    L.qdt_footprint.argtypes = [ctypes.POINTER(Request)]
    L.qdt_footprint.restype = ctypes.c_size_t
    L.qdt_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_size_t]
    L.qdt_server_destroy.argtypes = [vp]
    L.qdt_server_destroy.restype = None
    L.qdt_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.qdt_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
    L.qdt_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(Stats)]
    L.qdt_second_half_noalloc.argtypes = [vp, vp, ctypes.c_longlong, ctypes.c_longlong, vp, vp,
                                          ctypes.c_char_p, ctypes.c_size_t]
    L.qdt_transform_batch.argtypes = [ctypes.POINTER(BatchItem), ctypes.c_int, ctypes.c_uint]
    L.qdt_graph_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.qdt_alu_peak.argtypes = [ctypes.c_int, ctypes.c_int, dp]
    _LIB = L
    return L


def _ptr(x):
    """Address of a numpy array or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def blocks_mask(blocks):
    if isinstance(blocks, int):
        return blocks
    m = 0
    for b in blocks:
        m |= BLOCK_BITS[b]
    return m


class Context:
    """One qdt context on one CUDA device (and one stream)."""

    def __init__(self, device=0, stream=None):
        self.L = load()
        h = ctypes.c_void_p()
        sp = None
        if stream is not None:
            sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = self.L.qdt_create(ctypes.byref(h), int(device), sp)
        if rc != 0:
            raise QdtError(rc, "qdt_create failed")
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            self.L.qdt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise QdtError(rc, self.L.qdt_last_error(self.h).decode())

    def set_basis(self, basis):
        arrs = [np.ascontiguousarray(basis.xyz, np.float64), np.ascontiguousarray(basis.shell_center, np.int32),
                np.ascontiguousarray(basis.shell_l, np.int32), np.ascontiguousarray(basis.shell_nprim, np.int32),
                np.ascontiguousarray(basis.exps, np.float64), np.ascontiguousarray(basis.coefs, np.float64)]
        self._check(self.L.qdt_set_basis(self.h, int(arrs[0].shape[0]), _ptr(arrs[0]), int(arrs[1].shape[0]),
                                         _ptr(arrs[1]), _ptr(arrs[2]), _ptr(arrs[3]), _ptr(arrs[4]),
                                         _ptr(arrs[5])))

    def num_functions(self):
        return self.L.qdt_num_functions(self.h)

    def set_coefficients(self, CL, CS):
        """CL [nL, nK, 4], CS [3 nL, nK, 4] float64, numpy (host) or torch (host or cuda)."""
        if isinstance(CL, np.ndarray):
            CL = np.ascontiguousarray(CL, np.float64)
            CS = np.ascontiguousarray(CS, np.float64)
        nK = int(CL.shape[1])
        self._check(self.L.qdt_set_coefficients(self.h, nK, _ptr(CL), _ptr(CS)))

    def set_spinor_coefficients(self, CL, CS):
        """Kramers-unrestricted input: CL [nL, n, 4], CS [3 nL, n, 4] float64
        (Re alpha, Im alpha, Re beta, Im beta per row and spinor)."""
        if isinstance(CL, np.ndarray):
            CL = np.ascontiguousarray(CL, np.float64)
            CS = np.ascontiguousarray(CS, np.float64)
        n = int(CL.shape[1])
        self._check(self.L.qdt_set_spinor_coefficients(self.h, n, _ptr(CL), _ptr(CS)))

    def set_rkb_coefficients(self, CL, CS, c_light, spinors=False):
        """Restricted-kinetic-balance input: CL and CS both [nL, n, 4] float64;
        CS is expanded over the derivative functions on the device."""
        if isinstance(CL, np.ndarray):
            CL = np.ascontiguousarray(CL, np.float64)
            CS = np.ascontiguousarray(CS, np.float64)
        n = int(CL.shape[1])
        self._check(self.L.qdt_set_rkb_coefficients(self.h, n, _ptr(CL), _ptr(CS), float(c_light),
                                                    1 if spinors else 0))

    def set_route(self, route, mo_block=0):
        """'density' (default), 'quarter' (two-quarter Coulomb first half) or
        'mo' (MO-driven, integrals recomputed per block of mo_block outer MOs)."""
        code = {"density": 0, "quarter": 1, "mo": 2}[route]
        self._check(self.L.qdt_set_route(self.h, code, int(mo_block)))

    def f32_error_ratio(self, blocks, k_begin, k_end, tau):
        """[Coulomb, L-S class] max |FP32 - compensated FP32| / (Q_A Q_C) of the kept integrals."""
        r = (ctypes.c_double * 2)()
        self._check(self.L.qdt_f32_error_ratio(self.h, blocks_mask(blocks), int(k_begin), int(k_end), float(tau),
                                               ctypes.cast(r, ctypes.c_void_p)))
        return [r[0], r[1]]

    def check_bounded_wait(self, limit_s=0.05):
        """Status code of the bounded-wait self-check (QDT_ERR_TIMEOUT = -6 expected)."""
        return int(self.L.qdt_check_bounded_wait(self.h, float(limit_s)))

    def packed_size(self, blocks, k_begin, k_end):
        return int(self.L.qdt_packed_size(self.h, blocks_mask(blocks), int(k_begin), int(k_end)))

    def transform(self, blocks, k_begin, k_end, tau, precision, out):
        """Packed (pq|rs) into `out` (numpy or torch float64, host or device);
        returns the call's statistics as a dict."""
        st = Stats()
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        self._check(self.L.qdt_transform(self.h, blocks_mask(blocks), int(k_begin), int(k_end), float(tau),
                                         int(precision), _ptr(out), nbytes, ctypes.byref(st)))
        return st.as_dict()

    def unpack(self, packed, n_kramers, block, full):
        """packed/full: torch cuda float64 tensors; full holds (2n)^4 complex values
        (n^4 after set_spinor_coefficients, n counting spinors)."""
        self._check(self.L.qdt_unpack(self.h, _ptr(packed), int(n_kramers), blocks_mask([block]), _ptr(full)))


    def graph_counts(self):
        """(graphs captured, graph replays) of the batches this context owned."""
        c, r = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.L.qdt_graph_counts(self.h, ctypes.byref(c), ctypes.byref(r)))
        return c.value, r.value


def transform_batch(jobs, graph=False, raise_on_error=True):
    """Several transformations as one batch (qdt_transform_batch).

    jobs: list of (Context, blocks, k_begin, k_end, tau, precision, out), every
    Context distinct.  Returns (status list, stats dicts); with raise_on_error
    a failing item raises QdtError with its message instead."""
    L = load()
    n = len(jobs)
    items = (BatchItem * n)()
    stats = [Stats() for _ in range(n)]
    for i, (ctx, blocks, k0, k1, tau, prec, out) in enumerate(jobs):
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        items[i].ctx = ctx.h
        items[i].blocks = blocks_mask(blocks)
        items[i].k_begin, items[i].k_end = int(k0), int(k1)
        items[i].schwarz_tau = float(tau)
        items[i].precision = int(prec)
        items[i].out = _ptr(out)
        items[i].out_bytes = nbytes
        items[i].stats = ctypes.addressof(stats[i])
    rc = L.qdt_transform_batch(items, n, BATCH_GRAPH if graph else 0)
    status = [items[i].status for i in range(n)]
    if rc != 0 and raise_on_error:
        bad = next(i for i in range(n) if status[i] != 0)
        raise QdtError(rc, "item %d: %s" % (bad, L.qdt_last_error(jobs[bad][0].h).decode()))
    return status, [s.as_dict() for s in stats]


def version():
    return load().qdt_version().decode()


class Server:
    """Continuous-batching request server (qdt_server_*): n_slots concurrent
    contexts on one GPU, admission by device-memory footprint."""

    def __init__(self, device=0, n_slots=4, pool_bytes=0):
        self.L = load()
        h = ctypes.c_void_p()
        rc = self.L.qdt_server_create(ctypes.byref(h), int(device), int(n_slots), int(pool_bytes))
        if rc != 0:
            raise QdtError(rc, "qdt_server_create failed")
        self.h = h
        self._keep = {}

    def make_request(self, problem, blocks, k_begin, k_end, tau, precision, out, CL=None, CS=None):
        b = problem.basis
        arrs = [np.ascontiguousarray(b.xyz, np.float64), np.ascontiguousarray(b.shell_center, np.int32),
                np.ascontiguousarray(b.shell_l, np.int32), np.ascontiguousarray(b.shell_nprim, np.int32),
                np.ascontiguousarray(b.exps, np.float64), np.ascontiguousarray(b.coefs, np.float64),
                np.ascontiguousarray(problem.CL if CL is None else CL, np.float64),
                np.ascontiguousarray(problem.CS if CS is None else CS, np.float64)]
        nbytes = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
        r = Request(int(arrs[0].shape[0]), _ptr(arrs[0]), int(arrs[1].shape[0]), _ptr(arrs[1]), _ptr(arrs[2]),
                    _ptr(arrs[3]), _ptr(arrs[4]), _ptr(arrs[5]), int(arrs[6].shape[1]), _ptr(arrs[6]),
                    _ptr(arrs[7]), blocks_mask(blocks), int(k_begin), int(k_end), float(tau), int(precision),
                    _ptr(out), nbytes)
        return r, arrs + [out]

    def footprint(self, req):
        return int(self.L.qdt_footprint(ctypes.byref(req)))

    def submit(self, req, keep):
        hd = ctypes.c_uint64()
        rc = self.L.qdt_submit(self.h, ctypes.byref(req), ctypes.byref(hd))
        if rc != 0:
            raise QdtError(rc, "qdt_submit")
        self._keep[hd.value] = (req, keep)
        return hd.value

    def poll(self, handle):
        d = ctypes.c_int()
        rc = self.L.qdt_poll(self.h, ctypes.c_uint64(handle), ctypes.byref(d))
        if rc != 0:
            raise QdtError(rc, "qdt_poll")
        return bool(d.value)

    def wait(self, handle, timeout=-1.0):
        lat = ctypes.c_double()
        st = Stats()
        rc = self.L.qdt_wait(self.h, ctypes.c_uint64(handle), float(timeout), ctypes.byref(lat), ctypes.byref(st))
        if rc == -6 and timeout >= 0:
            raise TimeoutError("request %d still running" % handle)
        self._keep.pop(handle, None)
        if rc != 0:
            raise QdtError(rc, "request %d failed" % handle)
        return lat.value, st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.L.qdt_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def second_half_noalloc(Dq, V, O, stream=None):
    """O = Dq^T V (FP64, upper 64x64 tiles) through qdt_second_half_noalloc:
    no device allocation.  Dq, V: CUDA float64 contiguous [K, N] of the same
    shape; O: CUDA float64 contiguous [N, N].  The C entry point takes no size
    for V or O, so the shapes are checked here before anything is launched."""
    for name, t in (("Dq", Dq), ("V", V), ("O", O)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError("second_half_noalloc: %s must be a CUDA tensor" % name)
        if str(t.dtype) != "torch.float64":
            raise ValueError("second_half_noalloc: %s must be float64, not %s" % (name, t.dtype))
        if t.dim() != 2 or not t.is_contiguous():
            raise ValueError("second_half_noalloc: %s must be a contiguous 2-D tensor" % name)
    if tuple(V.shape) != tuple(Dq.shape):
        raise ValueError("second_half_noalloc: V %s must have Dq's shape %s" % (tuple(V.shape), tuple(Dq.shape)))
    N = int(Dq.shape[1])
    if tuple(O.shape) != (N, N):
        raise ValueError("second_half_noalloc: O %s must be (%d, %d)" % (tuple(O.shape), N, N))
    if Dq.device != V.device or Dq.device != O.device:
        raise ValueError("second_half_noalloc: Dq, V and O must be on one device")
    L = load()
    buf = ctypes.create_string_buffer(512)
    sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    rc = L.qdt_second_half_noalloc(_ptr(Dq), _ptr(V), int(Dq.shape[0]), N, _ptr(O), sp, buf, 512)
    if rc != 0:
        raise QdtError(rc, buf.value.decode())


def alu_peak(device=0, kind="fp32"):
    """Measured FMA throughput (TFLOP/s) of the CUDA cores: kind "fp32" or "fp64"."""
    L = load()
    v = ctypes.c_double()
    rc = L.qdt_alu_peak(int(device), {"fp32": 0, "fp64": 1}[kind], ctypes.byref(v))
    if rc != 0:
        raise QdtError(rc, "qdt_alu_peak")
    return v.value
