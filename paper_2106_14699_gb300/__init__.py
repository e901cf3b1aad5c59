"""Python binding of the GB300 CMIF library (``include/cmif.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libcmif.so``.  There is no CPU fallback; if the library is not
built, every call raises.  PyTorch is used for device memory and streams.

The names follow the C ABI: ``Plan`` wraps ``cmif_plan_create_ex`` /
``cmif_compute`` / ``cmif_compute_host`` / ``cmif_get_status`` /
``cmif_plan_destroy``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["FP32", "SPLIT32", "FP64", "AUTO", "Plan", "Peak", "CmifError", "lib", "STATUS_NAMES", "cmif"]

FP32, SPLIT32, FP64, AUTO = 0, 1, 2, 3
FLAG_DEBUG_COUNTS = 1
FLAG_GRAPH = 2
FLAG_WINDOW = 4
FLAG_NMI = 8
FLAG_WEIGHTED = 16
FLAG_AUTOTUNE = 32
FLAG_BATCH_ANGLES = 64
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "LABEL_RANGE", 3: "OOM", 4: "CUDA", 5: "PRECISION",
                6: "TIMEOUT", 7: "NOT_IMPLEMENTED", 8: "UNSUPPORTED"}


class CmifError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}" if what else STATUS_NAMES.get(code, str(code)))


class PairDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("M_A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("M_B", ctypes.c_void_p),
                ("H_A", ctypes.c_int), ("W_A", ctypes.c_int), ("H_B", ctypes.c_int), ("W_B", ctypes.c_int),
                ("K_A", ctypes.c_int), ("K_B", ctypes.c_int), ("angles_rad", ctypes.c_void_p),
                ("n_angles", ctypes.c_int), ("gamma", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("col_lanes", ctypes.c_int), ("tmem_rows", ctypes.c_int), ("cols_blocks_per_sm", ctypes.c_int),
                ("ms_per_map", ctypes.c_double), ("from_cache", ctypes.c_int), ("candidates", ctypes.c_int)]


class Peak(ctypes.Structure):
    _fields_ = [("angle_idx", ctypes.c_int32), ("dy", ctypes.c_int32), ("dx", ctypes.c_int32),
                ("n", ctypes.c_int32), ("mi", ctypes.c_double)]


EXPORTS = ["cmif_plan_create", "cmif_plan_create_ex", "cmif_plan_create_3d", "cmif_plan_destroy", "cmif_plan_workspace_bytes",
           "cmif_compute", "cmif_compute_host", "cmif_get_status", "cmif_plan_set_profiling",
           "cmif_plan_stage_times", "cmif_compute_noalloc", "cmif_rotate_nn", "cmif_align_rotations",
           "cmif_align_two_stage", "cmif_compute_weighted", "cmif_batch_create", "cmif_compute_batch", "cmif_batch_get_status",
           "cmif_batch_destroy", "cmif_entropy_terms", "cmif_plan_set_wait_test", "cmif_get_precision_report",
           "cmif_plan_autotune", "cmif_status_string"]

_lib = None


def lib():
    """Load libcmif.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIBPATH
        if not os.path.exists(path):
            raise CmifError(4, f"{path} is not built (run __graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(path)
        P, I, D, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint
        L.cmif_plan_create.argtypes = [ctypes.POINTER(P), I, I, I, I, I]
        L.cmif_plan_create_ex.argtypes = [ctypes.POINTER(P), I, I, I, I, I, I, I, U]
        L.cmif_plan_create_3d.argtypes = [ctypes.POINTER(P), I, I, I, I, I, I, I, I, I, U]
        L.cmif_plan_destroy.argtypes = [P]
        L.cmif_plan_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.cmif_compute.argtypes = [P, P, P, P, P, P, P, P, D, P, P]
        L.cmif_compute_host.argtypes = [P, P, P, P, P, P, P, D, P, P]
        L.cmif_get_status.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I)]
        L.cmif_plan_set_profiling.argtypes = [P, I]
        L.cmif_plan_stage_times.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(ctypes.c_char_p)]
        L.cmif_compute_noalloc.argtypes = [I, I, I, I, I, I, P, P, P, P, P, P, D, P, P, P]
        L.cmif_rotate_nn.argtypes = [P, P, I, I, D, P, P, P]
        L.cmif_align_rotations.argtypes = [P, P, P, P, P, P, I, D, I, P, P, P, P]
        L.cmif_compute_weighted.argtypes = [P, P, P, P, P, P, P, D, P, P]
        L.cmif_align_two_stage.argtypes = [P, P, P, P, P, I, P, I, D, ctypes.POINTER(Peak), ctypes.POINTER(D), P]
        L.cmif_batch_create.argtypes = [ctypes.POINTER(P), I, P, I, U]
        L.cmif_compute_batch.argtypes = [P, P, P, P]
        L.cmif_batch_get_status.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I)]
        L.cmif_batch_destroy.argtypes = [P]
        L.cmif_entropy_terms.argtypes = [I, I, P, P]
        L.cmif_plan_set_wait_test.argtypes = [P, I, I]
        L.cmif_plan_autotune.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(Tuning)]
        L.cmif_get_precision_report.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D),
                                                ctypes.POINTER(D)]
        L.cmif_status_string.argtypes = [I]
        L.cmif_status_string.restype = ctypes.c_char_p
        for name in EXPORTS[:-1]:
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(code, what):
    if code != 0:
        raise CmifError(code, what)


class Plan:
    """A CMIF plan for images H_A x W_A and H_B x W_B with K_A, K_B labels."""

    def __init__(self, H_A, W_A, H_B, W_B, K_A, K_B, precision=FP32, debug_counts=False, graph=False, window=False,
                 nmi=False, weighted=False, autotune=False, batch_angles=False):
        self._h = ctypes.c_void_p()
        flags = (FLAG_DEBUG_COUNTS if debug_counts else 0) | (FLAG_GRAPH if graph else 0) | \
            (FLAG_WINDOW if window else 0) | (FLAG_NMI if nmi else 0) | (FLAG_WEIGHTED if weighted else 0) | \
            (FLAG_AUTOTUNE if autotune else 0) | (FLAG_BATCH_ANGLES if batch_angles else 0)
        _check(lib().cmif_plan_create_ex(ctypes.byref(self._h), H_A, W_A, H_B, W_B, K_A, K_B, precision, flags),
               "cmif_plan_create_ex")
        self.H_A, self.W_A, self.H_B, self.W_B, self.K_A, self.K_B = H_A, W_A, H_B, W_B, K_A, K_B
        self.precision = precision
        self.R, self.C = H_A + H_B - 1, W_A + W_B - 1

    @property
    def handle(self):
        return self._h.value

    def workspace_bytes(self):
        n = ctypes.c_size_t()
        _check(lib().cmif_plan_workspace_bytes(self._h, ctypes.byref(n)), "cmif_plan_workspace_bytes")
        return n.value

    def compute(self, A, M_A, B, M_B, mi_map, n_map=None, counts=None, gamma=0.0, peak=None, stream=None):
        """Device-pointer call (torch CUDA tensors or raw addresses); asynchronous."""
        _check(lib().cmif_compute(self._h, _ptr(A), _ptr(M_A), _ptr(B), _ptr(M_B), _ptr(mi_map), _ptr(n_map),
                                  _ptr(counts), float(gamma), _ptr(peak), _stream(stream)), "cmif_compute")

    def compute_weighted(self, A, W_A, B, W_B, mi_map, nw_map=None, gamma=0.0, peak=None, stream=None):
        """Spatially weighted MI map (device tensors; weights float64 or None); asynchronous."""
        _check(lib().cmif_compute_weighted(self._h, _ptr(A), _ptr(W_A), _ptr(B), _ptr(W_B), _ptr(mi_map),
                                           _ptr(nw_map), float(gamma), _ptr(peak), _stream(stream)),
               "cmif_compute_weighted")

    def compute_host(self, A, M_A, B, M_B, mi_map, n_map=None, gamma=0.0, peak=None, stream=None):
        """Host-buffer call (numpy, ideally pinned); copies in and out, synchronises."""
        pk = ctypes.byref(peak) if peak is not None else None
        _check(lib().cmif_compute_host(self._h, _ptr(A), _ptr(M_A), _ptr(B), _ptr(M_B), _ptr(mi_map), _ptr(n_map),
                                       float(gamma), pk, _stream(stream)), "cmif_compute_host")

    def align_rotations(self, A, M_A, B, M_B, angles_rad, gamma, top_k, topk_dev, mi_maps=None, stream=None,
                        n_maps=None):
        """Alg. 1 over rotations (device tensors; angles: host sequence of radians); asynchronous."""
        ang = np.ascontiguousarray(np.asarray(angles_rad, dtype=np.float64))
        _check(lib().cmif_align_rotations(self._h, _ptr(A), _ptr(M_A), _ptr(B), _ptr(M_B), ang.ctypes.data,
                                          len(ang), float(gamma), int(top_k), _ptr(topk_dev), _ptr(mi_maps),
                                          _ptr(n_maps), _stream(stream)), "cmif_align_rotations")

    def align_two_stage(self, A, M_A, B, M_B, n_grid, refine_u, gamma, stream=None):
        """Two-stage rigid alignment; returns ((angle_idx, dy, dx, n, mi), angle_rad); synchronises."""
        u = np.ascontiguousarray(np.asarray(refine_u, dtype=np.float64))
        pk, ang = Peak(), ctypes.c_double()
        _check(lib().cmif_align_two_stage(self._h, _ptr(A), _ptr(M_A), _ptr(B), _ptr(M_B), int(n_grid),
                                          u.ctypes.data if len(u) else None, len(u), float(gamma), ctypes.byref(pk),
                                          ctypes.byref(ang), _stream(stream)), "cmif_align_two_stage")
        return (pk.angle_idx, pk.dy, pk.dx, pk.n, pk.mi), ang.value

    def set_wait_test(self, poll_limit=0, withhold_row=-1):
        """Diagnostics of the bounded device waits (cmif_plan_set_wait_test)."""
        _check(lib().cmif_plan_set_wait_test(self._h, int(poll_limit), int(withhold_row)), "cmif_plan_set_wait_test")

    def status(self):
        """(device status name, max residual, escalations) of the last call; synchronises."""
        ds, res, esc = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(lib().cmif_get_status(self._h, ctypes.byref(ds), ctypes.byref(res), ctypes.byref(esc)), "cmif_get_status")
        return STATUS_NAMES.get(ds.value, ds.value), res.value, esc.value

    def precision_report(self):
        """(pairs predicted, pairs escalated, FP32 residual, second-precision residual) of the last call."""
        pp, pe, r0, r1 = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(lib().cmif_get_precision_report(self._h, ctypes.byref(pp), ctypes.byref(pe), ctypes.byref(r0),
                                               ctypes.byref(r1)), "cmif_get_precision_report")
        return pp.value, pe.value, r0.value, r1.value

    def autotune(self, cache_path=None):
        """cmif_plan_autotune: time the launch-shape candidates, keep the fastest; returns the choice."""
        t = Tuning()
        _check(lib().cmif_plan_autotune(self._h, cache_path.encode() if cache_path else None, ctypes.byref(t)),
               "cmif_plan_autotune")
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_profiling(self, enable=True):
        _check(lib().cmif_plan_set_profiling(self._h, 1 if enable else 0), "cmif_plan_set_profiling")

    def stage_times(self, max_n=64):
        """[(kernel name, ms)] of the last call's launches (profiling on); synchronises."""
        n = ctypes.c_int()
        ms = (ctypes.c_double * max_n)()
        names = (ctypes.c_char_p * max_n)()
        _check(lib().cmif_plan_stage_times(self._h, max_n, ctypes.byref(n), ms, names), "cmif_plan_stage_times")
        return [(names[i].decode(), ms[i]) for i in range(min(n.value, max_n))]

    def close(self):
        if self._h and self._h.value:
            lib().cmif_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class VolumePlan(Plan):
    """A CMIF plan for volumes D_A x H_A x W_A and D_B x H_B x W_B (cmif_plan_create_3d);
    compute() then fills maps of (D_A + D_B - 1) * (H_A + H_B - 1) rows by W_A + W_B - 1
    columns (depth-offset major), and the peak's first field is dz."""

    def __init__(self, D_A, H_A, W_A, D_B, H_B, W_B, K_A, K_B, precision=FP32, debug_counts=False, graph=False,
                 nmi=False):
        self._h = ctypes.c_void_p()
        flags = (FLAG_DEBUG_COUNTS if debug_counts else 0) | (FLAG_GRAPH if graph else 0) | (FLAG_NMI if nmi else 0)
        _check(lib().cmif_plan_create_3d(ctypes.byref(self._h), D_A, H_A, W_A, D_B, H_B, W_B, K_A, K_B, precision,
                                         flags), "cmif_plan_create_3d")
        self.D_A, self.D_B = D_A, D_B
        self.H_A, self.W_A, self.H_B, self.W_B, self.K_A, self.K_B = H_A, W_A, H_B, W_B, K_A, K_B
        self.precision = precision
        self.R, self.C = (D_A + D_B - 1) * (H_A + H_B - 1), W_A + W_B - 1


class Batch:
    """cmif_batch over pairs given as dicts with device tensors A, M_A, B, M_B, K_A, K_B,
    host angle lists `angles` (radians) and `gamma`."""

    def __init__(self, pairs, precision=FP32, graph=True, window=False, nmi=False, autotune=False,
                 batch_angles=False):
        self._keep = []
        descs = (PairDesc * len(pairs))()
        for i, p in enumerate(pairs):
            ang = np.ascontiguousarray(np.asarray(p.get("angles", []), dtype=np.float64))
            self._keep.append(ang)
            H_A, W_A = p["A"].shape
            H_B, W_B = p["B"].shape
            descs[i] = PairDesc(_ptr(p["A"]), _ptr(p.get("M_A")), _ptr(p["B"]), _ptr(p.get("M_B")), H_A, W_A, H_B, W_B,
                                p["K_A"], p["K_B"], ang.ctypes.data if len(ang) else None, len(ang),
                                float(p.get("gamma", 0.5)))
        self._descs = descs
        self._h = ctypes.c_void_p()
        _check(lib().cmif_batch_create(ctypes.byref(self._h), len(pairs), ctypes.cast(descs, ctypes.c_void_p),
                                       precision, (FLAG_GRAPH if graph else 0) | (FLAG_WINDOW if window else 0) |
                                       (FLAG_NMI if nmi else 0) | (FLAG_AUTOTUNE if autotune else 0) |
                                       (FLAG_BATCH_ANGLES if batch_angles else 0)),
               "cmif_batch_create")
        self.n = len(pairs)

    def run(self, results_dev, status_dev=None, stream=None):
        _check(lib().cmif_compute_batch(self._h, _ptr(results_dev), _ptr(status_dev), _stream(stream)),
               "cmif_compute_batch")

    def status(self):
        ds, res, esc = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(lib().cmif_batch_get_status(self._h, ctypes.byref(ds), ctypes.byref(res), ctypes.byref(esc)),
               "cmif_batch_get_status")
        return STATUS_NAMES.get(ds.value, ds.value), res.value, esc.value

    def close(self):
        if self._h and self._h.value:
            lib().cmif_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rotate_nn(B, M_B, theta, B_out, M_out, stream=None):
    """cmif_rotate_nn on torch CUDA tensors."""
    H, W = B.shape
    _check(lib().cmif_rotate_nn(_ptr(B), _ptr(M_B), H, W, float(theta), _ptr(B_out), _ptr(M_out), _stream(stream)),
           "cmif_rotate_nn")


def peaks_from_bytes(buf, count):
    """Decode `count` cmif_peak records from a uint8 tensor / bytes."""
    raw = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
    out = []
    for i in range(count):
        pk = Peak.from_buffer_copy(raw[24 * i:24 * (i + 1)])
        out.append((pk.angle_idx, pk.dy, pk.dx, pk.n, pk.mi))
    return out


def entropy_terms(c0, n, out, stream=None):
    """cmif_entropy_terms: out (torch int64 CUDA tensor of n elements) = the epilogue's c log2 c
    for c = c0 .. c0 + n - 1, in units of 2^-ENTROPY_FIX_BITS."""
    _check(lib().cmif_entropy_terms(int(c0), int(n), _ptr(out), _stream(stream)), "cmif_entropy_terms")


ENTROPY_FIX_BITS = 23


def compute_noalloc(A, M_A, B, M_B, K_A, K_B, mi_map, n_map=None, gamma=0.0, peak=None, status=None,
                    stream=None):
    """cmif_compute_noalloc on torch CUDA tensors (no plan, no device allocation in the library).

    The tensors are checked here (dtype, shape, contiguity, device) because the C
    entry point writes through the raw pointers it is given; the call runs on A's device."""
    import torch
    H_A, W_A = A.shape
    H_B, W_B = B.shape
    R, C = H_A + H_B - 1, W_A + W_B - 1
    dev = A.device

    def need(t, dtype, numel, what, shape=None):
        ok = (t.device == dev and t.dtype == dtype and t.is_contiguous() and t.numel() >= numel and
              (shape is None or tuple(t.shape) == shape))
        if not ok:
            raise CmifError(1, f"cmif_compute_noalloc: {what} must be a contiguous {dtype} tensor on {dev}"
                               + (f" of shape {shape}" if shape else f" with at least {numel} elements"))

    if dev.type != "cuda":
        raise CmifError(1, "cmif_compute_noalloc: A must be a CUDA tensor")
    need(A, torch.int32, H_A * W_A, "A", (H_A, W_A))
    need(B, torch.int32, H_B * W_B, "B", (H_B, W_B))
    if M_A is not None:
        need(M_A, torch.uint8, H_A * W_A, "M_A", (H_A, W_A))
    if M_B is not None:
        need(M_B, torch.uint8, H_B * W_B, "M_B", (H_B, W_B))
    need(mi_map, torch.float64, R * C, "mi_map", (R, C))
    if n_map is not None:
        need(n_map, torch.int32, R * C, "n_map", (R, C))
    if peak is not None:
        need(peak, torch.uint8, 24, "peak")
    if status is not None:
        need(status, torch.int32, 1, "status")
    with torch.cuda.device(dev):
        _check(lib().cmif_compute_noalloc(H_A, W_A, H_B, W_B, K_A, K_B, _ptr(A), _ptr(M_A), _ptr(B), _ptr(M_B),
                                          _ptr(mi_map), _ptr(n_map), float(gamma), _ptr(peak), _ptr(status),
                                          _stream(stream)), "cmif_compute_noalloc")


def cmif(A, M_A, B, M_B, K_A, K_B, precision=FP32, gamma=0.0, with_counts=False, plan=None, stream=None):
    """Convenience: CMIF map of torch CUDA tensors.  Returns dict(mi, n, peak[, counts], status)."""
    import torch
    H_A, W_A = A.shape
    H_B, W_B = B.shape
    own = plan is None
    if own:
        plan = Plan(H_A, W_A, H_B, W_B, K_A, K_B, precision, debug_counts=with_counts)
    dev = A.device
    mi = torch.empty((plan.R, plan.C), dtype=torch.float64, device=dev)
    n = torch.empty((plan.R, plan.C), dtype=torch.int32, device=dev)
    counts = None
    if with_counts:
        counts = torch.empty((K_A * K_B + K_A + K_B, plan.R, plan.C), dtype=torch.int32, device=dev)
    peak = torch.empty(24, dtype=torch.uint8, device=dev)
    plan.compute(A, M_A, B, M_B, mi, n, counts, gamma, peak, stream)
    st = plan.status()
    pk = Peak.from_buffer_copy(peak.cpu().numpy().tobytes())
    out = dict(mi=mi, n=n, peak=(pk.angle_idx, pk.dy, pk.dx, pk.n, pk.mi), status=st)
    if with_counts:
        out["counts"] = counts
    if own:
        plan.close()
    return out
