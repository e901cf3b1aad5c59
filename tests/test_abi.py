"""CPU checks of the C ABI boundary: the library builds, loads, exports every
function declared in include/cmif.h, and rejects bad arguments on the host
before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2106_14699_gb300 as cm
from paper_2106_14699_gb300 import build as cmbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "cmif.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cmif_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libcmif():
    cmbuild.build()
    return cm.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cmif_plan_create", "cmif_plan_create_ex", "cmif_plan_destroy", "cmif_compute",
                     "cmif_get_status", "cmif_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libcmif):
    for name in _declared():
        assert hasattr(libcmif, name), f"{name} declared in cmif.h but not exported"
    assert set(_declared()) == set(cm.EXPORTS)


def test_host_side_argument_errors(libcmif):
    h = ctypes.c_void_p()
    P = ctypes.byref(h)
    assert libcmif.cmif_plan_create_ex(P, 0, 4, 4, 4, 2, 2, cm.FP32, 0) == 1     # H_A < 1
    assert libcmif.cmif_plan_create_ex(P, 4, 4, 4, 4, 0, 2, cm.FP32, 0) == 1     # K_A < 1
    assert libcmif.cmif_plan_create_ex(P, 4, 4, 4, 4, 65, 2, cm.FP32, 0) == 1    # K_A > 64
    assert libcmif.cmif_plan_create_ex(P, 4, 4, 4, 4, 2, 2, 9, 0) == 1           # bad precision
    assert libcmif.cmif_plan_create_ex(P, 4, 4, 4, 4, 2, 2, cm.FP32, 0x80) == 1  # unknown flag
    assert libcmif.cmif_plan_create_ex(P, 4096, 1025, 8, 8, 2, 2, cm.FP32, 0) == 1  # H*W > 2^22
    assert libcmif.cmif_plan_create_ex(P, 2049, 2, 2049, 2, 2, 2, cm.FP32, 0) == 8  # P > 4096
    assert libcmif.cmif_plan_create_ex(None, 4, 4, 4, 4, 2, 2, cm.FP32, 0) == 1
    assert libcmif.cmif_compute(None, None, None, None, None, None, None, None, 0.0, None, None) == 1
    assert libcmif.cmif_plan_destroy(None) == 0
    assert libcmif.cmif_status_string(2) == b"label outside [0, K) under mask"


def test_host_side_argument_errors_of_the_extensions(libcmif):
    """Volume, weighted, rotation and batch entry points reject bad arguments on
    the host, before any CUDA call (status codes of include/cmif.h)."""
    h = ctypes.c_void_p()
    P = ctypes.byref(h)
    INVALID, UNSUPPORTED = 1, 8
    c3 = libcmif.cmif_plan_create_3d
    assert c3(P, 0, 4, 4, 2, 4, 4, 2, 2, cm.FP32, 0) == INVALID                          # D_A < 1
    assert c3(P, 2, 4, 4, 1025, 4, 4, 2, 2, cm.FP32, 0) == INVALID                       # D_B > 1024
    assert c3(P, 65, 256, 256, 2, 4, 4, 2, 2, cm.FP32, 0) == INVALID                     # D*H*W > 2^22
    assert c3(P, 2, 4, 4, 2, 4, 4, 2, 2, cm.FP32, cm.FLAG_WINDOW) == UNSUPPORTED         # no window in 3-D
    assert c3(P, 2, 4, 4, 1, 4, 4, 2, 2, cm.FP64, cm.FLAG_WEIGHTED) == UNSUPPORTED       # no weights in 3-D
    assert not h.value
    ce = libcmif.cmif_plan_create_ex
    assert ce(P, 4, 4, 4, 4, 2, 2, cm.FP32, cm.FLAG_WEIGHTED) == UNSUPPORTED                   # SWMI is FP64
    assert ce(P, 4, 4, 4, 4, 2, 2, cm.FP64, cm.FLAG_WEIGHTED | cm.FLAG_NMI) == UNSUPPORTED     # MI only
    assert ce(P, 4, 4, 4, 4, 2, 2, cm.FP64, cm.FLAG_WEIGHTED | cm.FLAG_DEBUG_COUNTS) == UNSUPPORTED
    assert libcmif.cmif_compute_weighted(None, None, None, None, None, None, None, 0.0, None, None) == INVALID
    assert libcmif.cmif_align_rotations(None, None, None, None, None, None, 1, 0.5, 1, None, None, None, None) == INVALID
    pk, th = cm.Peak(), ctypes.c_double()
    assert libcmif.cmif_align_two_stage(None, None, None, None, None, 8, None, 0, 0.5, ctypes.byref(pk),
                                        ctypes.byref(th), None) == INVALID
    assert libcmif.cmif_rotate_nn(None, None, 4, 4, 0.1, None, None, None) == INVALID
    b = ctypes.c_void_p()
    assert libcmif.cmif_batch_create(ctypes.byref(b), 0, None, cm.FP32, 0) == INVALID          # no pairs
    assert libcmif.cmif_batch_create(None, 1, None, cm.FP32, 0) == INVALID
    assert not b.value
    assert libcmif.cmif_entropy_terms(0, 4, None, None) == INVALID                              # no output
    assert libcmif.cmif_entropy_terms(-1, 4, ctypes.c_void_p(16), None) == INVALID              # c0 < 0
    assert libcmif.cmif_entropy_terms((1 << 22) - 2, 4, ctypes.c_void_p(16), None) == INVALID  # beyond 2^22
    assert libcmif.cmif_plan_set_wait_test(None, 0, -1) == INVALID
    assert libcmif.cmif_plan_autotune(None, None, None) == INVALID


_LAYOUT_PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "cmif.h"
#define OFF(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
    printf("sizeof.cmif_peak %zu\nsizeof.cmif_pair_desc %zu\n", sizeof(cmif_peak), sizeof(cmif_pair_desc));
    OFF(cmif_peak, angle_idx); OFF(cmif_peak, dy); OFF(cmif_peak, dx); OFF(cmif_peak, n); OFF(cmif_peak, mi);
    OFF(cmif_pair_desc, A); OFF(cmif_pair_desc, M_A); OFF(cmif_pair_desc, B); OFF(cmif_pair_desc, M_B);
    OFF(cmif_pair_desc, H_A); OFF(cmif_pair_desc, W_A); OFF(cmif_pair_desc, H_B); OFF(cmif_pair_desc, W_B);
    OFF(cmif_pair_desc, K_A); OFF(cmif_pair_desc, K_B); OFF(cmif_pair_desc, angles_rad);
    OFF(cmif_pair_desc, n_angles); OFF(cmif_pair_desc, gamma);
    printf("prec %d %d %d %d\n", CMIF_FP32, CMIF_SPLIT32, CMIF_FP64, CMIF_AUTO);
    printf("flags %u %u %u %u %u %u %u\n", CMIF_FLAG_DEBUG_COUNTS, CMIF_FLAG_GRAPH, CMIF_FLAG_WINDOW, CMIF_FLAG_NMI,
           CMIF_FLAG_WEIGHTED, CMIF_FLAG_AUTOTUNE, CMIF_FLAG_BATCH_ANGLES);
    printf("sizeof.cmif_tuning %zu\n", sizeof(cmif_tuning));
    OFF(cmif_tuning, col_lanes); OFF(cmif_tuning, tmem_rows); OFF(cmif_tuning, cols_blocks_per_sm);
    OFF(cmif_tuning, ms_per_map); OFF(cmif_tuning, from_cache); OFF(cmif_tuning, candidates);
    printf("status %d %d %d %d %d %d %d %d %d\n", CMIF_OK, CMIF_ERR_INVALID_ARG, CMIF_ERR_LABEL_RANGE, CMIF_ERR_OOM,
           CMIF_ERR_CUDA, CMIF_ERR_PRECISION, CMIF_ERR_TIMEOUT, CMIF_ERR_NOT_IMPLEMENTED, CMIF_ERR_UNSUPPORTED);
    printf("fixbits %d\n", CMIF_ENTROPY_FIX_BITS);
    return 0;
}
"""


def test_binding_mirrors_the_header(tmp_path, libcmif):
    """The ctypes structs, precision and flag constants and status names of the
    binding match what a C compiler makes of include/cmif.h, and every status
    has its string."""
    import subprocess
    src, exe = tmp_path / "probe.c", tmp_path / "probe"
    src.write_text(_LAYOUT_PROBE)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    out = dict(line.split(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(out["sizeof.cmif_peak"]) == ctypes.sizeof(cm.Peak)
    assert int(out["sizeof.cmif_pair_desc"]) == ctypes.sizeof(cm.PairDesc)
    assert int(out["sizeof.cmif_tuning"]) == ctypes.sizeof(cm.Tuning)
    for T, S in (("cmif_peak", cm.Peak), ("cmif_pair_desc", cm.PairDesc), ("cmif_tuning", cm.Tuning)):
        for name, _ in S._fields_:
            assert int(out[f"{T}.{name}"]) == getattr(S, name).offset, (T, name)
    assert [int(v) for v in out["prec"].split()] == [cm.FP32, cm.SPLIT32, cm.FP64, cm.AUTO]
    assert [int(v) for v in out["flags"].split()] == [cm.FLAG_DEBUG_COUNTS, cm.FLAG_GRAPH, cm.FLAG_WINDOW,
                                                      cm.FLAG_NMI, cm.FLAG_WEIGHTED, cm.FLAG_AUTOTUNE,
                                                      cm.FLAG_BATCH_ANGLES]
    assert int(out["fixbits"]) == cm.ENTROPY_FIX_BITS
    codes = [int(v) for v in out["status"].split()]
    assert codes == sorted(cm.STATUS_NAMES)
    for c in codes:
        s = libcmif.cmif_status_string(c)
        assert s and s != libcmif.cmif_status_string(99)


def test_peaks_from_bytes_decodes_the_record_layout():
    import struct
    recs = [(3, -7, 12, 4096, 1.25), (-1, 0, 0, 0, 0.0), (0, 1023, -1023, 1, 2.0 ** -22)]
    raw = b"".join(struct.pack("<iiiid", *r) for r in recs)
    assert len(raw) == 24 * len(recs)
    assert cm.peaks_from_bytes(raw, len(recs)) == recs
    assert cm.peaks_from_bytes(raw, 1) == recs[:1]
