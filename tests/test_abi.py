"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, its parameter block matches the ctypes mirror byte for byte,
and host-side validation rejects bad arguments before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2512_11086_gb300 as rc
from paper_2512_11086_gb300 import build as rbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rcbf.h")


@pytest.fixture(scope="module")
def lib():
    rbuild.build()
    return rc.load_library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(rcbf_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_expected_entry_points():
    names = _declared_functions()
    for n in ("rcbf_plan", "rcbf_decode", "rcbf_das", "rcbf_das_backward", "rcbf_destroy",
              "rcbf_last_error", "rcbf_batch_create", "rcbf_batch_run"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared_functions()) <= set(rc.SIGNATURES)


def test_params_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rcbf.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(rcbf_params),"
        " offsetof(rcbf_params, fs), offsetof(rcbf_params, xdc_transform),"
        " offsetof(rcbf_params, voxel_transform), offsetof(rcbf_params, f_number),"
        " offsetof(rcbf_params, decode_matrix)); return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    P = rc.Params
    want = [ctypes.sizeof(P), P.fs.offset, P.xdc_transform.offset, P.voxel_transform.offset,
            P.f_number.offset, P.decode_matrix.offset]
    assert got == want


def test_plan_info_layout_matches_header(tmp_path):
    src = tmp_path / "info.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rcbf.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu\\n\", sizeof(rcbf_plan_info),"
        " offsetof(rcbf_plan_info, workspace_bytes), offsetof(rcbf_plan_info, bwd_tile),"
        " offsetof(rcbf_plan_info, bwd_mode)); return 0;}\n")
    exe = tmp_path / "info"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    I = rc.PlanInfo
    assert got == [ctypes.sizeof(I), I.workspace_bytes.offset, I.bwd_tile.offset, I.bwd_mode.offset]


def test_ceilings_layout_matches_header(tmp_path):
    src = tmp_path / "ceil.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "rcbf.h"\n'
        "int main(void){printf(\"%zu %zu %zu\\n\", sizeof(rcbf_ceilings),"
        " offsetof(rcbf_ceilings, red_shared_per_s), offsetof(rcbf_ceilings, sm_clock_hz)); return 0;}\n")
    exe = tmp_path / "ceil"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    C = rc.Ceilings
    assert got == [ctypes.sizeof(C), C.red_shared_per_s.offset, C.sm_clock_hz.offset]


def test_measure_ceilings_rejects_null():
    lib = rc.load_library()
    assert lib.rcbf_measure_ceilings(None, None) == rc.EINVAL


def _good_params():
    import synth
    return rc.make_params(synth.tiny_bscan_geometry(), decoded_dtype="f32")


@pytest.mark.parametrize("mutate,code", [
    (lambda p: setattr(p, "n_samples", 1001), rc.EINVAL),
    (lambda p: setattr(p, "n_samples", 0), rc.EINVAL),
    (lambda p: setattr(p, "n_tx", 0), rc.EINVAL),
    (lambda p: setattr(p, "n_tx", 300), rc.EINVAL),
    (lambda p: setattr(p, "hadamard_order", 16), rc.EINVAL),
    (lambda p: (setattr(p, "n_tx", 48), setattr(p, "hadamard_order", 48)), rc.EINVAL),
    (lambda p: setattr(p, "interp", 2), rc.EUNSUPPORTED),
    (lambda p: setattr(p, "decoded_dtype", 9), rc.EUNSUPPORTED),
    (lambda p: setattr(p, "decoded_dtype", rc.CF32), rc.EUNSUPPORTED),
    (lambda p: setattr(p, "fs", 0.0), rc.EINVAL),
    (lambda p: setattr(p, "c", -1.0), rc.EINVAL),
    (lambda p: setattr(p, "f_number", -0.5), rc.EINVAL),
    (lambda p: setattr(p, "tx_orientation", 3), rc.EINVAL),
    (lambda p: p.out_dims.__setitem__(1, 0), rc.EINVAL),
    (lambda p: (p.tile.__setitem__(0, 64), p.tile.__setitem__(1, 1), p.tile.__setitem__(2, 8)), rc.EINVAL),
    (lambda p: (p.tile.__setitem__(0, 48), p.tile.__setitem__(1, 1), p.tile.__setitem__(2, 21)), rc.EINVAL),
])
def test_plan_rejects_bad_params_on_host(lib, mutate, code):
    p = _good_params()
    mutate(p)
    h = ctypes.c_void_p()
    assert lib.rcbf_plan(ctypes.byref(p), ctypes.byref(h)) == code
    assert not h.value
    assert lib.rcbf_last_error()


def test_plan_rejects_non_pm1_matrix(lib):
    import numpy as np
    p = _good_params()
    m = np.ones((32, 32), dtype=np.int8)
    m[3, 4] = 0
    p.decode_matrix = m.ctypes.data
    h = ctypes.c_void_p()
    assert lib.rcbf_plan(ctypes.byref(p), ctypes.byref(h)) == rc.EINVAL
    assert b"+1 or -1" in lib.rcbf_last_error()


def test_null_arguments_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.rcbf_plan(None, ctypes.byref(h)) == rc.EINVAL
    assert lib.rcbf_plan(ctypes.byref(_good_params()), None) == rc.EINVAL
    assert lib.rcbf_decode(None, None, None, None) == rc.EINVAL
    assert lib.rcbf_das(None, None, None, ctypes.c_float(0), None, None) == rc.EINVAL
    assert lib.rcbf_das_backward(None, None, None, ctypes.c_float(0), None, None, None, None, None) == rc.EINVAL
    assert lib.rcbf_batch_run(None, None) == rc.EINVAL
    assert lib.rcbf_plan_query(None, None) == rc.EINVAL
    assert lib.rcbf_batch_status(None, None) == rc.EINVAL
    assert lib.rcbf_batch_set_wait(None, 1000, -1) == rc.EINVAL
    h = ctypes.c_void_p()
    assert lib.rcbf_batch_create(None, 0, None, None, None, ctypes.byref(h)) == rc.EINVAL
    assert lib.rcbf_batch_create(None, 1, None, None, None, None) == rc.EINVAL
    lib.rcbf_destroy(None)
    lib.rcbf_batch_destroy(None)


def test_status_entry_points_reject_null(lib):
    assert lib.rcbf_plan_status(None, None) == rc.EINVAL
    assert lib.rcbf_plan_set_wait(None, 1000, 0) == rc.EINVAL


def test_noalloc_rejects_what_rcbf_das_rejects_before_any_cuda_call(lib):
    # the tiled form on a geometry that does not admit it (12 channels: not a
    # multiple of the 8-channel chunk) is RCBF_EUNSUPPORTED for both entry
    # points; the check runs on the host, so no device is needed here
    p = _good_params()
    p.n_ch = 12
    fake = ctypes.c_void_p(1 << 20)          # never dereferenced: rejected first
    assert lib.rcbf_das_noalloc(ctypes.byref(p), fake, None, ctypes.c_float(0), fake, None) == rc.EUNSUPPORTED
    assert b"tiled form" in lib.rcbf_last_error()
    p = _good_params()
    p.tx_wave = rc.TX_PLANE
    ang = (ctypes.c_double * p.n_tx)(*([0.0] * p.n_tx))
    p.tx_angles = ctypes.cast(ang, ctypes.c_void_p)
    assert lib.rcbf_das_noalloc(ctypes.byref(p), fake, None, ctypes.c_float(0), fake, None) == rc.EUNSUPPORTED


def test_version_string(lib):
    assert b"rcbf" in lib.rcbf_version()
