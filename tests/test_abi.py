"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point that include/dfp2s.h declares; pure host logic agrees
with the oracle."""
import os
import re
import subprocess

import pytest

import paper_2210_06713_gb300 as dfp2s
from oracle import sampler

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dfp2s_\w+)\s*\(", txt))
    return names


def test_library_loads_and_exports_every_declared_symbol():
    lib = dfp2s.load()
    declared = _declared()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", dfp2s.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dfp2s_\w+)", out))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(lib, name)
    # the binding wraps every declared entry point
    assert declared <= set(dfp2s.SIGNATURES)


def test_version_and_grid_size_match_oracle():
    assert b"sm_103a" in dfp2s.load().dfp2s_version()
    for (H, W, ppd) in [(64, 64, 8.0), (256, 256, 8.0), (512, 512, 8.0), (2160, 3840, 8.0), (768, 768, 8.0),
                        (1024, 1024, 8.0), (50, 37, 2.0), (100, 3, 4.5)]:
        assert dfp2s.grid_size(H, W, ppd) == sampler.grid_size(H, W, ppd)


def test_grid_size_rejects_bad_arguments():
    with pytest.raises(dfp2s.DFP2SError) as e:
        dfp2s.grid_size(0, 10, 8.0)
    assert e.value.code == -1
    with pytest.raises(dfp2s.DFP2SError):
        dfp2s.grid_size(4090, 4090, 8.0)  # grid would exceed 4096
    with pytest.raises(dfp2s.DFP2SError):
        dfp2s.grid_size(64, 64, -1.0)


def test_null_handles_are_rejected_without_a_gpu():
    lib = dfp2s.load()
    import ctypes
    assert lib.dfp2s_sample_zernike_fields(None, 1.0, 0, 0, 8, 8, None, None) == -1
    assert lib.dfp2s_p2s_weights(None, 0, None, 8, 8, None, 0, None) == -1
    assert lib.dfp2s_tilt_warp(None, 1, 8, 8, None, None, None, None) == -1
    assert lib.dfp2s_simulate_frame(None, None, 1, 8, 8, 1.0, 0, 0, 0, None, None) == -1
    buf = ctypes.create_string_buffer(256)
    assert lib.dfp2s_last_error(buf, 256) == -1
    assert b"null" in buf.value


def test_new_entry_points_validate_arguments_without_a_gpu():
    lib = dfp2s.load()
    import ctypes
    lags = (ctypes.c_int * 2)(0, 0)
    # field statistics: null pointers, J out of range, a lag that does not fit
    assert lib.dfp2s_field_covariance(None, 4, 8, 8, lags, 1, None, None) == -1
    dummy = ctypes.c_void_p(16)
    assert lib.dfp2s_field_covariance(dummy, 0, 8, 8, lags, 1, dummy, None) == -1
    assert lib.dfp2s_field_covariance(dummy, 65, 8, 8, lags, 1, dummy, None) == -1
    assert lib.dfp2s_field_covariance(dummy, 4, 8, 8, lags, 0, dummy, None) == -1
    far = (ctypes.c_int * 2)(8, 0)
    assert lib.dfp2s_field_covariance(dummy, 4, 8, 8, far, 1, dummy, None) == -1
    # network files and frame stage timing: null handles
    assert lib.dfp2s_mlp_save(None, b"/nonexistent/x") == -1
    assert lib.dfp2s_mlp_load(None, b"/nonexistent/x") == -1
    assert lib.dfp2s_ctx_stage_timing(None, 4) == -1
    out = (ctypes.c_float * 4)()
    assert lib.dfp2s_ctx_stage_times(None, 1, out) == -1
