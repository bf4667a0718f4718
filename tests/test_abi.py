"""The C-ABI library loads and exports every entry point of include/sn.h (CPU only).

No compute call is made here: without a GPU only argument validation (which
returns before any CUDA call) can run.
"""
import ctypes
import os
import re

import pytest

from paper_1909_08354_b300 import sn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sn_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sn_create_grid", "sn_set_kernel", "sn_set_state", "sn_get_state", "sn_step",
                     "sn_observables", "sn_destroy_grid", "sn_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(sn.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    wrapped = {name for name, _, _ in sn._SIGNATURES}
    assert set(declared_functions()) <= wrapped


@pytest.mark.parametrize("n,L", [((8, 12), (1.0, 1.0)), ((4, 8), (1.0, 1.0)),
                                 ((8, 8, 8, 8), (1.0,) * 4), ((16, 16), (1.0, -1.0)),
                                 ((16, 16), (1.0, float("nan"))), ((8,), (1.0,))])
def test_invalid_grids_are_rejected_before_any_cuda_call(n, L):
    with pytest.raises(sn.SNError) as e:
        sn.sn_create_grid(n, L)
    assert e.value.status == sn.SN_EINVAL
    assert "sn_create_grid" in sn.sn_last_error(None)


def test_oversized_axis_is_not_supported():
    with pytest.raises(sn.SNError) as e:
        sn.sn_create_grid((2048, 8), (1.0, 1.0))
    assert e.value.status == sn.SN_ENOTSUP


def test_null_handles_are_rejected():
    L = sn.lib()
    assert L.sn_step(None, 0.1, 1) == sn.SN_EINVAL
    assert L.sn_set_state(None, None, 0) == sn.SN_EINVAL
    assert L.sn_set_fluid(None, None) == sn.SN_EINVAL
    assert L.sn_set_fields(None, 2) == sn.SN_EINVAL
    assert L.sn_get_fields(None) == 0
    assert L.sn_observables(None, None) == sn.SN_EINVAL
    assert L.sn_launch_count(None) == 0
    L.sn_destroy_grid(None)
    assert sn.sn_kind_names()[0] == "psi_pass"


def test_binding_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "sn.h")).read()
    assert int(re.search(r"#define SN_MAX_FIELDS (\d+)", text).group(1)) == sn.SN_MAX_FIELDS


def test_schedule_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "sn.h")).read()
    assert int(re.search(r"#define SN_SCHED_KINDS (\d+)", text).group(1)) == sn.SN_SCHED_KINDS
    assert int(re.search(r"#define SN_SCHED_MAX_CTAS (\d+)", text).group(1)) == sn.SN_SCHED_MAX_CTAS
    m = re.search(r"#define SN_SCHED_VALUES \((\d+) \* SN_SCHED_KINDS\)", text)
    assert int(m.group(1)) * sn.SN_SCHED_KINDS == sn.SN_SCHED_VALUES
    m = re.search(r"SN_STAGING_TMA = (\d+), SN_STAGING_REGISTERS = (\d+), SN_STAGING_RESIDENT = (\d+)", text)
    assert tuple(map(int, m.groups())) == (sn.SN_STAGING_TMA, sn.SN_STAGING_REGISTERS, sn.SN_STAGING_RESIDENT)
    # the schedule kinds are the first kernel kinds, in order
    assert sn.sn_kind_names()[:sn.SN_SCHED_KINDS] == ["psi_pass", "psi_pass_nphase",
                                                      "psi_pass_density", "rho_fwd", "rho_green",
                                                      "rho_inv"]


def test_schedule_calls_reject_null_grids():
    L = sn.lib()
    buf = (ctypes.c_int * 18)()
    assert L.sn_get_schedule(None, buf, 18) == sn.SN_EINVAL
    assert L.sn_set_schedule(None, buf, 18) == sn.SN_EINVAL
    assert L.sn_autotune(None, 0.01, 1) == sn.SN_EINVAL


def test_schedule_cache_round_trip(tmp_path):
    path = str(tmp_path / "sched.json")
    k1 = sn.schedule_key("B300", (256, 256, 256), sn.SN_ENGINE_FP32, 1)
    k2 = sn.schedule_key("B300", (256, 256, 256), sn.SN_ENGINE_FP32, 2)
    assert k1 != k2 and "256x256x256" in k1
    assert sn.load_schedule(path, k1) is None  # no file yet
    v1 = [0, 1, 2] * 6 + [-1, 0, 1] * 6
    sn.store_schedule(path, k1, v1)
    sn.store_schedule(path, k2, [-1] * sn.SN_SCHED_VALUES)
    assert sn.load_schedule(path, k1) == v1
    assert sn.load_schedule(path, k2) == [-1] * sn.SN_SCHED_VALUES
    # malformed entries and files are ignored, not trusted
    sn.store_schedule(path, k1, [0] * (sn.SN_SCHED_VALUES - 1))
    assert sn.load_schedule(path, k1) is None
    sn.store_schedule(path, k1, [0] * 18)  # a schedule without its staging part
    assert sn.load_schedule(path, k1) is None
    sn.store_schedule(path, k1, [99] * 18 + [0] * 18)
    assert sn.load_schedule(path, k1) is None
    sn.store_schedule(path, k1, [0] * 18 + [2] * 18)  # no staging mode 2
    assert sn.load_schedule(path, k1) is None
    with open(path, "w") as f:
        f.write("not json")
    assert sn.load_schedule(path, k2) is None
    sn.store_schedule(path, k2, v1)  # a broken file is replaced
    assert sn.load_schedule(path, k2) == v1


def test_later_calls_reject_bad_arguments_before_any_cuda_call():
    """The grid options, the batch's register budget and tuner, the fused FNO
    layer form and the measurement hooks check their arguments first."""
    L = sn.lib()
    assert L.sn_set_staging(None, 0) == sn.SN_EINVAL
    assert L.sn_set_blocking(None, 4) == sn.SN_EINVAL
    assert L.sn_set_obs_mode(None, sn.SN_OBS_FP32) == sn.SN_EINVAL
    assert L.sn_set_batch_ctas(None, 2) == sn.SN_EINVAL
    assert L.sn_set_batch_schedule(None, sn.SN_BATCH_GRAPH) == sn.SN_EINVAL
    assert L.sn_get_batch_schedule(None) == -1
    dt = (ctypes.c_double * 1)(0.01)
    assert L.sn_autotune_batch(None, dt, 5, None) == sn.SN_EINVAL
    assert L.sn_fno_set_layer_form(None, sn.SN_FNO_LAYER_UMMA) == sn.SN_EINVAL
    ms = ctypes.c_double(0.0)
    # NULL data, a bad length, a bad sign, the tcgen05 engine off 256 points, reps < 1
    assert L.sn_test_line_fft_engines(None, 8, 256, -1, sn.SN_ENGINE_FP32, 1, ctypes.byref(ms), None) == sn.SN_EINVAL
    dummy = ctypes.c_void_p(16)
    assert L.sn_test_line_fft_engines(dummy, 8, 100, -1, sn.SN_ENGINE_FP32, 1, ctypes.byref(ms), None) == sn.SN_EINVAL
    assert L.sn_test_line_fft_engines(dummy, 8, 256, 2, sn.SN_ENGINE_FP32, 1, ctypes.byref(ms), None) == sn.SN_EINVAL
    assert L.sn_test_line_fft_engines(dummy, 8, 128, -1, sn.SN_ENGINE_UMMA, 1, ctypes.byref(ms), None) == sn.SN_EINVAL
    assert L.sn_test_line_fft_engines(dummy, 8, 256, -1, sn.SN_ENGINE_UMMA, 0, ctypes.byref(ms), None) == sn.SN_EINVAL
    rates = (ctypes.c_double * 3)()
    for bad in (1, 3, 16):
        assert L.sn_test_dsmem_rates(bad, rates) == sn.SN_EINVAL
    assert L.sn_test_dsmem_rates(4, None) == sn.SN_EINVAL
    cyc = (ctypes.c_double * 5)()
    tiles = ctypes.c_longlong(0)
    assert L.sn_test_umma_phases(None, 8, -1, cyc, ctypes.byref(tiles), None) == sn.SN_EINVAL
    assert L.sn_test_umma_phases(dummy, 0, -1, cyc, ctypes.byref(tiles), None) == sn.SN_EINVAL
    assert L.sn_test_umma_phases(dummy, 8, 3, cyc, ctypes.byref(tiles), None) == sn.SN_EINVAL
    assert L.sn_test_umma_phases(dummy, 8, -1, None, ctypes.byref(tiles), None) == sn.SN_EINVAL


def test_new_header_enums_match_the_binding():
    text = open(os.path.join(ROOT, "include", "sn.h")).read()
    m = re.search(r"SN_OBS_FP64 = (\d+), SN_OBS_FP32 = (\d+)", text)
    assert tuple(map(int, m.groups())) == (sn.SN_OBS_FP64, sn.SN_OBS_FP32)
    m = re.search(r"SN_FNO_LAYER_GEMMS = (\d+), SN_FNO_LAYER_UMMA = (\d+)", text)
    assert tuple(map(int, m.groups())) == (sn.SN_FNO_LAYER_GEMMS, sn.SN_FNO_LAYER_UMMA)
    m = re.search(r"SN_BATCH_PERSISTENT = (\d+),\s*/\*[^*]*\*/\s*SN_BATCH_GRAPH = (\d+),"
                  r"\s*/\*[^*]*\*/\s*SN_BATCH_CLASSES = (\d+)", text)
    assert tuple(map(int, m.groups())) == (sn.SN_BATCH_PERSISTENT, sn.SN_BATCH_GRAPH,
                                           sn.SN_BATCH_CLASSES)
    m = re.search(r"SN_ENGINE_FP32 = (\d+), SN_ENGINE_TC16 = (\d+), SN_ENGINE_UMMA = (\d+)", text)
    assert tuple(map(int, m.groups())) == (sn.SN_ENGINE_FP32, sn.SN_ENGINE_TC16, sn.SN_ENGINE_UMMA)
