"""C-ABI checks that need no GPU: the library loads, exports every call the
header declares, answers pure-host queries, and rejects invalid arguments
with a status instead of crashing."""
import os
import re

import numpy as np
import pytest

from oracle.lattice import D2Q9, D3Q19
from tests.conftest import gpu_available

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ibl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibl_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_core_calls():
    names = _declared()
    for must in ["ibl_create", "ibl_set_markers", "ibl_set_kinematics", "ibl_step", "ibl_forces",
                 "ibl_destroy", "ibl_get_field", "ibl_force_history", "ibl_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(ibl):
    import ctypes
    lib = ctypes.CDLL(ibl.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(ibl.exported_symbols())


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_lattice_velocities_match_oracle_sets(ibl, lat):
    c, w = ibl.lattice_velocities(lat.Q)
    mine = {tuple(v): wi for v, wi in zip(c.tolist(), w)}
    ref = {tuple(v): wi for v, wi in zip(lat.c.tolist(), lat.w)}
    assert mine.keys() == ref.keys()
    for k in ref:
        assert mine[k] == ref[k]


def test_invalid_arguments_are_statuses(ibl):
    g = {"nx": 8, "ny": 8, "nz": 2, "bc": [0] * 6}
    with pytest.raises(ibl.IblError) as e:
        ibl.Context(g, 0.8, 9)                  # D2Q9 with nz != 1
    assert e.value.status == ibl.IBL_EINVAL
    with pytest.raises(ibl.IblError) as e:
        ibl.Context({"nx": 8, "ny": 8, "nz": 1, "bc": [0] * 6}, 0.5, 9)   # tau <= 1/2
    assert e.value.status == ibl.IBL_EINVAL
    with pytest.raises(ibl.IblError) as e:
        ibl.Context({"nx": 8, "ny": 8, "nz": 8, "bc": [0, 1, 0, 0, 0, 0]}, 0.8, 19)  # unpaired periodic
    assert e.value.status == ibl.IBL_EINVAL
    with pytest.raises(ibl.IblError) as e:
        ibl.Context({"nx": 8, "ny": 8, "nz": 8, "bc": [2, 3, 1, 1, 0, 0]}, 0.8, 19)  # Zou-He + wall corner
    assert e.value.status == ibl.IBL_EINVAL


@pytest.mark.skipif(gpu_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error(ibl):
    with pytest.raises(ibl.IblError) as e:
        ibl.Context({"nx": 8, "ny": 8, "nz": 8, "bc": [0] * 6}, 0.8, 19)
    assert e.value.status in (ibl.IBL_ECUDA, ibl.IBL_ENOMEM)


def test_null_context_calls_are_einval(ibl):
    """Every call that takes a context answers NULL with IBL_EINVAL (no GPU
    needed: the check comes before any device work)."""
    import ctypes as C
    lib = C.CDLL(ibl.LIB_PATH)
    d = C.c_double()
    i32 = C.c_int32()
    calls = [
        lambda: lib.ibl_step(None, C.c_int64(1)),
        lambda: lib.ibl_sync(None),
        lambda: lib.ibl_set_overlap(None, C.c_int32(1)),
        lambda: lib.ibl_solver_blocks(None, C.c_int32(8)),
        lambda: lib.ibl_solver_config(None, C.c_int32(64), C.c_double(0.0), C.c_int32(1)),
        lambda: lib.ibl_profile(None, C.c_int32(1)),
        lambda: lib.ibl_profile_phases(None, C.byref(d), C.c_int32(1)),
        lambda: lib.ibl_mass(None, C.byref(d)),
        lambda: lib.ibl_mass_noalloc(None, C.c_int32(16), C.byref(d)),
        lambda: lib.ibl_interpolate_points(None, C.c_int32(1), None, None, None),
        lambda: lib.ibl_spread_points(None, C.c_int32(1), None, None, None, None),
        lambda: lib.ibl_forces(None, C.c_int32(0), C.byref(d), C.byref(d), C.byref(d)),
        lambda: lib.ibl_solver_stats(None, C.byref(i32), C.byref(d), None),
    ]
    for call in calls:
        assert call() == ibl.IBL_EINVAL
