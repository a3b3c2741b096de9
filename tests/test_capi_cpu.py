"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that include/storm.h declares, and rejects bad arguments
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2104_13542_b300 import binding
from paper_2104_13542_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(storm_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    binding.build()
    return binding.lib()


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= set(binding.EXPORTED) | set(), declared - set(binding.EXPORTED)
    for name in declared:
        assert hasattr(L, name), f"{name} not exported"


def test_status_strings(L):
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert binding.status_string(code)
    assert binding.status_string(99) == "unknown status"


def _structs(wl):
    m = binding._Marshal()
    return m, m.robot(wl.robot), m.world(wl.world), m.params(wl.params)


@pytest.mark.parametrize("mutate", [
    lambda r, w, p: setattr(r, "dof", 0),
    lambda r, w, p: setattr(r, "dof", 8),
    lambda r, w, p: setattr(p, "N", 0),
    lambda r, w, p: setattr(p, "N", 16385),
    lambda r, w, p: setattr(p, "H", 65),
    lambda r, w, p: setattr(p, "K", 0),
    lambda r, w, p: setattr(p, "n_knots", 3),
    lambda r, w, p: setattr(p, "sampler", 7),
    lambda r, w, p: setattr(p, "n_null", -1),
    lambda r, w, p: setattr(p, "beta", -1.0),
    lambda r, w, p: setattr(p, "instance", 1 << 24),
    lambda r, w, p: setattr(r, "n_spheres", 65),
    lambda r, w, p: setattr(r, "n_pairs", 2049),
    lambda r, w, p: setattr(w, "n_boxes", 65),
    lambda r, w, p: setattr(p, "dt", None),
    lambda r, w, p: setattr(p, "filter", 7),
    lambda r, w, p: (setattr(p, "filter", 2), setattr(p, "n_knots", 0)),
    lambda r, w, p: setattr(p, "mix_bspline", 1.5),
    lambda r, w, p: setattr(p, "w_ee_vel", -1.0),
    lambda r, w, p: setattr(p, "ee_acc_max", float("nan")),
    lambda r, w, p: setattr(p, "w_ball", float("inf")),
    lambda r, w, p: (setattr(p, "grad_steps", 2), setattr(p, "filter", 1)),
    lambda r, w, p: (setattr(p, "grad_steps", 2), setattr(p, "w_ball", 1.0)),
])
def test_create_rejects_bad_arguments(L, mutate):
    wl = W.config_paper(0, N=8, H=10)
    keep, r, w, p = _structs(wl)
    mutate(r, w, p)
    h = C.c_void_p(123)
    rc = L.storm_create(C.byref(r), C.byref(w), C.byref(p), None, C.byref(h))
    assert rc == binding.STORM_ERR_INVALID_ARG
    assert h.value is None


def test_create_rejects_bad_indices(L):
    wl = W.config_paper(0, N=8, H=10)
    wl.robot.pairs = wl.robot.pairs.copy()
    wl.robot.pairs[3, 1] = 49  # one past the last sphere
    keep, r, w, p = _structs(wl)
    h = C.c_void_p()
    assert L.storm_create(C.byref(r), C.byref(w), C.byref(p), None, C.byref(h)) == -1
    wl = W.config_paper(0, N=8, H=10)
    wl.robot.sphere_link = wl.robot.sphere_link.copy()
    wl.robot.sphere_link[0] = 8
    keep, r, w, p = _structs(wl)
    assert L.storm_create(C.byref(r), C.byref(w), C.byref(p), None, C.byref(h)) == -1
    wl = W.config_paper(0, N=8, H=10)
    wl.world.boxes = wl.world.boxes.copy()
    wl.world.boxes[0, 0] = np.nan
    keep, r, w, p = _structs(wl)
    assert L.storm_create(C.byref(r), C.byref(w), C.byref(p), None, C.byref(h)) == -1


def test_null_handle_calls_fail_cleanly(L):
    assert L.storm_reset(None) == -1
    assert L.storm_sync(None, None) == -1
    assert L.storm_shift(None) == -1
    assert L.storm_step(None, None, None, None, None) == -1
    assert L.storm_create(None, None, None, None, None) == -1
    L.storm_destroy(None)
    assert L.storm_last_error(None) == b"NULL handle"


def test_oracle_and_library_share_nothing():
    """The oracle and the CUDA path have separate sources and headers."""
    cu = open(os.path.join(ROOT, "paper_2104_13542_b300", "csrc", "storm.cu")).read()
    cuh = open(os.path.join(ROOT, "paper_2104_13542_b300", "csrc", "storm_device.cuh")).read()
    for src in (cu, cuh):
        assert "storm_oracle" not in src and "orc_" not in src
    orc = open(os.path.join(ROOT, "oracle", "storm_oracle.c")).read()
    assert "storm.h" not in orc and "storm_device" not in orc
    for py in ("binding.py", "__init__.py", "workloads.py"):
        src = open(os.path.join(ROOT, "paper_2104_13542_b300", py)).read()
        assert "import oracle" not in src and "from oracle" not in src


def test_batch_rejects_ball_term(L):
    wls = [W.config_paper(0, N=8, H=10), W.config_ball(1, N=8, H=10)]
    m = binding._Marshal()
    R = (binding.storm_robot * 2)(*[m.robot(w.robot) for w in wls])
    Wd = (binding.storm_world * 2)(*[m.world(w.world) for w in wls])
    P = (binding.storm_params * 2)(*[m.params(w.params) for w in wls])
    h = C.c_void_p()
    L.storm_batch_create.argtypes = [C.c_int, C.POINTER(binding.storm_robot),
                                     C.POINTER(binding.storm_world), C.POINTER(binding.storm_params),
                                     C.c_void_p, C.POINTER(C.c_void_p)]
    assert L.storm_batch_create(2, R, Wd, P, None, C.byref(h)) == binding.STORM_ERR_INVALID_ARG
    assert h.value is None


def test_batch_create_rejects_bad_instance(L):
    wls = [W.config_paper(0, N=8, H=10), W.config_paper(1, N=8, H=10)]
    m = binding._Marshal()
    wls[1].params = wls[1].params.replace(K=0)
    R = (binding.storm_robot * 2)(*[m.robot(w.robot) for w in wls])
    Wd = (binding.storm_world * 2)(*[m.world(w.world) for w in wls])
    P = (binding.storm_params * 2)(*[m.params(w.params) for w in wls])
    h = C.c_void_p()
    L.storm_batch_create.argtypes = [C.c_int, C.POINTER(binding.storm_robot),
                                     C.POINTER(binding.storm_world), C.POINTER(binding.storm_params),
                                     C.c_void_p, C.POINTER(C.c_void_p)]
    assert L.storm_batch_create(2, R, Wd, P, None, C.byref(h)) == binding.STORM_ERR_INVALID_ARG
    assert L.storm_batch_create(0, R, Wd, P, None, C.byref(h)) == binding.STORM_ERR_INVALID_ARG
    assert h.value is None
