"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point include/bpm.h declares, and rejects invalid
arguments on the host before touching the device."""

import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "bpm.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(bpm_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert "sm_103a" in binding.bpm_version()


def _problem(**kw):
    e = np.array([8000.0])
    args = dict(nx=1024, nz=10, dx_um=0.4, dz_um=0.05, x0_um=-200.0, n_energy=1,
                energy_ev=e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                e_ref_ev=8000.0, theta_b_ref_rad=math.radians(23.65), chi0_re=-1.5e-5,
                chi0_im=3.5e-7, chih_re=-9.1e-6, chih_im=3.4e-7, record_every=0,
                precision=binding.BPM_FP32_FUSED)
    args.update(kw)
    return binding.bpm_problem(**args), e


@pytest.mark.parametrize("field,value,needle", [
    ("nx", 1000, "power of two"),
    ("nx", 4, "power of two"),
    ("nx", 1 << 20, "power of two"),
    ("nz", 0, "nz"),
    ("dz_um", 0.0, "dz_um"),
    ("dx_um", -1.0, "dx_um"),
    ("n_energy", 0, "n_energy"),
    ("theta_b_ref_rad", 2.0, "theta_b_ref_rad"),
    ("record_every", -1, "record_every"),
    ("precision", 7, "precision"),
    ("chi0_re", float("nan"), "finite"),
    ("dx_um", 1e-5, "evanescent"),
    ("dz_um", 100.0, "coupling expansion"),
])
def test_plan_rejects_invalid_problems_on_the_host(lib, field, value, needle):
    prob, keep = _problem(**{field: value})
    h = ctypes.c_void_p()
    rc = lib.bpm_plan(ctypes.byref(prob), ctypes.byref(h))
    assert rc == binding.BPM_ERR_INVALID
    assert needle in binding.bpm_last_error()
    assert h.value is None


def test_long_free_space_step_is_valid_without_a_crystal(lib):
    """A far-field step (chi = 0, dz of metres) passes validation; it is only
    the coupling expansion that bounds dz."""
    from paper_2601_06340_gb300 import inputs
    prob, keep = _problem(dz_um=2.0e6, chi0_re=0.0, chi0_im=0.0, chih_re=0.0, chih_im=0.0,
                          nz=1)
    # validation happens before any device work: without a GPU the call gets
    # past it and fails on the device (or succeeds on a GPU machine)
    h = ctypes.c_void_p()
    rc = lib.bpm_plan(ctypes.byref(prob), ctypes.byref(h))
    assert rc != binding.BPM_ERR_INVALID, binding.bpm_last_error()
    if h.value:
        lib.bpm_destroy(h)
    assert inputs.slit_field(256, -25.6, 0.2, 0.0, 5.0).shape == (1, 2, 256)


def test_null_arguments_are_rejected(lib):
    assert lib.bpm_plan(None, None) == binding.BPM_ERR_INVALID
    assert lib.bpm_set_crystal(None, 0, 0, 0, 0, 0, None, None, 0) == binding.BPM_ERR_INVALID
    assert lib.bpm_set_strain(None, 0, None, None, 0) == binding.BPM_ERR_INVALID
    assert lib.bpm_propagate(None, None, None, None, None, 0, 1) == binding.BPM_ERR_INVALID
    assert lib.bpm_destroy(None) == binding.BPM_ERR_INVALID
    assert lib.bpm_set_splitting(None, 1) == binding.BPM_ERR_INVALID
    assert lib.bpm_set_crystal_box(None, None) == binding.BPM_ERR_INVALID
    assert lib.bpm_launch_shape(None, None, None) == binding.BPM_ERR_INVALID
    assert lib.bpm_slice_form(None, None, None) == binding.BPM_ERR_INVALID
    assert lib.bpm_selftest_wait_expiry(None, None) == binding.BPM_ERR_INVALID
    assert lib.bpm_device_status(None, None) == binding.BPM_ERR_INVALID
    assert lib.bpm_server_inject_launch_failure(1000, 1) == binding.BPM_ERR_INVALID
    assert lib.bpm_server_inject_launch_failure(1 << 15, 1) == binding.BPM_ERR_INVALID
    assert lib.bpm_server_inject_launch_failure(1024, -1) == binding.BPM_ERR_INVALID
    assert lib.bpm_server_inject_launch_failure(1024, 0) == binding.BPM_OK
    assert lib.bpm_poll(ctypes.c_uint64(12345), 0) == binding.BPM_ERR_INVALID
    assert "ticket" in binding.bpm_last_error()


def test_omega_to_t_argument_checks(lib):
    assert lib.bpm_omega_to_t_device(None, None, 256, 64, 1, None) == binding.BPM_ERR_INVALID
    dummy = ctypes.c_void_p(16)
    assert lib.bpm_omega_to_t_device(dummy, dummy, 300, 64, 1, None) == binding.BPM_ERR_INVALID
    assert "power of two" in binding.bpm_last_error()


def test_last_error_is_thread_local(lib):
    import threading
    lib.bpm_destroy(None)
    seen = {}

    def other():
        seen["msg"] = binding.bpm_last_error()
    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["msg"] == ""
    assert binding.bpm_last_error() != ""


def test_workloads_are_seeded_and_shaped():
    a = inputs.asym_dislocation(nx=256, nz=100)
    b = inputs.asym_dislocation(nx=256, nz=100)
    assert np.array_equal(a.crystal["polygon"], b.crystal["polygon"])
    assert 5 <= a.meta["nv"] <= 8 and 50 <= a.meta["extent_um"] <= 300
    p = inputs.pulse_batched(nx=64, nz=10, n_energy=16)
    assert p.psi0.shape == (16, 2, 64) and np.all(np.diff(p.energies_ev) > 0)
    assert abs(p.energies_ev[0] - 8995.0) < 1e-9
    reqs = inputs.serving_requests(20)
    assert all(r2.arrival_s > r1.arrival_s for r1, r2 in zip(reqs, reqs[1:]))
    assert {r.workload.nx for r in inputs.serving_requests(200)} <= {
        512, 1024, 2048, 4096, 8192, 16384}


def test_fp_peak_argument_checks(lib):
    rate, sec = ctypes.c_double(), ctypes.c_double()
    assert lib.bpm_fp_peak(1, 100, None, ctypes.byref(sec)) == binding.BPM_ERR_INVALID
    assert lib.bpm_fp_peak(3, 100, ctypes.byref(rate), ctypes.byref(sec)) == binding.BPM_ERR_INVALID
    assert lib.bpm_fp_peak(1, 0, ctypes.byref(rate), ctypes.byref(sec)) == binding.BPM_ERR_INVALID
