"""Repeat runs are bitwise equal on every kernel family.

A data race inside a kernel (a shared-memory slot read before its writer is
done with it, a peer's exchange buffer overwritten early, a slice copy that
lands late) shows up as run-to-run differences.  Every case here marches
twice on the same plan and input and compares the exit fields, the records
and the band powers bit for bit: the one-CTA kernels at N = 64 and N = 512
(a batch larger than one launch, so rotated), the second-order form of the
band-per-thread kernel, the 2-CTA cluster (N = 1024), the split-band cluster
kernels (N = 4096, 8192, 16384), the plain FP64 path and the 3D march."""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

FP32, FP64 = binding.BPM_FP32_FUSED, binding.BPM_FP64_PLAIN


def _serving(nx, nz=300, seed=3):
    return inputs.serving_request(np.random.default_rng(seed), nx, nz)


CASES = {
    "fused N=64": (lambda: _serving(64), FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "fused2 N=512 batch of 200": (lambda: inputs.rocking_scan(nx=512, nz=300, n_angles=200),
                                  FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "Verlet N=4096 (half-band split)": (lambda: _serving(4096), FP32, binding.BPM_SPLIT_VERLET),
    "Verlet batch of 200 (one CTA per row)": (lambda: inputs.rocking_scan(nx=512, nz=300, n_angles=200),
                                              FP32, binding.BPM_SPLIT_VERLET),
    "fused3 N=1024": (lambda: _serving(1024), FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "fused4e N=4096": (lambda: _serving(4096), FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "fused4e N=8192": (lambda: _serving(8192), FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "fused4t N=16384": (lambda: _serving(16384), FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "plain FP64 N=1024": (lambda: _serving(1024), FP64, binding.BPM_SPLIT_FIRST_ORDER),
    "3D 256x256": (lambda: inputs.cube_dislocation_3d(nx=256, ny=256, nz=40, dx_um=0.08,
                                                      dy_um=0.08, dz_um=0.1, cube_um=5.0,
                                                      fwhm_um=1.5, record_every=10),
                   FP32, binding.BPM_SPLIT_FIRST_ORDER),
    "3D 256x256 Verlet": (lambda: inputs.cube_dislocation_3d(nx=256, ny=256, nz=40, dx_um=0.08,
                                                             dy_um=0.08, dz_um=0.1, cube_um=5.0,
                                                             fwhm_um=1.5, record_every=10),
                          FP32, binding.BPM_SPLIT_VERLET),
}


@pytest.mark.parametrize("name", list(CASES))
def test_repeat_runs_are_bitwise_equal(bpm_lib, name):
    make, precision, split = CASES[name]
    wl = make()
    with binding.Plan(wl, precision, splitting=split) as plan:
        first = plan.propagate()
        second = plan.propagate()
    assert np.array_equal(first.psi, second.psi)
    assert np.array_equal(first.records, second.records)
    assert np.array_equal(first.powers, second.powers)
    assert np.isfinite(first.psi).all() and np.abs(first.psi).max() > 0
