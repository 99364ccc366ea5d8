"""Rocking-curve scan: incidence angles as the rows of one batched launch.

Every row is the same photon energy with its own tilted incident beam; the
reflectivity of a row is its final psi_- power over its incident psi_+
power (FP64 band sums).  Compared with the FP64 oracle row by row.
"""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP32, TOL_FP64, band_errors, run_gpu, run_ref

pytestmark = pytest.mark.gpu

FP32, FP64 = binding.BPM_FP32_FUSED, binding.BPM_FP64_PLAIN


def _reflectivity(wl, powers, rows=None):
    psi0 = wl.psi0 if rows is None else wl.psi0[rows]
    p_in = wl.dx_um * np.sum(np.abs(psi0[:, 0]) ** 2, axis=-1)
    return powers[:, -1, 1] / p_in


def test_rocking_scan_every_row(bpm_lib):
    wl = inputs.rocking_scan(nx=512, nz=600, n_angles=16, fwhm_um=60.0)
    ref = run_ref(wl)
    r_ref = _reflectivity(wl, ref.powers)
    assert r_ref.max() > 0.05          # the scan crosses the reflection
    for prec, tol in ((FP64, TOL_FP64), (FP32, TOL_FP32)):
        out = run_gpu(wl, prec)
        assert max(band_errors(out.psi, ref.psi)) <= tol, prec
        r = _reflectivity(wl, out.powers)
        assert np.max(np.abs(r - r_ref)) <= 2 * tol * r_ref.max(), (prec, r, r_ref)


def test_rocking_scan_full_size_sampled_rows(bpm_lib):
    """256 angles x Nx=2048 x Nz=2000 in one FP32 batch; the oracle checks
    three rows (the curve's centre and two flanks)."""
    wl = inputs.rocking_scan()
    out = run_gpu(wl, FP32)
    rows = [0, 128, 140]
    ref = run_ref(wl, rows=rows)
    assert max(band_errors(out.psi[rows], ref.psi)) <= TOL_FP32
    r = _reflectivity(wl, out.powers)
    r_ref = _reflectivity(wl, ref.powers, rows)
    assert np.max(np.abs(r[rows] - r_ref)) <= 2 * TOL_FP32 * r.max()
    # symmetric Laue, perfect crystal: the reflectivity is even in the
    # angle offset (rows b and 256 - b are +-dtheta) and peaks near zero
    angles = wl.meta["angles_urad"]
    b = np.arange(1, 256)
    assert np.allclose(angles[b], -angles[256 - b])
    assert np.max(np.abs(r[b] - r[256 - b])) <= 1e-3 * r.max()
    assert abs(angles[int(np.argmax(r))]) <= 6.0
