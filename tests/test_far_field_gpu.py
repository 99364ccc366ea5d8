"""Far field: one free-space step of metres behind the crystal (Secs. 5-6
take far-field images 2-4 m from the crystal), on both GPU paths against the
oracle, for a crystal's exit field and for a slit-shaped beam."""

import numpy as np
import pytest

from oracle import run as orun
from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP32, TOL_FP64, band_errors, run_gpu, run_ref

pytestmark = pytest.mark.gpu

FP32, FP64 = binding.BPM_FP32_FUSED, binding.BPM_FP64_PLAIN


def test_far_field_of_a_laue_exit_field(bpm_lib):
    wl = inputs.laue_perfect(nx=1024, nz=600, record_every=0)
    exit_field = run_ref(wl).psi
    ff = inputs.far_field_step(exit_field, wl.nx, wl.dx_um, wl.x0_um, 2.0e6)
    ref = run_ref(ff)
    for prec, tol in ((FP64, TOL_FP64), (FP32, TOL_FP32)):
        out = run_gpu(ff, prec)
        assert max(band_errors(out.psi, ref.psi)) <= tol, prec
    # free space: each band keeps its power
    p0 = wl.dx_um * np.sum(np.abs(exit_field) ** 2, axis=-1)
    assert np.allclose(ref.powers[:, -1], p0, rtol=1e-12)


def test_far_field_of_a_slit(bpm_lib):
    """A 5 um slit (section topography) seen 4 m away: GPU = oracle, and the
    central lobe spreads to the Fraunhofer width lambda L / w."""
    nx, dx = 4096, 0.1
    x0 = -0.5 * nx * dx
    slit = inputs.slit_field(nx, x0, dx, 0.0, 5.0)
    ff = inputs.far_field_step(slit, nx, dx, x0, 4.0e6)
    ref = run_ref(ff)
    for prec, tol in ((FP64, TOL_FP64), (FP32, TOL_FP32)):
        out = run_gpu(ff, prec)
        assert max(band_errors(out.psi, ref.psi)) <= tol, prec
    inten = np.abs(ref.psi[0, 0]) ** 2
    lam = 12398.419843320026 / inputs.E_REF_EV * 1e-4
    # first zeros of the sinc^2 lobe are lambda L / w apart (along the beam,
    # projected on x by 1 / cos(theta_B)); measure the lobe's width at 1/2
    peak = int(np.argmax(inten))
    above = np.where(np.roll(inten, nx // 2 - peak) >= 0.5 * inten.max())[0]
    fwhm_um = (above.max() - above.min() + 1) * dx
    fraunhofer_fwhm = 0.886 * lam * 4.0e6 / 5.0
    assert 0.5 * fraunhofer_fwhm < fwhm_um < 2.0 * fraunhofer_fwhm
