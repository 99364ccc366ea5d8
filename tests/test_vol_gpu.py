"""3D march (both transverse coordinates) on the GPU against the 3D oracle."""

import numpy as np
import pytest

from oracle import run as orun
from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP32

pytestmark = pytest.mark.gpu

FP32 = binding.BPM_FP32_FUSED


def _rel(got, ref):
    """max over bands of the relative L2 error (fields and records)."""
    out = 0.0
    for b in range(2):
        den = np.linalg.norm(ref[:, b])
        if den > 0:
            out = max(out, np.linalg.norm(got[:, b] - ref[:, b]) / den)
    return out


def _small(nx=256, ny=256, nz=80, record_every=20):
    return inputs.cube_dislocation_3d(nx=nx, ny=ny, nz=nz, dx_um=0.08, dy_um=0.08,
                                      dz_um=0.1, cube_um=5.0, fwhm_um=1.5,
                                      record_every=record_every)


def test_vol_small_fields_records_powers(bpm_lib):
    wl = _small()
    ref = orun.run_workload3d(wl)
    with binding.Plan(wl, FP32) as plan:
        out = plan.propagate()
    assert _rel(out.psi, ref.psi) <= TOL_FP32
    for r in range(ref.records.shape[1]):
        assert _rel(out.records[:, r], ref.records[:, r]) <= TOL_FP32, r
    assert np.allclose(out.powers, ref.powers, rtol=2 * TOL_FP32, atol=1e-12 * ref.powers.max())
    assert ref.powers[0, -1, 1] > 1e-3 * ref.powers[0, -1, 0]   # the box reflects


@pytest.mark.parametrize("shape", [(512, 256), (256, 512), (1024, 256), (256, 1024)])
def test_vol_sizes(bpm_lib, shape):
    nx, ny = shape
    wl = _small(nx=nx, ny=ny, nz=24, record_every=0)
    ref = orun.run_workload3d(wl)
    with binding.Plan(wl, FP32) as plan:
        out = plan.propagate(records=False)
    assert _rel(out.psi, ref.psi) <= TOL_FP32


def test_vol_mask_is_bit_exact_and_phasor_fp32(bpm_lib):
    wl = _small(nz=40, record_every=0)
    with binding.Plan(wl, FP32) as plan:
        mask, ph = plan.slices()
    from oracle import bpm, bpm3d
    cr = bpm3d.Crystal3D(wl.nx, wl.ny, wl.x0_um, wl.y0_um, wl.dx_um, wl.dy_um, wl.dz_um,
                         bpm.d_spacing_um(wl.e_ref_ev, wl.theta_b_ref_rad))
    cr.set_crystal(bpm3d.CRYSTAL_BOX, box=wl.crystal["box_um"])
    cr.set_strain(wl.strain["kind"], params=wl.strain["params"])
    for n in range(wl.nz):
        inside, theta = cr(n)
        assert np.array_equal(mask[n].astype(bool), inside), n
        ref = np.where(inside, np.exp(1j * theta), 0)
        assert np.max(np.abs(ph[n] - ref)) < 4e-6, n


def test_vol_resume_equals_whole_march(bpm_lib):
    wl = _small(nz=60, record_every=0)
    with binding.Plan(wl, FP32) as plan:
        whole = plan.propagate(records=False).psi.copy()
        half = plan.propagate(n_end=25, records=False).psi.copy()
        rest = plan.propagate(psi_in=half, n_begin=25, records=False).psi
    assert _rel(rest, whole) < 1e-6


def test_vol_full_size_against_oracle(bpm_lib):
    """512 x 256 x 300 cells (the 3D stand-in workload) in one march."""
    wl = inputs.cube_dislocation_3d()
    ref = orun.run_workload3d(wl)
    with binding.Plan(wl, FP32) as plan:
        out = plan.propagate(records=False)
    assert _rel(out.psi, ref.psi) <= TOL_FP32
    assert np.allclose(out.powers[:, -1], ref.powers[:, -1], rtol=2 * TOL_FP32)


def test_vol_rejects_bad_sizes_and_server(bpm_lib):
    wl = _small(nx=128, nz=4)
    with pytest.raises(binding.BpmError):
        binding.Plan(wl, FP32)
    wl = _small(nz=4)
    with pytest.raises(binding.BpmError):
        binding.Plan(wl, binding.BPM_FP64_PLAIN)
    with binding.Plan(wl, FP32) as plan:
        out = np.empty_like(wl.psi0)
        with pytest.raises(binding.BpmError):
            binding.bpm_submit(plan.handle, wl.psi0, out)


def test_vol_verlet_matches_oracle(bpm_lib):
    """Second-order (Verlet) splitting on the 3D path against the 3D
    oracle's Verlet march: fields, records, powers; a resumed march equals
    the whole one; and the scheme differs from the first-order step."""
    wl = _small(nz=60, record_every=20)
    ref = orun.run_workload3d(wl, method="verlet")
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_VERLET) as plan:
        out = plan.propagate()
        half = plan.propagate(n_end=30, records=False).psi
        rest = plan.propagate(psi_in=half, n_begin=30, records=False).psi
    err = _rel(out.psi, ref.psi)
    assert err <= TOL_FP32, err
    for r in range(ref.records.shape[1]):
        assert _rel(out.records[:, r], ref.records[:, r]) <= TOL_FP32, r
    assert np.allclose(out.powers, ref.powers, rtol=2 * TOL_FP32, atol=1e-12 * ref.powers.max())
    assert _rel(rest, out.psi) <= 1e-5
    first = orun.run_workload3d(wl)
    assert _rel(first.psi, ref.psi) > max(1e-6, 10 * err)
