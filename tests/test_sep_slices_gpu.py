"""Separable slices: for a vacuum, bulk or slab crystal with no strain or the
bent-crystal strain, h u = h x'^2/(2R) + h nu z'^2/(2R) is a column term
plus a row term and the mask is one column interval per z-step, so the plan
keeps one row per step and one phasor per column and the fused kernels form
each cell's phasor as they couple, instead of reading a per-cell stream.

Both forms hold the same cells (the same FP64-reduced column and row
phasors, the same mask decisions: the stream expanded from the separable
tables equals the stream form bit for bit).  The kernels fold the row
phasor into the step's coupling coefficient, (b row) col instead of
b (col row), so the two forms march equal up to FP32 rounding: every kernel
family, with the first-order step and the splittings of Eq. split-op, must
give the same fields in both forms to far below the FP32 bound, and match
the oracle within it.
"""

import dataclasses
import math

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP32, band_errors, submit_ref

pytestmark = pytest.mark.gpu

# separable against stream form: rounding-order differences only
TOL_FORMS = 2e-5

FP32 = binding.BPM_FP32_FUSED
FIRST = binding.BPM_SPLIT_FIRST_ORDER
VERLET = binding.BPM_SPLIT_VERLET
FR = binding.BPM_SPLIT_FOREST_RUTH


def _bent(nx, nz, geometry, record_every=50):
    """A bent slab seen by the whole window: asymmetric Bragg (the inside
    interval moves with z; rows before the surface have none) or Laue
    (every row inside or outside)."""
    wl = inputs.bragg_bent(nx=nx, nz=nz, dx_um=0.1, dz_um=0.1, record_every=record_every,
                           radius_um=0.4e6)
    z_hit = wl.meta["z_hit_um"]
    if geometry == "bragg":
        crystal = dict(kind=inputs.CRYSTAL_SLAB, asym_angle_rad=math.radians(15.0),
                       thickness_um=200.0, surf_x_um=0.0, surf_z_um=z_hit)
    else:
        crystal = dict(kind=inputs.CRYSTAL_SLAB, asym_angle_rad=math.pi / 2,
                       thickness_um=200.0, surf_x_um=0.0, surf_z_um=0.3 * nz * 0.1)
    return dataclasses.replace(wl, crystal=crystal)


def _march(wl, monkeypatch, stream, layout=None, split=FIRST):
    # either form forced (the rule takes the stream at small nx)
    monkeypatch.setenv("BPM_SLICE_STREAM", "1" if stream else "0")
    if layout:
        monkeypatch.setenv("BPM_FUSED_LAYOUT", layout)
    else:
        monkeypatch.delenv("BPM_FUSED_LAYOUT", raising=False)
    with binding.Plan(wl, FP32, splitting=split) as plan:
        out = plan.propagate()
        shape = binding.bpm_launch_shape(plan.handle)
        form = binding.bpm_slice_form(plan.handle)
    return out, shape, form


# (nx, nz, BPM_FUSED_LAYOUT, splitting, launch layout or None): every fused
# kernel family with each step form it runs (first-order single rows report
# the fixed rule, -1, which BPM_FUSED_LAYOUT steers)
CASES = [
    (64, 300, None, FIRST, None),        # both bands per thread
    (64, 300, None, VERLET, None),
    (64, 300, None, FR, None),
    (1024, 300, "cta", FIRST, -1),       # band per thread, one CTA per row
    (1024, 300, "cta", VERLET, 3),
    (1024, 300, "cta", FR, 6),
    (1024, 300, "cluster", FIRST, -1),   # 2-CTA cluster
    (1024, 300, "cluster", VERLET, 4),
    (1024, 300, None, FR, 10),
    (4096, 400, None, FIRST, 2),         # half-band split, 8 points per thread
    (4096, 400, "split16", FIRST, 8),    # half-band split, 16 points per thread
    (4096, 400, None, VERLET, 5),        # the 8-point split's Verlet form
    (4096, 200, None, FR, 9),            # the 8-point split's Forest-Ruth form
    (4096, 400, "split16", VERLET, 5),   # the 16-point split's Verlet form
    (8192, 300, None, FIRST, -1),        # split band, two parts
    (8192, 300, None, VERLET, 5),
    (8192, 120, None, FR, 9),            # the split band's Forest-Ruth form
    (8192, 120, "staged", FR, 7),        # stage by stage (coupling-only launches)
    (16384, 300, None, FIRST, -1),       # split band, four parts (TMEM tables)
    (16384, 300, None, VERLET, 5),
]


METHOD = {FIRST: "first_order", VERLET: "verlet", FR: "forest_ruth"}
GEOMETRIES = ["bragg", "laue"]


@pytest.fixture(scope="module")
def sep_refs():
    """The oracle marches of every case, started at once in the spawn pool."""
    keys = {(g, c[0], c[1], c[3]) for g in GEOMETRIES for c in CASES}
    return {k: submit_ref(_bent(k[1], k[2], k[0]), method=METHOD[k[3]]) for k in sorted(keys)}


@pytest.mark.parametrize("geometry", GEOMETRIES)
@pytest.mark.parametrize("nx,nz,layout,split,want", CASES)
def test_separable_against_stream_and_oracle(bpm_lib, monkeypatch, sep_refs, geometry, nx, nz,
                                             layout, split, want):
    wl = _bent(nx, nz, geometry)
    sep, sep_shape, sep_form = _march(wl, monkeypatch, False, layout, split)
    st, st_shape, st_form = _march(wl, monkeypatch, True, layout, split)
    assert sep_form[0] == 1 and st_form[0] == 0, (sep_form, st_form)
    assert sep_form[1] == nz * 96 + nx * 8 and st_form[1] == nz * nx * 8
    assert sep_shape == st_shape, (sep_shape, st_shape)
    if want is not None:
        assert sep_shape[0] == want, sep_shape
    forms = band_errors(sep.psi, st.psi, sep.records, st.records)
    assert max(forms) <= TOL_FORMS, forms
    assert np.allclose(sep.powers, st.powers, rtol=TOL_FORMS, atol=1e-9 * st.powers.max())
    ref = sep_refs[(geometry, nx, nz, split)].result()
    errs = band_errors(sep.psi, ref.psi, sep.records, ref.records)
    assert max(errs) <= TOL_FP32, errs


@pytest.mark.parametrize("nx", [512, 4096, 8192, 16384])
def test_fetched_slices_are_identical(bpm_lib, monkeypatch, nx):
    """The cells expanded from the separable tables equal the stream's (in
    the natural order, whatever the per-part layout of the plan)."""
    wl = _bent(nx, 200, "bragg")
    got = {}
    for stream in (False, True):
        monkeypatch.setenv("BPM_SLICE_STREAM", "1" if stream else "0")
        with binding.Plan(wl, FP32) as plan:
            mask, ph = plan.slices()
            got[stream] = (mask, ph, binding.bpm_slice_form(plan.handle)[0])
    assert got[False][2] == 1 and got[True][2] == 0
    assert np.array_equal(got[False][0], got[True][0])
    assert np.array_equal(got[False][1], got[True][1])
    inside = got[False][0].astype(bool)
    assert inside.any() and (~inside).any()
    assert np.allclose(np.abs(got[False][1][inside]), 1.0, atol=1e-6)


def test_which_plans_are_separable(bpm_lib, monkeypatch):
    """Bent or unstrained slabs take the separable form at nx = 4096 (first
    order) while every row gets four SMs and at nx >= 8192 while every row
    gets two; a
    smaller nx, a dislocation, a polygon cut, an FP64 plan, a batch that
    fills the GPU or BPM_SLICE_STREAM=1 keep the stream; BPM_SLICE_STREAM=0
    gives them the separable form where the crystal allows it."""
    monkeypatch.delenv("BPM_SLICE_STREAM", raising=False)

    def form(wl, precision=FP32, split=FIRST):
        with binding.Plan(wl, precision, splitting=split) as plan:
            assert binding.bpm_slice_form(plan.handle)[0] == -1   # prepared at the first march
            plan.propagate(n_end=2)
            return binding.bpm_slice_form(plan.handle)

    assert form(inputs.bragg_bent(nx=4096, nz=50)) == (1, 50 * 96 + 4096 * 8)
    # the N = 4096 Verlet form marches faster on the stream
    assert form(inputs.bragg_bent(nx=4096, nz=50), split=VERLET)[0] == 0
    assert form(inputs.bragg_bent(nx=8192, nz=50), split=VERLET)[0] == 1
    assert form(inputs.bragg_bent(nx=8192, nz=50))[0] == 1
    assert form(inputs.laue_perfect(nx=16384, nz=50))[0] == 1
    assert form(inputs.bragg_bent(nx=1024, nz=50)) == (0, 50 * 1024 * 8)
    assert form(inputs.asym_dislocation(nx=8192, nz=50))[0] == 0
    assert form(inputs.bragg_bent(nx=4096, nz=50), binding.BPM_FP64_PLAIN)[0] == 0
    wl = inputs.asym_dislocation(nx=8192, nz=50)
    assert form(dataclasses.replace(wl, strain=dict(kind=inputs.STRAIN_NONE)))[0] == 0
    batch = inputs.pulse_batched(nx=4096, nz=50, n_energy=256)
    assert form(batch)[0] == 0
    monkeypatch.setenv("BPM_SLICE_STREAM", "0")
    assert form(batch)[0] == 1
    assert form(inputs.bragg_bent(nx=1024, nz=50))[0] == 1


def test_separable_rotated_batch(bpm_lib, monkeypatch):
    """A 256-energy bent batch in the separable form (forced), marched by
    the rotated one-CTA-per-row schedule with several launches per march,
    against the stream form and the oracle on sampled rows."""
    wb = inputs.pulse_batched(nx=4096, nz=400, n_energy=256, record_every=200)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("BPM_SLICE_STREAM", mode)
        with binding.Plan(wb, FP32) as plan:
            out[mode] = plan.propagate()
            assert binding.bpm_slice_form(plan.handle)[0] == (1 if mode == "0" else 0)
            assert binding.bpm_launch_shape(plan.handle)[1] > 0   # rotated
    forms = band_errors(out["0"].psi, out["1"].psi, out["0"].records, out["1"].records)
    assert max(forms) <= TOL_FORMS, forms
    rows = [0, 97, 255]
    ref = submit_ref(wb, rows=rows).result()
    errs = band_errors(out["0"].psi[rows], ref.psi, out["0"].records[rows], ref.records)
    assert max(errs) <= TOL_FP32, errs


def test_splitting_change_reprepares_the_slices(bpm_lib, monkeypatch):
    """The N = 4096 slice form follows the step form: switching a prepared
    first-order plan to Verlet prepares the stream at its next march."""
    monkeypatch.delenv("BPM_SLICE_STREAM", raising=False)
    wl = inputs.bragg_bent(nx=4096, nz=40)
    with binding.Plan(wl, FP32) as plan:
        plan.propagate(n_end=2)
        assert binding.bpm_slice_form(plan.handle)[0] == 1
        binding.bpm_set_splitting(plan.handle, VERLET)
        assert binding.bpm_slice_form(plan.handle)[0] == -1
        plan.propagate(n_end=2)
        assert binding.bpm_slice_form(plan.handle)[0] == 0
