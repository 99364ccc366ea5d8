"""Operator splitting of Eq. split-op (Verlet, Forest-Ruth) on the plain
FP64 GPU path, and Verlet and Forest-Ruth on the fused FP32 path
(N = 8..4096), against the oracle; other combinations are refused."""

import pytest

from paper_2601_06340_gb300 import binding, inputs
import numpy as np

from parity_util import TOL_FP32, TOL_FP64, band_errors, run_ref

pytestmark = pytest.mark.gpu

FP32, FP64 = binding.BPM_FP32_FUSED, binding.BPM_FP64_PLAIN
METHODS = {"verlet": binding.BPM_SPLIT_VERLET, "forest_ruth": binding.BPM_SPLIT_FOREST_RUTH}


@pytest.mark.parametrize("method", sorted(METHODS))
@pytest.mark.parametrize("name", ["laue_perfect", "bragg_bent", "asym_dislocation"])
def test_splitting_fp64_matches_oracle(bpm_lib, method, name):
    wl = {"laue_perfect": lambda: inputs.laue_perfect(nx=512, nz=400, record_every=50),
          "bragg_bent": lambda: inputs.bragg_bent(nx=1024, nz=600, record_every=100),
          "asym_dislocation": lambda: inputs.asym_dislocation(nx=1024, nz=500,
                                                              record_every=100)}[name]()
    ref = run_ref(wl, method=method)
    with binding.Plan(wl, FP64, splitting=METHODS[method]) as plan:
        out = plan.propagate()
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP64, errs
    # the method changes the result (it is not silently the first-order step)
    first = run_ref(wl)
    assert max(band_errors(first.psi, ref.psi)) > 1e3 * TOL_FP64


def test_splitting_refused_where_not_built(bpm_lib):
    wl = inputs.laue_perfect(nx=256, nz=10)
    with binding.Plan(wl, FP32) as plan:
        binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_FIRST_ORDER)
        binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_VERLET)
        binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_FOREST_RUTH)
    with binding.Plan(inputs.serving_request(np.random.default_rng(1), 8192, 10), FP32) as plan:
        binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_VERLET)
        binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_FOREST_RUTH)
    with binding.Plan(wl, FP64) as plan:
        with pytest.raises(binding.BpmError):
            binding.bpm_set_splitting(plan.handle, 7)


def _verlet_layout(wl, layout):
    """Launch layout the Verlet rule (or a forced layout) gives: 5 the
    N = 4096 half-band split, 4 the 2-CTA cluster, 3 one CTA per row."""
    if layout == "cta" or wl.batch > 1:
        return 3
    if layout == "cluster":
        return 4
    if wl.nx == 4096:
        return 5
    return 3 if wl.nx == 2048 else 4


@pytest.mark.parametrize("layout", ["rule", "cta", "cluster"])
@pytest.mark.parametrize("name", ["laue_perfect", "bragg_bent", "asym_dislocation", "pulse"])
def test_verlet_fp32_matches_oracle(bpm_lib, monkeypatch, name, layout):
    """The fused kernels' second-order step (half coupling, propagation, half
    coupling on the slice of the step) against the oracle's Verlet march,
    fields and records; rows of a batch included.  A single row takes the
    half-band split at N = 4096 by rule, the 2-CTA cluster form elsewhere
    except at N = 2048, batches the one-CTA form; BPM_FUSED_LAYOUT=cta|cluster
    forces either of the latter (the cluster form only while every row gets
    two SMs)."""
    if layout != "rule":
        monkeypatch.setenv("BPM_FUSED_LAYOUT", layout)
    wl = {"laue_perfect": lambda: inputs.laue_perfect(nx=512, nz=400, record_every=50),
          "bragg_bent": lambda: inputs.bragg_bent(nx=4096, nz=1000, record_every=150),
          "asym_dislocation": lambda: inputs.asym_dislocation(nx=1024, nz=500,
                                                              record_every=100),
          # more rows than one launch keeps resident: the rotation schedule
          "pulse": lambda: inputs.pulse_batched(nx=4096, nz=300, n_energy=160,
                                                record_every=100)}[name]()
    rows = [0, wl.batch - 1]
    ref = run_ref(wl, method="verlet", rows=rows)
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_VERLET) as plan:
        out = plan.propagate()
        shape = binding.bpm_launch_shape(plan.handle)
    assert shape[0] == _verlet_layout(wl, layout), shape
    errs = band_errors(out.psi[rows], ref.psi, out.records[rows], ref.records)
    assert max(errs) <= TOL_FP32, errs
    final = band_errors(out.psi[rows], ref.psi)
    assert max(final) <= TOL_FP32, final
    assert np.allclose(out.powers[rows], ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
    # and it is not the first-order step
    first = run_ref(wl, rows=rows)
    diff = max(band_errors(first.psi, ref.psi))
    assert diff > 1e-6 and diff > max(errs), (diff, errs)


def test_verlet_fp32_full_size_bragg(bpm_lib):
    """The full-size single-solve workload (Bragg, bent, Nx = 4096,
    Nz = 8000) with second-order splitting on the half-band split kernel
    against the oracle's Verlet march: fields, records and powers."""
    wl = inputs.bragg_bent()
    ref = run_ref(wl, method="verlet")
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_VERLET) as plan:
        out = plan.propagate()
        assert binding.bpm_launch_shape(plan.handle)[0] == 5
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP32, errs
    assert np.allclose(out.powers, ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())


@pytest.mark.parametrize("nx", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("method", ["verlet", "forest_ruth"])
def test_small_n_splitting_fp32_matches_oracle(bpm_lib, nx, method):
    """N <= 128 (both bands per thread, several rows per CTA): Verlet and
    Forest-Ruth on random two-band fields through a masked, strained bulk
    with a ragged record tail, a batch of rows with different energies."""
    rng = np.random.default_rng(nx + 7)
    nz = 37
    wl = inputs.pulse_batched(nx=nx, nz=nz, n_energy=5, dx_um=0.4, record_every=12)
    wl.psi0 = rng.standard_normal((5, 2, nx)) + 1j * rng.standard_normal((5, 2, nx))
    wl.crystal = dict(kind=inputs.CRYSTAL_MASK, mask=(rng.uniform(size=(nz, nx)) < 0.8))
    wl.strain = dict(kind=inputs.STRAIN_ARRAY, ux=rng.uniform(-1e-3, 1e-3, (nz, nx)))
    ref = run_ref(wl, method=method)
    with binding.Plan(wl, FP32, splitting=METHODS[method]) as plan:
        out = plan.propagate()
        shape = binding.bpm_launch_shape(plan.handle)
    assert shape[0] == (3 if method == "verlet" else 6), shape
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= 2e-6, errs
    assert np.allclose(out.powers, ref.powers, rtol=1e-5, atol=1e-9 * ref.powers.max())
    first = run_ref(wl)
    assert max(band_errors(first.psi, ref.psi)) > 1e3 * max(errs)


@pytest.mark.parametrize("name", ["n256", "laue_perfect", "bragg_bent", "asym_dislocation",
                                  "pulse"])
def test_forest_ruth_fp32_matches_oracle(bpm_lib, name):
    """The fused kernels' fourth-order step (the band-per-thread kernel, the
    2-CTA cluster for single rows with 512 <= N <= 2048, and the N = 4096
    half-band split for a single row; coupling t/2,
    then propagate t dz / couple (1-t)/2, propagate (1-2t) dz / couple
    (1-t)/2, propagate t dz / couple t/2, all on the slice of the step)
    against the oracle's Forest-Ruth march: fields, records and powers, rows
    of a rotated batch included.  It must differ from both the first-order
    and the Verlet march by more than its own error."""
    wl = {"n256": lambda: inputs.laue_perfect(nx=256, nz=300, dx_um=0.8, record_every=70),
          "laue_perfect": lambda: inputs.laue_perfect(nx=512, nz=400, record_every=50),
          "bragg_bent": lambda: inputs.bragg_bent(nx=4096, nz=1000, record_every=150),
          "asym_dislocation": lambda: inputs.asym_dislocation(nx=1024, nz=500,
                                                              record_every=100),
          # more rows than one launch keeps resident: the rotation schedule
          "pulse": lambda: inputs.pulse_batched(nx=4096, nz=300, n_energy=160,
                                                record_every=100)}[name]()
    rows = [0, wl.batch - 1]
    ref = run_ref(wl, method="forest_ruth", rows=rows)
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_FOREST_RUTH) as plan:
        out = plan.propagate()
        shape = binding.bpm_launch_shape(plan.handle)
    # a single N = 4096 row marches on the half-band split (layout 9), other
    # single rows from N = 512 on the 2-CTA cluster (layout 10)
    want = 6 if wl.batch > 1 or wl.nx < 512 else 9 if wl.nx == 4096 else 10
    assert shape[0] == want, shape
    if wl.batch > 1:
        assert shape[1] > 0, shape       # rotated
    errs = band_errors(out.psi[rows], ref.psi, out.records[rows], ref.records)
    assert max(errs) <= TOL_FP32, errs
    final = band_errors(out.psi[rows], ref.psi)
    assert max(final) <= TOL_FP32, final
    assert np.allclose(out.powers[rows], ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
    for other in ("first_order", "verlet"):
        alt = run_ref(wl, rows=rows, method=other)
        diff = max(band_errors(alt.psi, ref.psi))
        assert diff > 1e-6 and diff > max(errs), (other, diff, errs)


@pytest.mark.parametrize("nx", [8192, 16384])
@pytest.mark.parametrize("seed", [11, 2])
def test_verlet_split_band_matches_oracle(bpm_lib, nx, seed):
    """N = 8192 and 16384 (bands split over 2 and 4 CTAs per band) with the
    second-order step: the couplings of step n's second half and step
    n + 1's first half after the psi_p swap, step n + 1's slice staged in
    the peer spectrum buffer.  A bent symmetric Bragg request (seed 11) and
    a dislocated asymmetric one (seed 2) against the oracle's Verlet march:
    fields, records and powers, and a resumed march equal to the whole."""
    wl = inputs.serving_request(np.random.default_rng(seed), nx, 600)
    wl.record_every = 150
    ref = run_ref(wl, method="verlet")
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_VERLET) as plan:
        out = plan.propagate()
        assert binding.bpm_launch_shape(plan.handle)[0] == 5
        first = plan.propagate(n_begin=0, n_end=250)
        rest = plan.propagate(psi_in=first.psi, n_begin=250, n_end=wl.nz)
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP32, errs
    assert np.allclose(out.powers, ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
    assert max(band_errors(rest.psi, ref.psi)) <= TOL_FP32
    fo = run_ref(wl)
    diff = max(band_errors(fo.psi, ref.psi))
    assert diff > 1e-6 and diff > max(errs), (diff, errs)


@pytest.mark.parametrize("nx,layout,want", [
    (8192, None, 9),        # the split band's fused fourth-order form
    (8192, "staged", 7),    # stage by stage, forced
    (16384, None, 7),       # stage by stage
])
def test_forest_ruth_split_band_matches_oracle(bpm_lib, monkeypatch, nx, layout, want):
    """N = 8192 with the fourth-order step fused into the split-band kernel
    (three propagations per step, each with its own tables, in one launch),
    and N = 16384 (or 8192, forced) run stage by stage (a coupling launch
    and three one-step launches of the split-band kernel per step): a
    dislocated asymmetric Bragg request against the oracle's Forest-Ruth
    march, fields, records and powers, and a resumed march equal to the
    whole; different from the first-order and Verlet marches by more than
    its own error."""
    if layout:
        monkeypatch.setenv("BPM_FUSED_LAYOUT", layout)
    else:
        monkeypatch.delenv("BPM_FUSED_LAYOUT", raising=False)
    wl = inputs.serving_request(np.random.default_rng(2), nx, 200)
    wl.record_every = 60
    ref = run_ref(wl, method="forest_ruth")
    with binding.Plan(wl, FP32, splitting=binding.BPM_SPLIT_FOREST_RUTH) as plan:
        out = plan.propagate()
        assert binding.bpm_launch_shape(plan.handle) == (want, 0)
        first = plan.propagate(n_begin=0, n_end=77)
        rest = plan.propagate(psi_in=first.psi, n_begin=77, n_end=wl.nz)
    assert max(band_errors(rest.psi, ref.psi)) <= TOL_FP32
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP32, errs
    assert np.allclose(out.powers, ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
    for other in ("first_order", "verlet"):
        alt = run_ref(wl, method=other)
        diff = max(band_errors(alt.psi, ref.psi))
        assert diff > 1e-6 and diff > max(errs), (other, diff, errs)


def test_forest_ruth_split_band_batch(bpm_lib, monkeypatch):
    """Several N = 8192 rows on the split band's fused fourth-order form (one
    4-CTA cluster per row, each row with its own energy and stage tables):
    sampled rows against the oracle's Forest-Ruth march."""
    monkeypatch.delenv("BPM_FUSED_LAYOUT", raising=False)
    wb = inputs.pulse_batched(nx=8192, nz=150, n_energy=3, record_every=50)
    rows = [0, 2]
    ref = run_ref(wb, method="forest_ruth", rows=rows)
    with binding.Plan(wb, FP32, splitting=binding.BPM_SPLIT_FOREST_RUTH) as plan:
        out = plan.propagate()
        assert binding.bpm_launch_shape(plan.handle) == (9, 0)
    errs = band_errors(out.psi[rows], ref.psi, out.records[rows], ref.records)
    assert max(errs) <= TOL_FP32, errs
    assert np.allclose(out.powers[rows], ref.powers, rtol=1e-4, atol=1e-9 * ref.powers.max())
