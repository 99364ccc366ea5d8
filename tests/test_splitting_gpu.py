"""Operator splitting of Eq. split-op (Verlet, Forest-Ruth) on the plain
FP64 GPU path, and Verlet on the fused FP32 path (N = 256..4096), against
the oracle; other combinations are refused."""

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
        with pytest.raises(binding.BpmError):
            binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_FOREST_RUTH)
    with binding.Plan(inputs.laue_perfect(nx=128, nz=10), FP32) as plan:
        with pytest.raises(binding.BpmError):
            binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_VERLET)
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
