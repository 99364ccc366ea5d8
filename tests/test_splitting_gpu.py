"""Operator splitting of Eq. split-op (Verlet, Forest-Ruth) on the plain
FP64 GPU path against the oracle; FP32 plans refuse it."""

import pytest

from paper_2601_06340_gb300 import binding, inputs
from parity_util import TOL_FP64, band_errors, run_ref

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
        with pytest.raises(binding.BpmError):
            binding.bpm_set_splitting(plan.handle, binding.BPM_SPLIT_VERLET)
    with binding.Plan(wl, FP64) as plan:
        with pytest.raises(binding.BpmError):
            binding.bpm_set_splitting(plan.handle, 7)
