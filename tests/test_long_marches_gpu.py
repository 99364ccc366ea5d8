"""Long fused FP32 marches at the split-band sizes against the oracle.

N = 8192 and 16384 run as bands split over 2 and 4 CTAs per band.  Their
circulant tables once carried a fixed error on the modes that hold the beam,
repeated every step, which grew to 7e-4 over 20000 steps; each table value
is now rounded relative to itself.  These are the marches the request server
runs at its largest sizes: 20000 steps (1 mm of march at dz = 0.05 um) of a
symmetric Bragg request with a bent crystal and of an asymmetric Bragg
request with an edge dislocation, per size, against the oracle at the FP32
bound over the final fields and the records every 5000 steps."""

import numpy as np
import pytest

from paper_2601_06340_gb300 import binding, inputs

from parity_util import TOL_FP32, band_errors, submit_ref

pytestmark = pytest.mark.gpu

FP32 = binding.BPM_FP32_FUSED
NZ = 20000
REC = 5000
# (nx, seed): seed 11 draws a symmetric Bragg slab with a bend, seed 2 an
# asymmetric Bragg slab with an edge dislocation (inputs.serving_request)
CASES = [(8192, 11), (8192, 2), (16384, 11), (16384, 2)]


def _request(nx, seed):
    wl = inputs.serving_request(np.random.default_rng(seed), nx, NZ)
    wl.record_every = REC
    return wl


@pytest.fixture(scope="module")
def long_refs():
    """All four oracle marches start at once in the spawn pool and run while
    the GPU tests of this module proceed."""
    return {case: submit_ref(_request(*case)) for case in CASES}


def test_cases_are_the_intended_geometries():
    assert [inputs.serving_request(np.random.default_rng(s), 8192, NZ).meta["geometry"]
            for s in (11, 2)] == [0, 2]
    kinds = [inputs.serving_request(np.random.default_rng(s), 8192, NZ).strain["kind"]
             for s in (11, 2)]
    assert kinds == [inputs.STRAIN_BENT, inputs.STRAIN_EDGE_DISLOCATION]


@pytest.mark.parametrize("nx,seed", CASES)
def test_20000_step_split_band_march_matches_oracle(bpm_lib, long_refs, nx, seed):
    wl = _request(nx, seed)
    with binding.Plan(wl, FP32) as plan:
        out = plan.propagate()
        form, nbytes = binding.bpm_slice_form(plan.handle)
    # the bent request keeps separable slices (about 2 MB instead of the
    # 1.3-2.6 GB per-cell stream), the dislocated one the stream
    if wl.strain["kind"] == inputs.STRAIN_BENT:
        assert (form, nbytes) == (1, NZ * 96 + nx * 8)
    else:
        assert (form, nbytes) == (0, NZ * nx * 8)
    ref = long_refs[(nx, seed)].result()
    errs = band_errors(out.psi, ref.psi, out.records, ref.records)
    assert max(errs) <= TOL_FP32, (nx, seed, errs)
    # the final fields alone (the stricter reading when a band has decayed)
    final = band_errors(out.psi, ref.psi)
    assert max(final) <= TOL_FP32, (nx, seed, final)
