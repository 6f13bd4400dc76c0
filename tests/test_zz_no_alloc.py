"""The allocation-free Coulomb entry point against the regular one.

npsim_coulomb_forces_noalloc is for callers that cannot allocate device memory
when they need forces (inside an open stream capture, under a framework whose
pool owns all device memory, or in a real-time loop).  Its partial sums live in
a fixed device array that every call reuses.  Two calls in a row, on different
inputs and sizes, must each match the regular entry point
npsim_forces(sim, 3), whose scratch npsim_create allocates, within the force
tolerance the other parity tests use.  This file is collected last so that a
run stopping at its first failure has run every other test already.
"""
import numpy as np
import pytest

import workloads as wl
from gpu_helpers import FORCE_TOL, force_error, library, small, with_

pytestmark = pytest.mark.gpu


def _case(P, torch, n, seed):
    sc = with_(small(wl.config3(seed=seed), n), lj_mode=0)  # Coulomb only
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    stream = torch.cuda.current_stream()
    sim = P.Sim(sc, x, v, types, stream=stream)
    ref = sim.forces(3)
    xq = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    P.npsim_positions_device(sim.h, xq.data_ptr())
    return sc, sim, ref, xq


def test_noalloc_matches_regular_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    P = library()
    cases = [_case(P, torch, 3001, 0), _case(P, torch, 1500, 1)]
    try:
        for sc, sim, ref, xq in cases:
            n = xq.shape[0]
            F = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
            P.npsim_coulomb_forces_noalloc(xq.data_ptr(), n, sc.bjerrum, F.data_ptr(),
                                           torch.cuda.current_stream())
            torch.cuda.synchronize()
            got = F.cpu().numpy()
            assert np.isfinite(got).all()
            err = force_error(got, ref)
            assert err.max() <= FORCE_TOL, float(err.max())
    finally:
        for _, sim, _, _ in cases:
            sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    P = library()
    n = 32769
    xq = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.NpsimError) as e:
        P.npsim_coulomb_forces_noalloc(xq.data_ptr(), n, 0.7, F.data_ptr())
    assert e.value.code == -1
