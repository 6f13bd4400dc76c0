"""The allocation-free Coulomb entry point against the regular one and the oracle.

npsim_coulomb_forces_noalloc is for callers that cannot allocate device memory
when they need forces: code under a framework whose own pool owns all device
memory and forbids raw allocations, or a real-time loop that cannot risk an
allocation's latency or failure.  Its partial sums live in a fixed device
array that every call reuses.

Two calls in a row, on different inputs and sizes, must each match the regular
entry point npsim_forces(sim, 3) (whose scratch npsim_create allocates) and the
float64 oracle's Coulomb sum at the same float32 positions, within the force
tolerance the other parity tests use.  A third case runs at the documented
maximum n = 32768, where the fixed scratch is used to its last slot, and
compares sampled rows with the oracle.  This file is collected last so that a
run stopping at its first failure has run every other test already.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import FORCE_TOL, force_error, library, small, with_

pytestmark = pytest.mark.gpu

MAX_N = 32768  # the largest n the fixed scratch holds


def _case(P, torch, n, seed):
    sc = with_(small(wl.config3(seed=seed), n), lj_mode=0)  # Coulomb only
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    stream = torch.cuda.current_stream()
    sim = P.Sim(sc, x, v, types, stream=stream)
    ref = sim.forces(3)
    xq = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    P.npsim_positions_device(sim.h, xq.data_ptr())
    return sc, sim, ref, xq, x, types


def _oracle_coulomb(sc, x, types, sel=None):
    return oracle.pair_forces(x, types, [t.sigma for t in sc.types],
                              [t.eps for t in sc.types], [t.charge for t in sc.types],
                              sc.bjerrum, lj=False, coulomb=True, sel=sel)


def _noalloc(P, torch, sc, xq):
    n = xq.shape[0]
    F = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    P.npsim_coulomb_forces_noalloc(xq.data_ptr(), n, sc.bjerrum, F.data_ptr(),
                                   torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = F.cpu().numpy()
    assert np.isfinite(got).all()
    return got


def test_noalloc_matches_regular_entry_point_and_oracle_on_two_calls():
    torch = pytest.importorskip("torch")
    P = library()
    cases = [_case(P, torch, 3001, 0), _case(P, torch, 1500, 1)]
    try:
        for sc, sim, ref, xq, x, types in cases:
            got = _noalloc(P, torch, sc, xq)
            err = force_error(got, ref)
            assert err.max() <= FORCE_TOL, ("vs npsim_forces", float(err.max()))
            err = force_error(got, _oracle_coulomb(sc, x, types))
            assert err.max() <= FORCE_TOL, ("vs oracle", float(err.max()))
    finally:
        for case in cases:
            case[1].close()


def test_noalloc_at_its_maximum_size():
    """n = 32768 needs every slot of the fixed scratch (64 row tiles of 512 plus
    one slot per CTA): sampled rows against the oracle, all rows against the
    regular entry point, and Newton's third law on the sum."""
    torch = pytest.importorskip("torch")
    P = library()
    sc, sim, ref, xq, x, types = _case(P, torch, MAX_N, 2)
    try:
        got = _noalloc(P, torch, sc, xq)
    finally:
        sim.close()
    assert force_error(got, ref).max() <= FORCE_TOL
    rng = np.random.default_rng(3)
    sel = np.unique(np.concatenate([[0, 511, 512, MAX_N - 1],
                                    rng.choice(MAX_N, 120, replace=False)]))
    o = _oracle_coulomb(sc, x, types, sel=sel)
    rms = np.sqrt((ref ** 2).sum(1).mean())
    err = np.linalg.norm(got[sel] - o, axis=1) / np.maximum(np.linalg.norm(o, axis=1), rms)
    assert err.max() <= FORCE_TOL, float(err.max())
    assert np.abs(got.sum(0)).max() <= 1e-6 * np.abs(got).sum()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    P = library()
    n = MAX_N + 1
    xq = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.NpsimError) as e:
        P.npsim_coulomb_forces_noalloc(xq.data_ptr(), n, 0.7, F.data_ptr())
    assert e.value.code == -1
