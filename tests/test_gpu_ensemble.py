"""Batched ensemble of droplets of uneven N (one launch per force pass for all
droplets) against the FP64 oracle and against single-droplet runs."""
import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import FORCE_TOL, TRAJ_TOL, cutoff_ambiguous, force_error, library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return library()


@pytest.fixture(scope="module")
def drops():
    scs = wl.ensemble_config(n_droplets=6, master_seed=7, n_min=300, n_max=3000)
    out = []
    for sc in scs:
        types, x, v = wl.initial_state(sc, fp32_positions=True)
        out.append((sc, x, v, types))
    return out


def test_ensemble_forces_match_oracle(P, drops):
    with P.Ensemble(drops) as ens:
        for d, (sc, x, v, types) in enumerate(drops):
            F = ens.forces(d)
            ref = oracle.total_forces(sc, x, types, 0.0)
            amb = cutoff_ambiguous(x, types, sc)
            err = force_error(F, ref)[~amb]
            assert err.max() <= FORCE_TOL, (d, sc.n, float(err.max()))


def test_ensemble_every_shape(P, drops, monkeypatch):
    sc, x, v, types = drops[2]
    ref = [oracle.total_forces(s, xx, tt, 0.0) for s, xx, _, tt in drops]
    for idx in range(8):  # the ensemble kernel's eight launch shapes
        monkeypatch.setenv("NPSIM_ENS_SHAPE", str(idx))
        with P.Ensemble(drops) as ens:
            assert ens.config()["index"] == idx
            for d, (s, xx, vv, tt) in enumerate(drops):
                amb = cutoff_ambiguous(xx, tt, s)
                err = force_error(ens.forces(d), ref[d])[~amb]
                assert err.max() <= FORCE_TOL, (idx, d, float(err.max()))


def test_ensemble_trajectories_match_oracle_and_single_runs(P, drops):
    steps = 60
    with P.Ensemble(drops) as ens:
        n_tot, pairs = ens.info()
        assert n_tot == sum(len(d[1]) for d in drops)
        assert pairs == sum(len(d[1]) * (len(d[1]) - 1) for d in drops)
        ens.step(steps)
        states = [ens.state(d) for d in range(len(drops))]
    for d, (sc, x, v, types) in enumerate(drops):
        xe, ve, Fe, st = states[d]
        assert st == steps
        xo, vo, Fo = oracle.run(sc, x, v, types, 0, steps)
        assert np.abs(xe - xo).max() <= TRAJ_TOL, d
        with P.Sim(sc, x, v, types) as sim:
            sim.step(steps)
            xs, vs, _, _ = sim.state()
        # same physics, same Philox keys; the pair sums differ only in float
        # summation order (type groups padded to 256 here, to 512 in a single
        # run), which 60 steps amplify to a few 1e-8; a wrong key or counter
        # would differ by the noise amplitude itself (~1e-2)
        assert np.abs(xe - xs).max() <= 1e-6, d


def test_ensemble_large_droplets_sampled(P):
    """Droplets large enough that most (warp, segment) pairs are beyond the LJ
    cutoff (culled to the Coulomb-only sweep): sampled rows of every droplet
    against the oracle."""
    scs = wl.ensemble_config(n_droplets=3, master_seed=11, n_min=9000, n_max=16000)
    drops = []
    for sc in scs:
        types, x, v = wl.initial_state(sc, fp32_positions=True)
        drops.append((sc, x, v, types))
    rng = np.random.default_rng(2)
    with P.Ensemble(drops) as ens:
        for d, (sc, x, v, types) in enumerate(drops):
            F = ens.forces(d)
            sel = np.unique(rng.choice(sc.n, 100, replace=False))
            ref = oracle.pair_forces(x, types, [t.sigma for t in sc.types],
                                     [t.eps for t in sc.types], [t.charge for t in sc.types],
                                     sc.bjerrum, lj_cut=sc.lj_cut, lj=sc.lj_mode != 0,
                                     coulomb=sc.coulomb, eps_override=sc.eps_override, sel=sel)
            ref = ref + oracle.external_forces(sc, x[sel], types[sel], 0.0)
            keep = ~cutoff_ambiguous(x, types, sc)[sel]
            rms = np.sqrt((F ** 2).sum(1).mean())
            err = np.linalg.norm(F[sel] - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)
            assert err[keep].max() <= FORCE_TOL, (d, sc.n, float(err.max()))


def test_ensemble_runs_are_bit_reproducible(P, drops):
    """CTAs draw work items in whatever order they reach the counter, but every
    item writes its own slot and a row's items are summed in item order: two
    runs of the same ensemble agree bit for bit (and the item counter is reset
    between launches, or the second run would find no work).  The second
    ensemble of the same geometry reuses the first one's launch shape."""
    states, shapes = [], []
    for _ in range(2):
        with P.Ensemble(drops) as ens:
            shapes.append(ens.config()["index"])
            ens.step(25)
            states.append([ens.state(d) for d in range(len(drops))])
    assert shapes[0] == shapes[1]
    for a, b in zip(*states):
        for u, w in zip(a[:3], b[:3]):
            assert np.array_equal(u, w)
