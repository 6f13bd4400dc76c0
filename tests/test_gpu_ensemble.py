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
    steps = 100  # the step count the 1e-4 sigma trajectory tolerance is stated for
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
        # run), which 100 steps amplify to ~1e-7 at most; a wrong key or counter
        # would differ by the noise amplitude itself (~1e-2)
        assert np.abs(xe - xs).max() <= 1e-6, d


def test_ensemble_large_droplets_sampled(P):
    """Droplets large enough that most (warp, segment) pairs are beyond the LJ
    cutoff (culled to the Coulomb-only sweep), up to the largest N of the
    256-droplet ensemble (32768, many more j-tiles per work item row): sampled
    rows of every droplet against the oracle."""
    scs = wl.ensemble_config(n_droplets=3, master_seed=11, n_min=9000, n_max=16000)
    scs += wl.ensemble_config(n_droplets=1, master_seed=13, n_min=32768, n_max=32768)
    assert scs[-1].n == 32768
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


def test_ensemble_stats_match_oracle(P, drops):
    """npsim_ens_stats (the statistics of Sec. 3 straight from the ensemble's
    device state) for droplets of uneven N after some steps, against the oracle
    on the same float64 positions: integer histograms and box counts exactly,
    g, C_NPs, R_g and both D_f to float64 rounding."""
    steps = 20
    sizes = [len(d[1]) for d in drops]
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), 2]
    with P.Ensemble(drops) as ens:
        ens.step(steps)
        got = {d: (ens.state(d)[0], ens.stats(d, r_max=8.0, n_bins=64, radial_bins=16,
                                               boxcount=True)) for d in picks}
        # a second call on the first droplet reuses the scratch grown for the largest
        again = ens.stats(picks[0], r_max=8.0, n_bins=64, radial_bins=16, boxcount=True)
    assert np.array_equal(again["rdf_counts"], got[picks[0]][1]["rdf_counts"])
    assert np.array_equal(again["nbox"], got[picks[0]][1]["nbox"])
    for d in picks:
        sc, _, _, types = drops[d]
        xg, st = got[d]
        R = oracle.radius(sc.R0, sc.k_evap, steps * sc.dt)
        assert st["R"] == pytest.approx(R, rel=1e-14)
        sig = np.array([t.sigma for t in sc.types])
        d_mean = float(sig[types].mean())
        assert st["d_mean"] == pytest.approx(d_mean, rel=1e-14)
        c_o, g_o = oracle.rdf(xg, 8.0, 64, R)
        assert np.array_equal(st["rdf_counts"], c_o), d
        assert np.allclose(st["rdf_g"], g_o, rtol=1e-12, atol=0)
        rc_o, C_o = oracle.radial_concentration(xg, R, 16, R)
        assert np.array_equal(st["radial_counts"], rc_o)
        assert np.allclose(st["radial_c"], C_o, rtol=1e-12)
        Rg, Df, r0 = oracle.rg(xg, d_mean)
        assert st["Rg"] == pytest.approx(Rg, rel=1e-12)
        assert st["Df_rg"] == pytest.approx(Df, rel=1e-10)
        assert np.allclose(st["center"], r0, rtol=1e-10, atol=1e-12)
        Dfb, nb = oracle.boxcount_df(xg, d_mean, Rg)
        assert np.array_equal(st["nbox"], nb)
        if np.isfinite(Dfb):
            assert st["Df_box"] == pytest.approx(Dfb, rel=1e-10)
        assert st["n_surf"] == oracle.surface_count(xg, types, sig, st["R"])


def test_ensemble_stats_rejects_a_bad_droplet_index(P, drops):
    with P.Ensemble(drops[:2]) as ens:
        for d in (-1, 2):
            with pytest.raises(P.NpsimError) as e:
                ens.stats(d, r_max=8.0, n_bins=16)
            assert e.value.code == -1  # NPSIM_ERR_INVALID_ARG
        with pytest.raises(P.NpsimError):
            ens.stats(0, r_max=-1.0, n_bins=16)  # bins need a positive range


def test_ensemble_reports_an_escaped_np(P, drops):
    """An NP of one droplet farther than 2 max(R0, R(t)) from its centre (spring
    on) makes npsim_ens_step return NPSIM_ERR_ESCAPED; the other droplets' NPs
    are inside theirs, and an ensemble without it steps without error."""
    sc, x, v, types = drops[1]
    xb = x.copy()
    xb[3] = [0.0, 0.0, -3.0 * sc.R0]
    bad = list(drops[:3])
    bad[1] = (sc, xb, v, types)
    with P.Ensemble(bad) as ens:
        with pytest.raises(P.NpsimError) as e:
            ens.step(2)
        assert e.value.code == -8
    with P.Ensemble(drops[:3]) as ens:
        ens.step(2)


def test_ensemble_kernel_times_leave_results_unchanged(P, drops):
    """The measurement hook: with CUDA event records in its step graphs an
    ensemble gives the same states bit for bit as one without, and reports
    positive durations of its all-pairs and integrator launches over the
    steps of the last chunk; without profiling the hook is refused."""
    with P.Ensemble(drops[:3]) as a, P.Ensemble(drops[:3]) as b:
        with pytest.raises(P.NpsimError) as e:
            a.kernel_times()
        assert e.value.code == -1
        b.profile(True)
        a.step(20)
        b.step(20)  # a chunk of 16 steps, then one of 4
        kt, k = b.kernel_times()
        assert k == 4 and kt["allpairs"] > 0.0 and kt["integrate"] > 0.0
        n_items, itile = b.work()
        assert itile == b.config()["block"] * b.config()["i_per_thread"]
        rows = sum(-(-n // itile) for n in b.sizes)  # row tiles, at least one item each
        assert n_items >= rows
        for d in range(3):
            xa, va, _, _ = a.state(d)
            xb, vb, _, _ = b.state(d)
            assert np.array_equal(xa, xb) and np.array_equal(va, vb)
