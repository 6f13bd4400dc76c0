"""GPU path vs the FP64 oracle, through the C ABI.

Forces are compared at float32-representable positions (the positions the
float32 pair kernels see exactly), with the metric
max_i |dF_i| / max(|F_i|, rms_j |F_j|) <= 1e-5.  Trajectories are compared after
100 steps to 1e-4 sigma.  Philox words are compared bit for bit; integer
histogram counts exactly.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_helpers import (FORCE_TOL, TRAJ_TOL, cutoff_ambiguous, force_error, library,
                         small, with_)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return library()


# --------------------------------------------------------------------------
# Philox and normals


def test_philox_bit_exact(P):
    for seed in (0, 1, 0x123456789, 0xFFFFFFFFFFFFFFFF):
        for ctr in ([0, 0, 0, 0], [0xFFFFFF00, 7, 3, 1], [5, 0xFFFFFFFF, 0, 2]):
            g = P.npsim_philox(seed, ctr, 4096)
            o = oracle.philox_blocks(seed, ctr, 4096)
            assert np.array_equal(g, o), (seed, ctr)


def test_normals_match_oracle(P):
    for seed, step in ((3, 0), (0xABCDEF, 123456789012)):
        g = P.npsim_normals(seed, step, 50000)
        o = oracle.normals(seed, step, 0, 50000)
        d = np.abs(g - o)
        # float32 Box-Muller: ~1e-7 relative; the worst case is at tiny radii
        assert np.median(d) < 1e-6
        assert d.max() < 2e-4


# --------------------------------------------------------------------------
# Forces


def _scen(name):
    if name == "lj1000_cell":
        return wl.config1()
    if name == "coul_lj_allpairs_3001":
        return small(wl.config2(), 3001)
    if name == "coul_allpairs_lj_cell_5003":
        return small(wl.config3(), 5003)
    if name == "lj_allpairs_only_1537":
        return with_(small(wl.config2(), 1537), coulomb=False)
    if name == "coul_only_2049":
        return with_(small(wl.config3(), 2049), lj_mode=0)
    if name == "eps_matrix_1200":
        sc = small(wl.config2(), 1200)
        return with_(sc, eps_override=np.array([[0.155, 1.26], [1.26, 0.155]]) * 4)
    if name == "truncated_coul_lj_cell_5003":  # the printed range 4 sigma_ab, cell list
        return with_(small(wl.config3(), 5003), coulomb_cut=4.0)
    if name == "isotropic_centrifugal_coul_lj_2000":
        # the tumbling droplet of Sec. 1.2 (Fig. 2: omega = 1, isotropic): the
        # centrifugal force m omega^2 x in every direction, no gravity
        return with_(small(wl.config2(), 2000), rot_mode=2, omega=1.0, g=0.0)
    raise KeyError(name)


SCENARIOS = ["lj1000_cell", "coul_lj_allpairs_3001", "coul_allpairs_lj_cell_5003",
             "lj_allpairs_only_1537", "coul_only_2049", "eps_matrix_1200",
             "truncated_coul_lj_cell_5003", "isotropic_centrifugal_coul_lj_2000"]


def _oracle_pair(sc, x, types, lj=True, coul=True, sel=None):
    sig = [t.sigma for t in sc.types]
    eps = [t.eps for t in sc.types]
    q = [t.charge for t in sc.types]
    return oracle.pair_forces(x, types, sig, eps, q, sc.bjerrum, lj_cut=sc.lj_cut,
                              lj=lj and sc.lj_mode != 0, coulomb=coul and sc.coulomb,
                              eps_override=sc.eps_override, sel=sel,
                              coulomb_cut=sc.coulomb_cut)


@pytest.mark.parametrize("name", SCENARIOS)
def test_forces_parity(P, name):
    sc = _scen(name)
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    amb = cutoff_ambiguous(x, types, sc)
    assert amb.sum() <= max(2, len(x) // 500)
    keep = ~amb
    with P.Sim(sc, x, v, types) as sim:
        F_pair = sim.forces(1)
        F_lj = sim.forces(2)
        F_coul = sim.forces(3)
        F_tot = sim.forces(0)
        _, _, F_state, _ = sim.state()
    o_pair = _oracle_pair(sc, x, types)
    o_lj = _oracle_pair(sc, x, types, coul=False)
    o_coul = _oracle_pair(sc, x, types, lj=False)
    o_tot = oracle.total_forces(sc, x, types, 0.0)
    for got, ref, what in ((F_pair, o_pair, "pair"), (F_lj, o_lj, "lj"),
                           (F_coul, o_coul, "coulomb"), (F_tot, o_tot, "total"),
                           (F_state, o_tot, "state")):
        if not np.any(ref):
            assert np.all(got == 0), what
            continue
        err = force_error(got, ref)[keep]
        assert err.max() <= FORCE_TOL, (what, float(err.max()), int(err.argmax()))
    # Newton's third law on the GPU pair forces
    assert np.abs(F_pair.sum(0)).max() <= 1e-6 * np.abs(F_pair).sum()


def test_every_launch_shape(P, monkeypatch):
    """Each all-pairs launch shape of the autotuner's table (scalar, packed
    float32x2, charge-grouped Coulomb, type-grouped LJ + Coulomb), forced in
    turn, gives the oracle's forces on a ragged size, for a Coulomb-only and an
    LJ + Coulomb sum."""
    sc_c = with_(small(wl.config3(), 1531), lj_mode=0)          # Coulomb only
    sc_l = with_(small(wl.config2(), 1531), coulomb=True)        # Coulomb + LJ
    st_c = wl.initial_state(sc_c, fp32_positions=True)
    st_l = wl.initial_state(sc_l, fp32_positions=True)
    ref_c = _oracle_pair(sc_c, st_c[1], st_c[0])
    ref_l = _oracle_pair(sc_l, st_l[1], st_l[0])
    amb_l = cutoff_ambiguous(st_l[1], st_l[0], sc_l)
    ref_lo = _oracle_pair(sc_l, st_l[1], st_l[0], coul=False)
    ref_co = _oracle_pair(sc_l, st_l[1], st_l[0], lj=False)
    seen = set()
    for idx in range(P.npsim_allpairs_num_configs()):
        monkeypatch.setenv("NPSIM_AUTOTUNE", f"1:{idx}")
        with P.Sim(sc_c, st_c[1], st_c[2], st_c[0]) as sim:
            cfg = sim.allpairs_config()
            assert cfg["index"] == idx  # every shape can sum Coulomb alone
            seen.add(cfg["packed"])
            err = force_error(sim.forces(1), ref_c)
            assert err.max() <= FORCE_TOL, (idx, float(err.max()))
        with P.Sim(sc_l, st_l[1], st_l[2], st_l[0]) as sim:
            cfg = sim.allpairs_config()
            # the LJ sum runs on the scalar or on the type-grouped kernels
            assert cfg["packed"] in (0, 3)
            if cfg["index"] == idx:
                seen.add(10 + cfg["packed"])
            for what, ref in ((1, ref_l), (2, ref_lo), (3, ref_co)):
                err = force_error(sim.forces(what), ref)[~amb_l]
                assert err.max() <= FORCE_TOL, (idx, what, float(err.max()))
    assert seen == {0, 1, 2, 3, 10, 13}


def test_dynamic_ranges(P, monkeypatch):
    """The grouped kernels cut their work into several ranges per CTA and hand
    them out at run time.  For 1, 3 and 16 ranges per CTA, on droplets large
    enough that there are more ranges than CTAs, every grouped shape gives the
    oracle's forces on sampled rows, and a second evaluation (the CTAs taking
    other ranges) is bit-identical."""
    sc_c = with_(small(wl.config3(), 60001), lj_mode=0)      # Coulomb only
    sc_l = with_(small(wl.config2(), 20011), coulomb=True)   # Coulomb + LJ
    rng = np.random.default_rng(5)
    checked = set()
    for sc, packed in ((sc_c, 2), (sc_l, 3)):
        types, x, v = wl.initial_state(sc, fp32_positions=True)
        sel = np.unique(np.concatenate([[0, sc.n - 1], rng.choice(sc.n, 150, replace=False)]))
        ref = _oracle_pair(sc, x, types, sel=sel)
        amb = cutoff_ambiguous(x, types, sc)[sel]
        for idx in range(P.npsim_allpairs_num_configs()):
            for m in (1, 3, 16):
                monkeypatch.setenv("NPSIM_AUTOTUNE", f"1:{idx}:{m}")
                with P.Sim(sc, x, v, types) as sim:
                    cfg = sim.allpairs_config()
                    if cfg["index"] != idx or cfg["packed"] != packed:
                        break
                    F1 = sim.forces(1)
                    F2 = sim.forces(1)
                assert np.array_equal(F1, F2), (idx, m)
                rms = np.sqrt((F1 ** 2).sum(1).mean())
                err = np.linalg.norm(F1[sel] - ref, axis=1) / np.maximum(
                    np.linalg.norm(ref, axis=1), rms)
                assert err[~amb].max() <= FORCE_TOL, (idx, m, float(err.max()))
                checked.add((packed, m))
    assert checked == {(p, m) for p in (2, 3) for m in (1, 3, 16)}


def test_neutral_elision_forces_and_steps(P):
    """By default the neutral NPs are left out of the all-pairs Coulomb sum
    (their terms are exactly zero): the forces are the oracle's, a neutral NP's
    Coulomb force is exactly zero, and the trajectory equals that of the full
    sum over all N(N-1) pairs (sum_neutral) to float32 summation order.  The two
    are not bit-identical: the stream-K split of a shorter j-range groups the
    charged partners' float32 partial sums differently."""
    sc = small(wl.config3(), 3001)  # 60 % neutral NPs
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    sc_full = with_(sc, sum_neutral=True)
    amb = cutoff_ambiguous(x, types, sc)
    with P.Sim(sc, x, v, types) as sim:
        F = sim.forces(0)
        Fc = sim.forces(3)
        sim.step(20)
        xs, _, _, _ = sim.state()
    assert force_error(F, oracle.total_forces(sc, x, types, 0.0))[~amb].max() <= FORCE_TOL
    assert force_error(Fc, _oracle_pair(sc, x, types, lj=False)).max() <= FORCE_TOL
    neutral = np.array([sc.types[t].charge == 0 for t in types])
    assert np.all(Fc[neutral] == 0)
    with P.Sim(sc_full, x, v, types) as sim:
        Fc_full = sim.forces(3)
        sim.step(20)
        xa, _, _, _ = sim.state()
    assert np.all(Fc_full[neutral] == 0)
    assert force_error(Fc, Fc_full).max() <= 1e-6
    assert np.abs(xs - xa).max() < 1e-9


def test_forces_full_size_sampled(P):
    """The 250000-NP scenario at full size, in the launch configuration the benchmark
    times: sampled rows against the oracle row by row."""
    sc = wl.config3()
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    with P.Sim(sc, x, v, types) as sim:
        F = sim.forces(0)
        cfg = sim.allpairs_config()
    rng = np.random.default_rng(0)
    it = cfg["block"] * cfg["i_per_thread"]
    sel = np.unique(np.concatenate([[0, 1, sc.n - 1, sc.n - 2, it - 1, it, it + 1],
                                    rng.choice(sc.n, 41, replace=False)]))
    o = _oracle_pair(sc, x, types, sel=sel) + oracle.external_forces(sc, x[sel], types[sel], 0.0)
    amb = cutoff_ambiguous(x, types, sc)[sel]
    rms = np.sqrt((F ** 2).sum(1).mean())
    err = np.linalg.norm(F[sel] - o, axis=1) / np.maximum(np.linalg.norm(o, axis=1), rms)
    assert err[~amb].max() <= FORCE_TOL, float(err.max())
    # zero net internal force over all rows
    Fp = None
    with P.Sim(sc, x, v, types) as sim:
        Fp = sim.forces(1)
    assert np.abs(Fp.sum(0)).max() <= 1e-6 * np.abs(Fp).sum()


@pytest.mark.parametrize("coul", [True, False])
def test_lj_in_allpairs_large_droplet_sampled(P, monkeypatch, coul):
    """LJ inside the all-pairs sum on a droplet large enough that most (warp,
    64-partner segment) pairs lie beyond the LJ cutoff: those take the culled
    Coulomb-only sweep (charged types) or are skipped (no charges).  Sampled
    rows against the oracle row by row, for a type-grouped shape forced and for
    the autotuned one."""
    sc = with_(small(wl.config2(), 24000), coulomb=coul)
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    rng = np.random.default_rng(5)
    sel = np.unique(np.concatenate([[0, sc.n - 1], rng.choice(sc.n, 150, replace=False)]))
    ref = _oracle_pair(sc, x, types, sel=sel)
    keep = ~cutoff_ambiguous(x, types, sc)[sel]
    n_cfg = P.npsim_allpairs_num_configs()
    ljg = None
    for idx in range(n_cfg - 1, -1, -1):  # the type-grouped shapes close the table
        monkeypatch.setenv("NPSIM_AUTOTUNE", f"1:{idx}")
        with P.Sim(sc, x, v, types) as sim:
            if sim.allpairs_config()["packed"] != 3:
                break
            ljg = idx
    assert ljg is not None
    for forced in (f"1:{ljg}", None):
        if forced:
            monkeypatch.setenv("NPSIM_AUTOTUNE", forced)
        else:
            monkeypatch.delenv("NPSIM_AUTOTUNE", raising=False)
        with P.Sim(sc, x, v, types) as sim:
            F = sim.forces(1)
        rms = np.sqrt((F ** 2).sum(1).mean())
        err = np.linalg.norm(F[sel] - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), rms)
        assert err[keep].max() <= FORCE_TOL, (forced, float(err.max()))
        assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum()


# --------------------------------------------------------------------------
# Trajectories


TRAJ = ["lj1000_cell", "coul_lj_allpairs_2048", "coul_allpairs_lj_cell_4096",
        "overdamped_lj_1000", "printed_kick_band_coul_lj_2048", "printed_kick_band_lj1000_cell",
        "truncated_coul_lj_cell_4096", "isotropic_centrifugal_coul_lj_2048",
        "isotropic_centrifugal_lj1000_cell"]


def _traj_scen(name):
    if name == "lj1000_cell":
        return wl.config1()
    if name == "coul_lj_allpairs_2048":
        return small(wl.config2(), 2048)
    if name == "coul_allpairs_lj_cell_4096":
        return small(wl.config3(), 4096)
    if name == "overdamped_lj_1000":
        return with_(wl.config1(), integrator=1)
    # the paper's printed steps (iv) and (vi): band-limited wall, drag + fixed kick
    if name == "printed_kick_band_coul_lj_2048":
        return with_(small(wl.config2(), 2048), integrator=2, v_kick=0.05, wall_band=True)
    if name == "printed_kick_band_lj1000_cell":
        return with_(wl.config1(), integrator=2, v_kick=0.1, wall_band=True)
    if name == "truncated_coul_lj_cell_4096":
        return with_(small(wl.config3(), 4096), coulomb_cut=4.0)
    # the isotropic centrifugal force of the tumbling droplet (Sec. 1.2, Fig. 2:
    # omega = 1) pushing every NP outward against the interface spring
    if name == "isotropic_centrifugal_coul_lj_2048":
        return with_(small(wl.config2(), 2048), rot_mode=2, omega=1.0, g=0.0)
    if name == "isotropic_centrifugal_lj1000_cell":
        return with_(wl.config1(), rot_mode=2, omega=1.0)
    raise KeyError(name)


@pytest.mark.parametrize("name", TRAJ)
def test_trajectory_parity_100_steps(P, name):
    sc = _traj_scen(name)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as sim:
        sim.step(100)
        xg, vg, Fg, st = sim.state()
    assert st == 100
    xo, vo, Fo = oracle.run(sc, x, v, types, 0, 100)
    dx = np.abs(xg - xo).max()
    assert dx <= TRAJ_TOL, dx
    if sc.integrator != 1:
        assert np.abs(vg - vo).max() <= 1e-2
    assert force_error(Fg, Fo).max() <= 1e-3


# --------------------------------------------------------------------------
# Determinism, chunking and checkpoints


def test_chunking_and_runs_are_bit_identical(P):
    sc = small(wl.config3(), 3000)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as a:
        a.step(37)
        xa, va, Fa, _ = a.state()
    with P.Sim(sc, x, v, types) as b:
        for k in (5, 16, 1, 15):
            b.step(k)
        xb, vb, Fb, st = b.state()
    assert st == 37
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(Fa, Fb)


@pytest.mark.parametrize("which", ["lj_allpairs", "cell_list", "printed_cell", "full_sum"])
def test_checkpoint_resume_is_bit_exact(P, tmp_path, which):
    # the cell-list case carries neighbour lists (and their rebuilds) across the
    # checkpoint: kT = 4 makes the NPs fast enough to rebuild several times;
    # full_sum: the Coulomb sum over all pairs (sum_neutral) travels with the
    # file (resumed with the default neutral elision, the summation order and
    # so the bits would differ)
    sc = (small(wl.config2(), 1500) if which == "lj_allpairs"
          else with_(small(wl.config3(), 3000), kT=4.0))
    if which == "full_sum":
        sc = with_(sc, sum_neutral=True)
    if which == "printed_cell":  # the printed variants' parameters travel with the file
        sc = with_(sc, coulomb_cut=4.0, integrator=2, v_kick=0.05, wall_band=True)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as a:
        a.step(40)
        xa, va, _, _ = a.state()
    path = str(tmp_path / "ck.bin")
    with P.Sim(sc, x, v, types) as b:
        b.step(20)
        b.save(path)
    c = P.Sim.load(path, sc.n, sc)
    try:
        _, _, _, st = c.state()
        assert st == 20
        c.step(20)
        xc, vc, _, st = c.state()
        assert st == 40
    finally:
        c.close()
    assert np.array_equal(xa, xc) and np.array_equal(va, vc)


def _hi_words(P, sim, n):
    torch = pytest.importorskip("torch")
    xq = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    P.npsim_positions_device(sim.h, xq.data_ptr())
    torch.cuda.synchronize()
    return xq[:, :3].cpu().double().numpy()


def test_neighbour_lists_rebuild_and_stay_exact(P):
    """The cell-list LJ runs from Verlet lists rebuilt only after an NP has moved
    half the skin: after several rebuilds the LJ forces still equal the
    oracle's at the same (float32) positions."""
    sc = with_(wl.config1(), kT=3.0)
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    with P.Sim(sc, x, v, types) as sim:
        _, _, b0 = sim.nbr_info()
        sim.step(300)
        cap, mean_len, b1 = sim.nbr_info()
        F = sim.forces(2)
        xh = _hi_words(P, sim, sc.n)
    assert b1 - b0 >= 2 and mean_len > 0
    ref = _oracle_pair(sc, xh, types, coul=False)
    amb = cutoff_ambiguous(xh, types, sc)
    assert force_error(F, ref)[~amb].max() <= FORCE_TOL


def test_neighbour_list_overflow_is_exact_and_grows(P):
    """A compact lattice has more list partners per NP than the initial list
    holds: those NPs are summed from the cells (exact) and the list grows."""
    m, a = 12, 1.12
    g = (np.arange(m) - (m - 1) / 2) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x.astype(np.float32).astype(np.float64)
    n = len(x)
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.0, charge=0.0, gamma=1.0, k_wall=100.0)
    sc = wl.Scenario(name="lattice", types=[t], n=n, seed=4, dt=1e-3, kT=0.1, R0=40.0,
                     lj_mode=2, coulomb=False)
    ty = np.zeros(n, np.int32)
    with P.Sim(sc, x, None, ty) as sim:
        cap, mean_len, _ = sim.nbr_info()
        F0 = sim.forces(2)
        sim.step(40)
        F1 = sim.forces(2)
        xh = _hi_words(P, sim, n)
    assert mean_len > 32 and cap >= mean_len  # grown past the initial 32
    for F, xx in ((F0, x), (F1, xh)):
        ref = _oracle_pair(sc, xx, ty, coul=False)
        amb = cutoff_ambiguous(xx, ty, sc)
        assert force_error(F, ref)[~amb].max() <= FORCE_TOL


# --------------------------------------------------------------------------
# Statistics


def test_stats_parity(P):
    sc = small(wl.config3(), 6000)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as sim:
        sim.step(10)
        xg, _, _, _ = sim.state()
        st = sim.stats(r_max=10.0, n_bins=128, radial_bins=32, boxcount=True)
    R = oracle.radius(sc.R0, sc.k_evap, 10 * sc.dt)
    assert st["R"] == pytest.approx(R, rel=1e-14)
    c_o = oracle.pair_hist(xg, 10.0, 128)
    assert np.array_equal(st["rdf_counts"], c_o)
    _, g_o = oracle.rdf(xg, 10.0, 128, R)
    assert np.allclose(st["rdf_g"], g_o, rtol=1e-12, atol=0)
    rc_o, C_o = oracle.radial_concentration(xg, R, 32, R)
    assert np.array_equal(st["radial_counts"], rc_o)
    assert np.allclose(st["radial_c"], C_o, rtol=1e-12)
    Rg, Df, r0 = oracle.rg(xg, st["d_mean"])
    assert st["Rg"] == pytest.approx(Rg, rel=1e-12)
    assert st["Df_rg"] == pytest.approx(Df, rel=1e-10)
    assert np.allclose(st["center"], r0, rtol=1e-10, atol=1e-12)
    Dfb, nb = oracle.boxcount_df(xg, st["d_mean"], Rg)
    assert np.array_equal(st["nbox"], nb)
    assert st["Df_box"] == pytest.approx(Dfb, rel=1e-10)
    # the surface band is decided in float64 on both sides, at the library's R
    sig = [t.sigma for t in sc.types]
    assert st["n_surf"] == oracle.surface_count(xg, types, sig, st["R"])


def test_scattering_matches_oracle(P):
    """I(q) of Sec. 3.3 on the GPU from a simulated RDF, and the fractal form."""
    sc = small(wl.config3(), 4000)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as sim:
        sim.step(5)
        st = sim.stats(r_max=12.0, n_bins=96, boxcount=False)
    q = np.concatenate([[0.0, 1e-3, 0.02], np.linspace(0.1, 12.0, 61)])
    n_surf = max(st["n_surf"], 7)
    I, If = P.npsim_scattering(st["rdf_g"], 12.0, n_surf, q, Rg=st["Rg"], Df=st["Df_rg"])
    ref = oracle.scattering(st["rdf_g"], 12.0, n_surf, q)
    assert np.allclose(I, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())
    with np.errstate(divide="ignore"):
        frac = n_surf ** 2 * (q * st["Rg"]) ** (-st["Df_rg"])
    assert np.allclose(If[1:], frac[1:], rtol=1e-12)


def test_frame_recorder_matches_stepping(P):
    """Frames recorded every 5 steps (asynchronous copies) are the float32 position
    words and charges of the states reached by plain stepping, and recording
    leaves the trajectory bit-identical."""
    sc = small(wl.config3(), 3000)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as a:
        frames = a.record(23, every=5)           # after steps 5, 10, 15, 20; then 3 more
        xa, va, _, st = a.state()
    assert frames.shape == (4, sc.n, 4) and st == 23
    q = np.array([t.charge for t in sc.types], np.float32)[types]
    with P.Sim(sc, x, v, types) as b:
        for k in range(4):
            b.step(5)
            xb, _, _, _ = b.state()
            x32 = xb.astype(np.float32)           # the hi word is the float nearest x
            f = frames[k, :, :3]
            assert np.mean(f == x32) >= 0.9999
            assert np.all(np.abs(f - x32) <= np.spacing(np.abs(x32)))
            assert np.array_equal(frames[k, :, 3], q)
        b.step(3)
        xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_stats_surface_count_hand_placed(P):
    """N_surf on the GPU for NPs placed on both sides of both band edges."""
    ts = [wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.0, charge=0.0, gamma=1.0, k_wall=10.0),
          wl.TypeSpec(sigma=3.0, eps=1.0, mass=27.0, charge=0.0, gamma=1.0 / 9, k_wall=10.0)]
    cases = [(0, 9.4, 0), (0, 9.6, 1), (0, 10.0, 1), (0, 10.4, 1), (0, 10.6, 0),
             (1, 8.4, 0), (1, 8.6, 1), (1, 11.4, 1), (1, 11.6, 0), (1, 0.0, 0)]
    rng = np.random.default_rng(4)
    u = rng.standard_normal((len(cases), 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    ty = np.array([c[0] for c in cases], np.int32)
    x = u * np.array([c[1] for c in cases])[:, None]
    sc = wl.Scenario(name="band", types=ts, n=len(cases), R0=10.0, k_evap=0.0,
                     lj_mode=0, coulomb=False)
    with P.Sim(sc, x, None, ty) as sim:
        st = sim.stats(r_max=2.0, n_bins=4, boxcount=False)
    assert st["R"] == 10.0
    assert st["n_surf"] == sum(c[2] for c in cases) == 5


def test_stats_boxcount_lattice_on_gpu(P):
    """A filled cubic lattice gives N_box = (L/2^k)^3 and D_f = 3 on the GPU path."""
    L = 32
    g = (np.arange(L) - L / 2 + 0.5) * 1.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xl = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.0, charge=0.0, gamma=1.0, k_wall=0.0)
    sc = wl.Scenario(name="lattice", types=[t], n=len(xl), R0=100.0, wall=False,
                     lj_mode=0, coulomb=False)
    with P.Sim(sc, xl, None, np.zeros(len(xl), np.int32)) as sim:
        st = sim.stats(r_max=3.0, n_bins=30, boxcount=True)
    # 2 R_g = 2 sqrt(3 (L^2 - 1)/12) = 31.98: scales eps = 1 .. 16
    assert len(st["nbox"]) == 5
    for k in range(5):
        assert st["nbox"][k] == (L // 2 ** k) ** 3
    assert st["Df_box"] == pytest.approx(3.0, abs=0.02)


# --------------------------------------------------------------------------
# Edge cases


def test_single_and_two_particles(P):
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=2.0, charge=1.0, gamma=3.0, k_wall=40.0)
    sc = wl.Scenario(name="two", types=[t], n=2, seed=0, dt=0.01, kT=0.0, R0=2.0,
                     k_evap=1.0, bjerrum=0.5, coulomb=True, lj_mode=1, lj_cut=2.5)
    x0 = np.array([[0.0, 0.0, 0.9], [0.0, 0.0, -0.4]])
    v0 = np.array([[0.1, 0.0, 0.0], [0.0, 0.0, 0.2]])
    ty = np.zeros(2, np.int32)
    with P.Sim(sc, x0, v0, ty) as sim:
        assert force_error(sim.forces(0), oracle.total_forces(sc, x0, ty, 0.0)).max() < FORCE_TOL
        sim.step(3)
        xg, vg, _, _ = sim.state()
    xo, vo, _ = oracle.run(sc, x0, v0, ty, 0, 3)
    assert np.abs(xg - xo).max() < 1e-9
    sc1 = with_(sc, n=1)
    with P.Sim(sc1, x0[:1], v0[:1], ty[:1]) as sim:
        F = sim.forces(0)
        assert np.allclose(F, oracle.external_forces(sc1, x0[:1], ty[:1], 0.0), rtol=1e-14)
        assert np.all(sim.forces(1) == 0)
        sim.step(5)


@pytest.mark.parametrize("n", [511, 512, 513, 2047])
def test_ragged_sizes(P, n):
    sc = small(wl.config2(), n)
    types, x, v = wl.initial_state(sc, fp32_positions=True)
    with P.Sim(sc, x, v, types) as sim:
        F = sim.forces(1)
    amb = cutoff_ambiguous(x, types, sc)
    err = force_error(F, _oracle_pair(sc, x, types))[~amb]
    assert err.max() <= FORCE_TOL


def test_invalid_arguments_are_errors(P):
    sc = wl.config1()
    types, x, v = wl.initial_state(sc)
    with pytest.raises(P.NpsimError) as e:
        P.Sim(sc, x[:0], None, types[:0])
    assert e.value.code == -1
    bad = types.copy()
    bad[3] = 7
    with pytest.raises(P.NpsimError) as e:
        P.Sim(sc, x, v, bad)
    assert e.value.code == -1
    with pytest.raises(P.NpsimError):
        P.Sim(with_(sc, dt=0.0), x, v, types)


def test_band_wall_forces_match_oracle(P):
    """The printed step (iv) wall on the GPU: NPs of two sizes placed inside,
    across and beyond the band (-r, r) about the surface."""
    ts = [wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.0, charge=0.0, gamma=1.0, k_wall=40.0),
          wl.TypeSpec(sigma=3.0, eps=1.0, mass=27.0, charge=0.0, gamma=1.0 / 9, k_wall=90.0)]
    rng = np.random.default_rng(8)
    n = 400
    ty = (np.arange(n) % 2).astype(np.int32)
    rad = 10.0 + rng.uniform(-2.5, 2.5, n)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    x = wl.fp32_representable(u * rad[:, None])
    for band in (False, True):
        sc = wl.Scenario(name="band", types=ts, n=n, R0=10.0, k_evap=0.0, lj_mode=0,
                         coulomb=False, g=0.3, wall_band=band)
        with P.Sim(sc, x, None, ty) as sim:
            F = sim.forces(0)
        ref = oracle.total_forces(sc, x, ty, 0.0)
        assert force_error(F, ref).max() <= FORCE_TOL, band


def test_printed_kick_has_fixed_magnitude_gpu(P):
    """Printed step (vi) on the GPU with gamma = 0 and no force: one step from
    rest gives |v| = v_kick for every NP, in the oracle's directions."""
    n, A = 4096, 0.3
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.5, charge=0.0, gamma=0.0, k_wall=0.0)
    sc = wl.Scenario(name="kick", types=[t], n=n, seed=23, kT=0.0, R0=1e9, wall=False,
                     lj_mode=0, coulomb=False, integrator=2, v_kick=A)
    ty = np.zeros(n, np.int32)
    x0 = np.zeros((n, 3))
    with P.Sim(sc, x0, None, ty) as sim:
        sim.step(1)
        _, v, _, _ = sim.state()
    assert np.allclose(np.linalg.norm(v, axis=1), A, rtol=1e-6)
    _, vo, _ = oracle.run(sc, x0, np.zeros((n, 3)), ty, 0, 1)
    # directions: the float32 Box-Muller normals differ from the float64 ones by
    # ~1e-7 relative, rarely ~1e-5 at small radii (test_normals_match_oracle)
    assert np.abs(v - vo).max() <= 2e-5 * A
    assert np.median(np.abs(v - vo)) <= 1e-6 * A


def test_free_particles_msd_and_equipartition_gpu(P):
    """Same closed forms as the oracle pins, on the GPU integrator."""
    n, steps = 20000, 300
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.5, charge=0.0, gamma=2.0, k_wall=0.0)
    sc = wl.Scenario(name="free", types=[t], n=n, seed=21, dt=2e-3, kT=1.3, R0=1e9,
                     wall=False, lj_mode=0, coulomb=False)
    ty = np.zeros(n, np.int32)
    x0 = np.zeros((n, 3))
    v0 = wl.maxwell_velocities(sc, ty, seed=1)
    with P.Sim(sc, x0, v0, ty) as sim:
        sim.step(steps)
        x, v, _, _ = sim.state()
    T = steps * sc.dt
    D = 1.3 / (1.5 * 2.0)
    msd_th = 6 * D * (T - (1 - math.exp(-2.0 * T)) / 2.0)
    d2 = (x ** 2).sum(1)
    assert abs(d2.mean() - msd_th) < 4 * d2.std() / math.sqrt(n) + 0.01 * msd_th
    ke = 1.5 * (v ** 2).sum(1) / 3
    assert abs(ke.mean() - 1.3) < 4 * ke.std() / math.sqrt(n)
    xo, vo, _ = oracle.run(sc, x0, v0, ty, 0, steps)
    # Velocities are float32 on the device: each step rounds v by <= 2^-24 |v|
    # (|v| <= ~5 here), and the Langevin damping remembers a velocity error for
    # ~1/(gamma dt) = 250 steps, so v differs from the float64 oracle by ~1e-6 and
    # x = sum of v dt by a few 1e-6 at most over 300 steps (the 100-step
    # position bound of the method is 1e-4 sigma).
    assert np.abs(v - vo).max() < 1e-5
    assert np.abs(x - xo).max() < 1e-5


def test_position_keeps_increments_below_float32_resolution(P):
    """Positions are hi + lo float pairs: a drift of 1e-7 sigma per step along z
    at z in [150, 250] sigma, 76x below half a float32 ulp there (7.6e-6), must
    accumulate as in float64; a plain float32 position would not move."""
    n, steps = 1024, 2000
    t = wl.TypeSpec(sigma=1.0, eps=0.0, mass=1.0, charge=0.0, gamma=1.0, k_wall=0.0)
    sc = wl.Scenario(name="drift", types=[t], n=n, seed=5, dt=1e-3, kT=0.0, g=1e-4,
                     R0=1e9, wall=False, lj_mode=0, coulomb=False, integrator=1)
    rng = np.random.default_rng(3)
    x0 = np.column_stack([rng.uniform(-250, 250, n), rng.uniform(-250, 250, n),
                          rng.uniform(150, 250, n)])
    x0 = x0.astype(np.float32).astype(np.float64)
    ty = np.zeros(n, np.int32)
    with P.Sim(sc, x0, None, ty) as sim:
        sim.step(steps)
        x, _, _, st = sim.state()
    assert st == steps
    xo, _, _ = oracle.run(sc, x0, np.zeros_like(x0), ty, 0, steps)
    dz, dzo = x[:, 2] - x0[:, 2], xo[:, 2] - x0[:, 2]
    # float64 oracle: 2000 adds at |z| <= 250 round by <= 2000 * 1.5e-14
    assert np.allclose(dzo, -steps * sc.dt * sc.g / t.gamma, rtol=1e-6, atol=0)
    # the per-step increment is rounded to float32 (~6e-8 relative) and each
    # compensated add is exact to ~2^-48 |x|: 2000 adds at |x| <= 250 give < 2e-9
    assert np.abs(dz - dzo).max() <= 1e-8
    assert np.array_equal(x[:, :2], x0[:, :2])


def test_nonfinite_position_is_reported(P):
    sc = small(wl.config2(), 600)
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as sim:
        xb = x.copy()
        xb[5] = [1e300, 0.0, 0.0]  # float32 mirror overflows -> non-finite forces
        sim.set_state(xb, v, 0)
        with pytest.raises(P.NpsimError) as e:
            sim.step(2)
        assert e.value.code == -3


def test_escaped_np_is_reported(P):
    """With the full interface spring on, an NP farther than 2 max(R0, R(t))
    from the centre (where only an unstable step could have left it) makes npsim_step
    return NPSIM_ERR_ESCAPED; the steps were still taken and the word is
    cleared, so the next steps (the spring pulling the NP back in) succeed.
    Without the spring the same position is no error."""
    sc = wl.config1()
    types, x, v = wl.initial_state(sc)
    xb = x.copy()
    xb[7] = [3.0 * sc.R0, 0.0, 0.0]
    with P.Sim(sc, x, v, types) as sim:
        sim.set_state(xb, v, 0)
        with pytest.raises(P.NpsimError) as e:
            sim.step(2)
        assert e.value.code == -8
        assert sim.state()[3] == 2
        x2 = sim.state()[0]
        assert np.linalg.norm(x2[7]) < 3.0 * sc.R0  # pulled back towards the droplet
    with P.Sim(with_(sc, wall=False), xb, v, types) as sim:
        sim.step(2)
        assert sim.state()[3] == 2


def test_cell_grid_follows_the_shrinking_droplet(P):
    """The droplet of config 1 shrinks from R = 30 to 20: at step 1024 the cell
    grid (sized at creation for R0) is more than a quarter too wide and is
    replaced by one sized for R(t).  After the regrid the LJ forces still equal
    the oracle's at the same float32 positions, and the steps are cut at the
    regrid period whatever the calls' sizes, so 1500 steps in one call equal
    700 + 800 bit for bit."""
    sc = wl.config1()
    types, x, v = wl.initial_state(sc)
    with P.Sim(sc, x, v, types) as a:
        dim0, _ = a.cell_grid()
        a.step(1500)
        dim1, _ = a.cell_grid()
        xa, va, _, st = a.state()
        F = a.forces(2)
        xh = _hi_words(P, a, sc.n)
    assert st == 1500 and dim1 < dim0
    ref = _oracle_pair(sc, xh, types, coul=False)
    amb = cutoff_ambiguous(xh, types, sc)
    assert force_error(F, ref)[~amb].max() <= FORCE_TOL
    with P.Sim(sc, x, v, types) as b:
        b.step(700)
        b.step(800)
        xb, vb, _, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
