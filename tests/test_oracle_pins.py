"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these tests re-derives the oracle's own formula: each compares the
oracle with something independent of it -- a published generator run from a
library, a closed form, a potential whose numerical derivative must equal the
force, a conservation law, an exact symmetry, brute-force integer counting, or
a statistical law with its standard error.  A dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import ctypes
import ctypes.util
import json
import math
import os

import numpy as np
import pytest

import oracle
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# --------------------------------------------------------------------------
# Philox4x32-10


def _curand_host():
    for name in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand"),
                 "libcurand.so.10", "libcurand.so"):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """cuRAND's host Philox4_32_10 generator keyed by the 64-bit seed emits, as its
    b-th block of four words, Philox4x32-10 of counter (0, 0, b, 0); the oracle must
    reproduce 16384 such blocks bit for bit."""
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        for seed in (0, 0x123456789, 0xFEDCBA9876543210):
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(0)) == 0
            n = 4 * 16384
            out = np.zeros(n, np.uint32)
            assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_size_t(n)) == 0
            out = out.reshape(-1, 4)
            for b in list(range(64)) + list(range(16384 - 64, 16384)):
                mine = oracle.philox_blocks(seed, [0, 0, b, 0], 1)[0]
                assert np.array_equal(mine, out[b]), (seed, b)
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_uniform_and_counter_sensitivity():
    u = oracle.philox_blocks(7, [0, 0, 0, 0], 1 << 15).ravel()
    # chi-square on the top 8 bits, 255 dof: mean 255, sd ~22.6
    h = np.bincount(u >> 24, minlength=256)
    e = len(u) / 256
    chi2 = ((h - e) ** 2 / e).sum()
    assert 150 < chi2 < 380
    # every output bit flips with probability ~1/2 when one counter bit flips
    a = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for word in range(4):
        for bit in (0, 13, 31):
            c = [1, 2, 3, 4]
            c[word] ^= 1 << bit
            b = oracle.philox4x32_10(c, [5, 6])
            flips = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b))
            assert 30 < flips < 98


def test_philox_block_helper_carry():
    """Block helper: counter word 0 carries into word 1."""
    a = oracle.philox_blocks(3, [0xFFFFFFFF, 5, 6, 7], 2)
    assert np.array_equal(a[0], oracle.philox4x32_10([0xFFFFFFFF, 5, 6, 7], [3, 0]))
    assert np.array_equal(a[1], oracle.philox4x32_10([0, 6, 6, 7], [3, 0]))


def test_normals_moments_and_cdf():
    from scipy import stats
    z = oracle.normals(11, 5, 0, 40000)
    flat = z.ravel()
    n = len(flat)
    assert abs(flat.mean()) < 4 / math.sqrt(n)
    assert abs(flat.var() - 1) < 4 * math.sqrt(2 / n)
    assert abs(stats.kurtosis(flat)) < 4 * math.sqrt(24 / n)
    for k in range(3):
        assert stats.kstest(z[:, k], "norm").pvalue > 1e-4
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c - np.eye(3)) < 4 / math.sqrt(len(z)))
    # distinct streams for another step / purpose / seed
    assert not np.allclose(z[:100], oracle.normals(11, 6, 0, 100))
    assert not np.allclose(z[:100], oracle.normals(11, 5, 1, 100))
    assert not np.allclose(z[:100], oracle.normals(12, 5, 0, 100))


def test_normals_are_box_muller_of_the_stream():
    """Row i of step s is the Box-Muller image of block philox((i, s_lo, s_hi, p), seed)."""
    seed, step, purpose = 0xABCDEF0123, (1 << 33) + 17, 0
    z = oracle.normals(seed, step, purpose, 8)
    for i in range(8):
        r = oracle.philox4x32_10([i, step & 0xFFFFFFFF, step >> 32, purpose],
                                 [seed & 0xFFFFFFFF, seed >> 32]).astype(np.float64)
        u = (r + 0.5) / 2.0 ** 32
        # the polar radius of (n0, n1) recovers u0; the angle recovers u1
        assert math.isclose(z[i, 0] ** 2 + z[i, 1] ** 2, -2 * math.log(u[0]), rel_tol=1e-12)
        ang = math.atan2(z[i, 1], z[i, 0]) % (2 * math.pi)
        assert math.isclose(ang, 2 * math.pi * u[1], rel_tol=1e-10, abs_tol=1e-10)
        assert abs(z[i, 2]) <= math.sqrt(-2 * math.log(u[2])) + 1e-12


# --------------------------------------------------------------------------
# Forces


def _lj_U(r, s, e):
    return 4 * e * ((s / r) ** 12 - (s / r) ** 6)


def _two_body(r, t=(0, 0), sigma=(1.0, 1.0), eps=(1.0, 1.0), q=(0.0, 0.0), lb=0.0,
              lj=True, coul=False, cut=2.5, ov=None):
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    F = oracle.pair_forces(x, np.array(t), sigma, eps, q, lb, lj_cut=cut, lj=lj,
                           coulomb=coul, eps_override=ov)
    return F


def test_lj_two_body_zero_at_minimum_and_sign():
    rmin = 2 ** (1 / 6)
    F = _two_body(rmin)
    assert abs(F[0, 0]) < 1e-12 and abs(F[1, 0]) < 1e-12
    assert _two_body(0.95 * rmin)[1, 0] > 0  # repulsive: particle 1 pushed to +x
    assert _two_body(1.05 * rmin)[1, 0] < 0  # attractive
    # mixed pair: minimum at 2^(1/6) sigma_ab
    smix = 0.5 * (1.0 + 3.0)
    F = _two_body(rmin * smix, t=(0, 1), sigma=(1.0, 3.0), eps=(1.0, 2.0))
    assert abs(F[1, 0]) < 1e-12


@pytest.mark.parametrize("r", [0.9, 1.0, 1.5, 2.0, 2.49])
def test_lj_two_body_equals_minus_dU_dr(r):
    """Force = -dU/dr of 4 eps ((s/r)^12 - (s/r)^6), by a central difference."""
    s, e = 1.25, 0.7
    h = 1e-6
    dU = (_lj_U(r * s / 1.25 + h, s, e) - _lj_U(r * s / 1.25 - h, s, e)) / (2 * h)
    F = _two_body(r * s / 1.25, sigma=(s, s), eps=(e, e))
    assert F[1, 0] == pytest.approx(-dU, rel=1e-7, abs=1e-9)
    assert F[0, 0] == pytest.approx(dU, rel=1e-7, abs=1e-9)


def test_lj_truncated_not_shifted():
    """Zero at and beyond r_c = 2.5 sigma_ab; the full (nonzero) force just inside."""
    assert np.all(_two_body(2.5000001) == 0)
    assert np.all(_two_body(3.0) == 0)
    inside = _two_body(2.4999999)[1, 0]
    h = 1e-6
    dU = (_lj_U(2.4999999 + h, 1, 1) - _lj_U(2.4999999 - h, 1, 1)) / (2 * h)
    assert inside == pytest.approx(-dU, rel=1e-6)
    # cutoff follows sigma_ab: a 1-3 pair (sigma_ab = 2) still interacts at 4.9
    F = _two_body(4.9, t=(0, 1), sigma=(1.0, 3.0))
    assert F[1, 0] != 0
    assert np.all(_two_body(5.01, t=(0, 1), sigma=(1.0, 3.0)) == 0)


def test_eps_override_matrix():
    """The Table 1 / Fig. 9 epsilon matrix replaces the mixing rule (scales the force)."""
    ov = np.array([[0.155, 1.26], [1.26, 0.155]])
    F1 = _two_body(1.5, t=(0, 1), sigma=(1.0, 1.0), ov=ov)
    F2 = _two_body(1.5, t=(0, 1), sigma=(1.0, 1.0), eps=(1.0, 1.0))
    assert F1[1, 0] == pytest.approx(1.26 * F2[1, 0], rel=1e-14)
    s, e, rc = oracle.mix_tables([1.0, 3.0], [1.0, 4.0], None, 2.5)
    assert np.allclose(s, [[1, 2], [2, 3]]) and np.allclose(e, [[1, 2], [2, 4]])
    assert np.allclose(rc, 2.5 * s)


@pytest.mark.parametrize("r", [0.8, 3.0, 17.0])
def test_coulomb_two_body_inverse_square(r):
    q = (0.5, -2.0)
    lb = 0.7
    F = _two_body(r, t=(0, 1), q=q, lb=lb, lj=False, coul=True)
    # -dU/dr of U = lb q1 q2 / r
    h = 1e-6 * r
    dU = (lb * q[0] * q[1] / (r + h) - lb * q[0] * q[1] / (r - h)) / (2 * h)
    assert F[1, 0] == pytest.approx(-dU, rel=1e-7)
    assert F[1, 0] < 0  # opposite charges attract
    F2 = _two_body(2 * r, t=(0, 1), q=q, lb=lb, lj=False, coul=True)
    assert F2[1, 0] == pytest.approx(F[1, 0] / 4, rel=1e-13)
    assert np.all(F[:, 1:] == 0)


@pytest.mark.parametrize("frac,inside", [(0.5, True), (0.999, True), (1.001, False),
                                           (1.5, False)])
def test_coulomb_truncated_two_body(frac, inside):
    """Truncated Coulomb (the printed range 4 sigma_ab, not shifted): inside the
    range the force is the full C q1 q2 / r^2, beyond it exactly 0; sigma_ab of
    a 1-3 pair is 2, so the range is 8."""
    q, lb, cut = (0.5, -2.0), 0.7, 4.0
    sig = (1.0, 3.0)
    r = frac * cut * 2.0
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    F = oracle.pair_forces(x, np.array([0, 1]), sig, (1.0, 1.0), q, lb, lj=False,
                           coulomb=True, coulomb_cut=cut)
    expect = lb * q[0] * q[1] / (r * r) if inside else 0.0
    assert F[1, 0] == pytest.approx(expect, rel=1e-13, abs=1e-300)
    assert F[0, 0] == -F[1, 0]


def test_coulomb_truncated_cluster_newton_and_subset():
    """Truncated Coulomb on a random cluster: Newton's third law holds and every
    pair's contribution is either the untruncated one (r < 4 sigma_ab) or 0,
    checked by removing the far pairs one NP at a time."""
    rng = np.random.default_rng(6)
    n = 40
    x = rng.uniform(-6, 6, (n, 3))
    ty = rng.integers(0, 2, n).astype(np.int32)
    sig, q = (1.0, 3.0), (0.7, -0.4)
    Ft = oracle.pair_forces(x, ty, sig, (1.0, 1.0), q, 0.7, lj=False, coulomb=True,
                            coulomb_cut=4.0)
    assert np.abs(Ft.sum(0)).max() <= 1e-12 * np.abs(Ft).sum()
    s = np.array(sig)
    for i in range(0, n, 7):
        d = np.linalg.norm(x - x[i], axis=1)
        near = d < 4.0 * 0.5 * (s[ty[i]] + s[ty])
        keep = near.copy()
        keep[i] = True
        Fi = oracle.pair_forces(x[keep], ty[keep], sig, (1.0, 1.0), q, 0.7, lj=False,
                                coulomb=True)            # untruncated, near partners only
        assert np.allclose(Ft[i], Fi[np.flatnonzero(keep).tolist().index(i)], rtol=1e-12,
                           atol=1e-14)


def test_coulomb_ring_axis_exact():
    """M equal charges on a ring of radius a: on the axis at height z the force is
    exactly C q Q z / (a^2 + z^2)^(3/2) along z (transverse parts cancel)."""
    M, a, z, lb = 12, 3.0, 1.7, 0.7
    ang = 2 * np.pi * np.arange(M) / M
    ring = np.stack([a * np.cos(ang), a * np.sin(ang), np.zeros(M)], 1)
    x = np.vstack([ring, [[0, 0, z]]])
    t = np.array([0] * M + [1])
    F = oracle.pair_forces(x, t, [1, 1], [1, 1], [0.5, 2.0], lb, lj=False, coulomb=True)
    Q = 0.5 * M
    expect = lb * 2.0 * Q * z / (a * a + z * z) ** 1.5
    assert F[M, 2] == pytest.approx(expect, rel=1e-13)
    assert abs(F[M, 0]) < 1e-13 and abs(F[M, 1]) < 1e-13


def _random_cluster(n, seed, R=4.0, T=3):
    rng = np.random.default_rng(seed)
    sc = wl.Scenario(name="t", types=[wl.stokes_type(1.0, 0.3, frac=0.5),
                                      wl.stokes_type(1.5, -0.6, frac=0.3),
                                      wl.stokes_type(2.0, 1.0, frac=0.2)][:T],
                     n=n, seed=seed, R0=R)
    ty = wl.assign_types(sc)
    x = wl.place(sc, ty)
    return sc, ty, x


def test_newton_third_law():
    sc, ty, x = _random_cluster(300, 5, R=10.0)
    sig = [t.sigma for t in sc.types]
    eps = [1.0, 0.5, 2.0]
    q = [t.charge for t in sc.types]
    F = oracle.pair_forces(x, ty, sig, eps, q, 0.7)
    assert np.abs(F.sum(0)).max() <= 1e-12 * np.abs(F).sum()


def test_forces_are_minus_gradient_of_potential():
    """F_i = -dU/dx_i for U = sum_{i<j} [C q_i q_j / r + 4 eps (...) [r < rc]],
    by central differences on a configuration with no pair near the cutoff."""
    sc, ty, x = _random_cluster(40, 9, R=4.5)
    sig = np.array([t.sigma for t in sc.types])
    eps = np.array([1.0, 0.5, 2.0])
    q = np.array([t.charge for t in sc.types])
    lb = 0.7

    def U(xx):
        tot = 0.0
        for i in range(len(xx)):
            for j in range(i + 1, len(xx)):
                r = np.linalg.norm(xx[i] - xx[j])
                s = 0.5 * (sig[ty[i]] + sig[ty[j]])
                e = math.sqrt(eps[ty[i]] * eps[ty[j]])
                tot += lb * q[ty[i]] * q[ty[j]] / r
                if r < 2.5 * s:
                    tot += _lj_U(r, s, e)
        return tot

    # keep the test away from the LJ discontinuity at the cutoff
    d = np.linalg.norm(x[:, None] - x[None], axis=-1)
    S = 0.5 * (sig[ty][:, None] + sig[ty][None])
    assert np.all(np.abs(d - 2.5 * S)[~np.eye(len(x), dtype=bool)] > 1e-3)
    F = oracle.pair_forces(x, ty, sig, eps, q, lb)
    h = 1e-6
    for i in (0, 7, 23, 39):
        for k in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            g = (U(xp) - U(xm)) / (2 * h)
            assert F[i, k] == pytest.approx(-g, rel=2e-5, abs=2e-5 * np.abs(F).max())


def test_forces_rotate_with_configuration():
    sc, ty, x = _random_cluster(120, 3, R=8.0)
    sig = [t.sigma for t in sc.types]
    q = [t.charge for t in sc.types]
    from scipy.spatial.transform import Rotation
    Rm = Rotation.from_euler("zyx", [0.3, -1.1, 2.0]).as_matrix()
    F = oracle.pair_forces(x, ty, sig, [1, 1, 1], q, 0.7)
    Fr = oracle.pair_forces(x @ Rm.T, ty, sig, [1, 1, 1], q, 0.7)
    assert np.allclose(Fr, F @ Rm.T, rtol=1e-9, atol=1e-10 * np.abs(F).max())


def test_selected_rows_equal_full_rows():
    sc, ty, x = _random_cluster(200, 4, R=9.0)
    sig = [t.sigma for t in sc.types]
    q = [t.charge for t in sc.types]
    F = oracle.pair_forces(x, ty, sig, [1, 1, 1], q, 0.7)
    sel = np.array([199, 0, 57, 57, 3])
    Fs = oracle.pair_forces(x, ty, sig, [1, 1, 1], q, 0.7, sel=sel)
    assert np.array_equal(Fs, F[sel])


# --------------------------------------------------------------------------
# Radius law and external forces


def test_radius_square_law():
    R0, k = 30.0, 500.0
    for t in (0.0, 0.3, 1.0):
        assert oracle.radius(R0, k, t) == pytest.approx(math.sqrt(R0 * R0 - k * t), rel=1e-15)
    assert oracle.radius(R0, k, 1.0) == pytest.approx(20.0, rel=1e-15)  # 900 - 500 = 400
    assert oracle.radius(R0, k, 10.0) == 0.0          # dried up
    assert oracle.radius(R0, -100.0, 5.0) > R0        # condensation grows the droplet
    sc = wl.config1()
    assert oracle.radius(sc.R0, sc.k_evap, sc.n_steps * sc.dt) == pytest.approx(20.0, rel=1e-12)


def _one_type_scenario(**kw):
    t = wl.TypeSpec(sigma=2.0, eps=1.0, mass=3.0, charge=0.0, gamma=1.0, k_wall=50.0)
    base = dict(name="ext", types=[t], n=1, R0=10.0, k_evap=0.0, wall=True)
    base.update(kw)
    return wl.Scenario(**base)


def test_wall_spring_closed_form():
    sc = _one_type_scenario()
    R, r_np = 10.0, 1.0
    for rad in (8.5, 9.0, 9.5, 12.0):
        u = np.array([0.48, -0.6, 0.64])
        x = (rad * u)[None]
        F = oracle.external_forces(sc, x, np.zeros(1, np.int32), 0.0)
        s = rad - (R - r_np)
        expect = -50.0 * max(s, 0.0) * u
        assert np.allclose(F[0], expect, rtol=1e-14, atol=1e-14)
    # the equilibrium point follows R(t)
    sc2 = _one_type_scenario(k_evap=10.0)
    t = 1.9
    Rt = math.sqrt(100 - 10 * t)
    x = np.array([[0, 0, Rt - r_np + 0.25]])
    F = oracle.external_forces(sc2, x, np.zeros(1, np.int32), t)
    assert F[0, 2] == pytest.approx(-50.0 * 0.25, rel=1e-12)


def test_band_wall_closed_form():
    """wall_band: the spring acts only within the band (-r, r) about the surface,
    i.e. for 0 < s < sigma with s = |x| - (R - r); beyond it the force is 0, where
    the default wall keeps pulling (-k s x/|x|)."""
    import dataclasses
    sc1 = _one_type_scenario()                       # sigma 2, k_wall 50, R 10
    sc2 = dataclasses.replace(sc1, wall_band=True)
    u = np.array([0.48, -0.6, 0.64])
    for rad, in_band in ((8.5, False), (9.5, True), (10.5, True), (10.99, True),
                         (11.01, False), (11.5, False)):
        x = (rad * u)[None]
        s = rad - 9.0
        full = -50.0 * max(s, 0.0) * u
        F1 = oracle.external_forces(sc1, x, np.zeros(1, np.int32), 0.0)[0]
        F2 = oracle.external_forces(sc2, x, np.zeros(1, np.int32), 0.0)[0]
        assert np.allclose(F1, full, rtol=1e-14, atol=1e-14)
        assert np.allclose(F2, full if in_band else 0.0 * u, rtol=1e-14, atol=1e-14)


def test_gravity_and_centrifugal_closed_form():
    x = np.array([[1.0, -2.0, 3.0]])
    ty = np.zeros(1, np.int32)
    F = oracle.external_forces(_one_type_scenario(wall=False, g=0.5), x, ty, 0.0)
    assert np.allclose(F[0], [0, 0, -1.5])
    F = oracle.external_forces(_one_type_scenario(wall=False, omega=0.2, rot_mode=1), x, ty, 0.0)
    assert np.allclose(F[0], 3.0 * 0.04 * np.array([1.0, -2.0, 0.0]), rtol=1e-14)
    F = oracle.external_forces(_one_type_scenario(wall=False, omega=0.2, rot_mode=2), x, ty, 0.0)
    assert np.allclose(F[0], 3.0 * 0.04 * x[0], rtol=1e-14)


# --------------------------------------------------------------------------
# Integrator


def _free_scenario(n, integrator=0, g=0.0, omega=0.0, rot_mode=0, dt=2e-3, gamma=2.0,
                   mass=1.5, kT=1.3):
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=mass, charge=0.0, gamma=gamma, k_wall=0.0)
    return wl.Scenario(name="free", types=[t], n=n, seed=21, dt=dt, kT=kT, R0=1e9,
                       wall=False, lj_mode=0, coulomb=False, integrator=integrator, g=g,
                       omega=omega, rot_mode=rot_mode)


def test_free_particle_msd_and_equipartition_baoab():
    """No forces: MSD(t) = 6 (kT/(m gamma)) [t - (1 - e^{-gamma t})/gamma] for Maxwellian
    v0, and <m v^2>/3 = kT at every step (the O step is exact)."""
    n, steps = 20000, 300
    sc = _free_scenario(n)
    m, gam, kT = 1.5, 2.0, 1.3
    ty = np.zeros(n, np.int32)
    x0 = np.zeros((n, 3))
    v0 = wl.maxwell_velocities(sc, ty, seed=1)
    x, v, _ = oracle.run(sc, x0, v0, ty, 0, steps)
    t = steps * sc.dt
    D = kT / (m * gam)
    msd_th = 6 * D * (t - (1 - math.exp(-gam * t)) / gam)
    d2 = ((x - x0) ** 2).sum(1)
    se = d2.std() / math.sqrt(n)
    assert abs(d2.mean() - msd_th) < 4 * se + 0.01 * msd_th  # BAOAB O(dt^2) bias
    ke = (m * (v ** 2).sum(1) / 3)
    assert abs(ke.mean() - kT) < 4 * ke.std() / math.sqrt(n)


def test_free_particle_msd_overdamped():
    """Overdamped: MSD = 6 D t exactly in distribution, D = kT/(m gamma)."""
    n, steps = 20000, 50
    sc = _free_scenario(n, integrator=1, dt=1e-2)
    ty = np.zeros(n, np.int32)
    x0 = np.zeros((n, 3))
    x, _, _ = oracle.run(sc, x0, np.zeros((n, 3)), ty, 0, steps)
    D = 1.3 / (1.5 * 2.0)
    d2 = ((x - x0) ** 2).sum(1)
    assert abs(d2.mean() - 6 * D * steps * sc.dt) < 4 * d2.std() / math.sqrt(n)


def test_sedimentation_and_centrifugal_drift():
    """Constant force -m g: terminal <v_z> = -g/gamma.  Overdamped rotation about z:
    radial drift d<rho>/dt = omega^2 rho / gamma (linear in rho, so exact on average)."""
    n = 20000
    sc = _free_scenario(n, g=0.8, dt=5e-3)
    ty = np.zeros(n, np.int32)
    v0 = wl.maxwell_velocities(sc, ty, seed=2)
    _, v, _ = oracle.run(sc, np.zeros((n, 3)), v0, ty, 0, 1500)  # t = 7.5 = 15/gamma
    assert abs(v[:, 2].mean() + 0.8 / 2.0) < 4 * v[:, 2].std() / math.sqrt(n)
    sc = _free_scenario(n, integrator=1, omega=0.5, rot_mode=1, dt=1e-3, kT=0.0)
    x0 = np.tile([[2.0, 0.0, 1.0]], (n, 1))
    x, _, _ = oracle.run(sc, x0, np.zeros((n, 3)), ty, 0, 200)
    # d rho/dt = omega^2 rho / gamma -> rho(t) = rho0 exp(omega^2 t / gamma) (Euler: (1+h)^k)
    h = 0.25 * 1e-3 / 2.0
    assert x[0, 0] == pytest.approx(2.0 * (1 + h) ** 200, rel=1e-12)
    assert x[0, 2] == pytest.approx(1.0, rel=1e-15)


def _boltzmann_wall_cdf(R_eff, k, kT):
    """CDF of the radius for an ideal gas held by the one-sided interface spring:
    p(r) ~ r^2 exp(-k max(r - R_eff, 0)^2 / (2 kT)), by trapezoidal quadrature."""
    w = math.sqrt(kT / k)
    r = np.linspace(0.0, R_eff + 12.0 * w, 400001)
    p = r * r * np.exp(-0.5 * np.maximum(r - R_eff, 0.0) ** 2 / (w * w))
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (p[1:] + p[:-1]) * np.diff(r))])
    return r, cdf / cdf[-1], w


@pytest.mark.parametrize("integrator,dt", [(1, 1e-3), (0, 2e-3)])
def test_wall_ideal_gas_keeps_boltzmann_radial_density(integrator, dt):
    """An ideal gas (no pair forces) in a static droplet has Boltzmann's stationary
    radial density under the interface spring (Sec. 2.2 step (iv)): flat inside
    R - sigma/2, a Gaussian tail of width sqrt(kT/k_wall) beyond it.  Sampled from
    that law, the gas must stay in it: a wrong spring constant, sign or noise
    amplitude moves the tail within a few gamma/k_wall (here 0.1 of the 2 time
    units run).  Checked by a chi-square over radial bins and the tail fraction."""
    n, k, kT, R, sigma = 20000, 10.0, 1.0, 3.0, 1.0
    R_eff = R - sigma / 2
    t = wl.TypeSpec(sigma=sigma, eps=0.0, mass=1.0, charge=0.0, gamma=1.0, k_wall=k)
    sc = wl.Scenario(name="gas", types=[t], n=n, seed=5, dt=dt, kT=kT, R0=R, k_evap=0.0,
                     wall=True, lj_mode=0, coulomb=False, integrator=integrator)
    grid, cdf, w = _boltzmann_wall_cdf(R_eff, k, kT)
    rng = np.random.default_rng(11)
    rad = np.interp(rng.random(n), cdf, grid)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    ty = np.zeros(n, np.int32)
    v0 = wl.maxwell_velocities(sc, ty, seed=3) if integrator == 0 else np.zeros((n, 3))
    x, _, _ = oracle.run(sc, rad[:, None] * u, v0, ty, 0, int(round(2.0 / dt)))
    r = np.linalg.norm(x, axis=1)
    edges = np.array([0.0, R_eff - 1.0, R_eff - 0.5, R_eff - 0.25, R_eff, R_eff + 0.5 * w,
                      R_eff + w, R_eff + 1.5 * w, R_eff + 2.0 * w, R_eff + 3.0 * w, np.inf])
    prob = np.diff(np.interp(edges, grid, cdf, right=1.0))
    obs = np.histogram(r, bins=edges)[0]
    chi2 = float((((obs - n * prob) ** 2) / (n * prob)).sum())
    dof = len(prob) - 1
    assert chi2 < dof + 6.0 * math.sqrt(2.0 * dof), (chi2, obs, n * prob)
    p_out = 1.0 - float(np.interp(R_eff, grid, cdf))
    se = math.sqrt(p_out * (1.0 - p_out) / n)
    assert abs((r > R_eff).mean() - p_out) < 5.0 * se


def _kick_scenario(n, v_kick, gamma, g=0.0, dt=2e-3, mass=1.5):
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=mass, charge=0.0, gamma=gamma, k_wall=0.0)
    return wl.Scenario(name="kick", types=[t], n=n, seed=23, dt=dt, kT=0.0, R0=1e9,
                       wall=False, lj_mode=0, coulomb=False, integrator=2,
                       v_kick=v_kick, g=g)


def test_printed_step_drag_closed_form():
    """Printed step (vi) without kick: v_{k+1} = (1 - gamma dt) v_k, so
    v_n = q^n v_0 and x_n = x_0 + dt v_0 q (1 - q^n)/(1 - q), q = 1 - gamma dt;
    under a constant force -m g the terminal velocity -g/gamma is a fixed point."""
    n_p, steps, gam, dt = 50, 300, 2.0, 2e-3
    sc = _kick_scenario(n_p, 0.0, gam, dt=dt)
    rng = np.random.default_rng(3)
    x0, v0 = rng.standard_normal((n_p, 3)), rng.standard_normal((n_p, 3))
    ty = np.zeros(n_p, np.int32)
    x, v, _ = oracle.run(sc, x0, v0, ty, 0, steps)
    q = 1.0 - gam * dt
    assert np.allclose(v, v0 * q ** steps, rtol=1e-12, atol=1e-15)
    assert np.allclose(x, x0 + dt * v0 * q * (1 - q ** steps) / (1 - q), rtol=1e-11, atol=1e-13)
    sc = _kick_scenario(n_p, 0.0, gam, g=0.8, dt=dt)
    vt = np.tile([[0.0, 0.0, -0.8 / gam]], (n_p, 1))
    _, v, _ = oracle.run(sc, x0, vt, ty, 0, 50)
    assert np.allclose(v, vt, rtol=1e-13, atol=1e-15)


def test_printed_step_kick_has_fixed_magnitude_and_uniform_direction():
    """Printed step (vi) with gamma = 0 and no force: every step adds exactly
    v_kick in a direction uniform on the sphere (mean 0, second moment I/3), so
    |v_n|^2 grows by v_kick^2 per step on average."""
    n_p, A = 20000, 0.3
    sc = _kick_scenario(n_p, A, 0.0)
    ty = np.zeros(n_p, np.int32)
    x0 = np.zeros((n_p, 3))
    v0 = np.zeros((n_p, 3))
    _, v1, _ = oracle.run(sc, x0, v0, ty, 0, 1)
    assert np.allclose(np.linalg.norm(v1, axis=1), A, rtol=1e-13)
    _, v2, _ = oracle.run(sc, x0, v1, ty, 1, 1)        # the next step, alone
    assert np.allclose(np.linalg.norm(v2 - v1, axis=1), A, rtol=1e-12)
    u = v1 / A
    se = 1.0 / math.sqrt(3 * n_p)
    assert np.all(np.abs(u.mean(0)) < 5 * se)
    M = u.T @ u / n_p
    assert np.allclose(M, np.eye(3) / 3, atol=5 * math.sqrt(2.0 / 15 / n_p) + 1e-3)
    steps = 40
    _, v, _ = oracle.run(sc, x0, v0, ty, 0, steps)
    s2 = (v ** 2).sum(1)
    assert abs(s2.mean() - steps * A * A) < 5 * s2.std() / math.sqrt(n_p)


def test_velocity_verlet_limit_reversible_and_energy():
    """gamma = 0, kT = 0 turns BAOAB into velocity Verlet: running n steps, negating v
    and running n more returns to the start (time reversibility), and the total
    energy of an LJ cluster is conserved to O(dt^2)."""
    sc0, ty, x = _random_cluster(27, 2, R=3.5, T=1)
    t = wl.TypeSpec(sigma=1.0, eps=1.0, mass=1.0, charge=0.0, gamma=0.0, k_wall=0.0)
    sc = wl.Scenario(name="nve", types=[t], n=len(x), seed=0, dt=1e-3, kT=0.0, R0=1e9,
                     wall=False, lj_mode=1, coulomb=False, lj_cut=1e6)
    rng = np.random.default_rng(0)
    v0 = 0.3 * rng.standard_normal(x.shape)
    x1, v1, _ = oracle.run(sc, x, v0, ty, 0, 400)
    x2, v2, _ = oracle.run(sc, x1, -v1, ty, 400, 400)
    assert np.abs(x2 - x).max() < 1e-9
    assert np.abs(v2 + v0).max() < 1e-9

    def energy(xx, vv):
        U = 0.0
        for i in range(len(xx)):
            for j in range(i + 1, len(xx)):
                U += _lj_U(np.linalg.norm(xx[i] - xx[j]), 1.0, 1.0)
        return U + 0.5 * (vv ** 2).sum()

    E0 = energy(x, v0)
    E1 = energy(x1, v1)
    scale = np.abs(oracle.pair_forces(x, ty, [1.0], [1.0], [0.0], 0.0, lj_cut=1e6)).max()
    assert abs(E1 - E0) < 1e-3 * max(1.0, abs(E0))
    # halving dt cuts the drift by ~4 (second order)
    sc_h = wl.Scenario(**{**sc.__dict__, "dt": 5e-4})
    xh, vh, _ = oracle.run(sc_h, x, v0, ty, 0, 800)
    assert abs(energy(xh, vh) - E0) < 0.5 * abs(E1 - E0) + 1e-12 * scale


def test_resume_is_bit_exact():
    sc = wl.config2(n=256)
    ty, x, v = wl.initial_state(sc)
    xa, va, Fa = oracle.run(sc, x, v, ty, 0, 6)
    xb, vb, _ = oracle.run(sc, x, v, ty, 0, 3)
    xb, vb, Fb = oracle.run(sc, xb, vb, ty, 3, 3)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(Fa, Fb)


def test_single_step_brute_force_two_particles():
    """One BAOAB step of two charged NPs in a droplet, followed by hand on paper:
    with kT = 0 there is no noise, so the step is deterministic."""
    t0 = wl.TypeSpec(sigma=1.0, eps=1.0, mass=2.0, charge=1.0, gamma=3.0, k_wall=40.0)
    sc = wl.Scenario(name="two", types=[t0], n=2, seed=0, dt=0.01, kT=0.0, R0=2.0,
                     k_evap=1.0, bjerrum=0.5, coulomb=True, lj_mode=1, lj_cut=2.5)
    x0 = np.array([[0.0, 0.0, 0.9], [0.0, 0.0, -0.4]])
    v0 = np.array([[0.1, 0.0, 0.0], [0.0, 0.0, 0.2]])
    ty = np.zeros(2, np.int32)

    def force(x, t):
        d = x[0] - x[1]
        r = np.linalg.norm(d)
        f = 0.5 / r ** 3 + 24 * (2 / r ** 12 - 1 / r ** 6) / r ** 2
        F = np.array([f * d, -f * d])
        R = math.sqrt(4.0 - t)
        for i in range(2):
            ri = np.linalg.norm(x[i])
            s = ri - (R - 0.5)
            if s > 0:
                F[i] -= 40.0 * s * x[i] / ri
        return F

    dt, m, c1 = 0.01, 2.0, math.exp(-0.03)
    v = v0 + 0.5 * dt * force(x0, 0.0) / m
    x = x0 + 0.5 * dt * v
    v = c1 * v
    x = x + 0.5 * dt * v
    v = v + 0.5 * dt * force(x, dt) / m
    xo, vo, Fo = oracle.run(sc, x0, v0, ty, 0, 1)
    assert np.allclose(xo, x, rtol=1e-13, atol=1e-15)
    assert np.allclose(vo, v, rtol=1e-12, atol=1e-14)
    assert np.allclose(Fo, force(x, dt), rtol=1e-12)


# --------------------------------------------------------------------------
# Statistics


def test_rdf_uniform_ball_chord_law():
    """Uniform points in a ball of radius R with V = 4 pi R^3/3: g(r) tends to
    1 - 3r/(4R) + r^3/(16 R^3) (distance distribution of two uniform points)."""
    rng = np.random.default_rng(3)
    n, R = 3000, 10.0
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = v * (R * rng.random(n) ** (1 / 3))[:, None]
    nb, rmax = 20, 20.0
    counts, g = oracle.rdf(x, rmax, nb, R)
    dr = rmax / nb
    for b in range(1, nb - 1):
        # expected counts from the exact shell average of the chord law
        r0, r1 = b * dr, (b + 1) * dr
        rr = np.linspace(r0, r1, 2001)
        law = 1 - 3 * rr / (4 * R) + rr ** 3 / (16 * R ** 3)
        shell = np.trapezoid(4 * np.pi * rr ** 2 * law, rr)
        expect = n * (n - 1) * shell / (4 / 3 * np.pi * R ** 3)
        # ordered pairs double the variance of the unordered count
        assert abs(counts[b] - expect) < 5 * math.sqrt(2 * expect) + 1
    assert counts.sum() == n * (n - 1)  # all pairs within 2R


def test_pair_hist_fcc_first_shell_integer_count():
    """FCC points = integer triples with even coordinate sum (spacing a = 2):
    ordered pairs at distance sqrt(2) counted by integer arithmetic."""
    L = 6
    P = np.array([(i, j, k) for i in range(L) for j in range(L) for k in range(L)
                  if (i + j + k) % 2 == 0], float)
    D2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1).round().astype(int)
    n_first = int((D2 == 2).sum())
    n_second = int((D2 == 4).sum())
    c = oracle.pair_hist(P, 2.2, 11)  # bins of 0.2: sqrt(2)=1.414 in bin 7, 2 in bin 10
    assert c[7] == n_first and c[10] == n_second
    assert c.sum() == n_first + n_second
    interior = sum(1 for p in P if np.all((p >= 1) & (p <= L - 2)))
    assert n_first >= 12 * interior


def test_radial_concentration_uniform_ball_flat():
    rng = np.random.default_rng(4)
    n, R = 200000, 5.0
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = v * (R * rng.random(n) ** (1 / 3))[:, None]
    counts, Cc = oracle.radial_concentration(x, R, 10, R)
    assert counts.sum() == n
    for b in range(10):
        assert abs(Cc[b] - 1) < 5 / math.sqrt(counts[b])


def test_surface_count_band_edges():
    """N_surf counts NP i when | |x_i| - R | < sigma_i / 2: NPs placed just
    inside and just outside both edges of the band, for two diameters, in random
    directions (a band of sigma instead of sigma/2, or a one-sided test, fails)."""
    R = 10.0
    sigma = np.array([1.0, 3.0])
    cases = [(0, 9.4, 0), (0, 9.6, 1), (0, 10.0, 1), (0, 10.4, 1), (0, 10.6, 0),
             (1, 8.4, 0), (1, 8.6, 1), (1, 11.4, 1), (1, 11.6, 0), (1, 0.0, 0),
             (0, 12.0, 0), (1, 10.0, 1)]
    rng = np.random.default_rng(4)
    u = rng.standard_normal((len(cases), 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    ty = np.array([c[0] for c in cases], np.int32)
    x = u * np.array([c[1] for c in cases])[:, None]
    assert oracle.surface_count(x, ty, sigma, R) == sum(c[2] for c in cases)
    for k in range(len(cases)):  # one NP at a time
        assert oracle.surface_count(x[k:k + 1], ty[k:k + 1], sigma, R) == cases[k][2]


def test_scattering_uniform_sphere_closed_form():
    """g = 1 on [0, R): the transform is the volume integral of a uniform sphere,
    4 pi (sin qR - qR cos qR)/q^3, and 4 pi R^3/3 at q = 0 (whatever the binning),
    times N_surf^2."""
    R = 7.5
    q = np.array([0.05, 0.3, 1.0, 2.7, 9.0])
    for n_bins in (1, 16, 128):
        I = oracle.scattering(np.ones(n_bins), R, 3, q)
        ref = 9 * 4 * np.pi * (np.sin(q * R) - q * R * np.cos(q * R)) / q ** 3
        assert np.allclose(I, ref, rtol=1e-11, atol=0)
        assert oracle.scattering(np.ones(n_bins), R, 3, [0.0])[0] == pytest.approx(
            9 * 4 * np.pi * R ** 3 / 3, rel=1e-13)


def test_scattering_matches_numerical_quadrature():
    """A random piecewise-constant g: every bin's r^2 sin(qr)/(qr) integral by
    adaptive quadrature agrees with the oracle's antiderivative form, small q
    (series branch) included."""
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(12)
    n_bins, r_max = 24, 6.0
    g = rng.uniform(0.0, 3.0, n_bins)
    dr = r_max / n_bins
    for q in (0.01, 0.08, 0.37, 2.5, 11.0):
        tot = 0.0
        for b in range(n_bins):
            val, _ = integrate.quad(lambda r: r * r * np.sinc(q * r / np.pi), b * dr,
                                    (b + 1) * dr, epsabs=0, epsrel=1e-13, limit=200)
            tot += g[b] * val
        assert oracle.scattering(g, r_max, 1, [q])[0] == pytest.approx(4 * np.pi * tot,
                                                                       rel=1e-10)


def test_rg_closed_forms_and_fractal_equation():
    golden = json.load(open(GOLDEN))
    assert oracle.K_F == golden["fractal_prefactor_k_f"]["value"]
    # symmetric shell: +-R along each axis -> R_g = R exactly, centre 0
    R = 2.5
    x = np.array([[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]]) + 7.0
    Rg, Df, r0 = oracle.rg(x, 1.0)
    assert Rg == pytest.approx(R, rel=1e-14)
    assert np.allclose(r0, 7.0)
    # D_f solves N = k_f (2 Rg / d)^Df
    assert oracle.K_F * (2 * Rg / 1.0) ** Df == pytest.approx(len(x), rel=1e-12)
    # solid ball: R_g = sqrt(3/5) R
    rng = np.random.default_rng(5)
    n = 200000
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x = v * (4.0 * rng.random(n) ** (1 / 3))[:, None]
    Rg, _, _ = oracle.rg(x, 1.0)
    assert Rg == pytest.approx(math.sqrt(3 / 5) * 4.0, rel=3e-3)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_boxcount_lattice_dimension(dim):
    """Filled lattices of spacing d: N_box(d 2^k) = (L/2^k)^dim exactly, D_f = dim."""
    L = 32 if dim == 3 else 256
    g = (np.arange(L) + 0.5)
    if dim == 1:
        P = np.stack([g, np.zeros(L), np.zeros(L)], 1)
    elif dim == 2:
        X, Y = np.meshgrid(g, g, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    else:
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    nb = oracle.boxcount(P, 1.0, 5)
    for k in range(5):
        assert nb[k] == (L // 2 ** k) ** dim
    Rg, _, _ = oracle.rg(P, 1.0)
    Df, nbs = oracle.boxcount_df(P, 1.0, Rg)
    assert Df == pytest.approx(dim, abs=0.02)


def test_lsq_slope_exact_line():
    xs = np.array([0.0, 1.0, 2.5, 4.0])
    assert oracle.lsq_slope(xs, 3.0 - 2.0 * xs) == pytest.approx(-2.0, rel=1e-14)
