"""Seeded synthetic inputs for the nanoparticle-aggregation step.

This module holds scenario descriptions (per-type NP properties, droplet and
integrator parameters) and the seeded initial state (types, positions,
velocities).  It contains none of the method's arithmetic: no forces, no
integrator, no statistics.  Both the FP64 oracle and the GPU library take
their inputs from here, so both start from identical float64 arrays.

Scenarios follow the paper's set-up (Sec. 2.1: NPs of several types placed at
random in a sphere, a droplet whose radius follows the radius-square law,
Table 1 for the flavour of the parameters) at the sizes of the benchmark
workloads: a 1000-NP LJ droplet, a 16384-NP two-type charged droplet, a
250000-NP three-type droplet and a 256-droplet ensemble.  Units are reduced:
length sigma (the diameter of the smallest NP), energy kT_ref = 1, mass of a
sigma = 1 NP = 1.  Masses scale as sigma^3 (uniform density) and the Stokes
friction coefficient m*gamma scales as sigma (Sec. 2.1: the dissipative force
"conforms to Stokes' law"), so gamma = 1/sigma^2.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = ["TypeSpec", "Scenario", "config1", "config2", "config3", "ensemble_config",
           "assign_types", "place", "maxwell_velocities", "initial_state",
           "scaled", "fp32_representable"]


@dataclass
class TypeSpec:
    sigma: float = 1.0      # NP diameter
    eps: float = 1.0        # LJ well depth of the like pair
    mass: float = 1.0
    charge: float = 0.0
    gamma: float = 1.0      # Langevin friction rate (1/time)
    k_wall: float = 100.0   # interface spring constant
    frac: float = 1.0       # number fraction


def stokes_type(sigma, charge=0.0, eps=1.0, k_wall=100.0, frac=1.0) -> TypeSpec:
    """NP of diameter sigma: m = sigma^3, m*gamma = sigma (Stokes)."""
    m = sigma ** 3
    return TypeSpec(sigma=sigma, eps=eps, mass=m, charge=charge, gamma=sigma / m,
                    k_wall=k_wall, frac=frac)


@dataclass
class Scenario:
    name: str
    types: List[TypeSpec]
    n: int
    seed: int = 0
    dt: float = 1e-3
    kT: float = 1.0
    R0: float = 30.0
    k_evap: float = 0.0          # R(t)^2 = R0^2 - k_evap t
    g: float = 0.0               # gravity along -z
    omega: float = 0.0
    rot_mode: int = 0            # 0 none, 1 about z, 2 isotropic
    bjerrum: float = 0.0         # Coulomb prefactor (Bjerrum length, kT_ref = 1)
    lj_cut: float = 2.5          # LJ cutoff in units of sigma_ab
    coulomb: bool = False
    lj_mode: int = 1             # 0 off, 1 inside the all-pairs kernel, 2 cell list
    integrator: int = 0          # 0 BAOAB Langevin, 1 overdamped, 2 printed step (vi) + kick
    wall: bool = True
    wall_band: bool = False      # spring only within (-r, r) of the surface (printed step iv)
    v_kick: float = 0.0          # integrator 2: magnitude of the random velocity per step
    coulomb_cut: float = 0.0     # > 0: Coulomb truncated at coulomb_cut * sigma_ab (cell list)
    eps_override: Optional[np.ndarray] = None
    n_steps: int = 1000          # length of the full run
    min_gap: float = 0.9         # placement: no pair closer than min_gap*sigma_ab
    sum_neutral: bool = False    # all-pairs Coulomb over all pairs, charge-0 NPs included
                                 # (default: they are left out; their terms are exactly 0)

    @property
    def T(self) -> int:
        return len(self.types)

    def radius_at(self, step: int) -> float:
        """Droplet radius at a step (scenario bookkeeping for sizing, not physics)."""
        R2 = self.R0 ** 2 - self.k_evap * step * self.dt
        return math.sqrt(R2) if R2 > 0 else 0.0


def _k_for(R0, Rf, n_steps, dt):
    return (R0 * R0 - Rf * Rf) / (n_steps * dt)


def config1(seed: int = 0) -> Scenario:
    """1000 one-type LJ NPs, cutoff 2.5 sigma (cell list), R 30 -> 20 over 1000 steps."""
    return Scenario(name="lj1000", types=[TypeSpec(1.0, 1.0, 1.0, 0.0, 1.0, 100.0, 1.0)],
                    n=1000, seed=seed, dt=1e-3, kT=1.0, R0=30.0,
                    k_evap=_k_for(30.0, 20.0, 1000, 1e-3), coulomb=False, lj_mode=2,
                    n_steps=1000)


def config2(seed: int = 0, n: int = 16384) -> Scenario:
    """16384 NPs, diameters 1 and 2 (3:1), charges +1/-1, Bjerrum length 0.7,
    all-pairs Coulomb + LB-mixed LJ, g = 0.01, omega = 0.05 about z,
    R 80 -> 30 over 20000 steps at dt = 5e-4."""
    types = [stokes_type(1.0, +1.0, frac=0.75), stokes_type(2.0, -1.0, frac=0.25)]
    sc = Scenario(name="coulomb_lj16384", types=types, n=16384, seed=seed, dt=5e-4,
                  kT=1.0, R0=80.0, k_evap=_k_for(80.0, 30.0, 20000, 5e-4), g=0.01,
                  omega=0.05, rot_mode=1, bjerrum=0.7, coulomb=True, lj_mode=1,
                  n_steps=20000)
    return scaled(sc, n) if n != 16384 else sc


def config3(kT: float = 1.0, seed: int = 0, n: int = 250000) -> Scenario:
    """250000 NPs, diameters 1/1.5/3 (0.6/0.3/0.1), charges 0/+0.5/-0.5, all-pairs
    Coulomb + cell-list LJ at 2.5 sigma_ab, R 200 -> 60 over 50000 steps."""
    types = [stokes_type(1.0, 0.0, frac=0.6), stokes_type(1.5, +0.5, frac=0.3),
             stokes_type(3.0, -0.5, frac=0.1)]
    sc = Scenario(name="paper_scale250000", types=types, n=250000, seed=seed, dt=5e-4,
                  kT=kT, R0=200.0, k_evap=_k_for(200.0, 60.0, 50000, 5e-4),
                  bjerrum=0.7, coulomb=True, lj_mode=2, n_steps=50000)
    return scaled(sc, n) if n != 250000 else sc


def scaled(sc: Scenario, n: int) -> Scenario:
    """Same scenario with n NPs and R0 (and k) scaled to keep the packing fraction."""
    f = (n / sc.n) ** (1.0 / 3.0)
    R0 = sc.R0 * f
    Rf = sc.radius_at(sc.n_steps) * f
    out = dataclasses.replace(sc, n=n, R0=R0,
                              k_evap=_k_for(R0, Rf, sc.n_steps, sc.dt),
                              name=f"{sc.name.rstrip('0123456789')}{n}")
    return out


def ensemble_config(n_droplets: int = 256, master_seed: int = 12345,
                    n_min: int = 512, n_max: int = 32768, n_steps: int = 10000,
                    phi0: float = 0.01) -> List[Scenario]:
    """Independent droplets: N log-uniform in [n_min, n_max], |q| ~ U[0,1] with the
    two types carrying +|q| and -|q|, eps ~ U[0.5, 2], final R/R0 ~ U[0.2, 0.6],
    R0 chosen for an initial packing fraction phi0, own seed per droplet.
    Physics otherwise as the 16384-NP two-type scenario."""
    rng = np.random.default_rng(master_seed)
    out = []
    for d in range(n_droplets):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        q = float(rng.uniform(0.0, 1.0))
        eps = float(rng.uniform(0.5, 2.0))
        ratio = float(rng.uniform(0.2, 0.6))
        types = [stokes_type(1.0, +q, eps=eps, frac=0.75),
                 stokes_type(2.0, -q, eps=eps, frac=0.25)]
        vol = sum(t.frac * math.pi / 6.0 * t.sigma ** 3 for t in types) * n
        R0 = (vol / phi0 / (4.0 / 3.0 * math.pi)) ** (1.0 / 3.0)
        dt = 5e-4
        out.append(Scenario(name=f"drop{d}", types=types, n=n, seed=d, dt=dt, kT=1.0,
                            R0=R0, k_evap=_k_for(R0, ratio * R0, n_steps, dt), g=0.01,
                            omega=0.05, rot_mode=1, bjerrum=0.7, coulomb=True,
                            lj_mode=1, n_steps=n_steps))
    return out


# --------------------------------------------------------------------------
# Initial state


def assign_types(sc: Scenario) -> np.ndarray:
    """Deterministic split: the first round(f_0 n) indices get type 0, and so on;
    the last type takes the remainder."""
    t = np.zeros(sc.n, np.int32)
    start = 0
    for a, ts in enumerate(sc.types):
        cnt = sc.n - start if a == sc.T - 1 else int(round(ts.frac * sc.n))
        t[start:start + cnt] = a
        start += cnt
    return t


def _uniform_ball(rng, m, radii):
    v = rng.standard_normal((m, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = radii * rng.random(m) ** (1.0 / 3.0)
    return v * r[:, None]


def place(sc: Scenario, types: np.ndarray, seed: Optional[int] = None,
          R: Optional[float] = None, batch: int = 4096) -> np.ndarray:
    """Uniform random positions in |x| <= R - sigma_i/2 (R defaults to R0) with no
    pair closer than min_gap * sigma_ab (random sequential addition).

    Candidates are drawn in batches in index order; a candidate is rejected if
    it overlaps an accepted NP or an earlier candidate of the same batch, and is
    redrawn.  Deterministic for a given seed."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(sc.seed if seed is None else seed)
    R = sc.R0 if R is None else R
    sig = np.array([t.sigma for t in sc.types])
    s_i = sig[types]
    n = sc.n
    x = np.zeros((n, 3))
    placed = np.zeros(n, bool)
    acc_idx = np.zeros(0, np.int64)
    tree = None
    todo = np.arange(n)
    gmax = sc.min_gap * sig.max()
    rounds = 0
    while len(todo):
        cur = todo[:batch]
        pending = cur
        while len(pending):
            rounds += 1
            if rounds > 20000:
                raise RuntimeError("placement jammed: packing fraction too high for "
                                   "random sequential addition")
            cand = _uniform_ball(rng, len(pending), R - 0.5 * s_i[pending])
            ok = np.ones(len(pending), bool)
            if tree is not None:
                hits = tree.query_ball_point(cand, gmax)
                for k, h in enumerate(hits):
                    if h:
                        j = acc_idx[np.asarray(h)]
                        d = np.linalg.norm(x[j] - cand[k], axis=1)
                        lim = sc.min_gap * 0.5 * (s_i[j] + s_i[pending[k]])
                        if np.any(d < lim):
                            ok[k] = False
            # conflicts inside the batch: keep the earlier index
            if len(pending) > 1:
                bt = cKDTree(cand)
                pairs = bt.query_pairs(gmax, output_type="ndarray")
                if len(pairs):
                    a, b = pairs[:, 0], pairs[:, 1]
                    d = np.linalg.norm(cand[a] - cand[b], axis=1)
                    lim = sc.min_gap * 0.5 * (s_i[pending[a]] + s_i[pending[b]])
                    bad = d < lim
                    for aa, bb in zip(a[bad], b[bad]):
                        lo, hi = (aa, bb) if aa < bb else (bb, aa)
                        if ok[lo]:
                            ok[hi] = False
            x[pending[ok]] = cand[ok]
            placed[pending[ok]] = True
            acc_idx = np.concatenate([acc_idx, pending[ok]])
            tree = cKDTree(x[acc_idx])
            pending = pending[~ok]
        todo = todo[batch:]
    assert placed.all()
    return x


def maxwell_velocities(sc: Scenario, types: np.ndarray, seed: Optional[int] = None):
    """Velocities with each component ~ N(0, kT/m_i)."""
    rng = np.random.default_rng((sc.seed if seed is None else seed) + 0x5EED)
    m = np.array([t.mass for t in sc.types])[types]
    return rng.standard_normal((sc.n, 3)) * np.sqrt(sc.kT / m)[:, None]


def fp32_representable(x: np.ndarray) -> np.ndarray:
    """Round float64 positions to the nearest float32 value (kept as float64)."""
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def initial_state(sc: Scenario, fp32_positions: bool = False):
    """(types, x0, v0) for a scenario; x0 optionally rounded to float32 values."""
    types = assign_types(sc)
    x = place(sc, types)
    if fp32_positions:
        x = fp32_representable(x)
    v = maxwell_velocities(sc, types)
    return types, x, v
