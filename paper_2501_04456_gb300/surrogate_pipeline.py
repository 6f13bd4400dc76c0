"""Learned surrogate of the final aggregate's statistics over scenario parameters.

The simulation maps a scenario -- number of NPs, composition, charge, LJ
depth, droplet radius, evaporation rate, temperature -- to an aggregate whose
fractal dimension (Sec. 3.1, Eq. N with k_f = 1.593) and RDF (Sec. 3.2) the
paper reports.  This module generates training data with the batched
ensemble (many droplets per launch), fits the deep ensemble of MLPs of
npsim_surr_* (BF16 tcgen05 kernels), and predicts new scenarios, sending the
ones whose ensemble spread is too large back to the simulation, which also
scores the surrogate's error.

Inputs (8): log N, fraction of type 1, fraction of type 2, charge magnitude q
(types carry 0, +q, -q), LJ eps, R0, evaporation rate k, kT.
Outputs (65): D_f from the fractal equation, then g(r) in 64 bins over
[0, r_max).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

FEATURES = ("log_n", "f1", "f2", "q", "eps", "R0", "k_evap", "kT")
N_OUT = 65


@dataclass
class Ranges:
    n_min: int = 256
    n_max: int = 2048
    f1: tuple = (0.4, 0.8)
    q: tuple = (0.0, 1.0)
    eps: tuple = (0.5, 2.0)
    phi0: tuple = (0.01, 0.04)     # initial packing fraction (sets R0 for the N)
    shrink: tuple = (0.4, 0.8)     # final R / R0 (sets k for the run length)
    kT: tuple = (0.5, 2.0)


def config5_ranges() -> Ranges:
    """Scenario ranges of the surrogate's training data in the regime of the
    batched ensemble: N log-uniform in [512, 8192], final R/R0 in [0.2, 0.6],
    initial packing fraction in [0.006, 0.012] (the ensemble's 0.01 with some
    spread), the other inputs as in Ranges."""
    return Ranges(n_min=512, n_max=8192, phi0=(0.006, 0.012), shrink=(0.2, 0.6))


def calibrate_tau(spread, err, tol=0.05, target=0.98):
    """Largest spread threshold tau such that, on a validation set, at least
    `target` of the predictions with spread <= tau are within `tol` of the
    simulation (err = |prediction - simulation|).  Returns tau (0.0 if no
    threshold qualifies: everything falls back to the simulation)."""
    order = np.argsort(spread, kind="stable")
    sp = np.asarray(spread)[order]
    ok = (np.asarray(err)[order] <= tol).astype(np.float64)
    frac = np.cumsum(ok) / np.arange(1, len(ok) + 1)
    good = np.nonzero(frac >= target)[0]
    if len(good) == 0:
        return 0.0
    k = good[-1]
    # keep every prediction tied with the last accepted spread on the same side
    while k + 1 < len(sp) and sp[k + 1] == sp[k] and frac[k + 1] >= target:
        k += 1
    return float(sp[k])


def scenario_from(feat, steps, dt=5e-4, seed=0):
    """Scenario of one droplet: three types of diameters 1, 1.5, 3 (fractions f1,
    f2, 1 - f1 - f2), charges 0, +q, -q, LJ eps, Bjerrum length 0.7, all-pairs
    Coulomb and LJ, interface spring 100, Stokes friction."""
    import workloads as wl
    log_n, f1, f2, q, eps, R0, k, kT = [float(v) for v in feat]
    n = int(round(math.exp(log_n)))
    types = [wl.stokes_type(1.0, 0.0, eps=eps, frac=f1),
             wl.stokes_type(1.5, +q, eps=eps, frac=f2),
             wl.stokes_type(3.0, -q, eps=eps, frac=max(0.0, 1.0 - f1 - f2))]
    return wl.Scenario(name=f"surr{seed}", types=types, n=n, seed=seed, dt=dt, kT=kT, R0=R0,
                       k_evap=k, bjerrum=0.7, coulomb=True, lj_mode=1, n_steps=steps)


def sample_features(n, rng, steps, ranges=Ranges(), dt=5e-4):
    """n random scenarios as an (n, 8) feature array."""
    out = np.zeros((n, 8))
    for i in range(n):
        N = math.exp(rng.uniform(math.log(ranges.n_min), math.log(ranges.n_max)))
        f1 = rng.uniform(*ranges.f1)
        f2 = rng.uniform(0.1, 0.9) * (1.0 - f1)
        q = rng.uniform(*ranges.q)
        eps = rng.uniform(*ranges.eps)
        vol = N * math.pi / 6.0 * (f1 * 1.0 + f2 * 1.5 ** 3 + (1 - f1 - f2) * 27.0)
        R0 = (vol / rng.uniform(*ranges.phi0) / (4.0 / 3.0 * math.pi)) ** (1.0 / 3.0)
        Rf = R0 * rng.uniform(*ranges.shrink)
        k = (R0 * R0 - Rf * Rf) / (steps * dt)
        kT = rng.uniform(*ranges.kT)
        out[i] = (math.log(N), f1, f2, q, eps, R0, k, kT)
    return out


def simulate(P, feats, steps, seed0=0, batch=256, stream=None, r_max=8.0):
    """Simulate every scenario for `steps` steps with the batched ensemble and
    return (Y, seconds): Y[i] = (D_f, g(r) in 64 bins), both computed on the GPU
    from the ensemble's final state by npsim_ens_stats (no copy of the positions
    to the host).  `seconds` is the simulation time (creation and steps)."""
    import workloads as wl
    Y = np.zeros((len(feats), N_OUT))
    t_sim = 0.0
    for b0 in range(0, len(feats), batch):
        scs = [scenario_from(f, steps, seed=seed0 + b0 + i)
               for i, f in enumerate(feats[b0:b0 + batch])]
        drops = []
        for sc in scs:
            t, x, v = wl.initial_state(sc)
            drops.append((sc, x, v, t))
        t0 = time.perf_counter()
        with P.Ensemble(drops, stream=stream) as ens:
            ens.step(steps)
            t_sim += time.perf_counter() - t0
            for i in range(len(scs)):
                st = ens.stats(i, r_max=r_max, n_bins=N_OUT - 1, boxcount=False)
                Y[b0 + i, 0] = st["Df_rg"]
                Y[b0 + i, 1:] = st["rdf_g"]
    return Y, t_sim


def rdf_spread(mean, spread):
    """Relative spread of the predicted g(r) across the networks:
    ||spread of the 64 bins||_2 / ||mean g||_2 per sample."""
    g = np.asarray(mean)[:, 1:]
    return np.linalg.norm(np.asarray(spread)[:, 1:], axis=1) / np.maximum(
        np.linalg.norm(g, axis=1), 1e-30)


def rdf_rel_error(pred, sim):
    """||g_pred - g_sim||_2 / ||g_sim||_2 per sample (the 64 RDF bins)."""
    a, b = np.asarray(pred)[:, 1:], np.asarray(sim)[:, 1:]
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-30)


class SurrogateModel:
    """Deep ensemble of MLPs (8 -> 4 x 256 SiLU -> 65) with a spread-gated
    fallback to simulation."""

    def __init__(self, P, n_nets=4, seed=0):
        self.P = P
        self.net = P.Surrogate(n_in=8, n_hidden=256, n_layers=4, n_out=N_OUT, n_nets=n_nets,
                               seed=seed)

    def fit(self, X, Y, epochs=200, batch=256, lr=1e-3, wd=1e-4, seed=0):
        xs = X.std(0)
        ys = Y.std(0)
        self.net.set_norm(X.mean(0), np.where(xs > 0, xs, 1.0), Y.mean(0),
                          np.where(ys > 1e-6, ys, 1.0))
        return self.net.train(X, Y, epochs=epochs, batch=batch, lr=lr, wd=wd, seed=seed)

    def predict(self, X):
        return self.net.predict(X)

    def predict_or_simulate(self, X, steps, tau, seed0=10 ** 6, stream=None, tau_rdf=None):
        """Surrogate prediction where the spread of D_f across the networks is at
        most tau (and, with tau_rdf, the relative spread of g(r) at most
        tau_rdf); the plain simulation elsewhere.  Returns (Y, fallback mask)."""
        m, sp = self.predict(X)
        fb = sp[:, 0] > tau
        if tau_rdf is not None:
            fb |= rdf_spread(m, sp) > tau_rdf
        Y = m.astype(np.float64)
        if fb.any():
            Ys, _ = simulate(self.P, X[fb], steps, seed0=seed0, stream=stream)
            Y[fb] = Ys
        return Y, fb

    def close(self):
        self.net.close()
