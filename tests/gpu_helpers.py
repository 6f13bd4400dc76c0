"""Shared helpers of the GPU parity tests: build the library, create a simulation
from a workloads scenario, and the force-error metric."""
import dataclasses

import numpy as np

import workloads as wl

# Force parity tolerance: max_i |dF_i| / max(|F_i|, rms_j |F_j|) <= 1e-5 with the
# oracle evaluated at the same float32-representable positions.
FORCE_TOL = 1e-5
# Trajectory parity: max |x_gpu - x_oracle| <= 1e-4 sigma after 100 steps.
TRAJ_TOL = 1e-4


def library():
    from paper_2501_04456_gb300 import build
    build.build()
    import paper_2501_04456_gb300 as P
    return P


def make_sim(P, sc, x, v, types, stream=None):
    return P.Sim(sc, x, v, types, stream=stream)


def force_error(F_gpu, F_ref, rows=None):
    """Per-row error |dF_i| / max(|F_i|, rms_j |F_j|) (rows: subset to report)."""
    F_gpu = np.asarray(F_gpu)
    F_ref = np.asarray(F_ref)
    rms = np.sqrt((F_ref ** 2).sum(1).mean())
    mag = np.linalg.norm(F_ref, axis=1)
    err = np.linalg.norm(F_gpu - F_ref, axis=1) / np.maximum(np.maximum(mag, rms), 1e-300)
    return err if rows is None else err[rows]


def cutoff_ambiguous(x, types, sc, rel=2e-6):
    """Rows with a pair whose distance lies within float32 rounding of its LJ
    cutoff (or of its Coulomb cutoff, when Coulomb is truncated): both
    classifications of such a pair are correct, so the strict comparison leaves
    these rows out (the caller checks they are few)."""
    sig = np.array([t.sigma for t in sc.types])
    sab = 0.5 * (sig[:, None] + sig[None, :])
    cuts = []
    if sc.lj_mode != 0:
        cuts.append(sc.lj_cut * sab)
    if sc.coulomb and getattr(sc, "coulomb_cut", 0.0) > 0:
        cuts.append(sc.coulomb_cut * sab)
    out = np.zeros(len(x), bool)
    if not cuts:
        return out
    from scipy.spatial import cKDTree
    tree = cKDTree(x)
    pairs = tree.query_pairs(max(c.max() for c in cuts) * (1 + 1e-4), output_type="ndarray")
    if len(pairs):
        d = np.linalg.norm(x[pairs[:, 0]] - x[pairs[:, 1]], axis=1)
        for rc in cuts:
            r = rc[types[pairs[:, 0]], types[pairs[:, 1]]]
            amb = np.abs(d - r) <= rel * r
            out[pairs[amb, 0]] = True
            out[pairs[amb, 1]] = True
    return out


def small(sc, n):
    """Scenario at n particles with its packing fraction kept."""
    return wl.scaled(sc, n)


def with_(sc, **kw):
    return dataclasses.replace(sc, **kw)
