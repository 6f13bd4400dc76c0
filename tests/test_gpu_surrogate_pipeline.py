"""The learned surrogate end to end: training data from the batched ensemble,
fit on the GPU, prediction with a spread-gated fallback to the simulation, and
what the network gains over the method without it."""
import time

import numpy as np
import pytest

from gpu_helpers import library

pytestmark = pytest.mark.gpu


def test_surrogate_gains_over_simulation_and_baseline():
    P = library()
    from paper_2501_04456_gb300 import surrogate_pipeline as sp_

    rng = np.random.default_rng(0)
    steps = 400
    r = sp_.Ranges(n_min=256, n_max=1024)
    Xtr = sp_.sample_features(2048, rng, steps, r)
    Ytr, t_tr = sp_.simulate(P, Xtr, steps, seed0=0)
    Xte = sp_.sample_features(256, rng, steps, r)
    Yte, t_te = sp_.simulate(P, Xte, steps, seed0=100000)
    Yrep, _ = sp_.simulate(P, Xte, steps, seed0=200000)  # same scenarios, other seeds
    assert np.all(np.isfinite(Ytr)) and np.all(np.isfinite(Yte))

    model = sp_.SurrogateModel(P, n_nets=4, seed=1)
    try:
        model.fit(Xtr, Ytr, epochs=100, batch=256, lr=1e-3)
        t0 = time.perf_counter()
        m, spread = model.predict(Xte)
        t_pred = time.perf_counter() - t0

        err = np.abs(m[:, 0] - Yte[:, 0])
        base = np.abs(Ytr[:, 0].mean() - Yte[:, 0])      # the method without the network
        rep = np.abs(Yrep[:, 0] - Yte[:, 0])               # simulation vs simulation
        # the network predicts D_f much better than the data mean, and about as
        # well as a second simulation with another seed
        assert err.mean() <= 0.25 * base.mean()
        assert err.mean() <= 1.5 * rep.mean() + 0.005
        # RDF: L2 error relative to the simulated g(r) no larger than the
        # seed-to-seed L2 variation of the simulation itself
        rel = np.linalg.norm(m[:, 1:] - Yte[:, 1:], axis=1) / np.linalg.norm(Yte[:, 1:], axis=1)
        rel_rep = (np.linalg.norm(Yrep[:, 1:] - Yte[:, 1:], axis=1) /
                   np.linalg.norm(Yte[:, 1:], axis=1))
        assert np.median(rel) <= np.median(rel_rep)
        # spread-gated acceptance: accepted predictions within +-0.05 in D_f
        tau = 0.02
        acc = spread[:, 0] <= tau
        assert acc.mean() >= 0.6
        assert np.mean(err[acc] <= 0.05) >= 0.98
        # speed: a prediction costs far less than a simulation of the droplet
        assert t_pred / len(Xte) <= 0.1 * (t_te / len(Xte))
        # fallback: rejected scenarios are re-simulated
        few = Xte[:32]
        Yf, fb = model.predict_or_simulate(few, steps, tau=np.median(spread[:32, 0]))
        assert fb.any() and (~fb).any()
        assert np.all(np.isfinite(Yf))
        assert np.allclose(Yf[~fb], m[:32][~fb], rtol=1e-6, atol=1e-6)
    finally:
        model.close()
