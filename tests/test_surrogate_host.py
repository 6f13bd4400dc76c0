"""Host logic of the surrogate's spread-gated acceptance (no GPU)."""
import numpy as np

from paper_2501_04456_gb300 import surrogate_pipeline as sp


def test_calibrate_tau_picks_the_largest_qualifying_threshold():
    spread = np.array([0.4, 0.1, 0.3, 0.2])
    err = np.array([0.01, 0.01, 0.10, 0.02])
    # sorted by spread: ok, ok, bad, ok -> 100 %, 100 %, 67 %, 75 %
    assert sp.calibrate_tau(spread, err, tol=0.05, target=0.98) == 0.2
    assert sp.calibrate_tau(spread, err, tol=0.05, target=0.75) == 0.4
    assert sp.calibrate_tau(spread, err, tol=0.2, target=0.98) == 0.4
    # nothing qualifies: every prediction falls back to the simulation
    assert sp.calibrate_tau(np.array([0.1, 0.2]), np.array([0.1, 0.1])) == 0.0


def test_rdf_error_and_spread_measures():
    sim = np.zeros((2, 65))
    sim[:, 1:] = 1.0
    pred = sim.copy()
    pred[0, 1:] += 0.1  # 10 % off in every bin
    e = sp.rdf_rel_error(pred, sim)
    assert np.allclose(e, [0.1, 0.0])
    spread = np.zeros_like(sim)
    spread[1, 1:] = 0.5
    assert np.allclose(sp.rdf_spread(sim, spread), [0.0, 0.5])


def test_config5_ranges_and_features():
    r = sp.config5_ranges()
    rng = np.random.default_rng(0)
    steps, dt = 10000, 5e-4
    X = sp.sample_features(500, rng, steps, r, dt=dt)
    n = np.exp(X[:, 0])
    assert n.min() >= 512 * 0.999 and n.max() <= 8192 * 1.001
    f1, f2 = X[:, 1], X[:, 2]
    assert np.all(f1 + f2 < 1.0)
    R0, k = X[:, 5], X[:, 6]
    ratio = np.sqrt(R0 ** 2 - k * steps * dt) / R0  # final R / R0 by the radius law
    assert ratio.min() >= 0.2 - 1e-9 and ratio.max() <= 0.6 + 1e-9
