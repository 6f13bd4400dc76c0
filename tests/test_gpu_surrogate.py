"""The surrogate's tcgen05 BF16 kernels against the FP64 MLP oracle."""
import numpy as np
import pytest

from oracle import mlp
from gpu_helpers import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return library()


def _bits(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def _val(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K,nt", [(128, 16, 16, 16), (300, 80, 80, 80), (512, 256, 256, 64),
                                      (256, 256, 512, 256), (129, 48, 272, 48)])
def test_gemm_bf16_tcgen05(P, M, N, K, nt):
    rng = np.random.default_rng(M + N + K)
    A = _bits(rng.standard_normal((M, K)))
    B = _bits(rng.standard_normal((N, K)))
    Cg = P.npsim_gemm_bf16(A, B, nt)
    a, b = _val(A), _val(B)
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(Cg - ref) <= 2e-5 * scale + 1e-30)


DIMS = [(256, 16), (256, 256), (256, 256), (256, 256), (80, 256)]


def _pad(X, w):
    out = np.zeros((X.shape[0], w))
    out[:, :X.shape[1]] = X
    return out


def test_surrogate_forward_backward_vs_oracle(P):
    with P.Surrogate(n_in=8, n_hidden=256, n_layers=4, n_out=65, n_nets=2, seed=3) as s:
        rng = np.random.default_rng(4)
        X = rng.standard_normal((300, 8)).astype(np.float32)
        Y = rng.standard_normal((300, 65)).astype(np.float32)
        flat, _ = s.get_params(1)
        g, loss, yh = s.grads(1, X, Y)
    layers = mlp.unflatten(flat, DIMS)
    lo, go, yo = mlp.loss_and_grads(layers, _pad(X, 16), _pad(Y, 80), n_valid=65, m_valid=300,
                                    bf=True)
    assert np.abs(yh - yo[:, :65]).max() <= 1e-2 * max(1.0, np.abs(yo).max())
    assert loss == pytest.approx(lo, rel=1e-3)
    gg = mlp.unflatten(g, DIMS)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(gg, go)):
        assert np.linalg.norm(gW - oW) <= 1e-2 * np.linalg.norm(oW), l
        assert np.linalg.norm(gb - ob) <= 1e-2 * np.linalg.norm(ob) + 1e-12, l


def test_fused_inference_equals_layered_and_oracle(P, monkeypatch):
    """Prediction runs every layer of every network in one fused tcgen05 launch;
    it gives the same bits as the layer-by-layer GEMMs (same MMA sequence, same
    epilogue) and matches the float64 oracle's networks within BF16 rounding.
    300 rows: three 128-row tiles, the last one ragged."""
    rng = np.random.default_rng(9)
    X = rng.standard_normal((300, 8)).astype(np.float32)
    with P.Surrogate(n_in=8, n_hidden=256, n_layers=4, n_out=65, n_nets=3, seed=5) as s:
        m_f, sp_f = s.predict(X)
        monkeypatch.setenv("NPSIM_SURR_LAYERED", "1")
        m_l, sp_l = s.predict(X)
        monkeypatch.delenv("NPSIM_SURR_LAYERED")
        flats = [s.get_params(k)[0] for k in range(3)]
    assert np.array_equal(m_f, m_l) and np.array_equal(sp_f, sp_l)
    outs = []
    for flat in flats:
        _, _, yo = mlp.loss_and_grads(mlp.unflatten(flat, DIMS), _pad(X, 16),
                                      np.zeros((300, 80)), n_valid=65, m_valid=300, bf=True)
        outs.append(yo[:, :65])
    mean_o = np.mean(outs, axis=0)
    assert np.abs(m_f - mean_o).max() <= 1e-2 * max(1.0, np.abs(mean_o).max())


def test_surrogate_adamw_step_vs_oracle(P):
    lr, wd = 1e-3, 1e-2
    with P.Surrogate(n_in=8, n_hidden=256, n_layers=4, n_out=65, n_nets=1, seed=5) as s:
        rng = np.random.default_rng(6)
        X = rng.standard_normal((256, 8)).astype(np.float32)
        Y = rng.standard_normal((256, 65)).astype(np.float32)
        p0, _ = s.get_params(0)
        s.train(X, Y, epochs=1, batch=256, lr=lr, wd=wd, seed=0)  # one minibatch: all rows
        p1, g1 = s.get_params(0)
    # decay on weights only; padded (all-zero) entries are masked and stay zero
    dec = np.concatenate([np.concatenate([np.full(o * i, wd), np.zeros(o)]) for o, i in DIMS])
    valid = np.concatenate([np.concatenate([np.ones(o * i), np.ones(o)]) for o, i in DIMS]) > 0
    w1, _, _ = mlp.adamw(p0.astype(np.float64), g1.astype(np.float64), 0.0, 0.0, 1, lr,
                         wd=dec)
    live = (p0 != 0) | (g1 != 0)
    sel = live & (np.abs(g1) > 1e-6)
    assert np.abs(p1[sel] - w1[sel]).max() <= 1e-3 * lr + 1e-6 * np.abs(p0[sel]).max()
    assert np.all(p1[~live] == 0)


def test_surrogate_learns_smooth_function(P):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((8, 65)) / np.sqrt(8)
    X = rng.uniform(-1, 1, (4096, 8)).astype(np.float32)
    Xt = rng.uniform(-1, 1, (1024, 8)).astype(np.float32)
    f = lambda x: (np.sin(2 * x @ A) + 0.5 * (x @ A) ** 2).astype(np.float32)
    Y, Yt = f(X), f(Xt)
    with P.Surrogate(8, 256, 4, 65, n_nets=3, seed=8) as s:
        s.set_norm(X.mean(0), X.std(0), Y.mean(0), Y.std(0))
        _, loss0, _ = s.grads(0, X[:512], Y[:512])
        final = s.train(X, Y, epochs=40, batch=512, lr=2e-3, wd=1e-4, seed=1)
        m, sp = s.predict(Xt)
    assert final < 0.05 * loss0
    rmse = np.sqrt(((m - Yt) ** 2).mean(0))
    assert np.all(rmse <= 0.15 * Yt.std(0) + 1e-3)
    assert np.all(np.isfinite(sp)) and np.all(sp >= 0) and sp.mean() > 0


def test_bounded_wait_expiry_reports_timeout_and_recovers(P):
    """Failure path of the tensor-core kernels without a stuck GPU: with the
    bound of the GEMM kernel's main-loop waits cut to one SM cycle, the waits
    give up (a TMA copy or an MMA always takes longer), the kernel drains its
    copies and MMAs in flight with the default bound, frees its tensor memory
    and flags the timeout: npsim_gemm_bf16 and the surrogate's training return
    NPSIM_ERR_TIMEOUT.  With the default bound back, the same GEMM is correct
    and a fresh surrogate trains."""
    rng = np.random.default_rng(9)
    A = _bits(rng.standard_normal((256, 128)))
    B = _bits(rng.standard_normal((64, 128)))
    a, b = _val(A), _val(B)
    ref, scale = a @ b.T, np.abs(a) @ np.abs(b).T
    X = rng.standard_normal((256, 8)).astype(np.float32)
    Y = rng.standard_normal((256, 16)).astype(np.float32)
    try:
        P.npsim_test_wait_cycles(1)
        with pytest.raises(P.NpsimError) as e:
            P.npsim_gemm_bf16(A, B, 64)
        assert e.value.code == -4  # NPSIM_ERR_TIMEOUT
        with P.Surrogate(n_in=8, n_hidden=64, n_layers=2, n_out=16, n_nets=1, seed=0) as s:
            with pytest.raises(P.NpsimError) as e:
                s.train(X, Y, epochs=1, batch=128)
            assert e.value.code == -4
    finally:
        P.npsim_test_wait_cycles(0)
    Cg = P.npsim_gemm_bf16(A, B, 64)
    assert np.all(np.abs(Cg - ref) <= 2e-5 * scale + 1e-30)
    with P.Surrogate(n_in=8, n_hidden=64, n_layers=2, n_out=16, n_nets=1, seed=0) as s:
        loss = s.train(X, Y, epochs=2, batch=128)
        assert np.isfinite(loss)
    with pytest.raises(P.NpsimError):
        P.npsim_test_wait_cycles(-1)
