"""Warm-start network: CUDA forward / backward / Adam against the FP64 oracle.

Tolerances (FP32 kernels vs FP64 oracle on identical parameters): forward
outputs within 1e-5 of the output scale; every parameter-gradient tensor
within 1e-4 of that tensor's largest oracle entry; five Adam steps within
1e-4 relative in the parameters.
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1509_08391_gb300 import llr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_08391_gb300 import build
    build.build()


def flat_to_list(flat):
    out, k = [], 0
    for s in omlp.SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(flat[k:k + n], dtype=np.float64).reshape(s))
        k += n
    return out


def list_to_flat(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    L = rng.choice([8.0, 12.0, 16.0], size=n)
    e = rng.uniform(0.58, 0.68, size=n)
    d = 8.0 * (L / 8.0) ** 2 / (6.0 * L ** 4)
    t = -1.0 - 1.5 * (e - 0.63) + 0.1 * np.sin(30 * e) + 0.05 / L
    return L, e, d, t


def _oracle_features(L, e, d, mean, std):
    raw = omlp.features(L, e, d)
    return (raw - mean) / std


def test_forward_matches_oracle():
    L, e, d, _ = _data(333, 1)
    with llr.MLP(seed=7) as net:
        raw = omlp.features(L, e, d)
        mean, std = raw.mean(axis=0), raw.std(axis=0)
        net.set_norm(mean, std)
        p = flat_to_list(net.get_params().astype(np.float64))
        y_gpu = net.predict(L, e, d)
        y_or, _ = omlp.forward(p, _oracle_features(L, e, d, mean, std))
        scale = max(1.0, np.max(np.abs(y_or)))
        assert np.max(np.abs(y_gpu - y_or)) <= 1e-5 * scale


def test_gradients_match_oracle():
    L, e, d, t = _data(257, 2)
    rng = np.random.default_rng(3)
    with llr.MLP(seed=11) as net:
        raw = omlp.features(L, e, d)
        mean, std = raw.mean(axis=0), raw.std(axis=0)
        net.set_norm(mean, std)
        p = flat_to_list(net.get_params().astype(np.float64))
        p = [q + 0.05 * rng.normal(size=q.shape) for q in p]   # nonzero biases too
        flat = list_to_flat(p)
        net.set_params(flat)
        p = flat_to_list(flat.astype(np.float64))              # exactly what the GPU holds
        g_gpu, loss_gpu = net.grad(L, e, d, t)
        x = _oracle_features(L, e, d, mean, std)
        g_or = omlp.backward(p, x, t)
        assert abs(loss_gpu - omlp.loss(p, x, t)) <= 1e-5 * max(1.0, omlp.loss(p, x, t))
        for k, (gg, go) in enumerate(zip(flat_to_list(g_gpu.astype(np.float64)), g_or)):
            scale = max(np.max(np.abs(go)), 1e-12)
            assert np.max(np.abs(gg - go)) <= 1e-4 * scale, (k, np.max(np.abs(gg - go)), scale)


def test_adam_steps_match_oracle():
    L, e, d, t = _data(200, 4)
    with llr.MLP(seed=5) as net:
        raw = omlp.features(L, e, d)
        mean, std = raw.mean(axis=0), raw.std(axis=0)
        p = flat_to_list(net.get_params().astype(np.float64))
        net.set_params(list_to_flat(p))
        net.fit(L, e, d, t, epochs=5, lr=1e-3, standardise=True)
        m_gpu, s_gpu = net.get_norm()
        assert np.allclose(m_gpu, mean, rtol=1e-12) and np.allclose(s_gpu, std, rtol=1e-12)
        x = _oracle_features(L, e, d, mean, std)
        opt = omlp.Adam(p, lr=1e-3)
        for _ in range(5):
            p = opt.step(p, omlp.backward(p, x, t))
        got = flat_to_list(net.get_params().astype(np.float64))
        for a, b in zip(got, p):
            assert np.max(np.abs(a - b)) <= 1e-4 * max(1.0, np.max(np.abs(b)))


def test_training_fits_a_smooth_slope_curve():
    L, e, d, t = _data(600, 6)
    with llr.MLP(seed=9) as net:
        raw = omlp.features(L, e, d)
        var = np.var(t)
        loss = net.fit(L, e, d, t, epochs=3000, lr=2e-3, standardise=True)
        assert loss < 0.02 * var
        Lh, eh, dh, th = _data(200, 60)
        pred = net.predict(Lh, eh, dh)
        assert np.sqrt(np.mean((pred - th) ** 2)) < 0.2 * np.sqrt(var)
