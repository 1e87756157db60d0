"""Pins of the FP64 MLP oracle (no GPU): backprop against central finite
differences, Adam's closed-form first step, ensemble statistics, and that
training lowers the loss on a smooth target."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def rand_params(rng, scale=0.5):
    return rng.normal(size=M.N_PARAMS) * scale


def test_layout():
    assert M.N_PARAMS == 4 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    p = np.arange(M.N_PARAMS, dtype=float)
    assert np.array_equal(M.pack(*M.unpack(p)), p)


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rand_params(rng, 0.3)
    z = rng.uniform(-1, 1, size=(16, 4))
    t = rng.normal(size=16)
    loss, g = M.loss_and_grad(p, z, t)
    idx = rng.choice(M.N_PARAMS, 300, replace=False)
    idx = np.concatenate([idx, [M.OFF_B3, M.OFF_W1, M.OFF_B1, M.OFF_W2 + 5, M.OFF_B2 + 7, M.OFF_W3 + 3]])
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = 1e-6
        fd = (M.loss_and_grad(p + e, z, t)[0] - M.loss_and_grad(p - e, z, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_output_bias_gradient_closed_form():
    """With W2 = 0 and b2 = 0 the hidden layer is 0, y = b3 and
    dL/db3 = 2 mean(y - t), dL/dw3 = 0."""
    rng = np.random.default_rng(2)
    W1, b1, W2, b2, w3, b3 = M.unpack(rand_params(rng))
    p = M.pack(W1, b1, np.zeros_like(W2), np.zeros_like(b2), w3, 0.7)
    z = rng.uniform(-1, 1, size=(32, 4))
    t = rng.normal(size=32)
    loss, g = M.loss_and_grad(p, z, t)
    assert loss == pytest.approx(np.mean((0.7 - t) ** 2), rel=1e-14)
    assert g[M.OFF_B3] == pytest.approx(2 * np.mean(0.7 - t), rel=1e-13)
    assert np.all(g[M.OFF_W3:M.OFF_B3] == 0.0)


def test_adam_first_step_moves_by_lr_sign():
    rng = np.random.default_rng(3)
    p = rand_params(rng)
    g = rng.normal(size=M.N_PARAMS)
    p1, m, v = M.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    # bias-corrected first moments are g and g^2: the step is lr g / (|g| + eps)
    np.testing.assert_allclose(p - p1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)


def test_ensemble_of_identical_members_has_zero_spread():
    rng = np.random.default_rng(4)
    p = rand_params(rng)
    z = rng.uniform(-1, 1, size=(10, 4))
    mean, spread = M.ensemble_predict(np.stack([p, p, p]), z)
    np.testing.assert_allclose(mean, M.forward(p, z)[0], rtol=1e-15)
    assert np.all(spread == 0.0)


def test_training_lowers_the_loss():
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, size=(2000, 4))
    t = np.sin(2 * z[:, 0]) + 0.5 * z[:, 1] * z[:, 2] + 2.0
    p0 = rand_params(rng, 0.2)
    p, losses = M.train(p0, z, t, 600, 128, 3e-3, rng)
    assert losses[-50:].mean() < 0.05 * losses[:10].mean()


def test_adam_constant_gradient_moves_lr_per_step():
    """Under a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step (Kingma & Ba 2015, Sec. 3), so t steps move each
    parameter by t lr g / (|g| + eps): pins the step count in both bias
    corrections."""
    rng = np.random.default_rng(6)
    p0 = rand_params(rng)
    g = rng.normal(size=M.N_PARAMS)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 6):
        p, m, v = M.adam_step(p, g, m, v, t, 2e-3)
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-13)
        np.testing.assert_allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)
    np.testing.assert_allclose(p0 - p, 5 * 2e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_splitmix64_published_sequence():
    """SplitMix64 from state 0 (Steele, Lea & Flood 2014; the reference C
    implementation's generator): the first four outputs."""
    x, out = 0, []
    for _ in range(4):
        out.append(M.splitmix64(x))
        x = (x + M.GOLDEN_GAMMA) & M.MASK64
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_batch_rows_are_uniform_and_distinct_per_member_and_step():
    n = 1000
    rows = np.concatenate([M.batch_rows(99, k, t, n) for k in range(4) for t in range(1, 41)])
    assert rows.min() >= 0 and rows.max() < n
    # 20,480 draws over 10 bins of 100 rows: chi-square with 9 dof, p ~ 1e-4 at 33
    counts = np.bincount(rows // 100, minlength=10)
    chi2 = np.sum((counts - rows.size / 10) ** 2 / (rows.size / 10))
    assert chi2 < 33.0, counts
    a, b, c = M.batch_rows(99, 0, 1, n), M.batch_rows(99, 1, 1, n), M.batch_rows(99, 0, 2, n)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(a, M.batch_rows(99, 0, 1, n))


def _adam_variant(p, g, m, v, step, lr, kind, beta1=0.9, beta2=0.999, eps=1e-8):
    """adam_step with one planted mistake (for the criterion's power only)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    if kind == "no_bias_correction":
        mhat, vhat = m, v
    elif kind == "step_from_zero":
        mhat, vhat = m / (1.0 - beta1 ** (step + 1)), v / (1.0 - beta2 ** (step + 1))
    else:
        mhat, vhat = m / (1.0 - beta1 ** step), v / (1.0 - beta2 ** step)
    if kind == "eps_inside_sqrt":
        return p - lr * mhat / np.sqrt(vhat + eps), m, v
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


@pytest.mark.parametrize("kind", ["no_bias_correction", "step_from_zero", "eps_inside_sqrt"])
def test_adam_parity_criterion_catches_planted_mistakes(kind):
    """The GPU Adam test's criterion -- >= 99 % of the parameter updates within
    1e-3 lr per step of the oracle's, after 1 and 5 steps -- fails for an
    update with a missing or mis-stepped bias correction or with eps inside
    the square root, on gradients of the test's scale (the network's own
    gradients of a random minibatch)."""
    rng = np.random.default_rng(8)
    p0 = rand_params(rng, 0.3)
    z = rng.uniform(-1, 1, size=(128, 4))
    t = 2.0 + rng.normal(size=128)
    lr = 1e-3
    caught = []
    for steps in (1, 5):
        p_ok, m_ok, v_ok = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
        p_bad, m_bad, v_bad = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
        for k in range(1, steps + 1):
            _, g_ok = M.loss_and_grad(p_ok, z, t)
            _, g_bad = M.loss_and_grad(p_bad, z, t)
            p_ok, m_ok, v_ok = M.adam_step(p_ok, g_ok, m_ok, v_ok, k, lr)
            p_bad, m_bad, v_bad = _adam_variant(p_bad, g_bad, m_bad, v_bad, k, lr, kind)
        within = np.abs((p_bad - p0) - (p_ok - p0)) <= 1e-3 * lr * steps
        caught.append(within.mean() < 0.99)
    assert any(caught), kind
