"""Pins of the surrogate oracle (oracle/surrogate.py): bfloat16 rounding against its
definition, backpropagation against central finite differences, closed forms of a
network with zero weights, the first Adam step, and a short fit."""
import numpy as np
import pytest

from oracle import surrogate as S


def test_bf16_is_the_nearest_bfloat16():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5]])
    r = S.bf16(x)
    bits = r.astype(np.float32).view(np.uint32)
    assert (bits & 0xFFFF == 0).all()                       # a bfloat16 value
    # both bfloat16 neighbours of x are at least as far as r
    up = (x.astype(np.float32).view(np.uint32) & 0xFFFF0000).astype(np.uint32)
    lo = up.view(np.float32).astype(np.float64)
    hi = (up + 0x10000).view(np.float32).astype(np.float64)
    assert (np.abs(r - x) <= np.minimum(np.abs(lo - x), np.abs(hi - x)) + 0.0).all()
    assert r[-4] == 1.0 and r[-3] == 1.0                    # tie to even
    assert r[-2] == 1.0 + 2.0 ** -7 and r[-1] == -2.5


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = S.init_params(3, 1)[0] + 0.05 * rng.standard_normal(S.NPARAM)
    x = rng.standard_normal((7, 2))
    t = rng.standard_normal((7, 2))
    _, g = S.loss_and_grad(p, x, t, bf16_mode=False)
    idx = rng.choice(S.NPARAM, 300, replace=False)
    idx = np.concatenate([idx, np.arange(S.NPARAM - 2, S.NPARAM), np.arange(0, 4)])
    h = 1e-6
    for k in idx:
        e = np.zeros(S.NPARAM)
        e[k] = h
        lp, _ = S.loss_and_grad(p + e, x, t, bf16_mode=False)
        lm, _ = S.loss_and_grad(p - e, x, t, bf16_mode=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_zero_weight_network_closed_form():
    d = {name: np.zeros(shp) for name, shp in S.SHAPES}
    d["b1"][:] = 0.3
    d["b3"][:] = -0.2
    d["b4"][:] = [0.5, -1.0]
    p = S.pack(d)
    x = np.array([[1.0, 2.0], [-1.0, 0.5], [0.0, 0.0]])
    t = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, -1.0]])
    y, _ = S.forward(p, x, bf16_mode=False)
    assert np.allclose(y, [[0.5, -1.0]] * 3, rtol=0, atol=0)
    loss, g = S.loss_and_grad(p, x, t, bf16_mode=False)
    gd = S.unpack(g)
    dy = 2 * (y - t) / 6.0
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-15)
    assert np.allclose(gd["b4"], dy.sum(axis=0), rtol=1e-15)
    assert np.allclose(gd["W4"], np.outer(dy.sum(axis=0), np.tanh(-0.2) * np.ones(S.H)), rtol=1e-14)
    for name in ("W1", "W2", "W3", "b1", "b2", "b3"):  # nothing flows back through W4 = 0
        assert not gd[name].any()


def test_first_adam_step_has_size_lr():
    g = np.array([1e-3, -2.0, 5.0, 0.0])
    p, m, v = S.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=1e-2)
    assert np.allclose(p[:3], -1e-2 * np.sign(g[:3]), rtol=1e-4)
    assert p[3] == 0.0 and np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_gradient_close_to_fp64_and_short_fit_converges():
    rng = np.random.default_rng(2)
    p = S.init_params(4, 1)[0]
    x = rng.uniform(-1, 1, (256, 2))
    t = np.stack([np.sin(2 * x[:, 0]) + x[:, 1] ** 2, x[:, 0] * x[:, 1]], axis=1)
    l0, g16 = S.loss_and_grad(p, x, t, bf16_mode=True)
    _, g64 = S.loss_and_grad(p, x, t, bf16_mode=False)
    assert np.linalg.norm(g16 - g64) <= 0.05 * np.linalg.norm(g64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for k in range(1, 301):
        _, g = S.loss_and_grad(p, x, t)
        p, m, v = S.adam_step(p, g, m, v, k, lr=3e-3)
    l1, _ = S.loss_and_grad(p, x, t)
    assert l1 < 0.1 * l0
