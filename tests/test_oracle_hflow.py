"""Pins of the oracle's Alg. 1 pieces (Sec. 4.1): the change of variable
u = div A + m0, the Gaussian blur, G(A) = F_eps(k * u) and its gradient, and
the Adam update."""
import numpy as np
import pytest

import oracle
from paper_2103_04856_gb300 import inputs as I


def P(a=(1.0, 0.3, 0.7, 0.2, -0.1, 0.1), eps=1.5, xi=1e-6, h=1.0, well=0):
    return {"a": a, "eps": eps, "xi": xi, "h": h, "well": well}


def test_gauss_weights_moments():
    for sigma in (1.0, 2.0, 3.5):
        R = int(np.ceil(3 * sigma))
        w = oracle.gauss_weights(sigma, R)
        j = np.arange(-R, R + 1)
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        np.testing.assert_allclose(w, w[::-1], rtol=0, atol=0)
        assert np.sum(j**2 * w) == pytest.approx(sigma**2, rel=0.03)   # truncated at 3 sigma
        np.testing.assert_allclose(w / w[R], np.exp(-j**2 / (2 * sigma**2)), rtol=1e-14)


def test_blur_delta_is_separable_gaussian():
    shape = (16, 18, 20)
    fp = {"blur_sigma": 2.0}
    d = np.zeros(shape)
    d[3, 5, 7] = 1.0
    b = oracle.blur(d, P(), fp)
    w = oracle.gauss_weights(2.0, 6)
    ref = np.zeros(shape)
    for dz in range(-6, 7):
        for dy in range(-6, 7):
            for dx in range(-6, 7):
                ref[(3 + dz) % 16, (5 + dy) % 18, (7 + dx) % 20] += w[dz + 6] * w[dy + 6] * w[dx + 6]
    np.testing.assert_allclose(b, ref, rtol=0, atol=1e-16)


def test_blur_self_adjoint_and_constant():
    rng = np.random.default_rng(1)
    shape = (9, 10, 11)
    a, c = rng.standard_normal(shape), rng.standard_normal(shape)
    fp = {"blur_sigma": 1.3}
    ka, kc = oracle.blur(a, P(), fp), oracle.blur(c, P(), fp)
    assert np.sum(ka * c) == pytest.approx(np.sum(a * kc), rel=1e-13)
    np.testing.assert_allclose(oracle.blur(np.full(shape, 0.37), P(), fp), 0.37, rtol=1e-15)


@pytest.mark.parametrize("sigma", [0.0, 1.5])
def test_field_keeps_mass_exactly(sigma):
    rng = np.random.default_rng(2)
    A = 0.05 * rng.standard_normal((3, 8, 9, 10))
    ut = oracle.hflow_field(A, P(h=0.7), {"m0": -0.31, "blur_sigma": sigma})
    assert ut.mean() == pytest.approx(-0.31, abs=1e-15)
    assert np.std(ut) > 1e-3


def test_flow_gradient_matches_central_differences():
    """dG/dA against central differences of G for every component of every
    voxel (smooth softplus width so a 1e-6 step never crosses its kink)."""
    rng = np.random.default_rng(3)
    A = 0.03 * rng.standard_normal((3, 5, 6, 4))
    p = P(xi=1e-2, h=0.8)
    fp = {"m0": 0.3, "blur_sigma": 1.0}
    G, gA = oracle.hflow_grad(A, p, fp)
    fd = np.empty_like(A)
    flat, d = A.reshape(-1), 1e-6
    for i in range(flat.size):
        v = flat[i]
        flat[i] = v + d
        gp, _ = oracle.hflow_grad(A, p, fp)
        flat[i] = v - d
        gm, _ = oracle.hflow_grad(A, p, fp)
        flat[i] = v
        fd.reshape(-1)[i] = (gp - gm) / (2 * d)
    assert np.max(np.abs(fd - gA)) < 1e-6 * np.max(np.abs(gA))
    assert G == pytest.approx(oracle.energy(oracle.hflow_field(A, p, fp), p), rel=1e-15)


def test_first_adam_step_closed_form():
    """From zero moments, bias correction makes the first step
    A1 = A0 - lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    A0 = 0.03 * rng.standard_normal((3, 6, 6, 6))
    p, fp = P(), {"m0": 0.3, "blur_sigma": 1.0, "lr": 2e-3}
    _, g = oracle.hflow_grad(A0, p, fp)
    A1, m, v, t, tr = oracle.hflow_run(A0, np.zeros_like(A0), np.zeros_like(A0), p, fp, 1)
    np.testing.assert_allclose(A1, A0 - 2e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-14)
    assert t == 1 and tr[0, 4] == 1
    assert tr[0, 1] == pytest.approx(np.max(np.abs(g))) and tr[0, 3] == pytest.approx(0.3, abs=1e-15)


def test_flow_descends():
    rng = np.random.default_rng(5)
    A = 0.02 * rng.standard_normal((3, 12, 12, 12))
    p, fp = P(a=(1, 2, 1, 0, 0, 0)), {"m0": 0.3, "blur_sigma": 1.0, "lr": 1e-2}
    A1, m, v, t, tr = oracle.hflow_run(A, np.zeros_like(A), np.zeros_like(A), p, fp, 60)
    assert tr[-1, 0] < 0.7 * tr[0, 0]              # Willmore energy of the blurred field decreases
    assert np.all(np.abs(tr[:, 3] - 0.3) < 1e-14)  # and the mass never moves
    assert t == 60
