"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term of
eq. Feps, a wrong sign or index, kappa1/kappa2 swapped, a wrong factor of eps,
a wrong adjoint) fails at least one of them:

  closed forms       tanh sphere / cylinder / slab energies tend to sigma times
                     the sharp-interface value under refinement (Thm. gamma_limsup,
                     Sec. 3.3) -- pins c1..c6 as a whole and the eps scaling
  ordering           cylinder: p = k1^2 >> p = k2^2 and p = k1 -> 2 pi L while
                     p = k2 -> 0 -- pins kappa1 >= kappa2 (Sec. 2.1) and the
                     signs of the c3 and c5 terms
  Willmore / Helfrich  eq. Feps with a_W / a_H equals the separately coded
                     eqs. Willmore_eps / Helfrich_eps (Sec. 3.2 comparison)
  phase swap         F[a](1-u) = F[a'](u) with a' = (a02, a11, a20, -a01, -a10, a00)
  double well        F_pm1(2u - 1) = 4 F_01(u)
  constant field     E = N h^3 (a10 - a01)/2 xi sqrt(xi ln 2), g = 0
  gradient           central finite differences on every voxel, and torch
                     FP64 autograd of the forward formula
  step / run         mass conservation, lambda = mean(g), energy decrease
  invariants         translation, axis permutation and reflection
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2103_04856_gb300 import inputs as I

SIGMA01 = math.sqrt(2.0) / 6.0          # int_0^1 sqrt(2 W(u)) du for W = u^2 (1-u)^2
HERE = os.path.dirname(os.path.abspath(__file__))


def prob(a, eps=1.5, h=1.0, xi=1e-6, well=0):
    return {"a": tuple(float(x) for x in a), "eps": eps, "h": h, "xi": xi, "well": well}


def rand_a(rng):
    return rng.uniform(-1.0, 1.0, 6)


# ---------------------------------------------------------------- tables

def test_b_to_a_printed_tables():
    rows = json.load(open(os.path.join(HERE, "golden", "b_to_a_tables.json")))["rows"]
    assert len(rows) == 8
    for r in rows:
        np.testing.assert_allclose(oracle.b_to_a(r["b"]), r["a"], rtol=0, atol=1e-9, err_msg=r["name"])


# ---------------------------------------------------------------- closed forms

def test_constant_field_closed_form():
    rng = np.random.default_rng(3)
    for well in (0, 1):
        a = rand_a(rng)
        u = np.full((6, 5, 7), 0.37)
        p = prob(a, eps=1.3, h=0.7, xi=1e-6, well=well)
        E, g = oracle.energy_and_grad(u, p)
        xi = p["xi"]
        expect = u.size * p["h"] ** 3 * (a[3] - a[4]) / 2.0 * xi * math.sqrt(xi * math.log(2.0))
        assert E == pytest.approx(expect, rel=1e-12)
        assert np.max(np.abs(g)) < 1e-14


def test_sphere_willmore_refines_to_8pi():
    # p = k1^2 + k2^2, sphere R = n/4, eps = n/64, i.e. fixed R/eps = 16
    ratios = []
    for n in (64, 96, 128):
        u = I.tanh_sphere((n, n, n), n / 4, n / 64)
        ratios.append(oracle.energy(u, prob((1, 0, 1, 0, 0, 0), eps=n / 64)) / SIGMA01 / (8 * math.pi))
    assert ratios[0] > ratios[1] > ratios[2] > 1.0
    assert ratios[2] == pytest.approx(1.1198, abs=2e-3)     # 8 pi within 12% at eps = 2h
    # the error shrinks faster than linearly in h/eps
    assert (ratios[2] - 1) < 0.5 * (ratios[1] - 1)


def test_sphere_gauss_and_area():
    n = 128
    u = I.tanh_sphere((n, n, n), 32, 2.0)
    K = oracle.energy(u, prob((0, 1, 0, 0, 0, 0), eps=2.0)) / SIGMA01
    A = oracle.energy(u, prob((0, 0, 0, 0, 0, 1), eps=2.0)) / SIGMA01
    assert K / (4 * math.pi) == pytest.approx(0.889, abs=0.01)     # Gauss-Bonnet 4 pi
    assert A / (4 * math.pi * 32 ** 2) == pytest.approx(1.0, abs=0.02)


def test_cylinder_orders_kappa1_above_kappa2():
    n, r, eps = 96, 15.0, 1.5
    u = I.tanh_cylinder((n, n, n), r, eps)
    L = n

    def F(a):
        return oracle.energy(u, prob(a, eps=eps)) / SIGMA01

    k1sq, k2sq = F((1, 0, 0, 0, 0, 0)), F((0, 0, 1, 0, 0, 0))
    k1, k2 = F((0, 0, 0, 1, 0, 0)), F((0, 0, 0, 0, 1, 0))
    area = F((0, 0, 0, 0, 0, 1))
    assert k1sq / (2 * math.pi * L / r) == pytest.approx(1.0, abs=0.1)
    assert k2sq < 0.25 * k1sq
    assert k1 / (2 * math.pi * L) == pytest.approx(1.0, abs=0.03)   # u high inside: H > 0
    assert abs(k2) < 0.03 * k1
    assert area / (2 * math.pi * r * L) == pytest.approx(1.0, abs=0.05)


def test_slab_area_refines():
    vals = []
    for eps in (1.5, 3.0):
        n = 64
        u = I.tanh_slab((n, 8, 8), n / 2, eps)
        vals.append(oracle.energy(u, prob((0, 0, 0, 0, 0, 1), eps=eps)) / SIGMA01 / (2 * 8 * 8))
    assert abs(vals[1] - 1) < abs(vals[0] - 1) < 0.07
    assert vals[1] == pytest.approx(1.0, abs=0.02)


# ---------------------------------------------------------------- reductions

def _np_sh(u, dx, dy, dz):
    return np.roll(u, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def _np_M(u, eps, xi, h, well):
    G = [(_np_sh(u, 1, 0, 0) - _np_sh(u, -1, 0, 0)) / (2 * h),
         (_np_sh(u, 0, 1, 0) - _np_sh(u, 0, -1, 0)) / (2 * h),
         (_np_sh(u, 0, 0, 1) - _np_sh(u, 0, 0, -1)) / (2 * h)]
    lap = sum(_np_sh(u, *s) - 2 * u + _np_sh(u, *[-x for x in s]) for s in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]) / h**2
    g2 = G[0] ** 2 + G[1] ** 2 + G[2] ** 2
    Wp = u**3 - u if well == 1 else 2 * u * (1 - u) * (1 - 2 * u)
    return G, lap, g2, Wp


def test_willmore_reduction():
    """eq. Feps with a = (1,2,1,0,0,0) equals eq. Willmore_eps, (1/eps) int (eps Lap u - W'/eps)^2,
    up to the xi offset inside n_u (relative size xi^2/|grad u|^2)."""
    # off-grid centre: no voxel has grad u = 0 exactly, where the regularised
    # normal vanishes instead of being a unit vector
    sph = I.tanh_sphere((24, 24, 24), 7, 1.5, center=(11.3, 12.1, 11.7), well=1)
    for well, u in ((0, I.noise((10, 12, 14), 0.3, 0.1, 5)), (1, sph)):
        eps, h = 1.5, 1.0
        _, lap, g2, Wp = _np_M(u, eps, 1e-6, h, well)
        Weps = (1 / eps) * np.sum((eps * lap - Wp / eps) ** 2) * h**3
        F = oracle.energy(u, prob((1, 2, 1, 0, 0, 0), eps=eps, well=well))
        assert F == pytest.approx(Weps, rel=1e-8)


def test_helfrich_reduction():
    """eq. Feps with a_H = (chi_b/2, chi_b + chi_G, chi_b/2, -chi_b H0, -chi_b H0, chi_b H0^2/2)
    equals eq. Helfrich_eps evaluated by its own formula."""
    rng = np.random.default_rng(11)
    u = I.noise((9, 10, 11), 0.35, 0.12, 6)
    eps, h, xi = 1.5, 1.0, 1e-6
    G, lap, g2, Wp = _np_M(u, eps, xi, h, 0)
    e3 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    Hs = [[None] * 3 for _ in range(3)]
    for c in range(3):
        Hs[c][c] = (_np_sh(u, *e3[c]) - 2 * u + _np_sh(u, *[-x for x in e3[c]])) / h**2
        for d in range(c + 1, 3):
            s, t = np.array(e3[c]), np.array(e3[d])
            Hs[c][d] = Hs[d][c] = (_np_sh(u, *(s + t)) - _np_sh(u, *(s - t)) - _np_sh(u, *(-s + t))
                                   + _np_sh(u, *(-s - t))) / (4 * h**2)
    rho = g2 + xi**2
    M = [[-eps * Hs[i][j] + Wp / eps * G[i] * G[j] / rho for j in range(3)] for i in range(3)]
    TrM = M[0][0] + M[1][1] + M[2][2]
    M2 = sum(M[i][j] ** 2 for i in range(3) for j in range(3))
    for _ in range(3):
        chib, chiG, H0 = rng.uniform(0.2, 2.0), rng.uniform(-1.0, 1.0), rng.uniform(-0.5, 0.5)
        Heps = np.sum(chib / (2 * eps) * (TrM - eps * np.sqrt(rho) * H0) ** 2
                      + chiG / (2 * eps) * (TrM**2 - M2)) * h**3
        aH = (chib / 2, chib + chiG, chib / 2, -chib * H0, -chib * H0, chib * H0**2 / 2)
        F = oracle.energy(u, prob(aH, eps=eps, xi=xi))
        # expanding the square gives eps^2 H0^2 |grad u|^2 with the regularised norm,
        # while eq. Feps's a00 term uses the plain |grad u|^2: remove the xi^2 part
        Heps_plain = Heps - np.sum(chib / (2 * eps) * (eps * H0) ** 2 * (rho - g2)) * h**3
        assert F == pytest.approx(Heps_plain, rel=1e-10)


def test_phase_swap_identity():
    rng = np.random.default_rng(21)
    u = I.noise((8, 9, 10), 0.4, 0.15, 7)
    for _ in range(3):
        a = rand_a(rng)
        asw = (a[2], a[1], a[0], -a[4], -a[3], a[5])
        E1, g1 = oracle.energy_and_grad(1.0 - u, prob(a))
        E2, g2 = oracle.energy_and_grad(u, prob(asw))
        assert E1 == pytest.approx(E2, rel=1e-11)
        np.testing.assert_allclose(-g1, g2, rtol=0, atol=1e-11 * np.max(np.abs(g2)))


def test_double_well_plumbing():
    # symmetric p: exact up to the xi offsets
    u = I.tanh_sphere((20, 20, 20), 6, 1.5)
    a = (1.0, 0.3, 1.0, 0.2, 0.2, 0.5)
    F01 = oracle.energy(u, prob(a))
    Fpm = oracle.energy(2 * u - 1, prob(a, well=1))
    assert Fpm == pytest.approx(4 * F01, rel=1e-8)
    # asymmetric p on noise: the softplus of 4D and 4 softplus(D) differ only where |D| ~ xi
    u = I.noise((10, 10, 10), 0.3, 0.1, 8)
    a = (0.7, -0.2, 0.1, 0.5, -0.3, 0.2)
    assert oracle.energy(2 * u - 1, prob(a, well=1)) == pytest.approx(4 * oracle.energy(u, prob(a)), rel=1e-5)


# ---------------------------------------------------------------- gradient

def _fd_grad(u, p, delta):
    g = np.empty_like(u)
    flat = u.reshape(-1)
    for i in range(flat.size):
        v = flat[i]
        flat[i] = v + delta
        ep = oracle.energy(u, p)
        flat[i] = v - delta
        em = oracle.energy(u, p)
        flat[i] = v
        g.reshape(-1)[i] = (ep - em) / (2 * delta)
    return g


@pytest.mark.parametrize("well", [0, 1])
def test_gradient_matches_central_differences(well):
    """Every voxel, with a softplus width xi = 1e-2 so that a perturbation of
    1e-5 never crosses the kink of sqrt(x^+) (the adjoint formulas do not
    depend on xi)."""
    rng = np.random.default_rng(31 + well)
    shape = (6, 7, 8)          # ragged, every wrap path
    u = I.noise(shape, 0.3, 0.1, 9) if well == 0 else I.noise(shape, -0.2, 0.3, 9)
    p = prob(rand_a(rng), eps=1.5, h=0.9, xi=1e-2, well=well)
    _, g = oracle.energy_and_grad(u, p)
    gfd = _fd_grad(u.copy(), p, 1e-5)
    err = np.abs(g - gfd)
    assert np.max(err) < 1e-6 * np.max(np.abs(g)), np.max(err)


def test_gradient_central_differences_default_xi():
    """xi = 1e-6: voxels whose neighbourhood sits on the kink (where two step
    sizes disagree) are left out; at least 90% must remain and all agree."""
    rng = np.random.default_rng(35)
    u = I.noise((6, 7, 8), 0.3, 0.1, 13)
    p = prob(rand_a(rng), eps=1.5)
    _, g = oracle.energy_and_grad(u, p)
    f1 = _fd_grad(u.copy(), p, 1e-5)
    f2 = _fd_grad(u.copy(), p, 1e-6)
    scale = np.max(np.abs(g))
    smooth = np.abs(f1 - f2) < 1e-7 * scale
    assert smooth.mean() > 0.9
    assert np.max(np.abs(g - f1)[smooth]) < 1e-6 * scale


def _fd_grad_local(u, p, delta):
    """Central differences of the energy with respect to every voxel, each
    from the densities of the 3 x 3 x 3 voxels around it (periodic): the
    19-point stencils of eq. Feps reach no further, so the rest of the sum
    cancels exactly and only the window's change is differenced."""
    nz, ny, nx = u.shape
    g = np.empty_like(u)
    off = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                wz, wy, wx = (z + off[:, 0]) % nz, (y + off[:, 1]) % ny, (x + off[:, 2]) % nx
                v = u[z, y, x]
                u[z, y, x] = v + delta
                ep = oracle.density(u, p)[wz, wy, wx].sum()
                u[z, y, x] = v - delta
                em = oracle.density(u, p)[wz, wy, wx].sum()
                u[z, y, x] = v
                g[z, y, x] = (ep - em) / (2 * delta)
    return g


def test_gradient_central_differences_all_voxels_16():
    """All 4096 voxels of a 16^3 noise field (asymmetric p, FP64): with a
    smooth softplus (xi = 1e-2) every voxel agrees with its central
    difference (delta 1e-5); at the default xi = 1e-6 the voxels whose two
    step sizes (1e-5, 1e-6) disagree sit at the sqrt(x^+) kink and are left
    out, at least 90 % remain (96 % here), and they agree too.  (A step of
    1e-3 crosses the kink, whose width is xi, at one voxel in ten.)"""
    rng = np.random.default_rng(47)
    a = rand_a(rng)
    u = I.noise((16, 16, 16), 0.3, 0.1, 17)
    p = prob(a, eps=1.5, xi=1e-2)
    _, g = oracle.energy_and_grad(u, p)
    gfd = _fd_grad_local(u.copy(), p, 1e-5)
    assert np.max(np.abs(g - gfd)) < 1e-6 * np.max(np.abs(g))
    p = prob(a, eps=1.5)
    _, g = oracle.energy_and_grad(u, p)
    f1 = _fd_grad_local(u.copy(), p, 1e-5)
    f2 = _fd_grad_local(u.copy(), p, 1e-6)
    scale = np.max(np.abs(g))
    smooth = np.abs(f1 - f2) < 1e-7 * scale
    assert smooth.mean() > 0.9
    assert np.max(np.abs(g - f1)[smooth]) < 1e-6 * scale


def test_gradient_matches_torch_autograd():
    ref_torch = pytest.importorskip("ref_torch")
    rng = np.random.default_rng(41)
    for shape, well in (((8, 10, 12), 0), ((5, 6, 7), 1)):
        u = I.noise(shape, 0.3 if well == 0 else 0.0, 0.1 if well == 0 else 0.4, 10)
        p = prob(rand_a(rng), eps=1.7, h=1.1, well=well)
        E, g = oracle.energy_and_grad(u, p)
        Et, gt = ref_torch.energy_and_grad(u, p)
        assert E == pytest.approx(Et, rel=1e-12)
        np.testing.assert_allclose(g, gt, rtol=0, atol=1e-11 * np.max(np.abs(gt)))


def test_grad_sampled_equals_full():
    rng = np.random.default_rng(51)
    u = I.noise((9, 8, 7), 0.3, 0.1, 11)
    p = prob(rand_a(rng))
    _, g = oracle.energy_and_grad(u, p)
    idx = rng.integers(0, u.size, 40)
    np.testing.assert_allclose(oracle.grad_sampled(u, p, idx), g.reshape(-1)[idx], rtol=0, atol=1e-14)


# ---------------------------------------------------------------- step / run

def test_step_conserves_mass_and_descends():
    inst = I.willmore_descent_32()
    u0 = inst.field()[:16, :16, :16].copy()
    p = inst.problem()
    u, tr = oracle.run(u0, p, 12, 1e-3)
    m0 = u0.mean()
    assert abs(u.mean() - m0) < 1e-14
    np.testing.assert_allclose(tr[:, 1], m0, rtol=0, atol=1e-14)
    assert np.all(np.diff(tr[:, 0]) < 0)            # gradient descent with a small step
    # lambda is the mean gradient of the state the row evaluates
    _, g = oracle.energy_and_grad(u0, p)
    assert tr[0, 2] == pytest.approx(g.mean(), rel=1e-12, abs=1e-18)
    assert tr[0, 3] == pytest.approx(np.max(np.abs(g)), rel=1e-14)
    assert tr[0, 4] == pytest.approx(np.mean(np.abs(g)), rel=1e-12)
    # one explicit step by hand
    u1, sc = oracle.step(u0, p, 1e-3)
    np.testing.assert_allclose(u1, u0 - 1e-3 * (g - g.mean()), rtol=0, atol=1e-15)


# ---------------------------------------------------------------- invariants

def test_translation_permutation_reflection():
    rng = np.random.default_rng(61)
    u = I.noise((8, 9, 10), 0.3, 0.1, 12)
    p = prob(rand_a(rng))
    E, g = oracle.energy_and_grad(u, p)
    ur = np.roll(u, (2, -3, 1), axis=(0, 1, 2))
    Er, gr = oracle.energy_and_grad(ur, p)
    assert Er == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(gr, np.roll(g, (2, -3, 1), axis=(0, 1, 2)), rtol=0, atol=1e-12 * np.max(np.abs(g)))
    ut = np.ascontiguousarray(np.transpose(u, (2, 0, 1)))
    Et, gt = oracle.energy_and_grad(ut, p)
    assert Et == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(gt, np.transpose(g, (2, 0, 1)), rtol=0, atol=1e-12 * np.max(np.abs(g)))
    uf = np.ascontiguousarray(u[:, ::-1, :])
    Ef, gf = oracle.energy_and_grad(uf, p)
    assert Ef == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(gf, g[:, ::-1, :], rtol=0, atol=1e-12 * np.max(np.abs(g)))


def test_curvatures_on_shapes():
    n = 64
    u = I.tanh_sphere((n, n, n), 16, 1.5)
    k1, k2 = oracle.curvatures(u, prob((1, 0, 1, 0, 0, 0)))
    band = np.abs(u - 0.5) < 0.2
    assert np.all(k1 >= k2)
    # sum of the curvatures (the diffuse mean curvature H^eps) is 2/R; sqrt(D^+)
    # picks up the discretisation error of D, so kappa1 alone is biased upward
    assert np.median(k1[band] + k2[band]) * 16 / 2 == pytest.approx(1.0, abs=0.15)
    assert np.median(k2[band]) * 16 == pytest.approx(1.0, abs=0.05)
    u = I.tanh_cylinder((16, n, n), 12, 1.5)
    k1, k2 = oracle.curvatures(u, prob((1, 0, 1, 0, 0, 0)))
    band = np.abs(u - 0.5) < 0.2
    assert np.median(k1[band]) * 12 == pytest.approx(1.0, abs=0.05)
    assert abs(np.median(k2[band])) * 12 < 0.05
