"""Pins of the oracle's extensions (Sec. 5.2) and diagnostics (Sec. 4.5).

  orientation term  eps mu (theta . grad u)^2: closed form on a sine field (the
                    central difference of sin is sin(k) cos(kx)), the axis-sum
                    identity sum over theta = e_x, e_y, e_z equals the a00 term
                    with a00 = mu, and central differences of the gradient
  a(x)              the integrand is linear in a, so E(a(x)) equals the sum over
                    k of a_k(x) times the density with a = e_k; central
                    differences of the gradient with a random a(x)
  m(x)              u = div A + m(x): with A = 0 and no blur u is m(x), and the
                    mean of u is the mean of m for any A
  diagnostics       constant field (discrepancy = Cahn-Hilliard = N h^3 W(c)/eps),
                    tanh slab (equipartition: the ratio vanishes like (h/eps)^2
                    and the Cahn-Hilliard energy tends to sigma times the area)
  surface cells     flat interfaces along each axis: exact area, zero curvature;
                    tanh sphere: area -> 4 pi R^2 under refinement, mean of
                    kappa1 + kappa2 -> 2/R; tanh cylinder: area -> 2 pi r L,
                    kappa1 -> 1/r, kappa2 -> 0
"""
import math

import numpy as np
import pytest

import oracle
from paper_2103_04856_gb300 import inputs as I


def prob(a, eps=1.5, h=1.0, xi=1e-6, well=0, **kw):
    d = {"a": tuple(float(x) for x in a), "eps": eps, "h": h, "xi": xi, "well": well}
    d.update(kw)
    return d


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


# ------------------------------------------------------------ orientation

@pytest.mark.parametrize("h", [1.0, 0.7])
def test_orientation_sine_closed_form(h):
    """u = c + s sin(2 pi x / L): G_x = s sin(2 pi / L) cos(2 pi x / L) / h, so
    h^3 sum eps mu (theta . G)^2 = h eps mu s^2 sin^2(2 pi / L) theta_x^2 N / 2."""
    nz, ny, nx = 3, 4, 10
    s, c, eps, mu = 0.3, 0.4, 1.3, 2.5
    x = np.arange(nx)
    u = np.broadcast_to(c + s * np.sin(2 * math.pi * x / nx), (nz, ny, nx)).copy()
    a = (0.7, -0.2, 0.4, 0.3, -0.1, 0.2)
    base = oracle.energy(u, prob(a, eps=eps, h=h))
    N = nx * ny * nz
    for phi in (0.0, 0.4, 1.1, math.pi / 2):
        th = (math.cos(phi), math.sin(phi) * 0.6, math.sin(phi) * 0.8)
        E = oracle.energy(u, prob(a, eps=eps, h=h, mu=mu, theta=th))
        want = h * eps * mu * s * s * math.sin(2 * math.pi / nx) ** 2 * th[0] ** 2 * N / 2
        assert E - base == pytest.approx(want, rel=1e-10, abs=1e-12)


def test_orientation_axis_sum_equals_a00_term():
    rng = np.random.default_rng(5)
    u = I.noise((5, 6, 7), 0.3, 0.2, 4)
    a = rng.uniform(-1, 1, 6)
    mu = 1.7
    p0 = prob(a, h=0.8)
    E0, g0 = oracle.energy_and_grad(u, p0)
    Es, gs = 0.0, np.zeros_like(u)
    for th in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        E, g = oracle.energy_and_grad(u, prob(a, h=0.8, mu=mu, theta=th))
        Es += E - E0
        gs += g - g0
    Ea, ga = oracle.energy_and_grad(u, prob((0, 0, 0, 0, 0, mu), h=0.8))
    assert Es == pytest.approx(Ea, rel=1e-11)
    np.testing.assert_allclose(gs, ga, rtol=0, atol=1e-11 * np.max(np.abs(ga)))


def test_orientation_gradient_central_differences():
    rng = np.random.default_rng(8)
    u = I.noise((6, 7, 8), 0.3, 0.1, 21)
    th = rng.normal(size=3)
    th /= np.linalg.norm(th)
    p = prob(rng.uniform(-1, 1, 6), eps=1.5, h=0.9, xi=1e-2, mu=3.0, theta=tuple(th))
    _, g = oracle.energy_and_grad(u, p)
    gfd = _fd_grad(u.copy(), p, 1e-5)
    assert np.max(np.abs(g - gfd)) < 1e-6 * np.max(np.abs(g))


# ------------------------------------------------------------ a(x)

def test_spatial_coefficients_linearity():
    rng = np.random.default_rng(9)
    shape = (5, 6, 7)
    u = I.noise(shape, 0.3, 0.15, 6)
    af = rng.uniform(-1, 1, (6,) + shape)
    h = 0.9
    E = oracle.energy(u, prob((0,) * 6, h=h, a_field=af))
    want = 0.0
    for k in range(6):
        ek = np.zeros(6)
        ek[k] = 1.0
        want += np.sum(af[k] * oracle.density(u, prob(ek, h=h)))
    assert E == pytest.approx(h ** 3 * want, rel=1e-12)
    # a constant field is the constant a
    a = rng.uniform(-1, 1, 6)
    afc = np.broadcast_to(a[:, None, None, None], (6,) + shape).copy()
    Ec, gc = oracle.energy_and_grad(u, prob((0,) * 6, h=h, a_field=afc))
    Ea, ga = oracle.energy_and_grad(u, prob(a, h=h))
    assert Ec == Ea
    np.testing.assert_array_equal(gc, ga)


def test_spatial_coefficients_gradient_central_differences():
    rng = np.random.default_rng(10)
    shape = (6, 7, 8)
    u = I.noise(shape, 0.3, 0.1, 22)
    af = rng.uniform(-1, 1, (6,) + shape)
    p = prob((0,) * 6, eps=1.5, h=1.1, xi=1e-2, a_field=af)
    _, g = oracle.energy_and_grad(u, p)
    gfd = _fd_grad(u.copy(), p, 1e-5)
    assert np.max(np.abs(g - gfd)) < 1e-6 * np.max(np.abs(g))


# ------------------------------------------------------------ m(x)

def test_spatial_mass_field():
    rng = np.random.default_rng(11)
    shape = (6, 7, 8)
    m = rng.uniform(-0.7, -0.3, shape)
    p = prob((1, 0, 1, 0, 0, 0))
    A0 = np.zeros((3,) + shape)
    np.testing.assert_array_equal(oracle.hflow_field(A0, p, {"m_field": m}), m)
    A = rng.normal(size=(3,) + shape)
    ut = oracle.hflow_field(A, p, {"m_field": m, "blur_sigma": 1.0})
    assert ut.mean() == pytest.approx(m.mean(), abs=1e-13)
    np.testing.assert_allclose(oracle.hflow_field(A0, p, {"m_field": m, "blur_sigma": 1.0}),
                               oracle.blur(m, p, {"blur_sigma": 1.0}), rtol=0, atol=1e-15)


# ------------------------------------------------------------ diagnostics

@pytest.mark.parametrize("well", [0, 1])
def test_diagnostics_constant_field(well):
    c, eps, h = 0.37, 1.3, 0.8
    u = np.full((4, 5, 6), c)
    W = c * c * (1 - c) ** 2 if well == 0 else (1 - c * c) ** 2 / 4
    d = oracle.diagnostics(u, prob((0,) * 6, eps=eps, h=h, well=well))
    want = 120 * h ** 3 * W / eps
    assert d["discrepancy"] == pytest.approx(want, rel=1e-13)
    assert d["cahn_hilliard"] == pytest.approx(want, rel=1e-13)
    assert d["ratio"] == pytest.approx(1.0, rel=1e-13)
    assert d["max"] == d["min"] == c


@pytest.mark.parametrize("well", [0, 1])
def test_diagnostics_tanh_slab_equipartition(well):
    """On the tanh profile eps/2 |grad u|^2 = W(u)/eps (equipartition), so the
    normalised discrepancy vanishes like (h/eps)^2, and the Cahn-Hilliard
    energy tends to sigma x area (two interfaces of 8 x 8)."""
    sigma = math.sqrt(2) / 6 if well == 0 else 2 * math.sqrt(2) / 3
    ratios, areas = [], []
    for n, eps in ((32, 2.0), (48, 3.0), (64, 4.0)):
        u = I.tanh_slab((n, 8, 8), n / 2, eps, 1.0, well=well)
        d = oracle.diagnostics(u, prob((0,) * 6, eps=eps, well=well))
        ratios.append(d["ratio"])
        areas.append(d["cahn_hilliard"] / (sigma * 2 * 64))
        assert 0.0 <= d["ratio"] <= 1.0
    assert ratios[0] < 0.03 and ratios[0] > ratios[1] > ratios[2]
    scaled = [r * e * e for r, e in zip(ratios, (2.0, 3.0, 4.0))]
    assert max(scaled) / min(scaled) < 1.1
    assert abs(areas[0] - 1) < 0.02 and abs(areas[2] - 1) < 0.005
    assert abs(areas[0] - 1) > abs(areas[1] - 1) > abs(areas[2] - 1)


# ------------------------------------------------------------ curvature diagram

@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("well", [0, 1])
def test_surface_cells_flat_interfaces_exact(axis, well):
    """A slab normal to one axis: {u = level} is two flat planes, which the
    linear edge interpolation reproduces exactly: area 2 L1 L2 h^2, zero
    diffuse curvature (the profile varies along one axis only)."""
    L, h = 32, 0.7
    prof = I.tanh_slab((L, 1, 1), 16.0, 2.0, 1.0, well=well)[:, 0, 0]
    shape = {0: (10, 12, L), 1: (10, L, 12), 2: (L, 10, 12)}[axis]      # (nz, ny, nx)
    bshape = [1, 1, 1]
    bshape[2 - axis] = L
    u = np.broadcast_to(prof.reshape(bshape), shape).copy()
    cells = oracle.surface_cells(u, prob((0,) * 6, eps=2.0 * h, h=h, well=well), 0.5 if well == 0 else 0.0)
    other = [s for k, s in enumerate(shape) if k != 2 - axis]
    assert cells[:, 0].sum() == pytest.approx(2 * other[0] * other[1] * h * h, rel=1e-12)
    assert np.max(np.abs(cells[:, 1:])) < 1e-9


def test_surface_cells_sphere_area_and_mean_curvature():
    """tanh sphere (off-grid centre): area -> 4 pi R^2 under refinement, the
    area-weighted mean of kappa1 + kappa2 -> 2/R, kappa1 >= kappa2 per cell."""
    errs = []
    for R, n, eps in ((12, 48, 2.0), (16, 64, 2.0), (24, 96, 3.0)):
        u = I.tanh_sphere((n, n, n), R, eps, 1.0, center=(n / 2 + 0.31, n / 2 + 0.17, n / 2 + 0.23), well=1)
        c = oracle.surface_cells(u, prob((0,) * 6, eps=eps, well=1), 0.0)
        A = c[:, 0].sum()
        errs.append(abs(A / (4 * math.pi * R * R) - 1))
        H = (c[:, 0] * (c[:, 1] + c[:, 2])).sum() / A
        assert H * R == pytest.approx(2.0, rel=0.01)
        assert np.all(c[:, 1] >= c[:, 2])
    assert errs[0] < 2e-3 and errs[0] > errs[1] > errs[2]


def test_surface_cells_cylinder_curvatures():
    """z-periodic tanh cylinder: area -> 2 pi r L, kappa1 -> 1/r, kappa2 -> 0."""
    for r, n, eps in ((10, 40, 2.0), (24, 96, 3.0)):
        L = 8
        u = I.tanh_cylinder((L, n, n), r, eps, 1.0, center=(n / 2 + 0.31, n / 2 + 0.17), well=0)
        c = oracle.surface_cells(u, prob((0,) * 6, eps=eps), 0.5)
        A = c[:, 0].sum()
        assert A / (2 * math.pi * r * L) == pytest.approx(1.0, abs=5e-4)
        assert (c[:, 0] * c[:, 1]).sum() / A * r == pytest.approx(1.0, abs=0.02)
        assert abs((c[:, 0] * c[:, 2]).sum() / A * r) < 0.02


# ------------------------------------------------------------ tangent-projected M

def test_projected_planar_profile_closed_form():
    """u depends on z only: Hess u = H e_z e_z^T and G = G e_z, so
    P Hess P = (xi^2/rho)^2 H e_z e_z^T: M_P is rank one with T = -eps
    (xi^2/rho)^2 H, S = D = T^2 (M_P vanishes where G != 0 and is -eps Hess u
    where G = 0, the slab's mid-planes), and
    e = (c1 + c2) T^2 + c3 T r + c4 q T + c5 q r + c6 G^2, r = sqrt(softplus(T^2))."""
    rng = np.random.default_rng(12)
    h, eps, xi = 0.8, 1.6, 1e-6
    u = I.tanh_slab((32, 5, 6), 16.0, eps / h, 1.0, well=0)
    a = rng.uniform(-1, 1, 6)
    E = oracle.energy(u, prob(a, eps=eps, h=h, xi=xi, proj=1))
    G = (np.roll(u, -1, axis=0) - np.roll(u, 1, axis=0)) / (2 * h)
    H = (np.roll(u, -1, axis=0) - 2 * u + np.roll(u, 1, axis=0)) / (h * h)
    rho = G * G + xi * xi
    q = np.sqrt(rho)
    T = -eps * (xi * xi / rho) ** 2 * H
    D = T * T
    r = np.sqrt(D + xi * np.log1p(np.exp(-D / xi)))
    c1, c2, c3 = (a[0] + a[2] - a[1]) / (2 * eps), a[1] / (2 * eps), (a[0] - a[2]) / (2 * eps)
    c4, c5, c6 = (a[3] + a[4]) / 2, (a[3] - a[4]) / 2, a[5] * eps
    e = (c1 + c2) * T * T + c3 * T * r + c4 * q * T + c5 * q * r + c6 * G * G
    assert np.any(G == 0) and np.any(np.abs(T) > 1e-3)      # both regimes occur
    assert E == pytest.approx(h ** 3 * e.sum(), rel=1e-12)


def test_projected_sphere_and_permutations():
    """tanh sphere R = 32, eps = 2h, p = k1^2 + k2^2: F/(sigma 8 pi) close to 1
    (the W' term of eq. Meps is replaced by the projection, which removes the
    normal direction exactly); axis permutations leave E unchanged."""
    n = 128
    u = I.tanh_sphere((n, n, n), 32.0, 2.0, 1.0, center=(64.3, 64.1, 64.2))
    ratio = oracle.energy(u, prob((1, 0, 1, 0, 0, 0), eps=2.0, proj=1)) / (math.sqrt(2) / 6 * 8 * math.pi)
    assert abs(ratio - 1) < 0.01
    rng = np.random.default_rng(13)
    v = I.noise((5, 6, 7), 0.3, 0.2, 14)
    p = prob(rng.uniform(-1, 1, 6), h=0.9, proj=1)
    E = oracle.energy(v, p)
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert oracle.energy(np.ascontiguousarray(np.transpose(v, perm)), p) == pytest.approx(E, rel=1e-12)


@pytest.mark.parametrize("well", [0, 1])
def test_projected_gradient_central_differences(well):
    rng = np.random.default_rng(15 + well)
    u = I.noise((6, 7, 8), 0.3 if well == 0 else -0.1, 0.1 if well == 0 else 0.3, 23)
    th = rng.normal(size=3)
    p = prob(rng.uniform(-1, 1, 6), eps=1.5, h=0.9, xi=1e-2, well=well, proj=1, mu=0.7,
             theta=tuple(th / np.linalg.norm(th)))
    _, g = oracle.energy_and_grad(u, p)
    gfd = _fd_grad(u.copy(), p, 1e-5)
    assert np.max(np.abs(g - gfd)) < 1e-6 * np.max(np.abs(g))
