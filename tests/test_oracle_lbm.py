"""Pins of the oracle's LBM core (no GPU).

Each test checks the oracle against a fact fixed by the mathematics, not by
re-typing its formula: exact moment identities of the equilibrium (Eq. 4) and
of the Guo term (Eq. 8), exact conservation of collision (Eq. 7) and
streaming, the Zou-He faces reproducing their prescribed velocity / density,
the Chapman-Enskog viscosity nu = (tau - 1/2)/3 (Eq. 3) from Taylor-Green /
shear-wave decay, and the body-force Poiseuille profile between halfway
bounce-back walls.
"""
import math

import numpy as np
import pytest

from oracle import lbm
from oracle.lattice import D2Q9, D3Q19
import workloads as W

LATS = [D2Q9, D3Q19]


def _rand_state(lat, shape=(3, 4, 5), seed=1, umax=0.08):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * rng.standard_normal(shape)
    u = umax * rng.uniform(-1, 1, size=(lat.d,) + shape)
    F = 1e-3 * rng.standard_normal((lat.d,) + shape)
    return rho, u, F


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_lattice_isotropy(lat):
    # sum w = 1, sum w c = 0, sum w c_a c_b = cs^2 delta_ab, 4th order isotropy
    c = lat.c[:, :lat.d].astype(float)
    assert abs(lat.w.sum() - 1.0) < 1e-15
    assert np.allclose(lat.w @ c, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", lat.w, c, c), np.eye(lat.d) / 3.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", lat.w, c, c, c, c)
    I = np.eye(lat.d)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(M4, iso, atol=1e-16)
    for i in range(lat.Q):
        assert (lat.c[lat.opp[i]] == -lat.c[i]).all()


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_equilibrium_moments(lat):
    rho, u, _ = _rand_state(lat)
    feq = lbm.equilibrium(lat, rho, u)
    c = lat.c[:, :lat.d].astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    mom = np.einsum("ia,i...->a...", c, feq)
    assert np.allclose(mom, rho * u, rtol=0, atol=1e-14)
    Pi = np.einsum("ia,ib,i...->ab...", c, c, feq)
    expect = rho * np.eye(lat.d)[:, :, None, None, None] / 3.0 + rho * np.einsum("a...,b...->ab...", u, u)
    assert np.allclose(Pi, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_guo_source_moments(lat):
    rho, u, F = _rand_state(lat)
    tau = 0.73
    S = lbm.guo_source(lat, u, F, tau)
    c = lat.c[:, :lat.d].astype(float)
    pref = 1.0 - 0.5 / tau
    assert np.allclose(S.sum(0), 0.0, atol=1e-17)
    assert np.allclose(np.einsum("ia,i...->a...", c, S), pref * F, rtol=0, atol=1e-17)
    second = np.einsum("ia,ib,i...->ab...", c, c, S)
    expect = pref * (np.einsum("a...,b...->ab...", u, F) + np.einsum("a...,b...->ab...", F, u))
    assert np.allclose(second, expect, rtol=0, atol=1e-17)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_collision_conserves_mass_and_adds_force(lat):
    rho, u, F = _rand_state(lat)
    f = lbm.equilibrium(lat, rho, u)
    rng = np.random.default_rng(7)
    f = f + 1e-3 * rng.standard_normal(f.shape)      # non-equilibrium part
    fs = lbm.collide(lat, f, F, 0.61)
    c = lat.c[:, :lat.d].astype(float)
    assert np.allclose(fs.sum(0), f.sum(0), rtol=0, atol=1e-14)
    dm = np.einsum("ia,i...->a...", c, fs - f)
    assert np.allclose(dm, F, rtol=0, atol=1e-14)


def test_equilibrium_is_fixed_point_without_force():
    lat = D3Q19
    rho, u, _ = _rand_state(lat)
    feq = lbm.equilibrium(lat, rho, u)
    out = lbm.collide(lat, feq, np.zeros_like(u), 0.8)
    assert np.allclose(out, feq, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_periodic_streaming_is_a_permutation(lat):
    shape = (4, 5, 6) if lat.d == 3 else (1, 5, 6)
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(lat.Q,) + shape)
    out = lbm.stream(lat, f, [W.PERIODIC] * 6)
    for i in range(lat.Q):
        assert np.array_equal(np.sort(out[i].ravel()), np.sort(f[i].ravel()))
        cx, cy, cz = lat.c[i]
        # spot check: value at x comes from x - c_i
        z, y, x = (1 if lat.d == 3 else 0), 2, 3
        assert out[i, z, y, x] == f[i, (z - cz) % shape[0], (y - cy) % shape[1], (x - cx) % shape[2]]


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_bounce_back_conserves_mass(lat):
    shape = (3, 6, 5) if lat.d == 3 else (1, 6, 5)
    rng = np.random.default_rng(4)
    f = rng.uniform(size=(lat.Q,) + shape)
    bc = [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC]
    if lat.d == 3:
        bc[4] = bc[5] = W.BOUNCEBACK
    out = lbm.stream(lat, f, bc)
    assert abs(out.sum() - f.sum()) < 1e-12
    # a population leaving through the bottom wall comes back reversed at the same node
    i_up = int(np.where((lat.c == [0, 1, 0]).all(1))[0][0])
    assert np.array_equal(out[i_up][:, 0, :], f[lat.opp[i_up]][:, 0, :])


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
@pytest.mark.parametrize("face", [0, 1])
def test_zou_he_reproduces_prescribed_moments(lat, face):
    shape = (3, 4, 5) if lat.d == 3 else (1, 4, 5)
    rho, u, _ = _rand_state(lat, shape, seed=11, umax=0.03)
    rng = np.random.default_rng(5)
    f = lbm.equilibrium(lat, rho, u) + 1e-3 * rng.standard_normal((lat.Q,) + shape)
    u_in = (0.031, -0.012, 0.007)
    bc = [W.PERIODIC] * 6
    bc[0], bc[1] = W.VEL_INLET, W.PRESS_OUTLET
    out = lbm.stream(lat, f, bc, u_in=u_in, rho_out=1.02)
    c = lat.c[:, :lat.d].astype(float)
    x = 0 if face == 0 else shape[2] - 1
    fn = out[:, :, :, x]
    rho_n = fn.sum(0)
    mom = np.einsum("ia,i...->a...", c, fn)
    if face == 0:
        for a in range(lat.d):
            assert np.allclose(mom[a] / rho_n, u_in[a], rtol=0, atol=1e-15)
    else:
        assert np.allclose(rho_n, 1.02, rtol=0, atol=1e-14)
        for a in range(1, lat.d):
            assert np.allclose(mom[a], 0.0, atol=1e-15)


def test_zou_he_rejects_wall_corners():
    bc = [W.VEL_INLET, W.PRESS_OUTLET, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC]
    with pytest.raises(ValueError):
        lbm.check_bc(D2Q9, bc)
    with pytest.raises(ValueError):
        lbm.check_bc(D2Q9, [W.PERIODIC, W.BOUNCEBACK] + [W.PERIODIC] * 4)


def _run(lat, f, steps, tau, bc, F=None):
    for _ in range(steps):
        Fz = np.zeros((lat.d,) + f.shape[1:]) if F is None else F
        f = lbm.stream(lat, lbm.collide(lat, f, Fz, tau), bc)
    return f


def test_tgv2d_decay_gives_chapman_enskog_viscosity():
    # u(t) = u0 exp(-2 nu k^2 t) for the 2D Taylor-Green vortex
    lat, n, u0, tau, steps = D2Q9, 32, 1e-3, 0.8, 200
    u = W.tgv2d_velocity(n, n, u0)
    k = 2 * math.pi / n
    X = 2 * math.pi * np.arange(n) / n
    Y, Xg = np.meshgrid(X, X, indexing="ij")
    p = -0.25 * u0 ** 2 * (np.cos(2 * Xg) + np.cos(2 * Y))      # exact pressure
    rho = 1.0 + 3.0 * p[None]
    f = lbm.equilibrium(lat, rho, u)
    f = _run(lat, f, steps, tau, [W.PERIODIC] * 6)
    _, uu = lbm.velocity(lat, f)
    amp = np.sum(uu[0] * u[0]) / np.sum(u[0] * u[0])
    nu_fit = -math.log(amp) / (2 * k * k * steps)
    nu = (tau - 0.5) / 3.0
    assert abs(nu_fit - nu) / nu < 5e-3


def _shear_wave_nu(n, tau, u0=1e-3):
    # u_x = u0 sin(kz) exp(-nu k^2 t); the rate is fitted between two times so
    # that the start-up transient of an equilibrium initial state drops out
    lat = D3Q19
    k = 2 * math.pi / n
    z = np.arange(n)
    u = np.zeros((3, n, 1, 1))
    u[0, :, 0, 0] = u0 * np.sin(k * z)
    f = lbm.equilibrium(lat, np.ones((n, 1, 1)), u)
    f = _run(lat, f, 50, tau, [W.PERIODIC] * 6)
    a1 = np.sum(lbm.velocity(lat, f)[1][0] * u[0])
    T = int(0.3 / ((tau - 0.5) / 3.0 * k * k))
    f = _run(lat, f, T, tau, [W.PERIODIC] * 6)
    a2 = np.sum(lbm.velocity(lat, f)[1][0] * u[0])
    return -math.log(a2 / a1) / (k * k * T)


def test_d3q19_shear_wave_decay():
    """The fitted viscosity converges to (tau - 1/2)/3 at second order in k."""
    tau = 0.7
    nu = (tau - 0.5) / 3.0
    e32 = abs(_shear_wave_nu(32, tau) - nu) / nu
    e64 = abs(_shear_wave_nu(64, tau) - nu) / nu
    assert e64 < 1e-3
    assert 3.0 < e32 / e64 < 5.0


@pytest.mark.parametrize("lat", LATS, ids=lambda l: l.name)
def test_body_force_poiseuille(lat):
    """Steady channel flow between halfway bounce-back walls at y=-1/2 and H-1/2.

    Navier-Stokes gives u(y) = G/(2 nu) (y + 1/2)(H - 1/2 - y).  For BGK with
    halfway bounce-back the discrete profile has exactly this curvature at
    any tau; it is exact, walls included, when (tau - 1/2)^2 = 3/16 (the
    "magic" value of the TRT literature, which for BGK is Lambda =
    (tau - 1/2)^2; Ginzburg and d'Humieres 2003).
    """
    H, G = 8, 1e-6
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    shape = (1, H, 1) if lat.d == 2 else (1, H, 1)
    u = np.zeros((lat.d,) + shape)
    u[0, 0, :, 0] = exact
    f = lbm.equilibrium(lat, np.ones(shape), u)
    F = np.zeros((lat.d,) + shape)
    F[0] = G
    bc = [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC]
    f = _run(lat, f, 3000, tau, bc, F)
    rho, uu = lbm.velocity(lat, f, F)
    prof = uu[0, 0, :, 0]
    curv = prof[2:] - 2 * prof[1:-1] + prof[:-2]
    assert np.allclose(curv, -G / nu, rtol=1e-9, atol=0)
    assert np.allclose(prof, exact, rtol=1e-9, atol=0)


def test_poiseuille_curvature_any_tau():
    lat, H, G, tau = D2Q9, 10, 1e-6, 0.65
    nu = (tau - 0.5) / 3.0
    shape = (1, H, 1)
    y = np.arange(H)
    u = np.zeros((2,) + shape)
    u[0, 0, :, 0] = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    f = lbm.equilibrium(lat, np.ones(shape), u)
    F = np.zeros((2,) + shape)
    F[0] = G
    bc = [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC]
    f = _run(lat, f, 4000, tau, bc, F)
    _, uu = lbm.velocity(lat, f, F)
    prof = uu[0, 0, :, 0]
    curv = prof[2:] - 2 * prof[1:-1] + prof[:-2]
    assert np.allclose(curv, -G / nu, rtol=1e-7, atol=0)


def test_d3q19_reduces_to_d2q9_on_z_invariant_flow():
    """A z-invariant D3Q19 run projects exactly onto D2Q9 (weights sum per (cx,cy))."""
    nx, ny, nz, tau = 10, 8, 3, 0.7
    rng = np.random.default_rng(9)
    u2 = 0.03 * rng.uniform(-1, 1, size=(2, 1, ny, nx))
    rho2 = 1.0 + 0.01 * rng.standard_normal((1, ny, nx))
    G = np.array([2e-5, -1e-5])
    bc = [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC]
    f2 = lbm.equilibrium(D2Q9, rho2, u2)
    u3 = np.zeros((3, nz, ny, nx))
    u3[:2] = u2
    f3 = lbm.equilibrium(D3Q19, np.broadcast_to(rho2, (nz, ny, nx)), u3)
    F2 = np.broadcast_to(G[:, None, None, None], (2, 1, ny, nx))
    F3 = np.zeros((3, nz, ny, nx))
    F3[:2] = G[:, None, None, None]
    for _ in range(40):
        f2 = lbm.stream(D2Q9, lbm.collide(D2Q9, f2, F2, tau), bc)
        f3 = lbm.stream(D3Q19, lbm.collide(D3Q19, f3, F3, tau), bc)
    r2, v2 = lbm.velocity(D2Q9, f2, F2)
    r3, v3 = lbm.velocity(D3Q19, f3, F3)
    for z in range(nz):
        assert np.allclose(r3[z], r2[0], rtol=0, atol=1e-13)
        assert np.allclose(v3[:2, z], v2[:, 0], rtol=0, atol=1e-13)
    assert np.abs(v3[2]).max() < 1e-15


def test_d2q9_weights_match_paper_eq5():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "d2q9_weights.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for idx, num, den in rows:
        i = int(idx)
        assert D2Q9.w[i] == int(num) / int(den)
    # index classes of Eq. 5: rest, axis (|c|=1), diagonal (|c|^2=2)
    norms = (D2Q9.c ** 2).sum(1)
    assert list(norms) == [0, 1, 1, 1, 1, 2, 2, 2, 2]
