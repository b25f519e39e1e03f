"""Pins of the oracle's immersed boundary and kinematics (no GPU).

* cosine delta (Eq. 14): partition of unity, the even/odd half sums, the
  sum of squares 3/8, and the first moment's closed form
  sum_j (x-j) phi(x-j) = x - 1/2 - sin(pi x/2)/2 + cos(pi x/2)/2 on [0,1)
  (the kernel does NOT have a vanishing first moment);
* interpolation (Eq. 17), spreading (Eq. 15) and the system matrix
  (Eq. 18) against a brute-force double loop over every grid node with the
  minimum-image distance on periodic axes;
* the solve: no-slip E(u* + du) = U_B (Eq. 17) after a step;
* the Lagrangian force sum equals minus the Eulerian force-density sum
  (Eq. 26 with the interpolated density);
* kinematics: wall velocity = time derivative of the marker positions.
"""
import math

import numpy as np
import pytest

from oracle import ib, kinematics
from oracle.sim import Simulation
import workloads as W


def test_phi_values():
    assert ib.phi(0.0) == 0.5
    assert ib.phi(2.0) == 0.0 and ib.phi(-2.0) == 0.0 and ib.phi(2.5) == 0.0
    assert abs(ib.phi(1.0) - 0.25) < 1e-16


@pytest.mark.parametrize("x", np.linspace(0.0, 0.999, 37))
def test_delta_discrete_moments(x):
    j = np.arange(-3, 5)
    w = ib.phi(x - j)
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs(w[j % 2 == 0].sum() - 0.5) < 1e-15
    assert abs(w[j % 2 == 1].sum() - 0.5) < 1e-15
    assert abs((w * w).sum() - 0.375) < 1e-15
    m1 = ((x - j) * w).sum()
    closed = x - 0.5 - 0.5 * math.sin(0.5 * math.pi * x) + 0.5 * math.cos(0.5 * math.pi * x)
    assert abs(m1 - closed) < 1e-15


def test_first_moment_is_not_zero():
    xs = np.linspace(0, 1, 1001)[:-1]
    m1 = [((x - np.arange(-3, 5)) * ib.phi(x - np.arange(-3, 5))).sum() for x in xs]
    assert 0.02 < max(np.abs(m1)) < 0.0215


def _brute_delta(shape_zyx, X, periodic):
    """Literal D(x - X_l) on every node, distances taken as the minimum image on periodic axes."""
    nz, ny, nx = shape_zyx
    m, d = X.shape
    n_ax = [nx, ny, nz]
    D = np.zeros((nz * ny * nx, m))
    for l in range(m):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    node = [x, y, z]
                    val = 1.0
                    for a in range(d):
                        r = node[a] - X[l, a]
                        if periodic[a]:
                            r = (r + n_ax[a] / 2) % n_ax[a] - n_ax[a] / 2
                        val *= ib.phi(r)
                    D[(z * ny + y) * nx + x, l] = val
    return D


@pytest.mark.parametrize("d", [2, 3])
def test_spread_interp_system_against_brute_force(d):
    rng = np.random.default_rng(21)
    if d == 2:
        shape = (1, 9, 12)
        X = np.column_stack([rng.uniform(0, 12, 5), rng.uniform(2.2, 5.8, 5)])
        periodic = [True, False]
    else:
        shape = (7, 8, 9)
        X = np.column_stack([rng.uniform(0, 9, 4), rng.uniform(2.1, 4.9, 4), rng.uniform(0, 7, 4)])
        periodic = [True, False, True]
    ds = rng.uniform(0.5, 1.5, X.shape[0])
    Dm = ib.spread_matrix(X, shape, periodic)
    Db = _brute_delta(shape, X, periodic)
    assert np.allclose(Dm.toarray(), Db, rtol=0, atol=1e-15)
    u = rng.standard_normal((d,) + shape)
    ul = ib.interpolate(Dm, u)
    for l in range(X.shape[0]):
        for a in range(d):
            assert abs(ul[l, a] - (u[a].ravel() * Db[:, l]).sum()) < 1e-13
    v = rng.standard_normal((X.shape[0], d))
    du = ib.spread(Dm, v, ds, shape)
    brute = np.einsum("xl,la->ax", Db, v * ds[:, None]).reshape((d,) + shape)
    assert np.allclose(du, brute, rtol=0, atol=1e-14)
    A = ib.system_matrix(Dm, ds)
    m = X.shape[0]
    for l in range(m):
        for k in range(m):
            lit = sum(Db[x, l] * Db[x, k] for x in range(Db.shape[0])) * ds[k]
            assert abs(A[l, k] - lit) < 1e-14
    # adjointness <E u, v> = <u, D v> with ds = 1
    du1 = ib.spread(Dm, v, np.ones(m), shape)
    assert abs(np.sum(ul * v) - np.sum(u * du1)) < 1e-12


def test_stencil_outside_nonperiodic_axis_is_rejected():
    with pytest.raises(ValueError):
        ib.spread_matrix(np.array([[5.0, 0.7]]), (1, 10, 10), [True, False])


def test_partition_of_unity_of_spreading():
    rng = np.random.default_rng(2)
    shape = (6, 7, 8)
    X = rng.uniform(0, 6, size=(6, 3))
    Dm = ib.spread_matrix(X, shape, [True, True, True])
    v = rng.standard_normal((6, 3))
    ds = rng.uniform(0.5, 2.0, 6)
    du = ib.spread(Dm, v, ds, shape)
    assert np.allclose(du.reshape(3, -1).sum(1), (v * ds[:, None]).sum(0), rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", [W.WAVE_COS, W.WAVE_SIN, W.WAVE_ABS_SIN])
def test_wall_velocity_is_time_derivative(kind):
    X0, ds = W.elliptic_planform_markers(8.0, 16.0)
    body = {"X0": X0, "hinge": (4.0, 0.0, 0.0), "axis": (0.2, 0.1, 1.0), "origin": (20.0, 10.0, 11.0),
            "A": {"kind": W.WAVE_COS, "amp": 3.0, "offset": 0.5},
            "alpha": {"kind": kind, "amp": 1.0, "offset": 0.1},
            "beta": 0.4, "phi": 0.3, "f": 1.0 / 500.0}
    h = 1e-4
    for t in (17.0, 130.0, 333.3):
        X, U = kinematics.marker_state(body, t, 3)
        Xp, _ = kinematics.marker_state(body, t + h, 3)
        Xm, _ = kinematics.marker_state(body, t - h, 3)
        assert np.allclose((Xp - Xm) / (2 * h), U, rtol=0, atol=1e-9)


def test_rigid_motion_preserves_distances_and_hinge():
    X0, _ = W.elliptic_planform_markers(10.0, 20.0)
    body = {"X0": X0, "hinge": (5.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0), "origin": (30.0, 20.0, 15.0),
            "A": {"kind": W.WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "alpha": {"kind": W.WAVE_ABS_SIN, "amp": math.pi / 3, "offset": 0.0},
            "beta": 0.0, "phi": 0.0, "f": 1.0 / 400.0}
    X, _ = kinematics.marker_state(body, 100.0, 3)     # quarter period: alpha = 60 degrees
    d0 = np.linalg.norm(X0[:, None] - X0[None], axis=-1)
    d1 = np.linalg.norm(X[:, None] - X[None], axis=-1)
    assert np.allclose(d0, d1, atol=1e-12)
    # the trailing-edge hinge line stays at x = origin_x + 5, the leading edge swings by 60 deg
    le = X0[:, 0].argmin()
    v = X[le] - np.array([35.0, 20.0, X[le, 2]])
    assert abs(math.degrees(math.atan2(-v[1], -v[0])) - 60.0) < 1e-9


def _cylinder_sim(steps=0):
    cfg = W.cylinder_channel(nx=60, ny=40, diameter=10.0, center=(20.0, 20.0), m=31)
    sim = Simulation(9, cfg["grid"], cfg["tau"])
    sim.init_fluid()
    sim.add_body(cfg["bodies"][0])
    sim.set_reference(**cfg["reference"])
    sim.step(steps)
    return sim


def test_step_enforces_no_slip_and_force_balance():
    sim = _cylinder_sim(steps=30)
    sim.step(1)
    L = sim.last
    # no-slip (Eq. 17): the corrected field u* + du, interpolated afresh, equals U_B
    Dm = ib.spread_matrix(L["X"], sim.shape, sim.periodic)
    u_corr = ib.interpolate(Dm, L["ustar"] + L["du"])
    assert np.abs(u_corr - L["U"]).max() < 1e-12
    # Lagrangian sum of 2 rho_l y_l ds_l equals the Eulerian sum of 2 rho du
    ds = np.asarray(sim.bodies[0]["ds"])
    lag = (2.0 * L["rho_l"][:, None] * L["y"] * ds[:, None]).sum(0)
    eul = (2.0 * L["rho"][None] * L["du"]).reshape(2, -1).sum(1)
    assert np.allclose(lag, eul, rtol=1e-12, atol=1e-18)
    G = np.asarray(sim.grid["body_force"])[:2]
    assert np.allclose((sim.last_F - G[:, None, None, None]), 2.0 * L["rho"][None] * L["du"],
                       rtol=0, atol=1e-18)


def test_step_conserves_mass_with_walls_and_markers():
    sim = _cylinder_sim()
    m0 = sim.f.sum()
    sim.step(40)
    assert abs(sim.f.sum() - m0) < 1e-10


def test_cylinder_drag_is_positive_and_lift_small():
    """Sanity of the sign convention: flow along +x drags the cylinder along +x."""
    sim = _cylinder_sim(steps=300)
    CL, CT, CD = sim.history[0][-1]
    assert CD > 0 and abs(CT + CD) < 1e-15
    assert abs(CL) < 0.05 * CD


def test_figure_eight_kinematics():
    """Sec. 3.2 hovering wing (Eqs. 20-22): the centre sweeps +-A0/2 along the
    stroke plane at beta = 60 deg, the pitch is 45 deg at t = 0 and 0 at
    t = T/4, and the largest centre speed is Eq. 22's U_tip = pi f A0."""
    from oracle.kinematics import marker_state
    cfg = W.figure_eight_2d(chord=16.0, Re=75.0, period=2000.0)
    b = cfg["bodies"][0]
    p = cfg["params"]
    org = np.array(b["origin"][:2])
    es = np.array([0.5, math.sqrt(3.0) / 2.0])
    T = 2000.0
    probe = dict(b, X0=np.array([[0.0, 0.0], [-1.0, 0.0]]))   # centre, a point towards the leading edge
    for t, A, alpha in ((0.0, p["A0"] / 2, math.pi / 4), (T / 4, 0.0, 0.0), (T / 2, -p["A0"] / 2, math.pi / 4)):
        X, _ = marker_state(probe, t, 2)
        assert np.abs(X[0] - (org + A * es)).max() < 1e-9
        v = X[1] - X[0]
        ang = math.atan2(v[1], v[0])
        assert abs(((ang - (math.pi + alpha)) + math.pi) % (2 * math.pi) - math.pi) < 1e-9
    speeds = []
    for t in np.linspace(0.0, T, 401):
        _, U = marker_state(probe, t, 2)
        speeds.append(np.linalg.norm(U[0]))
    assert abs(max(speeds) - p["u_tip"]) < 1e-12
    assert abs(p["u_tip"] - math.pi * p["f"] * p["A0"]) < 1e-15


def test_table_wave_values_and_rates():
    """TABLE wave: value table[n mod len] at step n, rate by the central
    difference of the neighbouring samples, wrapping at both ends.  Expected
    values worked by hand for the table 0, 1, 4, 9, 16."""
    w = {"kind": W.WAVE_TABLE, "table": [0.0, 1.0, 4.0, 9.0, 16.0]}
    cases = {0: (0.0, -7.5), 1: (1.0, 2.0), 2: (4.0, 4.0), 4: (16.0, -4.5), 7: (4.0, 4.0), -1: (16.0, -4.5)}
    for t, (v, vd) in cases.items():
        assert kinematics.wave(w, float(t), 0.0, 0.0) == (v, vd)


def test_table_wave_drives_the_rotation():
    """A rotation angle given as a table turns the body by table[n mod len]
    at step n (a marker one unit behind the hinge lands at angle pi + alpha)
    and its wall velocity is the table's central difference times e x r."""
    angles = [0.0, 0.1, 0.3, 0.6]
    body = {"X0": np.array([[-1.0, 0.0, 0.0]]), "hinge": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0),
            "origin": (5.0, 6.0, 7.0), "A": {"kind": W.WAVE_CONST},
            "alpha": {"kind": W.WAVE_TABLE, "table": angles}, "beta": 0.0, "phi": 0.0, "f": 0.0}
    for n, (al, rate) in {1: (0.1, 0.15), 2: (0.3, 0.25), 5: (0.1, 0.15)}.items():
        X, U = kinematics.marker_state(body, float(n), 3)
        r = np.array([-math.cos(al), -math.sin(al), 0.0])
        assert np.abs(X[0] - (np.array([5.0, 6.0, 7.0]) + r)).max() < 1e-15
        assert np.abs(U[0] - rate * np.array([-r[1], r[0], 0.0])).max() < 1e-15


def test_coefficient_normalisation_by_hand():
    """C = F / (rho_ref U_ref^2 L / 2): with rho_ref = 0.5, U_ref = 2, L = 3
    the dynamic-pressure scale is 3, so a body force (6, -1.5) gives
    C_D = 2 (along +x), C_T = -2 and C_L = -0.5 along +y, +0.5 along -y."""
    grid = W.grid(16, 16, 1, [W.PERIODIC] * 6, precision="fp64")
    sim = Simulation(9, grid, 0.8)
    for axis in ((0.0, 1.0, 0.0), (0.0, -1.0, 0.0)):
        sim.add_body({"X0": np.zeros((1, 2)), "ds": np.ones(1), "hinge": (0, 0, 0), "axis": (0, 0, 1),
                      "origin": (8.0, 8.0, 0.0), "A": {"kind": W.WAVE_CONST},
                      "alpha": {"kind": W.WAVE_CONST}, "beta": 0.0, "phi": 0.0, "f": 0.0,
                      "lift_axis": axis})
    sim.set_reference(2.0, 3.0, 0.5)
    F = np.array([6.0, -1.5])
    assert sim.coefficients(0, F) == (-0.5, -2.0, 2.0)
    assert sim.coefficients(1, F) == (0.5, -2.0, 2.0)
