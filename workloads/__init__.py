"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and bench.py.

This module only produces *inputs*: marker geometry (body-frame coordinates and
element sizes), initial velocity fields, random marker clouds and the run
parameters of each workload.  It contains none of the IB-LBM step arithmetic
(equilibrium, forcing, streaming, delta kernel, solve, forces); those live,
written independently, in ``oracle/`` and in the CUDA sources.

The paper (arXiv 2102.01305) measures on no public dataset, so every workload
here is synthetic, with the shapes of the paper's cases:

* cylinder in a body-force-driven channel (Sec. 3.1 benchmark, 2D, D2Q9);
* two rigid elliptic wings hinged at the trailing edge performing clap and
  fling (Sec. 3.3, Eq. 23, Eq. 24), extended to a 3D planform on D3Q19;
* a periodic Taylor-Green vortex (pure LBM roofline sweep);
* a cloud of random markers (interpolate/spread throughput sweep).

All random draws use numpy's PCG64 seeded with ``SEED``.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20210203

# Boundary-condition codes, identical to the C ABI's ``ibl_bc`` enum.
PERIODIC, BOUNCEBACK, VEL_INLET, PRESS_OUTLET = 0, 1, 2, 3

# Wave kinds, identical to the C ABI's ``ibl_wave_kind`` enum.
WAVE_CONST, WAVE_COS, WAVE_SIN, WAVE_ABS_SIN, WAVE_TABLE = 0, 1, 2, 3, 4


# --------------------------------------------------------------------------- geometry
def cylinder_markers(diameter: float, m: int):
    """Circle of ``m`` equally spaced markers (Sec. 3.1), body frame centred at 0.

    Returns (X0 [m,2], ds [m]); ds is the arc length per marker, pi*D/m.
    """
    theta = 2.0 * math.pi * np.arange(m) / m
    r = 0.5 * diameter
    X0 = np.stack([r * np.cos(theta), r * np.sin(theta)], axis=1)
    ds = np.full(m, math.pi * diameter / m)
    return X0, ds


def elliptic_planform_markers(chord: float, span: float, spacing: float = 1.0):
    """Flat elliptic planform: a unit-spaced marker mesh clipped to the ellipse.

    Body frame: x chordwise (leading edge at -chord/2, trailing edge at
    +chord/2), y normal to the wing, z spanwise.  Mesh points sit at cell
    centres (i+1/2, k+1/2)*spacing; each marker carries the area of its mesh
    cell, ds = spacing**2.
    """
    a, b = 0.5 * chord, 0.5 * span
    ni = int(math.ceil(a / spacing)) + 1
    nk = int(math.ceil(b / spacing)) + 1
    xs = (np.arange(-ni, ni) + 0.5) * spacing
    zs = (np.arange(-nk, nk) + 0.5) * spacing
    xx, zz = np.meshgrid(xs, zs, indexing="ij")
    keep = (xx / a) ** 2 + (zz / b) ** 2 <= 1.0
    X0 = np.stack([xx[keep], np.zeros(keep.sum()), zz[keep]], axis=1)
    ds = np.full(X0.shape[0], spacing * spacing)
    return X0, ds


def ellipse_foil_markers(chord: float, thickness: float, spacing: float = 1.0):
    """2D elliptic foil perimeter (Sec. 3.2/3.3 foils), markers at ~equal arc length.

    Body frame: x chordwise (leading edge at -chord/2), y thickness.  ds is half
    the sum of the two adjacent chord lengths of the marker polygon.
    """
    a, b = 0.5 * chord, 0.5 * thickness
    t = np.linspace(0.0, 2.0 * math.pi, 20001)
    px, py = a * np.cos(t), b * np.sin(t)
    seg = np.hypot(np.diff(px), np.diff(py))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    m = max(8, int(round(s[-1] / spacing)))
    targets = np.arange(m) * s[-1] / m
    tt = np.interp(targets, s, t)
    X0 = np.stack([a * np.cos(tt), b * np.sin(tt)], axis=1)
    nxt = np.roll(X0, -1, axis=0)
    prv = np.roll(X0, 1, axis=0)
    ds = 0.5 * (np.hypot(*(nxt - X0).T) + np.hypot(*(X0 - prv).T))
    return X0, ds


def random_markers(m: int, n: int, lo: float = 2.0, hi: float | None = None,
                   umax: float = 0.05, seed: int = SEED):
    """Uniform random marker cloud in [lo, hi)^3 with velocities in [-umax, umax]^3."""
    hi = (n - 2.0) if hi is None else hi
    rng = np.random.default_rng(seed)
    X = rng.uniform(lo, hi, size=(m, 3))
    U = rng.uniform(-umax, umax, size=(m, 3))
    return X, U


# --------------------------------------------------------------------------- fields
def tgv3d_velocity(nx: int, ny: int, nz: int, u0: float):
    """3D Taylor-Green initial velocity, u=(u0 s c c, -u0 c s c, 0), k=2*pi/n per axis.

    Returns u with shape [3, nz, ny, nx] (x fastest).
    """
    x = 2.0 * math.pi * np.arange(nx) / nx
    y = 2.0 * math.pi * np.arange(ny) / ny
    z = 2.0 * math.pi * np.arange(nz) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    return u


def tgv2d_velocity(nx: int, ny: int, u0: float):
    """2D Taylor-Green initial velocity u=(u0 sin x cos y, -u0 cos x sin y), shape [2,1,ny,nx]."""
    x = 2.0 * math.pi * np.arange(nx) / nx
    y = 2.0 * math.pi * np.arange(ny) / ny
    Y, X = np.meshgrid(y, x, indexing="ij")
    u = np.zeros((2, 1, ny, nx))
    u[0, 0] = u0 * np.sin(X) * np.cos(Y)
    u[1, 0] = -u0 * np.cos(X) * np.sin(Y)
    return u


def random_velocity(shape, d: int, umax: float, seed: int = SEED):
    """Smooth-free random velocity field in [-umax, umax], shape [d, *shape]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-umax, umax, size=(d,) + tuple(shape))


# --------------------------------------------------------------------------- parameters
def clap_fling_parameters(Re: float, period: float, chord: float, J: float,
                          opening_deg: float = 120.0):
    """Run parameters of a clap-and-fling case.

    Tip speed U_tip = 2*Phi*f*c with Phi the maximum opening angle (Eq. 24 and
    Sec. 3.4); Re = U_tip*c/nu (Eq. 22 with the clap-and-fling tip speed);
    tau = 3*nu + 1/2 (Eq. 3, lattice units); free stream U_inf = J*U_tip (Eq. 24).
    """
    phi_max = math.radians(opening_deg)
    f = 1.0 / period
    u_tip = 2.0 * phi_max * f * chord
    nu = u_tip * chord / Re
    tau = 3.0 * nu + 0.5
    return {"u_tip": u_tip, "nu": nu, "tau": tau, "u_inf": J * u_tip, "f": f}


def grid(nx, ny, nz, bc, u_in=(0.0, 0.0, 0.0), rho_out=1.0,
         body_force=(0.0, 0.0, 0.0), precision="fp32"):
    """Grid description shared by both sides (bc order: -x,+x,-y,+y,-z,+z)."""
    return {"nx": int(nx), "ny": int(ny), "nz": int(nz), "bc": list(bc),
            "u_in": tuple(float(v) for v in u_in), "rho_out": float(rho_out),
            "body_force": tuple(float(v) for v in body_force), "precision": precision}


def cylinder_channel(nx=200, ny=100, diameter=20.0, center=(50.0, 50.0), m=63,
                     tau=0.8, u_mean=0.05, precision="fp64"):
    """Cylinder in a channel: D2Q9, x periodic with a uniform body force, y walls.

    The body force G is the one that drives an empty channel of height H=ny
    (halfway bounce-back walls) at mean speed u_mean: G = 12*nu*u_mean/H^2
    with nu = (tau-1/2)/3.  The fluid starts at rest, rho=1.
    """
    nu = (tau - 0.5) / 3.0
    G = 12.0 * nu * u_mean / (ny * ny)
    X0, ds = cylinder_markers(diameter, m)
    body = {"X0": X0, "ds": ds, "hinge": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0),
            "origin": (center[0], center[1], 0.0),
            "A": {"kind": WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "alpha": {"kind": WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "beta": 0.0, "phi": 0.0, "f": 0.0, "J": 0.0}
    return {"lattice": 9, "tau": tau,
            "grid": grid(nx, ny, 1, [PERIODIC, PERIODIC, BOUNCEBACK, BOUNCEBACK,
                                     PERIODIC, PERIODIC], body_force=(G, 0.0, 0.0),
                         precision=precision),
            "bodies": [body], "rho0": 1.0, "u0": (0.0, 0.0, 0.0),
            "reference": {"U_ref": u_mean, "L": diameter, "rho_ref": 1.0}}


def cylinder_50d(diameter=8.0, Re=20.0, u_in=0.05, precision="fp64"):
    """Sec. 3.1 validation case: a stationary cylinder in a 50D x 50D box,
    uniform velocity inlet (Zou-He) at -x and pressure outlet at +x.  The
    lateral faces are periodic (reading: with a blockage of 1/50 the walls
    are 25 D away; Zou-He faces meeting walls are not supported).  The
    cylinder sits 12.5 D behind the inlet on the centre line; nu = U D / Re;
    the fluid starts uniform at the inflow velocity."""
    n = int(round(50 * diameter))
    nu = u_in * diameter / Re
    m = max(8, int(round(math.pi * diameter)))
    X0, ds = cylinder_markers(diameter, m)
    body = {"X0": X0, "ds": ds, "hinge": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0),
            "origin": (12.5 * diameter, 0.5 * n, 0.0),
            "A": {"kind": WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "alpha": {"kind": WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "beta": 0.0, "phi": 0.0, "f": 0.0, "J": 0.0}
    return {"lattice": 9, "tau": 3.0 * nu + 0.5,
            "grid": grid(n, n, 1, [VEL_INLET, PRESS_OUTLET, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                         u_in=(u_in, 0.0, 0.0), precision=precision),
            "bodies": [body], "rho0": 1.0, "u0": (u_in, 0.0, 0.0),
            "reference": {"U_ref": u_in, "L": diameter, "rho_ref": 1.0}}


def clap_fling_3d(nx=256, ny=192, nz=160, chord=20.0, Re=100.0, J=1e-2, period=4000.0,
                  precision="fp32", spacing=1.0, span_ratio=5.0, hinge_x=None,
                  gap_ratio=0.5, alpha_kind=WAVE_ABS_SIN, phase=0.0, faces="inlet-outlet"):
    """Two flat elliptic wings (chord c, span 5c) doing clap and fling on D3Q19.

    Wings hinge at the trailing edge (Sec. 3.3) about spanwise axes; at clap
    (alpha=0) they are parallel planes y = y_mid -/+ gap/2, gap = c/2.  The
    opening angle of each wing is alpha(t) = (pi/3)|sin(2 pi f t + phi)|, so the
    pair opens to 120 degrees and claps twice per period.  Inlet at -x with
    U_inf = J*U_tip, pressure outlet at +x, periodic in y and z.
    """
    p = clap_fling_parameters(Re, period, chord, J)
    X0, ds = elliptic_planform_markers(chord, span_ratio * chord, spacing)
    hx = float(round(nx / 3.0)) if hinge_x is None else float(hinge_x)
    ymid = 0.5 * ny
    gap = gap_ratio * chord
    zc = 0.5 * nz
    bodies = []
    for side, axis_z in ((-1.0, 1.0), (1.0, -1.0)):
        bodies.append({
            "X0": X0.copy(), "ds": ds.copy(),
            "hinge": (0.5 * chord, 0.0, 0.0), "axis": (0.0, 0.0, axis_z),
            # body-frame trailing edge lands at x = hx
            "origin": (hx - 0.5 * chord, ymid + side * 0.5 * gap, zc),
            "A": {"kind": WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "alpha": {"kind": alpha_kind, "amp": math.pi / 3.0, "offset": 0.0},
            "beta": 0.0, "phi": phase, "f": p["f"], "J": J,
            "lift_axis": (0.0, side, 0.0)})
    u_inf = p["u_inf"]
    area = float(ds.sum())
    xb = [VEL_INLET, PRESS_OUTLET] if faces == "inlet-outlet" else [PERIODIC, PERIODIC]
    return {"lattice": 19, "tau": p["tau"],
            "grid": grid(nx, ny, nz, xb + [PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                         u_in=(u_inf, 0.0, 0.0), rho_out=1.0, precision=precision),
            "bodies": bodies, "rho0": 1.0, "u0": (u_inf, 0.0, 0.0),
            "reference": {"U_ref": p["u_tip"], "L": area, "rho_ref": 1.0},
            "params": p}


def clap_fling_2d(chord=20.0, Re=100.0, J=1.67e-3, period=4000.0, thickness_ratio=5.0,
                  domain=(50, 25), precision="fp64"):
    """Paper-faithful 2D clap and fling: two elliptic foils (chord/thickness 5)."""
    p = clap_fling_parameters(Re, period, chord, J)
    nx, ny = int(domain[0] * chord), int(domain[1] * chord)
    X0, ds = ellipse_foil_markers(chord, chord / thickness_ratio)
    hx = float(round(nx / 3.0))
    ymid = 0.5 * ny
    gap = 0.5 * chord
    bodies = []
    for side, axis_z in ((-1.0, 1.0), (1.0, -1.0)):
        bodies.append({
            "X0": X0.copy(), "ds": ds.copy(),
            "hinge": (0.5 * chord, 0.0, 0.0), "axis": (0.0, 0.0, axis_z),
            "origin": (hx - 0.5 * chord, ymid + side * 0.5 * gap, 0.0),
            "A": {"kind": WAVE_CONST, "amp": 0.0, "offset": 0.0},
            "alpha": {"kind": WAVE_ABS_SIN, "amp": math.pi / 3.0, "offset": 0.0},
            "beta": 0.0, "phi": 0.0, "f": p["f"], "J": J,
            "lift_axis": (0.0, side, 0.0)})
    return {"lattice": 9, "tau": p["tau"],
            "grid": grid(nx, ny, 1, [VEL_INLET, PRESS_OUTLET, PERIODIC, PERIODIC,
                                     PERIODIC, PERIODIC], u_in=(p["u_inf"], 0.0, 0.0),
                         precision=precision),
            "bodies": bodies, "rho0": 1.0, "u0": (p["u_inf"], 0.0, 0.0),
            "reference": {"U_ref": p["u_tip"], "L": chord, "rho_ref": 1.0},
            "params": p}


def figure_eight_2d(chord=16.0, Re=75.0, period=2000.0, domain=(50, 25), precision="fp64"):
    """Sec. 3.2 hovering wing: an elliptic foil (chord/thickness 7.5) pitching
    about its centre while sweeping along a stroke plane inclined at beta:
    A(t) = (A0/2) cos(2 pi t/T + phi) (Eq. 20), alpha(t) = pi/4 - (pi/4)
    sin(2 pi t/T + phi) (Eq. 21), A0/c = 2.5, beta = pi/3, phi = 0; Re =
    pi f A0 c / nu (Eq. 22); fluid at rest in a periodic 50c x 25c box."""
    f = 1.0 / period
    A0 = 2.5 * chord
    u_tip = math.pi * f * A0
    nu = u_tip * chord / Re
    nx, ny = int(domain[0] * chord), int(domain[1] * chord)
    X0, ds = ellipse_foil_markers(chord, chord / 7.5)
    body = {"X0": X0, "ds": ds, "hinge": (0.0, 0.0, 0.0), "axis": (0.0, 0.0, 1.0),
            "origin": (0.5 * nx, 0.5 * ny, 0.0),
            "A": {"kind": WAVE_COS, "amp": 0.5 * A0, "offset": 0.0},
            "alpha": {"kind": WAVE_SIN, "amp": -0.25 * math.pi, "offset": 0.25 * math.pi},
            "beta": math.pi / 3.0, "phi": 0.0, "f": f, "J": 0.0, "lift_axis": (0.0, 1.0, 0.0)}
    return {"lattice": 9, "tau": 3.0 * nu + 0.5,
            "grid": grid(nx, ny, 1, [PERIODIC] * 6, precision=precision),
            "bodies": [body], "rho0": 1.0, "u0": (0.0, 0.0, 0.0),
            "reference": {"U_ref": u_tip, "L": chord, "rho_ref": 1.0},
            "params": {"f": f, "A0": A0, "u_tip": u_tip, "nu": nu, "Re": Re}}


def taylor_green_3d(n=64, u0=0.05, tau=0.6, precision="fp32"):
    """Periodic D3Q19 Taylor-Green vortex on an n^3 cube (pure LBM, no markers)."""
    return {"lattice": 19, "tau": tau,
            "grid": grid(n, n, n, [PERIODIC] * 6, precision=precision),
            "bodies": [], "rho0": 1.0, "u_field": tgv3d_velocity(n, n, n, u0)}
