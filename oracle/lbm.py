"""Lattice Boltzmann core of the oracle (FP64; test infrastructure only).

Arrays: populations f have shape [Q, nz, ny, nx] (x fastest, nz = 1 in 2D);
vector fields (u, F) have shape [d, nz, ny, nx].  Lattice units throughout:
dx = dt = 1, c_s^2 = 1/3.

Readings of garbled passages (the PDF extraction mangled several equations):

* Eq. 4 (equilibrium) prints "(c_i - u)^2" and "u/c_s^2"; it is read as the
  standard second-order expansion
  f_eq = w_i rho [1 + c.u/c_s^2 + (c.u)^2/(2 c_s^4) - u.u/(2 c_s^2)].
* Eq. 8 (Guo forcing) lacks the trailing c_i in the second term; it is read
  as Guo et al.'s source
  F_i = (1 - 1/(2 tau)) w_i [(c_i - u)/c_s^2 + (c_i.u) c_i/c_s^4] . F.
* Eq. 2 prints "sum c_i f"; with Eq. 9 the velocity used in both f_eq and
  F_i is rho u = sum_i c_i f_i + F/2.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice

PERIODIC, BOUNCEBACK, VEL_INLET, PRESS_OUTLET = 0, 1, 2, 3


def _cdot(lat: Lattice, i: int, v: np.ndarray) -> np.ndarray:
    """c_i . v for a vector field v of shape [d, ...]."""
    out = np.zeros(v.shape[1:])
    for a in range(lat.d):
        if lat.c[i, a] != 0:
            out = out + lat.c[i, a] * v[a]
    return out


def equilibrium(lat: Lattice, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Second-order Maxwellian f_eq (Eq. 4, reading above)."""
    cs2 = lat.cs2
    usq = np.zeros_like(rho)
    for a in range(lat.d):
        usq = usq + u[a] * u[a]
    feq = np.empty((lat.Q,) + rho.shape)
    for i in range(lat.Q):
        cu = _cdot(lat, i, u)
        feq[i] = lat.w[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2)
                                   - usq / (2.0 * cs2))
    return feq


def guo_source(lat: Lattice, u: np.ndarray, F: np.ndarray, tau: float) -> np.ndarray:
    """Guo forcing term F_i (Eq. 8, reading above)."""
    cs2 = lat.cs2
    pref = 1.0 - 1.0 / (2.0 * tau)
    S = np.empty((lat.Q,) + u.shape[1:])
    for i in range(lat.Q):
        cu = _cdot(lat, i, u)
        acc = np.zeros(u.shape[1:])
        for a in range(lat.d):
            ca = float(lat.c[i, a])
            acc = acc + ((ca - u[a]) / cs2 + cu * ca / (cs2 * cs2)) * F[a]
        S[i] = pref * lat.w[i] * acc
    return S


def density(f: np.ndarray) -> np.ndarray:
    """rho = sum_i f_i (Eq. 2 / Eq. 9)."""
    return f.sum(axis=0)


def momentum(lat: Lattice, f: np.ndarray) -> np.ndarray:
    """sum_i c_i f_i, shape [d, ...]."""
    m = np.zeros((lat.d,) + f.shape[1:])
    for i in range(lat.Q):
        for a in range(lat.d):
            if lat.c[i, a] != 0:
                m[a] += lat.c[i, a] * f[i]
    return m


def velocity(lat: Lattice, f: np.ndarray, F: np.ndarray | None = None):
    """rho and u with rho u = sum c_i f_i + F/2 (Eq. 9)."""
    rho = density(f)
    mom = momentum(lat, f)
    if F is not None:
        mom = mom + 0.5 * F
    return rho, mom / rho


def collide(lat: Lattice, f: np.ndarray, F: np.ndarray, tau: float) -> np.ndarray:
    """BGK collision with the Guo term (Eq. 7): f* = f - (f - f_eq)/tau + F_i.

    F is the total force density on the fluid at this step; u follows Eq. 9.
    """
    rho, u = velocity(lat, f, F)
    feq = equilibrium(lat, rho, u)
    return f - (f - feq) / tau + guo_source(lat, u, F, tau)


def _face_slice(face: int, shape3):
    """Index tuple of the node layer on ``face`` (0..5 = -x,+x,-y,+y,-z,+z) of a [nz,ny,nx] array."""
    a, side = divmod(face, 2)
    ax = 2 - a
    sl = [slice(None)] * 3
    sl[ax] = 0 if side == 0 else shape3[ax] - 1
    return tuple(sl)


def check_bc(lat: Lattice, bc) -> None:
    """Periodic faces come in pairs; Zou-He faces need periodic side axes."""
    zh_axes = []
    for a in range(lat.d):
        lo, hi = bc[2 * a], bc[2 * a + 1]
        if (lo == PERIODIC) != (hi == PERIODIC):
            raise ValueError(f"axis {a}: periodic must be set on both faces")
        if lo in (VEL_INLET, PRESS_OUTLET) or hi in (VEL_INLET, PRESS_OUTLET):
            zh_axes.append(a)
    for a in zh_axes:
        for b in range(lat.d):
            if b != a and bc[2 * b] != PERIODIC:
                raise ValueError("Zou-He faces need periodic lateral axes")


def stream(lat: Lattice, fpost: np.ndarray, bc, u_in=(0.0, 0.0, 0.0),
           rho_out: float = 1.0) -> np.ndarray:
    """Streaming f_i(x + c_i, t+1) = f*_i(x, t) (left side of Eq. 1) with the faces' conditions.

    Written in pull form: f_i(x) <- f*_i(x - c_i).
    * periodic faces wrap;
    * halfway bounce-back walls (Sec. 2.1 "bounce back"): a population whose
      source x - c_i lies beyond a wall face is the reflected post-collision
      population of the same node, f_i(x) = f*_{opp(i)}(x);
    * velocity inlet / pressure outlet faces (Sec. 3.1, Zou and He) rebuild
      the populations that enter from outside, see ``zou_he``.
    """
    check_bc(lat, bc)
    shape3 = fpost.shape[1:]
    fnew = np.empty_like(fpost)
    for i in range(lat.Q):
        cx, cy, cz = (int(v) for v in lat.c[i])
        fnew[i] = np.roll(fpost[i], shift=(cz, cy, cx), axis=(0, 1, 2))
    for i in range(lat.Q):
        for a in range(lat.d):
            ca = int(lat.c[i, a])
            if ca == 0:
                continue
            face = 2 * a if ca > 0 else 2 * a + 1   # face the source lies beyond
            if bc[face] == BOUNCEBACK:
                sl = _face_slice(face, shape3)
                fnew[i][sl] = fpost[lat.opp[i]][sl]
    for face in range(2 * lat.d):
        if bc[face] in (VEL_INLET, PRESS_OUTLET):
            zou_he(lat, fnew, face, bc[face], u_in, rho_out)
    return fnew


def zou_he(lat: Lattice, f: np.ndarray, face: int, kind: int, u_in, rho_out: float) -> None:
    """Zou-He reconstruction of the unknown populations on one face (in place).

    Zou and He's non-equilibrium bounce-back, generalised to D3Q19 with the
    transverse-momentum correction of Hecht and Harting (2010).  With n the
    inward normal, the populations with c_i.n = +1 are unknown:
      rho (1 - u.n) = sum_{c.n=0} f + 2 sum_{c.n=-1} f        (mass)
      N_t = 1/2 sum_{c.n=0} (c.t) f - rho (u.t)/3           (each tangent t)
      f_i = f_opp(i) + 2 w_i rho (c_i.u)/c_s^2 - sum_t (c_i.t) N_t.
    A velocity inlet prescribes u (rho follows); a pressure outlet prescribes
    rho with zero tangential velocity (u.n follows).
    """
    a, side = divmod(face, 2)
    sgn = 1 if side == 0 else -1
    sl = _face_slice(face, f.shape[1:])
    fs = [f[i][sl] for i in range(lat.Q)]
    cn = lat.c[:, a] * sgn
    S0 = sum(fs[i] for i in range(lat.Q) if cn[i] == 0)
    Sm = sum(fs[i] for i in range(lat.Q) if cn[i] == -1)
    if kind == VEL_INLET:
        u = [np.full(S0.shape, float(u_in[b])) for b in range(lat.d)]
        un = u[a] * sgn
        rho = (S0 + 2.0 * Sm) / (1.0 - un)
    else:
        rho = np.full(S0.shape, float(rho_out))
        un = 1.0 - (S0 + 2.0 * Sm) / rho
        u = [np.zeros(S0.shape) for _ in range(lat.d)]
        u[a] = un * sgn
    tangents = [b for b in range(lat.d) if b != a]
    N = {}
    for b in tangents:
        N[b] = 0.5 * sum(lat.c[i, b] * fs[i] for i in range(lat.Q) if cn[i] == 0) \
            - rho * u[b] / 3.0
    for i in range(lat.Q):
        if cn[i] != 1:
            continue
        cu = sum(lat.c[i, b] * u[b] for b in range(lat.d))
        val = fs[lat.opp[i]] + 2.0 * lat.w[i] * rho * cu / lat.cs2
        for b in tangents:
            if lat.c[i, b] != 0:
                val = val - lat.c[i, b] * N[b]
        f[i][sl] = val
