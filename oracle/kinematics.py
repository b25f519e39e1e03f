"""Prescribed rigid-body kinematics of the oracle (FP64; test infrastructure only).

Wave forms, with theta(t) = 2 pi f t + phi (f in cycles per lattice step):

* CONST    value = offset
* COS      value = offset + amp cos(theta)        (Eq. 20: amp = A0/2)
* SIN      value = offset + amp sin(theta)        (Eq. 21: offset = pi/4, amp = -pi/4;
                                                   Eq. 23: offset = 0, amp = pi/3)
* ABS_SIN  value = offset + amp |sin(theta)|      (reading of Sec. 3.3: each wing
                                                   opens 0..60 degrees, the pair
                                                   claps twice per period)
* TABLE    value = table[n mod len], rate = central difference of the table

A body's markers move rigidly: with body-frame coordinates X0, hinge h,
rotation axis e (unit), placement ``origin`` and stroke direction
e_s = (cos beta, sin beta, 0) (Sec. 3.2, stroke plane inclined at beta):
    r(t) = R(e, alpha(t)) (X0 - h)
    X(t) = origin + h + r(t) + A(t) e_s
    U(t) = A'(t) e_s + alpha'(t) e x r(t)
The rotation rate term is the "rotational velocities ... given in addition"
of Sec. 3.3.  Both are evaluated at the step's own time t_n = n (the paper is
silent on the time level; the same level as the fluid velocity u*(t_n)).
"""
from __future__ import annotations

import math

import numpy as np

CONST, COS, SIN, ABS_SIN, TABLE = 0, 1, 2, 3, 4


def wave(w: dict, t: float, f: float, phi: float):
    """(value, d value / dt) of a wave at time t."""
    kind = w["kind"]
    amp = float(w.get("amp", 0.0))
    off = float(w.get("offset", 0.0))
    om = 2.0 * math.pi * f
    th = om * t + phi
    if kind == CONST:
        return off, 0.0
    if kind == COS:
        return off + amp * math.cos(th), -amp * om * math.sin(th)
    if kind == SIN:
        return off + amp * math.sin(th), amp * om * math.cos(th)
    if kind == ABS_SIN:
        s = math.sin(th)
        sgn = 1.0 if s >= 0.0 else -1.0
        return off + amp * abs(s), amp * om * math.cos(th) * sgn
    if kind == TABLE:
        tab = np.asarray(w["table"], dtype=np.float64)
        n = len(tab)
        k = int(round(t))
        return float(tab[k % n]), 0.5 * float(tab[(k + 1) % n] - tab[(k - 1) % n])
    raise ValueError(f"unknown wave kind {kind}")


def rotation(axis, angle: float) -> np.ndarray:
    """Rotation matrix about a unit axis (Rodrigues' formula)."""
    e = np.asarray(axis, dtype=np.float64)
    e = e / np.linalg.norm(e)
    K = np.array([[0.0, -e[2], e[1]], [e[2], 0.0, -e[0]], [-e[1], e[0], 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def marker_state(body: dict, t: float, d: int):
    """Marker positions X [m,d] and wall velocities U_B [m,d] of a rigid body at time t."""
    X0 = np.asarray(body["X0"], dtype=np.float64)
    m = X0.shape[0]
    X03 = np.zeros((m, 3))
    X03[:, :X0.shape[1]] = X0
    h = np.asarray(body["hinge"], dtype=np.float64)
    e = np.asarray(body["axis"], dtype=np.float64)
    e = e / np.linalg.norm(e)
    org = np.asarray(body["origin"], dtype=np.float64)
    f, ph = float(body["f"]), float(body["phi"])
    A, Ad = wave(body["A"], t, f, ph)
    al, ald = wave(body["alpha"], t, f, ph)
    beta = float(body["beta"])
    es = np.array([math.cos(beta), math.sin(beta), 0.0])
    r = (X03 - h) @ rotation(e, al).T
    X = org + h + r + A * es
    U = Ad * es + ald * np.cross(e, r)
    return X[:, :d], U[:, :d]
