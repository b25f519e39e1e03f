"""Discrete velocity sets (oracle; test infrastructure only).

D2Q9: Sec. 2.1 ("D2Q9 ... arrangement") with the weights of Eq. 5:
w0 = 4/9, w1..w4 = 1/9, w5..w8 = 1/36; sound speed c_s = 1/sqrt(3) (Eq. 3's
surrounding text), i.e. c_s^2 = 1/3 in lattice units.

D3Q19: not given by the paper, which runs in 2D only; the 3D wing cases use
the textbook D3Q19 set: rest weight 1/3, six face neighbours 1/18, twelve
edge neighbours 1/36, same c_s^2 = 1/3.

Velocities are stored with three components (c_z = 0 for D2Q9) so that the
rest of the oracle is dimension-agnostic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Lattice:
    name: str
    d: int              # spatial dimension
    c: np.ndarray       # [Q, 3] integer velocities
    w: np.ndarray       # [Q] weights
    opp: np.ndarray     # [Q] index of -c_i

    @property
    def Q(self) -> int:
        return self.c.shape[0]

    cs2: float = 1.0 / 3.0


def _make(name, d, vel, wts):
    c = np.array(vel, dtype=np.int64)
    w = np.array(wts, dtype=np.float64)
    opp = np.array([int(np.where((c == -ci).all(axis=1))[0][0]) for ci in c])
    return Lattice(name=name, d=d, c=c, w=w, opp=opp)


D2Q9 = _make(
    "D2Q9", 2,
    [(0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0),
     (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)],
    [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

D3Q19 = _make(
    "D3Q19", 3,
    [(0, 0, 0),
     (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
     (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
     (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
     (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)],
    [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def get(q: int) -> Lattice:
    if q == 9:
        return D2Q9
    if q == 19:
        return D3Q19
    raise ValueError(f"unknown lattice Q={q}")
