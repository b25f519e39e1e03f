"""Implicit velocity-correction immersed boundary of the oracle (FP64; test infrastructure only).

Follows Sec. 2.2 (Wu and Shu's formulation) in lattice units (dx = dy = dz = 1):

* delta function: D(x - X) = prod_d phi(x_d - X_d) (Eq. 13; its tensor
  product extends to 3D) with the 4-point cosine kernel
  phi(r) = (1 + cos(pi |r| / 2)) / 4 for |r| <= 2, else 0 (Eq. 14);
* spreading: du(x) = sum_l du_B^l D(x - X_l) ds_l (Eq. 15);
* interpolation: U(X_l) = sum_x u(x) D(x - X_l) (Eq. 17, dx dy = 1);
* implicit system A X = B (Eqs. 18-19): A_lk = sum_x D(x - X_l) D(x - X_k) ds_k,
  B_l = U_B^l - sum_x u*(x) D(x - X_l); Eq. 18's garbled double sum is read as
  this product (the second marker index is k);
* force density on the fluid F = 2 rho du / dt (Eq. 26); a marker's share is
  2 rho_l du_B^l ds_l with rho_l the interpolated density, and the body force
  is minus the sum over the body's markers (Sec. 3.7).

Stencil: every axis uses the 4 nodes floor(X_d)-1 .. floor(X_d)+2, which hold
the whole support |x_d - X_d| < 2.  Periodic axes wrap; on a non-periodic axis
a stencil that leaves the domain is an error (the paper is silent).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def phi(r):
    """4-point cosine kernel (Eq. 14)."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    return np.where(r <= 2.0, 0.25 * (1.0 + np.cos(0.5 * math.pi * r)), 0.0)


def stencil_1d(Xd: np.ndarray, n: int, periodic: bool):
    """Node indices [m,4] and weights [m,4] of one axis for marker coordinates Xd [m]."""
    base = np.floor(Xd).astype(np.int64) - 1
    nodes = base[:, None] + np.arange(4)[None, :]
    w = phi(nodes - Xd[:, None])
    if periodic:
        nodes = np.mod(nodes, n)
    elif (nodes < 0).any() or (nodes >= n).any():
        raise ValueError("marker stencil leaves a non-periodic axis")
    return nodes, w


def spread_matrix(X: np.ndarray, shape_zyx, periodic) -> sp.csr_matrix:
    """Sparse delta matrix Dm [N_cells, m] with Dm[x, l] = D(x - X_l) (Eq. 13).

    X has shape [m, d]; cells are flattened as (z*ny + y)*nx + x.
    """
    nz, ny, nx = shape_zyx
    m, d = X.shape
    n_axis = [nx, ny, nz]
    idx, wts = [], []
    for a in range(d):
        nodes, w = stencil_1d(X[:, a], n_axis[a], bool(periodic[a]))
        idx.append(nodes)
        wts.append(w)
    if d == 2:
        idx.append(np.zeros((m, 1), dtype=np.int64))
        wts.append(np.ones((m, 1)))
    ix, iy, iz = idx
    wx, wy, wz = wts
    rows = (iz[:, :, None, None] * ny + iy[:, None, :, None]) * nx + ix[:, None, None, :]
    vals = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
    cols = np.broadcast_to(np.arange(m)[:, None, None, None], rows.shape)
    Dm = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())),
                       shape=(nx * ny * nz, m))
    return Dm.tocsr()


def interpolate(Dm: sp.csr_matrix, field: np.ndarray) -> np.ndarray:
    """Marker values sum_x field(x) D(x - X_l) (Eq. 17). field [c, nz, ny, nx] -> [m, c]."""
    flat = field.reshape(field.shape[0], -1)
    return np.stack([Dm.T @ flat[k] for k in range(flat.shape[0])], axis=1)


def spread(Dm: sp.csr_matrix, values: np.ndarray, ds: np.ndarray, shape_zyx) -> np.ndarray:
    """Eulerian field sum_l values_l D(x - X_l) ds_l (Eq. 15). values [m, c] -> [c, nz, ny, nx]."""
    out = [Dm @ (values[:, k] * ds) for k in range(values.shape[1])]
    return np.stack(out, axis=0).reshape((values.shape[1],) + tuple(shape_zyx))


def system_matrix(Dm: sp.csr_matrix, ds: np.ndarray) -> np.ndarray:
    """Dense A with A_lk = sum_x D(x - X_l) D(x - X_k) ds_k (Eq. 18, reading above)."""
    G = (Dm.T @ Dm).toarray()
    return G * ds[None, :]


def solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Direct dense solve of A X = B for every velocity component (Eq. 19, Sec. 2.2).

    LU with partial pivoting (numpy's LAPACK gesv) - the paper solves the
    system exactly at every step.
    """
    return np.linalg.solve(A, B)


def marker_force(rho_l: np.ndarray, du_B: np.ndarray, ds: np.ndarray) -> np.ndarray:
    """Force each marker applies to the fluid: 2 rho_l du_B^l ds_l (Eq. 26 times ds), [m, d]."""
    return 2.0 * rho_l[:, None] * du_B * ds[:, None]
