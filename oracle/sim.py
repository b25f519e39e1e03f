"""Whole IB-LBM time step of the oracle, in the paper's order (FP64; test infrastructure only).

Per step n (Sec. 2.2; the order "solve, spread, force density, new
equilibrium" is the one stated right after Eq. 19):

1. marker positions X_l and wall velocities U_B^l at t_n (kinematics);
2. moments of the current populations: rho = sum f_i and the intermediate
   velocity u* = (sum c_i f_i + G/2)/rho (Eq. 11; G is an optional uniform
   body force, zero in the paper's cases);
3. interpolation of u* and rho to the markers (Eq. 17);
4. B = U_B - u*_l and the dense solve A du_B = B, one column per velocity
   component (Eqs. 18-19);
5. spreading du(x) = sum_l du_B^l D ds_l (Eq. 15);
6. corrected velocity u = u* + du (Eq. 16) and force density
   F = 2 rho du + G (Eq. 26), so that rho u = sum c_i f_i + F/2 (Eq. 9);
7. BGK collision with the Guo term (Eqs. 7-8);
8. streaming with the boundary conditions;
9. body forces F_w = -sum_{l in w} 2 rho_l du_B^l ds_l (Sec. 3.7) and the
   coefficients C = F / (rho_ref U_ref^2 L / 2): C_D along the free stream
   (+x), C_T = -C_D, C_L along the body's lateral lift axis.
"""
from __future__ import annotations

import numpy as np

from . import ib, kinematics, lbm
from .lattice import get as get_lattice


class Simulation:
    def __init__(self, lattice_q: int, grid: dict, tau: float):
        self.lat = get_lattice(lattice_q)
        self.grid = grid
        self.tau = float(tau)
        self.shape = (int(grid["nz"]), int(grid["ny"]), int(grid["nx"]))
        self.bc = list(grid["bc"])
        lbm.check_bc(self.lat, self.bc)
        d = self.lat.d
        self.periodic = [self.bc[2 * a] == lbm.PERIODIC for a in range(d)]
        self.G = np.asarray(grid.get("body_force", (0, 0, 0)), dtype=np.float64)[:d]
        self.u_in = tuple(grid.get("u_in", (0.0, 0.0, 0.0)))
        self.rho_out = float(grid.get("rho_out", 1.0))
        self.bodies: list[dict] = []
        self.t = 0
        self.f = None
        self.history: list[list] = []
        self.reference = {"U_ref": 1.0, "L": 1.0, "rho_ref": 1.0}
        self.last = {}

    # ------------------------------------------------------------------ set-up
    def init_fluid(self, rho=None, u=None):
        d = self.lat.d
        rho = np.ones(self.shape) if rho is None else np.broadcast_to(
            np.asarray(rho, dtype=np.float64), self.shape).copy()
        if u is None:
            u = np.zeros((d,) + self.shape)
        else:
            u = np.asarray(u, dtype=np.float64)
            if u.ndim == 1:
                u = np.broadcast_to(u[:d, None, None, None], (d,) + self.shape).copy()
            u = u.reshape((d,) + self.shape)
        self.f = lbm.equilibrium(self.lat, rho, u)
        self.t = 0

    def set_populations(self, f):
        self.f = np.array(f, dtype=np.float64).reshape((self.lat.Q,) + self.shape)

    def add_body(self, body: dict) -> int:
        b = dict(body)
        b.setdefault("lift_axis", (0.0, 1.0, 0.0))
        b["prescribed"] = None
        self.bodies.append(b)
        self.history.append([])
        return len(self.bodies) - 1

    def set_marker_state(self, body_id: int, X, U):
        """Caller-supplied positions and wall velocities for the next step only."""
        self.bodies[body_id]["prescribed"] = (np.asarray(X, dtype=np.float64),
                                             np.asarray(U, dtype=np.float64))

    def set_reference(self, U_ref, L, rho_ref=1.0):
        self.reference = {"U_ref": float(U_ref), "L": float(L), "rho_ref": float(rho_ref)}

    # ------------------------------------------------------------------ step
    def markers(self, t):
        d = self.lat.d
        Xs, Us = [], []
        for b in self.bodies:
            if b["prescribed"] is not None:
                X, U = b["prescribed"]
            else:
                X, U = kinematics.marker_state(b, t, d)
            Xs.append(X[:, :d])
            Us.append(U[:, :d])
        return Xs, Us

    def step(self, n: int = 1):
        for _ in range(n):
            self._step_once()

    def _step_once(self):
        lat, d = self.lat, self.lat.d
        # 1. kinematics
        Xs, Us = self.markers(self.t)
        for b in self.bodies:
            b["prescribed"] = None
        # 2. moments: rho and intermediate velocity u* (Eq. 11, + G/2)
        rho = lbm.density(self.f)
        Gfield = np.broadcast_to(self.G[:, None, None, None], (d,) + self.shape)
        ustar = (lbm.momentum(lat, self.f) + 0.5 * Gfield) / rho
        F = np.array(Gfield)
        forces = []
        if self.bodies:
            X = np.concatenate(Xs, axis=0)
            U = np.concatenate(Us, axis=0)
            ds = np.concatenate([np.asarray(b["ds"], dtype=np.float64) for b in self.bodies])
            Dm = ib.spread_matrix(X, self.shape, self.periodic)
            # 3. interpolation
            u_l = ib.interpolate(Dm, ustar)
            rho_l = ib.interpolate(Dm, rho[None])[:, 0]
            # 4. implicit system
            A = ib.system_matrix(Dm, ds)
            B = U - u_l
            y = ib.solve(A, B)
            # 5-6. spreading and force density
            du = ib.spread(Dm, y, ds, self.shape)
            F = F + 2.0 * rho[None] * du
            fm = ib.marker_force(rho_l, y, ds)
            k = 0
            for b in self.bodies:
                m = len(b["ds"])
                forces.append(-fm[k:k + m].sum(axis=0))
                k += m
            self.last = {"X": X, "U": U, "u_l": u_l, "rho_l": rho_l, "B": B, "y": y,
                         "A": A, "du": du, "ustar": ustar, "rho": rho}
        # 7. collision, 8. streaming
        fpost = lbm.collide(lat, self.f, F, self.tau)
        self.f = lbm.stream(lat, fpost, self.bc, self.u_in, self.rho_out)
        self.last_F = F
        # 9. forces and coefficients
        for bid, Fw in enumerate(forces):
            self.history[bid].append(self.coefficients(bid, Fw))
        self.t += 1

    def coefficients(self, body_id: int, Fw: np.ndarray):
        d = self.lat.d
        ref = self.reference
        q = 0.5 * ref["rho_ref"] * ref["U_ref"] ** 2 * ref["L"]
        e_inf = np.zeros(d)
        e_inf[0] = 1.0
        e_l = np.asarray(self.bodies[body_id]["lift_axis"], dtype=np.float64)[:d]
        CD = float(Fw @ e_inf) / q
        CL = float(Fw @ e_l) / q
        return (CL, -CD, CD)

    # ------------------------------------------------------------------ outputs
    def fields(self):
        """rho and u = (sum c_i f_i + G/2)/rho of the current populations."""
        d = self.lat.d
        rho = lbm.density(self.f)
        Gfield = np.broadcast_to(self.G[:, None, None, None], (d,) + self.shape)
        u = (lbm.momentum(self.lat, self.f) + 0.5 * Gfield) / rho
        return rho, u
