"""x-slab decomposition of the oracle's IB-LBM step over CPU ranks (FP64; test infrastructure only).

This is the multi-GPU partition of the hot path, written on the oracle and
run as torch.distributed ranks (gloo, CPU), so that the partition - what each
rank owns, what it exchanges each step, and where the global sums are formed
- is checked against the undivided oracle (``oracle.sim``) bit for bit.

Partition (x is split, y and z are whole on every rank; x must be periodic):

* fluid: rank r owns the cells with x in [x0_r, x1_r) (nx split as evenly as
  possible); moments, forcing and the BGK collision (Eqs. 2, 7-9, 11) are
  per cell and run on the owned cells only;
* ghost layer of (rho, u*) two planes deep on each side, exchanged after the
  moments: a marker's 4-node stencil (Eq. 14) reaches one node below and two
  above floor(X_x);
* markers: every rank knows every marker's position (the kinematics,
  Eqs. 20-23, are evaluated everywhere); marker l is owned by the rank whose
  slab holds floor(X_l,x); the owner interpolates rho_l and u*_l (Eq. 17)
  from its owned and ghost cells, and a sum over ranks (all-reduce) gives
  every rank all markers' values - each value is contributed by one rank,
  the others add exact zeros, so the sums are exact;
* the system A X = B (Eqs. 18-19) depends on the marker positions only, so
  every rank assembles it and solves it itself (replicated owner-computes;
  no exchange); the solution and the body forces (Eq. 26, Sec. 3.7) are then
  identical everywhere;
* spreading (Eq. 15) fills the owned cells from all markers;
* streaming: the populations with c_x != 0 that leave a slab (5 of 19 per
  face for D3Q19, 3 of 9 for D2Q9) are exchanged as one plane per face.

Per step a rank sends 2 x 2 planes of 4 doubles (rho, u*; 3 in 2D), one
plane of the crossing populations per face, and one all-reduce of 4 m
doubles.  Every sum that the undivided oracle forms over the grid (the
interpolation's sum over a stencil, the spreading's sum over markers) is
formed here on one rank in the same order, which is why the two agree
bitwise.
"""
from __future__ import annotations

import numpy as np

from . import ib, kinematics, lbm
from .lattice import get as get_lattice


def slab_bounds(nx: int, world: int, rank: int) -> tuple[int, int]:
    """[x0, x1) of rank's slab: nx split as evenly as possible, lower ranks first."""
    base, extra = divmod(nx, world)
    x0 = rank * base + min(rank, extra)
    return x0, x0 + base + (1 if rank < extra else 0)


class SlabSimulation:
    """One rank's share of ``oracle.sim.Simulation`` (same step, same results)."""

    GHOST = 2

    def __init__(self, lattice_q: int, grid: dict, tau: float, dist, rank: int, world: int):
        self.lat = get_lattice(lattice_q)
        self.grid = grid
        self.tau = float(tau)
        self.dist, self.rank, self.world = dist, rank, world
        self.shape = (int(grid["nz"]), int(grid["ny"]), int(grid["nx"]))
        self.bc = list(grid["bc"])
        lbm.check_bc(self.lat, self.bc)
        if self.bc[0] != lbm.PERIODIC:
            raise ValueError("the slab partition splits x, which must be periodic")
        d = self.lat.d
        self.periodic = [self.bc[2 * a] == lbm.PERIODIC for a in range(d)]
        self.G = np.asarray(grid.get("body_force", (0, 0, 0)), dtype=np.float64)[:d]
        self.x0, self.x1 = slab_bounds(self.shape[2], world, rank)
        if self.x1 - self.x0 < self.GHOST:
            raise ValueError("every slab needs at least two planes")
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.bodies: list[dict] = []
        self.history: list[list] = []
        self.reference = {"U_ref": 1.0, "L": 1.0, "rho_ref": 1.0}
        self.t = 0
        self.f = None

    # ------------------------------------------------------------------ set-up
    def init_fluid(self, u_global: np.ndarray):
        """f = f_eq(1, u) on the owned cells; u_global [d, nz, ny, nx] (or a [d] constant)."""
        d = self.lat.d
        u = np.asarray(u_global, dtype=np.float64)
        if u.ndim == 1:
            u = np.broadcast_to(u[:d, None, None, None], (d,) + self.shape)
        u = np.ascontiguousarray(u[:d, :, :, self.x0:self.x1])
        rho = np.ones(u.shape[1:])
        self.f = lbm.equilibrium(self.lat, rho, u)
        self.t = 0

    def add_body(self, body: dict) -> int:
        b = dict(body)
        b.setdefault("lift_axis", (0.0, 1.0, 0.0))
        self.bodies.append(b)
        self.history.append([])
        return len(self.bodies) - 1

    def set_reference(self, U_ref, L, rho_ref=1.0):
        self.reference = {"U_ref": float(U_ref), "L": float(L), "rho_ref": float(rho_ref)}

    # ------------------------------------------------------------------ exchange
    def _exchange_x(self, arr: np.ndarray, depth: int) -> np.ndarray:
        """arr [..., nloc] extended by `depth` planes from each neighbour: [..., depth + nloc + depth]."""
        import torch
        send_l = torch.from_numpy(np.ascontiguousarray(arr[..., :depth]))
        send_r = torch.from_numpy(np.ascontiguousarray(arr[..., -depth:]))
        recv_l = torch.empty_like(send_l)
        recv_r = torch.empty_like(send_r)
        if self.world == 1:
            recv_l.copy_(send_r)
            recv_r.copy_(send_l)
        else:
            # tag 1: planes travelling left, tag 2: travelling right (with two
            # ranks the left and right neighbour are the same rank)
            reqs = [self.dist.isend(send_l, self.left, tag=1), self.dist.isend(send_r, self.right, tag=2),
                    self.dist.irecv(recv_l, self.left, tag=2), self.dist.irecv(recv_r, self.right, tag=1)]
            for q in reqs:
                q.wait()
        return np.concatenate([recv_l.numpy(), arr, recv_r.numpy()], axis=-1)

    def _allreduce(self, a: np.ndarray) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.ascontiguousarray(a))
        if self.world > 1:
            self.dist.all_reduce(t)
        return t.numpy()

    # ------------------------------------------------------------------ step
    def step(self, n: int = 1):
        for _ in range(n):
            self._step_once()

    def _owned_interpolation(self, Dm, ext: np.ndarray, owned: np.ndarray) -> np.ndarray:
        """For the owned markers: sum over their stencil cells, in ascending
        global cell index (the order of the undivided oracle's sparse
        transpose product), of D(x - X_l) times ext's value at the cell;
        ext [c, nz, ny, nloc + 2 GHOST] holds the owned and ghost planes."""
        nz, ny, nx = self.shape
        Dc = Dm.tocsc()
        out = np.zeros((len(owned), ext.shape[0]))
        for r, l in enumerate(owned):
            lo, hi = Dc.indptr[l], Dc.indptr[l + 1]
            cells, vals = Dc.indices[lo:hi], Dc.data[lo:hi]
            order = np.argsort(cells, kind="stable")
            cells, vals = cells[order], vals[order]
            x = cells % nx
            yz = cells // nx
            xl = (x - self.x0 + self.GHOST) % nx          # position in the extended slab
            acc = np.zeros(ext.shape[0])
            for cidx, xi, w in zip(yz, xl, vals):
                acc = acc + w * ext[:, cidx // ny, cidx % ny, xi]
            out[r] = acc
        return out

    def _step_once(self):
        lat, d = self.lat, self.lat.d
        nz, ny, nx = self.shape
        nloc = self.x1 - self.x0
        # 1. kinematics (every rank, every marker)
        Xs, Us = [], []
        for b in self.bodies:
            X, U = kinematics.marker_state(b, self.t, d)
            Xs.append(X[:, :d])
            Us.append(U[:, :d])
        # 2. moments on the owned cells (Eq. 11, + G/2), then the ghost layer
        rho = lbm.density(self.f)
        Gfield = np.broadcast_to(self.G[:, None, None, None], (d,) + rho.shape)
        ustar = (lbm.momentum(lat, self.f) + 0.5 * Gfield) / rho
        F = np.array(Gfield)
        forces = []
        if self.bodies:
            X = np.concatenate(Xs, axis=0)
            U = np.concatenate(Us, axis=0)
            ds = np.concatenate([np.asarray(b["ds"], dtype=np.float64) for b in self.bodies])
            ext = self._exchange_x(np.concatenate([rho[None], ustar], axis=0), self.GHOST)
            Dm = ib.spread_matrix(X, self.shape, self.periodic)     # geometry only: replicated
            # 3. interpolation by each marker's owner, completed by an exact all-reduce
            base_x = np.floor(X[:, 0]).astype(np.int64) % nx
            owned = np.nonzero((base_x >= self.x0) & (base_x < self.x1))[0]
            vals = np.zeros((X.shape[0], 1 + d))
            vals[owned] = self._owned_interpolation(Dm, ext, owned)
            vals = self._allreduce(vals)
            rho_l, u_l = vals[:, 0], vals[:, 1:]
            # 4. the implicit system, assembled and solved by every rank
            A = ib.system_matrix(Dm, ds)
            B = U - u_l
            y = ib.solve(A, B)
            # 5-6. spreading onto the owned cells and force density
            cols = np.arange(self.x0, self.x1)
            rows = ((np.arange(nz)[:, None, None] * ny + np.arange(ny)[None, :, None]) * nx
                    + cols[None, None, :]).ravel()
            Dloc = Dm[rows]
            du = np.stack([Dloc @ (y[:, k] * ds) for k in range(d)], axis=0).reshape((d, nz, ny, nloc))
            F = F + 2.0 * rho[None] * du
            fm = ib.marker_force(rho_l, y, ds)
            k = 0
            for b in self.bodies:
                m = len(b["ds"])
                forces.append(-fm[k:k + m].sum(axis=0))
                k += m
        # 7. collision on the owned cells
        fpost = lbm.collide(lat, self.f, F, self.tau)
        # 8. streaming: one plane of the populations crossing each x face,
        # y and z whole on this rank (rolled or bounced as in the oracle)
        ext = self._exchange_x(fpost, 1)
        fnew = np.empty_like(fpost)
        for i in range(lat.Q):
            cx, cy, cz = (int(v) for v in lat.c[i])
            src = ext[i][:, :, 1 - cx:1 - cx + nloc]
            fnew[i] = np.roll(src, shift=(cz, cy), axis=(0, 1))
        for i in range(lat.Q):
            for a in range(1, d):
                ca = int(lat.c[i, a])
                if ca == 0:
                    continue
                face = 2 * a if ca > 0 else 2 * a + 1
                if self.bc[face] == lbm.BOUNCEBACK:
                    sl = lbm._face_slice(face, fpost.shape[1:])
                    fnew[i][sl] = fpost[lat.opp[i]][sl]
        for face in range(2, 2 * d):
            if self.bc[face] in (lbm.VEL_INLET, lbm.PRESS_OUTLET):
                raise ValueError("Zou-He faces on the unsplit axes are not supported by the slab partition")
        self.f = fnew
        # 9. forces (identical on every rank)
        for bid, Fw in enumerate(forces):
            self.history[bid].append(self._coefficients(bid, Fw))
        self.t += 1

    def _coefficients(self, body_id: int, Fw: np.ndarray):
        d = self.lat.d
        ref = self.reference
        q = 0.5 * ref["rho_ref"] * ref["U_ref"] ** 2 * ref["L"]
        e_inf = np.zeros(d)
        e_inf[0] = 1.0
        e_l = np.asarray(self.bodies[body_id]["lift_axis"], dtype=np.float64)[:d]
        CD = float(Fw @ e_inf) / q
        CL = float(Fw @ e_l) / q
        return (CL, -CD, CD)

    def gather_populations(self) -> np.ndarray | None:
        """The whole grid's populations on rank 0 (None elsewhere)."""
        import torch
        t = torch.from_numpy(np.ascontiguousarray(self.f))
        if self.world == 1:
            return self.f.copy()
        parts = [torch.empty((self.lat.Q,) + self.shape[:2] + (b1 - b0,), dtype=t.dtype)
                 for b0, b1 in (slab_bounds(self.shape[2], self.world, r) for r in range(self.world))]
        if self.rank == 0:
            parts[0].copy_(t)
            for r in range(1, self.world):
                self.dist.recv(parts[r], r)
            return np.concatenate([p.numpy() for p in parts], axis=-1)
        self.dist.send(t, 0)
        return None
