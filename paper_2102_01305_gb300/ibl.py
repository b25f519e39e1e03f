"""Thin ctypes binding of libibl (the C ABI in include/ibl.h), same names.

Only argument marshalling happens here: numpy arrays are passed as host
pointers and every step of the IB-LBM path runs in the library's CUDA
kernels.  There is no fallback: if ``libibl.so`` is missing or fails to load,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibl.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2102_01305_gb300.build.build() "
                      "(nvcc, sm_103a); there is no CPU fallback")
_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------ enums (ibl.h)
(IBL_OK, IBL_EINVAL, IBL_ENOMEM, IBL_ECUDA, IBL_EDIVERGED, IBL_ENOTCONV, IBL_ETIMEOUT, IBL_ESTATE,
 IBL_ECANCELED, IBL_EUNSTABLE) = range(10)
IBL_D2Q9, IBL_D3Q19 = 9, 19
IBL_PERIODIC, IBL_BOUNCEBACK, IBL_VEL_INLET, IBL_PRESS_OUTLET = range(4)
IBL_FP64, IBL_FP32, IBL_FP16DEV, IBL_BF16DEV = range(4)
IBL_WAVE_CONST, IBL_WAVE_COS, IBL_WAVE_SIN, IBL_WAVE_ABS_SIN, IBL_WAVE_TABLE = range(5)
IBL_FIELD_RHO, IBL_FIELD_U, IBL_FIELD_FORCE = range(3)
STATUS_NAMES = ["IBL_OK", "IBL_EINVAL", "IBL_ENOMEM", "IBL_ECUDA", "IBL_EDIVERGED",
                "IBL_ENOTCONV", "IBL_ETIMEOUT", "IBL_ESTATE", "IBL_ECANCELED", "IBL_EUNSTABLE"]
PRECISIONS = {"fp64": IBL_FP64, "fp32": IBL_FP32, "fp16dev": IBL_FP16DEV, "bf16dev": IBL_BF16DEV}


class ibl_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("bc", C.c_int32 * 6), ("u_in", C.c_double * 3), ("rho_out", C.c_double),
                ("body_force", C.c_double * 3), ("precision", C.c_int32)]


class ibl_wave(C.Structure):
    _fields_ = [("kind", C.c_int32), ("amp", C.c_double), ("offset", C.c_double),
                ("table", C.POINTER(C.c_double)), ("n_table", C.c_int64)]


class ibl_server_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_active", C.c_int32), ("chunk_steps", C.c_int32),
                ("tune", C.c_int32)]


class ibl_run_request(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("chord", C.c_double),
                ("Re", C.c_double), ("period", C.c_double), ("J", C.c_double), ("precision", C.c_int32),
                ("faces", C.c_int32), ("steps", C.c_int64)]


class ibl_run_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("done", C.c_int32), ("steps_done", C.c_int64),
                ("submit_s", C.c_double), ("start_s", C.c_double), ("finish_s", C.c_double),
                ("CL_max", C.c_double * 2), ("CL_mean", C.c_double * 2), ("CT_max", C.c_double * 2),
                ("CT_mean", C.c_double * 2), ("CL_last", C.c_double * 2), ("CT_last", C.c_double * 2),
                ("solve_blocks", C.c_int32), ("overlap", C.c_int32), ("collide_bx", C.c_int32),
                ("collide_by", C.c_int32), ("collide_pairs", C.c_int32), ("tuned", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)

_SIGS = {
    "ibl_create": ([C.POINTER(ibl_grid), C.c_double, C.c_int32, C.POINTER(_P)], C.c_int),
    "ibl_destroy": ([_P], C.c_int),
    "ibl_init_fluid": ([_P, _D, _D], C.c_int),
    "ibl_set_populations": ([_P, _D], C.c_int),
    "ibl_set_markers": ([_P, C.c_int32, _D, _D, _D, _D, _D, _I32], C.c_int),
    "ibl_set_kinematics": ([_P, C.c_int32, C.POINTER(ibl_wave), C.POINTER(ibl_wave), C.c_double,
                            C.c_double, C.c_double, C.c_double], C.c_int),
    "ibl_set_marker_state": ([_P, C.c_int32, _D, _D], C.c_int),
    "ibl_set_lift_axis": ([_P, C.c_int32, _D], C.c_int),
    "ibl_set_reference": ([_P, C.c_double, C.c_double, C.c_double], C.c_int),
    "ibl_step": ([_P, C.c_int64], C.c_int),
    "ibl_sync": ([_P], C.c_int),
    "ibl_forces": ([_P, C.c_int32, _D, _D, _D], C.c_int),
    "ibl_force_history": ([_P, C.c_int32, C.c_int64, _D, _I64], C.c_int),
    "ibl_get_field": ([_P, C.c_int32, _D], C.c_int),
    "ibl_get_populations": ([_P, _D], C.c_int),
    "ibl_get_markers": ([_P, C.c_int32, _D, _D, _D], C.c_int),
    "ibl_mass": ([_P, _D], C.c_int),
    "ibl_mass_noalloc": ([_P, C.c_int32, _D], C.c_int),
    "ibl_set_mass_check": ([_P, C.c_int32, C.c_double], C.c_int),
    "ibl_mass_check_read": ([_P, _D, _D, _I64], C.c_int),
    "ibl_set_overlap": ([_P, C.c_int32], C.c_int),
    "ibl_set_collide_shape": ([_P, C.c_int32, C.c_int32, C.c_int32], C.c_int),
    "ibl_profile_phases": ([_P, _D, C.c_int32], C.c_int),
    "ibl_solver_blocks": ([_P, C.c_int32], C.c_int),
    "ibl_interpolate_points": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "ibl_spread_points": ([_P, C.c_int32, _P, _P, _P, _P], C.c_int),
    "ibl_lattice_velocities": ([C.c_int32, _I32, _I32, _D], C.c_int),
    "ibl_solver_stats": ([_P, _I32, _D, _I64], C.c_int),
    "ibl_solver_trace": ([_P, _I64, C.c_int32, _I32], C.c_int),
    "ibl_solver_config": ([_P, C.c_int32, C.c_double, C.c_int32], C.c_int),
    "ibl_solver_preconditioner": ([_P, C.c_int32, C.c_int32], C.c_int),
    "ibl_profile": ([_P, C.c_int32], C.c_int),
    "ibl_profile_read": ([_P, _D, _D, _I64], C.c_int),
    "ibl_launch_count": ([_P, _I64], C.c_int),
    "ibl_stream": ([_P, C.POINTER(_P)], C.c_int),
    "ibl_last_error": ([_P], C.c_char_p),
    "ibl_server_create": ([C.POINTER(ibl_server_config), C.POINTER(_P)], C.c_int),
    "ibl_server_submit": ([_P, C.POINTER(ibl_run_request), _I64], C.c_int),
    "ibl_server_poll": ([_P, C.c_int64, C.POINTER(ibl_run_result)], C.c_int),
    "ibl_server_load": ([_P, _D, _D, _D, _D, _D], C.c_int),
    "ibl_server_cancel": ([_P, C.c_int64], C.c_int),
    "ibl_server_wait_all": ([_P, C.c_double], C.c_int),
    "ibl_server_stats": ([_P, _I32, _I32, _I32, _I64], C.c_int),
    "ibl_server_destroy": ([_P], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


class IblError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(ctx, status, allow=()):
    if status != IBL_OK and status not in allow:
        raise IblError(status, last_error(ctx))
    return status


def last_error(ctx=None) -> str:
    return (_lib.ibl_last_error(ctx) or b"").decode()


def exported_symbols():
    return list(_SIGS)


def lattice_velocities(lattice: int):
    q = C.c_int32()
    c = np.zeros((lattice, 3), dtype=np.int32)
    w = np.zeros(lattice)
    _check(None, _lib.ibl_lattice_velocities(lattice, C.byref(q), c.ctypes.data_as(_I32), _dptr(w)))
    return c, w


def _wave(w: dict | None):
    if w is None:
        return None, None
    wv = ibl_wave()
    wv.kind = int(w.get("kind", IBL_WAVE_CONST))
    wv.amp = float(w.get("amp", 0.0))
    wv.offset = float(w.get("offset", 0.0))
    keep = None
    if wv.kind == IBL_WAVE_TABLE:
        keep = _f64(w["table"])
        wv.table = _dptr(keep)
        wv.n_table = keep.size
    return wv, keep


def _torch():
    import torch
    return torch


def _device_f64(t, name, ndim, last):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if t.dim() != ndim or (last is not None and t.shape[-1] != last):
        raise ValueError(f"{name} has shape {tuple(t.shape)}")
    return t.contiguous()


def _device_out(t, shape, like):
    torch = _torch()
    if t is None:
        return torch.empty(shape, dtype=torch.float64, device=like.device)
    t = _device_f64(t, "output", len(shape), shape[-1])
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"output must be a contiguous {shape} tensor")
    return t


PHASES = ["kinematics", "counter_reset", "tile_mark", "slot_assign", "marker_lists", "interpolation",
          "assembly", "solve", "spreading", "collide"]


class Context:
    """Owning wrapper around an ibl_ctx*; methods map 1:1 onto the C calls."""

    def __init__(self, grid: dict, tau: float, lattice: int):
        g = ibl_grid()
        g.nx, g.ny, g.nz = int(grid["nx"]), int(grid["ny"]), int(grid["nz"])
        for i, b in enumerate(grid["bc"]):
            g.bc[i] = int(b)
        for a in range(3):
            g.u_in[a] = float(grid.get("u_in", (0, 0, 0))[a])
            g.body_force[a] = float(grid.get("body_force", (0, 0, 0))[a])
        g.rho_out = float(grid.get("rho_out", 1.0))
        prec = grid.get("precision", "fp32")
        g.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.lattice = int(lattice)
        self.d = 2 if self.lattice == IBL_D2Q9 else 3
        self.shape = (g.nz, g.ny, g.nx)
        self.N = g.nx * g.ny * g.nz
        h = _P()
        _check(None, _lib.ibl_create(C.byref(g), float(tau), self.lattice, C.byref(h)))
        self.h = h
        self.nbodies = 0

    def close(self):
        if getattr(self, "h", None):
            _lib.ibl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- set-up
    def ibl_init_fluid(self, rho=None, u=None):
        r = None if rho is None else _f64(np.broadcast_to(rho, self.shape))
        uu = None
        if u is not None:
            u = np.asarray(u, dtype=np.float64)
            if u.ndim == 1:
                u = np.broadcast_to(u[:self.d, None, None, None], (self.d,) + self.shape)
            uu = _f64(u.reshape((self.d,) + self.shape))
        _check(self.h, _lib.ibl_init_fluid(self.h, _dptr(r), _dptr(uu)))

    def ibl_set_populations(self, f):
        f = _f64(f)
        assert f.size == self.lattice * self.N
        _check(self.h, _lib.ibl_set_populations(self.h, _dptr(f)))

    def ibl_set_markers(self, X0, ds, hinge, axis, origin) -> int:
        X0 = _f64(np.asarray(X0)[:, :self.d])
        ds = _f64(ds)
        bid = C.c_int32()
        _check(self.h, _lib.ibl_set_markers(self.h, X0.shape[0], _dptr(X0), _dptr(ds),
                                            _dptr(_f64(hinge)), _dptr(_f64(axis)), _dptr(_f64(origin)),
                                            C.byref(bid)))
        self.nbodies += 1
        return bid.value

    def ibl_set_kinematics(self, body_id, A, alpha, beta=0.0, phi=0.0, f=0.0, J=0.0):
        wa, ka = _wave(A)
        wb, kb = _wave(alpha)
        _check(self.h, _lib.ibl_set_kinematics(self.h, body_id, C.byref(wa) if wa else None,
                                               C.byref(wb) if wb else None, float(beta), float(phi),
                                               float(f), float(J)))
        del ka, kb

    def ibl_set_marker_state(self, body_id, X, U):
        X = _f64(np.asarray(X)[:, :self.d])
        U = _f64(np.asarray(U)[:, :self.d])
        _check(self.h, _lib.ibl_set_marker_state(self.h, body_id, _dptr(X), _dptr(U)))

    def ibl_set_lift_axis(self, body_id, e):
        _check(self.h, _lib.ibl_set_lift_axis(self.h, body_id, _dptr(_f64(e))))

    def ibl_set_reference(self, U_ref, L_or_S, rho_ref=1.0):
        _check(self.h, _lib.ibl_set_reference(self.h, float(U_ref), float(L_or_S), float(rho_ref)))

    def add_body(self, body: dict) -> int:
        """Convenience: markers + kinematics (+ lift axis) from a workload body dict."""
        bid = self.ibl_set_markers(body["X0"], body["ds"], body["hinge"], body["axis"], body["origin"])
        self.ibl_set_kinematics(bid, body["A"], body["alpha"], body.get("beta", 0.0), body.get("phi", 0.0),
                                body.get("f", 0.0), body.get("J", 0.0))
        if "lift_axis" in body:
            self.ibl_set_lift_axis(bid, body["lift_axis"])
        return bid

    # ---------------------------------------------------------------- stepping
    def ibl_step(self, n: int = 1, allow=()):
        return _check(self.h, _lib.ibl_step(self.h, int(n)), allow)

    def ibl_sync(self, allow=()):
        return _check(self.h, _lib.ibl_sync(self.h), allow)

    # ---------------------------------------------------------------- outputs
    def ibl_forces(self, body_id, allow=()):
        cl, ct, cd = C.c_double(), C.c_double(), C.c_double()
        _check(self.h, _lib.ibl_forces(self.h, body_id, C.byref(cl), C.byref(ct), C.byref(cd)), allow)
        return cl.value, ct.value, cd.value

    def ibl_force_history(self, body_id, max_n, allow=()):
        out = np.zeros((max(int(max_n), 1), 3))
        n = C.c_int64()
        _check(self.h, _lib.ibl_force_history(self.h, body_id, int(max_n), _dptr(out), C.byref(n)), allow)
        return out[:n.value]

    def ibl_get_field(self, what, allow=()):
        comps = 1 if what == IBL_FIELD_RHO else self.d
        out = np.zeros((comps,) + self.shape)
        _check(self.h, _lib.ibl_get_field(self.h, int(what), _dptr(out)), allow)
        return out[0] if what == IBL_FIELD_RHO else out

    def ibl_get_populations(self, allow=()):
        out = np.zeros((self.lattice,) + self.shape)
        _check(self.h, _lib.ibl_get_populations(self.h, _dptr(out)), allow)
        return out

    def ibl_get_markers(self, body_id, m, allow=()):
        X = np.zeros((m, self.d))
        U = np.zeros((m, self.d))
        F = np.zeros((m, self.d))
        _check(self.h, _lib.ibl_get_markers(self.h, body_id, _dptr(X), _dptr(U), _dptr(F)), allow)
        return X, U, F

    def ibl_mass(self, allow=()):
        m = C.c_double()
        _check(self.h, _lib.ibl_mass(self.h, C.byref(m)), allow)
        return m.value

    def ibl_mass_noalloc(self, nparts=1024, allow=()):
        """Total mass without any device allocation (static scratch, see ibl.h)."""
        m = C.c_double()
        _check(self.h, _lib.ibl_mass_noalloc(self.h, int(nparts), C.byref(m)), allow)
        return m.value

    def ibl_set_mass_check(self, every=500, rel_tol=0.0):
        """FP64 mass check every `every` steps (0: off); rel_tol 0: default for the precision."""
        _check(self.h, _lib.ibl_set_mass_check(self.h, int(every), float(rel_tol)))

    def ibl_mass_check_read(self, allow=()):
        """(reference total, last checked total, checks so far)."""
        m0, m1, n = C.c_double(), C.c_double(), C.c_int64()
        _check(self.h, _lib.ibl_mass_check_read(self.h, C.byref(m0), C.byref(m1), C.byref(n)), allow)
        return m0.value, m1.value, n.value

    def ibl_solver_blocks(self, blocks):
        """Blocks of the cooperative solve (0: half the SMs)."""
        _check(self.h, _lib.ibl_solver_blocks(self.h, int(blocks)))

    def ibl_profile_phases(self):
        """Per-phase milliseconds (ibl_profile level 2): dict phase name -> ms."""
        ms = np.zeros(10)
        _check(self.h, _lib.ibl_profile_phases(self.h, ms.ctypes.data_as(_D), 10))
        return dict(zip(PHASES, ms.tolist()))

    def ibl_set_overlap(self, mode):
        """-1 automatic, 0 one collide kernel after the IB chain, 1 split step, 2 serial split."""
        _check(self.h, _lib.ibl_set_overlap(self.h, int(mode)))

    def ibl_set_collide_shape(self, bx=64, by=2, pairs=3):
        """Thread block (bx x by) of the one-kernel collide; 16-bit storage: pairs 3 two cells and
        8 z-planes per thread, 1 two cells per thread, 2 the same on planes staged in shared memory,
        0 one cell per thread."""
        _check(self.h, _lib.ibl_set_collide_shape(self.h, int(bx), int(by), int(pairs)))

    def ibl_interpolate_points(self, X, U=None, rho=None):
        """rho and u* of the current populations at points X (Eq. 17).

        X: CUDA float64 tensor [m, 3]; returns (U [m, d], rho [m]), freshly
        allocated unless given.  Torch's current stream is synchronised first.
        """
        X = _device_f64(X, "X", 2, 3)
        m = X.shape[0]
        U = _device_out(U, (m, self.d), X)
        rho = _device_out(rho, (m,), X)
        _torch().cuda.current_stream(X.device).synchronize()
        _check(self.h, _lib.ibl_interpolate_points(self.h, m, X.data_ptr(), U.data_ptr(), rho.data_ptr()))
        return U, rho

    def ibl_spread_points(self, X, V, ds, out=None):
        """sum_l V_l ds_l D(x - X_l) on the grid (Eq. 15): [d, nz, ny, nx] float64.

        X [m, 3], V [m, d], ds [m]: CUDA float64 tensors.
        """
        X = _device_f64(X, "X", 2, 3)
        m = X.shape[0]
        V = _device_f64(V, "V", 2, self.d)
        ds = _device_f64(ds, "ds", 1, None)
        if V.shape[0] != m or ds.shape[0] != m:
            raise ValueError("X, V and ds need the same number of points")
        out = _device_out(out, (self.d,) + self.shape, X)
        _torch().cuda.current_stream(X.device).synchronize()
        _check(self.h, _lib.ibl_spread_points(self.h, m, X.data_ptr(), V.data_ptr(), ds.data_ptr(),
                                              out.data_ptr()))
        return out

    def ibl_solver_stats(self, allow=()):
        it, res, ref = C.c_int32(), C.c_double(), C.c_int64()
        _check(self.h, _lib.ibl_solver_stats(self.h, C.byref(it), C.byref(res), C.byref(ref)), allow)
        return it.value, res.value, ref.value

    def ibl_solver_config(self, refresh_every=384, tol=0.0, extrapolate=True):
        """extrapolate: 2 (3 w_n-1 - 3 w_n-2 + w_n-3), True or 1 (2 w_n-1 - w_n-2),
        False or 0 (w_n-1), None or -1 (zero)."""
        if extrapolate is None:
            mode = -1
        elif isinstance(extrapolate, bool):
            mode = 1 if extrapolate else 0
        else:
            mode = int(extrapolate)
        _check(self.h, _lib.ibl_solver_config(self.h, int(refresh_every), float(tol), mode))

    def ibl_solver_preconditioner(self, kind=-1, resident_rows=-1):
        """kind: -1 automatic, 0 dense per-body inverse, 1 separable factors;
        resident_rows: -1 when they fit, 0 always read from L2/HBM."""
        _check(self.h, _lib.ibl_solver_preconditioner(self.h, int(kind), int(resident_rows)))

    def ibl_solver_trace(self, allow=()):
        out = np.zeros(256, dtype=np.int64)
        n = C.c_int32()
        _check(self.h, _lib.ibl_solver_trace(self.h, out.ctypes.data_as(_I64), 256, C.byref(n)), allow)
        return out[:n.value]

    def ibl_profile(self, enable):
        """0 off, 1 (or True) collide / IB chain totals, 2 also per-phase events."""
        _check(self.h, _lib.ibl_profile(self.h, int(enable)))

    def ibl_profile_read(self):
        a, b, n = C.c_double(), C.c_double(), C.c_int64()
        _check(self.h, _lib.ibl_profile_read(self.h, C.byref(a), C.byref(b), C.byref(n)))
        return a.value, b.value, n.value

    def ibl_launch_count(self):
        n = C.c_int64()
        _check(self.h, _lib.ibl_launch_count(self.h, C.byref(n)))
        return n.value

    def ibl_stream(self):
        s = _P()
        _check(self.h, _lib.ibl_stream(self.h, C.byref(s)))
        return s.value


def ibl_create(grid: dict, tau: float, lattice: int) -> Context:
    return Context(grid, tau, lattice)


def from_workload(cfg: dict, init: bool = True) -> Context:
    """Create a context for a workload dict of ``workloads`` and initialise it."""
    ctx = Context(cfg["grid"], cfg["tau"], cfg["lattice"])
    for b in cfg.get("bodies", []):
        ctx.add_body(b)
    if "reference" in cfg:
        r = cfg["reference"]
        ctx.ibl_set_reference(r["U_ref"], r["L"], r.get("rho_ref", 1.0))
    if init:
        if "u_field" in cfg:
            ctx.ibl_init_fluid(None, cfg["u_field"][:ctx.d])
        else:
            ctx.ibl_init_fluid(None, np.asarray(cfg.get("u0", (0.0, 0.0, 0.0)))[:ctx.d])
    return ctx


class Server:
    """Continuous-batching server of clap-and-fling runs (ibl_server_* calls)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, chunk_steps: int = 50, tune: int = 1):
        cfg = ibl_server_config(int(hbm_budget_bytes), int(max_active), int(chunk_steps), int(tune))
        h = _P()
        st = _lib.ibl_server_create(C.byref(cfg), C.byref(h))
        if st != IBL_OK:
            raise IblError(st, "ibl_server_create failed")
        self.h = h

    def ibl_server_submit(self, nx, ny, nz, chord, Re, period, J, precision="fp32", steps=1000, faces=0):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        req = ibl_run_request(int(nx), int(ny), int(nz), float(chord), float(Re), float(period), float(J),
                              prec, int(faces), int(steps))
        rid = C.c_int64()
        st = _lib.ibl_server_submit(self.h, C.byref(req), C.byref(rid))
        if st != IBL_OK:
            raise IblError(st, "ibl_server_submit rejected the request")
        return rid.value

    def ibl_server_poll(self, run_id):
        r = ibl_run_result()
        st = _lib.ibl_server_poll(self.h, int(run_id), C.byref(r))
        if st != IBL_OK:
            raise IblError(st, "unknown run id")
        return {"status": r.status, "done": bool(r.done), "steps_done": r.steps_done,
                "submit_s": r.submit_s, "start_s": r.start_s, "finish_s": r.finish_s,
                "CL_max": list(r.CL_max), "CL_mean": list(r.CL_mean), "CT_max": list(r.CT_max),
                "CT_mean": list(r.CT_mean), "CL_last": list(r.CL_last), "CT_last": list(r.CT_last),
                "solve_blocks": r.solve_blocks, "overlap": r.overlap, "collide_shape": (r.collide_bx, r.collide_by),
                "collide_pairs": r.collide_pairs, "tuned": bool(r.tuned)}

    def ibl_server_cancel(self, run_id):
        st = _lib.ibl_server_cancel(self.h, int(run_id))
        if st != IBL_OK:
            raise IblError(st, "unknown run id")

    def ibl_server_wait_all(self, timeout_s=3600.0):
        st = _lib.ibl_server_wait_all(self.h, float(timeout_s))
        if st != IBL_OK:
            raise IblError(st, "ibl_server_wait_all timed out")

    def ibl_server_stats(self):
        q, a, f, b = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        _lib.ibl_server_stats(self.h, C.byref(q), C.byref(a), C.byref(f), C.byref(b))
        return {"queued": q.value, "active": a.value, "finished": f.value, "hbm_in_use": b.value}

    def ibl_server_load(self):
        v = [C.c_double() for _ in range(5)]
        _check(None, _lib.ibl_server_load(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("wall_s", "busy_s", "enqueue_s", "build_s", "retire_s"), (x.value for x in v)))

    def close(self):
        if getattr(self, "h", None):
            _lib.ibl_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
