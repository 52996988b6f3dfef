"""FP64 CPU oracle of one FishGym IB-LBM time step -- TEST INFRASTRUCTURE.

A ctypes wrapper around ``lbm_oracle.c``.  The oracle is the plain, slow,
double-precision definition of what the CUDA path computes (arXiv 2206.01683
Sec. III-B, Eq. 3, with the readings stated in the C file).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the product library never does.
"""
import ctypes
import os

import numpy as np

from . import build as _build

PERIODIC, VELOCITY, OUTFLOW, FREESLIP = 0, 1, 2, 3

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        P = ctypes.POINTER
        L.orc_create.restype = vp
        L.orc_create.argtypes = [i, i, i, d, P(i), P(d), d]
        L.orc_destroy.argtypes = [vp]
        L.orc_lattice.argtypes = [P(i), P(d)]
        L.orc_init_fields.argtypes = [vp, P(d), P(d)]
        L.orc_set_markers.restype = i
        L.orc_set_markers.argtypes = [vp, i, P(d), P(d), P(d), P(i), i, P(d)]
        L.orc_step.restype = i
        L.orc_step.argtypes = [vp, P(d)]
        for name in ("orc_get_populations", "orc_set_populations", "orc_get_force_torque",
                     "orc_get_marker_force", "orc_get_fib"):
            getattr(L, name).argtypes = [vp, P(d)]
        L.orc_get_fields.argtypes = [vp, P(d), P(d)]
        L.orc_get_post_stream_moments.argtypes = [vp, P(d), P(d), P(d)]
        L.orc_mass.restype = d
        L.orc_mass.argtypes = [vp]
        L.orc_mass_deviation.restype = d
        L.orc_mass_deviation.argtypes = [vp]
        L.orc_phi.restype = d
        L.orc_phi.argtypes = [d]
        L.orc_interp.restype = i
        L.orc_interp.argtypes = [vp, P(d), i, P(d), P(d)]
        L.orc_spread.restype = i
        L.orc_spread.argtypes = [vp, i, P(d), P(d), P(d)]
        L.orc_collide_cell.argtypes = [P(d), P(d), P(d), P(d), d, i, P(d)]
        L.orc_set_eq_order.restype = i
        L.orc_set_eq_order.argtypes = [vp, i]
        L.orc_frame_accel.argtypes = [P(d), d, d, d, P(d)]
        L.orc_set_threads.restype = i
        L.orc_set_threads.argtypes = [i]
        L.orc_set_ib_iters.restype = i
        L.orc_set_ib_iters.argtypes = [vp, i]
        L.orc_set_body_force.argtypes = [vp, P(d)]
        L.orc_region_momentum.argtypes = [vp, P(d), d, P(d), P(d)]
        L.orc_set_segment_refs.restype = i
        L.orc_set_segment_refs.argtypes = [vp, i, P(d)]
        L.orc_set_slip.restype = i
        L.orc_set_slip.argtypes = [vp, i, i, P(d)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n):
    """OpenMP threads of the oracle's loops (0: keep); returns the count in use."""
    return lib().orc_set_threads(int(n))


def lattice():
    """Velocities (27, 3) int and weights (27,) in the oracle's own order."""
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().orc_lattice(_ip(c), _dp(w))
    return c, w


def phi(r):
    return lib().orc_phi(float(r))


def frame_accel(frame, x):
    out = np.zeros(3)
    fr = _f64(frame, (12,))
    lib().orc_frame_accel(_dp(fr), float(x[0]), float(x[1]), float(x[2]), _dp(out))
    return out


def collide_cell(fs, a0, fib, omega, tau, eq_order=2):
    out = np.zeros(27)
    fs, a0, fib, om = _f64(fs, (27,)), _f64(a0, (3,)), _f64(fib, (3,)), _f64(omega, (3,))
    lib().orc_collide_cell(_dp(fs), _dp(a0), _dp(fib), _dp(om), float(tau), int(eq_order), _dp(out))
    return out


def make_frame(acc=(0, 0, 0), omega=(0, 0, 0), domega=(0, 0, 0), origin=(0, 0, 0)):
    return np.array(list(acc) + list(omega) + list(domega) + list(origin), dtype=np.float64)


class Oracle:
    """One FP64 domain.  Fields use cell index x + nx*(y + ny*z)."""

    def __init__(self, shape, tau, faces=(PERIODIC,) * 6, u_in=(0.0, 0.0, 0.0), rho_out=1.0, ib_iters=1,
                 slip=False, eq_order=2):
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        self.ncell = nx * ny * nz
        faces = np.ascontiguousarray(faces, dtype=np.int32)
        uin = _f64(u_in, (3,))
        self._h = lib().orc_create(nx, ny, nz, float(tau), _ip(faces), _dp(uin), float(rho_out))
        if not self._h:
            raise ValueError("oracle: invalid domain description")
        if lib().orc_set_ib_iters(self._h, int(ib_iters)) != 0:
            lib().orc_destroy(self._h)
            self._h = None
            raise ValueError("oracle: ib_iters must be in [1, 64]")
        self.slip = bool(slip)
        if lib().orc_set_eq_order(self._h, int(eq_order)) != 0:
            raise ValueError("oracle: eq_order must be 2 or 3")
        self.tau = tau
        self.faces = tuple(int(f) for f in faces)
        self.nm = 0
        self.nseg = 1
        self.init_fields()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init_fields(self, rho=None, u=None):
        r = _f64(rho, (self.ncell,)) if rho is not None else None
        v = _f64(u, (self.ncell, 3)) if u is not None else None
        lib().orc_init_fields(self._h, _dp(r) if r is not None else None,
                              _dp(v) if v is not None else None)

    def set_markers(self, X, U, dV, seg=None, nseg=1, ref=(0.0, 0.0, 0.0), normals=None):
        """normals: unit surface normals (n, 3), required with slip=True."""
        X = _f64(X).reshape(-1, 3)
        n = X.shape[0]
        U = _f64(U, (n, 3))
        dV = _f64(dV, (n,))
        ref = _f64(ref, (3,))
        s = np.ascontiguousarray(seg, dtype=np.int32) if seg is not None else None
        rc = lib().orc_set_markers(self._h, n, _dp(X), _dp(U), _dp(dV),
                                   _ip(s) if s is not None else None, int(nseg), _dp(ref))
        if rc != 0:
            raise ValueError("oracle: invalid markers")
        self.nm = n
        self.nseg = max(int(nseg), 1)
        if self.slip:
            if normals is None:
                raise ValueError("oracle: slip forcing needs marker normals")
            N = _f64(normals, (n, 3))
            if lib().orc_set_slip(self._h, 1, n, _dp(N)) != 0:
                raise ValueError("oracle: invalid normals")

    def region_momentum(self, center, radius):
        """(P[3], L[3], sum alpha) of the fluid inside the sphere."""
        out = np.zeros(6)
        a = ctypes.c_double()
        c = _f64(center, (3,))
        lib().orc_region_momentum(self._h, _dp(c), float(radius), _dp(out), ctypes.byref(a))
        return out[:3].copy(), out[3:].copy(), a.value

    def set_body_force(self, G):
        """External body-force density G (ncell, 3), cell order x fastest,
        entering the Guo forcing as the IB force does (pins only); None
        removes it."""
        if G is None:
            lib().orc_set_body_force(self._h, None)
            return
        g = _f64(G).reshape(self.ncell, 3)
        if lib().orc_set_body_force(self._h, _dp(g)) != 0:
            raise MemoryError("oracle: body force")

    def set_segment_refs(self, refs):
        """Torque reference point per segment row (nseg, 3); None: common ref."""
        if refs is None:
            lib().orc_set_segment_refs(self._h, 0, None)
            return
        r = _f64(refs).reshape(-1, 3)
        if lib().orc_set_segment_refs(self._h, r.shape[0], _dp(r)) != 0:
            raise ValueError("oracle: one reference point per segment")

    def step(self, frame=None, n=1):
        fr = make_frame() if frame is None else _f64(frame, (12,))
        for _ in range(n):
            if lib().orc_step(self._h, _dp(fr)) != 0:
                raise ValueError("oracle: step refused (slip forcing without normals)")

    def populations(self):
        f = np.zeros((self.ncell, 27))
        lib().orc_get_populations(self._h, _dp(f))
        return f

    def set_populations(self, f):
        f = _f64(f, (self.ncell, 27))
        lib().orc_set_populations(self._h, _dp(f))

    def fields(self):
        rho = np.zeros(self.ncell)
        u = np.zeros((self.ncell, 3))
        lib().orc_get_fields(self._h, _dp(rho), _dp(u))
        return rho, u

    def force_torque(self):
        out = np.zeros((self.nseg + 1, 6))
        lib().orc_get_force_torque(self._h, _dp(out))
        return out

    def marker_force(self):
        F = np.zeros((max(self.nm, 1), 3))
        lib().orc_get_marker_force(self._h, _dp(F))
        return F[: self.nm]

    def fib(self):
        g = np.zeros((self.ncell, 3))
        lib().orc_get_fib(self._h, _dp(g))
        return g

    def post_stream_moments(self):
        rho = np.zeros(self.ncell)
        j = np.zeros((self.ncell, 3))
        Pi = np.zeros((self.ncell, 6))
        lib().orc_get_post_stream_moments(self._h, _dp(rho), _dp(j), _dp(Pi))
        return rho, j, Pi

    def mass(self):
        return lib().orc_mass(self._h)

    def mass_deviation(self):
        """sum over cells of (rho - 1) after the last step."""
        return lib().orc_mass_deviation(self._h)

    def interp(self, g, X):
        g = _f64(g, (self.ncell, 3))
        X = _f64(X).reshape(-1, 3)
        out = np.zeros_like(X)
        if lib().orc_interp(self._h, _dp(g), X.shape[0], _dp(X), _dp(out)) != 0:
            raise ValueError("oracle: invalid markers")
        return out

    def spread(self, X, F):
        X = _f64(X).reshape(-1, 3)
        F = _f64(F, X.shape)
        g = np.zeros((self.ncell, 3))
        if lib().orc_spread(self._h, X.shape[0], _dp(X), _dp(F), _dp(g)) != 0:
            raise ValueError("oracle: invalid markers")
        return g
