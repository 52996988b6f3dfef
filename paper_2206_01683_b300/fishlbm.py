"""Thin Python binding of the C ABI in include/fishlbm.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``libfishlbm.so`` next to this file.  If that library is missing or cannot be
loaded the import of the binding fails loudly; there is no fallback path.

The ``fg_*`` functions mirror the C names one to one.  ``Domain`` is a small
convenience wrapper over them that accepts numpy arrays (host) or torch CUDA
tensors (device pointers) for marker data.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FISHLBM_LIB selects another build of the library (the debug build in tests)
LIB_PATH = os.environ.get("FISHLBM_LIB") or os.path.join(HERE, "libfishlbm.so")

FG_OK, FG_ERR_INVALID, FG_ERR_CUDA, FG_ERR_OOM = 0, -1, -2, -3
FG_ERR_TIMEOUT, FG_ERR_NUMERIC, FG_ERR_STATE = -4, -5, -6
FG_F32, FG_F16, FG_BF16 = 0, 1, 2
FG_PERIODIC, FG_VELOCITY, FG_OUTFLOW, FG_FREESLIP = 0, 1, 2, 3
FG_K_IB, FG_K_STREAM_COLLIDE, FG_K_REDUCE, FG_K_COUNT = 0, 1, 2, 3
FG_KERNEL_AUTO, FG_KERNEL_PLAIN, FG_KERNEL_STAGED, FG_KERNEL_STAGED512 = 0, 1, 2, 3
FG_KERNEL_FUSED, FG_KERNEL_OVERLAP = 4, 5
FG_K1_PLAIN, FG_K1_STAGED256, FG_K1_STAGED512, FG_K1_FUSED, FG_K1_OVERLAP, FG_K1_NVARIANTS = 0, 1, 2, 3, 4, 5
K1_NAMES = {0: "plain", 1: "staged256", 2: "staged512", 3: "fused", 4: "overlap"}
VARIANT = {"auto": FG_KERNEL_AUTO, "plain": FG_KERNEL_PLAIN, "staged": FG_KERNEL_STAGED,
           "staged512": FG_KERNEL_STAGED512, "fused": FG_KERNEL_FUSED, "overlap": FG_KERNEL_OVERLAP}
STORAGE = {"f32": FG_F32, "f16": FG_F16, "bf16": FG_BF16}
FG_LAYOUT_PULL, FG_LAYOUT_AA = 0, 1
LAYOUT = {"pull": FG_LAYOUT_PULL, "aa": FG_LAYOUT_AA}


class FgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("fishlbm status %d: %s" % (status, msg))
        self.status = status


class fg_env_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("tau", ctypes.c_double), ("face", ctypes.c_int * 6),
                ("u_in", ctypes.c_double * 3), ("rho0", ctypes.c_double),
                ("u0", ctypes.c_double * 3)]


class fg_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("layout", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("ib_iters", ctypes.c_int),
                ("record_history", ctypes.c_int), ("kernel_variant", ctypes.c_int),
                ("autotune", ctypes.c_int), ("ib_slip", ctypes.c_int), ("eq_order", ctypes.c_int),
                ("use_graphs", ctypes.c_int)]


class fg_frame(ctypes.Structure):
    _fields_ = [("acc", ctypes.c_double * 3), ("omega", ctypes.c_double * 3),
                ("domega", ctypes.c_double * 3), ("origin", ctypes.c_double * 3)]


# name -> (restype, argtypes); the exported symbols of include/fishlbm.h
_V, _I, _D, _LL, _ULL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_ulonglong
_P = ctypes.POINTER
SIGNATURES = {
    "fg_create_domain": (_I, [_P(fg_env_desc), _I, _P(fg_options), _V, _P(_V)]),
    "fg_set_markers": (_I, [_V, _I, _I, _V, _V, _V, _V, _I, _P(_D), _I]),
    "fg_set_marker_normals": (_I, [_V, _I, _I, _V, _I]),
    "fg_set_segment_refs": (_I, [_V, _I, _I, _P(_D)]),
    "fg_set_markers_all": (_I, [_V, _I, _V, _V, _I]),
    "fg_selftest_waits": (_I, [ctypes.c_uint, _P(_I)]),
    "fg_debug_flags": (_I, [_P(ctypes.c_uint), _I]),
    "fg_region_momentum": (_I, [_V, _I, _P(_D), _D, _P(_D), _P(_D)]),
    "fg_attach_sphere": (_I, [_V, _I, _D, _P(_D), _D, _P(_D), _I, _P(_D), _P(ctypes.c_float), _I]),
    "fg_sphere_state": (_I, [_V, _I, _P(_D)]),
    "fg_detach_sphere": (_I, [_V, _I]),
    "fg_step": (_I, [_V, _I, _P(fg_frame)]),
    "fg_get_body_force_torque": (_I, [_V, _I, _P(_D)]),
    "fg_step_io": (_I, [_V, _V, _V, _I, _P(fg_frame), _V]),
    "fg_step_markers": (_I, [_V, _V, _V, _I, _P(fg_frame)]),
    "fg_destroy": (None, [_V]),
    "fg_last_error": (ctypes.c_char_p, []),
    "fg_lattice": (_I, [_P(_I), _P(_D)]),
    "fg_init_fields": (_I, [_V, _I, _P(_D), _P(_D)]),
    "fg_get_fields": (_I, [_V, _I, _P(_D), _P(_D)]),
    "fg_get_populations": (_I, [_V, _I, _P(_D)]),
    "fg_set_populations": (_I, [_V, _I, _P(_D)]),
    "fg_get_marker_force": (_I, [_V, _I, _P(ctypes.c_float)]),
    "fg_watch_mass": (_I, [_V, _I, _D]),
    "fg_set_alloc_cap": (_I, [_ULL]),
    "fg_get_mass": (_I, [_V, _I, _P(_D)]),
    "fg_get_history": (_I, [_V, _I, _P(_D), _I, _P(_I)]),
    "fg_state_bytes": (_I, [_V, _I, _P(_ULL)]),
    "fg_save_state": (_I, [_V, _I, _V]),
    "fg_load_state": (_I, [_V, _I, _V]),
    "fg_get_status": (_I, [_V, _P(_I)]),
    "fg_step_count": (_I, [_V, _P(_LL)]),
    "fg_profile": (_I, [_V, _I]),
    "fg_profile_read": (_I, [_V, _P(_D), _P(_LL)]),
    "fg_stream_collide_bytes": (_I, [_V, _P(_ULL)]),
    "fg_autotune": (_I, [_V, _P(_I), _P(_D)]),
    "fg_copy_state": (_I, [_V, _I, _V, _I]),
    "fg_step_state": (_I, [_V, _V, _V, _P(fg_frame)]),
    "fg_adjoint_reset": (_I, [_V]),
    "fg_adjoint_step": (_I, [_V, _P(fg_frame), _P(_D), _V, _V]),
    "fg_adjoint_step_state": (_I, [_V, _V, _P(fg_frame), _P(_D), _V, _V]),
    "fg_get_adjoint": (_I, [_V, _P(_D)]),
    "fg_set_adjoint": (_I, [_V, _P(_D)]),
    "fg_stream_collide_variant": (_I, [_V, _P(_I)]),
    "fg_body_force_noalloc": (_I, [_P(fg_env_desc), _V, _V, _V, _V, _V, _I, _I, _P(_D),
                                   _P(fg_frame), _V, _V]),
}
FG_NOALLOC_MAX_MARKERS = 65536

_lib = None


def lib():
    """Load libfishlbm.so (raises if it is absent: build it with build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfishlbm.so is not built (run paper_2206_01683_b300/build.py); "
                              "there is no fallback implementation")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != FG_OK:
        raise FgError(status, lib().fg_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(_P(_D))


# ----------------------------------------------------- C-named functions

def fg_create_domain(envs, opt=None, stream=None):
    arr = (fg_env_desc * len(envs))(*envs)
    out = _V()
    _check(lib().fg_create_domain(arr, len(envs), ctypes.byref(opt) if opt is not None else None,
                                  _V(stream or 0), ctypes.byref(out)))
    return out


def fg_set_markers(d, env, n, X, U, dV, seg, n_seg, ref, device_ptrs):
    refa = (_D * 3)(*ref) if ref is not None else None
    _check(lib().fg_set_markers(d, env, n, X, U, dV, seg, n_seg, refa, device_ptrs))


def fg_step(d, n_steps=1, frames=None):
    fr = None
    if frames is not None:
        fr = (fg_frame * len(frames))(*frames)
    _check(lib().fg_step(d, n_steps, fr))


def fg_get_body_force_torque(d, env, n_seg):
    out = np.zeros((n_seg + 1, 6))
    _check(lib().fg_get_body_force_torque(d, env, _dp(out)))
    return out


def fg_body_force_noalloc(env, g, X, U, dV, seg, n, n_seg, ref, frame, out, stream=None):
    """Allocation-free body force from a caller-owned FP32 state (device
    pointers as ints or None); see include/fishlbm.h."""
    refa = (_D * 3)(*ref) if ref is not None else None
    _check(lib().fg_body_force_noalloc(ctypes.byref(env), _V(g), _V(X), _V(U), _V(dV),
                                       _V(seg) if seg else None, n, n_seg, refa,
                                       ctypes.byref(frame) if frame is not None else None,
                                       _V(out), _V(stream or 0)))


def fg_destroy(d):
    if d:
        lib().fg_destroy(d)


def fg_lattice():
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    _check(lib().fg_lattice(c.ctypes.data_as(_P(_I)), _dp(w)))
    return c, w


def make_frame(acc=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), domega=(0.0, 0.0, 0.0),
               origin=(0.0, 0.0, 0.0)):
    f = fg_frame()
    for a in range(3):
        f.acc[a], f.omega[a], f.domega[a], f.origin[a] = acc[a], omega[a], domega[a], origin[a]
    return f


def frame_from_array(v):
    """fg_frame from the 12 numbers (p'', omega, domega, origin)."""
    v = [float(x) for x in v]
    return make_frame(v[0:3], v[3:6], v[6:9], v[9:12])


def env_desc(shape, tau, faces=(FG_PERIODIC,) * 6, u_in=(0.0, 0.0, 0.0), rho0=1.0,
             u0=(0.0, 0.0, 0.0)):
    e = fg_env_desc()
    e.nx, e.ny, e.nz = shape
    e.tau = tau
    for k in range(6):
        e.face[k] = faces[k]
    for a in range(3):
        e.u_in[a] = u_in[a]
        e.u0[a] = u0[a]
    e.rho0 = rho0
    return e


def _check_shape(name, a, shape):
    """The C ABI takes bare pointers: a wrong shape would make it read past
    the caller's array, so the binding refuses it."""
    if a is not None and tuple(a.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, not %s" % (name, tuple(shape), tuple(a.shape)))


def _ptr_and_keep(a, dtype):
    """(pointer, is_device, keepalive) for a numpy array or a torch tensor
    (a CUDA tensor is passed as a device pointer, a CPU tensor, e.g. pinned,
    as a host pointer; tensors must be contiguous and of the right dtype)."""
    if a is None:
        return None, None, None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or a.element_size() != np.dtype(dtype).itemsize:
            raise ValueError("marker tensors must be contiguous float32 / int32")
        return _V(a.data_ptr()), bool(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(_V), False, arr


def set_alloc_cap(nbytes):
    """Largest single device allocation the library may make (0: no limit);
    larger requests fail with FG_ERR_OOM (fg_set_alloc_cap)."""
    _check(lib().fg_set_alloc_cap(int(nbytes)))


def debug_flags(reset=True):
    """Index-check flags of the debug build (see fg_debug_flags)."""
    f = ctypes.c_uint()
    _check(lib().fg_debug_flags(ctypes.byref(f), 1 if reset else 0))
    return f.value


def selftest_waits(limit=4096):
    """Run the bounded device waits on conditions that never come; returns
    (mbarrier wait gave up, grid barrier gave up, status timeout bit, work
    queue wait gave up and set the abort word)."""
    out = (_I * 4)()
    _check(lib().fg_selftest_waits(int(limit), out))
    return bool(out[0]), bool(out[1]), bool(out[2]), bool(out[3])


class Domain:
    """Owns one fg_domain (one or many environments)."""

    def __init__(self, envs, storage="f32", record_history=0, stream=None, variant="auto",
                 graphs=True, autotune=False, ib_iters=1, deterministic=False, slip=False, eq_order=2,
                 layout="pull"):
        self.envs = list(envs)
        opt = fg_options()
        opt.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        opt.layout = LAYOUT[layout] if isinstance(layout, str) else int(layout)
        opt.deterministic = 1 if deterministic else 0
        opt.ib_iters = int(ib_iters)
        opt.record_history = int(record_history)
        opt.kernel_variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
        opt.ib_slip = 1 if slip else 0
        opt.eq_order = int(eq_order)
        opt.use_graphs = 1 if graphs else 0
        opt.autotune = 1 if autotune else 0
        self.storage = opt.storage
        self.h = fg_create_domain(self.envs, opt, stream)
        self.nseg = [1] * len(self.envs)
        self.nmark = [0] * len(self.envs)

    def close(self):
        if getattr(self, "h", None):
            fg_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def ncell(self, env=0):
        e = self.envs[env]
        return e.nx * e.ny * e.nz

    def set_markers(self, X, U, dV=None, seg=None, n_seg=1, ref=None, env=0):
        n = int(X.shape[0])
        _check_shape("X", X, (n, 3))
        _check_shape("U", U, (n, 3))
        _check_shape("dV", dV, (n,))
        _check_shape("seg", seg, (n,))
        pX, devX, kX = _ptr_and_keep(X, np.float32)
        pU, devU, kU = _ptr_and_keep(U, np.float32)
        pd, devd, kd = _ptr_and_keep(dV, np.float32)
        ps, devs, ks = _ptr_and_keep(seg, np.int32)
        dev = bool(devX)
        for flag in (devU, devd, devs):
            if flag is not None and flag != dev:
                raise ValueError("marker arrays must all be host or all be device")
        fg_set_markers(self.h, env, n, pX, pU, pd, ps, int(n_seg), ref, 1 if dev else 0)
        self._keep = (kX, kU, kd, ks)
        self.nseg[env] = int(n_seg)
        self.nmark[env] = n

    def region_momentum(self, center, radius, env=0):
        """(P[3], L[3], sum alpha) of the fluid inside a sphere."""
        c = np.ascontiguousarray(center, dtype=np.float64).reshape(3)
        out = np.zeros(6)
        a = _D()
        _check(lib().fg_region_momentum(self.h, env, _dp(c), float(radius), _dp(out), ctypes.byref(a)))
        return out[:3].copy(), out[3:].copy(), a.value

    def set_markers_all(self, X, U):
        """Positions and velocities (n_total, 3) of all environments' markers,
        environment after environment (numpy, torch CPU or CUDA tensors)."""
        n = int(X.shape[0])
        _check_shape("X", X, (n, 3))
        _check_shape("U", U, (n, 3))
        pX, devX, kX = _ptr_and_keep(X, np.float32)
        pU, devU, kU = _ptr_and_keep(U, np.float32)
        if devX != devU:
            raise ValueError("X and U must both be host or both be device arrays")
        _check(lib().fg_set_markers_all(self.h, n, pX, pU, 1 if devX else 0))
        self._keep_all = (kX, kU)

    def attach_sphere(self, radius, center, density_ratio, gravity, dirs, dV, env=0, box_reaction=True):
        """Advance a free rigid sphere of the given radius on the device,
        two-way coupled every step (fg_attach_sphere): markers on the shell
        along the unit directions dirs (n, 3) with weights dV (n,)."""
        c = np.ascontiguousarray(center, dtype=np.float64).reshape(3)
        g = np.ascontiguousarray(gravity, dtype=np.float64).reshape(3)
        d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(dV, dtype=np.float32).reshape(-1)
        if w.shape[0] != d.shape[0]:
            raise ValueError("dirs and dV must have the same length")
        _check(lib().fg_attach_sphere(self.h, env, float(radius), _dp(c), float(density_ratio), _dp(g),
                                      d.shape[0], _dp(d), w.ctypes.data_as(_P(ctypes.c_float)),
                                      1 if box_reaction else 0))
        self.nmark[env] = d.shape[0]

    def sphere_state(self, env=0):
        """(centre, velocity, spin) of the sphere attached to env."""
        out = np.zeros(9)
        _check(lib().fg_sphere_state(self.h, env, _dp(out)))
        return out[0:3].copy(), out[3:6].copy(), out[6:9].copy()

    def detach_sphere(self, env=0):
        _check(lib().fg_detach_sphere(self.h, env))

    def set_segment_refs(self, refs, env=0):
        """Torque point per segment row (n_seg, 3); None: the common point."""
        if refs is None:
            _check(lib().fg_set_segment_refs(self.h, env, 0, None))
            return
        r = np.ascontiguousarray(refs, dtype=np.float64).reshape(-1, 3)
        _check(lib().fg_set_segment_refs(self.h, env, r.shape[0], _dp(r)))

    def set_marker_normals(self, N, env=0):
        """Unit normals (n, 3) of env's current markers (slip forcing);
        numpy, torch CPU or CUDA tensors."""
        n = int(N.shape[0])
        _check_shape("N", N, (n, 3))
        p, dev, keep = _ptr_and_keep(N, np.float32)
        _check(lib().fg_set_marker_normals(self.h, env, n, p, 1 if dev else 0))
        self._keep_n = keep

    def step(self, n=1, frames=None):
        if frames is not None and not isinstance(frames, (list, tuple)):
            frames = [frames]
        if frames is not None:
            frames = [f if isinstance(f, fg_frame) else frame_from_array(f) for f in frames]
        fg_step(self.h, n, frames)

    def get_body_force_torque(self, env=0):
        return fg_get_body_force_torque(self.h, env, self.nseg[env])

    def step_markers(self, X=None, U=None, frames=None):
        """New markers and one step in one asynchronous call
        (fg_step_markers): positions and velocities of all environments'
        markers as for step_io (None keeps them), then one step."""
        pX, pU, dev, fr = self._io_args(X, U, frames)
        _check(lib().fg_step_markers(self.h, pX, pU, 1 if dev else 0, fr))

    def _io_args(self, X, U, frames):
        """Marker pointers (kept alive until the next call), device flag and
        frames argument of fg_step_io / fg_step_markers."""
        if (X is None) != (U is None):
            raise ValueError("X and U must both be given or both be None")
        pX = pU = None
        dev = False
        if X is not None:
            n = sum(self.nmark)
            if tuple(X.shape) != (n, 3) or tuple(U.shape) != (n, 3):
                raise ValueError("X and U must be (%d, 3): every environment's markers, in order" % n)
            pX, devX, kX = _ptr_and_keep(X, np.float32)
            pU, devU, kU = _ptr_and_keep(U, np.float32)
            if devX != devU:
                raise ValueError("X and U must both be host or both be device arrays")
            dev = bool(devX)
            self._keep_io = (kX, kU)
        fr = None
        if frames is not None:
            if not isinstance(frames, (list, tuple)):
                frames = [frames]
            if len(frames) == 1 and isinstance(frames[0], fg_frame):
                fr = ctypes.byref(frames[0])   # the per-step case, without building an array
            else:
                fr = (fg_frame * len(frames))(*[f if isinstance(f, fg_frame) else frame_from_array(f)
                                                 for f in frames])
        return pX, pU, dev, fr

    def step_io(self, X=None, U=None, frames=None):
        """One coupled step in one call (fg_step_io): new positions and
        velocities of all environments' markers (numpy, torch CPU/pinned or
        CUDA tensors, environment after environment; None keeps them), one
        step, and the force/torque rows read back.  Returns the (n_seg + 1, 6)
        rows of a single environment, else a list of them."""
        pX, pU, dev, fr = self._io_args(X, U, frames)
        rows = [self.nseg[e] + 1 for e in range(len(self.nseg))]
        total = sum(rows)
        if getattr(self, "_io_out", None) is None or self._io_out.shape[0] != total:
            self._io_out = np.zeros((total, 6))          # landing buffer, its address cached
            self._io_addr = self._io_out.ctypes.data
        _check(lib().fg_step_io(self.h, pX, pU, 1 if dev else 0, fr, self._io_addr))
        out = self._io_out.copy()
        if len(rows) == 1:
            return out
        return np.split(out, np.cumsum(rows)[:-1])

    def init_fields(self, rho=None, u=None, env=0):
        r = np.ascontiguousarray(rho, dtype=np.float64) if rho is not None else None
        v = np.ascontiguousarray(u, dtype=np.float64) if u is not None else None
        _check(lib().fg_init_fields(self.h, env, _dp(r) if r is not None else None,
                                    _dp(v) if v is not None else None))

    def fields(self, env=0):
        n = self.ncell(env)
        rho = np.zeros(n)
        u = np.zeros((n, 3))
        _check(lib().fg_get_fields(self.h, env, _dp(rho), _dp(u)))
        return rho, u

    def populations(self, env=0):
        f = np.zeros((self.ncell(env), 27))
        _check(lib().fg_get_populations(self.h, env, _dp(f)))
        return f

    def set_populations(self, f, env=0):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.ncell(env), 27)
        _check(lib().fg_set_populations(self.h, env, _dp(f)))

    def marker_force(self, env=0):
        F = np.zeros((max(self.nmark[env], 1), 3), dtype=np.float32)
        _check(lib().fg_get_marker_force(self.h, env, F.ctypes.data_as(_P(ctypes.c_float))))
        return F[: self.nmark[env]]

    def watch_mass(self, rel_tol, env=0):
        """Mass-drift watchdog (fg_watch_mass): the current mass becomes the
        reference; rel_tol <= 0 switches it off."""
        _check(lib().fg_watch_mass(self.h, env, float(rel_tol)))

    def mass(self, env=0):
        m = _D()
        _check(lib().fg_get_mass(self.h, env, ctypes.byref(m)))
        return m.value

    def history(self, max_steps, env=0):
        w = 6 * (self.nseg[env] + 1) + 1
        out = np.zeros((max_steps, w))
        n = _I()
        _check(lib().fg_get_history(self.h, env, _dp(out), max_steps, ctypes.byref(n)))
        return out[: n.value]

    def state_bytes(self, env=0):
        b = _ULL()
        _check(lib().fg_state_bytes(self.h, env, ctypes.byref(b)))
        return b.value

    def save_state(self, env=0):
        buf = np.zeros(self.state_bytes(env), dtype=np.uint8)
        _check(lib().fg_save_state(self.h, env, buf.ctypes.data_as(_V)))
        return buf

    def load_state(self, buf, env=0):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().fg_load_state(self.h, env, buf.ctypes.data_as(_V)))

    def status(self):
        s = _I()
        _check(lib().fg_get_status(self.h, ctypes.byref(s)))
        return s.value

    def step_count(self):
        s = _LL()
        _check(lib().fg_step_count(self.h, ctypes.byref(s)))
        return s.value

    def profile(self, enable=True):
        _check(lib().fg_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        ms = np.zeros(FG_K_COUNT)
        n = np.zeros(FG_K_COUNT, dtype=np.int64)
        _check(lib().fg_profile_read(self.h, _dp(ms), n.ctypes.data_as(_P(_LL))))
        return ms, n

    def copy_state(self, buf, to_buf, env=0):
        """Copy the raw state to / from a device buffer (an int pointer or a
        CUDA tensor of state_bytes() bytes)."""
        p = buf.data_ptr() if hasattr(buf, "data_ptr") else int(buf)
        _check(lib().fg_copy_state(self.h, env, _V(p), 1 if to_buf else 0))

    def step_state(self, src, dst, frames=None):
        """One step from the device state buffer src into dst (CUDA tensors
        or int pointers of state_bytes() bytes), leaving the domain's own
        populations alone (fg_step_state)."""
        fr = None
        if frames is not None:
            if not isinstance(frames, (list, tuple)):
                frames = [frames]
            fr = (fg_frame * len(frames))(*[f if isinstance(f, fg_frame) else frame_from_array(f) for f in frames])
        ps = src.data_ptr() if hasattr(src, "data_ptr") else int(src)
        pd = dst.data_ptr() if hasattr(dst, "data_ptr") else int(dst)
        _check(lib().fg_step_state(self.h, _V(ps), _V(pd), fr))

    def adjoint_reset(self):
        _check(lib().fg_adjoint_reset(self.h))

    def adjoint_step(self, frame=None, gF=None, gX=None, gU=None):
        """One adjoint step; gX, gU are CUDA float tensors (n, 3) to fill."""
        fr = None
        if frame is not None:
            fr = ctypes.byref(frame if isinstance(frame, fg_frame) else frame_from_array(frame))
        g = None
        if gF is not None:
            g = np.ascontiguousarray(gF, dtype=np.float64).ravel()
        _check(lib().fg_adjoint_step(self.h, fr, _dp(g) if g is not None else None,
                                     _V(gX.data_ptr()) if gX is not None else None,
                                     _V(gU.data_ptr()) if gU is not None else None))

    def adjoint_step_state(self, state, frame=None, gF=None, gX=None, gU=None):
        """adjoint_step with the step's forward state read from a device
        buffer (CUDA tensor or int pointer of state_bytes() bytes)."""
        fr = None
        if frame is not None:
            fr = ctypes.byref(frame if isinstance(frame, fg_frame) else frame_from_array(frame))
        g = None
        if gF is not None:
            g = np.ascontiguousarray(gF, dtype=np.float64).ravel()
        p = state.data_ptr() if hasattr(state, "data_ptr") else int(state)
        _check(lib().fg_adjoint_step_state(self.h, _V(p), fr, _dp(g) if g is not None else None,
                                           _V(gX.data_ptr()) if gX is not None else None,
                                           _V(gU.data_ptr()) if gU is not None else None))

    def adjoint(self):
        lam = np.zeros((self.ncell(0), 27))
        _check(lib().fg_get_adjoint(self.h, _dp(lam)))
        return lam

    def set_adjoint(self, lam):
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(self.ncell(0), 27)
        _check(lib().fg_set_adjoint(self.h, _dp(lam)))

    def autotune(self):
        """Time the stream-collide variants, keep the fastest; returns
        (name of the kept variant, {name: ms per launch})."""
        choice = _I()
        ms = np.zeros(FG_K1_NVARIANTS)
        _check(lib().fg_autotune(self.h, ctypes.byref(choice), _dp(ms)))
        return K1_NAMES[choice.value], {K1_NAMES[k]: float(ms[k]) for k in range(FG_K1_NVARIANTS) if ms[k] >= 0}

    def stream_collide_variant(self):
        v = _I()
        _check(lib().fg_stream_collide_variant(self.h, ctypes.byref(v)))
        return K1_NAMES[v.value]

    def stream_collide_bytes(self):
        b = _ULL()
        _check(lib().fg_stream_collide_bytes(self.h, ctypes.byref(b)))
        return b.value
