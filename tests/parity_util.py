"""Run the CUDA path (through the C ABI) and the FP64 oracle side by side on
identical inputs and measure their difference.

Both sides receive the same float32-rounded marker and frame data, since the
C ABI takes markers in float and rounds frames to float.  Nothing fed to the
oracle ever comes from the CUDA path: both start from the same seeded fields.
"""
import numpy as np

import oracle
from paper_2206_01683_b300 import fishlbm

# FP32 parity bar: relative L2 error <= 1e-5 in density, velocity and body
# force against the FP64 oracle; the same bar holds for the velocity and the
# populations restricted to the open-face boundary layer and to the markers'
# stencil support
TOL_F32 = 1e-5
# FP32 per-cell bar: no cell's velocity (or population) may differ by more
# than this fraction of the field's largest magnitude
TOL_MAX = 1e-5
LOCAL_KEYS = ("u_bl", "u_ib", "pop_bl", "pop_ib")
MAX_KEYS = ("u_max", "pop_max")


def assert_local(err, tol=TOL_F32, tol_max=TOL_MAX, where=""):
    """The local bars: rel-L2 on the boundary layer and on the stencil
    support, and the per-cell bound (keys absent for a case are skipped)."""
    print("local errors", where, {k: "%.3g" % err[k] for k in LOCAL_KEYS + MAX_KEYS + ("drho_max",) if k in err})
    for k in LOCAL_KEYS:
        if k in err:
            assert err[k] <= tol, (where, k, err)
    for k in MAX_KEYS:
        if k in err:
            assert err[k] <= tol_max, (where, k, err)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gpu_to_oracle_perm():
    cg, _ = fishlbm.fg_lattice()
    co, _ = oracle.lattice()
    idx = []
    for v in co:
        j = [k for k in range(27) if tuple(cg[k]) == tuple(v)]
        assert len(j) == 1
        idx.append(j[0])
    return np.array(idx)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_rel(a, b):
    """Largest per-element difference over the largest reference magnitude:
    the L-infinity analogue of rel_l2, which a domain-wide L2 norm cannot
    dilute."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b)) / (nb if nb > 0 else 1.0)) if a.size else 0.0


def boundary_layer_mask(shape, faces):
    """Cells (index x + nx (y + ny z)) in the two outermost layers of every
    non-periodic face: the boundary nodes the open-face rule rebuilds and the
    inward neighbours it extrapolates from.  None when every face is
    periodic."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = np.zeros((nz, ny, nx), dtype=bool)
    for axis, (c, n) in enumerate(((x, nx), (y, ny), (z, nz))):
        if faces[2 * axis] != 0:
            m |= c <= 1
        if faces[2 * axis + 1] != 0:
            m |= c >= n - 2
    return m.ravel() if m.any() else None


def ib_support_mask(shape, faces, X):
    """Cells within one cell of some marker's 4x4x4 delta stencil (nodes
    floor(X) - 1 .. floor(X) + 2 per axis, widened to floor(X) - 2 ..
    floor(X) + 3): where the spread force lands and the cells it streams to
    in one step.  Periodic axes wrap.  None without markers."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    if X.shape[0] == 0:
        return None
    nx, ny, nz = shape
    off = np.arange(-2, 4)
    idx = []
    for axis, n in enumerate((nx, ny, nz)):
        k = np.floor(X[:, axis]).astype(np.int64)[:, None] + off[None, :]
        periodic = faces[2 * axis] == 0 and faces[2 * axis + 1] == 0
        idx.append(np.mod(k, n) if periodic else np.clip(k, 0, n - 1))
    ix, iy, iz = idx
    cells = ix[:, None, None, :] + nx * (iy[:, None, :, None] + ny * iz[:, :, None, None])
    m = np.zeros(nx * ny * nz, dtype=bool)
    m[cells.ravel()] = True
    return m


def local_errors(shape, faces, X, rg, ug, ro, uo, fg=None, fo=None):
    """Errors a domain-wide rel-L2 can dilute: rel-L2 of u (and of the
    populations f - w) restricted to the open-face boundary layer (_bl) and
    to the markers' stencil support (_ib), and the largest per-cell error of
    u, rho - 1 and f - w over the reference's largest magnitude (_max)."""
    out = dict(u_max=max_rel(ug, uo), drho_max=max_rel(rg - 1.0, ro - 1.0))
    if fg is not None:
        out["pop_max"] = max_rel(fg, fo)
    for tag, m in (("bl", boundary_layer_mask(shape, faces)),
                   ("ib", ib_support_mask(shape, faces, X) if X is not None else None)):
        if m is None:
            continue
        out["u_" + tag] = rel_l2(ug[m], uo[m])
        if fg is not None:
            out["pop_" + tag] = rel_l2(fg[m], fo[m])
    return out


class Pair:
    """One GPU domain (single environment) and one oracle, stepped together."""

    def __init__(self, shape, tau, faces=(0,) * 6, u_in=(0.0, 0.0, 0.0), rho0=1.0, storage="f32",
                 variant="auto", ib_iters=1, deterministic=False, slip=False, eq_order=2, layout="pull"):
        self.shape = tuple(shape)
        self.faces = tuple(int(f) for f in faces)
        self.X = None
        self.o = oracle.Oracle(shape, tau, faces=faces, u_in=f32(u_in), rho_out=rho0, ib_iters=ib_iters,
                               slip=slip, eq_order=eq_order)
        self.g = fishlbm.Domain([fishlbm.env_desc(shape, tau, faces, f32(u_in), rho0)], storage=storage,
                                variant=variant, ib_iters=ib_iters, deterministic=deterministic, slip=slip,
                                eq_order=eq_order, layout=layout)
        self.perm = gpu_to_oracle_perm()
        _, self.w = oracle.lattice()
        self.nseg = 1
        self.force_hist_o = []
        self.force_hist_g = []

    def init(self, rho=None, u=None):
        self.o.init_fields(rho, u)
        self.g.init_fields(rho, u)

    def markers(self, X, U, dV, seg=None, nseg=1, ref=(0.0, 0.0, 0.0), normals=None):
        X32, U32, dV32 = (np.asarray(a, dtype=np.float32) for a in (X, U, dV))
        N32 = None
        if normals is not None:
            N32 = np.asarray(normals, dtype=np.float64)
            N32 = (N32 / np.linalg.norm(N32, axis=1, keepdims=True)).astype(np.float32)
        self.o.set_markers(X32.astype(np.float64), U32.astype(np.float64), dV32.astype(np.float64),
                           seg=seg, nseg=nseg, ref=ref,
                           normals=None if N32 is None else N32.astype(np.float64))
        self.g.set_markers(X32, U32, dV32, seg=seg, n_seg=nseg, ref=ref)
        self.X = X32.astype(np.float64)
        if N32 is not None:
            self.g.set_marker_normals(N32)
        self.nseg = nseg

    def step(self, frame=None, record=True):
        fr = oracle.make_frame() if frame is None else np.asarray(frame, dtype=np.float64)
        fr = f32(fr)
        self.o.step(fr)
        self.g.step(1, [fishlbm.frame_from_array(fr)])
        if record:
            self.force_hist_o.append(self.o.force_torque())
            self.force_hist_g.append(self.g.get_body_force_torque())

    def errors(self):
        ro, uo = self.o.fields()
        rg, ug = self.g.fields()
        fo = self.o.populations() - self.w
        fg = self.g.populations()[:, self.perm] - self.w
        out = dict(rho=rel_l2(rg, ro), drho=rel_l2(rg - 1.0, ro - 1.0), u=rel_l2(ug, uo),
                   pop=rel_l2(fg, fo))
        out.update(local_errors(self.shape, self.faces, self.X, rg, ug, ro, uo, fg, fo))
        if self.force_hist_o:
            Fo = np.array([h[-1, :3] for h in self.force_hist_o])
            Fg = np.array([h[-1, :3] for h in self.force_hist_g])
            To = np.array([h[:, 3:] for h in self.force_hist_o])
            Tg = np.array([h[:, 3:] for h in self.force_hist_g])
            Fso = np.array([h[:, :3] for h in self.force_hist_o])
            Fsg = np.array([h[:, :3] for h in self.force_hist_g])
            out.update(force=rel_l2(Fg, Fo), torque=rel_l2(Tg, To), seg_force=rel_l2(Fsg, Fso))
        out["mass"] = abs(self.g.mass() - self.o.mass()) / self.o.mass()
        return out

