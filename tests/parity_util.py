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
# force against the FP64 oracle
TOL_F32 = 1e-5


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


class Pair:
    """One GPU domain (single environment) and one oracle, stepped together."""

    def __init__(self, shape, tau, faces=(0,) * 6, u_in=(0.0, 0.0, 0.0), rho0=1.0, storage="f32",
                 variant="auto", ib_iters=1, deterministic=False, slip=False, eq_order=2):
        self.shape = tuple(shape)
        self.o = oracle.Oracle(shape, tau, faces=faces, u_in=f32(u_in), rho_out=rho0, ib_iters=ib_iters,
                               slip=slip, eq_order=eq_order)
        self.g = fishlbm.Domain([fishlbm.env_desc(shape, tau, faces, f32(u_in), rho0)], storage=storage,
                                variant=variant, ib_iters=ib_iters, deterministic=deterministic, slip=slip,
                                eq_order=eq_order)
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

