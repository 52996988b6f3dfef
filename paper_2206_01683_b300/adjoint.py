"""Gradients of the swimmer's time-averaged thrust with respect to its
joint-wave parameters, through the discrete adjoint of the IB-LBM step.

The loss is  L = (1/N) sum_{n<N} thrust_n,  thrust_n = -F^n_x,  the force the
fluid exerts on the body along -x in step n (paper Sec. III-B; the tau_ext of
Eq. 1).  The parameters are the amplitudes A_j and phases phi_j of the joint
wave theta_j(t) = A_j sin(2 pi t / period - phi_j); they drive the markers
through linear blend skinning (Sec. III-A), written here in torch so that
autograd maps dL/dX, dL/dU of every step to dL/dA, dL/dphi.

The forward pass runs the CUDA step and keeps the state every `checkpoint`
steps; the backward pass walks the segments in reverse, recomputes the states
of a segment from its checkpoint (fg_step_state, from buffer to buffer, so no
state is copied), and runs the library's adjoint step on each of them
(fg_adjoint_step_state) from the last step of the segment to its first.  Only the
skinning (a small dense map) is differentiated by torch; the fluid's adjoint
is the library's.
"""
import math

import numpy as np
import torch

from . import fishlbm, inputs


def fish_poses_torch(fish, ts, A, phi):
    """Marker positions and velocities (T, n, 3) for times ts, as a
    differentiable function of A (4,) and phi (4,) (float64 tensors); the same
    skinning as inputs.Fish.poses."""
    dev = A.device
    ts = torch.as_tensor(np.asarray(ts, dtype=np.float64), device=dev)
    T = ts.shape[0]
    NS = inputs.N_SEGMENTS
    w = 2.0 * math.pi / fish.period
    th = A[None, :] * torch.sin(w * ts[:, None] - phi[None, :])           # (T, 4)
    dth = A[None, :] * w * torch.cos(w * ts[:, None] - phi[None, :])
    ang = torch.cat([torch.zeros(T, 1, dtype=A.dtype, device=dev), torch.cumsum(th, dim=1)], dim=1)
    c, s = torch.cos(ang), torch.sin(ang)
    J = torch.as_tensor(fish.joints_rest, device=dev)
    trans = [torch.zeros(T, 2, dtype=A.dtype, device=dev)]
    joint_world = []
    for k in range(1, NS):
        Pk = J[k - 1, :2]
        cp, sp = c[:, k - 1], s[:, k - 1]
        jw = torch.stack([cp * Pk[0] - sp * Pk[1], sp * Pk[0] + cp * Pk[1]], dim=1) + trans[k - 1]
        joint_world.append(jw)
        ck, sk = c[:, k], s[:, k]
        trans.append(jw - torch.stack([ck * Pk[0] - sk * Pk[1], sk * Pk[0] + ck * Pk[1]], dim=1))
    rest = torch.as_tensor(fish.rest, device=dev)
    Wt = torch.as_tensor(fish.W, device=dev)
    p = rest[:, :2]
    Xx = torch.zeros(T, fish.n, dtype=A.dtype, device=dev)
    Xy = torch.zeros_like(Xx)
    Ux = torch.zeros_like(Xx)
    Uy = torch.zeros_like(Xx)
    for k in range(NS):
        qx = c[:, k, None] * p[None, :, 0] - s[:, k, None] * p[None, :, 1] + trans[k][:, None, 0]
        qy = s[:, k, None] * p[None, :, 0] + c[:, k, None] * p[None, :, 1] + trans[k][:, None, 1]
        vx = torch.zeros_like(qx)
        vy = torch.zeros_like(qy)
        for jj in range(1, k + 1):
            dx = qx - joint_world[jj - 1][:, None, 0]
            dy = qy - joint_world[jj - 1][:, None, 1]
            vx = vx - dth[:, jj - 1, None] * dy
            vy = vy + dth[:, jj - 1, None] * dx
        wk = Wt[None, :, k]
        Xx = Xx + wk * qx
        Xy = Xy + wk * qy
        Ux = Ux + wk * vx
        Uy = Uy + wk * vy
    Xz = rest[None, :, 2].expand(T, fish.n)
    X = torch.stack([Xx, Xy, Xz], dim=2)
    U = torch.stack([Ux, Uy, torch.zeros_like(Ux)], dim=2)
    return X, U


class ThrustProblem:
    """One swimmer in a periodic box, fluid initially at rest, FP32.

    frames: None (frame at rest) or an array (steps, 12) of p'', omega,
    domega, origin per step."""

    def __init__(self, shape, tau, length, n_markers, steps, checkpoint=20, frames=None, variant="auto"):
        self.shape = tuple(shape)
        self.tau = tau
        self.steps = int(steps)
        self.C = int(checkpoint)
        self.fish = inputs.fish_for_grid(shape, length, n_markers)
        self.nseg = inputs.N_SEGMENTS
        self.ref = tuple(float(v) for v in self.fish.joints_rest[0])
        self.frames = None
        if frames is not None:
            self.frames = [fishlbm.frame_from_array(f) for f in np.asarray(frames)]
        self.dom = fishlbm.Domain([fishlbm.env_desc(shape, tau)], record_history=self.steps, variant=variant)
        self.state_bytes = self.dom.state_bytes()
        dev = "cuda"
        self.dV = torch.tensor(self.fish.dV, dtype=torch.float32, device=dev)
        self.seg = torch.tensor(self.fish.seg, dtype=torch.int32, device=dev)
        nck = (self.steps + self.C - 1) // self.C
        self.ckpt = torch.empty((nck, self.state_bytes), dtype=torch.uint8, device=dev)
        self.seg_states = torch.empty((self.C, self.state_bytes), dtype=torch.uint8, device=dev)
        self.forward_ms = None
        self.backward_ms = None

    def _frame(self, n):
        return [self.frames[n]] if self.frames is not None else None

    def _markers(self, X, U, n, first=False):
        self.dom.set_markers(X[n], U[n], self.dV if first else None, self.seg if first else None,
                             n_seg=self.nseg, ref=self.ref)

    def forward(self, X, U):
        """Run N steps with markers X, U (float32 CUDA, (N, n, 3)); keep
        checkpoints; return L (float)."""
        d = self.dom
        d.init_fields(None, None)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        for n in range(self.steps):
            if n % self.C == 0:
                d.copy_state(self.ckpt[n // self.C], True)
            self._markers(X, U, n, first=(n == 0))
            d.step(1, self._frame(n))
        ev[1].record()
        torch.cuda.synchronize()
        self.forward_ms = ev[0].elapsed_time(ev[1])
        h = d.history(self.steps)
        fx_total = h[:, 6 * self.nseg]          # total row, F_x
        return float(np.mean(-fx_total))

    def backward(self, X, U):
        """dL/dX and dL/dU of every step (float32 CUDA, (N, n, 3))."""
        d = self.dom
        N = self.steps
        gX = torch.zeros_like(X)
        gU = torch.zeros_like(U)
        gF = np.zeros((self.nseg + 1, 6))
        gF[self.nseg, 0] = -1.0 / N                # d L / d F_x(total) of every step
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        d.adjoint_reset()
        for s in reversed(range(0, N, self.C)):
            e = min(s + self.C, N)
            # the input state of step n: the checkpoint for n = s, else the
            # recomputed seg_states[n - s]; each recompute step writes the
            # next buffer directly (no state copies)
            state = [self.ckpt[s // self.C]] + [self.seg_states[k] for k in range(1, e - s)]
            for n in range(s, e - 1):              # recompute f*^{s+1} .. f*^{e-1}
                self._markers(X, U, n)
                d.step_state(state[n - s], state[n - s + 1], self._frame(n))
            for n in reversed(range(s, e)):
                self._markers(X, U, n)
                d.adjoint_step_state(state[n - s], self._frame(n)[0] if self.frames is not None else None, gF,
                                     gX[n], gU[n])
        ev[1].record()
        torch.cuda.synchronize()
        self.backward_ms = ev[0].elapsed_time(ev[1])
        return gX, gU


class SwimThrust(torch.autograd.Function):
    """L = SwimThrust.apply(theta, problem): theta = (A_1..A_4, phi_1..phi_4)
    as a float64 tensor; L is the time-averaged thrust (a 0-d tensor)."""

    @staticmethod
    def forward(ctx, theta, problem):
        with torch.no_grad():
            X, U = fish_poses_torch(problem.fish, np.arange(problem.steps), theta[:4], theta[4:])
        X32 = X.float().cuda().contiguous()
        U32 = U.float().cuda().contiguous()
        L = problem.forward(X32, U32)
        ctx.problem = problem
        ctx.save_for_backward(theta)
        ctx.XU = (X32, U32)
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        (theta,) = ctx.saved_tensors
        problem = ctx.problem
        X32, U32 = ctx.XU
        gX, gU = problem.backward(X32, U32)
        with torch.enable_grad():
            th = theta.detach().requires_grad_(True)
            X, U = fish_poses_torch(problem.fish, np.arange(problem.steps), th[:4], th[4:])
            (g,) = torch.autograd.grad((X, U), (th,), (gX.double().to(X.device) * gL.to(X.device),
                                                       gU.double().to(U.device) * gL.to(U.device)))
        return g, None


def default_theta():
    """The joint wave theta_j(t) = 0.3 (j/4) sin(2 pi t/400 - 0.8 j)."""
    j = np.arange(1, 5, dtype=np.float64)
    return torch.tensor(np.concatenate([0.3 * j / 4.0, 0.8 * j]), dtype=torch.float64)
