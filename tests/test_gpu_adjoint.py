"""The discrete adjoint of the step against the FP64 oracle.

Dot-product tests: for the step map Phi (populations, marker positions and
velocities -> next populations) and a force/torque loss of the step, the
oracle's directional derivative J v (FP64 central differences) must equal
<v, J^T w> from the CUDA adjoint, at the same linearisation point, with the
frame's rotation and acceleration on.  Then the whole pipeline -- forward with
checkpoints, recompute, adjoint steps, torch skinning -- gives the gradient of
the time-averaged thrust w.r.t. the joint-wave amplitudes and phases, checked
against central differences of the oracle (FP64) and, at the full
128x64x64 / 1500-marker / 200-step size, of the CUDA forward (FP32).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2206_01683_b300 import fishlbm, inputs

from parity_util import gpu_to_oracle_perm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPE = (10, 8, 6)
TAU = 0.7
FRAME = oracle.make_frame(acc=(2e-4, -1e-4, 5e-5), omega=(1e-3, -2e-3, 3e-3), domega=(1e-5, 2e-5, -1e-5),
                          origin=(4.5, 3.5, 2.5))


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def base_case(seed=3):
    """A generic state (equilibrium of smooth random fields plus a small
    non-equilibrium part), 6 markers on two segments; everything
    float32-representable so both sides start from the same point."""
    rng = np.random.default_rng(seed)
    o = oracle.Oracle(SHAPE, TAU)
    rho, u = inputs.random_fields(SHAPE, seed=seed, u_amp=0.03, rho_amp=0.01)
    o.init_fields(rho, u)
    _, w = oracle.lattice()
    f = o.populations()
    f = f + 1e-3 * w * rng.standard_normal(f.shape)
    f = w + f32(f - w)
    X = f32(rng.uniform(0, 1, (6, 3)) * np.array(SHAPE))
    U = f32(0.02 * rng.standard_normal((6, 3)))
    dV = f32(np.full(6, 0.7))
    seg = np.array([0, 1, 0, 1, 1, 0], dtype=np.int32)
    return f, X, U, dV, seg


def oracle_step(f, X, U, dV, seg, ref):
    o = oracle.Oracle(SHAPE, TAU)
    o.set_populations(f)
    o.set_markers(X, U, dV, seg=seg, nseg=2, ref=ref)
    o.step(f32(FRAME))
    return o.populations(), o.force_torque()


def gpu_adjoint(f, X, U, dV, seg, ref, lam_next=None, gF=None):
    perm = gpu_to_oracle_perm()
    d = fishlbm.Domain([fishlbm.env_desc(SHAPE, TAU)], variant="plain")
    inv = np.argsort(perm)
    d.set_populations(f[:, inv])                   # oracle order -> library order
    d.set_markers(np.float32(X), np.float32(U), np.float32(dV), seg=seg, n_seg=2, ref=ref)
    d.adjoint_reset()
    if lam_next is not None:
        d.set_adjoint(lam_next[:, inv])
    gX = torch.zeros((6, 3), device="cuda")
    gU = torch.zeros((6, 3), device="cuda")
    d.adjoint_step(fishlbm.frame_from_array(f32(FRAME)), gF, gX, gU)
    lam = d.adjoint()[:, perm]                      # library order -> oracle order
    torch.cuda.synchronize()
    return lam, gX.cpu().numpy().astype(np.float64), gU.cpu().numpy().astype(np.float64)


def rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


def test_adjoint_of_the_population_update():
    f, X, U, dV, seg = base_case()
    ref = (4.0, 3.0, 2.0)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(f.shape) * 1e-2
    w = rng.standard_normal(f.shape)
    eps = 1e-5
    fp, _ = oracle_step(f + eps * v, X, U, dV, seg, ref)
    fm, _ = oracle_step(f - eps * v, X, U, dV, seg, ref)
    Jv = (fp - fm) / (2 * eps)
    lam, _, _ = gpu_adjoint(f, X, U, dV, seg, ref, lam_next=w)
    assert rel((Jv * w).sum(), (v * lam).sum()) < 2e-4
    # and along the markers (positions, velocities)
    vX = rng.standard_normal(X.shape)
    vU = rng.standard_normal(U.shape) * 1e-2
    fp, _ = oracle_step(f, X + eps * vX, U, dV, seg, ref)
    fm, _ = oracle_step(f, X - eps * vX, U, dV, seg, ref)
    _, gX, gU = gpu_adjoint(f, X, U, dV, seg, ref, lam_next=w)
    assert rel((((fp - fm) / (2 * eps)) * w).sum(), (vX * gX).sum()) < 2e-4
    fp, _ = oracle_step(f, X, U + eps * vU, dV, seg, ref)
    fm, _ = oracle_step(f, X, U - eps * vU, dV, seg, ref)
    assert rel((((fp - fm) / (2 * eps)) * w).sum(), (vU * gU).sum()) < 2e-4


def test_adjoint_of_force_and_torque_loss():
    f, X, U, dV, seg = base_case(seed=5)
    ref = (4.0, 3.0, 2.0)
    rng = np.random.default_rng(9)
    gF = rng.standard_normal((3, 6))               # rows: segment 0, segment 1, total

    def loss(f_, X_, U_):
        _, ft = oracle_step(f_, X_, U_, dV, seg, ref)
        return (gF * ft).sum()

    lam, gX, gU = gpu_adjoint(f, X, U, dV, seg, ref, gF=gF)
    eps = 1e-5
    v = rng.standard_normal(f.shape) * 1e-2
    vX = rng.standard_normal(X.shape)
    vU = rng.standard_normal(U.shape) * 1e-2
    fd = (loss(f + eps * v, X, U) - loss(f - eps * v, X, U)) / (2 * eps)
    assert rel(fd, (v * lam).sum()) < 2e-4
    fd = (loss(f, X + eps * vX, U) - loss(f, X - eps * vX, U)) / (2 * eps)
    assert rel(fd, (vX * gX).sum()) < 2e-4
    fd = (loss(f, X, U + eps * vU) - loss(f, X, U - eps * vU)) / (2 * eps)
    assert rel(fd, (vU * gU).sum()) < 2e-4


def test_adjoint_rejects_what_it_does_not_cover():
    d = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7, (1, 2, 3, 3, 3, 3))])
    with pytest.raises(fishlbm.FgError) as ei:
        d.adjoint_reset()
    assert ei.value.status == fishlbm.FG_ERR_INVALID
    d = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7)], storage="f16")
    with pytest.raises(fishlbm.FgError):
        d.adjoint_reset()


# ------------------------------------------------------ end-to-end gradient

def oracle_thrust(shape, tau, fish_len, nm, steps, theta):
    """Time-averaged thrust of the same run in the FP64 oracle, exact markers."""
    th = np.asarray(theta, dtype=np.float64)
    fish = inputs.fish_for_grid(shape, fish_len, nm, amplitudes=th[:4], phases=th[4:])
    X, U = fish.poses(np.arange(steps))
    o = oracle.Oracle(shape, tau)
    total = 0.0
    for n in range(steps):
        o.set_markers(X[n], U[n], fish.dV, seg=fish.seg, nseg=5, ref=fish.joints_rest[0])
        o.step()
        total += -o.force_torque()[-1, 0]
    return total / steps


def test_thrust_gradient_matches_oracle_central_differences():
    from paper_2206_01683_b300 import adjoint
    shape, tau, L, nm, steps = (48, 24, 24), 0.6, 12.0, 300, 40
    prob = adjoint.ThrustProblem(shape, tau, L, nm, steps, checkpoint=10)
    theta = adjoint.default_theta().requires_grad_(True)
    Lgpu = adjoint.SwimThrust.apply(theta, prob)
    (g,) = torch.autograd.grad(Lgpu, theta)
    g = g.numpy()
    th0 = theta.detach().numpy()
    L0 = oracle_thrust(shape, tau, L, nm, steps, th0)
    assert abs(Lgpu.item() - L0) < 1e-4 * abs(L0) + 1e-9
    h = 1e-3
    fd = np.zeros(8)
    for k in range(8):
        e = np.zeros(8)
        e[k] = h
        fd[k] = (oracle_thrust(shape, tau, L, nm, steps, th0 + e) -
                 oracle_thrust(shape, tau, L, nm, steps, th0 - e)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    err = np.abs(g - fd)
    print("thrust gradient: adjoint", g, "oracle FD", fd, "rel", err / np.abs(fd))
    # 1e-3 relative per component, above a floor for what neither side
    # resolves: the oracle's central difference carries O(h^2) truncation
    # (about 1e-7 of the largest component at h = 1e-3) and the CUDA forward
    # sees float32 marker data (rounding 6e-8 relative), so a component below
    # about 1e-5 of the largest is compared at that absolute level
    floor = 1e-5 * scale
    assert np.all(err <= 1e-3 * np.abs(fd) + floor), (g, fd, err)


def test_thrust_gradient_full_size_matches_gpu_central_differences():
    """128x64x64, one fish of 1500 markers (body length 32), 200 steps,
    checkpoint every 20: adjoint vs central differences (h = 1e-3) of the FP32
    CUDA forward."""
    from paper_2206_01683_b300 import adjoint
    cfg = inputs.ADJOINT_CHANNEL
    prob = adjoint.ThrustProblem(cfg["shape"], cfg["tau"], cfg["length"], cfg["n_markers"], cfg["steps"],
                                 checkpoint=cfg["checkpoint"])
    theta = adjoint.default_theta().requires_grad_(True)
    Lgpu = adjoint.SwimThrust.apply(theta, prob)
    (g,) = torch.autograd.grad(Lgpu, theta)
    g = g.numpy()
    th0 = theta.detach()
    h = 1e-3
    fd = np.zeros(8)
    for k in range(8):
        e = torch.zeros(8, dtype=torch.float64)
        e[k] = h
        fd[k] = (adjoint.SwimThrust.apply(th0 + e, prob).item() -
                 adjoint.SwimThrust.apply(th0 - e, prob).item()) / (2 * h)
    # 1e-2 relative per component (central differences of an FP32 forward),
    # above the differences' own noise: the loss is resolved to about 1e-7 of
    # |L| (FP32 dynamics, FP64 force rows), so a difference quotient carries
    # about 1e-7 |L| / h; the floor is ten times that
    floor = 10 * 1e-7 * abs(Lgpu.item()) / h
    err = np.abs(g - fd)
    print("full-size thrust gradient: adjoint", g, "GPU FD", fd, "floor", floor)
    assert np.all(err <= 1e-2 * np.abs(fd) + floor), (g, fd, err, floor)
    assert prob.backward_ms is not None and prob.forward_ms > 0
