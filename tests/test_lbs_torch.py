"""The differentiable skinning used by the adjoint equals the numpy skinning
of the input generators, and its autograd derivative w.r.t. the joint-wave
parameters matches central differences (CPU only)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_01683_b300 import adjoint, inputs


def test_torch_poses_equal_numpy_poses():
    fish = inputs.fish_for_grid((64, 32, 32), 16.0, 400)
    th = adjoint.default_theta()
    X, U = adjoint.fish_poses_torch(fish, np.arange(0, 60, 7), th[:4], th[4:])
    Xn, Un = fish.poses(np.arange(0, 60, 7))
    assert np.max(np.abs(X.numpy() - Xn)) < 1e-12
    assert np.max(np.abs(U.numpy() - Un)) < 1e-12


def test_torch_pose_gradient_matches_central_differences():
    fish = inputs.fish_for_grid((64, 32, 32), 16.0, 200)
    th = adjoint.default_theta().requires_grad_(True)
    ts = np.arange(0, 50, 5)
    rng = np.random.default_rng(0)
    wX = torch.tensor(rng.standard_normal((len(ts), 200, 3)))
    wU = torch.tensor(rng.standard_normal((len(ts), 200, 3)))

    def scalar(t):
        X, U = adjoint.fish_poses_torch(fish, ts, t[:4], t[4:])
        return (X * wX).sum() + 100.0 * (U * wU).sum()

    (g,) = torch.autograd.grad(scalar(th), th)
    h = 1e-6
    for k in range(8):
        e = torch.zeros(8, dtype=torch.float64)
        e[k] = h
        fd = (scalar(th.detach() + e) - scalar(th.detach() - e)) / (2 * h)
        assert abs(fd.item() - g[k].item()) <= 1e-6 * max(1.0, abs(g[k].item())), k
