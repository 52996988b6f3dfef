"""Allocation-free body force, checked against the domain path.

fg_body_force_noalloc serves callers that cannot allocate device memory when
they need the force on the body: a program whose GPU memory is all held by
another framework's memory pool, or a control loop that cannot afford the
device-wide synchronisation cudaMalloc and cudaFree imply.  Its scratch is a
static device array inside the library.  Here it is called through the C ABI
twice in a row, each time on a state saved from a domain, and must report
the same force and torque as fg_step + fg_get_body_force_torque from that
state, within the FP32 parity tolerance.  This file is collected last so a
failure here cannot hide the other tests' results.
"""
import numpy as np
import pytest

from paper_2206_01683_b300 import fishlbm, inputs

from parity_util import TOL_F32, rel_l2

pytestmark = pytest.mark.gpu

OPEN_X = (1, 2, 3, 3, 3, 3)


def test_noalloc_force_matches_step_force_twice():
    torch = pytest.importorskip("torch")
    shape = (96, 48, 48)
    env = fishlbm.env_desc(shape, 0.52, OPEN_X, (0.02, 0.0, 0.0), 1.0, (0.02, 0.0, 0.0))
    d = fishlbm.Domain([env])
    rho, u = inputs.random_fields(shape, seed=77, u_amp=0.01, rho_amp=0.004)
    u[:, 0] += 0.02
    d.init_fields(rho, u)
    fish = inputs.fish_for_grid(shape, 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    ref = tuple(float(v) for v in fish.joints_rest[0])
    dV = torch.tensor(fish.dV, dtype=torch.float32, device="cuda")
    seg = torch.tensor(fish.seg, dtype=torch.int32, device="cuda")
    for n in range(5):                       # a non-trivial flow to start from
        X, U = fish.pose(n)
        d.set_markers(np.float32(X), np.float32(U), np.float32(fish.dV), seg=fish.seg, n_seg=5, ref=ref)
        d.step(1, [traj.at(n)])
    d.get_body_force_torque()

    for n in (10, 11):                       # two calls in a row
        state = torch.from_numpy(d.save_state().view(np.float32).copy()).cuda()
        X, U = (torch.tensor(a, dtype=torch.float32, device="cuda") for a in fish.pose(n))
        frame = fishlbm.frame_from_array(traj.at(n))
        out = torch.full((6, 6), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        fishlbm.fg_body_force_noalloc(env, state.data_ptr(), X.data_ptr(), U.data_ptr(), dV.data_ptr(),
                                      seg.data_ptr(), X.shape[0], 5, ref, frame, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()

        d.set_markers(X, U, dV, seg, n_seg=5, ref=ref)
        d.step(1, [frame])
        want = d.get_body_force_torque()
        assert np.all(np.isfinite(got))
        assert np.abs(want[-1, :3]).max() > 1e-4          # a real force, not zeros
        assert rel_l2(got, want) <= TOL_F32, (got, want)


def test_noalloc_rejects_more_markers_than_its_scratch():
    torch = pytest.importorskip("torch")
    env = fishlbm.env_desc((16, 16, 16), 0.6)
    buf = torch.zeros(16, device="cuda")
    p = buf.data_ptr()
    with pytest.raises(fishlbm.FgError) as ei:
        fishlbm.fg_body_force_noalloc(env, p, p, p, p, None, fishlbm.FG_NOALLOC_MAX_MARKERS + 1, 1,
                                      None, None, p)
    assert ei.value.status == fishlbm.FG_ERR_INVALID
    assert "FG_NOALLOC_MAX_MARKERS" in fishlbm.lib().fg_last_error().decode()
