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

import oracle
from paper_2206_01683_b300 import fishlbm, inputs

from parity_util import TOL_F32, f32, rel_l2

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


def _noalloc(env, state, X, U, dV, seg, n_seg, ref, frame):
    """One call through the C ABI on device tensors; the rows as numpy."""
    import torch
    out = torch.full((n_seg + 1, 6), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    fishlbm.fg_body_force_noalloc(env, state.data_ptr(), X.data_ptr(), U.data_ptr(), dV.data_ptr(),
                                  seg.data_ptr() if seg is not None else None, X.shape[0], n_seg, ref, frame,
                                  out.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _seeded_state(shape, env, seed, u_in=0.0):
    """The same seeded (rho, u) fields as a GPU state buffer (the library's
    own equilibrium initialisation) and as host arrays for the oracle."""
    import torch
    rho, u = inputs.random_fields(shape, seed=seed, u_amp=0.01, rho_amp=0.004)
    u[:, 0] += u_in
    d = fishlbm.Domain([env])
    d.init_fields(rho, u)
    state = torch.from_numpy(d.save_state().view(np.float32).copy()).cuda()
    d.close()
    return state, rho, u


def test_noalloc_rejected_marker_then_valid_call():
    """A marker half a cell from the open -x face is rejected: every row of
    that call is NaN.  The next call, with the valid pose, must not see the
    previous call's flag (the scratch keeps its contents between calls): its
    rows are finite and match the domain's step from the same state."""
    torch = pytest.importorskip("torch")
    shape = (48, 32, 32)
    env = fishlbm.env_desc(shape, 0.52, OPEN_X, (0.02, 0.0, 0.0), 1.0, (0.02, 0.0, 0.0))
    state, rho, u = _seeded_state(shape, env, seed=78, u_in=0.02)
    fish = inputs.fish_for_grid(shape, 16.0, 400)
    ref = tuple(float(v) for v in fish.joints_rest[0])
    X, U = (np.float32(a) for a in fish.pose(7))
    dV = torch.tensor(fish.dV, dtype=torch.float32, device="cuda")
    seg = torch.tensor(fish.seg, dtype=torch.int32, device="cuda")
    frame = fishlbm.make_frame(origin=tuple(inputs.domain_centre(shape)))
    bad = X.copy()
    bad[0] = (0.5, 16.0, 16.0)
    got_bad = _noalloc(env, state, torch.from_numpy(bad).cuda(), torch.from_numpy(U).cuda(), dV, seg, 5, ref, frame)
    assert np.all(np.isnan(got_bad)), got_bad
    got = _noalloc(env, state, torch.from_numpy(X).cuda(), torch.from_numpy(U).cuda(), dV, seg, 5, ref, frame)
    assert np.all(np.isfinite(got)), got
    d = fishlbm.Domain([env])
    d.init_fields(rho, u)
    d.set_markers(X, U, np.float32(fish.dV), seg=fish.seg, n_seg=5, ref=ref)
    d.step(1, [frame])
    want = d.get_body_force_torque()
    assert rel_l2(got, want) <= TOL_F32, (got, want)


@pytest.mark.parametrize("case", ["periodic_wrap", "open_channel"])
def test_noalloc_against_oracle(case):
    """The rows against the FP64 oracle's first step from the same seeded
    fields (both sides initialise their own state from them): a sphere whose
    stencils straddle the periodic x and y wraps of a box in a rotating
    frame, two segments about a common point; and the swimmer in its open
    channel and moving frame, five segments."""
    torch = pytest.importorskip("torch")
    if case == "periodic_wrap":
        shape, tau, faces, u_in = (32, 24, 20), 0.6, (0,) * 6, 0.0
        X, dV = inputs.fibonacci_sphere(150, 3.0, (0.6, 23.3, 10.0))
        U = np.tile([0.01, -0.005, 0.002], (150, 1))
        seg = (X[:, 2] > 10.0).astype(np.int32)
        n_seg, ref = 2, (1.0, 23.0, 10.0)
        fr = oracle.make_frame(acc=(1e-5, -2e-5, 0.0), omega=(1e-4, 2e-4, -1e-4), domega=(1e-6, 0.0, 2e-6),
                               origin=(16.0, 12.0, 10.0))
    else:
        shape, tau, faces, u_in = (64, 32, 32), 0.52, OPEN_X, 0.02
        fish = inputs.fish_for_grid(shape, 16.0, 400)
        X, U = fish.pose(5)
        dV, seg, n_seg, ref = fish.dV, fish.seg.astype(np.int32), 5, tuple(fish.joints_rest[0])
        fr = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape)).at(5)
    X32, U32, dV32, fr32 = np.float32(X), np.float32(U), np.float32(dV), f32(fr)
    env = fishlbm.env_desc(shape, tau, faces, f32((u_in, 0, 0)), 1.0, f32((u_in, 0, 0)))
    state, rho, u = _seeded_state(shape, env, seed=79, u_in=u_in)
    got = _noalloc(env, state, torch.from_numpy(X32).cuda(), torch.from_numpy(U32).cuda(),
                   torch.from_numpy(dV32).cuda(), torch.from_numpy(seg).cuda(), n_seg, ref,
                   fishlbm.frame_from_array(fr32))
    o = oracle.Oracle(shape, tau, faces=faces, u_in=f32((u_in, 0, 0)))
    o.init_fields(rho, u)
    o.set_markers(X32.astype(np.float64), U32.astype(np.float64), dV32.astype(np.float64), seg=seg, nseg=n_seg,
                  ref=ref)
    o.step(fr32)
    want = o.force_torque()
    assert np.abs(want[-1, :3]).max() > 1e-4
    assert rel_l2(got[:, :3], want[:, :3]) <= TOL_F32, (case, got, want)
    assert rel_l2(got[:, 3:], want[:, 3:]) <= TOL_F32, (case, got, want)
