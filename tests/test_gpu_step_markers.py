"""fg_step_markers: new markers and one step in one call, the markers read by
the step's IB kernel straight from the caller's arrays (no copy launch before
the step).  It must give exactly what fg_set_markers_all + fg_step give, for
every stream-collide variant and layout, one and several environments, more
markers than the IB kernel has half-warps, several direct-forcing passes,
and the arrays as device or pinned host memory (the paths that fall back to
a copy included)."""
import numpy as np
import pytest

from paper_2206_01683_b300 import fishlbm, inputs

pytestmark = pytest.mark.gpu

OPEN_X = (1, 2, 3, 3, 3, 3)   # inlet, outflow, free-slip walls


def _case(shapes, n_markers, variant, layout="pull", ib_iters=1, storage="f32"):
    fishes = [inputs.fish_for_grid(s, 0.45 * s[0], n) for s, n in zip(shapes, n_markers)]
    trajs = [inputs.FrameTrajectory(inputs.seed_for(2) + k, inputs.domain_centre(s)) for k, s in enumerate(shapes)]

    def make():
        d = fishlbm.Domain([fishlbm.env_desc(s, 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)) for s in shapes],
                           deterministic=True, variant=variant, layout=layout, ib_iters=ib_iters,
                           storage=storage)   # the deterministic spread: runs compare bit for bit
        for e, f in enumerate(fishes):
            X, U = f.pose(0)
            d.set_markers(np.float32(X), np.float32(U), np.float32(f.dV), seg=f.seg, n_seg=5,
                          ref=f.joints_rest[0], env=e)
        return d
    return fishes, trajs, make


@pytest.mark.parametrize("variant,layout,storage", [("plain", "pull", "f32"), ("staged", "pull", "f32"),
                                                    ("staged512", "pull", "f32"), ("plain", "aa", "f32"),
                                                    ("fused", "pull", "f32"), ("overlap", "pull", "f32"),
                                                    ("staged512", "pull", "f16"), ("plain", "aa", "bf16")])
def test_step_markers_equals_set_then_step(variant, layout, storage):
    """Seven steps of three environments (the markers kept unchanged on one
    step): force/torque rows after every step, then the populations, fields
    and marker forces, bit for bit against fg_set_markers_all + fg_step, with
    device arrays and with pinned host arrays, in FP32 and 16-bit storage."""
    torch = pytest.importorskip("torch")
    shapes = [(40, 24, 24), (48, 20, 28), (32, 32, 24)]
    fishes, trajs, make = _case(shapes, [300, 420, 260], variant, layout, storage=storage)
    ref, dev, pin = make(), make(), make()
    for n in range(1, 8):
        poses = [f.pose(n) for f in fishes]
        frames = [fishlbm.frame_from_array(t.at(n)) for t in trajs]
        Xall = np.concatenate([p[0] for p in poses]).astype(np.float32)
        Uall = np.concatenate([p[1] for p in poses]).astype(np.float32)
        if n == 4:   # this step keeps the previous markers
            ref.step(1, frames)
            dev.step_markers(None, None, frames)
            pin.step_markers(None, None, frames)
        else:
            ref.set_markers_all(Xall, Uall)
            ref.step(1, frames)
            Xd, Ud = torch.from_numpy(Xall).cuda(), torch.from_numpy(Uall).cuda()
            Xp, Up = torch.from_numpy(Xall).pin_memory(), torch.from_numpy(Uall).pin_memory()
            dev.step_markers(Xd, Ud, frames)
            pin.step_markers(Xp, Up, frames)
            torch.cuda.synchronize()   # the arrays stay unchanged until the step has run
        for e in range(len(shapes)):
            want = ref.get_body_force_torque(e)
            assert np.array_equal(dev.get_body_force_torque(e), want), (n, e)
            assert np.array_equal(pin.get_body_force_torque(e), want), (n, e)
    for e in range(len(shapes)):
        for d in (dev, pin):
            assert np.array_equal(d.populations(e), ref.populations(e))
            assert np.array_equal(d.marker_force(e), ref.marker_force(e))
    # a step without new markers after a posted one uses what that step copied
    frames = [fishlbm.frame_from_array(t.at(9)) for t in trajs]
    for d in (ref, dev, pin):
        d.step(1, frames)
    for e in range(len(shapes)):
        assert np.array_equal(dev.get_body_force_torque(e), ref.get_body_force_torque(e))
        assert np.array_equal(pin.get_body_force_torque(e), ref.get_body_force_torque(e))


@pytest.mark.parametrize("ib_iters", [1, 3])
def test_step_markers_more_markers_than_half_warps(ib_iters):
    """More markers than the IB kernel's half-warps (each walks several; the
    later ones reloaded from the domain's arrays the first phase filled),
    with one and three direct-forcing passes: device arrays are posted,
    pinned host arrays fall back to the copy; both equal set + step."""
    torch = pytest.importorskip("torch")
    shapes = [(96, 48, 48), (96, 48, 48), (96, 48, 48)]
    fishes, trajs, make = _case(shapes, [4000, 4000, 4000], "plain", ib_iters=ib_iters)
    ref, dev, pin = make(), make(), make()
    for n in range(1, 5):
        poses = [f.pose(n) for f in fishes]
        frames = [fishlbm.frame_from_array(t.at(n)) for t in trajs]
        Xall = np.concatenate([p[0] for p in poses]).astype(np.float32)
        Uall = np.concatenate([p[1] for p in poses]).astype(np.float32)
        ref.set_markers_all(Xall, Uall)
        ref.step(1, frames)
        dev.step_markers(torch.from_numpy(Xall).cuda(), torch.from_numpy(Uall).cuda(), frames)
        pin.step_markers(torch.from_numpy(Xall).pin_memory(), torch.from_numpy(Uall).pin_memory(), frames)
        torch.cuda.synchronize()
        for e in range(len(shapes)):
            want = ref.get_body_force_torque(e)
            assert np.array_equal(dev.get_body_force_torque(e), want), (n, e)
            assert np.array_equal(pin.get_body_force_torque(e), want), (n, e)
    for e in range(len(shapes)):
        for d in (dev, pin):
            assert np.array_equal(d.populations(e), ref.populations(e))


def test_step_markers_checks():
    """Refused calls launch and post nothing: a frame that is not finite,
    one array without the other, a wrong count; invalid host markers are
    refused like fg_set_markers_all's; invalid device markers are reported
    by the step (FG_ERR_INVALID when the force is read)."""
    torch = pytest.importorskip("torch")
    shapes = [(40, 24, 24)]
    fishes, trajs, make = _case(shapes, [300], "plain")
    ref, d = make(), make()
    X, U = (np.float32(v) for v in fishes[0].pose(1))
    bad = fishlbm.make_frame(acc=(float("nan"), 0.0, 0.0))
    with pytest.raises(fishlbm.FgError) as ei:
        d.step_markers(torch.from_numpy(X + 0.25).cuda(), torch.from_numpy(U).cuda(), [bad])
    assert ei.value.status == fishlbm.FG_ERR_INVALID
    with pytest.raises(ValueError):
        d.step_markers(X, None)
    with pytest.raises(ValueError):
        d.step_markers(X[:-1], U[:-1])
    Xo = X.copy()
    Xo[7, 0] = 0.5   # inside the open -x face's two-cell margin
    with pytest.raises(fishlbm.FgError) as ei:
        d.step_markers(torch.from_numpy(Xo).pin_memory(), torch.from_numpy(U).pin_memory())
    assert ei.value.status == fishlbm.FG_ERR_INVALID
    # nothing ran: the next posted step equals the reference's first step
    frames = [fishlbm.frame_from_array(trajs[0].at(1))]
    ref.set_markers_all(X, U)
    ref.step(1, frames)
    d.step_markers(torch.from_numpy(X).cuda(), torch.from_numpy(U).cuda(), frames)
    torch.cuda.synchronize()
    assert np.array_equal(d.get_body_force_torque(0), ref.get_body_force_torque(0))
    assert np.array_equal(d.populations(0), ref.populations(0))
    # an invalid device marker: the step reports it
    d.step_markers(torch.from_numpy(Xo).cuda(), torch.from_numpy(U).cuda(), frames)
    with pytest.raises(fishlbm.FgError):
        d.get_body_force_torque(0)
