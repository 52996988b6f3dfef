"""The in-place (AA) population layout: one population array updated in
place, against the plain kernel in the two-buffer pull layout and the FP64
oracle.

The AA kernels inline the plain kernel's per-cell arithmetic in the same
order; like the plain and staged kernels, they agree with it to rounding
(the compiler's choice of fused multiply-adds differs between kernels:
measured, single units in the last place of FP32 deviations).  The bars are
those of the kernel-variant agreement test.  Where the arithmetic is the
same kernel's (state access, region sums, the state-buffer format), the
tests compare bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import FREESLIP, OUTFLOW, PERIODIC, VELOCITY
from paper_2206_01683_b300 import fishlbm, inputs

from parity_util import TOL_F32, Pair, assert_local, rel_l2

pytestmark = pytest.mark.gpu

OPEN_X = (VELOCITY, OUTFLOW, FREESLIP, FREESLIP, FREESLIP, FREESLIP)
ALL_OPEN = (VELOCITY, OUTFLOW, FREESLIP, OUTFLOW, FREESLIP, FREESLIP)
# mass sums of the two layouts group FP32 partial sums differently: the
# difference is bounded by 1e-9 per cell (a block partial of <= 512 values
# of |rho - 1| < 0.05 rounds by < 2e-6; over N / 256 blocks that is < 1e-8 N
# in the worst case and about 1e-11 N for independent roundings)
TOL_MASS_PER_CELL = 1e-9


def _pair_of_domains(envs, **kw):
    """The plain kernel in the pull layout (the kernel whose in-place form
    the AA layout runs) and the AA layout."""
    return [fishlbm.Domain(envs, layout=lay, variant="plain", **kw) for lay in ("pull", "aa")]


def _assert_agree(ref, got, storage, where):
    """The populations of two kernels agree to rounding (the bars of the
    kernel-variant agreement test)."""
    cl, w = fishlbm.fg_lattice()
    g, r = got - w, ref - w
    if storage == "f32":
        assert rel_l2(g, r) < 1e-6 and np.abs(g - r).max() < 1e-7, where
    else:
        scale = 4.0 ** (1 + (cl ** 2).sum(axis=1))
        ulp = 2.0 ** -10 if storage == "f16" else 2.0 ** -7
        dh = np.abs(g - r) * scale
        hmax = np.abs(r * scale).max(axis=1, keepdims=True)
        assert (dh / (ulp * hmax + 2.0 ** -24)).max() <= 4.0, where
        assert np.mean(g != r) < 1e-2, where


def _assert_same(doms, n_envs, steps, where="", storage="f32"):
    a, b = doms
    for e in range(n_envs):
        _assert_agree(a.populations(env=e), b.populations(env=e), storage, (where, e))
        ra, ua = a.fields(env=e)
        rb, ub = b.fields(env=e)
        assert np.abs(ra - rb).max() < (1e-6 if storage == "f32" else 1e-3), (where, e)
        assert rel_l2(ub, ua) < (1e-5 if storage == "f32" else 2e-3), (where, e)
        if steps:
            ha, hb = a.history(steps, env=e), b.history(steps, env=e)
            assert rel_l2(hb[:, :-1], ha[:, :-1]) <= (1e-5 if storage == "f32" else 2e-3), (where, e)
            ncell = a.ncell(e)
            assert np.max(np.abs(ha[:, -1] - hb[:, -1])) <= TOL_MASS_PER_CELL * ncell * (
                1 if storage == "f32" else 1e3), (where, e)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("eq_order", [2, 3])
def test_aa_agrees_with_pull(storage, eq_order):
    """Three environments in one batch -- the swimmer channel with open faces
    and a moving frame (96x48x48), a periodic box with a sphere, a ragged
    grid with every face open and a rotating frame -- stepped 1, 2 and 11
    steps (both phases of the in-place layout, ending on either)."""
    fish = inputs.fish_for_grid((96, 48, 48), 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre((96, 48, 48)))
    envs = [fishlbm.env_desc((96, 48, 48), 0.52, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)),
            fishlbm.env_desc((40, 32, 24), 0.6),
            fishlbm.env_desc((37, 23, 11), 0.7, ALL_OPEN, (0.01, 0.0, 0.0), 1.002, (0.01, 0.0, 0.0))]
    Xs, dVs = inputs.fibonacci_sphere(200, 4.0, (20.0, 16.0, 12.0))
    Xr, dVr = inputs.fibonacci_sphere(60, 2.2, (18.0, 11.0, 5.5))
    rho, u = inputs.random_fields((37, 23, 11), seed=21, u_amp=0.01)
    doms = _pair_of_domains(envs, storage=storage, eq_order=eq_order, deterministic=True, record_history=16)
    for d in doms:
        d.init_fields(rho, u, env=2)
    n = 0
    for chunk in (1, 1, 9):
        for _ in range(chunk):
            X, U = fish.pose(n)
            Us = np.tile([0.02, -0.01 * math.sin(0.2 * n), 0.0], (200, 1))
            frames = [fishlbm.frame_from_array(traj.at(n)), fishlbm.make_frame(origin=(20, 16, 12)),
                      fishlbm.make_frame(acc=(1e-5, -2e-5, 5e-6), omega=(2e-4, -1e-4, 3e-4),
                                         domega=(1e-6, 2e-6, -1e-6), origin=(18.0, 11.0, 5.0))]
            for d in doms:
                d.set_markers(np.float32(X), np.float32(U), np.float32(fish.dV), seg=fish.seg, n_seg=5,
                              ref=fish.joints_rest[0], env=0)
                d.set_markers(np.float32(Xs + Us * n), np.float32(Us), np.float32(dVs), env=1)
                d.set_markers(np.float32(Xr), np.zeros((60, 3), np.float32), np.float32(dVr), env=2)
                d.step(1, frames)
            n += 1
        _assert_same(doms, 3, n, where="after %d steps" % n, storage=storage)
        for e in range(3):
            fa, fb = doms[0].marker_force(env=e), doms[1].marker_force(env=e)
            assert rel_l2(fb, fa) <= (1e-5 if storage == "f32" else 2e-3), (n, e)


@pytest.mark.parametrize("shape,faces", [
    ((3, 5, 4), (VELOCITY, OUTFLOW, PERIODIC, PERIODIC, FREESLIP, FREESLIP)),   # an open axis of 3 cells
    ((4, 3, 3), (OUTFLOW, OUTFLOW, FREESLIP, VELOCITY, OUTFLOW, FREESLIP)),     # three short open axes
    ((2, 1, 6), (PERIODIC, PERIODIC, PERIODIC, PERIODIC, VELOCITY, OUTFLOW)),   # periodic axes of 2 and 1
    ((1, 1, 1), (PERIODIC,) * 6),                                               # a single cell
    ((9, 7, 5), (VELOCITY, OUTFLOW, FREESLIP, FREESLIP, OUTFLOW, VELOCITY)),    # odd rows, every face open
])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_aa_small_and_degenerate_grids(shape, faces, storage):
    """Grids where one cell serves boundary cells on both sides of an axis,
    periodic axes shorter than the stencil, and a single cell: 1 and 6
    steps from seeded fields against the pull layout."""
    env = fishlbm.env_desc(shape, 0.8, faces, (0.01, -0.004, 0.006), 1.001, (0.0, 0.0, 0.0))
    rho, u = inputs.random_fields(shape, seed=7, u_amp=0.02)
    doms = _pair_of_domains([env], storage=storage, record_history=8)
    for d in doms:
        d.init_fields(rho, u)
    fr = fishlbm.make_frame(acc=(2e-5, 0, -1e-5), omega=(1e-4, 2e-4, 0), origin=(1.0, 1.0, 1.0))
    for steps in (1, 5):
        for d in doms:
            d.step(steps, [fr])
        _assert_same(doms, 1, 1 + (steps == 5) * 5, where=(shape, steps), storage=storage)


@pytest.mark.parametrize("steps", [149, 150])
def test_aa_swimmer_open_channel_against_oracle(steps):
    """The in-place layout against the FP64 oracle on the reduced swimmer
    channel (96x48x48, inlet/outflow/free-slip faces, moving frame, 900
    markers), ending on either phase: the FP32 bars of the pull layout."""
    shape = (96, 48, 48)
    fish = inputs.fish_for_grid(shape, 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    p = Pair(shape, 0.52, faces=OPEN_X, u_in=(0.02, 0.0, 0.0), layout="aa")
    p.init(None, np.tile([0.02, 0.0, 0.0], (p.o.ncell, 1)))
    for n in range(steps):
        X, U = fish.pose(n)
        p.markers(X, U, fish.dV, seg=fish.seg, nseg=5, ref=fish.joints_rest[0])
        p.step(traj.at(n))
    err = p.errors()
    for k in ("rho", "u", "pop", "force", "torque", "seg_force"):
        assert err[k] <= TOL_F32, (k, err)
    assert_local(err)


def test_aa_ragged_grid_rotating_frame_against_oracle():
    """37x23x11 (odd rows, one cell per thread), periodic x, free-slip y,
    inlet/outflow z, rotating and accelerating frame, markers across the
    periodic wrap, 61 steps."""
    shape = (37, 23, 11)
    faces = (PERIODIC, PERIODIC, FREESLIP, FREESLIP, VELOCITY, OUTFLOW)
    p = Pair(shape, 0.7, faces=faces, u_in=(0.005, 0.0, 0.01), rho0=1.002, layout="aa")
    rho, u = inputs.random_fields(shape, seed=21, u_amp=0.01)
    p.init(rho, u)
    X, dV = inputs.fibonacci_sphere(60, 2.2, (35.5, 11.0, 5.0))
    frame = oracle.make_frame(acc=(1e-5, -2e-5, 5e-6), omega=(2e-4, -1e-4, 3e-4),
                              domega=(1e-6, 2e-6, -1e-6), origin=(18.0, 11.0, 5.0))
    for n in range(61):
        p.markers(X + np.array([0.01 * n, 0.0, 0.0]), np.tile([0.01, 0.0, 0.0], (60, 1)), dV,
                  ref=(18.0, 11.0, 5.0))
        p.step(frame)
    err = p.errors()
    for k in ("rho", "u", "pop", "force", "torque"):
        assert err[k] <= TOL_F32, (k, err)
    assert_local(err)


def test_aa_state_buffers_cross_layouts_and_phases():
    """fg_save_state / fg_load_state / fg_copy_state use one format in both
    layouts: a state saved from either layout at either phase loads into the
    other unchanged and steps on as in the layout it came from (to
    rounding); set_populations / populations round-trip at both phases."""
    torch = pytest.importorskip("torch")
    shape = (24, 16, 12)
    env = fishlbm.env_desc(shape, 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0))
    rho, u = inputs.random_fields(shape, seed=3, u_amp=0.02)
    X, dV = inputs.fibonacci_sphere(50, 2.5, (12.0, 8.0, 6.0))
    U = np.tile([0.01, 0.0, 0.0], (50, 1)).astype(np.float32)

    def dom(layout):
        d = fishlbm.Domain([env], layout=layout, variant="plain", deterministic=True)
        d.init_fields(rho, u)
        d.set_markers(np.float32(X), U, np.float32(dV))
        return d

    for k in (3, 4):   # the in-place domain ends on phase 1, then on phase 0
        pull, aa = dom("pull"), dom("aa")
        pull.step(k)
        aa.step(k)
        s_pull, s_aa = pull.save_state(), aa.save_state()
        _assert_agree(pull.populations(), aa.populations(), "f32", k)
        for m in (1, 2):   # load into a domain of the other layout at either phase
            a2, p2 = dom("aa"), dom("pull")
            a2.step(m)
            p2.step(m)
            a2.load_state(s_pull)
            p2.load_state(s_aa)
            assert np.array_equal(a2.populations(), pull.populations()), (k, m)
            assert np.array_equal(p2.populations(), aa.populations()), (k, m)
            assert np.array_equal(a2.save_state(), s_pull) and np.array_equal(p2.save_state(), s_aa), (k, m)
            a2.step(3)
            p2.step(3)
            pull.step(3)
            aa.step(3)
            _assert_agree(pull.populations(), a2.populations(), "f32", (k, m))
            _assert_agree(aa.populations(), p2.populations(), "f32", (k, m))
            pull.load_state(s_pull)
            aa.load_state(s_aa)
        buf = torch.zeros(aa.state_bytes(), dtype=torch.uint8, device="cuda")
        aa.copy_state(buf, True)
        assert np.array_equal(buf.cpu().numpy(), s_aa), k
        other = dom("aa")
        other.step(1)
        other.copy_state(buf, False)
        assert np.array_equal(other.populations(), aa.populations()), k
        f = aa.populations()
        other.set_populations(f)
        assert np.array_equal(other.populations(), f), k


def test_aa_region_momentum_and_fields_match_pull():
    """The sphere-interior momentum sums and the macroscopic fields read the
    post-collision state where each phase keeps it: on the same state
    (loaded into both layouts) they equal the pull layout's bit for bit at
    both phases, including a sphere cut by an open face."""
    shape = (32, 24, 20)
    env = fishlbm.env_desc(shape, 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0))
    rho, u = inputs.random_fields(shape, seed=5, u_amp=0.02)
    doms = _pair_of_domains([env])
    for d in doms:
        d.init_fields(rho, u)
    for k in (1, 1, 1):
        for d in doms:
            d.step(k)
        doms[0].load_state(doms[1].save_state())   # the in-place domain's state in both
        for c, r in (((16.0, 12.0, 10.0), 5.0), ((1.5, 3.0, 18.5), 3.0)):
            a = doms[0].region_momentum(c, r)
            b = doms[1].region_momentum(c, r)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2], (c, r)
        ra, ua = doms[0].fields()
        rb, ub = doms[1].fields()
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub)


def test_aa_halves_population_memory_and_refuses_two_buffer_calls():
    """An in-place domain allocates one population array (the pull layout
    two): device memory taken at creation differs by one array.  The calls
    that need two buffers (fg_step_state, the adjoint) refuse it."""
    import torch
    shape = (128, 96, 96)
    env = fishlbm.env_desc(shape, 0.6)
    pop_bytes = 27 * 128 * 96 * 96 * 4
    torch.cuda.synchronize()
    taken = {}
    for lay in ("pull", "aa"):
        free0 = torch.cuda.mem_get_info()[0]
        d = fishlbm.Domain([env], layout=lay)
        torch.cuda.synchronize()
        taken[lay] = free0 - torch.cuda.mem_get_info()[0]
        d.close()
        torch.cuda.synchronize()
    saved = taken["pull"] - taken["aa"]
    assert abs(saved - pop_bytes) <= 0.02 * pop_bytes, (taken, pop_bytes)
    aa = fishlbm.Domain([fishlbm.env_desc((16, 16, 16), 0.6)], layout="aa")
    buf = torch.zeros(aa.state_bytes(), dtype=torch.uint8, device="cuda")
    buf2 = torch.zeros_like(buf)
    with pytest.raises(fishlbm.FgError):
        aa.step_state(buf, buf2)
    with pytest.raises(fishlbm.FgError):
        aa.adjoint_reset()
    assert aa.stream_collide_variant() == "plain"
    choice, _ = aa.autotune()
    assert choice == "plain"


def test_aa_options_step_io_slip_multi_pass():
    """The in-place layout under fg_step_io (pinned host markers), three
    direct-forcing passes and slip forcing, against the plain kernel in the
    pull layout (the variant bars) over 12 steps of the open swimmer
    channel."""
    torch = pytest.importorskip("torch")
    shape = (96, 48, 48)
    fish = inputs.fish_for_grid(shape, 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    env = fishlbm.env_desc(shape, 0.52, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0))
    for kw in (dict(ib_iters=3, deterministic=True), dict(slip=True, deterministic=True)):
        doms = _pair_of_domains([env], **kw)
        X0, U0 = fish.pose(0)
        normals = np.float32(np.asarray(X0) - np.asarray(X0).mean(axis=0))
        normals /= np.linalg.norm(normals, axis=1, keepdims=True)
        for d in doms:
            d.set_markers(np.float32(X0), np.float32(U0), np.float32(fish.dV), seg=fish.seg, n_seg=5,
                          ref=fish.joints_rest[0])
            if kw.get("slip"):
                d.set_marker_normals(normals)
        rows = [[], []]
        for n in range(12):
            X, U = fish.pose(n)
            Xh = torch.from_numpy(np.float32(X)).pin_memory()
            Uh = torch.from_numpy(np.float32(U)).pin_memory()
            for k, d in enumerate(doms):
                rows[k].append(d.step_io(Xh, Uh, [fishlbm.frame_from_array(traj.at(n))]))
        _assert_agree(doms[0].populations(), doms[1].populations(), "f32", kw)
        assert rel_l2(np.array(rows[1]), np.array(rows[0])) <= 1e-5, kw
