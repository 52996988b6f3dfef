"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Element-by-element comparisons on identical seeded inputs: populations,
density, velocity, per-step body force/torque and mass, at sizes the oracle
runs in seconds (several 256-cell blocks, ragged tails), the full-size
swimmer channel for a few steps from a seeded state, the batched form, and
the edge cases (no markers, a single cell, invalid markers, NaN input).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import FREESLIP, OUTFLOW, PERIODIC, VELOCITY
from paper_2206_01683_b300 import fishlbm, inputs

from parity_util import TOL_F32, Pair, assert_local, f32, rel_l2

pytestmark = pytest.mark.gpu
VARIANTS = ["plain", "staged", "staged512", "fused", "overlap"]

OPEN_X = (VELOCITY, OUTFLOW, FREESLIP, FREESLIP, FREESLIP, FREESLIP)


def assert_parity(err, tol=TOL_F32, keys=("rho", "u", "force")):
    for k in keys:
        if k in err:
            assert err[k] <= tol, (k, err)
    assert_local(err)


@pytest.mark.parametrize("variant", VARIANTS)
def test_taylor_green_periodic(variant):
    shape = (32, 24, 8)
    rho, u = inputs.taylor_green(shape, (0, 1), U0=0.02)
    r2, u2 = inputs.random_fields(shape, seed=3, u_amp=0.01, rho_amp=0.005)
    p = Pair(shape, 0.56, variant=variant)
    p.init(rho + r2 - 1.0, u + u2)
    for _ in range(100):
        p.step(record=False)
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop"))


@pytest.mark.parametrize("variant", VARIANTS)
def test_sphere_in_periodic_box_full_run(variant):
    """Rigid sphere (452 Fibonacci markers, R = 6) translating at 0.05 lu/step
    through a 48x32x32 periodic box at tau = 0.56, 200 steps."""
    cfg = inputs.SPHERE_BOX
    p = Pair(cfg["shape"], cfg["tau"], variant=variant)
    for n in range(cfg["steps"]):
        X, U, dV = inputs.translating_sphere(cfg["n_markers"], cfg["radius"], cfg["center"],
                                             cfg["velocity"], n)
        p.markers(X, U, dV)
        p.step()
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque"))
    assert err["mass"] < 1e-9
    drag = np.array([h[-1, 0] for h in p.force_hist_g])
    assert drag[-1] < 0          # the fluid resists the motion


def test_fixed_sphere_in_oncoming_flow_parity_and_frame_equivalence():
    """The fixed sphere in fluid that starts at -U against the oracle, and on
    the GPU the frame equivalence the oracle pins: its mean drag equals that
    of the sphere translating at U through fluid at rest."""
    shape, tau, U, nm = (48, 32, 32), 0.6, 0.02, 400
    c0 = np.array([20.0, 15.5, 15.5])
    X0, dV = inputs.fibonacci_sphere(nm, 5.0, c0)
    p = Pair(shape, tau)
    p.init(None, np.tile([-U, 0.0, 0.0], (p.o.ncell, 1)))
    moving = fishlbm.Domain([fishlbm.env_desc(shape, tau)])
    Fm = []
    for n in range(120):
        p.markers(X0, np.zeros((nm, 3)), dV)
        p.step()
        moving.set_markers(np.float32(X0 + np.array([U * n, 0.0, 0.0])), np.tile(np.float32([U, 0, 0]), (nm, 1)),
                           np.float32(dV))
        moving.step(1)
        Fm.append(moving.get_body_force_torque()[-1, 0])
    assert_parity(p.errors(), keys=("rho", "u", "pop", "force", "torque"))
    Ff = np.array([h[-1, 0] for h in p.force_hist_g])[40:]
    Fm = np.array(Fm[40:])
    assert abs(Fm.mean() - Ff.mean()) < 2e-4 * abs(Ff.mean())


def _fish_case(shape, tau, length, n_markers, steps, seed, amps=None, variant="auto", ib_iters=1):
    fish = inputs.fish_for_grid(shape, length, n_markers, amplitudes=amps)
    traj = inputs.FrameTrajectory(seed, inputs.domain_centre(shape))
    p = Pair(shape, tau, faces=OPEN_X, u_in=(0.02, 0.0, 0.0), variant=variant, ib_iters=ib_iters)
    p.init(None, np.tile([0.02, 0.0, 0.0], (p.o.ncell, 1)))
    ref = fish.joints_rest[0]
    for n in range(steps):
        X, U = fish.pose(n)
        p.markers(X, U, fish.dV, seg=fish.seg, nseg=5, ref=ref)
        p.step(traj.at(n))
    return p


@pytest.mark.parametrize("variant", VARIANTS)
def test_swimmer_open_channel_reduced(variant):
    """Skinned swimmer in the moving frame with inlet/outflow/free-slip faces
    (the full workload's physics at 96x48x48, body length 24, 900 markers)."""
    p = _fish_case((96, 48, 48), 0.52, 24.0, 900, 150, seed=inputs.seed_for(2), variant=variant)
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque", "seg_force"))


@pytest.mark.parametrize("M", [2, 3, 8])
def test_multi_direct_forcing_sphere_box(M):
    """Multi-direct forcing (M passes per step) on the translating sphere in
    the periodic box, 60 steps: populations, fields, forces and the marker
    forces against the oracle with the same M."""
    cfg = inputs.SPHERE_BOX
    p = Pair(cfg["shape"], cfg["tau"], ib_iters=M)
    for n in range(60):
        X, U, dV = inputs.translating_sphere(cfg["n_markers"], cfg["radius"], cfg["center"],
                                             cfg["velocity"], n)
        p.markers(X, U, dV)
        p.step()
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque"))
    Fo = p.o.marker_force()
    Fg = p.g.marker_force().astype(np.float64)
    assert rel_l2(Fg, Fo) <= TOL_F32


@pytest.mark.parametrize("variant", ["plain", "staged", "fused", "overlap"])
def test_multi_direct_forcing_swimmer_open_channel(variant):
    """Three passes on the skinned swimmer in the moving frame with open
    faces (96x48x48, 900 markers, 80 steps)."""
    p = _fish_case((96, 48, 48), 0.52, 24.0, 900, 80, seed=inputs.seed_for(2), variant=variant, ib_iters=3)
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque", "seg_force"))


def test_multi_direct_forcing_reduces_gpu_marker_slip():
    """On the GPU too, more passes leave less slip: the body force of the
    sphere's first step grows towards the converged value with M while the
    populations stay finite (steps taken from the same state)."""
    cfg = inputs.SPHERE_BOX
    X, U, dV = inputs.translating_sphere(cfg["n_markers"], cfg["radius"], cfg["center"], cfg["velocity"], 0)
    drag = []
    for M in (1, 2, 4, 8):
        d = fishlbm.Domain([fishlbm.env_desc(cfg["shape"], cfg["tau"])], ib_iters=M)
        d.set_markers(np.float32(X), np.float32(U), np.float32(dV))
        d.step(1)
        drag.append(-d.get_body_force_torque()[-1, 0])
    assert all(b > a for a, b in zip(drag, drag[1:])), drag


@pytest.mark.parametrize("M", [1, 3])
def test_deterministic_spread_parity(M):
    """The fixed-point (deterministic) spread against the oracle: sphere box,
    60 steps, one and three direct-forcing passes."""
    cfg = inputs.SPHERE_BOX
    p = Pair(cfg["shape"], cfg["tau"], ib_iters=M, deterministic=True)
    for n in range(60):
        X, U, dV = inputs.translating_sphere(cfg["n_markers"], cfg["radius"], cfg["center"],
                                             cfg["velocity"], n)
        p.markers(X, U, dV)
        p.step()
    assert_parity(p.errors(), keys=("rho", "u", "pop", "force", "torque"))


@pytest.mark.parametrize("variant", ["plain", "staged"])
def test_two_fish_school_parity(variant):
    """Two fish in tandem (one marker set, ten segments, each fish's segments
    about its own first joint) in an open channel with the leader's moving
    frame: 75x25x50, body length 18, 2 x 600 markers, 60 steps; fields,
    populations, the total and the ten per-segment force/torque rows."""
    shape = (75, 25, 50)
    school = inputs.School(shape, 18.0, 600, 27.0)
    traj = inputs.FrameTrajectory(inputs.seed_for(6), inputs.domain_centre(shape))
    p = Pair(shape, 0.52, faces=OPEN_X, u_in=(0.02, 0.0, 0.0), variant=variant)
    p.init(None, np.tile([0.02, 0.0, 0.0], (p.o.ncell, 1)))
    for n in range(60):
        X, U = school.pose(n)
        p.markers(X, U, school.dV, seg=school.seg, nseg=school.n_seg, ref=school.ref)
        if n == 0:
            p.o.set_segment_refs(school.seg_refs)
            p.g.set_segment_refs(school.seg_refs)
        p.step(traj.at(n))
    assert_parity(p.errors(), keys=("rho", "u", "pop", "force", "torque", "seg_force"))
    ft = p.g.get_body_force_torque()
    assert ft.shape == (11, 6)
    # per-fish sums of the segment rows give each fish's force
    lead, follow = ft[:5, :3].sum(axis=0), ft[5:10, :3].sum(axis=0)
    assert np.allclose(lead + follow, ft[10, :3], rtol=1e-5, atol=1e-9)


def test_segment_refs_validation_and_reset():
    d = fishlbm.Domain([fishlbm.env_desc((16, 16, 16), 0.7)])
    X, dV = inputs.fibonacci_sphere(60, 3.0, (8.0, 8.0, 8.0))
    seg = (np.arange(60) % 2).astype(np.int32)
    d.set_markers(np.float32(X), np.zeros((60, 3), np.float32), np.float32(dV), seg=seg, n_seg=2)
    with pytest.raises(fishlbm.FgError):
        d.set_segment_refs(np.zeros((3, 3)))               # one point per segment
    d.set_segment_refs(np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]]))
    d.set_segment_refs(None)
    d.step(1)


def test_maximum_segment_count_parity():
    """16 segments (the most a marker set may have), each with its own torque
    point: a rotating, translating sphere cut into 16 longitude sectors in the
    periodic box, 40 steps; every segment's force and torque row against the
    oracle."""
    cfg = inputs.SPHERE_BOX
    nseg = 16
    p = Pair(cfg["shape"], cfg["tau"])
    c0 = np.asarray(cfg["center"], dtype=np.float64)
    X0, dV = inputs.fibonacci_sphere(cfg["n_markers"], cfg["radius"], c0)
    phi = np.arctan2(X0[:, 1] - c0[1], X0[:, 0] - c0[0])
    seg = np.minimum(((phi + np.pi) / (2 * np.pi) * nseg).astype(np.int32), nseg - 1)
    assert set(seg.tolist()) == set(range(nseg))
    om = np.array([0.0, 0.0, 4e-3])
    v = np.asarray(cfg["velocity"], dtype=np.float64)
    for n in range(40):
        c = c0 + v * n
        X = X0 - c0 + c
        U = v + np.cross(om, X - c)
        p.markers(X, U, dV, seg=seg, nseg=nseg, ref=tuple(c))
        refs = np.array([c + 2.0 * np.array([np.cos(a), np.sin(a), 0.0])
                         for a in (np.arange(nseg) + 0.5) * 2 * np.pi / nseg - np.pi])
        p.o.set_segment_refs(f32(refs))
        p.g.set_segment_refs(f32(refs))
        p.step()
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque", "seg_force"))
    assert p.force_hist_g[-1].shape == (nseg + 1, 6)


def test_segment_count_and_ids_are_checked():
    d = fishlbm.Domain([fishlbm.env_desc((16, 16, 16), 0.7)])
    X, dV = inputs.fibonacci_sphere(40, 3.0, (8.0, 8.0, 8.0))
    X, U, dV = np.float32(X), np.zeros((40, 3), np.float32), np.float32(dV)
    for n_seg, seg in ((17, np.arange(40) % 17), (0, None), (4, np.full(40, 4)), (4, np.full(40, -1))):
        with pytest.raises(fishlbm.FgError) as ei:
            d.set_markers(X, U, dV, seg=None if seg is None else seg.astype(np.int32), n_seg=n_seg)
        assert ei.value.status == fishlbm.FG_ERR_INVALID
    d.set_markers(X, U, dV, seg=(np.arange(40) % 16).astype(np.int32), n_seg=16)
    d.step(1)
    assert d.get_body_force_torque().shape == (17, 6)
    # shapes the bare-pointer ABI cannot check are refused by the binding
    for bad in ((X[:, :2], U, dV), (X, U[:39], dV), (X, U, dV[:39])):
        with pytest.raises(ValueError):
            d.set_markers(*bad)
    with pytest.raises(ValueError):
        d.set_markers_all(X.reshape(-1), U.reshape(-1))


@pytest.mark.parametrize("M", [1, 3])
def test_slip_forcing_parity(M):
    """Slip (normal-only) forcing on the translating sphere in the periodic
    box, 60 steps, with the sphere's outward normals."""
    cfg = inputs.SPHERE_BOX
    p = Pair(cfg["shape"], cfg["tau"], ib_iters=M, slip=True)
    c0 = np.asarray(cfg["center"], dtype=np.float64)
    for n in range(60):
        X, U, dV = inputs.translating_sphere(cfg["n_markers"], cfg["radius"], cfg["center"],
                                             cfg["velocity"], n)
        centre = c0 + np.asarray(cfg["velocity"]) * n
        p.markers(X, U, dV, normals=X - centre)
        p.step()
    assert_parity(p.errors(), keys=("rho", "u", "pop", "force", "torque"))
    assert rel_l2(p.g.marker_force().astype(np.float64), p.o.marker_force()) <= TOL_F32


def test_slip_forcing_needs_normals():
    d = fishlbm.Domain([fishlbm.env_desc((16, 16, 16), 0.7)], slip=True)
    X, dV = inputs.fibonacci_sphere(60, 3.0, (8.0, 8.0, 8.0))
    d.set_markers(np.float32(X), np.zeros((60, 3), np.float32), np.float32(dV))
    with pytest.raises(fishlbm.FgError) as ei:
        d.step(1)
    assert ei.value.status == fishlbm.FG_ERR_STATE
    with pytest.raises(fishlbm.FgError):
        d.set_marker_normals(np.ones((59, 3), np.float32))        # wrong count
    d.set_marker_normals(np.float32((X - 8.0) / 3.0))
    d.step(1)
    d.set_markers(np.float32(X[:50]), np.zeros((50, 3), np.float32), np.float32(dV[:50]))
    with pytest.raises(fishlbm.FgError):                         # a new count drops the normals
        d.step(1)


def _swimmer_run(deterministic, ib_iters, steps=30, variant="staged"):
    shape = (96, 48, 48)
    fish = inputs.fish_for_grid(shape, 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    d = fishlbm.Domain([fishlbm.env_desc(shape, 0.52, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0))],
                       record_history=steps, variant=variant, ib_iters=ib_iters, deterministic=deterministic)
    for n in range(steps):
        X, U = fish.pose(n)
        d.set_markers(np.float32(X), np.float32(U), np.float32(fish.dV), seg=fish.seg, n_seg=5,
                      ref=fish.joints_rest[0])
        d.step(1, [fishlbm.frame_from_array(traj.at(n))])
    return d.populations(), d.history(steps)


@pytest.mark.parametrize("M", [1, 3])
def test_deterministic_spread_is_bit_reproducible(M):
    """Two fresh runs of the swimmer channel (30 steps, moving frame, open
    faces) with the deterministic spread give identical populations and force
    histories, bit for bit; they agree with the atomic spread to rounding."""
    f1, h1 = _swimmer_run(True, M)
    f2, h2 = _swimmer_run(True, M)
    assert np.array_equal(f1, f2)
    assert np.array_equal(h1, h2)
    fa, ha = _swimmer_run(False, M)
    assert rel_l2(f1, fa) < 1e-6
    assert rel_l2(h1, ha) < 1e-5


@pytest.mark.parametrize("variant", VARIANTS)
def test_ragged_grid_mixed_faces_rotating_frame(variant):
    """37x23x11 (rows padded to a pitch of 40, not a multiple of 32 or 256):
    periodic x, free-slip y walls, inlet at -z and outflow at +z, rotating +
    accelerating frame, markers straddling the periodic x wrap."""
    shape = (37, 23, 11)
    faces = (PERIODIC, PERIODIC, FREESLIP, FREESLIP, VELOCITY, OUTFLOW)
    p = Pair(shape, 0.7, faces=faces, u_in=(0.005, 0.0, 0.01), rho0=1.002, variant=variant)
    rho, u = inputs.random_fields(shape, seed=21, u_amp=0.01)
    p.init(rho, u)
    X, dV = inputs.fibonacci_sphere(60, 2.2, (35.5, 11.0, 5.0))   # straddles the x wrap
    frame = oracle.make_frame(acc=(1e-5, -2e-5, 5e-6), omega=(2e-4, -1e-4, 3e-4),
                              domega=(1e-6, 2e-6, -1e-6), origin=(18.0, 11.0, 5.0))
    for n in range(60):
        Xn = X + np.array([0.01 * n, 0.0, 0.0])
        p.markers(Xn, np.tile([0.01, 0.0, 0.0], (60, 1)), dV, ref=(18.0, 11.0, 5.0))
        p.step(frame)
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque"))


def test_full_size_swimmer_channel_few_steps():
    """The 256x128x128 swimmer channel (6000 markers, body length 64) in the
    launch configuration of the benchmark (automatic kernel choice: staged),
    3 steps from a seeded state."""
    cfg = inputs.FISH_CHANNEL
    shape = cfg["shape"]
    p = Pair(shape, cfg["tau"], faces=OPEN_X, u_in=(cfg["u_in"], 0.0, 0.0))
    rho, u = inputs.random_fields(shape, seed=inputs.seed_for(2), u_amp=0.02, rho_amp=0.004)
    u[:, 0] += cfg["u_in"]
    p.init(rho, u)
    fish = inputs.fish_for_grid(shape, cfg["length"], cfg["n_markers"])
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    for n in range(100, 103):
        X, U = fish.pose(n)
        p.markers(X, U, fish.dV, seg=fish.seg, nseg=5, ref=fish.joints_rest[0])
        p.step(traj.at(n))
    err = p.errors()
    assert_parity(err, keys=("rho", "u", "pop", "force", "torque", "seg_force"))


@pytest.mark.parametrize("variant", VARIANTS)
def test_batched_environments_match_separate_oracles(variant):
    shapes = [(40, 24, 24), (32, 32, 16), (21, 20, 28)]
    taus = [0.52, 0.6, 0.8]
    faces = [OPEN_X, (PERIODIC,) * 6, (PERIODIC, PERIODIC, FREESLIP, FREESLIP, PERIODIC, PERIODIC)]
    envs = [fishlbm.env_desc(s, t, f, f32((0.02, 0, 0))) for s, t, f in zip(shapes, taus, faces)]
    dom = fishlbm.Domain(envs, variant=variant)
    ors = [oracle.Oracle(s, t, faces=f, u_in=f32((0.02, 0, 0))) for s, t, f in zip(shapes, taus, faces)]
    from parity_util import gpu_to_oracle_perm
    perm = gpu_to_oracle_perm()
    marks = []
    for e, s in enumerate(shapes):
        X, dV = inputs.fibonacci_sphere(80 + 20 * e, 3.0, (s[0] / 2, s[1] / 2, s[2] / 2))
        U = np.tile([0.01 * (e + 1), 0.0, -0.005], (X.shape[0], 1))
        X32, U32, dV32 = (np.asarray(a, np.float32) for a in (X, U, dV))
        dom.set_markers(X32, U32, dV32, env=e)
        ors[e].set_markers(X32.astype(float), U32.astype(float), dV32.astype(float))
        marks.append(X.shape[0])
    trajs = [inputs.FrameTrajectory(100 + e, inputs.domain_centre(s)) for e, s in enumerate(shapes)]
    for n in range(40):
        frs = [f32(t.at(n)) for t in trajs]
        dom.step(1, [fishlbm.frame_from_array(f) for f in frs])
        for e in range(3):
            ors[e].step(frs[e])
    _, w = oracle.lattice()
    for e in range(3):
        ro, uo = ors[e].fields()
        rg, ug = dom.fields(env=e)
        assert rel_l2(rg, ro) <= TOL_F32 and rel_l2(ug, uo) <= TOL_F32, e
        fo = ors[e].populations() - w
        fg = dom.populations(env=e)[:, perm] - w
        assert rel_l2(fg, fo) <= TOL_F32, e
        assert rel_l2(dom.get_body_force_torque(env=e), ors[e].force_torque()) <= TOL_F32, e


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("even", [True, False])
def test_many_small_environments(variant, even):
    """96 small environments of four shapes and mixed faces in one domain
    (environment tables, binary searches, per-environment blocks and row
    groups; with every row length even the kernels take two cells per
    thread), each against its own oracle after 12 steps, two markers in
    every periodic environment."""
    rng = np.random.default_rng(inputs.seed_for(9))
    shapes_even = [(8, 8, 8), (10, 7, 6), (12, 5, 7), (16, 4, 4)]
    shapes = shapes_even if even else [(8, 8, 8), (9, 7, 6), (12, 5, 7), (15, 4, 4)]
    faces_set = [(PERIODIC,) * 6, OPEN_X, (PERIODIC, PERIODIC, FREESLIP, FREESLIP, PERIODIC, PERIODIC)]
    envs, ors, periodic_envs = [], [], []
    for e in range(96):
        sh = shapes[int(rng.integers(0, 4))]
        fc = faces_set[int(rng.integers(0, 3))]
        if fc == faces_set[0]:
            periodic_envs.append(e)
        tau = float(rng.uniform(0.55, 0.9))
        envs.append(fishlbm.env_desc(sh, tau, fc, f32((0.01, 0, 0)), 1.0, f32((0.01, 0, 0))))
        o = oracle.Oracle(sh, tau, faces=fc, u_in=f32((0.01, 0, 0)))
        o.init_fields(None, np.tile(f32((0.01, 0, 0)), (o.ncell, 1)))
        ors.append(o)
    dom = fishlbm.Domain(envs, variant=variant)
    for e in periodic_envs:
        X = f32(np.array([[3.3, 3.1, 2.6], [4.2, 2.7, 2.4]]))
        U = f32(np.array([[0.01, 0.0, 0.0], [0.0, 0.005, 0.0]]))
        dV = f32(np.array([1.0, 1.0]))
        dom.set_markers(np.float32(X), np.float32(U), np.float32(dV), env=e)
        ors[e].set_markers(X, U, dV)
    for n in range(12):
        dom.step(1)
        for o in ors:
            o.step()
    for e in range(96):
        ro, uo = ors[e].fields()
        rg, ug = dom.fields(env=e)
        assert rel_l2(rg, ro) <= TOL_F32 and rel_l2(ug, uo) <= TOL_F32, (e, rel_l2(ug, uo))
    dom.get_body_force_torque(env=0)


def test_environment_tables_beyond_shared_memory():
    """140 environments, more than the IB kernel keeps in shared memory (it
    then reads the environment tables and frames from global memory), give
    exactly what the same environments give as two domains of 70 (tables in
    shared memory): deterministic spread, markers in every environment, ten
    steps in a moving frame, populations and force/torque rows bit for bit."""
    rng = np.random.default_rng(inputs.seed_for(10))
    shapes = [(8, 8, 8), (10, 8, 6), (12, 6, 8)]
    envs, marks, frames = [], [], []
    for e in range(140):
        sh = shapes[int(rng.integers(0, 3))]
        envs.append(fishlbm.env_desc(sh, float(rng.uniform(0.55, 0.9)), (PERIODIC,) * 6, (0.0, 0.0, 0.0), 1.0,
                                     f32((0.01, 0, 0))))
        c = np.array(sh, float) / 2.0 + rng.uniform(-0.5, 0.5, 3)
        X = f32(c + np.array([[0.4, 0.1, -0.3], [-0.6, 0.2, 0.5], [0.1, -0.7, 0.2]]))
        U = f32(rng.uniform(-0.01, 0.01, (3, 3)))
        marks.append((X, U, f32(np.ones(3))))
        frames.append(fishlbm.make_frame(acc=tuple(rng.uniform(-1e-5, 1e-5, 3)), omega=(0.0, 0.0, 1e-4)))
    one = fishlbm.Domain(envs, deterministic=True)
    halves = [fishlbm.Domain(envs[:70], deterministic=True), fishlbm.Domain(envs[70:], deterministic=True)]
    for e, (X, U, dV) in enumerate(marks):
        one.set_markers(X, U, dV, env=e)
        halves[e // 70].set_markers(X, U, dV, env=e % 70)
    for n in range(10):
        one.step(1, frames)
        halves[0].step(1, frames[:70])
        halves[1].step(1, frames[70:])
    for e in range(140):
        h, k = halves[e // 70], e % 70
        assert np.array_equal(one.get_body_force_torque(e), h.get_body_force_torque(k)), e
        assert np.array_equal(one.populations(e), h.populations(k)), e


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("variant", VARIANTS)
def test_no_markers_and_single_cell(variant):
    for shape in ((1, 1, 1), (2, 1, 1), (1, 3, 2), (9, 1, 1)):
        p = Pair(shape, 0.8, variant=variant)
        rho, u = inputs.random_fields(shape, seed=5)
        p.init(rho, u)
        for _ in range(5):
            p.step(oracle.make_frame(acc=(1e-4, 0, 0)), record=False)
        err = p.errors()
        assert_parity(err, keys=("rho", "u", "pop"))
        assert np.all(p.g.get_body_force_torque() == 0.0)


def test_host_marker_validation():
    d = fishlbm.Domain([fishlbm.env_desc((16, 12, 12), 0.7, OPEN_X)])
    bad = np.array([[1.5, 6.0, 6.0]], np.float32)
    with pytest.raises(fishlbm.FgError) as ei:
        d.set_markers(bad, np.zeros_like(bad), np.ones(1, np.float32))
    assert ei.value.status == fishlbm.FG_ERR_INVALID
    with pytest.raises(fishlbm.FgError):
        d.set_markers(np.array([[5, 6, 6]], np.float32), np.zeros((1, 3), np.float32),
                      np.ones(1, np.float32), seg=np.array([3], np.int32), n_seg=2)


def test_device_marker_outside_domain_is_skipped_and_reported():
    torch = pytest.importorskip("torch")
    d = fishlbm.Domain([fishlbm.env_desc((16, 12, 12), 0.7, OPEN_X)])
    X = torch.tensor([[6.0, 6.0, 6.0], [14.0, 6.0, 6.0]], device="cuda")   # second is too close to +x
    U = torch.zeros_like(X)
    dV = torch.ones(2, device="cuda")
    d.set_markers(X, U, dV)
    d.step(1)
    with pytest.raises(fishlbm.FgError) as ei:
        d.get_body_force_torque()
    assert ei.value.status == fishlbm.FG_ERR_INVALID
    assert np.all(d.marker_force()[1] == 0.0)
    d.set_markers(X[:1].contiguous(), U[:1].contiguous(), dV[:1].contiguous())
    d.step(1)
    d.get_body_force_torque()        # usable again


def test_numeric_watchdog_poison_and_reset():
    d = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7)])
    rho = np.ones(512)
    rho[77] = np.nan
    d.init_fields(rho, None)
    d.step(1)
    with pytest.raises(fishlbm.FgError) as ei:
        d.get_body_force_torque()
    assert ei.value.status == fishlbm.FG_ERR_NUMERIC
    with pytest.raises(fishlbm.FgError) as ei:
        d.step(1)
    assert ei.value.status == fishlbm.FG_ERR_STATE
    d.init_fields(None, None)
    d.step(2)
    d.get_body_force_torque()
    assert abs(d.mass() - 512.0) < 1e-9


def test_mass_drift_watchdog():
    """fg_watch_mass: a periodic box with a translating sphere conserves mass
    to rounding, so a tight watch stays quiet for 60 steps; mass injected
    into the state trips it (FG_ERR_NUMERIC, domain poisoned); switched off,
    the same injection passes; an open channel passes a tolerance that bounds
    its net inflow."""
    cfg = inputs.SPHERE_BOX
    d = fishlbm.Domain([fishlbm.env_desc(cfg["shape"], cfg["tau"])])
    d.step(1)
    d.watch_mass(1e-9)
    m0 = d.mass()
    for n in range(60):
        X, U, dV = inputs.translating_sphere(cfg["n_markers"], cfg["radius"], cfg["center"], cfg["velocity"], n)
        d.set_markers(np.float32(X), np.float32(U), np.float32(dV))
        d.step(1)
    d.get_body_force_torque()
    assert abs(d.mass() - m0) <= 1e-9 * m0
    f = d.populations()
    f[:, 13] += 1e-6                      # +1e-6 per cell in the rest population: relative drift 1e-6
    d.set_populations(f)
    d.step(1)
    with pytest.raises(fishlbm.FgError) as ei:
        d.get_body_force_torque()
    assert ei.value.status == fishlbm.FG_ERR_NUMERIC and "mass" in str(ei.value)
    with pytest.raises(fishlbm.FgError) as ei:
        d.step(1)
    assert ei.value.status == fishlbm.FG_ERR_STATE
    d.watch_mass(0.0)
    d.init_fields(None, None)
    d.set_populations(f)
    d.step(2)
    d.get_body_force_torque()
    ch = fishlbm.Domain([fishlbm.env_desc((48, 24, 24), 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0))])
    ch.step(1)
    ch.watch_mass(0.05)
    ch.step(50)
    ch.get_body_force_torque()
    with pytest.raises(fishlbm.FgError):
        ch.watch_mass(float("nan"))


def test_out_of_memory_paths_leave_domains_usable():
    """With a per-allocation cap (fg_set_alloc_cap) standing in for a full
    device: creating a domain whose population buffers exceed it fails with
    FG_ERR_OOM and frees what it had allocated; growing a live domain's
    marker buffers past it fails with FG_ERR_OOM and leaves the domain's
    markers and state as they were, so it steps on exactly like a twin that
    never saw the failure."""
    torch = pytest.importorskip("torch")
    shape = (64, 64, 64)
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        fishlbm.set_alloc_cap(1 << 20)
        with pytest.raises(fishlbm.FgError) as ei:
            fishlbm.Domain([fishlbm.env_desc(shape, 0.6)])
        assert ei.value.status == fishlbm.FG_ERR_OOM
        torch.cuda.synchronize()
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
        fishlbm.set_alloc_cap(0)
        a, b = (fishlbm.Domain([fishlbm.env_desc((32, 24, 20), 0.6)], deterministic=True) for _ in range(2))
        X, dV = inputs.fibonacci_sphere(100, 4.0, (16, 12, 10))
        U = np.tile(np.float32([0.01, 0, 0]), (100, 1))
        for d in (a, b):
            d.set_markers(np.float32(X), U, np.float32(dV))
            d.step(2)
        fishlbm.set_alloc_cap(16 << 10)
        X2, dV2 = inputs.fibonacci_sphere(20000, 6.0, (16, 12, 10))
        with pytest.raises(fishlbm.FgError) as ei:
            b.set_markers(np.float32(X2), np.tile(np.float32([0.01, 0, 0]), (20000, 1)), np.float32(dV2))
        assert ei.value.status == fishlbm.FG_ERR_OOM
    finally:
        fishlbm.set_alloc_cap(0)
    for d in (a, b):
        d.step(3)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.get_body_force_torque(), b.get_body_force_torque())


def test_history_checkpoint_and_profile():
    shape = (24, 16, 16)
    d = fishlbm.Domain([fishlbm.env_desc(shape, 0.6)], record_history=8)
    X, dV = inputs.fibonacci_sphere(100, 3.0, (12, 8, 8))
    d.set_markers(np.float32(X), np.float32(np.tile([0.02, 0, 0], (100, 1))), np.float32(dV))
    d.profile(True)
    forces = []
    for _ in range(12):
        d.step(1)
        forces.append(d.get_body_force_torque()[-1].copy())
    ms, n = d.profile_read()
    assert n[fishlbm.FG_K_IB] == 12 and n[fishlbm.FG_K_STREAM_COLLIDE] == 12 and n[fishlbm.FG_K_REDUCE] == 12
    assert np.all(ms > 0)
    h = d.history(100)
    assert h.shape == (8, 13)
    assert np.allclose(h[:, :6 * 2][:, 6:], np.array(forces[-8:]), rtol=0, atol=0)
    assert np.all(np.abs(h[:, -1] - d.mass()) < 1e-6)
    snap = d.save_state()
    d.step(5)
    a = d.populations()
    d.load_state(snap)
    d.step(5)
    b = d.populations()
    assert np.max(np.abs(a - b)) < 1e-6
    assert d.step_count() == 22


def test_long_rows_fall_back_to_plain_and_staged_rejects_them():
    """Rows longer than 512 cells go to the plain kernel under AUTO; asking
    for the staged kernel explicitly is an argument error."""
    e = fishlbm.env_desc((600, 4, 3), 0.7)
    d = fishlbm.Domain([e])          # AUTO -> plain
    d.step(2)
    d.get_body_force_torque()
    with pytest.raises(fishlbm.FgError) as ei:
        fishlbm.Domain([e], variant="staged")
    assert ei.value.status == fishlbm.FG_ERR_INVALID


def test_long_rows_parity():
    p = Pair((520, 5, 4), 0.6)
    rho, u = inputs.random_fields((520, 5, 4), seed=31)
    p.init(rho, u)
    for _ in range(10):
        p.step(oracle.make_frame(acc=(1e-5, 0, 0), omega=(0, 0, 1e-4), origin=(260, 2, 1.5)), record=False)
    assert_parity(p.errors(), keys=("rho", "u", "pop"))


def test_graph_replay_matches_direct_launches():
    """The same steps replayed from captured graphs and launched directly give
    identical states (no markers: every kernel is then deterministic), and
    with markers agree to rounding; the step counter and history advance the
    same way."""
    shape = (40, 24, 20)
    rho, u = inputs.random_fields(shape, seed=41)
    frame = fishlbm.make_frame(acc=(1e-5, 0, 0), omega=(0, 1e-4, 0), origin=(20, 12, 10))
    doms = [fishlbm.Domain([fishlbm.env_desc(shape, 0.6)], graphs=g, record_history=16) for g in (True, False)]
    for d in doms:
        d.init_fields(rho, u)
        d.step(7, [frame])
    assert np.array_equal(doms[0].populations(), doms[1].populations())
    X, dV = inputs.fibonacci_sphere(200, 4.0, (20, 12, 10))
    U = np.tile([0.01, 0.0, 0.0], (200, 1))
    for d in doms:
        for n in range(9):
            d.set_markers(np.float32(X + U * n), np.float32(U), np.float32(dV))
            d.step(1, [frame])
    assert rel_l2(doms[0].populations(), doms[1].populations()) < 1e-9
    assert doms[0].step_count() == doms[1].step_count() == 16
    h0, h1 = doms[0].history(16), doms[1].history(16)
    assert h0.shape == h1.shape == (16, 13)
    assert rel_l2(h0, h1) < 1e-6


@pytest.mark.parametrize("storage", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("nx", [64, 63])
def test_stream_collide_variants_agree(storage, nx):
    """The plain and staged stream-collide kernels agree to rounding, with
    two neighbouring cells per thread where every row length is even (nx =
    64: the plain kernel in every storage, the staged kernels with 16-bit
    storage) and one otherwise (nx = 63).  The kernels inline the same
    per-cell arithmetic, and the compiler's choice of fused multiply-adds
    may differ between them (measured: FP32 deviations differ by at most a
    few 1e-9, FP16 stores in about 1e-4 of the entries).  Open x faces, a
    moving frame, markers with the deterministic spread, 12 steps."""
    shape = (nx, 20, 18)
    rho, u = inputs.random_fields(shape, seed=61, u_amp=0.02, rho_amp=0.01)
    c = np.array([nx / 2.0, 10.0, 9.0])
    X0, dV = inputs.fibonacci_sphere(150, 4.0, c)
    frame = fishlbm.make_frame(acc=(1e-5, 2e-6, 0.0), omega=(0.0, 1e-4, 2e-4), domega=(1e-6, 0.0, 0.0),
                               origin=tuple(c))
    doms = [fishlbm.Domain([fishlbm.env_desc(shape, 0.56, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0))],
                           storage=storage, variant=v, deterministic=True) for v in ("plain", "staged", "staged512")]
    for d in doms:
        d.init_fields(rho, u)
    for n in range(12):
        U = np.tile([0.01, 0.003 * math.sin(0.3 * n), 0.0], (150, 1))
        for d in doms:
            d.set_markers(np.float32(X0 + U * n), np.float32(U), np.float32(dV))
            d.step(1, [frame])
    cl, w = fishlbm.fg_lattice()                   # library velocity order
    scale = 4.0 ** (1 + (cl ** 2).sum(axis=1))     # the 16-bit stores keep s_i g_i
    ref = doms[0].populations() - w
    for d in doms[1:]:
        g = d.populations() - w
        v = d.stream_collide_variant()
        if storage == "f32":
            assert rel_l2(g, ref) < 1e-6 and np.abs(g - ref).max() < 1e-7, v
        else:
            # the stored values s_i g_i differ by at most a few units in the
            # last place of the cell's largest stored value (a rounding of a
            # moment moves every output of the cell), in a small fraction of
            # the entries; one unit is 2^-10 (FP16) or 2^-7 (BF16) relative
            ulp = 2.0 ** -10 if storage == "f16" else 2.0 ** -7
            dh = np.abs(g - ref) * scale
            hmax = np.abs(ref * scale).max(axis=1, keepdims=True)
            ratio = (dh / (ulp * hmax + 2.0 ** -24)).max()
            assert ratio <= 4.0, (v, float(ratio))
            assert np.mean(g != ref) < 1e-2, (v, float(np.mean(g != ref)))


def test_autotune_keeps_a_runnable_variant_and_the_state():
    """The autotuner times the candidates on the domain's own buffers without
    changing the state, keeps the fastest (a staged variant by a margin of
    more than 2%), and steps continue identically."""
    shape = (96, 40, 24)
    rho, u = inputs.random_fields(shape, seed=51)
    a = fishlbm.Domain([fishlbm.env_desc(shape, 0.6)], variant="plain")
    b = fishlbm.Domain([fishlbm.env_desc(shape, 0.6)])
    for d in (a, b):
        d.init_fields(rho, u)
        d.step(3)
    before = b.populations()
    kept, ms = b.autotune()
    assert set(ms) == {"plain", "staged256", "staged512", "fused", "overlap"} and all(v > 0 for v in ms.values())
    # a staged variant is kept only when more than 2% faster than the plain one
    score = {k: (v / 0.98 if k.startswith("staged") else v) for k, v in ms.items()}
    assert kept == min(score, key=score.get) == b.stream_collide_variant()
    assert np.array_equal(b.populations(), before)
    for d in (a, b):
        d.step(4)
    assert rel_l2(b.populations(), a.populations()) < 1e-6
    big = fishlbm.Domain([fishlbm.env_desc((300, 4, 4), 0.6)], autotune=True)
    big.step(1)   # the autotune option runs before the first step
    assert big.stream_collide_variant() in ("plain", "staged512", "fused", "overlap")


def test_region_momentum_matches_oracle():
    """fg_region_momentum against the oracle on a seeded state, for a sphere
    straddling the periodic x faces and one cut by the open faces of a
    channel."""
    shape = (40, 24, 20)
    rho, u = inputs.random_fields(shape, seed=41, u_amp=0.03, rho_amp=0.01)
    for faces in ((PERIODIC,) * 6, OPEN_X):
        p = Pair(shape, 0.7, faces=faces, u_in=(0.02, 0.0, 0.0))
        p.init(rho, u)
        for c, R in (((1.3, 11.7, 9.6), 5.2), ((20.4, 12.0, 10.1), 7.9), ((38.2, 3.0, 17.5), 4.0)):
            Po, Lo, ao = p.o.region_momentum(c, R)
            Pg, Lg, ag = p.g.region_momentum(c, R)
            assert abs(ag - ao) <= 1e-6 * ao
            assert np.linalg.norm(Pg - Po) <= 1e-5 * np.linalg.norm(Po) + 1e-12
            assert np.linalg.norm(Lg - Lo) <= 1e-5 * np.linalg.norm(Lo) + 1e-12


def test_free_sphere_matches_oracle_reference():
    """The library's free sphere (rigid.FreeSphere) against the oracle's
    reference integrator on a 24^3 periodic box: density ratio 1.08, skewed
    gravity, 120 steps; centre, velocity and spin agree."""
    from oracle.rigid import OracleFreeSphere
    from paper_2206_01683_b300 import rigid
    L, R, g = 24, 4.0, np.array([2e-4, -3e-4, -1e-3])
    c0 = (11.3, 12.1, 10.7)
    d = fishlbm.Domain([fishlbm.env_desc((L, L, L), 1.0)])
    s_g = rigid.FreeSphere(d, R, c0, 1.08, g)
    o = oracle.Oracle((L, L, L), 1.0)
    N = s_g.dirs
    s_o = OracleFreeSphere(o, N, s_g.dV.astype(np.float64), R, c0, 1.08, g)
    for _ in range(120):
        s_g.step()
        s_o.step()
    assert np.linalg.norm(s_g.vel - s_o.V) <= 2e-4 * np.linalg.norm(s_o.V)
    assert np.linalg.norm(s_g.centre - s_o.c) <= 1e-6 * L
    assert np.linalg.norm(s_g.spin - s_o.W) <= 2e-3 * np.linalg.norm(s_o.W) + 1e-10


def test_set_markers_all_equals_per_environment_updates():
    """One fg_set_markers_all call (device and host arrays) moves the markers
    of three environments exactly as three fg_set_markers calls do."""
    torch = pytest.importorskip("torch")
    shapes = [(32, 24, 20), (40, 16, 24), (24, 24, 24)]
    fishes = [inputs.fish_for_grid(s, 0.4 * s[0], 300 + 50 * k) for k, s in enumerate(shapes)]

    def make():
        d = fishlbm.Domain([fishlbm.env_desc(s, 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)) for s in shapes],
                           deterministic=True)   # bit-reproducible, so the runs compare exactly
        for e, f in enumerate(fishes):
            X, U = f.pose(0)
            d.set_markers(np.float32(X), np.float32(U), np.float32(f.dV), seg=f.seg, n_seg=5,
                          ref=f.joints_rest[0], env=e)
        return d

    a, b, c = make(), make(), make()
    for n in range(1, 6):
        poses = [f.pose(n) for f in fishes]
        for e, f in enumerate(fishes):
            a.set_markers(np.float32(poses[e][0]), np.float32(poses[e][1]), None, None, n_seg=5,
                          ref=f.joints_rest[0], env=e)
        Xall = np.concatenate([p[0] for p in poses]).astype(np.float32)
        Uall = np.concatenate([p[1] for p in poses]).astype(np.float32)
        b.set_markers_all(torch.from_numpy(Xall).cuda(), torch.from_numpy(Uall).cuda())
        c.set_markers_all(Xall, Uall)
        for d in (a, b, c):
            d.step(1)
    for e in range(3):
        fa = a.populations(e)
        assert np.array_equal(fa, b.populations(e)) and np.array_equal(fa, c.populations(e))
        assert np.array_equal(a.get_body_force_torque(e), b.get_body_force_torque(e))
    with pytest.raises(fishlbm.FgError):
        b.set_markers_all(Xall[:-1], Uall[:-1])             # wrong total


@pytest.mark.parametrize("n_envs", [1, 3])
def test_step_io_equals_separate_calls(n_envs):
    """fg_step_io (markers in, one step, force/torque out, one call) gives
    exactly what fg_set_markers_all + fg_step + fg_get_body_force_torque
    give, with pageable, pinned and device marker arrays, for one environment
    and for three, and so do per-environment fg_set_markers calls with pinned
    arrays (read in place by the copy kernel); a failing check (a frame that
    is not finite) launches nothing, so the steps that follow are
    unchanged."""
    torch = pytest.importorskip("torch")
    shapes = [(32, 24, 20), (40, 16, 24), (24, 24, 24)][:n_envs]
    fishes = [inputs.fish_for_grid(s, 0.4 * s[0], 300 + 50 * k) for k, s in enumerate(shapes)]
    trajs = [inputs.FrameTrajectory(inputs.seed_for(2) + k, inputs.domain_centre(s)) for k, s in enumerate(shapes)]

    def make():
        d = fishlbm.Domain([fishlbm.env_desc(s, 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)) for s in shapes],
                           deterministic=True)   # bit-reproducible, so the runs compare exactly
        for e, f in enumerate(fishes):
            X, U = f.pose(0)
            d.set_markers(np.float32(X), np.float32(U), np.float32(f.dV), seg=f.seg, n_seg=5,
                          ref=f.joints_rest[0], env=e)
        return d

    a, b, c, p, q = make(), make(), make(), make(), make()
    bad = fishlbm.make_frame(acc=(float("nan"), 0.0, 0.0))
    for n in range(1, 6):
        poses = [f.pose(n) for f in fishes]
        frames = [fishlbm.frame_from_array(t.at(n)) for t in trajs]
        Xall = np.concatenate([p[0] for p in poses]).astype(np.float32)
        Uall = np.concatenate([p[1] for p in poses]).astype(np.float32)
        keep = n == 3   # this step keeps the previous markers
        if not keep:
            a.set_markers_all(Xall, Uall)
        a.step(1, frames)
        ref = [a.get_body_force_torque(e) for e in range(n_envs)]
        if keep:
            # valid markers with a bad frame: refused before any copy
            with pytest.raises(fishlbm.FgError) as ei:
                b.step_io(Xall + 0.25, Uall, [bad] * n_envs)
            assert ei.value.status == fishlbm.FG_ERR_INVALID
            got_b, got_c = b.step_io(None, None, frames), c.step_io(None, None, frames)
            got_p = p.step_io(None, None, frames)
        else:
            got_b = b.step_io(Xall, Uall, frames)
            got_c = c.step_io(torch.from_numpy(Xall).cuda(), torch.from_numpy(Uall).cuda(), frames)
            got_p = p.step_io(torch.from_numpy(Xall).pin_memory(), torch.from_numpy(Uall).pin_memory(), frames)
            for e, f in enumerate(fishes):
                q.set_markers(torch.from_numpy(np.float32(poses[e][0])).pin_memory(),
                              torch.from_numpy(np.float32(poses[e][1])).pin_memory(), None, None, n_seg=5,
                              ref=f.joints_rest[0], env=e)
        q.step(1, frames)
        got_q = [q.get_body_force_torque(e) for e in range(n_envs)]
        if n_envs == 1:
            got_b, got_c, got_p = [got_b], [got_c], [got_p]
        for e in range(n_envs):
            assert got_b[e].shape == (6, 6)
            for got in (got_b, got_c, got_p, got_q):
                assert np.array_equal(got[e], ref[e])
    for e in range(n_envs):
        for d in (b, c, p, q):
            assert np.array_equal(a.populations(e), d.populations(e))
    with pytest.raises(ValueError):
        b.step_io(Xall, None)
    with pytest.raises(ValueError):
        b.step_io(Xall[:-1], Uall[:-1])                    # the binding checks the marker count


@pytest.mark.parametrize("variant", ["plain", "staged"])
def test_third_order_equilibrium_parity(variant):
    """eq_order = 3 against the oracle: a perturbed Taylor-Green field with a
    uniform carrier velocity (periodic, 100 steps) and the swimmer channel
    (open faces, moving frame, 60 steps)."""
    shape = (32, 24, 8)
    rho, u = inputs.taylor_green(shape, (0, 1), U0=0.02)
    r2, u2 = inputs.random_fields(shape, seed=13, u_amp=0.01, rho_amp=0.005)
    p = Pair(shape, 0.56, variant=variant, eq_order=3)
    p.init(rho + r2 - 1.0, u + u2 + np.array([0.05, -0.03, 0.02]))
    for _ in range(100):
        p.step(record=False)
    assert_parity(p.errors(), keys=("rho", "u", "pop"))
    fish = inputs.fish_for_grid((96, 48, 48), 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre((96, 48, 48)))
    p = Pair((96, 48, 48), 0.52, faces=OPEN_X, u_in=(0.02, 0.0, 0.0), variant=variant, eq_order=3)
    p.init(None, np.tile([0.02, 0.0, 0.0], (p.o.ncell, 1)))
    for n in range(60):
        X, U = fish.pose(n)
        p.markers(X, U, fish.dV, seg=fish.seg, nseg=5, ref=fish.joints_rest[0])
        p.step(traj.at(n))
    assert_parity(p.errors(), keys=("rho", "u", "pop", "force", "torque", "seg_force"))


def test_third_order_equilibrium_galilean_shear_on_gpu():
    """The advected shear wave of the oracle pin, on the GPU: with eq_order = 3
    the decay rate at U0 = 0.1 equals the one at rest; with 2 it drops by
    about 3 U0^2."""
    L, tau, steps = 64, 0.8, 400

    def rate(order, U0):
        d = fishlbm.Domain([fishlbm.env_desc((L, 4, 4), tau)], eq_order=order)
        n = L * 16
        x = np.tile(np.arange(L), 16).astype(float)
        u = np.zeros((n, 3))
        u[:, 0] = U0
        u[:, 1] = 1e-3 * np.sin(2 * math.pi * x / L)
        d.init_fields(np.ones(n), u)

        def amp():
            _, uu = d.fields()
            return abs(np.fft.rfft(uu[:, 1].reshape(4, 4, L).mean(axis=(0, 1)))[1])

        a0 = amp()
        d.step(steps)
        nu, k = (tau - 0.5) / 3.0, 2 * math.pi / L
        return -math.log(amp() / a0) / steps / (nu * k * k)

    r0 = rate(3, 0.0)
    assert abs(rate(3, 0.1) - r0) < 2e-4 * r0
    assert abs((rate(2, 0.1) - r0) / (-0.03) - 1.0) < 0.15


def test_step_state_steps_between_buffers():
    """fg_step_state from a state buffer into another gives exactly the step
    fg_step takes from the same state (deterministic spread, markers, moving
    frame), records the same force/torque, and leaves the domain's own
    populations untouched; in == out and several environments are refused."""
    torch = pytest.importorskip("torch")
    shape = (40, 24, 20)
    rho, u = inputs.random_fields(shape, seed=71, u_amp=0.02)
    X, dV = inputs.fibonacci_sphere(200, 4.0, (20, 12, 10))
    frame = fishlbm.make_frame(acc=(1e-5, 0, 2e-6), omega=(0, 1e-4, 0), origin=(20, 12, 10))
    a, b = (fishlbm.Domain([fishlbm.env_desc(shape, 0.6)], deterministic=True) for _ in range(2))
    for d in (a, b):
        d.init_fields(rho, u)
        d.set_markers(np.float32(X), np.tile(np.float32([0.01, 0, 0]), (200, 1)), np.float32(dV))
    nb = b.state_bytes()
    bufs = [torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(3)]
    b.copy_state(bufs[0], True)
    before = b.populations()
    for n in range(3):
        U = np.tile(np.float32([0.01, 0.002 * n, 0]), (200, 1))
        for d in (a, b):
            d.set_markers(np.float32(X + U * n), U, None)
        a.step(1, [frame])
        b.step_state(bufs[n], bufs[n + 1] if n < 2 else bufs[0], [frame])
        assert np.array_equal(a.get_body_force_torque(), b.get_body_force_torque())
    assert np.array_equal(b.populations(), before)            # the domain's state is untouched
    b.copy_state(bufs[0], False)
    assert np.array_equal(a.populations(), b.populations())
    with pytest.raises(fishlbm.FgError):
        b.step_state(bufs[1], bufs[1])
    two = fishlbm.Domain([fishlbm.env_desc(shape, 0.6)] * 2)
    with pytest.raises(fishlbm.FgError):
        two.step_state(bufs[1], bufs[2])


@pytest.mark.parametrize("other", ["fused", "overlap"])
@pytest.mark.parametrize("M", [1, 3])
def test_fused_step_equals_plain_bit_for_bit(M, other):
    """The fused step kernel (IB phases and cell blocks from one work queue,
    one persistent launch), and the plain kernel with the IB beside it (a
    second stream), against the plain chain (IB kernel, plain stream-collide
    kernel, reduction) with the deterministic spread: the same populations,
    force/torque rows of every segment and mass, bit for bit, over 25 steps of
    three environments (the swimmer channel with open faces and a moving
    frame, a periodic box with a sphere, one without markers), with one and
    three direct-forcing passes."""
    fish = inputs.fish_for_grid((96, 48, 48), 24.0, 900)
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre((96, 48, 48)))
    envs = [fishlbm.env_desc((96, 48, 48), 0.52, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)),
            fishlbm.env_desc((40, 32, 24), 0.6), fishlbm.env_desc((24, 16, 16), 0.7)]
    Xs, dVs = inputs.fibonacci_sphere(200, 4.0, (20.0, 16.0, 12.0))
    doms = [fishlbm.Domain(envs, variant=v, deterministic=True, ib_iters=M, record_history=25)
            for v in ("plain", other)]
    for n in range(25):
        X, U = fish.pose(n)
        Us = np.tile([0.02, -0.01 * math.sin(0.2 * n), 0.0], (200, 1))
        frames = [fishlbm.frame_from_array(traj.at(n)), fishlbm.make_frame(origin=(20, 16, 12)),
                  fishlbm.make_frame(acc=(1e-5, 0, 0), origin=(12, 8, 8))]
        for d in doms:
            d.set_markers(np.float32(X), np.float32(U), np.float32(fish.dV), seg=fish.seg, n_seg=5,
                          ref=fish.joints_rest[0], env=0)
            d.set_markers(np.float32(Xs + Us * n), np.float32(Us), np.float32(dVs), env=1)
            d.step(1, frames)
    assert doms[1].stream_collide_variant() == other
    for e in range(3):
        assert np.array_equal(doms[0].populations(env=e), doms[1].populations(env=e)), e
        assert np.array_equal(doms[0].history(25, env=e), doms[1].history(25, env=e)), e
    assert np.array_equal(doms[0].marker_force(env=0), doms[1].marker_force(env=0))


@pytest.mark.parametrize("variant", ["plain", "fused", "overlap"])
def test_removed_markers_give_zero_rows(variant):
    """An environment whose markers are removed reports zero force/torque
    rows from its next step on, in every variant: the fused kernel writes no
    chunk sums for an environment without markers, and the reduction must
    add none (the scratch still holds the previous steps' sums).  The other
    environment's rows and every population equal the plain chain's, bit for
    bit."""
    envs = [fishlbm.env_desc((40, 32, 24), 0.6), fishlbm.env_desc((32, 24, 24), 0.7)]
    Xs, dVs = inputs.fibonacci_sphere(600, 5.0, (20.0, 16.0, 12.0))
    Xt, dVt = inputs.fibonacci_sphere(400, 4.0, (16.0, 12.0, 12.0))
    doms = [fishlbm.Domain(envs, variant=v, deterministic=True, record_history=8) for v in ("plain", variant)]
    for n in range(8):
        Us = np.tile([0.02, -0.01 * math.sin(0.3 * n), 0.0], (600, 1))
        for d in doms:
            d.set_markers(np.float32(Xs + Us * n), np.float32(Us), np.float32(dVs), env=0)
            if n < 4:
                Ut = np.tile([0.0, 0.015, 0.0], (400, 1))
                d.set_markers(np.float32(Xt), np.float32(Ut), np.float32(dVt), env=1)
            elif n == 4:   # removed: no markers from this step on
                d.set_markers(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                              np.zeros(0, np.float32), env=1)
            d.step(1)
            if n >= 4:
                assert not np.any(d.get_body_force_torque(1)), (n, variant)
            elif n > 0:
                assert np.any(d.get_body_force_torque(1)), (n, variant)
    assert doms[1].stream_collide_variant() == variant
    for e in range(2):
        assert np.array_equal(doms[0].populations(env=e), doms[1].populations(env=e)), e
        assert np.array_equal(doms[0].history(8, env=e), doms[1].history(8, env=e)), e
