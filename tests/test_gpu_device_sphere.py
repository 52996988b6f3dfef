"""The free rigid sphere advanced on the device (fg_attach_sphere) against
the host-coupled sphere (rigid.FreeSphere: the same update in numpy with two
synchronisations per step) and the oracle's reference integrator.

With the deterministic spread both GPU paths compute the same IB sums, and
the device update runs the host's FP64 sequence of operations with every
rounding explicit, so centre, velocity and spin agree bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2206_01683_b300 import fishlbm, inputs, rigid

pytestmark = pytest.mark.gpu

L, R, G = 24, 4.0, np.array([2e-4, -3e-4, -1e-3])
C0 = (11.3, 12.1, 10.7)
OPEN_X = (1, 2, 3, 3, 3, 3)


def _host_and_device(steps, layout="pull", storage="f32", env_list=None, env=0):
    envs = env_list or [fishlbm.env_desc((L, L, L), 1.0)]
    dh = fishlbm.Domain(envs, deterministic=True, storage=storage, variant="plain")
    dd = fishlbm.Domain(envs, deterministic=True, storage=storage, layout=layout, variant="plain")
    h = rigid.FreeSphere(dh, R, C0, 1.08, G, env=env)
    d = rigid.DeviceFreeSphere(dd, R, C0, 1.08, G, env=env)
    traj_h, traj_d = [], []
    for _ in range(steps):
        h.step()
        traj_h.append(np.concatenate([h.centre, h.vel, h.spin]))
    for _ in range(steps):
        d.step()
        traj_d.append(np.concatenate(d.state()))
    return np.array(traj_h), np.array(traj_d), dh, dd


def test_device_sphere_equals_host_coupled_sphere_bit_for_bit():
    """120 steps of the 24^3 periodic box (density ratio 1.08, skewed
    gravity): the device update and the host update give the same centre,
    velocity and spin after every step."""
    th, td, dh, dd = _host_and_device(120)
    assert np.array_equal(th, td), np.max(np.abs(th - td))
    assert np.array_equal(dh.populations(), dd.populations())
    assert np.array_equal(dh.get_body_force_torque(), dd.get_body_force_torque())


def test_device_sphere_in_place_layout():
    """The same sphere over the in-place population layout (whose kernels
    agree with the plain kernel to rounding): velocity within 1e-5 of its
    scale, centre within 1e-7 of the box, spin (driven by small torques)
    within the oracle test's 2e-3 of its scale, of the host-coupled run."""
    th, td, _, _ = _host_and_device(120, layout="aa")
    vs = np.abs(th[:, 3:6]).max()
    assert np.abs(td[:, 3:6] - th[:, 3:6]).max() <= 1e-5 * vs
    assert np.abs(td[:, 0:3] - th[:, 0:3]).max() <= 1e-7 * L
    ws = np.abs(th[:, 6:9]).max()
    assert np.abs(td[:, 6:9] - th[:, 6:9]).max() <= 2e-3 * ws


def test_device_sphere_every_step_and_graphs_off():
    """The state read back after every step matches the host sphere step by
    step; direct launches (graphs off) give the same trajectory."""
    envs = [fishlbm.env_desc((L, L, L), 1.0)]
    dh = fishlbm.Domain(envs, deterministic=True)
    h = rigid.FreeSphere(dh, R, C0, 1.08, G)
    runs = []
    for graphs in (True, False):
        dd = fishlbm.Domain(envs, deterministic=True, graphs=graphs)
        runs.append((dd, rigid.DeviceFreeSphere(dd, R, C0, 1.08, G)))
    for n in range(40):
        h.step()
        ref = np.concatenate([h.centre, h.vel, h.spin])
        for dd, s in runs:
            s.step()
            assert np.array_equal(np.concatenate(s.state()), ref), n


def test_device_sphere_matches_oracle_reference():
    """The device sphere against the oracle's reference integrator (the
    bars of the host-coupled test): 120 steps."""
    from oracle.rigid import OracleFreeSphere
    d = fishlbm.Domain([fishlbm.env_desc((L, L, L), 1.0)])
    s_g = rigid.DeviceFreeSphere(d, R, C0, 1.08, G)
    o = oracle.Oracle((L, L, L), 1.0)
    s_o = OracleFreeSphere(o, s_g.dirs, s_g.dV.astype(np.float64), R, C0, 1.08, G)
    for _ in range(120):
        s_g.step()
        s_o.step()
    c, v, w = s_g.state()
    assert np.linalg.norm(v - s_o.V) <= 2e-4 * np.linalg.norm(s_o.V)
    assert np.linalg.norm(c - s_o.c) <= 1e-6 * L
    assert np.linalg.norm(w - s_o.W) <= 2e-3 * np.linalg.norm(s_o.W) + 1e-10


def test_device_sphere_in_a_batch_with_moving_marker_layout():
    """A sphere on environment 1 of three, next to a swimmer channel whose
    marker set grows mid-run (the marker regions move): the sphere's
    trajectory equals that of the sphere alone in its own domain, and the
    other environments equal a domain without the sphere."""
    envs = [fishlbm.env_desc((48, 24, 24), 0.6, OPEN_X, (0.02, 0, 0), 1.0, (0.02, 0, 0)),
            fishlbm.env_desc((L, L, L), 1.0), fishlbm.env_desc((16, 16, 16), 0.7)]
    fish_a = inputs.fish_for_grid((48, 24, 24), 12.0, 200)
    fish_b = inputs.fish_for_grid((48, 24, 24), 12.0, 700)
    alone = fishlbm.Domain([envs[1]], deterministic=True)
    s_alone = rigid.DeviceFreeSphere(alone, R, C0, 1.08, G)
    batch = fishlbm.Domain(envs, deterministic=True)
    s_batch = rigid.DeviceFreeSphere(batch, R, C0, 1.08, G, env=1)
    plain = fishlbm.Domain([envs[0], envs[2]], deterministic=True)
    for n in range(30):
        fish = fish_a if n < 12 else fish_b
        X, U = fish.pose(n)
        for d, e in ((batch, 0), (plain, 0)):
            d.set_markers(np.float32(X), np.float32(U), np.float32(fish.dV), seg=fish.seg, n_seg=5,
                          ref=fish.joints_rest[0], env=e)
        batch.step(1)
        plain.step(1)
        s_alone.step()
    for a, b in zip(s_batch.state(), s_alone.state()):
        assert np.array_equal(a, b)
    assert np.array_equal(batch.populations(env=1), alone.populations())
    assert np.array_equal(batch.populations(env=0), plain.populations(env=0))
    assert np.array_equal(batch.populations(env=2), plain.populations(env=1))


def test_device_sphere_rules():
    """While attached the environment's markers and segment points belong to
    the body; a second sphere on the same environment, bad arguments and
    a shell outside an open domain's limits are rejected; after detaching,
    markers can be set again and the box reaction is gone from the frame."""
    d = fishlbm.Domain([fishlbm.env_desc((L, L, L), 1.0), fishlbm.env_desc((16, 16, 16), 0.7, OPEN_X)])
    s = rigid.DeviceFreeSphere(d, R, C0, 1.08, G)
    X = np.float32([[8.0, 8.0, 8.0]])
    for call in (lambda: d.set_markers(X, np.zeros_like(X), np.float32([1.0])),
                 lambda: d.set_segment_refs([[1.0, 2.0, 3.0]]),
                 lambda: d.set_markers_all(np.zeros((s.dirs.shape[0], 3), np.float32),
                                           np.zeros((s.dirs.shape[0], 3), np.float32)),
                 lambda: d.attach_sphere(R, C0, 1.08, G, s.dirs, s.dV)):
        with pytest.raises(fishlbm.FgError) as e:
            call()
        assert e.value.status == fishlbm.FG_ERR_STATE
    for bad in (dict(radius=-1.0), dict(density_ratio=0.0), dict(center=(np.nan, 1.0, 1.0)),
                dict(center=(1.0, 8.0, 8.0))):   # the last: the shell leaves the open x range
        kw = dict(radius=2.0, center=(8.0, 8.0, 8.0), density_ratio=1.1, gravity=(0, 0, -1e-4),
                  dirs=s.dirs, dV=s.dV, env=1)
        kw.update(bad)
        with pytest.raises(fishlbm.FgError) as e:
            d.attach_sphere(**kw)
        assert e.value.status == fishlbm.FG_ERR_INVALID, bad
    with pytest.raises(fishlbm.FgError) as e:
        d.sphere_state(env=1)
    assert e.value.status == fishlbm.FG_ERR_STATE
    d.step(3)
    c_before = s.centre.copy()
    s.detach()
    d.set_markers(X, np.zeros_like(X), np.float32([1.0]))
    d.step(2)
    with pytest.raises(fishlbm.FgError):
        d.sphere_state()
    assert np.all(np.isfinite(c_before))


@pytest.mark.parametrize("variant", ["fused", "overlap"])
def test_device_sphere_with_other_step_kernels(variant):
    """The device sphere around the fused step kernel and around the IB
    beside the cell blocks: the same trajectory bit for bit as around the
    plain chain (deterministic spread), in a two-environment batch."""
    envs = [fishlbm.env_desc((L, L, L), 1.0), fishlbm.env_desc((32, 24, 24), 0.6)]
    states = []
    for v in ("plain", variant):
        d = fishlbm.Domain(envs, deterministic=True, variant=v)
        s = rigid.DeviceFreeSphere(d, R, C0, 1.08, G)
        X, dV = inputs.fibonacci_sphere(120, 3.0, (16.0, 12.0, 12.0))
        d.set_markers(np.float32(X), np.tile(np.float32([0.01, 0, 0]), (120, 1)), np.float32(dV), env=1)
        s.step(30)
        states.append(np.concatenate(s.state()))
        assert d.stream_collide_variant() == v
    assert np.array_equal(states[0], states[1])
