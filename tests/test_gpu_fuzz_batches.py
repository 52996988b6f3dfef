"""Seeded random batches: the three ways of running a step that must agree
bit for bit with the deterministic spread -- the plain chain (IB kernel,
stream-collide kernel, reduction), the fused persistent kernel, and the IB
beside the cell blocks -- over batches drawn at random: one to five
environments of random shapes (odd row lengths included, which take the
one-cell kernels), periodic or open faces, an accelerating and rotating
frame, zero to 1200 markers in one to three segments, one to three
direct-forcing passes, FP32, FP16 or BF16 storage, second- or third-order
equilibrium, and marker sets that grow, shrink, appear and go away
between steps; and the plain chain with its markers posted with the step
(fg_step_markers, device arrays the IB kernel reads in place) on the steps
that keep every marker count, and launched without graphs.  Compared after
every step: every environment's force/torque history row and mass; at the
end: the populations and the marker forces.

An environment without markers once read force sums its step had not
written (the fused kernel writes none for it); a fixed batch missed that
whenever the scratch happened to hold zeros."""
import math

import numpy as np
import pytest

from paper_2206_01683_b300 import fishlbm, inputs

pytestmark = pytest.mark.gpu

P, V, O, S = fishlbm.FG_PERIODIC, 1, 2, 3   # periodic, velocity inlet, outflow, free slip
FACE_SETS = [(P,) * 6, (V, O, S, S, S, S), (V, O, P, P, S, S), (P, P, S, S, P, P)]
STEPS = 10


@pytest.fixture(autouse=True)
def _index_checks_clean():
    """Run on the debug build (FISHLBM_LIB, as test_gpu_debug_bounds.py
    does), no index check of any kernel may have fired in a case."""
    yield
    try:
        flags = fishlbm.debug_flags()
    except fishlbm.FgError:   # the release build carries no index checks
        flags = 0
    assert flags == 0, flags


def _draw(seed):
    """A batch: per environment its shape, faces, tau, frame and the marker
    counts and segment counts of the two halves of the run."""
    rng = np.random.default_rng(seed)
    envs = []
    for _ in range(int(rng.integers(1, 6))):
        shape = tuple(int(v) for v in rng.integers(16, 41, 3))
        faces = FACE_SETS[int(rng.integers(0, len(FACE_SETS)))]
        counts = [int(rng.choice([0, 50, 300, 1200])) for _ in range(2)]
        envs.append(dict(shape=shape, faces=faces, tau=float(rng.uniform(0.52, 0.9)),
                         n_seg=int(rng.integers(1, 4)), counts=counts,
                         acc=tuple(float(v) for v in rng.normal(0, 2e-5, 3)),
                         omega=tuple(float(v) for v in rng.normal(0, 2e-4, 3)),
                         seed=int(rng.integers(0, 2 ** 31))))
    opts = dict(ib_iters=int(rng.integers(1, 4)), storage=str(rng.choice(["f32", "f16", "bf16"])),
                eq_order=int(rng.choice([2, 3])))
    return envs, opts


def _markers(env, n, step):
    """n markers on a sphere at the domain centre (radius a quarter of the
    smallest extent, clear of every face), moving with a seeded velocity."""
    if n == 0:
        z = np.zeros((0, 3), np.float32)
        return z, z, np.zeros(0, np.float32), np.zeros(0, np.int32)
    c = [0.5 * (v - 1) for v in env["shape"]]
    X, dV = inputs.fibonacci_sphere(n, 0.25 * min(env["shape"]), c)
    rng = np.random.default_rng(env["seed"] + n)
    seg = rng.integers(0, env["n_seg"], n).astype(np.int32)
    U = np.tile([0.02 * math.cos(0.3 * step), 0.01 * math.sin(0.2 * step), -0.005], (n, 1))
    U = U + rng.normal(0, 1e-3, (n, 3))
    return np.float32(X + U * step), np.float32(U), np.float32(dV), seg


@pytest.mark.parametrize("seed", list(range(11, 23)))
def test_random_batches_agree_across_step_kernels(seed):
    envs, opts = _draw(seed)
    descs = [fishlbm.env_desc(e["shape"], e["tau"], e["faces"], (0.02, 0, 0) if e["faces"][0] == V else (0, 0, 0))
             for e in envs]
    torch = pytest.importorskip("torch")
    doms = {v: fishlbm.Domain(descs, variant=v, deterministic=True, record_history=STEPS, **opts)
            for v in ("plain", "fused", "overlap")}
    # the plain chain again, its markers posted with the step (fg_step_markers,
    # device arrays read in place by the IB kernel) whenever no environment's
    # marker count changes
    doms["posted"] = fishlbm.Domain(descs, variant="plain", deterministic=True, record_history=STEPS, **opts)
    # and launched directly instead of replayed from a captured graph
    doms["direct"] = fishlbm.Domain(descs, variant="plain", deterministic=True, record_history=STEPS,
                                    graphs=False, **opts)
    for n in range(STEPS):
        half = 0 if n < STEPS // 2 else 1
        frames = [fishlbm.make_frame(acc=e["acc"], omega=e["omega"],
                                     origin=tuple(0.5 * (v - 1) for v in e["shape"])) for e in envs]
        recount = n == 0 or (n == STEPS // 2 and any(e["counts"][1] != e["counts"][0] for e in envs))
        sets = [_markers(e, e["counts"][half], n) for e in envs]
        for name, d in doms.items():
            if name == "posted" and not recount:
                if sum(e["counts"][half] for e in envs) > 0:
                    Xd = torch.from_numpy(np.concatenate([m[0] for m in sets])).cuda()
                    Ud = torch.from_numpy(np.concatenate([m[1] for m in sets])).cuda()
                    d.step_markers(Xd, Ud, frames)
                    torch.cuda.synchronize()   # the arrays live until the step has run
                else:
                    d.step(1, frames)
                continue
            for k, e in enumerate(envs):
                cnt = e["counts"][half]
                if n == 0 or (n == STEPS // 2 and cnt != e["counts"][0]) or cnt > 0:
                    X, U, dV, seg = sets[k]
                    d.set_markers(X, U, dV, seg=seg, n_seg=e["n_seg"], env=k)
            d.step(1, frames)
        want = [doms["plain"].history(STEPS, env=k) for k in range(len(envs))]
        for v in ("fused", "overlap", "posted", "direct"):
            for k in range(len(envs)):
                got = doms[v].history(STEPS, env=k)
                assert np.array_equal(got, want[k]), (seed, v, n, k, envs[k]["counts"])
    for k, e in enumerate(envs):
        ref = doms["plain"].populations(env=k)
        for v in ("fused", "overlap", "posted", "direct"):
            assert np.array_equal(doms[v].populations(env=k), ref), (seed, v, k)
            if e["counts"][1] > 0:
                assert np.array_equal(doms[v].marker_force(env=k), doms["plain"].marker_force(env=k)), (seed, v, k)
        if e["counts"][1] == 0:   # markers gone: zero force/torque rows
            assert not np.any(doms["plain"].history(STEPS, env=k)[-1][:-1]), (seed, k)
    for d in doms.values():
        d.close()
