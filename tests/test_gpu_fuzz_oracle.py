"""Seeded random configurations against the FP64 oracle (FP32 storage, the
FP32 bars): per case a random grid (odd extents included), per axis periodic
faces, a velocity inlet with an outflow, or free-slip walls, a random
relaxation time, smooth random initial fields, an accelerating and rotating
frame, zero to 200 sphere markers (straddling a periodic wrap where the axis
allows) in one or two segments, one to three direct-forcing passes, no-slip
or slip forcing, second- or third-order equilibrium, the kernel variant and
the population layout.  Eight steps, then density, velocity, populations,
force and torque within the FP32 bar, and the local bars (open-face boundary
layer, the markers' stencil support, the largest per-cell error); and the
same draws with FP16 or BF16 storage at those dtypes' bars."""
import numpy as np
import pytest

import oracle
from oracle import FREESLIP, OUTFLOW, PERIODIC, VELOCITY
from paper_2206_01683_b300 import fishlbm, inputs

from parity_util import Pair, assert_local

pytestmark = pytest.mark.gpu

AXIS_FACES = [(PERIODIC, PERIODIC), (VELOCITY, OUTFLOW), (FREESLIP, FREESLIP)]
VARIANTS = ["plain", "staged", "staged512", "fused", "overlap"]
STEPS = 8
TOL = 1e-5


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
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(14, 37, 3))
    faces = ()
    for a in range(3):
        faces += AXIS_FACES[int(rng.integers(0, 3))]
    layout = "aa" if rng.random() < 0.25 else "pull"
    variant = "plain" if layout == "aa" else VARIANTS[int(rng.integers(0, len(VARIANTS)))]
    n = int(rng.choice([0, 40, 200]))
    r = 0.2 * min(shape)
    centre = []
    for a in range(3):
        if faces[2 * a] == PERIODIC:
            centre.append(float(rng.uniform(0, shape[a])))   # may straddle the wrap
        else:
            centre.append(float(rng.uniform(r + 3.0, shape[a] - 1 - r - 3.0)))
    return dict(shape=shape, faces=faces, layout=layout, variant=variant, n=n, r=r, centre=centre,
                tau=float(rng.uniform(0.52, 0.9)), u_in=tuple(float(v) for v in rng.normal(0, 0.006, 3)),
                rho0=float(rng.choice([1.0, 1.001])), ib_iters=int(rng.integers(1, 4)),
                slip=bool(n > 0 and rng.random() < 0.3), eq_order=int(rng.choice([2, 3])),
                nseg=int(rng.integers(1, 3)), U=rng.normal(0, 0.01, 3),
                acc=rng.normal(0, 2e-5, 3), omega=rng.normal(0, 2e-4, 3), domega=rng.normal(0, 2e-6, 3),
                field_seed=int(rng.integers(0, 2 ** 31)))


# the frozen per-dtype bars of the precision form (velocity, force, torque,
# the local rel-L2 bars and the per-cell bound)
TOL16 = {"f16": 2e-3, "bf16": 5e-2}


def _run(c, storage="f32"):
    """Eight steps of configuration c on both sides; the errors."""
    p = Pair(c["shape"], c["tau"], faces=c["faces"], u_in=c["u_in"], rho0=c["rho0"], variant=c["variant"],
             ib_iters=c["ib_iters"], slip=c["slip"], eq_order=c["eq_order"], layout=c["layout"], storage=storage)
    rho, u = inputs.random_fields(c["shape"], seed=c["field_seed"], u_amp=0.01, rho_amp=0.005)
    p.init(rho, u)
    origin = tuple(0.5 * (v - 1) for v in c["shape"])
    frame = oracle.make_frame(acc=tuple(c["acc"]), omega=tuple(c["omega"]), domega=tuple(c["domega"]),
                              origin=origin)
    if c["n"] > 0:
        X0, dV = inputs.fibonacci_sphere(c["n"], c["r"], c["centre"])
        seg = (np.arange(c["n"]) % c["nseg"]).astype(np.int32)
        # torques about a point off the sphere's centre: slip forcing pushes
        # along the sphere's normals, so about the centre the torque is a
        # cancellation down to rounding on both sides
        ref = tuple(np.asarray(c["centre"]) + c["r"] * np.array([0.7, -0.4, 0.3]))
    for k in range(STEPS):
        if c["n"] > 0:
            X = X0 + 0.02 * k * c["U"]
            U = np.tile(c["U"], (c["n"], 1))
            normals = (X0 - np.asarray(c["centre"])) if c["slip"] else None
            p.markers(X, U, dV, seg=seg, nseg=c["nseg"], ref=ref, normals=normals)
        p.step(frame)
    return p.errors()


def _where(c):
    return {k: c[k] for k in ("shape", "faces", "layout", "variant", "n", "ib_iters", "slip", "eq_order")}


@pytest.mark.parametrize("seed", list(range(31, 55)))
def test_random_configuration_against_oracle(seed):
    c = _draw(seed)
    err = _run(c)
    for key in ("rho", "u", "pop", "force", "torque", "seg_force"):
        assert err[key] <= TOL, (key, err[key], _where(c))
    assert_local(err, where=str(_where(c)))


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("seed", list(range(61, 73)))
def test_random_configuration_reduced_storage_against_oracle(seed, storage):
    """The same draws with FP16 or BF16 storage of f - w (FP32 arithmetic):
    velocity, force and torque within the dtype's frozen bar, and its local
    bars."""
    c = _draw(seed)
    err = _run(c, storage)
    for key in ("u", "force", "torque"):
        assert err[key] <= TOL16[storage], (key, err[key], storage, _where(c))
    assert_local(err, tol=TOL16[storage], tol_max=TOL16[storage], where=str((storage, _where(c))))
