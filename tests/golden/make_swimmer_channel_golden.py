"""Write the FP64 oracle's reference history of the full swimmer channel.

The workload is the skinned swimmer in its accelerating frame on the
256x128x128 D3Q27 channel (velocity inlet u = 0.02 at -x, outflow at +x,
free-slip side walls), tau = 0.52, a 6000-marker fish of body length 64 on
a 5-segment spine driven by the travelling joint wave, the seeded frame
trajectory of Eq. 3, fluid starting uniform at the inflow velocity, 2000
steps.  Every marker position, velocity and frame value is rounded to
float32 first, as the C ABI rounds them, so that both sides see the same
inputs.

Only the oracle computes anything here.  Output (gzip text):

  swimmer_channel_history.txt.gz  one row per step: the (n_seg + 1) x 6
      force/torque rows (segments 0..4, then the total; F, T) and the mass
  swimmer_channel_fields.txt.gz   at steps 500, 1000 and 2000: rho and u of
      a seeded set of cells (uniform over the grid, over the open-face
      boundary layer, and over the fish's stencil support at that step)

Run: python tests/golden/make_swimmer_channel_golden.py [steps]
(about 25 minutes on 8 cores).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2206_01683_b300 import inputs  # noqa: E402
from parity_util import boundary_layer_mask, ib_support_mask  # noqa: E402

OPEN_X = (oracle.VELOCITY, oracle.OUTFLOW, oracle.FREESLIP, oracle.FREESLIP, oracle.FREESLIP, oracle.FREESLIP)
CHECKPOINTS = (500, 1000, 2000)
N_UNIFORM, N_BL, N_IB = 4096, 1024, 1024


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def sample_cells(shape, X, rng):
    """Seeded cell indices: uniform, boundary layer, stencil support."""
    n = shape[0] * shape[1] * shape[2]
    uni = rng.choice(n, N_UNIFORM, replace=False)
    bl = np.flatnonzero(boundary_layer_mask(shape, OPEN_X))
    ib = np.flatnonzero(ib_support_mask(shape, OPEN_X, X))
    return np.concatenate([uni, rng.choice(bl, N_BL, replace=False), rng.choice(ib, N_IB, replace=False)])


def main(steps=2000):
    cfg = inputs.FISH_CHANNEL
    shape, tau, u_in = cfg["shape"], cfg["tau"], cfg["u_in"]
    o = oracle.Oracle(shape, tau, faces=OPEN_X, u_in=f32((u_in, 0.0, 0.0)))
    o.init_fields(None, np.tile(f32((u_in, 0.0, 0.0)), (o.ncell, 1)))
    fish = inputs.fish_for_grid(shape, cfg["length"], cfg["n_markers"])
    traj = inputs.FrameTrajectory(inputs.seed_for(2), inputs.domain_centre(shape))
    rng = np.random.default_rng(inputs.seed_for(2) + 2000)
    hist, fields = [], []
    t0 = time.time()
    for n in range(steps):
        X, U = fish.pose(n)
        X, U = f32(X), f32(U)
        o.set_markers(X, U, f32(fish.dV), seg=fish.seg, nseg=5, ref=fish.joints_rest[0])
        o.step(f32(traj.at(n)))
        hist.append(np.concatenate([o.force_torque().ravel(), [o.mass()]]))
        if n + 1 in CHECKPOINTS:
            rho, u = o.fields()
            cells = sample_cells(shape, X, rng)
            fields.append(np.column_stack([np.full(cells.size, n + 1), cells, rho[cells], u[cells]]))
        if (n + 1) % 50 == 0:
            print("step %d  %.0f s" % (n + 1, time.time() - t0), flush=True)
    head = ("FP64 oracle, swimmer channel 256x128x128 (tau 0.52, inflow 0.02, 6000 markers, seeded frame); "
            "written by tests/golden/make_swimmer_channel_golden.py")
    np.savetxt(os.path.join(HERE, "swimmer_channel_history.txt.gz"), np.array(hist), fmt="%.12e",
               header=head + "\nper step: force/torque rows of segments 0..4 and the total (Fx Fy Fz Tx Ty Tz "
                             "each), then the mass")
    if fields:
        np.savetxt(os.path.join(HERE, "swimmer_channel_fields.txt.gz"), np.concatenate(fields),
                   fmt=["%d", "%d", "%.12e", "%.12e", "%.12e", "%.12e"],
                   header=head + "\ncolumns: step, cell (x + nx (y + ny z)), rho, ux, uy, uz")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2000)
