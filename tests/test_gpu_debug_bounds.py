"""Index checks of the debug build on tiny grids (the stand-in for a memory
sanitizer, which is closed on this machine).

libfishlbm_debug.so is the library compiled with -DFG_DEBUG_BOUNDS: every
kernel checks the indices it computes and records a flag instead of making
an out-of-range access.  A child process loads it (FISHLBM_LIB) and runs
tiny periodic and open domains through every stream-collide variant and
population layout and option (multi-direct forcing, deterministic spread, slip forcing, third-order
equilibrium, FP16/BF16 storage with two cells per thread and one, several
environments, fg_step_io, region momentum, 1- and 2-cell domains) against
the oracle; no flag may be set and the FP32 cases
must stay within the parity bar.
"""
import json
import os
import re
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, math, sys
import numpy as np
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import oracle
from paper_2206_01683_b300 import fishlbm, inputs
from parity_util import Pair
out = {"errors": {}}
OPEN = (1, 2, 3, 3, 3, 3)

def run(name, shape, faces, markers, steps, frame=None, **kw):
    p = Pair(shape, 0.7, faces=faces, u_in=(0.01, 0.0, 0.0), **kw)
    rho, u = inputs.random_fields(shape, seed=3, u_amp=0.01, rho_amp=0.005)
    p.init(rho, u)
    for n in range(steps):
        if markers is not None:
            X, U, dV, N = markers(n)
            p.markers(X, U, dV, normals=N if kw.get("slip") else None)
        p.step(frame)
    e = p.errors()
    out["errors"][name] = max(e["rho"], e["u"], e.get("force", 0.0))

def ball(c, R, n):
    def f(step):
        X, dV = inputs.fibonacci_sphere(n, R, c)
        X = X + np.array([0.01 * step, 0.0, 0.0])
        return X, np.tile([0.01, 0.0, 0.0], (n, 1)), dV, X - (np.asarray(c) + [0.01 * step, 0, 0])
    return f

fr = oracle.make_frame(acc=(1e-5, 0, 0), omega=(1e-4, -2e-4, 1e-4), domega=(1e-6, 0, 0), origin=(4, 3, 3))
for v in ("plain", "staged", "staged512", "fused", "overlap"):
    for M in (1, 2):
        run("periodic_%s_M%d" % (v, M), (8, 8, 8), (0,) * 6, ball((4.0, 3.5, 4.2), 1.5, 4), 20, variant=v, ib_iters=M)
    run("open_%s_eq3_det" % v, (9, 7, 6), OPEN, ball((4.3, 3.1, 2.6), 0.4, 3), 20, fr, variant=v, eq_order=3,
        deterministic=True)
    run("periodic_%s_slip" % v, (8, 8, 8), (0,) * 6, ball((4.0, 3.5, 4.2), 1.5, 6), 10, variant=v, slip=True)
# the in-place layout: both phases, open faces on every axis, short axes
for M in (1, 2):
    run("aa_periodic_M%d" % M, (8, 8, 8), (0,) * 6, ball((4.0, 3.5, 4.2), 1.5, 4), 21, layout="aa", ib_iters=M)
run("aa_open_eq3_det", (9, 7, 6), OPEN, ball((4.3, 3.1, 2.6), 0.4, 3), 21, fr, layout="aa", eq_order=3,
    deterministic=True)
run("aa_open_even", (10, 7, 6), OPEN, ball((4.3, 3.1, 2.6), 0.4, 3), 20, fr, layout="aa")
run("aa_all_open", (6, 5, 4), (1, 2, 3, 2, 2, 3), None, 9, fr, layout="aa")
run("aa_open3", (3, 3, 3), (2, 2, 3, 1, 3, 3), None, 8, layout="aa")
for st in ("f16", "bf16"):
    for nx in (10, 9):
        a = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7),
                            fishlbm.env_desc((nx, 7, 6), 0.7, OPEN, (0.01, 0, 0), 1.0, (0.01, 0, 0))],
                           storage=st, layout="aa")
        a.set_markers(np.float32([[4.3, 3.1, 2.6]]), np.zeros((1, 3), np.float32), np.float32([1.0]), env=1)
        a.step(5)
        a.region_momentum((1.0, 3.0, 2.0), 3.0, env=1)
        s_ = a.save_state(env=1)
        a.step(1)
        a.load_state(s_, env=1)
        a.step(2)
for shape in ((1, 1, 1), (2, 1, 1), (4, 3, 3)):
    t = fishlbm.Domain([fishlbm.env_desc(shape, 0.8, (0, 0, 0, 0, 0, 0) if shape[1] == 1 else
                                         (1, 2, 3, 3, 2, 1))], layout="aa")
    t.step(3)
    t.populations()
# several environments, FP16, region momentum, tiny domains
d = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7), fishlbm.env_desc((9, 7, 6), 0.7, OPEN, (0.01, 0, 0))])
X, dV = inputs.fibonacci_sphere(4, 1.5, (4.0, 3.5, 4.2))
d.set_markers(np.float32(X), np.zeros((4, 3), np.float32), np.float32(dV), env=0)
d.set_markers(np.float32([[4.3, 3.1, 2.6]]), np.zeros((1, 3), np.float32), np.float32([1.0]), env=1)
d.step(10)
d.region_momentum((1.0, 7.5, 4.0), 3.0, env=0)
d.region_momentum((4.0, 3.0, 3.0), 5.0, env=1)
for st in ("f16", "bf16"):
    g = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7)], storage=st, variant="staged512")
    g.set_markers(np.float32(X), np.zeros((4, 3), np.float32), np.float32(dV))
    g.step(10)
    # two cells per thread with open x faces and environment switches (even
    # rows), and one cell per thread (an odd row)
    for nx in (10, 9):
        h = fishlbm.Domain([fishlbm.env_desc((8, 8, 8), 0.7),
                            fishlbm.env_desc((nx, 7, 6), 0.7, OPEN, (0.01, 0, 0), 1.0, (0.01, 0, 0))],
                           storage=st, variant="staged512")
        h.set_markers(np.float32(X), np.zeros((4, 3), np.float32), np.float32(dV), env=0)
        h.set_markers(np.float32([[4.3, 3.1, 2.6]]), np.zeros((1, 3), np.float32), np.float32([1.0]), env=1)
        h.step_io(np.float32(np.concatenate([X, [[4.4, 3.1, 2.6]]])), np.zeros((5, 3), np.float32))
        h.step(5, [fishlbm.make_frame(acc=(1e-5, 0, 0), omega=(0, 1e-4, 0))] * 2)
for shape in ((1, 1, 1), (2, 1, 1)):
    t = fishlbm.Domain([fishlbm.env_desc(shape, 0.8)])
    t.step(3)
out["flags"] = fishlbm.debug_flags()
print("RESULT " + json.dumps(out))
'''


def test_debug_build_index_checks_stay_clean():
    sys.path.insert(0, ROOT)
    from paper_2206_01683_b300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, FISHLBM_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res["flags"] == 0, res
    bad = {k: v for k, v in res["errors"].items() if not v <= 1e-5}
    assert not bad, bad


def test_debug_build_random_configurations_stay_clean():
    """The seeded random configurations and batches (test_gpu_fuzz_oracle.py,
    test_gpu_fuzz_batches.py: every variant, layout and storage type, marker
    sets that change between steps, posted markers, direct launches) on the
    debug build: every case passes its bars and no index check fires."""
    sys.path.insert(0, ROOT)
    from paper_2206_01683_b300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, FISHLBM_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_fuzz_oracle.py", "tests/test_gpu_fuzz_batches.py"],
                       env=env, capture_output=True, text=True, timeout=1500, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    summary = r.stdout.strip().splitlines()[-1]
    print("debug build:", summary)
    m = re.search(r"(\d+) passed", summary)
    assert m and int(m.group(1)) == 60 and "skipped" not in summary, summary
