"""Seeded synthetic inputs shared by the CUDA path's callers and the oracle.

Nothing here computes any part of the lattice Boltzmann / immersed-boundary
step; these are the problem descriptions both sides are fed:

* marker sets: a Fibonacci sphere, and a skinned fish surface (an ellipsoid of
  revolution on a 5-segment spine with 4 yaw joints, linear blend skinning as
  in Sec. III-A / Eq. 1's skin) driven by a travelling joint wave;
* frame trajectories p''(n), omega(n), domega(n) for Eq. 3;
* Taylor-Green initial fields;
* the per-environment draws of the batched workload.

All draws use ``numpy.random.default_rng(seed)``.  Positions are in lattice
units with cell centres at integer coordinates.
"""
import math

import numpy as np

SEED_BASE = 220601683

# Workloads by their sizes (lattice units).
SPHERE_BOX = dict(shape=(48, 32, 32), tau=0.56, radius=6.0, n_markers=452,
                  center=(24.0, 16.0, 16.0), velocity=(0.05, 0.0, 0.0), steps=200)
FISH_CHANNEL = dict(shape=(256, 128, 128), tau=0.52, u_in=0.02, length=64.0,
                    n_markers=6000, steps=2000)
SPHERE_BIG = dict(shape=(384, 192, 192), tau=0.56, n_markers=13500, steps=1000)
BATCH_SHAPES = ((96, 64, 64), (128, 64, 64), (160, 80, 80), (192, 96, 96))
ADJOINT_CHANNEL = dict(shape=(128, 64, 64), tau=0.52, length=32.0, n_markers=1500,
                       steps=200, checkpoint=20)

SCHOOL_CHANNEL = dict(shape=(150, 50, 100), tau=0.52, u_in=0.02, length=36.0, n_markers=2500,
                      gap=54.0, phase_lag=math.pi / 2.0, steps=2000)

WAVE_PERIOD = 400.0
N_SEGMENTS = 5


def seed_for(workload_id):
    return SEED_BASE + int(workload_id)


# ------------------------------------------------------------------ spheres

def fibonacci_sphere(n, radius, center):
    """n points on a sphere by the golden-angle spiral; equal area per point.

    Returns X (n, 3) and dV (n,) = 4 pi R^2 / n (surface area x unit width)."""
    i = np.arange(n, dtype=np.float64)
    zc = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    th = golden * i
    X = np.stack([r * np.cos(th), r * np.sin(th), zc], axis=1) * radius
    X += np.asarray(center, dtype=np.float64)
    dV = np.full(n, 4.0 * math.pi * radius * radius / n)
    return X, dV


def translating_sphere(n, radius, center0, velocity, step):
    """Rigid sphere moving at constant velocity: X(n) = X0 + U n, U_l = U."""
    X0, dV = fibonacci_sphere(n, radius, center0)
    U = np.tile(np.asarray(velocity, dtype=np.float64), (n, 1))
    return X0 + U * step, U, dV


# --------------------------------------------------------------------- fish

class Fish:
    """Skinned fish surface: prolate spheroid (semi-axes L/2, L/8, L/8) on a
    spine of 5 equal segments joined by 4 yaw joints (axis = frame z).  The
    head segment is the root and stays fixed in the frame; the head tip sits
    at ``head`` and the body extends along +x.  Joint angles follow
    theta_j(t) = A_j sin(2 pi t / period - phi_j).  Skin weights are linear
    hats in the axial coordinate between adjacent segment centres."""

    def __init__(self, length, n_markers, head, amplitudes=None, phases=None,
                 period=WAVE_PERIOD):
        self.L = float(length)
        self.n = int(n_markers)
        self.head = np.asarray(head, dtype=np.float64)
        j = np.arange(1, 5, dtype=np.float64)
        self.A = np.asarray(amplitudes if amplitudes is not None else 0.3 * j / 4.0, dtype=np.float64)
        self.phi = np.asarray(phases if phases is not None else 0.8 * j, dtype=np.float64)
        self.period = float(period)
        self._sample_surface()

    def _sample_surface(self):
        L, n = self.L, self.n
        a, b = L / 2.0, L / 8.0
        # area-uniform sampling: invert the cumulative lateral area along the axis
        s_fine = np.linspace(0.0, L, 200001)
        xi = (s_fine - a) / a
        r = b * np.sqrt(np.maximum(0.0, 1.0 - xi * xi))
        # dA/ds = 2 pi r sqrt(1 + r'^2) = 2 pi sqrt(r^2 + (r r')^2), r r' = -b^2 xi / a
        dA = 2.0 * math.pi * np.sqrt(r * r + (b * b * xi / a) ** 2)
        A = np.concatenate([[0.0], np.cumsum(0.5 * (dA[1:] + dA[:-1]) * np.diff(s_fine))])
        self.area = float(A[-1])
        i = np.arange(n, dtype=np.float64)
        s = np.interp((i + 0.5) / n * self.area, A, s_fine)
        golden = math.pi * (3.0 - math.sqrt(5.0))
        th = golden * i
        xi = (s - a) / a
        rs = b * np.sqrt(np.maximum(0.0, 1.0 - xi * xi))
        self.s = s
        self.rest = np.stack([self.head[0] + s, self.head[1] + rs * np.cos(th),
                              self.head[2] + rs * np.sin(th)], axis=1)
        self.dV = np.full(n, self.area / n)
        seglen = L / N_SEGMENTS
        centres = (np.arange(N_SEGMENTS) + 0.5) * seglen
        W = np.zeros((n, N_SEGMENTS))
        for k in range(N_SEGMENTS):
            if k == 0:
                W[:, 0] = np.where(s <= centres[0], 1.0, 0.0)
            if k == N_SEGMENTS - 1:
                W[:, k] += np.where(s >= centres[-1], 1.0, 0.0)
        for k in range(N_SEGMENTS - 1):
            inside = (s > centres[k]) & (s < centres[k + 1])
            t = (s - centres[k]) / seglen
            W[inside, k] += 1.0 - t[inside]
            W[inside, k + 1] += t[inside]
        self.W = W
        self.seg = np.argmax(W, axis=1).astype(np.int32)
        self.joints_rest = np.stack([self.head[0] + np.arange(1, N_SEGMENTS) * seglen,
                                     np.full(N_SEGMENTS - 1, self.head[1]),
                                     np.full(N_SEGMENTS - 1, self.head[2])], axis=1)

    def angles(self, t):
        w = 2.0 * math.pi / self.period
        th = self.A * np.sin(w * t - self.phi)
        dth = self.A * w * np.cos(w * t - self.phi)
        return th, dth

    def pose(self, t):
        """Marker positions X (n,3) and velocities U (n,3) at time t (steps)."""
        th, dth = self.angles(t)
        n = self.n
        # bone transforms as (rotation angle, translation) in the xy-plane
        ang = np.zeros(N_SEGMENTS)
        R = [np.eye(2)]
        trans = [np.zeros(2)]
        joint_world = []
        for k in range(1, N_SEGMENTS):
            Pk = self.joints_rest[k - 1, :2]
            jw = R[k - 1] @ Pk + trans[k - 1]      # world position of joint k
            joint_world.append(jw)
            ang[k] = ang[k - 1] + th[k - 1]
            c, s = math.cos(ang[k]), math.sin(ang[k])
            Rk = np.array([[c, -s], [s, c]])
            R.append(Rk)
            trans.append(jw - Rk @ Pk)
        p = self.rest[:, :2]
        X = np.zeros((n, 3))
        U = np.zeros((n, 3))
        X[:, 2] = self.rest[:, 2]
        for k in range(N_SEGMENTS):
            q = p @ R[k].T + trans[k]
            # revolute-chain velocity: sum_{j<=k} dtheta_j z x (q - joint_j)
            v = np.zeros((n, 2))
            for jj in range(1, k + 1):
                d = q - joint_world[jj - 1]
                v += dth[jj - 1] * np.stack([-d[:, 1], d[:, 0]], axis=1)
            X[:, :2] += self.W[:, k:k + 1] * q
            U[:, :2] += self.W[:, k:k + 1] * v
        return X, U


    def poses(self, ts):
        """Marker positions and velocities for many times at once:
        X, U of shape (len(ts), n, 3), float64."""
        ts = np.asarray(ts, dtype=np.float64)
        T = ts.size
        w = 2.0 * math.pi / self.period
        th = self.A[None, :] * np.sin(w * ts[:, None] - self.phi[None, :])          # (T, 4)
        dth = self.A[None, :] * w * np.cos(w * ts[:, None] - self.phi[None, :])
        ang = np.concatenate([np.zeros((T, 1)), np.cumsum(th, axis=1)], axis=1)    # (T, 5)
        c, s = np.cos(ang), np.sin(ang)
        trans = np.zeros((T, N_SEGMENTS, 2))
        joint_world = np.zeros((T, N_SEGMENTS - 1, 2))
        for k in range(1, N_SEGMENTS):
            Pk = self.joints_rest[k - 1, :2]
            cp, sp = c[:, k - 1], s[:, k - 1]
            jw = np.stack([cp * Pk[0] - sp * Pk[1], sp * Pk[0] + cp * Pk[1]], axis=1) + trans[:, k - 1]
            joint_world[:, k - 1] = jw
            ck, sk = c[:, k], s[:, k]
            trans[:, k] = jw - np.stack([ck * Pk[0] - sk * Pk[1], sk * Pk[0] + ck * Pk[1]], axis=1)
        p = self.rest[:, :2]
        X = np.zeros((T, self.n, 3))
        U = np.zeros((T, self.n, 3))
        X[:, :, 2] = self.rest[None, :, 2]
        for k in range(N_SEGMENTS):
            qx = c[:, k, None] * p[None, :, 0] - s[:, k, None] * p[None, :, 1] + trans[:, k, None, 0]
            qy = s[:, k, None] * p[None, :, 0] + c[:, k, None] * p[None, :, 1] + trans[:, k, None, 1]
            vx = np.zeros_like(qx)
            vy = np.zeros_like(qy)
            for jj in range(1, k + 1):
                dx = qx - joint_world[:, jj - 1, None, 0]
                dy = qy - joint_world[:, jj - 1, None, 1]
                vx += -dth[:, jj - 1, None] * dy
                vy += dth[:, jj - 1, None] * dx
            wk = self.W[None, :, k]
            X[:, :, 0] += wk * qx
            X[:, :, 1] += wk * qy
            U[:, :, 0] += wk * vx
            U[:, :, 1] += wk * vy
        return X, U


def fish_for_grid(shape, length, n_markers, amplitudes=None, phases=None):
    """Fish with its head tip at x = nx/4, centred in y and z."""
    nx, ny, nz = shape
    head = (nx / 4.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    return Fish(length, n_markers, head, amplitudes, phases)


class School:
    """Two fish in tandem along x in one marker set: the leader's head tip at
    x = nx/5, the follower's ``gap`` cells behind it, both centred in y and z;
    the follower's joint wave lags the leader's by ``phase_lag``.  Segments
    0-4 are the leader's, 5-9 the follower's; ``seg_refs`` gives each
    segment's torque point (its fish's first joint) and ``ref`` the leader's
    first joint for the total row."""

    def __init__(self, shape, length, n_each, gap, phase_lag=math.pi / 2.0):
        nx, ny, nz = shape
        y0, z0 = (ny - 1) / 2.0, (nz - 1) / 2.0
        j = np.arange(1, 5, dtype=np.float64)
        self.fish = [Fish(length, n_each, (nx / 5.0, y0, z0)),
                     Fish(length, n_each, (nx / 5.0 + gap, y0, z0), phases=0.8 * j + phase_lag)]
        self.n = 2 * int(n_each)
        self.n_seg = 2 * N_SEGMENTS
        self.dV = np.concatenate([f.dV for f in self.fish])
        self.seg = np.concatenate([self.fish[0].seg, self.fish[1].seg + N_SEGMENTS]).astype(np.int32)
        self.seg_refs = np.concatenate([np.tile(f.joints_rest[0], (N_SEGMENTS, 1)) for f in self.fish])
        self.ref = self.fish[0].joints_rest[0].copy()

    def pose(self, t):
        XA, UA = self.fish[0].pose(t)
        XB, UB = self.fish[1].pose(t)
        return np.concatenate([XA, XB]), np.concatenate([UA, UB])


# ------------------------------------------------------------------- frame

class FrameTrajectory:
    """Seeded smooth frame motion for Eq. 3.  Per component,
    p''(n) = sum_{k=1..3} a_k sin(2 pi n / T_k + psi_k), a_k ~ U(0, acc_max),
    omega(n) = sum_{k=1..3} b_k sin(2 pi n / S_k + chi_k), b_k ~ U(0, om_max/3),
    domega(n) its analytic derivative; T_k, S_k ~ U(200, 2000)."""

    def __init__(self, seed, origin, acc_max=2e-6, om_max=1e-4):
        rng = np.random.default_rng(seed)
        self.a = rng.uniform(0.0, acc_max, (3, 3))
        self.T = rng.uniform(200.0, 2000.0, (3, 3))
        self.psi = rng.uniform(0.0, 2 * math.pi, (3, 3))
        self.b = rng.uniform(0.0, om_max / 3.0, (3, 3))
        self.S = rng.uniform(200.0, 2000.0, (3, 3))
        self.chi = rng.uniform(0.0, 2 * math.pi, (3, 3))
        self.origin = np.asarray(origin, dtype=np.float64)

    def at(self, n):
        """The 12 frame numbers (p'', omega, domega, origin) at step n."""
        acc = (self.a * np.sin(2 * math.pi * n / self.T + self.psi)).sum(axis=1)
        ph = 2 * math.pi * n / self.S + self.chi
        om = (self.b * np.sin(ph)).sum(axis=1)
        dom = (self.b * (2 * math.pi / self.S) * np.cos(ph)).sum(axis=1)
        return np.concatenate([acc, om, dom, self.origin])


def domain_centre(shape):
    return np.array([(s - 1) / 2.0 for s in shape], dtype=np.float64)


def still_frame(origin=(0.0, 0.0, 0.0)):
    return np.concatenate([np.zeros(9), np.asarray(origin, dtype=np.float64)])


# --------------------------------------------------------------- fields

def taylor_green(shape, plane=(0, 1), U0=0.01, k=None):
    """2-D Taylor-Green vortex in the given axis plane (a, b):
    u_a = U0 sin(k x_a) cos(k x_b), u_b = -U0 cos(k x_a) sin(k x_b),
    rho = 1 - (3 U0^2 / 4)(cos 2k x_a + cos 2k x_b)   (p = cs2 rho).
    Returns rho (ncell,), u (ncell, 3) with cell index x + nx (y + ny z)."""
    nx, ny, nz = shape
    a, b = plane
    L = shape[a]
    if k is None:
        k = 2 * math.pi / L
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = [x.ravel().astype(np.float64), y.ravel().astype(np.float64), z.ravel().astype(np.float64)]
    xa, xb = pos[a], pos[b]
    u = np.zeros((x.size, 3))
    u[:, a] = U0 * np.sin(k * xa) * np.cos(k * xb)
    u[:, b] = -U0 * np.cos(k * xa) * np.sin(k * xb)
    rho = 1.0 - 0.75 * U0 * U0 * (np.cos(2 * k * xa) + np.cos(2 * k * xb))
    return rho, u


def random_fields(shape, seed, u_amp=0.02, rho_amp=0.01):
    """Smooth random (rho, u) fields: a few low Fourier modes per component."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    out = np.zeros((x.size, 4))
    for comp in range(4):
        for _ in range(3):
            kx, ky, kz = rng.integers(0, 3, 3)
            ph = rng.uniform(0, 2 * math.pi)
            out[:, comp] += rng.uniform(-1, 1) * np.cos(
                2 * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    rho = 1.0 + rho_amp * out[:, 0] / 3.0
    u = u_amp * out[:, 1:] / 3.0
    return rho, u


# ---------------------------------------------------------- batched draws

def batch_envs(n_envs, seed):
    """Per-environment draws of the batched workload: grid shape, marker
    count in [1500, 4000], joint-wave amplitude in [0.1, 0.4] rad, and a
    frame-trajectory seed."""
    rng = np.random.default_rng(seed)
    envs = []
    for e in range(n_envs):
        shape = BATCH_SHAPES[int(rng.integers(0, len(BATCH_SHAPES)))]
        envs.append(dict(shape=shape,
                         n_markers=int(rng.integers(1500, 4001)),
                         amplitude=float(rng.uniform(0.1, 0.4)),
                         frame_seed=int(rng.integers(0, 2**31 - 1))))
    return envs
