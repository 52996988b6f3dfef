"""Free rigid sphere two-way coupled to the lattice Boltzmann domain.

The smallest instance of the paper's body update (Eq. 1): a rigid body whose
only generalised forces are the fluid's tau_ext, gravity and buoyancy, here a
sphere of density ratio rho_p / rho_f (the fish of the paper have 1080/1000,
Sec. IV-A).  Each step the sphere's markers move with the body (positions on
the shell, velocities V + W x r), the library advances the fluid, and the
body is advanced explicitly from the force and torque the fluid exerted on it
(fg_get_body_force_torque).  The immersed shell encloses simulated fluid, and
the reported force includes what it took to move that inner fluid, so the
inner fluid's change of momentum and angular momentum (fg_region_momentum)
is added back, after Kempe & Froehlich (J. Comput. Phys. 231, 2012):

    m_p dV = F + dP_in + (m_p - m_f) g,   I_p dW = T + dL_in,
    centre += (V_old + V_new) / 2.

In a periodic box nothing else holds the body's excess weight, so the fluid
is given the reaction -(m_p - m_f) g each step as a uniform frame
acceleration of the library's Eq. 3 term (``box_reaction``).
"""
import math

import numpy as np

from . import fishlbm, inputs


class FreeSphere:
    """One free sphere in environment ``env`` of a Domain (single-body use of
    the domain's marker set)."""

    def __init__(self, domain, radius, center, density_ratio, gravity, n_markers=None, env=0,
                 box_reaction=True):
        self.dom = domain
        self.env = env
        self.R = float(radius)
        n = int(n_markers) if n_markers else int(round(4.0 * math.pi * self.R ** 2))
        unit, w = inputs.fibonacci_sphere(n, 1.0, (0.0, 0.0, 0.0))
        self.dirs = unit
        self.dV = (w * self.R ** 2).astype(np.float32)       # shell area per marker x unit width
        self.centre = np.array(center, dtype=np.float64)
        self.vel = np.zeros(3)
        self.spin = np.zeros(3)
        self.gravity = np.array(gravity, dtype=np.float64)
        volume = 4.0 * math.pi * self.R ** 3 / 3.0
        self.m_body = float(density_ratio) * volume
        self.m_fluid = volume
        self.inertia = 0.4 * self.m_body * self.R ** 2
        e = domain.envs[env]
        self.fluid_mass = float(e.nx * e.ny * e.nz)
        self.box_reaction = bool(box_reaction)
        self._p_in, self._l_in, _ = domain.region_momentum(self.centre, self.R, env)
        self._first = True

    def _frame(self):
        acc = (self.m_body - self.m_fluid) * self.gravity / self.fluid_mass if self.box_reaction else np.zeros(3)
        return fishlbm.make_frame(acc=tuple(acc))

    def step(self):
        """Advance fluid and body by one step; returns the fluid's force and
        torque on the body (about its centre) for the step."""
        X = self.centre + self.R * self.dirs
        U = self.vel + np.cross(self.spin, X - self.centre)
        self.dom.set_markers(X.astype(np.float32), U.astype(np.float32), self.dV if self._first else None,
                             env=self.env, ref=tuple(self.centre))
        self._first = False
        frames = [fishlbm.make_frame() for _ in self.dom.envs]
        frames[self.env] = self._frame()
        self.dom.step(1, frames)
        ft = self.dom.get_body_force_torque(self.env)[-1]
        p_in, l_in, _ = self.dom.region_momentum(self.centre, self.R, self.env)
        dv = (ft[:3] + (p_in - self._p_in) + (self.m_body - self.m_fluid) * self.gravity) / self.m_body
        dw = (ft[3:] + (l_in - self._l_in)) / self.inertia
        new_vel = self.vel + dv
        self.centre = self.centre + 0.5 * (self.vel + new_vel)
        self.vel = new_vel
        self.spin = self.spin + dw
        self._p_in, self._l_in = p_in, l_in
        return ft


class DeviceFreeSphere:
    """The same free sphere advanced on the device (fg_attach_sphere): the
    markers, the inner-fluid sums and the body update run in the step's own
    kernels, so stepping needs no synchronisation; ``centre``, ``vel`` and
    ``spin`` read the body state back (and synchronise).  Same constructor
    arguments as FreeSphere; the environment's frame is the box reaction
    unless the caller passes frames of its own to the domain."""

    def __init__(self, domain, radius, center, density_ratio, gravity, n_markers=None, env=0,
                 box_reaction=True):
        self.dom = domain
        self.env = env
        self.R = float(radius)
        n = int(n_markers) if n_markers else int(round(4.0 * math.pi * self.R ** 2))
        unit, w = inputs.fibonacci_sphere(n, 1.0, (0.0, 0.0, 0.0))
        self.dirs = unit
        self.dV = (w * self.R ** 2).astype(np.float32)
        domain.attach_sphere(self.R, center, density_ratio, gravity, self.dirs, self.dV, env=env,
                             box_reaction=box_reaction)

    def step(self, n=1):
        """Advance fluid and body by n steps (no synchronisation)."""
        self.dom.step(n)

    def state(self):
        return self.dom.sphere_state(self.env)

    @property
    def centre(self):
        return self.state()[0]

    @property
    def vel(self):
        return self.state()[1]

    @property
    def spin(self):
        return self.state()[2]

    def detach(self):
        self.dom.detach_sphere(self.env)
