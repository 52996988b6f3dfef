"""Free rigid sphere coupled to the FP64 oracle -- TEST INFRASTRUCTURE.

The reference for the library's free-body coupling (``paper_2206_01683_b300
/rigid.py``); it shares no code with it.  Newton-Euler equations of a rigid
sphere (Eq. 1 restricted to one rigid body: the generalised force is the
fluid's tau_ext plus gravity and buoyancy), with the fluid inside the
immersed-boundary shell treated as in Kempe & Froehlich 2012 (J. Comput.
Phys. 231): the force the markers report includes what it takes to move the
simulated inner fluid, so the inner fluid's momentum change is added back:

    m_p (V' - V) = F + (P_in' - P_in) + (m_p - m_f) g
    I_p (W' - W) = T + (L_in' - L_in)
    c' = c + (V + V') / 2

F, T: force and torque the fluid exerts on the body in the step (about the
centre); P_in, L_in: momentum and angular momentum of the fluid inside the
sphere after the step; m_p = rho_p V_p, m_f = V_p (fluid density 1),
I_p = 2/5 m_p R^2, V_p = 4/3 pi R^3.  In a periodic box the fluid carries the
reaction to the excess weight: a uniform frame acceleration p'' =
(m_p - m_f) g / M gives the fluid the force -(m_p - m_f) g each step.
"""
import math

import numpy as np

import oracle


class OracleFreeSphere:
    def __init__(self, o, directions, dV, radius, center, density_ratio, gravity, box_mass=None):
        self.o = o
        self.N = np.asarray(directions, dtype=np.float64)
        self.dV = np.asarray(dV, dtype=np.float64)
        self.R = float(radius)
        self.c = np.asarray(center, dtype=np.float64).copy()
        self.V = np.zeros(3)
        self.W = np.zeros(3)
        self.g = np.asarray(gravity, dtype=np.float64)
        vol = 4.0 / 3.0 * math.pi * self.R ** 3
        self.mp, self.mf = density_ratio * vol, vol
        self.Ip = 0.4 * self.mp * self.R ** 2
        self.M = float(box_mass) if box_mass is not None else float(o.ncell)
        self.P_in, self.L_in, _ = o.region_momentum(self.c, self.R)

    def step(self):
        X = self.c + self.R * self.N
        U = self.V + np.cross(self.W, X - self.c)
        self.o.set_markers(X, U, self.dV, ref=self.c)
        self.o.step(oracle.make_frame(acc=(self.mp - self.mf) * self.g / self.M))
        ft = self.o.force_torque()[-1]
        P, L, _ = self.o.region_momentum(self.c, self.R)
        Vn = self.V + (ft[:3] + (P - self.P_in) + (self.mp - self.mf) * self.g) / self.mp
        Wn = self.W + (ft[3:] + (L - self.L_in)) / self.Ip
        self.c = self.c + 0.5 * (self.V + Vn)
        self.V, self.W, self.P_in, self.L_in = Vn, Wn, P, L
        return ft
