"""Discrete energy of the planar-string scheme (test helper, NumPy FP64).

Written from the energy method, independently of the oracle's update code:
multiplying the transverse line of Eq. 4 by h_t delta_t. u and the
longitudinal line by h_l delta_t. z and summing by parts gives

  H^{n+1/2} = 1/2 <dtu, Theta dtu>_t + 1/2 ||dtz||_l^2
            + gamma^2/2 <q^{n+1}, q^n>_t + kappa^2/2 <u^{n+1}, D4 u^n>_t
            + gamma^2 alpha^2/2 <p^{n+1}, p^n>_l
            + phi' ( 1/4 <(q^{n+1})^2, (q^n)^2>_t
                     + 1/2 <q^{n+1} q^n, pt^{n+1} + pt^n>_t )

with dtu = (u^{n+1}-u^n)/k, q = D_x- u, p = D_x- z, pt = D_x- (P z) where P
is the piecewise-linear interpolant of z at the transverse nodes, and
phi' = gamma^2 (alpha^2-1)/2.  Without loss or excitation it is constant;
with loss it decreases by exactly k times the dissipated power at step n.
"""

from __future__ import annotations

import numpy as np


class Grid:
    def __init__(self, n_t: int, n_l: int, d: dict):
        self.nt, self.nl = n_t, n_l
        self.ht, self.hl = 1.0 / n_t, 1.0 / n_l
        self.k = 1.0 / d["fs"]
        self.gamma = d["gamma"] if d.get("gamma") else 2.0 * d["f0"]
        self.kappa, self.alpha = d["kappa"], d["alpha"]
        self.theta = d["theta"]
        self.sigma0, self.sigma1 = d["sigma0"], d["sigma1"]
        self.boundary = d.get("boundary", 0)
        xt = np.arange(n_t + 1) * self.ht
        # P: z interior (n_l - 1) -> all transverse nodes (n_t + 1), hat functions
        nz = max(n_l - 1, 0)
        self.P = np.zeros((n_t + 1, nz))
        for m in range(1, n_l):
            xm = m * self.hl
            self.P[:, m - 1] = np.maximum(0.0, 1.0 - np.abs(xt - xm) / self.hl)
        # D4 on the interior transverse nodes with the boundary ghosts
        nu = n_t - 1
        D2 = (np.diag(-2.0 * np.ones(nu)) + np.diag(np.ones(nu - 1), 1) + np.diag(np.ones(nu - 1), -1))
        D4 = D2 @ D2
        # D2 @ D2 is the simply-supported operator (ghost u_{-1} = -u_1, corner 5);
        # the clamped ghost u_{-1} = u_1 gives corner 7.
        corr = 2.0 if self.boundary == 0 else 0.0
        D4[0, 0] += corr
        D4[-1, -1] += corr
        self.D4 = D4 / self.ht ** 4

    def strain_t(self, u):
        ue = np.concatenate([[0.0], u, [0.0]])
        return np.diff(ue) / self.ht

    def strain_l(self, z):
        ze = np.concatenate([[0.0], z, [0.0]])
        return np.diff(ze) / self.hl

    def ptilde(self, z):
        if len(z) == 0:
            return np.zeros(self.nt)
        return np.diff(self.P @ z) / self.ht

    def theta_mul(self, v):
        ve = np.concatenate([[0.0], v, [0.0]])
        return self.theta * v + (1.0 - self.theta) * 0.5 * (ve[2:] + ve[:-2])


def energy(g: Grid, u0, u1, z0, z1, gamma: float | None = None) -> float:
    """H^{n+1/2} from (u^n, u^{n+1}, z^n, z^{n+1}) (normalised units)."""
    gam = g.gamma if gamma is None else gamma
    ht, hl, k = g.ht, g.hl, g.k
    dtu = (u1 - u0) / k
    kin = 0.5 * ht * np.dot(dtu, g.theta_mul(dtu))
    if len(z0):
        dtz = (z1 - z0) / k
        kin += 0.5 * hl * np.dot(dtz, dtz)
    q0, q1 = g.strain_t(u0), g.strain_t(u1)
    pot = 0.5 * gam ** 2 * ht * np.dot(q1, q0)
    pot += 0.5 * g.kappa ** 2 * ht * np.dot(u1, g.D4 @ u0)
    if len(z0):
        p0, p1 = g.strain_l(z0), g.strain_l(z1)
        pot += 0.5 * gam ** 2 * g.alpha ** 2 * hl * np.dot(p1, p0)
    phi = 0.5 * gam ** 2 * (g.alpha ** 2 - 1.0)
    if phi != 0.0:
        pt0, pt1 = g.ptilde(z0), g.ptilde(z1)
        pot += phi * (0.25 * ht * np.dot(q1 ** 2, q0 ** 2) + 0.5 * ht * np.dot(q1 * q0, pt1 + pt0))
    return kin + pot


def dissipation(g: Grid, um, up, zm, zp) -> float:
    """Power removed by the loss terms at step n, from u^{n-1}, u^{n+1}:
    2 sigma0 (|dt.u|^2 + |dt.z|^2) + 2 sigma1 (|D_x- dt.u|^2 + |D_x- dt.z|^2)."""
    k = g.k
    du = (up - um) / (2 * k)
    out = 2 * g.sigma0 * g.ht * np.dot(du, du)
    out += 2 * g.sigma1 * g.ht * np.sum(g.strain_t(du) ** 2)
    if len(zm):
        dz = (zp - zm) / (2 * k)
        out += 2 * g.sigma0 * g.hl * np.dot(dz, dz)
        out += 2 * g.sigma1 * g.hl * np.sum(g.strain_l(dz) ** 2)
    return out
