"""Dense matrix-vector form of the scheme (Sec. 3.4, Eqs. 7-9), NumPy FP64.

Test helper for tiny grids (N_t, N_l <= ~12).  Every block of Eqs. 8-9 is
built literally as a dense matrix product and each step solves
A^n w^{n+1} = -(B^n w^n + C w^{n-1} + Gamma^n) with numpy.linalg.solve.
Readings applied (each differs from a literal transcription only where the
paper is inconsistent with its own Eq. 4):
  * Q_+- use sigma0 k and sigma1 k (Eq. 4), not 2 sigma k;
  * I_(l->t) is piecewise-linear interpolation P from the z nodes to the
    transverse nodes, and K^(lt) = (h_t/h_l) K^(tl)^T (the t->l transfer is
    the h-weighted adjoint of the l->t one);
  * Lambda^n = diag(D_x- u^n) over all N_t intervals;
  * the force enters as Gamma = -k^2 F J (Eq. 4 is k^2-scaled into Eq. 7).
The hammer is an extra unknown (u_H) appended to w; the bow force is found
by bracketing the scalar friction equation with scipy's brentq, each trial
velocity costing one dense solve.
"""

from __future__ import annotations

import math

import numpy as np


def _dminus(n_int: int, n_nodes_interior: int, h: float) -> np.ndarray:
    """D_x- : interior node values (zero ends) -> interval values."""
    D = np.zeros((n_int, n_nodes_interior))
    for i in range(n_int):          # interval i+1 between nodes i and i+1
        if i < n_nodes_interior:
            D[i, i] += 1.0 / h
        if i - 1 >= 0:
            D[i, i - 1] -= 1.0 / h
    return D


class Brute:
    def __init__(self, d: dict, n_t: int, n_l: int):
        self.d = d
        self.nt, self.nl = n_t, n_l
        self.ht, self.hl = 1.0 / n_t, 1.0 / n_l
        self.k = 1.0 / d["fs"]
        self.gamma = d["gamma"] if d.get("gamma") else 2.0 * d["f0"]
        th, k = d["theta"], self.k
        nu, nz = n_t - 1, max(n_l - 1, 0)
        self.nu, self.nz = nu, nz
        ht, hl = self.ht, self.hl
        I_t, I_l = np.eye(nu), np.eye(nz)
        self.Dm_t = _dminus(n_t, nu, ht)                 # N_t x (N_t-1)
        self.Dp_t = -self.Dm_t.T                          # (N_t-1) x N_t
        self.Dxx_t = self.Dp_t @ self.Dm_t
        Dm_l = _dminus(n_l, nz, hl)
        self.Dxx_l = (-Dm_l.T) @ Dm_l if nz else np.zeros((0, 0))
        Dxxxx = self.Dxx_t @ self.Dxx_t                   # simply supported
        if d.get("boundary", 0) == 0:                     # clamped ghost u_{-1} = u_1
            Dxxxx[0, 0] += 2.0 / ht ** 4
            Dxxxx[-1, -1] += 2.0 / ht ** 4
        M = np.zeros((nu, nu))
        for i in range(nu - 1):
            M[i, i + 1] = M[i + 1, i] = 0.5
        self.Theta = th * I_t + (1 - th) * M
        s0k, s1k = d["sigma0"] * k, d["sigma1"] * k
        self.Qp_t = self.Theta + s0k * I_t - s1k * self.Dxx_t
        self.Qm_t = self.Theta - s0k * I_t + s1k * self.Dxx_t
        self.Qp_l = (1 + s0k) * I_l - s1k * self.Dxx_l
        self.Qm_l = (1 - s0k) * I_l + s1k * self.Dxx_l
        self.S_t = d["kappa"] ** 2 * k ** 2 * Dxxxx
        # P: z interior -> all transverse nodes; D_x- on all transverse nodes
        xt = np.arange(n_t + 1) * ht
        P = np.zeros((n_t + 1, nz))
        for m in range(1, n_l):
            P[:, m - 1] = np.maximum(0.0, 1.0 - np.abs(xt - m * hl) / hl)
        Dm_full = np.zeros((n_t, n_t + 1))
        for i in range(n_t):
            Dm_full[i, i + 1] = 1.0 / ht
            Dm_full[i, i] = -1.0 / ht
        self.DmI = Dm_full @ P                            # D_x- I_(l->t): N_t x nz
        self.x_t = np.arange(1, n_t) * ht

    def interp_row(self, x: float) -> np.ndarray:
        """I(x): linear interpolation on the interior transverse nodes."""
        r = np.maximum(0.0, 1.0 - np.abs(self.x_t - x) / self.ht)
        return r

    def matrices(self, u, gam):
        k = self.k
        al = self.d["alpha"]
        phi2 = gam ** 2 * k ** 2 * (al ** 2 - 1.0) / 4.0
        Lam = np.diag(self.Dm_t @ u)
        V = -phi2 * self.Dp_t @ Lam @ Lam @ self.Dm_t
        Ktl = -phi2 * self.Dp_t @ Lam @ self.DmI
        Klt = (self.ht / self.hl) * Ktl.T
        G_t = gam ** 2 * k ** 2 * self.Dxx_t
        G_l = gam ** 2 * k ** 2 * self.Dxx_l
        nu, nz = self.nu, self.nz
        A = np.block([[self.Qp_t + V, Ktl], [Klt, self.Qp_l]])
        B = np.block([[-2 * self.Theta - G_t + self.S_t, 2 * Ktl],
                      [np.zeros((nz, nu)), -2 * np.eye(nz) - al ** 2 * G_l]])
        C = np.block([[self.Qm_t + V, Ktl], [Klt, self.Qm_l]])
        return A, B, C

    def run(self, n_samples: int, u0=None, z0=None, gamma_fn=None):
        """Outputs y^0..y^{n-1} = L I(x_o) u^j and the u trajectory."""
        d, k, L = self.d, self.k, d_len(self.d)
        nu, nz = self.nu, self.nz
        ex = d["excitation"]
        u_prev = np.zeros(nu); u = np.zeros(nu)
        z_prev = np.zeros(nz); z = np.zeros(nz)
        uh_prev = uh = 0.0
        if ex["kind"] == "pluck":
            c0, xp = ex["amp"] / L, ex["pos"]
            tri = np.where(self.x_t <= xp, c0 * self.x_t / xp, c0 * (1 - self.x_t) / (1 - xp))
            u_prev, u = tri.copy(), tri.copy()
        elif ex["kind"] == "hammer":
            uh = ex["vel"] / L * k
        Io = self.interp_row(d["pickup"])
        ys = [L * Io @ u_prev, L * Io @ u]
        n = 1
        while len(ys) < n_samples:
            gam = self.gamma if gamma_fn is None else gamma_fn(n)
            A, B, C = self.matrices(u, gam)
            w, wp = np.concatenate([u, z]), np.concatenate([u_prev, z_prev])
            rhs = -(B @ w + C @ wp)
            if ex["kind"] == "pluck":
                sol = np.linalg.solve(A, rhs)
            elif ex["kind"] == "hammer":
                sol, uh_new = self._hammer(A, rhs, u, u_prev, uh, uh_prev)
                uh_prev, uh = uh, uh_new
            else:
                sol = self._bow(A, rhs, u_prev, n)
            u_prev, u = u, sol[:nu]
            z_prev, z = z, sol[nu:]
            n += 1
            ys.append(L * Io @ u)
        return np.array(ys[:n_samples])

    def _hammer(self, A, rhs, u, u_prev, uh, uh_prev):
        d, k = self.d, self.k
        ex = d["excitation"]
        L = d_len(d)
        M = ex["mass"] / (d["rho_a"] * L)
        Ih = np.concatenate([self.interp_row(ex["pos"]), np.zeros(self.nz)])
        J = Ih / self.ht
        eta = uh - Ih[: self.nu] @ u
        eta_prev = uh_prev - Ih[: self.nu] @ u_prev
        G = ex["omega"] ** (1 + ex["alpha"]) * max(eta, 0.0) ** (ex["alpha"] - 1) if eta > 0 else 0.0
        # unknowns [w^{n+1}; u_H^{n+1}], force k^2 M F_H J with F_H = G (eta^{n+1}+eta^{n-1})/2
        nn = A.shape[0]
        Aa = np.zeros((nn + 1, nn + 1))
        Aa[:nn, :nn] = A
        cg = 0.5 * k * k * G
        Aa[:nn, :nn] += M * cg * np.outer(J, Ih)
        Aa[:nn, nn] = -M * cg * J
        Aa[nn, nn] = 1 + cg
        Aa[nn, :nn] = -cg * Ih
        b = np.concatenate([rhs + M * cg * eta_prev * J, [2 * uh - uh_prev - cg * eta_prev]])
        sol = np.linalg.solve(Aa, b)
        return sol[:nn], sol[nn]

    def _bow(self, A, rhs, u_prev, n):
        from scipy.optimize import brentq
        d, k = self.d, self.k
        ex = d["excitation"]
        L = d_len(d)
        force, vel, pos = ex["force"], ex["vel"], ex["pos"]
        env = ex.get("envelope")
        if env:   # controls at t = n k, piecewise linear, held outside the breakpoints
            t = n * k
            force = np.interp(t, env["t"], env["force"]) if "force" in env else force
            vel = np.interp(t, env["t"], env["vel"]) if "vel" in env else vel
            pos = np.interp(t, env["t"], env["pos"]) if "pos" in env else pos
        FB = force / (d["rho_a"] * L * L)
        if ex.get("release", -1.0) >= 0 and n * k >= ex["release"]:
            FB = 0.0
        vB, aN, eps = vel / L, ex["a"] * L, ex["eps"]
        Ib = np.concatenate([self.interp_row(pos), np.zeros(self.nz)])
        J = Ib / self.ht

        def w_of(phi):
            return np.linalg.solve(A, rhs + k * k * (-FB * phi) * J)

        def vrel(w):
            return (Ib[: self.nu] @ w[: self.nu] - Ib[: self.nu] @ u_prev) / (2 * k) - vB

        b = vrel(w_of(0.0))
        if FB == 0.0:
            return w_of(0.0)
        c = b - vrel(w_of(1.0))          # v = b - c phi, c = (k F/2) I A^-1 J
        if abs(b) <= c:                  # sticking: phi = b / c gives v = 0
            return w_of(b / c)
        sg = math.copysign(1.0, b)

        def g(wv):
            return wv + c * (eps + (1 - eps) * math.exp(-aN * wv)) - abs(b)

        wv = brentq(g, 0.0, abs(b), xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
        phi = sg * (eps + (1 - eps) * math.exp(-aN * wv))
        return w_of(phi)


def d_len(d: dict) -> float:
    return d.get("length", 1.0)
