"""Per-step power budgets of forced strings from the states alone (test
helper, NumPy FP64).

Written from the energy method (tests/fdtd_energy.py gives H^{n+1/2}): over
one step n -> n+1 a lossless string's energy changes by exactly the work of
the excitation force on it,

  H^{n+1/2} - H^{n-1/2} = k F^n I(x_e) delta_t. u^n,
  delta_t. u^n = (u^{n+1} - u^{n-1}) / 2k,

with F^n the (normalised) force and I the linear interpolation at the
excitation point.  The force is not taken from the synthesizer but from the
states and the excitation's own law:

* hammer (Sec. 3.3.2, Eq. 6): F^n = -M delta_tt u_H (the force on the
  string is minus the force on the hammer), and it must also equal the
  contact law M G^n (eta^{n+1} + eta^{n-1}) / 2, G^n = omega_H^{1+alpha_H}
  [eta^n]_+^{alpha_H - 1}, eta = u_H - I u;
* bow (Sec. 3.3.1, Eq. 5): with v = I delta_t. u - v_B, a slipping step has
  F^n = -F_B phi(v), phi(v) = sign(v)(eps + (1 - eps) e^{-a|v|}); a sticking
  step (v = 0) any |F^n| <= F_B.

States come as levels: level n holds (u^n, D^n = u^n - u^{n-1}, z^n, Dz^n)
and for a hammer (u_H^n, u_H^n - u_H^{n-1}), so both time levels of each
energy are read from one state and delta_t. u^n = (D^{n+1} + D^n) / 2k.
Applied to the FP64 oracle's states the budgets hold to rounding; applied to
the GPU kernel's FP32 states they measure its per-step energy error.
"""

from __future__ import annotations

import math

import numpy as np

from fdtd_energy import Grid, energy


def interp_weights(n_t: int, x: float):
    """(node l, weight w): I(x) u = (1 - w) u_l + w u_{l+1} (u_0 = u_N = 0)."""
    pos = x * n_t
    l = min(int(math.floor(pos)), n_t - 1)
    return l, pos - l


def interp(u: np.ndarray, lw) -> float:
    l, w = lw
    node = lambda j: float(u[j - 1]) if 1 <= j <= len(u) else 0.0
    return (1.0 - w) * node(l) + w * node(l + 1)


def level_energies(g: Grid, levels) -> np.ndarray:
    """H^{n-1/2} of every level (from u^{n-1} = u^n - D^n, u^n)."""
    out = []
    for lv in levels:
        u, du, z, dz = (np.asarray(a, np.float64) for a in lv[:4])
        out.append(energy(g, u - du, u, z - dz, z))
    return np.array(out)


def hammer_budget(d: dict, n_t: int, n_l: int, levels):
    """Residuals of the string's budget and of the contact law for each step
    between consecutive levels: (r, c, F, H) with r_n the energy residual,
    c_n = F^n - (contact law), F^n = -M delta_tt u_H and H the energies."""
    g = Grid(n_t, n_l, d)
    k = g.k
    ex = d["excitation"]
    L, rho = d.get("length", 1.0), d.get("rho_a", 5e-3)
    M = ex["mass"] / (rho * L)
    lw = interp_weights(n_t, ex["pos"])
    wk = ex.get("omega", 3000.0) ** (1.0 + ex.get("alpha", 2.5))
    expo = ex.get("alpha", 2.5) - 1.0
    H = level_energies(g, levels)
    r, c, F = [], [], []
    for i in range(1, len(levels) - 1):
        un, dn = np.asarray(levels[i][0], np.float64), np.asarray(levels[i][1], np.float64)
        up1, dp1 = np.asarray(levels[i + 1][0], np.float64), np.asarray(levels[i + 1][1], np.float64)
        uh, duh = levels[i][4], levels[i][5]
        uh1, duh1 = levels[i + 1][4], levels[i + 1][5]
        Fn = -M * (duh1 - duh) / (k * k)
        vI = (interp(dp1, lw) + interp(dn, lw)) / (2.0 * k)
        r.append((H[i + 1] - H[i]) - k * Fn * vI)
        eta = uh - interp(un, lw)
        eta_p = uh1 - interp(up1, lw)
        eta_m = (uh - duh) - interp(un - dn, lw)
        G = wk * max(eta, 0.0) ** expo if eta > 0 else 0.0
        c.append(Fn - M * G * 0.5 * (eta_p + eta_m))
        F.append(Fn)
    return np.array(r), np.array(c), np.array(F), H


def bow_budget(d: dict, n_t: int, n_l: int, levels, n0: int, slip_rel: float = 1e-9):
    """Residuals of the string's budget for each step between consecutive
    levels (level i at time n0 + i): (r_slip, excess_stick, n_slip, n_stick, H)
    where r_slip are the energy residuals of slipping steps with F = -F_B
    phi(v) and excess_stick the amounts by which sticking steps exceed the
    bound |dH| <= k F_B |I delta_t. u| (<= 0 when met).  A step sticks when
    |v| <= slip_rel |v_B|; with a time-varying bow the controls are those at
    t_n = n k (linear between breakpoints), I at x_B(t_n)."""
    g = Grid(n_t, n_l, d)
    k = g.k
    ex = d["excitation"]
    L, rho = d.get("length", 1.0), d.get("rho_a", 5e-3)
    a, eps = ex.get("a", 100.0) * L, ex.get("eps", 0.1)
    env = ex.get("envelope")
    rel = ex.get("release", -1.0)
    H = level_energies(g, levels)
    r_slip, stick_excess = [], []
    for i in range(1, len(levels) - 1):
        t = (n0 + i) * k
        if env:
            vB = float(np.interp(t, env["t"], env.get("vel", [ex["vel"]] * len(env["t"])))) / L
            FB = float(np.interp(t, env["t"], env.get("force", [ex["force"]] * len(env["t"])))) / (rho * L * L)
            xB = float(np.interp(t, env["t"], env.get("pos", [ex["pos"]] * len(env["t"]))))
        else:
            vB, FB, xB = ex["vel"] / L, ex["force"] / (rho * L * L), ex["pos"]
        if rel >= 0 and n0 + i >= math.ceil(rel * d["fs"] - 1e-9):
            FB = 0.0
        lw = interp_weights(n_t, xB)
        dn, dp1 = np.asarray(levels[i][1], np.float64), np.asarray(levels[i + 1][1], np.float64)
        vI = (interp(dp1, lw) + interp(dn, lw)) / (2.0 * k)
        v = vI - vB
        dH = H[i + 1] - H[i]
        if abs(v) <= slip_rel * abs(vB):
            stick_excess.append(abs(dH) - k * FB * abs(vI))
        else:
            phi = math.copysign(eps + (1.0 - eps) * math.exp(-a * abs(v)), v)
            r_slip.append(dH - k * (-FB * phi) * vI)
    return np.array(r_slip), np.array(stick_excess), len(r_slip), len(stick_excess), H
