"""Modal closed forms for the linear scheme (test helper, NumPy FP64).

With alpha = 1 the scheme is linear.  With simply supported ends the sine
vectors s_p(l) = sin(p pi l h), p = 1..N-1, diagonalise every operator of
Eq. 4 (Fourier symbols; s = sin^2(p pi h / 2)):
  delta_xx -> -4 s / h^2,   delta_xxxx -> 16 s^2 / h^4,
  Theta    -> Theta_s = 1 - 2 (1 - theta) s,
so each modal amplitude obeys the two-term recurrence
  (Theta_s + Sig) a^{n+1} = (2 Theta_s - Om2) a^n - (Theta_s - Sig) a^{n-1}
with Om2 = 4 gamma^2 k^2 s/h^2 + 16 kappa^2 k^2 s^2/h^4 and
Sig = sigma0 k + 4 sigma1 k s / h^2, solved here in closed form through the
roots of its characteristic polynomial (no time stepping).
"""

from __future__ import annotations

import math

import numpy as np


def symbols(n_t: int, d: dict):
    h, k = 1.0 / n_t, 1.0 / d["fs"]
    gam = d["gamma"] if d.get("gamma") else 2.0 * d["f0"]
    p = np.arange(1, n_t)
    s = np.sin(p * math.pi * h / 2.0) ** 2
    th = 1.0 - 2.0 * (1.0 - d["theta"]) * s
    om2 = 4 * gam ** 2 * k ** 2 * s / h ** 2 + 16 * d["kappa"] ** 2 * k ** 2 * s ** 2 / h ** 4
    sig = d["sigma0"] * k + 4 * d["sigma1"] * k * s / h ** 2
    return p, s, th, om2, sig


def dst_solution(n_t: int, d: dict, u0: np.ndarray, u1: np.ndarray, n_samples: int,
                 x_o: float) -> np.ndarray:
    """y^j = L I(x_o) u^j, j = 0..n-1, of the linear simply-supported scheme
    with initial levels u^0, u^1 (interior nodes)."""
    h = 1.0 / n_t
    L = d.get("length", 1.0)
    p, s, th, om2, sig = symbols(n_t, d)
    l = np.arange(1, n_t)
    Sm = np.sin(np.outer(p, l) * math.pi * h)          # (modes, nodes), orthogonal
    a0 = (2.0 / n_t) * Sm @ u0
    a1 = (2.0 / n_t) * Sm @ u1
    # roots of (th+sig) r^2 - (2 th - om2) r + (th - sig) = 0
    A = th + sig
    Bc = -(2 * th - om2)
    Cc = th - sig
    disc = (Bc ** 2 - 4 * A * Cc).astype(complex)
    r1 = (-Bc + np.sqrt(disc)) / (2 * A)
    r2 = (-Bc - np.sqrt(disc)) / (2 * A)
    # a^n = c1 r1^n + c2 r2^n with a^0, a^1
    c2 = (a1 - a0 * r1) / (r2 - r1)
    c1 = a0 - c2
    # pickup row I(x_o) on the interior nodes, projected on the modes
    Io = np.maximum(0.0, 1.0 - np.abs(l * h - x_o) / h)
    w = Sm.T  # node values of mode p
    Ip = Io @ w                                           # I(x_o) s_p
    n = np.arange(n_samples)[:, None]
    amp = c1[None, :] * r1[None, :] ** n + c2[None, :] * r2[None, :] ** n
    return L * np.real(amp @ Ip)


def discrete_frequency(n_t: int, d: dict, p: int) -> float:
    """Frequency [Hz] of lossless mode p from cos(w k) = 1 - Om2/(2 Theta_s)."""
    _, _, th, om2, _ = symbols(n_t, d)
    c = 1.0 - om2[p - 1] / (2.0 * th[p - 1])
    return math.acos(c) * d["fs"] / (2.0 * math.pi)


def fletcher_clamped(f0: float, K: float, p: int) -> float:
    """Eq. 10: p-th (0-based) mode of a lossless clamped stiff string."""
    return f0 * (p + 1) * (1 + 2 / math.pi * math.sqrt(K) + 4 / math.pi ** 2 * K) * math.sqrt(1 + K * (p + 1) ** 2)


def simply_supported(f0: float, K: float, n: int) -> float:
    """Continuum simply-supported stiff string: f_n = n f0 sqrt(1 + K n^2)."""
    return n * f0 * math.sqrt(1 + K * n * n)


def modulated_solution(n_t: int, d: dict, gammas: np.ndarray, u0: np.ndarray, u1: np.ndarray,
                       n_samples: int, x_o: float) -> np.ndarray:
    """y^j of the linear simply-supported scheme when the wave speed of the
    step n -> n+1 is gammas[n]: each sine mode follows the same two-term
    recurrence with Om2 built from gammas[n], stepped in time."""
    h, k = 1.0 / n_t, 1.0 / d["fs"]
    L = d.get("length", 1.0)
    p = np.arange(1, n_t)
    s = np.sin(p * math.pi * h / 2.0) ** 2
    th = 1.0 - 2.0 * (1.0 - d["theta"]) * s
    stiff = 16 * d["kappa"] ** 2 * k ** 2 * s ** 2 / h ** 4
    sig = d["sigma0"] * k + 4 * d["sigma1"] * k * s / h ** 2
    l = np.arange(1, n_t)
    Sm = np.sin(np.outer(p, l) * math.pi * h)
    a_prev, a = (2.0 / n_t) * Sm @ u0, (2.0 / n_t) * Sm @ u1
    Io = np.maximum(0.0, 1.0 - np.abs(l * h - x_o) / h)
    Ip = Io @ Sm.T
    y = np.zeros(n_samples)
    if n_samples > 0:
        y[0] = L * a_prev @ Ip
    if n_samples > 1:
        y[1] = L * a @ Ip
    for n in range(1, n_samples - 1):
        om2 = 4 * gammas[n] ** 2 * k ** 2 * s / h ** 2 + stiff
        a_next = ((2 * th - om2) * a - (th - sig) * a_prev) / (th + sig)
        a_prev, a = a, a_next
        y[n + 1] = L * a @ Ip
    return y
