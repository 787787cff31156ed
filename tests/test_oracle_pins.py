"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, invariants, the stability bound, dense brute force on tiny
grids and special cases (arXiv 2311.18505, Secs. 3-4).  CPU only."""

import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2311_18505_gb300 import workloads as W
from brute_matrix import Brute
from fdtd_energy import Grid, dissipation, energy
from modal import discrete_frequency, dst_solution, fletcher_clamped, modulated_solution, simply_supported
from pitch import peak_frequency

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _states(s: oracle.OracleString, n_steps: int):
    """State after each of n_steps further steps (the first entry is the
    current state)."""
    out = [s.state()]
    for _ in range(n_steps):
        s.run(1)
        out.append(s.state())
    return out


def _fresh(d):
    s = oracle.OracleString(d)
    s.run(2)          # outputs y^0, y^1 come from the initial levels
    return s


# ----------------------------------------------------------------- grid

def test_theta_value_printed():
    assert W.THETA_DEFAULT == pytest.approx(GOLD["theta"]["value"], abs=1e-15)


def _amplification_max(n_t, d, theta):
    """Largest eigenvalue of Theta^{-1}(gamma^2 k^2 (-D_xx) + kappa^2 k^2 D_xxxx)
    for simply supported ends (dense NumPy), the quantity that must stay
    below 4 for the lossless linear scheme to be stable (von Neumann)."""
    h, k = 1.0 / n_t, 1.0 / d["fs"]
    nu = n_t - 1
    D2 = (np.diag(-2.0 * np.ones(nu)) + np.diag(np.ones(nu - 1), 1) + np.diag(np.ones(nu - 1), -1)) / h ** 2
    Mx = (np.diag(np.ones(nu - 1), 1) + np.diag(np.ones(nu - 1), -1)) / 2.0
    Th = theta * np.eye(nu) + (1 - theta) * Mx
    gam = 2 * d["f0"]
    K = gam ** 2 * k ** 2 * (-D2) + d["kappa"] ** 2 * k ** 2 * (D2 @ D2)
    return float(np.max(np.real(np.linalg.eigvals(np.linalg.solve(Th, K)))))


@pytest.mark.parametrize("f0,kappa", [(110.0, 1.0), (40.0, 0.5), (1000.0, 3.0), (300.0, 6.08), (2000.0, 3.0)])
def test_grid_is_the_stability_bound(f0, kappa):
    d = W.make(f0=f0, kappa=kappa)
    n_t, _ = oracle.grid(d)
    assert _amplification_max(n_t, d, d["theta"]) < 4.0
    # one more interval crosses the bound: the rule is tight
    assert _amplification_max(n_t + 1, d, d["theta"]) > 4.0 * (1 - 1e-3) or n_t + 1 > 400


def test_config1_grid_sizes():
    assert oracle.grid(W.single_string(1.0)) == (101, 218)
    assert oracle.grid(W.single_string(3.0)) == (101, 72)


def test_printed_spacing_rule_is_theta_one_bound():
    """The printed h_t (Sec. 3.2) gives N = 136 at f0 = 110, kappa = 1: stable
    with theta = 1, unstable with the printed theta = 0.70 (reading A5)."""
    d = W.make(grid_rule=1)
    n_t, _ = oracle.grid(d)
    assert n_t == 136
    assert _amplification_max(n_t, d, 1.0) < 4.0
    assert _amplification_max(n_t, d, d["theta"]) > 4.0


def test_printed_rule_blows_up_with_printed_theta():
    d = W.make(grid_rule=1, sigma0=0.0, sigma1=0.0)
    s = oracle.OracleString(d)
    with pytest.raises(FloatingPointError):
        for _ in range(200):
            y = s.run(1000)
            if not np.all(np.isfinite(y)) or np.abs(y).max() > 1e6:
                raise FloatingPointError("grew without bound")


# -------------------------------------------------------- linear modes

def test_single_mode_closed_form():
    """Simply supported, lossless, alpha = 1: u^0 = u^1 = sin(p pi x) gives
    y^j = A cos(w (j - 1/2)) / cos(w/2), cos w = 1 - Om2 / (2 Theta_s)."""
    d = W.make(boundary=1, sigma0=0.0, sigma1=0.0, kappa=1.5)
    s = oracle.OracleString(d)
    n_t = s.n_t
    for p in (1, 3, 17):
        x = np.arange(1, n_t) / n_t
        mode = 1e-3 * np.sin(p * math.pi * x)
        s2 = oracle.OracleString(d)
        s2.set_state(mode, mode)
        y = s2.run(6000)
        f = discrete_frequency(n_t, d, p)
        w = 2 * math.pi * f / d["fs"]
        Io = np.maximum(0.0, 1.0 - np.abs(x - d["pickup"]) * n_t)
        A = Io @ mode
        j = np.arange(6000)
        ref = A * np.cos(w * (j - 0.5)) / math.cos(w / 2)
        assert np.max(np.abs(y - ref)) <= 1e-10 * abs(A)


@pytest.mark.parametrize("sigma0,sigma1,kappa", [(0.0, 0.0, 1.0), (0.5, 1e-5, 1.0), (2.0, 1e-4, 3.0)])
def test_dst_modal_solution(sigma0, sigma1, kappa):
    """The oracle equals the closed-form modal (DST) solution of the linear
    simply-supported scheme, lossless or lossy, for a pluck."""
    d = W.make(boundary=1, sigma0=sigma0, sigma1=sigma1, kappa=kappa)
    s = oracle.OracleString(d)
    up, u, *_ = s.state()
    y = s.run(12000)
    ym = dst_solution(s.n_t, d, up, u, 12000, d["pickup"])
    assert np.max(np.abs(y - ym)) <= 1e-10 * np.max(np.abs(ym))


# ---------------------------------------------------------- f0 modulation

def _wave_speeds(d, n):
    """gamma^n of the step n -> n+1 (reading A14): vibrato
    gamma 2^{(c/1200) sin(2 pi f_v n k + phi)}, glissando gamma 2^{D min(n k, T) / T}."""
    g, t = 2.0 * d["f0"], np.arange(n) / d["fs"]
    m = d["modulation"]
    if m["kind"] == "vibrato":
        return g * 2.0 ** (m["depth"] / 1200.0 * np.sin(2 * math.pi * m["rate"] * t + m["phase"]))
    if m["kind"] == "gliss":
        return g * 2.0 ** (m["depth"] * np.minimum(t, m["duration"]) / m["duration"])
    return np.full(n, g)


@pytest.mark.parametrize("mod", [{"kind": "vibrato", "rate": 6.0, "depth": 40.0, "phase": 0.7},
                                 {"kind": "gliss", "depth": 1.0, "duration": 0.25},
                                 {"kind": "gliss", "depth": -0.5, "duration": 0.25},
                                 {"kind": "gliss", "depth": 0.7, "duration": 0.1}])
def test_modulated_modal_recursion(mod):
    """A linear simply-supported string with a modulated wave speed: each sine
    mode's recurrence, stepped with the step's gamma^n, gives the oracle's
    output to 1e-9 (on the grid sized for the peak gamma)."""
    d = W.make(boundary=1, sigma0=0.3, sigma1=2e-5, kappa=1.5, modulation=mod)
    s = oracle.OracleString(d)
    up, u, *_ = s.state()
    n = 12000
    y = s.run(n)
    ym = modulated_solution(s.n_t, d, _wave_speeds(d, n), up, u, n, d["pickup"])
    assert np.max(np.abs(y - ym)) <= 1e-9 * np.max(np.abs(ym))


@pytest.mark.parametrize("mod", [{"kind": "vibrato", "rate": 150.0, "depth": 300.0, "phase": 0.4},
                                 {"kind": "gliss", "depth": 1.0, "duration": 0.00625},
                                 {"kind": "gliss", "depth": 0.6, "duration": 0.003}])
@pytest.mark.parametrize("alpha,exi", [(3.0, 0), (6.0, 1), (2.0, 2)])
def test_modulated_brute_force(mod, alpha, exi):
    """Nonlinear strings (plucked, struck, bowed) with a fast vibrato or
    glissando on tiny grids: the dense matrix form (Eqs. 7-9) with every
    gamma^2 term taken at the step's gamma^n (transverse and longitudinal
    wave terms, phi') equals the oracle to 1e-11 over 300 steps."""
    d = W.make(f0=2500.0, alpha=alpha, kappa=1.0, excitation=EXCS[exi], modulation=mod)
    n_t, n_l = oracle.grid(d)
    assert n_t <= 16
    y_o = oracle.run(d, 300)
    g = _wave_speeds(d, 300)
    y_b = Brute(d, n_t, n_l).run(300, gamma_fn=lambda n: g[n])
    assert np.max(np.abs(y_o - y_b)) <= 1e-11 * np.max(np.abs(y_b))


BOW_ENV = {"t": [0.0, 0.002, 0.004, 0.006], "vel": [0.1, 0.4, 0.25, 0.3], "force": [0.5, 2.0, 1.0, 0.0],
           "pos": [0.15, 0.3, 0.45, 0.2]}


@pytest.mark.parametrize("alpha", [1.0, 4.0])
def test_bow_envelope_brute_force(alpha):
    """Time-varying bow velocity, force and position (Sec. 3.3.1): the dense
    matrix form with the controls of step n at t = n k (linear between
    breakpoints) and I, J at the step's x_B equals the oracle to 1e-11."""
    ex = dict(EXCS[2], release=-1.0, envelope=BOW_ENV)
    d = W.make(f0=2500.0, alpha=alpha, kappa=1.0, excitation=ex)
    n_t, n_l = oracle.grid(d)
    y_o = oracle.run(d, 400)
    y_b = Brute(d, n_t, n_l).run(400)
    assert np.max(np.abs(y_o - y_b)) <= 1e-11 * np.max(np.abs(y_b))
    # the envelope matters: constant controls give another waveform
    y_c = oracle.run(dict(d, excitation=EXCS[2]), 400)
    assert np.max(np.abs(y_o - y_c)) > 1e-3 * np.max(np.abs(y_o))


def test_bow_envelope_with_vibrato_brute_force():
    """Time-varying bow controls and a fast vibrato together: the dense
    matrix form with the step's controls and gamma^n equals the oracle to
    1e-11 over 400 steps."""
    ex = dict(EXCS[2], release=-1.0, envelope=BOW_ENV)
    mod = {"kind": "vibrato", "rate": 150.0, "depth": 300.0, "phase": 0.4}
    d = W.make(f0=2500.0, alpha=3.0, kappa=1.0, excitation=ex, modulation=mod)
    n_t, n_l = oracle.grid(d)
    y_o = oracle.run(d, 400)
    g = _wave_speeds(d, 400)
    y_b = Brute(d, n_t, n_l).run(400, gamma_fn=lambda n: g[n])
    assert np.max(np.abs(y_o - y_b)) <= 1e-11 * np.max(np.abs(y_b))


def test_constant_bow_envelope_is_no_envelope():
    ex = EXCS[2]
    flat = {"t": [0.0, 0.01], "vel": [ex["vel"]] * 2, "force": [ex["force"]] * 2, "pos": [ex["pos"]] * 2}
    d = W.make(alpha=3.0, f0=196.0, excitation=ex, n_samples=2000)
    assert np.array_equal(oracle.run(dict(d, excitation=dict(ex, envelope=flat))), oracle.run(d))


def test_glissando_pitch_rises_an_octave():
    """An octave glissando over 1 s: the fundamental measured near the end is
    2^0.8 times the one measured near the start (window centres 0.1 s and
    0.9 s), within 0.5 %."""
    d = W.make(kappa=0.1, sigma0=0.2, sigma1=1e-6, modulation={"kind": "gliss", "depth": 1.0, "duration": 1.0},
               excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3}, n_samples=48000)
    y = oracle.run(d)
    f_a = peak_frequency(y[:9600], d["fs"], 80.0, 160.0)
    f_b = peak_frequency(y[38400:], d["fs"], 160.0, 280.0)
    assert f_b / f_a == pytest.approx(2.0 ** 0.8, rel=5e-3)


def test_glissando_holds_at_its_end():
    """After its duration T an octave glissando holds at 2^D: from then on the
    string steps with gamma 2^1 = 2 gamma on the grid sized for that peak,
    which is the unmodulated string an octave up (same grid, same
    coefficients), so the fundamental measured after T is that string's
    (within 0.2 %), and the held note stays bounded for 12 T (a glide that
    kept rising would reach 2^12 and leave the grid's stability bound)."""
    d = W.make(kappa=0.1, sigma0=0.2, sigma1=1e-6, modulation={"kind": "gliss", "depth": 1.0, "duration": 0.1},
               excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3}, n_samples=57600)
    up = W.make(kappa=0.1, sigma0=0.2, sigma1=1e-6, f0=2.0 * d["f0"],
                excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3}, n_samples=57600)
    assert oracle.grid(d) == oracle.grid(up)
    y, y_up = oracle.run(d), oracle.run(up)
    assert np.all(np.isfinite(y))
    f_held = peak_frequency(y[9600:], d["fs"], 160.0, 280.0)
    f_up = peak_frequency(y_up[9600:], d["fs"], 160.0, 280.0)
    assert f_held == pytest.approx(f_up, rel=2e-3)
    assert np.max(np.abs(y[28800:])) <= np.max(np.abs(y[:28800]))


def test_zero_depth_modulation_is_none():
    base = W.make(alpha=3.0, n_samples=3000)
    y = oracle.run(base)
    for mod in ({"kind": "vibrato", "rate": 6.0, "depth": 0.0, "phase": 1.0},
                {"kind": "gliss", "depth": 0.0, "duration": 0.5}):
        assert np.array_equal(oracle.run(dict(base, modulation=mod)), y)


def test_decay_rate_per_mode():
    """A single lossy sine mode decays by r = sqrt((Theta_s - Sig)/(Theta_s + Sig))
    per step (roots of the modal recurrence), and -ln(r) fs approaches the
    continuum rate sigma0 + sigma1 (p pi)^2 within the O(h^2) dispersion."""
    d = W.make(boundary=1, sigma0=1.0, sigma1=1e-4, kappa=0.5)
    n_t = oracle.grid(d)[0]
    x = np.arange(1, n_t) / n_t
    h, k = 1.0 / n_t, 1.0 / d["fs"]
    for p in (1, 5):
        sp = math.sin(p * math.pi * h / 2) ** 2
        th = 1 - 2 * (1 - d["theta"]) * sp
        sig = d["sigma0"] * k + 4 * d["sigma1"] * k * sp / h ** 2
        om2 = 4 * (2 * d["f0"]) ** 2 * k ** 2 * sp / h ** 2 + 16 * d["kappa"] ** 2 * k ** 2 * sp ** 2 / h ** 4
        r = math.sqrt((th - sig) / (th + sig))
        cw = (2 * th - om2) / (2 * r * (th + sig))

        def envelope(a_prev, a_cur):
            # a^n = R r^n cos(n w + c)  =>  this equals R^2 r^{2n} sin^2 w
            return a_cur ** 2 - 2 * cw * r * a_cur * a_prev + (r * a_prev) ** 2

        basis = np.sin(p * math.pi * x)
        s2 = oracle.OracleString(d)
        s2.set_state(1e-3 * basis, 1e-3 * basis)
        up0, u0, *_ = s2.state()
        e0 = envelope((2 / n_t) * basis @ up0, (2 / n_t) * basis @ u0) / r ** 2   # level 1
        n_steps = 24000
        s2.run(2 + n_steps)
        up1, u1, *_ = s2.state()
        e1 = envelope((2 / n_t) * basis @ up1, (2 / n_t) * basis @ u1) / r ** (2 * (1 + n_steps))
        assert e1 == pytest.approx(e0, rel=1e-8)
        sigma_c = d["sigma0"] + d["sigma1"] * (p * math.pi) ** 2
        assert -math.log(r) * d["fs"] == pytest.approx(sigma_c, rel=0.02)


def test_clamped_fundamental_eq10_config1():
    """Sec. 4.1: lossless plucked string, estimated f0 within 2 Hz of Eq. 10."""
    d = W.make(sigma0=0.0, sigma1=0.0, n_samples=48000)
    y = oracle.run(d)
    f_est = peak_frequency(y, d["fs"], 60.0, 160.0)
    K = (math.pi * d["kappa"] / (2 * d["f0"])) ** 2
    assert abs(f_est - fletcher_clamped(d["f0"], K, 0)) < GOLD["detune_max_hz"]["value"]


@pytest.mark.parametrize("alpha,c0", [(1.0, 1e-3), (4.0, 1e-3), (1.0, 1e-2), (2.5, 5e-3)])
def test_detune_sweep_eq10(alpha, c0):
    """Sec. 4.1 detune figure: kappa = 5.88, alpha in [1,4], c0 in [1e-3,1e-2]."""
    sw = GOLD["detune_sweep"]
    f0 = 110.0
    d = W.make(f0=f0, kappa=sw["kappa"], alpha=alpha, sigma0=0.0, sigma1=0.0,
               excitation={"kind": "pluck", "amp": c0, "pos": 0.3}, n_samples=24000)
    y = oracle.run(d)
    f_est = peak_frequency(y, d["fs"], 0.5 * f0, 1.5 * f0)
    K = (math.pi * d["kappa"] / (2 * f0)) ** 2
    assert abs(f_est - fletcher_clamped(f0, K, 0)) < GOLD["detune_max_hz"]["value"]


def test_simply_supported_partials():
    """Partials n = 1..10 against f_n = n f0 sqrt(1 + K n^2): within 0.01 Hz of
    the discrete dispersion relation and within its O(h^2) dispersion of the
    continuum (the bound below is the discrete-vs-continuum gap plus 0.05%)."""
    d = W.make(boundary=1, sigma0=0.0, sigma1=0.0, excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.13},
               pickup=0.91, n_samples=96000)
    s = oracle.OracleString(d)
    y = s.run(96000)
    K = (math.pi * d["kappa"] / (2 * d["f0"])) ** 2
    for n in range(1, 11):
        fd = discrete_frequency(s.n_t, d, n)
        fc = simply_supported(d["f0"], K, n)
        f_est = peak_frequency(y, d["fs"], fd - 20, fd + 20)
        assert abs(f_est - fd) < 0.01
        assert abs(fd - fc) / fc < 0.005


# --------------------------------------------------------------- energy

@pytest.mark.parametrize("alpha,amp", [(1.0, 1e-3), (3.0, 2e-3), (10.0, 1e-2), (1.3, 2e-2)])
def test_energy_conserved_lossless(alpha, amp):
    """Lossless unexcited (pluck initial condition only): H^{n+1/2} constant
    to 1e-10 relative over 24,000 steps, for the nonlinear coupled scheme."""
    d = W.make(alpha=alpha, sigma0=0.0, sigma1=0.0, excitation={"kind": "pluck", "amp": amp, "pos": 0.3})
    s = _fresh(d)
    g = Grid(s.n_t, s.n_l, d)
    prev = s.state()
    H0 = None
    worst = 0.0
    for n in range(24000):
        s.run(1)
        cur = s.state()
        H = energy(g, prev[1], cur[1], prev[3], cur[3])
        if H0 is None:
            H0 = H
        worst = max(worst, abs(H - H0))
        prev = cur
    assert worst <= 1e-10 * abs(H0)


@pytest.mark.parametrize("alpha", [1.0, 4.0])
def test_energy_dissipation_budget(alpha):
    """Lossy: H^{n+1/2} - H^{n-1/2} = -k (2 sigma0 |dt.w|^2 + 2 sigma1 |D dt.w|^2)."""
    d = W.make(alpha=alpha, sigma0=1.5, sigma1=8e-5, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.21})
    s = _fresh(d)
    g = Grid(s.n_t, s.n_l, d)
    st = _states(s, 400)
    H = [energy(g, st[i][1], st[i + 1][1], st[i][3], st[i + 1][3]) for i in range(len(st) - 1)]
    for i in range(1, len(H)):
        D = dissipation(g, st[i - 1][1], st[i + 1][1], st[i - 1][3], st[i + 1][3])
        assert abs((H[i] - H[i - 1]) + g.k * D) <= 1e-10 * abs(H[0])
        assert D >= 0


def test_hammer_power_budget():
    """Lossless string + hammer (Eq. 6): the string gains k F I(dt.u) per
    step and the hammer's kinetic energy changes by -k M F_H dt.u_H."""
    ex = {"kind": "hammer", "mass": 6e-3, "vel": 2.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}
    d = W.make(alpha=3.0, sigma0=0.0, sigma1=0.0, excitation=ex)
    s = _fresh(d)
    g = Grid(s.n_t, s.n_l, d)
    M = ex["mass"] / (d["rho_a"] * d["length"])
    st = _states(s, 300)
    k = g.k
    contact = 0
    for i in range(1, len(st) - 1):
        Hm = energy(g, st[i - 1][1], st[i][1], st[i - 1][3], st[i][3])
        Hp = energy(g, st[i][1], st[i + 1][1], st[i][3], st[i + 1][3])
        ex_n = st[i + 1][4]          # power/force of the step i -> i+1
        assert abs((Hp - Hm) - k * ex_n[2]) <= 1e-10 * max(abs(Hp), 1e-30) + 1e-18
        uhm, uh = st[i - 1][4][1], st[i][4][1]
        uhp = st[i + 1][4][1]
        Km = 0.5 * M * ((uh - uhm) / k) ** 2
        Kp = 0.5 * M * ((uhp - uh) / k) ** 2
        FH = ex_n[5] / M
        assert abs((Kp - Km) + k * M * FH * (uhp - uhm) / (2 * k)) <= 1e-10 * max(Kp, Km, 1e-30)
        contact += ex_n[3] > 0
    assert contact > 5


def test_bow_power_budget_and_friction():
    """Lossless bowed string (Eq. 5): the string gains exactly k F I(dt.u)
    with F = -F_B phi(v_rel) and I(dt.u) = v_rel + v_B; slipping steps satisfy
    the friction law, sticking steps have v_rel = 0 and |phi| <= 1."""
    ex = {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0}
    d = W.make(alpha=2.0, sigma0=0.0, sigma1=0.0, excitation=ex)
    s = _fresh(d)
    g = Grid(s.n_t, s.n_l, d)
    st = _states(s, 1500)
    k = g.k
    FB = ex["force"] / (d["rho_a"] * d["length"] ** 2)
    vB = ex["vel"] / d["length"]
    stick = slip = 0
    for i in range(1, len(st) - 1):
        Hm = energy(g, st[i - 1][1], st[i][1], st[i - 1][3], st[i][3])
        Hp = energy(g, st[i][1], st[i + 1][1], st[i][3], st[i + 1][3])
        P, v, F = st[i + 1][4][2], st[i + 1][4][4], st[i + 1][4][5]
        assert abs((Hp - Hm) - k * P) <= 1e-10 * max(abs(Hp), 1e-30) + 1e-18
        assert P == pytest.approx(F * (v + vB), rel=1e-9, abs=1e-18)
        phi = -F / FB
        if v == 0.0:
            stick += 1
            assert abs(phi) <= 1 + 1e-12
        else:
            slip += 1
            mag = ex["eps"] + (1 - ex["eps"]) * math.exp(-ex["a"] * d["length"] * abs(v))
            assert phi == pytest.approx(math.copysign(mag, v), rel=1e-12)
    assert stick > 10 and slip > 10


def test_bow_envelope_power_budget():
    """Time-varying bow (Sec. 3.3.1, reading A20), from the states alone: a
    lossless bowed string whose v_B, F_B and x_B move changes its energy
    over each step n -> n+1 by exactly k F I_n(dt.u), where I_n interpolates
    linearly at x_B(t_n) and the controls are linear in time at t_n = n k.
    Slipping steps obey F = -F_B(t_n) phi(I_n(dt.u) - v_B(t_n)); sticking
    steps have I_n(dt.u) = v_B(t_n) and |F| <= F_B(t_n)."""
    env = {"t": [0.0, 0.004, 0.01, 0.02], "vel": [0.05, 0.4, 0.15, 0.3], "force": [0.2, 2.0, 1.0, 0.6],
           "pos": [0.12, 0.31, 0.2, 0.44]}
    ex = {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0,
          "envelope": env}
    d = W.make(alpha=2.0, sigma0=0.0, sigma1=0.0, excitation=ex)
    s = _fresh(d)
    n0 = s.time_level
    g = Grid(s.n_t, s.n_l, d)
    st = _states(s, 1100)
    k, L = g.k, d["length"]

    def interp(u, x):
        pos = x * s.n_t
        l = min(int(math.floor(pos)), s.n_t - 1)
        w = pos - l
        node = lambda j: u[j - 1] if 1 <= j <= s.n_t - 1 else 0.0
        return (1.0 - w) * node(l) + w * node(l + 1)

    stick = slip = 0
    for i in range(1, len(st) - 1):
        t = (n0 + i) * k                           # u^n = st[i][1], step n -> n+1
        vB = np.interp(t, env["t"], env["vel"]) / L
        FB = np.interp(t, env["t"], env["force"]) / (d["rho_a"] * L * L)
        xB = np.interp(t, env["t"], env["pos"])
        vI = (interp(st[i + 1][1], xB) - interp(st[i - 1][1], xB)) / (2.0 * k)
        v = vI - vB
        Hm = energy(g, st[i - 1][1], st[i][1], st[i - 1][3], st[i][3])
        Hp = energy(g, st[i][1], st[i + 1][1], st[i][3], st[i + 1][3])
        tol = 1e-10 * abs(Hp) + 1e-18
        if abs(v) <= 1e-9 * abs(vB):
            stick += 1
            assert abs(Hp - Hm) <= k * FB * abs(vI) * (1 + 1e-9) + tol
        else:
            slip += 1
            phi = math.copysign(ex["eps"] + (1 - ex["eps"]) * math.exp(-ex["a"] * L * abs(v)), v)
            assert abs((Hp - Hm) - k * (-FB * phi) * vI) <= tol
    assert stick > 50 and slip > 50
    assert s.time_level == n0 + len(st) - 1


# ---------------------------------------------------------- brute force

EXCS = [
    {"kind": "pluck", "amp": 2e-2, "pos": 0.3},
    {"kind": "hammer", "mass": 5e-3, "vel": 4.0, "pos": 0.37, "omega": 3000.0, "alpha": 2.5},
    {"kind": "bow", "vel": 0.3, "force": 1.5, "pos": 0.23, "a": 100.0, "eps": 0.1, "release": 0.004},
]


@pytest.mark.parametrize("alpha", [1.0, 3.0, 10.0])
@pytest.mark.parametrize("exi", [0, 1, 2])
@pytest.mark.parametrize("boundary", [0, 1])
def test_brute_force_tiny_grids(alpha, exi, boundary):
    """Stencil oracle == dense matrix form of Eqs. 7-9 on N_t = 8 grids."""
    n_l = 6 if alpha < 5 else 3
    d = W.make(alpha=alpha, excitation=EXCS[exi], boundary=boundary, f0=400.0, kappa=2.0,
               n_t=8, n_l=n_l, sigma0=0.7, sigma1=3e-5)
    y_o = oracle.run(d, 400)
    y_b = Brute(d, 8, n_l).run(400)
    assert np.max(np.abs(y_o - y_b)) <= 1e-11 * np.max(np.abs(y_b))


@pytest.mark.parametrize("f0,alpha", [(2500.0, 1.2), (3000.0, 2.0), (1800.0, 6.0)])
def test_brute_force_derived_grids(f0, alpha):
    """Grids from the spacing rules themselves (no override) at high f0."""
    d = W.make(f0=f0, alpha=alpha, kappa=1.0, excitation={"kind": "pluck", "amp": 1e-2, "pos": 0.4})
    n_t, n_l = oracle.grid(d)
    assert n_t <= 12
    y_o = oracle.run(d, 300)
    y_b = Brute(d, n_t, n_l).run(300)
    assert np.max(np.abs(y_o - y_b)) <= 1e-11 * np.max(np.abs(y_b))


# -------------------------------------------------------- special cases

def test_alpha_one_no_longitudinal_motion():
    """Sec. 4.1: alpha = 1 nullifies the coupling, so z stays exactly zero."""
    for ex in EXCS:
        d = W.make(alpha=1.0, excitation=ex)
        s = oracle.OracleString(d)
        s.run(3000)
        _, _, zp, z, _ = s.state()
        assert np.all(z == 0.0) and np.all(zp == 0.0)


def test_dalembert_exact_period():
    """kappa = 0, theta = 1, gamma k / h = 1: the scheme is the exact
    travelling-wave recursion, so u returns to itself after 2 N steps."""
    N = 100
    d = W.make(f0=48000.0 / N / 2.0, kappa=0.0, theta=1.0, sigma0=0.0, sigma1=0.0, n_t=N,
               excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3})
    s = oracle.OracleString(d)
    up0, u0, *_ = s.state()
    s.run(2 + 2 * N)
    up1, u1, *_ = s.state()
    # levels: after 2 + 2N outputs the state holds (u^{2N}, u^{2N+1})
    assert np.max(np.abs(u1 - u0)) <= 1e-14
    assert np.max(np.abs(up1 - up0)) <= 1e-14


def test_mirror_symmetry():
    """(x_P, x_o) -> (1 - x_P, 1 - x_o) gives the same output (nonlinear too)."""
    a = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.3}, pickup=0.7)
    b = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.7}, pickup=0.3)
    ya, yb = oracle.run(a, 4000), oracle.run(b, 4000)
    assert np.max(np.abs(ya - yb)) <= 1e-12 * np.max(np.abs(ya))


def test_linear_in_amplitude_at_alpha_one():
    a = W.make(excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3})
    b = W.make(excitation={"kind": "pluck", "amp": 2e-3, "pos": 0.3})
    ya, yb = oracle.run(a, 4000), oracle.run(b, 4000)
    assert np.max(np.abs(yb - 2 * ya)) <= 1e-12 * np.max(np.abs(yb))


def test_longitudinal_motion_quadratic_in_amplitude():
    """Sec. 4.2: z is driven by the transverse strain squared, so doubling a
    small pluck quadruples z (to leading order)."""
    zs = []
    for amp in (1e-4, 2e-4):
        d = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": amp, "pos": 0.14})
        s = oracle.OracleString(d)
        s.run(2000)
        zs.append(np.max(np.abs(s.state()[3])))
    assert zs[1] / zs[0] == pytest.approx(4.0, rel=1e-3)


# ------------------------------------------- longitudinal output channel

def test_longitudinal_output_zero_at_alpha_one():
    for ex in EXCS:
        y = oracle.run(W.make(alpha=1.0, excitation=ex, output="longitudinal"), 2000)
        assert np.all(y == 0.0)


def test_longitudinal_output_reads_zeta_at_the_pickup():
    """The sample is L times the linear interpolation of zeta^j at x_o on
    the longitudinal grid (nodes m h_l, fixed ends)."""
    d = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.3}, pickup=0.63,
               output="longitudinal")
    _, n_l = oracle.grid(d)
    s = oracle.OracleString(d)
    for n in (1, 7, 500):
        y = s.run(n)
        _, _, _, z, _ = s.state()
        node = np.concatenate([[0.0], z, [0.0]])          # node values zeta_0 .. zeta_{N_l}
        want = d["length"] * np.interp(0.63, np.arange(n_l + 1) / n_l, node)
        assert y[-1] == pytest.approx(want, rel=1e-13, abs=1e-300)


def test_longitudinal_output_antisymmetric_under_mirror():
    """(x_P, x_o) -> (1 - x_P, 1 - x_o) mirrors the string: u keeps its sign,
    the longitudinal displacement changes it."""
    a = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.3}, pickup=0.7,
               output="longitudinal")
    b = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.7}, pickup=0.3,
               output="longitudinal")
    ya, yb = oracle.run(a, 4000), oracle.run(b, 4000)
    assert np.max(np.abs(ya)) > 0
    assert np.max(np.abs(ya + yb)) <= 1e-12 * np.max(np.abs(ya))


def test_longitudinal_output_quadratic_in_amplitude():
    ys = [oracle.run(W.make(alpha=3.0, excitation={"kind": "hammer", "mass": 5e-3, "vel": v,
                                                     "pos": 0.2, "omega": 3000.0, "alpha": 1.0},
                            output="longitudinal"), 2000) for v in (1e-3, 2e-3)]
    assert np.max(np.abs(ys[1] - 4 * ys[0])) <= 1e-3 * np.max(np.abs(ys[1]))


@pytest.mark.parametrize("kappa,c0", [(6.08, 0.0078), (9.63, 0.0085)])
def test_longitudinal_spectrum_fig2(kappa, c0):
    """Sec. 4.2 / Fig. 2 (f0 = 300 Hz, alpha = 3, x_P = 0.14, lossless): zeta
    is forced by the square of the transverse strain, so its strongest
    component lies at the sum f_1 + f_2 of the first two transverse partials
    (near the longitudinal fundamental alpha f0 = 900 Hz), and it is far
    weaker than u."""
    d = W.make(f0=300.0, alpha=3.0, kappa=kappa, sigma0=0.0, sigma1=0.0,
               excitation={"kind": "pluck", "amp": c0, "pos": 0.14}, n_samples=24000)
    yu = oracle.run(d)
    yz = oracle.run(dict(d, output="longitudinal"))
    f1 = peak_frequency(yu, d["fs"], 200.0, 400.0)
    f2 = peak_frequency(yu, d["fs"], 500.0, 700.0)
    assert peak_frequency(yz, d["fs"], 100.0, 2000.0) == pytest.approx(f1 + f2, abs=0.5)
    assert np.std(yz) < 0.2 * np.std(yu)


def test_pitch_rises_with_amplitude():
    """Tension modulation (the '+' sign of Eq. 4): a loud pluck of a string
    with alpha > 1 sounds sharper than a soft one."""
    fs = []
    for amp in (1e-4, 2e-2):
        d = W.make(alpha=4.0, sigma0=0.0, sigma1=0.0, excitation={"kind": "pluck", "amp": amp, "pos": 0.3},
                   n_samples=24000)
        fs.append(peak_frequency(oracle.run(d), d["fs"], 60.0, 170.0))
    assert fs[1] > fs[0] + 0.05


def test_chunked_run_equals_single_run():
    d = W.make(alpha=3.0, excitation=EXCS[1])
    a = oracle.OracleString(d)
    y1 = np.concatenate([a.run(1), a.run(2), a.run(997)])
    y2 = oracle.run(d, 1000)
    assert np.array_equal(y1, y2)


def test_batch_matches_single():
    ss = W.batch_mixed(6, seconds=0.02, seed=11)
    ys, used = oracle.run_batch(ss, threads=2)
    assert used >= 1
    for s, y in zip(ss, ys):
        assert np.array_equal(y, oracle.run(s))


def test_linear_solve_residual_small():
    d = W.make(alpha=7.0, excitation=EXCS[1])
    s = oracle.OracleString(d)
    s.run(500)
    assert s.residual() < 1e-12
