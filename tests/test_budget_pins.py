"""The per-step power-budget checker (tests/budget.py) pinned on the FP64
oracle's states before it judges the GPU's: a lossless struck or bowed
string's energy changes by exactly the work of the excitation force
(Secs. 3.3.1-3.3.2, Eqs. 5-6), and planted mistakes (a hammer mass off by
1 %, bow controls taken one step late) break the budget."""

import numpy as np

import oracle
from budget import bow_budget, hammer_budget
from paper_2311_18505_gb300 import workloads as W

HAMMER = {"kind": "hammer", "mass": 6e-3, "vel": 2.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}
BOW = {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0}
ENV = {"t": [0.0, 0.004, 0.01, 0.02], "vel": [0.05, 0.4, 0.15, 0.3], "force": [0.2, 2.0, 1.0, 0.6],
       "pos": [0.12, 0.31, 0.2, 0.44]}


def oracle_levels(d, n_steps):
    """Levels 1 .. n_steps + 1 of the oracle as (u, D, z, Dz, u_H, Du_H)."""
    s = oracle.OracleString(d)
    s.run(2)
    lv = []
    for i in range(n_steps + 1):
        up, u, zp, z, ex = s.state()
        lv.append((u, u - up, z, z - zp, ex[1], ex[1] - ex[0]))
        if i < n_steps:
            s.run(1)
    return s, lv


def test_hammer_budget_on_the_oracle():
    d = W.make(alpha=3.0, sigma0=0.0, sigma1=0.0, excitation=HAMMER)
    s, lv = oracle_levels(d, 800)
    r, c, F, H = hammer_budget(d, s.n_t, s.n_l, lv)
    assert (F > 0).sum() > 50                       # the contact lasts many steps
    assert np.abs(r).max() <= 1e-12 * np.abs(H).max()
    assert np.abs(c).max() <= 1e-10 * np.abs(F).max()
    wrong = dict(d, excitation=dict(HAMMER, mass=HAMMER["mass"] * 1.01))
    r2, _, _, _ = hammer_budget(wrong, s.n_t, s.n_l, lv)
    assert np.abs(r2).max() > 1e-5 * np.abs(H).max()


def test_bow_budget_on_the_oracle():
    for ex in (BOW, dict(BOW, envelope=ENV)):
        d = W.make(alpha=2.0, sigma0=0.0, sigma1=0.0, excitation=ex)
        s, lv = oracle_levels(d, 1200)
        rs, stick, n_slip, n_stick, H = bow_budget(d, s.n_t, s.n_l, lv, n0=1)
        assert n_slip > 100 and n_stick > 100
        assert np.abs(rs).max() <= 1e-12 * np.abs(H).max()
        assert stick.max() <= 1e-12 * np.abs(H).max()
    late_r, _, _, _, H = bow_budget(d, s.n_t, s.n_l, lv, n0=2)
    assert np.abs(late_r).max() > 1e-4 * np.abs(H).max()
