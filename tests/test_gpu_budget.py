"""Energy and power budgets of forced strings on the GPU, from the FP32
states the kernels keep (Secs. 3.3.1-3.3.2, Eqs. 5-6; tests/budget.py, pinned
on the oracle in tests/test_budget_pins.py).

Each lossless string is stepped one sample per call for 2,400 steps and its
state read after every step.  Per step, the energy change must equal the
work of the excitation force, with the force taken from the states and the
excitation's own law (hammer: -M delta_tt u_H, checked against the contact
law; bow: -F_B phi(v) while slipping, |F| <= F_B while sticking).

Tolerance, from FP32 rounding: the kernel stores u^{n+1} = fl(u^n + D^{n+1}),
so the level n seen by H^{n+1/2} and by H^{n-1/2} differ by the rounding of
u, eps |u| per node (eps = 2^-24); the energy terms linear in u^{n+1} move by
about 2 eps H per step (H the largest energy), and the FP32 solve adds
errors proportional to the small accelerations.  The bar per step is
16 eps H (measured: at most 6 eps); over the steps without force the summed
change (the energy drift of the free string) must stay within 1e-5 H
(measured: 3e-7).  The hammer's force is the second difference of u_H,
whose increments lose log2(|u_H| / |D u_H|) bits, so the contact law is
held to 2^-14 of the largest force (measured: 1.6e-5 at most)."""

import numpy as np
import pytest

from budget import bow_budget, hammer_budget
from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -24
STEPS = 2400


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


@pytest.fixture(scope="module")
def ctx(sfd):
    c = sfd.sfd_ctx_create(0, None, 256 << 20)
    yield c
    sfd.sfd_ctx_destroy(c)


def gpu_levels(sfd, ctx, d, n_steps):
    """Levels 1 .. n_steps + 1 as (u, D, z, Dz, u_H, Du_H) in FP64 (exact
    widenings of the kernel's FP32 state), the grid and the kernel class."""
    s = sfd.string_from_dict(ctx, d)
    try:
        n_t, n_l, _, _ = sfd.sfd_string_info(s)
        cls = sfd.sfd_string_kernel_class(s)
        hammer = d["excitation"]["kind"] == "hammer"
        sfd.sfd_synthesize(s, 2)                    # the two initial levels, no step
        lv = []
        for i in range(n_steps + 1):
            u, du, z, dz = (a.astype(np.float64) for a in sfd.sfd_string_delta_state(s))
            uhp, uh = sfd.sfd_string_hammer(s) if hammer else (0.0, 0.0)
            lv.append((u, du, z, dz, uh, uh - uhp))
            if i < n_steps:
                sfd.sfd_synthesize(s, 1)
        return lv, n_t, n_l, cls
    finally:
        sfd.sfd_string_destroy(s)


HAMMER = {"kind": "hammer", "mass": 6e-3, "vel": 2.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}
BOW = {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0}
ENV = {"t": [0.0, 0.004, 0.01, 0.02], "vel": [0.05, 0.4, 0.15, 0.3], "force": [0.2, 2.0, 1.0, 0.6],
       "pos": [0.12, 0.31, 0.2, 0.44]}
SMEM_CLASS = 5


@pytest.mark.parametrize("f0,kappa,alpha,vel,smem", [(110.0, 1.0, 3.0, 2.0, False),
                                                     (80.0, 1.5, 1.0, 3.0, False),
                                                     (35.0, 0.1, 4.0, 3.0, True)])
def test_hammer_power_budget(sfd, ctx, f0, kappa, alpha, vel, smem):
    d = W.make(f0=f0, kappa=kappa, alpha=alpha, sigma0=0.0, sigma1=0.0,
               excitation=dict(HAMMER, vel=vel))
    lv, n_t, n_l, cls = gpu_levels(sfd, ctx, d, STEPS)
    assert (cls == SMEM_CLASS) == smem
    r, c, F, H = hammer_budget(d, n_t, n_l, lv)
    Hmax = np.abs(H).max()
    contact = F != 0.0
    print(f"hammer f0 {f0} alpha {alpha} N_t {n_t}: max|r|/H {np.abs(r).max() / Hmax:.3e} "
          f"({np.abs(r).max() / Hmax / EPS:.1f} eps), contact law {np.abs(c).max() / np.abs(F).max():.3e}, "
          f"contact steps {contact.sum()}, free drift {abs(r[~contact].sum()) / Hmax:.3e}")
    assert contact.sum() > 20 and (~contact).sum() > 1000
    assert np.abs(r).max() <= 16 * EPS * Hmax
    assert abs(r[~contact].sum()) <= 1e-5 * Hmax
    assert np.abs(c).max() <= 2.0 ** -14 * np.abs(F).max()


@pytest.mark.parametrize("f0,kappa,alpha,env,smem", [(196.0, 1.0, 2.0, False, False),
                                                     (196.0, 1.0, 2.0, True, False),
                                                     (30.0, 0.1, 2.0, False, True)])
def test_bow_power_budget(sfd, ctx, f0, kappa, alpha, env, smem):
    ex = dict(BOW, envelope=ENV) if env else BOW
    d = W.make(f0=f0, kappa=kappa, alpha=alpha, sigma0=0.0, sigma1=0.0, excitation=ex)
    lv, n_t, n_l, cls = gpu_levels(sfd, ctx, d, STEPS)
    assert (cls == SMEM_CLASS) == smem
    # a step sticks when its relative velocity is zero to FP32 rounding
    rs, stick, n_slip, n_stick, H = bow_budget(d, n_t, n_l, lv, n0=1, slip_rel=1e-4)
    Hmax = np.abs(H).max()
    print(f"bow f0 {f0} env {env} N_t {n_t}: slip {n_slip} stick {n_stick}, max|r|/H "
          f"{np.abs(rs).max() / Hmax:.3e} ({np.abs(rs).max() / Hmax / EPS:.1f} eps), stick excess "
          f"{(stick.max() / Hmax / EPS) if n_stick else 0:.1f} eps")
    assert n_slip > 100
    assert np.abs(rs).max() <= 16 * EPS * Hmax
    if n_stick:
        assert stick.max() <= 16 * EPS * Hmax
