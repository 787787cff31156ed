"""The oracle's exact gradient: the same C source built with a complex scalar
(complex step, dy/dp = Im y(p + i h) / h) differentiates the scheme to
rounding on smooth paths.  Pinned against things other than itself:

* its real part is the real build's output;
* on a linear simply-supported string the derivatives with respect to
  kappa, sigma0 and sigma1 equal those of the closed-form modal solution
  (tests/modal.py, no time stepping), and the one with respect to the pluck
  amplitude is y / amplitude (the scheme is linear in the amplitude);
* on nonlinear plucked, struck and vibrato strings every derivative equals
  a fourth-order central difference of the real build.

(A second-order central difference is not enough: kappa and alpha move the
high partials' phase by an amount that grows with time, so its truncation
error over 1500 samples is ~1e-4 at a relative step of 1e-6.  Differences
also have a rounding floor, which the complex step does not: sigma0 and
sigma1 change the output little, so their quotients carry the outputs'
rounding divided by a small change, 1e-6 - 1e-4 of the derivative here.
The tolerances sit just above those floors; a derivative that loses a term,
or a parameter that loses its imaginary part somewhere, is off by O(1).)"""

import math

import numpy as np
import pytest

import modal
import oracle
from paper_2311_18505_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def central4(f, p0, e):
    """(-f(p+2e) + 8 f(p+e) - 8 f(p-e) + f(p-2e)) / 12e."""
    return (-f(p0 + 2 * e) + 8 * f(p0 + e) - 8 * f(p0 - e) + f(p0 - 2 * e)) / (12 * e)


def with_param(d, key, v):
    if key == "amplitude":
        ex = dict(d["excitation"])
        ex["amp" if ex["kind"] == "pluck" else "vel"] = v
        return dict(d, excitation=ex)
    return dict(d, **{key: v})


def param(d, key):
    if key == "amplitude":
        ex = d["excitation"]
        return ex["amp" if ex["kind"] == "pluck" else "vel"]
    return d[key]


def test_real_part_is_the_real_build():
    cases = [dict(W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 4e-3, "pos": 0.23}), n_samples=800),
             dict(W.make(alpha=2.0, f0=90.0, excitation={"kind": "hammer", "mass": 5e-3, "vel": 2.5, "pos": 0.3,
                                                          "omega": 3000.0, "alpha": 2.5}), n_samples=800),
             dict(W.make(alpha=1.5, modulation={"kind": "vibrato", "rate": 6.0, "depth": 40.0, "phase": 0.3}),
                  n_samples=800)]
    for d in cases:
        for w in range(len(oracle.GRAD_PARAMS)):
            y, _ = oracle.complex_step(d, w)
            ref = oracle.run(d)
            # complex products and quotients round differently from real ones
            assert np.max(np.abs(y - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_linear_derivatives_equal_the_modal_closed_form():
    d = dict(W.make(alpha=1.0, boundary=1, sigma0=0.8, sigma1=3e-5, kappa=1.3,
                    excitation={"kind": "pluck", "amp": 2e-3, "pos": 0.31}), n_samples=1500)
    n_t, _ = oracle.grid(d)
    x = np.arange(1, n_t) / n_t
    c0, xp = d["excitation"]["amp"] / d["length"], d["excitation"]["pos"]
    u0 = np.where(x <= xp, c0 * x / xp, c0 * (1 - x) / (1 - xp))

    def closed(key):
        return lambda v: modal.dst_solution(n_t, with_param(d, key, v), u0, u0, d["n_samples"], d["pickup"])

    for w, key in enumerate(oracle.GRAD_PARAMS):
        y, dy = oracle.complex_step(d, w)
        if key == "alpha":
            continue   # no alpha in the linear closed form (pinned below on nonlinear strings)
        if key == "amplitude":
            assert rel(dy, y / d["excitation"]["amp"]) <= 1e-13
            continue
        step, tol = {"kappa": (3e-6, 1e-6), "sigma0": (1e-5, 1e-5), "sigma1": (1e-4, 5e-4)}[key]
        ref = central4(closed(key), d[key], step * d[key])
        assert rel(dy, ref) <= tol, (key, rel(dy, ref))


@pytest.mark.parametrize("case", ["pluck", "hammer", "vibrato"])
def test_nonlinear_derivatives_equal_fourth_order_differences(case):
    if case == "pluck":
        d = W.make(alpha=3.0, sigma0=0.7, sigma1=2e-5, excitation={"kind": "pluck", "amp": 4e-3, "pos": 0.23})
    elif case == "hammer":
        # contact from the first step to its end: smooth in every parameter
        # as long as the perturbation does not move the step contact ends
        d = W.make(alpha=2.0, f0=90.0, kappa=1.4, sigma0=0.6, sigma1=4e-5,
                   excitation={"kind": "hammer", "mass": 5e-3, "vel": 2.5, "pos": 0.3, "omega": 3000.0,
                               "alpha": 2.5})
    else:
        d = W.make(alpha=1.5, kappa=0.9, sigma0=0.4, sigma1=1e-5,
                   modulation={"kind": "vibrato", "rate": 6.0, "depth": 40.0, "phase": 0.3})
    d = dict(d, n_samples=1500)
    n_t, n_l = oracle.grid(d)
    for w, key in enumerate(oracle.GRAD_PARAMS):
        _, dy = oracle.complex_step(d, w, n_t=n_t, n_l=n_l)
        p0 = param(d, key)
        e = 1e-5 * (p0 - 1.0 if key == "alpha" else p0)
        ref = central4(lambda v: oracle.run(with_param(d, key, v), n_t=n_t, n_l=n_l), p0, e)
        tol = {"sigma0": 2e-4, "sigma1": 2e-3}.get(key, 1e-4)
        assert rel(dy, ref) <= tol, (case, key, rel(dy, ref))
        assert np.linalg.norm(dy) > 0


def test_loss_gradient_is_the_sum_of_output_derivatives():
    d = dict(W.make(alpha=2.5, excitation={"kind": "pluck", "amp": 3e-3, "pos": 0.27}), n_samples=600)
    tgt = oracle.run(with_param(d, "kappa", d["kappa"] * 1.03))
    g = oracle.loss_gradient_cs(d, tgt)
    y = oracle.run(d)
    for w in range(len(oracle.GRAD_PARAMS)):
        _, dy = oracle.complex_step(d, w)
        assert g[w] == pytest.approx(float(np.sum(2 * (y - tgt) * dy)), rel=1e-12)
    assert math.isfinite(float(np.sum(g)))
