"""Seeded synthetic string workloads.

This module only draws parameters; it holds none of the scheme's arithmetic
(no grid rule, no coefficient, no update).  The CUDA path and the FP64 oracle
both read the same parameter dictionaries and each converts them into its own
structures.

A string is a plain dict with SI units:

    f0 [Hz], kappa [1/s], alpha, sigma0 [1/s], sigma1, theta, fs [Hz],
    length [m], rho_a [kg/m], boundary (0 clamped, 1 simply supported),
    grid_rule (0 theta bound, 1 printed rule), pickup (fraction of L),
    excitation: {"kind": "pluck", "amp": m, "pos": frac}
              | {"kind": "hammer", "mass": kg, "vel": m/s, "pos": frac,
                 "omega": 1/s, "alpha": -}
              | {"kind": "bow", "vel": m/s, "force": N, "pos": frac,
                 "a": s/m, "eps": -, "release": s (<0: never)}
    modulation: {"kind": "none"} | {"kind": "vibrato", "rate": Hz,
                 "depth": cents, "phase": rad}
              | {"kind": "gliss", "depth": octaves, "duration": s}
    n_samples: output samples requested.

Parameter ranges follow the paper's Table 1 and its experiments (Sec. 4) and
the five benchmark workloads; the draws are uniform or log-uniform as named.
"""

from __future__ import annotations

import copy
import math

import numpy as np

THETA_DEFAULT = 0.5 * (1.0 + 4.0 / math.pi ** 2)   # Sec. 3.2

BASE = dict(
    f0=110.0, kappa=1.0, alpha=1.0, sigma0=0.5, sigma1=1e-5,
    theta=THETA_DEFAULT, fs=48000.0, length=1.0, rho_a=5e-3,
    boundary=0, grid_rule=0, pickup=0.7,
    excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3},
    modulation={"kind": "none"},
    n_samples=48000,
)


def make(**kw) -> dict:
    """A string dict: BASE overridden by keyword arguments."""
    d = copy.deepcopy(BASE)
    for k, v in kw.items():
        d[k] = copy.deepcopy(v)
    return d


def single_string(alpha: float = 1.0, seconds: float = 1.0) -> dict:
    """Single plucked string: f0 = 110 Hz, kappa = 1, sigma0 = 0.5,
    sigma1 = 1e-5, 1 mm pluck at 0.3 L, pickup 0.7 L, 48 kHz."""
    return make(alpha=alpha, n_samples=int(round(48000 * seconds)))


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _excitation(rng, kind: str) -> dict:
    if kind == "pluck":
        return {"kind": "pluck", "amp": float(rng.uniform(0.1e-3, 2e-3)),
                "pos": float(rng.uniform(0.1, 0.5))}
    if kind == "hammer":
        return {"kind": "hammer", "mass": float(rng.uniform(1e-3, 10e-3)),
                "vel": float(rng.uniform(0.5, 5.0)), "pos": float(rng.uniform(0.1, 0.5)),
                "omega": 3000.0, "alpha": 2.5}
    if kind == "bow":
        return {"kind": "bow", "vel": float(rng.uniform(0.05, 0.5)),
                "force": float(rng.uniform(0.1, 2.0)), "pos": float(rng.uniform(0.1, 0.5)),
                "a": 100.0, "eps": 0.1, "release": -1.0}
    raise ValueError(kind)


def random_string(rng, f0_lo=40.0, f0_hi=1000.0, kinds=("pluck", "hammer", "bow"),
                  seconds=2.0, fs=48000.0) -> dict:
    """One string drawn from the mixed-excitation distribution:
    f0 log-uniform, kappa U[0.5,3], alpha U[1,10], sigma0 U[0.1,2],
    sigma1 U[1e-6,1e-4], excitation uniform over `kinds`, pickup U[0.55,0.9]."""
    kind = kinds[int(rng.integers(len(kinds)))]
    return make(
        f0=float(_loguniform(rng, f0_lo, f0_hi)),
        kappa=float(rng.uniform(0.5, 3.0)),
        alpha=float(rng.uniform(1.0, 10.0)),
        sigma0=float(rng.uniform(0.1, 2.0)),
        sigma1=float(rng.uniform(1e-6, 1e-4)),
        pickup=float(rng.uniform(0.55, 0.9)),
        excitation=_excitation(rng, kind),
        fs=fs,
        n_samples=int(round(fs * seconds)),
    )


def batch_mixed(n: int = 256, seconds: float = 2.0, seed: int = 2) -> list[dict]:
    """Batch of n strings with mixed pluck / hammer / bow excitation,
    f0 log-uniform 40-1000 Hz (256 strings x 2 s is the headline workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [random_string(rng, seconds=seconds) for _ in range(n)]


def batch_modulated(n: int = 4096, seconds: float = 4.0, seed: int = 3) -> list[dict]:
    """Uneven-N batch with f0 modulation: f0 log-uniform 30-2000 Hz, half the
    strings with vibrato (rate U[5,7] Hz, +-20 cents, random phase), half with
    a glissando of +-1 octave (linear in log f over the note)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        d = random_string(rng, f0_lo=30.0, f0_hi=2000.0, seconds=seconds)
        if i % 2 == 0:
            d["modulation"] = {"kind": "vibrato", "rate": float(rng.uniform(5.0, 7.0)),
                               "depth": 20.0, "phase": float(rng.uniform(0, 2 * math.pi))}
        else:
            d["modulation"] = {"kind": "gliss", "depth": float(rng.choice([-1.0, 1.0])),
                               "duration": seconds}
        out.append(d)
    return out


def batch_gradient(n: int = 64, seconds: float = 0.5, seed: int = 4):
    """Differentiation workload: n plucked or hammered strings and their
    targets, the same strings with every differentiable parameter scaled by
    (1 + U[-5%, 5%])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base, target = [], []
    for _ in range(n):
        d = random_string(rng, kinds=("pluck", "hammer"), seconds=seconds)
        t = copy.deepcopy(d)
        for key in ("kappa", "alpha", "sigma0", "sigma1"):
            t[key] = d[key] * float(1.0 + rng.uniform(-0.05, 0.05))
        t["alpha"] = max(1.0, t["alpha"])
        ex = t["excitation"]
        amp_key = "amp" if ex["kind"] == "pluck" else "vel"
        ex[amp_key] = ex[amp_key] * float(1.0 + rng.uniform(-0.05, 0.05))
        base.append(d)
        target.append(t)
    return base, target


def serving_trace(rate_hz: float = 2000.0, seconds: float = 60.0, seed: int = 5,
                  fs: float = 48000.0) -> list[tuple[float, dict]]:
    """Poisson note requests: (arrival time [s], string dict); f0 log-uniform
    40-1000 Hz, duration U[0.25,4] s, excitation and parameters as in
    `random_string`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= seconds:
            break
        dur = float(rng.uniform(0.25, 4.0))
        out.append((t, random_string(rng, seconds=dur, fs=fs)))
    return out
