"""FP32 storage floor of the scheme, measured with the oracle (test helper).

The GPU kernel keeps each string's state in FP32: u, D = u^n - u^{n-1}, the
longitudinal z and Dz.  Running the FP64 oracle with exactly that state
rounded to FP32 after every step gives the deviation that FP32 storage alone
causes for a string; a strongly nonlinear string struck hard (alpha of 5-9,
millimetre amplitudes) can amplify it far above the 1e-4 parity tolerance,
which no FP32 implementation can then meet.
"""

import numpy as np

import oracle


def fp32_state_floor(d: dict, n: int) -> float:
    """rel-L2 over n samples between the oracle and the oracle whose state is
    rounded to FP32 (in the kernel's u, D, z, Dz form) after every step."""
    ref = oracle.run(d, n)
    s = oracle.OracleString(d)
    y = list(s.run(min(n, 2)))
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    for _ in range(2, n):
        y.extend(s.run(1))
        up, u, zp, z, _ = s.state()
        u32, d32 = r32(u), r32(u - up)
        z32, dz32 = r32(z), r32(z - zp)
        s.set_state(u32 - d32, u32, z32 - dz32, z32)
    y = np.asarray(y)
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


def coefficient_floor(d: dict, n: int) -> float:
    """Largest rel-L2 change over n samples when one of f0, alpha, kappa,
    sigma0, sigma1 moves by 2^-24 relative (the rounding of an FP64 value to
    FP32), on the string's own grid.  The kernel's coefficients are FP32
    roundings of FP64 expressions in these parameters, so this is the
    problem's own conditioning at FP32 input precision.  It is large for the
    longitudinal output when a sum of transverse partials lies near a
    longitudinal mode (a near resonance of the forced zeta)."""
    n_t, n_l = oracle.grid(d)
    ref = oracle.run(d, n)
    norm = np.linalg.norm(ref)
    if norm == 0:
        return 0.0
    worst = 0.0
    for key in ("f0", "alpha", "kappa", "sigma0", "sigma1"):
        if d[key] == 0:
            continue
        p = dict(d, n_t=n_t, n_l=n_l)
        p[key] = d[key] * (1.0 + 2.0 ** -24)
        worst = max(worst, float(np.linalg.norm(oracle.run(p, n) - ref) / norm))
    return worst


def fp32_floor(d: dict, n: int) -> float:
    """FP32 state storage plus FP32 coefficient rounding (both measured with
    the oracle)."""
    return fp32_state_floor(d, n) + coefficient_floor(d, n)
