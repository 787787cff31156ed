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
