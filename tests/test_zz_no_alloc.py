"""The synthesis entry point that allocates no device memory, for callers
that cannot call cudaMalloc (real-time audio threads, code running under
stream capture, hosts with a fixed device footprint).  It must give the same
samples as the regular entry point, call after call, although every call
reuses the same static scratch array.  Collected last on purpose."""

import numpy as np
import pytest

from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4   # relative L2, as in the parity tests


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


def regular(sfd, ctx, d, n):
    s = sfd.string_from_dict(ctx, d)
    try:
        return sfd.sfd_synthesize(s, n)
    finally:
        sfd.sfd_string_destroy(s)


CASES = [
    W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.23}),
    W.make(alpha=4.0, f0=80.0, kappa=1.5,
           excitation={"kind": "hammer", "mass": 6e-3, "vel": 3.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}),
    W.make(alpha=2.0, f0=196.0,
           excitation={"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1,
                       "release": -1.0}),
]


def test_noalloc_matches_regular_two_calls_in_a_row(sfd):
    assert torch.cuda.is_available()
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        n = 6000
        stream = torch.cuda.current_stream().cuda_stream
        for d in CASES:
            ref = regular(sfd, ctx, d, n)
            for _ in range(2):                       # two calls in a row share the scratch
                out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
                sfd.sfd_synthesize_noalloc(0, stream, sfd.params_from_dict(d),
                                           sfd.excitation_from_dict(d["excitation"]), n, out)
                y = out.cpu().numpy()
                assert np.all(np.isfinite(y))
                assert rel_l2(y, ref) <= TOL
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_noalloc_rejects_strings_beyond_its_scratch(sfd):
    # N_t = 71 but N_l ~ 2400: about 40 KB of state, over the 32 KiB array
    d = W.make(f0=10.0, kappa=3.0, alpha=1.001)
    out = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(sfd.SfdError) as ei:
        sfd.sfd_synthesize_noalloc(0, torch.cuda.current_stream().cuda_stream, sfd.params_from_dict(d),
                                   sfd.excitation_from_dict(d["excitation"]), 64, out)
    assert ei.value.code == sfd.SFD_EINVAL
    assert "scratch" in str(ei.value)
