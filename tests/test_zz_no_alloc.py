"""The synthesis entry point that allocates no device memory, for callers
that cannot call cudaMalloc: a real-time audio thread (cudaMalloc may
synchronise the device and block for an unbounded time) or a host that fixes
a library's device footprint in advance.  It runs the same kernels on the
same state as the regular entry point, so its samples must be bit for bit the
same, call after call, although every call reuses one static scratch array.
It refuses what it cannot do (a string beyond the scratch or beyond one
warp's shared memory, a capturing stream) without enqueueing anything.
Collected last on purpose."""

import ctypes

import numpy as np
import pytest

from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


HAMMER = {"kind": "hammer", "mass": 6e-3, "vel": 3.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}
CASES = [
    W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.23}),
    W.make(alpha=4.0, f0=80.0, kappa=1.5, excitation=HAMMER),
    W.make(alpha=2.0, f0=196.0,
           excitation={"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1,
                       "release": -1.0}),
]


def raw_call(sfd, stream, d, n, out):
    """The C entry point itself: (status, message)."""
    p, e = sfd.params_from_dict(d), sfd.excitation_from_dict(d["excitation"])
    ptr = out.data_ptr() if out is not None else None
    rc = sfd.lib().sfd_synthesize_noalloc(0, stream, ctypes.byref(p), ctypes.byref(e), n, ptr)
    return rc, sfd.sfd_last_error()


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
                assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_noalloc_rejects_strings_beyond_its_scratch(sfd):
    # N_t = 71 but N_l ~ 2400: about 40 KB of state, over the 32 KiB array
    d = W.make(f0=10.0, kappa=3.0, alpha=1.001)
    out = torch.zeros(64, dtype=torch.float32, device="cuda")
    rc, msg = raw_call(sfd, torch.cuda.current_stream().cuda_stream, d, 64, out)
    assert rc == sfd.SFD_EINVAL and "scratch" in msg


def test_noalloc_rejects_grids_beyond_one_warps_shared_memory(sfd):
    # a linear string with N_t ~ 3050: its state fits the scratch array, but
    # the shared-memory step kernel would need ~236 KB for one warp
    d = W.make(f0=5.0, kappa=0.0, alpha=1.0)
    n_t, n_l = sfd.sfd_grid(sfd.params_from_dict(d))
    assert n_t > 3000
    out = torch.full((64,), 7.0, dtype=torch.float32, device="cuda")
    rc, msg = raw_call(sfd, torch.cuda.current_stream().cuda_stream, d, 64, out)
    assert rc == sfd.SFD_EINVAL and "shared memory" in msg
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0))


def test_noalloc_zero_samples_writes_nothing_but_validates(sfd):
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full((16,), 3.0, dtype=torch.float32, device="cuda")
    rc, _ = raw_call(sfd, stream, CASES[1], 0, out)
    assert rc == sfd.SFD_OK
    torch.cuda.synchronize()
    assert bool(torch.all(out == 3.0))
    bad = dict(CASES[1], alpha=0.5)            # alpha < 1: refused even with nothing to write
    rc, msg = raw_call(sfd, stream, bad, 0, out)
    assert rc == sfd.SFD_EINVAL and "alpha" in msg


def test_noalloc_reports_the_string_status(sfd):
    """A string on the printed grid (reading A5: unstable with theta = 0.70)
    ends with SFD_EUNSTABLE, plucked or struck, as through a context."""
    stream = torch.cuda.current_stream().cuda_stream
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        for ex in ({"kind": "pluck", "amp": 1e-3, "pos": 0.3}, HAMMER):
            d = W.make(grid_rule=1, sigma0=0.0, sigma1=0.0, excitation=ex)
            n = 4000
            out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
            rc, _ = raw_call(sfd, stream, d, n, out)
            assert rc == sfd.SFD_EUNSTABLE
            s = sfd.string_from_dict(ctx, d)
            try:
                y = np.zeros(n, dtype=np.float32)
                rc2 = sfd.lib().sfd_synthesize(s, n, y.ctypes.data, 0)
            finally:
                sfd.sfd_string_destroy(s)
            assert rc2 == sfd.SFD_EUNSTABLE
            assert np.array_equal(out.cpu().numpy(), y)
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_noalloc_refuses_a_capturing_stream(sfd):
    """The call copies from host memory and waits for its stream, which a
    CUDA graph cannot hold: on a capturing stream it returns SFD_EINVAL and
    enqueues nothing.  The first call on the device (the scratch address
    look-up) comes before the capture."""
    d, n = CASES[0], 512
    s = torch.cuda.Stream()
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    rc, _ = raw_call(sfd, s.cuda_stream, d, n, out)
    assert rc == sfd.SFD_OK
    torch.cuda.synchronize()
    out.fill_(5.0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc, msg = raw_call(sfd, s.cuda_stream, d, n, out)
    assert rc == sfd.SFD_EINVAL and "capturing" in msg
    torch.cuda.synchronize()
    assert bool(torch.all(out == 5.0))
    # the stream is usable afterwards, with the same result as before
    rc, _ = raw_call(sfd, s.cuda_stream, d, n, out)
    assert rc == sfd.SFD_OK
    torch.cuda.synchronize()
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        assert np.array_equal(out.cpu().numpy(), regular(sfd, ctx, d, n))
    finally:
        sfd.sfd_ctx_destroy(ctx)
