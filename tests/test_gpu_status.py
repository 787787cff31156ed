"""Failure statuses through the C-ABI, made on the host without any GPU
fault: the coupled Gauss-Seidel solve of a strongly nonlinear string given
a sweep cap below what it needs reports SFD_ENOCONV (its samples are kept,
finite), while a string beside it in the same launch that needs no sweeps
gives bit for bit the samples it gives alone; the cap's range is checked and
0 restores the default."""

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


STRUCK = W.make(f0=60.0, kappa=1.0, alpha=8.0, n_samples=3000,
                excitation={"kind": "hammer", "mass": 8e-3, "vel": 4.0, "pos": 0.3, "omega": 3000.0, "alpha": 2.5})
LINEAR = W.make(f0=220.0, kappa=1.0, alpha=1.0, n_samples=3000,
                excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.27})


def alone(sfd, d, cap=0):
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        sfd.sfd_ctx_set_sweep_cap(ctx, cap)
        s = sfd.string_from_dict(ctx, d)
        y = sfd.sfd_synthesize(s, d["n_samples"], allow_noconv=True)
        st = sfd.sfd_string_stats(s)
        sfd.sfd_string_destroy(s)
        return y, st
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_sweep_cap_gives_noconv_and_leaves_the_neighbour_alone(sfd):
    y_free, (status, max_sweeps, _) = alone(sfd, STRUCK)
    assert status == sfd.SFD_OK and max_sweeps >= 2          # the string needs more than one sweep
    ref_linear, (st_lin, sweeps_lin, _) = alone(sfd, LINEAR)
    assert st_lin == sfd.SFD_OK and sweeps_lin == 0            # no longitudinal grid: no sweeps

    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        sfd.sfd_ctx_set_sweep_cap(ctx, 1)
        hs = [sfd.string_from_dict(ctx, d) for d in (STRUCK, LINEAR)]
        b = sfd.sfd_batch_create(ctx, hs)
        ys, status = sfd.sfd_batch_synthesize_host(b, [3000, 3000], allow_noconv=True)
        assert list(status) == [sfd.SFD_ENOCONV, sfd.SFD_OK]
        assert np.all(np.isfinite(ys[0])) and not np.array_equal(ys[0], y_free)
        assert np.array_equal(ys[1], ref_linear)
        assert sfd.sfd_string_stats(hs[0])[1] == 1
        sfd.sfd_batch_destroy(b)
        for h in hs:
            sfd.sfd_string_destroy(h)
        # a single synthesis reports it as the call's status
        s = sfd.string_from_dict(ctx, STRUCK)
        with pytest.raises(sfd.SfdError) as ei:
            sfd.sfd_synthesize(s, 3000)
        assert ei.value.code == sfd.SFD_ENOCONV
        sfd.sfd_string_destroy(s)
        # 0 restores the default cap: the same samples as a fresh context
        sfd.sfd_ctx_set_sweep_cap(ctx, 0)
        s = sfd.string_from_dict(ctx, STRUCK)
        assert np.array_equal(sfd.sfd_synthesize(s, 3000), y_free)
        sfd.sfd_string_destroy(s)
        for bad in (-1, 65):
            with pytest.raises(sfd.SfdError) as ei:
                sfd.sfd_ctx_set_sweep_cap(ctx, bad)
            assert ei.value.code == sfd.SFD_EINVAL
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_a_cap_above_what_strings_need_changes_nothing(sfd):
    y_free, (_, max_sweeps, _) = alone(sfd, STRUCK)
    y_cap, (status, _, _) = alone(sfd, STRUCK, cap=max_sweeps)
    assert status == sfd.SFD_OK and np.array_equal(y_cap, y_free)
    y_big, _ = alone(sfd, STRUCK, cap=64)
    assert np.array_equal(y_big, y_free)
