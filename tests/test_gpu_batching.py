"""Batching of uneven strings with f0 modulation (4096 strings of uneven N in
one launch per kernel class, CUDA-graph replay, autotuned warps per CTA):
results must not depend on how a batch is launched, and a subset of the
modulated workload must match the FP64 oracle."""

import numpy as np
import pytest

import oracle
from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def make_batch(sfd, ctx, strings):
    hs = [sfd.string_from_dict(ctx, d) for d in strings]
    return hs, sfd.sfd_batch_create(ctx, hs)


def free(sfd, hs, b):
    sfd.sfd_batch_destroy(b)
    for h in hs:
        sfd.sfd_string_destroy(h)


def test_graph_replay_equals_direct_chunks(sfd):
    """Chunks of 1024 samples: a captured CUDA graph replayed 6 times gives
    bitwise the samples of 6 direct batch calls."""
    stream = torch.cuda.Stream()
    ctx = sfd.sfd_ctx_create(0, stream.cuda_stream, 256 << 20)
    try:
        strings = W.batch_modulated(48, seconds=0.2, seed=31)
        n, chunks = 1024, 6
        ns = np.full(len(strings), n, np.int64)
        offs = np.arange(len(strings), dtype=np.int64) * n
        # direct
        hs, b = make_batch(sfd, ctx, strings)
        out = torch.zeros(len(strings) * n, device="cuda")
        direct = []
        with torch.cuda.stream(stream):
            for _ in range(chunks):
                sfd.sfd_batch_synthesize(b, ns, out, offs)
                direct.append(out.cpu().numpy().copy())
        free(sfd, hs, b)
        # captured
        hs, b = make_batch(sfd, ctx, strings)
        out2 = torch.zeros(len(strings) * n, device="cuda")
        sfd.sfd_batch_prepare(b, ns, out2, offs)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sfd.sfd_batch_launch(b)
        graphed = []
        for _ in range(chunks):
            g.replay()
            torch.cuda.synchronize()
            graphed.append(out2.cpu().numpy().copy())
        # the capture itself did not run the kernels: state advanced only by replays
        free(sfd, hs, b)
        for a, c in zip(direct, graphed):
            assert np.array_equal(a, c)
    finally:
        torch.cuda.synchronize()
        sfd.sfd_ctx_destroy(ctx)


def test_string_changed_after_prepare_is_uploaded_at_launch(sfd):
    """A string excited again after sfd_batch_prepare (allowed until it first
    runs) starts from its new initial state when sfd_batch_launch runs the
    batch; every string equals its own synthesis alone."""
    ctx = sfd.sfd_ctx_create(0, None, 128 << 20)
    try:
        strings = W.batch_mixed(6, seconds=0.05, seed=7)
        n = 1000
        ns = np.full(len(strings), n, np.int64)
        offs = np.arange(len(strings), dtype=np.int64) * n
        hs, b = make_batch(sfd, ctx, strings)
        out = torch.zeros(len(strings) * n, device="cuda")
        torch.cuda.synchronize()
        sfd.sfd_batch_prepare(b, ns, out, offs)
        assert strings[2]["excitation"]["kind"] == "hammer"
        hit = {"kind": "hammer", "mass": 7e-3, "vel": 4.5, "pos": 0.41, "omega": 2500.0, "alpha": 2.2}
        sfd.sfd_excite_hammer(hs[2], hit["mass"], hit["vel"], hit["pos"], hit["omega"], hit["alpha"])
        sfd.sfd_batch_launch(b)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(len(strings), n)
        free(sfd, hs, b)
        for i, d in enumerate(strings):
            s = sfd.string_from_dict(ctx, dict(d, excitation=hit) if i == 2 else d)
            try:
                assert np.array_equal(got[i], sfd.sfd_synthesize(s, n)), i
            finally:
                sfd.sfd_string_destroy(s)
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_autotune_does_not_advance_strings(sfd):
    ctx = sfd.sfd_ctx_create(0, None, 256 << 20)
    try:
        strings = W.batch_mixed(40, seconds=0.05, seed=41)
        ns = [d["n_samples"] for d in strings]
        hs, b = make_batch(sfd, ctx, strings)
        best = sfd.sfd_batch_autotune(b, 256)
        assert best in (1, 2, 4)
        ys, _ = sfd.sfd_batch_synthesize_host(b, ns)
        free(sfd, hs, b)
        hs, b = make_batch(sfd, ctx, strings)
        ref, _ = sfd.sfd_batch_synthesize_host(b, ns)
        free(sfd, hs, b)
        for a, c in zip(ys, ref):
            assert np.array_equal(a, c)
    finally:
        sfd.sfd_ctx_destroy(ctx)


@pytest.mark.parametrize("wpc", [1, 2, 4])
def test_warps_per_cta_does_not_change_results(sfd, wpc):
    ctx = sfd.sfd_ctx_create(0, None, 256 << 20)
    try:
        strings = W.batch_mixed(20, seconds=0.03, seed=43)
        ns = [d["n_samples"] for d in strings]
        hs, b = make_batch(sfd, ctx, strings)
        sfd.sfd_batch_set_warps_per_cta(b, wpc)
        ys, _ = sfd.sfd_batch_synthesize_host(b, ns)
        free(sfd, hs, b)
        for d, y in zip(strings, ys):
            s = sfd.string_from_dict(ctx, d)
            assert np.array_equal(y, sfd.sfd_synthesize(s, d["n_samples"]))
            sfd.sfd_string_destroy(s)
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_modulated_uneven_subset_matches_oracle(sfd):
    """Strings of the 4096-string modulated workload (f0 30-2000 Hz, vibrato
    and glissando, uneven N) synthesized together in one batch: the first
    0.25 s of a spread of them against the oracle (bowed: 150 samples)."""
    ctx = sfd.sfd_ctx_create(0, None, 512 << 20)
    try:
        full = W.batch_modulated(4096, seconds=4.0, seed=3)
        picks = [0, 1, 2, 3, 100, 101, 777, 1500, 2048, 3001, 4094, 4095]
        strings = [dict(full[i], n_samples=12000) for i in picks]
        grids = [oracle.grid(d) for d in strings]
        assert min(g[0] for g in grids) < 20 and max(g[0] for g in grids) > 60   # uneven N
        hs, b = make_batch(sfd, ctx, strings)
        ys, st = sfd.sfd_batch_synthesize_host(b, [12000] * len(strings))
        free(sfd, hs, b)
        assert np.all(st == 0)
        for d, y in zip(strings, ys):
            n = 150 if d["excitation"]["kind"] == "bow" else 12000
            ref = oracle.run(d, n)
            assert rel_l2(y[:n], ref) <= (1e-3 if n == 150 else TOL), (d["f0"], d["modulation"])
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_highest_f0_modulated_strings_match_oracle(sfd):
    """The 24 highest non-bowed notes of the modulated workload (f0 about
    1.9-2 kHz, grids of 3-8 intervals): the most periods in 0.25 s, so the
    largest phase error FP32 coefficients or factors could accumulate."""
    ctx = sfd.sfd_ctx_create(0, None, 256 << 20)
    try:
        full = W.batch_modulated(4096, seconds=4.0, seed=3)
        order = sorted((i for i in range(len(full)) if full[i]["excitation"]["kind"] != "bow"),
                       key=lambda i: -full[i]["f0"])[:24]
        strings = [dict(full[i], n_samples=12000) for i in order]
        assert min(d["f0"] for d in strings) > 1800
        hs, b = make_batch(sfd, ctx, strings)
        ys, st = sfd.sfd_batch_synthesize_host(b, [12000] * len(strings))
        free(sfd, hs, b)
        assert np.all(st == 0)
        refs, _ = oracle.run_batch(strings, n_samples=12000)
        for d, y, ref in zip(strings, ys, refs):
            assert rel_l2(y, ref) <= TOL, (d["f0"], d["modulation"])
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_modulated_batch_all_finite(sfd):
    """512 strings of the modulated workload, 0.5 s, graph-replayed in 4
    chunks: every sample finite and every string's status OK."""
    stream = torch.cuda.Stream()
    ctx = sfd.sfd_ctx_create(0, stream.cuda_stream, 512 << 20)
    try:
        strings = W.batch_modulated(512, seconds=0.5, seed=3)
        n = 6000
        ns = np.full(len(strings), n, np.int64)
        offs = np.arange(len(strings), dtype=np.int64) * n
        hs, b = make_batch(sfd, ctx, strings)
        out = torch.zeros(len(strings) * n, device="cuda")
        sfd.sfd_batch_prepare(b, ns, out, offs)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sfd.sfd_batch_launch(b)
        for _ in range(4):
            g.replay()
            torch.cuda.synchronize()
            assert torch.isfinite(out).all().item()
        for h in hs:
            assert sfd.sfd_string_stats(h)[0] == 0
        free(sfd, hs, b)
    finally:
        torch.cuda.synchronize()
        sfd.sfd_ctx_destroy(ctx)


def test_warp_pairs_change_nothing(sfd):
    """Strings stepped by a pair of warps give the same bits as on one warp:
    the mixed batch (both channels) and a fine longitudinal grid alone."""
    ctx = sfd.sfd_ctx_create(0, None, 512 << 20)
    try:
        strings = W.batch_mixed(48, seconds=0.05, seed=29)
        strings += [dict(d, output="longitudinal") for d in strings[:16]]
        strings.append(W.make(f0=45.0, alpha=1.3, kappa=0.6, excitation={"kind": "hammer", "mass": 6e-3,
                              "vel": 3.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}, n_samples=2400))
        out = []
        for pairs in (True, False):
            sfd.sfd_ctx_set_warp_pairs(ctx, pairs)
            hs = [sfd.string_from_dict(ctx, d) for d in strings]
            b = sfd.sfd_batch_create(ctx, hs)
            ys, st = sfd.sfd_batch_synthesize_host(b, [d["n_samples"] for d in strings], allow_noconv=True)
            sfd.sfd_batch_destroy(b)
            states = [sfd.sfd_string_state(h) for h in hs]
            for h in hs:
                sfd.sfd_string_destroy(h)
            out.append((ys, st, states))
        (ya, sa, za), (yb, sb, zb) = out
        assert np.array_equal(sa, sb)
        for a, b in zip(ya, yb):
            assert np.array_equal(a, b)
        for a, b in zip(za, zb):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    finally:
        sfd.sfd_ctx_destroy(ctx)


def test_modulation_grows_the_grid_before_the_first_synthesis(sfd):
    """A string created without room for its modulation's peak (f0_max_ratio
    1, a grid too fine to be stable at the peak wave speed) gets the grid of
    that peak from sfd_set_modulation (reading A14), with
    its hammer at the same position: grid and samples equal a string sized
    for the peak at creation, bit for bit.  In a batch the grid can no
    longer change (SFD_EBUSY)."""
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        d = W.make(f0=150.0, kappa=1.2, alpha=3.0, n_samples=3000,
                   excitation={"kind": "hammer", "mass": 5e-3, "vel": 2.0, "pos": 0.27, "omega": 3000.0,
                               "alpha": 2.5},
                   modulation={"kind": "gliss", "depth": 1.0, "duration": 0.0625})
        sized = sfd.string_from_dict(ctx, d)
        late = sfd.string_from_dict(ctx, dict(d, gamma_max_ratio=1.0, modulation={"kind": "none"}))
        small = sfd.sfd_string_info(late)[:2]
        sfd.sfd_set_modulation(late, sfd.SFD_MOD_GLISS, 0.0, 1.0, 0.0, 0.0625)
        assert sfd.sfd_string_info(late)[:2] == sfd.sfd_string_info(sized)[:2] == sfd.sfd_grid(sfd.params_from_dict(d))
        assert sfd.sfd_string_info(late)[0] < small[0]   # a faster peak wave: a coarser grid
        assert np.array_equal(sfd.sfd_synthesize(late, 3000), sfd.sfd_synthesize(sized, 3000))
        sfd.sfd_string_destroy(late)
        sfd.sfd_string_destroy(sized)
        s = sfd.string_from_dict(ctx, dict(d, gamma_max_ratio=1.0, modulation={"kind": "none"}))
        b = sfd.sfd_batch_create(ctx, [s])
        with pytest.raises(sfd.SfdError) as ei:
            sfd.sfd_set_modulation(s, sfd.SFD_MOD_GLISS, 0.0, 1.0, 0.0, 0.0625)
        assert ei.value.code == sfd.SFD_EBUSY
        sfd.sfd_batch_destroy(b)
        sfd.sfd_string_destroy(s)
        # a refused modulation leaves the string as it was: grid, block and samples
        plain = dict(d, gamma_max_ratio=1.0, modulation={"kind": "none"})
        s = sfd.string_from_dict(ctx, plain)
        grid = sfd.sfd_string_info(s)[:2]
        with pytest.raises(sfd.SfdError) as ei:
            sfd.sfd_set_modulation(s, sfd.SFD_MOD_VIBRATO, float("nan"), 300.0, 0.0, 0.0)
        assert ei.value.code == sfd.SFD_EINVAL
        assert sfd.sfd_string_info(s)[:2] == grid
        ref = sfd.string_from_dict(ctx, plain)
        assert np.array_equal(sfd.sfd_synthesize(s, 3000), sfd.sfd_synthesize(ref, 3000))
        sfd.sfd_string_destroy(ref)
        sfd.sfd_string_destroy(s)
    finally:
        sfd.sfd_ctx_destroy(ctx)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_output_copies_each_class_and_nothing_else(sfd, pinned):
    """sfd_batch_synthesize_host copies each class's strings as its kernel
    ends: every string's range equals the device-output launch bit for bit,
    in any offset order, with gaps between ranges and strings of zero
    samples left unwritten, into pinned or pageable host memory."""
    ctx = sfd.sfd_ctx_create(0, None, 256 << 20)
    try:
        strings = W.batch_modulated(24, seconds=0.02, seed=47)
        ns = np.array([d["n_samples"] for d in strings], np.int64)
        ns[5] = 0
        order = np.arange(len(ns))[::-1]            # offsets in reverse string order, 37-sample gaps
        offs = np.zeros(len(ns), np.int64)
        pos = 11
        for i in order:
            offs[i] = pos
            pos += int(ns[i]) + 37
        total = pos
        hs, b = make_batch(sfd, ctx, strings)
        classes = {sfd.sfd_string_kernel_class(h) for h in hs}
        dev = torch.full((total,), 7.0, dtype=torch.float32, device="cuda")
        sfd.sfd_batch_synthesize(b, ns, dev, offs)
        torch.cuda.synchronize()
        ref = dev.cpu().numpy()
        free(sfd, hs, b)
        hs, b = make_batch(sfd, ctx, strings)
        host = torch.full((total,), 7.0, dtype=torch.float32)
        if pinned:
            host = host.pin_memory()
        rc = sfd.lib().sfd_batch_synthesize_host(
            b, ns.ctypes.data_as(sfd.ctypes.POINTER(sfd.ctypes.c_int64)), host.data_ptr(),
            offs.ctypes.data_as(sfd.ctypes.POINTER(sfd.ctypes.c_int64)), None)
        free(sfd, hs, b)
        assert rc == sfd.SFD_OK, sfd.sfd_last_error()
        got = host.numpy()
        assert len(classes) >= 2
        written = np.zeros(total, bool)
        for o, n in zip(offs, ns):
            written[o:o + n] = True
        assert np.array_equal(got[written], ref[written])
        assert np.all(got[~written] == 7.0)
    finally:
        sfd.sfd_ctx_destroy(ctx)
