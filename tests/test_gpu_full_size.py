"""The 4096-string x 4 s modulated batch, the largest one-GPU workload, in the
launch configuration bench.py times (warps per CTA autotuned on throwaway
copies, the prepared launch captured as one CUDA graph and replayed, output
in device memory): every output sample finite and every string's status OK
(properties that hold at any size), and a spread of 40 strings (both
modulation kinds, every excitation, every kernel class) against the FP64
oracle sample by sample.

Bars: a plucked or struck string within 1e-4 relative L2 over the first
0.25 s and over its whole 4 s note (measured on a spread of 20 such strings:
at most 8.5e-6 and 5.5e-5).  Over a whole note, phase drift grows with
f0 t: for a note whose inputs' own conditioning at FP32 precision over 4 s
(the coefficient floor: the FP64 oracle's output moved by rounding one of
f0, alpha, kappa, sigma0, sigma1 to FP32) exceeds 1e-4, the whole-note bar
is that floor (a vibrato note at 1.64 kHz: 1.02e-4 against a floor of
1.3e-3; its first 0.25 s at 1.4e-5 meets 1e-4).  A bowed string within 1e-4 over its first
0.125 s (the bar of the 256-string batch's bowed strings).  Over whole notes
a bowed string near a bifurcation can settle into another periodic regime
under FP32-sized perturbations (several did, at relative L2 ~1 over 4 s),
so bowed notes are held to the short window only.  The one exception is the
256-string batch's: a struck string whose hammer chatters (four or more
separate contacts within 0.25 s, counted on the oracle) and whose FP32
state floor (the oracle's own output moved by rounding its state to FP32)
exceeds 1e-4 is held to three times that floor over 0.25 s; at most two of
the spread may use it."""

import numpy as np
import pytest

import oracle
from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
HEAD = 12000        # 0.25 s
BOW_WINDOW = 6000   # 0.125 s
PICKS = list(range(5, 4096, 103))   # 40 strings, both parities (vibrato and glissando)


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def contact_episodes(d, n):
    """Separate hammer contacts of the oracle's trajectory over n samples."""
    s = oracle.OracleString(d)
    s.run(2)
    episodes, inside = 0, False
    for _ in range(n - 2):
        s.run(1)
        c = s.state()[4][3] > 0          # the contact stiffness of the last step
        episodes += c and not inside
        inside = c
    return episodes


def test_full_size_batch_in_the_benchmark_configuration(sfd):
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    strings = W.batch_modulated(4096, seconds=4.0, seed=3)
    ctx = sfd.sfd_ctx_create(0, stream.cuda_stream, 1 << 30)
    try:
        ns = np.array([d["n_samples"] for d in strings], np.int64)
        offs = np.zeros(len(ns), np.int64)
        offs[1:] = np.cumsum(ns)[:-1]
        out = torch.empty(int(ns.sum()), dtype=torch.float32, device="cuda")
        hs = [sfd.string_from_dict(ctx, d) for d in strings]
        b = sfd.sfd_batch_create(ctx, hs)
        wpc = sfd.sfd_batch_autotune(b, 2048)
        sfd.sfd_batch_set_warps_per_cta(b, wpc)
        sfd.sfd_batch_prepare(b, ns, out, offs)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sfd.sfd_batch_launch(b)
        g.replay()
        torch.cuda.synchronize()
        assert bool(torch.isfinite(out).all().item())
        assert all(sfd.sfd_string_stats(h)[0] == sfd.SFD_OK for h in hs)
        classes = {sfd.sfd_string_kernel_class(hs[i]) for i in PICKS}
        ys = {i: out[offs[i]:offs[i] + ns[i]].cpu().numpy() for i in PICKS}
        del g
        sfd.sfd_batch_destroy(b)
        for h in hs:
            sfd.sfd_string_destroy(h)
    finally:
        sfd.sfd_ctx_destroy(ctx)
        torch.cuda.set_stream(torch.cuda.default_stream())

    sel = [strings[i] for i in PICKS]
    kinds = {d["excitation"]["kind"] for d in sel}
    mods = {d["modulation"]["kind"] for d in sel}
    assert kinds == {"pluck", "hammer", "bow"} and mods == {"vibrato", "gliss"} and len(classes) >= 3
    refs, _ = oracle.run_batch(sel)
    worst, beyond, drift = {}, [], []
    for i, d, ref in zip(PICKS, sel, refs):
        y = ys[i]
        kind = d["excitation"]["kind"]
        if kind == "bow":
            e = rel_l2(y[:BOW_WINDOW], ref[:BOW_WINDOW])
            worst["bow"] = max(worst.get("bow", 0.0), e)
            assert e <= TOL, (i, d["f0"], d["modulation"], e)
        else:
            e_head, e_all = rel_l2(y[:HEAD], ref[:HEAD]), rel_l2(y, ref)
            if e_head <= TOL and e_all <= TOL:
                worst["head"] = max(worst.get("head", 0.0), e_head)
                worst["note"] = max(worst.get("note", 0.0), e_all)
                continue
            if e_head <= TOL:   # whole-note drift: within the note's coefficient floor
                from fp32_floor import coefficient_floor
                cf = coefficient_floor(d, d["n_samples"])
                assert cf > TOL and e_all <= cf, (i, kind, d["f0"], e_all, cf)
                drift.append((i, e_all, cf))
                continue
            # the chatter exception (see the module docstring)
            from fp32_floor import fp32_state_floor
            dd = dict(d, n_samples=HEAD)
            assert kind == "hammer" and contact_episodes(dd, HEAD) >= 4, (i, kind, d["f0"], e_head, e_all)
            floor = fp32_state_floor(dd, HEAD)
            assert floor > TOL and e_head <= 3 * floor, (i, d["f0"], e_head, floor)
            beyond.append((i, e_head, floor))
    assert len(beyond) <= 2, beyond
    print("worst rel-L2:", {k: f"{v:.2e}" for k, v in worst.items()}, "chatter:", beyond, "drift:", drift)
