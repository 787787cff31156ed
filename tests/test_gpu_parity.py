"""GPU parity: the sm_103a kernels through the C-ABI against the FP64 oracle.

Bar (from the method's accuracy target): relative L2 error of the output
waveform <= 1e-4 over the first 0.25 s, energy drift <= 1e-5 for the
lossless scheme.  Bowed strings are compared at 1e-4 over 0.125 s (every
bowed string of the 256-string batch), and over 0.5 s at 1e-3 wherever the
FP64 trajectory is itself stable under FP32-sized state noise; a bowed note
near a bifurcation, which that noise moves into another periodic regime, is
compared by its level."""

import math

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


@pytest.fixture(scope="module")
def ctx(sfd):
    assert torch.cuda.is_available()
    c = sfd.sfd_ctx_create(0, None, 1 << 30)
    yield c
    sfd.sfd_ctx_destroy(c)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def gpu_run(sfd, ctx, d, n=None, chunks=None):
    s = sfd.string_from_dict(ctx, d)
    try:
        n = d["n_samples"] if n is None else n
        if chunks is None:
            return sfd.sfd_synthesize(s, n)
        return np.concatenate([sfd.sfd_synthesize(s, c) for c in chunks])
    finally:
        sfd.sfd_string_destroy(s)


HAMMER = {"kind": "hammer", "mass": 6e-3, "vel": 3.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5}
BOW = {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0}


@pytest.mark.parametrize("alpha", [1.0, 3.0])
def test_single_string_quarter_second(sfd, ctx, alpha):
    """f0 = 110 Hz, kappa = 1, sigma0 = 0.5, sigma1 = 1e-5, 1 mm pluck at 0.3,
    pickup 0.7: rel-L2 <= 1e-4 over 0.25 s (12,000 samples)."""
    d = W.single_string(alpha=alpha, seconds=0.25)
    y = gpu_run(sfd, ctx, d)
    assert rel_l2(y, oracle.run(d)) <= TOL


@pytest.mark.parametrize("alpha,amp", [(3.0, 5e-3), (10.0, 2e-3), (1.2, 1e-2)])
def test_nonlinear_pluck(sfd, ctx, alpha, amp):
    d = W.make(alpha=alpha, excitation={"kind": "pluck", "amp": amp, "pos": 0.23}, n_samples=12000)
    assert rel_l2(gpu_run(sfd, ctx, d), oracle.run(d)) <= TOL


@pytest.mark.parametrize("alpha", [1.0, 4.0])
def test_hammer(sfd, ctx, alpha):
    d = W.make(alpha=alpha, f0=80.0, kappa=1.5, excitation=HAMMER, n_samples=12000)
    assert rel_l2(gpu_run(sfd, ctx, d), oracle.run(d)) <= TOL


@pytest.mark.parametrize("alpha", [1.0, 2.5])
def test_bow_short_window(sfd, ctx, alpha):
    d = W.make(alpha=alpha, f0=196.0, excitation=BOW, n_samples=600)
    y = gpu_run(sfd, ctx, d)
    ref = oracle.run(d)
    assert rel_l2(y[:150], ref[:150]) <= 1e-3
    assert np.all(np.isfinite(y)) and np.max(np.abs(y)) < 10 * np.max(np.abs(ref)) + 1e-9


def oracle_with_state_noise(d, n, eps, seed):
    """The oracle's output with every level of u and zeta multiplied by
    (1 + eps N(0, 1)) noise after each step: an FP64 trajectory perturbed
    at the size of FP32 rounding."""
    rng = np.random.default_rng(seed)
    s = oracle.OracleString(d)
    y = list(s.run(2))
    for _ in range(2, n):
        up, u, zp, z, _ = s.state()
        s.set_state(up, u * (1 + eps * rng.standard_normal(u.shape)), zp,
                    z * (1 + eps * rng.standard_normal(z.shape)) if len(z) else None)
        y.extend(s.run(1))
    return np.array(y)


def test_bowed_notes_over_half_a_second(sfd, ctx):
    """Bowed notes over 0.5 s, the first 8 bowed strings of the 256-string
    batch.  Where the FP64 trajectory is stable under FP32-sized state noise
    (1e-7 relative per step keeps the oracle within 1e-3), the GPU waveform
    is within 1e-3 of the oracle over the whole note and the second half's
    fundamental within 0.2 %.  Where that noise itself moves the note into
    another periodic regime (a bowed string near a bifurcation), no FP32
    run can follow the FP64 one; there the level is what every correct run
    shares: the second half's RMS within 5 %.  Most of these strings are
    stable (at least 6 of 8 required)."""
    from pitch import peak_frequency
    n = 24000
    strings = [dict(d, n_samples=n) for d in W.batch_mixed(256, seconds=2.0, seed=2)
               if d["excitation"]["kind"] == "bow"][:8]
    refs, _ = oracle.run_batch(strings)
    stable = 0
    for i, (d, ref) in enumerate(zip(strings, refs)):
        ref = np.asarray(ref, np.float64)
        noisy = oracle_with_state_noise(d, n, 1e-7, seed=100 + i)
        y = np.asarray(gpu_run(sfd, ctx, d), np.float64)
        h = n // 2
        rms = lambda v: float(np.sqrt(np.mean(v[h:] ** 2)))
        if rel_l2(noisy, ref) <= 1e-3:
            stable += 1
            assert rel_l2(y, ref) <= 1e-3, i
            band = (0.8 * d["f0"], 1.25 * d["f0"])
            fy, fr = peak_frequency(y[h:], d["fs"], *band), peak_frequency(ref[h:], d["fs"], *band)
            assert abs(fy - fr) <= 2e-3 * fr, (i, fy, fr)
        else:
            assert abs(rms(y) - rms(ref)) <= 0.05 * rms(ref), (i, rms(y), rms(ref))
    assert stable >= 6


@pytest.mark.parametrize("case", [
    dict(f0=3000.0, alpha=3.0),                 # N_t ~ 5, one longitudinal unknown
    dict(f0=2000.0, alpha=10.0),                # N_l = 1: cubic term only, no z
    dict(f0=40.0, alpha=1.05, kappa=0.5),       # N_l ~ 570, N_t ~ 165
    dict(f0=30.0, alpha=1.01, kappa=0.5),       # N_l = 792, N_t = 169: the largest grids of the workloads
    dict(f0=110.0, alpha=3.0, boundary=1),      # simply supported ends
    dict(f0=55.0, alpha=6.0, kappa=2.7, sigma0=2.0, sigma1=1e-4),
    dict(f0=110.0, alpha=1.0, kappa=0.0, theta=1.0),
    dict(f0=55.0, alpha=2.0, kappa=0.0),        # N_t ~ 277: 9 transverse rows per lane
    dict(f0=40.0, alpha=2.0, kappa=0.0),        # N_t ~ 382: shared-memory path
    dict(f0=40.0, alpha=1.0, kappa=0.0),        # shared-memory path, linear
    dict(f0=48000.0 / 6.0 / 3.14, alpha=1.5, kappa=0.0),   # N_t = 2-3: a single unknown
])
def test_grid_edge_cases(sfd, ctx, case):
    d = W.make(excitation={"kind": "pluck", "amp": 2e-3, "pos": 0.37}, n_samples=6000, **case)
    assert rel_l2(gpu_run(sfd, ctx, d), oracle.run(d)) <= TOL


@pytest.mark.parametrize("exc", [HAMMER, BOW])
def test_forced_shared_memory_path(sfd, ctx, exc):
    """Hammer and bow on a grid too large for the register path."""
    d = W.make(f0=40.0, alpha=2.0, kappa=0.0, excitation=exc, n_samples=3000)
    y, ref = gpu_run(sfd, ctx, d), oracle.run(d)
    if exc["kind"] == "hammer":
        assert rel_l2(y, ref) <= TOL
    else:
        assert rel_l2(y[:150], ref[:150]) <= 1e-3


def test_grid_sizes_match_oracle(sfd, ctx):
    rng = np.random.default_rng(7)
    for _ in range(40):
        d = W.random_string(rng, f0_lo=30.0, f0_hi=2000.0, seconds=0.01)
        s = sfd.string_from_dict(ctx, d)
        nt, nl, _, _ = sfd.sfd_string_info(s)
        sfd.sfd_string_destroy(s)
        assert (nt, nl) == oracle.grid(d)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 33, 65])
def test_short_requests(sfd, ctx, n):
    d = W.make(alpha=3.0, excitation=HAMMER)
    ref = oracle.run(d, n)
    y = gpu_run(sfd, ctx, d, n=n)
    assert y.shape == (n,)
    if n:
        assert np.max(np.abs(y - ref)) <= 1e-4 * max(np.max(np.abs(ref)), 1e-12) + 1e-12


def test_chunked_equals_single_call_bitwise(sfd, ctx):
    d = W.make(alpha=4.0, f0=80.0, excitation=HAMMER, n_samples=5000)
    a = gpu_run(sfd, ctx, d, chunks=[1, 2, 29, 968, 1000, 3000])
    b = gpu_run(sfd, ctx, d)
    assert np.array_equal(a, b)


def test_batch_equals_alone_bitwise(sfd, ctx):
    """Each string's samples are identical alone and inside a mixed batch."""
    strings = W.batch_mixed(24, seconds=0.05, seed=21)
    hs = [sfd.string_from_dict(ctx, d) for d in strings]
    b = sfd.sfd_batch_create(ctx, hs)
    ys, st = sfd.sfd_batch_synthesize_host(b, [d["n_samples"] for d in strings])
    sfd.sfd_batch_destroy(b)
    for h in hs:
        sfd.sfd_string_destroy(h)
    for d, y in zip(strings, ys):
        assert np.array_equal(y, gpu_run(sfd, ctx, d))


def test_modulation(sfd, ctx):
    vib = W.make(alpha=2.0, modulation={"kind": "vibrato", "rate": 6.0, "depth": 20.0, "phase": 1.0},
                 n_samples=12000)
    gl = W.make(alpha=2.0, f0=90.0, modulation={"kind": "gliss", "depth": 1.0, "duration": 0.25},
                n_samples=12000)
    # glides that end within the run and hold at 2^D (up and down)
    held_up = W.make(alpha=2.0, f0=90.0, modulation={"kind": "gliss", "depth": 1.0, "duration": 0.08},
                     n_samples=12000)
    held_down = W.make(alpha=3.0, f0=150.0, modulation={"kind": "gliss", "depth": -0.6, "duration": 0.05},
                       excitation={"kind": "hammer", "mass": 0.01, "vel": 1.0, "pos": 0.2, "omega": 3e3,
                                   "alpha": 2.3}, n_samples=12000)
    for d in (vib, gl, held_up, held_down):
        assert rel_l2(gpu_run(sfd, ctx, d), oracle.run(d)) <= TOL


def test_energy_drift_lossless(sfd, ctx):
    """Lossless nonlinear string: the discrete energy of the FP32 state stays
    within 1e-5 of its initial value over 24,000 steps."""
    from fdtd_energy import Grid, energy
    d = W.make(alpha=3.0, sigma0=0.0, sigma1=0.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.3})
    s = sfd.string_from_dict(ctx, d)
    nt, nl, _, _ = sfd.sfd_string_info(s)
    g = Grid(nt, nl, d)
    sfd.sfd_synthesize(s, 3)
    up, u, zp, z = [a.astype(np.float64) for a in sfd.sfd_string_state(s)]
    H0 = energy(g, up, u, zp, z)
    worst = 0.0
    for _ in range(8):
        sfd.sfd_synthesize(s, 3000)
        up, u, zp, z = [a.astype(np.float64) for a in sfd.sfd_string_state(s)]
        worst = max(worst, abs(energy(g, up, u, zp, z) - H0) / H0)
    sfd.sfd_string_destroy(s)
    assert worst <= 1e-5


def test_state_matches_oracle(sfd, ctx):
    d = W.make(alpha=3.0, excitation={"kind": "pluck", "amp": 5e-3, "pos": 0.3})
    s = sfd.string_from_dict(ctx, d)
    sfd.sfd_synthesize(s, 2001)
    up, u, zp, z = sfd.sfd_string_state(s)
    sfd.sfd_string_destroy(s)
    o = oracle.OracleString(d)
    o.run(2001)
    oup, ou, ozp, oz, _ = o.state()
    assert rel_l2(u, ou) <= TOL
    assert rel_l2(z, oz) <= 1e-3


def test_errors_are_reported(sfd, ctx):
    p = sfd.sfd_params_default()
    p.alpha = 0.5
    with pytest.raises(sfd.SfdError) as ei:
        sfd.sfd_string_create(ctx, p)
    assert ei.value.code == sfd.SFD_EINVAL
    s = sfd.string_from_dict(ctx, W.make())
    sfd.sfd_synthesize(s, 10)
    with pytest.raises(sfd.SfdError) as ei:
        sfd.sfd_excite_pluck(s, 1e-3, 0.3)
    assert ei.value.code == sfd.SFD_ESTATE
    b = sfd.sfd_batch_create(ctx, [s])
    with pytest.raises(sfd.SfdError) as ei:
        sfd.sfd_string_destroy(s)
    assert ei.value.code == sfd.SFD_EBUSY
    sfd.sfd_batch_destroy(b)
    sfd.sfd_string_destroy(s)


def test_pool_exhaustion_is_enomem(sfd):
    c = sfd.sfd_ctx_create(0, None, 64 << 10)
    try:
        hs = []
        with pytest.raises(sfd.SfdError) as ei:
            for _ in range(1000):
                hs.append(sfd.string_from_dict(c, W.make(f0=40.0, alpha=1.05, kappa=0.5)))
        assert ei.value.code == sfd.SFD_ENOMEM
        used, total = sfd.sfd_ctx_memory(c)
        assert used <= total
        for h in hs:
            sfd.sfd_string_destroy(h)
        assert sfd.sfd_ctx_memory(c)[0] == 0
    finally:
        sfd.sfd_ctx_destroy(c)


def contact_episodes(d, n):
    """Separate hammer contacts of the oracle's trajectory over n samples."""
    s = oracle.OracleString(d)
    s.run(2)
    episodes, inside = 0, False
    for _ in range(n - 2):
        s.run(1)
        c = s.state()[4][3] > 0          # the contact stiffness G of the last step
        episodes += c and not inside
        inside = c
    return episodes


BOW_WINDOW = 6000   # 0.125 s


def test_full_batch_parity(sfd, ctx):
    """The 256-string, 2 s mixed batch in the benchmark's launch configuration:
    the first 0.25 s of every plucked or struck string against the oracle
    within 1e-4, and the first 0.125 s of every bowed string within 1e-4
    (measured: at most 3.4e-5 over the 96 bowed strings; over 0.25 s five of
    them cross a bifurcation, see test_bowed_notes_over_half_a_second); every
    output finite; the whole 2 s note within 1e-4 for every 10th of the
    plucked or struck strings.

    The one exception, measured and physical: a struck string whose hammer
    chatters (four or more separate contacts within the window, the string
    swinging back into the slower hammer) has a trajectory that grows
    FP32-sized perturbations ~10^5-fold, so running the FP64 oracle with its
    state rounded to FP32 after every step already moves it past 1e-4; such
    a string is held to three times that floor.  Two of the 160 are."""
    strings = W.batch_mixed(256, seconds=2.0, seed=2)
    hs = [sfd.string_from_dict(ctx, d) for d in strings]
    b = sfd.sfd_batch_create(ctx, hs)
    ns = np.array([d["n_samples"] for d in strings])
    offs = np.zeros(len(ns), np.int64)
    offs[1:] = np.cumsum(ns)[:-1]
    out = torch.zeros(int(ns.sum()), dtype=torch.float32, device="cuda")
    st = sfd.sfd_batch_synthesize(b, ns, out, offs, per_string_status=True)
    sfd.sfd_batch_destroy(b)
    for h in hs:
        sfd.sfd_string_destroy(h)
    y = out.cpu().numpy()
    assert np.all(np.isfinite(y))
    assert np.all(st == 0)
    lens = [BOW_WINDOW if d["excitation"]["kind"] == "bow" else 12000 for d in strings]
    refs, _ = oracle.run_batch(strings, n_samples=lens)
    from fp32_floor import fp32_state_floor
    beyond = []
    for i, (n, ref) in enumerate(zip(lens, refs)):
        e = rel_l2(y[offs[i]:offs[i] + n], ref)
        if e <= TOL:
            continue
        d = strings[i]
        assert d["excitation"]["kind"] == "hammer", (i, e)
        assert contact_episodes(d, n) >= 4, (i, e, "no chatter")
        floor = fp32_state_floor(d, n)
        assert floor > TOL and e <= 3 * floor, (i, e, floor)
        beyond.append(i)
    assert len(beyond) <= 2, beyond
    # the whole 2 s note, for every 10th of the others (phase errors grow
    # with time: measured 2e-6 - 1.3e-5 over 2 s)
    full = [i for i, d in enumerate(strings) if d["excitation"]["kind"] != "bow" and i not in beyond][::10]
    refs_full, _ = oracle.run_batch([strings[i] for i in full])
    for i, ref in zip(full, refs_full):
        assert rel_l2(y[offs[i]:offs[i] + ns[i]], ref) <= TOL, (i, "whole note")
