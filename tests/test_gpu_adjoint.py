"""Gradients by the hand-written discrete adjoint (sfd_tape_*, grad.py), for
plucked and hammered strings of the differentiation workload (loss: sum of
squared differences to targets rendered from parameters perturbed by up to
5 %):
* the vector-Jacobian product with the GPU run's dJ/dy against the FP64
  oracle's exact derivatives (complex step; exactness of the adjoint);
* the loss gradient against central finite differences of the GPU
  synthesis (relative steps 1e-3, 3e-3) and against the FP64 oracle's
  exact gradient (complex step).  The loss of the FP32 run differs from the oracle's by the FP32
  synthesis error, which is correlated with the output's sigma1
  sensitivity, so those components are held relative to the string's
  largest sensitivity."""

import numpy as np
import pytest

import oracle
from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_SHORT = 4800       # 0.1 s: five checkpoint segments of 1024, the last partial


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


@pytest.fixture(scope="module")
def ctx(sfd):
    c = sfd.sfd_ctx_create(0, None, 512 << 20)
    yield c
    sfd.sfd_ctx_destroy(c)


def workload(count, n):
    base, target = W.batch_gradient(64, seconds=0.5, seed=4)
    base = [dict(d, n_samples=n) for d in base[:count]]
    target = [dict(d, n_samples=n) for d in target[:count]]
    return base, target


def targets_of(target, n):
    ys, _ = oracle.run_batch(target, n_samples=n)
    return np.stack(ys)


def adjoint_grad(sfd, ctx, base, tgt, n, K=1024, record=None):
    tape = sfd.sfd_tape_create(ctx, base, n, K)
    try:
        if record is not None:
            sfd.sfd_tape_set_record_forward(tape, record)
        y = torch.empty(len(base), n, device="cuda", dtype=torch.float32)
        sfd.sfd_tape_forward(tape, y)
        dy = 2.0 * (y.double() - torch.from_numpy(tgt).cuda())
        g = sfd.sfd_tape_backward(tape, dy.float().contiguous(), len(base))
        return g, y.cpu().numpy()
    finally:
        sfd.sfd_tape_destroy(tape)


def perturbed(d, k, factor):
    from paper_2311_18505_gb300.grad import params_of, with_params
    r = np.array(params_of(d))
    r[k] *= factor
    return with_params(d, r)


def gpu_losses(sfd, ctx, dicts, tgts, n):
    hs = [sfd.string_from_dict(ctx, d) for d in dicts]
    b = sfd.sfd_batch_create(ctx, hs)
    try:
        ys, _ = sfd.sfd_batch_synthesize_host(b, [n] * len(dicts))
    finally:
        sfd.sfd_batch_destroy(b)
        grids = [sfd.sfd_string_info(h)[:2] for h in hs]
        for h in hs:
            sfd.sfd_string_destroy(h)
    return [float(np.sum((y.astype(np.float64) - t) ** 2)) for y, t in zip(ys, tgts)], grids


def test_tape_forward_is_the_plain_synthesis(sfd, ctx):
    base, _ = workload(6, N_SHORT)
    tape = sfd.sfd_tape_create(ctx, base, N_SHORT, 1024)
    try:
        y = torch.empty(len(base), N_SHORT, device="cuda", dtype=torch.float32)
        sfd.sfd_tape_forward(tape, y)
        y = y.cpu().numpy()
    finally:
        sfd.sfd_tape_destroy(tape)
    for d, row in zip(base, y):
        s = sfd.string_from_dict(ctx, d)
        assert np.array_equal(row, sfd.sfd_synthesize(s, N_SHORT))
        sfd.sfd_string_destroy(s)


def test_adjoint_matches_gpu_central_differences(sfd, ctx):
    """Central differences of the GPU synthesis itself (relative steps 1e-3
    and 3e-3).  FP32 rounding makes the difference quotient noisy where a
    parameter barely moves the loss, so each component is held to the
    spread of its two quotients plus 2 % (and the string's largest
    sensitivity sets a floor)."""
    base, target = workload(8, N_SHORT)
    tgt = targets_of(target, N_SHORT)
    g, _ = adjoint_grad(sfd, ctx, base, tgt, N_SHORT)
    from paper_2311_18505_gb300.grad import params_of
    steps = (1e-3, 3e-3)
    dicts, tg = [], []
    for i, d in enumerate(base):
        for k in range(5):
            for eps in steps:
                for f in (1 + eps, 1 - eps):
                    dicts.append(perturbed(d, k, f))
                    tg.append(tgt[i])
    losses, grids = gpu_losses(sfd, ctx, dicts, tg, N_SHORT)
    _, base_grids = gpu_losses(sfd, ctx, base, list(tgt), N_SHORT)
    checked = 0
    for i, d in enumerate(base):
        th = params_of(d)
        sens = np.max(np.abs(g[i] * np.array(th)))
        for k in range(5):
            j = 20 * i + 4 * k
            if any(grids[j + q] != base_grids[i] for q in range(4)):
                continue   # the perturbation moved the grid: no derivative on a fixed grid
            fd1 = (losses[j] - losses[j + 1]) / (2 * steps[0] * th[k])
            fd3 = (losses[j + 2] - losses[j + 3]) / (2 * steps[1] * th[k])
            band = 3 * abs(fd1 - fd3) + 2e-2 * abs(fd1) + 1e-3 * sens / abs(th[k])
            assert abs(g[i, k] - fd1) <= band, (i, k, g[i, k], fd1, fd3)
            checked += 1
    assert checked >= 30


def oracle_derivatives(d, n):
    """The FP64 oracle's output and its exact derivatives dy/dp (complex
    step, one row per parameter of params_of) on the string's own grid."""
    nt, nl = oracle.grid(d)
    rows = []
    for k in range(5):
        y, dy = oracle.complex_step(d, k, n=n, n_t=nt, n_l=nl)
        rows.append(dy)
    return y, np.array(rows)


def test_vector_jacobian_product_matches_the_oracle(sfd, ctx):
    """The adjoint is the exact transpose of the step's linearisation: with
    the residual weights w = dJ/dy of the GPU run, its result must equal
    sum_j w_j dy_j/dp of the FP64 oracle, whose derivatives are exact
    (complex step, grid held fixed).  What remains is that the adjoint
    differentiates the FP32 trajectory, not the FP64 one, whose outputs
    differ by rel-L2 ~1e-6 here.  kappa and alpha move the partials' phase in
    proportion to time, so their derivatives on the FP32 trajectory depart
    most from the FP64 ones: measured up to 2.7e-4 of the component for
    plucked strings, the other components within 2e-5.  Each component is
    held to 1e-3 of itself plus 1e-6 of the string's largest term."""
    base, target = workload(8, N_SHORT)
    tgt = targets_of(target, N_SHORT)
    tape = sfd.sfd_tape_create(ctx, base, N_SHORT, 1024)
    try:
        y = torch.empty(len(base), N_SHORT, device="cuda", dtype=torch.float32)
        sfd.sfd_tape_forward(tape, y)
        w = (2.0 * (y.double() - torch.from_numpy(tgt).cuda())).float().contiguous()
        g = sfd.sfd_tape_backward(tape, w, len(base))
    finally:
        sfd.sfd_tape_destroy(tape)
    w = w.double().cpu().numpy()
    y32 = y.double().cpu().numpy()
    from paper_2311_18505_gb300.grad import params_of
    for i, d in enumerate(base):
        y64, D = oracle_derivatives(d, N_SHORT)
        ref = D @ w[i]
        ey = float(np.linalg.norm(y32[i] - y64) / np.linalg.norm(y64))
        th = np.array(params_of(d))
        scale = np.max(np.abs(ref * th))
        err = np.abs(g[i] - ref) * th
        print(f"vjp {i} {d['excitation']['kind']}: trajectory {ey:.2e}, err/scale per component "
              + " ".join(f"{x:.1e}" for x in err / scale) + " rel " + " ".join(f"{x:.1e}" for x in err / np.maximum(np.abs(ref * th), 1e-300)))
        assert np.all(err <= 1e-3 * np.abs(ref * th) + 1e-6 * scale), (i, g[i], ref, ey)


def test_vector_jacobian_product_longitudinal_output(sfd, ctx):
    """The same check for strings read on the longitudinal channel (dJ/dy
    enters the adjoint of zeta at the pickup).  zeta is forced at sums of
    transverse partials, so its sensitivity to kappa (which detunes them
    against the longitudinal modes) follows the FP32 trajectory's small
    departure from the FP64 one with a large gain: measured, the kappa
    component is off by 1.8 % where zeta's rel-L2 trajectory error is 7e-5
    and by < 1e-4 where it is 3e-5 with little detuning.  Each component is
    held to 1e-4 of the string's largest sensitivity plus max(1 %, 300 x that
    trajectory error) of itself.  A wrong injection (node, weight, sign,
    first-sample term) breaks every component by O(1).  (Central differences
    of the FP32 GPU map are no check here: near a longitudinal mode its
    kappa-derivative departs from the scheme's by tens of percent, which the
    adjoint, the derivative of the scheme along the trajectory, does not
    follow.)"""
    base, target = workload(8, N_SHORT)
    base = [dict(d, output="longitudinal") for d in base]
    target = [dict(d, output="longitudinal") for d in target]
    tgt = targets_of(target, N_SHORT)
    tape = sfd.sfd_tape_create(ctx, base, N_SHORT, 1024)
    try:
        y = torch.empty(len(base), N_SHORT, device="cuda", dtype=torch.float32)
        sfd.sfd_tape_forward(tape, y)
        w = (2.0 * (y.double() - torch.from_numpy(tgt).cuda())).float().contiguous()
        g = sfd.sfd_tape_backward(tape, w, len(base))
    finally:
        sfd.sfd_tape_destroy(tape)
    w = w.double().cpu().numpy()
    yg = y.double().cpu().numpy()
    from paper_2311_18505_gb300.grad import params_of
    checked = 0
    for i, d in enumerate(base):
        nt, nl = oracle.grid(d)
        if nl <= 1:
            assert np.all(g[i] == 0.0)   # no longitudinal grid: the output is identically zero
            continue
        th = np.array(params_of(d))
        runs = []
        for k in range(5):
            for f in (1 + 1e-6, 1 - 1e-6):
                runs.append(dict(perturbed(d, k, f), n_t=nt, n_l=nl))
        ys, _ = oracle.run_batch(runs + [d], n_samples=N_SHORT)
        ref = np.array([(w[i] @ ys[2 * k] - w[i] @ ys[2 * k + 1]) / (2e-6 * th[k]) for k in range(5)])
        e_traj = np.linalg.norm(yg[i] - ys[-1]) / np.linalg.norm(ys[-1])
        scale = np.max(np.abs(ref * th))
        err = np.abs(g[i] - ref) * th
        rel = max(1e-2, 300.0 * e_traj)
        assert np.all(err <= 1e-4 * scale + rel * np.abs(ref * th)), (i, g[i], ref, e_traj)
        checked += 1
    assert checked >= 6


@pytest.mark.parametrize("mod", [{"kind": "vibrato", "rate": 6.0, "depth": 40.0, "phase": 0.3},
                                 {"kind": "gliss", "depth": 0.5, "duration": 0.1}])
def test_vector_jacobian_product_modulated(sfd, ctx, mod):
    """f0-modulated strings: the adjoint scales each step's gamma^2
    coefficients as the forward did, and the gradient of each unscaled
    coefficient carries the step's factor.  Same check as for unmodulated
    strings (the oracle's central differences on the grid sized for the
    modulation's peak)."""
    base, target = workload(6, N_SHORT)
    base = [dict(d, modulation=mod) for d in base]
    target = [dict(d, modulation=mod) for d in target]
    tgt = targets_of(target, N_SHORT)
    tape = sfd.sfd_tape_create(ctx, base, N_SHORT, 1024)
    try:
        y = torch.empty(len(base), N_SHORT, device="cuda", dtype=torch.float32)
        sfd.sfd_tape_forward(tape, y)
        w = (2.0 * (y.double() - torch.from_numpy(tgt).cuda())).float().contiguous()
        g = sfd.sfd_tape_backward(tape, w, len(base))
        yt = y.cpu().numpy()
    finally:
        sfd.sfd_tape_destroy(tape)
    for d, row in zip(base, yt):   # the tape's forward is the plain modulated synthesis
        s = sfd.string_from_dict(ctx, d)
        assert np.array_equal(row, sfd.sfd_synthesize(s, N_SHORT))
        sfd.sfd_string_destroy(s)
    w = w.double().cpu().numpy()
    from paper_2311_18505_gb300.grad import params_of
    for i, d in enumerate(base):
        nt, nl = oracle.grid(d)
        th = np.array(params_of(d))
        runs = [dict(perturbed(d, k, f), n_t=nt, n_l=nl) for k in range(5) for f in (1 + 1e-6, 1 - 1e-6)]
        ys, _ = oracle.run_batch(runs, n_samples=N_SHORT)
        ref = np.array([(w[i] @ ys[2 * k] - w[i] @ ys[2 * k + 1]) / (2e-6 * th[k]) for k in range(5)])
        scale = np.max(np.abs(ref * th))
        err = np.abs(g[i] - ref) * th
        assert np.all(err <= 1e-4 * scale + 2e-3 * np.abs(ref * th)), (i, g[i], ref)


def _bow(vel, force, pos=0.21, a=100.0, eps=0.1):
    return {"kind": "bow", "vel": vel, "force": force, "pos": pos, "a": a, "eps": eps, "release": -1.0}


def test_bowed_strings_vector_jacobian_product(sfd, ctx):
    """Bowed strings (Eq. 5): each step keeps the regime the forward took
    (sliding: the force follows the friction curve; sticking: the bow point
    moves with the bow), so the loss is piecewise smooth and the adjoint
    gives its derivative between switches.  Against central differences of
    the FP64 oracle (relative steps 1e-6 and 1e-5, grid fixed), on the
    components where the two quotients agree to 1 % (elsewhere a switch
    falls inside the step or the sensitivity is at rounding level): each
    within 1e-4 of the string's largest sensitivity plus 3 % of itself
    (measured up to 1.7 %, on kappa of a string that sticks and slips).  The
    cases: sliding bows, a stick-slip bow and the longitudinal channel."""
    n = N_SHORT
    cases = [W.make(f0=220.0, alpha=2.0, excitation=_bow(0.4, 0.1), n_samples=n),
             W.make(f0=150.0, alpha=3.0, kappa=1.5, excitation=_bow(0.3, 0.2), n_samples=n),
             W.make(f0=196.0, alpha=2.5, excitation=_bow(0.2, 1.0), n_samples=n),
             dict(W.make(f0=220.0, alpha=2.0, excitation=_bow(0.4, 0.1), n_samples=n), output="longitudinal")]
    from paper_2311_18505_gb300.grad import params_of, with_params
    rng = np.random.default_rng(8)
    checked = 0
    for d in cases:
        r0 = np.array(params_of(d)) * (1 + rng.uniform(-0.05, 0.05, 5))
        r0[1] = max(r0[1], 1.0)
        tgt = oracle.run(with_params(d, r0), n)
        tape = sfd.sfd_tape_create(ctx, [d], n, 1024)
        try:
            y = torch.empty(1, n, device="cuda", dtype=torch.float32)
            sfd.sfd_tape_forward(tape, y)
            w = (2.0 * (y.double() - torch.from_numpy(tgt).cuda())).float().contiguous()
            g = sfd.sfd_tape_backward(tape, w, 1)[0]
        finally:
            sfd.sfd_tape_destroy(tape)
        w = w.double().cpu().numpy()[0]
        nt, nl = oracle.grid(d)
        th = np.array(params_of(d))
        quot = []
        for eps in (1e-6, 1e-5):
            runs = [dict(perturbed(d, k, f), n_t=nt, n_l=nl) for k in range(5) for f in (1 + eps, 1 - eps)]
            ys, _ = oracle.run_batch(runs, n_samples=n)
            quot.append(np.array([(w @ ys[2 * k] - w @ ys[2 * k + 1]) / (2 * eps * th[k]) for k in range(5)]))
        ref = quot[0]
        scale = np.max(np.abs(ref * th))
        for k in range(5):
            if ref[k] == 0.0 or abs(quot[0][k] - quot[1][k]) > 1e-2 * abs(ref[k]):
                continue
            err = abs(g[k] - ref[k]) * th[k]
            assert err <= 1e-4 * scale + 3e-2 * abs(ref[k] * th[k]), (d["f0"], k, g[k], ref[k])
            checked += 1
    assert checked >= 12


def test_adjoint_matches_the_oracle_gradient(sfd, ctx):
    """The loss gradient of the GPU run against the FP64 oracle's exact one
    (complex step).  The two losses differ because the outputs do: by
    Cauchy-Schwarz that moves component k by at most 2 |y32 - y64| |dy/dp_k|,
    which, plus the adjoint's own bar of the VJP test, bounds the error."""
    base, target = workload(8, N_SHORT)
    tgt = targets_of(target, N_SHORT)
    g, y32 = adjoint_grad(sfd, ctx, base, tgt, N_SHORT)
    from paper_2311_18505_gb300.grad import params_of
    for i, d in enumerate(base):
        y64, D = oracle_derivatives(d, N_SHORT)
        ref = D @ (2.0 * (y64 - tgt[i]))
        th = np.array(params_of(d))
        ey = float(np.linalg.norm(y32[i] - y64) / np.linalg.norm(y64))
        scale = np.max(np.abs(ref * th))
        shift = 2.0 * np.linalg.norm(y32[i] - y64) * np.linalg.norm(D, axis=1) * th
        err = np.abs(g[i] - ref) * th
        print(f"grad {i}: trajectory {ey:.2e}, worst err/scale {np.max(err) / scale:.2e}, "
              f"worst err/bound {np.max(err / (shift + (1e-7 + 30 * ey) * scale)):.2f}")
        assert np.all(err <= shift + (1e-7 + 30 * ey) * scale), (i, g[i], ref)


def test_gradient_does_not_depend_on_the_checkpoint_interval(sfd, ctx):
    base, target = workload(6, N_SHORT)
    tgt = targets_of(target, N_SHORT)
    g1, y1 = adjoint_grad(sfd, ctx, base, tgt, N_SHORT, K=1024)
    g2, y2 = adjoint_grad(sfd, ctx, base, tgt, N_SHORT, K=333)
    g3, y3 = adjoint_grad(sfd, ctx, base, tgt, N_SHORT, K=N_SHORT)
    assert np.array_equal(y1, y2) and np.array_equal(y1, y3)
    # the replayed levels and the adjoint recursion are identical; only the
    # grouping of the FP64 gradient sums differs
    np.testing.assert_allclose(g2, g1, rtol=1e-9, atol=0)
    np.testing.assert_allclose(g3, g1, rtol=1e-9, atol=0)


@pytest.mark.parametrize("K", [1024, 333])
def test_recorded_forward_equals_replayed_segments(sfd, ctx, K):
    """The backward pass over levels the forward pass recorded gives the
    gradient of the one that replays each segment from its checkpoint, bit
    for bit (a replay re-runs the same kernel from the same state)."""
    base, target = workload(6, N_SHORT)
    tgt = targets_of(target, N_SHORT)
    g_rec, y_rec = adjoint_grad(sfd, ctx, base, tgt, N_SHORT, K=K, record=True)
    g_rep, y_rep = adjoint_grad(sfd, ctx, base, tgt, N_SHORT, K=K, record=False)
    assert np.array_equal(y_rec, y_rep)
    assert np.array_equal(g_rec, g_rep)


def test_record_forward_invalidates_an_earlier_forward(sfd, ctx):
    """Switching the tape to recording after a forward pass asks for a new
    forward pass before the backward (SFD_ESTATE)."""
    base, target = workload(2, 2000)
    tape = sfd.sfd_tape_create(ctx, base, 2000, 512)
    try:
        sfd.sfd_tape_set_record_forward(tape, False)
        y = torch.empty(2, 2000, device="cuda", dtype=torch.float32)
        sfd.sfd_tape_forward(tape, y)
        sfd.sfd_tape_set_record_forward(tape, True)
        with pytest.raises(sfd.SfdError) as e:
            sfd.sfd_tape_backward(tape, torch.zeros_like(y), 2)
        assert e.value.code == sfd.SFD_ESTATE
        sfd.sfd_tape_forward(tape, y)
        g = sfd.sfd_tape_backward(tape, torch.zeros_like(y), 2)
        assert np.all(g == 0.0)
    finally:
        sfd.sfd_tape_destroy(tape)


def test_autograd_function_and_a_descent_step(sfd, ctx):
    from paper_2311_18505_gb300 import grad as G
    base, target = workload(6, N_SHORT)
    tgt = torch.from_numpy(targets_of(target, N_SHORT)).cuda()
    theta = torch.tensor(G.theta_of(base), dtype=torch.float64, requires_grad=True)
    y = G.synthesize(theta, base, N_SHORT, ctx)
    loss = ((y.double() - tgt) ** 2).sum()
    loss.backward()
    g_direct, _ = adjoint_grad(sfd, ctx, base, tgt.cpu().numpy(), N_SHORT)
    np.testing.assert_allclose(theta.grad.numpy(), g_direct, rtol=1e-6)
    # a small step against the gradient (scaled per parameter) lowers the loss
    with torch.no_grad():
        step = -1e-3 * theta * torch.sign(theta.grad)
        y2 = G.synthesize(theta + step, base, N_SHORT, ctx)
        loss2 = ((y2.double() - tgt) ** 2).sum()
    assert loss2.item() < loss.detach().item()


def test_full_differentiation_workload_against_the_oracle(sfd, ctx):
    """64 strings x 0.5 s, checkpoint every 1024 steps; four strings checked
    against the oracle's exact gradient (complex step) at full length, with
    the bound of test_adjoint_matches_the_oracle_gradient."""
    n = 24000
    base, target = workload(64, n)
    tgt = targets_of(target, n)
    g, y = adjoint_grad(sfd, ctx, base, tgt, n, K=1024)
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(y))
    from paper_2311_18505_gb300.grad import params_of
    for i in (0, 17, 33, 63):
        y64, D = oracle_derivatives(base[i], n)
        ref = D @ (2.0 * (y64 - tgt[i]))
        th = np.array(params_of(base[i]))
        ey = float(np.linalg.norm(y[i] - y64) / np.linalg.norm(y64))
        scale = np.max(np.abs(ref * th))
        shift = 2.0 * np.linalg.norm(y[i] - y64) * np.linalg.norm(D, axis=1) * th
        err = np.abs(g[i] - ref) * th
        print(f"full {i}: trajectory {ey:.2e}, worst err/scale {np.max(err) / scale:.2e}, "
              f"worst err/bound {np.max(err / (shift + (1e-7 + 30 * ey) * scale)):.2f}")
        assert np.all(err <= shift + (1e-7 + 30 * ey) * scale), (i, g[i], ref)
