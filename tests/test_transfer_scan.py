"""The register path's transfer of transverse node values to the
longitudinal grid (the spreading P^T of the coupling terms of Eq. 4, P the
linear interpolation from the longitudinal to the transverse nodes), as a
lane-level model of the kernel's segmented warp scan, against the direct
sum (P^T F)_m = sum_l P[l, m] F_l.

The model follows the kernel step by step: the transfer map (interval m_l =
floor(l N_l / N_t) and weight of every transverse row, pad rows in interval
N_l + 1), the in-lane running sums over consecutive rows of one interval,
the shuffle levels that close every interval across lanes, the carry from
the previous lane, and the two slot stores (S0[m], S1[m + 1]) made by the
last row of each interval.  Checked: every store lands inside the slot
arrays (32 m_z + 4 words, 2 guard cells), no slot is written twice, and the
longitudinal rows read the direct sum.  No GPU needed.
"""

import numpy as np
import pytest

W = 32


def shfl_up(v, s):
    return [v[l - s] if l >= s else v[l] for l in range(W)]


def shfl_down(v, s):
    return [v[l + s] if l + s < W else v[l] for l in range(W)]


def scan_transfer(n_t: int, n_l: int, mu: int, f: np.ndarray, cross_lane: bool = True):
    """Slot sums S0[m + 1] + S1[m + 1] read by longitudinal row m, and the
    number of shuffle levels the scan needed (cross_lane=False drops the
    shuffle levels and the carry: a planted mistake)."""
    n_u = n_t - 1
    m_z = 1
    while W * m_z < n_l:          # odd rows per lane, 32 m_z >= N_l - 1 + 1
        m_z += 2
    rz = W * m_z + 4
    tmi = np.zeros(W * mu, int)
    tmw = np.zeros(W * mu)
    for i in range(W * mu):
        pos = (i + 1) * n_l
        mm = pos // n_t if i < n_u else n_l + 1
        tmi[i] = mm
        tmw[i] = (pos - mm * n_t) / n_t if i < n_u else 0.0
    mmr = [[tmi[l * mu + r] for r in range(mu)] for l in range(W)]
    wr = [[tmw[l * mu + r] for r in range(mu)] for l in range(W)]
    nxt = shfl_down([m[0] for m in mmr], 1)
    prv = shfl_up([m[mu - 1] for m in mmr], 1)
    lastm, carry_ok, flag = [0] * W, [False] * W, [True] * W
    for l in range(W):
        for r in range(mu - 1):
            if mmr[l][r + 1] != mmr[l][r]:
                lastm[l] |= 1 << r
        if l == W - 1 or nxt[l] != mmr[l][mu - 1]:
            lastm[l] |= 1 << (mu - 1)
        for r in range(mu):
            if l * mu + r >= n_u:
                lastm[l] &= ~(1 << r)        # pad rows store nothing
        carry_ok[l] = l > 0 and prv[l] == mmr[l][0]
        flag[l] = not (l > 0 and prv[l] == mmr[l][mu - 1])
    # levels that close every interval, and per lane the levels at which it
    # adds the partial sum from lane - 2^level (computed once per job)
    fs, levels, add_mask = list(flag), 0, [0] * W
    for lv in range(5):
        if all(fs):
            break
        sh = 1 << lv
        fu = shfl_up(fs, sh)
        for l in range(W):
            if l >= sh and not fs[l]:
                add_mask[l] |= 1 << lv
        fs = [fs[l] or fu[l] if l >= sh else fs[l] for l in range(W)]
        levels = lv + 1
    assert all(fs)
    fl = [[f[l * mu + r] if l * mu + r < n_u else 0.0 for r in range(mu)] for l in range(W)]
    a0 = [[0.0] * mu for _ in range(W)]
    a1 = [[0.0] * mu for _ in range(W)]
    for l in range(W):
        for r in range(mu):
            p0, p1 = (1 - wr[l][r]) * fl[l][r], wr[l][r] * fl[l][r]
            cont = r > 0 and mmr[l][r] == mmr[l][r - 1]
            a0[l][r] = a0[l][r - 1] + p0 if cont else p0
            a1[l][r] = a1[l][r - 1] + p1 if cont else p1
    v0 = [a0[l][mu - 1] for l in range(W)]
    v1 = [a1[l][mu - 1] for l in range(W)]
    for lv in range(levels if cross_lane else 0):
        sh = 1 << lv
        u0, u1 = shfl_up(v0, sh), shfl_up(v1, sh)
        for l in range(W):
            if (add_mask[l] >> lv) & 1:
                v0[l] += u0[l]
                v1[l] += u1[l]
    c0, c1 = shfl_up(v0, 1), shfl_up(v1, 1)
    if not cross_lane:
        c0, c1 = [0.0] * W, [0.0] * W
    s0, s1 = np.zeros(rz), np.zeros(rz)
    written = set()
    for l in range(W):
        for r in range(mu):
            if not (lastm[l] >> r) & 1:
                continue
            add = carry_ok[l] and mmr[l][r] == mmr[l][0]
            i0, i1 = mmr[l][r] + 2, mmr[l][r] + 3          # +2: the arrays' guard cells
            assert 0 <= i0 < rz and 0 <= i1 < rz, (n_t, n_l, mu, i0, i1, rz)
            for key in (("S0", i0), ("S1", i1)):
                assert key not in written, ("slot written twice", n_t, n_l, mu, key)
                written.add(key)
            s0[i0] = a0[l][r] + c0[l] if add else a0[l][r]
            s1[i1] = a1[l][r] + c1[l] if add else a1[l][r]
    return np.array([s0[m + 3] + s1[m + 3] for m in range(n_l - 1)]), levels


def direct_transfer(n_t: int, n_l: int, f: np.ndarray) -> np.ndarray:
    l = np.arange(1, n_t)[:, None]
    m = np.arange(1, n_l)[None, :]
    p = np.maximum(0.0, 1.0 - np.abs(l * n_l - m * n_t) / n_t)     # P[l, m]
    return p.T @ f


def grids():
    rng = np.random.default_rng(1)
    for mu in (1, 3, 5, 7, 9):
        lo = 2 if mu == 1 else 32 * (mu - 2) + 2                    # rows per lane of the class
        for n_t in sorted({lo + 1, lo + 7, (lo + 32 * mu) // 2, 32 * mu, 32 * mu + 1}):
            if not (n_t - 1 <= 32 * mu and n_t >= 3):
                continue
            cands = {2, 3, 5, 32, 33, 64, n_t // 3 + 1, n_t // 2, n_t - 1, n_t, n_t + 1, 2 * n_t}
            cands |= set(int(x) for x in rng.integers(2, 3 * n_t + 3, 2))
            for n_l in sorted(c for c in cands if 2 <= c <= 600):
                yield mu, n_t, n_l


CASES = list(grids())


def test_case_set_spans_every_class_and_ratio():
    assert {c[0] for c in CASES} == {1, 3, 5, 7, 9}
    assert any(n_l < n_t // 2 for _, n_t, n_l in CASES)   # intervals spanning several lanes
    assert any(n_l > n_t for _, n_t, n_l in CASES)        # plain scatter
    assert len(CASES) > 150


@pytest.mark.parametrize("mu", [1, 3, 5, 7, 9])
def test_segmented_scan_equals_direct_transfer(mu):
    rng = np.random.default_rng(mu)
    levels_seen = set()
    for m, n_t, n_l in CASES:
        if m != mu:
            continue
        f = rng.standard_normal(n_t - 1)
        got, levels = scan_transfer(n_t, n_l, mu, f)
        want = direct_transfer(n_t, n_l, f)
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want))), (n_t, n_l)
        levels_seen.add(levels)
    assert levels_seen - {0}          # some grids need cross-lane levels


def test_planted_mistake_is_caught():
    """Dropping the cross-lane levels and the carry from the previous lane
    (a plausible slip) breaks the sums of intervals that begin in an
    earlier lane, and the comparison with the direct sum sees it."""
    n_t, n_l, mu = 280, 20, 9          # ~14 transverse rows per interval: intervals cross lanes
    f = np.random.default_rng(3).standard_normal(n_t - 1)
    want = direct_transfer(n_t, n_l, f)
    got, levels = scan_transfer(n_t, n_l, mu, f)
    assert levels > 0 and np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    cut, _ = scan_transfer(n_t, n_l, mu, f, cross_lane=False)
    assert np.max(np.abs(cut - want)) > 0.1 * np.max(np.abs(want))
