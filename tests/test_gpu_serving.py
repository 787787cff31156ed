"""Serving with continuous batching: notes that arrive while others are on the
GPU are admitted as slots and device memory free up, their chunks overlap on
the device, and each note's audio is the same alone and in the mix."""

import numpy as np
import pytest

import oracle
from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHUNK = 1024


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


def short_notes(n_rate_s: float, seed: int, lo: int = 1500, hi: int = 6000):
    """Notes of the serving trace (f0 40-1000 Hz, pluck / hammer / bow) with
    lengths of a few chunks, none a multiple of the chunk."""
    trace = W.serving_trace(2000.0, n_rate_s, seed=seed)
    rng = np.random.default_rng(seed)
    notes = []
    for _, d in trace:
        n = int(rng.integers(lo, hi))
        if n % CHUNK == 0:
            n += 1
        notes.append(dict(d, n_samples=n))
    return notes


def alone(sfd, ctx, d):
    s = sfd.string_from_dict(ctx, d)
    try:
        return sfd.sfd_synthesize(s, d["n_samples"])
    finally:
        sfd.sfd_string_destroy(s)


def collect(sfd, sv, audio, stats_log, finished):
    for tag, first, data, last, status, ready, arrival in sfd.sfd_server_pump(sv):
        parts = audio.setdefault(tag, [])
        expect = sum(len(p) for p in parts)
        assert first == expect, (tag, first, expect)
        parts.append(data)
        assert ready >= arrival
        if last:
            assert tag not in finished
            finished[tag] = status
    stats_log.append(sfd.sfd_server_stats_get(sv))


def drain(sfd, sv, audio, stats_log, finished, limit=10000):
    for _ in range(limit):
        st = sfd.sfd_server_stats_get(sv)
        if st.queued == 0 and st.live == 0 and st.in_flight == 0:
            return
        collect(sfd, sv, audio, stats_log, finished)
    raise AssertionError("server did not drain")


def test_served_notes_equal_alone(sfd):
    ctx = sfd.sfd_ctx_create(0, None, 256 << 20)
    sv = sfd.sfd_server_create(ctx, CHUNK, 64)
    try:
        notes = short_notes(0.03, seed=11)
        assert len(notes) >= 30
        waves = [notes[i::3] for i in range(3)]
        audio, stats_log, finished = {}, [], {}
        tags = {}
        for w, wave in enumerate(waves):
            for d in wave:
                tag = len(tags)
                tags[tag] = d
                sfd.sfd_server_submit(sv, sfd.request_from_dict(d, tag))
            for _ in range(2):   # the next wave arrives while this one is mid-note
                collect(sfd, sv, audio, stats_log, finished)
        drain(sfd, sv, audio, stats_log, finished)
        # continuous batching: notes of a later wave were live beside unfinished earlier ones
        assert max(st.live for st in stats_log) > len(waves[0])
        assert sorted(finished) == sorted(tags)
        for tag, d in tags.items():
            y = np.concatenate(audio[tag])
            assert len(y) == d["n_samples"]
            assert finished[tag] == sfd.SFD_OK
            assert np.array_equal(y, alone(sfd, ctx, d)), tag
        # and against the oracle for a few non-bowed notes
        picks = [t for t, d in tags.items() if d["excitation"]["kind"] != "bow"][:4]
        for t in picks:
            ref = oracle.run(tags[t], tags[t]["n_samples"])
            y = np.concatenate(audio[t]).astype(np.float64)
            assert np.linalg.norm(y - ref) <= 1e-4 * np.linalg.norm(ref)
    finally:
        sfd.sfd_server_destroy(sv)
        sfd.sfd_ctx_destroy(ctx)


def server_reservation(max_live: int, chunk: int) -> int:
    rnd = lambda n: (n + 255) // 256 * 256
    return 2 * (rnd(4 * max_live * chunk) + rnd(40 * max_live))   # output rows + job table (40 B jobs)


def test_admission_by_device_memory(sfd):
    max_live = 32
    pool = server_reservation(max_live, CHUNK) + 16 * 1024   # room for a few notes' state
    ctx = sfd.sfd_ctx_create(0, None, pool)
    sv = sfd.sfd_server_create(ctx, CHUNK, max_live)
    try:
        base = sfd.sfd_server_stats_get(sv).pool_used
        notes = short_notes(0.03, seed=12, lo=1200, hi=3000)[:40]
        assert len(notes) == 40
        for tag, d in enumerate(notes):
            sfd.sfd_server_submit(sv, sfd.request_from_dict(d, tag))
        audio, stats_log, finished = {}, [], {}
        drain(sfd, sv, audio, stats_log, finished)
        peak_live = max(st.live for st in stats_log)
        assert 0 < peak_live < len(notes)              # memory, not slots, limited admission
        assert all(st.pool_used <= st.pool_size for st in stats_log)
        assert any(st.queued > 0 and st.live > 0 for st in stats_log)
        assert sfd.sfd_server_stats_get(sv).pool_used == base   # every note's block returned
        assert sorted(finished) == list(range(len(notes)))
        for tag in (0, len(notes) // 2, len(notes) - 1):
            assert np.array_equal(np.concatenate(audio[tag]), alone(sfd, ctx, notes[tag]))
    finally:
        sfd.sfd_server_destroy(sv)
        sfd.sfd_ctx_destroy(ctx)


def test_submit_rejects_invalid_and_never_fitting_notes(sfd):
    max_live = 8
    pool = server_reservation(max_live, CHUNK) + 4096
    ctx = sfd.sfd_ctx_create(0, None, pool)
    sv = sfd.sfd_server_create(ctx, CHUNK, max_live)
    try:
        bad = dict(W.make(alpha=0.5), n_samples=2000)
        with pytest.raises(sfd.SfdError) as ei:
            sfd.sfd_server_submit(sv, sfd.request_from_dict(bad, 0))
        assert ei.value.code == sfd.SFD_EINVAL
        big = dict(W.make(f0=40.0, alpha=1.5), n_samples=2000)   # 399 longitudinal unknowns
        with pytest.raises(sfd.SfdError) as ei:
            sfd.sfd_server_submit(sv, sfd.request_from_dict(big, 1))
        assert ei.value.code == sfd.SFD_ENOMEM
        st = sfd.sfd_server_stats_get(sv)
        assert st.queued == 0 and st.submitted == 0
        ok = dict(W.make(f0=880.0, alpha=2.0), n_samples=1500)
        sfd.sfd_server_submit(sv, sfd.request_from_dict(ok, 2))
        audio, stats_log, finished = {}, [], {}
        drain(sfd, sv, audio, stats_log, finished)
        assert finished == {2: sfd.SFD_OK}
    finally:
        sfd.sfd_server_destroy(sv)
        sfd.sfd_ctx_destroy(ctx)


def test_unstable_note_is_isolated(sfd):
    """A note on the printed grid (N_t from the theta = 1 rule with theta =
    0.70, unstable: reading A5) ends with SFD_EUNSTABLE; the notes served
    beside it are unaffected."""
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    sv = sfd.sfd_server_create(ctx, CHUNK, 16)
    try:
        bad = dict(W.make(grid_rule=1, sigma0=0.0, sigma1=0.0), n_samples=4000)
        good = short_notes(0.004, seed=13, lo=2000, hi=4000)[:5]
        sfd.sfd_server_submit(sv, sfd.request_from_dict(bad, 100))
        for tag, d in enumerate(good):
            sfd.sfd_server_submit(sv, sfd.request_from_dict(d, tag))
        audio, stats_log, finished = {}, [], {}
        drain(sfd, sv, audio, stats_log, finished)
        assert finished[100] == sfd.SFD_EUNSTABLE
        for tag, d in enumerate(good):
            assert finished[tag] == sfd.SFD_OK
            assert np.array_equal(np.concatenate(audio[tag]), alone(sfd, ctx, d))
    finally:
        sfd.sfd_server_destroy(sv)
        sfd.sfd_ctx_destroy(ctx)


def test_longitudinal_notes_served(sfd):
    """Notes read on the longitudinal channel, served beside transverse ones,
    equal the same notes alone."""
    ctx = sfd.sfd_ctx_create(0, None, 128 << 20)
    sv = sfd.sfd_server_create(ctx, CHUNK, 32)
    try:
        notes = short_notes(0.004, seed=17, lo=1500, hi=4000)[:8]
        notes = [dict(d, output="longitudinal") if i % 2 else d for i, d in enumerate(notes)]
        for tag, d in enumerate(notes):
            sfd.sfd_server_submit(sv, sfd.request_from_dict(d, tag))
        audio, stats_log, finished = {}, [], {}
        drain(sfd, sv, audio, stats_log, finished)
        assert sorted(finished) == list(range(len(notes)))
        for tag, d in enumerate(notes):
            assert finished[tag] == sfd.SFD_OK
            assert np.array_equal(np.concatenate(audio[tag]), alone(sfd, ctx, d)), tag
    finally:
        sfd.sfd_server_destroy(sv)
        sfd.sfd_ctx_destroy(ctx)


def test_bow_envelope_notes_served(sfd):
    """Bowed notes with time-varying velocity, force and position (Sec.
    3.3.1), served beside plain notes, equal the same notes alone; a
    non-bowed request with an envelope is refused."""
    ctx = sfd.sfd_ctx_create(0, None, 128 << 20)
    sv = sfd.sfd_server_create(ctx, CHUNK, 32)
    try:
        notes = short_notes(0.004, seed=19, lo=1500, hi=4000)[:8]
        env = {"t": [0.0, 0.01, 0.03], "vel": [0.05, 0.4, 0.2], "force": [0.3, 2.0, 0.8], "pos": [0.12, 0.3, 0.2]}
        bow = {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0}
        notes = [dict(d, excitation=dict(bow, envelope=env)) if i % 2 else d for i, d in enumerate(notes)]
        for tag, d in enumerate(notes):
            sfd.sfd_server_submit(sv, sfd.request_from_dict(d, tag))
        pluck = dict(notes[0], excitation={"kind": "pluck", "amp": 1e-3, "pos": 0.3, "envelope": env})
        with pytest.raises(sfd.SfdError) as e:
            sfd.sfd_server_submit(sv, sfd.request_from_dict(pluck, 99))
        assert e.value.code == sfd.SFD_EINVAL
        audio, stats_log, finished = {}, [], {}
        drain(sfd, sv, audio, stats_log, finished)
        assert sorted(finished) == list(range(len(notes)))
        for tag, d in enumerate(notes):
            assert finished[tag] == sfd.SFD_OK
            assert np.array_equal(np.concatenate(audio[tag]), alone(sfd, ctx, d)), tag
    finally:
        sfd.sfd_server_destroy(sv)
        sfd.sfd_ctx_destroy(ctx)
