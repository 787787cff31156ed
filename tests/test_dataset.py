"""Host logic of the dataset generator (no GPU): the per-item draws, the
shard plan, the files, retries of failed strings and the merge.  A stand-in
renderer replaces the GPU: it returns, for each string, samples that encode
the string's own parameters, so every row can be traced back to its item."""

import json
import os

import numpy as np
import pytest

from paper_2311_18505_gb300 import dataset as D


def fake_renderer(bad_f0=frozenset()):
    calls = []

    def render(dicts):
        calls.append(len(dicts))
        n = dicts[0]["n_samples"] if dicts else 0
        audio = np.zeros((len(dicts), n), np.float32)
        for r, d in enumerate(dicts):
            audio[r] = np.float32(d["f0"]) + (np.float32(1000.0) if d.get("output") == "longitudinal" else 0)
        status = np.array([-3 if d["f0"] in bad_f0 else 0 for d in dicts], np.int32)
        grids = [(int(d["f0"]) % 97 + 2, int(d["alpha"] * 10)) for d in dicts]
        return audio, status, grids

    render.calls = calls
    return render


SMALL = D.Distribution(seconds=0.001)


def test_draw_depends_only_on_seed_index_attempt():
    a = D.draw(SMALL, 7, 5)
    assert a == D.draw(SMALL, 7, 5)
    assert a != D.draw(SMALL, 7, 6)
    assert a != D.draw(SMALL, 8, 5)
    assert a != D.draw(SMALL, 7, 5, attempt=1)
    assert a["n_samples"] == 48


def test_draws_stay_in_their_ranges():
    dist = D.Distribution()
    kinds, mods, f0 = {}, {}, []
    for i in range(3000):
        d = D.draw(dist, 1, i)
        assert dist.f0[0] <= d["f0"] <= dist.f0[1]
        f0.append(d["f0"])
        for key in ("kappa", "alpha", "sigma0", "sigma1", "pickup"):
            lo, hi = getattr(dist, key)
            assert lo <= d[key] <= hi, key
        ex = d["excitation"]
        kinds[ex["kind"]] = kinds.get(ex["kind"], 0) + 1
        if ex["kind"] == "bow":
            assert dist.bow_a[0] <= ex["a"] <= dist.bow_a[1]
            assert dist.bow_eps[0] <= ex["eps"] <= dist.bow_eps[1]
            assert ex["release"] == -1.0 or 0 < ex["release"] < dist.seconds
        if ex["kind"] == "hammer":
            assert dist.hammer_alpha[0] <= ex["alpha"] <= dist.hammer_alpha[1]
        m = d["modulation"]
        mods[m["kind"]] = mods.get(m["kind"], 0) + 1
        if m["kind"] == "gliss":
            assert 0 < m["duration"] <= dist.seconds
    assert set(kinds) == {"pluck", "hammer", "bow"} and min(kinds.values()) > 800
    assert abs(mods["vibrato"] / 3000 - 0.25) < 0.04 and abs(mods["gliss"] / 3000 - 0.25) < 0.04
    # f0 log-uniform: the median near the geometric mean of the range
    assert abs(np.log(np.median(f0)) - 0.5 * np.log(40.0 * 1000.0)) < 0.15


def test_bow_envelopes_are_drawn_on_their_own_stream():
    """With p_bow_envelope > 0 bowed items get velocity, force and position
    envelopes (Sec. 3.3.1) spanning the note, in the bow ranges; every other
    parameter of every item is the draw of p_bow_envelope = 0."""
    plain = D.Distribution()
    env = D.Distribution(p_bow_envelope=0.5, bow_env_points=5)
    n_env = n_bow = 0
    for i in range(600):
        a, b = D.draw(plain, 3, i), D.draw(env, 3, i)
        eb = dict(b["excitation"])
        e = eb.pop("envelope", None)
        assert dict(b, excitation=eb) == a
        if a["excitation"]["kind"] != "bow":
            assert e is None
            continue
        n_bow += 1
        if e is None:
            continue
        n_env += 1
        assert e["t"] == [0.0, 0.25, 0.5, 0.75, 1.0]
        for key, rng in (("vel", env.bow_vel), ("force", env.bow_force), ("pos", env.bow_pos)):
            assert len(e[key]) == 5 and all(rng[0] <= v <= rng[1] for v in e[key]), key
    assert abs(n_env / n_bow - 0.5) < 0.1


def test_shard_plan_partitions_the_items():
    assert D.shard_ranges(0, 4) == []
    assert D.shard_ranges(10, 4) == [(0, 4), (4, 8), (8, 10)]
    with pytest.raises(ValueError):
        D.shard_ranges(10, 0)
    for world in (1, 2, 3, 5):
        got = sorted(k for r in range(world) for k in D.shards_of_rank(7, r, world))
        assert got == list(range(7))


def test_generate_writes_shards_and_metadata(tmp_path):
    out = str(tmp_path / "ds")
    render = fake_renderer()
    written = D.generate(out, 10, SMALL, seed=3, shard_size=4, render=render, render_items_max=4)
    assert written == [0, 1, 2] and render.calls == [4, 4, 2]
    assert D.merge_metadata(out) == 10
    audio, index, status = D.load(out)
    assert audio.shape == (10, 48) and list(index) == list(range(10)) and not status.any()
    info = json.load(open(os.path.join(out, "dataset.json")))
    assert info["shards"] == 3 and info["channels"] == ["transverse"]
    assert D.Distribution.from_json(info["distribution"]) == SMALL
    lines = [json.loads(l) for l in open(os.path.join(out, "metadata.jsonl"))]
    for i, m in enumerate(lines):
        d = D.draw(SMALL, 3, i)
        assert m["index"] == i and m["params"] == d and m["attempt"] == 0
        assert np.all(audio[i] == np.float32(d["f0"]))
        assert m["peak"] == pytest.approx(float(np.float32(d["f0"])))
    assert not [f for f in os.listdir(out) if ".tmp" in f]


def test_both_channels(tmp_path):
    out = str(tmp_path / "ds")
    dist = D.Distribution(seconds=0.001, output="both")
    D.generate(out, 5, dist, seed=4, shard_size=2, render=fake_renderer())
    audio, _, _ = D.load(out)
    assert audio.shape == (5, 2, 48)
    for i in range(5):
        f0 = np.float32(D.draw(dist, 4, i)["f0"])
        assert np.all(audio[i, 0] == f0) and np.all(audio[i, 1] == f0 + np.float32(1000.0))


def test_failed_strings_are_drawn_again(tmp_path):
    out = str(tmp_path / "ds")
    bad = frozenset(D.draw(SMALL, 5, i)["f0"] for i in (1, 6))
    D.generate(out, 8, SMALL, seed=5, shard_size=4, render=fake_renderer(bad))
    D.merge_metadata(out)
    lines = [json.loads(l) for l in open(os.path.join(out, "metadata.jsonl"))]
    for m in lines:
        if m["index"] in (1, 6):
            assert m["attempt"] == 1 and m["params"] == D.draw(SMALL, 5, m["index"], 1)
            assert m["status"] == 0
        else:
            assert m["attempt"] == 0


def test_persistent_failure_is_kept_and_flagged(tmp_path):
    out = str(tmp_path / "ds")
    bad = frozenset(D.draw(SMALL, 6, 2, a)["f0"] for a in range(3))
    D.generate(out, 4, SMALL, seed=6, shard_size=4, render=fake_renderer(bad), max_attempts=3)
    _, _, status = D.load(out)
    assert list(status) == [0, 0, -3, 0]


def test_shards_are_rendered_in_groups(tmp_path):
    render = fake_renderer()
    D.generate(str(tmp_path / "a"), 10, SMALL, seed=3, shard_size=3, render=render, render_items_max=7)
    assert render.calls == [6, 4]        # shards {0, 1} then {2, 3}: a group never splits a shard
    render = fake_renderer()
    D.generate(str(tmp_path / "b"), 10, SMALL, seed=3, shard_size=3, render=render)
    assert render.calls == [10]
    a, _, _ = D.load(str(tmp_path / "a"))
    b, _, _ = D.load(str(tmp_path / "b"))
    assert np.array_equal(a, b)


def test_dataset_does_not_depend_on_shard_size_or_ranks(tmp_path):
    ref = None
    for shard, world, group in ((3, 1, 4096), (4, 1, 4), (10, 1, 1), (3, 2, 6), (2, 3, 4096)):
        out = str(tmp_path / f"ds{shard}_{world}_{group}")
        for rank in range(world):
            D.generate(out, 10, SMALL, seed=9, shard_size=shard, rank=rank, world=world, render=fake_renderer(),
                       render_items_max=group)
        D.merge_metadata(out)
        audio, index, _ = D.load(out)
        assert list(index) == list(range(10))
        meta = open(os.path.join(out, "metadata.jsonl")).read()
        meta = [{k: v for k, v in json.loads(l).items() if k not in ("shard", "row")} for l in meta.splitlines()]
        if ref is None:
            ref = (audio, meta)
        else:
            assert np.array_equal(audio, ref[0]) and meta == ref[1]


def test_merge_reports_a_missing_shard(tmp_path):
    out = str(tmp_path / "ds")
    D.generate(out, 10, SMALL, seed=3, shard_size=4, rank=0, world=2, render=fake_renderer())
    with pytest.raises(FileNotFoundError):
        D.merge_metadata(out)


def test_writer_error_is_raised(tmp_path, monkeypatch):
    def boom(*a, **k):
        raise OSError("disk full")
    monkeypatch.setattr(D, "_write_shard", boom)
    with pytest.raises(OSError):
        D.generate(str(tmp_path / "ds"), 10, SMALL, seed=3, shard_size=4, render=fake_renderer())


def test_unknown_output_is_rejected(tmp_path):
    with pytest.raises(ValueError):
        D.generate(str(tmp_path / "ds"), 2, D.Distribution(output="sideways"), render=fake_renderer())


def test_cli_writes_a_dataset(tmp_path, monkeypatch, capsys):
    """The command line (python -m paper_2311_18505_gb300.dataset) with a
    stand-in for the GPU renderer: the flags reach the distribution, every
    item is written once, and bowed items get envelopes when asked."""
    class Fake:
        def __init__(self, device):
            self.render = fake_renderer()

        def __call__(self, dicts):
            return self.render(dicts)

        def close(self):
            pass

    monkeypatch.setattr(D, "GpuRenderer", Fake)
    for var in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(var, raising=False)
    out = str(tmp_path / "cli")
    D.main(["--out", out, "--count", "5", "--seconds", "0.001", "--shard-size", "2", "--kinds", "bow",
            "--p-bow-envelope", "1", "--no-modulation"])
    assert json.loads(capsys.readouterr().out.strip().splitlines()[-1]) == {"out": out, "items": 5}
    audio, index, status = D.load(out)
    assert list(index) == list(range(5)) and audio.shape == (5, 48) and not status.any()
    meta = [json.loads(l) for l in open(os.path.join(out, "metadata.jsonl"))]
    assert all(m["params"]["excitation"]["kind"] == "bow" and "envelope" in m["params"]["excitation"]
               for m in meta)
    assert all(m["params"]["modulation"]["kind"] == "none" for m in meta)
    info = json.load(open(os.path.join(out, "dataset.json")))
    assert info["distribution"]["p_bow_envelope"] == 1.0 and info["shards"] == 3
