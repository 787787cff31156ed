"""The dataset generator on the GPU: every stored row is the string's own
synthesis bit for bit (alone, on either channel), the dataset does not
depend on the shard size, and a few items match the FP64 oracle."""

import json
import os

import numpy as np
import pytest

import oracle
from fp32_floor import fp32_floor
from paper_2311_18505_gb300 import dataset as D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIST = D.Distribution(seconds=0.05, output="both")


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


@pytest.fixture(scope="module")
def renderer(sfd):
    r = D.GpuRenderer(0, 1 << 30)
    yield r
    r.close()


@pytest.fixture(scope="module")
def dataset(tmp_path_factory, renderer):
    out = str(tmp_path_factory.mktemp("ds") / "a")
    D.generate(out, 21, DIST, seed=31, shard_size=8, render=renderer)
    assert D.merge_metadata(out) == 21
    return out


def test_rows_are_each_strings_own_synthesis(sfd, renderer, dataset):
    audio, index, status = D.load(dataset)
    assert audio.shape == (21, 2, 2400) and list(index) == list(range(21))
    meta = [json.loads(l) for l in open(os.path.join(dataset, "metadata.jsonl"))]
    assert not status.any()
    for i, m in enumerate(meta):
        d = m["params"]
        for c, ch in enumerate(("transverse", "longitudinal")):
            s = sfd.string_from_dict(renderer.ctx, dict(d, output=ch))
            try:
                assert (m["n_t"], m["n_l"]) == tuple(sfd.sfd_string_info(s)[:2])
                assert np.array_equal(audio[i, c], sfd.sfd_synthesize(s, d["n_samples"])), (i, ch)
            finally:
                sfd.sfd_string_destroy(s)


def test_shard_size_does_not_change_the_dataset(renderer, dataset, tmp_path):
    out = str(tmp_path / "b")
    D.generate(out, 21, DIST, seed=31, shard_size=5, render=renderer)
    a, _, _ = D.load(dataset)
    b, _, _ = D.load(out)
    assert np.array_equal(a, b)


def test_items_match_the_oracle(dataset):
    audio, _, _ = D.load(dataset)
    meta = [json.loads(l) for l in open(os.path.join(dataset, "metadata.jsonl"))]
    picks = [m for m in meta if m["params"]["excitation"]["kind"] != "bow"][:4]
    assert len(picks) >= 3
    for m in picks:
        for c, ch in enumerate(("transverse", "longitudinal")):
            d = dict(m["params"], output=ch)
            ref = oracle.run(d)
            if not np.any(ref):
                assert not np.any(audio[m["index"], c])
                continue
            e = np.linalg.norm(audio[m["index"], c] - ref) / np.linalg.norm(ref)
            assert e <= 1e-4 or e <= 3 * fp32_floor(d, d["n_samples"]), (m["index"], ch, e)


def test_bow_envelope_items(sfd, renderer, tmp_path):
    """Bowed items with time-varying velocity, force and position: each row
    is the string's own synthesis, and its first 150 samples (the window
    before FP32 and FP64 may take a stick/slip switch a step apart) match
    the oracle to 1e-3."""
    dist = D.Distribution(seconds=0.0125, kinds=("bow",), p_bow_envelope=1.0, p_vibrato=0.0, p_gliss=0.0)
    out = str(tmp_path / "bow")
    D.generate(out, 6, dist, seed=5, shard_size=4, render=renderer)
    assert D.merge_metadata(out) == 6
    audio, _, status = D.load(out)
    assert not status.any()
    meta = [json.loads(l) for l in open(os.path.join(out, "metadata.jsonl"))]
    for i, m in enumerate(meta):
        d = m["params"]
        assert "envelope" in d["excitation"]
        s = sfd.string_from_dict(renderer.ctx, d)
        try:
            assert np.array_equal(audio[i], sfd.sfd_synthesize(s, d["n_samples"])), i
        finally:
            sfd.sfd_string_destroy(s)
        ref = oracle.run(d)
        assert np.linalg.norm(audio[i, :150] - ref[:150]) <= 1e-3 * np.linalg.norm(ref[:150]), i
