"""String checkpoints (sfd_string_save / sfd_string_load): a note saved at any
time level continues in another context bit for bit, alone or in a batch,
with its statistics; a buffer that is not an intact checkpoint of this
library is refused.

The full state of a string is its two time levels (Sec. 3.4) in the
increment form the kernel keeps, the hammer's two levels (Eq. 6), the bow's
friction-root warm start (Eq. 5), the coupled solve's warm starts and the
time level, which also fixes the modulation phase and the bow envelope."""

import ctypes
import struct

import numpy as np
import pytest

from paper_2311_18505_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENV = {"t": [0.0, 0.004, 0.01], "vel": [0.1, 0.35, 0.2], "force": [0.4, 1.5, 0.8], "pos": [0.2, 0.3, 0.25]}


@pytest.fixture(scope="module")
def sfd():
    from paper_2311_18505_gb300 import build as B
    B.build()
    from paper_2311_18505_gb300 import sfd as S
    return S


@pytest.fixture(scope="module")
def ctxs(sfd):
    assert torch.cuda.is_available()
    a = sfd.sfd_ctx_create(0, None, 256 << 20)
    b = sfd.sfd_ctx_create(0, None, 256 << 20)
    yield a, b
    sfd.sfd_ctx_destroy(a)
    sfd.sfd_ctx_destroy(b)


def cases():
    """Every excitation, both output channels, linear and nonlinear strings,
    vibrato, a glissando that ends and holds inside the run, a bow envelope,
    and a long longitudinal grid."""
    out = W.batch_mixed(9, seconds=0.1, seed=41)
    out.append(W.make(alpha=3.0, f0=200.0, modulation={"kind": "vibrato", "rate": 40.0, "depth": 50.0,
                                                       "phase": 0.3}, n_samples=4800))
    out.append(W.make(alpha=2.0, f0=90.0, modulation={"kind": "gliss", "depth": 1.0, "duration": 0.03},
                      excitation={"kind": "hammer", "mass": 0.01, "vel": 2.0, "pos": 0.2, "omega": 3e3,
                                  "alpha": 2.5}, n_samples=4800))
    out.append(W.make(alpha=4.0, f0=150.0, excitation={"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.2,
                                                       "a": 100.0, "eps": 0.1, "release": 0.05,
                                                       "envelope": ENV}, n_samples=4800))
    out.append(W.make(alpha=1.0, f0=110.0, n_samples=4800))
    out.append(W.make(alpha=1.05, f0=85.0, output="longitudinal", n_samples=4800))
    return out


def split_points(n):
    return [0, 1, 2, 3, 33, n // 3, n - 1]


def test_resume_in_another_context_bitwise(sfd, ctxs):
    """Synthesize m samples, save, load the checkpoint into a second context
    and synthesize the rest: the samples equal one uninterrupted call, for
    checkpoints taken before the first sample, at the initial levels and
    mid-note; the saved string itself continues unchanged too."""
    a, b = ctxs
    for d in cases():
        n = d["n_samples"]
        s = sfd.string_from_dict(a, d)
        ref = sfd.sfd_synthesize(s, n)
        sfd.sfd_string_destroy(s)
        for m in split_points(n):
            s = sfd.string_from_dict(a, d)
            head = sfd.sfd_synthesize(s, m) if m else np.zeros(0, np.float32)
            blob = sfd.sfd_string_save(s)
            t = sfd.sfd_string_load(b, blob)
            assert sfd.sfd_string_position(t) == sfd.sfd_string_position(s)
            tail_b = sfd.sfd_synthesize(t, n - m)
            tail_a = sfd.sfd_synthesize(s, n - m)
            sfd.sfd_string_destroy(t)
            sfd.sfd_string_destroy(s)
            assert np.array_equal(np.concatenate([head, tail_b]), ref), (d["excitation"]["kind"], m)
            assert np.array_equal(tail_a, tail_b)


def test_resume_inside_a_batch(sfd, ctxs):
    """Checkpoints of several notes loaded into one context and advanced as a
    batch give each note's uninterrupted samples."""
    a, b = ctxs
    ds = cases()
    m = 1500
    refs, blobs = [], []
    for d in ds:
        s = sfd.string_from_dict(a, d)
        refs.append(sfd.sfd_synthesize(s, d["n_samples"]))
        sfd.sfd_string_destroy(s)
        s = sfd.string_from_dict(a, d)
        sfd.sfd_synthesize(s, m)
        blobs.append(sfd.sfd_string_save(s))
        sfd.sfd_string_destroy(s)
    hs = [sfd.sfd_string_load(b, x) for x in blobs]
    bt = sfd.sfd_batch_create(b, hs)
    ys, _ = sfd.sfd_batch_synthesize_host(bt, [d["n_samples"] - m for d in ds])
    sfd.sfd_batch_destroy(bt)
    for h in hs:
        sfd.sfd_string_destroy(h)
    for y, r in zip(ys, refs):
        assert np.array_equal(y, r[m:])


def test_checkpoint_after_a_regrid(sfd, ctxs):
    """A string created with a grid too fine for its modulation gets the
    peak's grid from sfd_set_modulation; its checkpoint reloads on that grid
    and continues bit for bit."""
    a, b = ctxs
    d = W.make(alpha=2.0, f0=120.0, gamma_max_ratio=1.0,
               modulation={"kind": "vibrato", "rate": 7.0, "depth": 80.0, "phase": 1.1}, n_samples=4000)
    s = sfd.string_from_dict(a, d)
    ref = sfd.sfd_synthesize(s, 4000)
    grid = sfd.sfd_string_info(s)[:2]
    sfd.sfd_string_destroy(s)
    s = sfd.string_from_dict(a, d)
    head = sfd.sfd_synthesize(s, 1234)
    t = sfd.sfd_string_load(b, sfd.sfd_string_save(s))
    sfd.sfd_string_destroy(s)
    assert sfd.sfd_string_info(t)[:2] == grid
    tail = sfd.sfd_synthesize(t, 4000 - 1234)
    sfd.sfd_string_destroy(t)
    assert np.array_equal(np.concatenate([head, tail]), ref)


def test_statistics_and_state_carry_over(sfd, ctxs):
    """Status, sweep statistics, state and hammer position of a loaded string
    equal the saved string's; a loaded note that had started refuses a new
    excitation like the original (SFD_ESTATE)."""
    a, b = ctxs
    d = W.make(alpha=3.0, f0=140.0, excitation={"kind": "hammer", "mass": 0.008, "vel": 2.5, "pos": 0.15,
                                                "omega": 3e3, "alpha": 2.5}, n_samples=3000)
    s = sfd.string_from_dict(a, d)
    sfd.sfd_synthesize(s, 777)
    t = sfd.sfd_string_load(b, sfd.sfd_string_save(s))
    assert sfd.sfd_string_stats(t) == sfd.sfd_string_stats(s)
    assert sfd.sfd_string_hammer(t) == sfd.sfd_string_hammer(s)
    for x, y in zip(sfd.sfd_string_delta_state(t), sfd.sfd_string_delta_state(s)):
        assert np.array_equal(x, y)
    with pytest.raises(sfd.SfdError) as e:
        sfd.sfd_excite_pluck(t, 1e-3, 0.3)
    assert e.value.code == sfd.SFD_ESTATE
    sfd.sfd_string_destroy(t)
    sfd.sfd_string_destroy(s)


def test_refused_checkpoints(sfd, ctxs):
    """Not a checkpoint, truncated, a size that disagrees with the header, a
    changed descriptor byte, a changed parameter and an inconsistent time
    level are all refused with SFD_EINVAL, and the context keeps working."""
    a, b = ctxs
    d = W.make(alpha=3.0, f0=160.0, n_samples=2000)
    s = sfd.string_from_dict(a, d)
    sfd.sfd_synthesize(s, 500)
    blob = bytearray(sfd.sfd_string_save(s))
    used0 = sfd.sfd_ctx_memory(b)[0]

    def refused(buf):
        with pytest.raises(sfd.SfdError) as e:
            sfd.sfd_string_load(b, bytes(buf))
        assert e.value.code == sfd.SFD_EINVAL
        assert sfd.sfd_ctx_memory(b)[0] == used0   # nothing left allocated

    bad = bytearray(blob); bad[0] ^= 0xFF
    refused(bad)                                   # magic
    refused(blob[:100])                            # truncated
    refused(blob[:-4])                             # size differs from the header
    refused(blob + b"\0" * 8)
    # header: magic[8], version, header_bytes (u32), total (u64), 4 x u32,
    # state offset and size (u64), n_t, n_l, started, pad (i32)
    hdr = struct.calcsize("<8sIIQIIIIQQiiii")
    params = ctypes.sizeof(sfd.sfd_string_params)
    rec = int(struct.unpack_from("<I", blob, 36)[0])
    desc_at = hdr + rec
    state_at = desc_at + int(struct.unpack_from("<I", blob, 28)[0])
    # a coefficient of the descriptor (dg, offset 48)
    bad = bytearray(blob); bad[desc_at + 48] ^= 0x01
    refused(bad)
    # kappa (the third double of the parameters, first in the record) moved
    # by 0.4 %: a valid string whose descriptor is not the saved one
    bad = bytearray(blob); bad[hdr + 16 + 5] ^= 0x10
    refused(bad)
    # time level n (Scalars: uh, duh floats, then n) moved far from the next sample
    bad = bytearray(blob)
    struct.pack_into("<q", bad, state_at + 8, 10 ** 6)
    refused(bad)
    assert params > 0
    # the intact checkpoint still loads and continues
    t = sfd.sfd_string_load(b, bytes(blob))
    assert np.array_equal(sfd.sfd_synthesize(t, 300), sfd.sfd_synthesize(s, 300))
    sfd.sfd_string_destroy(t)
    sfd.sfd_string_destroy(s)


def test_save_size_query(sfd, ctxs):
    """With no buffer the call reports the size; a buffer one byte short is
    refused with the size needed."""
    a, _ = ctxs
    s = sfd.string_from_dict(a, W.make(alpha=2.0, n_samples=100))
    L = sfd.lib()
    n = ctypes.c_size_t()
    assert L.sfd_string_save(s, None, ctypes.byref(n)) == sfd.SFD_OK
    need = n.value
    buf = ctypes.create_string_buffer(need)
    n.value = need - 1
    assert L.sfd_string_save(s, buf, ctypes.byref(n)) == sfd.SFD_EINVAL
    assert n.value == need
    n.value = need
    assert L.sfd_string_save(s, buf, ctypes.byref(n)) == sfd.SFD_OK and n.value == need
    sfd.sfd_string_destroy(s)
