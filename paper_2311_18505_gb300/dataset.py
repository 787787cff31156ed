"""Dataset construction with the GPU synthesizer.

The synthesizer's randomised control parameters and material properties
(Sec. 1; the concluding Sec. 5 names dataset construction as its use) are
drawn here per item and rendered in GPU batches into sharded files:

    <out>/dataset.json            the distribution, seed, count, layout
    <out>/shard-00000.npz         audio float32 [rows, n_samples] (or
                                  [rows, 2, n_samples] with both channels,
                                  transverse first), index int64 [rows],
                                  status int32 [rows]
    <out>/shard-00000.jsonl       one line per row: index, parameters, grid,
                                  status, attempt, peak and rms
    <out>/metadata.jsonl          every shard's lines, in index order
                                  (merge_metadata)

Item i's parameters depend only on (seed, i, attempt), and a string's
samples do not depend on the batch it is rendered in, so a dataset is the
same bit for bit whatever the shard size or the number of ranks.  Shards
are dealt to ranks round-robin (shard k to rank k mod N); ranks share no
data, so N GPUs scale weakly with no collective.

A string whose run fails (SFD_EUNSTABLE, SFD_ENOCONV) is drawn again with
the next attempt number, up to `max_attempts`; the last failure is kept and
flagged in its status.

Marshalling and file I/O only: every sample is computed by the CUDA library
(`sfd`).  This module holds no arithmetic of the scheme.
"""

from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import queue
import threading
from typing import Callable, Sequence

import numpy as np

from . import workloads as W

FORMAT_VERSION = 1
GROUP_BYTES = 1 << 30      # output bytes of one rendered group (device pool and host copies)


@dataclasses.dataclass
class Distribution:
    """Ranges of the randomised parameters (Table 1 notation).  Pairs are
    (low, high) of a uniform draw; f0 and sigma1 are drawn log-uniform."""
    f0: tuple = (40.0, 1000.0)
    kappa: tuple = (0.5, 3.0)
    alpha: tuple = (1.0, 10.0)
    sigma0: tuple = (0.1, 2.0)
    sigma1: tuple = (1e-6, 1e-4)
    pickup: tuple = (0.55, 0.9)
    kinds: tuple = ("pluck", "hammer", "bow")
    # pluck: peak amplitude c0 [m], position x_P
    pluck_amp: tuple = (0.1e-3, 2e-3)
    pluck_pos: tuple = (0.1, 0.5)
    # hammer: mass [kg], velocity v_H [m/s], position x_H, omega_H, alpha_H
    hammer_mass: tuple = (1e-3, 10e-3)
    hammer_vel: tuple = (0.5, 5.0)
    hammer_pos: tuple = (0.1, 0.5)
    hammer_omega: tuple = (1000.0, 5000.0)
    hammer_alpha: tuple = (1.5, 3.5)
    # bow: v_B [m/s], F_B [N], x_B, and the friction curve's a and epsilon,
    # which the paper also randomises (Sec. 3.3.1)
    bow_vel: tuple = (0.05, 0.5)
    bow_force: tuple = (0.1, 2.0)
    bow_pos: tuple = (0.1, 0.5)
    bow_a: tuple = (20.0, 200.0)
    bow_eps: tuple = (0.05, 0.3)
    bow_release: tuple = (0.5, 1.5)      # release time as a fraction of the note; >= 1: held
    # time-varying bow controls (Sec. 3.3.1): with this probability a bowed
    # item's v_B, F_B and x_B are envelopes through bow_env_points values
    # drawn from the ranges above, evenly spaced over the note, linear between
    p_bow_envelope: float = 0.0
    bow_env_points: int = 4
    # f0 modulation: probabilities of a vibrato and of a glissando
    p_vibrato: float = 0.25
    p_gliss: float = 0.25
    vibrato_rate: tuple = (4.0, 8.0)     # Hz
    vibrato_depth: tuple = (5.0, 50.0)   # cents
    gliss_depth: tuple = (-1.0, 1.0)     # octaves
    gliss_duration: tuple = (0.25, 1.0)  # fraction of the note
    seconds: float = 1.0
    fs: float = 48000.0
    output: str = "transverse"           # "transverse", "longitudinal" or "both"

    def to_json(self) -> dict:
        return dataclasses.asdict(self)

    @classmethod
    def from_json(cls, d: dict) -> "Distribution":
        return cls(**{k: tuple(v) if isinstance(v, list) else v for k, v in d.items()})


def _u(rng, lo_hi):
    return float(rng.uniform(lo_hi[0], lo_hi[1]))


def _logu(rng, lo_hi):
    return float(math.exp(rng.uniform(math.log(lo_hi[0]), math.log(lo_hi[1]))))


def draw(dist: Distribution, seed: int, index: int, attempt: int = 0) -> dict:
    """Parameters of item `index` (a string dict of `workloads`), a function
    of (seed, index, attempt) alone."""
    rng = np.random.Generator(np.random.PCG64([int(seed), int(index), int(attempt)]))
    n = int(round(dist.fs * dist.seconds))
    kind = dist.kinds[int(rng.integers(len(dist.kinds)))]
    if kind == "pluck":
        ex = {"kind": "pluck", "amp": _u(rng, dist.pluck_amp), "pos": _u(rng, dist.pluck_pos)}
    elif kind == "hammer":
        ex = {"kind": "hammer", "mass": _u(rng, dist.hammer_mass), "vel": _u(rng, dist.hammer_vel),
              "pos": _u(rng, dist.hammer_pos), "omega": _u(rng, dist.hammer_omega),
              "alpha": _u(rng, dist.hammer_alpha)}
    elif kind == "bow":
        rel = _u(rng, dist.bow_release)
        ex = {"kind": "bow", "vel": _u(rng, dist.bow_vel), "force": _u(rng, dist.bow_force),
              "pos": _u(rng, dist.bow_pos), "a": _u(rng, dist.bow_a), "eps": _u(rng, dist.bow_eps),
              "release": rel * dist.seconds if rel < 1.0 else -1.0}
        if dist.p_bow_envelope > 0.0:
            # a stream of its own, so the other draws stay those of p_bow_envelope = 0
            erng = np.random.Generator(np.random.PCG64([int(seed), int(index), int(attempt), 1]))
            if float(erng.uniform()) < dist.p_bow_envelope:
                m = min(16, max(2, int(dist.bow_env_points)))
                ex["envelope"] = {"t": [dist.seconds * j / (m - 1) for j in range(m)],
                                  "vel": [_u(erng, dist.bow_vel) for _ in range(m)],
                                  "force": [_u(erng, dist.bow_force) for _ in range(m)],
                                  "pos": [_u(erng, dist.bow_pos) for _ in range(m)]}
    else:
        raise ValueError(f"unknown excitation kind {kind!r}")
    r = float(rng.uniform())
    if r < dist.p_vibrato:
        mod = {"kind": "vibrato", "rate": _u(rng, dist.vibrato_rate), "depth": _u(rng, dist.vibrato_depth),
               "phase": float(rng.uniform(0.0, 2.0 * math.pi))}
    elif r < dist.p_vibrato + dist.p_gliss:
        mod = {"kind": "gliss", "depth": _u(rng, dist.gliss_depth),
               "duration": _u(rng, dist.gliss_duration) * dist.seconds}
    else:
        mod = {"kind": "none"}
    return W.make(
        f0=_logu(rng, dist.f0), kappa=_u(rng, dist.kappa), alpha=_u(rng, dist.alpha),
        sigma0=_u(rng, dist.sigma0), sigma1=_logu(rng, dist.sigma1), pickup=_u(rng, dist.pickup),
        excitation=ex, modulation=mod, fs=dist.fs, n_samples=n)


def channels(dist: Distribution) -> list[str]:
    if dist.output == "both":
        return ["transverse", "longitudinal"]
    if dist.output in ("transverse", "longitudinal"):
        return [dist.output]
    raise ValueError(f"unknown output {dist.output!r}")


def shard_ranges(count: int, shard_size: int) -> list[tuple[int, int]]:
    """[first, end) item ranges of the shards; the last may be short."""
    if count < 0 or shard_size <= 0:
        raise ValueError("count must be >= 0 and shard_size > 0")
    return [(a, min(a + shard_size, count)) for a in range(0, count, shard_size)]


def shards_of_rank(n_shards: int, rank: int, world: int) -> list[int]:
    return list(range(rank, n_shards, world))


# A renderer takes string dicts of one length and returns (audio [n,
# n_samples] float32, status [n] int32, grids [(n_t, n_l)] * n).
Renderer = Callable[[Sequence[dict]], tuple]


class GpuRenderer:
    """Renders batches with the CUDA library on one device."""

    def __init__(self, device: int = 0, pool_bytes: int = 2 << 30):
        from . import sfd
        self.sfd = sfd
        self.ctx = sfd.sfd_ctx_create(device, None, pool_bytes)

    def __call__(self, dicts: Sequence[dict]):
        sfd = self.sfd
        if not dicts:
            return np.zeros((0, 0), np.float32), np.zeros(0, np.int32), []
        n = dicts[0]["n_samples"]
        if any(d["n_samples"] != n for d in dicts):
            raise ValueError("a renderer batch has one note length")
        hs = []
        try:
            for d in dicts:
                hs.append(sfd.string_from_dict(self.ctx, d))
            grids = [tuple(sfd.sfd_string_info(h)[:2]) for h in hs]
            b = sfd.sfd_batch_create(self.ctx, hs)
            try:
                offs = np.arange(len(hs), dtype=np.int64) * n
                ys, st = sfd.sfd_batch_synthesize_host(b, [n] * len(hs), offs, check=False)
            finally:
                sfd.sfd_batch_destroy(b)
            audio = np.stack(ys) if n else np.zeros((len(hs), 0), np.float32)
            return audio, st.astype(np.int32), grids
        finally:
            for h in hs:
                sfd.sfd_string_destroy(h)

    def close(self):
        if self.ctx:
            self.sfd.sfd_ctx_destroy(self.ctx)
            self.ctx = None


def render_items(render: Renderer, dist: Distribution, seed: int, indices: Sequence[int],
                 max_attempts: int = 3):
    """Audio [rows, (channels,) n_samples], status, attempts, params, grids of
    the items `indices`; failed items are drawn again (next attempt)."""
    chans = channels(dist)
    rows = len(indices)
    attempts = np.zeros(rows, np.int32)
    params = [draw(dist, seed, i, 0) for i in indices]
    n = int(round(dist.fs * dist.seconds))
    audio = np.zeros((rows, len(chans), n), np.float32)
    status = np.zeros(rows, np.int32)
    grids = [None] * rows
    todo = list(range(rows))
    while todo:
        dicts = [dict(params[r], output=c) for r in todo for c in chans]
        a, st, g = render(dicts)
        a = np.asarray(a).reshape(len(todo), len(chans), n)
        st = np.asarray(st).reshape(len(todo), len(chans))
        retry = []
        for k, r in enumerate(todo):
            audio[r] = a[k]
            status[r] = next((int(s) for s in st[k] if s != 0), 0)
            grids[r] = g[k * len(chans)]
            if status[r] != 0 and attempts[r] + 1 < max_attempts:
                attempts[r] += 1
                params[r] = draw(dist, seed, indices[r], int(attempts[r]))
                retry.append(r)
        todo = retry
    if len(chans) == 1:
        audio = audio[:, 0]
    return audio, status, attempts, params, grids


def _shard_name(k: int) -> str:
    return f"shard-{k:05d}"


def _write_shard(out: str, k: int, indices, audio, status, attempts, params, grids) -> None:
    base = os.path.join(out, _shard_name(k))
    tmp = base + ".tmp.npz"
    np.savez(tmp, audio=audio, index=np.asarray(indices, np.int64), status=status)
    os.replace(tmp, base + ".npz")
    with open(base + ".jsonl.tmp", "w") as f:
        for row, i in enumerate(indices):
            a = audio[row].astype(np.float64)
            f.write(json.dumps({
                "index": int(i), "shard": k, "row": row, "status": int(status[row]),
                "attempt": int(attempts[row]), "n_t": int(grids[row][0]), "n_l": int(grids[row][1]),
                "peak": float(np.max(np.abs(a))) if a.size else 0.0,
                "rms": float(np.sqrt(np.mean(a * a))) if a.size else 0.0,
                "params": params[row]}) + "\n")
    os.replace(base + ".jsonl.tmp", base + ".jsonl")


def generate(out: str, count: int, dist: Distribution | None = None, seed: int = 0,
             shard_size: int = 256, rank: int = 0, world: int = 1,
             render: Renderer | None = None, max_attempts: int = 3, device: int = 0,
             render_items_max: int = 4096) -> list[int]:
    """Render this rank's shards of a `count`-item dataset into `out`.
    Consecutive shards of the rank are rendered together, up to
    `render_items_max` items per GPU batch (a batch takes about as long as
    its slowest string, so larger batches keep more of the GPU busy), and
    the writing of one group overlaps the rendering of the next.  A group
    also holds at most `GROUP_BYTES` of output (the batch's device output
    buffer comes from the renderer's pool).  Returns the shard numbers
    written."""
    dist = dist or Distribution()
    channels(dist)
    os.makedirs(out, exist_ok=True)
    ranges = shard_ranges(count, shard_size)
    mine = shards_of_rank(len(ranges), rank, world)
    if rank == 0:
        with open(os.path.join(out, "dataset.json"), "w") as f:
            json.dump({"format": FORMAT_VERSION, "count": count, "seed": seed, "shard_size": shard_size,
                       "shards": len(ranges), "channels": channels(dist),
                       "distribution": dist.to_json()}, f, indent=1)
    own = render is None
    if own:
        render = GpuRenderer(device)
    pending: queue.Queue = queue.Queue(maxsize=max(1, render_items_max // max(shard_size, 1)))
    errors: list[BaseException] = []

    def writer():
        while True:
            job = pending.get()
            if job is None:
                return
            try:
                _write_shard(out, *job)
            except BaseException as e:   # reported after the join
                errors.append(e)

    th = threading.Thread(target=writer, daemon=True)
    th.start()
    per_item = len(channels(dist)) * int(round(dist.fs * dist.seconds)) * 4
    cap = max(1, min(render_items_max, GROUP_BYTES // max(per_item, 1)))
    groups, cur, size = [], [], 0
    for k in mine:
        n = ranges[k][1] - ranges[k][0]
        if cur and size + n > cap:
            groups.append(cur)
            cur, size = [], 0
        cur.append(k)
        size += n
    if cur:
        groups.append(cur)
    try:
        for grp in groups:
            idx = [i for k in grp for i in range(*ranges[k])]
            audio, status, attempts, params, grids = render_items(render, dist, seed, idx, max_attempts)
            o = 0
            for k in grp:
                n = ranges[k][1] - ranges[k][0]
                pending.put((k, idx[o:o + n], audio[o:o + n], status[o:o + n], attempts[o:o + n],
                             params[o:o + n], grids[o:o + n]))
                o += n
            if errors:
                break
    finally:
        pending.put(None)
        th.join()
        if own:
            render.close()
    if errors:
        raise errors[0]
    return mine


def merge_metadata(out: str) -> int:
    """Concatenate the shards' metadata into metadata.jsonl in index order;
    returns the number of items.  Raises if a shard is missing."""
    with open(os.path.join(out, "dataset.json")) as f:
        info = json.load(f)
    lines = []
    for k in range(info["shards"]):
        with open(os.path.join(out, _shard_name(k) + ".jsonl")) as f:
            lines.extend(f.readlines())
    lines.sort(key=lambda s: json.loads(s)["index"])
    with open(os.path.join(out, "metadata.jsonl"), "w") as f:
        f.writelines(lines)
    return len(lines)


def load(out: str):
    """(audio, index, status) of the whole dataset, in index order."""
    with open(os.path.join(out, "dataset.json")) as f:
        info = json.load(f)
    parts = [np.load(os.path.join(out, _shard_name(k) + ".npz")) for k in range(info["shards"])]
    if not parts:
        return np.zeros((0,), np.float32), np.zeros(0, np.int64), np.zeros(0, np.int32)
    return (np.concatenate([p["audio"] for p in parts]), np.concatenate([p["index"] for p in parts]),
            np.concatenate([p["status"] for p in parts]))


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description="Render a synthetic string dataset on the GPU.")
    ap.add_argument("--out", required=True)
    ap.add_argument("--count", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--seconds", type=float, default=1.0)
    ap.add_argument("--fs", type=float, default=48000.0)
    ap.add_argument("--shard-size", type=int, default=256)
    ap.add_argument("--output", choices=("transverse", "longitudinal", "both"), default="transverse")
    ap.add_argument("--kinds", default="pluck,hammer,bow")
    ap.add_argument("--f0", type=float, nargs=2, default=(40.0, 1000.0))
    ap.add_argument("--no-modulation", action="store_true")
    ap.add_argument("--p-bow-envelope", type=float, default=0.0,
                    help="probability that a bowed item's velocity, force and position vary in time")
    ap.add_argument("--device", type=int, default=None)
    args = ap.parse_args(argv)
    dist = Distribution(seconds=args.seconds, fs=args.fs, output=args.output,
                        kinds=tuple(args.kinds.split(",")), f0=tuple(args.f0))
    if args.no_modulation:
        dist.p_vibrato = dist.p_gliss = 0.0
    dist.p_bow_envelope = args.p_bow_envelope
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    device = args.device if args.device is not None else int(os.environ.get("LOCAL_RANK", "0"))
    generate(args.out, args.count, dist, args.seed, args.shard_size, rank, world, device=device)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("gloo")
        tdist.barrier()   # every shard on disk before the merge
        tdist.destroy_process_group()
    if rank == 0:
        n = merge_metadata(args.out)
        print(json.dumps({"out": args.out, "items": n}))


if __name__ == "__main__":
    main()
