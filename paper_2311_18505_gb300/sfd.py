"""Python binding of the C-ABI in include/sfd.h (ctypes).

Argument marshalling only: every step of the time-stepping runs in the CUDA
library ``_build/libsfd.so``.  There is no CPU fallback; importing this
module raises if the library has not been built.

The functions keep the C names.  ``string_from_dict`` marshals a parameter
dictionary (see ``workloads``) into create / excite / modulation calls.
"""

from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfd.so")

SFD_OK, SFD_EINVAL, SFD_ENOMEM, SFD_EUNSTABLE, SFD_ENOCONV = 0, -1, -2, -3, -4
SFD_ECUDA, SFD_ETIMEOUT, SFD_EBUSY, SFD_ESTATE = -5, -6, -7, -8
STATUS_NAMES = {0: "SFD_OK", -1: "SFD_EINVAL", -2: "SFD_ENOMEM", -3: "SFD_EUNSTABLE", -4: "SFD_ENOCONV",
                -5: "SFD_ECUDA", -6: "SFD_ETIMEOUT", -7: "SFD_EBUSY", -8: "SFD_ESTATE"}
SFD_MOD_NONE, SFD_MOD_VIBRATO, SFD_MOD_GLISS = 0, 1, 2
MOD_KINDS = {"none": SFD_MOD_NONE, "vibrato": SFD_MOD_VIBRATO, "gliss": SFD_MOD_GLISS}
SFD_OUTPUT_TRANSVERSE, SFD_OUTPUT_LONGITUDINAL = 0, 1
OUTPUTS = {"transverse": SFD_OUTPUT_TRANSVERSE, "longitudinal": SFD_OUTPUT_LONGITUDINAL}


class SfdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class sfd_string_params(ctypes.Structure):
    _fields_ = [
        ("f0", ctypes.c_double), ("gamma", ctypes.c_double), ("kappa", ctypes.c_double),
        ("alpha", ctypes.c_double), ("sigma0", ctypes.c_double), ("sigma1", ctypes.c_double),
        ("length_m", ctypes.c_double), ("fs", ctypes.c_double), ("linear_density", ctypes.c_double),
        ("theta", ctypes.c_double), ("boundary", ctypes.c_int32), ("grid_rule", ctypes.c_int32),
        ("pickup_pos", ctypes.c_double), ("f0_max_ratio", ctypes.c_double),
        ("output", ctypes.c_int32), ("pad_", ctypes.c_int32),
    ]


class sfd_excitation(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("amp_m", ctypes.c_double), ("pos", ctypes.c_double),
        ("mass_kg", ctypes.c_double), ("vel_mps", ctypes.c_double), ("omega_h", ctypes.c_double),
        ("alpha_h", ctypes.c_double), ("force_n", ctypes.c_double), ("a_s_per_m", ctypes.c_double),
        ("eps", ctypes.c_double), ("release_time_s", ctypes.c_double),
    ]


SFD_NOALLOC_SCRATCH_BYTES = 32 * 1024


class sfd_modulation(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("rate_hz", ctypes.c_double), ("depth", ctypes.c_double),
        ("phase_rad", ctypes.c_double), ("duration_s", ctypes.c_double),
    ]


class sfd_request(ctypes.Structure):
    _fields_ = [
        ("params", sfd_string_params), ("exc", sfd_excitation),
        ("mod_kind", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("mod_rate_hz", ctypes.c_double), ("mod_depth", ctypes.c_double),
        ("mod_phase_rad", ctypes.c_double), ("mod_duration_s", ctypes.c_double),
        ("n_samples", ctypes.c_int64), ("arrival_s", ctypes.c_double), ("tag", ctypes.c_uint64),
    ]


class sfd_chunk(ctypes.Structure):
    _fields_ = [
        ("tag", ctypes.c_uint64), ("first_sample", ctypes.c_int64), ("n", ctypes.c_int32),
        ("last", ctypes.c_int32), ("status", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("samples", ctypes.POINTER(ctypes.c_float)), ("ready_s", ctypes.c_double), ("arrival_s", ctypes.c_double),
    ]


class sfd_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("queued", "live", "submitted", "admitted", "completed", "chunks",
                                               "samples", "in_flight")] + \
               [("pool_used", ctypes.c_uint64), ("pool_size", ctypes.c_uint64)]

_lib = None


def lib() -> ctypes.CDLL:
    """Load libsfd.so; raise if it is missing (the CUDA path is mandatory)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2311_18505_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "sfd_params_default": (None, [P(sfd_string_params)]),
        "sfd_ctx_create": (i32, [ctypes.c_int, vp, ctypes.c_size_t, P(vp)]),
        "sfd_ctx_destroy": (None, [vp]),
        "sfd_ctx_memory": (i32, [vp, P(ctypes.c_size_t), P(ctypes.c_size_t)]),
        "sfd_string_create": (i32, [vp, P(sfd_string_params), P(vp)]),
        "sfd_string_info": (i32, [vp, P(i32), P(i32), P(dbl), P(dbl)]),
        "sfd_grid": (i32, [P(sfd_string_params), P(i32), P(i32)]),
        "sfd_excite_pluck": (i32, [vp, dbl, dbl]),
        "sfd_excite_hammer": (i32, [vp, dbl, dbl, dbl, dbl, dbl]),
        "sfd_excite_bow": (i32, [vp, dbl, dbl, dbl, dbl, dbl, dbl]),
        "sfd_bow_envelope": (i32, [vp, i32, P(dbl), P(dbl), P(dbl), P(dbl)]),
        "sfd_set_modulation": (i32, [vp, i32, dbl, dbl, dbl, dbl]),
        "sfd_modulation_peak": (i32, [i32, dbl, P(dbl)]),
        "sfd_synthesize": (i32, [vp, i64, vp, i32]),
        "sfd_string_position": (i32, [vp, P(i64), P(i64)]),
        "sfd_string_state": (i32, [vp, vp, vp, vp, vp]),
        "sfd_string_destroy": (i32, [vp]),
        "sfd_string_stats": (i32, [vp, P(i32), P(i32), P(i64)]),
        "sfd_string_delta_state": (i32, [vp, vp, vp, vp, vp]),
        "sfd_string_hammer": (i32, [vp, P(dbl), P(dbl)]),
        "sfd_string_save": (i32, [vp, vp, P(ctypes.c_size_t)]),
        "sfd_string_load": (i32, [vp, vp, ctypes.c_size_t, P(vp)]),
        "sfd_ctx_set_sweep_cap": (i32, [vp, i32]),
        "sfd_batch_create": (i32, [vp, i32, P(vp), P(vp)]),
        "sfd_batch_synthesize": (i32, [vp, P(i64), vp, P(i64), P(i32)]),
        "sfd_batch_synthesize_host": (i32, [vp, P(i64), vp, P(i64), P(i32)]),
        "sfd_batch_destroy": (i32, [vp]),
        "sfd_batch_set_warps_per_cta": (i32, [vp, i32]),
        "sfd_batch_autotune": (i32, [vp, i64, P(i32)]),
        "sfd_batch_prepare": (i32, [vp, P(i64), vp, P(i64)]),
        "sfd_batch_launch": (i32, [vp]),
        "sfd_last_launch_count": (i32, [vp]),
        "sfd_ctx_transfer_bytes": (i32, [vp, P(ctypes.c_uint64), P(ctypes.c_uint64)]),
        "sfd_ctx_set_timing": (i32, [vp, i32]),
        "sfd_ctx_set_warp_pairs": (i32, [vp, i32]),
        "sfd_ctx_kernel_times": (i32, [vp, P(ctypes.c_float), P(i32)]),
        "sfd_string_kernel_class": (i32, [vp, P(i32)]),
        "sfd_synthesize_noalloc": (i32, [ctypes.c_int, vp, P(sfd_string_params), P(sfd_excitation), i64, vp]),
        "sfd_server_create": (i32, [vp, i32, i32, P(vp)]),
        "sfd_server_submit": (i32, [vp, P(sfd_request)]),
        "sfd_server_submit_bow_envelope": (i32, [vp, P(sfd_request), i32, P(dbl), P(dbl), P(dbl), P(dbl)]),
        "sfd_server_pump": (i32, [vp, P(P(sfd_chunk)), P(i32)]),
        "sfd_server_clock": (dbl, [vp]),
        "sfd_server_stats_get": (i32, [vp, P(sfd_server_stats)]),
        "sfd_server_destroy": (i32, [vp]),
        "sfd_tape_create": (i32, [vp, i32, P(sfd_string_params), P(sfd_excitation), P(sfd_modulation), i64, i32,
                                  P(vp)]),
        "sfd_tape_forward": (i32, [vp, vp]),
        "sfd_tape_backward": (i32, [vp, vp, P(dbl)]),
        "sfd_tape_destroy": (i32, [vp]),
        "sfd_tape_set_record_forward": (i32, [vp, i32]),
        "sfd_measure_peaks": (i32, [ctypes.c_int, P(dbl), P(dbl), P(dbl)]),
        "sfd_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def _check(rc: int, allow=()) -> int:
    if rc != SFD_OK and rc not in allow:
        raise SfdError(rc, lib().sfd_last_error().decode(errors="replace"))
    return rc


def _i64p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


# ---------------------------------------------------------------- C names

def sfd_params_default() -> sfd_string_params:
    p = sfd_string_params()
    lib().sfd_params_default(ctypes.byref(p))
    return p


def sfd_ctx_create(device: int = 0, stream: int | None = None, mem_budget_bytes: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfd_ctx_create(device, stream, mem_budget_bytes, ctypes.byref(h)))
    return h.value


def sfd_ctx_destroy(ctx: int) -> None:
    lib().sfd_ctx_destroy(ctx)


def sfd_ctx_memory(ctx: int) -> tuple[int, int]:
    u, t = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().sfd_ctx_memory(ctx, ctypes.byref(u), ctypes.byref(t)))
    return u.value, t.value


def sfd_string_create(ctx: int, params: sfd_string_params) -> int:
    h = ctypes.c_void_p()
    _check(lib().sfd_string_create(ctx, ctypes.byref(params), ctypes.byref(h)))
    return h.value


def sfd_grid(params: sfd_string_params) -> tuple[int, int]:
    """(N_t, N_l) of a string with these parameters; host arithmetic, no device."""
    nt, nl = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sfd_grid(ctypes.byref(params), ctypes.byref(nt), ctypes.byref(nl)))
    return nt.value, nl.value


def sfd_string_info(s: int) -> tuple[int, int, float, float]:
    nt, nl, ht, hl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sfd_string_info(s, ctypes.byref(nt), ctypes.byref(nl), ctypes.byref(ht), ctypes.byref(hl)))
    return nt.value, nl.value, ht.value, hl.value


def sfd_excite_pluck(s: int, amp_m: float, pos: float) -> None:
    _check(lib().sfd_excite_pluck(s, amp_m, pos))


def sfd_excite_hammer(s: int, mass_kg: float, vel_mps: float, pos: float, omega_h: float = 3000.0,
                      alpha_h: float = 2.5) -> None:
    _check(lib().sfd_excite_hammer(s, mass_kg, vel_mps, pos, omega_h, alpha_h))


def sfd_excite_bow(s: int, vel_mps: float, force_n: float, pos: float, a_s_per_m: float = 100.0,
                   eps: float = 0.1, release_time_s: float = -1.0) -> None:
    _check(lib().sfd_excite_bow(s, vel_mps, force_n, pos, a_s_per_m, eps, release_time_s))


def sfd_bow_envelope(s: int, t_s, vel_mps=None, force_n=None, pos=None) -> None:
    """Breakpoint envelopes of the bow velocity, force and position (None:
    that control stays at its sfd_excite_bow value)."""
    t, v, f, x = _env_arrays(t_s, vel_mps, force_n, pos)
    _check(lib().sfd_bow_envelope(s, len(t), _dptr(t), _dptr(v), _dptr(f), _dptr(x)))


def sfd_set_modulation(s: int, kind: int, rate_hz: float = 0.0, depth: float = 0.0, phase_rad: float = 0.0,
                       duration_s: float = 0.0) -> None:
    _check(lib().sfd_set_modulation(s, kind, rate_hz, depth, phase_rad, duration_s))


def sfd_modulation_peak(kind: int, depth: float) -> float:
    """Grid-sizing ratio (largest gamma^n / gamma) of an f0 modulation."""
    r = ctypes.c_double()
    _check(lib().sfd_modulation_peak(kind, depth, ctypes.byref(r)))
    return r.value


def sfd_synthesize(s: int, n_samples: int, out=None, allow_noconv: bool = False):
    """Next n_samples samples.  `out` may be None (a NumPy array is returned),
    a float32 NumPy array (host) or a CUDA float32 torch tensor (device)."""
    allow = (SFD_ENOCONV,) if allow_noconv else ()
    if out is None:
        out = np.zeros(n_samples, dtype=np.float32)
    if isinstance(out, np.ndarray):
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size >= n_samples
        _check(lib().sfd_synthesize(s, n_samples, out.ctypes.data, 0), allow)
    else:
        assert out.is_cuda and out.dtype.is_floating_point and out.element_size() == 4 and out.is_contiguous()
        _check(lib().sfd_synthesize(s, n_samples, out.data_ptr(), 1), allow)
    return out


def sfd_string_position(s: int) -> tuple[int, int]:
    n, j = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sfd_string_position(s, ctypes.byref(n), ctypes.byref(j)))
    return n.value, j.value


def sfd_string_state(s: int):
    nt, nl, _, _ = sfd_string_info(s)
    up = np.zeros(nt - 1, np.float32); u = np.zeros(nt - 1, np.float32)
    zp = np.zeros(max(nl - 1, 1), np.float32); z = np.zeros(max(nl - 1, 1), np.float32)
    _check(lib().sfd_string_state(s, up.ctypes.data, u.ctypes.data, zp.ctypes.data, z.ctypes.data))
    return up, u, zp[: nl - 1], z[: nl - 1]


def sfd_string_delta_state(s: int):
    """(u^n, D, z^n, Dz) as the kernel keeps them (FP32, normalised)."""
    nt, nl, _, _ = sfd_string_info(s)
    u = np.zeros(nt - 1, np.float32); du = np.zeros(nt - 1, np.float32)
    z = np.zeros(max(nl - 1, 1), np.float32); dz = np.zeros(max(nl - 1, 1), np.float32)
    _check(lib().sfd_string_delta_state(s, u.ctypes.data, du.ctypes.data, z.ctypes.data, dz.ctypes.data))
    return u, du, z[: nl - 1], dz[: nl - 1]


def sfd_string_hammer(s: int) -> tuple[float, float]:
    """Hammer position u_H / L at levels n-1 and n."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().sfd_string_hammer(s, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def sfd_string_save(s: int) -> bytes:
    """Checkpoint of a string (state, parameters and set-up calls)."""
    n = ctypes.c_size_t()
    _check(lib().sfd_string_save(s, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().sfd_string_save(s, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def sfd_string_load(ctx: int, blob: bytes) -> int:
    """A new string in ctx that continues the checkpointed one."""
    h = ctypes.c_void_p()
    _check(lib().sfd_string_load(ctx, blob, len(blob), ctypes.byref(h)))
    return h.value


def sfd_string_stats(s: int) -> tuple[int, int, int]:
    """(status, max sweeps, total sweeps) of the coupled solve."""
    st, mx, tot = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().sfd_string_stats(s, ctypes.byref(st), ctypes.byref(mx), ctypes.byref(tot)))
    return st.value, mx.value, tot.value


def sfd_string_destroy(s: int) -> None:
    _check(lib().sfd_string_destroy(s))


def sfd_batch_create(ctx: int, strings) -> int:
    arr = (ctypes.c_void_p * len(strings))(*strings)
    h = ctypes.c_void_p()
    _check(lib().sfd_batch_create(ctx, len(strings), arr, ctypes.byref(h)))
    return h.value


def sfd_batch_synthesize(b: int, n_samples, out_device, out_offsets, per_string_status: bool = False,
                         allow_noconv: bool = False):
    """Device output (CUDA torch tensor or raw pointer); asynchronous on the
    context's stream unless per_string_status is requested."""
    ns = np.ascontiguousarray(n_samples, dtype=np.int64)
    offs = np.ascontiguousarray(out_offsets, dtype=np.int64)
    ptr = out_device if isinstance(out_device, int) else out_device.data_ptr()
    st = np.zeros(len(ns), dtype=np.int32) if per_string_status else None
    stp = st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if st is not None else None
    _check(lib().sfd_batch_synthesize(b, _i64p(ns), ptr, _i64p(offs), stp))
    if st is not None:
        bad = [int(x) for x in st if x != SFD_OK and not (allow_noconv and x == SFD_ENOCONV)]
        if bad:
            raise SfdError(bad[0], f"{len(bad)} string(s) reported {STATUS_NAMES.get(bad[0])}")
    return st


def sfd_batch_synthesize_host(b: int, n_samples, out_offsets=None, allow_noconv: bool = False,
                              check: bool = True):
    """Host output: (list of per-string sample arrays, per-string status).
    With check=False a string's failure is reported in the status only."""
    ns = np.ascontiguousarray(n_samples, dtype=np.int64)
    if out_offsets is None:
        offs = np.zeros(len(ns), dtype=np.int64)
        offs[1:] = np.cumsum(ns)[:-1]
    else:
        offs = np.ascontiguousarray(out_offsets, dtype=np.int64)
    total = int((offs + ns).max()) if len(ns) else 0
    out = np.zeros(max(total, 1), dtype=np.float32)
    st = np.zeros(len(ns), dtype=np.int32)
    _check(lib().sfd_batch_synthesize_host(b, _i64p(ns), out.ctypes.data, _i64p(offs),
                                           st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    bad = [int(x) for x in st if x != SFD_OK and not (allow_noconv and x == SFD_ENOCONV)]
    if bad and check:
        raise SfdError(bad[0], f"{len(bad)} string(s) reported {STATUS_NAMES.get(bad[0])}")
    return [out[o:o + n] for o, n in zip(offs, ns)], st


def sfd_batch_set_warps_per_cta(b: int, wpc: int) -> None:
    _check(lib().sfd_batch_set_warps_per_cta(b, wpc))


def sfd_batch_autotune(b: int, probe_samples: int) -> int:
    best = ctypes.c_int32()
    _check(lib().sfd_batch_autotune(b, probe_samples, ctypes.byref(best)))
    return best.value


def sfd_batch_prepare(b: int, n_samples, out_device, out_offsets) -> None:
    ns = np.ascontiguousarray(n_samples, dtype=np.int64)
    offs = np.ascontiguousarray(out_offsets, dtype=np.int64)
    ptr = out_device if isinstance(out_device, int) else out_device.data_ptr()
    _check(lib().sfd_batch_prepare(b, _i64p(ns), ptr, _i64p(offs)))


def sfd_batch_launch(b: int) -> None:
    _check(lib().sfd_batch_launch(b))


def sfd_batch_destroy(b: int) -> None:
    _check(lib().sfd_batch_destroy(b))


def sfd_last_launch_count(ctx: int) -> int:
    return lib().sfd_last_launch_count(ctx)


def sfd_ctx_transfer_bytes(ctx: int) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().sfd_ctx_transfer_bytes(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


SFD_KERNEL_CLASSES = 6


def sfd_ctx_set_timing(ctx: int, enable: bool) -> None:
    _check(lib().sfd_ctx_set_timing(ctx, 1 if enable else 0))


def sfd_ctx_set_warp_pairs(ctx: int, enable: bool) -> None:
    _check(lib().sfd_ctx_set_warp_pairs(ctx, 1 if enable else 0))


def sfd_ctx_set_sweep_cap(ctx: int, cap: int) -> None:
    _check(lib().sfd_ctx_set_sweep_cap(ctx, cap))


def sfd_ctx_kernel_times(ctx: int):
    """(ms per class, jobs per class) of the last launch (timing enabled)."""
    ms = (ctypes.c_float * SFD_KERNEL_CLASSES)()
    nj = (ctypes.c_int32 * SFD_KERNEL_CLASSES)()
    _check(lib().sfd_ctx_kernel_times(ctx, ms, nj))
    return list(ms), list(nj)


def sfd_string_kernel_class(s: int) -> int:
    c = ctypes.c_int32()
    _check(lib().sfd_string_kernel_class(s, ctypes.byref(c)))
    return c.value


def sfd_measure_peaks(device: int = 0) -> dict:
    """Measured FP32 / FP64 FMA throughput [TFLOP/s] and shared-memory load
    bandwidth [TB/s] of the device (the roofline denominators)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sfd_measure_peaks(device, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"fp32_tflops": a.value, "fp64_tflops": b.value, "smem_tbs": c.value}


def sfd_last_error() -> str:
    return lib().sfd_last_error().decode(errors="replace")


def excitation_from_dict(ex: dict) -> sfd_excitation:
    if ex.get("envelope"):
        raise ValueError("bow envelopes apply to strings and server requests, not to tapes")
    e = sfd_excitation()
    e.pos = ex["pos"]
    if ex["kind"] == "pluck":
        e.kind, e.amp_m = 0, ex["amp"]
    elif ex["kind"] == "hammer":
        e.kind, e.mass_kg, e.vel_mps = 1, ex["mass"], ex["vel"]
        e.omega_h, e.alpha_h = ex.get("omega", 3000.0), ex.get("alpha", 2.5)
    else:
        e.kind, e.vel_mps, e.force_n = 2, ex["vel"], ex["force"]
        e.a_s_per_m, e.eps, e.release_time_s = ex.get("a", 100.0), ex.get("eps", 0.1), ex.get("release", -1.0)
    return e


def sfd_synthesize_noalloc(device: int, stream, params: sfd_string_params, exc: sfd_excitation,
                           n_samples: int, out_device) -> None:
    """First n_samples samples of one string into device memory, with no
    device allocation (scratch in the library's static device array)."""
    ptr = out_device if isinstance(out_device, int) else out_device.data_ptr()
    _check(lib().sfd_synthesize_noalloc(device, stream, ctypes.byref(params), ctypes.byref(exc), n_samples, ptr))


# ------------------------------------------------------------ serving

def sfd_server_create(ctx: int, chunk_samples: int = 1024, max_live: int = 4096) -> int:
    out = ctypes.c_void_p()
    _check(lib().sfd_server_create(ctx, chunk_samples, max_live, ctypes.byref(out)))
    return out.value


def _env_arrays(t_s, vel_mps, force_n, pos):
    """Breakpoint arrays as contiguous float64 (None for an absent control)."""
    t = np.ascontiguousarray(t_s, dtype=np.float64)
    out = []
    for a in (vel_mps, force_n, pos):
        if a is not None:
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.shape != t.shape:
                raise ValueError("every envelope array needs one value per breakpoint time")
        out.append(a)
    return [t] + out


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def sfd_server_submit(sv: int, req: sfd_request) -> None:
    """Queue a request; one made by request_from_dict from a bowed string
    with an "envelope" carries it (sfd_server_submit_bow_envelope)."""
    env = getattr(req, "bow_envelope", None)
    if env is None:
        _check(lib().sfd_server_submit(sv, ctypes.byref(req)))
        return
    t, v, f, x = _env_arrays(env["t"], env.get("vel"), env.get("force"), env.get("pos"))
    _check(lib().sfd_server_submit_bow_envelope(sv, ctypes.byref(req), len(t), _dptr(t), _dptr(v), _dptr(f),
                                                _dptr(x)))


def sfd_server_pump(sv: int, copy: bool = True):
    """One admission + launch + delivery round.  Returns a list of
    (tag, first_sample, samples, last, status, ready_s, arrival_s); samples
    is a numpy copy (copy=True) or the sample count (copy=False)."""
    ptr = ctypes.POINTER(sfd_chunk)()
    n = ctypes.c_int32()
    _check(lib().sfd_server_pump(sv, ctypes.byref(ptr), ctypes.byref(n)))
    res = []
    for i in range(n.value):
        c = ptr[i]
        data = np.ctypeslib.as_array(c.samples, shape=(c.n,)).copy() if copy else c.n
        res.append((c.tag, c.first_sample, data, bool(c.last), c.status, c.ready_s, c.arrival_s))
    return res


def sfd_server_clock(sv: int) -> float:
    return lib().sfd_server_clock(sv)


def sfd_server_stats_get(sv: int) -> sfd_server_stats:
    st = sfd_server_stats()
    _check(lib().sfd_server_stats_get(sv, ctypes.byref(st)))
    return st


def sfd_server_destroy(sv: int) -> None:
    _check(lib().sfd_server_destroy(sv))


# ------------------------------------------------------------ gradients

SFD_GRAD_PARAMS = 5
GRAD_PARAM_NAMES = ("kappa", "alpha", "sigma0", "sigma1", "amplitude")


def modulation_from_dict(mod: dict | None) -> sfd_modulation:
    m = sfd_modulation()
    mod = mod or {"kind": "none"}
    if mod["kind"] == "vibrato":
        m.kind, m.rate_hz, m.depth, m.phase_rad = SFD_MOD_VIBRATO, mod["rate"], mod["depth"], mod.get("phase", 0.0)
    elif mod["kind"] == "gliss":
        m.kind, m.depth, m.duration_s = SFD_MOD_GLISS, mod["depth"], mod["duration"]
    return m


def sfd_tape_create(ctx: int, strings, n_samples: int, checkpoint_every: int = 1024) -> int:
    """Tape of strings (parameter dicts: any excitation, f0 modulation and
    output channel)."""
    n = len(strings)
    params = (sfd_string_params * n)(*[params_from_dict(d) for d in strings])
    excs = (sfd_excitation * n)(*[excitation_from_dict(d["excitation"]) for d in strings])
    mods = (sfd_modulation * n)(*[modulation_from_dict(d.get("modulation")) for d in strings])
    out = ctypes.c_void_p()
    _check(lib().sfd_tape_create(ctx, n, params, excs, mods, n_samples, checkpoint_every, ctypes.byref(out)))
    return out.value


def sfd_tape_forward(tape: int, y_device, allow_noconv: bool = False) -> None:
    ptr = y_device if isinstance(y_device, int) else y_device.data_ptr()
    _check(lib().sfd_tape_forward(tape, ptr), allow=(SFD_ENOCONV,) if allow_noconv else ())


def sfd_tape_backward(tape: int, dy_device, n: int) -> np.ndarray:
    """dJ/d(kappa, alpha, sigma0, sigma1, amplitude) per string, shape (n, 5)."""
    ptr = dy_device if isinstance(dy_device, int) else dy_device.data_ptr()
    g = np.zeros((n, SFD_GRAD_PARAMS), dtype=np.float64)
    _check(lib().sfd_tape_backward(tape, ptr, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return g


def sfd_tape_set_record_forward(tape: int, enable: bool) -> None:
    """Record every level on the forward pass (True) or replay segments (False)."""
    _check(lib().sfd_tape_set_record_forward(tape, 1 if enable else 0))


def sfd_tape_destroy(tape: int) -> None:
    _check(lib().sfd_tape_destroy(tape))


def request_from_dict(d: dict, tag: int, n_samples: int | None = None, arrival_s: float = -1.0) -> sfd_request:
    r = sfd_request()
    r.params = params_from_dict(d)
    ex = dict(d["excitation"])
    env = ex.pop("envelope", None)
    r.exc = excitation_from_dict(ex)
    if env:
        r.bow_envelope = env   # sent by sfd_server_submit
    mod = d.get("modulation", {"kind": "none"})
    if mod.get("kind") == "vibrato":
        r.mod_kind, r.mod_rate_hz, r.mod_depth, r.mod_phase_rad = SFD_MOD_VIBRATO, mod["rate"], mod["depth"], \
            mod.get("phase", 0.0)
    elif mod.get("kind") == "gliss":
        r.mod_kind, r.mod_depth, r.mod_duration_s = SFD_MOD_GLISS, mod["depth"], mod["duration"]
    r.n_samples = d["n_samples"] if n_samples is None else n_samples
    r.arrival_s = arrival_s
    r.tag = tag
    return r


# ------------------------------------------------------ dict marshalling

def params_from_dict(d: dict) -> sfd_string_params:
    p = sfd_params_default()
    if d.get("gamma"):
        p.gamma = d["gamma"]
    else:
        p.f0 = d["f0"]
    p.kappa, p.alpha, p.sigma0, p.sigma1 = d["kappa"], d["alpha"], d["sigma0"], d["sigma1"]
    p.length_m = d.get("length", 1.0)
    p.fs = d.get("fs", 48000.0)
    p.linear_density = d.get("rho_a", 5e-3)
    p.theta = d.get("theta", 0.5 * (1 + 4 / math.pi ** 2))
    p.boundary = d.get("boundary", 0)
    p.grid_rule = d.get("grid_rule", 0)
    p.pickup_pos = d.get("pickup", 0.7)
    p.output = OUTPUTS[d.get("output", "transverse")]
    mod = d.get("modulation", {"kind": "none"})
    kind = MOD_KINDS[mod.get("kind", "none")]
    p.f0_max_ratio = d.get("gamma_max_ratio", sfd_modulation_peak(kind, mod.get("depth", 0.0)))
    return p


def string_from_dict(ctx: int, d: dict) -> int:
    s = sfd_string_create(ctx, params_from_dict(d))
    try:
        ex = d["excitation"]
        if ex["kind"] == "pluck":
            sfd_excite_pluck(s, ex["amp"], ex["pos"])
        elif ex["kind"] == "hammer":
            sfd_excite_hammer(s, ex["mass"], ex["vel"], ex["pos"], ex.get("omega", 3000.0), ex.get("alpha", 2.5))
        else:
            sfd_excite_bow(s, ex["vel"], ex["force"], ex["pos"], ex.get("a", 100.0), ex.get("eps", 0.1),
                           ex.get("release", -1.0))
            env = ex.get("envelope")
            if env:   # breakpoint times [s]; an absent key keeps that control constant
                sfd_bow_envelope(s, env["t"], env.get("vel"), env.get("force"), env.get("pos"))
        mod = d.get("modulation", {"kind": "none"})
        if mod.get("kind") == "vibrato":
            sfd_set_modulation(s, SFD_MOD_VIBRATO, mod["rate"], mod["depth"], mod.get("phase", 0.0), 0.0)
        elif mod.get("kind") == "gliss":
            sfd_set_modulation(s, SFD_MOD_GLISS, 0.0, mod["depth"], 0.0, mod["duration"])
    except Exception:
        sfd_string_destroy(s)
        raise
    return s
