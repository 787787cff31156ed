"""FP64 CPU oracle of the nonlinear planar stiff-string scheme (arXiv 2311.18505).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never does.

The numerics live in ``sfd_oracle.c`` (plain C, FP64, one step = assemble the
linearly-implicit system of Eq. 4 / Eqs. 7-9 and solve it exactly).  This
module compiles it with gcc and marshals the parameter dictionaries of
``paper_2311_18505_gb300.workloads`` into the C structure.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfd_oracle.c")
_HDR = os.path.join(_HERE, "sfd_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libsfd_oracle.so")
_OUT_CS = os.path.join(_HERE, "_build", "libsfd_oracle_cs.so")

EXC = {"pluck": 0, "hammer": 1, "bow": 2}
MOD = {"none": 0, "vibrato": 1, "gliss": 2}


class Spec(ctypes.Structure):
    """Mirror of ``sfdo_spec`` (same field order and types)."""

    _fields_ = [
        ("gamma", ctypes.c_double), ("kappa", ctypes.c_double), ("alpha", ctypes.c_double),
        ("sigma0", ctypes.c_double), ("sigma1", ctypes.c_double), ("theta", ctypes.c_double),
        ("fs", ctypes.c_double), ("length", ctypes.c_double), ("rho_a", ctypes.c_double),
        ("boundary", ctypes.c_int32), ("grid_rule", ctypes.c_int32),
        ("n_t_override", ctypes.c_int32), ("n_l_override", ctypes.c_int32),
        ("gamma_max_ratio", ctypes.c_double), ("pickup", ctypes.c_double),
        ("exc_kind", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("pluck_amp", ctypes.c_double), ("pluck_pos", ctypes.c_double),
        ("ham_mass", ctypes.c_double), ("ham_vel", ctypes.c_double), ("ham_pos", ctypes.c_double),
        ("ham_omega", ctypes.c_double), ("ham_alpha", ctypes.c_double),
        ("bow_vel", ctypes.c_double), ("bow_force", ctypes.c_double), ("bow_pos", ctypes.c_double),
        ("bow_a", ctypes.c_double), ("bow_eps", ctypes.c_double), ("bow_release", ctypes.c_double),
        ("mod_kind", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("mod_rate", ctypes.c_double), ("mod_depth", ctypes.c_double),
        ("mod_phase", ctypes.c_double), ("mod_duration", ctypes.c_double),
        ("out_channel", ctypes.c_int32), ("bow_env_n", ctypes.c_int32),
        ("bow_env_t", ctypes.c_double * 16), ("bow_env_v", ctypes.c_double * 16),
        ("bow_env_f", ctypes.c_double * 16), ("bow_env_x", ctypes.c_double * 16),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it also builds on Arm)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def build_cs(force: bool = False) -> str:
    """Compile the same source a second time with a complex scalar
    (-DSFDO_COMPLEX): the complex-step derivative library."""
    os.makedirs(os.path.dirname(_OUT_CS), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OUT_CS) or os.path.getmtime(_OUT_CS) < newest:
        tmp = _OUT_CS + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-DSFDO_COMPLEX",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT_CS)
    return _OUT_CS


_lib = None
_lib_cs = None


def lib_cs():
    global _lib_cs
    if _lib_cs is None:
        L = ctypes.CDLL(build_cs())
        P = ctypes.POINTER
        L.sfdo_cs_run.argtypes = [P(Spec), ctypes.c_int, ctypes.c_double, ctypes.c_int64, P(ctypes.c_double),
                                  P(ctypes.c_double)]
        L.sfdo_cs_run.restype = ctypes.c_int
        _lib_cs = L
    return _lib_cs


GRAD_PARAMS = ("kappa", "alpha", "sigma0", "sigma1", "amplitude")


def complex_step(d: dict, which: int, n: int | None = None, h: float = 1e-30, n_t: int = 0, n_l: int = 0):
    """(y, dy/dp) of one string for parameter GRAD_PARAMS[which] by the
    complex step (exact to rounding on a smooth path).  The grid is held at
    the parameters' own grid (or n_t, n_l)."""
    n = d["n_samples"] if n is None else n
    if not (n_t and n_l):
        n_t, n_l = grid(d)
    sp = spec(d, n_t, n_l)
    y = np.zeros(n)
    dy = np.zeros(n)
    rc = lib_cs().sfdo_cs_run(ctypes.byref(sp), which, h, n, _ptr(y), _ptr(dy))
    if rc != 0:
        raise FloatingPointError(f"complex-step run failed (code {rc})")
    return y, dy


def loss_gradient_cs(d: dict, target: np.ndarray, n: int | None = None) -> np.ndarray:
    """Gradient of J = sum (y - target)^2 with respect to GRAD_PARAMS by the
    complex step, on the string's own grid."""
    g = np.zeros(len(GRAD_PARAMS))
    for w in range(len(GRAD_PARAMS)):
        y, dy = complex_step(d, w, n)
        g[w] = float(np.sum(2.0 * (y - target[: len(y)]) * dy))
    return g


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        L.sfdo_grid.argtypes = [P(Spec), P(ctypes.c_int32), P(ctypes.c_int32)]
        L.sfdo_grid.restype = ctypes.c_int
        L.sfdo_create.argtypes = [P(Spec)]
        L.sfdo_create.restype = ctypes.c_void_p
        L.sfdo_destroy.argtypes = [ctypes.c_void_p]
        L.sfdo_destroy.restype = None
        L.sfdo_run.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_double)]
        L.sfdo_run.restype = ctypes.c_int
        L.sfdo_time_level.argtypes = [ctypes.c_void_p]
        L.sfdo_time_level.restype = ctypes.c_int64
        L.sfdo_get_state.argtypes = [ctypes.c_void_p] + [P(ctypes.c_double)] * 5
        L.sfdo_get_state.restype = ctypes.c_int
        L.sfdo_set_state.argtypes = [ctypes.c_void_p] + [P(ctypes.c_double)] * 4
        L.sfdo_set_state.restype = ctypes.c_int
        L.sfdo_last_residual.argtypes = [ctypes.c_void_p]
        L.sfdo_last_residual.restype = ctypes.c_double
        L.sfdo_run_batch.argtypes = [P(Spec), ctypes.c_int32, P(ctypes.c_int64), P(ctypes.c_int64),
                                     P(ctypes.c_double), ctypes.c_int32]
        L.sfdo_run_batch.restype = ctypes.c_int
        _lib = L
    return _lib


def gamma_max_ratio(mod: dict) -> float:
    """Grid sizing factor for a modulated note: the grid is derived from the
    largest gamma the modulation reaches."""
    kind = mod.get("kind", "none")
    if kind == "vibrato":
        return 2.0 ** (abs(mod["depth"]) / 1200.0)
    if kind == "gliss":
        return 2.0 ** max(0.0, mod["depth"])
    return 1.0


def spec(d: dict, n_t: int = 0, n_l: int = 0) -> Spec:
    """Parameter dictionary -> C structure (SI units at this boundary)."""
    s = Spec()
    s.gamma = d["gamma"] if d.get("gamma") else 2.0 * d["f0"]   # f0 = gamma/2 (Sec. 4.1)
    s.kappa, s.alpha = d["kappa"], d["alpha"]
    s.sigma0, s.sigma1 = d["sigma0"], d["sigma1"]
    s.theta = d.get("theta", 0.5 * (1 + 4 / math.pi ** 2))
    s.fs, s.length, s.rho_a = d["fs"], d.get("length", 1.0), d.get("rho_a", 5e-3)
    s.boundary, s.grid_rule = d.get("boundary", 0), d.get("grid_rule", 0)
    s.n_t_override, s.n_l_override = n_t or d.get("n_t", 0), n_l or d.get("n_l", 0)
    mod = d.get("modulation", {"kind": "none"})
    s.gamma_max_ratio = d.get("gamma_max_ratio", gamma_max_ratio(mod))
    s.pickup = d.get("pickup", 0.7)
    s.out_channel = 1 if d.get("output", "transverse") == "longitudinal" else 0
    ex = d["excitation"]
    s.exc_kind = EXC[ex["kind"]]
    if ex["kind"] == "pluck":
        s.pluck_amp, s.pluck_pos = ex["amp"], ex["pos"]
    elif ex["kind"] == "hammer":
        s.ham_mass, s.ham_vel, s.ham_pos = ex["mass"], ex["vel"], ex["pos"]
        s.ham_omega, s.ham_alpha = ex.get("omega", 3000.0), ex.get("alpha", 2.5)
    else:
        s.bow_vel, s.bow_force, s.bow_pos = ex["vel"], ex["force"], ex["pos"]
        s.bow_a, s.bow_eps = ex.get("a", 100.0), ex.get("eps", 0.1)
        s.bow_release = ex.get("release", -1.0)
        env = ex.get("envelope")
        if env:   # time-varying controls: breakpoint times and values (constant where a key is absent)
            t = list(env["t"])
            s.bow_env_n = len(t)
            for j, tj in enumerate(t):
                s.bow_env_t[j] = tj
                s.bow_env_v[j] = env["vel"][j] if "vel" in env else ex["vel"]
                s.bow_env_f[j] = env["force"][j] if "force" in env else ex["force"]
                s.bow_env_x[j] = env["pos"][j] if "pos" in env else ex["pos"]
    s.mod_kind = MOD[mod.get("kind", "none")]
    if s.mod_kind == 1:
        s.mod_rate, s.mod_depth, s.mod_phase = mod["rate"], mod["depth"], mod.get("phase", 0.0)
    elif s.mod_kind == 2:
        s.mod_depth, s.mod_duration = mod["depth"], mod["duration"]
    return s


def grid(d: dict) -> tuple[int, int]:
    nt, nl = ctypes.c_int32(), ctypes.c_int32()
    s = spec(d)
    rc = lib().sfdo_grid(ctypes.byref(s), ctypes.byref(nt), ctypes.byref(nl))
    if rc != 0:
        raise ValueError(f"invalid string parameters (code {rc})")
    return nt.value, nl.value


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleString:
    """One string advanced by the FP64 oracle, sample by sample."""

    def __init__(self, d: dict, n_t: int = 0, n_l: int = 0):
        self._spec = spec(d, n_t, n_l)
        ntc, nlc = ctypes.c_int32(), ctypes.c_int32()
        if lib().sfdo_grid(ctypes.byref(self._spec), ctypes.byref(ntc), ctypes.byref(nlc)) != 0:
            raise ValueError("invalid string parameters")
        self.n_t, self.n_l = ntc.value, nlc.value
        self._h = lib().sfdo_create(ctypes.byref(self._spec))
        if not self._h:
            raise ValueError("invalid string parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().sfdo_destroy(h)
            self._h = None

    @property
    def n_u(self) -> int:
        return self.n_t - 1

    @property
    def n_z(self) -> int:
        return max(self.n_l - 1, 0)

    def run(self, n: int) -> np.ndarray:
        y = np.zeros(n, dtype=np.float64)
        rc = lib().sfdo_run(self._h, n, _ptr(y))
        if rc != 0:
            raise FloatingPointError(f"oracle step failed (code {rc})")
        return y

    @property
    def time_level(self) -> int:
        return lib().sfdo_time_level(self._h)

    def state(self):
        """(u^{n-1}, u^n, z^{n-1}, z^n, exc) with exc = [u_H^{n-1}, u_H^n,
        power, G, v_rel, force] of the last step (normalised units)."""
        up = np.zeros(self.n_u); u = np.zeros(self.n_u)
        zp = np.zeros(max(self.n_z, 1)); z = np.zeros(max(self.n_z, 1))
        ex = np.zeros(6)
        lib().sfdo_get_state(self._h, _ptr(up), _ptr(u), _ptr(zp), _ptr(z), _ptr(ex))
        return up, u, zp[: self.n_z], z[: self.n_z], ex

    def set_state(self, up, u, zp=None, zn=None):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                for a in (up, u, zp, zn)]
        ptrs = [_ptr(a) if a is not None else None for a in arrs]
        lib().sfdo_set_state(self._h, *ptrs)

    def residual(self) -> float:
        return lib().sfdo_last_residual(self._h)


def run(d: dict, n: int | None = None, **kw) -> np.ndarray:
    """Output samples y^0 .. y^{n-1} of one string (n defaults to d["n_samples"])."""
    return OracleString(d, **kw).run(d["n_samples"] if n is None else n)


def run_batch(strings: list[dict], n_samples=None, threads: int = 0):
    """Run independent strings with OpenMP; returns (list of outputs, threads used)."""
    ns = np.array([s["n_samples"] if n_samples is None else
                   (n_samples[i] if hasattr(n_samples, "__len__") else n_samples)
                   for i, s in enumerate(strings)], dtype=np.int64)
    offs = np.zeros(len(strings), dtype=np.int64)
    offs[1:] = np.cumsum(ns)[:-1]
    y = np.zeros(int(ns.sum()), dtype=np.float64)
    specs = (Spec * len(strings))(*[spec(s) for s in strings])
    used = lib().sfdo_run_batch(specs, len(strings), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(y), threads)
    if used < 0:
        raise RuntimeError(f"oracle batch failed (code {used})")
    return [y[o:o + n] for o, n in zip(offs, ns)], used
