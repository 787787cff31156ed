"""Host-side checks of the C-ABI library (no GPU compute): it builds for
sm_103a, loads, exports every function include/sfd.h declares, and reports
a CUDA error (rather than falling back to the CPU) when no GPU is present."""

import ctypes
import os
import re

import pytest

import torch

from paper_2311_18505_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sfd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(sfd_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sfd_ctx_create", "sfd_string_create", "sfd_excite_pluck", "sfd_excite_hammer",
                 "sfd_excite_bow", "sfd_synthesize", "sfd_string_destroy", "sfd_batch_create",
                 "sfd_batch_synthesize", "sfd_batch_destroy", "sfd_last_error"):
        assert must in names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    L = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in sfd.h but not exported"


def test_binding_covers_every_declared_function():
    """The Python binding gives every function of the header a signature
    (argtypes stay None for a function the binding never declared)."""
    B.build()
    from paper_2311_18505_gb300 import sfd
    L = sfd.lib()
    missing = [n for n in declared_functions() if getattr(L, n).argtypes is None]
    assert not missing, f"no binding for {missing}"


def test_binding_loads_and_defaults():
    from paper_2311_18505_gb300 import sfd
    p = sfd.sfd_params_default()
    assert p.f0 == 110.0 and p.fs == 48000.0 and p.pickup_pos == 0.7
    assert abs(p.theta - 0.5 * (1 + 4 / 3.141592653589793 ** 2)) < 1e-15


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_no_gpu_is_an_error_not_a_fallback():
    from paper_2311_18505_gb300 import sfd
    with pytest.raises(sfd.SfdError) as ei:
        sfd.sfd_ctx_create(0, None, 1 << 20)
    assert ei.value.code == sfd.SFD_ECUDA


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    from paper_2311_18505_gb300 import sfd
    monkeypatch.setattr(sfd, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(sfd, "_lib", None)
    with pytest.raises(ImportError):
        sfd.lib()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_18505_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "sfd_oracle" not in txt, f


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes across the boundary has the C layout:
    size and field offsets from a C program compiled against sfd.h."""
    import shutil
    import subprocess
    from paper_2311_18505_gb300 import sfd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [sfd.sfd_string_params, sfd.sfd_excitation, sfd.sfd_request, sfd.sfd_chunk, sfd.sfd_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sfd.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln)}
    for st in structs:
        name = st.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (compiled with the host C compiler; no GPU)."""
    import shutil
    import subprocess
    from paper_2311_18505_gb300 import sfd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"sfd_string_params": sfd.sfd_string_params, "sfd_excitation": sfd.sfd_excitation,
               "sfd_request": sfd.sfd_request, "sfd_chunk": sfd.sfd_chunk,
               "sfd_server_stats": sfd.sfd_server_stats, "sfd_modulation": sfd.sfd_modulation}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sfd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                   text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


def test_host_grid_matches_the_oracle():
    """sfd_grid (host arithmetic, no device) gives the oracle's grid for
    random strings, modulated or not, and refuses invalid parameters."""
    import numpy as np
    import oracle
    from paper_2311_18505_gb300 import sfd
    from paper_2311_18505_gb300 import workloads as W
    rng = np.random.default_rng(3)
    for i in range(200):
        d = W.random_string(rng, f0_lo=30.0, f0_hi=2000.0, seconds=0.01)
        if i % 2:
            d["modulation"] = {"kind": "vibrato", "rate": 6.0, "depth": 30.0, "phase": 0.0}
        assert sfd.sfd_grid(sfd.params_from_dict(d)) == oracle.grid(d)
    p = sfd.params_from_dict(W.make())
    p.alpha = 0.5
    with pytest.raises(sfd.SfdError) as ei:
        sfd.sfd_grid(p)
    assert ei.value.code == sfd.SFD_EINVAL


def test_modulation_peak_matches_the_oracle():
    """The library's grid-sizing ratio of a modulation (host arithmetic)
    equals the oracle's own reading of it, and refuses bad input."""
    import oracle
    from paper_2311_18505_gb300 import sfd
    cases = [("vibrato", 20.0), ("vibrato", -35.0), ("gliss", 1.0), ("gliss", -1.0), ("gliss", 0.37),
             ("none", 0.0)]
    for kind, depth in cases:
        assert sfd.sfd_modulation_peak(sfd.MOD_KINDS[kind], depth) == \
            oracle.gamma_max_ratio({"kind": kind, "depth": depth})
    for kind, depth in ((7, 1.0), (1, float("nan"))):
        with pytest.raises(sfd.SfdError) as ei:
            sfd.sfd_modulation_peak(kind, depth)
        assert ei.value.code == sfd.SFD_EINVAL


def test_lpt_partition():
    """Every string on exactly one rank, the same split however often it is
    computed, and the greedy bound: no rank above the mean load plus the
    largest single cost."""
    from paper_2311_18505_gb300 import partition
    from paper_2311_18505_gb300 import workloads as W
    strings = W.batch_modulated(512, seconds=0.5, seed=3)
    costs = [partition.string_cost(d) for d in strings]
    for world in (1, 2, 3, 8):
        parts = partition.partition_lpt(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(strings)))
        assert parts == partition.partition_lpt(costs, world)
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)
        assert [partition.shard(strings, r, world) for r in range(world)] == parts
    with pytest.raises(ValueError):
        partition.partition_lpt(costs, 0)
