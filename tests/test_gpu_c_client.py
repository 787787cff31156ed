"""The C-ABI used from plain C: tests/c_client.c, compiled with the host C
compiler against include/sfd.h and linked to libsfd.so, synthesizes three
strings alone (two calls each) and as one batch; its samples equal the
Python binding's bit for bit."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2311_18505_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
N = 4000


def test_c_client_matches_the_binding(tmp_path):
    from paper_2311_18505_gb300 import build as B
    lib = B.build()
    from paper_2311_18505_gb300 import sfd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    exe = tmp_path / "c_client"
    subprocess.run([cc, "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "c_client.c"),
                    "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    out = tmp_path / "samples.f32"
    r = subprocess.run([str(exe), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    y = np.fromfile(out, dtype=np.float32).reshape(2, 3, N)
    assert np.array_equal(y[0], y[1])          # alone == in the batch
    ctx = sfd.sfd_ctx_create(0, None, 64 << 20)
    try:
        exc = [{"kind": "pluck", "amp": 1e-3, "pos": 0.3},
               {"kind": "hammer", "mass": 6e-3, "vel": 3.0, "pos": 0.31, "omega": 3000.0, "alpha": 2.5},
               {"kind": "bow", "vel": 0.2, "force": 1.0, "pos": 0.17, "a": 100.0, "eps": 0.1, "release": -1.0}]
        for w in range(3):
            d = W.make(f0=110.0 + 40.0 * w, alpha=3.0, excitation=exc[w], n_samples=N,
                       output="longitudinal" if w == 2 else "transverse")
            s = sfd.string_from_dict(ctx, d)
            try:
                assert np.array_equal(sfd.sfd_synthesize(s, N), y[0, w]), w
            finally:
                sfd.sfd_string_destroy(s)
    finally:
        sfd.sfd_ctx_destroy(ctx)
