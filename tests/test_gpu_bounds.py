"""The bounds-checked build (-DTEM_CHECK_BOUNDS): the hot kernels check every global index and the
start of every TMA box before the access and record a failing check instead of faulting.  The
solver reports a recorded failure as an error.  Here it runs forward models on a grid that takes
the TMA stencil (even nx) and one that takes the cp.async stencil (odd nx), in FP64 and mixed
precision, in a process that loads the checked library: every call must finish with TEM_OK and
agree with the normal build to the parity tolerances (the checks change no arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_11657_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [((20, 14, 18), "mixed"), ((20, 14, 18), "fp64"), ((17, 12, 15), "mixed"), ((17, 12, 15), "fp64")]

SCRIPT = """
import json, sys
sys.path.insert(0, {root!r})
from paper_2506_11657_gb300 import tem, workloads as W
out = []
for (nx, ny, nz), prec in {cases!r}:
    m = W.uniform_model(nx, 10.0, nz // 3, 0.02, 40.0, 1e-5, 1e-3, 9, 10, ny=ny, nz=nz)
    sh, c, _ = tem.poles_residues(m.t, m.degree)
    g = tem.Grid(m.hx, m.hy, m.hz, m.origin, m.sigma)
    r = tem.forward(g, m.loop_xy, m.z_loop, m.rx, sh, c, tem.default_options(precision=prec, tol=1e-13))
    out.append([int(r.status), r.d.tolist()])
print(json.dumps(out))
"""


def _run(lib_path):
    env = dict(os.environ)
    env["TEM_LIB"] = lib_path
    p = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, cases=CASES)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_runs_clean_and_agrees():
    from paper_2506_11657_gb300 import build as B
    checked = B.build_checked()
    normal = os.path.join(ROOT, "paper_2506_11657_gb300", "libtem.so")
    a, b = _run(checked), _run(normal)
    for ((dims, prec), (sa, da), (sb, db)) in zip(CASES, a, b):
        assert sa == 0 and sb == 0, (dims, prec, sa, sb)
        da, db = np.asarray(da), np.asarray(db)
        rel = np.max(np.abs(da - db) / np.abs(db))
        print(f"checked vs normal build {dims} {prec}: max rel diff {rel:.2e}")
        assert rel <= (1e-9 if prec == "fp64" else 1e-5), (dims, prec, rel)
