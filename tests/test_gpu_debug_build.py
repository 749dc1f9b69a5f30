"""The debug build (libsph_debug.so, -DSPH_DEBUG): its index checks guard the
neighbour walks (cell range, list entries, cell offsets), the reorder and the
wall gather, and record SPH_E_INDEX instead of making the access.  In a child
process (so that the debug library is the one loaded) the parity workloads
run under the checks: no check fails, and the results meet the oracle at the
parity bars.  The checks replace a memory checker, which this pool does not
offer; a failing check is not provoked here, since the release path of the
same input would read out of bounds."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2603_11868_gb300 import build, cases
from paper_2603_11868_gb300 import sph as S
S.load(build.build(debug=True))
from oracle import oracle as O

def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)

def against_oracle(case, precision, steps, tol):
    s = S.Solver(case, precision=precision)
    s.step(steps)
    got = s.fields("pos", "rho")
    s.synchronize()
    s.close()
    o = O.Oracle.from_case(case)
    o.step(steps)
    assert np.abs(got["pos"] - o.field(O.POS)).max() <= tol * case.dp, case.name
    assert rel(got["rho"], o.field(O.RHO)) <= tol, case.name

against_oracle(cases.dam_break_2d(), "fp64", 40, 1e-8)
against_oracle(cases.dam_break_2d(), "mixed", 40, 1e-4)
against_oracle(cases.dam_break_3d(dp=0.02), "mixed", 25, 1e-4)
against_oracle(cases.sliding_lid_channel_2d(), "mixed", 60, 1e-4)
against_oracle(cases.piston_channel_2d(V=2.0), "fp64", 130, 1e-8)

tanks = [cases.batched_tank(n, dp=0.02, seed=70 + k) for k, n in enumerate((400, 1500, 900))]
b = S.Batch(tanks, precision="mixed")
b.step(30)
f = b.fields("pos", "rho")
b.synchronize()
b.close()
for t, c in enumerate(tanks):
    s = S.Solver(c, precision="mixed")
    s.step(30)
    want = s.fields("pos", "rho")
    s.close()
    sl = slice(int(b.offsets[t]), int(b.offsets[t + 1]))
    assert np.array_equal(f["pos"][sl], want["pos"]) and np.array_equal(f["rho"][sl], want["rho"])

c = cases.dam_break_2d()
a = S.Solver(c, precision="mixed")
a.step(20)
buf = a.checkpoint()
a.close()
r = S.Solver(c, precision="mixed")
r.restore(buf)
r.step(10)
r.synchronize()
r.close()
print("debug build ok")
'''


def test_debug_build_runs_clean():
    code = SCRIPT.replace("ROOT", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=1500, cwd=ROOT)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "debug build ok" in r.stdout
