"""Writes the stored expected series under tests/golden/ by running the FP64
oracle (oracle/) on the seeded dam-break inputs.  Calls nothing but oracle/
and the input generators; no value here comes from the CUDA path.

    python tests/golden/make_golden.py dam_break_2d     # 200 steps, seconds
    python tests/golden/make_golden.py dam_break_3d     # 1000 steps, minutes

Each file holds one line per acoustic step: n_ac, t, front, kinetic energy.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_2603_11868_gb300 import cases  # noqa: E402

RUNS = {
    "dam_break_2d": (lambda: cases.dam_break_2d(), 200),
    "dam_break_3d": (lambda: cases.dam_break_3d(), 1000),
}


def run(name: str) -> str:
    make, steps = RUNS[name]
    case = make()
    o = oracle.Oracle.from_case(case)
    lines = ["# oracle FP64 series for %s (n=%d fluid, %d wall): n_ac t front ke"
             % (name, case.n, case.nw)]
    f, k = o.front_ke()
    lines.append("0 %.17g %.17g %.17g" % (0.0, f, k))
    for i in range(steps):
        o.step(1)
        s = o.scalars()
        f, k = o.front_ke()
        lines.append("%d %.17g %.17g %.17g" % (s["n_ac"], s["t"], f, k))
    path = os.path.join(HERE, f"{name}_front_ke.txt")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    return path


if __name__ == "__main__":
    for name in sys.argv[1:] or list(RUNS):
        print(run(name))
