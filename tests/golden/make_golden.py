"""Write the stored expected values under tests/golden/ by calling only the
CPU oracle (oracle/). Run: python tests/golden/make_golden.py

box33_fp64_J.txt: converged J of the 33^3 periodic box (vertical chi
profile, B = 1, eps = 1e-2, 8 x 16 angles, linear interpolation, I_top = 0,
I_bottom = B), iterated with the ALI (Eq. alo) to max rel dJ < 1e-13. The
medium is horizontally uniform, so J depends on z only: one value per layer.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2102_01734_gb300 import inputs  # noqa: E402


def box33():
    chi, eps, B, bc = inputs.cartesian_config(33, 1e-2)
    t = time.time()
    J, it, hist, _ = oracle.ali_solve(chi, eps, B, 8, 16, False, bc, tol=1e-13, max_iter=1000)
    assert it > 0, "oracle ALI did not converge"
    prof = J.reshape(33, -1)
    spread = float(np.max(np.ptp(prof, axis=1) / prof.mean(axis=1)))
    path = os.path.join(HERE, "box33_fp64_J.txt")
    with open(path, "w") as f:
        f.write("# converged J per layer z = 0..32 (bottom to top) of the 33^3 box,\n")
        f.write("# eps=1e-2, B=1, chi=10^(-4+6(32-z)/32), 8x16 angles, linear, I_top=0,\n")
        f.write(f"# I_bottom=B; oracle ALI to rel dJ<1e-13 in {it} iterations "
                f"({time.time() - t:.0f} s); horizontal spread {spread:.1e}\n")
        for z in range(33):
            f.write(f"{prof[z].mean():.17e}\n")
    print(path, it)


if __name__ == "__main__":
    box33()
