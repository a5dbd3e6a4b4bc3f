"""Writes the stored oracle fixtures under tests/golden/ (calls only the oracle
and the seeded input generator).  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import bse_oracle as O  # noqa: E402
from paper_1601_07728_gb300 import synth as S  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    s = S.make_system("k_edge_small")
    b = S.make_start_vectors(s, 1)[0]
    for reorth in (True, False):
        a, bb, nd, brk = O.haydock(lambda v: O.apply_h(s, v), b, 100, reorth=reorth)
        name = "k_edge_small_haydock_%s.txt" % ("reorth" if reorth else "plain")
        with open(os.path.join(HERE, name), "w") as f:
            f.write("# Haydock coefficients (Sec. 3.2, Eq. 9) of the FP64 oracle on the 1s-edge\n")
            f.write("# workload (1 core state, 2^3 k, 16 bands, 8^3 grid, erf W eps=5, cell 7.4 bohr),\n")
            f.write("# seeded start vector 0, 100 steps, reorth=%d.  Columns: i a_i b_i (b_0 = |b|).\n" % reorth)
            f.write("# steps_done=%d breakdown=%d\n" % (nd, int(brk)))
            for i in range(nd + 1):
                ai = a[i] if i < nd else float("nan")
                f.write("%d %.17e %.17e\n" % (i, ai, bb[i]))


if __name__ == "__main__" and len(sys.argv) == 1:
    main()


def l23_spectrum(n_steps=200):
    """Oracle Haydock run (plain Lanczos, like the benchmark) on the full
    L2,3-edge workload; stores a_i, b_i and the spectrum on the 2000-point grid."""
    s = S.make_system("l23_multiplet")
    b = S.make_start_vectors(s, 1)[0]
    a, bb, nd, brk = O.haydock(lambda v: O.apply_h(s, v), b, n_steps)
    sig = O.cf_spectrum(a, bb, S.omega_grid(), 0.5)
    np.savez_compressed(os.path.join(HERE, "l23_multiplet_haydock200.npz"), a=a, b=bb, sigma=sig,
                        omega=S.omega_grid(), steps=nd)


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "l23":
    l23_spectrum()
