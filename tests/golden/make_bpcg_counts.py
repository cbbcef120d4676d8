"""Writes tests/golden/bpcg_iterations_annulus6x6_p3_n64.txt: the oracle's
FP64 MG-MG-S (Bramble-Pasciak CG on Eq. 2, three V-cycles in the K~
preconditioner, Sec. 3.3 and 4) and MG-MG (dual PCG on Eq. 4) iteration
counts on the full-size 6x6 quarter annulus, p = 3, 64 x 64 elements per
patch.  Calls only oracle/ and the input description; minutes of CPU time.

    python tests/golden/make_bpcg_counts.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ietidp as O  # noqa: E402
from oracle import saddle  # noqa: E402
from paper_1705_04531_gb300 import workloads as W  # noqa: E402


def main():
    dom = W.annulus_6x6(64, 3)
    t0 = time.time()
    orc = O.IETIDP(dom, O.Options(mode="mg"))
    _, ost = saddle.bpcg(orc)
    orc.stats = O.Stats()
    orc.solve()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bpcg_iterations_annulus6x6_p3_n64.txt")
    with open(out, "w") as fh:
        fh.write("# Oracle (oracle/saddle.py, oracle/ietidp.py), FP64, on the quarter annulus 6x6,\n"
                 "# p = 3, 64 x 64 elements per patch, tolerance 1e-10; written by\n"
                 "# tests/golden/make_bpcg_counts.py (oracle only).\n"
                 "# method iterations\n")
        fh.write(f"mg_mg_s_bpcg {ost['iterations']}\n")
        fh.write(f"mg_mg_dual_pcg {orc.stats.outer_it}\n")
    print(out, ost["iterations"], orc.stats.outer_it, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
