"""Writes plain_2x2x2_chi8.txt: the oracle's energies for one sweep of the
plain-method workload (2x2x2 open lattice, t = m = 1, g^2 = 1 -> g_e^2 = 1,
c_B = 1/2, nu = 10, Q = 0, chi = 8, seed 0, Lanczos tolerance 1e-12), one
line per node update in sweep order.  Calls only oracle/ and the preset
module; run from the repository root:  python tests/golden/make_plain_2x2x2.py"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import model, tree, ttn  # noqa: E402


def main():
    c = workloads.qed_couplings(1.0)
    p = model.Params(2, 2, 2, Q=0, **c)
    s = ttn.TTN(p, 8, 0)
    order = tree.sweep_order(s.nodes)
    energies = s.sweep(tol=1e-12)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plain_2x2x2_chi8.txt")
    with open(out, "w") as f:
        f.write("# Oracle (oracle/ttn.py) sweep of the plain-method workload: 2x2x2 open lattice,\n")
        f.write("# t = m = 1, g^2 = 1 (ge2 = 1, cB = 0.5, nu = 10), Q = 0, chi = 8, seed 0, tol 1e-12.\n")
        f.write("# Written by tests/golden/make_plain_2x2x2.py.  Columns: update index, node, energy.\n")
        for i, (node, e) in enumerate(zip(order, energies)):
            f.write(f"{i} {node} {float(e)!r}\n")


if __name__ == "__main__":
    main()
