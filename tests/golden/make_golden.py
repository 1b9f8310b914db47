"""Writes the stored expected values under tests/golden/ from the oracle only.

Run:  python tests/golden/make_golden.py
Each file states what it holds and which passage of the paper it follows.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import element  # noqa: E402


def write_fraction_matrix(path, Kq, header):
    with open(path, "w") as f:
        for h in header:
            f.write("# " + h + "\n")
        for row in Kq:
            f.write(" ".join(str(v) for v in row) + "\n")


def main():
    write_fraction_matrix(
        os.path.join(HERE, "k0_q4_nu0.3.txt"), element.k0_q4_exact(),
        ["Exact unit-square Q4 plane-stress stiffness K0, E = 1, nu = 3/10 (rational).",
         "Energy density of Section 2.1 (Eq. str_energy) with plane-stress lambda;",
         "node order (0,0),(1,0),(1,1),(0,1); DOF order node-major, component-minor."])
    write_fraction_matrix(
        os.path.join(HERE, "k0_h8_nu0.3.txt"), element.k0_h8_exact(),
        ["Exact unit-cube H8 isotropic stiffness K0, E = 1, nu = 3/10 (rational).",
         "Energy density of Section 2.1 (Eq. str_energy); node order: the Q4 order at",
         "z = 0 then at z = 1; DOF order node-major, component-minor."])


if __name__ == "__main__":
    main()
