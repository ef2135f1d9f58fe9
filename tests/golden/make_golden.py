"""Writes tests/golden/paper_systems_pairs.txt using only the CPU oracle.

Systems are the paper's molecular shapes (spin orbitals N, electrons N_e): N2, PH3 and
LiCl of Table I, and Fe2S2, H50 and C6H6 of Sec. IV-B (C6H6's electron count is not
given there; half filling is used).  For each, the oracle enumerates every S_z-conserving
single and double excitation of the closed-shell Aufbau determinant and reports the
count (the size of the connected set entering Eq. 5 for one sample).

Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

SYSTEMS = [
    ("N2", 20, 14, "Table I"),
    ("PH3", 24, 18, "Table I"),
    ("LiCl", 28, 20, "Table I"),
    ("Fe2S2", 40, 30, "Sec. IV-B"),
    ("H50", 100, 50, "Sec. IV-B"),
    ("C6H6", 120, 60, "Sec. IV-B (electrons: half filling, not stated)"),
]


def main():
    lines = ["# name n_orb n_elec pairs_per_determinant  (source of the shape)"]
    for name, n, ne, src in SYSTEMS:
        K = n // 2
        h = np.zeros((K, K))
        eri = np.zeros((K, K, K, K))
        x = np.zeros((1, 2), dtype=np.uint64)
        for k in range(ne // 2):
            for s in (0, 1):
                b = 2 * k + s
                x[0, b >> 6] |= np.uint64(1) << np.uint64(b & 63)
        _, det = oracle.eloc(h, eri, 0.0, n, x, np.ones(1, complex), details=True)
        lines.append(f"{name} {n} {ne} {int(det['pairs'][0])}  ({src})")
    with open(os.path.join(HERE, "paper_systems_pairs.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
