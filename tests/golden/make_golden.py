"""Writes tests/golden/tiny_spectrum.txt: the five lowest eigenvalues of the
Hamiltonian of the tiny workload (16 spin orbitals, 4 alpha + 4 beta, all 4900
determinants, integrals from seed 0), built by term-by-term second
quantization (oracle/fci_brute.c).  The paper prints no worked example, so this
is a regression anchor computed by the oracle only.

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2604_15768_gb300 import synth  # noqa: E402


def main():
    s = synth.config_system("tiny")
    H, outside = O.brute_hamiltonian(s.norb, s.h1, s.h2, s.dets)
    assert outside == 0
    w = np.linalg.eigvalsh(H)[:5]
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_spectrum.txt")
    with open(path, "w") as f:
        f.write("# lowest eigenvalues, tiny workload (16 spin orbitals, 4a+4b, seed 0), "
                "brute-force second-quantized H\n")
        for x in w:
            f.write(f"{x:.15e}\n")
    print(path)


if __name__ == "__main__":
    main()
