"""Writes the stored expected values under tests/golden/ from the oracle only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import pw_oracle as O  # noqa: E402


def dense_lowest(species, n, ecut, seed, k):
    ci = synth.cell_inputs(species, n, seed)
    cell = O.make_cell(ci["L"], ci["tau"], ci["depth"], ci["dkb"], ecut)
    w, _ = O.dense_eigs(cell, k)
    return cell, w


def write(name, header, values):
    with open(os.path.join(HERE, name), "w") as f:
        for h in header:
            f.write("# " + h + "\n")
        for v in values:
            f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    cell, w = dense_lowest("Si", 1, 10.0, 0, 32)
    write("si8_ecut10_seed0_eigs.txt",
          ["Si 8-atom diamond cell, a = 10.26 bohr, Ecut = 10 Ha, seed 0 (synth.py draws)",
           f"npw = {cell.npw}, grid = {cell.Ns}; lowest 32 eigenvalues (Ha) of the dense H,",
           "the Kohn-Sham eigenproblem H X = X Lambda of Sec. II-A Eq. 1; written by make_golden.py"],
          w)
    cell, w = dense_lowest("C", 1, 8.0, 0, 24)
    write("c8_ecut8_seed0_eigs.txt",
          ["C 8-atom diamond cell, a = 6.74 bohr, Ecut = 8 Ha, seed 0 (synth.py draws)",
           f"npw = {cell.npw}, grid = {cell.Ns}; lowest 24 eigenvalues (Ha) of the dense H,",
           "Sec. II-A Eq. 1; written by make_golden.py"],
          w)
