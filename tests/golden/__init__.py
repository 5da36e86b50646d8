"""Small text fixtures taken from the paper, each with its citation."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ANGSTROM = 1.0 / 0.529177210903   # bohr per Angstrom (CODATA 2018 Bohr radius)
_Z = {"H": 1, "C": 6, "N": 7, "O": 8}


def water_sample_input():
    """(Z, xyz in bohr) of the paper's sample-input water molecule."""
    Z, xyz = [], []
    for line in open(os.path.join(HERE, "water_sample_input.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        Z.append(_Z[line[0]])
        xyz.append([float(v) * ANGSTROM for v in line[1:4]])
    return np.array(Z, np.int32), np.array(xyz)
