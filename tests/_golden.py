"""Reader of the hand-derived fixtures under tests/golden/ (exact solutions of
small Poisson problems, each block citing the passage it follows)."""

import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BC_CODES = {"P": 0, "DR": 1, "DS": 2, "NR": 3, "NS": 4}
APPROX_CODES = {"SPECTRAL": 0, "FD2": 1}


def _parse_block(lines, fname):
    case = {"file": fname}
    for ln in lines:
        key, _, val = ln.partition(":")
        case[key.strip()] = val.strip()
    n = [int(v) for v in case["n"].split()]
    Ls = [float(v) for v in case["L"].split()]
    bcs = [BC_CODES[v] for v in case["bc"].split()]
    g = [Fraction(v) for v in case["g"].split()]
    phi = [Fraction(v) for v in case["phi"].split()]
    if not (len(n) == len(Ls) == len(bcs)) or len(g) != int(np.prod(n)) or len(phi) != len(g):
        raise ValueError(f"{fname}: case {case.get('case')}: inconsistent sizes")
    shape = tuple(reversed(n))  # numpy shape, x the last axis
    return {
        "name": case["case"],
        "file": fname,
        "approx": APPROX_CODES[case["approx"]],
        "n": tuple(n),
        "Ls": tuple(Ls),
        "bcs": tuple(bcs),
        "g_exact": g,
        "phi_exact": phi,
        "g": np.array([float(v) for v in g]).reshape(shape),
        "phi": np.array([float(v) for v in phi]).reshape(shape),
    }


def load_cases():
    cases = []
    for fname in sorted(os.listdir(GOLDEN)):
        if not fname.endswith(".txt"):
            continue
        block = []
        with open(os.path.join(GOLDEN, fname)) as f:
            for raw in f:
                ln = raw.strip()
                if ln.startswith("#"):
                    continue
                if not ln:
                    if block:
                        cases.append(_parse_block(block, fname))
                        block = []
                    continue
                block.append(ln)
        if block:
            cases.append(_parse_block(block, fname))
    return cases
