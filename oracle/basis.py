"""Dressed-site basis (Methods, Eq. (12)-(14)).  Test infrastructure only.

A site x carries one staggered matter mode (occupation phi in {0,1}) and six
half-links (rishon modes) j = 1..6 in the order -x, -y, -z, +x, +y, +z, each
with occupation k_j in {0,1,2}.  Gauss's law, Eq. (14), keeps the rows with

    phi + sum_j k_j = 6 + (1 - p)/2,     p = (-1)^(i+j+k) the site parity.

Eq. (12) attaches the sign (-1)^([k1=2] + [k2=2] + [k3=2]) to each row.  The
site charge is q = phi - (1 - p)/2 (Eq. (1) text: Q = N - L^3/2).

Row order (a reading: the paper fixes none): phi outer (0 then 1), then
(k1, ..., k6) lexicographic with k1 the most significant digit.
"""
import itertools

import numpy as np

N_HALF = 6
D_LOCAL = 267

# column layout of a basis table row
COL_PHI = 0
COL_K = slice(1, 7)
COL_SIGN = 7
COL_Q = 8


def enumerate_basis(parity):
    """Return the int8 table [267, 9] = (phi, k1..k6, sign, q) for a site of
    parity +1 (even) or -1 (odd), following Eq. (12) and Eq. (14)."""
    if parity not in (1, -1):
        raise ValueError("parity must be +1 or -1")
    target = 6 + (1 - parity) // 2
    rows = []
    for phi in (0, 1):
        for ks in itertools.product((0, 1, 2), repeat=N_HALF):
            if phi + sum(ks) != target:
                continue
            n_two = sum(1 for k in ks[:3] if k == 2)
            sign = -1 if n_two % 2 else 1
            q = phi - (1 - parity) // 2
            rows.append((phi,) + ks + (sign, q))
    table = np.array(rows, dtype=np.int8)
    return table


def all_configurations():
    """All 2 * 3^6 = 1458 (phi, k1..k6) before Gauss's law (Methods text
    after Eq. (14))."""
    return [(phi,) + ks for phi in (0, 1) for ks in itertools.product((0, 1, 2), repeat=N_HALF)]


def charges(parity):
    """Site charge of each basis row (int array of length 267)."""
    return enumerate_basis(parity)[:, COL_Q].astype(np.int64)
