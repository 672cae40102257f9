"""Test helpers: move oracle tensors (dense with masks) into the native block
layout and back.  The native layout orders blocks by (parent sector
ascending, left charge ascending); each block is row-major (left, right,
parent) over the indices of those sectors."""
import numpy as np


def layout_index(ql, qr, qc):
    """Flat dense indices (a, b, c) in native layout order."""
    idx_a, idx_b, idx_c = [], [], []
    qr_set = set(np.unique(qr).tolist())
    for q in sorted(np.unique(qc).tolist()):
        cols = np.nonzero(qc == q)[0]
        for qa in sorted(np.unique(ql).tolist()):
            qb = q - qa
            if qb not in qr_set:
                continue
            A = np.nonzero(ql == qa)[0]
            B = np.nonzero(qr == qb)[0]
            a, b, c = np.meshgrid(A, B, cols, indexing="ij")
            idx_a.append(a.ravel())
            idx_b.append(b.ravel())
            idx_c.append(c.ravel())
    if not idx_a:
        return (np.zeros(0, int),) * 3
    return np.concatenate(idx_a), np.concatenate(idx_b), np.concatenate(idx_c)


def to_layout(T, labels):
    a, b, c = layout_index(*labels)
    return T[a, b, c].copy()


def from_layout(v, labels, shape):
    a, b, c = layout_index(*labels)
    T = np.zeros(shape)
    T[a, b, c] = v
    return T
