"""Binary 3D tree, U(1) sector table and seeded isometric initialisation.
Test infrastructure only.

Tree (Methods, "Tensor Networks"): bottom tensors merge pairs of
x-neighbouring sites; the next layer merges pairs along y, then z, and the
cycle repeats (an axis whose blocks already span the lattice is skipped).
Every tensor has three legs (left child, right child, parent); the left child
is the block with the lower coordinate along the merge axis.  Nodes are
numbered layer by layer from the bottom, and inside a layer by the lowest
corner of their block in (z, y, x) lexicographic order.

Sectors (a reading; the paper initialises them at random): a bond whose
lower subtree S holds n of the N sites gets, for each charge q,
    w_q = D_S(q) * D_comp(Q - q),
D_X(q) the number of product states of region X with charge q.  Bond
dimensions are chi_q = min(floor(chi' w_q / W), cap_q), chi' = min(chi,
sum cap_q), cap_q = min(D_comp(Q - q), rows_q), rows_q the number of child
index pairs with charge q; the units still missing go one at a time to the
sector with the largest chi' w_q / W - chi_q among those below their cap,
ties to the smaller |q N - Q n|, then to the lower q.  The two bonds below
the root are then trimmed to their common part, chi_left(q) = chi_right(Q -
q) = min of the two, since the root's parent leg has dimension one.  All
arithmetic is exact (Python integers and Fractions).

Initialisation (a reading): SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),
one stream seeded with ``seed``; value = 2 * (x >> 11) * 2^-53 - 1.  Nodes
are filled in number order; inside a node, parent sectors in ascending q,
and for each one the (rows x chi_q) matrix row-major, rows ordered by
(q_left ascending, left index, right index).  Each parent-sector matrix is
then replaced by the Q factor of its QR decomposition with diag(R) > 0.
"""
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

from . import basis as _basis
from . import model as _model


@dataclass
class Node:
    index: int
    layer: int
    lo: tuple          # block lower corner (x, y, z)
    hi: tuple          # block upper corner, exclusive
    axis: int          # merge axis of this node
    children: tuple    # ((kind, id), (kind, id)), kind 'site' or 'node'
    parent: int = -1
    sites: tuple = ()


def build_tree(Lx, Ly, Lz):
    lat = _model.Lattice(Lx, Ly, Lz)
    dims = (Lx, Ly, Lz)
    blocks = []
    for s in range(lat.n_sites):
        c = lat.coords(s)
        blocks.append((("site", s), c, tuple(v + 1 for v in c), (s,)))
    nodes = []
    layer = 0
    axis = 0
    while len(blocks) > 1:
        # next axis (cycle x, y, z) along which blocks do not yet span the lattice
        for _ in range(3):
            ext = blocks[0][2][axis] - blocks[0][1][axis]
            if ext < dims[axis]:
                break
            axis = (axis + 1) % 3
        ext = blocks[0][2][axis] - blocks[0][1][axis]
        by_lo = {b[1]: b for b in blocks}
        merged = []
        for b in blocks:
            lo = b[1]
            if (lo[axis] // ext) % 2 != 0:
                continue
            partner_lo = list(lo)
            partner_lo[axis] += ext
            partner = by_lo[tuple(partner_lo)]
            hi = list(b[2])
            hi[axis] = partner[2][axis]
            merged.append((lo, tuple(hi), b, partner))
        merged.sort(key=lambda m: (m[0][2], m[0][1], m[0][0]))
        new_blocks = []
        for (lo, hi, left, right) in merged:
            idx = len(nodes)
            nd = Node(idx, layer, lo, hi, axis, (left[0], right[0]), sites=tuple(sorted(left[3] + right[3])))
            nodes.append(nd)
            new_blocks.append((("node", idx), lo, hi, nd.sites))
        for nd in nodes:
            for (kind, cid) in nd.children:
                if kind == "node":
                    nodes[cid].parent = nd.index
        blocks = new_blocks
        layer += 1
        axis = (axis + 1) % 3
    return nodes


def site_multiplicities(parity):
    """{charge: number of dressed rows}: 141/126 per the Gauss-law count."""
    q = _basis.charges(parity)
    vals, cnt = np.unique(q, return_counts=True)
    return {int(v): int(c) for v, c in zip(vals, cnt)}


def _convolve(a, b):
    out = {}
    for qa, da in a.items():
        for qb, db in b.items():
            out[qa + qb] = out.get(qa + qb, 0) + da * db
    return out


def region_counts(lat, sites):
    """D_X(q): number of product states of the sites with total charge q."""
    dist = {0: 1}
    for s in sites:
        dist = _convolve(dist, site_multiplicities(lat.parity(s)))
    return dist


def allocate(chi, w, cap, n, N, Q):
    """Largest-remainder allocation of chi' units over sectors (see module
    docstring).  w, cap: dicts over q with w_q > 0 and cap_q > 0."""
    qs = sorted(q for q in w if w[q] > 0 and cap.get(q, 0) > 0)
    if not qs:
        return {}
    W = sum(w[q] for q in qs)
    chi_p = min(chi, sum(cap[q] for q in qs))
    ideal = {q: Fraction(chi_p * w[q], W) for q in qs}
    out = {q: min(int(ideal[q]), cap[q]) for q in qs}
    missing = chi_p - sum(out.values())
    while missing > 0:
        cands = [q for q in qs if out[q] < cap[q]]
        best = min(cands, key=lambda q: (-(ideal[q] - out[q]), abs(q * N - Q * n), q))
        out[best] += 1
        missing -= 1
    return {q: c for q, c in out.items() if c > 0}


def sweep_order(nodes):
    """Order of the node updates within one sweep.  The Methods section runs
    each sweep from the lowest to the highest layer and fixes no order
    inside a layer.  Reading taken here: inside a layer the nodes follow a
    depth-first walk of the tree (first child before second child), and the
    direction alternates from one layer to the next, so that consecutive
    updates sit few bonds apart and each layer starts next to where the
    previous one ended."""
    root = len(nodes) - 1
    rank = {}
    stack = [root]
    while stack:
        i = stack.pop()
        rank[i] = len(rank)
        kids = [c for (kind, c) in nodes[i].children if kind == "node"]
        stack.extend(reversed(kids))
    order = []
    layers = sorted({nd.layer for nd in nodes})
    for li, layer in enumerate(layers):
        row = sorted((nd.index for nd in nodes if nd.layer == layer), key=rank.get)
        order.extend(row if li % 2 == 0 else row[::-1])
    return order


def sector_table(p: _model.Params, chi, nodes=None):
    """Bond sectors {q: chi_q} for the bond above each node, bottom-up.
    The root's parent bond is {Q: 1}."""
    lat = _model.Lattice(p.Lx, p.Ly, p.Lz)
    if nodes is None:
        nodes = build_tree(p.Lx, p.Ly, p.Lz)
    N = lat.n_sites
    all_sites = set(range(N))
    bonds = [None] * len(nodes)
    for nd in nodes:
        legs = [leg_sectors(lat, bonds, c) for c in nd.children]
        rows = {}
        for qa, da in legs[0].items():
            for qb, db in legs[1].items():
                rows[qa + qb] = rows.get(qa + qb, 0) + da * db
        if nd.parent < 0:
            bonds[nd.index] = {p.Q: 1} if rows.get(p.Q, 0) > 0 else {}
            continue
        dS = region_counts(lat, nd.sites)
        dC = region_counts(lat, sorted(all_sites - set(nd.sites)))
        w = {q: dS[q] * dC.get(p.Q - q, 0) for q in dS}
        cap = {q: min(dC.get(p.Q - q, 0), rows.get(q, 0)) for q in dS}
        bonds[nd.index] = allocate(chi, w, cap, len(nd.sites), N, p.Q)
    # The root has a one-dimensional parent leg, so its two child bonds must
    # pair up sector by sector (q, Q - q); keep the common part of both.
    root = nodes[-1]
    kids = [cid for (kind, cid) in root.children if kind == "node"]
    if len(kids) == 2:
        left, right = bonds[kids[0]], bonds[kids[1]]
        new_left = {q: min(c, right.get(p.Q - q, 0)) for q, c in left.items()}
        new_right = {q: min(c, left.get(p.Q - q, 0)) for q, c in right.items()}
        bonds[kids[0]] = {q: c for q, c in new_left.items() if c > 0}
        bonds[kids[1]] = {q: c for q, c in new_right.items() if c > 0}
    return bonds


def leg_sectors(lat, bonds, child):
    kind, cid = child
    if kind == "site":
        return site_multiplicities(lat.parity(cid))
    return bonds[cid]


def leg_charges(lat, bonds, child):
    """Charge label of every index of a leg (sector-contiguous, ascending)."""
    sec = leg_sectors(lat, bonds, child)
    if child[0] == "site":
        return _basis.charges(lat.parity(child[1]))
    return np.concatenate([np.full(sec[q], q, dtype=np.int64) for q in sorted(sec)]) if sec else np.zeros(0, np.int64)


def parent_charges(bonds, idx):
    sec = bonds[idx]
    return np.concatenate([np.full(sec[q], q, dtype=np.int64) for q in sorted(sec)]) if sec else np.zeros(0, np.int64)


# SplitMix64 constants from Steele, Lea & Flood (2014)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, start, count):
    """Outputs number start+1 .. start+count of SplitMix64 seeded with seed
    (state_i = seed + i * gamma; output = mix(state_i))."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(raw):
    """2 * (x >> 11) * 2^-53 - 1 in [-1, 1)."""
    return 2.0 * (raw >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 1.0


def sector_rows(qa_labels, qb_labels, q):
    """Flat (a, b) row indices of parent sector q, ordered by (q_a, a, b)."""
    A, B = np.meshgrid(np.arange(len(qa_labels)), np.arange(len(qb_labels)), indexing="ij")
    A = A.ravel()
    B = B.ravel()
    sel = qa_labels[A] + qb_labels[B] == q
    A, B = A[sel], B[sel]
    order = np.lexsort((B, A, qa_labels[A]))
    return A[order], B[order]


def qr_positive(M):
    """Reduced QR with diag(R) > 0 (numpy Householder QR + sign fix)."""
    Qm, R = np.linalg.qr(M, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Qm * d[None, :], R * d[:, None]


# Rank handling of the centre-move QR (a reading: the paper keeps the bond
# dimensions fixed only implicitly).  A sector matrix whose QR diagonal
# falls below QR_FALLBACK * (largest column norm) is factorised by
# classical Gram-Schmidt applied twice per column; a column whose remainder
# is at most QR_DEPENDENT * (largest column norm) is dependent: R_jj = 0 and
# q_j is the first unit vector e_k (k increasing over the rows, never reused)
# whose remainder after two projections exceeds QR_ACCEPT.
QR_FALLBACK = 1e-6
QR_DEPENDENT = 1e-9
QR_ACCEPT = 0.5


def qr_gram_schmidt(X):
    """Column-by-column Gram-Schmidt (two passes) with deterministic
    completion of dependent columns; returns Q (orthonormal columns), R."""
    m, n = X.shape
    if n > m:
        raise ValueError("sector has fewer rows than columns")
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    scale = max(float(np.max(np.linalg.norm(X, axis=0))), 0.0) if n else 0.0
    next_k = 0
    for j in range(n):
        v = X[:, j].copy()
        for _ in range(2):
            c = Q[:, :j].T @ v
            v = v - Q[:, :j] @ c
            R[:j, j] += c
        nv = float(np.linalg.norm(v))
        if nv > QR_DEPENDENT * scale:
            Q[:, j] = v / nv
            R[j, j] = nv
            continue
        while True:
            w = np.zeros(m)
            w[next_k] = 1.0
            next_k += 1
            for _ in range(2):
                w = w - Q[:, :j] @ (Q[:, :j].T @ w)
            nw = float(np.linalg.norm(w))
            if nw > QR_ACCEPT:
                Q[:, j] = w / nw
                break
    return Q, R


def qr_sector(X):
    """QR of one sector matrix for a centre move: the unique QR with
    positive diag(R) when every diagonal entry exceeds QR_FALLBACK times the
    largest column norm, else ``qr_gram_schmidt``."""
    if X.shape[1] > X.shape[0]:
        raise ValueError("sector has fewer rows than columns")
    Qm, R = qr_positive(X)
    scale = float(np.max(np.linalg.norm(X, axis=0))) if X.size else 0.0
    if X.shape[1] and np.min(np.abs(np.diag(R))) <= QR_FALLBACK * scale:
        return qr_gram_schmidt(X)
    return Qm, R
