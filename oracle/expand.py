"""Single-tensor optimisation with subspace expansion, written plainly.  Test
infrastructure only.

Methods, "Tensor Networks": the single-tensor optimisation is run with a
subspace expansion that lets the bond dimension grow during the sweeps and
the symmetry sectors adapt; the paper names the technique and cites it, with
no equations.  This module takes the usual form of it (the enrichment of
Hubig, McCulloch, Schollwoeck and Wolf, 2015), written for this tree and
its operators:

When the centre leaves node c across bond b towards its neighbour t, the
tensor A of c is enlarged along b by alpha * P.  P holds what the
Hamiltonian does on c's side of b: the part of H_eff(c) that acts only on
c's other legs, applied to A (one block of columns), and, for every term
that acts on both sides of b, its factors on c's other legs applied to A
(one block of columns per term, with the bond index now carrying the charge
those factors leave on it).  The tensor of t is padded with zeros along b,
so the state does not change.  The enlarged A is split per charge sector of
the enlarged bond by an SVD; the chi_max largest singular values over all
sectors are kept (values at or below cutoff times the largest are dropped),
which fixes the new sector dimensions of b; A becomes the isometry U and
S V^T is absorbed into t.

Readings: a column of P keeps its charge even where the neighbour's other
legs cannot form it yet (its block in t starts empty); that is how sectors
grow through a node whose two other bonds must match, such as the root
(two-step adaptation: one bond gains the sector empty, the next expanded
move fills the other); only the first bond of each centre path is expanded
(the one the
freshly optimised tensor leaves through); the later bonds of the path are
crossed by the same SVD move with alpha = 0, so every bond dimension follows
the rank of its tensors (a truncated bond elsewhere can leave a bond with
more columns than the state needs, which the SVD drops); ties between equal
singular values go to the lower charge, then to the lower index; alpha,
chi_max and cutoff are inputs (the paper gives none).
"""
import numpy as np

from . import tree as _tree
from .ttn import apply_leg


def _implied_labels(labels, X, leg):
    """Charge each index of ``leg`` of X must carry for X's nonzero entries
    to obey q_left + q_right = q_parent; None for an all-zero index."""
    ql, qr, qc = labels
    others = [l for l in (0, 1, 2) if l != leg]
    Xm = np.moveaxis(X, leg, 2)
    q0 = labels[others[0]][:, None]
    q1 = labels[others[1]][None, :]
    if leg == 2:
        implied = q0 + q1
    elif leg == 0:
        implied = q1 - q0        # others = (1, 2): q_left = q_parent - q_right
    else:
        implied = q1 - q0        # others = (0, 2): q_right = q_parent - q_left
    out = []
    for i in range(Xm.shape[2]):
        nz = Xm[:, :, i] != 0.0
        if not nz.any():
            out.append(None)
            continue
        vals = np.unique(implied[nz])
        if len(vals) != 1:
            raise ValueError("expansion block without a definite charge")
        out.append(int(vals[0]))
    return out


def expansion_blocks(state, c, leg):
    """The blocks of P at node c for the bond on ``leg``: a list of dense
    tensors of A's shape (before the factor alpha)."""
    A = state.T[c]
    own = np.zeros_like(A)
    blocks = []
    for coef, ops in state.heff_terms(c):
        rest = {l: op for l, op in ops.items() if l != leg}
        if not rest:
            continue                      # acts on t's side only
        Z = A
        for l, op in rest.items():
            Z = apply_leg(op, Z, l)
        if leg in ops:
            blocks.append(coef * Z)       # a term acting on both sides of b
        else:
            own = own + coef * Z          # c's side alone
    return [own] + blocks


def expand_move(state, target, alpha, chi_max, cutoff=1e-13):
    """Move the centre from state.center to the neighbour ``target`` with
    subspace expansion of the bond between them.  Returns the new sector
    dimensions {q: dim} of that bond."""
    c = state.center
    leg_c = state._neighbour_leg(c, target)
    leg_t = state._neighbour_leg(target, c)
    A = state.T[c]
    lab_c = state.labels[c]
    old = lab_c[leg_c]
    # columns of the enlarged A: A's own, then alpha * P block by block
    cols, col_q, col_src = [], [], []
    Am = np.moveaxis(A, leg_c, 2)
    for i in range(Am.shape[2]):
        cols.append(Am[:, :, i])
        col_q.append(int(old[i]))
        col_src.append(i)
    if alpha != 0.0:
        for X in expansion_blocks(state, c, leg_c):
            q = _implied_labels(lab_c, X, leg_c)
            Xm = np.moveaxis(X, leg_c, 2)
            for i in range(Xm.shape[2]):
                if q[i] is None:
                    continue
                cols.append(alpha * Xm[:, :, i])
                col_q.append(q[i])
                col_src.append(-1)
    col_q = np.array(col_q)
    col_src = np.array(col_src)
    others = [l for l in (0, 1, 2) if l != leg_c]
    q0 = lab_c[others[0]][:, None]
    q1 = lab_c[others[1]][None, :]
    implied = q0 + q1 if leg_c == 2 else q1 - q0
    # SVD per charge sector of the enlarged bond
    cand = []        # (-s, q, j) for every singular value
    per_q = {}
    for q in sorted(set(col_q.tolist())):
        sel = np.nonzero(col_q == q)[0]
        rows = np.nonzero(implied == q)
        M = np.stack([cols[j][rows] for j in sel], axis=1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        per_q[q] = (rows, sel, U, S, Vt)
        for j, s in enumerate(S):
            cand.append((-s, q, j))
    cand.sort()
    smax = -cand[0][0] if cand else 0.0
    kept = [(q, j) for (ms, q, j) in cand if -ms > cutoff * smax][:chi_max]
    dims = {}
    for q, j in kept:
        dims[q] = dims.get(q, 0) + 1
    new_lab = np.concatenate([np.full(dims[q], q, dtype=np.int64) for q in sorted(dims)])
    off = {}
    o = 0
    for q in sorted(dims):
        off[q] = o
        o += dims[q]
    # new isometry at c and the matrix R (new index x old index) for t
    shape = list(Am.shape[:2]) + [len(new_lab)]
    newA = np.zeros(shape)
    R = np.zeros((len(new_lab), len(old)))
    for q in sorted(dims):
        rows, sel, U, S, Vt = per_q[q]
        js = sorted(j for (qq, j) in kept if qq == q)
        for k, j in enumerate(js):
            newA[rows[0], rows[1], off[q] + k] = U[:, j]
            for p, src in enumerate(col_src[sel]):
                if src >= 0:
                    R[off[q] + k, src] = S[j] * Vt[j, p]
    state.T[c] = np.moveaxis(newA, 2, leg_c)
    state.T[target] = apply_leg(R, state.T[target], leg_t)
    lc = list(state.labels[c])
    lc[leg_c] = new_lab
    state.labels[c] = tuple(lc)
    lt = list(state.labels[target])
    lt[leg_t] = new_lab
    state.labels[target] = tuple(lt)
    child = c if leg_c == 2 else target
    state.bonds[child] = dict(dims)
    state.center = target
    if leg_c == 2:
        state.up[c] = state._up_ops(c)
    else:
        state.down[target] = state._down_ops(target)
    return dict(dims)


def optimize_node_expanded(state, idx, tol, alpha, chi_max, cutoff=1e-13):
    """Move the centre to idx (the first bond of the path expanded) and
    replace T[idx] by the lowest eigenvector of its H_eff."""
    path = state.path(state.center, idx)
    for k, nxt in enumerate(path[1:]):
        expand_move(state, nxt, alpha if k == 0 else 0.0, chi_max, cutoff)
    e, v = state.local_ground_state(idx, tol)
    M = state.mask(idx)
    T = np.zeros(M.shape)
    T[M] = v
    state.T[idx] = T
    state.energies.append(e)
    return e


def sweep_expanded(state, tol, alpha, chi_max, cutoff=1e-13):
    """One sweep (tree.sweep_order) of expanded single-tensor updates."""
    return [optimize_node_expanded(state, i, tol, alpha, chi_max, cutoff) for i in _tree.sweep_order(state.nodes)]
