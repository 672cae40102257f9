"""Tree Tensor Network ground-state search, written plainly.  Test
infrastructure only.

This follows the three-step single-tensor optimisation of the Methods
("Tensor Networks"):
  (i)   H_eff of one tensor is the full Hamiltonian contracted with every
        other tensor of the tree,
  (ii)  its lowest eigenpair is found by an Arnoldi/Lanczos-type solver
        (here scipy's ARPACK ``eigsh``, the paper's solver family, or dense
        ``eigh`` for small problems),
  (iii) the tensor is replaced by that eigenvector; tensors are visited
        from the lowest to the highest layer, and the sweep repeats.

Representation: every node tensor is a DENSE array T[a, b, c] (left child,
right child, parent) with zeros wherever q_a + q_b != q_c; the global U(1)
symmetry (Methods: total charge conserved through global sectors) enters
only through those masks and through per-sector QR.  Renormalized
operators are dense bond x bond matrices.  Physical site operators are
scipy CSR matrices from ``oracle.fock``.

Gauge: all tensors except the centre are isometries pointing at the
centre.  Moving the centre across a bond is a per-sector QR
(``tree.qr_sector``: positive diag(R), with a deterministic completion of
rank-deficient sectors); R is absorbed by the neighbour.  Rows of a sector
matrix are ordered lexicographically in the two other legs.

Bond operators: ``up[n]`` holds, for the bond above node n, the
renormalized restriction to subtree(n) of every term that crosses the bond
(key = term index) and the block Hamiltonian of the terms inside subtree(n)
(key 'H').  ``down[n]`` holds the same for the complement of subtree(n).

Parity unpinned: absolute TTN energies at a given bond dimension (a
variational result) are pinned only by the variational bound, exactness at
large bond dimension on 2x2x1 (``oracle.ed``), the invariants, and parity
with the GPU path.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis as _basis
from . import fock as _fock
from . import model as _model
from . import tree as _tree


def apply_leg(op, X, leg):
    """Contract a matrix op[i', i] into leg ``leg`` of the 3-tensor X."""
    d0, d1, d2 = X.shape
    if leg == 0:
        return np.asarray(op @ X.reshape(d0, d1 * d2)).reshape(op.shape[0], d1, d2)
    if leg == 2:
        return np.asarray(X.reshape(d0 * d1, d2) @ op.T).reshape(d0, d1, op.shape[0])
    Y = np.asarray(op @ X.transpose(1, 0, 2).reshape(d1, d0 * d2))
    return Y.reshape(op.shape[0], d0, d2).transpose(1, 0, 2)


def renormalize(T, ops, out_leg):
    """Sum_{others} T[..i'..] (ops applied) T[..i..] with the free leg
    ``out_leg``: returns R[i', i] = <i'| O |i> for the isometry T.
    ``ops`` maps leg -> matrix (legs other than out_leg); missing = 1."""
    Y = T
    for leg, op in ops.items():
        if op is not None:
            Y = apply_leg(op, Y, leg)
    # R[i', i] = sum over the two other legs of T[.., i', ..] * Y[.., i, ..]
    A = np.moveaxis(T, out_leg, 0).reshape(T.shape[out_leg], -1)
    B = np.moveaxis(Y, out_leg, 0).reshape(Y.shape[out_leg], -1)
    return A @ B.T


class TTN:
    def __init__(self, p: _model.Params, chi, seed, build_ops=True):
        self.p = p
        self.chi = chi
        self.lat = _model.lattice(p)
        self.nodes = _tree.build_tree(p.Lx, p.Ly, p.Lz)
        self.bonds = _tree.sector_table(p, chi, self.nodes)
        self.terms, self.const = _model.build_terms(p)
        n = len(self.nodes)
        self.labels = []
        for nd in self.nodes:
            ql = _tree.leg_charges(self.lat, self.bonds, nd.children[0])
            qr = _tree.leg_charges(self.lat, self.bonds, nd.children[1])
            qc = _tree.parent_charges(self.bonds, nd.index)
            self.labels.append((ql, qr, qc))
        self.region = [set(nd.sites) for nd in self.nodes]
        self.all_sites = set(range(self.lat.n_sites))
        self.T = [None] * n
        self._init_random(seed)
        self.center = n - 1
        self.up = [None] * n
        self.down = [None] * n
        if build_ops:
            for nd in self.nodes:
                if nd.parent >= 0:
                    self.up[nd.index] = self._up_ops(nd.index)
        self.energies = []

    # ------------------------------------------------------------ setup
    def mask(self, idx):
        ql, qr, qc = self.labels[idx]
        return (ql[:, None, None] + qr[None, :, None]) == qc[None, None, :]

    def _init_random(self, seed):
        pos = 0
        self.prefill = []
        for nd in self.nodes:
            ql, qr, qc = self.labels[nd.index]
            T = np.zeros((len(ql), len(qr), len(qc)))
            pre = np.zeros_like(T)
            for q in sorted(self.bonds[nd.index]):
                cols = np.nonzero(qc == q)[0]
                A, B = _tree.sector_rows(ql, qr, q)
                cnt = len(A) * len(cols)
                vals = _tree.uniform_pm1(_tree.splitmix64(seed, pos, cnt)).reshape(len(A), len(cols))
                pos += cnt
                pre[A[:, None], B[:, None], cols[None, :]] = vals
                Qm, _ = _tree.qr_positive(vals)
                T[A[:, None], B[:, None], cols[None, :]] = Qm
            self.prefill.append(pre)
            self.T[nd.index] = T

    # ------------------------------------------------------------ operators
    def _leg_region(self, child):
        kind, cid = child
        return {cid} if kind == "site" else self.region[cid]

    def _crosses(self, term, region):
        sites = {s for (s, _) in term.ops}
        return bool(sites & region) and bool(sites - region)

    def _site_factor(self, term, s):
        for (site, key) in term.ops:
            if site == s:
                return _fock.site_op(key, self.lat.parity(s))
        return None

    def _leg_factor(self, child, term_idx, term, upward=True):
        """Factor of a term on a child leg: the site op, or the renormalized
        restriction stored on the child's bond; None if the term misses it."""
        kind, cid = child
        region = self._leg_region(child)
        sites = {s for (s, _) in term.ops}
        if not (sites & region):
            return None
        if kind == "site":
            return self._site_factor(term, cid)
        return self.up[cid][term_idx]

    def _leg_hamiltonian(self, child):
        kind, cid = child
        if kind == "node":
            return self.up[cid]["H"]
        # single-site terms of this site
        d = _basis.D_LOCAL
        H = sp.csr_matrix((d, d))
        for tm in self.terms:
            if len(tm.ops) == 1 and tm.ops[0][0] == cid:
                H = H + tm.coef * _fock.site_op(tm.ops[0][1], self.lat.parity(cid))
        return H

    def _up_ops(self, idx):
        nd = self.nodes[idx]
        T = self.T[idx]
        S = self.region[idx]
        l, r = nd.children
        Sl, Sr = self._leg_region(l), self._leg_region(r)
        out = {}
        for k, tm in enumerate(self.terms):
            if self._crosses(tm, S):
                A = self._leg_factor(l, k, tm)
                B = self._leg_factor(r, k, tm)
                out[k] = renormalize(T, {0: A, 1: B}, 2)
        H = renormalize(T, {0: self._leg_hamiltonian(l)}, 2) + renormalize(T, {1: self._leg_hamiltonian(r)}, 2)
        for k, tm in enumerate(self.terms):
            sites = {s for (s, _) in tm.ops}
            if sites <= S and sites & Sl and sites & Sr:
                H = H + tm.coef * renormalize(T, {0: self._leg_factor(l, k, tm), 1: self._leg_factor(r, k, tm)}, 2)
        out["H"] = H
        return out

    def _down_ops(self, idx):
        """Environment operators of the bond above node idx, from its parent."""
        nd = self.nodes[idx]
        par = self.nodes[nd.parent]
        T = self.T[par.index]
        leg = 0 if par.children[0] == ("node", idx) else 1
        sib = par.children[1 - leg]
        Ssib = self._leg_region(sib)
        Sp = self.region[par.index]
        comp_p = self.all_sites - Sp
        comp_n = self.all_sites - self.region[idx]
        out = {}
        for k, tm in enumerate(self.terms):
            if not self._crosses(tm, self.region[idx]):
                continue
            sites = {s for (s, _) in tm.ops}
            B = self._leg_factor(sib, k, tm)
            C = self.down[par.index][k] if (sites & comp_p) else None
            out[k] = renormalize(T, {1 - leg: B, 2: C}, leg)
        H = renormalize(T, {1 - leg: self._leg_hamiltonian(sib)}, leg)
        if par.parent >= 0:
            H = H + renormalize(T, {2: self.down[par.index]["H"]}, leg)
        for k, tm in enumerate(self.terms):
            sites = {s for (s, _) in tm.ops}
            if sites <= comp_n and sites & Ssib and sites & comp_p:
                H = H + tm.coef * renormalize(T, {1 - leg: self._leg_factor(sib, k, tm), 2: self.down[par.index][k]}, leg)
        out["H"] = H
        return out

    # ------------------------------------------------------------ H_eff
    def heff_terms(self, idx):
        """(coef, {leg: op}) list whose sum is H_eff at node idx (without
        the constant), following step (i) of the Methods."""
        nd = self.nodes[idx]
        l, r = nd.children
        Sl, Sr = self._leg_region(l), self._leg_region(r)
        S = self.region[idx]
        comp = self.all_sites - S
        out = [(1.0, {0: self._leg_hamiltonian(l)}), (1.0, {1: self._leg_hamiltonian(r)})]
        if nd.parent >= 0:
            out.append((1.0, {2: self.down[idx]["H"]}))
        for k, tm in enumerate(self.terms):
            sites = {s for (s, _) in tm.ops}
            touched = [bool(sites & Sl), bool(sites & Sr), bool(sites & comp)]
            if sum(touched) < 2:
                continue
            ops = {}
            if touched[0]:
                ops[0] = self._leg_factor(l, k, tm)
            if touched[1]:
                ops[1] = self._leg_factor(r, k, tm)
            if touched[2]:
                ops[2] = self.down[idx][k]
            out.append((tm.coef, ops))
        return out

    def heff_apply(self, idx, X, terms=None):
        """y = H_eff X (dense 3-tensor in, dense out), constant included."""
        if terms is None:
            terms = self.heff_terms(idx)
        y = self.const * X
        for coef, ops in terms:
            Z = X
            for leg, op in ops.items():
                Z = apply_leg(op, Z, leg)
            y += coef * Z
        return y

    def local_ground_state(self, idx, tol=1e-12, dense_limit=1500):
        """Step (ii): lowest eigenpair of H_eff restricted to the flux mask,
        started from the current tensor.  Eigenvector sign: <v0, v> >= 0."""
        M = self.mask(idx)
        shape = M.shape
        terms = self.heff_terms(idx)
        v0 = self.T[idx][M]

        def mv(v):
            X = np.zeros(shape)
            X[M] = v
            return self.heff_apply(idx, X, terms)[M]

        n = v0.size
        if n <= dense_limit:
            Hm = np.stack([mv(e) for e in np.eye(n)], axis=1)
            Hm = 0.5 * (Hm + Hm.T)
            w, V = np.linalg.eigh(Hm)
            e, v = w[0], V[:, 0]
        else:
            op = spla.LinearOperator((n, n), matvec=mv, dtype=np.float64)
            w, V = spla.eigsh(op, k=1, which="SA", v0=v0, tol=tol, ncv=min(n, 40), maxiter=100000)
            e, v = w[0], V[:, 0]
        v = v / np.linalg.norm(v)
        if np.dot(v, v0) < 0:
            v = -v
        return e, v

    # ------------------------------------------------------------ gauge moves
    def _qr_toward(self, idx, leg):
        """Per-sector QR of T[idx] with ``leg`` as the column index.
        Returns R (block diagonal over the sectors of that leg)."""
        T = self.T[idx]
        M = self.mask(idx)
        lab = self.labels[idx][leg]
        Tm = np.moveaxis(T, leg, 2)
        Mm = np.moveaxis(M, leg, 2)
        dim = T.shape[leg]
        R = np.zeros((dim, dim))
        newT = np.zeros_like(Tm)
        for q in np.unique(lab):
            cols = np.nonzero(lab == q)[0]
            rows = np.nonzero(Mm[:, :, cols[0]])
            A = Tm[rows[0], rows[1], :][:, cols]
            if A.shape[0] < A.shape[1]:
                raise ValueError("sector has fewer rows than columns")
            Qm, Rq = _tree.qr_sector(A)
            newT[rows[0][:, None], rows[1][:, None], cols[None, :]] = Qm
            R[np.ix_(cols, cols)] = Rq
        self.T[idx] = np.moveaxis(newT, 2, leg)
        return R

    def _neighbour_leg(self, a, b):
        """Leg of node a that connects to node b."""
        nd = self.nodes[a]
        if nd.parent == b:
            return 2
        for leg in (0, 1):
            if nd.children[leg] == ("node", b):
                return leg
        raise ValueError("not neighbours")

    def move(self, target):
        """Move the centre one bond to neighbouring node ``target``."""
        c = self.center
        leg_c = self._neighbour_leg(c, target)
        leg_t = self._neighbour_leg(target, c)
        R = self._qr_toward(c, leg_c)
        self.T[target] = apply_leg(R, self.T[target], leg_t)
        self.center = target
        if leg_c == 2:
            self.up[c] = self._up_ops(c)
        else:
            self.down[target] = self._down_ops(target)

    def path(self, a, b):
        """Node path from a to b along the tree."""
        def ancestors(x):
            out = [x]
            while self.nodes[x].parent >= 0:
                x = self.nodes[x].parent
                out.append(x)
            return out
        pa, pb = ancestors(a), ancestors(b)
        common = next(x for x in pa if x in pb)
        up = pa[: pa.index(common) + 1]
        down = pb[: pb.index(common)]
        return up + list(reversed(down))

    def move_to(self, target):
        for nxt in self.path(self.center, target)[1:]:
            self.move(nxt)

    def set_couplings(self, **couplings):
        """New couplings (any of t, m, ge2, cB, nu) on the same lattice and
        charge: the centre moves to the root, the term list is rebuilt for
        the new couplings and every upward operator is recomputed from the
        current tensors (downward ones follow the centre as it moves down
        again, as after construction).  Used by the driven optimisation of
        the penalty (Methods, "Numerical Convergence")."""
        self.move_to(len(self.nodes) - 1)
        self.p = _model.with_couplings(self.p, **couplings)
        self.terms, self.const = _model.build_terms(self.p)
        n = len(self.nodes)
        self.up = [None] * n
        self.down = [None] * n
        for nd in self.nodes:
            if nd.parent >= 0:
                self.up[nd.index] = self._up_ops(nd.index)

    # ------------------------------------------------------------ sweep
    def optimize_node(self, idx, tol=1e-12):
        self.move_to(idx)
        e, v = self.local_ground_state(idx, tol)
        M = self.mask(idx)
        T = np.zeros(M.shape)
        T[M] = v
        self.T[idx] = T
        self.energies.append(e)
        return e

    def sweep(self, tol=1e-12):
        """One sweep: layer by layer from the bottom, in tree.sweep_order."""
        out = []
        for i in _tree.sweep_order(self.nodes):
            out.append(self.optimize_node(i, tol))
        return out

    # ------------------------------------------------------------ measurement
    def norm_at_center(self):
        return float(np.linalg.norm(self.T[self.center]))

    def energy_at_center(self):
        """<psi|H_eff|psi> / <psi|psi> at the current centre."""
        X = self.T[self.center]
        return float(np.vdot(X, self.heff_apply(self.center, X)) / np.vdot(X, X))

    def site_probabilities(self):
        """p[s][i] = <P_i> for each dressed row i of each site, via reduced
        density matrices pushed down from the root (centre moved there)."""
        self.move_to(len(self.nodes) - 1)
        n = len(self.nodes)
        rho = [None] * n
        root = n - 1
        rho[root] = np.ones((1, 1)) / 1.0
        probs = {}
        for idx in reversed(range(n)):
            T = self.T[idx]
            r = rho[idx]
            # rho_child[a', a] = sum T[a', b, c'] r[c', c] T[a, b, c]
            Y = apply_leg(r, T, 2)
            for leg in (0, 1):
                A = np.moveaxis(T, leg, 0).reshape(T.shape[leg], -1)
                B = np.moveaxis(Y, leg, 0).reshape(Y.shape[leg], -1)
                red = A @ B.T
                kind, cid = self.nodes[idx].children[leg]
                if kind == "site":
                    probs[cid] = np.diag(red).copy()
                else:
                    rho[cid] = red
        return [probs[s] for s in range(self.lat.n_sites)]

    def observables(self):
        """Single-site diagonal expectations: <psi^dag psi>, n_x, q_x, link E
        (Eq. (10) at the lower site), delta_L (Eq. (17b) text) and the surface
        charge density sigma(l) (Eq. (16a))."""
        probs = self.site_probabilities()
        lat = self.lat
        out = {"phi": [], "n": [], "q": [], "k": []}
        for s in range(lat.n_sites):
            table = _basis.enumerate_basis(lat.parity(s))
            pr = probs[s]
            phi = float(pr @ table[:, 0])
            par = lat.parity(s)
            out["phi"].append(phi)
            out["n"].append((1 + par) / 2 - par * phi)
            out["q"].append(float(pr @ table[:, _basis.COL_Q]))
            out["k"].append(pr @ table[:, _basis.COL_K].astype(np.float64))
        E = []
        dL = 0.0
        for (x, mu, y) in lat.links():
            kx = out["k"][x][_model.plus(mu)]
            ky = out["k"][y][_model.minus(mu)]
            E.append(1.0 - kx)
            dL += abs(kx + ky - 2.0)
        out["E_link"] = E
        out["delta_L"] = dL
        out["rho"] = float(np.mean(out["n"]))
        out["Q"] = float(np.sum(out["q"]))
        # sigma(l): mean <psi^dag psi> over the sites of surface layer l
        layers = {}
        for s in range(lat.n_sites):
            layers.setdefault(surface_layer(lat, s), []).append(out["phi"][s])
        out["sigma"] = [float(np.mean(layers[l])) for l in sorted(layers)]
        return out


def surface_layer(lat, s):
    """Layer index l of site s for the surface charge density sigma(l) of
    Eq. (16a): l = 1 on the outer surface of the open lattice, l = 2 one
    site further in, and so on (one plus the number of sites between s and
    the closest boundary face)."""
    c = lat.coords(s)
    dims = lat.dims()
    return 1 + min(min(c[a], dims[a] - 1 - c[a]) for a in range(3))


def bottom_heff_flops(state: TTN, idx):
    """Algorithmic flops of one H_eff x at bottom node ``idx``: every term
    with an environment factor (and the environment block Hamiltonian) is a
    row selection of the node tensor by the monomial site operators
    followed by a dense product with one environment block per output
    charge sector, 2 * (nonzero rows) * chi_out * chi_in flops; terms that
    act on the two sites only are row rescalings and count no flops.  A row
    is nonzero when both site operators have an entry in it and its source
    row lies in a charge block the parent bond carries."""
    nd = state.nodes[idx]
    assert all(kind == "site" for kind, _ in nd.children)
    ql, qr, qc = state.labels[idx]
    chi_q = {q: int(np.sum(qc == q)) for q in np.unique(qc)}
    sites = [cid for _, cid in nd.children]
    comp = state.all_sites - state.region[idx]
    d = _basis.D_LOCAL

    def row_source(op):
        # source index of every row of a monomial operator (-1: zero row)
        src = np.full(d, -1)
        if op is None:
            return np.arange(d)
        op = op.tocsr()
        for r in range(d):
            lo, hi = op.indptr[r], op.indptr[r + 1]
            if hi > lo:
                src[r] = op.indices[lo]
        return src

    def count(srcA, srcB):
        flops = 0.0
        qs = ql[:, None] + qr[None, :]
        ok = (srcA[:, None] >= 0) & (srcB[None, :] >= 0)
        sa, sb = np.maximum(srcA, 0), np.maximum(srcB, 0)
        qsrc = ql[sa][:, None] + qr[sb][None, :]
        ok &= np.isin(qsrc, list(chi_q))
        for q_out, c_out in chi_q.items():
            sel = ok & (qs == q_out)
            if not sel.any():
                continue
            for q_in in np.unique(qsrc[sel]):
                flops += 2.0 * np.sum(sel & (qsrc == q_in)) * c_out * chi_q[int(q_in)]
        return flops

    total = 0.0
    if nd.parent >= 0:
        total += count(np.arange(d), np.arange(d))   # environment block Hamiltonian
    for tm in state.terms:
        on = {s for s, _ in tm.ops}
        if not (on & comp) or not (on & set(sites)):
            continue
        A = state._site_factor(tm, sites[0])
        B = state._site_factor(tm, sites[1])
        total += count(row_source(A), row_source(B))
    return total


def expectation(state: TTN, p: _model.Params):
    """<psi|H(p)|psi> for the state's tensors under another coupling set p on
    the same lattice, by renormalizing every bond from scratch (centre moved
    to the root).  Used for E without penalty and for <H_class>."""
    state.move_to(len(state.nodes) - 1)
    other = TTN.__new__(TTN)
    other.__dict__.update(state.__dict__)
    other.p = p
    other.terms, other.const = _model.build_terms(p)
    other.up = [None] * len(state.nodes)
    other.down = [None] * len(state.nodes)
    for nd in state.nodes:
        if nd.parent >= 0:
            other.up[nd.index] = other._up_ops(nd.index)
    return other.energy_at_center()


def energy_gradient(state: TTN, X=None):
    """E(X) = <X|H_eff|X> / <X|X> at the current centre (X defaults to the
    centre tensor) and dE/dX = 2 (H_eff X - E X) / <X|X>: the gradient of a
    Rayleigh quotient of the real symmetric H_eff of Eq. (1) + Eq. (16).
    Test infrastructure (differentiation row)."""
    idx = state.center
    if X is None:
        X = state.T[idx]
    HX = state.heff_apply(idx, X)
    nrm = float(np.vdot(X, X))
    e = float(np.vdot(X, HX)) / nrm
    return e, 2.0 * (HX - e * X) / nrm


COUPLINGS = ("t", "m", "ge2", "cB", "nu")


def coupling_gradient(state: TTN, p: _model.Params):
    """dE/dc for c in (t, m, ge2, cB, nu) at fixed tensors.  Eq. (1) + Eq. (16)
    is linear in each coupling, so dE/dc = <H_c> / c with H_c the terms of
    class c (Hellmann-Feynman); NaN for a zero coupling."""
    out = {}
    for c in COUPLINGS:
        val = getattr(p, c)
        out[c] = expectation(state, _model.class_only(p, c)) / val if val != 0.0 else float("nan")
    return out
