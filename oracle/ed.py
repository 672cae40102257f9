"""Exact-diagonalisation references.  Test infrastructure only.

Two independent constructions of the ground-state energy of Eq. (1) on tiny
open lattices:

``dressed_ed``  the full tensor product of 267-dimensional dressed sites with
                the product terms of ``oracle.model`` (penalty included),
                restricted to total charge Q.  Feasible for two sites
                (71289 states).

``config_ed``   a configuration basis that never mentions rishons: matter
                occupations with global Jordan-Wigner ordering (site index
                order), link electric fields E in {-1, 0, 1} with U raising
                E by one with unit amplitude (Eq. (4)-(5)), Gauss's law of
                Eq. (3) at every site.  Net flux F_x leaving site x through
                its dangling half-links is fixed by Gauss's law; the cheapest
                dangling configuration realising F_x costs (ge2/2)|F_x|, and
                dangling occupations are conserved, so the ground energy is
                the minimum over F-blocks.  This shares no operator code with
                the dressed construction, so agreement pins the signs of
                Eq. (6), (8), (12) and of the plaquette factorisation.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis as _basis
from . import fock as _fock
from . import model as _model


def dressed_hamiltonian(p):
    """Sparse H on the full dressed space of a lattice with N sites
    (267^N states; use N <= 2).  Returns (H, charge vector, constant)."""
    lat = _model.lattice(p)
    n = lat.n_sites
    if n > 2:
        raise ValueError("dressed ED is limited to two sites")
    terms, const = _model.build_terms(p)
    eye = sp.identity(_basis.D_LOCAL, format="csr")
    dim = _basis.D_LOCAL ** n
    H = sp.csr_matrix((dim, dim))
    for tm in terms:
        factors = [eye] * n
        for (s, key) in tm.ops:
            factors[s] = _fock.site_op(key, lat.parity(s))
        op = factors[0]
        for f in factors[1:]:
            op = sp.kron(op, f, format="csr")
        H = H + tm.coef * op
    H = H + const * sp.identity(dim, format="csr")
    q = np.zeros(1, dtype=np.int64)
    for s in range(n):
        q = (q[:, None] + _basis.charges(lat.parity(s))[None, :]).ravel()
    return H.tocsr(), q, const


def dressed_ed(p, k=1):
    """Lowest k eigenvalues of the dressed-space H in charge sector p.Q."""
    H, q, _ = dressed_hamiltonian(p)
    sel = np.nonzero(q == p.Q)[0]
    Hq = H[sel][:, sel]
    if Hq.shape[0] <= 2000:
        return np.linalg.eigvalsh(Hq.toarray())[:k]
    vals = spla.eigsh(Hq, k=k, which="SA", tol=1e-13, return_eigenvectors=False)
    return np.sort(vals)


def _config_blocks(p):
    """Enumerate Gauss-law configurations (phi, E) grouped by dangling flux F."""
    lat = _model.lattice(p)
    n = lat.n_sites
    links = lat.links()
    ndang = [len(lat.dangling(s)) for s in range(n)]
    par = [lat.parity(s) for s in range(n)]
    blocks = {}
    for phis in itertools.product((0, 1), repeat=n):
        qs = [phis[s] - (1 - par[s]) // 2 for s in range(n)]
        if sum(qs) != p.Q:
            continue
        for Es in itertools.product((-1, 0, 1), repeat=len(links)):
            # Gauss, Eq. (3): q_x = sum of outgoing internal E + dangling outflow
            div = [0] * n
            for (x, mu, y), e in zip(links, Es):
                div[x] += e
                div[y] -= e
            F = tuple(qs[s] - div[s] for s in range(n))
            if any(abs(F[s]) > ndang[s] for s in range(n)):
                continue
            blocks.setdefault(F, []).append((phis, Es))
    return lat, links, blocks


def _jw_sign(occ, s):
    """(-1)^(number of occupied modes with index < s)."""
    return -1 if sum(occ[:s]) % 2 else 1


def config_block_hamiltonian(p, lat, links, states):
    index = {st: i for i, st in enumerate(states)}
    n = lat.n_sites
    link_id = {(x, mu): li for li, (x, mu, y) in enumerate(links)}
    rows, cols, vals = [], [], []

    def add(i, j, v):
        rows.append(i)
        cols.append(j)
        vals.append(v)

    for i, (phis, Es) in enumerate(states):
        diag = sum(p.m * lat.parity(s) * phis[s] for s in range(n))
        diag += 0.5 * p.ge2 * sum(e * e for e in Es)
        add(i, i, diag)
        # hopping psi_x^dag U_{x,mu} psi_y + h.c.
        for li, (x, mu, y) in enumerate(links):
            # forward: needs phi_y = 1, phi_x = 0, E < 1
            if phis[y] == 1 and phis[x] == 0 and Es[li] < 1:
                occ = list(phis)
                sgn = _jw_sign(occ, y)
                occ[y] = 0
                sgn *= _jw_sign(occ, x)
                occ[x] = 1
                E2 = list(Es)
                E2[li] += 1
                j = index.get((tuple(occ), tuple(E2)))
                if j is not None:
                    add(j, i, -p.t * sgn)
                    add(i, j, -p.t * sgn)
        # plaquette -cB (box + box^dag); box raises E on (x,mu), (x+mu,nu),
        # lowers E on (x+nu,mu), (x,nu)
        for (x, mu, nu, a, c, b) in lat.plaquettes():
            up1 = link_id[(x, mu)]
            up2 = link_id[(a, nu)]
            dn1 = link_id[(b, mu)]
            dn2 = link_id[(x, nu)]
            E2 = list(Es)
            ok = E2[up1] < 1 and E2[up2] < 1 and E2[dn1] > -1 and E2[dn2] > -1
            if ok:
                E2[up1] += 1
                E2[up2] += 1
                E2[dn1] -= 1
                E2[dn2] -= 1
                j = index.get((phis, tuple(E2)))
                if j is not None:
                    add(j, i, -p.cB)
                    add(i, j, -p.cB)
    m = len(states)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def config_ed(p, return_blocks=False):
    """Ground energy of Eq. (1) (L = 2 on every internal link, so no
    penalty) on an open lattice, minimised over dangling-flux blocks."""
    lat, links, blocks = _config_blocks(p)
    best = np.inf
    per_block = {}
    for F, states in blocks.items():
        H = config_block_hamiltonian(p, lat, links, states)
        e0 = np.linalg.eigvalsh(H.toarray())[0] if H.shape[0] <= 3000 else spla.eigsh(H, k=1, which="SA")[0][0]
        e0 += 0.5 * p.ge2 * sum(abs(f) for f in F)
        per_block[F] = e0
        best = min(best, e0)
    if return_blocks:
        return best, per_block
    return best


def dressed_ed_fixed_dangling(p, dangling_k, k=1):
    """Lowest eigenvalues of the dressed-space H restricted to one dangling
    configuration.  ``dangling_k[s]`` maps each dangling half-link of site s
    to its fixed occupation k.  Dangling occupations are conserved by every
    term, so this block is an exact invariant subspace.  Feasible for a few
    sites (each site keeps only its rows matching ``dangling_k[s]``)."""
    lat = _model.lattice(p)
    n = lat.n_sites
    keep = []
    for s in range(n):
        table = _basis.enumerate_basis(lat.parity(s))
        ok = np.ones(table.shape[0], dtype=bool)
        for j, kv in dangling_k[s].items():
            ok &= table[:, 1 + j] == kv
        keep.append(np.nonzero(ok)[0])
    terms, const = _model.build_terms(p)
    dims = [len(kk) for kk in keep]
    dim = int(np.prod(dims))
    H = sp.csr_matrix((dim, dim))
    for tm in terms:
        factors = [sp.identity(d, format="csr") for d in dims]
        for (s, key) in tm.ops:
            full = _fock.site_op(key, lat.parity(s))
            factors[s] = full[keep[s]][:, keep[s]]
        op = factors[0]
        for f in factors[1:]:
            op = sp.kron(op, f, format="csr")
        H = H + tm.coef * op
    H = H + const * sp.identity(dim, format="csr")
    q = np.zeros(1, dtype=np.int64)
    for s in range(n):
        qs = _basis.charges(lat.parity(s))[keep[s]]
        q = (q[:, None] + qs[None, :]).ravel()
    sel = np.nonzero(q == p.Q)[0]
    Hq = H.tocsr()[sel][:, sel]
    if Hq.shape[0] <= 3000:
        return np.linalg.eigvalsh(Hq.toarray())[:k]
    return np.sort(spla.eigsh(Hq, k=k, which="SA", tol=1e-13, return_eigenvectors=False))
