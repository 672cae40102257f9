"""Pins of the oracle's dressed basis and local operators against what the
paper fixes: the 1458 -> 267 count (Methods, after Eq. (14)), the link
algebra of Eq. (5) rebuilt from the rishons of Eq. (6) and the link states
of Eq. (8), Eq. (9) = Eq. (10) on L = 2, the plaquette factorisation
box = -C C C C, Gauss-law closure and monomial structure."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import basis, fock, model


def trinomial(n, s):
    """Coefficient of x^s in (1 + x + x^2)^n, by direct counting."""
    return sum(1 for ks in itertools.product(range(3), repeat=n) if sum(ks) == s)


@pytest.mark.parametrize("parity", [1, -1])
def test_basis_counts(parity):
    table = basis.enumerate_basis(parity)
    assert table.shape == (267, 9)
    assert len(basis.all_configurations()) == 1458
    phi = table[:, 0]
    target = 6 + (1 - parity) // 2
    # phi = 0 rows have sum k = target, phi = 1 rows target - 1
    assert (phi == 0).sum() == trinomial(6, target)
    assert (phi == 1).sum() == trinomial(6, target - 1)
    if parity == 1:
        assert ((phi == 0).sum(), (phi == 1).sum()) == (141, 126)
    else:
        assert ((phi == 0).sum(), (phi == 1).sum()) == (126, 141)
    assert np.all(phi + table[:, 1:7].sum(1) == target)
    assert len({tuple(r) for r in table[:, :7]}) == 267


@pytest.mark.parametrize("parity", [1, -1])
def test_basis_sign_and_charge(parity):
    table = basis.enumerate_basis(parity)
    for row in table:
        n2 = sum(1 for k in row[1:4] if k == 2)
        assert row[7] == (-1) ** n2
        assert row[8] == row[0] - (1 - parity) // 2
    # order: phi outer, then k1..k6 lexicographic
    keys = [tuple(r[:7]) for r in table]
    assert keys == sorted(keys)


def test_link_algebra_eq5_from_rishons():
    """U = eta_x eta_y^dag on the L = 2 link states of Eq. (8) acts as
    Eq. (5) with unit elements; E of Eq. (9) equals Eq. (10)."""
    jx, jy = 0, 3  # two half-links standing in for (x,+mu) and (x+mu,-mu)
    vac = np.zeros(fock.DIM)
    vac[0] = 1.0
    ax, bx = fock.creation(2 * jx + 1), fock.creation(2 * jx + 2)
    ay, by = fock.creation(2 * jy + 1), fock.creation(2 * jy + 2)
    right = -(by @ (ay @ vac))       # |->> = -|0,2>, |2> = b^dag a^dag |0>
    zero = ax @ (ay @ vac)           # |0>  = |1,1> = a_x^dag a_y^dag |0>
    left = bx @ (ax @ vac)           # |<-> = |2,0>
    U = fock.eta(jx) @ fock.eta_dag(jy)
    np.testing.assert_allclose(U @ left, zero, atol=1e-15)
    np.testing.assert_allclose(U @ zero, right, atol=1e-15)
    np.testing.assert_allclose(U @ right, 0.0, atol=1e-15)
    one = fock.identity()
    nx = fock.number(2 * jx + 1) + fock.number(2 * jx + 2)
    ny = fock.number(2 * jy + 1) + fock.number(2 * jy + 2)
    E9 = 0.5 * (ny - nx)
    E10 = one - nx
    for state, e in ((right, 1.0), (zero, 0.0), (left, -1.0)):
        np.testing.assert_allclose(E9 @ state, e * state, atol=1e-15)
        np.testing.assert_allclose(E10 @ state, e * state, atol=1e-15)


def test_eta_is_three_level_raising():
    """Eq. (6): eta^dag maps |0> -> |1> -> |2> -> 0 with unit amplitude
    (alone on the half-link, no other mode occupied)."""
    vac = np.zeros(fock.DIM)
    vac[0] = 1.0
    j = 2
    s1 = fock.creation(2 * j + 1) @ vac
    s2 = fock.creation(2 * j + 2) @ s1
    np.testing.assert_allclose(fock.eta_dag(j) @ vac, s1, atol=1e-15)
    np.testing.assert_allclose(fock.eta_dag(j) @ s1, s2, atol=1e-15)
    np.testing.assert_allclose(fock.eta_dag(j) @ s2, 0.0, atol=1e-15)
    eta3 = fock.eta_dag(j) @ fock.eta_dag(j) @ fock.eta_dag(j)
    assert abs(eta3).max() == 0
    eta2 = fock.eta_dag(j) @ fock.eta_dag(j)
    assert abs(eta2).max() > 0


def test_odd_operator_leaves_gauge_span():
    with pytest.raises(ValueError):
        fock.project(fock.eta_dag(1), 1)


KEYS = [("M", j) for j in range(6)] + [("Md", j) for j in range(6)] + \
       [("C", i, j) for i in range(6) for j in range(6) if i != j] + \
       [("P", j, k) for j in range(6) for k in range(3)] + [("PC", j, k) for j in range(6) for k in range(3)] + \
       [("n",)]


@pytest.mark.parametrize("parity", [1, -1])
def test_local_ops_monomial_and_charge(parity):
    q = basis.charges(parity)
    shift = {"M": 1, "Md": -1, "C": 0, "P": 0, "PC": 0, "n": 0}
    for key in KEYS:
        M = fock.site_op(key, parity).toarray()
        nz = M != 0
        assert nz.sum(0).max() <= 1 and nz.sum(1).max() <= 1
        vals = np.unique(M[nz])
        assert set(vals.tolist()) <= {-1.0, 1.0}
        rows, cols = np.nonzero(M)
        assert np.all(q[rows] - q[cols] == shift[key[0]])
    # hermitian-conjugate pairs
    for j in range(6):
        np.testing.assert_array_equal(fock.site_op(("Md", j), parity).toarray(), fock.site_op(("M", j), parity).toarray().T)
    for i in range(6):
        for j in range(6):
            if i != j:
                np.testing.assert_array_equal(fock.site_op(("C", i, j), parity).toarray(), fock.site_op(("C", j, i), parity).toarray().T)


@pytest.mark.parametrize("parity", [1, -1])
def test_projectors_and_electric(parity):
    table = basis.enumerate_basis(parity)
    for j in range(6):
        tot = sum(fock.site_op(("P", j, k), parity) for k in range(3)).toarray()
        np.testing.assert_array_equal(tot, np.eye(267))
        for k in range(3):
            d = fock.site_op(("P", j, k), parity).diagonal()
            np.testing.assert_array_equal(d, (table[:, 1 + j] == k).astype(float))
    mask = (0, 4, 5)
    d = fock.site_op(("E2", mask), parity).diagonal()
    expect = sum((1 - table[:, 1 + j].astype(float)) ** 2 for j in mask)
    np.testing.assert_array_equal(d, expect)


def _plaquette_space():
    """16-mode Fock space of the 8 half-links of one plaquette."""
    n = 16
    dim = 1 << n
    states = np.arange(dim, dtype=np.int64)

    def cdag(m):
        occ = (states >> m) & 1
        below = states & ((1 << m) - 1)
        par = np.zeros(dim, dtype=np.int64)
        v = below.copy()
        while v.any():
            par ^= v & 1
            v >>= 1
        src = states[occ == 0]
        return sp.csr_matrix((np.where(par[occ == 0] == 1, -1.0, 1.0), (src | (1 << m), src)), shape=(dim, dim))

    def eta_dag(h):
        a, b = cdag(2 * h), cdag(2 * h + 1)
        na, nb = a @ a.T, b @ b.T
        return (na @ b + (sp.identity(dim) - nb) @ a).tocsr()

    return dim, eta_dag


def test_plaquette_factorisation():
    """box = U_{x,mu} U_{x+mu,nu} U^dag_{x+nu,mu} U^dag_{x,nu} equals
    -C_x C_{x+mu} C_{x+mu+nu} C_{x+nu} with the C keys the term list uses,
    as an operator identity on all 2^16 states of the plaquette's
    half-links (any mode order)."""
    dim, eta_dag = _plaquette_space()
    lat = model.Lattice(2, 2, 1)
    (x, mu, nu, a, c, b), = lat.plaquettes()
    # half-link slots: (site, half-link index) -> mode pair id
    slots = [(x, model.plus(mu)), (a, model.minus(mu)), (a, model.plus(nu)), (c, model.minus(nu)),
             (b, model.plus(mu)), (c, model.minus(mu)), (x, model.plus(nu)), (b, model.minus(nu))]
    hid = {s: i for i, s in enumerate(slots)}
    ed = {s: eta_dag(hid[s]) for s in slots}
    e = {s: ed[s].T.tocsr() for s in slots}

    def U(site, m, other):
        return e[(site, model.plus(m))] @ ed[(other, model.minus(m))]

    box = U(x, mu, a) @ U(a, nu, c) @ U(b, mu, c).T @ U(x, nu, b).T
    p = model.Params(2, 2, 1, t=0.0, m=0.0, ge2=0.0, cB=1.0, nu=0.0)
    terms, _ = model.build_terms(p)
    plaq = [tm for tm in terms if tm.cls == "cB"]
    assert len(plaq) == 2
    prods = []
    for tm in plaq:
        op = sp.identity(dim, format="csr")
        for (site, key) in tm.ops:
            _, i, j = key
            op = op @ (ed[(site, i)] @ e[(site, j)])
        prods.append(op)
    # H_plaq = -cB (box + box^dag) must equal the two product terms (coef +cB)
    diff = (prods[0] + prods[1]) + (box + box.T)
    assert abs(diff).max() < 1e-12
    assert abs(box).max() > 0
