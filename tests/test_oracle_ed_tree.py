"""Pins of the oracle's Hamiltonian (through exact diagonalisation), tree,
sector table and seeded initialisation."""
import os

import numpy as np
import pytest

from oracle import ed, model, tree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def closed_form_2x1x1(t, m, ge2):
    """Two sites, one link, Q = 0: {vacuum (-m), pair with E = 1 (m + ge2/2)}
    coupled by -t (Eq. (1) with U of Eq. (5))."""
    return ge2 / 4 - np.sqrt((m + ge2 / 4) ** 2 + t * t)


@pytest.mark.parametrize("t,m,ge2", [(1.0, 1.0, 1.0), (0.7, -0.3, 2.0), (1.3, 0.4, 0.5)])
def test_two_site_closed_form(t, m, ge2):
    p = model.Params(2, 1, 1, t=t, m=m, ge2=ge2, cB=0.0, nu=20.0, Q=0)
    e_closed = closed_form_2x1x1(t, m, ge2)
    assert abs(ed.config_ed(p) - e_closed) < 1e-12
    assert abs(ed.dressed_ed(p)[0] - e_closed) < 1e-10


def test_two_site_reference_value():
    """t = m = ge2 = 1: E0 = 1/4 - sqrt(41)/4."""
    p = model.Params(2, 1, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)
    assert abs(ed.dressed_ed(p)[0] - (-1.3507810593582121)) < 1e-10


def _dangling_all(lat, k=1):
    return [{j: k for j in lat.dangling(s)} for s in range(lat.n_sites)]


@pytest.mark.parametrize("Q", [0, 1, -1])
def test_dressed_vs_configuration_basis_2x2x1(Q):
    """The dressed tensor-product construction (rishons, Eq. (6), (12), the
    factorised plaquette) against a configuration basis with global
    Jordan-Wigner matter and link E fields (Eq. (1), (3)-(5)), block by
    block in the dangling flux."""
    p = model.Params(2, 2, 1, t=0.8, m=0.3, ge2=1.5, cB=0.9, nu=30.0, Q=Q)
    lat = model.Lattice(2, 2, 1)
    best, blocks = ed.config_ed(p, return_blocks=True)
    rng = np.random.default_rng(5 + Q)
    checked = 0
    for F, e_cfg in sorted(blocks.items()):
        if checked >= 4:
            break
        dk = _dangling_all(lat)
        extra = 0.0
        for s, f in enumerate(F):
            d = list(lat.dangling(s))
            for i in range(abs(f)):
                dk[s][d[i]] = 0 if f > 0 else 2
        # spend one non-minimal realisation on a random site: (0, 2) pair
        s = int(rng.integers(lat.n_sites))
        free = [j for j in lat.dangling(s) if dk[s][j] == 1]
        if len(free) >= 2:
            dk[s][free[0]] = 0
            dk[s][free[1]] = 2
            extra = p.ge2
        e_dr = ed.dressed_ed_fixed_dangling(p, dk)[0]
        assert abs(e_dr - (e_cfg + extra)) < 1e-9, (F, e_dr, e_cfg + extra)
        checked += 1
    assert checked >= 2


def test_static_limit():
    """t = 0, no plaquette: E = min(-m N/2, (m + ge2/2) N/2) (Methods,
    scaling analysis), on both sides of m_c = -ge2/4."""
    for m in (0.8, -0.2, -0.6):
        p = model.Params(2, 2, 1, t=0.0, m=m, ge2=1.0, cB=0.0, nu=10.0, Q=0)
        N = 4
        expect = min(-m * N / 2, (m + 0.5) * N / 2)
        assert abs(ed.config_ed(p) - expect) < 1e-12
        lat = model.Lattice(2, 2, 1)
        assert ed.dressed_ed_fixed_dangling(p, _dangling_all(lat))[0] >= expect - 1e-12


def test_hamiltonian_symmetric():
    p = model.Params(2, 1, 1, t=0.9, m=0.4, ge2=1.2, cB=0.3, nu=10.0, Q=0)
    H, _, _ = ed.dressed_hamiltonian(p)
    assert abs(H - H.T).max() < 1e-14


@pytest.mark.parametrize("L,counts", [((2, 1, 1), (2, 1, 0, 10, 1, 1)), ((2, 2, 1), (4, 4, 1, 16, 3, 2)),
                                      ((2, 2, 2), (8, 12, 6, 24, 7, 3)), ((4, 4, 4), (64, 144, 108, 96, 63, 6))])
def test_lattice_and_tree_counts(L, counts):
    lat = model.Lattice(*L)
    nodes = tree.build_tree(*L)
    got = (lat.n_sites, len(lat.links()), len(lat.plaquettes()), sum(len(lat.dangling(s)) for s in range(lat.n_sites)),
           len(nodes), max(n.layer for n in nodes) + 1)
    assert got == counts
    terms, const = model.build_terms(model.Params(*L))
    n_links, n_plaq = counts[1], counts[2]
    assert len(terms) == 2 * lat.n_sites + 5 * n_links + 2 * n_plaq
    assert const == 0.0


def test_tree_structure_4x4x4():
    nodes = tree.build_tree(4, 4, 4)
    lat = model.Lattice(4, 4, 4)
    # bottom nodes pair x-neighbours, left = lower x
    for nd in nodes[:32]:
        (k0, s0), (k1, s1) = nd.children
        assert k0 == k1 == "site"
        c0, c1 = lat.coords(s0), lat.coords(s1)
        assert c1[0] == c0[0] + 1 and c0[1:] == c1[1:]
    axes = [nodes[i].axis for i in (0, 32, 48, 56, 60, 62)]
    assert axes == [0, 1, 2, 0, 1, 2]
    # numbering inside a layer: lowest corner in (z, y, x) order
    for lo_, hi_ in ((0, 32), (32, 48), (48, 56)):
        keys = [(n.lo[2], n.lo[1], n.lo[0]) for n in nodes[lo_:hi_]]
        assert keys == sorted(keys)
    assert nodes[-1].parent == -1
    assert sorted(nodes[-1].sites) == list(range(64))


def test_splitmix64_reference_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            seed, *outs = line.split()
            got = tree.splitmix64(int(seed), 0, len(outs))
            assert [int(v) for v in got] == [int(o, 16) for o in outs]
    # counter form: outputs start+1.. equal the tail of a longer stream
    np.testing.assert_array_equal(tree.splitmix64(7, 3, 5), tree.splitmix64(7, 0, 8)[3:])
    u = tree.uniform_pm1(tree.splitmix64(3, 0, 100000))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


def test_region_counts_total():
    lat = model.Lattice(2, 2, 2)
    d = tree.region_counts(lat, range(8))
    assert sum(d.values()) == 267 ** 8
    # charge-conjugation-like symmetry of the count: D(q) = D(-q) for equal parities
    assert all(d[q] == d[-q] for q in d)


@pytest.mark.parametrize("L,chi,Q", [((2, 2, 2), 8, 0), ((4, 4, 4), 64, 0), ((4, 4, 4), 48, 16), ((4, 4, 4), 32, 4)])
def test_sector_table_properties(L, chi, Q):
    p = model.Params(*L, Q=Q)
    nodes = tree.build_tree(*L)
    bonds = tree.sector_table(p, chi, nodes)
    lat = model.Lattice(*L)
    for nd in nodes:
        legs = [tree.leg_sectors(lat, bonds, c) for c in nd.children]
        rows = {}
        for qa, da in legs[0].items():
            for qb, db in legs[1].items():
                rows[qa + qb] = rows.get(qa + qb, 0) + da * db
        for q, c in bonds[nd.index].items():
            assert 0 < c <= rows.get(q, 0), (nd.index, q)
        if nd.parent >= 0:
            assert sum(bonds[nd.index].values()) <= chi
    root = nodes[-1]
    l, r = [cid for (_, cid) in root.children]
    assert {q: c for q, c in bonds[l].items()} == {Q - q: c for q, c in bonds[r].items()}
    assert bonds[root.index] == {Q: 1}


def test_allocation_rule_small():
    """Largest remainder by hand: w = (1, 2, 1), chi = 4 -> ideal 1, 2, 1;
    chi = 5 -> 1.25, 2.5, 1.25 -> floors 1, 2, 1, remainder to q = 0."""
    w = {-1: 1, 0: 2, 1: 1}
    cap = {-1: 10, 0: 10, 1: 10}
    assert tree.allocate(4, w, cap, 1, 2, 0) == {-1: 1, 0: 2, 1: 1}
    assert tree.allocate(5, w, cap, 1, 2, 0) == {-1: 1, 0: 3, 1: 1}
    # ties in remainder and distance: lower q wins
    assert tree.allocate(6, w, cap, 1, 2, 0) == {-1: 2, 0: 3, 1: 1}
    # caps bind and the surplus moves on
    assert tree.allocate(6, w, {-1: 10, 0: 1, 1: 10}, 1, 2, 0) == {-1: 3, 0: 1, 1: 2}


def test_penalty_rewrite_equals_eq16():
    """nu sum_k P^k_x (1 - P^{2-k}_y) equals nu (1 - delta_{2, k_x + k_y}) on
    every two-site state (Eq. (16))."""
    from oracle import fock
    p = model.Params(2, 1, 1, t=0.0, m=0.0, ge2=0.0, cB=0.0, nu=7.0, Q=0)
    terms, const = model.build_terms(p)
    assert const == 0.0
    tabs = [np.asarray(fock.site_op(("P", 3, 0), s).diagonal()) for s in (1, -1)]
    from oracle import basis
    b0, b1 = basis.enumerate_basis(1), basis.enumerate_basis(-1)
    H = np.zeros((267, 267))
    for tm in terms:
        (s0, k0), (s1, k1) = tm.ops
        d0 = fock.site_op(k0, 1).diagonal()
        d1 = fock.site_op(k1, -1).diagonal()
        H += tm.coef * np.outer(d0, d1)
    L = b0[:, 1 + 3][:, None] + b1[:, 1 + 0][None, :]
    np.testing.assert_array_equal(H, 7.0 * (L != 2))


def test_qr_positive():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((40, 7))
    Qm, R = tree.qr_positive(A)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Qm @ R, A, atol=1e-13)
    np.testing.assert_allclose(Qm.T @ Qm, np.eye(7), atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0)


def test_qr_sector_full_rank_equals_householder():
    rng = np.random.default_rng(3)
    for m, n in ((50, 7), (9, 9), (300, 32)):
        A = rng.standard_normal((m, n))
        Q1, R1 = tree.qr_positive(A)
        Q2, R2 = tree.qr_gram_schmidt(A)
        np.testing.assert_allclose(Q2, Q1, atol=1e-12)
        np.testing.assert_allclose(R2, R1, atol=1e-12)
        Q3, R3 = tree.qr_sector(A)
        np.testing.assert_array_equal(Q3, Q1)


def test_qr_sector_rank_deficient():
    # hand example: second column zero -> R_11 = 0, q_1 completed by e_1
    X = np.array([[2.0, 0.0], [0.0, 0.0], [0.0, 0.0]])
    Q, R = tree.qr_sector(X)
    np.testing.assert_array_equal(Q, np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]]))
    np.testing.assert_array_equal(R, np.array([[2.0, 0.0], [0.0, 0.0]]))
    # general: rank 3 of 6 columns, noise far below the dependency threshold
    rng = np.random.default_rng(4)
    B = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 6))
    B += 1e-13 * rng.standard_normal(B.shape)
    Q, R = tree.qr_sector(B)
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(Q @ R, B, atol=1e-8)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.all(np.diag(R) >= 0)
    assert np.sum(np.diag(R) == 0) == 3
    with pytest.raises(ValueError):
        tree.qr_sector(rng.standard_normal((3, 5)))


def test_sweep_order_2x2x2_by_hand():
    """2x2x2: bottom nodes 0,1 (children of 4) and 2,3 (children of 5) in
    depth-first order, layer 1 walked backwards, then the root."""
    assert tree.sweep_order(tree.build_tree(2, 2, 2)) == [0, 1, 2, 3, 5, 4, 6]


@pytest.mark.parametrize("L", [(4, 4, 4), (8, 8, 8)])
def test_sweep_order_properties(L):
    """A permutation of the nodes, layers bottom-up, siblings adjacent in
    the bottom layer, and fewer bond moves than number order."""
    nodes = tree.build_tree(*L)
    order = tree.sweep_order(nodes)
    assert sorted(order) == list(range(len(nodes)))
    layers = [nodes[i].layer for i in order]
    assert layers == sorted(layers)
    parent = {nd.index: nd.parent for nd in nodes}
    bottom = [i for i in order if nodes[i].layer == 0]
    for a, b in zip(bottom[0::2], bottom[1::2]):
        assert parent[a] == parent[b]

    def dist(a, b):
        up = []
        while a >= 0:
            up.append(a)
            a = parent[a]
        steps = 0
        while b not in up:
            b = parent[b]
            steps += 1
        return steps + up.index(b)

    def moves(seq):
        return sum(dist(x, y) for x, y in zip([len(nodes) - 1] + list(seq[:-1]), seq))

    assert moves(order) < moves(list(range(len(nodes))))


def _strong(g2, Q=0):
    c = dict(t=1.0, m=1.0, ge2=g2, cB=1.0 / (2.0 * g2), nu=10.0 * max(1.0, g2 / 2.0))
    return model.Params(2, 2, 1, Q=Q, **c)


def test_strong_coupling_second_order():
    """g^2 -> infinity (Q = 0): the ground state is the bare staggered vacuum,
    E0 = -m N / 2, and second-order perturbation theory in t adds, per link,
    -t^2 / (2 m + g^2 / 2) (one hop creates a particle-antiparticle pair, cost
    2m, joined by one unit of electric flux, cost g^2/2).  The exact energy's
    second-order part tends to that value with a relative error that falls
    at least 4x for every 4x in g^2."""
    n_sites, n_links, m, t = 4, 4, 1.0, 1.0
    e0 = -m * n_sites / 2.0
    errs = []
    for g2 in (10.0, 40.0, 160.0):
        e = ed.config_ed(_strong(g2))
        ept = e0 - n_links * t * t / (2.0 * m + g2 / 2.0)
        errs.append(abs((e - e0) / (ept - e0) - 1.0))
        assert e < e0
    assert errs[2] < 1e-3
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4
