"""CPU tests of the C-ABI library: it loads, exports every entry point that
include/qedttn.h declares, and its host-side model (basis, monomial site
operators, term list, tree, sector table) equals the oracle's bit for bit.
No GPU call is made here."""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import basis as obasis
from oracle import fock as ofock
from oracle import model as omodel
from oracle import tree as otree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qedttn.h")


@pytest.fixture(scope="module")
def q():
    import paper_2011_10658_gb300 as pkg
    from paper_2011_10658_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2011_10658_gb300 import build
        build.build()
    pkg.lib()
    return pkg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:qed|ttn)_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(q):
    from paper_2011_10658_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T ((?:qed|ttn)_\w+)", out))
    assert set(names) <= exported, set(names) - exported
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(names) == bound


@pytest.mark.parametrize("parity", [1, -1])
def test_basis_bit_exact(q, parity):
    np.testing.assert_array_equal(q.basis(parity), obasis.enumerate_basis(parity))


def _dense(src, val):
    M = np.zeros((267, 267))
    for r in range(267):
        if src[r] >= 0:
            M[r, src[r]] = val[r]
    return M


KEYS = [(("M", j), ("M", j, 0)) for j in range(6)] + [(("Md", j), ("MD", j, 0)) for j in range(6)] + \
       [(("C", i, j), ("C", i, j)) for i in range(6) for j in range(6) if i != j] + \
       [(("P", j, k), ("P", j, k)) for j in range(6) for k in range(3)] + \
       [(("PC", j, k), ("PC", j, k)) for j in range(6) for k in range(3)] + [(("n",), ("N", 0, 0))]


@pytest.mark.parametrize("parity", [1, -1])
def test_local_ops_bit_exact(q, parity):
    """Closed-form Jordan-Wigner signs (native) against the literal Fock
    construction of Eq. (6) and Eq. (12) (oracle)."""
    for okey, (kind, j1, j2) in KEYS:
        src, val = q.local_op(parity, kind, j1, j2)
        np.testing.assert_array_equal(_dense(src, val), ofock.site_op(okey, parity).toarray(), err_msg=str(okey))
    mask = (1 << 0) | (1 << 4) | (1 << 5)
    src, val = q.local_op(parity, "E2", mask, 0)
    np.testing.assert_array_equal(_dense(src, val), ofock.site_op(("E2", (0, 4, 5)), parity).toarray())


def test_local_op_errors(q):
    from paper_2011_10658_gb300 import QedError
    with pytest.raises(QedError):
        q.local_op(2, "M", 0)
    with pytest.raises(QedError):
        q.local_op(1, "M", 7)
    with pytest.raises(QedError):
        q.local_op(1, "C", 2, 2)


KIND = {"M": 1, "Md": 2, "C": 3, "P": 4, "n": 5, "E2": 6, "PC": 8}
CLS = {"t": 0, "m": 1, "ge2": 2, "cB": 3, "nu": 4, "mu": 5}


def _oracle_terms(p):
    terms, const = omodel.build_terms(p)
    rows = []
    for tm in terms:
        ops = []
        for (s, key) in tm.ops:
            k = key[0]
            if k in ("M", "Md"):
                ops.append((s, KIND[k], key[1], 0))
            elif k == "C":
                ops.append((s, KIND[k], key[1], key[2]))
            elif k in ("P", "PC"):
                ops.append((s, KIND[k], key[1], key[2]))
            elif k == "n":
                ops.append((s, KIND[k], 0, 0))
            else:
                ops.append((s, KIND[k], sum(1 << j for j in key[1]), 0))
        # factors act on different sites and commute: compare them in site order
        rows.append((tm.coef, CLS[tm.cls], tuple(sorted(ops))))
    return rows, const


@pytest.mark.parametrize("L,Q,boundary,with_mu", [((2, 1, 1), 0, 0, False), ((2, 2, 1), 1, 0, False),
                                                  ((2, 2, 2), 0, 0, False), ((4, 4, 4), 4, 0, False),
                                                  ((2, 1, 1), 0, 1, False), ((2, 2, 1), 0, 1, True),
                                                  ((2, 2, 2), 0, 1, False), ((4, 2, 2), 2, 1, True),
                                                  ((4, 4, 4), 0, 1, False), ((4, 4, 4), 0, 0, True)])
def test_term_list_equal(q, L, Q, boundary, with_mu):
    kw = dict(t=0.9, m=-0.4, ge2=1.3, cB=0.35, nu=12.0, Q=Q)
    n = L[0] * L[1] * L[2]
    mu = tuple(np.round(np.random.default_rng(n).uniform(-2, 2, n), 3)) if with_mu else ()
    if with_mu:
        mu = tuple(0.0 if i % 5 == 0 else float(v) for i, v in enumerate(mu))   # zeros give no term
    m = q.Model(*L, boundary=boundary, mu=(mu if with_mu else None), **kw)
    coef, cls, nops, ops = m.terms()
    native = []
    for i in range(len(coef)):
        native.append((coef[i], int(cls[i]), tuple(tuple(int(v) for v in ops[i, f]) for f in range(nops[i]))))
    ref, const = _oracle_terms(omodel.Params(*L, boundary=boundary, mu=mu, **kw))
    assert native == ref
    assert m.info()["constant"] == const


@pytest.mark.parametrize("L", [(2, 1, 1), (2, 2, 1), (2, 2, 2), (4, 4, 4), (8, 8, 8)])
def test_tree_equal(q, L):
    t = q.Model(*L).tree()
    nodes = otree.build_tree(*L)
    assert t.shape[0] == len(nodes)
    for row, nd in zip(t, nodes):
        kinds = [0 if k == "site" else 1 for (k, _) in nd.children]
        ids = [c for (_, c) in nd.children]
        assert tuple(row) == (nd.layer, nd.axis, kinds[0], ids[0], kinds[1], ids[1], nd.parent)


@pytest.mark.parametrize("L,chi,Q", [((2, 2, 2), 8, 0), ((2, 2, 1), 12, 0), ((4, 4, 4), 64, 0),
                                     ((4, 4, 4), 48, 16), ((4, 4, 4), 32, 4), ((4, 4, 4), 48, 6),
                                     ((4, 4, 4), 48, 2), ((4, 4, 4), 48, 10), ((4, 4, 4), 48, 14),
                                     ((4, 4, 4), 1, 0), ((2, 2, 1), 4, 2)])
def test_sector_table_equal(q, L, chi, Q):
    assert q.Model(*L, Q=Q).sectors(chi) == otree.sector_table(omodel.Params(*L, Q=Q), chi)


def test_model_errors(q):
    from paper_2011_10658_gb300 import QedError
    with pytest.raises(QedError):
        q.Model(3, 2, 2)
    with pytest.raises(QedError):
        q.Model(2, 2, 2, boundary=2)
    with pytest.raises(QedError):
        q.Model(2, 2, 2, mu=[0.5] * 7)
    with pytest.raises(QedError):
        q.Model(2, 2, 2, mu=[0.5] * 7 + [float("inf")])
    with pytest.raises(QedError):
        q.Model(2, 2, 2, t=float("nan"))


@pytest.mark.parametrize("L", [(2, 1, 1), (2, 2, 1), (2, 2, 2), (4, 4, 4), (8, 8, 8)])
def test_sweep_order_equal(q, L):
    assert q.Model(*L).sweep_order().tolist() == otree.sweep_order(otree.build_tree(*L))
