"""Degenerate cases of the method on the GPU against the oracle: bond
dimension 1 (a product of bottom-node pairs) deep in the strong-coupling
regime, the largest charge a 2x2x1 lattice holds (one sector per bond), and
the smallest Krylov space (two vectors, explicit restarts)."""
import numpy as np
import pytest

from oracle import model as omodel, ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as pkg
    pkg.lib()
    return pkg


def _sweep_pair(q, L, chi, seed, kw, tol=1e-12, max_krylov=64, sweeps=1):
    p = omodel.Params(*L, **kw)
    ref = ottn.TTN(p, chi, seed)
    s = q.TTN(q.Model(*L, **kw), chi, seed=seed)
    for _ in range(sweeps):
        e_ref = ref.sweep(tol=tol)[-1]
        e = s.sweep(1, tol=tol, max_krylov=max_krylov, allow_noconv=True)["energy"]
    return e, e_ref


def test_chi1_strong_coupling(q):
    g2 = 40.0
    kw = dict(t=1.0, m=1.0, ge2=g2, cB=1.0 / (2.0 * g2), nu=20.0, Q=0)
    e, e_ref = _sweep_pair(q, (2, 2, 1), 1, 0, kw, sweeps=2)
    assert abs(e - e_ref) < 1e-10 * abs(e_ref)
    assert e <= -2.0


def test_largest_charge_2x2x1(q):
    """Q = 2 on 2x2x1: both even sites occupied and both odd sites empty of
    antiparticles is the only matter content; every bond has one sector."""
    kw = dict(t=1.0, m=0.5, ge2=1.0, cB=0.5, nu=10.0, Q=2)
    m = q.Model(2, 2, 1, **kw)
    assert all(len(b) == 1 for b in m.sectors(4)[:-1])
    e, e_ref = _sweep_pair(q, (2, 2, 1), 4, 1, kw)
    assert abs(e - e_ref) < 1e-10 * abs(e_ref)


def test_two_vector_krylov_space(q):
    """max_krylov = 2: no room for a thick restart, explicit restarts from the
    Ritz vector (close to steepest descent).  Fifty restarts do not converge a
    two-site update, which the stats must flag; the energies stay variational
    (above the exact ground state) and the state stays isometric."""
    from oracle import ed
    kw = dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)
    p = omodel.Params(2, 2, 1, **kw)
    s = q.TTN(q.Model(2, 2, 1, **kw), 6, seed=2)
    e_start = s.energy()[0]
    st = s.sweep(1, tol=1e-6, max_krylov=2, allow_noconv=True)
    assert np.isfinite(st["energy"])
    assert st["not_converged"] > 0
    assert ed.config_ed(p) - 1e-9 <= st["energy"] < e_start
    assert abs(s.energy()[0] - st["energy"]) < 1e-9 * abs(st["energy"])
