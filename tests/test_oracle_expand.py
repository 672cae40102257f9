"""Pins of the oracle's single-tensor optimisation with subspace expansion
(Methods, "Tensor Networks": the bond dimension grows during the sweeps and
the symmetry sectors adapt): an expanded move leaves the state unchanged
when nothing is truncated, in both directions of a bond; the new tensor is an
isometry and both ends of the bond carry the same charges; from bond
dimension 2 (where plain sweeps stay far above the exact energy) and from a
single charge sector per bond, expanded sweeps reach the independent
configuration-basis ground energy; truncation respects chi_max and stays
variational."""
import numpy as np
import pytest

from oracle import ed, expand, model, ttn

P = model.Params(2, 2, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)


@pytest.fixture(scope="module")
def e_ed():
    return ed.config_ed(P)


def _isometric(T, leg):
    Tm = np.moveaxis(T, leg, 2).reshape(-1, T.shape[leg])
    return np.max(np.abs(Tm.T @ Tm - np.eye(T.shape[leg])))


@pytest.mark.parametrize("start,target", [(0, 2), (2, 1)])
def test_expanded_move_keeps_the_state(start, target):
    s = ttn.TTN(P, 4, 0)
    s.move_to(start)
    e0, n0 = s.energy_at_center(), s.norm_at_center()
    c = s.center
    leg_c = s._neighbour_leg(c, target)
    leg_t = s._neighbour_leg(target, c)
    dims = expand.expand_move(s, target, 0.05, 1000, 0.0)
    assert s.center == target
    assert abs(s.energy_at_center() - e0) < 1e-11 * abs(e0)
    assert abs(s.norm_at_center() - n0) < 1e-12
    assert _isometric(s.T[c], leg_c) < 1e-12
    assert np.array_equal(s.labels[c][leg_c], s.labels[target][leg_t])
    assert sum(dims.values()) == s.T[c].shape[leg_c]
    if start == 0:
        # leaving a bottom node upwards the bond grows and gains charge sectors
        assert sum(dims.values()) > 3 and len(dims) > 1


def test_zero_alpha_keeps_the_bond():
    s = ttn.TTN(P, 4, 0)
    s.move_to(0)
    before = dict(s.bonds[0])
    e0 = s.energy_at_center()
    dims = expand.expand_move(s, 2, 0.0, 1000)
    assert dims == before
    assert abs(s.energy_at_center() - e0) < 1e-11 * abs(e0)


def test_expansion_reaches_exact_energy_from_chi_2(e_ed):
    plain = ttn.TTN(P, 2, 0)
    plain.sweep(tol=1e-10)
    assert plain.sweep(tol=1e-10)[-1] > e_ed + 0.1
    s = ttn.TTN(P, 2, 0)
    es = expand.sweep_expanded(s, 1e-10, 1e-3, 12)
    assert abs(es[-1] - e_ed) < 1e-10 * abs(e_ed)
    for idx in (0, 1):
        assert _isometric(s.T[idx], 2) < 1e-12


def test_sectors_adapt_from_one_sector_per_bond(e_ed):
    s = ttn.TTN(P, 1, 0)
    assert all(len(b) == 1 for b in s.bonds)
    for _ in range(3):
        es = expand.sweep_expanded(s, 1e-10, 1e-3, 12)
    assert len(s.bonds[0]) == 3 and len(s.bonds[1]) == 3
    assert abs(es[-1] - e_ed) < 1e-9 * abs(e_ed)


def test_truncation_respects_chi_max(e_ed):
    s = ttn.TTN(P, 4, 0)
    es = expand.sweep_expanded(s, 1e-10, 1e-3, 3)
    assert all(sum(b.values()) <= 3 for b in s.bonds)
    assert es[-1] > e_ed


@pytest.mark.parametrize("start,target,boundary", [(4, 0, 0), (4, 6, 0), (1, 4, 1)])
def test_expanded_move_deep_tree(start, target, boundary):
    """2x2x2 (three layers), open and periodic: untruncated expanded moves
    down from a middle node, up to the root and up from a bottom node keep
    the state; the operators rebuilt on the new bond give the same H_eff
    expectation as a from-scratch recomputation."""
    p = model.Params(2, 2, 2, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0, boundary=boundary)
    s = ttn.TTN(p, 4, 1)
    s.move_to(start)
    e0 = s.energy_at_center()
    expand.expand_move(s, target, 0.05, 1000, 0.0)
    assert abs(s.energy_at_center() - e0) < 1e-11 * abs(e0)
    # back to the root with SVD moves (a new sector may still be empty on
    # one side, which a plain QR move cannot factorise), then every bond
    # operator recomputed from scratch
    for nxt in s.path(s.center, len(s.nodes) - 1)[1:]:
        expand.expand_move(s, nxt, 0.0, 1000)
    assert abs(ttn.expectation(s, p) - e0) < 1e-11 * abs(e0)


@pytest.mark.parametrize("Q", [1, -1])
def test_expansion_at_finite_charge(Q):
    """2x2x1 with one net charge: from chi = 2 one expanded sweep reaches the
    configuration-basis ground energy of that charge sector, with bond
    sectors that are no longer symmetric about zero."""
    p = model.Params(2, 2, 1, t=0.8, m=0.3, ge2=1.5, cB=0.9, nu=20.0, Q=Q)
    s = ttn.TTN(p, 2, 3)
    es = expand.sweep_expanded(s, 1e-10, 1e-3, 16)
    e_ed = ed.config_ed(p)
    assert abs(es[-1] - e_ed) < 1e-10 * abs(e_ed)
    assert s.bonds[-1] == {Q: 1}
    assert s.bonds[1].get(Q, 0) > s.bonds[1].get(-Q, 0)
