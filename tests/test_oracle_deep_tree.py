"""Pins of the oracle's renormalized operators on trees of three and four
layers (2x2x2 and 4x2x2), where the environment operators of a node are
built from its parent's environment (the grandparent branch of
``TTN._down_ops``) and the upward operators of a node from its children's
upward operators.

Energy seen from every centre: with all other tensors isometric towards the
centre, <psi|H|psi> is the same number wherever the centre sits (Methods,
"Tensor Networks": the tree is kept in the isometric gauge).  The reference
value comes from ``expectation``, which rebuilds only the upward operators
from scratch and evaluates at the root; the value at a deep node goes
through the chain of downward operators.  A crossing term dropped from, or
counted twice in, any downward operator changes the energy at the nodes
below it by that term's expectation value in the (random, non-eigen) start
state, so the check fails; ``test_planted_*`` shows that it does.

Surface layers of sigma(l) (Eq. (16a)): counted by hand on 4x4x4 (56
surface sites, 8 interior) and 8x8x8 (296, 152, 56, 8)."""
import numpy as np
import pytest

import workloads
from oracle import model, ttn


def _state(L, chi, seed=0):
    p = model.Params(*L, Q=0, **workloads.qed_couplings(1.0))
    return p, ttn.TTN(p, chi, seed)


def _isometric_towards_centre(s):
    worst = 0.0
    for nd in s.nodes:
        if nd.index == s.center:
            continue
        T = s.T[nd.index]
        leg = s._neighbour_leg(nd.index, s.path(nd.index, s.center)[1])
        A = np.moveaxis(T, leg, 2).reshape(-1, T.shape[leg])
        worst = max(worst, float(np.max(np.abs(A.T @ A - np.eye(A.shape[1])))))
    return worst


def _centre_errors(s, e_ref):
    errs = {}
    for c in range(len(s.nodes)):
        s.move_to(c)
        errs[c] = abs(s.energy_at_center() - e_ref) / abs(e_ref)
    return errs


@pytest.mark.parametrize("L,chi", [((2, 2, 2), 6), ((4, 2, 2), 4)])
def test_energy_at_every_centre_equals_upward_only_value(L, chi):
    p, s = _state(L, chi)
    layers = {nd.layer for nd in s.nodes}
    assert len(layers) >= 3
    e_ref = ttn.expectation(s, p)
    for c in range(len(s.nodes)):
        s.move_to(c)
        e = s.energy_at_center()
        assert abs(e - e_ref) <= 1e-11 * abs(e_ref), (c, e, e_ref)
        assert abs(s.norm_at_center() - 1.0) < 1e-12
        assert _isometric_towards_centre(s) < 1e-12


@pytest.mark.parametrize("L,chi", [((2, 2, 2), 6), ((4, 2, 2), 4)])
def test_class_energies_add_up_at_deep_nodes(L, chi):
    """Eq. (1) + Eq. (16) are linear in the couplings: the class energies sum
    to the total, from the root (upward operators) and from a bottom node
    (downward operators of a class-only copy)."""
    p, s = _state(L, chi)
    total = ttn.expectation(s, p)
    parts = [ttn.expectation(s, model.class_only(p, c)) for c in ttn.COUPLINGS]
    assert abs(sum(parts) - total) <= 1e-11 * abs(total)
    # the same split seen from bottom node 0 through the downward operators
    got = []
    for c in ttn.COUPLINGS:
        q = model.class_only(p, c)
        other = ttn.TTN(q, chi, 0)
        other.move_to(0)
        got.append(other.energy_at_center())
    np.testing.assert_allclose(got, parts, rtol=1e-11, atol=1e-11 * abs(total))


def test_planted_dropped_crossing_term_is_detected(monkeypatch):
    """Drop one crossing term from the downward operators of every node whose
    parent is not the root; the energy seen from those nodes moves away
    from the upward-only value."""
    p, s = _state((2, 2, 2), 6)
    e_ref = ttn.expectation(s, p)
    original = ttn.TTN._down_ops

    def dropped(self, idx):
        out = original(self, idx)
        if self.nodes[self.nodes[idx].parent].parent >= 0:
            # the crossing operator of largest norm (a penalty projector)
            k = max((key for key in out if key != "H"), key=lambda key: np.linalg.norm(out[key]))
            out[k] = np.zeros_like(out[k])
        return out

    monkeypatch.setattr(ttn.TTN, "_down_ops", dropped)
    errs = _centre_errors(s, e_ref)
    bottom = [nd.index for nd in s.nodes if nd.layer == 0]
    assert max(errs[c] for c in bottom) > 1e-6


def test_planted_missing_grandparent_hamiltonian_is_detected(monkeypatch):
    """Leave out the parent's environment Hamiltonian (the grandparent
    branch); the energy at the bottom nodes changes."""
    p, s = _state((2, 2, 2), 6)
    e_ref = ttn.expectation(s, p)
    original = ttn.TTN._down_ops

    def no_grandparent(self, idx):
        out = original(self, idx)
        par = self.nodes[self.nodes[idx].parent]
        if par.parent >= 0:
            leg = 0 if par.children[0] == ("node", idx) else 1
            out["H"] = out["H"] - ttn.renormalize(self.T[par.index], {2: self.down[par.index]["H"]}, leg)
        return out

    monkeypatch.setattr(ttn.TTN, "_down_ops", no_grandparent)
    errs = _centre_errors(s, e_ref)
    assert max(errs[nd.index] for nd in s.nodes if nd.layer == 0) > 1e-6


def test_planted_double_counted_upward_term_is_detected(monkeypatch):
    """Count one crossing term twice in the upward operators of the layer-1
    nodes (children that are nodes); the root energy moves."""
    p, s = _state((2, 2, 2), 6)
    e_ok = ttn.expectation(s, p)
    original = ttn.TTN._up_ops

    def doubled(self, idx):
        out = original(self, idx)
        if self.nodes[idx].children[0][0] == "node":
            k = max((key for key in out if key != "H"), key=lambda key: np.linalg.norm(out[key]))
            out[k] = 2.0 * out[k]
        return out

    monkeypatch.setattr(ttn.TTN, "_up_ops", doubled)
    assert abs(ttn.expectation(s, p) - e_ok) > 1e-6 * abs(e_ok)


@pytest.mark.parametrize("L,counts", [((2, 2, 2), {1: 8}), ((4, 4, 4), {1: 56, 2: 8}),
                                      ((8, 8, 8), {1: 296, 2: 152, 3: 56, 4: 8}),
                                      ((4, 4, 2), {1: 32})])
def test_surface_layers_hand_counted(L, counts):
    lat = model.Lattice(*L)
    got = {}
    for x in range(lat.n_sites):
        got[ttn.surface_layer(lat, x)] = got.get(ttn.surface_layer(lat, x), 0) + 1
    assert got == counts
    # corners and face centres by hand on 4x4x4
    if L == (4, 4, 4):
        assert ttn.surface_layer(lat, lat.index(0, 0, 0)) == 1
        assert ttn.surface_layer(lat, lat.index(1, 1, 0)) == 1
        assert ttn.surface_layer(lat, lat.index(1, 2, 1)) == 2
        assert ttn.surface_layer(lat, lat.index(3, 3, 3)) == 1
