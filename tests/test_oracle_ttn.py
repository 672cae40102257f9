"""Pins of the oracle's TTN sweep: the exact two-site energy, exactness
against independent ED at sufficient bond dimension on 2x2x1, the
variational bound below it, and the invariants (isometry, charge, Gauss sum
rule, centre independence, monotone energy)."""
import numpy as np
import pytest

from oracle import ed, model, ttn


def test_single_node_closed_form():
    p = model.Params(2, 1, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)
    s = ttn.TTN(p, 8, 0)
    e = s.sweep(tol=1e-12)
    assert abs(e[-1] - (0.25 - np.sqrt(41.0) / 4.0)) < 1e-10


@pytest.fixture(scope="module")
def swept_2x2x1():
    p = model.Params(2, 2, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)
    s = ttn.TTN(p, 12, 0)
    energies = s.sweep(tol=1e-10)
    return p, s, energies


def test_reaches_exact_diagonalisation(swept_2x2x1):
    p, s, energies = swept_2x2x1
    e_ed = ed.config_ed(p)
    assert abs(energies[-1] - e_ed) < 1e-9 * abs(e_ed)


def test_variational_bound_small_chi():
    p = model.Params(2, 2, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)
    s = ttn.TTN(p, 4, 1)
    e = s.sweep(tol=1e-10)
    assert e[-1] > ed.config_ed(p) + 1e-3


def test_energy_monotone(swept_2x2x1):
    _, _, energies = swept_2x2x1
    assert all(b <= a + 1e-9 for a, b in zip(energies, energies[1:]))


def test_isometry_and_centre_independence(swept_2x2x1):
    p, s, energies = swept_2x2x1
    e_root = s.energy_at_center()
    assert abs(e_root - energies[-1]) < 1e-9
    for target in (0, 1, 2):
        s.move_to(target)
        assert abs(s.energy_at_center() - e_root) < 1e-10
        assert abs(s.norm_at_center() - 1.0) < 1e-12
        for nd in s.nodes:
            if nd.index == s.center:
                continue
            T = s.T[nd.index]
            leg = s._neighbour_leg(nd.index, s.path(nd.index, s.center)[1])
            A = np.moveaxis(T, leg, 2).reshape(-1, T.shape[leg])
            np.testing.assert_allclose(A.T @ A, np.eye(A.shape[1]), atol=1e-12)


def test_charge_and_gauss_sum_rule(swept_2x2x1):
    p, s, _ = swept_2x2x1
    obs = s.observables()
    assert abs(obs["Q"] - p.Q) < 1e-12
    lat = s.lat
    # Q - sum <dangling outflow> = sum_links <2 - L>  (sum of Eq. (11) over sites)
    flux = 0.0
    for x in range(lat.n_sites):
        for j in lat.dangling(x):
            flux += 1.0 - obs["k"][x][j]
    links = sum(2.0 - obs["k"][x][model.plus(mu)] - obs["k"][y][model.minus(mu)] for (x, mu, y) in lat.links())
    assert abs((p.Q - flux) - links) < 1e-12
    assert obs["delta_L"] < 1e-2
    assert 0.0 <= obs["rho"] <= 1.0


def test_energy_split_by_class(swept_2x2x1):
    """E is linear in the couplings at fixed psi (Eq. (1) + (16)):
    sum_class <H_class> + nu N_links = <H>."""
    p, s, energies = swept_2x2x1
    total = ttn.expectation(s, p)
    parts = sum(ttn.expectation(s, model.class_only(p, c)) for c in ("t", "m", "ge2", "cB"))
    pen = ttn.expectation(s, model.class_only(p, "nu"))
    assert abs(total - energies[-1]) < 1e-9
    assert abs(parts + pen - total) < 1e-10


def test_plain_workload_stored_sweep_reproduces():
    """The stored plain-workload sweep (tests/golden/plain_2x2x2_chi8.txt) is
    what the oracle computes; the GPU test reads the stored file."""
    import os
    import workloads
    from oracle import model as _model, ttn as _ttn
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "plain_2x2x2_chi8.txt")
    rows = [line.split() for line in open(path) if not line.startswith("#")]
    s = _ttn.TTN(_model.Params(2, 2, 2, Q=0, **workloads.qed_couplings(1.0)), 8, 0)
    energies = s.sweep(tol=1e-12)
    assert len(energies) == len(rows)
    for (_, _, e), got in zip(rows, energies):
        assert abs(got - float(e)) < 1e-10 * abs(float(e))


def test_strong_coupling_chi1_pair_product():
    """chi = 1 on 2x2x1 makes the TTN a product of the two bottom-node pairs
    (x-neighbours).  As g^2 grows it tends to the confined vacuum dressed by
    the pair fluctuations of the two links inside the pairs: E0 - 2 t^2 /
    (2 m + g^2 / 2) to second order, between the exact energy and E0."""
    from oracle import ed
    errs = []
    for g2, tol in ((40.0, 5e-3), (160.0, 5e-4)):
        c = dict(t=1.0, m=1.0, ge2=g2, cB=1.0 / (2.0 * g2), nu=10.0 * max(1.0, g2 / 2.0))
        p = model.Params(2, 2, 1, Q=0, **c)
        s = ttn.TTN(p, 1, 0)
        s.sweep(tol=1e-12)
        e = s.sweep(tol=1e-12)[-1]
        e0 = -2.0
        ept = e0 - 2.0 / (2.0 + g2 / 2.0)
        assert ed.config_ed(p) - 1e-9 <= e <= e0
        errs.append(abs((e - e0) / (ept - e0) - 1.0))
        assert errs[-1] < tol
    assert errs[1] < errs[0] / 4


def test_site_observables_against_dressed_ed():
    """Two sites: the TTN (one node holding both sites, exact) gives the same
    single-site occupations <psi^dag psi>_x as the ground vector of the full
    dressed-space Hamiltonian, and each site's probabilities sum to one."""
    import scipy.sparse.linalg as spla
    from oracle import basis
    p = model.Params(2, 1, 1, t=0.8, m=0.6, ge2=1.2, cB=0.5, nu=12.0, Q=0)
    H, qv, _ = ed.dressed_hamiltonian(p)
    sel = np.nonzero(qv == p.Q)[0]
    vals, vecs = spla.eigsh(H[sel][:, sel], k=1, which="SA", tol=1e-14)
    v = np.zeros(H.shape[0])
    v[sel] = vecs[:, 0]
    w = (v * v).reshape(basis.D_LOCAL, basis.D_LOCAL)
    lat = model.Lattice(2, 1, 1)
    phi_ed = [float(w.sum(axis=1) @ basis.enumerate_basis(lat.parity(0))[:, 0]),
              float(w.sum(axis=0) @ basis.enumerate_basis(lat.parity(1))[:, 0])]
    s = ttn.TTN(p, 8, 0)
    e = s.sweep(tol=1e-12)[-1]
    assert abs(e - vals[0]) < 1e-10 * abs(vals[0])
    obs = s.observables()
    for x in range(2):
        assert abs(obs["phi"][x] - phi_ed[x]) < 1e-8, (x, obs["phi"][x], phi_ed[x])
    # the link field of Eq. (10) at the lower site: E = 1 - k_{x,+x}
    k_plus_x = basis.enumerate_basis(lat.parity(0))[:, basis.COL_K][:, model.plus(0)].astype(float)
    e_link_ed = 1.0 - float(w.sum(axis=1) @ k_plus_x)
    assert abs(obs["E_link"][0] - e_link_ed) < 1e-8
    probs = s.site_probabilities()
    for x in range(2):
        assert abs(np.sum(probs[x]) - 1.0) < 1e-12
        assert np.min(probs[x]) > -1e-14
