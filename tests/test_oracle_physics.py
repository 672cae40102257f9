"""Pins of the oracle's periodic boundaries and local chemical potentials
(Results, "Transition at zero charge" and "Quantum capacitor"; Methods,
"Fermionic compact representation": diagonal local terms that pin
charges): closed-form term counts, the dressed two-site problem against the
independent configuration-basis diagonalisation on a ring, the static
strong-coupling limit, and a two-level closed form with potentials."""
import numpy as np
import pytest

from oracle import ed, model, ttn


def _counts(p):
    terms, _ = model.build_terms(p)
    out = {}
    for tm in terms:
        out[tm.cls] = out.get(tm.cls, 0) + 1
    return out


@pytest.mark.parametrize("L", [(2, 2, 2), (4, 2, 2), (4, 4, 4)])
def test_periodic_term_counts(L):
    """All extents >= 2: 3N links, 3N plaquettes, no dangling half-link;
    N mass + N electric + 2 x 3N hopping + 2 x 3N plaquette + 3 x 3N penalty
    = 23N product terms."""
    N = L[0] * L[1] * L[2]
    p = model.Params(*L, boundary=1)
    lat = model.lattice(p)
    assert len(lat.links()) == 3 * N and len(lat.plaquettes()) == 3 * N
    assert all(lat.dangling(s) == () for s in range(N))
    assert _counts(p) == {"m": N, "ge2": N, "t": 6 * N, "cB": 6 * N, "nu": 9 * N}


def test_periodic_with_a_flat_direction_counts():
    """2x2x1 periodic: x and y wrap (2N links, N plaquettes), z stays open
    with two dangling half-links per site: 14N terms."""
    p = model.Params(2, 2, 1, boundary=1)
    lat = model.lattice(p)
    N = 4
    assert len(lat.links()) == 2 * N and len(lat.plaquettes()) == N
    assert all(lat.dangling(s) == (2, 5) for s in range(N))
    assert _counts(p) == {"m": N, "ge2": N, "t": 4 * N, "cB": 2 * N, "nu": 6 * N}


def test_extent_two_ring_has_two_links_per_pair():
    lat = model.lattice(model.Params(2, 1, 1, boundary=1))
    assert lat.links() == [(0, 0, 1), (1, 0, 0)]
    assert lat.dangling(0) == (1, 2, 4, 5)


@pytest.mark.parametrize("t,m,ge2,cB", [(1.0, 1.0, 1.0, 0.5), (0.7, -0.3, 2.0, 0.25)])
def test_periodic_two_sites_equal_configuration_ed(t, m, ge2, cB):
    """2x1x1 ring (two links between the sites): the single-node TTN is the
    exact ground state of the dressed, penalised two-site problem; it must
    equal the configuration-basis diagonalisation with global
    Jordan-Wigner matter, a construction that shares nothing with the
    rishon operators."""
    p = model.Params(2, 1, 1, t=t, m=m, ge2=ge2, cB=cB, nu=10.0, Q=0, boundary=1)
    e = ttn.TTN(p, 8, 0).sweep(tol=1e-12)[-1]
    assert abs(e - ed.config_ed(p)) < 1e-10 * abs(e)


@pytest.mark.parametrize("m,want", [(1.0, -2.0), (-1.0, -1.0)])
def test_periodic_static_limit(m, want):
    """t = 0, cB = 0 (diagonal H): E = min(-m N/2, (m + ge2/2) N/2), bare
    vacuum against the charge crystal whose fields cost ge2/2 per pair;
    2x2x1 ring, N = 4, ge2 = 1."""
    p = model.Params(2, 2, 1, t=0.0, m=m, ge2=1.0, cB=0.0, nu=10.0, Q=0, boundary=1)
    e = ttn.TTN(p, 4, 0).sweep(tol=1e-12)[-1]
    assert abs(e - want) < 1e-10
    assert want == min(-m * 4 / 2, (m + 0.5) * 4 / 2)


def test_site_potential_two_level_closed_form():
    """2x1x1 open, Q = 0, with potentials mu_0 (even) and mu_1 (odd): the
    link-constrained space is {bare vacuum (odd site filled): -m + mu_1,
    pair with E = +1 on the link: m + ge2/2 + mu_0} coupled by -t, so
    E0 = (a + b)/2 - sqrt(((b - a)/2)^2 + t^2)."""
    mu = (0.3, -0.7)
    p = model.Params(2, 1, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0, mu=mu)
    e = ttn.TTN(p, 8, 0).sweep(tol=1e-12)[-1]
    a, b = -1.0 + mu[1], 1.0 + 0.5 + mu[0]
    assert abs(e - ((a + b) / 2 - np.sqrt(((b - a) / 2) ** 2 + 1.0))) < 1e-10


def test_site_potential_class_is_its_own():
    """<H_mu> = sum_x mu_x <psi^dag psi>_x, and the other classes do not see
    the potentials (class_only drops them)."""
    mu = (0.3, -0.7)
    p = model.Params(2, 1, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0, mu=mu)
    s = ttn.TTN(p, 8, 0)
    e = s.sweep(tol=1e-12)[-1]
    obs = s.observables()
    e_mu = ttn.expectation(s, model.class_only(p, "mu"))
    assert abs(e_mu - sum(m_ * ph for m_, ph in zip(mu, obs["phi"]))) < 1e-12
    rest = sum(ttn.expectation(s, model.class_only(p, c)) for c in ("t", "m", "ge2", "cB", "nu"))
    assert abs(rest + e_mu - e) < 1e-10 * abs(e)
