"""Pins of the oracle's energy gradients (differentiation row): central
finite differences in the node tensor and in each coupling, and Euler's
identity E = sum_c c dE/dc for an energy linear in the couplings."""
import dataclasses

import numpy as np
import pytest

from oracle import model, ttn

KW = dict(t=0.9, m=0.7, ge2=1.1, cB=0.45, nu=8.0)


@pytest.fixture(scope="module")
def state():
    p = model.Params(2, 2, 1, **KW)
    s = ttn.TTN(p, 6, seed=5)
    s.move_to(1)
    return p, s


def test_psi_gradient_matches_central_differences(state):
    p, s = state
    M = s.mask(s.center)
    rng = np.random.default_rng(0)
    X = np.zeros(M.shape)
    X[M] = rng.standard_normal(M.sum())
    e, g = ttn.energy_gradient(s, X)
    assert np.linalg.norm(g) > 1e-3
    for _ in range(3):
        d = np.zeros_like(X)
        d[M] = rng.standard_normal(M.sum())
        h = 1e-5
        ep, _ = ttn.energy_gradient(s, X + h * d)
        em, _ = ttn.energy_gradient(s, X - h * d)
        fd = (ep - em) / (2 * h)
        assert abs(fd - float(np.vdot(g, d))) < 1e-7 * max(1.0, abs(fd))
    # the gradient is orthogonal to X (scale invariance of the quotient)
    assert abs(float(np.vdot(g, X))) < 1e-10 * np.linalg.norm(g) * np.linalg.norm(X)


def test_coupling_gradient_matches_central_differences(state):
    p, s = state
    grads = ttn.coupling_gradient(s, p)
    h = 1e-5
    for c in ttn.COUPLINGS:
        v = getattr(p, c)
        ep = ttn.expectation(s, dataclasses.replace(p, **{c: v + h}))
        em = ttn.expectation(s, dataclasses.replace(p, **{c: v - h}))
        fd = (ep - em) / (2 * h)
        assert abs(fd - grads[c]) < 1e-6 * max(1.0, abs(fd)), (c, fd, grads[c])


def test_euler_identity(state):
    """E is homogeneous of degree one in (t, m, ge2, cB, nu): E = sum c dE/dc."""
    p, s = state
    grads = ttn.coupling_gradient(s, p)
    e = ttn.expectation(s, p)
    assert abs(sum(getattr(p, c) * grads[c] for c in ttn.COUPLINGS) - e) < 1e-10 * abs(e)
