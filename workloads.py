"""Seeded workload presets shared by the tests, the benchmark and the oracle
legs.  Parameters only: lattice sizes, coupling presets, seeds and random
test vectors.  None of the method's arithmetic lives here.

Coupling preset for a QED coupling g^2 (a reading of the paper's couplings):
electric ge2 = g^2, plaquette coefficient cB = 1 / (2 g^2) (the plaquette
enters as -cB sum(box + h.c.)), hopping t = 1, mass m, and the link penalty
nu = 10 * max(|t|, |m|, ge2 / 2, |cB|) (the paper asks for nu much larger than
every other coupling and gives no number).
"""
import numpy as np


def qed_couplings(g2, t=1.0, m=1.0):
    ge2 = float(g2)
    cB = 1.0 / (2.0 * g2)
    nu = 10.0 * max(abs(t), abs(m), ge2 / 2.0, abs(cB))
    return dict(t=float(t), m=float(m), ge2=ge2, cB=cB, nu=nu)


# Plain method, FP64: 2x2x2, t = m = 1, g^2 = 1, Q = 0, chi = 8, seed 0, one sweep, tol 1e-12.
PLAIN_2X2X2 = dict(L=(2, 2, 2), chi=8, seed=0, Q=0, g2=1.0, tol=1e-12, sweeps=1)

# Precision workload: 4x4x4, t = m = 1, g^2 in {0.5, 1, 2, 4}, Q = 0, chi = 64, seed 1, 4 sweeps.
PRECISION_4X4X4 = dict(L=(4, 4, 4), chi=64, seed=1, Q=0, g2_values=(0.5, 1.0, 2.0, 4.0), sweeps=4)


def random_vector(n, seed):
    """Seeded standard-normal test vector (numpy default_rng)."""
    return np.random.default_rng(seed).standard_normal(n)
