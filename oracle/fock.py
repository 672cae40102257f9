"""Site operators built literally in a Fock space.  Test infrastructure only.

One dressed site holds 13 Dirac modes: the matter mode psi (mode 0) and, for
each half-link j = 1..6, the two species a_j (mode 2j-1) and b_j (mode 2j)
of the Methods' three-level rishon construction.  Creation operators are
Jordan-Wigner matrices on the 2^13 occupation basis (bit m = occupation of
mode m).  From them this module writes out, with no shortcut:

* the three-level rishon raising operator of Eq. (6),
      eta_j^dag = n^a_j b_j^dag + (1 - n^b_j) a_j^dag,
* the half-link states |0>, |1> = a^dag|0>, |2> = b^dag a^dag|0> (text after
  Eq. (6)),
* the dressed basis vectors of Eq. (12): the sign of Eq. (12) times
  (psi^dag)^phi c_1 ... c_6 |vac>, c_j the creation string of |k_j>,
* the genuinely local (fermion-even) operators used by the Hamiltonian:
  M_j = psi^dag eta_j and M'_j = eta_j^dag psi of Eq. (15), C_ij =
  eta_i^dag eta_j of the plaquette factorisation, half-link projectors P^k_j
  and the matter number psi^dag psi.

Each operator is projected onto the 267 dressed rows, O_dressed = V^T O V.
The result is returned as a scipy CSR matrix (267 x 267, float64).
"""
import functools

import numpy as np
import scipy.sparse as sp

from . import basis as _basis

N_MODES = 13
DIM = 1 << N_MODES


def _mode_a(j):
    """Mode index of species a on half-link j (0-based j = 0..5)."""
    return 2 * j + 1


def _mode_b(j):
    return 2 * j + 2


@functools.lru_cache(maxsize=None)
def creation(mode):
    """Jordan-Wigner creation operator c_mode^dag on 2^13 states."""
    states = np.arange(DIM, dtype=np.int64)
    occupied = (states >> mode) & 1
    below = states & ((1 << mode) - 1)
    parity = np.array([bin(int(v)).count("1") & 1 for v in below], dtype=np.int64)
    src = states[occupied == 0]
    dst = src | (1 << mode)
    val = np.where(parity[occupied == 0] == 1, -1.0, 1.0)
    return sp.csr_matrix((val, (dst, src)), shape=(DIM, DIM))


def annihilation(mode):
    return creation(mode).T.tocsr()


def number(mode):
    return (creation(mode) @ annihilation(mode)).tocsr()


def identity():
    return sp.identity(DIM, format="csr")


@functools.lru_cache(maxsize=None)
def eta_dag(j):
    """Eq. (6): eta_j^dag = n^a_j b_j^dag + (1 - n^b_j) a_j^dag."""
    a_dag = creation(_mode_a(j))
    b_dag = creation(_mode_b(j))
    n_a = number(_mode_a(j))
    n_b = number(_mode_b(j))
    return (n_a @ b_dag + (identity() - n_b) @ a_dag).tocsr()


def eta(j):
    return eta_dag(j).T.tocsr()


def psi_dag():
    return creation(0)


def psi():
    return annihilation(0)


def _halflink_string(j, k):
    """Creation string of half-link state |k>_j: 1, a^dag, b^dag a^dag."""
    if k == 0:
        return identity()
    if k == 1:
        return creation(_mode_a(j))
    return (creation(_mode_b(j)) @ creation(_mode_a(j))).tocsr()


@functools.lru_cache(maxsize=None)
def dressed_vectors(parity):
    """V [8192, 267]: column i is the Fock vector of dressed row i, Eq. (12)."""
    table = _basis.enumerate_basis(parity)
    vac = np.zeros(DIM)
    vac[0] = 1.0
    cols = []
    for row in table:
        phi = int(row[_basis.COL_PHI])
        ks = [int(v) for v in row[_basis.COL_K]]
        sign = float(row[_basis.COL_SIGN])
        vec = vac.copy()
        # (psi^dag)^phi c_1 c_2 ... c_6 |vac>: apply c_6 first.
        for j in reversed(range(6)):
            vec = _halflink_string(j, ks[j]) @ vec
        if phi:
            vec = psi_dag() @ vec
        cols.append(sign * vec)
    return np.stack(cols, axis=1)


def project(op_fock, parity, check_closure=True):
    """Matrix elements <i|O|i'> of a Fock operator in the dressed basis.

    With ``check_closure`` the operator must map the dressed span into itself
    (Gauss's law preserved, Eq. (13)); otherwise ValueError is raised."""
    V = dressed_vectors(parity)
    OV = op_fock @ V
    M = V.T @ OV
    if check_closure:
        leak = OV - V @ M
        if np.abs(leak).max() > 1e-12:
            raise ValueError("operator leaves the gauge-invariant span")
    M[np.abs(M) < 1e-14] = 0.0
    return sp.csr_matrix(M)


def fock_op(key):
    """Fock-space operator for a local op key (see module docstring).

    Keys: ('M', j) = psi^dag eta_j; ('Md', j) = eta_j^dag psi;
    ('C', i, j) = eta_i^dag eta_j; ('P', j, k) = projector on k_j = k;
    ('PC', j, k) = 1 - ('P', j, k); ('n',) = psi^dag psi.  Half-link indices are 0-based (0..5 for
    -x, -y, -z, +x, +y, +z)."""
    kind = key[0]
    if kind == "M":
        return (psi_dag() @ eta(key[1])).tocsr()
    if kind == "Md":
        return (eta_dag(key[1]) @ psi()).tocsr()
    if kind == "C":
        return (eta_dag(key[1]) @ eta(key[2])).tocsr()
    if kind == "P":
        j, k = key[1], key[2]
        na = number(_mode_a(j))
        nb = number(_mode_b(j))
        one = identity()
        if k == 0:
            return ((one - na) @ (one - nb)).tocsr()
        if k == 1:
            return (na @ (one - nb)).tocsr()
        return (na @ nb).tocsr()
    if kind == "PC":
        return (identity() - fock_op(("P", key[1], key[2]))).tocsr()
    if kind == "n":
        return number(0)
    raise KeyError(key)


def electric_sq(mask):
    """Sum over the half-links in ``mask`` of E_j^2 with E_j = 1 - n^a_j -
    n^b_j, the one-sided field of Eq. (10)."""
    total = sp.csr_matrix((DIM, DIM))
    for j in mask:
        e = (identity() - number(_mode_a(j)) - number(_mode_b(j))).tocsr()
        total = total + e @ e
    return total.tocsr()


@functools.lru_cache(maxsize=None)
def site_op(key, parity):
    """Dressed-basis CSR matrix (267 x 267) of a local op key on a site of
    the given parity.  ('E2', mask) is the diagonal electric energy of the
    masked half-links (see ``electric_sq``)."""
    if key[0] == "E2":
        return project(electric_sq(key[1]), parity)
    return project(fock_op(key), parity)
