"""FP64 CPU oracle for the TTN ground-state method of lattice QED in (3+1)D.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of the method (Magnifico, Felser, Silvi, Montangero, "Lattice
Quantum Electrodynamics in (3+1)-dimensions at finite density with Tensor
Networks", arXiv:2011.10658).  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import it.  The product library never imports, links or executes anything
in here, and this package imports nothing from the product library.

Modules
-------
basis   dressed-site basis of Eq. (12)-(14) (Methods, "Fermionic compact
        representation of local gauge-invariant site").
fock    site operators built literally in the Fock space of one matter mode
        and twelve Dirac modes, from Eq. (6) and the state definitions that
        follow it.
model   lattice, couplings and the product-term list of Eq. (1) + Eq. (16).
tree    binary 3D tree (Methods, "Tensor Networks"), U(1) sector table,
        SplitMix64 initialisation, per-sector QR.
ttn     dense-with-mask TTN: renormalized operators, H_eff, eigensolver,
        sweep, energies and observables.
ed      exact diagonalisation references: the dressed tensor-product space
        and an independent configuration basis (link E, global
        Jordan-Wigner matter).

Parity pins live in ``tests/test_oracle_*.py``.  Functions whose result has
no pin other than GPU parity are marked "parity unpinned" in their
docstring.
"""
