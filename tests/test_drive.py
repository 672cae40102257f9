"""Driven optimisation of the penalty (Methods, "Numerical Convergence"):
the schedule of nu and of the Lanczos tolerance, pinned by hand on
synthetic energy sequences, the library's host-side schedule against the
oracle's on random sequences, and the oracle's coupling update against
the linearity of Eq. (1) + (16) in the couplings."""
import numpy as np
import pytest

from oracle import drive as odrive
from oracle import model as omodel
from oracle import ttn as ottn

SETTINGS = dict(nu_start=0.5, nu_step=0.5, quad_coef=0.25, nu_max=3.0, tol_start=1e-4, tol_factor=0.1,
                tol_final=1e-9, conv_rel=1e-6, rise_rel=1e-9, min_final_sweeps=2)
# energies after each sweep; sweep 3 rises above sweep 2 (-2.4 > -2.5)
ENERGIES = [-1.0, -2.0, -2.5, -2.4, -2.6, -2.7, -2.75, -2.8, -2.8000001]
# by hand: linear 0.5, 1.0, 1.5, 2.0; the rise after sweep 3 switches at nu = 2.0:
# 2.0 + 0.25 * 0.5 * k^2 = 2.125, 2.5, then 3.125 -> clamped to nu_max = 3.0
WANT_NU = [0.5, 1.0, 1.5, 2.0, 2.125, 2.5, 3.0, 3.0, 3.0]
WANT_STAGE = [0, 0, 0, 0, 1, 1, 2, 2, 2]
# converged after sweep 8: third sweep at nu_max, |dE| = 1e-7 <= 1e-6 * 2.8


def _oracle_trace(settings, energies):
    sch = odrive.Schedule(**settings)
    out = []
    for e in energies:
        if sch.converged:
            break
        out.append((sch.next_nu, odrive.STAGE_CODE[sch.next_stage], sch.tol()))
        sch.record(e)
    return out, sch.converged


def _library_trace(settings, energies):
    q = pytest.importorskip("paper_2011_10658_gb300")
    d = q.drive_settings(**settings)
    st = q.drive_start(d)
    out = []
    for e in energies:
        if st.done:
            break
        out.append((st.nu, st.stage, st.tol))
        q.drive_next(d, st, e)
    return out, bool(st.done)


def _check_hand(trace, converged):
    assert converged
    assert [t[0] for t in trace] == pytest.approx(WANT_NU, abs=1e-15)
    assert [t[1] for t in trace] == WANT_STAGE
    want_tol = [max(1e-9, 1e-4 * 0.1 ** s) for s in range(len(WANT_NU))]
    assert [t[2] for t in trace] == pytest.approx(want_tol, rel=1e-12)


def test_oracle_schedule_hand_pinned():
    _check_hand(*_oracle_trace(SETTINGS, ENERGIES))


def test_library_schedule_hand_pinned():
    _check_hand(*_library_trace(SETTINGS, ENERGIES))


def test_schedule_edge_cases():
    # nu_start at nu_max: constant from the first sweep; converged on the 2nd equal energy
    s = dict(SETTINGS, nu_start=3.0)
    for trace, conv in (_oracle_trace(s, [-1.0, -1.0, -1.0]), _library_trace(s, [-1.0, -1.0, -1.0])):
        assert [t[1] for t in trace] == [2, 2] and [t[0] for t in trace] == [3.0, 3.0] and conv
    # a rise below rise_rel is rounding, not a rise: the linear stage runs on to nu_max
    e = [-1.0, -1.0 + 1e-12, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0]
    for trace, conv in (_oracle_trace(SETTINGS, e), _library_trace(SETTINGS, e)):
        assert [t[1] for t in trace][:6] == [0, 0, 0, 0, 0, 2]
        assert [t[0] for t in trace][:6] == [0.5, 1.0, 1.5, 2.0, 2.5, 3.0]


def test_library_schedule_matches_oracle_on_random_sequences():
    rng = np.random.default_rng(7)
    for trial in range(200):
        s = dict(nu_start=float(rng.choice([0.25, 0.5, 1.0])), nu_step=float(rng.choice([0.25, 0.5, 2.0])),
                 quad_coef=float(rng.choice([0.125, 0.25, 0.5])), nu_max=float(rng.choice([2.0, 5.0, 10.0])),
                 tol_start=1e-4, tol_factor=float(rng.choice([0.1, 0.5, 1.0])), tol_final=1e-10,
                 conv_rel=float(rng.choice([0.0, 1e-3])), rise_rel=float(rng.choice([0.0, 1e-9])),
                 min_final_sweeps=int(rng.integers(2, 4)))
        e = list(np.cumsum(rng.normal(-0.1, 0.3, size=30)) - 5.0)
        if trial % 3 == 0:   # flat tails reach convergence
            e[12:] = [e[11]] * 18
        a, ca = _oracle_trace(s, e)
        b, cb = _library_trace(s, e)
        assert ca == cb and len(a) == len(b)
        for x, y in zip(a, b):
            assert x[1] == y[1] and x[0] == pytest.approx(y[0], rel=1e-14) and x[2] == pytest.approx(y[2], rel=1e-14)


def test_library_rejects_bad_settings():
    q = pytest.importorskip("paper_2011_10658_gb300")
    for bad in (dict(nu_start=0.0), dict(nu_step=-1.0), dict(nu_max=0.1), dict(tol_factor=1.5),
                dict(min_final_sweeps=1), dict(rise_rel=-1.0)):
        with pytest.raises(q.QedError):
            q.drive_start(q.drive_settings(**bad))


@pytest.fixture(scope="module")
def swept_2x2x1():
    p = omodel.Params(2, 2, 1, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)
    s = ottn.TTN(p, 4, 3)
    s.sweep(tol=1e-8)
    return p, s


def test_oracle_set_couplings_is_linear_in_nu(swept_2x2x1):
    """<H + H_pen> is linear in nu at fixed tensors: E(nu') = <H> + (nu'/nu) <H_pen(nu)>."""
    p, s = swept_2x2x1
    e_pen = ottn.expectation(s, omodel.class_only(p, "nu"))
    e_rest = sum(ottn.expectation(s, omodel.class_only(p, c)) for c in ("t", "m", "ge2", "cB"))
    for nu in (3.0, 0.5, 10.0):
        s.set_couplings(nu=nu)
        assert s.center == len(s.nodes) - 1
        for node in (0, 1, 2):
            s.move_to(node)
            e = s.energy_at_center()
            assert abs(e - (e_rest + nu / 10.0 * e_pen)) < 1e-11 * abs(e)


def test_oracle_set_couplings_switches_a_class_off(swept_2x2x1):
    p, s = swept_2x2x1
    s.set_couplings(nu=10.0, cB=0.0)
    e = s.energy_at_center()
    want = sum(ottn.expectation(s, omodel.class_only(p, c)) for c in ("t", "m", "ge2", "nu"))
    assert abs(e - want) < 1e-11 * abs(want)
    s.set_couplings(cB=0.5)


@pytest.mark.parametrize("L,boundary", [((4, 4, 4), 0), ((4, 2, 2), 1), ((2, 2, 1), 1)])
def test_bench_link_order_matches_the_lattice(L, boundary):
    """The capacitor profile E_c(d) of bench.py indexes ttn_measure's link
    list by (site, direction) in the lattice's link order."""
    import bench
    want = [(x, mu) for (x, mu, _) in omodel.lattice(omodel.Params(*L, boundary=boundary)).links()]
    assert bench._links(L, boundary == 1) == want


def test_oracle_driven_run_two_sites():
    """2x1x1, one node: the driven run's last energy is the two-site closed
    form (the link constraint is exact once nu is large enough, R6), delta_L
    vanishes, and the records follow the schedule (nu 0.5, 3.5, 6.5, 9.5,
    then 10 until two energies agree)."""
    c = dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=0.5)
    st = ottn.TTN(omodel.Params(2, 1, 1, Q=0, **c), 8, 0)
    recs, conv = odrive.run(st, nu_start=0.5, nu_step=3.0, quad_coef=0.25, nu_max=10.0, tol_start=1e-10,
                            tol_factor=0.1, tol_final=1e-12, conv_rel=1e-10, rise_rel=1e-9, min_final_sweeps=2,
                            max_sweeps=8)
    assert conv
    assert [r["nu"] for r in recs][:5] == [0.5, 3.5, 6.5, 9.5, 10.0]
    exact = 0.25 - np.sqrt(41.0) / 4.0
    assert abs(recs[-1]["energy"] - exact) < 1e-10
    assert recs[-1]["delta_L"] < 1e-10
    assert abs(recs[-1]["energy_without_penalty"] - recs[-1]["energy"]) < 1e-10
