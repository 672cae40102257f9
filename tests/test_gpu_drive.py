"""Coupling updates and the driven optimisation of the penalty on the GPU
(Methods, "Numerical Convergence"): a state whose couplings were changed
equals a state created with those couplings and loaded with the same
tensors, element by element; repeated changes give back their memory; the
driven sweeps follow the oracle's driven sweeps record by record."""
import numpy as np
import pytest

import workloads
from oracle import drive as odrive
from oracle import model as omodel
from oracle import ttn as ottn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_set_couplings_equals_fresh_state(q, precision):
    L, chi = (4, 2, 2), 16
    c = workloads.qed_couplings(1.0)
    a = q.TTN(q.Model(*L, Q=0, **c), chi, seed=5, precision=precision)
    a.sweep(1, tol=1e-8, allow_noconv=True)
    tensors = [a.node_export(i) for i in range(a.info()["n_nodes"])]
    new = dict(c, nu=3.0, cB=0.25, m=0.5)
    a.set_couplings(**new)
    b = q.TTN(q.Model(*L, Q=0, **new), chi, seed=5, precision=precision)
    b.load_tensors(tensors)
    ea, eb = a.energy(), b.energy()
    assert abs(ea[0] - eb[0]) < 1e-12 * abs(eb[0])
    for k in ea[2]:
        assert abs(ea[2][k] - eb[2][k]) < 1e-11 * max(1.0, abs(eb[2][k]))
    rng = np.random.default_rng(3)
    for node in (0, 8, 2, 12, 14):
        a.move_center(node)
        b.move_center(node)
        x = rng.standard_normal(a.node_size(node))
        for s in (a, b):
            s.set_precision("fp64")
        ya, yb = a.apply_heff(x), b.apply_heff(x)
        for s in (a, b):
            s.set_precision(precision)
        assert np.max(np.abs(ya - yb)) <= 1e-12 * np.max(np.abs(yb)), node
    a.close()
    b.close()


def test_set_couplings_gives_memory_back(q):
    import torch
    c = workloads.qed_couplings(1.0)
    s = q.TTN(q.Model(4, 2, 2, Q=0, **c), 16, seed=5, precision="tf32x3")
    s.sweep(1, tol=1e-6, allow_noconv=True)
    s.set_couplings(**dict(c, nu=2.0))
    s.sweep(1, tol=1e-6, allow_noconv=True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for nu in (3.0, 4.0, 5.0, 6.0):
        s.set_couplings(**dict(c, nu=nu))
        s.sweep(1, tol=1e-6, allow_noconv=True)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 16 << 20, (free0 - free1)
    s.close()


def test_set_couplings_rejects_a_class_absent_at_creation(q):
    c = dict(workloads.qed_couplings(1.0), cB=0.0)
    s = q.TTN(q.Model(2, 2, 1, Q=0, **c), 8, seed=0, precision="fp64")
    with pytest.raises(q.QedError):
        s.set_couplings(**dict(c, cB=0.5))
    # keeping the absent class at zero while another coupling changes is fine
    s.set_couplings(**dict(c, nu=4.0))
    s.sweep(1, tol=1e-10)
    s.close()


DRIVE = dict(nu_start=0.5, nu_step=3.0, quad_coef=0.25, nu_max=10.0, tol_start=1e-10, tol_factor=0.1, tol_final=1e-12,
             conv_rel=1e-9, rise_rel=1e-9, min_final_sweeps=2)


def test_drive_matches_oracle(q):
    """2x2x1, chi = 8, FP64: nu 0.5, 3.5, 6.5, 9.5, then 10 until two energies
    agree; every record equals the oracle's driven run."""
    c = dict(workloads.qed_couplings(1.0), nu=DRIVE["nu_start"])
    ref = ottn.TTN(omodel.Params(2, 2, 1, Q=0, **c), 8, 0)
    want, want_conv = odrive.run(ref, max_sweeps=6, **DRIVE)
    s = q.TTN(q.Model(2, 2, 1, Q=0, **c), 8, seed=0, precision="fp64")
    got, conv = s.drive(max_sweeps=6, max_krylov=64, allow_noconv=True, **DRIVE)
    assert conv == want_conv and len(got) == len(want)
    for g, w in zip(got, want):
        assert g["stage"] == w["stage"] and g["sweep"] == w["sweep"]
        assert g["nu"] == pytest.approx(w["nu"], rel=1e-15) and g["tol"] == pytest.approx(w["tol"], rel=1e-14)
        assert abs(g["energy"] - w["energy"]) < 1e-8 * abs(w["energy"])
        assert abs(g["energy_without_penalty"] - w["energy_without_penalty"]) < 1e-8 * abs(w["energy"])
        assert abs(g["delta_L"] - w["delta_L"]) < 1e-6
        assert g["not_converged"] == 0
    s.close()


def test_drive_mixed_precision_reaches_the_constraint(q):
    """2x2x2, chi = 8, split TF32: the driven run ends at nu_max with the link
    constraint met (delta_L small) and an energy within the mixed gate of
    the FP64 driven run."""
    c = dict(workloads.qed_couplings(1.0), nu=DRIVE["nu_start"])
    out = {}
    for prec in ("fp64", "tf32x3"):
        s = q.TTN(q.Model(2, 2, 2, Q=0, **c), 8, seed=0, precision=prec)
        out[prec] = s.drive(max_sweeps=12, max_krylov=64, allow_noconv=True, **dict(DRIVE, tol_final=1e-10))
        s.close()
    for prec, (recs, conv) in out.items():
        assert recs[-1]["nu"] == 10.0 and recs[-1]["delta_L"] < 1e-5, prec
        assert [r["nu"] for r in recs][:4] == [0.5, 3.5, 6.5, 9.5]
    e64, emx = out["fp64"][0][-1]["energy"], out["tf32x3"][0][-1]["energy"]
    assert abs(e64 - emx) < 1e-6 * abs(e64)
