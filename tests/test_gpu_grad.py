"""GPU tests of the differentiation entry points through the C ABI: the
adjoint H_eff product against the transpose identity and the forward
product, the energy gradient against the oracle's, and the autograd path
(dE/dg^2, dE/dm, dE/dpsi) against central finite differences and the
Hellmann-Feynman class energies on the 4x4x4, chi = 32, Q = 4 workload."""
import numpy as np
import pytest

from oracle import model as omodel, ttn as ottn

from ttn_layout import from_layout, to_layout

pytestmark = pytest.mark.gpu

KW = dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as pkg
    pkg.lib()
    return pkg


def dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_adjoint_transpose_identity(q):
    """<u, H v> = <H^T u, v> and H^T v = H v (H_eff is real symmetric), at a
    bottom, an upper and the root centre."""
    import torch
    s = q.TTN(q.Model(2, 2, 2, **KW), 8, seed=0)
    rng = np.random.default_rng(3)
    for node in (6, 0, 4, 3, 5):
        s.move_center(node)
        n = s.node_size(node)
        u, v = dev(rng.standard_normal(n)), dev(rng.standard_normal(n))
        hv, htu, htv = (torch.empty_like(u) for _ in range(3))
        s.apply_heff_device(v.data_ptr(), hv.data_ptr(), n)
        s.apply_heff_adjoint_device(u.data_ptr(), htu.data_ptr(), n)
        s.apply_heff_adjoint_device(v.data_ptr(), htv.data_ptr(), n)
        torch.cuda.synchronize()
        lhs, rhs = float(u @ hv), float(htu @ v)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)), node
        assert float((htv - hv).abs().max()) <= 1e-12 * float(hv.abs().max()), node


CASES = [((2, 2, 1), 12, 3, dict(t=0.8, m=0.3, ge2=1.5, cB=0.9, nu=20.0, Q=1)),
         ((2, 2, 2), 8, 0, KW)]


@pytest.mark.parametrize("L,chi,seed,kw", CASES, ids=["2x2x1", "2x2x2"])
def test_energy_grad_matches_oracle(q, L, chi, seed, kw):
    import torch
    p = omodel.Params(*L, **kw)
    ref = ottn.TTN(p, chi, seed)
    s = q.TTN(q.Model(*L, **kw), chi, seed=seed)
    rng = np.random.default_rng(4)
    for node in sorted({0, len(ref.nodes) // 2, len(ref.nodes) - 1}):
        ref.move_to(node)
        n = s.node_size(node)
        x = rng.standard_normal(n)
        g = torch.empty(n, dtype=torch.float64, device="cuda")
        e, _ = s.energy_grad_device(node, dev(x).data_ptr(), g.data_ptr(), n)
        X = from_layout(x, ref.labels[node], ref.T[node].shape)
        e_ref, g_ref = ottn.energy_gradient(ref, X)
        assert abs(e - e_ref) < 1e-10 * abs(e_ref)
        want = to_layout(g_ref, ref.labels[node])
        assert np.max(np.abs(g.cpu().numpy() - want)) < 1e-10 * np.max(np.abs(want)), node
    # coupling derivatives of the TTN state itself (psi = centre tensor)
    node = len(ref.nodes) - 1
    _, dc = s.energy_grad_device(node)
    want = ottn.coupling_gradient(ref, p)
    for c in ottn.COUPLINGS:
        assert abs(dc[c] - want[c]) < 1e-10 * max(1.0, abs(want[c])), c


def _config4(q, g2, mass):
    c = dict(t=1.0, m=mass, ge2=g2, cB=1.0 / (2.0 * g2), nu=10.0, Q=4)
    return q.TTN(q.Model(4, 4, 4, **c), 32, seed=3)


def test_autograd_couplings_match_finite_differences(q):
    """dE/dg^2 and dE/dm by reverse mode through EnergyFn (ge2 = g^2,
    cB = 1/(2 g^2), nu fixed) against central differences with step 1e-5 and
    against the Hellmann-Feynman class energies."""
    import torch
    from paper_2011_10658_gb300.autograd import EnergyFn
    s = _config4(q, 1.0, 1.0)
    root = s.info()["n_nodes"] - 1
    psi = dev(s.node_export(root))
    g2 = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    mass = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    one = torch.tensor(1.0, dtype=torch.float64)
    couplings = torch.stack([one, mass, g2, 0.5 / g2, 10.0 * one])
    e = EnergyFn.apply(psi, couplings, s, root)
    e.backward()
    et, _, parts = s.energy()
    assert abs(float(e.detach()) - et) < 1e-12 * abs(et)
    hf_m = parts["m"] / 1.0
    hf_g2 = parts["ge2"] / 1.0 - parts["cB"] / 0.5 * 0.5
    assert abs(float(mass.grad) - hf_m) < 1e-10 * max(1.0, abs(hf_m))
    assert abs(float(g2.grad) - hf_g2) < 1e-10 * max(1.0, abs(hf_g2))
    h = 1e-5
    fd_g2 = (_config4(q, 1.0 + h, 1.0).energy()[0] - _config4(q, 1.0 - h, 1.0).energy()[0]) / (2 * h)
    fd_m = (_config4(q, 1.0, 1.0 + h).energy()[0] - _config4(q, 1.0, 1.0 - h).energy()[0]) / (2 * h)
    assert abs(float(g2.grad) - fd_g2) < 1e-6 * max(1.0, abs(fd_g2)), (float(g2.grad), fd_g2)
    assert abs(float(mass.grad) - fd_m) < 1e-6 * max(1.0, abs(fd_m)), (float(mass.grad), fd_m)


def test_autograd_psi_matches_finite_differences(q):
    import torch
    from paper_2011_10658_gb300.autograd import EnergyFn
    s = _config4(q, 1.0, 1.0)
    node = 40   # an upper node
    s.move_center(node)
    psi = dev(s.node_export(node)).requires_grad_(True)
    couplings = torch.tensor([1.0, 1.0, 1.0, 0.5, 10.0], dtype=torch.float64)
    e = EnergyFn.apply(psi, couplings, s, node)
    e.backward()
    rng = np.random.default_rng(5)
    h = 1e-5
    for _ in range(3):
        d = dev(rng.standard_normal(psi.numel()))
        with torch.no_grad():
            ep = float(EnergyFn.apply((psi + h * d).contiguous(), couplings, s, node))
            em = float(EnergyFn.apply((psi - h * d).contiguous(), couplings, s, node))
        fd = (ep - em) / (2 * h)
        an = float(psi.grad @ d)
        assert abs(fd - an) < 1e-6 * max(1.0, abs(fd)), (fd, an)


def test_gradient_step_lowers_energy(q):
    s = q.TTN(q.Model(2, 2, 2, **KW), 8, seed=0)
    s.move_center(0)
    e_first = None
    for _ in range(5):
        e0, e1 = s.gradient_step(1e-3)
        e_first = e0 if e_first is None else e_first
        assert e1 < e0
    x = s.node_export(0)
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    # the Lanczos update from the same state reaches at least as low
    e_lz = s.optimize_node(0, tol=1e-12)
    assert e_lz <= e1 + 1e-12 * abs(e1)
