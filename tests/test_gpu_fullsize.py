"""Parity at the benchmark's full size (4x4x4 open lattice, chi = 64, seed 1,
Q = 0, the state bench.py times): the seeded isometric start equals the
oracle's at every node, and properties that hold at any size are checked
where the oracle's full operator contractions would take too long on the
host -- the adjoint equals the transpose and the forward product, the energy
does not depend on the centre position, the total charge is Q, and a
split-TF32 node update equals the FP64 one on the identical H_eff."""
import numpy as np
import pytest

import workloads
from oracle import model as omodel, ttn as ottn

from ttn_layout import to_layout

pytestmark = pytest.mark.gpu

L, CHI, SEED, Q = (4, 4, 4), 64, 1, 0


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as pkg
    pkg.lib()
    return pkg


def _model(q):
    return q.Model(*L, Q=Q, **workloads.qed_couplings(1.0))


def test_initial_tensors_full_size(q):
    ref = ottn.TTN(omodel.Params(*L, Q=Q, **workloads.qed_couplings(1.0)), CHI, SEED, build_ops=False)
    s = q.TTN(_model(q), CHI, seed=SEED)
    for idx in range(len(ref.nodes)):
        got = s.node_export(idx)
        want = to_layout(ref.T[idx], ref.labels[idx])
        assert got.shape == want.shape, idx
        assert np.max(np.abs(got - want)) < 1e-12, idx


def test_properties_full_size(q):
    import torch
    s = q.TTN(_model(q), CHI, seed=SEED)
    e_root = s.energy()[0]
    rng = np.random.default_rng(8)
    for node in (0, 40, 61):
        s.move_center(node)
        n = s.node_size(node)
        u = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
        v = torch.tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
        hv, htu, htv = (torch.empty_like(u) for _ in range(3))
        s.apply_heff_device(v.data_ptr(), hv.data_ptr(), n)
        s.apply_heff_adjoint_device(u.data_ptr(), htu.data_ptr(), n)
        s.apply_heff_adjoint_device(v.data_ptr(), htv.data_ptr(), n)
        torch.cuda.synchronize()
        lhs, rhs = float(u @ hv), float(htu @ v)
        assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs)), node
        assert float((htv - hv).abs().max()) <= 1e-11 * float(hv.abs().max()), node
        # the state's energy seen from this centre
        e_here, _ = s.energy_grad_device(node)
        assert abs(e_here - e_root) < 1e-10 * abs(e_root), node
    qx = s.measure("qx")
    assert abs(float(np.sum(qx)) - Q) < 1e-9


# element-wise budget of one product relative to max |y|: operands rounded
# to the format (BF16 2^-8, TF32 2^-11; split TF32 about FP32), FP32 sums
TOL = {"bf16": 2e-2, "tf32": 3e-3, "tf32x3": 2e-5}
NODES = (0, 17, 32, 45, 48, 56, 60, 62)   # bottom, layer 1 .. 4, root


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
def test_products_every_precision_full_size(q, prec):
    """The product that Lanczos calls in a mixed state (tensor cores at the
    bottom nodes, the state's precision at the upper nodes), with no Lanczos
    and no FP64 correction, element by element against the FP64 product of
    the same state on the same vector, at nodes of every layer."""
    import torch
    s = q.TTN(_model(q), CHI, seed=SEED, precision=prec)
    g = torch.Generator(device="cpu").manual_seed(21)
    for node in NODES:
        s.move_center(node)
        n = s.node_size(node)
        x = torch.randn(n, dtype=torch.float64, generator=g).cuda()
        y64, ym = torch.empty_like(x), torch.full_like(x, float("nan"))
        s.set_precision("fp64")
        s.apply_heff_device(x.data_ptr(), y64.data_ptr(), n)
        s.set_precision(prec)
        s.apply_heff_device(x.data_ptr(), ym.data_ptr(), n)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(ym).all()), (prec, node)
        err = float((ym - y64).abs().max() / y64.abs().max())
        assert err < TOL[prec], (prec, node, err)
        # and again, so that replayed plans and staged operands are exercised
        s.apply_heff_device(x.data_ptr(), ym.data_ptr(), n)
        torch.cuda.synchronize()
        assert float((ym - y64).abs().max() / y64.abs().max()) < TOL[prec], (prec, node)
    s.close()


# budget of the low-precision phase's Ritz value against the FP64 update
RITZ_TOL = {"tf32x3": 1e-5, "tf32": 3e-3, "bf16": 2e-2}


@pytest.mark.parametrize("prec", ["tf32x3", "tf32", "bf16"])
def test_mixed_update_full_size(q, prec):
    """Node updates from identical states and identical H_eff.  The Ritz
    value that the low-precision phase reaches on its own, before the FP64
    correction, must agree with the FP64 update within the product's
    rounding (a wrong tensor-core product fails here, where the corrected
    energy would still agree); the corrected energy must meet the 1e-6 gate
    of the benchmark's tolerance."""
    tol = 1e-6
    s = q.TTN(_model(q), CHI, seed=SEED, precision=prec)
    for node in (0, 48):
        s.move_center(node)
        t0 = s.node_export(node)
        s.set_precision("fp64")
        e64 = s.optimize_node(node, tol=tol, max_krylov=64)
        s.node_import(node, t0)
        s.set_precision(prec)
        em = s.optimize_node(node, tol=tol, max_krylov=64)
        lu = s.last_update()
        theta = lu["ritz_mixed"]
        assert lu["iters_mixed"] > 0, (prec, node)
        assert abs(theta - e64) < RITZ_TOL[prec] * abs(e64), (prec, node, theta, e64)
        assert abs(em - e64) < 1e-6 * abs(e64), (prec, node, em, e64)
        s.node_import(node, t0)
    s.close()


@pytest.mark.parametrize("L,chi,seed", [((2, 2, 2), 8, 0), ((4, 4, 4), 64, 1)])
def test_bottom_flop_count_matches_oracle(q, L, chi, seed):
    """The algorithmic flops the library books for one tensor-core product
    at bottom node 0 equal the oracle's own count of the same product (a
    row selection per term, then one dense environment block per charge
    sector: 2 x nonzero rows x chi_out x chi_in)."""
    c = workloads.qed_couplings(1.0)
    ref = ottn.TTN(omodel.Params(*L, Q=0, **c), chi, seed, build_ops=False)
    want = ottn.bottom_heff_flops(ref, 0)
    s = q.TTN(q.Model(*L, Q=0, **c), chi, seed=seed, precision="tf32x3")
    s.move_center(0)
    s.set_profiling(True)
    s.reset_timing()
    s.apply_heff(np.ones(s.node_size(0)))
    t = s.kernel_timing("tc_heff")
    s.close()
    got = t["flops_alg"] / max(1, t["launches"])
    assert abs(got - want) <= 1e-9 * want, (got, want)
