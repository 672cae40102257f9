"""GPU tests of the mixed-precision (tcgen05 TF32 / BF16) bottom-node path:
H_eff x against the FP64 path and the oracle within the operand rounding,
and mixed sweeps against FP64 sweeps within the mixed-path tolerance."""
import numpy as np
import pytest

from oracle import model as omodel, ttn as ottn

from ttn_layout import from_layout, to_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as pkg
    pkg.lib()
    return pkg


# relative error budget of one H_eff x: operands rounded to the format's
# unit roundoff (BF16 2^-8, TF32 2^-11), FP32 accumulation
TOL = {"bf16": 2e-2, "tf32": 3e-3, "tf32x3": 2e-5}
KW = dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("L,chi", [((2, 1, 1), 8), ((2, 2, 2), 8), ((4, 2, 2), 16)])
def test_heff_mixed_vs_fp64(q, prec, L, chi):
    ref = q.TTN(q.Model(*L, **KW), chi, seed=3, precision="fp64")
    mix = q.TTN(q.Model(*L, **KW), chi, seed=3, precision=prec)
    rng = np.random.default_rng(5)
    nodes = (0,) if L == (2, 1, 1) else (0, 1, len(ref.model.tree()) - 2)
    for node in nodes:
        ref.move_center(node)
        mix.move_center(node)
        n = ref.node_size(node)
        x = rng.standard_normal(n)
        y64 = ref.apply_heff(x)
        ym = mix.apply_heff(x)
        err = np.max(np.abs(ym - y64)) / np.max(np.abs(y64))
        assert err < TOL[prec], (prec, node, err)
        # the Rayleigh quotient: operator rounding (the same W for every
        # row) is systematic, so only the per-element budget applies
        rq64 = x @ y64 / (x @ x)
        rqm = x @ ym / (x @ x)
        assert abs(rqm - rq64) < TOL[prec] * abs(rq64)


def test_heff_mixed_vs_oracle_tail_tiles(q):
    """2x2x1 bottom node: sector row counts are not multiples of 128."""
    p = omodel.Params(2, 2, 1, **KW)
    ref = ottn.TTN(p, 12, 0)
    mix = q.TTN(q.Model(2, 2, 1, **KW), 12, seed=0, precision="tf32")
    ref.move_to(0)
    mix.move_center(0)
    x = np.random.default_rng(9).standard_normal(mix.node_size(0))
    ym = mix.apply_heff(x)
    want = to_layout(ref.heff_apply(0, from_layout(x, ref.labels[0], ref.T[0].shape)), ref.labels[0])
    assert np.max(np.abs(ym - want)) / np.max(np.abs(want)) < TOL["tf32"]


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3"])
def test_mixed_sweep_matches_fp64(q, prec):
    """Mixed Lanczos followed by the FP64 residual correction reaches the FP64
    path's energies: |dE|/|E| <= 1e-6 per node update."""
    L, chi = (2, 2, 2), 8
    ref = q.TTN(q.Model(*L, **KW), chi, seed=0, precision="fp64")
    mix = q.TTN(q.Model(*L, **KW), chi, seed=0, precision=prec)
    e_ref, e_mix, mixed_iters = [], [], 0
    for node in range(7):
        e_ref.append(ref.optimize_node(node, tol=1e-10, max_krylov=48))
        e_mix.append(mix.optimize_node(node, tol=1e-10, max_krylov=48))
        mixed_iters += mix.last_update()["iters_mixed"]
    e_ref, e_mix = np.array(e_ref), np.array(e_mix)
    assert np.max(np.abs(e_mix - e_ref) / np.abs(e_ref)) < 1e-6
    assert mixed_iters > 0


def test_upper_node_fp32_products(q):
    """Upper-node products of the low-precision phase (FP32 grouped GEMM whose
    FP64 operands are converted to FP32 on the integer pipes) against FP64 at
    every upper node: FP32 rounding only."""
    L, chi = (4, 2, 2), 16
    ref = q.TTN(q.Model(*L, **KW), chi, seed=4, precision="fp64")
    mix = q.TTN(q.Model(*L, **KW), chi, seed=4, precision="tf32x3")
    tree = ref.model.tree()
    rng = np.random.default_rng(6)
    upper = [i for i in range(len(tree)) if tree[i][2] == 1]
    assert upper
    for node in upper:
        ref.move_center(node)
        mix.move_center(node)
        x = rng.standard_normal(ref.node_size(node))
        y64 = ref.apply_heff(x)
        ym = mix.apply_heff(x)
        assert np.max(np.abs(ym - y64)) / np.max(np.abs(y64)) < 1e-5, node
