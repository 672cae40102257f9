"""FP64 parity against the oracle on lattices whose plans have many tiles,
many K chunks per output, split-K partial sums and ragged tail tiles:
4x2x2 at chi = 16 (four tree layers) and 4x4x2 at chi = 32 (five layers,
bottom sectors of 17 000-35 000 rows).  Element-wise: every tensor after
every centre move of a sweep's path, H_eff x at every centre (Methods,
"Tensor Networks", step (i)), node updates at the upper layers (steps
(ii)-(iii); the oracle's bottom-node eigensolves at this size take minutes
on the host, so bottom nodes are updated only at 2x2x2 in the other parity
tests), and the observables.  At 4x4x2 every tile shape of the grouped GEMM
is forced once (QED_KC_SHAPE), so each shape runs the operator updates and
the products of a full path against the oracle."""
import copy
import os

import numpy as np
import pytest

import workloads
from oracle import model as omodel, tree as otree, ttn as ottn

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


def _pair(q, L, chi, seed, shape=None):
    c = workloads.qed_couplings(1.0)
    ref = ottn.TTN(omodel.Params(*L, Q=0, **c), chi, seed)
    old = os.environ.get("QED_KC_SHAPE")
    if shape is not None:
        os.environ["QED_KC_SHAPE"] = str(shape)
    try:
        s = q.TTN(q.Model(*L, Q=0, **c), chi, seed=seed, precision="fp64")
    finally:
        if shape is not None:
            if old is None:
                del os.environ["QED_KC_SHAPE"]
            else:
                os.environ["QED_KC_SHAPE"] = old
    return ref, s


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def _check_centre(ref, s, node, rng):
    for idx in range(len(ref.nodes)):
        got = s.node_export(idx)
        want = to_layout(ref.T[idx], ref.labels[idx])
        assert np.max(np.abs(got - want)) < 1e-10, (node, idx)
    x = rng.standard_normal(s.node_size(node))
    y = s.apply_heff(x)
    want = to_layout(ref.heff_apply(node, from_layout(x, ref.labels[node], ref.T[node].shape)), ref.labels[node])
    assert _rel(y, want) < 1e-12, node


def test_4x2x2_chi16(q):
    ref, s = _pair(q, (4, 2, 2), 16, 2)
    rng = np.random.default_rng(31)
    order = otree.sweep_order(ref.nodes)
    for node in order:
        ref.move_to(node)
        s.move_center(node)
        _check_centre(ref, s, node, rng)
    # node updates at every upper node, in sweep order
    for node in [i for i in order if ref.nodes[i].layer > 0]:
        e_ref = ref.optimize_node(node, tol=1e-12)
        e = s.optimize_node(node, tol=1e-12, max_krylov=64)
        assert abs(e - e_ref) < 1e-10 * abs(e_ref), (node, e, e_ref)
        got = s.node_export(node)
        want = to_layout(ref.T[node], ref.labels[node])
        assert np.max(np.abs(got - want)) < 1e-8, node
    obs = ref.observables()
    assert abs(s.energy()[0] - ref.energy_at_center()) < 1e-10 * abs(ref.energy_at_center())
    np.testing.assert_allclose(s.measure("phi"), obs["phi"], atol=1e-10)
    np.testing.assert_allclose(s.measure("elink"), obs["E_link"], atol=1e-10)
    np.testing.assert_allclose(s.measure("sigma"), obs["sigma"], atol=1e-10)
    sc = s.measure("scalars")
    assert abs(sc[0] - obs["rho"]) < 1e-10 and abs(sc[1] - obs["delta_L"]) < 1e-9 and abs(sc[2] - obs["Q"]) < 1e-9
    s.close()


@pytest.fixture(scope="module")
def pristine_4x4x2():
    c = workloads.qed_couplings(1.0)
    return ottn.TTN(omodel.Params(4, 4, 2, Q=0, **c), 32, 2)


@pytest.fixture
def ref_4x4x2(pristine_4x4x2):
    # every test starts from the seeded state with the centre at the root
    return copy.deepcopy(pristine_4x4x2)


def test_4x4x2_chi32_path(q, ref_4x4x2):
    ref = ref_4x4x2
    _, s = _pair(q, (4, 4, 2), 32, 2)
    rng = np.random.default_rng(32)
    layers = {}
    for nd in ref.nodes:
        layers.setdefault(nd.layer, nd.index)
    path = [0, 1] + [layers[l] for l in sorted(layers) if l > 0] + [5]
    for node in path:
        ref.move_to(node)
        s.move_center(node)
        _check_centre(ref, s, node, rng)
    s.close()


@pytest.mark.parametrize("shape", [16, 32, 64, 1664, 6416])
def test_4x4x2_every_tile_shape(q, ref_4x4x2, shape):
    """One forced tile shape for every grouped-GEMM plan (operator updates,
    QR Gram matrices, products): the path root -> bottom node 3 and H_eff
    there and at the root against the oracle."""
    ref = ref_4x4x2
    _, s = _pair(q, (4, 4, 2), 32, 2, shape=shape)
    rng = np.random.default_rng(33)
    root = len(ref.nodes) - 1
    ref.move_to(root)
    _check_centre(ref, s, root, rng)
    ref.move_to(3)
    s.move_center(3)
    _check_centre(ref, s, 3, rng)
    s.close()
