"""FP64-accurate renormalized-operator updates on the BF16 tensor cores
(digit-plane splitting) against the FP64 path and the oracle.

A mixed-precision state forms the operators of the bond above a bottom
node with the digit-plane kernel when the centre moves up from that node
(Methods, "Tensor Networks": operators of every term crossing the bond,
renormalized by the node tensor).  At the parent the FP64 product of the
mixed state, which reads those operators, must equal the FP64 state's
product to FP64-level accuracy (the splitting keeps about 2^-38 of the
largest entry), element by element."""
import numpy as np
import pytest

import workloads
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


# chi = 96 on 2x2x2: bottom-bond sectors up to 55 wide (64-column tiles);
# chi = 128: a 74-wide sector, which the FP64 kernel takes instead
@pytest.mark.parametrize("L,chi,seed,path", [((2, 2, 2), 8, 0, (0, 4, 1, 5)), ((2, 2, 2), 96, 0, (0, 4, 1, 5)),
                                             ((2, 2, 2), 128, 0, (0, 4, 1, 5)),
                                             ((4, 4, 4), 64, 1, (0, 32, 1, 32, 17))])
def test_bottom_operator_update_matches_fp64(q, L, chi, seed, path):
    c = workloads.qed_couplings(1.0)
    a = q.TTN(q.Model(*L, Q=0, **c), chi, seed=seed, precision="fp64")
    b = q.TTN(q.Model(*L, Q=0, **c), chi, seed=seed, precision="tf32x3")
    rng = np.random.default_rng(41)
    for node in path:
        a.move_center(node)
        b.move_center(node)
        n = a.node_size(node)
        x = rng.standard_normal(n)
        ya = a.apply_heff(x)
        b.set_precision("fp64")
        yb = b.apply_heff(x)
        b.set_precision("tf32x3")
        err = float(np.max(np.abs(yb - ya)) / np.max(np.abs(ya)))
        assert err < 1e-11, (node, err)
    ea, eb = a.energy()[0], b.energy()[0]
    assert abs(ea - eb) < 1e-11 * abs(ea)
    a.close()
    b.close()


def test_bottom_operator_update_matches_oracle(q):
    """2x2x2: after the centre leaves bottom node 0 upwards in a mixed state,
    the FP64 product at its parent equals the oracle's."""
    c = workloads.qed_couplings(1.0)
    ref = ottn.TTN(omodel.Params(2, 2, 2, Q=0, **c), 8, 0)
    s = q.TTN(q.Model(2, 2, 2, Q=0, **c), 8, seed=0, precision="tf32x3")
    for node in (0, 4):
        ref.move_to(node)
        s.move_center(node)
    x = np.random.default_rng(42).standard_normal(s.node_size(4))
    s.set_precision("fp64")
    y = s.apply_heff(x)
    want = to_layout(ref.heff_apply(4, from_layout(x, ref.labels[4], ref.T[4].shape)), ref.labels[4])
    assert np.max(np.abs(y - want)) / np.max(np.abs(want)) < 1e-11
    s.close()
