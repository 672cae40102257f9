"""Checkpoint round trip through ttn_save / ttn_load (GPU)."""
import numpy as np
import pytest

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


def test_save_load_round_trip(q, tmp_path):
    m = q.Model(2, 2, 2, **KW)
    s = q.TTN(m, 8, seed=0)
    for node in (0, 1, 4):
        s.optimize_node(node, tol=1e-10)
    path = tmp_path / "state.ttn"
    s.save(path)
    r = q.TTN.load(m, path)
    n = s.info()["n_nodes"]
    assert r.info()["center"] == n - 1
    for i in range(n):
        np.testing.assert_array_equal(r.node_export(i), s.node_export(i))
    assert r.energy()[0] == pytest.approx(s.energy()[0], rel=1e-13)
    # both continue identically
    assert r.optimize_node(2, tol=1e-10) == pytest.approx(s.optimize_node(2, tol=1e-10), rel=1e-12)


def test_load_rejects_other_model_and_corruption(q, tmp_path):
    m = q.Model(2, 2, 2, **KW)
    s = q.TTN(m, 8, seed=0)
    path = tmp_path / "state.ttn"
    s.save(path)
    with pytest.raises(q.QedError):
        q.TTN.load(q.Model(2, 2, 2, **dict(KW, m=0.5)), path)
    raw = bytearray(path.read_bytes())
    raw[200] ^= 0x01
    bad = tmp_path / "bad.ttn"
    bad.write_bytes(bytes(raw))
    with pytest.raises(q.QedError):
        q.TTN.load(m, bad)
    short = tmp_path / "short.ttn"
    short.write_bytes(bytes(raw[:100]))
    with pytest.raises(q.QedError):
        q.TTN.load(m, short)
