"""The allocation-free H_eff entry point (ttn_apply_heff_device_noalloc),
for callers whose device memory belongs to another allocator and who cannot
let a library call cudaMalloc or cudaFree.  It must give the same product as
ttn_apply_heff_device on an FP64 state, call after call, whether it runs
first in a fresh process or after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)


@pytest.mark.parametrize("L,chi,node", [((2, 2, 2), 8, 0), ((4, 2, 2), 16, 1)])
def test_noalloc_matches_allocating_entry_point(L, chi, node):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as q
    s = q.TTN(q.Model(*L, **KW), chi, seed=2, precision="fp64")
    s.move_center(node)
    n = s.node_size(node)
    g = torch.Generator(device="cpu").manual_seed(7)
    for call in range(2):
        x = torch.randn(n, dtype=torch.float64, generator=g).cuda()
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, float("nan"))
        s.apply_heff_device(x.data_ptr(), y_ref.data_ptr(), n)
        s.apply_heff_device_noalloc(x.data_ptr(), y_new.data_ptr(), n)
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), call
    s.close()


def test_noalloc_rejects_upper_centre():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as q
    s = q.TTN(q.Model(2, 2, 2, **KW), 8, seed=2, precision="fp64")
    root = s.info()["center"]
    n = s.node_size(root)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(q.QedError):
        s.apply_heff_device_noalloc(x.data_ptr(), y.data_ptr(), n)
    s.close()


def test_noalloc_first_on_a_fresh_state():
    """The allocation-free call runs before any other product on a newly
    built state (centre moved to a bottom node), and agrees with the
    allocating entry point called afterwards, twice in a row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as q
    s = q.TTN(q.Model(2, 2, 2, **KW), 8, seed=5, precision="fp64")
    s.move_center(2)
    n = s.node_size(2)
    g = torch.Generator(device="cpu").manual_seed(11)
    for call in range(2):
        x = torch.randn(n, dtype=torch.float64, generator=g).cuda()
        y_new = torch.full_like(x, float("nan"))
        y_ref = torch.empty_like(x)
        s.apply_heff_device_noalloc(x.data_ptr(), y_new.data_ptr(), n)
        torch.cuda.synchronize()
        s.apply_heff_device(x.data_ptr(), y_ref.data_ptr(), n)
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), call
    s.close()
