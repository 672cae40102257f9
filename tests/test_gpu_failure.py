"""Failure detection on the GPU without a GPU fault.

* A bounded mbarrier wait that runs out: the wait bound of the tensor-core
  kernels is set to zero polls, so every wait gives up at once; the kernel
  drains its MMAs, frees its tensor memory and returns, and the node update
  reports QED_ETIMEOUT.  The state stays usable: with the default bound the
  same update then equals the FP64 update from the same tensor.
* Non-finite input: a NaN planted in an imported tensor (QED_ENAN), on the
  host path (ttn_node_import) and on the device path (ttn_load_tensors).
* Device memory exhaustion: QED_FAIL_ALLOC_AFTER makes an allocation fail
  as cudaMalloc would (a host-side fake of the failing call), in a child
  process; ttn_create returns QED_ENOMEM and names the allocation."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KW = dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0)


def _q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as q
    return q


@pytest.mark.parametrize("precision", ["tf32x3", "bf16"])
def test_wait_timeout_reported_and_state_usable(precision):
    q = _q()
    model = q.Model(2, 2, 1, **KW)
    s = q.TTN(model, 8, seed=4, precision=precision)
    s.move_center(0)
    t0 = s.node_export(0)
    s.set_wait_limit(0)
    with pytest.raises(q.QedError) as ei:
        s.optimize_node(0, tol=1e-10)
    assert ei.value.code == -6
    s.set_wait_limit(-1)
    s.node_import(0, t0)
    e_mixed = s.optimize_node(0, tol=1e-10)
    r = q.TTN(model, 8, seed=4, precision="fp64")
    r.move_center(0)
    r.node_import(0, t0)
    e64 = r.optimize_node(0, tol=1e-10)
    assert abs(e_mixed - e64) <= 1e-9 * abs(e64)
    s.close()
    r.close()


def test_nan_import_rejected():
    q = _q()
    s = q.TTN(q.Model(2, 2, 1, **KW), 8, seed=4, precision="fp64")
    t = s.node_export(1)
    bad = t.copy()
    bad[len(bad) // 2] = np.nan
    with pytest.raises(q.QedError) as ei:
        s.node_import(1, bad)
    assert ei.value.code == -5
    # the tensor on the device is unchanged
    np.testing.assert_array_equal(s.node_export(1), t)
    arrays = [s.node_export(i) for i in range(s.info()["n_nodes"])]
    planted = [a.copy() for a in arrays]
    planted[0][3] = np.inf
    with pytest.raises(q.QedError) as ei:
        s.load_tensors(planted)
    assert ei.value.code == -5
    s.load_tensors(arrays)
    np.testing.assert_array_equal(s.node_export(0), arrays[0])
    s.close()


def test_injected_allocation_failure_reports_enomem():
    pytest.importorskip("torch")
    code = ("import paper_2011_10658_gb300 as q\n"
            "try:\n"
            "    q.TTN(q.Model(2, 2, 1), 8, seed=0)\n"
            "    print('NO-ERROR')\n"
            "except q.QedError as e:\n"
            "    print('CODE', e.code, str(e))\n")
    env = dict(os.environ, QED_FAIL_ALLOC_AFTER="3")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "CODE -2" in out.stdout and "injected" in out.stdout, out.stdout
