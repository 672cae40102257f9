"""Batched sweeps (ttn_batch_sweep) against the same problems swept one by
one: independent problems with different charge sectors, couplings and
seeds, FP64 and mixed precision, with and without CUDA graphs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2011_10658_gb300 as pkg
    pkg.lib()
    return pkg


PROBLEMS_2x2x2 = [dict(t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0),
                  dict(t=1.0, m=0.5, ge2=2.0, cB=0.25, nu=20.0, Q=1),
                  dict(t=0.7, m=1.0, ge2=0.5, cB=1.0, nu=10.0, Q=-1)]


def make(q, L, chi, probs, prec, stream, seed0=7):
    return [q.TTN(q.Model(*L, **kw), chi, seed=seed0 + i, precision=prec, stream=stream)
            for i, kw in enumerate(probs)]


def run_case(q, L, chi, probs, prec, use_stream, sweeps, tol, rel):
    import torch
    st = torch.cuda.Stream() if use_stream else None
    handle = st.cuda_stream if st is not None else None
    batch = make(q, L, chi, probs, prec, handle)
    single = make(q, L, chi, probs, prec, handle)
    got = q.batch_sweep(batch, sweeps, tol=tol, max_krylov=32)
    for s, g in zip(single, got):
        want = s.sweep(sweeps, tol=tol, max_krylov=32)
        assert abs(g["energy"] - want["energy"]) < rel * abs(want["energy"]), (g, want)
        assert g["node_updates"] == want["node_updates"]
        assert g["not_converged"] == 0
    # the batch's states are ordinary states afterwards
    for s, b in zip(single, batch):
        assert abs(s.energy()[0] - b.energy()[0]) < rel * abs(s.energy()[0])
    return batch


@pytest.mark.parametrize("use_stream", [True, False], ids=["graphs", "default-stream"])
def test_batch_fp64_matches_single(q, use_stream):
    run_case(q, (2, 2, 2), 8, PROBLEMS_2x2x2, "fp64", use_stream, 2, 1e-12, 1e-10)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16"])
def test_batch_mixed_matches_single(q, prec):
    run_case(q, (2, 2, 2), 8, PROBLEMS_2x2x2, prec, True, 1, 1e-10, 1e-6)


def test_batch_4x4x4_uneven_sectors(q):
    """Charge sectors 0, 2, 4 and two couplings: uneven block counts."""
    probs = [dict(t=1.0, m=mm, ge2=g2, cB=1 / (2 * g2), nu=10.0 * max(1.0, g2 / 2), Q=qq)
             for qq, g2, mm in ((0, 0.5, 0.5), (2, 2.0, 1.0), (4, 0.5, 1.0))]
    run_case(q, (4, 4, 4), 12, probs, "tf32x3", True, 1, 1e-8, 1e-6)


def test_batch_rejects_mixed_sizes(q):
    a = q.TTN(q.Model(2, 2, 2), 8, seed=0)
    b = q.TTN(q.Model(2, 2, 1), 8, seed=0)
    with pytest.raises(q.QedError):
        q.batch_sweep([a, b], 1)
    with pytest.raises(q.QedError):
        q.batch_sweep([a, a], 1)
    c = q.TTN(q.Model(2, 2, 2), 8, seed=0, precision="tf32x3")
    with pytest.raises(q.QedError):
        q.batch_sweep([a, c], 1)
