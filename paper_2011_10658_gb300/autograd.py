"""torch.autograd.Function over the library's energy gradient.

E(psi; t, m, ge2, cB, nu) = psi^T H_eff psi / psi^T psi at one TTN node.
Forward and backward call ttn_energy_grad; the backward recomputes the
operator products (ttn_apply_heff and the adjoint ttn_apply_heff_adjoint)
instead of keeping them from the forward.  This module only marshals
arguments between torch tensors and the C ABI.
"""
import torch

from . import CLASSES


class EnergyFn(torch.autograd.Function):
    """E = EnergyFn.apply(psi, couplings, state, node).

    psi: contiguous CUDA float64 tensor in the centre layout of ``node``;
    couplings: float64 tensor (t, m, ge2, cB, nu) equal to the model's
    couplings (it carries the autograd graph of, e.g., g^2 -> (ge2, cB));
    state: a TTN; node: the node the centre is moved to.  Returns a 0-d
    float64 tensor on the CPU.  Gradients: dE/dpsi (device) and dE/dcouplings
    (Hellmann-Feynman values; E is linear in the couplings)."""

    @staticmethod
    def forward(ctx, psi, couplings, state, node):
        if not (psi.is_cuda and psi.dtype == torch.float64 and psi.is_contiguous()):
            raise ValueError("psi must be a contiguous CUDA float64 tensor")
        p = state.model.params
        want = torch.tensor([p.t, p.m, p.ge2, p.cB, p.nu], dtype=torch.float64)
        got = couplings.detach().to("cpu", torch.float64)
        if not torch.allclose(got, want, rtol=1e-12, atol=0.0):
            raise ValueError("couplings differ from the state's model")
        torch.cuda.current_stream().synchronize()
        e, _ = state.energy_grad_device(node, psi.data_ptr(), None, psi.numel())
        ctx.state, ctx.node = state, node
        ctx.save_for_backward(psi)
        return torch.tensor(e, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        (psi,) = ctx.saved_tensors
        grad = torch.empty_like(psi)
        torch.cuda.current_stream().synchronize()
        _, dc = ctx.state.energy_grad_device(ctx.node, psi.data_ptr(), grad.data_ptr(), psi.numel())
        gc = torch.tensor([dc[c] for c in CLASSES], dtype=torch.float64)
        g = g.detach().to(torch.float64)
        return grad * g.to(grad.device), gc * g.cpu(), None, None
