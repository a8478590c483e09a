"""torch.autograd.Function around la_step / la_backward (argument marshalling only).

``propagate(ctx, V0, pulse, amp, psi0, nsteps, t0)`` returns psi after ``nsteps`` least-action
steps; gradients flow to the pulse amplitudes ``amp`` (real, CPU or CUDA) and to ``psi0``.  The
backward pass is the library's discrete adjoint (a second relaxation on the forward factors),
not autograd through the kernels.  PyTorch passes complex gradients as 2 dL/dz^*; the library
works with dJ/dz^*, so the factor 2 is converted at the boundary.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch


class LeastActionPropagate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, amp, psi0, ctx, V0, pulse, nsteps, t0):
        if ctx.cfg.ckpt_every <= 0:
            raise ValueError("the context must be created with ckpt_every > 0 to differentiate")
        amp_list = [float(a) for a in amp.detach().cpu().numpy()]
        ctx.set_hamiltonian(V0, dataclasses.replace(pulse, amp=amp_list))
        psi = psi0.detach().clone().contiguous()
        ctx.step(psi, int(nsteps), float(t0))
        fctx.la = ctx
        fctx.ncomp = len(amp_list)
        fctx.amp_device = amp.device
        return psi

    @staticmethod
    def backward(fctx, grad_psi):
        dJ = (0.5 * grad_psi).contiguous()
        dpsi0 = torch.empty_like(grad_psi)
        g = fctx.la.backward(dJ, fctx.ncomp, dpsi0)
        grad_amp = torch.as_tensor(np.asarray(g), dtype=torch.float64, device=fctx.amp_device)
        return grad_amp, 2.0 * dpsi0, None, None, None, None, None


def propagate(ctx, V0, pulse, amp, psi0, nsteps: int, t0: float = 0.0):
    return LeastActionPropagate.apply(amp, psi0, ctx, V0, pulse, nsteps, t0)
