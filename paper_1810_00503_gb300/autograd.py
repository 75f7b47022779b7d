"""torch.autograd.Function over the fused objective + adjoint kernels.

WFChi2.apply(s, q, problem, band) returns chi^2 per map for the whitened
spectra s (complex, (B, C, n, n/2+1)) with the band amplitudes q (float64,
(n_b,)) applied to the problem's signal power (Sec. 2.3, eq. pilin).  The
backward pass uses the gradient and the band derivatives that the forward
kernels produce (one operator pass computes both; nothing large is stored
beyond the gradient itself):

    d chi2 / d s   in torch's convention for complex inputs, i.e. the
                   derivative with respect to the real and imaginary parts of
                   every stored half-plane value: c_k * g_k, with c_k = 1 on the
                   kx = 0 and kx = n/2 columns and 2 elsewhere (each stored
                   interior mode stands for the pair k, -k), g the full-plane
                   gradient wf_eval returns;
    d chi2 / d q_l = (d chi2 / d log q_l) / q_l.

Derivatives with respect to s are meaningful along Hermitian-consistent
directions (spectra of real fields), which is the space the objective is
defined on.
"""
from __future__ import annotations

import torch


class WFChi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, q, problem, band):
        problem.set_band_scale(band, q)
        chi2, grad, dlogq = problem.eval_bands(s.contiguous(), band, q.numel())
        w = torch.full((s.shape[-1],), 2.0, dtype=torch.float64, device=s.device)
        w[0] = 1.0
        w[-1] = 1.0
        gs = grad * w.to(grad.real.dtype)
        ctx.save_for_backward(gs, dlogq, q)
        return chi2

    @staticmethod
    def backward(ctx, gout):
        gs, dlogq, q = ctx.saved_tensors
        gs_out = gs * gout.to(gs.real.dtype).view(-1, 1, 1, 1)
        gq = (gout.view(-1, 1) * dlogq).sum(0) / q
        return gs_out, gq, None, None


def chi2(s, q, problem, band):
    """chi^2 per map as a differentiable function of (s, q)."""
    return WFChi2.apply(s, q, problem, band)
