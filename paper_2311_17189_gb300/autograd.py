"""torch.autograd.Function over the C ABI: the Monte Carlo mean Sigma_f of a diagram as a
differentiable function of the real frequencies omega_f (X_f = omega_f + i Gamma_f), the
chemical potential mu and the external momentum k_ext.

    sigma = SigmaMC.apply(diagram, omega, gamma, mu, kext, t, tp, beta, n, seed, offset[, save])

Forward calls tami_forward; backward calls tami_backward, which recomputes every term product
instead of storing them.  With save (default True) the forward also keeps each sample's line
energies and dE/dK factors (8 (N + 2 N_ext) bytes per sample) so that the backward need not
regenerate momenta and trig; the results are the same bits either way.  Gradients follow
PyTorch's convention for complex outputs.
"""
import torch


class SigmaMC(torch.autograd.Function):
    @staticmethod
    def forward(ctx, diagram, omega, gamma, mu, kext, t, tp, beta, n, seed, offset, save=True):
        X = torch.complex(omega.detach().to(torch.float64), gamma.detach().to(torch.float64).expand_as(omega))
        lat = (float(t), float(tp), float(mu), float(kext[0]), float(kext[1]))
        ctx.saved_rows = diagram.saved_buffer(n) if save and any(ctx.needs_input_grad) else None
        mean, _, _ = diagram.forward(lat, seed, offset, n, X, beta, save=ctx.saved_rows)
        ctx.diagram, ctx.X, ctx.lat, ctx.beta, ctx.n, ctx.seed, ctx.offset = diagram, X, lat, beta, n, seed, offset
        ctx.dev_kext = kext.device
        ctx.dtype_mu = mu.dtype
        return mean.clone()

    @staticmethod
    def backward(ctx, gout):
        out = ctx.diagram.backward(ctx.lat, ctx.seed, ctx.offset, ctx.n, ctx.X, ctx.beta,
                                   gout.to(torch.complex128).contiguous(), saved=ctx.saved_rows)
        g_omega = out["grad_X_re"]
        gp = out["grad_params"]
        g_mu = gp[0].to(ctx.dtype_mu)
        g_kext = gp[1:3].to(ctx.dev_kext)
        return None, g_omega, None, g_mu, g_kext, None, None, None, None, None, None, None
