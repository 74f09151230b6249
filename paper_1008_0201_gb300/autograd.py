"""torch.autograd.Function over the batched Jacobi eigensolver and its adjoint kernel.

JacobiEigh.apply(G, J, opts, deg_tol) takes a stack of square factors G (batch, n, n) of
H = G J G^T (J = I when J is None) and returns (lam, U): eigenvalues ascending (batch, n) and
orthonormal eigenvectors (batch, n, n), computed by jacobi_eig_batched.  Its backward maps
(lam_bar, U_bar) to G_bar = 2 H_bar G J through jacobi_eig_backward, where
H_bar = U sym(diag(lam_bar) + F o (U^T U_bar)) U^T.  Both directions run in the library's
kernels; this module only marshals tensors.
"""
import torch

from . import binding


class JacobiEigh(torch.autograd.Function):
    @staticmethod
    def forward(ctx, G, J=None, opts=None, deg_tol=1e-12):
        if opts is None:
            opts = binding.default_opts(want_v=0)
        out = binding.jacobi_eig_batched_uniform(G.detach(), J, opts, want_u=True)
        lam, U = out["lam"], out["U"]
        ctx.deg_tol = deg_tol
        ctx.save_for_backward(G.detach(), lam, U, J if J is not None else torch.empty(0))
        ctx.has_j = J is not None
        ctx.set_materialize_grads(False)  # an unused output passes None, not zeros
        return lam, U

    @staticmethod
    def backward(ctx, lam_bar, U_bar):
        G, lam, U, J = ctx.saved_tensors
        need_g = ctx.needs_input_grad[0]
        _, G_bar = binding.jacobi_eig_backward(lam, U, lam_bar, U_bar, ctx.deg_tol, G=G if need_g else None,
                                               J=J if ctx.has_j else None)
        return G_bar, None, None, None


def eigh_factor(G, J=None, opts=None, deg_tol=1e-12):
    """(lam, U) of H = G J G^T for a stack of square factors, differentiable w.r.t. G."""
    return JacobiEigh.apply(G, J, opts, deg_tol)


def eigh_backward_H(lam, U, lam_bar=None, U_bar=None, deg_tol=1e-12):
    """dL/dH for H = U diag(lam) U^T given dL/dlam and dL/dU (the adjoint kernel alone)."""
    H_bar, _ = binding.jacobi_eig_backward(lam, U, lam_bar, U_bar, deg_tol)
    return H_bar
