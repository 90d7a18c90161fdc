"""torch.autograd.Function around ns_solve / ns_backward.

``null_space(A, k, s)`` returns W (n x k), the k trailing right singular vectors
of the SRHT sketch of A (Algorithm 1), and sigma_k.  Gradients flow to A
through the hand-written adjoint (ns_backward): exact for losses that depend
on W only through W W^T (components of dL/dW along span(W) are ignored, since
they cannot change W W^T).  sigma_k is returned without a gradient.
"""
import torch

from . import api


class NullSpace(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, k, s, seed):
        d = api.desc(api.NS_SRHT, s=s, seed=seed)
        Acm = A if A.stride(0) == 1 else api.colmajor(A)
        Vk, sk, save, status = api.ns_solve(d, Acm, k, save=True)
        ctx.save_for_backward(save, Vk)
        ctx.dims = (A.shape[0], A.shape[1], k, s, seed)
        ctx.status = status
        ctx.mark_non_differentiable(sk)
        return Vk, sk

    @staticmethod
    def backward(ctx, dVk, dsk):
        save, Vk = ctx.saved_tensors
        m, n, k, s, seed = ctx.dims
        d = api.desc(api.NS_SRHT, s=s, seed=seed)
        g = api.colmajor(dVk)
        dA = api.ns_backward(d, m, n, k, save, Vk, g)
        return dA, None, None, None


def null_space(A, k, s, seed=0):
    """W, sigma_k = Algorithm 1 with an SRHT sketch of size s; differentiable in A."""
    return NullSpace.apply(A, int(k), int(s), int(seed))
