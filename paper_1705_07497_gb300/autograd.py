"""Differentiable forward and adjoint products, and an unrolled reconstruction.

``RadonForward`` (y = A x) and ``RadonAdjoint`` (x = A^T y) are
torch.autograd.Functions over the library's products: the backward of A is
the library's A^T product and the backward of A^T is its A product (the
adjoint identity <A x, y> = <x, A^T y>).  float32 tensors go through
ct_forward / ct_adjoint, float64 tensors through ct_forward_f64 /
ct_adjoint_f64.  Vectors are [N*N] or [N*N, B] (images) and [rows] or
[rows, B] (sinograms), the slice index innermost.

``split_bregman_unrolled`` writes anisotropic-TV split Bregman (Sec. 4 of the
paper, the system of Eq. SB_solve with "+ lambda K*K" and v = d - b) with a
fixed number of warm-started CG steps per update, in torch operations around
those Functions (and, for FP64 vectors, ``NormalOp``: the whole operator of
Eq. SB_solve in one library call), so that the reconstruction is
differentiable with respect to the data f.  Each Bregman update can be
wrapped in torch.utils.checkpoint, so the backward pass keeps one update's
graph at a time and recomputes it.
"""

import torch
from torch.utils.checkpoint import checkpoint


def _out(shape_like, rows, ref):
    extra = tuple(shape_like.shape[1:])
    return torch.empty((rows,) + extra, dtype=ref.dtype, device=ref.device)


class RadonForward(torch.autograd.Function):
    """y = A x (Sec. 1: the data term's M R); backward x_grad = A^T y_grad."""

    @staticmethod
    def forward(ctx, M, x):
        ctx.M = M
        x = x.contiguous()
        y = _out(x, M.rows, x)
        M.forward(x, y)
        return y

    @staticmethod
    def backward(ctx, g):
        M = ctx.M
        g = g.contiguous()
        gx = _out(g, M.cols, g)
        M.adjoint(g, gx)
        return None, gx


class RadonAdjoint(torch.autograd.Function):
    """x = A^T y; backward y_grad = A x_grad."""

    @staticmethod
    def forward(ctx, M, y):
        ctx.M = M
        y = y.contiguous()
        x = _out(y, M.cols, y)
        M.adjoint(y, x)
        return x

    @staticmethod
    def backward(ctx, g):
        M = ctx.M
        g = g.contiguous()
        gy = _out(g, M.rows, g)
        M.forward(g, gy)
        return None, gy


class NormalOp(torch.autograd.Function):
    """out = alpha A^T A x + lambda grad^T grad x on FP64 vectors, the library's
    fused ct_normal_f64 (two products and one stencil pass).  The operator is
    symmetric, so its backward is the same operator applied to the incoming
    gradient."""

    @staticmethod
    def forward(ctx, M, x, alpha, lam):
        ctx.M, ctx.alpha, ctx.lam = M, alpha, lam
        return _normal_f64(M, x.contiguous(), alpha, lam)

    @staticmethod
    def backward(ctx, g):
        return None, _normal_f64(ctx.M, g.contiguous(), ctx.alpha, ctx.lam), None, None


def _normal_f64(M, x, alpha, lam):
    from . import ct

    out = torch.empty_like(x)
    ct.ct_normal_f64(M.handle, alpha, lam, x, out, x.shape[1] if x.dim() == 2 else 1,
                     torch.cuda.current_stream(x.device).cuda_stream)
    return out


def radon(M, x):
    return RadonForward.apply(M, x)


def radon_adjoint(M, y):
    return RadonAdjoint.apply(M, y)


def _as_cols(t):
    return t if t.dim() == 2 else t.unsqueeze(1)


def grad2d(u, n):
    """Forward differences with a zero last difference, [N*N, B] -> two [N*N, B]."""
    U = u.view(n, n, -1)
    zx = torch.zeros_like(U[:, :1])
    zy = torch.zeros_like(U[:1])
    gx = torch.cat([U[:, 1:] - U[:, :-1], zx], dim=1)
    gy = torch.cat([U[1:] - U[:-1], zy], dim=0)
    return gx.reshape(n * n, -1), gy.reshape(n * n, -1)


def grad2d_adj(wx, wy, n):
    """Adjoint of grad2d."""
    WX = wx.view(n, n, -1)[:, :-1]
    WY = wy.view(n, n, -1)[:-1]
    zx = torch.zeros_like(WX[:, :1])
    zy = torch.zeros_like(WY[:1])
    out = torch.cat([zx, WX], dim=1) - torch.cat([WX, zx], dim=1)
    out = out + torch.cat([zy, WY], dim=0) - torch.cat([WY, zy], dim=0)
    return out.reshape(n * n, -1)


def shrink(x, gamma):
    return torch.sign(x) * torch.clamp(x.abs() - gamma, min=0.0)


def _normal_op(M, p, alpha, lam, n):
    """alpha A^T A p + lambda grad^T grad p: the fused library operator for FP64
    vectors; FP32 vectors compose the FP32 products with torch's differences."""
    if p.dtype == torch.float64:
        return NormalOp.apply(M, p, alpha, lam)
    return alpha * radon_adjoint(M, radon(M, p)) + lam * grad2d_adj(*grad2d(p, n), n)


def cg_unrolled(M, rhs, u, iters, alpha, lam, n):
    """`iters` steps of CG per slice on alpha A^T A + lambda grad^T grad, warm start u."""
    r = rhs - _normal_op(M, u, alpha, lam, n)
    p = r
    rr = (r * r).sum(dim=0)
    for _ in range(iters):
        q = _normal_op(M, p, alpha, lam, n)
        a = rr / (p * q).sum(dim=0)
        u = u + a * p
        r = r - a * q
        rn = (r * r).sum(dim=0)
        p = r + (rn / rr) * p
        rr = rn
    return u


def split_bregman_unrolled(M, f, alpha, lam, outer, inner, use_checkpoint=True):
    """Differentiable anisotropic-TV split Bregman with u0 = 0, d = b = 0.

    f: [rows] or [rows, B] (float32 or float64); returns u with f's layout
    ([N*N] or [N*N, B]).  Each update: rhs = alpha A^T f + lambda grad^T(d - b);
    u = CG_inner(rhs, warm start u); d = shrink(grad u + b, 1/lambda);
    b = b + grad u - d.
    """
    n = M.n
    squeeze = f.dim() == 1
    f2 = _as_cols(f)
    atf = alpha * radon_adjoint(M, f2)
    zeros = torch.zeros_like(atf)
    u, dx, dy, bx, by = zeros, zeros, zeros, zeros, zeros

    def update(u, dx, dy, bx, by, atf):
        rhs = atf + lam * grad2d_adj(dx - bx, dy - by, n)
        u = cg_unrolled(M, rhs, u, inner, alpha, lam, n)
        gx, gy = grad2d(u, n)
        dx = shrink(gx + bx, 1.0 / lam)
        dy = shrink(gy + by, 1.0 / lam)
        return u, dx, dy, bx + gx - dx, by + gy - dy

    for _ in range(outer):
        if use_checkpoint:
            u, dx, dy, bx, by = checkpoint(update, u, dx, dy, bx, by, atf, use_reentrant=False)
        else:
            u, dx, dy, bx, by = update(u, dx, dy, bx, by, atf)
    return u.squeeze(1) if squeeze else u
