"""Independent torch FP64 restatement of eq. Feps, differentiated by autograd.

Test infrastructure: it pins the hand-derived adjoint of the oracle.  The
forward is written from the paper (Sec. 2.3 eq. Meps, Sec. 3.1, Sec. 3.2 eq.
Feps, Sec. 4.1 implementation details) with torch.roll stencils; the gradient
is whatever autograd makes of it.  It shares no code with the oracle or with
the CUDA library.
"""
from __future__ import annotations

import torch


class _GuardedSqrt(torch.autograd.Function):
    """sqrt with derivative 0 where the argument is exactly 0 (the limit of
    d sqrt(softplus(D)) / dD as softplus underflows)."""

    @staticmethod
    def forward(ctx, x):
        r = torch.sqrt(x)
        ctx.save_for_backward(r)
        return r

    @staticmethod
    def backward(ctx, go):
        (r,) = ctx.saved_tensors
        safe = torch.where(r > 0, r, torch.ones_like(r))
        return torch.where(r > 0, go * 0.5 / safe, torch.zeros_like(r))


def _sh(u, dx, dy, dz):
    """value at (x,y,z) of u(x+dx, y+dy, z+dz), periodic; u is (nz, ny, nx)."""
    return torch.roll(u, shifts=(-dz, -dy, -dx), dims=(0, 1, 2))


def energy(u: torch.Tensor, p: dict) -> torch.Tensor:
    h, eps, xi = float(p.get("h", 1.0)), float(p["eps"]), float(p.get("xi", 1e-6))
    a20, a11, a02, a10, a01, a00 = [float(v) for v in p["a"]]
    well = int(p.get("well", 0))
    G = [(_sh(u, 1, 0, 0) - _sh(u, -1, 0, 0)) / (2 * h),
         (_sh(u, 0, 1, 0) - _sh(u, 0, -1, 0)) / (2 * h),
         (_sh(u, 0, 0, 1) - _sh(u, 0, 0, -1)) / (2 * h)]
    e3 = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    Hs = [[None] * 3 for _ in range(3)]
    for c in range(3):
        s = e3[c]
        Hs[c][c] = (_sh(u, *s) - 2 * u + _sh(u, -s[0], -s[1], -s[2])) / h**2
    for c in range(3):
        for d in range(c + 1, 3):
            s, t = e3[c], e3[d]
            pp = _sh(u, s[0] + t[0], s[1] + t[1], s[2] + t[2])
            pm = _sh(u, s[0] - t[0], s[1] - t[1], s[2] - t[2])
            mp = _sh(u, -s[0] + t[0], -s[1] + t[1], -s[2] + t[2])
            mm = _sh(u, -s[0] - t[0], -s[1] - t[1], -s[2] - t[2])
            Hs[c][d] = Hs[d][c] = (pp - pm - mp + mm) / (4 * h**2)
    g2 = G[0] ** 2 + G[1] ** 2 + G[2] ** 2
    rho = g2 + xi**2
    q = torch.sqrt(rho)
    Wp = u**3 - u if well == 1 else 2 * u * (1 - u) * (1 - 2 * u)
    w = Wp / eps
    M = [[-eps * Hs[i][j] + w * G[i] * G[j] / rho for j in range(3)] for i in range(3)]
    T = M[0][0] + M[1][1] + M[2][2]
    S = sum(M[i][j] ** 2 for i in range(3) for j in range(3))
    D = 2 * S - T**2
    P = torch.clamp(D, min=0) + xi * torch.log1p(torch.exp(-torch.abs(D) / xi))
    r = _GuardedSqrt.apply(P)
    e = ((a20 + a02 - a11) / (2 * eps) * S + a11 / (2 * eps) * T**2 + (a20 - a02) / (2 * eps) * T * r
         + (a10 + a01) / 2 * q * T + (a10 - a01) / 2 * q * r + a00 * eps * g2)
    return h**3 * e.sum()


def energy_and_grad(u_np, p):
    u = torch.tensor(u_np, dtype=torch.float64, requires_grad=True)
    E = energy(u, p)
    (g,) = torch.autograd.grad(E, u)
    return float(E.detach()), g.numpy()
