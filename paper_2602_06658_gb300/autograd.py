"""torch.autograd.Function around the GW energy (forward: lift + gw_solve;
backward: the hand-written adjoint gw_grad_x).  Argument marshalling only;
all arithmetic runs in libgw's kernels."""

from __future__ import annotations

import torch

from . import (EN, PEN_SQEUCLID, PREC_FP32, gw_grad_x, gw_lift, gw_sgw, gw_solve)


class GWEnergy(torch.autograd.Function):
    """E = GW_eps(alpha, beta) for alpha = sum a_i delta_{x_i}, beta = sum
    b_j delta_{y_j} (Eq. entropic_gromov_wasserstein), with the gradient with
    respect to the source points x through the converged plan (Appendix B.6).

    penalty = PEN_SQEUCLID: features are the centered points (D = d).
    Otherwise the features are Kernel PCA features of dimension D and the
    gradient goes through Kernel-Proj (Algorithms 12-13)."""

    @staticmethod
    def forward(ctx, x, y, a, b, eps, n_outer, n_inner, penalty=PEN_SQEUCLID, param=2.0, D=None,
                prec=PREC_FP32, eps_final=0.0, Gamma0=None, seed=0):
        x = x.detach().contiguous()
        y = y.detach().contiguous()
        lifted = penalty != PEN_SQEUCLID
        Dx = x.shape[1] if not lifted else int(D)
        Dy = y.shape[1] if not lifted else int(D)
        lx = gw_lift(x, Dx, kind=penalty, param=param, w=a, want_basis=lifted, seed=seed)
        ly = gw_lift(y, Dy, kind=penalty, param=param, w=b, seed=seed + 1)
        out = gw_solve(lx["X"], ly["X"], lx["s"], ly["s"], a, b, eps, n_outer, n_inner,
                       eps_final=eps_final, prec=prec, record=False, Gamma0=Gamma0)
        ctx.save_for_backward(x, lx["X"], ly["X"], lx["s"], ly["s"], a, b, out["f"], out["g"],
                              out["Gamma_plan"], out["Gamma"])
        ctx.basis = (lx["V"], lx["lam"]) if lifted else None
        ctx.cfg = (penalty, param, prec)
        ctx.eps_last = float(out["energy"][EN["eps"]].item())
        return out["energy"][EN["E"]].clone()

    @staticmethod
    def backward(ctx, gE):
        x, X, Y, s, t, a, b, f, g, Gp, G = ctx.saved_tensors
        penalty, param, prec = ctx.cfg
        if ctx.basis is None:
            dX, _ = gw_grad_x(X, Y, s, t, a, b, f, g, Gp, G, ctx.eps_last, prec=prec)
            dx = dX
        else:
            V, lam = ctx.basis
            _, dx = gw_grad_x(X, Y, s, t, a, b, f, g, Gp, G, ctx.eps_last, prec=prec, x=x,
                              kind=penalty, param=param, basis=V, eigvals=lam)
        return (gE * dx, None, None, None, None, None, None, None, None, None, None, None, None,
                None)


def gw_energy_fn(x, y, a, b, eps, n_outer, n_inner, **kw):
    """Functional form: GWEnergy.apply with keyword options."""
    return GWEnergy.apply(x, y, a, b, eps, n_outer, n_inner, kw.get("penalty", PEN_SQEUCLID),
                          kw.get("param", 2.0), kw.get("D"), kw.get("prec", PREC_FP32),
                          kw.get("eps_final", 0.0), kw.get("Gamma0"), kw.get("seed", 0))


class SGWDivergence(torch.autograd.Function):
    """SGW_eps(alpha, beta) = GW_eps(alpha, beta) - (GW_eps(alpha, alpha) +
    GW_eps(beta, beta)) / 2 (Section 4.1), with the gradient with respect to
    the source points x (envelope theorem, the self term through both of its
    sides).  gw_sgw computes the value and the gradient in one call; the
    backward pass scales the stored gradient.  Penalties as GWEnergy."""

    @staticmethod
    def forward(ctx, x, y, a, b, eps, n_outer, n_inner, penalty=PEN_SQEUCLID, param=2.0, D=None,
                prec=PREC_FP32, eps_final=0.0, seed=0):
        x = x.detach().contiguous()
        y = y.detach().contiguous()
        lifted = penalty != PEN_SQEUCLID
        Dx = x.shape[1] if not lifted else int(D)
        Dy = y.shape[1] if not lifted else int(D)
        lx = gw_lift(x, Dx, kind=penalty, param=param, w=a, want_basis=lifted, seed=seed)
        ly = gw_lift(y, Dy, kind=penalty, param=param, w=b, seed=seed + 1)
        if lifted:
            out = gw_sgw(lx["X"], ly["X"], lx["s"], ly["s"], a, b, eps, n_outer, n_inner,
                         eps_final=eps_final, prec=prec, grad=True, x=x, kind=penalty,
                         param=param, basis=lx["V"], eigvals=lx["lam"])
            dx = out["dx"]
        else:
            out = gw_sgw(lx["X"], ly["X"], lx["s"], ly["s"], a, b, eps, n_outer, n_inner,
                         eps_final=eps_final, prec=prec, grad=True)
            dx = out["dX"]
        ctx.save_for_backward(dx)
        return out["sgw"][0].clone()

    @staticmethod
    def backward(ctx, gS):
        (dx,) = ctx.saved_tensors
        return (gS * dx, None, None, None, None, None, None, None, None, None, None, None, None)


def sgw_fn(x, y, a, b, eps, n_outer, n_inner, **kw):
    """Functional form: SGWDivergence.apply with keyword options."""
    return SGWDivergence.apply(x, y, a, b, eps, n_outer, n_inner, kw.get("penalty", PEN_SQEUCLID),
                               kw.get("param", 2.0), kw.get("D"), kw.get("prec", PREC_FP32),
                               kw.get("eps_final", 0.0), kw.get("seed", 0))
