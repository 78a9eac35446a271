"""Differentiable NLL and fits on top of the C ABI.

`PwaNLL` is a torch.autograd.Function whose forward calls pwa_nll_grad (one
fused kernel evaluates the NLL of Eq. 3 and its Wirtinger gradient g =
dNLL/dV*) and whose backward returns the stored gradient; no arithmetic of
the likelihood happens here.

Gradient conventions (the paper asks for proper handling of derivatives with
respect to complex parameters, Sec. 6):
  * real parameters x = (Re V, Im V): dNLL/dRe V = 2 Re g, dNLL/dIm V = 2 Im g;
  * complex tensors: PyTorch stores, for a real loss, the conjugate Wirtinger
    derivative scaled as dL/dRe + i dL/dIm = 2 dL/dV*, i.e. 2 g.

`fit_lbfgs` minimises the NLL over x with torch.optim.LBFGS (strong-Wolfe
line search). `fit_fumili` is the fitter the paper uses (Sec. 4: FUMILI on
analytic gradients and Hessian, 5-10 iterations): Newton steps on the
library's FUMILI Hessian (pwa_hessian), damped Levenberg-Marquardt style.
"""
from __future__ import annotations

import numpy as np
import torch


class PwaNLL(torch.autograd.Function):
    """NLL(V) for one parameter set. V is either a real tensor of length 2N
    holding (Re V, Im V) or a complex tensor of length N; `lik` is a
    paper_1108_5673_gb300.Likelihood with events loaded and M built."""

    @staticmethod
    def forward(ctx, V, lik):
        v = V.detach().to("cpu")
        if v.is_complex():
            vc = v.to(torch.complex128).numpy()
        else:
            n = v.shape[0] // 2
            vc = v[:n].double().numpy() + 1j * v[n:].double().numpy()
        nll, g = lik.nll_grad(vc[None, :])
        ctx.complex_input = V.is_complex()
        ctx.g = g[0]
        ctx.device, ctx.dtype = V.device, V.dtype
        return torch.tensor(float(nll[0]), dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.g
        if ctx.complex_input:
            dv = torch.from_numpy(2.0 * g)
        else:
            dv = torch.from_numpy(np.concatenate([2.0 * g.real, 2.0 * g.imag]))
        dv = dv.to(device=ctx.device, dtype=ctx.dtype)
        return grad_out * dv, None


def nll(V, lik):
    """Differentiable NLL (see PwaNLL)."""
    return PwaNLL.apply(V, lik)


class PwaResNLL(torch.autograd.Function):
    """NLL(V, masses, widths) with free Breit-Wigner parameters. x is a real
    tensor (Re V [N], Im V [N], mass [R], width [R]); forward calls
    pwa_nll_grad_res (the amplitudes of the free waves are recomputed on the
    device from the stored m and Y on every call, nothing is cached between
    forward and backward but the gradient itself), backward returns
    (2 Re g, 2 Im g, dNLL/dM, dNLL/dGamma) with g = dNLL/dV*."""

    @staticmethod
    def forward(ctx, x, lik):
        v = x.detach().to("cpu").double().numpy()
        N, R = lik.n_waves, lik.n_free
        V = v[:N] + 1j * v[N:2 * N]
        nll, gV, gM, gW = lik.nll_grad_res(V, v[2 * N:2 * N + R], v[2 * N + R:2 * N + 2 * R])
        ctx.g = np.concatenate([2.0 * gV.real, 2.0 * gV.imag, gM, gW])
        ctx.device, ctx.dtype = x.device, x.dtype
        return torch.tensor(nll, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, grad_out):
        return grad_out * torch.from_numpy(ctx.g).to(device=ctx.device, dtype=ctx.dtype), None


def nll_res(x, lik):
    """Differentiable NLL with free masses and widths (see PwaResNLL)."""
    return PwaResNLL.apply(x, lik)


def fit_lbfgs(lik, V0, max_iter=500, history=10, grad_tol=None, change_tol=1e-10):
    """Minimise NLL over (Re V, Im V) from the complex start V0.

    torch.optim.LBFGS with a strong-Wolfe line search runs until
    |grad|_inf <= grad_tol (default 1e-6 * n_data), until the NLL or the
    parameters change by less than change_tol between iterations, or for
    max_iter iterations. Returns (V_hat complex128 [N], nll, info dict)."""
    V0 = np.asarray(V0, dtype=np.complex128)
    N = V0.shape[0]
    x = torch.tensor(np.concatenate([V0.real, V0.imag]), dtype=torch.float64, requires_grad=True)
    if grad_tol is None:
        grad_tol = 1e-6 * max(1, getattr(lik, "n_data", 1))
    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=max_iter, max_eval=4 * max_iter,
                            history_size=history, line_search_fn="strong_wolfe",
                            tolerance_grad=grad_tol, tolerance_change=change_tol)
    evals = [0]

    def closure():
        opt.zero_grad()
        f = nll(x, lik)
        f.backward()
        evals[0] += 1
        return f

    opt.step(closure)
    xv = x.detach().numpy().copy()
    V = xv[:N] + 1j * xv[N:]
    xt = torch.tensor(xv, requires_grad=True)
    f = nll(xt, lik)
    f.backward()
    st = opt.state[opt.param_groups[0]["params"][0]]
    return V, float(f.detach()), {"iterations": int(st.get("n_iter", 0)), "evaluations": evals[0],
                                  "grad_inf": float(xt.grad.abs().max())}


def fit_fumili(lik, V0, max_iter=50, grad_tol=None, change_tol=1e-12, damping=1e-3):
    """Minimise NLL over p = (Re V, Im V) from the complex start V0 with
    FUMILI steps on the library's Hessian (pwa_hessian, sum_i grad ln I_i
    grad ln I_i^T). The NLL does not depend on the global phase, and that
    direction is in the null space of H, so the phase is fixed first (V0
    rotated to a real positive V_0, Im V_0 held at zero) and the steps solve
    (H + lam diag(H)) dp = -grad NLL over the other 2N - 1 parameters. A step
    is accepted if the NLL falls (then lam /= 10), otherwise lam *= 10 and
    the step is retried. Stops when |grad|_inf <= grad_tol (default
    1e-6 * n_data), when an accepted step changes the NLL by less than
    change_tol relative, or after max_iter iterations.
    Returns (V_hat complex128 [N], nll, info dict)."""
    V = phase_fixed(np.asarray(V0, dtype=np.complex128))
    N = V.shape[0]
    keep = np.array([k for k in range(2 * N) if k != N])   # all but Im V_0
    if grad_tol is None:
        grad_tol = 1e-6 * max(1, getattr(lik, "n_data", 1))

    def value_grad(v):
        f, g = lik.nll_grad(v[None, :])
        return float(f[0]), np.concatenate([2.0 * g[0].real, 2.0 * g[0].imag])[keep]

    f, gr = value_grad(V)
    lam, it, evals, hessians = damping, 0, 1, 0
    while it < max_iter and np.abs(gr).max() > grad_tol:
        H = lik.hessian(V)[np.ix_(keep, keep)]
        hessians += 1
        d = np.diag(H).copy()
        accepted = False
        for _ in range(12):
            dp = np.zeros(2 * N)
            dp[keep] = np.linalg.solve(H + lam * np.diag(d), -gr)
            Vt = V + dp[:N] + 1j * dp[N:]
            ft, gt = value_grad(Vt)
            evals += 1
            if np.isfinite(ft) and ft < f:
                accepted = True
                break
            lam *= 10.0
        if not accepted:
            break
        it += 1
        change = f - ft
        V, f, gr = Vt, ft, gt
        lam = max(lam / 10.0, 1e-12)
        if change <= change_tol * max(1.0, abs(f)):
            break
    return V, f, {"iterations": it, "evaluations": evals, "hessians": hessians,
                  "grad_inf": float(np.abs(gr).max())}


def phase_fixed(V):
    """Remove the unobservable global phase: rotate so that V_0 is real and positive."""
    V = np.asarray(V, dtype=np.complex128)
    return V * np.exp(-1j * np.angle(V[..., :1]))
