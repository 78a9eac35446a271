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
line search), in variables scaled by each wave's MC integral. `fit_fumili` is the fitter the paper uses (Sec. 4: FUMILI on
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


def wave_scales(lik):
    """s_a = sqrt(M_aa), the scale of wave a's contribution to the predicted
    yield (V^H M V has the diagonal terms |s_a V_a|^2), or None when the
    likelihood has no normalisation matrix at hand."""
    M = getattr(lik, "M", None)
    if M is None:
        return None
    s = np.sqrt(np.maximum(np.real(np.diag(M)), 0.0))
    return np.where(s > 0, s, 1.0)


def fit_lbfgs(lik, V0, max_iter=500, history=10, grad_tol=None, change_tol=1e-10, scaled=True):
    """Minimise NLL over (Re V, Im V) from the complex start V0.

    torch.optim.LBFGS with a strong-Wolfe line search. With `scaled` (the
    default, when the likelihood holds M) it works in u_a = s_a V_a,
    s_a = sqrt(M_aa): every wave then contributes |u_a|^2 to the yield's
    diagonal, the curvature is O(1) in every u direction and a statistical
    error of u is ~1/2, whereas the V of waves with small amplitudes are
    orders of magnitude larger than the rest (at 1M events x 20 waves the
    Hessian in V spans eigenvalues 5e-5..2 and L-BFGS in V stops tens of NLL
    units above the minimum). It runs until |grad_u|_inf <= grad_tol (default
    1e-3, about 1e-3 of a statistical error; unscaled: |grad_V|_inf <= 1e-6
    n_data), until the NLL or the parameters change by less than change_tol
    between iterations, or for max_iter iterations. If the line search stops
    above grad_tol (the NLL's FP32 noise), Newton steps on a Hessian from
    differences of the gradient finish the fit (2(2N - 1) gradients each).
    Returns (V_hat complex128 [N], nll, info dict)."""
    V0 = np.asarray(V0, dtype=np.complex128)
    N = V0.shape[0]
    s = wave_scales(lik) if scaled else None
    if s is None:
        s = np.ones(N)
        if grad_tol is None:
            grad_tol = 1e-6 * max(1, getattr(lik, "n_data", 1))
    elif grad_tol is None:
        grad_tol = 1e-3
    s2 = torch.from_numpy(np.concatenate([s, s]))
    x = torch.tensor(np.concatenate([(V0 * s).real, (V0 * s).imag]), dtype=torch.float64,
                     requires_grad=True)
    opt = torch.optim.LBFGS([x], lr=1.0, max_iter=max_iter, max_eval=4 * max_iter,
                            history_size=history, line_search_fn="strong_wolfe",
                            tolerance_grad=grad_tol, tolerance_change=change_tol)
    evals = [0]

    def closure():
        opt.zero_grad()
        f = nll(x / s2, lik)
        f.backward()
        evals[0] += 1
        return f

    opt.step(closure)
    st = opt.state[opt.param_groups[0]["params"][0]]
    sv = s2.numpy()

    def grad_u(u):
        xt = torch.tensor(u / sv, requires_grad=True)
        f = nll(xt, lik)
        f.backward()
        evals[0] += 1
        return float(f.detach()), xt.grad.numpy() / sv

    u = x.detach().numpy().copy()
    f, g = grad_u(u)
    polish = 0
    if np.abs(g).max() > grad_tol:
        # The line search compares NLL values; near the minimum the decrease
        # per step reaches the NLL's FP32 evaluation noise (~1e-4 at 1M
        # events) and the search stops short. The gradient stays accurate and
        # costs one evaluation, so the last steps are Newton steps on a
        # Hessian from central differences of the gradient.
        u, f, g, polish = _newton_on_gradient(grad_u, u, f, g, N, grad_tol)
    xv = u / sv
    V = xv[:N] + 1j * xv[N:]
    return V, f, {"iterations": int(st.get("n_iter", 0)), "evaluations": evals[0],
                  "newton_steps": polish,
                  "grad_inf": float(np.abs(g * sv).max()),
                  "grad_inf_scaled": float(np.abs(g).max())}


def _newton_on_gradient(grad_u, u, f, g, N, grad_tol, h=1e-3, max_steps=6):
    """Newton steps in the scaled variables u = (Re u, Im u) with the Hessian
    from central differences of the gradient (step h; a statistical error of
    u is ~1/2), Im u_0 held (the global phase is a null direction); a step is
    halved up to four times until max|g| falls. Stops at grad_tol, when no
    step lowers max|g|, or after max_steps. Returns (u, f, g, steps)."""
    keep = np.array([k for k in range(2 * N) if k != N])
    steps = 0
    for steps in range(1, max_steps + 1):
        H = np.empty((keep.size, keep.size))
        for j, k in enumerate(keep):
            e = np.zeros(2 * N)
            e[k] = h
            H[:, j] = (grad_u(u + e)[1][keep] - grad_u(u - e)[1][keep]) / (2 * h)
        H = 0.5 * (H + H.T)
        w, Q = np.linalg.eigh(H)
        if w.min() <= 0:          # not yet in the convex region: no Newton step
            break
        d = np.zeros(2 * N)
        d[keep] = -(Q @ ((Q.T @ g[keep]) / w))
        t, moved = 1.0, False
        for _ in range(5):
            fn, gn = grad_u(u + t * d)
            if np.isfinite(fn) and np.abs(gn).max() < np.abs(g).max():
                u, f, g, moved = u + t * d, fn, gn, True
                break
            t *= 0.5
        if not moved or np.abs(g).max() <= grad_tol:
            break
    return u, f, g, steps


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
