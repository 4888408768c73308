"""Terminal voltage after a backward-Euler discharge as a differentiable
function of per-element bulk solid conductivity, solid diffusivity and
porosity (torch.autograd.Function), with checkpointed time steps.

Forward: Newton per step (p4d_newton_solve), states kept every
`checkpoint` steps.  Backward: per segment the states are recomputed, then
the discrete adjoint runs backwards in time:
    J_n^T lam_n = rhs_n          (p4d_jacobian_update + p4d_adjoint_solve)
    g += -lam_n^T dR_n/dp        (p4d_param_grad)
    rhs_{n-1} = -(dR_n/du_{n-1})^T lam_n   (p4d_adjoint_prev)
with rhs_N = dV/du_N (p4d_voltage_weights).  Every step is a libp4d call.
"""
import torch

from .solver import P4DSolver

_FIELDS = ("phis", "phie", "ce", "cs")


def _clone(st):
    return {k: v.clone() for k, v in st.items()}


class TerminalVoltage(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_e, Ds_e, eps_e, case, nsteps, checkpoint, opts):
        mesh = dict(case["mesh"])
        mesh["sigma_e"] = sigma_e.detach().cpu().double().numpy()
        mesh["Ds_e"] = Ds_e.detach().cpu().double().numpy()
        mesh["eps"] = eps_e.detach().cpu().double().numpy()
        c2 = dict(case)
        c2["mesh"] = mesh
        newton = dict(rtol=opts.pop("newton_rtol", 1e-11), maxit=opts.pop("newton_maxit", 20))
        s = P4DSolver(c2, **opts)
        st = s.state_tensors(case["state"])
        ckpt = {0: _clone(st)}
        for n in range(1, nsteps + 1):
            st["ce_prev"].copy_(st["ce"])
            st["cs_prev"].copy_(st["cs"])
            s.newton(st, **newton)
            if n % checkpoint == 0 or n == nsteps:
                ckpt[n] = _clone(st)
        q = s.voltage_weights()
        V = s.terminal_voltage(st["phis"])[0]
        ctx.solver, ctx.ckpt, ctx.nsteps, ctx.checkpoint, ctx.q, ctx.newton = s, ckpt, nsteps, checkpoint, q, newton
        ctx.in_device = sigma_e.device
        return V.detach().to(sigma_e.device)

    @staticmethod
    def backward(ctx, gV):
        s, ckpt, N, K = ctx.solver, ctx.ckpt, ctx.nsteps, ctx.checkpoint
        dev = s.device
        nel = s._nelem
        g = [torch.zeros(nel, dtype=torch.float64, device=dev) for _ in range(3)]
        rhs = ctx.q * gV.to(dev).double()
        starts = list(range(0, N, K))
        for a in reversed(starts):
            b = min(a + K, N)
            states = {a: _clone(ckpt[a])}
            st = _clone(ckpt[a])
            for n in range(a + 1, b + 1):
                st["ce_prev"].copy_(st["ce"])
                st["cs_prev"].copy_(st["cs"])
                s.newton(st, **ctx.newton)
                states[n] = _clone(st)
            for n in range(b, a, -1):
                sn = states[n]
                s.jacobian_update(sn)
                lam, info = s.solve(rhs, adjoint=True)
                s.param_grad(sn, lam, g[0], g[1], g[2])
                rhs = s.adjoint_prev(lam)
        out = [gi.to(ctx.in_device) for gi in g]
        return out[0], out[1], out[2], None, None, None, None


def terminal_voltage(sigma_e, Ds_e, eps_e, case, nsteps, checkpoint=5, **opts):
    """V(t_N) for per-element sigma, D_s, eps (tensors of nelem); solver
    options as P4DSolver keywords, plus newton_rtol / newton_maxit."""
    o = dict(precision=1, mode=1, rtol=1e-10, maxit=600)
    o.update(opts)
    return TerminalVoltage.apply(sigma_e, Ds_e, eps_e, case, int(nsteps), int(checkpoint), o)
