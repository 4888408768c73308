"""GPU adjoint: Newton time stepping, terminal-voltage gradient through
torch.autograd (checkpointed), against the oracle's adjoint and against
central finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

from p4d_inputs import make_box_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07225_gb300 import build
    build.build()


def _case():
    return make_box_case(3, 3, (3, 2, 3), 30e-6, (40e-6, 20e-6, 40e-6), 4, 21, state="initial")


def _params(case):
    region = case["mesh"]["region"]
    sig0 = np.where(region == 0, case["params"]["sigma_n"], np.where(region == 2, case["params"]["sigma_p"], 0.0))
    return sig0, np.full(region.size, 1e-14), case["mesh"]["eps"].copy()


@pytest.mark.parametrize("laws", ["linear", "paper_ocp", "paper"])
def test_newton_step_matches_oracle(laws):
    """One backward-Euler step by Newton, with the linear OCP and constant
    transport, with the paper's OCP curves, and with the paper's OCP and
    concentration-dependent kappa(c_e), D_e(c_e)."""
    from paper_2602_07225_gb300 import P4DSolver
    from oracle.fe import Disc
    from oracle.krylov import time_step, per_field_error
    case = _case()
    okw = {"linear": {}, "paper_ocp": dict(ocp="paper"), "paper": dict(material="paper")}[laws]
    lkw = {"linear": {}, "paper_ocp": dict(ocp_model=1), "paper": dict(ocp_model=1, transport_model=1)}[laws]
    d = Disc(case["mesh"], case["params"], **okw)
    st0 = d.state_from_case(case["state"])
    st1, _ = time_step(d, st0, rtol=1e-13)
    s = P4DSolver(case, precision=1, rtol=1e-10, **lkw)
    st = s.state_tensors(case["state"])
    it, info = s.newton(st, rtol=1e-11)
    x = np.concatenate([st[k].cpu().numpy().ravel() for k in ("phis", "phie", "ce", "cs")])
    assert per_field_error(d, x, d.pack(st1))[0] < 1e-8
    assert it <= 10


@pytest.mark.parametrize("checkpoint,laws", [(1, "linear"), (2, "linear"), (2, "paper_ocp"), (2, "paper")])
def test_gradient_matches_oracle_adjoint(checkpoint, laws):
    from paper_2602_07225_gb300 import terminal_voltage
    from oracle.adjoint import gradient
    case = _case()
    sig0, Ds0, eps0 = _params(case)
    nsteps = 3
    okw = {"linear": {}, "paper_ocp": dict(ocp="paper"), "paper": dict(material="paper")}[laws]
    lkw = {"linear": {}, "paper_ocp": dict(ocp_model=1), "paper": dict(ocp_model=1, transport_model=1)}[laws]
    V_ref, gs, gD, ge = gradient(case, nsteps, sigma_e=sig0, Ds_e=Ds0, eps_e=eps0, **okw)
    t = [torch.tensor(a, requires_grad=True) for a in (sig0, Ds0, eps0)]
    V = terminal_voltage(*t, case, nsteps, checkpoint=checkpoint, **lkw)
    V.backward()
    assert V.item() == pytest.approx(V_ref, rel=1e-10)
    for g, ref in zip((t[0].grad, t[1].grad, t[2].grad), (gs, gD, ge)):
        g = g.numpy()
        assert np.max(np.abs(g - ref)) <= 1e-6 * np.max(np.abs(ref)), (np.max(np.abs(g - ref)), np.max(np.abs(ref)))


def test_gradient_matches_central_differences():
    """Central finite differences of the GPU forward on seeded elements
    (relative step 1e-5, Newton to 1e-12); agreement to 1e-5 relative, or
    the finite-difference noise floor for sensitivities close to zero."""
    from paper_2602_07225_gb300 import terminal_voltage
    case = _case()
    sig0, Ds0, eps0 = _params(case)
    nsteps = 3
    t = [torch.tensor(a, requires_grad=True) for a in (sig0, Ds0, eps0)]
    V = terminal_voltage(*t, case, nsteps, checkpoint=2, newton_rtol=1e-12)
    V.backward()
    region = case["mesh"]["region"]
    rng = np.random.default_rng(1005)
    el = np.flatnonzero((region == 0) | (region == 2))
    picks = rng.choice(el, 6, replace=False)
    for e in picks:
        for k, base in enumerate((sig0, Ds0, eps0)):
            h = 1e-5 * base[e]
            vals = []
            for sgn in (1, -1):
                p = [a.copy() for a in (sig0, Ds0, eps0)]
                p[k][e] += sgn * h
                vals.append(terminal_voltage(*[torch.tensor(a) for a in p], case, nsteps, checkpoint=2,
                                             newton_rtol=1e-12).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            g = t[k].grad[e].item()
            noise = 1e-12 * abs(V.item()) / h
            assert abs(g - fd) <= 1e-5 * abs(fd) + noise, (k, e, g, fd)
