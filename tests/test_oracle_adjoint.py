"""Pin of the oracle's adjoint gradient against central finite differences
of the terminal voltage after a short backward-Euler discharge."""
import numpy as np
import pytest

from p4d_inputs import make_box_case
from oracle.adjoint import gradient, forward


def _case():
    return make_box_case(3, 3, (3, 2, 3), 30e-6, (40e-6, 20e-6, 40e-6), 4, 21, state="initial")


@pytest.mark.parametrize("material", ["constant", "paper"])
def test_adjoint_gradient_matches_central_differences(material):
    case = _case()
    nelem = 3 * 3 * 8
    region = case["mesh"]["region"]
    sig0 = np.where(region == 0, case["params"]["sigma_n"], np.where(region == 2, case["params"]["sigma_p"], 0.0))
    Ds0 = np.full(nelem, 1e-14)
    eps0 = case["mesh"]["eps"].copy()
    nsteps = 3
    V, gs, gD, ge = gradient(case, nsteps, sigma_e=sig0, Ds_e=Ds0, eps_e=eps0, material=material)
    rng = np.random.default_rng(5)
    el = np.flatnonzero((region == 0) | (region == 2))
    for e in rng.choice(el, 4, replace=False):
        for name, base, g in (("sigma", sig0, gs), ("Ds", Ds0, gD), ("eps", eps0, ge)):
            h = 1e-4 * base[e]
            vals = []
            for sgn in (+1, -1):
                p = base.copy()
                p[e] += sgn * h
                kw = dict(sigma_e=sig0, Ds_e=Ds0, eps_e=eps0)
                kw[{"sigma": "sigma_e", "Ds": "Ds_e", "eps": "eps_e"}[name]] = p
                vals.append(forward(case, nsteps, material=material, **kw)[2])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[e] == pytest.approx(fd, rel=2e-4, abs=1e-9 * abs(V) / base[e]), (name, e, g[e], fd)
