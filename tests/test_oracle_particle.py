"""Pins of the oracle's radial finite-difference operator (paper section 3,
eqs. L1, L2, Lh, L0, LR and Remark on second-order accuracy) against the
textbook series solution and exact discrete lithium conservation."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle.fe import radial_operator

F = 96485.33


def _series(r, t, R, D, F0, nterms=200):
    """Sphere of radius R, initially uniform, constant influx F0 = D dc/dr(R)
    (Crank, The Mathematics of Diffusion, sphere with constant surface flux):
    c - c0 = F0 R / D [3Dt/R^2 + r^2/(2R^2) - 3/10
                        - (2R/r) sum sin(a_n r/R) / (a_n^2 sin a_n) exp(-D a_n^2 t/R^2)],
    a_n the positive roots of a cot a = 1."""
    alphas = [brentq(lambda a: np.tan(a) - a, n * np.pi + 1e-9, n * np.pi + np.pi / 2 - 1e-9)
              for n in range(1, nterms + 1)]
    r = np.asarray(r, float)
    s = np.zeros_like(r)
    for a in alphas:
        with np.errstate(invalid="ignore", divide="ignore"):
            sr = np.where(r > 0, (2 * R / np.where(r > 0, r, 1)) * np.sin(a * r / R), 2 * a)
        s += sr / (a ** 2 * np.sin(a)) * np.exp(-D * a ** 2 * t / R ** 2)
    return F0 * R / D * (3 * D * t / R ** 2 + r ** 2 / (2 * R ** 2) - 0.3 - s)


def _march(nc, R, D, i_n, t_end, nsteps, c0):
    r = np.linspace(0.0, R, nc)
    lo, di, up, beta = radial_operator(r[None], np.array([D]), F)
    L = np.diag(di[0]) + np.diag(lo[0, 1:], -1) + np.diag(up[0, :-1], 1)
    dt = t_end / nsteps
    A = np.eye(nc) / dt - L
    Ainv = np.linalg.inv(A)
    flux = np.zeros(nc)
    flux[-1] = -beta[0] * i_n
    c = np.full(nc, c0)
    for _ in range(nsteps):
        c = Ainv @ (c / dt + flux)
    return r, c


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_series_solution_constant_flux(sign):
    R, D, c0 = 5e-6, 1e-14, 2e4
    i_n = sign * 2.0                       # A/m^2, anodic removes lithium
    t_end = 0.2 * R ** 2 / D
    F0 = -i_n / F                           # influx (flux condition -D dc/dr = i_n / F)
    errs = []
    for nc in (11, 21, 41):
        r, c = _march(nc, R, D, i_n, t_end, 8000, c0)
        exact = c0 + _series(r, t_end, R, D, F0)
        scale = np.max(np.abs(exact - c0))
        errs.append(np.max(np.abs(c - exact)) / scale)
    assert errs[-1] < 2e-3
    # observed spatial order ~2 (Remark on local regularity): error ratios ~4
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 2.5
    # direction: anodic current (i_n > 0) lowers the surface concentration
    r, c = _march(21, R, D, i_n, t_end, 2000, c0)
    assert np.sign(c[-1] - c0) == -np.sign(i_n)


@pytest.mark.parametrize("nc", [3, 4, 5, 10, 15, 20])
@pytest.mark.parametrize("grading", [None, 0.3])
def test_discrete_lithium_conservation(nc, grading):
    """There is a positive weight vector w with w^T L_noflux = 0 and
    w^T (surface flux row) = -3 i_n / (F R) sum(w): the particle's weighted
    average changes exactly as the flux through its surface dictates."""
    R, D = 7e-6, 3e-14
    if grading is None:
        r = np.linspace(0, R, nc)
    else:
        # geometric progression, elements shrinking toward the surface
        q = grading ** (1.0 / max(nc - 2, 1))
        dr = q ** np.arange(nc - 1)
        r = np.concatenate([[0.0], np.cumsum(dr)]) * R / dr.sum()
    lo, di, up, beta = radial_operator(r[None], np.array([D]), F)
    L = np.diag(di[0]) + np.diag(lo[0, 1:], -1) + np.diag(up[0, :-1], 1)
    u, s, vt = np.linalg.svd(L.T)
    w = vt[-1]
    w = w / w.sum()
    assert s[-1] < 1e-10 * s[0]
    assert np.all(w >= -1e-14)
    assert w[-1] * beta[0] == pytest.approx(3.0 / (F * R), rel=1e-10)
