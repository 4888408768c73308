"""Seeded generators for the synthetic cells (see package docstring)."""
import math
import numpy as np

# Physical constants and material data (paper, Appendix "Model Parameters":
# constants, electrolyte, cathode, anode and separator tables).  D_s, D_e,
# kappa, sigma and eps_e follow the homogeneous-cube workload definition.
PARAMS_DEFAULT = dict(
    F=96485.33, R=8.31446, T=298.15, tplus=0.4, brug=1.5,
    De=7.5e-10, kappa=1.0,
    sigma_n=100.0, sigma_p=10.0,
    k_n=2e-5, k_p=6e-7,
    cmax_n=2.5e4, cmax_p=5.12e4,
    alpha=0.5,
    # linear OCP U(theta) = c0 + c1*theta (secants, see ocp_linear_secants)
    ocp_n=(0.229016, -0.067279), ocp_p=(4.948384, -1.535617),
    dt=10.0, i_app=-40.2022,
    diffpot_sign=1.0,
)

CASES = ("tiny", "cube8", "cube128", "hetero128")


def ocp_curve_p(th):
    """The paper's LiCoO2 open-circuit potential (Appendix, eq. for the
    cathode), used here only to draw the linear secants."""
    t = 1.062 * th
    return (2.16216 + 0.07645 * math.tanh(30.834 - 54.4806 * t)
            + 2.1581 * math.tanh(52.294 - 50.294 * t)
            - 0.14169 * math.tanh(11.0923 - 19.8543 * t)
            + 0.2051 * math.tanh(1.4684 - 5.4888 * t)
            + 0.2531 * math.tanh((-t + 0.56478) / 0.1316)
            - 0.02167 * math.tanh((t - 0.525) / 0.006))


def ocp_curve_n(th):
    """The paper's graphite open-circuit potential (Appendix, eq. for the
    anode), used here only to draw the linear secants."""
    return (0.194 + 1.5 * math.exp(-120.0 * th)
            + 0.0351 * math.tanh((th - 0.286) / 0.083)
            - 0.0045 * math.tanh((th - 0.849) / 0.119)
            - 0.035 * math.tanh((th - 0.9233) / 0.05)
            - 0.0147 * math.tanh((th - 0.5) / 0.034)
            - 0.102 * math.tanh((th - 0.194) / 0.142)
            - 0.022 * math.tanh((th - 0.9) / 0.0164)
            - 0.011 * math.tanh((th - 0.124) / 0.0226)
            + 0.0155 * math.tanh((th - 0.105) / 0.029))


def ocp_linear_secants():
    """Secant lines of the paper's OCP curves over the stoichiometry ranges
    the seeded states draw from: anode theta in [0.5, 0.8], cathode theta in
    [0.4, 0.6].  Returns ((c0_n, c1_n), (c0_p, c1_p))."""
    def secant(f, a, b):
        s = (f(b) - f(a)) / (b - a)
        return (f(a) - s * a, s)
    return secant(ocp_curve_n, 0.5, 0.8), secant(ocp_curve_p, 0.4, 0.6)


def theoretical_iapp(Lx, Ly, Ln, Lp, eps_s_n, eps_s_p, cmax_n, cmax_p, F, crate=1.0):
    """Applied current density for a C-rate from the theoretical capacity
    (paper, Appendix: Q_i = F eps_s,i V_i c_max,i / 3600, Q = min, I = C Q).
    Returned negative: discharge makes the cathode reaction cathodic."""
    area = Lx * Ly
    q_n = F / 3600.0 * eps_s_n * area * Ln * cmax_n
    q_p = F / 3600.0 * eps_s_p * area * Lp * cmax_p
    return -crate * min(q_n, q_p) / area


def _layers(n_an, n_sep, n_ca, L_an, L_sep, L_ca):
    hz = np.concatenate([np.full(n_an, L_an / n_an), np.full(n_sep, L_sep / n_sep),
                         np.full(n_ca, L_ca / n_ca)])
    reg_z = np.concatenate([np.zeros(n_an, np.uint8), np.ones(n_sep, np.uint8),
                            np.full(n_ca, 2, np.uint8)])
    return hz, reg_z


def _node_types(nx, ny, nz, region):
    """Anode/cathode flags per node (used only to pick which stoichiometry
    range a node's seeded state is drawn from)."""
    r = region.reshape(nz, ny, nx)
    an = np.zeros((nz + 1, ny + 1, nx + 1), bool)
    ca = np.zeros_like(an)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                an[dk:dk + nz, dj:dj + ny, di:di + nx] |= (r == 0)
                ca[dk:dk + nz, dj:dj + ny, di:di + nx] |= (r == 2)
    return an.ravel(), ca.ravel()


def radial_grid(nc, theta_bar=None):
    """Radial node positions r / R_s, r_0 = 0 and r_{nc-1} = 1.  Uniform when
    theta_bar is None; otherwise a geometric progression (paper section 3,
    the regular graded particle mesh) whose spacings shrink toward the
    surface by the constant factor theta_bar^(1/(nc-2)), so that the last
    spacing is theta_bar times the first (0 < theta_bar < 1)."""
    if theta_bar is None:
        return np.linspace(0.0, 1.0, nc)
    q = theta_bar ** (1.0 / (nc - 2))
    dr = q ** np.arange(nc - 1)
    r = np.concatenate([[0.0], np.cumsum(dr)])
    r /= r[-1]
    r[-1] = 1.0
    return r


def make_box_case(nx, ny, nz_layers, L_lat, L_layers, nc, seed, *, params=None,
                  hetero=False, rs_cv=0.0, state="seeded", Rs=5e-6, Ds=1e-14,
                  eps_e=0.3, eps_s=(0.6, 0.5), theta_bar=None):
    """Layered anode/separator/cathode box.

    state="seeded": linearization state with c_e = 1000(1 + U(-0.05, 0.05)),
    anode theta ~ U(0.5, 0.8), cathode theta ~ U(0.4, 0.6) per node, c_s
    uniform in r, previous step equal to the state and open-circuit
    potentials (phi_s = 0 in the anode, phi_e = -U_n(0.65),
    phi_s = U_p(0.5) - U_n(0.65) in the cathode).
    state="initial": c_e = 1000, theta_n = 0.8, theta_p = 0.6, open circuit.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    p = dict(PARAMS_DEFAULT)
    if params:
        p.update(params)
    n_an, n_sep, n_ca = nz_layers
    L_an, L_sep, L_ca = L_layers
    nz = n_an + n_sep + n_ca
    Lx, Ly = (L_lat, L_lat) if np.isscalar(L_lat) else L_lat
    hx = np.full(nx, Lx / nx)
    hy = np.full(ny, Ly / ny)
    hz, reg_z = _layers(n_an, n_sep, n_ca, L_an, L_sep, L_ca)
    nelem = nx * ny * nz
    region = np.repeat(reg_z, nx * ny).astype(np.uint8)
    eps = np.where(region == 1, 1.0, eps_e).astype(np.float64)
    eps_s_arr = np.where(region == 0, eps_s[0], np.where(region == 2, eps_s[1], 0.0))
    if hetero:
        eps, eps_s_arr = _hetero_fields(nx, ny, nz, hx, hy, hz, region, rng)
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    Rs_node = np.full(nn, Rs)
    if rs_cv > 0:
        s2 = math.log(1 + rs_cv ** 2)
        Rs_node = np.exp(math.log(Rs) - s2 / 2 + math.sqrt(s2) * rng.standard_normal(nn))
        Rs_node = np.clip(Rs_node, 1e-6, 20e-6)
    Ds_node = np.full(nn, Ds)
    gamma_p = np.ones(nx * ny, np.uint8)
    gamma_n = np.ones(nx * ny, np.uint8)
    if "i_app" not in (params or {}):
        p["i_app"] = theoretical_iapp(Lx, Ly, L_an, L_ca, eps_s[0], eps_s[1],
                                      p["cmax_n"], p["cmax_p"], p["F"])
    an, ca = _node_types(nx, ny, nz, region)
    (c0n, c1n), (c0p, c1p) = p["ocp_n"], p["ocp_p"]
    if state == "seeded":
        ce = 1000.0 * (1.0 + rng.uniform(-0.05, 0.05, nn))
        th_n = rng.uniform(0.5, 0.8, nn)
        th_p = rng.uniform(0.4, 0.6, nn)
        thn_ref, thp_ref = 0.65, 0.5
    else:
        ce = np.full(nn, 1000.0)
        th_n = np.full(nn, 0.8)
        th_p = np.full(nn, 0.6)
        thn_ref, thp_ref = 0.8, 0.6
    cs_node = np.zeros((nn, nc))
    cs_node[an] = (th_n[an] * p["cmax_n"])[:, None]
    cs_node[ca] = (th_p[ca] * p["cmax_p"])[:, None]
    un_ref = c0n + c1n * thn_ref
    up_ref = c0p + c1p * thp_ref
    phis = np.zeros(nn)
    phis[ca] = up_ref - un_ref
    phie = np.full(nn, -un_ref)
    mesh = dict(nx=nx, ny=ny, nz=nz, hx=hx, hy=hy, hz=hz, region=region, eps=eps,
                eps_s=eps_s_arr, Rs=Rs_node, Ds=Ds_node, gamma_p=gamma_p,
                gamma_n=gamma_n, nc=nc, rgrid=radial_grid(nc, theta_bar))
    st = dict(phis=phis, phie=phie, ce=ce, cs_node=cs_node, ce_prev=ce.copy(),
              cs_prev_node=cs_node.copy())
    return dict(mesh=mesh, params=p, state=st, seed=seed)


def _hetero_fields(nx, ny, nz, hx, hy, hz, region, rng, corr=8, mean=0.3, cv=0.2):
    """Lognormal porosity with correlation length `corr` elements: Gaussian
    samples on a coarse grid of `corr`-element spacing, trilinearly
    interpolated to element centres, smoothed by a few Jacobi sweeps of
    (I - h_c^2 Lap) g~ = g on the element grid, normalised to zero mean and
    unit variance, then eps = exp(mu + s g~) with mean 0.3 and CV 0.2 in the
    electrodes (clamped to [0.05, 0.7]); eps_s = 1 - eps - eps_b with binder
    fractions 0.1 (anode) and 0.2 (cathode)."""
    cz, cy, cx = nz // corr + 2, ny // corr + 2, nx // corr + 2
    g = rng.standard_normal((cz, cy, cx))
    zc = (np.arange(nz) + 0.5) / corr
    yc = (np.arange(ny) + 0.5) / corr
    xc = (np.arange(nx) + 0.5) / corr
    def interp1(arr, coords, axis):
        i0 = np.floor(coords).astype(int)
        t = coords - i0
        a = np.take(arr, i0, axis=axis)
        b = np.take(arr, i0 + 1, axis=axis)
        shape = [1, 1, 1]
        shape[axis] = -1
        t = t.reshape(shape)
        return a * (1 - t) + b * t
    f = interp1(interp1(interp1(g, zc, 0), yc, 1), xc, 2)
    # smoothing: damped Jacobi on (I - hc^2 Lap) with hc = corr (element units)
    h2 = float(corr) ** 2
    gt = f.copy()
    for _ in range(40):
        lap = -6 * gt
        for ax in range(3):
            lap += np.roll(gt, 1, ax) + np.roll(gt, -1, ax)
        res = f - (gt - h2 * lap)
        gt = gt + 0.8 * res / (1 + 6 * h2)
    gt = (gt - gt.mean()) / gt.std()
    s2 = math.log(1 + cv ** 2)
    mu = math.log(mean) - s2 / 2
    eps_field = np.clip(np.exp(mu + math.sqrt(s2) * gt), 0.05, 0.7).ravel()
    eps = np.where(region == 1, 1.0, eps_field)
    eps_b = np.where(region == 0, 0.1, np.where(region == 2, 0.2, 0.0))
    eps_s = np.where((region == 0) | (region == 2), 1.0 - eps - eps_b, 0.0)
    return eps, eps_s


def make_slab_case(nx=2048, ny=16, layers=(20, 8, 20), nc=15, seed=1005, tab=64, crate=2.0,
                   h_lat=100e-6 / 128, L_layers=(100e-6, 25e-6, 100e-6), shell=(0.0, 0.0),
                   state="initial", width=None):
    """Flattened jelly-roll-like slab: nx x ny elements of h_lat x h_lat
    laterally, anode/separator/cathode layers in z.  The tabs are the
    strips of the first `tab` element columns along x: gamma_p (applied
    current, z = Lz) and gamma_n (grounded, z = 0) flag only them, so the
    current runs along the electrodes to the tabs.  i_app is the C-rate
    current of the whole slab (theoretical capacity) spread over the tab
    area.  shell = (cathode, anode) collector-foil surface conductances in S
    (0: none); real foils (aluminium 3.77e7 S/m x 15 um = 565 S, copper
    5.96e7 S/m x 10 um = 596 S) are ~1e8 times the bulk conductance of a
    sub-micron element.  width: the slab's extent along y (default ny h_lat)."""
    Ly = ny * h_lat if width is None else width
    case = make_box_case(nx, ny, layers, (nx * h_lat, Ly), L_layers, nc, seed, state=state)
    m, p = case["mesh"], case["params"]
    col = np.arange(nx * ny) % nx
    m["gamma_p"] = (col < tab).astype(np.uint8)
    m["gamma_n"] = (col < tab).astype(np.uint8)
    m["shell_sigma_t_p"], m["shell_sigma_t_n"] = float(shell[0]), float(shell[1])
    p["i_app"] = crate * theoretical_iapp(nx * h_lat, Ly, L_layers[0], L_layers[2], 0.6, 0.5,
                                          p["cmax_n"], p["cmax_p"], p["F"]) * nx / tab
    return case


def make_tiny_case(nx=2, ny=2, layers=(2, 1, 2), nc=4, seed=7, **kw):
    """Small box for brute-force checks (lateral 20 um, 20/10/20 um thick)."""
    return make_box_case(nx, ny, layers, 20e-6, (20e-6, 10e-6, 20e-6), nc, seed, **kw)


def make_case(name, **kw):
    """Named workloads.

    cube8:      8x8x24 elements (10/4/10), 100 um lateral, 100/25/100 um,
                N_c = 10, seeded linearization state (seed 1001).
    cube128:    128x128x96 (40/16/40), same physics, N_c = 20 (seed 1002).
    hetero128:  cube128 mesh with lognormal porosity (mean 0.3, CV 0.2,
                correlation 8 elements) and lognormal particle radius
                (mean 5 um, CV 0.3) (seed 1003).
    cube96:     96x96x72 (30/12/30), cube128's physics at three quarters of
                its resolution (seed 1002); a profiling case whose level-0
                working set still exceeds the 129 MB L2.
    tiny:       2x2x5 (2/1/2), N_c = 4 (seed 7).
    """
    if name == "tiny":
        return make_tiny_case(**kw)
    if name == "cube8":
        return make_box_case(8, 8, (10, 4, 10), 100e-6, (100e-6, 25e-6, 100e-6), 10,
                             kw.pop("seed", 1001), **kw)
    if name == "cube128":
        return make_box_case(128, 128, (40, 16, 40), 100e-6, (100e-6, 25e-6, 100e-6), 20,
                             kw.pop("seed", 1002), **kw)
    if name == "cube96":
        return make_box_case(96, 96, (30, 12, 30), 100e-6, (100e-6, 25e-6, 100e-6), 20,
                             kw.pop("seed", 1002), **kw)
    if name == "hetero128":
        return make_box_case(128, 128, (40, 16, 40), 100e-6, (100e-6, 25e-6, 100e-6), 20,
                             kw.pop("seed", 1003), hetero=True, rs_cv=0.3, **kw)
    raise KeyError(name)


def make_gyroid_cell(n, t, periods, nc, seed, L_lat=100e-6, L_layers=(100e-6, 25e-6, 100e-6)):
    """Layered cube (anode/separator/cathode split 10/4/10 of nz = 1.5 n)
    whose electrode elements become electrolyte-only (region 3, eps = 1,
    eps_s = 0) where the gyroid level set
        g = sin X cos Y + sin Y cos Z + sin Z cos X,  (X, Y, Z) = 2 pi p (x, y, z) / L
    at the element centre is >= t.  Gamma_p / Gamma_n flag only the top /
    bottom faces of cathode / anode elements."""
    nz = (3 * n) // 2
    if nz % 12:
        raise ValueError("nz = 1.5 n must be a multiple of 12")
    layers = (nz * 10 // 24, nz * 4 // 24, nz * 10 // 24)
    case = make_box_case(n, n, layers, L_lat, L_layers, nc, seed)
    m = case["mesh"]
    hx, hy, hz = m["hx"], m["hy"], m["hz"]
    xc = np.cumsum(hx) - hx / 2
    yc = np.cumsum(hy) - hy / 2
    zc = np.cumsum(hz) - hz / 2
    Lz = hz.sum()
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    k = 2 * np.pi * periods
    Xs, Ys, Zs = k * X / L_lat, k * Y / L_lat, k * Z / Lz
    g = (np.sin(Xs) * np.cos(Ys) + np.sin(Ys) * np.cos(Zs) + np.sin(Zs) * np.cos(Xs)).ravel()
    region = m["region"].copy()
    void = ((region == 0) | (region == 2)) & (g >= t)
    region[void] = 3
    m["region"] = region
    m["eps"] = np.where(void, 1.0, m["eps"])
    m["eps_s"] = np.where(void, 0.0, m["eps_s"])
    nx = ny = n
    r3 = region.reshape(nz, ny, nx)
    m["gamma_p"] = (r3[-1] == 2).astype(np.uint8).ravel()
    m["gamma_n"] = (r3[0] == 0).astype(np.uint8).ravel()
    # 1C from the theoretical capacity of the remaining active material
    p = case["params"]
    vol = (hx[None, None, :] * hy[None, :, None] * hz[:, None, None]).ravel()
    qn = p["F"] / 3600 * np.sum((m["eps_s"] * vol)[region == 0]) * p["cmax_n"]
    qp = p["F"] / 3600 * np.sum((m["eps_s"] * vol)[region == 2]) * p["cmax_p"]
    area = np.sum((hx[None, :] * hy[:, None]).ravel()[m["gamma_p"].astype(bool)])
    p["i_app"] = -min(qn, qp) / area if area > 0 else 0.0
    case["gyroid"] = dict(n=n, t=t, periods=periods, nc=nc)
    return case


def make_tpms_cell(nx, ny, nz, nc=6, seed=1006, L=(1e-3, 1e-3, 0.5e-3), t=1.104, state="seeded"):
    """The paper's interpenetrating gyroid electrodes (section 5, Case IV)
    voxelised on an nx x ny x nz box mesh of L = (1, 1, 0.5) mm: with
    (X, Y, Z) = (pi x/Lx, pi y/Ly, pi z/Lz) at the element centre,
        s_n = sin X cos Y + sin Y cos Z + sin Z cos X - 1.3,
        s_p = sin X cos(Y + pi) + sin(Y + pi) cos(-Z) + sin(-Z) cos X - 1.3,
    an element is anode where |s_n| <= t/2, cathode where |s_p| <= t/2
    (t = 1.104), electrolyte-only elsewhere.  Cathode elements that share a
    node with an anode element become electrolyte-only (the two electrodes
    never touch).  The grounded face Gamma_n is the bottom (z = 0) face of
    the anode elements, the applied-current face Gamma_p the top face of the
    cathode elements; i_app is 1C of the active material's theoretical
    capacity.  N_c = 6 as in the paper's Case IV (Table tab:meshes)."""
    Lx, Ly, Lz = L
    rng = np.random.Generator(np.random.PCG64(seed))
    p = dict(PARAMS_DEFAULT)
    hx = np.full(nx, Lx / nx)
    hy = np.full(ny, Ly / ny)
    hz = np.full(nz, Lz / nz)
    xc = (np.arange(nx) + 0.5) / nx
    yc = (np.arange(ny) + 0.5) / ny
    zc = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(np.pi * zc, np.pi * yc, np.pi * xc, indexing="ij")
    s_n = np.sin(X) * np.cos(Y) + np.sin(Y) * np.cos(Z) + np.sin(Z) * np.cos(X) - 1.3
    s_p = np.sin(X) * np.cos(Y + np.pi) + np.sin(Y + np.pi) * np.cos(-Z) + np.sin(-Z) * np.cos(X) - 1.3
    region = np.full((nz, ny, nx), 3, np.uint8)
    region[np.abs(s_p) <= t / 2] = 2
    region[np.abs(s_n) <= t / 2] = 0
    an, _ = _node_types(nx, ny, nz, region.ravel())
    an3 = an.reshape(nz + 1, ny + 1, nx + 1)
    touch = np.zeros((nz, ny, nx), bool)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                touch |= an3[dk:dk + nz, dj:dj + ny, di:di + nx]
    region[(region == 2) & touch] = 3
    region = region.ravel()
    el = (region == 0) | (region == 2)
    eps = np.where(el, 0.3, 1.0)
    eps_s = np.where(region == 0, 0.6, np.where(region == 2, 0.5, 0.0))
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    r3 = region.reshape(nz, ny, nx)
    gamma_p = (r3[-1] == 2).astype(np.uint8).ravel()
    gamma_n = (r3[0] == 0).astype(np.uint8).ravel()
    vol = (hx[None, None, :] * hy[None, :, None] * hz[:, None, None]).ravel()
    qn = p["F"] / 3600 * np.sum((eps_s * vol)[region == 0]) * p["cmax_n"]
    qp = p["F"] / 3600 * np.sum((eps_s * vol)[region == 2]) * p["cmax_p"]
    area = np.sum((hx[None, :] * hy[:, None]).ravel()[gamma_p.astype(bool)])
    p["i_app"] = -min(qn, qp) / area if area > 0 else 0.0
    an, ca = _node_types(nx, ny, nz, region)
    (c0n, c1n), (c0p, c1p) = p["ocp_n"], p["ocp_p"]
    if state == "seeded":
        ce = 1000.0 * (1.0 + rng.uniform(-0.05, 0.05, nn))
        th_n = rng.uniform(0.5, 0.8, nn)
        th_p = rng.uniform(0.4, 0.6, nn)
        thn_ref, thp_ref = 0.65, 0.5
    else:
        ce = np.full(nn, 1000.0)
        th_n = np.full(nn, 0.8)
        th_p = np.full(nn, 0.6)
        thn_ref, thp_ref = 0.8, 0.6
    cs_node = np.zeros((nn, nc))
    cs_node[an] = (th_n[an] * p["cmax_n"])[:, None]
    cs_node[ca] = (th_p[ca] * p["cmax_p"])[:, None]
    phis = np.zeros(nn)
    phis[ca] = (c0p + c1p * thp_ref) - (c0n + c1n * thn_ref)
    phie = np.full(nn, -(c0n + c1n * thn_ref))
    mesh = dict(nx=nx, ny=ny, nz=nz, hx=hx, hy=hy, hz=hz, region=region, eps=eps, eps_s=eps_s,
                Rs=np.full(nn, 5e-6), Ds=np.full(nn, 1e-14), gamma_p=gamma_p, gamma_n=gamma_n, nc=nc,
                rgrid=np.linspace(0.0, 1.0, nc))
    st = dict(phis=phis, phie=phie, ce=ce, cs_node=cs_node, ce_prev=ce.copy(), cs_prev_node=cs_node.copy())
    return dict(mesh=mesh, params=p, state=st, seed=seed, tpms=dict(nx=nx, ny=ny, nz=nz, t=t))


def make_gyroid_batch(ncells=64, seed=1004, sizes=(16, 24, 32, 40, 48, 56, 64)):
    """Seeded batch of gyroid cells of uneven sizes: lateral n uniform over
    `sizes` (nz = 1.5 n), t ~ U(-0.3, 0.3), periods in {1, 2, 3}, N_c in 10..20."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = []
    for c in range(ncells):
        n = int(rng.choice(sizes))
        t = float(rng.uniform(-0.3, 0.3))
        per = int(rng.integers(1, 4))
        nc = int(rng.integers(10, 21))
        cells.append(make_gyroid_cell(n, t, per, nc, seed * 1000 + c))
    return cells
