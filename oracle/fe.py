"""Residual and exact Jacobian of the P4D DFN discretization (FP64, plain).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What is computed, following the paper:
* electrode level (section 3, "Spatial discretization for the electrode-level
  equations", eqs. ce-weak, phie-weak, phis-weak): continuous Q1 finite
  elements on a structured box mesh, every volume integral by 2x2x2 Gauss
  quadrature, the reaction terms by vertex (lumped) quadrature;
* particle level (section 3, "Spatial discretization of the particle
  equation", eqs. L1, L2, Lh, L0, LR, FD): the finite-difference radial
  operator per electrode node, weighted by the node's lumped electrode
  volume as in the weak form of Appendix A (eq. particle-weak);
* backward Euler in time (section 3, "Temporal discretization");
* Butler-Volmer kinetics (section 2, "Interfacial kinetics").

Readings taken where the paper is silent or inconsistent:
* the particle state lives on electrode *nodes* (one particle per node);
* the surface flux term of eq. LR enters with a minus sign (derived from
  the flux condition -D dc/dr = i_n/F);
* discharge uses a negative applied current density in eq. phis-weak;
* the diffusion-potential term of eq. phie-weak keeps the printed sign
  (parameter ``diffpot_sign``, default +1) and is discretized through the
  identity grad(c_e)/c_e = grad(ln c_e) with ln c_e replaced by its Q1
  nodal interpolant (the quadrature of the quotient is not specified by the
  paper): the term becomes the kappa_eff-weighted stiffness matrix applied
  to the nodal values of ln c_e and its Jacobian block is
  K_kappa diag(gamma / c_e).  Unlike the quotient grad(c_h)/c_h taken at the
  Gauss points (``diffpot_form="quad"``, kept for comparison), this form
  carries no ionic current when phi_e + gamma ln c_e is uniform, as in the
  continuous equations; on smooth fields the two forms' solutions differ by
  a vanishing fraction of the discretization error;
* the separator regularisation of phi_s is taken to its sigma -> 0 limit:
  phi_s exists only at electrode nodes; other nodes and the grounded face
  carry identity rows, and their phi_s values are lifted to zero wherever
  another row reads them;
* a = 3 eps_s / R_s (matches the tables: 1.5e5 = 3*0.5/1e-5,
  1.8e5 = 3*0.6/1e-5);
* current collectors (optional, the jelly-roll slab): a thin conducting
  foil on the z = Lz face (cathode) and on the z = 0 face (anode), each a
  surface conductance sigma_t = sigma_foil * thickness (S) entering the
  phi_s rows as the 2D Q1 stiffness of the face (bilinear quads, 2x2 Gauss,
  exact), only between active phi_s nodes like the bulk term; the applied
  current enters through the faces flagged in gamma_p and the grounded
  (Dirichlet) nodes are those of the faces flagged in gamma_n (tab strips).
  The paper meshes its collectors as layers; the shell replaces them.
"""
import numpy as np
import scipy.sparse as sp

G0 = 0.5 - 0.5 / np.sqrt(3.0)
G1 = 0.5 + 0.5 / np.sqrt(3.0)


class DomainError(ValueError):
    """A concentration left the domain of the kinetics (c_surf outside
    (0, c_max) or c_e <= 0)."""


def _reference_q1():
    """Q1 basis values and reference derivatives at the 2x2x2 Gauss points of
    the unit cube.  Local node l = a + 2b + 4c, Gauss point q likewise."""
    pts = (G0, G1)
    N = np.zeros((8, 8))
    dN = np.zeros((8, 8, 3))
    phi = (lambda t: 1.0 - t, lambda t: t)
    dphi = (-1.0, 1.0)
    for q in range(8):
        xq, yq, zq = pts[q & 1], pts[(q >> 1) & 1], pts[(q >> 2) & 1]
        for l in range(8):
            a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
            N[q, l] = phi[a](xq) * phi[b](yq) * phi[c](zq)
            dN[q, l, 0] = dphi[a] * phi[b](yq) * phi[c](zq)
            dN[q, l, 1] = phi[a](xq) * dphi[b] * phi[c](zq)
            dN[q, l, 2] = phi[a](xq) * phi[b](yq) * dphi[c]
    return N, dN


NREF, DREF = _reference_q1()
# Gauss weights on the unit cube are all 1/8.
MREF = NREF.T @ NREF / 8.0                                 # unit-cube mass
KREF = np.stack([DREF[:, :, d].T @ DREF[:, :, d] / 8.0 for d in range(3)])  # per-axis stiffness


def radial_operator(r, D, F):
    """Tridiagonal coefficients of the radial operator L_h (eqs. L1, L2, Lh,
    L0, LR) for node radii r[..., nc] (r[...,0] = 0, r[...,-1] = R) and
    diffusivity D[...].

    Returns (lo, di, up, beta): L_h(c)_i = lo_i c_{i-1} + di_i c_i + up_i c_{i+1}
    for the no-flux part, and the surface row additionally carries
    -beta * i_n with beta = 2 (1 + dr/R) / (F dr), dr = r_N - r_{N-1}.
    """
    r = np.asarray(r, float)
    D = np.asarray(D, float)[..., None]
    nc = r.shape[-1]
    lo = np.zeros(r.shape)
    di = np.zeros(r.shape)
    up = np.zeros(r.shape)
    # centre (eq. L0): 6 D / dr1^2 (c2 - c1)
    dr1 = r[..., 1] - r[..., 0]
    di[..., 0] = -6.0 * D[..., 0] / dr1 ** 2
    up[..., 0] = 6.0 * D[..., 0] / dr1 ** 2
    # interior (eqs. L1 + L2) with dr_i = r_{i+1} - r_i, dr_{i-1} = r_i - r_{i-1}
    for i in range(1, nc - 1):
        dri = r[..., i + 1] - r[..., i]
        drm = r[..., i] - r[..., i - 1]
        th = dri / drm
        ri = r[..., i]
        Di = D[..., 0]
        a1 = 2.0 * Di / (ri * dri * (1.0 + th))          # L1 prefactor
        a2 = 2.0 * Di / (dri * drm * (1.0 + th))         # L2 prefactor
        up[..., i] = a1 + a2
        lo[..., i] = -a1 * th ** 2 + a2 * th
        di[..., i] = -a1 * (1.0 - th ** 2) - a2 * (1.0 + th)
    # surface (eq. LR): 2 D / dr^2 (c_{N-1} - c_N) - 2 i_n/(F dr) (1 + dr/R)
    drN = r[..., -1] - r[..., -2]
    lo[..., -1] = 2.0 * D[..., 0] / drN ** 2
    di[..., -1] = -2.0 * D[..., 0] / drN ** 2
    beta = 2.0 * (1.0 + drN / r[..., -1]) / (F * drN)
    return lo, di, up, beta


def ocp_paper(theta, cathode):
    """The paper's open-circuit potentials (Appendix "Model Parameters",
    eqs. ocp_cathode and ocp_anode) and their derivatives dU/dtheta, for the
    surface stoichiometry theta; `cathode` selects the LiCoO2 curve per entry
    (else graphite)."""
    theta = np.asarray(theta, float)
    cathode = np.broadcast_to(np.asarray(cathode, bool), theta.shape)
    # LiCoO2, with t = 1.062 theta
    t = 1.062 * theta
    ta = [np.tanh(30.834 - 54.4806 * t), np.tanh(52.294 - 50.294 * t), np.tanh(11.0923 - 19.8543 * t),
          np.tanh(1.4684 - 5.4888 * t), np.tanh((-t + 0.56478) / 0.1316), np.tanh((t - 0.525) / 0.006)]
    Up = 2.16216 + 0.07645 * ta[0] + 2.1581 * ta[1] - 0.14169 * ta[2] + 0.2051 * ta[3] + 0.2531 * ta[4] \
        - 0.02167 * ta[5]
    dUp_dt = (0.07645 * -54.4806 * (1 - ta[0] ** 2) + 2.1581 * -50.294 * (1 - ta[1] ** 2)
              - 0.14169 * -19.8543 * (1 - ta[2] ** 2) + 0.2051 * -5.4888 * (1 - ta[3] ** 2)
              + 0.2531 * (-1.0 / 0.1316) * (1 - ta[4] ** 2) - 0.02167 * (1.0 / 0.006) * (1 - ta[5] ** 2))
    dUp = 1.062 * dUp_dt
    # graphite
    terms = [(0.0351, 0.286, 0.083), (-0.0045, 0.849, 0.119), (-0.035, 0.9233, 0.05), (-0.0147, 0.5, 0.034),
             (-0.102, 0.194, 0.142), (-0.022, 0.9, 0.0164), (-0.011, 0.124, 0.0226), (0.0155, 0.105, 0.029)]
    ex = np.exp(-120.0 * theta)
    Un = 0.194 + 1.5 * ex
    dUn = -180.0 * ex
    for amp, c0, w in terms:
        th = np.tanh((theta - c0) / w)
        Un = Un + amp * th
        dUn = dUn + amp / w * (1 - th ** 2)
    return np.where(cathode, Up, Un), np.where(cathode, dUp, dUn)


def transport_paper(ce, T=298.15, R=8.31446):
    """Bulk electrolyte conductivity kappa(c_e) and diffusivity D_e(c_e) of
    the paper (Appendix "Model Parameters", eqs. kappa_app and De_app, with
    their Arrhenius factors exp(E/R (1/298.15 - 1/T)), E = 34700 and
    37040 J/mol), with their derivatives with respect to c_e (mol/m^3)."""
    c = np.asarray(ce, float) / 1000.0
    ak = np.exp(34700.0 / R * (1.0 / 298.15 - 1.0 / T))
    ad = np.exp(37040.0 / R * (1.0 / 298.15 - 1.0 / T))
    kap = ak * (0.0911 + 1.9101 * c - 1.052 * c ** 2 + 0.1554 * c ** 3)
    dkap = ak * (1.9101 - 2.104 * c + 0.4662 * c ** 2) / 1000.0
    De = ad * 5.34e-10 * np.exp(-0.65 * c)
    dDe = -0.65e-3 * De
    return kap, dkap, De, dDe


class Disc:
    """Mesh bookkeeping and coefficients of one cell.

    ocp = "linear": the secant OCP of the parameters (the benchmark
    workloads); "paper": the paper's OCP curves.  transport = "constant":
    kappa and D_e of the parameters; "paper": the paper's
    concentration-dependent kappa(c_e), D_e(c_e), taken per element at the
    element mean of the nodal c_e (a reading: one-point quadrature of the
    coefficient; the Q1 integrals stay exact for it).  material = "paper"
    selects both."""

    def __init__(self, mesh, params, diffpot_form="ln", material=None, ocp="linear", transport="constant"):
        self.mesh = mesh
        self.p = dict(params)
        if material == "paper":
            ocp, transport = "paper", "paper"
        elif material not in (None, "constant"):
            raise ValueError(material)
        if diffpot_form not in ("ln", "quad") or ocp not in ("linear", "paper") or \
                transport not in ("constant", "paper"):
            raise ValueError((diffpot_form, ocp, transport))
        self.diffpot_form = diffpot_form
        self.ocp_model = ocp
        self.transport_model = transport
        nx, ny, nz = int(mesh["nx"]), int(mesh["ny"]), int(mesh["nz"])
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nnx, self.nny, self.nnz = nx + 1, ny + 1, nz + 1
        self.nn = self.nnx * self.nny * self.nnz
        self.nelem = nx * ny * nz
        k, j, i = [a.ravel() for a in np.indices((nz, ny, nx))]
        conn = np.empty((self.nelem, 8), np.int64)
        for l in range(8):
            a, b, c = l & 1, (l >> 1) & 1, (l >> 2) & 1
            conn[:, l] = (i + a) + self.nnx * ((j + b) + self.nny * (k + c))
        self.conn = conn
        hx, hy, hz = (np.asarray(mesh[h], float) for h in ("hx", "hy", "hz"))
        # axis lengths, summed in element order (the multigrid's coarsening
        # rule compares mean element sizes)
        self.lengths = tuple(sum(float(v) for v in a) for a in (hx, hy, hz))
        self.h = np.stack([hx[i], hy[j], hz[k]], axis=1)          # (nelem, 3)
        self.vol = self.h.prod(axis=1)
        region = np.asarray(mesh["region"])
        self.region = region
        an_el, ca_el = region == 0, region == 2
        el = an_el | ca_el
        self.el = el
        node_an = np.zeros(self.nn, bool)
        node_ca = np.zeros(self.nn, bool)
        node_an[conn[an_el].ravel()] = True
        node_ca[conn[ca_el].ravel()] = True
        if np.any(node_an & node_ca):
            raise ValueError("anode and cathode elements share a node")
        self.enodes = np.flatnonzero(node_an | node_ca)
        self.NE = self.enodes.size
        self.eidx = np.full(self.nn, -1, np.int64)
        self.eidx[self.enodes] = np.arange(self.NE)
        self.etype = np.where(node_an[self.enodes], 0, 1)
        eps = np.asarray(mesh["eps"], float)
        eps_s = np.asarray(mesh["eps_s"], float)
        Mn = np.zeros(self.nn)
        Sn = np.zeros(self.nn)
        np.add.at(Mn, conn[el].ravel(), np.repeat(self.vol[el] / 8.0, 8))
        np.add.at(Sn, conn[el].ravel(), np.repeat(eps_s[el] * self.vol[el] / 8.0, 8))
        self.M = Mn[self.enodes]
        self.S = Sn[self.enodes]
        self.Rs = np.asarray(mesh["Rs"], float)[self.enodes]
        if mesh.get("Ds_e") is not None:
            # particle diffusivity = volume-weighted mean of the node's electrode elements
            Dn = np.zeros(self.nn)
            np.add.at(Dn, conn[el].ravel(), np.repeat(np.asarray(mesh["Ds_e"], float)[el] * self.vol[el] / 8.0, 8))
            self.Ds = Dn[self.enodes] / self.M
        else:
            self.Ds = np.asarray(mesh["Ds"], float)[self.enodes]
        self.A = 3.0 * self.S / self.Rs
        p = self.p
        an = self.etype == 0
        self.kr = np.where(an, p["k_n"], p["k_p"])
        self.cmax = np.where(an, p["cmax_n"], p["cmax_p"])
        self.u0 = np.where(an, p["ocp_n"][0], p["ocp_p"][0])
        self.u1 = np.where(an, p["ocp_n"][1], p["ocp_p"][1])
        b = p["brug"]
        sig_reg = np.where(an_el, p["sigma_n"], np.where(ca_el, p["sigma_p"], 0.0))
        if mesh.get("sigma_e") is not None:
            sig_reg = np.where(el, np.asarray(mesh["sigma_e"], float), 0.0)
        self.sig_bulk = sig_reg
        self.sig = np.where(el, eps_s ** b * sig_reg, 0.0)
        self.eps_s_e = eps_s
        self.kap = eps ** b * p["kappa"]
        self.Deff = eps ** b * p["De"]
        self.eps = eps
        # applied-current face Gamma_p (z = Lz), grounded face Gamma_n (z = 0)
        fj, fi = [a.ravel() for a in np.indices((ny, nx))]
        area = hx[fi] * hy[fj]
        gp = np.asarray(mesh["gamma_p"]).astype(bool)
        gn = np.asarray(mesh["gamma_n"]).astype(bool)
        self.gpw = np.zeros(self.nn)
        self.dirichlet = np.zeros(self.nn, bool)
        for a in (0, 1):
            for bb in (0, 1):
                top = (fi + a) + self.nnx * ((fj + bb) + self.nny * nz)
                bot = (fi + a) + self.nnx * (fj + bb)
                np.add.at(self.gpw, top[gp], area[gp] / 4.0)
                self.dirichlet[bot[gn]] = True
        self.act = np.zeros(self.nn, bool)
        self.act[self.enodes] = True
        self.act[self.dirichlet] = False
        # thin collector shells on the z = Lz (cathode) and z = 0 (anode) faces
        self.shell = []
        for key, kk in (("shell_sigma_t_p", nz), ("shell_sigma_t_n", 0)):
            st_ = float(mesh.get(key, 0.0) or 0.0)
            if st_ > 0.0:
                fconn = np.stack([(fi + (l & 1)) + self.nnx * ((fj + ((l >> 1) & 1)) + self.nny * kk)
                                  for l in range(4)], axis=1)
                self.shell.append((st_, fconn, hx[fi], hy[fj]))
        self.nc = int(mesh["nc"])
        self.r = self.Rs[:, None] * np.asarray(mesh["rgrid"], float)[None, :]
        self.lo, self.di, self.up, self.beta = radial_operator(self.r, self.Ds, p["F"])
        self.ndof = 3 * self.nn + self.NE * self.nc

    # ------------------------------------------------------------------ state
    def state_from_case(self, st):
        """Compact a generator state (c_s given per node) to electrode rows."""
        return dict(phis=np.asarray(st["phis"], float).copy(),
                    phie=np.asarray(st["phie"], float).copy(),
                    ce=np.asarray(st["ce"], float).copy(),
                    cs=np.asarray(st["cs_node"], float)[self.enodes].copy(),
                    ce_prev=np.asarray(st["ce_prev"], float).copy(),
                    cs_prev=np.asarray(st["cs_prev_node"], float)[self.enodes].copy())

    def pack(self, st):
        return np.concatenate([st["phis"], st["phie"], st["ce"], st["cs"].ravel()])

    def unpack(self, x):
        nn = self.nn
        return dict(phis=x[:nn], phie=x[nn:2 * nn], ce=x[2 * nn:3 * nn],
                    cs=x[3 * nn:].reshape(self.NE, self.nc))

    def with_values(self, st, x):
        out = dict(st)
        out.update({k: v.copy() for k, v in self.unpack(x).items()})
        return out

    # --------------------------------------------------------------- helpers
    def _lap(self, ue):
        """Unit-coefficient Q1 stiffness applied element-wise: (nelem, 8)."""
        out = np.zeros_like(ue)
        for d in range(3):
            out += (self.vol / self.h[:, d] ** 2)[:, None] * (ue @ KREF[d])
        return out

    @staticmethod
    def _shell_ke(sig_t, a, b):
        """2D Q1 stiffness of one face quad a x b times sig_t, local nodes
        l = x + 2 y: sig_t [(b/a) K1 (x) M1 + (a/b) M1 (x) K1] with
        K1 = [[1,-1],[-1,1]], M1 = [[1/3,1/6],[1/6,1/3]]."""
        K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
        M1 = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
        kx = np.kron(M1, K1)   # x fastest: index l = x + 2 y -> kron(Y, X)
        ky = np.kron(K1, M1)
        return sig_t * ((b / a)[:, None, None] * kx[None] + (a / b)[:, None, None] * ky[None])

    def _diffpot_quad(self, ce_e):
        """The diffusion-potential integrals with the quotient grad(c_h)/c_h
        of the Q1 field c_h evaluated at the 2x2x2 Gauss points (the other
        reading of eq. phie-weak): (nelem, 8) values of
        int_e grad(c_h)/c_h . grad(N_l)."""
        cq = ce_e @ NREF.T                                   # (nelem, 8 points)
        out = np.zeros_like(ce_e)
        for d in range(3):
            g = (ce_e @ DREF[:, :, d].T) / self.h[:, d][:, None]      # d c_h / dx_d at the points
            w = (self.vol / 8.0 / self.h[:, d])[:, None]
            out += (w * g / cq) @ DREF[:, :, d]
        return out

    def _diffpot_quad_jac(self, ce_e):
        """Derivative of ``_diffpot_quad`` with respect to the element's
        nodal c_e: (nelem, 8, 8), [row l, column m]."""
        cq = ce_e @ NREF.T
        out = np.zeros((ce_e.shape[0], 8, 8))
        for d in range(3):
            hd = self.h[:, d][:, None, None]
            g = (ce_e @ DREF[:, :, d].T)[:, :, None] / hd                # (e, q, 1)
            dNq = DREF[None, :, :, d] / hd                               # (e, q, m)
            dcol = dNq / cq[:, :, None] - g * NREF[None] / cq[:, :, None] ** 2
            w = (self.vol / 8.0)[:, None, None]
            out += w * np.einsum("eql,eqm->elm", np.broadcast_to(dNq, dcol.shape), dcol)
        return out

    def _scatter(self, vals):
        return np.bincount(self.conn.ravel(), weights=vals.ravel(), minlength=self.nn)

    def kinetics(self, phis_l, phie, ce, cs_surf):
        """Butler-Volmer at the electrode nodes (section 2, "Interfacial
        kinetics").  Returns i_n and its partial derivatives with respect to
        phi_s, c_e and c_surf (d/dphi_e = -d/dphi_s)."""
        p = self.p
        ph_s, ph_e, c_e = phis_l[self.enodes], phie[self.enodes], ce[self.enodes]
        if np.any(c_e <= 0) or np.any(cs_surf <= 0) or np.any(cs_surf >= self.cmax):
            raise DomainError("concentration outside the kinetics domain")
        al = p["alpha"]
        f = p["F"] / (p["R"] * p["T"])
        theta = cs_surf / self.cmax
        U, dU = self.ocp(theta)
        eta = ph_s - ph_e - U
        i0 = self.kr * c_e ** al * (self.cmax - cs_surf) ** al * cs_surf ** (1.0 - al)
        ea = np.exp(al * f * eta)
        ec = np.exp(-(1.0 - al) * f * eta)
        i_n = i0 * (ea - ec)
        g_eta = i0 * f * (al * ea + (1.0 - al) * ec)
        g_c = al * i_n / c_e
        g_s = i_n * ((1.0 - al) / cs_surf - al / (self.cmax - cs_surf)) - g_eta * dU / self.cmax
        return i_n, g_eta, g_c, g_s

    def ocp(self, theta):
        """Open-circuit potential U and dU/dtheta at the electrode nodes."""
        if self.ocp_model == "paper":
            return ocp_paper(theta, self.etype == 1)
        return self.u0 + self.u1 * theta, self.u1

    def transport(self, ce):
        """Per-element kappa_eff, D_eff and their derivatives with respect to
        the element-mean c_e (zero for constant coefficients)."""
        epb = self.eps ** self.p["brug"]
        if self.transport_model == "constant":
            z = np.zeros(self.nelem)
            return epb * self.p["kappa"], epb * self.p["De"], z, z
        kap, dkap, De, dDe = transport_paper(ce[self.conn].mean(axis=1), self.p["T"], self.p["R"])
        return epb * kap, epb * De, epb * dkap, epb * dDe

    def _gamma(self):
        p = self.p
        return p["diffpot_sign"] * 2.0 * p["R"] * p["T"] * (1.0 - p["tplus"]) / p["F"]

    # -------------------------------------------------------------- residual
    def residual(self, st):
        """Monolithic residual [R_phis; R_phie; R_ce; R_cs] (section 4 eq. of
        the block residual)."""
        p = self.p
        dt = p["dt"]
        phis_l = np.where(self.act, st["phis"], 0.0)
        phie, ce, cs = st["phie"], st["ce"], st["cs"]
        if np.any(ce <= 0):
            raise DomainError("c_e <= 0")
        # electronic charge (eq. phis-weak)
        # element matrices have zero row sums, so each element (and face) acts
        # on its values shifted by their mean: the same sums without the
        # rounding of large products of nearly equal potentials (collector
        # shells carry conductances ~1e7 times the bulk ones)
        pe = phis_l[self.conn]
        R_s = self._scatter(self.sig[:, None] * self._lap(pe - pe.mean(axis=1, keepdims=True)))
        for sig_t, fconn, a, b in self.shell:
            Ke = self._shell_ke(sig_t, a, b)
            pf = phis_l[fconn]
            R_s += np.bincount(fconn.ravel(),
                               weights=np.einsum("fij,fj->fi", Ke, pf - pf.mean(axis=1, keepdims=True)).ravel(),
                               minlength=self.nn)
        # ionic charge (eq. phie-weak); diffusion potential through the Q1
        # interpolant of ln c_e (or, for comparison, the quotient at the
        # Gauss points)
        kap, Deff, _, _ = self.transport(ce)
        if self.diffpot_form == "quad":
            dp = self._gamma() * kap[:, None] * self._diffpot_quad(ce[self.conn])
        else:
            dp = self._gamma() * kap[:, None] * self._lap(np.log(ce)[self.conn])
        R_e = self._scatter(kap[:, None] * self._lap(phie[self.conn]) + dp)
        # electrolyte transport (eq. ce-weak), consistent mass
        dce = (ce - st["ce_prev"])[self.conn]
        R_c = self._scatter((self.eps * self.vol)[:, None] * (dce @ MREF) / dt
                            + Deff[:, None] * self._lap(ce[self.conn]))
        # reactions (vertex quadrature)
        i_n, *_ = self.kinetics(phis_l, phie, ce, cs[:, -1])
        tau = (1.0 - p["tplus"]) / p["F"]
        en = self.enodes
        R_s[en] += self.A * i_n
        R_e[en] -= self.A * i_n
        R_c[en] -= tau * self.A * i_n
        R_s -= p["i_app"] * self.gpw
        R_s[~self.act] = st["phis"][~self.act]
        # particles (eqs. FD, particle-weak)
        L = self.di * cs
        L[:, 1:] += self.lo[:, 1:] * cs[:, :-1]
        L[:, :-1] += self.up[:, :-1] * cs[:, 1:]
        L[:, -1] -= self.beta * i_n
        R_p = self.M[:, None] * ((cs - st["cs_prev"]) / dt - L)
        return np.concatenate([R_s, R_e, R_c, R_p.ravel()])

    # -------------------------------------------------------------- Jacobian
    def jacobian(self, st):
        """Exact derivative of ``residual`` as a CSR matrix (section 4 eq.
        blocks)."""
        p = self.p
        dt = p["dt"]
        nn, NE, nc = self.nn, self.NE, self.nc
        phis_l = np.where(self.act, st["phis"], 0.0)
        phie, ce, cs = st["phie"], st["ce"], st["cs"]
        rows, cols, vals = [], [], []

        def add(r, c, v):
            rows.append(np.asarray(r).ravel())
            cols.append(np.asarray(c).ravel())
            vals.append(np.broadcast_to(v, np.shape(r)).ravel() if np.ndim(v) == 0 else np.asarray(v).ravel())

        R8 = np.broadcast_to(self.conn[:, :, None], (self.nelem, 8, 8))
        C8 = np.broadcast_to(self.conn[:, None, :], (self.nelem, 8, 8))
        Ke = np.zeros((self.nelem, 8, 8))
        for d in range(3):
            Ke += (self.vol / self.h[:, d] ** 2)[:, None, None] * KREF[d][None]
        Me = self.vol[:, None, None] * MREF[None]
        # phi_s - phi_s (active rows and columns only)
        keep = self.el[:, None, None] & self.act[R8] & self.act[C8]
        add(R8[keep], C8[keep], (self.sig[:, None, None] * Ke)[keep])
        for sig_t, fconn, a, b in self.shell:
            Kf = self._shell_ke(sig_t, a, b)
            R4 = np.broadcast_to(fconn[:, :, None], Kf.shape)
            C4 = np.broadcast_to(fconn[:, None, :], Kf.shape)
            kf = self.act[R4] & self.act[C4]
            add(R4[kf], C4[kf], Kf[kf])
        kap, Deff, dkap, dDeff = self.transport(ce)
        # phi_e - phi_e
        add(nn + R8, nn + C8, kap[:, None, None] * Ke)
        # phi_e - c_e: derivative of the diffusion-potential term, K_kappa diag(gamma / c_e)
        if self.diffpot_form == "quad":
            Be = (self._gamma() * kap)[:, None, None] * self._diffpot_quad_jac(ce[self.conn])
            ue = self._gamma() * self._diffpot_quad(ce[self.conn])
        else:
            Be = (self._gamma() * kap)[:, None, None] * Ke / ce[self.conn][:, None, :]
            ue = self._gamma() * self._lap(np.log(ce)[self.conn])
        # ... and of kappa(c_e) through the element mean: (dkappa/8) (K_e u)_l in every column
        ue = ue + self._lap(phie[self.conn])
        Be = Be + (dkap / 8.0)[:, None, None] * ue[:, :, None]
        add(nn + R8, 2 * nn + C8, Be)
        # c_e - c_e (with dD_e/dc_e through the element mean)
        Ce = (self.eps / dt)[:, None, None] * Me + Deff[:, None, None] * Ke
        Ce = Ce + (dDeff / 8.0)[:, None, None] * self._lap(ce[self.conn])[:, :, None]
        add(2 * nn + R8, 2 * nn + C8, Ce)
        # identity rows of phi_s
        ina = np.flatnonzero(~self.act)
        add(ina, ina, 1.0)
        # reactions
        i_n, ge, gc, gs = self.kinetics(phis_l, phie, ce, cs[:, -1])
        tau = (1.0 - p["tplus"]) / p["F"]
        en = self.enodes
        a_ = self.act[en]
        csN = 3 * nn + np.arange(NE) * nc + (nc - 1)
        A = self.A
        Mb = self.M * self.beta
        # rows: (row index, row weight) for phi_s, phi_e, c_e, c_s(N)
        for rix, w, only_act in ((en, A, True), (nn + en, -A, False),
                                 (2 * nn + en, -tau * A, False), (csN, Mb, False)):
            m = a_ if only_act else np.ones(NE, bool)
            ms = m & a_
            add(rix[ms], en[ms], (w * ge)[ms])                # d/dphi_s (lifted)
            add(rix[m], nn + en[m], -(w * ge)[m])             # d/dphi_e
            add(rix[m], 2 * nn + en[m], (w * gc)[m])          # d/dc_e
            add(rix[m], csN[m], (w * gs)[m])                  # d/dc_surf
        # particle tridiagonals: M (I/dt - L_h)
        base = 3 * nn + np.arange(NE)[:, None] * nc + np.arange(nc)[None, :]
        Mcol = self.M[:, None]
        add(base, base, Mcol * (1.0 / dt - self.di))
        add(base[:, 1:], base[:, :-1], -Mcol * self.lo[:, 1:])
        add(base[:, :-1], base[:, 1:], -Mcol * self.up[:, :-1])
        J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.ndof, self.ndof)).tocsr()
        J.sum_duplicates()
        return J

    # ------------------------------------------------------------- utilities
    def field_slices(self):
        nn = self.nn
        return [slice(0, nn), slice(nn, 2 * nn), slice(2 * nn, 3 * nn), slice(3 * nn, self.ndof)]
