// Concentration-dependent electrolyte transport (p4d_params.transport_model
// = 1): the paper's bulk conductivity kappa(c_e) and diffusivity D_e(c_e)
// (Appendix "Model Parameters", eqs. kappa_app and De_app, with their
// Arrhenius factors at the cell temperature T), Bruggeman-scaled per
// element and evaluated at the element mean of the nodal c_e:
//   kappa_eff,e = eps_e^b kappa(cbar_e),  D_eff,e = eps_e^b D_e(cbar_e),
//   cbar_e = (1/8) sum of the element's nodal c_e.
// The element integrals stay exact Q1 forms with an element-constant
// coefficient; their derivative with respect to c_e passes through the mean
// (1/8 per node).  Rows of eqs. phie-weak and ce-weak:
//   R_phie += sum_e kappa_eff,e (K_e u_e)_l,      u = phi_e + gamma ln c_e
//   R_ce   += sum_e D_eff,e (K_e c_e)_l            (plus the consistent mass)
//   J: K_kappa(cbar) and M/dt + K_D(cbar) re-assembled at every
//      linearization, plus the rank-structured terms
//      (kappa'_eff,e / 8) (K_e u_e)_l (sum_m dc_m) and the same with D.
// K_e is the unit-coefficient Q1 stiffness of the box element; per element
// it is diagonal in the butterfly basis (per axis s = a + b, d = a - b):
// the 1D stiffness has eigenvalues 0 and 2/h, the 1D mass h/2 and h/6, so
// K_e v = H^T diag(lambda) H v / 8 with
// lambda_(a,b,c) = Kx(a) My(b) Mz(c) + Mx(a) Ky(b) Mz(c) + Mx(a) My(b) Kz(c).
//
// The multigrid preconditioner keeps the coefficients at the reference
// concentration c_e = 1000 mol/m^3 (set at p4d_setup); only the operator
// (Jacobian products, residual) follows the state.
#include <cmath>
#include "p4d_common.cuh"

namespace p4d {

void transport_reference(const p4d_params& p, double* kap, double* De) {
  double dk, dd;
  transport_bulk(1000.0, p.T, p.R, *kap, dk, *De, dd);
}

namespace {

struct TrArgs {
  Grid g;
  int nx, ny, nz;
  double brug, T, Rg, gamma;
  const double *hx, *hy, *hz;
  const double* eps;
};

// Unit-coefficient stiffness of the box element applied to v (in place):
// H^T diag(lambda) H v / 8.
__device__ inline void unit_stiffness(double (&v)[8], double hx, double hy, double hz) {
  const double K[3] = {2.0 / hx, 2.0 / hy, 2.0 / hz};
  const double Ms[3] = {hx / 2.0, hy / 2.0, hz / 2.0};
  const double Md[3] = {hx / 6.0, hy / 6.0, hz / 6.0};
#pragma unroll
  for (int st = 1; st < 8; st <<= 1)
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (!(l & st)) {
        const double p = v[l], q = v[l | st];
        v[l] = p + q;
        v[l | st] = p - q;
      }
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    const int a = l & 1, b = (l >> 1) & 1, c = (l >> 2) & 1;
    const double mx = a ? Md[0] : Ms[0], my = b ? Md[1] : Ms[1], mz = c ? Md[2] : Ms[2];
    const double kx = a ? K[0] : 0.0, ky = b ? K[1] : 0.0, kz = c ? K[2] : 0.0;
    v[l] *= (kx * my * mz + mx * ky * mz + mx * my * kz) * 0.125;
  }
#pragma unroll
  for (int st = 1; st < 8; st <<= 1)
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (!(l & st)) {
        const double p = v[l], q = v[l | st];
        v[l] = p + q;
        v[l | st] = p - q;
      }
}

__device__ __forceinline__ int64_t elem_node(const Grid& g, int i, int j, int k, int l) {
  return (i + (l & 1)) + (int64_t)g.nnx * ((j + ((l >> 1) & 1)) + (int64_t)g.nny * (k + ((l >> 2) & 1)));
}

// Per element: coef = (kappa_eff, D_eff, dkappa_eff/dcbar, dD_eff/dcbar) and
// GH = (K_e u_e, K_e c_e) with u = phi_e + gamma ln c_e (lnce: nodal ln c_e).
__global__ void k_transport_elem(TrArgs a, const double* __restrict__ phie, const double* __restrict__ ce,
                                 const double* __restrict__ lnce, double* __restrict__ coef,
                                 double* __restrict__ GH) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  if (e >= ne) return;
  const int i = (int)(e % a.nx), j = (int)((e / a.nx) % a.ny), k = (int)(e / ((int64_t)a.nx * a.ny));
  double u[8], c[8], cbar = 0.0;
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    const int64_t n = elem_node(a.g, i, j, k, l);
    c[l] = ce[n];
    u[l] = phie[n] + a.gamma * lnce[n];
    cbar += c[l];
  }
  cbar *= 0.125;
  double kap, dkap, De, dDe;
  transport_bulk(cbar, a.T, a.Rg, kap, dkap, De, dDe);
  const double epb = pow(a.eps[e], a.brug);
  coef[e] = epb * kap;
  coef[ne + e] = epb * De;
  coef[2 * ne + e] = epb * dkap;
  coef[3 * ne + e] = epb * dDe;
  const double hx = a.hx[i], hy = a.hy[j], hz = a.hz[k];
  unit_stiffness(u, hx, hy, hz);
  unit_stiffness(c, hx, hy, hz);
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    GH[l * ne + e] = u[l];
    GH[(8 + l) * ne + e] = c[l];
  }
}

// K_kappa and C = M_eps/dt + K_D (slots 1 and 2 of the FP64 stencils) with
// the per-element coefficients of the linearization state; same element
// integrals as the fixed assembly (2x2x2 Gauss, exact on boxes).
__global__ void k_assemble_transport(TrArgs a, const double* __restrict__ coef, double idt,
                                     double* __restrict__ Jst) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const Grid g = a.g;
  if (n >= g.nn) return;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  const int i = (int)(n % g.nnx);
  const int j = (int)((n / g.nnx) % g.nny);
  const int k = (int)(n / ((int64_t)g.nnx * g.nny));
  double Kk[27], Cc[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) Kk[o] = Cc[o] = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < 2; ++p) {
        const int ei = i - 1 + p, ej = j - 1 + q, ek = k - 1 + s;
        if (ei < 0 || ej < 0 || ek < 0 || ei >= a.nx || ej >= a.ny || ek >= a.nz) continue;
        const int64_t e = ei + (int64_t)a.nx * (ej + (int64_t)a.ny * ek);
        const double hx = a.hx[ei], hy = a.hy[ej], hz = a.hz[ek];
        const double vol = hx * hy * hz;
        const double kap = coef[e], De = coef[ne + e], mcoef = a.eps[e] * idt;
        const double ix2 = 1.0 / (hx * hx), iy2 = 1.0 / (hy * hy), iz2 = 1.0 / (hz * hz);
        const int an = 1 - p, bn = 1 - q, cn = 1 - s;
        for (int cc = 0; cc < 2; ++cc)
          for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
              const int o = (p + aa) + 3 * (q + bb) + 9 * (s + cc);
              const double sx = aa == an ? 1.0 : -1.0, mx = aa == an ? 1.0 / 3.0 : 1.0 / 6.0;
              const double sy = bb == bn ? 1.0 : -1.0, my = bb == bn ? 1.0 / 3.0 : 1.0 / 6.0;
              const double sz = cc == cn ? 1.0 : -1.0, mz = cc == cn ? 1.0 / 3.0 : 1.0 / 6.0;
              const double kf = vol * (sx * ix2 * my * mz + mx * sy * iy2 * mz + mx * my * sz * iz2);
              Kk[o] += kap * kf;
              Cc[o] += mcoef * vol * mx * my * mz + De * kf;
            }
      }
  const int64_t nn = g.nn;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    Jst[(1 * 27 + o) * nn + n] = Kk[o];
    Jst[(2 * 27 + o) * nn + n] = Cc[o];
  }
}

// Node rows of the transport integrals: rows[0][n] = sum_e kappa_eff,e (K_e u_e)_l,
// rows[1][n] = sum_e D_eff,e (K_e c_e)_l (l: the node's corner in e).
__global__ void k_transport_rows(TrArgs a, const double* __restrict__ coef, const double* __restrict__ GH,
                                 double* __restrict__ rows) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const Grid g = a.g;
  if (n >= g.nn) return;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  const int i = (int)(n % g.nnx);
  const int j = (int)((n / g.nnx) % g.nny);
  const int k = (int)(n / ((int64_t)g.nnx * g.nny));
  double se = 0.0, sc = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < 2; ++p) {
        const int ei = i - 1 + p, ej = j - 1 + q, ek = k - 1 + s;
        if (ei < 0 || ej < 0 || ek < 0 || ei >= a.nx || ej >= a.ny || ek >= a.nz) continue;
        const int64_t e = ei + (int64_t)a.nx * (ej + (int64_t)a.ny * ek);
        const int l = (1 - p) + 2 * (1 - q) + 4 * (1 - s);
        se += coef[e] * GH[l * ne + e];
        sc += coef[ne + e] * GH[(8 + l) * ne + e];
      }
  rows[n] = se;
  rows[g.nn + n] = sc;
}

// JVP terms through the element means.  Forward: per element
// s_e = (dkappa_eff/8) sum_m x_ce,m and t_e = (dD_eff/8) sum_m x_ce,m;
// transposed: tau_e = (dkappa_eff/8) sum_l x_phie,l (K u)_l + (dD_eff/8) sum_l x_ce,l (K c)_l.
__global__ void k_transport_jvp_elem(TrArgs a, const double* __restrict__ coef, const double* __restrict__ GH,
                                     const double* __restrict__ x, int trans, double* __restrict__ sc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  if (e >= ne) return;
  const int i = (int)(e % a.nx), j = (int)((e / a.nx) % a.ny), k = (int)(e / ((int64_t)a.nx * a.ny));
  const int64_t nn = a.g.nn;
  const double dk = coef[2 * ne + e] * 0.125, dd = coef[3 * ne + e] * 0.125;
  if (!trans) {
    double sum = 0.0;
#pragma unroll
    for (int l = 0; l < 8; ++l) sum += x[2 * nn + elem_node(a.g, i, j, k, l)];
    sc[e] = dk * sum;
    sc[ne + e] = dd * sum;
  } else {
    double tu = 0.0, tc = 0.0;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int64_t n = elem_node(a.g, i, j, k, l);
      tu += x[nn + n] * GH[l * ne + e];
      tc += x[2 * nn + n] * GH[(8 + l) * ne + e];
    }
    sc[e] = dk * tu + dd * tc;
  }
}

// Node pass: forward y_phie += sum_e s_e (K u)_l, y_ce += sum_e t_e (K c)_l;
// transposed y_ce += sum_e tau_e.  Output form of the operator: y = w (J x)
// or w (b - J x), w the row's output scale (1 unscaled).
__global__ void k_transport_jvp_node(TrArgs a, const double* __restrict__ GH, const double* __restrict__ sc,
                                     int trans, const double* __restrict__ b, const double* __restrict__ rsqd,
                                     const double* __restrict__ wf, double* __restrict__ y) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const Grid g = a.g;
  if (n >= g.nn) return;
  const int64_t ne = (int64_t)a.nx * a.ny * a.nz;
  const int64_t nn = g.nn;
  const int i = (int)(n % g.nnx);
  const int j = (int)((n / g.nnx) % g.nny);
  const int k = (int)(n / ((int64_t)g.nnx * g.nny));
  double ye = 0.0, yc = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < 2; ++p) {
        const int ei = i - 1 + p, ej = j - 1 + q, ek = k - 1 + s;
        if (ei < 0 || ej < 0 || ek < 0 || ei >= a.nx || ej >= a.ny || ek >= a.nz) continue;
        const int64_t e = ei + (int64_t)a.nx * (ej + (int64_t)a.ny * ek);
        if (!trans) {
          const int l = (1 - p) + 2 * (1 - q) + 4 * (1 - s);
          ye += sc[e] * GH[l * ne + e];
          yc += sc[ne + e] * GH[(8 + l) * ne + e];
        } else {
          yc += sc[e];
        }
      }
  const double sgn = b ? -1.0 : 1.0;
  if (!trans) y[nn + n] += sgn * (rsqd ? wf[1] * rsqd[nn + n] : 1.0) * ye;
  y[2 * nn + n] += sgn * (rsqd ? wf[2] * rsqd[2 * nn + n] : 1.0) * yc;
}

TrArgs make_tr(const p4d_ctx* c) {
  TrArgs a;
  a.g = c->g;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.brug = c->prm.brug; a.T = c->prm.T; a.Rg = c->prm.R;
  a.gamma = c->prm.diffpot_sign * 2.0 * c->prm.R * c->prm.T * (1.0 - c->prm.tplus) / c->prm.F;
  a.hx = c->hx; a.hy = c->hy; a.hz = c->hz;
  a.eps = c->eps_e;
  return a;
}

}  // namespace

p4d_status transport_alloc(p4d_ctx* c) {
  if (c->prm.transport_model != 1) return P4D_OK;
  const size_t ne = (size_t)c->nelem, nn = (size_t)c->g.nn;
  P4D_TRYS(dalloc_t(c, &c->tr_coefL, 4 * ne));
  P4D_TRYS(dalloc_t(c, &c->tr_GHL, 16 * ne));
  P4D_TRYS(dalloc_t(c, &c->tr_coefR, 4 * ne));
  P4D_TRYS(dalloc_t(c, &c->tr_GHR, 16 * ne));
  P4D_TRYS(dalloc_t(c, &c->tr_sc, 2 * ne));
  P4D_TRYS(dalloc_t(c, &c->tr_rows, 2 * nn));
  return P4D_OK;
}

p4d_status transport_linearize(p4d_ctx* c, const p4d_state* st) {
  if (c->prm.transport_model != 1) return P4D_OK;
  const TrArgs a = make_tr(c);
  ::p4d::count_launch(), k_transport_elem<<<nblocks(c->nelem, 128), 128, 0, c->stream>>>(a, st->phie, st->ce, c->lnce, c->tr_coefL, c->tr_GHL);
  ::p4d::count_launch(), k_assemble_transport<<<nblocks(c->g.nn, 128), 128, 0, c->stream>>>(a, c->tr_coefL, 1.0 / c->prm.dt, c->Jst);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

const double* transport_residual_rows(p4d_ctx* c, const p4d_state* st, const double* lnce) {
  if (c->prm.transport_model != 1) return nullptr;
  const TrArgs a = make_tr(c);
  ::p4d::count_launch(), k_transport_elem<<<nblocks(c->nelem, 128), 128, 0, c->stream>>>(a, st->phie, st->ce, lnce, c->tr_coefR, c->tr_GHR);
  ::p4d::count_launch(), k_transport_rows<<<nblocks(c->g.nn), kBlock, 0, c->stream>>>(a, c->tr_coefR, c->tr_GHR, c->tr_rows);
  return c->tr_rows;
}

p4d_status transport_jvp(p4d_ctx* c, const double* x, double* y, int transpose, const double* b, bool scaled) {
  if (c->prm.transport_model != 1) return P4D_OK;
  const TrArgs a = make_tr(c);
  ::p4d::count_launch(), k_transport_jvp_elem<<<nblocks(c->nelem, 128), 128, 0, c->stream>>>(a, c->tr_coefL, c->tr_GHL, x, transpose, c->tr_sc);
  ::p4d::count_launch(), k_transport_jvp_node<<<nblocks(c->g.nn), kBlock, 0, c->stream>>>(
      a, c->tr_GHL, c->tr_sc, transpose, b, scaled ? c->rsqd : nullptr, c->wf, y);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

}  // namespace p4d
