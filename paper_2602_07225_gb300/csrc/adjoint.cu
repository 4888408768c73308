// Newton time step, terminal-voltage functional and the adjoint sensitivity
// pieces (per-element parameter gradients and the coupling to the previous
// time level) of the backward-Euler P4D DFN discretization (paper sections
// 3-4; the adjoint is the pyadjoint use the paper's implementation section
// motivates).
//
// Gradient formulas (R_n: residual of step n, lam_n its adjoint):
//   dV/dp = -sum_n lam_n^T dR_n/dp,
//   sigma_e (eps_s^b sigma_e multiplies the element stiffness of phi_s):
//     -eps_s^b  lam~_s^T K_e phi~_s            (lifted rows/values)
//   eps_e (kappa_eff = eps^b kappa, D_eff = eps^b D_e, mass eps M_e/dt):
//     -b eps^(b-1) kappa lam_e^T K_e (phi_e + gamma ln c_e)
//     -lam_c^T (M_e (c_e - c_e_prev)/dt + b eps^(b-1) D_e K_e c_e)
//   D_s,e (node value = volume-weighted mean over electrode elements):
//     +(vol_e/8) sum_{nodes j of e} lam_cs,j^T Lref c_s,j / R_j^2
#include <algorithm>
#include <cmath>
#include "p4d_common.cuh"

namespace p4d {
namespace {

// field norms^2 of a vector, optionally weighted row-wise (phi_s, phi_e,
// c_e, c_s): per-block partials, one contiguous range per field
__global__ void k_fnorm(const double* __restrict__ r, const double* __restrict__ wgt, int64_t nn, int64_t len,
                        double* __restrict__ partial) {
  double acc[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t lo = f * nn, hi = f < 3 ? (f + 1) * nn : len;
    acc[f] = hi <= lo ? 0.0 : (wgt ? sumsq_share<true>(r + lo, wgt + lo, hi - lo) : sumsq_share<false>(r + lo, nullptr, hi - lo));
  }
  block_sum4(acc, partial);
}

__global__ void k_fnorm_sum(const double* __restrict__ partial, int nblk, double* out) { sum4_warps(partial, nblk, out); }

// trial = u - lam * dlt, in the full layout, from the four state arrays
__global__ void k_newton_trial(int64_t nn, int64_t ncs, const double* __restrict__ phis,
                               const double* __restrict__ phie, const double* __restrict__ ce,
                               const double* __restrict__ cs, const double* __restrict__ dlt, double lam,
                               double* __restrict__ trial) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= 3 * nn + ncs) return;
  double u;
  if (q < nn) u = phis[q];
  else if (q < 2 * nn) u = phie[q - nn];
  else if (q < 3 * nn) u = ce[q - 2 * nn];
  else u = cs[q - 3 * nn];
  trial[q] = fma(-lam, dlt[q], u);
}

__global__ void k_voltage_weights(int64_t nn, int64_t ndof, const double* __restrict__ gpw, double inv_area,
                                  double* __restrict__ q) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ndof) return;
  q[i] = i < nn ? gpw[i] * inv_area : 0.0;
}

// V = sum_n gpw_n phi_s,n / |Gamma_p| in one block (fixed order: strided
// partial sums, then a tree over the threads).
__global__ void __launch_bounds__(256) k_terminal_voltage(int64_t nn, const double* __restrict__ gpw,
                                                          const double* __restrict__ phis, double inv_area,
                                                          double* __restrict__ v) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t n = threadIdx.x; n < nn; n += 256) acc = fma(gpw[n], phis[n], acc);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *v = red[0] * inv_area;
}

// P_j = lam_cs,j^T Lref c_s,j / R_j^2 per electrode node
__global__ void k_grad_particle(int64_t NE, int nc, int64_t nn, const double* __restrict__ lam,
                                const double* __restrict__ cs, const double* __restrict__ rref,
                                const double* __restrict__ Rj, double* __restrict__ P) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= NE) return;
  const double* l = lam + 3 * nn + e * nc;
  const double* c = cs + e * nc;
  double acc = 0.0;
  for (int i = 0; i < nc; ++i) {
    double Lc = rref[nc + i] * c[i];
    if (i > 0) Lc += rref[i] * c[i - 1];
    if (i < nc - 1) Lc += rref[2 * nc + i] * c[i + 1];
    acc = fma(l[i], Lc, acc);
  }
  P[e] = acc / (Rj[e] * Rj[e]);
}

struct GradArgs {
  Grid g;
  int nx, ny, nz;
  double brug, kappa, De, idt, gamma;
  int transport;         // 1: bulk kappa, D_e of the paper at the element mean of c_e
  double T, Rg;
  const double *hx, *hy, *hz;
  const uint8_t* region;
  const double *eps, *eps_s;
  const uint8_t* label;
  const int32_t* eidx;
};

// Element contributions to the sigma / eps / D_s gradients.
__global__ void k_grad_elem(GradArgs a, const double* __restrict__ lam, const double* __restrict__ phis,
                            const double* __restrict__ phie, const double* __restrict__ ce,
                            const double* __restrict__ ce_prev, const double* __restrict__ P,
                            double* __restrict__ g_sig, double* __restrict__ g_Ds, double* __restrict__ g_eps) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nelem = (int64_t)a.nx * a.ny * a.nz;
  if (e >= nelem) return;
  const int i = (int)(e % a.nx), j = (int)((e / a.nx) % a.ny), k = (int)(e / ((int64_t)a.nx * a.ny));
  const int64_t nn = a.g.nn;
  const double hx = a.hx[i], hy = a.hy[j], hz = a.hz[k];
  const double vol = hx * hy * hz;
  int64_t nd[8];
  double ls[8], us[8], le[8], ue[8], lc[8], uc[8], dc[8];
  for (int l = 0; l < 8; ++l) {
    const int64_t n = (i + (l & 1)) + (int64_t)a.g.nnx * ((j + ((l >> 1) & 1)) + (int64_t)a.g.nny * (k + ((l >> 2) & 1)));
    nd[l] = n;
    const bool act = a.label[n] & kLabActive;
    ls[l] = act ? lam[n] : 0.0;
    us[l] = act ? phis[n] : 0.0;
    le[l] = lam[nn + n];
    ue[l] = phie[n] + a.gamma * log(ce[n]);
    lc[l] = lam[2 * nn + n];
    uc[l] = ce[n];
    dc[l] = ce[n] - ce_prev[n];
  }
  double Ks = 0.0, Ke = 0.0, Kc = 0.0, Mc = 0.0;
  for (int l = 0; l < 8; ++l) {
    const int al = l & 1, bl = (l >> 1) & 1, cl = (l >> 2) & 1;
    for (int m = 0; m < 8; ++m) {
      const int am = m & 1, bm = (m >> 1) & 1, cm = (m >> 2) & 1;
      const double sx = al == am ? 1.0 : -1.0, mx = al == am ? 1.0 / 3.0 : 1.0 / 6.0;
      const double sy = bl == bm ? 1.0 : -1.0, my = bl == bm ? 1.0 / 3.0 : 1.0 / 6.0;
      const double sz = cl == cm ? 1.0 : -1.0, mz = cl == cm ? 1.0 / 3.0 : 1.0 / 6.0;
      const double kf = vol * (sx / (hx * hx) * my * mz + mx * sy / (hy * hy) * mz + mx * my * sz / (hz * hz));
      const double mf = vol * mx * my * mz;
      Ks += ls[l] * kf * us[m];
      Ke += le[l] * kf * ue[m];
      Kc += lc[l] * kf * uc[m];
      Mc += lc[l] * mf * dc[m];
    }
  }
  const uint8_t r = a.region[e];
  const bool el = r == 0 || r == 2;
  const double ep = a.eps[e];
  const double dpb = a.brug * pow(ep, a.brug - 1.0);
  double kb = a.kappa, Db = a.De;
  if (a.transport) {
    double cbar = 0.0, dk, dd;
    for (int l = 0; l < 8; ++l) cbar += uc[l];
    transport_bulk(0.125 * cbar, a.T, a.Rg, kb, dk, Db, dd);
  }
  if (g_sig && el) g_sig[e] += -pow(a.eps_s[e], a.brug) * Ks;
  if (g_eps) g_eps[e] += -(dpb * kb * Ke + Mc * a.idt + dpb * Db * Kc);
  if (g_Ds && el) {
    double s = 0.0;
    for (int l = 0; l < 8; ++l) s += P[a.eidx[nd[l]]];
    g_Ds[e] += vol / 8.0 * s;
  }
}

// out = [0; 0; (M_eps/dt) lam_ce; (M_j/dt) lam_cs]
__global__ void k_adjoint_prev(Grid g, int64_t NE, int nc, double idt, const double* __restrict__ Mst,
                               const double* __restrict__ Mj, const double* __restrict__ lam, double* __restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  if (q < nn) {
    const int64_t n = q;
    const int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((int64_t)g.nnx * g.nny));
    double acc = 0.0;
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int ii = i + dx, jj = j + dy, kk = k + dz;
      if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nnx || jj >= g.nny || kk >= g.nnz) continue;
      const int64_t m = n + dx + (int64_t)g.nnx * (dy + (int64_t)g.nny * dz);
      acc = fma(Mst[o * nn + n], lam[2 * nn + m], acc);
    }
    out[n] = 0.0;
    out[nn + n] = 0.0;
    out[2 * nn + n] = acc;
  } else if (q < nn + NE * nc) {
    const int64_t p = q - nn;
    out[3 * nn + p] = Mj[(uint32_t)p / (uint32_t)nc] * idt * lam[3 * nn + p];
  }
}

}  // namespace
}  // namespace p4d

using namespace p4d;

extern "C" {

p4d_status p4d_newton_solve(p4d_handle h, double* phis, double* phie, double* ce, double* cs,
                            const double* ce_prev, const double* cs_prev, double rtol, int32_t maxit,
                            int32_t* iters_out, p4d_info* info) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !phis || !phie || !ce || !cs || !ce_prev || !cs_prev || maxit < 1 || !(rtol > 0))
    return P4D_ERR_INVALID_ARG;
  const int64_t nn = h->g.nn, ndof = h->ndof, ncs = h->NE * h->nc;
  double* R = h->nwork;
  double* dlt = h->nwork + ndof;
  double* trial = h->nwork + 2 * ndof;
  double* Rt = h->nwork + 3 * ndof;
  double* wsc = h->nwork + 4 * ndof;   // Jacobi row scaling frozen at the first linearization
  double* fn = h->hs_h;
  double* fn_d = h->nrm4;
  // ||.||^2 per field, optionally with the frozen row scaling
  auto fnorms = [&](const double* r, const double* w, double* out) -> p4d_status {
    ::p4d::count_launch(), k_fnorm<<<4 * 152, kBlock, 0, h->stream>>>(r, w, nn, ndof, h->part);
    ::p4d::count_launch(), k_fnorm_sum<<<1, 128, 0, h->stream>>>(h->part, 4 * 152, fn_d);
    P4D_TRY(cudaMemcpyAsync(fn, fn_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    P4D_TRY(cudaStreamSynchronize(h->stream));
    for (int f = 0; f < 4; ++f) out[f] = fn[f];
    return P4D_OK;
  };
  auto total = [](const double* f) { return std::sqrt(f[0] + f[1] + f[2] + f[3]); };
  p4d_state st{phis, phie, ce, cs, ce_prev, cs_prev};
  P4D_TRYS(residual(h, &st, R));
  P4D_TRYS(p4d_jacobian_update(h, &st));
  P4D_TRY(cudaMemcpyAsync(wsc, h->rsqd, ndof * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  double f0[4], fc[4];
  P4D_TRYS(fnorms(R, wsc, f0));
  const double r0 = total(f0);
  double rel = r0 > 0 ? 1.0 : 0.0;
  int it = 0;
  int nsolves = 0, iters_total = 0;
  p4d_status result = P4D_ERR_NOT_CONVERGED;
  bool linearized_here = true;
  for (; it <= maxit; ++it) {
    if (rel <= rtol) { result = P4D_OK; break; }
    if (it == maxit) break;
    if (!linearized_here) P4D_TRYS(p4d_jacobian_update(h, &st));
    linearized_here = false;
    P4D_TRY(cudaMemsetAsync(dlt, 0, ndof * sizeof(double), h->stream));
    p4d_info li;
    const p4d_status ls = fgmres(h, R, dlt, &li, 0);   // J dlt = R, step = -dlt
    ++nsolves;
    iters_total += li.iters;
    li.nsolves = nsolves;
    li.iters_total = iters_total;
    if (info) *info = li;
    if (ls != P4D_OK && ls != P4D_ERR_NOT_CONVERGED) return ls;
    // step-length test: the residual has a rounding floor (the phi_s rows,
    // for example, sum 27 terms ~1e5 times larger than the applied-current
    // term), so a converged iterate is also recognised by a tiny step
    double fd[4], fu[4];
    P4D_TRYS(fnorms(dlt, nullptr, fd));
    ::p4d::count_launch(), k_newton_trial<<<nblocks(ndof), kBlock, 0, h->stream>>>(nn, ncs, phis, phie, ce, cs, dlt, 0.0, trial);
    P4D_TRYS(fnorms(trial, nullptr, fu));
    double step_rel = 0.0;
    for (int q = 0; q < 4; ++q)
      if (fu[q] > 0) step_rel = std::max(step_rel, std::sqrt(fd[q] / fu[q]));
    // full Newton steps (the basic line search of the paper's default
    // nonlinear solver settings), halved only while the trial state leaves
    // the kinetics' domain or gives a non-finite residual
    double lam = 1.0;
    bool accepted = false;
    for (int bt = 0; bt < 9; ++bt, lam *= 0.5) {
      ::p4d::count_launch(), k_newton_trial<<<nblocks(ndof), kBlock, 0, h->stream>>>(nn, ncs, phis, phie, ce, cs, dlt, lam, trial);
      p4d_state ts{trial, trial + nn, trial + 2 * nn, trial + 3 * nn, ce_prev, cs_prev};
      const p4d_status rs = residual(h, &ts, Rt);
      if (rs == P4D_ERR_DOMAIN) continue;
      if (rs != P4D_OK) return rs;
      P4D_TRYS(fnorms(Rt, wsc, fc));
      const double rt = total(fc) / r0;
      if (!std::isfinite(rt)) continue;
      {
        P4D_TRY(cudaMemcpyAsync(phis, trial, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        P4D_TRY(cudaMemcpyAsync(phie, trial + nn, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        P4D_TRY(cudaMemcpyAsync(ce, trial + 2 * nn, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        P4D_TRY(cudaMemcpyAsync(cs, trial + 3 * nn, ncs * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        P4D_TRY(cudaMemcpyAsync(R, Rt, ndof * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        rel = rt;
        accepted = true;
        break;
      }
    }
    if (!accepted) { result = P4D_ERR_DOMAIN; break; }
    if (step_rel <= rtol && lam == 1.0) { ++it; result = P4D_OK; break; }
  }
  P4D_TRY(cudaStreamSynchronize(h->stream));
  if (iters_out) *iters_out = it;
  return result;
}

p4d_status p4d_voltage_weights(p4d_handle h, double* q) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !q || !(h->gp_area > 0)) return P4D_ERR_INVALID_ARG;
  ::p4d::count_launch(), k_voltage_weights<<<nblocks(h->ndof), kBlock, 0, h->stream>>>(h->g.nn, h->ndof, h->gpw, 1.0 / h->gp_area, q);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status p4d_terminal_voltage(p4d_handle h, const double* phis, double* v) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !phis || !v || !(h->gp_area > 0)) return P4D_ERR_INVALID_ARG;
  ::p4d::count_launch(), k_terminal_voltage<<<1, 256, 0, h->stream>>>(h->g.nn, h->gpw, phis, 1.0 / h->gp_area, v);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status p4d_param_grad(p4d_handle h, const p4d_state* st, const double* lam, double* g_sigma, double* g_Ds,
                          double* g_eps) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !st || !lam || !st->phis || !st->phie || !st->ce || !st->cs || !st->ce_prev) return P4D_ERR_INVALID_ARG;
  double* P = h->tloc;   // per electrode node particle term
  if (h->NE > 0)
    ::p4d::count_launch(), k_grad_particle<<<nblocks(h->NE), kBlock, 0, h->stream>>>(h->NE, h->nc, h->g.nn, lam, st->cs, h->rref, h->Rj, P);
  GradArgs a;
  a.g = h->g; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
  a.brug = h->prm.brug; a.kappa = h->prm.kappa; a.De = h->prm.De; a.idt = 1.0 / h->prm.dt;
  a.gamma = h->prm.diffpot_sign * 2.0 * h->prm.R * h->prm.T * (1.0 - h->prm.tplus) / h->prm.F;
  a.hx = h->hx; a.hy = h->hy; a.hz = h->hz; a.region = h->region; a.eps = h->eps_e; a.eps_s = h->epss_e;
  a.label = h->label; a.eidx = h->eidx;
  a.transport = h->prm.transport_model; a.T = h->prm.T; a.Rg = h->prm.R;
  ::p4d::count_launch(), k_grad_elem<<<nblocks(h->nelem, 128), 128, 0, h->stream>>>(a, lam, st->phis, st->phie, st->ce, st->ce_prev, P,
                                                                g_sigma, g_Ds, g_eps);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status p4d_adjoint_prev(p4d_handle h, const double* lam, double* out) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !lam || !out || lam == out) return P4D_ERR_INVALID_ARG;
  ::p4d::count_launch(), k_adjoint_prev<<<nblocks(h->g.nn + h->NE * h->nc), kBlock, 0, h->stream>>>(
      h->g, h->NE, h->nc, 1.0 / h->prm.dt, h->Jst + (size_t)3 * 27 * h->g.nn, h->Mj, lam, out);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

}  // extern "C"
