// Fixed stencil assembly, linearization (Butler-Volmer derivatives, particle
// Schur scalars, Jacobi scaling) and the nonlinear residual.
//
// Q1 on boxes: for an element of widths (hx, hy, hz) and local corners
// a, a' in {0,1} per axis, the 1D factors are
//   stiffness  s(a,a') / h  with s = +1 (a == a'), -1 (a != a')
//   mass       h m(a,a')    with m = 1/3 (a == a'), 1/6 (a != a')
// so the element stiffness entry is vol * (s_x/hx^2 m_y m_z + m_x s_y/hy^2 m_z
// + m_x m_y s_z/hz^2) and the mass entry vol * m_x m_y m_z (exact integrals of
// the trilinear basis).  Per node the contributions of its <= 8 elements are
// gathered into 27-point stencils (paper section 3, eqs. ce-weak, phie-weak,
// phis-weak); these depend only on the mesh and dt and are built once.
#include <cmath>
#include <vector>
#include "p4d_common.cuh"

namespace p4d {
namespace {

struct Phys {
  double brug, sigma_n, sigma_p, kappa, De, dt;
  double shell_p, shell_n;   // collector-foil surface conductances of the z = Lz / z = 0 faces (S)
};

__global__ void k_assemble(Grid g, int nx, int ny, int nz, const double* __restrict__ hx,
                           const double* __restrict__ hy, const double* __restrict__ hz,
                           const uint8_t* __restrict__ region, const double* __restrict__ eps,
                           const double* __restrict__ eps_s, const double* __restrict__ sig_e,
                           const uint8_t* __restrict__ label, Phys ph, double* __restrict__ Jst,
                           double* __restrict__ sfix) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int i = (int)(n % g.nnx);
  const int j = (int)((n / g.nnx) % g.nny);
  const int k = (int)(n / ((int64_t)g.nnx * g.nny));
  double Ks[27], Kk[27], Cc[27], Mm[27];
#pragma unroll
  for (int o = 0; o < 27; ++o) Ks[o] = Kk[o] = Cc[o] = Mm[o] = 0.0;
  const bool act = label[n] & kLabActive;
  double sdrop = 0.0, mlump = 0.0;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < 2; ++p) {
        const int ei = i - 1 + p, ej = j - 1 + q, ek = k - 1 + s;
        if (ei < 0 || ej < 0 || ek < 0 || ei >= nx || ej >= ny || ek >= nz) continue;
        const int64_t e = ei + (int64_t)nx * (ej + (int64_t)ny * ek);
        const double a = hx[ei], b = hy[ej], cz = hz[ek];
        const double vol = a * b * cz;
        const uint8_t r = region[e];
        const double sig = (r == 0 || r == 2) ? pow(eps_s[e], ph.brug) * sig_e[e] : 0.0;
        const double epb = pow(eps[e], ph.brug);
        const double kap = epb * ph.kappa;
        const double Dd = epb * ph.De;
        const double mcoef = eps[e] / ph.dt;
        const int an = 1 - p, bn = 1 - q, cn = 1 - s;
        for (int cc = 0; cc < 2; ++cc)
          for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
              const int dx = p - 1 + aa, dy = q - 1 + bb, dz = s - 1 + cc;
              const int o = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
              const double sx = aa == an ? 1.0 : -1.0, mx = aa == an ? 1.0 / 3.0 : 1.0 / 6.0;
              const double sy = bb == bn ? 1.0 : -1.0, my = bb == bn ? 1.0 / 3.0 : 1.0 / 6.0;
              const double sz = cc == cn ? 1.0 : -1.0, mz = cc == cn ? 1.0 / 3.0 : 1.0 / 6.0;
              const double kf = vol * (sx / (a * a) * my * mz + mx * sy / (b * b) * mz + mx * my * sz / (cz * cz));
              const double mf = vol * mx * my * mz;
              if (sig > 0.0 && act) {
                const int64_t nb = n + dx + (int64_t)g.nnx * (dy + (int64_t)g.nny * dz);
                if (label[nb] & kLabActive) Ks[o] += sig * kf;
                else sdrop -= sig * kf;
              }
              Kk[o] += kap * kf;
              Cc[o] += mcoef * mf + Dd * kf;
              Mm[o] += mcoef * mf;
              mlump += mcoef * mf;
            }
      }
  // collector foil of a boundary face as a thin shell: the 2D Q1 stiffness of
  // the face quads a x b around the node, sig_t [(b/a) k_x m_y + (a/b) m_x k_y]
  // (k = +1 same / -1 other node along the axis, m = 1/3 same / 1/6 other)
  const double sht = k == nz ? ph.shell_p : (k == 0 ? ph.shell_n : 0.0);
  if (sht > 0.0 && act) {
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < 2; ++p) {
        const int ei = i - 1 + p, ej = j - 1 + q;
        if (ei < 0 || ej < 0 || ei >= nx || ej >= ny) continue;
        const double a = hx[ei], b = hy[ej];
        const int an = 1 - p, bn = 1 - q;
        for (int bb = 0; bb < 2; ++bb)
          for (int aa = 0; aa < 2; ++aa) {
            const int dx = p - 1 + aa, dy = q - 1 + bb;
            const int o = (dx + 1) + 3 * (dy + 1) + 9;
            const double kx = aa == an ? 1.0 : -1.0, mx = aa == an ? 1.0 / 3.0 : 1.0 / 6.0;
            const double ky = bb == bn ? 1.0 : -1.0, my = bb == bn ? 1.0 / 3.0 : 1.0 / 6.0;
            const double v = sht * (b / a * kx * my + a / b * mx * ky);
            const int64_t nb = n + dx + (int64_t)g.nnx * dy;
            if (label[nb] & kLabActive) Ks[o] += v;
            else sdrop -= v;
          }
      }
  }
  const int64_t nn = g.nn;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    Jst[(0 * 27 + o) * nn + n] = Ks[o];
    Jst[(1 * 27 + o) * nn + n] = Kk[o];
    Jst[(2 * 27 + o) * nn + n] = Cc[o];
    Jst[(3 * 27 + o) * nn + n] = Mm[o];
  }
  sfix[0 * nn + n] = act ? sdrop : 1.0;
  sfix[1 * nn + n] = 0.0;
  sfix[2 * nn + n] = mlump;
}

// max |centre| over the nodes of one field (for the FP32 scaling)
__global__ void k_maxdiag(const double* __restrict__ st, int64_t nn, unsigned long long* out) {
  double m = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nn; n += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(st[13 * nn + n]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

struct Kin {
  double F, Rg, T, alpha, tau, i_app, gamma;
  double k[2], cmax[2], u0[2], u1[2];
  int ocp_model;   // 0 linear, 1 the paper's curves
};

// Open-circuit potential U(theta) and dU/dtheta of electrode et (0 graphite
// anode, 1 LiCoO2 cathode).  ocp_model 1: the paper's curves (Appendix
// "Model Parameters"), written as base + sum_i amp_i tanh(a_i + b_i t) with
// t = 1.062 theta for the cathode and t = theta (plus 1.5 exp(-120 theta))
// for the anode; dU/dtheta = dt/dtheta sum_i amp_i b_i (1 - tanh^2).
__device__ inline void ocp_eval(const Kin& kn, int et, double theta, double& U, double& dU) {
  if (kn.ocp_model == 0) {
    U = kn.u0[et] + kn.u1[et] * theta;
    dU = kn.u1[et];
    return;
  }
  if (et == 1) {
    constexpr double amp[6] = {0.07645, 2.1581, -0.14169, 0.2051, 0.2531, -0.02167};
    constexpr double a[6] = {30.834, 52.294, 11.0923, 1.4684, 0.56478 / 0.1316, -0.525 / 0.006};
    constexpr double b[6] = {-54.4806, -50.294, -19.8543, -5.4888, -1.0 / 0.1316, 1.0 / 0.006};
    const double t = 1.062 * theta;
    double u = 2.16216, du = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double th = tanh(a[q] + b[q] * t);
      u += amp[q] * th;
      du += amp[q] * b[q] * (1.0 - th * th);
    }
    U = u;
    dU = 1.062 * du;
  } else {
    constexpr double amp[8] = {0.0351, -0.0045, -0.035, -0.0147, -0.102, -0.022, -0.011, 0.0155};
    constexpr double c0[8] = {0.286, 0.849, 0.9233, 0.5, 0.194, 0.9, 0.124, 0.105};
    constexpr double w[8] = {0.083, 0.119, 0.05, 0.034, 0.142, 0.0164, 0.0226, 0.029};
    const double ex = exp(-120.0 * theta);
    double u = 0.194 + 1.5 * ex, du = -180.0 * ex;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double th = tanh((theta - c0[q]) / w[q]);
      u += amp[q] * th;
      du += amp[q] / w[q] * (1.0 - th * th);
    }
    U = u;
    dU = du;
  }
}

// Butler-Volmer (paper section 2, "Interfacial kinetics") at one electrode
// node; returns false outside the domain of the exchange current.
__device__ inline bool kinetics(const Kin& kn, int et, double phis, double phie, double ce, double cs,
                                double& in, double& ge, double& gc, double& gs) {
  const double cmax = kn.cmax[et];
  if (!(ce > 0.0) || !(cs > 0.0) || !(cs < cmax)) {
    in = ge = gc = gs = 0.0;
    return false;
  }
  const double f = kn.F / (kn.Rg * kn.T);
  const double al = kn.alpha;
  double U, dU;
  ocp_eval(kn, et, cs / cmax, U, dU);
  const double eta = phis - phie - U;
  double i0;
  if (al == 0.5) i0 = kn.k[et] * sqrt(ce) * sqrt(cmax - cs) * sqrt(cs);
  else i0 = kn.k[et] * pow(ce, al) * pow(cmax - cs, al) * pow(cs, 1.0 - al);
  const double ea = exp(al * f * eta);
  const double ec = exp(-(1.0 - al) * f * eta);
  in = i0 * (ea - ec);
  ge = i0 * f * (al * ea + (1.0 - al) * ec);
  gc = al * in / ce;
  gs = in * ((1.0 - al) / cs - al / (cmax - cs)) - ge * dU / cmax;
  return true;
}

__global__ void k_node_ln(int64_t nn, const double* __restrict__ ce, double gamma, double* __restrict__ lnce,
                          double* __restrict__ gdc, unsigned* flags) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const double c = ce[n];
  if (!(c > 0.0)) {
    atomicOr(flags, kFlagDomain);
    lnce[n] = 0.0;
    if (gdc) gdc[n] = 0.0;
    return;
  }
  lnce[n] = log(c);
  if (gdc) gdc[n] = gamma / c;
}

// LU of T_j / M_j = I/dt - kap_j Lref + e_N e_N^T beta_j g_s without its
// surface term (unit lower L with multipliers mult_i, upper U with pivots
// piv_i): every pivot but the last and all multipliers depend only on dt,
// kap_j and the radial grid, so they are factored once.  Stored as 1/piv and
// mult, radial-major ([nc][NE]: coalesced over nodes), so that every later
// FP64 particle solve is division free; qfix_j is the last pivot without the
// surface term.
__global__ void k_particle_lu_fixed(int64_t NE, int nc, double dt, const double* __restrict__ kapj,
                                    const double* __restrict__ rref, double* __restrict__ ipiv,
                                    double* __restrict__ mult, double* __restrict__ qfix, float* __restrict__ f32) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= NE) return;
  const double kap = kapj[j];
  const double* lo = rref;
  const double* di = rref + nc;
  const double* up = rref + 2 * nc;
  const double idt = 1.0 / dt;
  double piv = idt - kap * di[0];
  mult[j] = 0.0;
  for (int i = 1; i < nc; ++i) {
    ipiv[(i - 1) * NE + j] = 1.0 / piv;
    const double mi = (-kap * lo[i]) / piv;
    piv = (idt - kap * di[i]) - mi * (-kap * up[i - 1]);
    mult[i * NE + j] = mi;
  }
  qfix[j] = piv;
  if (f32)   // FP32 copies: [nc][NE] 1/pivot, then [nc][NE] multipliers
    for (int i = 0; i < nc; ++i) {
      f32[i * NE + j] = (float)ipiv[i * NE + j];
      f32[(nc + i) * NE + j] = (float)mult[i * NE + j];
    }
}

// Linearization per electrode node: kinetics derivatives, the last pivot of
// the particle tridiagonal T_j = M_j (I/dt - kap_j Lref) + e_N e_N^T M_j
// beta_j g_s (the fixed part plus the surface term), z_j = 1 / (M_j pivot) =
// (T_j^-1)_NN and zeta_j = 1 - z_j g_s M_j beta_j.
__global__ void k_linearize(int64_t NE, int nc, Kin kn, const int32_t* __restrict__ enode,
                            const uint8_t* __restrict__ label, const uint8_t* __restrict__ etype,
                            const double* __restrict__ phis, const double* __restrict__ phie,
                            const double* __restrict__ ce, const double* __restrict__ cs,
                            const double* __restrict__ Mj, const double* __restrict__ betaj,
                            const double* __restrict__ qfix, double* __restrict__ in_, double* __restrict__ ge,
                            double* __restrict__ gc, double* __restrict__ gs, double* __restrict__ zj,
                            double* __restrict__ zeta, double* __restrict__ ipiv, float* __restrict__ ipiv32,
                            unsigned* flags) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= NE) return;
  const int64_t n = enode[j];
  const bool act = label[n] & kLabActive;
  double a, b, c, d;
  if (!kinetics(kn, etype[j], act ? phis[n] : 0.0, phie[n], ce[n], cs[j * nc + nc - 1], a, b, c, d))
    atomicOr(flags, kFlagDomain);
  in_[j] = a; ge[j] = b; gc[j] = c; gs[j] = d;
  const double M = Mj[j];
  const double piv = qfix[j] + betaj[j] * d;
  ipiv[(nc - 1) * NE + j] = 1.0 / piv;
  if (ipiv32) ipiv32[(nc - 1) * NE + j] = (float)(1.0 / piv);
  const double z = 1.0 / (M * piv);
  zj[j] = z;
  zeta[j] = 1.0 - z * d * M * betaj[j];
}

// Jacobi scaling of the Krylov solve per row: sqrt(|J_ii|) and its inverse.
// The square roots are taken in FP32 (FP64 square roots cost ~1 ms per
// Newton step on this GPU); the scaling only defines the norm of the
// residual and the preconditioner's input weighting, both of which are free
// to be any positive diagonal, so a relative 1e-7 perturbation changes
// nothing but that definition.
__device__ __forceinline__ void put_scale(double d, double* sqd, double* rsqd, int64_t row) {
  float a = (float)fabs(d);
  if (!(a > 0.f) || !isfinite(a)) a = 1.f;
  const float r = sqrtf(a);
  sqd[row] = (double)r;
  rsqd[row] = (double)(1.0f / r);
}

__global__ void k_diag(Grid g, int64_t NE, int nc, double tau, double idt, const double* __restrict__ Jst,
                       const uint8_t* __restrict__ label, const int32_t* __restrict__ eidx,
                       const double* __restrict__ Aj, const double* __restrict__ Mj,
                       const double* __restrict__ kapj, const double* __restrict__ betaj,
                       const double* __restrict__ rref, const double* __restrict__ ge,
                       const double* __restrict__ gc, const double* __restrict__ gs, double* __restrict__ sqd,
                       double* __restrict__ rsqd) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  if (t < nn) {
    const int64_t n = t;
    const int32_t e = eidx[n];
    put_scale((label[n] & kLabActive) ? Jst[(0 * 27 + 13) * nn + n] + Aj[e] * ge[e] : 1.0, sqd, rsqd, n);
    put_scale(Jst[(1 * 27 + 13) * nn + n] + (e >= 0 ? Aj[e] * ge[e] : 0.0), sqd, rsqd, nn + n);
    put_scale(Jst[(2 * 27 + 13) * nn + n] - (e >= 0 ? tau * Aj[e] * gc[e] : 0.0), sqd, rsqd, 2 * nn + n);
  } else if (t < nn + NE * nc) {
    const int64_t q = t - nn;
    const int64_t e = (uint32_t)q / (uint32_t)nc;   // NE nc < 2^31 (checked at setup)
    const int i = (int)(q - e * nc);
    double d = Mj[e] * (idt - kapj[e] * rref[nc + i]);
    if (i == nc - 1) d += Mj[e] * betaj[e] * gs[e];
    put_scale(d, sqd, rsqd, 3 * nn + q);
  }
}

// ||(sqrt(d) u)_f||^2 per field of the linearization state (the rounding
// scale of each field's residual terms, used to floor the Krylov weights).
__global__ void k_state_scale(int64_t nn, int64_t ncs, const double* __restrict__ sqd, const double* __restrict__ phis,
                              const double* __restrict__ phie, const double* __restrict__ ce,
                              const double* __restrict__ cs, double* __restrict__ partial) {
  double acc[4];
  acc[0] = sumsq_share<true>(phis, sqd, nn);
  acc[1] = sumsq_share<true>(phie, sqd + nn, nn);
  acc[2] = sumsq_share<true>(ce, sqd + 2 * nn, nn);
  acc[3] = sumsq_share<true>(cs, sqd + 3 * nn, ncs);
  block_sum4(acc, partial);
}

__global__ void k_state_sum(const double* __restrict__ partial, int nblk, double* out4) { sum4_warps(partial, nblk, out4); }

// Fixed off-diagonal sums of the level-0 multigrid operators (setup).
__global__ void k_fixed_sums(Grid g, const double* __restrict__ Jst, const uint8_t* __restrict__ label,
                             double* __restrict__ offsum, double* __restrict__ absoff) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  if (n >= nn) return;
  for (int f = 0; f < 3; ++f) {
    const double* st = Jst + (size_t)f * 27 * nn;
    double s = 0.0, a = 0.0;
    if (!(f == 0 && !(label[n] & kLabActive)))
      for (int o = 0; o < 27; ++o)
        if (o != 13) { s += st[o * nn + n]; a += fabs(st[o * nn + n]); }
    offsum[f * nn + n] = s;
    absoff[f * nn + n] = a;
  }
}

template <typename F>
__device__ inline double stencil_apply(const double* __restrict__ st, int64_t nn, const Grid& g, int64_t n,
                                       int i, int j, int k, F val) {
  double acc = 0.0;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nnx || jj >= g.nny || kk >= g.nnz) continue;
    const int64_t m = n + dx + (int64_t)g.nnx * (dy + (int64_t)g.nny * dz);
    acc += st[o * nn + n] * val(m);
  }
  return acc;
}

// Nonlinear residual (paper section 4, block residual) -- macro rows.
__global__ void k_residual_macro(Grid g, Kin kn, const double* __restrict__ Jst,
                                 const uint8_t* __restrict__ label, const int32_t* __restrict__ eidx,
                                 const double* __restrict__ Aj, const double* __restrict__ gpw,
                                 const double* __restrict__ phis, const double* __restrict__ phie,
                                 const double* __restrict__ ce, const double* __restrict__ ce_prev,
                                 const double* __restrict__ lnce, const double* __restrict__ rin,
                                 const double* __restrict__ sfix, const double* __restrict__ trows,
                                 double* __restrict__ r) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  if (n >= nn) return;
  const int i = (int)(n % g.nnx);
  const int j = (int)((n / g.nnx) % g.nny);
  const int k = (int)(n / ((int64_t)g.nnx * g.nny));
  const int32_t e = eidx[n];
  const double ain = e >= 0 ? Aj[e] * rin[e] : 0.0;
  const bool act = label[n] & kLabActive;
  // phi_s: lifted stencil (entries to inactive nodes are zero) in difference
  // form, sum_{m != n} K_nm (phi_m - phi_n) + s_n phi_n with s_n the row sum
  // of the lifted stencil (exactly 0 where no coupling was dropped): the
  // collector-shell rows couple nodes whose potentials agree to microvolts
  // through conductances ~1e7 times the bulk ones, and the standard form
  // would leave rounding of those large products in the residual
  if (act) {
    const double* Ks = Jst;
    const double pn = phis[n];
    double s = sfix[n] * pn;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      if (o == 13) continue;
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int ii = i + dx, jj = j + dy, kk = k + dz;
      if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nnx || jj >= g.nny || kk >= g.nnz) continue;
      const int64_t m = n + dx + (int64_t)g.nnx * (dy + (int64_t)g.nny * dz);
      if (label[m] & kLabActive) s += Ks[o * nn + n] * (phis[m] - pn);
    }
    r[n] = s + ain - kn.i_app * gpw[n];
  } else {
    r[n] = phis[n];
  }
  // transport rows: the fixed stencils, or (concentration-dependent
  // coefficients) the element integrals at this state, trows[0..1][n]
  const double se = trows ? trows[n]
                          : stencil_apply(Jst + 1 * 27 * nn, nn, g, n, i, j, k,
                                          [&](int64_t m) { return phie[m] + kn.gamma * lnce[m]; });
  r[nn + n] = se - ain;
  // mass part on (c_e - c_e_prev), diffusion part (C - M_eps/dt) on c_e: no cancellation between
  // the two time levels
  double sc = 0.0;
  {
    const double* Cc = Jst + 2 * 27 * nn;
    const double* Mm = Jst + 3 * 27 * nn;
#pragma unroll
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int ii = i + dx, jj = j + dy, kk = k + dz;
      if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nnx || jj >= g.nny || kk >= g.nnz) continue;
      const int64_t m = n + dx + (int64_t)g.nnx * (dy + (int64_t)g.nny * dz);
      const double mo = Mm[o * nn + n];
      sc += mo * (ce[m] - ce_prev[m]) + (trows ? 0.0 : (Cc[o * nn + n] - mo) * ce[m]);
    }
  }
  if (trows) sc += trows[nn + n];
  r[2 * nn + n] = sc - kn.tau * ain;
}

__global__ void k_kinetics_only(int64_t NE, int nc, Kin kn, const int32_t* __restrict__ enode,
                                const uint8_t* __restrict__ label, const uint8_t* __restrict__ etype,
                                const double* __restrict__ phis, const double* __restrict__ phie,
                                const double* __restrict__ ce, const double* __restrict__ cs,
                                double* __restrict__ rin, unsigned* flags) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= NE) return;
  const int64_t n = enode[j];
  const bool act = label[n] & kLabActive;
  double a, b, c, d;
  if (!kinetics(kn, etype[j], act ? phis[n] : 0.0, phie[n], ce[n], cs[j * nc + nc - 1], a, b, c, d))
    atomicOr(flags, kFlagDomain);
  rin[j] = a;
}

// Particle rows: R_cs = M [(c - c_prev)/dt - kap Lref c] + e_N M beta i_n.
__global__ void k_residual_particle(int64_t NE, int nc, double idt, const double* __restrict__ cs,
                                    const double* __restrict__ cs_prev, const double* __restrict__ Mj,
                                    const double* __restrict__ kapj, const double* __restrict__ betaj,
                                    const double* __restrict__ rref, const double* __restrict__ rin,
                                    double* __restrict__ r) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= NE * nc) return;
  const int64_t e = (uint32_t)q / (uint32_t)nc;   // NE nc < 2^31 (checked at setup)
  const int i = (int)(q - e * nc);
  const double* c = cs + e * nc;
  double L = rref[nc + i] * c[i];
  if (i > 0) L += rref[i] * c[i - 1];
  if (i < nc - 1) L += rref[2 * nc + i] * c[i + 1];
  double v = Mj[e] * ((c[i] - cs_prev[q]) * idt - kapj[e] * L);
  if (i == nc - 1) v += Mj[e] * betaj[e] * rin[e];
  r[q] = v;
}

Kin make_kin(const p4d_params& p) {
  Kin k;
  k.F = p.F; k.Rg = p.R; k.T = p.T; k.alpha = p.alpha; k.tau = (1.0 - p.tplus) / p.F;
  k.i_app = p.i_app;
  k.gamma = p.diffpot_sign * 2.0 * p.R * p.T * (1.0 - p.tplus) / p.F;
  k.k[0] = p.k_n; k.k[1] = p.k_p;
  k.cmax[0] = p.cmax_n; k.cmax[1] = p.cmax_p;
  k.u0[0] = p.ocp_n[0]; k.u0[1] = p.ocp_p[0];
  k.u1[0] = p.ocp_n[1]; k.u1[1] = p.ocp_p[1];
  k.ocp_model = p.ocp_model;
  return k;
}

}  // namespace

p4d_status assemble_fixed(p4d_ctx* c, const double* eps, const double* eps_s, const uint8_t* region) {
  const int64_t nn = c->g.nn;
  P4D_TRYS(dalloc_t(c, &c->Jst, (size_t)4 * 27 * nn));
  P4D_TRYS(dalloc_t(c, &c->sfix, (size_t)3 * nn));
  Phys ph{c->prm.brug, c->prm.sigma_n, c->prm.sigma_p, c->kappa_fix, c->De_fix, c->prm.dt, c->shell_p, c->shell_n};
  ::p4d::count_launch(), k_assemble<<<nblocks(nn, 128), 128, 0, c->stream>>>(c->g, c->nx, c->ny, c->nz, c->hx, c->hy, c->hz, region,
                                                       eps, eps_s, c->sig_e, c->label, ph, c->Jst, c->sfix);
  P4D_TRY(cudaGetLastError());
  P4D_TRYS(dalloc_t(c, &c->offsum, (size_t)3 * nn));
  P4D_TRYS(dalloc_t(c, &c->absoff, (size_t)3 * nn));
  ::p4d::count_launch(), k_fixed_sums<<<nblocks(nn), kBlock, 0, c->stream>>>(c->g, c->Jst, c->label, c->offsum, c->absoff);
  P4D_TRYS(dalloc_t(c, &c->tqfix, (size_t)std::max<int64_t>(1, c->NE)));
  if (c->NE > 0)
    ::p4d::count_launch(), k_particle_lu_fixed<<<nblocks(c->NE), kBlock, 0, c->stream>>>(
        c->NE, c->nc, c->prm.dt, c->kapj, c->rref, c->tfac, c->tfac + (size_t)c->NE * c->nc, c->tqfix, c->tfac32);
  unsigned long long* mx = nullptr;
  P4D_TRYS(dalloc_t(c, &mx, 3));
  P4D_TRY(cudaMemsetAsync(mx, 0, 3 * sizeof(unsigned long long), c->stream));
  for (int f = 0; f < 3; ++f)
    ::p4d::count_launch(), k_maxdiag<<<4 * 152, kBlock, 0, c->stream>>>(c->Jst + (size_t)f * 27 * nn, nn, mx + f);
  unsigned long long h[3];
  P4D_TRY(cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  P4D_TRY(cudaStreamSynchronize(c->stream));
  for (int f = 0; f < 3; ++f) {
    double v;
    memcpy(&v, &h[f], sizeof(double));
    // power of two so that scaling is exact
    c->scale_f[f] = v > 0 ? std::ldexp(1.0, -std::ilogb(v)) : 1.0;
  }
  return P4D_OK;
}

p4d_status linearize(p4d_ctx* c, const p4d_state* st) {
  const int64_t nn = c->g.nn, NE = c->NE;
  const int nc = c->nc;
  Kin kn = make_kin(c->prm);
  P4D_TRY(cudaMemsetAsync(c->flags, 0, sizeof(unsigned), c->stream));
  ::p4d::count_launch(), k_node_ln<<<nblocks(nn), kBlock, 0, c->stream>>>(nn, st->ce, kn.gamma, c->lnce, c->gdc, c->flags);
  P4D_TRYS(transport_linearize(c, st));   // K_kappa, C at the state (transport_model 1)
  if (NE > 0)
    ::p4d::count_launch(), k_linearize<<<nblocks(NE), kBlock, 0, c->stream>>>(NE, nc, kn, c->enode, c->label, c->etype,
                                                        st->phis, st->phie, st->ce, st->cs, c->Mj, c->betaj,
                                                        c->tqfix, c->in_, c->ge, c->gc, c->gs, c->zj, c->zeta,
                                                        c->tfac, c->tfac32, c->flags);
  ::p4d::count_launch(), k_diag<<<nblocks(nn + NE * nc), kBlock, 0, c->stream>>>(c->g, NE, nc, kn.tau, 1.0 / c->prm.dt, c->Jst, c->label,
                                                          c->eidx, c->Aj, c->Mj, c->kapj, c->betaj, c->rref,
                                                          c->ge, c->gc, c->gs, c->sqd, c->rsqd);
  ::p4d::count_launch(), k_state_scale<<<4 * 152, kBlock, 0, c->stream>>>(nn, NE * nc, c->sqd, st->phis, st->phie, st->ce,
                                                                         st->cs, c->part);
  ::p4d::count_launch(), k_state_sum<<<1, 128, 0, c->stream>>>(c->part, 4 * 152, c->unorm2);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status residual(p4d_ctx* c, const p4d_state* st, double* r) {
  const int64_t nn = c->g.nn, NE = c->NE;
  const int nc = c->nc;
  Kin kn = make_kin(c->prm);
  P4D_TRY(cudaMemsetAsync(c->flags, 0, sizeof(unsigned), c->stream));
  ::p4d::count_launch(), k_node_ln<<<nblocks(nn), kBlock, 0, c->stream>>>(nn, st->ce, kn.gamma, c->lnce_r, nullptr, c->flags);
  if (NE > 0)
    ::p4d::count_launch(), k_kinetics_only<<<nblocks(NE), kBlock, 0, c->stream>>>(NE, nc, kn, c->enode, c->label, c->etype, st->phis,
                                                            st->phie, st->ce, st->cs, c->rin, c->flags);
  const double* trows = transport_residual_rows(c, st, c->lnce_r);
  ::p4d::count_launch(), k_residual_macro<<<nblocks(nn, 128), 128, 0, c->stream>>>(c->g, kn, c->Jst, c->label, c->eidx, c->Aj, c->gpw,
                                                             st->phis, st->phie, st->ce, st->ce_prev,
                                                             c->lnce_r, c->rin, c->sfix, trows, r);
  if (NE > 0)
    ::p4d::count_launch(), k_residual_particle<<<nblocks(NE * nc), kBlock, 0, c->stream>>>(NE, nc, 1.0 / c->prm.dt, st->cs, st->cs_prev, c->Mj,
                                                                    c->kapj, c->betaj, c->rref, c->rin,
                                                                    r + 3 * nn);
  P4D_TRY(cudaGetLastError());
  return check_flags(c);
}

}  // namespace p4d
