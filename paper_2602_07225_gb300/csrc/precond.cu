// Block preconditioner (paper section 4, eqs. PJ / PGS) with the particle
// blocks eliminated exactly.
//
// FULL layout, non-transposed, for r = [r_m; r_c]:
//   y_c = T^-1 r_c                         (one tridiagonal per electrode node)
//   r_m' = r_m - A_mc y_c                  (A_mc: column c_N, = u_m g_s)
//   z_m = P_macro^-1 r_m'                  (BJ / BGS over multigrid V-cycles)
//   z_c = y_c - T^-1 A_cm z_m              (A_cm: row c_N, = M beta v_m)
// The transposed preconditioner swaps A_mc <-> A_cm^T, uses T^T, keeps the
// (symmetric) V-cycles and runs BGS upper-triangular in reverse order.
// Particle solves run in the preconditioner precision T on the tridiagonal
// T/M = I/dt - kap Lref + e_N e_N^T beta g_s (entries of order one).
// In the scaled Krylov space the input is multiplied by s^-1 = sqrt(d)/w_f.
#include "p4d_common.cuh"

namespace p4d {
namespace {

struct PcArgs {
  Grid g;
  int64_t NE;
  int nc;
  double tau, dt, idt;
  const uint8_t* label;
  const int32_t* eidx;
  const int32_t* enode;
  const double *Aj, *Mj, *betaj, *kapj, *rref;
  const double *ge, *gc, *gs, *zeta, *sqd, *iwf;
  double sc[3];
};

__device__ __forceinline__ double insc(const PcArgs& a, bool scaled, int f, int64_t row) {
  return scaled ? a.sqd[row] * a.iwf[f] : 1.0;
}

// Thomas on T/M (or its transpose) for one particle; rhs in-place in x[0..nc).
template <typename T, bool TRANS>
__device__ __forceinline__ void particle_thomas(const PcArgs& a, int64_t e, T* x) {
  const int nc = a.nc;
  const T kap = (T)a.kapj[e];
  const T idt = (T)a.idt;
  const double* lo = a.rref;
  const double* di = a.rref + nc;
  const double* up = a.rref + 2 * nc;
  T cp[kMaxNc];
  T dg = idt - kap * (T)di[0];
  T u0 = TRANS ? -kap * (T)lo[1] : -kap * (T)up[0];
  cp[0] = u0 / dg;
  x[0] = x[0] / dg;
  for (int i = 1; i < nc; ++i) {
    T dii = idt - kap * (T)di[i];
    if (i == nc - 1) dii += (T)(a.betaj[e] * a.gs[e]);
    const T l = TRANS ? -kap * (T)up[i - 1] : -kap * (T)lo[i];
    const T den = dii - l * cp[i - 1];
    if (i < nc - 1) cp[i] = (TRANS ? -kap * (T)lo[i + 1] : -kap * (T)up[i]) / den;
    x[i] = (x[i] - l * x[i - 1]) / den;
  }
  for (int i = nc - 2; i >= 0; --i) x[i] -= cp[i] * x[i + 1];
}

// Step 1 + condensation coefficient: y_c = T^-1 (s^-1 r_c) stored in yc.
template <typename T, bool TRANS>
__global__ void k_part_fwd(PcArgs a, const double* __restrict__ r, T* __restrict__ yc, bool scaled) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.NE) return;
  const int nc = a.nc;
  const int64_t nn = a.g.nn;
  T x[kMaxNc];
  const double iM = 1.0 / a.Mj[e];
  for (int i = 0; i < nc; ++i) {
    const int64_t row = 3 * nn + e * nc + i;
    x[i] = (T)(r[row] * insc(a, scaled, 3, row) * iM);
  }
  particle_thomas<T, TRANS>(a, e, x);
  for (int i = 0; i < nc; ++i) yc[e * nc + i] = x[i];
}

// Local vectors at electrode node e: u = (A act, -A, -tau A, M beta),
// v = (g_eta act, -g_eta, g_c, g_s).
__device__ __forceinline__ void local_uv(const PcArgs& a, int64_t e, bool act, double* u, double* v) {
  const double A = a.Aj[e];
  u[0] = act ? A : 0.0; u[1] = -A; u[2] = -a.tau * A; u[3] = a.Mj[e] * a.betaj[e];
  const double ge = a.ge[e];
  v[0] = act ? ge : 0.0; v[1] = -ge; v[2] = a.gc[e]; v[3] = a.gs[e];
}

// Load the level-0 multigrid right-hand sides of the fields in `fmask`
// (bit f): r_f = s^-1 r - condensation (FULL) - BGS couplings to the fields
// in `done` (bits, their z already written to zm).  phi_s rows without an
// unknown are identity rows: z = r directly.
template <typename T, bool TRANS, bool FULL>
__global__ void k_load(PcArgs a, const double* __restrict__ r, const T* __restrict__ yc,
                       const double* __restrict__ zm, double* __restrict__ zout, int fmask, int done, bool scaled,
                       T* b0, T* b1, T* b2) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = a.g.nn;
  if (n >= nn) return;
  const int32_t e = a.eidx[n];
  const bool act = a.label[n] & kLabActive;
  double u[4] = {0, 0, 0, 0}, v[4] = {0, 0, 0, 0};
  double yN = 0.0, coup = 0.0;
  if (e >= 0) {
    local_uv(a, e, act, u, v);
    if (FULL) yN = (double)yc[(int64_t)e * a.nc + a.nc - 1];
    if (done) {
      for (int g = 0; g < 3; ++g)
        if (done & (1 << g)) coup += (TRANS ? u[g] : v[g]) * zm[g * nn + n];
      coup *= a.zeta[e];
    }
  }
  T* bs[3] = {b0, b1, b2};
  for (int f = 0; f < 3; ++f) {
    if (!(fmask & (1 << f))) continue;
    double rf = r[f * nn + n] * insc(a, scaled, f, f * nn + n);
    if (e >= 0) {
      // A_mc y_c: column c_N is u_m g_s (transposed: M beta v_m)
      if (FULL) rf -= (TRANS ? u[3] * v[f] : u[f] * v[3]) * yN;
      rf -= (TRANS ? v[f] : u[f]) * coup;
    }
    if (f == 0 && !act) {
      zout[n] = rf;   // identity row
      continue;
    }
    bs[f][n] = (T)(a.sc[f] * rf);
  }
}

template <typename T>
__global__ void k_store(Grid g, const uint8_t* __restrict__ label, int fmask, const T* __restrict__ x0,
                        const T* __restrict__ x1, const T* __restrict__ x2, double* __restrict__ zm) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  if (n >= nn) return;
  const T* xs[3] = {x0, x1, x2};
  for (int f = 0; f < 3; ++f) {
    if (!(fmask & (1 << f))) continue;
    if (f == 0 && !(label[n] & kLabActive)) continue;
    zm[f * nn + n] = (double)xs[f][n];
  }
}

// z_c = y_c - T^-1 (A_cm z_m): A_cm z_m is nonzero only in the surface row.
template <typename T, bool TRANS>
__global__ void k_part_bwd(PcArgs a, const T* __restrict__ yc, const double* __restrict__ z, double* __restrict__ zc) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.NE) return;
  const int nc = a.nc;
  const int64_t nn = a.g.nn;
  const int64_t n = a.enode[e];
  const bool act = a.label[n] & kLabActive;
  double u[4], v[4];
  local_uv(a, e, act, u, v);
  double t = 0.0;
  for (int f = 0; f < 3; ++f) t += (TRANS ? u[f] * v[3] : u[3] * v[f]) * z[f * nn + n];
  T w[kMaxNc];
  for (int i = 0; i < nc; ++i) w[i] = (T)0;
  w[nc - 1] = (T)(1.0 / a.Mj[e]);
  particle_thomas<T, TRANS>(a, e, w);
  for (int i = 0; i < nc; ++i) zc[e * nc + i] = (double)yc[e * nc + i] - t * (double)w[i];
}

PcArgs make_pc(p4d_ctx* c) {
  PcArgs a;
  a.g = c->g; a.NE = c->NE; a.nc = c->nc;
  a.tau = (1.0 - c->prm.tplus) / c->prm.F; a.dt = c->prm.dt; a.idt = 1.0 / c->prm.dt;
  a.label = c->label; a.eidx = c->eidx; a.enode = c->enode;
  a.Aj = c->Aj; a.Mj = c->Mj; a.betaj = c->betaj; a.kapj = c->kapj; a.rref = c->rref;
  a.ge = c->ge; a.gc = c->gc; a.gs = c->gs; a.zeta = c->zeta; a.sqd = c->sqd; a.iwf = c->iwf;
  for (int f = 0; f < 3; ++f) a.sc[f] = c->scale_f[f];
  return a;
}

// fields of the multigrid hierarchies
const int kHOfField[3][2] = {{0, 1}, {2, -1}, {3, -1}};

template <typename T, bool TRANS, bool FULL>
p4d_status apply_t(p4d_ctx* c, const double* r, double* z, bool scaled) {
  PcArgs a = make_pc(c);
  const int64_t nn = c->g.nn;
  T* yc = (T*)c->yc;
  if (FULL && c->NE > 0)
    ::p4d::count_launch(), k_part_fwd<T, TRANS><<<nblocks(c->NE, 128), 128, 0, c->stream>>>(a, r, yc, scaled);
  MGLevel& l0 = c->lev[0];
  T* b[3] = {(T*)l0.b[0], (T*)l0.b[2], (T*)l0.b[3]};
  if (c->prm.combine == 0) {
    ::p4d::count_launch(), k_load<T, TRANS, FULL><<<nblocks(nn), kBlock, 0, c->stream>>>(a, r, yc, z, z, 7, 0, scaled, b[0], b[1], b[2]);
    const int hs[4] = {0, 1, 2, 3};
    P4D_TRYS(mg_vcycle(c, hs, 4));
    ::p4d::count_launch(), k_store<T><<<nblocks(nn), kBlock, 0, c->stream>>>(c->g, c->label, 7, (const T*)l0.x[0], (const T*)l0.x[2],
                                                      (const T*)l0.x[3], z);
  } else {
    int done = 0;
    for (int t = 0; t < 3; ++t) {
      const int f = TRANS ? c->prm.order[2 - t] : c->prm.order[t];
      ::p4d::count_launch(), k_load<T, TRANS, FULL><<<nblocks(nn), kBlock, 0, c->stream>>>(a, r, yc, z, z, 1 << f, done, scaled, b[0], b[1],
                                                                   b[2]);
      int hs[2];
      int nh = 0;
      for (int q = 0; q < 2; ++q)
        if (kHOfField[f][q] >= 0) hs[nh++] = kHOfField[f][q];
      P4D_TRYS(mg_vcycle(c, hs, nh));
      ::p4d::count_launch(), k_store<T><<<nblocks(nn), kBlock, 0, c->stream>>>(c->g, c->label, 1 << f, (const T*)l0.x[0], (const T*)l0.x[2],
                                                        (const T*)l0.x[3], z);
      done |= 1 << f;
    }
  }
  if (FULL && c->NE > 0)
    ::p4d::count_launch(), k_part_bwd<T, TRANS><<<nblocks(c->NE, 128), 128, 0, c->stream>>>(a, yc, z, z + 3 * nn);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

template <bool FULL>
p4d_status apply_dispatch(p4d_ctx* c, const double* r, double* z, int transpose, bool scaled) {
  if (c->prm.precision == 0)
    return transpose ? apply_t<double, true, FULL>(c, r, z, scaled) : apply_t<double, false, FULL>(c, r, z, scaled);
  return transpose ? apply_t<float, true, FULL>(c, r, z, scaled) : apply_t<float, false, FULL>(c, r, z, scaled);
}

// FP64 particle solve y = T^-1 (rc - e_N tN) (tN optional) for the reduced
// mode's condensation and back substitution, with the LU factors of T/M
// stored at the linearization (no divisions: FP64 divides run at 1/58 of the
// FP32 rate on this GPU).  T/M = L U; transposed: T^T/M = U^T L^T.
template <bool TRANS>
__global__ void k_part64(PcArgs a, const double* __restrict__ ipiv, const double* __restrict__ mult,
                         const double* __restrict__ rc, double* __restrict__ yc, const double* __restrict__ tN) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= a.NE) return;
  const int nc = a.nc;
  const double iM = 1.0 / a.Mj[e];
  const double kap = a.kapj[e];
  const double* up = a.rref + 2 * nc;
  const double* ip = ipiv + e * nc;
  const double* ml = mult + e * nc;
  const double* r = rc + e * nc;
  double* y = yc + e * nc;
  const double tl = tN ? tN[e] : 0.0;
  if (!TRANS) {
    // L z = r/M (forward), U y = z (backward); z kept in y
    double zp = r[0] * iM;
    y[0] = zp;
    for (int i = 1; i < nc; ++i) {
      double ri = r[i];
      if (i == nc - 1) ri -= tl;
      zp = fma(-ml[i], zp, ri * iM);
      y[i] = zp;
    }
    double yn = y[nc - 1] * ip[nc - 1];
    y[nc - 1] = yn;
    for (int i = nc - 2; i >= 0; --i) {
      yn = (y[i] + kap * up[i] * yn) * ip[i];   // U_{i,i+1} = -kap up_i
      y[i] = yn;
    }
  } else {
    // U^T z = r/M (forward), L^T y = z (backward)
    double zp = r[0] * iM * ip[0];
    y[0] = zp;
    for (int i = 1; i < nc; ++i) {
      double ri = r[i];
      if (i == nc - 1) ri -= tl;
      zp = (ri * iM + kap * up[i - 1] * zp) * ip[i];
      y[i] = zp;
    }
    double yn = y[nc - 1];
    for (int i = nc - 2; i >= 0; --i) {
      yn = fma(-ml[i + 1], yn, y[i]);
      y[i] = yn;
    }
  }
}

}  // namespace

p4d_status precond_full(p4d_ctx* c, const double* r, double* z, int transpose, bool scaled) {
  return apply_dispatch<true>(c, r, z, transpose, scaled);
}

p4d_status precond_macro(p4d_ctx* c, const double* rm, double* zm, int transpose, bool scaled) {
  return apply_dispatch<false>(c, rm, zm, transpose, scaled);
}

p4d_status particle_solve64(p4d_ctx* c, const double* rc, double* yc, const double* tN, int transpose) {
  if (c->NE == 0) return P4D_OK;
  PcArgs a = make_pc(c);
  const double* ip = c->tfac;
  const double* ml = c->tfac + (size_t)c->NE * c->nc;
  if (transpose) ::p4d::count_launch(), k_part64<true><<<nblocks(c->NE, 128), 128, 0, c->stream>>>(a, ip, ml, rc, yc, tN);
  else ::p4d::count_launch(), k_part64<false><<<nblocks(c->NE, 128), 128, 0, c->stream>>>(a, ip, ml, rc, yc, tN);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

}  // namespace p4d
