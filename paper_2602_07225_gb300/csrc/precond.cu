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
  const double *Aj, *Mj, *iMj, *betaj, *kapj, *rref;
  const double *ge, *gc, *gs, *zeta, *sqd, *iwf;
  const double* Kk;     // K_kappa stencil [27][nn] (FP64, fixed)
  const double* gdc;    // gamma / c_e per node
  double sc[3];
};

// The one stencil coupling between the electrode-level blocks: the
// diffusion-potential block S[phi_e][c_e] = K_kappa diag(gamma / c_e)
// (eq. phie-weak; every other coupling is node-local).  Forward:
// (K_kappa diag(gamma/c_e) z_ce)_n; transposed: (diag(gamma/c_e) K_kappa z_phie)_n
// (K_kappa is symmetric).  zsrc: the done field's solution.
template <bool TRANS>
__device__ __forceinline__ double diffpot_coupling(const PcArgs& a, int64_t n, const double* __restrict__ zsrc) {
  const int64_t nn = a.g.nn;
  const int i = (int)(n % a.g.nnx);
  const int j = (int)((n / a.g.nnx) % a.g.nny);
  const int k = (int)(n / ((int64_t)a.g.nnx * a.g.nny));
  double acc = 0.0;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || jj < 0 || kk < 0 || ii >= a.g.nnx || jj >= a.g.nny || kk >= a.g.nnz) continue;
    const int64_t m = n + dx + (int64_t)a.g.nnx * (dy + (int64_t)a.g.nny * dz);
    acc += a.Kk[o * nn + n] * (TRANS ? zsrc[m] : a.gdc[m] * zsrc[m]);
  }
  return TRANS ? a.gdc[n] * acc : acc;
}

__device__ __forceinline__ double insc(const PcArgs& a, bool scaled, int f, int64_t row) {
  return scaled ? a.sqd[row] * a.iwf[f] : 1.0;
}

constexpr int kPartBlock = 128;   // nodes per block of the staged particle kernels

// LU factors of T_j / M_j in precision T, radial-major ([nc][NE]): 1/pivot
// and multiplier (unit lower L, upper U with U_{i,i+1} = -kap_j up_i).
template <typename T>
struct PartLU {
  const T* ip;
  const T* ml;
};

// In-place solve of (T_j/M_j) y = x (TRANS: its transpose) for one particle
// with the stored factors, x[i] at x[i] (stride 1), factor entry i of node
// e at f[i * NE + e].  Division free.
template <typename T, bool TRANS>
__device__ __forceinline__ void particle_lu_solve(const PartLU<T>& F, int64_t NE, int64_t e, int nc, T kap,
                                                  const double* __restrict__ up, T* x) {
  const T* ip = F.ip + e;
  const T* ml = F.ml + e;
  if (!TRANS) {
    T zp = x[0];
    for (int i = 1; i < nc; ++i) {
      zp = x[i] - ml[i * NE] * zp;
      x[i] = zp;
    }
    T yn = x[nc - 1] * ip[(nc - 1) * NE];
    x[nc - 1] = yn;
    for (int i = nc - 2; i >= 0; --i) {
      yn = (x[i] + kap * (T)up[i] * yn) * ip[i * NE];
      x[i] = yn;
    }
  } else {
    T zp = x[0] * ip[0];
    x[0] = zp;
    for (int i = 1; i < nc; ++i) {
      zp = (x[i] + kap * (T)up[i - 1] * zp) * ip[i * NE];
      x[i] = zp;
    }
    T yn = x[nc - 1];
    for (int i = nc - 2; i >= 0; --i) {
      yn = x[i] - ml[(i + 1) * NE] * yn;
      x[i] = yn;
    }
  }
}

// Step 1 + condensation coefficient: y_c = T^-1 (s^-1 r_c), written to yc
// radial-major ([nc][NE], internal).  The block's node-major slab of r goes
// through shared memory (rows padded to an odd stride).
template <typename T, bool TRANS>
__global__ void __launch_bounds__(kPartBlock) k_part_fwd(PcArgs a, PartLU<T> F, VRef rref_, T* __restrict__ yc,
                                                         bool scaled) {
  __shared__ T sl[kPartBlock * (kMaxNc + 1)];
  const double* __restrict__ r = rref_.get();
  const int nc = a.nc, ld = nc | 1;
  const int64_t NE = a.NE, nn = a.g.nn;
  const int64_t e0 = (int64_t)blockIdx.x * kPartBlock;
  const int nb = NE - e0 < kPartBlock ? (int)(NE - e0) : kPartBlock;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < nb; q += kPartBlock / 32)
    if (lane < nc) {
      const int64_t row = 3 * nn + (e0 + q) * nc + lane;
      sl[q * ld + lane] = (T)(r[row] * insc(a, scaled, 3, row) * a.iMj[e0 + q]);
    }
  __syncthreads();
  if (threadIdx.x >= nb) return;
  const int64_t e = e0 + threadIdx.x;
  T* x = sl + threadIdx.x * ld;
  particle_lu_solve<T, TRANS>(F, NE, e, nc, (T)a.kapj[e], a.rref + 2 * nc, x);
  for (int i = 0; i < nc; ++i) yc[i * NE + e] = x[i];
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
__global__ void k_load(PcArgs a, VRef rref_, const T* __restrict__ yc, VRef zref_, int fmask, int done, bool scaled,
                       T* b0, T* b1, T* b2) {
  const double* __restrict__ r = rref_.get();
  const double* zm = zref_.get();
  double* zout = zref_.get();
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = a.g.nn;
  if (n >= nn) return;
  const int32_t e = a.eidx[n];
  const bool act = a.label[n] & kLabActive;
  // the node couplings are needed only for the FULL condensation and for
  // BGS corrections (the reduced block-Jacobi load is a pure scaling, and
  // FP64 arithmetic is the cost of this kernel)
  const bool coupled = e >= 0 && (FULL || done);
  double u[4] = {0, 0, 0, 0}, v[4] = {0, 0, 0, 0};
  double yN = 0.0, coup = 0.0;
  if (coupled) {
    local_uv(a, e, act, u, v);
    if (FULL) yN = (double)yc[(int64_t)(a.nc - 1) * a.NE + e];
    if (done) {
      for (int g = 0; g < 3; ++g)
        if (done & (1 << g)) coup += (TRANS ? u[g] : v[g]) * zm[g * nn + n];
      coup *= a.zeta[e];
    }
  }
  T* bs[3] = {b0, b1, b2};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (!(fmask & (1 << f))) continue;
    const int64_t row = f * nn + n;
    const bool dpc = (!TRANS && f == 1 && (done & 4)) || (TRANS && f == 2 && (done & 2));
    if (sizeof(T) == sizeof(float) && scaled && !coupled && !dpc && !(f == 0 && !act)) {
      // FP32 right-hand side of an FP32 cycle: the scaling in FP32 (FP64
      // multiplies are this kernel's cost)
      const float w = (float)(a.iwf[f] * a.sc[f]);
      bs[f][n] = (T)(((float)r[row] * (float)a.sqd[row]) * w);
      continue;
    }
    double rf = scaled ? (r[row] * a.sqd[row]) * a.iwf[f] : r[row];
    if (coupled) {
      // A_mc y_c: column c_N is u_m g_s (transposed: M beta v_m)
      if (FULL) rf -= (TRANS ? u[3] * v[f] : u[f] * v[3]) * yN;
      rf -= (TRANS ? v[f] : u[f]) * coup;
    }
    // BGS: the diffusion-potential block couples phi_e to c_e over the stencil
    if (dpc) rf -= TRANS ? diffpot_coupling<true>(a, n, zm + nn) : diffpot_coupling<false>(a, n, zm + 2 * nn);
    if (f == 0 && !act) {
      zout[n] = rf;   // identity row
      continue;
    }
    bs[f][n] = (T)(a.sc[f] * rf);
  }
}

template <typename T>
__global__ void k_store(Grid g, const uint8_t* __restrict__ label, int fmask, const T* __restrict__ x0,
                        const T* __restrict__ x1, const T* __restrict__ x2, VRef zref_) {
  double* __restrict__ zm = zref_.get();
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

// z_c = y_c - T^-1 (A_cm z_m): A_cm z_m is nonzero only in the surface row,
// so T^-1 A_cm z_m = t w with w = T^-1 e_N / M (one backward recurrence
// with the stored factors).  z_c (node-major) is written through shared
// memory for coalesced stores.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(kPartBlock) k_part_bwd(PcArgs a, PartLU<T> F, const T* __restrict__ yc,
                                                         VRef zref_) {
  __shared__ double sl[kPartBlock * (kMaxNc + 1)];
  const double* __restrict__ z = zref_.get();
  double* __restrict__ zc = zref_.get() + 3 * a.g.nn;
  const int nc = a.nc, ld = nc | 1;
  const int64_t NE = a.NE, nn = a.g.nn;
  const int64_t e0 = (int64_t)blockIdx.x * kPartBlock;
  const int nb = NE - e0 < kPartBlock ? (int)(NE - e0) : kPartBlock;
  if (threadIdx.x < nb) {
    const int64_t e = e0 + threadIdx.x;
    const int64_t n = a.enode[e];
    const bool act = a.label[n] & kLabActive;
    double u[4], v[4];
    local_uv(a, e, act, u, v);
    double t = 0.0;
    for (int f = 0; f < 3; ++f) t += (TRANS ? u[f] * v[3] : u[3] * v[f]) * z[f * nn + n];
    const T kap = (T)a.kapj[e];
    const double* up = a.rref + 2 * nc;
    const T* ip = F.ip + e;
    const T* ml = F.ml + e;
    double* out = sl + threadIdx.x * ld;
    const T iM = (T)a.iMj[e];
    if (!TRANS) {
      // L z' = e_N / M gives z' = e_N / M; U w = z'
      T w = iM * ip[(nc - 1) * NE];
      out[nc - 1] = (double)yc[(nc - 1) * NE + e] - t * (double)w;
      for (int i = nc - 2; i >= 0; --i) {
        w = kap * (T)up[i] * w * ip[i * NE];
        out[i] = (double)yc[i * NE + e] - t * (double)w;
      }
    } else {
      // U^T z' = e_N / M gives z' = e_N ip_N / M; L^T w = z'
      T w = iM * ip[(nc - 1) * NE];
      out[nc - 1] = (double)yc[(nc - 1) * NE + e] - t * (double)w;
      for (int i = nc - 2; i >= 0; --i) {
        w = -ml[(i + 1) * NE] * w;
        out[i] = (double)yc[i * NE + e] - t * (double)w;
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < nb; q += kPartBlock / 32)
    if (lane < nc) zc[(e0 + q) * nc + lane] = sl[q * ld + lane];
}

PcArgs make_pc(p4d_ctx* c) {
  PcArgs a;
  a.g = c->g; a.NE = c->NE; a.nc = c->nc;
  a.tau = (1.0 - c->prm.tplus) / c->prm.F; a.dt = c->prm.dt; a.idt = 1.0 / c->prm.dt;
  a.label = c->label; a.eidx = c->eidx; a.enode = c->enode;
  a.Aj = c->Aj; a.Mj = c->Mj; a.iMj = c->iMj; a.betaj = c->betaj; a.kapj = c->kapj; a.rref = c->rref;
  a.ge = c->ge; a.gc = c->gc; a.gs = c->gs; a.zeta = c->zeta; a.sqd = c->sqd; a.iwf = c->iwf;
  a.Kk = c->Jst + 27 * c->g.nn; a.gdc = c->gdc;
  for (int f = 0; f < 3; ++f) a.sc[f] = c->scale_f[f];
  return a;
}

// fields of the multigrid hierarchies
const int kHOfField[3][2] = {{0, 1}, {2, -1}, {3, -1}};

template <typename T, bool TRANS, bool FULL>
p4d_status apply_t(p4d_ctx* c, VRef r, VRef z, bool scaled) {
  PcArgs a = make_pc(c);
  const int64_t nn = c->g.nn;
  T* yc = (T*)c->yc;
  PartLU<T> F;
  const T* fac = sizeof(T) == sizeof(double) ? (const T*)c->tfac : (const T*)c->tfac32;
  F.ip = fac;
  F.ml = fac + (size_t)c->NE * c->nc;
  if (FULL && c->NE > 0)
    ::p4d::count_launch(), k_part_fwd<T, TRANS><<<nblocks(c->NE, kPartBlock), kPartBlock, 0, c->stream>>>(a, F, r, yc, scaled);
  MGLevel& l0 = c->lev[0];
  T* b[3] = {(T*)l0.b[0], (T*)l0.b[2], (T*)l0.b[3]};
  if (c->prm.combine == 0) {
    ::p4d::count_launch(), k_load<T, TRANS, FULL><<<nblocks(nn), kBlock, 0, c->stream>>>(a, r, yc, z, 7, 0, scaled, b[0], b[1], b[2]);
    const int hs[4] = {0, 1, 2, 3};
    P4D_TRYS(mg_vcycle(c, hs, 4));
    ::p4d::count_launch(), k_store<T><<<nblocks(nn), kBlock, 0, c->stream>>>(c->g, c->label, 7, (const T*)l0.x[0], (const T*)l0.x[2],
                                                      (const T*)l0.x[3], z);
  } else {
    int done = 0;
    for (int t = 0; t < 3; ++t) {
      const int f = TRANS ? c->prm.order[2 - t] : c->prm.order[t];
      ::p4d::count_launch(), k_load<T, TRANS, FULL><<<nblocks(nn), kBlock, 0, c->stream>>>(a, r, yc, z, 1 << f, done, scaled, b[0], b[1],
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
    ::p4d::count_launch(), k_part_bwd<T, TRANS><<<nblocks(c->NE, kPartBlock), kPartBlock, 0, c->stream>>>(a, F, yc, z);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

template <bool FULL>
p4d_status apply_dispatch(p4d_ctx* c, VRef r, VRef z, int transpose, bool scaled) {
  if (c->prm.precision == 0)
    return transpose ? apply_t<double, true, FULL>(c, r, z, scaled) : apply_t<double, false, FULL>(c, r, z, scaled);
  return transpose ? apply_t<float, true, FULL>(c, r, z, scaled) : apply_t<float, false, FULL>(c, r, z, scaled);
}

// FP64 particle solve y = T^-1 (rc - e_N tN) (tN optional) for the reduced
// mode's condensation and back substitution, with the LU factors of T/M
// stored at the linearization (no divisions: FP64 divides run at 1/58 of the
// FP32 rate on this GPU).  T/M = L U; transposed: T^T/M = U^T L^T.
template <bool TRANS>
__global__ void __launch_bounds__(kPartBlock) k_part64(PcArgs a, const double* __restrict__ ipiv,
                                                       const double* __restrict__ mult,
                                                       const double* __restrict__ rc, double* __restrict__ yc,
                                                       const double* __restrict__ tN) {
  // the block's node-major slab of r (contiguous) goes through shared memory,
  // node rows padded to an odd stride; each thread solves its node in place
  __shared__ double sl[kPartBlock * (kMaxNc + 1)];
  const int nc = a.nc, ld = nc | 1;
  const int64_t NE = a.NE;
  const int64_t e0 = (int64_t)blockIdx.x * kPartBlock;
  const int nb = NE - e0 < kPartBlock ? (int)(NE - e0) : kPartBlock;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < nb; q += kPartBlock / 32)
    if (lane < nc) sl[q * ld + lane] = rc[(e0 + q) * nc + lane];
  __syncthreads();
  if (threadIdx.x < nb) {
    const int64_t e = e0 + threadIdx.x;
    double* y = sl + threadIdx.x * ld;
    const double iM = a.iMj[e];
    const double kap = a.kapj[e];
    const double* up = a.rref + 2 * nc;
    const double* ip = ipiv + e;     // ip[i * NE]
    const double* ml = mult + e;
    const double tl = tN ? tN[e] : 0.0;
    if (!TRANS) {
      // L z = r/M (forward), U y = z (backward); z kept in y
      double zp = y[0] * iM;
      y[0] = zp;
      for (int i = 1; i < nc; ++i) {
        double ri = y[i];
        if (i == nc - 1) ri -= tl;
        zp = fma(-ml[i * NE], zp, ri * iM);
        y[i] = zp;
      }
      double yn = y[nc - 1] * ip[(nc - 1) * NE];
      y[nc - 1] = yn;
      for (int i = nc - 2; i >= 0; --i) {
        yn = (y[i] + kap * up[i] * yn) * ip[i * NE];   // U_{i,i+1} = -kap up_i
        y[i] = yn;
      }
    } else {
      // U^T z = r/M (forward), L^T y = z (backward)
      double zp = y[0] * iM * ip[0];
      y[0] = zp;
      for (int i = 1; i < nc; ++i) {
        double ri = y[i];
        if (i == nc - 1) ri -= tl;
        zp = (ri * iM + kap * up[i - 1] * zp) * ip[i * NE];
        y[i] = zp;
      }
      double yn = y[nc - 1];
      for (int i = nc - 2; i >= 0; --i) {
        yn = fma(-ml[(i + 1) * NE], yn, y[i]);
        y[i] = yn;
      }
    }
  }
  __syncthreads();
  for (int q = warp; q < nb; q += kPartBlock / 32)
    if (lane < nc) yc[(e0 + q) * nc + lane] = sl[q * ld + lane];
}

}  // namespace

p4d_status precond_full(p4d_ctx* c, const double* r, double* z, int transpose, bool scaled) {
  return apply_dispatch<true>(c, VRef{const_cast<double*>(r), 0, nullptr}, VRef{z, 0, nullptr}, transpose, scaled);
}

p4d_status precond_macro(p4d_ctx* c, const double* rm, double* zm, int transpose, bool scaled) {
  return apply_dispatch<false>(c, VRef{const_cast<double*>(rm), 0, nullptr}, VRef{zm, 0, nullptr}, transpose, scaled);
}

void drop_graphs(p4d_ctx* c) {
  ++c->graph_gen;
  auto drop = [](p4d_ctx::PcGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.kernels = 0;
  };
  for (auto& row : c->pcg)
    for (auto& g : row) drop(g);
  for (auto& row : c->cyc)
    for (auto& g : row) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      g.m = 0;
      g.kernels.clear();
    }
}

// The preconditioner of FGMRES iteration k: z_k = P^-1 (s^-1 v_k).  Every
// kernel of one application reads k from c->kdev, so one captured graph per
// (transpose, layout) serves every column; the Chebyshev coefficients are
// read from the device table, so the graph survives linearization updates.
// The multigrid ping-pong buffers return to their start after each V-cycle
// (2 d swaps per level), so the captured pointers stay those in use.
p4d_status precond_column(p4d_ctx* c, int transpose, bool use_graph) {
  const bool full = c->prm.mode == 0;
  const int64_t len = full ? c->ndof : 3 * c->g.nn;
  const VRef r{c->V, len, c->kdev}, z{c->Z, len, c->kdev};
  auto apply = [&]() {
    return full ? apply_dispatch<true>(c, r, z, transpose, true) : apply_dispatch<false>(c, r, z, transpose, true);
  };
  if (c->prm.profile || !use_graph) return apply();   // per-kernel events cannot sit inside a graph
  p4d_ctx::PcGraph& g = c->pcg[transpose ? 1 : 0][full ? 1 : 0];
  if (!g.exec) P4D_TRYS(capture_graph(c, g, apply));
  count_launches(g.kernels);
  P4D_TRY(cudaGraphLaunch(g.exec, c->stream));
  return P4D_OK;
}

p4d_status particle_solve64(p4d_ctx* c, const double* rc, double* yc, const double* tN, int transpose) {
  if (c->NE == 0) return P4D_OK;
  PcArgs a = make_pc(c);
  const double* ip = c->tfac;
  const double* ml = c->tfac + (size_t)c->NE * c->nc;
  if (transpose) ::p4d::count_launch(), k_part64<true><<<nblocks(c->NE, kPartBlock), kPartBlock, 0, c->stream>>>(a, ip, ml, rc, yc, tN);
  else ::p4d::count_launch(), k_part64<false><<<nblocks(c->NE, kPartBlock), kPartBlock, 0, c->stream>>>(a, ip, ml, rc, yc, tN);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

}  // namespace p4d
