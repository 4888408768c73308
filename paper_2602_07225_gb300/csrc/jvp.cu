// Coupled Jacobian-vector products (paper section 4, eq. blocks), FP64.
//
// Structure used: the electrode-level blocks are the fixed 27-point stencils
// K_sigma (lifted phi_s), K_kappa, C = M_eps/dt + K_D; the diffusion-potential
// block is K_kappa diag(gamma / c_e); every other coupling is node-local and,
// at electrode node j, of rank one:
//     L_j = u_j v_j^T,  u = (A act, -A, -tau A, M beta),  v = (g_eta act, -g_eta, g_c, g_s)
// over (phi_s, phi_e, c_e, c_s surface).  The particle rows add
// M (I/dt - kap Lref).  The reduced (Schur) operator replaces the local term by
// zeta_j u_m v_m^T with zeta_j = 1 - z_j g_s M_j beta_j.
//
// Output forms: y = sc .* (J x) or y = sc .* (b - J x), sc = w_f / sqrt(d) in
// the scaled Krylov space, 1 otherwise.
#include <mutex>
#include "p4d_common.cuh"

namespace p4d {
namespace {

struct JvpArgs {
  Grid g;
  int64_t NE;
  int nc;
  double tau, dt, idt;
  const double* Jst;
  const uint8_t* label;
  const int32_t* eidx;
  const double *Aj, *Mj, *betaj, *kapj, *rref;
  const double *ge, *gc, *gs, *zeta, *gdc, *rsqd, *wf;
  double* tloc;
  const double* u;     // optional precombined phi_e + gamma/c_e * c_e of the input (non-transposed)
};

__device__ __forceinline__ double outscale(const JvpArgs& a, bool scaled, int f, int64_t row) {
  return scaled ? a.wf[f] * a.rsqd[row] : 1.0;
}

// u = x_phie + (gamma / c_e) x_ce: the input of the K_kappa stencil in the
// phi_e rows, formed once per node instead of once per stencil neighbour.
__global__ void k_jvp_combine(int64_t nn, const double* __restrict__ x, const double* __restrict__ gdc,
                              double* __restrict__ u) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  u[n] = fma(gdc[n], x[2 * nn + n], x[nn + n]);
}

// Macro rows.  reduced: Schur operator on [phi_s | phi_e | c_e] only.
template <bool TRANS, bool REDUCED>
__global__ void __launch_bounds__(128) k_jvp_macro(JvpArgs a, const double* __restrict__ x,
                                                   const double* __restrict__ b, double* __restrict__ y,
                                                   bool scaled) {
  const int64_t nn = a.g.nn;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % a.g.nnx);
  const int j = (int)((n / a.g.nnx) % a.g.nny);
  const int k = (int)(n / ((int64_t)a.g.nnx * a.g.nny));
  const double* xs = x;
  const double* xe = x + nn;
  const double* xc = x + 2 * nn;
  const double* Ks = a.Jst;
  const double* Kk = a.Jst + 27 * nn;
  const double* Cc = a.Jst + 2 * 27 * nn;
  double ys = 0.0, ye = 0.0, yc = 0.0;
  const bool act = a.label[n] & kLabActive;
#pragma unroll
  for (int o = 0; o < 27; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || jj < 0 || kk < 0 || ii >= a.g.nnx || jj >= a.g.nny || kk >= a.g.nnz) continue;
    const int64_t m = n + dx + (int64_t)a.g.nnx * (dy + (int64_t)a.g.nny * dz);
    const int64_t so = o * nn + n;
    if (act) ys += Ks[so] * xs[m];
    const double kk_ = Kk[so];
    if (!TRANS) ye += kk_ * (a.u ? a.u[m] : fma(a.gdc[m], xc[m], xe[m]));
    else ye += kk_ * xe[m];
    yc += Cc[so] * xc[m];
  }
  if (TRANS) yc += a.gdc[n] * ye;   // (K_kappa diag(gamma/c_e))^T = diag(gamma/c_e) K_kappa
  if (!act) ys = xs[n];
  const int32_t e = a.eidx[n];
  if (e >= 0) {
    const double A = a.Aj[e];
    const double ge = a.ge[e];
    if (!TRANS) {
      // t = v . x  (c_s surface value only in the full operator)
      double t = (act ? ge * xs[n] : 0.0) - ge * xe[n] + a.gc[e] * xc[n];
      if (REDUCED) t *= a.zeta[e];
      else t += a.gs[e] * x[3 * nn + (int64_t)e * a.nc + a.nc - 1];
      if (act) ys += A * t;
      ye -= A * t;
      yc -= a.tau * A * t;
      if (!REDUCED) a.tloc[e] = t;
    } else {
      // t = u . x
      double t = (act ? A * xs[n] : 0.0) - A * xe[n] - a.tau * A * xc[n];
      if (REDUCED) t *= a.zeta[e];
      else t += a.Mj[e] * a.betaj[e] * x[3 * nn + (int64_t)e * a.nc + a.nc - 1];
      if (act) ys += ge * t;
      ye -= ge * t;
      yc += a.gc[e] * t;
      if (!REDUCED) a.tloc[e] = t;
    }
  }
  if (b) {
    ys = b[n] - ys;
    ye = b[nn + n] - ye;
    yc = b[2 * nn + n] - yc;
  }
  y[n] = outscale(a, scaled, 0, n) * ys;
  y[nn + n] = outscale(a, scaled, 1, nn + n) * ye;
  y[2 * nn + n] = outscale(a, scaled, 2, 2 * nn + n) * yc;
}

// Particle rows of the full operator (after k_jvp_macro wrote tloc).
template <bool TRANS>
__global__ void k_jvp_particle(JvpArgs a, const double* __restrict__ x, const double* __restrict__ b,
                               double* __restrict__ y, bool scaled) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nc = a.nc;
  if (q >= a.NE * nc) return;
  const int64_t e = (uint32_t)q / (uint32_t)nc;   // NE nc < 2^31 (checked at setup)
  const int i = (int)(q - e * nc);
  const int64_t nn = a.g.nn;
  const double* xc = x + 3 * nn + e * nc;
  const double* lo = a.rref;
  const double* di = a.rref + nc;
  const double* up = a.rref + 2 * nc;
  double L = di[i] * xc[i];
  if (!TRANS) {
    if (i > 0) L += lo[i] * xc[i - 1];
    if (i < nc - 1) L += up[i] * xc[i + 1];
  } else {
    if (i > 0) L += up[i - 1] * xc[i - 1];
    if (i < nc - 1) L += lo[i + 1] * xc[i + 1];
  }
  double v = a.Mj[e] * (xc[i] * a.idt - a.kapj[e] * L);
  if (i == nc - 1) v += (TRANS ? a.gs[e] : a.Mj[e] * a.betaj[e]) * a.tloc[e];
  if (b) v = b[3 * nn + q] - v;
  y[3 * nn + q] = outscale(a, scaled, 3, 3 * nn + q) * v;
}

JvpArgs make_args(p4d_ctx* c) {
  JvpArgs a;
  a.g = c->g; a.NE = c->NE; a.nc = c->nc;
  a.tau = (1.0 - c->prm.tplus) / c->prm.F; a.dt = c->prm.dt; a.idt = 1.0 / c->prm.dt;
  a.Jst = c->Jst; a.label = c->label; a.eidx = c->eidx;
  a.Aj = c->Aj; a.Mj = c->Mj; a.betaj = c->betaj; a.kapj = c->kapj; a.rref = c->rref;
  a.ge = c->ge; a.gc = c->gc; a.gs = c->gs; a.zeta = c->zeta; a.gdc = c->gdc; a.rsqd = c->rsqd; a.wf = c->wf;
  a.tloc = c->tloc;
  a.u = nullptr;
  return a;
}

}  // namespace

p4d_status jvp_full(p4d_ctx* c, const double* x, double* y, int transpose, const double* b, bool scaled) {
  JvpArgs a = make_args(c);
  const int64_t nn = c->g.nn;
  if (!transpose) {
    ::p4d::count_launch(), k_jvp_combine<<<nblocks(nn), kBlock, 0, c->stream>>>(nn, x, c->gdc, c->ujvp);
    a.u = c->ujvp;
  }
  if (transpose) ::p4d::count_launch(), k_jvp_macro<true, false><<<nblocks(nn, 128), 128, 0, c->stream>>>(a, x, b, y, scaled);
  else ::p4d::count_launch(), k_jvp_macro<false, false><<<nblocks(nn, 128), 128, 0, c->stream>>>(a, x, b, y, scaled);
  if (c->NE > 0) {
    const int64_t np = c->NE * c->nc;
    if (transpose) ::p4d::count_launch(), k_jvp_particle<true><<<nblocks(np), kBlock, 0, c->stream>>>(a, x, b, y, scaled);
    else ::p4d::count_launch(), k_jvp_particle<false><<<nblocks(np), kBlock, 0, c->stream>>>(a, x, b, y, scaled);
  }
  P4D_TRYS(transport_jvp(c, x, y, transpose, b, scaled));
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status jvp_reduced(p4d_ctx* c, const double* x, double* y, int transpose, const double* b, bool scaled) {
  JvpArgs a = make_args(c);
  const int64_t nn = c->g.nn;
  if (!transpose) {
    ::p4d::count_launch(), k_jvp_combine<<<nblocks(nn), kBlock, 0, c->stream>>>(nn, x, c->gdc, c->ujvp);
    a.u = c->ujvp;
  }
  if (transpose) ::p4d::count_launch(), k_jvp_macro<true, true><<<nblocks(nn, 128), 128, 0, c->stream>>>(a, x, b, y, scaled);
  else ::p4d::count_launch(), k_jvp_macro<false, true><<<nblocks(nn, 128), 128, 0, c->stream>>>(a, x, b, y, scaled);
  P4D_TRYS(transport_jvp(c, x, y, transpose, b, scaled));
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

}  // namespace p4d

// ---------------------------------------------------------------------------
// p4d_jvp_noalloc: the full-layout coupled JVP with its one piece of scratch
// (the node-local coupling scalar per electrode node, written by the
// macro-row kernel and read by the particle-row kernel) kept in a fixed
// device array of this file instead of the handle's workspace.  Every GPU
// that loads the library holds this array until the process exits.
namespace p4d {

static __device__ __align__(256) double g_noalloc_tloc[P4D_NOALLOC_MAX_NELEC];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of g_noalloc_tloc on the handle's device, looked up once per
// device with that device current (in host code the array's name is only a
// stand-in for the device symbol, never a device address).  The handle's
// kernels run on its stream, on the device it was set up on; a caller with
// another device current gets INVALID_ARG instead of another GPU's array.
p4d_status noalloc_scratch(const p4d_ctx* h, double** out) {
  int dev = -1;
  P4D_TRY(cudaGetDevice(&dev));
  if (dev != h->device) return P4D_ERR_INVALID_ARG;
  if (dev < 0 || dev >= kMaxDevices) return P4D_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_tloc) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return P4D_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = static_cast<double*>(g_noalloc_ptr[dev]);
  return P4D_OK;
}

}  // namespace
}  // namespace p4d

extern "C" p4d_status p4d_jvp_noalloc(p4d_handle h, const double* x, double* y, int transpose) {
  using namespace p4d;
  if (!h || !x || !y || x == y || !h->linearized) return P4D_ERR_INVALID_ARG;
  if (h->NE > (int64_t)P4D_NOALLOC_MAX_NELEC || h->prm.transport_model != 0) return P4D_ERR_INVALID_ARG;
  double* tloc = nullptr;
  P4D_TRYS(noalloc_scratch(h, &tloc));
  JvpArgs a = make_args(h);
  a.tloc = tloc;   // each entry read by the particle rows is written first by the macro rows
  const int64_t nn = h->g.nn;
  if (transpose) ::p4d::count_launch(), k_jvp_macro<true, false><<<nblocks(nn, 128), 128, 0, h->stream>>>(a, x, nullptr, y, false);
  else ::p4d::count_launch(), k_jvp_macro<false, false><<<nblocks(nn, 128), 128, 0, h->stream>>>(a, x, nullptr, y, false);
  if (h->NE > 0) {
    const int64_t np = h->NE * h->nc;
    if (transpose) ::p4d::count_launch(), k_jvp_particle<true><<<nblocks(np), kBlock, 0, h->stream>>>(a, x, nullptr, y, false);
    else ::p4d::count_launch(), k_jvp_particle<false><<<nblocks(np), kBlock, 0, h->stream>>>(a, x, nullptr, y, false);
  }
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}
