// Matrix-free fine-level (level-0) operator of the multigrid V-cycles: one
// Chebyshev smoothing step or the residual r = b - A x, evaluated from the
// per-element coefficients instead of stored 27-point stencils.
//
// Level-0 operator of each electrode-level block (paper section 3, eqs.
// phis-weak, phie-weak, ce-weak; section 4: the diagonal blocks of the
// Schur-reduced macro operator), in the multigrid's per-field scaling sc_f:
//   phi_s: sc_0 (K_sigma,lifted + diag(v_s))      phi_e: sc_1 (K_kappa + diag(v_e))
//   c_e:   sc_2 (M_eps/dt + K_D + diag(v_c))
// with K_coef = sum_e coef_e K_e the Q1 stiffness, M the consistent mass and
// v the node-diagonal reaction/Schur terms of the linearization.
//
// On a box element with edges (hx, hy, hz) the Q1 element matrices are
// tensor products of the 1D matrices K1 = (1/h)[1 -1; -1 1] and
// M1 = (h/6)[2 1; 1 2], which share the eigenvectors (1, 1) and (1, -1):
// K1 has eigenvalues 0 and 2/h, M1 has h/2 and h/6.  So with the butterfly
// transform H (per axis: s = a + b, d = a - b; H^T H = 8 I in 3D) every
// element operator is diagonal,
//   coef K_e + m M_e = H^T diag(lambda) H / 8,
//   lambda_(a,b,c) = coef [Kx(a) My(b) Mz(c) + Mx(a) Ky(b) Mz(c) + Mx(a) My(b) Kz(c)]
//                    + m Mx(a) My(b) Mz(c),
// and one element costs 24 additions forward, 8 products and 24 additions
// back.  A constant vector maps to the (s,s,s) coefficient only, whose
// stiffness eigenvalue is exactly 0, and the differences of nearly equal
// nodal values are formed exactly: the near-constant modes of the potential
// blocks are kept in FP32 as by the difference form of the stored stencils.
// phi_s is lifted by its zero values at the nodes without a phi_s unknown
// (the multigrid never writes them).
//
// Layout of a launch: each block owns a tile of W x H nodes (W, H up to
// twice the nominal 32 x 8: the last tile of an axis takes the remainder)
// and marches in z over a chunk of node planes.  Per plane it stages the
// (W+2) x (H+2) tile of x in shared memory, evaluates the (W+1) x (H+1)
// elements between that plane and the next (their lower-corner outputs go
// to this plane, the upper-corner outputs are kept for the next), and
// updates its nodes.  The phi_s work list covers only the node planes that
// hold phi_s unknowns.
#include <algorithm>
#include <cstdlib>
#include <vector>
#include "p4d_common.cuh"

namespace p4d {
namespace {

constexpr int kTX = 32, kTY = 8;        // nominal node tile (one thread per node)
constexpr int kMfThreads = kTX * kTY;
constexpr int kDefaultZChunk = 16;     // node planes per block (tunable: P4D_MF_ZCHUNK)

template <typename T>
struct MfField {
  const T* x;      // level-0 iterate (guarded vector)
  T* xo;           // Chebyshev output x + d
  const T* b;
  const T* dinv;
  T* d;
  T* r;            // residual output
  const T* svs;    // sc_f * variable node diagonal
  const T* kc;     // [nelem] sc_f * stiffness coefficient
  const T* mc;     // [nelem] sc_f * mass coefficient / dt, or nullptr
};

template <typename T>
struct MfArgs {
  int nnx, nny, nnz, nx, ny, nz;
  int ntx, nty;                // tiles per axis
  const T* gx;                 // [3][nx] (2/h, h/2, h/6) / 8 along x
  const T* gy;                 // [3][ny] (2/h, h/2, h/6) along y
  const T* gz;                 // [3][nz] along z
  const uint8_t* label;        // node labels (phi_s unknowns and electrode)
  const int4* items;           // (field, tile, k0, k1) per block
  MfField<T> f[3];
  const T* ctab;               // Chebyshev table (level 0 rows used)
  int step;                    // Chebyshev step of this launch (MODE 0)
  int fmask;                   // fields taking part
};

template <typename T>
__device__ __forceinline__ const MfField<T>& fsel(const MfArgs<T>& a, int f) {
  return f == 0 ? a.f[0] : (f == 1 ? a.f[1] : a.f[2]);
}

template <typename T>
__device__ __forceinline__ T cheb_coef(const T* tab, int step, int j, int h) {
  return tab[((0 * kMaxDeg + step) * 3 + j) * kNH + h];
}

// One element: v = the 8 nodal values (local node a + 2b + 4c), lam = the
// 8 eigenvalues; returns H^T diag(lam) H v in v (the 1/8 is in lam).
template <typename T>
__device__ __forceinline__ void element_apply(T (&v)[8], const T (&lam)[8]) {
#pragma unroll
  for (int st = 1; st < 8; st <<= 1)
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (!(l & st)) {
        const T p = v[l], q = v[l | st];
        v[l] = p + q;
        v[l | st] = p - q;
      }
#pragma unroll
  for (int l = 0; l < 8; ++l) v[l] *= lam[l];
#pragma unroll
  for (int st = 1; st < 8; st <<= 1)
#pragma unroll
    for (int l = 0; l < 8; ++l)
      if (!(l & st)) {
        const T p = v[l], q = v[l | st];
        v[l] = p + q;
        v[l | st] = p - q;
      }
}

// MODE 0: Chebyshev step on a nonzero x: d = c0 D^-1 (b - A x) (step 0) or
// d = ca d + cb D^-1 (b - A x), then x_out = x + d.  MODE 1: r = b - A x.
template <typename T, int MODE>
__global__ void __launch_bounds__(kMfThreads) k_mf_level0(MfArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int4 it = a.items[blockIdx.x];
  const int f = it.x;
  if (!(a.fmask & (1 << f))) return;
  const int tix = it.y % a.ntx, tiy = it.y / a.ntx;
  const int i0 = tix * kTX, j0 = tiy * kTY;
  const int W = tix == a.ntx - 1 ? a.nnx - i0 : kTX;
  const int H = tiy == a.nty - 1 ? a.nny - j0 : kTY;
  const int k0 = it.z, k1 = it.w;
  const int XW = W + 2, XH = H + 2, EW = W + 1, EH = H + 1;
  const int XN = XW * XH, EN = EW * EH;
  T* xs = reinterpret_cast<T*>(smem_raw);          // [2][XN] x planes (ring)
  T* lo = xs + 2 * XN;                              // [4][EN] lower-corner outputs of the current element plane
  T* upA = lo + 4 * EN;                             // [4][EN] upper-corner outputs (two buffers)
  T* upB = upA + 4 * EN;
  T* sgx = upB + 4 * EN;                            // [3][EW] x factors of the tile's element columns
  T* sgy = sgx + 3 * EW;                            // [3][EH]
  const MfField<T>& F = fsel(a, f);
  const int tid = threadIdx.x;
  const int64_t sxy = (int64_t)a.nnx * a.nny;
  const int hA = f == 0 ? 0 : f + 1;               // hierarchy of the field (phi_s: per node)

  for (int q = tid; q < EW; q += kMfThreads) {
    const int ie = i0 - 1 + q;
    const bool in = ie >= 0 && ie < a.nx;
    sgx[q] = in ? a.gx[ie] : (T)0;
    sgx[EW + q] = in ? a.gx[a.nx + ie] : (T)0;
    sgx[2 * EW + q] = in ? a.gx[2 * a.nx + ie] : (T)0;
  }
  for (int q = tid; q < EH; q += kMfThreads) {
    const int je = j0 - 1 + q;
    const bool in = je >= 0 && je < a.ny;
    sgy[q] = in ? a.gy[je] : (T)0;
    sgy[EH + q] = in ? a.gy[a.ny + je] : (T)0;
    sgy[2 * EH + q] = in ? a.gy[2 * a.ny + je] : (T)0;
  }

  // x plane k (nodes (i0-1 .. i0+W) x (j0-1 .. j0+H)) into ring slot k & 1;
  // nodes outside the grid read 0
  auto load_plane = [&](int k) {
    T* dst = xs + (k & 1) * XN;
    const bool kin = k >= 0 && k < a.nnz;
    for (int q = tid; q < XN; q += kMfThreads) {
      const int jj = q / XW, ii = q - jj * XW;
      const int gi = i0 - 1 + ii, gj = j0 - 1 + jj;
      T v = (T)0;
      if (kin && gi >= 0 && gi < a.nnx && gj >= 0 && gj < a.nny) v = F.x[gi + (int64_t)a.nnx * gj + sxy * k];
      dst[q] = v;
    }
  };

  // element plane ke (between node planes ke and ke + 1): lower corners to
  // lo, upper corners to up; elements outside the grid give zero
  auto element_plane = [&](int ke, T* up) {
    const T* xl = xs + (ke & 1) * XN;
    const T* xu = xs + ((ke + 1) & 1) * XN;
    const bool kin = ke >= 0 && ke < a.nz;
    T Ksz = 0, Msz = 0, Mdz = 0;
    if (kin) {
      Ksz = a.gz[ke];
      Msz = a.gz[a.nz + ke];
      Mdz = a.gz[2 * a.nz + ke];
    }
    for (int q = tid; q < EN; q += kMfThreads) {
      const int ej = q / EW, ei = q - ej * EW;
      const int gi = i0 - 1 + ei, gj = j0 - 1 + ej;
      T kc = 0, mc = 0;
      if (kin && gi >= 0 && gi < a.nx && gj >= 0 && gj < a.ny) {
        const int64_t e = gi + (int64_t)a.nx * (gj + (int64_t)a.ny * ke);
        kc = F.kc[e];
        if (F.mc) mc = F.mc[e];
      }
      T v[8];
      const int base = ei + XW * ej;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int off = base + (l & 1) + XW * (l >> 1);
        v[l] = xl[off];
        v[4 + l] = xu[off];
      }
      // eigenvalues (the x factors carry the 1/8)
      const T Kdx = sgx[ei], Msx = sgx[EW + ei], Mdx = sgx[2 * EW + ei];
      const T Kdy = sgy[ej], Msy = sgy[EH + ej], Mdy = sgy[2 * EH + ej];
      // per (y, z) component b + 2c: P = My Mz, Q = Ky Mz + My Kz
      const T P0 = Msy * Msz, P1 = Mdy * Msz, P2 = Msy * Mdz, P3 = Mdy * Mdz;
      const T Q0 = (T)0, Q1 = Kdy * Msz, Q2 = Msy * Ksz, Q3 = Kdy * Mdz + Mdy * Ksz;
      const T As = Msx * mc, Bs = Msx * kc;          // lambda(s, .) = As P + Bs Q
      const T Ad = kc * Kdx + mc * Mdx, Bd = kc * Mdx; // lambda(d, .) = Ad P + Bd Q
      T lam[8];
      lam[0] = As * P0 + Bs * Q0;
      lam[1] = Ad * P0 + Bd * Q0;
      lam[2] = As * P1 + Bs * Q1;
      lam[3] = Ad * P1 + Bd * Q1;
      lam[4] = As * P2 + Bs * Q2;
      lam[5] = Ad * P2 + Bd * Q2;
      lam[6] = As * P3 + Bs * Q3;
      lam[7] = Ad * P3 + Bd * Q3;
      element_apply<T>(v, lam);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        lo[l * EN + q] = v[l];
        up[l * EN + q] = v[4 + l];
      }
    }
  };

  T* upPrev = upA;
  T* upCur = upB;
  load_plane(k0 - 1);
  load_plane(k0);
  __syncthreads();
  if (k0 > 0) {
    element_plane(k0 - 1, upPrev);
  } else {
    for (int q = tid; q < 4 * EN; q += kMfThreads) upPrev[q] = (T)0;
  }
  __syncthreads();

  for (int k = k0; k < k1; ++k) {
    load_plane(k + 1);          // the slot of plane k - 1, no longer read
    __syncthreads();
    element_plane(k, upCur);    // zero outputs when k = nz (no element plane)
    __syncthreads();
    const T* xk = xs + (k & 1) * XN;
    for (int q = tid; q < W * H; q += kMfThreads) {
      const int jj = q / W, ii = q - jj * W;
      const int64_t n = (i0 + ii) + (int64_t)a.nnx * (j0 + jj) + sxy * k;
      int h = hA;
      if (f == 0) {
        const uint8_t lb = a.label[n];
        if (!(lb & kLabActive)) continue;
        h = (lb & kLabAnode) ? 0 : 1;
      }
      T ax = F.svs[n] * xk[(ii + 1) + XW * (jj + 1)];
#pragma unroll
      for (int qq = 0; qq < 2; ++qq)
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int corner = (1 - pp) + 2 * (1 - qq);
          const int e = (ii + pp) + EW * (jj + qq);
          ax += lo[corner * EN + e] + upPrev[corner * EN + e];
        }
      const T res = F.b[n] - ax;
      if (MODE == 1) {
        F.r[n] = res;
      } else {
        const T z = F.dinv[n] * res;
        const T dn = a.step == 0 ? cheb_coef(a.ctab, 0, 0, h) * z
                                 : cheb_coef(a.ctab, a.step, 1, h) * F.d[n] + cheb_coef(a.ctab, a.step, 2, h) * z;
        F.d[n] = dn;
        F.xo[n] = xk[(ii + 1) + XW * (jj + 1)] + dn;
      }
    }
    __syncthreads();            // lo, upPrev and plane k are reused below
    T* t = upPrev;
    upPrev = upCur;
    upCur = t;
  }
}

template <typename T>
__global__ void k_mf_coef(int64_t nelem, const uint8_t* __restrict__ region, const double* __restrict__ eps,
                          const double* __restrict__ eps_s, const double* __restrict__ sig_e, double brug,
                          double kappa, double De, double dt, double s0, double s1, double s2, T* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nelem) return;
  const uint8_t r = region[e];
  const double sig = (r == 0 || r == 2) ? pow(eps_s[e], brug) * sig_e[e] : 0.0;
  const double epb = pow(eps[e], brug);
  out[e] = (T)(s0 * sig);
  out[nelem + e] = (T)(s1 * epb * kappa);
  out[2 * nelem + e] = (T)(s2 * epb * De);
  out[3 * nelem + e] = (T)(s2 * eps[e] / dt);
}

template <typename T>
p4d_status mf_setup_t(p4d_ctx* c) {
  const int nx = c->nx, ny = c->ny, nz = c->nz;
  const int64_t nelem = c->nelem;
  T* coef = nullptr;
  P4D_TRYS(dalloc_t(c, &coef, (size_t)4 * nelem));
  ::p4d::count_launch(), k_mf_coef<T><<<nblocks(nelem), kBlock, 0, c->stream>>>(
      nelem, c->region, c->eps_e, c->epss_e, c->sig_e, c->prm.brug, c->prm.kappa, c->prm.De, c->prm.dt,
      c->scale_f[0], c->scale_f[1], c->scale_f[2], coef);
  c->mf_coef = coef;
  // per-axis factors (2/h, h/2, h/6), the x ones divided by 8
  std::vector<double> hx(nx), hy(ny), hz(nz);
  P4D_TRY(cudaMemcpy(hx.data(), c->hx, nx * sizeof(double), cudaMemcpyDeviceToHost));
  P4D_TRY(cudaMemcpy(hy.data(), c->hy, ny * sizeof(double), cudaMemcpyDeviceToHost));
  P4D_TRY(cudaMemcpy(hz.data(), c->hz, nz * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<T> g(3 * (size_t)(nx + ny + nz));
  size_t o = 0;
  auto put = [&](const std::vector<double>& h, double w) {
    const size_t n = h.size();
    for (size_t i = 0; i < n; ++i) {
      g[o + i] = (T)(w * 2.0 / h[i]);
      g[o + n + i] = (T)(w * h[i] / 2.0);
      g[o + 2 * n + i] = (T)(w * h[i] / 6.0);
    }
    o += 3 * n;
  };
  put(hx, 0.125);
  put(hy, 1.0);
  put(hz, 1.0);
  T* gd = nullptr;
  P4D_TRYS(dalloc_t(c, &gd, g.size()));
  P4D_TRY(cudaMemcpy(gd, g.data(), g.size() * sizeof(T), cudaMemcpyHostToDevice));
  c->mf_geo = gd;
  T* svs = nullptr;
  P4D_TRYS(dalloc_t(c, &svs, (size_t)3 * c->g.nn));
  P4D_TRY(cudaMemset(svs, 0, sizeof(T) * 3 * c->g.nn));
  c->mf_svs = svs;
  return P4D_OK;
}

}  // namespace

// Work list, coefficients and factors of the matrix-free level 0.  phi_s is
// matrix-free only without collector shells (their face stiffness lives in
// the stored stencils).
p4d_status mf_setup(p4d_ctx* c) {
  const int nnx = c->g.nnx, nny = c->g.nny, nnz = c->g.nnz;
  c->mf_phis = !(c->shell_p > 0.0) && !(c->shell_n > 0.0);
  c->mf_ntx = std::max(1, (nnx - 1) / kTX);
  c->mf_nty = std::max(1, (nny - 1) / kTY);
  const int mw = nnx - (c->mf_ntx - 1) * kTX, mh = nny - (c->mf_nty - 1) * kTY;
  int zc = kDefaultZChunk;
  if (const char* s = std::getenv("P4D_MF_ZCHUNK")) zc = std::max(1, std::atoi(s));
  // planes holding phi_s unknowns
  std::vector<uint8_t> lab(c->g.nn);
  P4D_TRY(cudaMemcpy(lab.data(), c->label, c->g.nn, cudaMemcpyDeviceToHost));
  std::vector<int> act(nnz, 0);
  for (int64_t n = 0; n < c->g.nn; ++n)
    if (lab[n] & kLabActive) act[n / ((int64_t)nnx * nny)] = 1;
  std::vector<int4> items;
  const int ntiles = c->mf_ntx * c->mf_nty;
  for (int f = 0; f < 3; ++f) {
    c->mf_off[f] = (int)items.size();
    int k = 0;
    while (k < nnz) {
      if (f == 0 && !act[k]) { ++k; continue; }
      int k1 = k;
      while (k1 < nnz && k1 - k < zc && (f != 0 || act[k1])) ++k1;
      for (int t = 0; t < ntiles; ++t) items.push_back(make_int4(f, t, k, k1));
      k = k1;
    }
    c->mf_cnt[f] = (int)items.size() - c->mf_off[f];
  }
  int4* d = nullptr;
  P4D_TRYS(dalloc_t(c, &d, std::max<size_t>(1, items.size())));
  if (!items.empty()) P4D_TRY(cudaMemcpy(d, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
  c->mf_items = d;
  const size_t ts = c->prm.precision == 0 ? sizeof(double) : sizeof(float);
  const size_t xn = (size_t)(mw + 2) * (mh + 2), en = (size_t)(mw + 1) * (mh + 1);
  c->mf_smem = ts * (2 * xn + 12 * en + 3 * (mw + 1) + 3 * (mh + 1));
  // The kernels' shared-memory limit is a process-wide attribute shared by
  // every handle: set it to the largest tile any grid can have (64 x 16
  // nodes), never to this handle's size, which would fail the launches of
  // larger handles set up before.
  const size_t smax = sizeof(double) * (2 * 66 * 18 + 12 * 65 * 17 + 3 * 65 + 3 * 17);
  if (c->mf_smem > smax) return P4D_ERR_INVALID_ARG;   // cannot happen: tiles are at most 64 x 16 nodes
  P4D_TRY(cudaFuncSetAttribute(k_mf_level0<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  P4D_TRY(cudaFuncSetAttribute(k_mf_level0<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  P4D_TRY(cudaFuncSetAttribute(k_mf_level0<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  P4D_TRY(cudaFuncSetAttribute(k_mf_level0<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  if (c->prm.precision == 0) return mf_setup_t<double>(c);
  return mf_setup_t<float>(c);
}

// The FP64 preconditioner keeps the stored stencils: in FP64 the element
// arithmetic (~100 operations per element) runs at GB300's FP64 rate, 58x
// below FP32, and costs more than the 27 stored coefficients' traffic.
bool mf_field_on(const p4d_ctx* c, int f) {
  return c->mf_items && c->prm.precision != 0 && (f != 0 || c->mf_phis);
}

namespace {
template <typename T, int MODE>
p4d_status mf_launch(p4d_ctx* c, int fmask, int step) {
  MGLevel& L = c->lev[0];
  MfArgs<T> a;
  a.nnx = c->g.nnx; a.nny = c->g.nny; a.nnz = c->g.nnz;
  a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
  a.ntx = c->mf_ntx; a.nty = c->mf_nty;
  const T* g = (const T*)c->mf_geo;
  a.gx = g; a.gy = g + 3 * c->nx; a.gz = g + 3 * (c->nx + c->ny);
  a.label = c->label;
  a.items = c->mf_items;
  const T* coef = (const T*)c->mf_coef;
  const int64_t ne = c->nelem, nn = c->g.nn;
  const int hof[3] = {0, 2, 3};
  for (int f = 0; f < 3; ++f) {
    const int h = hof[f];
    MfField<T>& F = a.f[f];
    F.x = (const T*)L.x[h]; F.xo = (T*)L.x2[h]; F.b = (const T*)L.b[h]; F.dinv = (const T*)L.dinv[h];
    F.d = (T*)L.d[h]; F.r = (T*)L.r[h];
    F.svs = (const T*)c->mf_svs + f * nn;
    F.kc = coef + f * ne;
    F.mc = f == 2 ? coef + 3 * ne : nullptr;
  }
  a.ctab = sizeof(T) == sizeof(double) ? (const T*)c->cheb_dev : (const T*)c->cheb_dev32;
  a.step = step;
  a.fmask = fmask;
  int lo = -1, hi = -1;
  for (int f = 0; f < 3; ++f)
    if (fmask & (1 << f)) {
      if (lo < 0) lo = c->mf_off[f];
      hi = c->mf_off[f] + c->mf_cnt[f];
    }
  if (lo < 0 || hi <= lo) return P4D_OK;
  a.items = c->mf_items + lo;
  ::p4d::count_launch(), k_mf_level0<T, MODE><<<hi - lo, kMfThreads, c->mf_smem, c->stream>>>(a);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}
}  // namespace

p4d_status mf_level0(p4d_ctx* c, int fmask, int mode, int step) {
  if (c->prm.precision == 0)
    return mode == 0 ? mf_launch<double, 0>(c, fmask, step) : mf_launch<double, 1>(c, fmask, step);
  return mode == 0 ? mf_launch<float, 0>(c, fmask, step) : mf_launch<float, 1>(c, fmask, step);
}

}  // namespace p4d
