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
// Layout of a launch: each block owns a tile of W x H nodes (15 x 15; the
// last tile of an axis takes the remainder, 1 to 15 nodes) and marches in z
// over a chunk of node planes.  Per plane it stages the (W+2) x (H+2) tile
// of x, the element coefficients and the node data in shared memory
// (asynchronous copies one plane ahead), evaluates the (W+1) x (H+1)
// elements between that plane and the next (their lower-corner outputs go
// to this plane, the upper-corner outputs are kept in registers for the
// next), and updates its nodes.  The phi_s work list covers only
// the node planes that hold phi_s unknowns.
#include <algorithm>
#include <type_traits>
#include <vector>
#include "p4d_common.cuh"

namespace p4d {
namespace {

// Node tile: at most 15 x 15 nodes, which have at most (15 + 1)^2 = 256
// elements: one element and one node of a plane per thread, so that no
// warp evaluates a second element before the per-plane barrier.  The last
// tile of an axis takes the remainder (1 to 15 nodes).
constexpr int kTX = 15, kTY = 15;
constexpr int kMfThreads = 256;
// planes of asynchronous copies in flight ahead of their use: one keeps the
// rings small (35 KB of shared memory per block) for five blocks per SM,
// which measured faster than deeper rings at fewer blocks per SM
constexpr int kMfDepth = 1;
static_assert((kTX + 2) * (kTY + 2) <= 2 * kMfThreads, "two x entries per thread at most");
static_assert((kTX + 1) * (kTY + 1) <= kMfThreads, "one element per thread");
constexpr int kDefaultZChunk = 8;      // node planes per block when p4d_params.mf_zchunk = 0

template <typename T>
struct MfField {
  const T* x;      // level-0 iterate (guarded vector)
  T* xo;           // Chebyshev output x + d
  const T* b;
  T* d;
  T* r;            // residual output
  const float2* sd;   // [nn] (sc_f * variable node diagonal, 1/diag)
  const float2* kcm;  // [nelem] (sc_f * stiffness coefficient, sc_f * mass coefficient / dt or 0)
  bool mass;          // the field has a mass term
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

// 4-byte asynchronous copy global -> shared (zero-filled when !valid; the
// source is then not read).
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The same operator with packed FP32x2 arithmetic (float): the pair m =
// b + 2c holds the local nodes (a = 0, 1) of one (y, z) position, so the y
// and z butterfly stages, the eigenvalues and the scaling are lane-wise
// pair operations and only the x stage is scalar.  Every lane rounds as the
// scalar operation; a - b is formed as fma(b, -1, a), exact like a
// subtraction.  P[m], Q[m]: the (y, z) factors of pair m (Q[0] = 0).
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void f2_butterfly(float2& a, float2& b) {
  const float2 t = a;
  a = __fadd2_rn(t, b);
  b = f2_sub(t, b);
}
__device__ __forceinline__ void element_apply_x2(float (&v)[8], float As, float Ad, float Bs, float Bd,
                                                 const float (&P)[4], const float (&Q)[4]) {
  float2 w[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float p = v[2 * m], q = v[2 * m + 1];
    w[m] = make_float2(p + q, p - q);
  }
  f2_butterfly(w[0], w[1]);
  f2_butterfly(w[2], w[3]);
  f2_butterfly(w[0], w[2]);
  f2_butterfly(w[1], w[3]);
  const float2 A2 = make_float2(As, Ad), B2 = make_float2(Bs, Bd);
  w[0] = __fmul2_rn(w[0], __fmul2_rn(A2, make_float2(P[0], P[0])));
#pragma unroll
  for (int m = 1; m < 4; ++m)
    w[m] = __fmul2_rn(w[m], __ffma2_rn(B2, make_float2(Q[m], Q[m]), __fmul2_rn(A2, make_float2(P[m], P[m]))));
  f2_butterfly(w[0], w[2]);
  f2_butterfly(w[1], w[3]);
  f2_butterfly(w[0], w[1]);
  f2_butterfly(w[2], w[3]);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[2 * m] = w[m].x + w[m].y;
    v[2 * m + 1] = w[m].x - w[m].y;
  }
}

// MODE 0: Chebyshev step on a nonzero x: d = c0 D^-1 (b - A x) (step 0) or
// d = ca d + cb D^-1 (b - A x), then x_out = x + d.  MODE 1: r = b - A x.
//
// Every thread owns at most two x entries, one element and one node of a
// plane (x entry slot r: index tid + 256 r).  The global data of the march
// (x planes, the element coefficients, the node data b, diag, 1/diag, d)
// reach shared memory by asynchronous copies kMfDepth planes ahead of their
// use, in rings counted from the first step ks = k0 - 2 of the march (plane
// j in slot (j - ks) mod the ring size): the loads in flight hold no
// registers, and the x tile is not copied through registers into shared
// memory.  Each thread evaluates the same element column in every plane, so
// it keeps the upper-corner outputs of element plane ke - 1 in registers and
// adds them to the lower-corner outputs of element plane ke: the sums S
// (per corner, lower + upper) are what node plane ke gathers.
template <typename T, int MODE>
__global__ void __launch_bounds__(kMfThreads, 5) k_mf_level0(MfArgs<T> a) {
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
  const int XN = XW * XH, EN = EW * EH, NN = W * H;
  // shared memory, laid out with the largest tile's strides (compile-time
  // constants): rings of x planes [RX][XP] (rows of XS), element
  // coefficient pairs [RC][EP][2] (rows of ES), node data [RN][NP + 2 NP +
  // NP] (b, the (variable diagonal, 1/diag) pairs, d; rows of NW), then the
  // element planes' corner sums [2][4][EP]
  constexpr int XS = kTX + 3, XP = XS * (kTY + 3), ES = kTX + 2, EP = ES * (kTY + 2);
  constexpr int NW = kTX + 1, NP = NW * (kTY + 1);
  constexpr unsigned DP = kMfDepth, RX = DP + 4, RC = DP + 2, RN = DP + 2;
  T* xs = reinterpret_cast<T*>(smem_raw);
  T* cs = xs + RX * XP;
  T* ns = cs + RC * 2 * EP;
  T* Sb = ns + RN * 4 * NP;
  // the block's field pointers, selected once (not per access)
  const T* __restrict__ Fx = fsel(a, f).x;
  T* __restrict__ Fxo = fsel(a, f).xo;
  const T* __restrict__ Fb = fsel(a, f).b;
  T* __restrict__ Fd = fsel(a, f).d;
  T* __restrict__ Fr = fsel(a, f).r;
  const float2* __restrict__ Fsd = fsel(a, f).sd;
  const float2* __restrict__ Fkcm = fsel(a, f).kcm;
  const int tid = threadIdx.x;
  // 32-bit offsets: every level-0 array has fewer than 2^31 entries
  const int sxy = a.nnx * a.nny;
  const int sexy = a.nx * a.ny;

  // warp-uniform: does any lane of this warp own a second x entry (most
  // warps do not; they skip the second slot's code)
  const bool wx2 = (tid & ~31) + kMfThreads < XN;
  // per-thread constants, computed once for the whole z march
  int xoff[2], xsm[2];   // x entry: in-plane offset (-1 outside the grid), tile index (-1: none)
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int q = tid + r * kMfThreads;
    xoff[r] = -1;
    xsm[r] = -1;
    if (q < XN) {
      const int jj = q / XW, ii = q - jj * XW;
      xsm[r] = ii + XS * jj;
      const int gi = i0 - 1 + ii, gj = j0 - 1 + jj;
      if (gi >= 0 && gi < a.nnx && gj >= 0 && gj < a.nny) xoff[r] = gi + a.nnx * gj;
    }
  }
  // element: in-plane offset (-1 outside the grid), x-tile index of its
  // lower-left node, element tile index (-1: none), x factors (2/h, h/2,
  // h/6)/8 and y factors (2/h, h/2, h/6)
  int eoff = -1, ebase = 0, eq = -1;
  T ex[3] = {0, 0, 0}, ey[3] = {0, 0, 0};
  if (tid < EN) {
    const int ej = tid / EW, ei = tid - ej * EW;
    eq = ei + ES * ej;
    ebase = ei + XS * ej;
    const int gi = i0 - 1 + ei, gj = j0 - 1 + ej;
    if (gi >= 0 && gi < a.nx && gj >= 0 && gj < a.ny) {
      eoff = gi + a.nx * gj;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        ex[t] = a.gx[t * a.nx + gi];
        ey[t] = a.gy[t * a.ny + gj];
      }
    }
  }
  // node: in-plane offset (-1: none), element tile index of the element it
  // is the upper corner of, x-tile index, node-data tile index
  int noff = -1, nq = 0, nsm = 0, nid = 0;
  if (tid < NN) {
    const int jj = tid / W, ii = tid - jj * W;
    noff = (i0 + ii) + a.nnx * (j0 + jj);
    nq = ii + ES * jj;
    nsm = (ii + 1) + XS * (jj + 1);
    nid = ii + NW * jj;
  }
  // Chebyshev coefficients of the block's hierarchies (phi_s: both electrodes)
  T cA[2], cB[2];
  {
    const int hs0 = f == 0 ? 0 : f + 1, hs1 = f == 0 ? 1 : f + 1;
    if (MODE == 0) {
      cA[0] = a.step == 0 ? (T)0 : cheb_coef(a.ctab, a.step, 1, hs0);
      cB[0] = a.step == 0 ? cheb_coef(a.ctab, 0, 0, hs0) : cheb_coef(a.ctab, a.step, 2, hs0);
      cA[1] = a.step == 0 ? (T)0 : cheb_coef(a.ctab, a.step, 1, hs1);
      cB[1] = a.step == 0 ? cheb_coef(a.ctab, 0, 0, hs1) : cheb_coef(a.ctab, a.step, 2, hs1);
    }
  }

  const int ks = k0 - 2;   // first step of the march (element plane k0 - 1)
  // The march evaluates element planes k0 - 1 .. k1 - 1 (node planes k0 ..
  // k1 - 1 need no other), so it reads x planes k0 - 1 .. k1 and the
  // coefficients of element planes k0 - 1 .. k1 - 1.
  // asynchronous copies of x plane j (planes outside the grid: zeros)
  auto issue_x = [&](int j) {
    if (j > k1) return;
    T* dst = xs + ((unsigned)(j - ks) % RX) * XP;
    const bool kin = j >= 0 && j < a.nnz;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (r == 1 && !wx2) break;
      if (xsm[r] < 0) continue;
      const bool on = kin && xoff[r] >= 0;
      cp_async4(dst + xsm[r], on ? Fx + (xoff[r] + j * sxy) : Fx, on);
    }
  };
  // element coefficients of element plane ke (outside the grid: zeros)
  auto issue_coef = [&](int ke) {
    if (ke >= k1 || eq < 0) return;
    T* dst = cs + ((unsigned)(ke - ks) % RC) * 2 * EP;
    const bool on = ke >= 0 && ke < a.nz && eoff >= 0;
    cp_async8(dst + 2 * eq, on ? Fkcm + (eoff + ke * sexy) : Fkcm, on);
  };
  // node data of node plane k (only the march's planes [k0, k1))
  auto issue_nodes = [&](int k) {
    if (k < k0 || k >= k1 || noff < 0) return;
    T* dst = ns + ((unsigned)(k - ks) % RN) * 4 * NP;
    const int n = noff + k * sxy;
    cp_async4(dst + nid, Fb + n, true);
    cp_async8(dst + NP + 2 * nid, Fsd + n, true);
    if (MODE == 0) cp_async4(dst + 3 * NP + nid, a.step != 0 ? Fd + n : Fd, a.step != 0);
  };
  int lr = 0;   // label of the next node plane (phi_s), in a register
  auto fetch_labels = [&](int k) {
    if (f != 0) return;
    lr = (k < k1 && noff >= 0) ? (int)a.label[noff + k * sxy] : 0;
  };

  // element plane ke between x planes ke and ke + 1: corner sums (lower
  // corners of ke + upper corners of ke - 1) to S[(ke - ks) & 1]; the upper
  // corners of ke stay in up[] for element plane ke + 1
  T up[4] = {0, 0, 0, 0};
  auto element_plane = [&](int ke) {
    if (eq < 0) return;
    const unsigned rx = (unsigned)(ke - ks);
    const T* xl = xs + (rx % RX) * XP;
    const T* xu = xs + ((rx + 1) % RX) * XP;
    const T* cf = cs + (rx % RC) * 2 * EP;
    T* so = Sb + (rx & 1) * 4 * EP;
    T Ksz = 0, Msz = 0, Mdz = 0;
    if (ke >= 0 && ke < a.nz) {
      Ksz = a.gz[ke];
      Msz = a.gz[a.nz + ke];
      Mdz = a.gz[2 * a.nz + ke];
    }
    const float2 km = *reinterpret_cast<const float2*>(cf + 2 * eq);   // (kc, mc); mc = 0 without mass
    const T kc = km.x, mc = km.y;
    T v[8];
    v[0] = xl[ebase];
    v[1] = xl[ebase + 1];
    v[2] = xl[ebase + XS];
    v[3] = xl[ebase + XS + 1];
    v[4] = xu[ebase];
    v[5] = xu[ebase + 1];
    v[6] = xu[ebase + XS];
    v[7] = xu[ebase + XS + 1];
    // eigenvalues (the x factors carry the 1/8); per (y, z) component
    // b + 2c: P = My Mz, Q = Ky Mz + My Kz
    const T Kdx = ex[0], Msx = ex[1], Mdx = ex[2];
    const T Kdy = ey[0], Msy = ey[1], Mdy = ey[2];
    const T P0 = Msy * Msz, P1 = Mdy * Msz, P2 = Msy * Mdz, P3 = Mdy * Mdz;
    const T Q1 = Kdy * Msz, Q2 = Msy * Ksz, Q3 = Kdy * Mdz + Mdy * Ksz;
    const T As = Msx * mc, Bs = Msx * kc;            // lambda(s, .) = As P + Bs Q
    const T Ad = kc * Kdx + mc * Mdx, Bd = kc * Mdx; // lambda(d, .) = Ad P + Bd Q
    if constexpr (std::is_same<T, float>::value) {
      const float Pm[4] = {P0, P1, P2, P3}, Qm[4] = {0.f, Q1, Q2, Q3};
      element_apply_x2(v, As, Ad, Bs, Bd, Pm, Qm);
    } else {
      T lam[8];
      lam[0] = As * P0;
      lam[1] = Ad * P0;
      lam[2] = As * P1 + Bs * Q1;
      lam[3] = Ad * P1 + Bd * Q1;
      lam[4] = As * P2 + Bs * Q2;
      lam[5] = Ad * P2 + Bd * Q2;
      lam[6] = As * P3 + Bs * Q3;
      lam[7] = Ad * P3 + Bd * Q3;
      element_apply<T>(v, lam);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      so[l * EP + eq] = v[l] + up[l];
      up[l] = v[4 + l];
    }
  };

  // Step k of the march (k = ks .. k1 - 1): issue the copies of x plane
  // k + 2 + DP, coefficients k + 1 + DP and node data k + DP; wait for the
  // copies issued DP steps earlier; one barrier; evaluate element plane
  // k + 1 (x planes k + 1, k + 2; none at the last step) and, for k >= k0,
  // update node plane k from the corner sums of element plane k.  Between
  // two barriers the slots written (x plane k + 1 + DP + 2 of a thread
  // already in the next step: the slot of plane k - 1; S of element plane
  // k + 1; the coefficient and node slots of planes k and k - 1) and the
  // slots read (x planes k .. k + 2, coefficients k + 1, node data k, S of
  // element plane k) differ.
  issue_x(ks + 1);
#pragma unroll
  for (int g = 0; g < (int)DP; ++g) {
    const int k = ks - (int)DP + g;
    issue_x(k + 2 + DP);
    issue_coef(k + 1 + DP);
    issue_nodes(k + DP);
    cp_async_commit();
  }
  fetch_labels(k0);
  for (int k = ks; k < k1; ++k) {
    issue_x(k + 2 + DP);
    issue_coef(k + 1 + DP);
    issue_nodes(k + DP);
    cp_async_commit();
    cp_async_wait<DP>();
    __syncthreads();
    if (k + 1 < k1) element_plane(k + 1);   // zero outputs when k + 1 is outside the element planes
    if (k < k0) continue;
    if (noff >= 0) {
      int hsel = 0;
      bool act = true;
      if (f == 0) {
        act = lr & kLabActive;
        hsel = (lr & kLabAnode) ? 0 : 1;
      }
      if (act) {
        const unsigned rk = (unsigned)(k - ks);
        const T* xk = xs + (rk % RX) * XP;
        const T* nd = ns + (rk % RN) * 4 * NP;
        const T* S = Sb + (rk & 1) * 4 * EP;
        const T xn = xk[nsm];
        const float2 sdv = *reinterpret_cast<const float2*>(nd + NP + 2 * nid);   // (variable diagonal, 1/diag)
        T ax = sdv.x * xn;
        ax += S[3 * EP + nq] + S[2 * EP + nq + 1];
        ax += S[1 * EP + nq + ES] + S[nq + ES + 1];
        const T res = nd[nid] - ax;
        const int n = noff + k * sxy;
        if (MODE == 1) {
          Fr[n] = res;
        } else {
          const T dn = (hsel ? cA[1] : cA[0]) * nd[3 * NP + nid] + (hsel ? cB[1] : cB[0]) * (sdv.y * res);
          Fd[n] = dn;
          Fxo[n] = xn + dn;
        }
      }
    }
    fetch_labels(k + 1);
  }
  cp_async_wait<0>();   // no copy into this block's shared memory outlives it
}

// Shared memory of k_mf_level0 (FP32): the x, coefficient and node-data
// rings and the element planes' corner sums.
constexpr size_t mf_smem_bytes() {
  return sizeof(float) * ((size_t)(kMfDepth + 4) * (kTX + 3) * (kTY + 3) +
                          (size_t)(kMfDepth + 2) * 2 * (kTX + 2) * (kTY + 2) +
                          (size_t)(kMfDepth + 2) * 4 * (kTX + 1) * (kTY + 1) + (size_t)8 * (kTX + 2) * (kTY + 2));
}

// Per field and element the (stiffness, mass) coefficient pair; only c_e
// has a mass term.
__global__ void k_mf_coef(int64_t nelem, const uint8_t* __restrict__ region, const double* __restrict__ eps,
                          const double* __restrict__ eps_s, const double* __restrict__ sig_e, double brug,
                          double kappa, double De, double dt, double s0, double s1, double s2,
                          float2* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nelem) return;
  const uint8_t r = region[e];
  const double sig = (r == 0 || r == 2) ? pow(eps_s[e], brug) * sig_e[e] : 0.0;
  const double epb = pow(eps[e], brug);
  out[e] = make_float2((float)(s0 * sig), 0.f);
  out[nelem + e] = make_float2((float)(s1 * epb * kappa), 0.f);
  out[2 * nelem + e] = make_float2((float)(s2 * epb * De), (float)(s2 * eps[e] / dt));
}

template <typename T>
p4d_status mf_setup_t(p4d_ctx* c) {
  const int nx = c->nx, ny = c->ny, nz = c->nz;
  const int64_t nelem = c->nelem;
  float2* coef = nullptr;
  P4D_TRYS(dalloc_t(c, &coef, (size_t)3 * nelem));
  ::p4d::count_launch(), k_mf_coef<<<nblocks(nelem), kBlock, 0, c->stream>>>(
      nelem, c->region, c->eps_e, c->epss_e, c->sig_e, c->prm.brug, c->kappa_fix, c->De_fix, c->prm.dt,
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
  float2* svs = nullptr;   // (variable diagonal, 1/diag) pairs, written per linearization
  P4D_TRYS(dalloc_t(c, &svs, (size_t)3 * c->g.nn));
  P4D_TRY(cudaMemset(svs, 0, sizeof(float2) * 3 * c->g.nn));
  c->mf_svs = svs;
  return P4D_OK;
}

}  // namespace

// Work list, coefficients and factors of the matrix-free level 0.  phi_s is
// matrix-free only without collector shells (their face stiffness lives in
// the stored stencils).
p4d_status mf_setup(p4d_ctx* c) {
  // The FP64 preconditioner keeps the stored stencils: in FP64 the element
  // arithmetic (~100 operations per element) runs at GB300's FP64 rate, 58x
  // below FP32, and costs more than the 27 stored coefficients' traffic.
  if (c->prm.precision == 0) return P4D_OK;
  const int nnx = c->g.nnx, nny = c->g.nny, nnz = c->g.nnz;
  c->mf_phis = !(c->shell_p > 0.0) && !(c->shell_n > 0.0);
  // tiles of kTX x kTY nodes; the last of an axis takes the remainder (1 to
  // kTX nodes)
  c->mf_ntx = (nnx + kTX - 1) / kTX;
  c->mf_nty = (nny + kTY - 1) / kTY;
  const int mw = nnx - (c->mf_ntx - 1) * kTX, mh = nny - (c->mf_nty - 1) * kTY;
  const int zc = c->prm.mf_zchunk > 0 ? c->prm.mf_zchunk : kDefaultZChunk;
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
  // the kernel lays shared memory out with the largest tile's strides
  c->mf_smem = mf_smem_bytes();
  if (mw > kTX || mh > kTY || mw < 1 || mh < 1) return P4D_ERR_INVALID_ARG;   // cannot happen
  // The kernels' shared-memory limit is a process-wide attribute shared by
  // every handle: set it to the kernel's fixed layout (the largest tile's),
  // never to a size of this handle's, which could fail the launches of
  // handles set up before.
  const size_t smax = mf_smem_bytes();
  P4D_TRY(cudaFuncSetAttribute(k_mf_level0<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  P4D_TRY(cudaFuncSetAttribute(k_mf_level0<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  return mf_setup_t<float>(c);
}

bool mf_field_on(const p4d_ctx* c, int f) { return c->mf_items && (f != 0 || c->mf_phis); }

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
  const float2* coef = (const float2*)c->mf_coef;
  const int64_t ne = c->nelem, nn = c->g.nn;
  const int hof[3] = {0, 2, 3};
  for (int f = 0; f < 3; ++f) {
    const int h = hof[f];
    MfField<T>& F = a.f[f];
    F.x = (const T*)L.x[h]; F.xo = (T*)L.x2[h]; F.b = (const T*)L.b[h];
    F.d = (T*)L.d[h]; F.r = (T*)L.r[h];
    F.sd = (const float2*)c->mf_svs + f * nn;
    F.kcm = coef + f * ne;
    F.mass = f == 2;
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
  if (!c->mf_items) return P4D_ERR_INVALID_ARG;   // FP64 preconditioner: stored stencils only
  return mode == 0 ? mf_launch<float, 0>(c, fmask, step) : mf_launch<float, 1>(c, fmask, step);
}

}  // namespace p4d
