// Geometric multigrid on the Schur-reduced electrode blocks (paper section 4:
// one V-cycle approximates each electrode-level block inverse; the paper uses
// BoomerAMG, here the structured hex grid gives the hierarchy directly).
//
// Hierarchies h: 0 phi_s anode, 1 phi_s cathode, 2 phi_e, 3 c_e.  The two
// electrodes' phi_s never couple, and the thin separator leaves no coarse
// grid that could represent both electrodes' near-constant modes, so phi_s
// gets one masked hierarchy per electrode (they share the level-0 arrays).
//
// Per level: trilinear prolongation P (rows of masked-out fine nodes zero),
// Galerkin operators A_{l+1} = P^T A_l P split into a fixed part (built once
// at setup from the fixed stencils) and a linearization-dependent part
// (Schur/reaction row sums, rebuilt per Newton step), Chebyshev smoothing on
// D^-1 A over [lam/ratio, lam] (lam: Gershgorin bound), and an explicit FP64
// inverse on the coarsest level.  Stencils are in difference form (slot 13
// = row sum), see p4d_common.cuh.
#include <algorithm>
#include <type_traits>
#include <vector>
#include <cmath>
#include "p4d_common.cuh"

namespace p4d {
namespace {

template <typename T> __device__ __forceinline__ T fromd(double v);
template <> __device__ __forceinline__ double fromd<double>(double v) { return v; }
template <> __device__ __forceinline__ float fromd<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 fromd<__nv_bfloat16>(double v) {
  return __float2bfloat16((float)v);
}
// stencil entry -> compute precision (identity for float/double, widen bf16)
template <typename T> __device__ __forceinline__ T tof(T v) { return v; }
__device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }


struct LevelDims {
  int nnx, nny, nnz;
  int64_t n;
};

struct HList {
  int h[kNH];
};

__device__ __forceinline__ void node_ijk(const LevelDims& d, int64_t n, int& i, int& j, int& k) {
  i = (int)(n % d.nnx);
  j = (int)((n / d.nnx) % d.nny);
  k = (int)(n / ((int64_t)d.nnx * d.nny));
}

// One-dimensional linear interpolation between a fine node line (ne
// elements) and its coarsening: coarse nodes sit on the even fine nodes and,
// when ne is odd, also on the last fine node (that coarse element spans one
// fine element), so every element count >= 2 can be coarsened.  Per fine
// node: up to two parents; per coarse node: up to three support nodes.
// (struct Axis / Xfer: p4d_common.cuh)

// ---------------------------------------------------------------- masks
__global__ void k_mask0(int64_t nn, const uint8_t* __restrict__ label, uint8_t* m0, uint8_t* m1, uint8_t* m2,
                        uint8_t* m3) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const uint8_t l = label[n];
  const bool act = l & kLabActive;
  m0[n] = act && (l & kLabAnode);
  m1[n] = act && (l & kLabCathode);
  m2[n] = 1;
  m3[n] = 1;
}

// First and last node of each hierarchy's mask: ext[2 h] = min, ext[2 h + 1]
// = max (initialised to n and -1).
__global__ void k_mask_extent(int64_t n, Ptr4<const uint8_t> m, int* __restrict__ ext) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  if (i >= n || !pk(m.p, h)[i]) return;
  atomicMin(ext + 2 * h, (int)i);
  atomicMax(ext + 2 * h + 1, (int)i);
}

__global__ void k_mask_coarse(LevelDims fd, LevelDims cd, Xfer X, Ptr4<const uint8_t> fm, Ptr4<uint8_t> cm) {
  const int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  if (C >= cd.n) return;
  int I, J, K;
  node_ijk(cd, C, I, J, K);
  uint8_t any = 0;
  for (int tz = 0; tz < 3; ++tz) {
    const int fk = X.a[2].sup[K * 3 + tz];
    if (fk < 0) continue;
    for (int ty = 0; ty < 3; ++ty) {
      const int fj = X.a[1].sup[J * 3 + ty];
      if (fj < 0) continue;
      for (int tx = 0; tx < 3; ++tx) {
        const int fi = X.a[0].sup[I * 3 + tx];
        if (fi < 0) continue;
        any |= pk(fm.p, h)[fi + (int64_t)fd.nnx * (fj + (int64_t)fd.nny * fk)];
      }
    }
  }
  pk(cm.p, h)[C] = any ? 1 : 0;
}

// ---------------------------------------------------------------- Galerkin
// Source operator in difference form: off-diagonals O[o][n] (o != 13) and
// row sums s[n] (slot 13, or a separate array at level 0).
struct SrcOp {
  const double* st;      // [27][n] (slot 13 ignored when rs != nullptr)
  const double* rs;      // optional separate row sums [n]
};

// A_c = P^T diag(m) A diag(m) P for one hierarchy; writes difference form.
// identity_out: coarse nodes without support get an identity row (fixed part)
// or a zero row (variable part).  TV: the precision of input, accumulation
// and output (FP64 for the fixed part and the FP64 preconditioner).
//
// One warp per coarse node, lane t < 27 owning fine support node t: each
// lane scatters its row's products into its own column of 27 accumulators
// in shared memory, then lane o sums slot o over the 27 columns in a fixed
// order (deterministic, no atomics).
constexpr int kRapWarps = 4;     // coarse nodes per block
constexpr int kRapLd = 28;       // accumulator column stride (27 lanes, padded)

// acc[stride * oo] += a * w(g -> D) over the (up to 8) coarse parents D of
// fine node (gi, gj, gk), oo the slot of D in the coarse row of (I, J, K).
template <typename TV>
__device__ __forceinline__ void rap_scatter(const Xfer& X, int gi, int gj, int gk, int I, int J, int K, TV a,
                                            TV* acc, int stride) {
  const TV* pwx = parw_t<TV>(X.a[0]);
  const TV* pwy = parw_t<TV>(X.a[1]);
  const TV* pwz = parw_t<TV>(X.a[2]);
  int oyz[4];
  TV wyz[4];
  int nyz = 0;
  for (int c3 = 0; c3 < 2; ++c3) {
    const int pz = X.a[2].par[gk * 2 + c3];
    if (pz < 0) continue;
    for (int c2 = 0; c2 < 2; ++c2) {
      const int py = X.a[1].par[gj * 2 + c2];
      if (py < 0) continue;
      oyz[nyz] = 3 * (py - J + 1) + 9 * (pz - K + 1);
      wyz[nyz] = pwy[gj * 2 + c2] * pwz[gk * 2 + c3];
      ++nyz;
    }
  }
  for (int c1 = 0; c1 < 2; ++c1) {
    const int px = X.a[0].par[gi * 2 + c1];
    if (px < 0) continue;
    const TV t = a * pwx[gi * 2 + c1];
    for (int q = 0; q < nyz; ++q) acc[(oyz[q] + px - I + 1) * stride] += t * wyz[q];
  }
}

// Fine support node of lane t (t < 27) of coarse node (I, J, K): index f and
// weight, or false when absent or masked out.
template <typename TV>
__device__ __forceinline__ bool rap_support(const LevelDims& fd, const Xfer& X, const uint8_t* m, int I, int J, int K,
                                            int t, int& fi, int& fj, int& fk, int64_t& f, TV& wf) {
  const int tx = t % 3, ty = (t / 3) % 3, tz = t / 9;
  fi = X.a[0].sup[I * 3 + tx];
  fj = X.a[1].sup[J * 3 + ty];
  fk = X.a[2].sup[K * 3 + tz];
  if (fi < 0 || fj < 0 || fk < 0) return false;
  f = fi + (int64_t)fd.nnx * (fj + (int64_t)fd.nny * fk);
  if (!m[f]) return false;
  wf = supw_t<TV>(X.a[0])[I * 3 + tx] * (supw_t<TV>(X.a[1])[J * 3 + ty] * supw_t<TV>(X.a[2])[K * 3 + tz]);
  return true;
}

// Slot totals of one warp's accumulator block and the row sum: lane o < 27
// writes slot o of coarse node C.
template <typename TV>
__device__ __forceinline__ void rap_finish(const TV* my, TV rs_lane, bool cin, int identity_out, int lane,
                                           TV* o_, int64_t cn, int64_t C) {
  TV rsum = rs_lane;
  for (int o = 16; o > 0; o >>= 1) rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
  if (lane >= 27) return;
  TV v;
  if (!cin) {
    v = (lane == 13 && identity_out) ? (TV)1 : (TV)0;
  } else if (lane == 13) {
    v = rsum;
  } else {
    v = 0;
    for (int l = 0; l < 27; ++l) v += my[lane * kRapLd + l];
  }
  o_[lane * cn + C] = v;
}

template <typename TV>
__global__ void __launch_bounds__(32 * kRapWarps) k_rap(LevelDims fd, LevelDims cd, Xfer X, Ptr4<const TV> fst,
                                                        Ptr4<const TV> frs, Ptr4<const uint8_t> fm,
                                                        Ptr4<const uint8_t> cm, Ptr4<TV> out, int identity_out) {
  __shared__ TV part[kRapWarps][27 * kRapLd];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t C = (int64_t)blockIdx.x * kRapWarps + warp;
  const int h = blockIdx.y;
  if (C >= cd.n) return;   // per warp
  TV* my = part[warp];
  if (lane < 27)
    for (int o = 0; o < 27; ++o) my[o * kRapLd + lane] = (TV)0;
  int I, J, K;
  node_ijk(cd, C, I, J, K);
  const bool cin = pk(cm.p, h)[C];
  const TV* st = pk(fst.p, h);
  const TV* rs = pk(frs.p, h);
  const int64_t fn = fd.n;
  TV rs_l = 0;
  int fi, fj, fk;
  int64_t f;
  TV wf;
  if (cin && lane < 27 && rap_support<TV>(fd, X, pk(fm.p, h), I, J, K, lane, fi, fj, fk, f, wf)) {
    const uint8_t* m = pk(fm.p, h);
    const TV sf = rs ? rs[f] : st[13 * fn + f];
    rs_l = wf * sf;
    // full-form diagonal of row f
    TV diag = sf;
    for (int o = 0; o < 27; ++o)
      if (o != 13) diag -= st[o * fn + f];
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int gi = fi + dx, gj = fj + dy, gk = fk + dz;
      if (gi < 0 || gj < 0 || gk < 0 || gi >= fd.nnx || gj >= fd.nny || gk >= fd.nnz) continue;
      const int64_t gidx = gi + (int64_t)fd.nnx * (gj + (int64_t)fd.nny * gk);
      if (!m[gidx]) continue;
      const TV a = (o == 13 ? diag : st[o * fn + f]) * wf;
      if (a == (TV)0) continue;
      rap_scatter<TV>(X, gi, gj, gk, I, J, K, a, my + lane, kRapLd);
    }
  }
  __syncwarp();
  rap_finish<TV>(my, rs_l, cin, identity_out, lane, pk(out.p, h), cd.n, C);
}

// V_1 = P^T diag(m s) P by gathering: with a diagonal operator and a
// tensor-product P, entry (C, C + o) is sum_f w_C(f) m_f s_f w_{C+o}(f) over
// the fine nodes f in both supports, and it factors by axis.  One thread per
// coarse node: the m s values of its (at most 3 x 3 x 3) support nodes, the
// per-axis weight products q_a[d][t] = w_C(t) w_{C+d-1}(t) of support entry t,
// then three passes (x, y, z) give all 27 slots.  Slot 13 holds the row sum
// sum_f w_C(f) m_f s_f (a fine node's interpolation weights sum to one).
template <typename TV>
__global__ void __launch_bounds__(128) k_rap_diag_g(LevelDims fd, LevelDims cd, Xfer X, Ptr4<const double> s,
                                                    Ptr4<const uint8_t> fm, Ptr4<const uint8_t> cm,
                                                    Ptr4<TV> out) {
  const int C = blockIdx.x * blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  if (C >= (int)cd.n) return;
  TV* o_ = pk(out.p, h);
  const int64_t cn = cd.n;
  if (!pk(cm.p, h)[C]) {
#pragma unroll
    for (int o = 0; o < 27; ++o) o_[o * cn + C] = (TV)0;
    return;
  }
  int I, J, K;
  node_ijk(cd, (int64_t)C, I, J, K);
  const int Ic[3] = {I, J, K};
  const int ncd[3] = {cd.nnx, cd.nny, cd.nnz};
  int f[3][3];      // support fine index per axis and entry (-1: none)
  TV w[3][3];       // its weight w_C
  TV q[3][3][3];    // [axis][offset d][entry t]: w_C(t) w_{C+d-1}(t)
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int* sup = X.a[a].sup;
    const TV* sw = supw_t<TV>(X.a[a]);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      f[a][t] = sup[Ic[a] * 3 + t];
      w[a][t] = f[a][t] >= 0 ? sw[Ic[a] * 3 + t] : (TV)0;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int I2 = Ic[a] + d - 1;
      const bool in = I2 >= 0 && I2 < ncd[a];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        TV wv = (TV)0;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          const int g = in ? sup[I2 * 3 + u] : -1;
          if (f[a][t] >= 0 && g == f[a][t]) wv = sw[I2 * 3 + u];
        }
        q[a][d][t] = w[a][t] * wv;
      }
    }
  }
  // m s of the support nodes
  const double* sv = pk(s.p, h);
  const uint8_t* m = pk(fm.p, h);
  TV S[3][3][3];   // [tz][ty][tx]
#pragma unroll
  for (int tz = 0; tz < 3; ++tz)
#pragma unroll
    for (int ty = 0; ty < 3; ++ty)
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) {
        TV v = (TV)0;
        if (f[0][tx] >= 0 && f[1][ty] >= 0 && f[2][tz] >= 0) {
          const int64_t fi = f[0][tx] + (int64_t)fd.nnx * (f[1][ty] + (int64_t)fd.nny * f[2][tz]);
          if (m[fi]) v = (TV)sv[fi];
        }
        S[tz][ty][tx] = v;
      }
  // row sum
  TV rs = (TV)0;
#pragma unroll
  for (int tz = 0; tz < 3; ++tz)
#pragma unroll
    for (int ty = 0; ty < 3; ++ty)
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) rs += w[2][tz] * (w[1][ty] * (w[0][tx] * S[tz][ty][tx]));
  // x pass: T1[dx][tz][ty]; y pass: T2[dx][dy][tz]; z pass: the slots
  TV T1[3][3][3];
#pragma unroll
  for (int dx = 0; dx < 3; ++dx)
#pragma unroll
    for (int tz = 0; tz < 3; ++tz)
#pragma unroll
      for (int ty = 0; ty < 3; ++ty) {
        TV acc = (TV)0;
#pragma unroll
        for (int tx = 0; tx < 3; ++tx) acc += q[0][dx][tx] * S[tz][ty][tx];
        T1[dx][tz][ty] = acc;
      }
  TV T2[3][3][3];
#pragma unroll
  for (int dx = 0; dx < 3; ++dx)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int tz = 0; tz < 3; ++tz) {
        TV acc = (TV)0;
#pragma unroll
        for (int ty = 0; ty < 3; ++ty) acc += q[1][dy][ty] * T1[dx][tz][ty];
        T2[dx][dy][tz] = acc;
      }
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int o = dx + 3 * dy + 9 * dz;
        TV v;
        if (o == 13) {
          v = rs;
        } else {
          TV acc = (TV)0;
#pragma unroll
          for (int tz = 0; tz < 3; ++tz) acc += q[2][dz][tz] * T2[dx][dy][tz];
          v = acc;
        }
        o_[o * cn + C] = v;
      }
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Block-wide maximum of a non-negative value, one atomic per block (all
// threads of the block must call it).
__device__ __forceinline__ void block_max_to(double* addr, double v) {
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (blockDim.x + 31) / 32 ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0 && v > 0.0) atomic_max_pos(addr, v);
  }
}

// Level 0: variable row sums, storage stencil slot 13, inverse diagonal, lam.
// The fixed off-diagonal sums come from setup; only node-local arithmetic
// remains (the reciprocal and the Gershgorin ratio in the compute precision).
template <typename TS, typename T>
__global__ void k_level0_update(Grid g, double tau, const double* __restrict__ sfix,
                                const double* __restrict__ offsum, const double* __restrict__ absoff,
                                const uint8_t* __restrict__ label, const int32_t* __restrict__ eidx,
                                const double* __restrict__ Aj, const double* __restrict__ ge,
                                const double* __restrict__ gc, const double* __restrict__ zeta, double s0,
                                double s1, double s2, TS* st0, TS* st1, TS* st2, T* di0, T* di1, T* di2,
                                double* __restrict__ svar, double* lam, float2* __restrict__ sd) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  double gl[kNH] = {0.0, 0.0, 0.0, 0.0};
  if (n < nn) {
    const int32_t e = eidx[n];
    const uint8_t l = label[n];
    const bool act = l & kLabActive;
    double sv[3] = {0.0, 0.0, 0.0};
    if (e >= 0) {
      const double zA = zeta[e] * Aj[e];
      if (act) sv[0] = zA * ge[e];
      sv[1] = zA * ge[e];
      sv[2] = -tau * zA * gc[e];
    }
    TS* sts[3] = {st0, st1, st2};
    T* dis[3] = {di0, di1, di2};
    const double sc[3] = {s0, s1, s2};
    for (int f = 0; f < 3; ++f) {
      const double s = sfix[f * nn + n] + sv[f];
      double diag = (f == 0 && !act) ? 1.0 : s - offsum[f * nn + n];
      const double ab = absoff[f * nn + n];
      if (!(diag > 0.0)) diag = fmax(ab, 1e-300);   // keep the smoother finite on a degenerate row
      svar[f * nn + n] = sv[f];
      sts[f][13 * nn + n] = fromd<TS>(sc[f] * s);
      const T dsc = (T)(sc[f] * diag);
      dis[f][n] = (T)1 / dsc;
      // the matrix-free level 0 adds the variable diagonal to the element part;
      // it reads it with 1/diag as one pair
      if (sd) sd[f * nn + n] = make_float2((float)(T)(sc[f] * sv[f]), (float)((T)1 / dsc));
      int h = f + 1;
      if (f == 0) {
        if (!act) continue;
        h = (l & kLabAnode) ? 0 : 1;
      }
      // Gershgorin ratio in FP64: the Chebyshev interval must not depend on
      // the preconditioner precision
      gl[h] = (ab + diag) / diag;
    }
  }
  for (int h = 0; h < kNH; ++h) block_max_to(lam + h, gl[h]);
}

// Level >= 1: A = F + V into storage precision, inverse diagonal and lam.
template <typename TS, typename T, typename TV>
__global__ void k_level_combine(LevelDims d, Ptr4<const double> F, Ptr4<const TV> V, Ptr4<TS> st,
                                Ptr4<T> dinv, Ptr4<const uint8_t> mask, double sc0, double sc1, double sc2,
                                double sc3, double* lam) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  double gl = 0.0;
  if (n < d.n) {
    const double sc = h == 0 ? sc0 : (h == 1 ? sc1 : (h == 2 ? sc2 : sc3));
    const double* f = pk(F.p, h);
    const TV* v = pk(V.p, h);
    if (std::is_same<T, float>::value) {
      // FP32 cycle: the sum of the fixed and variable parts, the scaling, the
      // diagonal and the Gershgorin sums in FP32 (the results are stored in
      // FP32 or BF16; the row sum in slot 13 adds its two parts directly)
      const float scf = (float)sc;
      float diag = 0.f, absoff = 0.f, s = 0.f;
#pragma unroll
      for (int o = 0; o < 27; ++o) {
        const float a = (float)f[o * d.n + n] + (float)v[o * d.n + n];
        pk(st.p, h)[o * d.n + n] = (TS)(scf * a);
        if (o == 13) s = a;
        else { diag -= a; absoff += fabsf(a); }
      }
      diag += s;
      if (!(diag > 0.f)) diag = fmaxf(absoff, 1e-30f);
      pk(dinv.p, h)[n] = (T)(1.0f / (scf * diag));
      if (pk(mask.p, h)[n]) gl = (double)((absoff + fabsf(diag)) / diag);
    } else {
      double diag = 0.0, absoff = 0.0, s = 0.0;
      for (int o = 0; o < 27; ++o) {
        const double a = f[o * d.n + n] + (double)v[o * d.n + n];
        pk(st.p, h)[o * d.n + n] = fromd<TS>(sc * a);
        if (o == 13) s = a;
        else { diag -= a; absoff += fabs(a); }
      }
      diag += s;
      if (!(diag > 0.0)) diag = fmax(absoff, 1e-300);
      pk(dinv.p, h)[n] = fromd<T>(1.0 / (sc * diag));
      if (pk(mask.p, h)[n]) gl = (absoff + fabs(diag)) / diag;
    }
  }
  block_max_to(lam + h, gl);
}

// Dense scaled coarsest operator [n][n] (row major) from difference form.
template <typename TV>
__global__ void k_dense(LevelDims d, Ptr4<const double> F, Ptr4<const TV> V, double sc0, double sc1,
                        double sc2, double sc3, double* out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  if (n >= d.n) return;
  const double sc = h == 0 ? sc0 : (h == 1 ? sc1 : (h == 2 ? sc2 : sc3));
  double* A = out + (size_t)h * d.n * d.n;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  for (int64_t m = 0; m < d.n; ++m) A[n * d.n + m] = 0.0;
  double diag = 0.0;
  for (int o = 0; o < 27; ++o) {
    const double a = pk(F.p, h)[o * d.n + n] + (double)pk(V.p, h)[o * d.n + n];
    if (o == 13) { diag += a; continue; }
    diag -= a;
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || jj < 0 || kk < 0 || ii >= d.nnx || jj >= d.nny || kk >= d.nnz) continue;
    A[n * d.n + (ii + (int64_t)d.nnx * (jj + (int64_t)d.nny * kk))] = sc * a;
  }
  A[n * d.n + n] = sc * diag;
}

// Single-level hierarchy: dense scaled level-0 operator of hierarchy h from
// the fixed stencil (off-diagonals), fixed + variable row sums and the mask
// (masked-out rows/columns become identity).
__global__ void k_dense0(Grid g, const double* __restrict__ Jst, const double* __restrict__ sfix,
                         const double* __restrict__ svar, Ptr4<const uint8_t> mask, double sc0, double sc1,
                         double sc2, double* out) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int h = blockIdx.y;
  const int64_t nn = g.nn;
  if (n >= nn) return;
  const int f = h == 0 || h == 1 ? 0 : h - 1;
  const double sc = f == 0 ? sc0 : (f == 1 ? sc1 : sc2);
  double* A = out + (size_t)h * nn * nn;
  for (int64_t m = 0; m < nn; ++m) A[n * nn + m] = 0.0;
  if (!pk(mask.p, h)[n]) {
    A[n * nn + n] = 1.0;
    return;
  }
  const int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny), k = (int)(n / ((int64_t)g.nnx * g.nny));
  const double* st = Jst + (size_t)f * 27 * nn;
  double diag = sfix[f * nn + n] + svar[f * nn + n];
  for (int o = 0; o < 27; ++o) {
    if (o == 13) continue;
    const double a = st[o * nn + n];
    diag -= a;
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nnx || jj >= g.nny || kk >= g.nnz) continue;
    const int64_t m = ii + (int64_t)g.nnx * (jj + (int64_t)g.nny * kk);
    if (pk(mask.p, h)[m]) A[n * nn + m] = sc * a;
  }
  A[n * nn + n] = sc * diag;
}

// In-place Gauss-Jordan inversion with partial pivoting, one block per matrix.
// Coarsest-level inverse, n <= kLuMax: LU with partial pivoting of each
// hierarchy's matrix in one block (row-major, in place in lu; perm[i] = the
// original row now at row i), then the columns of the inverse, one warp
// each, by forward and backward substitution.  FP64 throughout.
constexpr int kLuMax = 256;

__global__ void __launch_bounds__(256) k_lu_factor(int n, const double* __restrict__ mats, double* __restrict__ lu,
                                                   int* __restrict__ perm) {
  const double* A0 = mats + (size_t)blockIdx.x * n * n;
  double* A = lu + (size_t)blockIdx.x * n * n;
  int* P = perm + (size_t)blockIdx.x * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ int piv;
  __shared__ double inv_d;
  for (int r = warp; r < n; r += nw)
    for (int cc = lane; cc < n; cc += 32) A[(size_t)r * n + cc] = A0[(size_t)r * n + cc];
  for (int r = threadIdx.x; r < n; r += blockDim.x) P[r] = r;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int idx = k;
      for (int r = k + lane; r < n; r += 32) {
        const double v = fabs(A[(size_t)r * n + k]);
        if (v > best) { best = v; idx = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
      }
      if (lane == 0) {
        piv = idx;
        const double d = A[(size_t)idx * n + k];
        inv_d = d != 0.0 ? 1.0 / d : 0.0;
      }
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {
      for (int cc = threadIdx.x; cc < n; cc += blockDim.x) {
        const double t = A[(size_t)k * n + cc];
        A[(size_t)k * n + cc] = A[(size_t)p * n + cc];
        A[(size_t)p * n + cc] = t;
      }
      if (threadIdx.x == 0) {
        const int t = P[k];
        P[k] = P[p];
        P[p] = t;
      }
    }
    __syncthreads();
    const double id = inv_d;
    for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) A[(size_t)r * n + k] *= id;
    __syncthreads();
    for (int r = k + 1 + warp; r < n; r += nw) {
      const double l = A[(size_t)r * n + k];
      if (l == 0.0) continue;
      for (int cc = k + 1 + lane; cc < n; cc += 32) A[(size_t)r * n + cc] -= l * A[(size_t)k * n + cc];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(128) k_lu_inverse(int n, const double* __restrict__ lu, const int* __restrict__ perm,
                                                    double* __restrict__ inv) {
  __shared__ double xs[4][kLuMax];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 4 + warp;
  if (j >= n) return;   // per warp
  const double* A = lu + (size_t)blockIdx.y * n * n;
  const int* P = perm + (size_t)blockIdx.y * n;
  double* x = xs[warp];
  // x = P e_j, then L y = x (unit lower), then U x = y
  for (int i = lane; i < n; i += 32) x[i] = P[i] == j ? 1.0 : 0.0;
  __syncwarp();
  for (int k = 0; k < n - 1; ++k) {
    const double xk = x[k];
    __syncwarp();
    if (xk != 0.0)
      for (int i = k + 1 + lane; i < n; i += 32) x[i] -= A[(size_t)i * n + k] * xk;
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {
    double xk = 0.0;
    if (lane == 0) {
      const double d = A[(size_t)k * n + k];
      xk = d != 0.0 ? x[k] / d : 0.0;
      x[k] = xk;
    }
    xk = __shfl_sync(0xffffffffu, xk, 0);
    __syncwarp();
    if (xk != 0.0)
      for (int i = lane; i < k; i += 32) x[i] -= A[(size_t)i * n + k] * xk;
    __syncwarp();
  }
  double* Inv = inv + (size_t)blockIdx.y * n * n;
  for (int i = lane; i < n; i += 32) Inv[(size_t)i * n + j] = x[i];
}

__global__ void k_gauss_jordan(int n, double* mats, double* work) {
  double* A = mats + (size_t)blockIdx.x * n * n;
  double* Inv = work + (size_t)blockIdx.x * n * n;
  __shared__ int piv;
  __shared__ double pval;
  for (int r = threadIdx.x >> 5; r < n; r += blockDim.x >> 5)
    for (int cc = threadIdx.x & 31; cc < n; cc += 32) Inv[(size_t)r * n + cc] = r == cc ? 1.0 : 0.0;
  __syncthreads();
  for (int col = 0; col < n; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double best = fabs(A[(size_t)col * n + col]);
      for (int r = col + 1; r < n; ++r) {
        const double v = fabs(A[(size_t)r * n + col]);
        if (v > best) { best = v; p = r; }
      }
      piv = p;
      pval = A[(size_t)p * n + col];
    }
    __syncthreads();
    const int p = piv;
    if (p != col)
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double a = A[(size_t)col * n + t]; A[(size_t)col * n + t] = A[(size_t)p * n + t]; A[(size_t)p * n + t] = a;
        double b = Inv[(size_t)col * n + t]; Inv[(size_t)col * n + t] = Inv[(size_t)p * n + t]; Inv[(size_t)p * n + t] = b;
      }
    __syncthreads();
    const double inv_p = pval != 0.0 ? 1.0 / pval : 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      A[(size_t)col * n + t] *= inv_p;
      Inv[(size_t)col * n + t] *= inv_p;
    }
    __syncthreads();
    // rows over warps, columns over lanes (no 64-bit index division)
    for (int r = threadIdx.x >> 5; r < n; r += blockDim.x >> 5) {
      if (r == col) continue;
      const double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int cc = threadIdx.x & 31; cc < n; cc += 32) {
        if (cc != col) A[(size_t)r * n + cc] -= f * A[(size_t)col * n + cc];
        Inv[(size_t)r * n + cc] -= f * Inv[(size_t)col * n + cc];
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != col) A[(size_t)r * n + col] = 0.0;
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) A[t] = Inv[t];
}

// ---------------------------------------------------------------- cycle kernels
template <typename TS, typename T>
struct LvlPtrs {
  const TS* st[kNH];
  const T* dinv[kNH];
  const uint8_t* mask[kNH];
  const T* x[kNH];
  T* xo[kNH];
  const T* b[kNH];
  T* r[kNH];
  T* d[kNH];
};

// Stencil kernels: kNpt rows per thread, blockDim apart (each load
// instruction stays coalesced), and the loads of one z-plane of the stencil
// (9 coefficients and 9 neighbour values per row) issued before their
// updates.  The kernels are bound by memory latency unless enough loads are
// in flight; on cube128 level 0 one row per thread with plane-batched loads
// was fastest (two rows per thread with per-offset loads came close, four or
// more were slower from register pressure).  The block ranges of the masks
// are shared with the one-row-per-thread transfer kernels.
constexpr int kNpt = 1;

// ax[q] = (A x)_{n[q]} in difference form, for the rows with on[q]:
// ax = s_13 x_n + sum_{o != 13} s_o (x_{n+off(o)} - x_n).  Every row takes
// the same unchecked path: the stencils hold exact zeros in the slots of
// neighbours outside the grid, and the x vectors carry zeroed guard zones
// (see alloc_x), so the loads of boundary rows stay in bounds and such a
// slot adds fma(0, finite, acc) = acc.  Indices are 32-bit (every level has
// fewer than 2^31/27 nodes).
template <typename TS, typename T>
__device__ __forceinline__ void stencil_rows(const TS* __restrict__ st, const T* __restrict__ x, const LevelDims& dd,
                                             const int (&n)[kNpt], const bool (&on)[kNpt], T (&ax)[kNpt]) {
  const int N = (int)dd.n;
  const int sy = dd.nnx, sz = dd.nnx * dd.nny;
  T xn[kNpt];
#pragma unroll
  for (int q = 0; q < kNpt; ++q) {
    xn[q] = on[q] ? x[n[q]] : (T)0;
    ax[q] = on[q] ? (T)tof(st[13 * N + n[q]]) * xn[q] : (T)0;
  }
  // one z-plane of the stencil at a time: all of its loads first, then the
  // updates, summed in offset order
#pragma unroll
  for (int pz = 0; pz < 3; ++pz) {
    TS sv[9][kNpt];
    T xv[9][kNpt];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int o = 9 * pz + t;
      if (o == 13) continue;
      const int off = (o % 3 - 1) + ((o / 3) % 3 - 1) * sy + (o / 9 - 1) * sz;
#pragma unroll
      for (int q = 0; q < kNpt; ++q)
        if (on[q]) {
          sv[t][q] = st[o * N + n[q]];
          xv[t][q] = x[n[q] + off];
        }
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      if (9 * pz + t == 13) continue;
#pragma unroll
      for (int q = 0; q < kNpt; ++q)
        if (on[q]) ax[q] += (T)tof(sv[t][q]) * (xv[t][q] - xn[q]);
    }
  }
}

// Chebyshev coefficients, on the device (so that captured graphs stay valid
// across linearizations): for level l, step s and hierarchy h,
// tab[((l kMaxDeg + s) 3 + j) kNH + h], j = 0: c0, 1: ca, 2: cb.  Step 0:
// d = c0 z; later steps: d = ca d + cb z, with z = D^-1 (b - A x).
template <typename T>
__device__ __forceinline__ T cheb_at(const T* tab, int level, int step, int j, int h) {
  return tab[((level * kMaxDeg + step) * 3 + j) * kNH + h];
}

// Rows of this thread: n[q] = base + q blockDim + tid with base the first
// row of block blo[h] + blockIdx.x (the launch covers only the blocks that
// hold rows of the hierarchy's mask).  ld[q]: the row is in range, so its
// loads are issued at once -- every array of a level is finite at every
// node, and a row outside the mask computes a value that is never stored;
// on[q]: the row is also inside the mask and its results are written.
// all_on: the hierarchy's mask is all ones (phi_e, c_e at every level), no
// mask load.
__device__ __forceinline__ void stencil_nodes(int N, const uint8_t* __restrict__ mask, bool all_on, int blo,
                                              int (&n)[kNpt], bool (&ld)[kNpt], bool (&on)[kNpt]) {
  const int base = (blo + (int)blockIdx.x) * (blockDim.x * kNpt) + threadIdx.x;
#pragma unroll
  for (int q = 0; q < kNpt; ++q) {
    n[q] = base + q * blockDim.x;
    ld[q] = n[q] < N;
    on[q] = ld[q] && (all_on || mask[n[q]]);
  }
}

// Block ranges of the listed hierarchies for one launch.
struct BRange {
  int lo[kNH];
  int cnt[kNH];
};

// One Chebyshev step, x_out = x + d.
template <typename TS, typename T>
__global__ void __launch_bounds__(256) k_cheb(LevelDims dd, LvlPtrs<TS, T> P, HList hl, BRange br,
                                              const T* __restrict__ ctab, int level, int step, int first) {
  const int hi = blockIdx.y;
  const int h = pk(hl.h, hi);
  if ((int)blockIdx.x >= pk(br.cnt, h)) return;
  int n[kNpt];
  bool ld[kNpt], on[kNpt];
  stencil_nodes((int)dd.n, pk(P.mask, h), h >= 2, pk(br.lo, h), n, ld, on);
  const T* __restrict__ b = pk(P.b, h);
  const T* __restrict__ dinv = pk(P.dinv, h);
  const T* __restrict__ x = pk(P.x, h);
  T* __restrict__ d = pk(P.d, h);
  T* __restrict__ xo = pk(P.xo, h);
  // the row's own values, loaded before the stencil so that their latency
  // overlaps with the stencil loads
  T bq[kNpt], dq[kNpt], iq[kNpt];
#pragma unroll
  for (int q = 0; q < kNpt; ++q) {
    bq[q] = ld[q] ? b[n[q]] : (T)0;
    iq[q] = ld[q] ? dinv[n[q]] : (T)0;
    dq[q] = (ld[q] && step != 0) ? d[n[q]] : (T)0;
  }
  T ax[kNpt];
  if (!first) stencil_rows<TS, T>(pk(P.st, h), x, dd, n, ld, ax);
  const T c0 = cheb_at(ctab, level, step, 0, h), ca = cheb_at(ctab, level, step, 1, h),
          cb = cheb_at(ctab, level, step, 2, h);
#pragma unroll
  for (int q = 0; q < kNpt; ++q) {
    if (!on[q]) continue;
    const int m = n[q];
    T res = bq[q];
    if (!first) res -= ax[q];
    const T z = iq[q] * res;
    const T dn = step == 0 ? c0 * z : ca * dq[q] + cb * z;
    d[m] = dn;
    xo[m] = (first ? (T)0 : x[m]) + dn;
  }
}

template <typename TS, typename T>
__global__ void __launch_bounds__(256) k_resid(LevelDims dd, LvlPtrs<TS, T> P, HList hl, BRange br) {
  const int h = pk(hl.h, blockIdx.y);
  if ((int)blockIdx.x >= pk(br.cnt, h)) return;
  int n[kNpt];
  bool ld[kNpt], on[kNpt];   // level-0 phi_s hierarchies share r: never write masked-out nodes
  stencil_nodes((int)dd.n, pk(P.mask, h), h >= 2, pk(br.lo, h), n, ld, on);
  T ax[kNpt];
  stencil_rows<TS, T>(pk(P.st, h), pk(P.x, h), dd, n, ld, ax);
  const T* __restrict__ b = pk(P.b, h);
  T* __restrict__ r = pk(P.r, h);
#pragma unroll
  for (int q = 0; q < kNpt; ++q)
    if (on[q]) r[n[q]] = b[n[q]] - ax[q];
}


// 32-bit (i, j, k) of node n of a level (every level has < 2^31 nodes).
__device__ __forceinline__ void node_ijk_i32(const LevelDims& d, int n, int& i, int& j, int& k) {
  const int sxy = d.nnx * d.nny;
  k = n / sxy;
  const int r = n - k * sxy;
  j = r / d.nnx;
  i = r - j * d.nnx;
}

// Full-weighting restriction b_c = P^T r over the fine nodes of the mask.
// The phi_e / c_e masks are all ones (no mask load); elsewhere a masked-out
// residual is selected away (never multiplied: it may hold stale values).
template <typename T>
__global__ void k_restrict(LevelDims fd, LevelDims cd, Xfer X, Ptr4<const T> fr, Ptr4<const uint8_t> fm, Ptr4<T> cb,
                           HList hl, BRange br) {
  const int h = pk(hl.h, blockIdx.y);
  if ((int)blockIdx.x >= pk(br.cnt, h)) return;   // coarse blocks without rows of the coarse mask
  const int C = (pk(br.lo, h) + (int)blockIdx.x) * blockDim.x + threadIdx.x;
  if (C >= (int)cd.n) return;
  int I, J, K;
  node_ijk_i32(cd, C, I, J, K);
  const T* __restrict__ r = pk(fr.p, h);
  const uint8_t* __restrict__ m = pk(fm.p, h);
  const bool all_on = h >= 2;
  const T* swx = supw_t<T>(X.a[0]);
  const T* swy = supw_t<T>(X.a[1]);
  const T* swz = supw_t<T>(X.a[2]);
  T acc = 0;
#pragma unroll
  for (int tz = 0; tz < 3; ++tz) {
    const int fk = X.a[2].sup[K * 3 + tz];
    if (fk < 0) continue;
    const T wz = swz[K * 3 + tz];
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) {
      const int fj = X.a[1].sup[J * 3 + ty];
      if (fj < 0) continue;
      const T wy = swy[J * 3 + ty];
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) {
        const int fi = X.a[0].sup[I * 3 + tx];
        if (fi < 0) continue;
        const int f = fi + fd.nnx * (fj + fd.nny * fk);
        const T v = r[f];
        const bool on = all_on || m[f];
        acc += on ? swx[I * 3 + tx] * wy * wz * v : (T)0;
      }
    }
  }
  pk(cb.p, h)[C] = acc;
}

template <typename T>
__global__ void k_prolong(LevelDims fd, LevelDims cd, Xfer X, Ptr4<const T> cx_, Ptr4<const uint8_t> fm, Ptr4<T> fx,
                          HList hl, BRange br) {
  const int h = pk(hl.h, blockIdx.y);
  if ((int)blockIdx.x >= pk(br.cnt, h)) return;   // fine blocks without rows of the mask
  const int f = (pk(br.lo, h) + (int)blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= (int)fd.n) return;
  // the mask gates only the write: the interpolation's loads do not wait on it
  // (phi_e / c_e masks are all ones)
  const bool on = h >= 2 || pk(fm.p, h)[f];
  const T xf = pk(fx.p, h)[f];
  int i, j, k;
  node_ijk_i32(fd, f, i, j, k);
  const T* __restrict__ cx = pk(cx_.p, h);
  const T* pwx = parw_t<T>(X.a[0]);
  const T* pwy = parw_t<T>(X.a[1]);
  const T* pwz = parw_t<T>(X.a[2]);
  T acc = 0;
#pragma unroll
  for (int c3 = 0; c3 < 2; ++c3) {
    const int pz = X.a[2].par[k * 2 + c3];
    if (pz < 0) continue;
    const T wz = pwz[k * 2 + c3];
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
      const int py = X.a[1].par[j * 2 + c2];
      if (py < 0) continue;
      const T wy = pwy[j * 2 + c2];
#pragma unroll
      for (int c1 = 0; c1 < 2; ++c1) {
        const int px = X.a[0].par[i * 2 + c1];
        if (px < 0) continue;
        acc += pwx[i * 2 + c1] * wy * wz * cx[px + cd.nnx * (py + cd.nny * pz)];
      }
    }
  }
  if (on) pk(fx.p, h)[f] = xf + acc;
}

// x = A^-1 b at the coarsest level (dense FP64 inverse): one warp per row,
// lanes over the columns, a fixed-order warp reduction.
constexpr int kCoarseWarps = 8;
template <typename T>
__global__ void __launch_bounds__(32 * kCoarseWarps) k_coarse_solve(int n, const double* __restrict__ inv,
                                                                    Ptr4<const T> b, Ptr4<const uint8_t> mask,
                                                                    Ptr4<T> x, HList hl) {
  const int h = pk(hl.h, blockIdx.y);
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kCoarseWarps + (threadIdx.x >> 5);
  if (r >= n) return;   // per warp
  const double* A = inv + (size_t)h * n * n + (size_t)r * n;
  const T* bb = pk(b.p, h);
  double acc = 0.0;
  for (int cidx = lane; cidx < n; cidx += 32) acc += A[cidx] * (double)bb[cidx];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && pk(mask.p, h)[r]) pk(x.p, h)[r] = (T)acc;   // masked-out rows are never read (and may be shared)
}

size_t tsize(int precision, int level) {
  if (precision == 0) return sizeof(double);
  if (precision == 2 && level > 0) return sizeof(__nv_bfloat16);
  return sizeof(float);
}

template <typename T>
HList make_hl(const int* hs, int nhs) {
  HList l{};
  for (int i = 0; i < kNH; ++i) l.h[i] = i < nhs ? hs[i] : hs[0];
  return l;
}

LevelDims dims(const MGLevel& L) { return LevelDims{L.nnx, L.nny, L.nnz, L.n}; }

template <typename TS, typename T>
LvlPtrs<TS, T> ptrs(const MGLevel& L) {
  LvlPtrs<TS, T> P;
  for (int h = 0; h < kNH; ++h) {
    P.st[h] = (const TS*)L.st[h];
    P.dinv[h] = (const T*)L.dinv[h];
    P.mask[h] = L.mask[h];
    P.x[h] = (const T*)L.x[h];
    P.xo[h] = (T*)L.x2[h];
    P.b[h] = (const T*)L.b[h];
    P.r[h] = (T*)L.r[h];
    P.d[h] = (T*)L.d[h];
  }
  return P;
}

void swap_x(MGLevel& L, const int* hs, int nhs) {
  bool done[kNH] = {false, false, false, false};
  for (int t = 0; t < nhs; ++t) {
    int h = hs[t];
    // level-0 hierarchies 0/1 alias one buffer pair: swap it once
    if (L.x[h] == L.x[h ^ 1] && h < 2) {
      if (done[0]) continue;
      done[0] = done[1] = true;
      std::swap(L.x[0], L.x2[0]);
      L.x[1] = L.x[0];
      L.x2[1] = L.x2[0];
      continue;
    }
    if (done[h]) continue;
    done[h] = true;
    std::swap(L.x[h], L.x2[h]);
  }
}


// The Chebyshev coefficient table in the smoother's precision.
template <typename T> const T* cheb_tab(const p4d_ctx* c);
template <> const double* cheb_tab<double>(const p4d_ctx* c) { return c->cheb_dev; }
template <> const float* cheb_tab<float>(const p4d_ctx* c) { return c->cheb_dev32; }

// Block ranges of a level for the listed hierarchies, and the launch's
// grid width (the widest range).  The transfer kernels take one row per
// thread in blocks of kBlock and share these ranges.
static_assert(kNpt == 1, "block ranges are shared by the one-row-per-thread transfer kernels");
BRange brange(const MGLevel& A, const int* hs, int nhs, unsigned* gx) {
  BRange r{};
  int w = 1;
  for (int h = 0; h < kNH; ++h) {
    r.lo[h] = A.blo[h];
    r.cnt[h] = A.bcnt[h];
  }
  for (int t = 0; t < nhs; ++t) w = std::max(w, A.bcnt[hs[t]]);
  *gx = (unsigned)w;
  return r;
}

// A level-0 step that applies the operator to a nonzero x (mode 0: a
// Chebyshev step, mode 1: the residual) for the hierarchies hs: the fields
// with a matrix-free operator in one mf launch, the others (phi_s with
// collector shells) with the stored stencils.
template <typename TS0, typename T>
p4d_status level0_stencil_step(p4d_ctx* c, MGLevel& A, const int* hs, int nhs, const HList& hl, const BRange& br,
                               dim3 grid, int mode, int step) {
  int fmask = 0, shs[kNH], ns = 0;
  for (int t = 0; t < nhs; ++t) {
    const int f = hs[t] < 2 ? 0 : hs[t] - 1;
    if (mf_field_on(c, f)) fmask |= 1 << f;
    else shs[ns++] = hs[t];
  }
  if (fmask) P4D_TRYS(mf_level0(c, fmask, mode, step));
  if (ns) {
    const HList hl2 = make_hl<T>(shs, ns);
    const dim3 g2(grid.x, ns);
    if (mode == 0)
      ::p4d::count_launch(), k_cheb<TS0, T><<<g2, kBlock, 0, c->stream>>>(dims(A), ptrs<TS0, T>(A), hl2, br, cheb_tab<T>(c), 0, step, 0);
    else
      ::p4d::count_launch(), k_resid<TS0, T><<<g2, kBlock, 0, c->stream>>>(dims(A), ptrs<TS0, T>(A), hl2, br);
  }
  (void)hl;
  return P4D_OK;
}

template <typename TS0, typename TS, typename T>
p4d_status vcycle_t(p4d_ctx* c, const int* hs, int nhs) {
  const int L = c->nlev;
  const int deg = c->prm.cheb_degree;
  HList hl = make_hl<T>(hs, nhs);
  for (int l = 0; l < L - 1; ++l) {
    MGLevel& A = c->lev[l];
    MGLevel& B = c->lev[l + 1];
    unsigned gx = 1;
    const BRange br = brange(A, hs, nhs, &gx);
    const dim3 grid(gx, nhs);
    for (int s = 0; s < deg; ++s) {
      if (l == 0 && s > 0) prof_mark(c, 3);
      if (l == 0 && s > 0) P4D_TRYS((level0_stencil_step<TS0, T>(c, A, hs, nhs, hl, br, grid, 0, s)));
      else if (l == 0) ::p4d::count_launch(), k_cheb<TS0, T><<<grid, kBlock, 0, c->stream>>>(dims(A), ptrs<TS0, T>(A), hl, br, cheb_tab<T>(c), l, s, 1);
      else ::p4d::count_launch(), k_cheb<TS, T><<<grid, kBlock, 0, c->stream>>>(dims(A), ptrs<TS, T>(A), hl, br, cheb_tab<T>(c), l, s, s == 0);
      if (l == 0 && s > 0) prof_mark(c, 3);
      swap_x(A, hs, nhs);
    }
    if (l == 0) P4D_TRYS((level0_stencil_step<TS0, T>(c, A, hs, nhs, hl, br, grid, 1, 0)));
    else ::p4d::count_launch(), k_resid<TS, T><<<grid, kBlock, 0, c->stream>>>(dims(A), ptrs<TS, T>(A), hl, br);
    Ptr4<const T> fr;
    Ptr4<const uint8_t> fm;
    Ptr4<T> cb;
    for (int h = 0; h < kNH; ++h) { fr.p[h] = (const T*)A.r[h]; fm.p[h] = A.mask[h]; cb.p[h] = (T*)B.b[h]; }
    unsigned gxc = 1;
    const BRange brc = brange(B, hs, nhs, &gxc);
    ::p4d::count_launch(), k_restrict<T><<<dim3(gxc, nhs), kBlock, 0, c->stream>>>(dims(A), dims(B), A.X, fr, fm, cb, hl, brc);
  }
  {
    MGLevel& C = c->lev[L - 1];
    Ptr4<const T> b;
    Ptr4<const uint8_t> m;
    Ptr4<T> x;
    for (int h = 0; h < kNH; ++h) { b.p[h] = (const T*)C.b[h]; m.p[h] = C.mask[h]; x.p[h] = (T*)C.x[h]; }
    ::p4d::count_launch(), k_coarse_solve<T><<<dim3((unsigned)((C.n + kCoarseWarps - 1) / kCoarseWarps), nhs), 32 * kCoarseWarps, 0, c->stream>>>((int)C.n, C.inv, b, m, x, hl);
  }
  for (int l = L - 2; l >= 0; --l) {
    MGLevel& A = c->lev[l];
    MGLevel& B = c->lev[l + 1];
    Ptr4<const T> cxp;
    Ptr4<const uint8_t> fm;
    Ptr4<T> fx;
    for (int h = 0; h < kNH; ++h) { cxp.p[h] = (const T*)B.x[h]; fm.p[h] = A.mask[h]; fx.p[h] = (T*)A.x[h]; }
    unsigned gx = 1;
    const BRange br = brange(A, hs, nhs, &gx);
    const dim3 grid(gx, nhs);
    ::p4d::count_launch(), k_prolong<T><<<grid, kBlock, 0, c->stream>>>(dims(A), dims(B), A.X, cxp, fm, fx, hl, br);
    for (int s = 0; s < deg; ++s) {
      if (l == 0) prof_mark(c, 3);
      if (l == 0) P4D_TRYS((level0_stencil_step<TS0, T>(c, A, hs, nhs, hl, br, grid, 0, s)));
      else ::p4d::count_launch(), k_cheb<TS, T><<<grid, kBlock, 0, c->stream>>>(dims(A), ptrs<TS, T>(A), hl, br, cheb_tab<T>(c), l, s, 0);
      if (l == 0) prof_mark(c, 3);
      swap_x(A, hs, nhs);
    }
  }
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

}  // namespace

// ---------------------------------------------------------------- planning
// An x vector of a level (the input of the unchecked stencil loads) with a
// zeroed guard of at least nnx nny + nnx + 1 entries on both sides, rounded
// to 64 entries so that the vector keeps the allocation's alignment.
p4d_status alloc_x(p4d_ctx* c, void** p, size_t ts, const MGLevel& lv) {
  const int64_t G = ((int64_t)lv.nnx * lv.nny + lv.nnx + 1 + 63) / 64 * 64;
  const size_t bytes = ts * (size_t)(lv.n + 2 * G);
  void* base = nullptr;
  P4D_TRYS(dalloc(c, &base, bytes));
  P4D_TRY(cudaMemset(base, 0, bytes));
  *p = static_cast<char*>(base) + ts * G;
  return P4D_OK;
}

p4d_status mg_plan(p4d_ctx* c) {
  const int prec = c->prm.precision;
  const size_t tv = prec == 0 ? sizeof(double) : sizeof(float);
  int nnx = c->g.nnx, nny = c->g.nny, nnz = c->g.nnz;
  int L = 0;
  while (true) {
    MGLevel& lv = c->lev[L];
    lv.nnx = nnx; lv.nny = nny; lv.nnz = nnz;
    lv.n = (int64_t)nnx * nny * nnz;
    // coarsened axes: those with >= 2 elements (odd counts included) whose
    // mean element size is at most twice the smallest among them -- the
    // stiffness couples most strongly across short element edges, and the
    // point smoother reduces only errors smooth along the weak directions,
    // so weakly coupled axes stay fine until the elements are near isotropic
    const int nd[3] = {nnx, nny, nnz};
    int can[3];
    double hm[3], hmin = 0.0;
    bool any = false;
    for (int a = 0; a < 3; ++a) {
      can[a] = (nd[a] - 1) >= 2;
      hm[a] = nd[a] >= 2 ? c->len[a] / (nd[a] - 1) : 0.0;
      if (can[a] && (!any || hm[a] < hmin)) hmin = hm[a];
      any = any || can[a];
    }
    const int cx = can[0] && hm[0] <= 2.0 * hmin, cy = can[1] && hm[1] <= 2.0 * hmin,
              cz = can[2] && hm[2] <= 2.0 * hmin;
    ++L;
    if (lv.n <= c->prm.coarse_max || !(cx || cy || cz) || L >= kMaxLevels) break;
    lv.cx = cx; lv.cy = cy; lv.cz = cz;
    const int dn[3] = {nnx, nny, nnz}, fl[3] = {cx, cy, cz};
    int cn[3];
    for (int a = 0; a < 3; ++a) {
      const int nf = dn[a], ne = nf - 1;
      const int nc = fl[a] ? (ne + 1) / 2 + 1 : nf;
      cn[a] = nc;
      std::vector<int> par(2 * nf, -1), sup(3 * nc, -1);
      std::vector<double> parw(2 * nf, 0.0), supw(3 * nc, 0.0);
      for (int i = 0; i < nf; ++i) {
        if (!fl[a]) { par[2 * i] = i; parw[2 * i] = 1.0; continue; }
        if ((ne & 1) && i == ne) { par[2 * i] = (ne + 1) / 2; parw[2 * i] = 1.0; }
        else if ((i & 1) == 0) { par[2 * i] = i / 2; parw[2 * i] = 1.0; }
        else { par[2 * i] = (i - 1) / 2; par[2 * i + 1] = (i + 1) / 2; parw[2 * i] = parw[2 * i + 1] = 0.5; }
      }
      std::vector<int> cnt(nc, 0);
      for (int i = 0; i < nf; ++i)
        for (int q = 0; q < 2; ++q) {
          const int C = par[2 * i + q];
          if (C < 0) continue;
          if (cnt[C] >= 3) return P4D_ERR_INVALID_ARG;
          sup[3 * C + cnt[C]] = i;
          supw[3 * C + cnt[C]] = parw[2 * i + q];
          ++cnt[C];
        }
      int* dp = nullptr;
      double* dw = nullptr;
      P4D_TRYS(dalloc_t(c, &dp, par.size() + sup.size()));
      P4D_TRYS(dalloc_t(c, &dw, parw.size() + supw.size()));
      P4D_TRY(cudaMemcpy(dp, par.data(), par.size() * sizeof(int), cudaMemcpyHostToDevice));
      P4D_TRY(cudaMemcpy(dp + par.size(), sup.data(), sup.size() * sizeof(int), cudaMemcpyHostToDevice));
      P4D_TRY(cudaMemcpy(dw, parw.data(), parw.size() * sizeof(double), cudaMemcpyHostToDevice));
      P4D_TRY(cudaMemcpy(dw + parw.size(), supw.data(), supw.size() * sizeof(double), cudaMemcpyHostToDevice));
      std::vector<float> wf(parw.size() + supw.size());
      for (size_t q = 0; q < parw.size(); ++q) wf[q] = (float)parw[q];
      for (size_t q = 0; q < supw.size(); ++q) wf[parw.size() + q] = (float)supw[q];
      float* dwf = nullptr;
      P4D_TRYS(dalloc_t(c, &dwf, wf.size()));
      P4D_TRY(cudaMemcpy(dwf, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice));
      lv.X.a[a] = Axis{dp, dw, dp + par.size(), dw + parw.size(), dwf, dwf + parw.size()};
    }
    nnx = cn[0];
    nny = cn[1];
    nnz = cn[2];
  }
  c->nlev = L;
  if (c->lev[L - 1].n > 4096) return P4D_ERR_INVALID_ARG;   // coarsest level too large for a dense inverse
  for (int l = 0; l < L; ++l) {
    MGLevel& lv = c->lev[l];
    const int64_t n = lv.n;
    const size_t ts = tsize(prec, l);
    P4D_TRYS(dalloc_t(c, &lv.lam, kNH));
    for (int h = 0; h < kNH; ++h) P4D_TRYS(dalloc_t(c, &lv.mask[h], n));
    if (l == 0) {
      // fields: phi_s (hierarchies 0,1 share), phi_e (2), c_e (3)
      void *st[3], *di[3], *x[3], *x2[3], *b[3], *r[3], *d[3];
      for (int f = 0; f < 3; ++f) {
        P4D_TRYS(dalloc(c, &st[f], ts * 27 * n));
        P4D_TRYS(dalloc(c, &di[f], tv * n));
        P4D_TRYS(alloc_x(c, &x[f], tv, lv));
        P4D_TRYS(alloc_x(c, &x2[f], tv, lv));
        P4D_TRYS(dalloc(c, &b[f], tv * n));
        P4D_TRYS(dalloc(c, &r[f], tv * n));
        P4D_TRYS(dalloc(c, &d[f], tv * n));
        P4D_TRY(cudaMemset(x[f], 0, tv * n));
        P4D_TRY(cudaMemset(x2[f], 0, tv * n));
        P4D_TRY(cudaMemset(b[f], 0, tv * n));
        P4D_TRY(cudaMemset(d[f], 0, tv * n));
      }
      const int fh[kNH] = {0, 0, 1, 2};
      for (int h = 0; h < kNH; ++h) {
        lv.st[h] = st[fh[h]]; lv.dinv[h] = di[fh[h]]; lv.x[h] = x[fh[h]]; lv.x2[h] = x2[fh[h]];
        lv.b[h] = b[fh[h]]; lv.r[h] = r[fh[h]]; lv.d[h] = d[fh[h]];
      }
      ::p4d::count_launch(), k_mask0<<<nblocks(n), kBlock, 0, c->stream>>>(n, c->label, lv.mask[0], lv.mask[1], lv.mask[2], lv.mask[3]);
    } else {
      P4D_TRYS(dalloc_t(c, &lv.Ffix, (size_t)kNH * 27 * n));
      P4D_TRYS(dalloc(c, &lv.Vvar, (prec == 0 ? sizeof(double) : sizeof(float)) * (size_t)kNH * 27 * n));
      for (int h = 0; h < kNH; ++h) {
        P4D_TRYS(dalloc(c, &lv.st[h], ts * 27 * n));
        P4D_TRYS(dalloc(c, &lv.dinv[h], tv * n));
        P4D_TRYS(alloc_x(c, &lv.x[h], tv, lv));
        P4D_TRYS(alloc_x(c, &lv.x2[h], tv, lv));
        P4D_TRYS(dalloc(c, &lv.b[h], tv * n));
        P4D_TRYS(dalloc(c, &lv.r[h], tv * n));
        P4D_TRYS(dalloc(c, &lv.d[h], tv * n));
        P4D_TRY(cudaMemset(lv.x[h], 0, tv * n));
        P4D_TRY(cudaMemset(lv.x2[h], 0, tv * n));
        P4D_TRY(cudaMemset(lv.d[h], 0, tv * n));
      }
      MGLevel& fl = c->lev[l - 1];
      Ptr4<const uint8_t> fm;
      Ptr4<uint8_t> cm;
      for (int h = 0; h < kNH; ++h) { fm.p[h] = fl.mask[h]; cm.p[h] = lv.mask[h]; }
      ::p4d::count_launch(), k_mask_coarse<<<dim3(nblocks(n), kNH), kBlock, 0, c->stream>>>(dims(fl), dims(lv), fl.X, fm, cm);
    }
    if (l == L - 1) {
      P4D_TRYS(dalloc_t(c, &lv.inv, (size_t)2 * kNH * n * n));
      P4D_TRYS(dalloc_t(c, &lv.perm, (size_t)kNH * n));
    }
  }
  // per level and hierarchy, the stencil-kernel blocks that hold mask rows
  {
    int* ext = nullptr;
    P4D_TRYS(dalloc_t(c, &ext, (size_t)2 * kNH * L));
    std::vector<int> init(2 * kNH * L);
    for (int l = 0; l < L; ++l)
      for (int h = 0; h < kNH; ++h) {
        init[2 * (l * kNH + h)] = (int)c->lev[l].n;
        init[2 * (l * kNH + h) + 1] = -1;
      }
    P4D_TRY(cudaMemcpyAsync(ext, init.data(), init.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    for (int l = 0; l < L; ++l) {
      Ptr4<const uint8_t> m;
      for (int h = 0; h < kNH; ++h) m.p[h] = c->lev[l].mask[h];
      ::p4d::count_launch(), k_mask_extent<<<dim3(nblocks(c->lev[l].n), kNH), kBlock, 0, c->stream>>>(
          c->lev[l].n, m, ext + 2 * kNH * l);
    }
    P4D_TRY(cudaMemcpyAsync(init.data(), ext, init.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    P4D_TRY(cudaStreamSynchronize(c->stream));
    const int rows = kBlock * kNpt;
    for (int l = 0; l < L; ++l)
      for (int h = 0; h < kNH; ++h) {
        const int lo = init[2 * (l * kNH + h)], hi = init[2 * (l * kNH + h) + 1];
        c->lev[l].blo[h] = hi < 0 ? 0 : lo / rows;
        c->lev[l].bcnt[h] = hi < 0 ? 0 : hi / rows - lo / rows + 1;
      }
  }
  // level-0 particle work and variable row sums
  P4D_TRYS(dalloc(c, &c->yc, (prec == 0 ? sizeof(double) : sizeof(float)) * (size_t)std::max<int64_t>(1, c->NE) * c->nc));
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

namespace {
template <typename TS>
__global__ void k_level0_offdiag(Grid g, const double* __restrict__ Jst, double s0, double s1, double s2, TS* st0,
                                 TS* st1, TS* st2) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int64_t nn = g.nn;
  TS* sts[3] = {st0, st1, st2};
  const double sc[3] = {s0, s1, s2};
  for (int f = 0; f < 3; ++f)
    for (int o = 0; o < 27; ++o)
      if (o != 13) sts[f][o * nn + n] = fromd<TS>(sc[f] * Jst[((size_t)f * 27 + o) * nn + n]);
}
}  // namespace

p4d_status mg_setup_fixed(p4d_ctx* c) {
  const int prec = c->prm.precision;
  MGLevel& l0 = c->lev[0];
  if (prec == 0)
    ::p4d::count_launch(), k_level0_offdiag<double><<<nblocks(l0.n), kBlock, 0, c->stream>>>(c->g, c->Jst, c->scale_f[0], c->scale_f[1], c->scale_f[2],
                                                                  (double*)l0.st[0], (double*)l0.st[2], (double*)l0.st[3]);
  else
    ::p4d::count_launch(), k_level0_offdiag<float><<<nblocks(l0.n), kBlock, 0, c->stream>>>(c->g, c->Jst, c->scale_f[0], c->scale_f[1], c->scale_f[2],
                                                                 (float*)l0.st[0], (float*)l0.st[2], (float*)l0.st[3]);
  const int64_t nn = c->g.nn;
  for (int l = 0; l + 1 < c->nlev; ++l) {
    MGLevel& A = c->lev[l];
    MGLevel& B = c->lev[l + 1];
    Ptr4<const double> fst, frs;
    Ptr4<const uint8_t> fm, cm;
    Ptr4<double> out;
    const int fh[kNH] = {0, 0, 1, 2};
    for (int h = 0; h < kNH; ++h) {
      if (l == 0) {
        fst.p[h] = c->Jst + (size_t)fh[h] * 27 * nn;
        frs.p[h] = c->sfix + (size_t)fh[h] * nn;
      } else {
        fst.p[h] = A.Ffix + (size_t)h * 27 * A.n;
        frs.p[h] = nullptr;
      }
      fm.p[h] = A.mask[h];
      cm.p[h] = B.mask[h];
      out.p[h] = B.Ffix + (size_t)h * 27 * B.n;
    }
    ::p4d::count_launch(), k_rap<double><<<dim3(nblocks(B.n, kRapWarps), kNH), 32 * kRapWarps, 0, c->stream>>>(dims(A), dims(B), A.X, fst, frs, fm, cm, out, 1);
  }
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

// Inverse of the coarsest dense matrices in mats (overwritten with it);
// work: scratch of the same size.
p4d_status coarse_inverse(p4d_ctx* c, MGLevel& C, double* mats, double* work) {
  const int n = (int)C.n;
  if (n <= kLuMax) {
    ::p4d::count_launch(), k_lu_factor<<<kNH, 256, 0, c->stream>>>(n, mats, work, C.perm);
    ::p4d::count_launch(), k_lu_inverse<<<dim3((n + 3) / 4, kNH), 128, 0, c->stream>>>(n, work, C.perm, mats);
  } else {
    ::p4d::count_launch(), k_gauss_jordan<<<kNH, 256, 0, c->stream>>>(n, mats, work);
  }
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

// Variable part of levels >= 1 (Galerkin products in precision TV), the
// stored level operators, and the coarsest dense inverse (FP64).
template <typename TV>
p4d_status mg_update_levels(p4d_ctx* c, const double* svar, const double* sch) {
  const int prec = c->prm.precision;
  const int64_t nn = c->g.nn;
  const double* sf = c->scale_f;
  const int fh[kNH] = {0, 0, 1, 2};
  for (int l = 1; l < c->nlev; ++l) {
    MGLevel& A = c->lev[l - 1];
    MGLevel& B = c->lev[l];
    Ptr4<const uint8_t> fm, cm;
    Ptr4<TV> out;
    for (int h = 0; h < kNH; ++h) { fm.p[h] = A.mask[h]; cm.p[h] = B.mask[h]; out.p[h] = (TV*)B.Vvar + (size_t)h * 27 * B.n; }
    if (l == 1) {
      Ptr4<const double> s;
      for (int h = 0; h < kNH; ++h) s.p[h] = svar + (size_t)fh[h] * nn;
      ::p4d::count_launch(), k_rap_diag_g<TV><<<dim3(nblocks(B.n, 128), kNH), 128, 0, c->stream>>>(dims(A), dims(B), A.X, s, fm, cm, out);
    } else {
      Ptr4<const TV> fst, frs;
      for (int h = 0; h < kNH; ++h) { fst.p[h] = (const TV*)A.Vvar + (size_t)h * 27 * A.n; frs.p[h] = nullptr; }
      ::p4d::count_launch(), k_rap<TV><<<dim3(nblocks(B.n, kRapWarps), kNH), 32 * kRapWarps, 0, c->stream>>>(dims(A), dims(B), A.X, fst, frs, fm, cm, out, 0);
    }
    Ptr4<const double> F;
    Ptr4<const TV> V;
    Ptr4<const uint8_t> m;
    for (int h = 0; h < kNH; ++h) {
      F.p[h] = B.Ffix + (size_t)h * 27 * B.n;
      V.p[h] = (const TV*)B.Vvar + (size_t)h * 27 * B.n;
      m.p[h] = B.mask[h];
    }
    const dim3 grid(nblocks(B.n), kNH);
    if (prec == 0) {
      Ptr4<double> st, di;
      for (int h = 0; h < kNH; ++h) { st.p[h] = (double*)B.st[h]; di.p[h] = (double*)B.dinv[h]; }
      ::p4d::count_launch(), k_level_combine<double, double, TV><<<grid, kBlock, 0, c->stream>>>(dims(B), F, V, st, di, m, sch[0], sch[1], sch[2], sch[3], B.lam);
    } else if (prec == 1) {
      Ptr4<float> st, di;
      for (int h = 0; h < kNH; ++h) { st.p[h] = (float*)B.st[h]; di.p[h] = (float*)B.dinv[h]; }
      ::p4d::count_launch(), k_level_combine<float, float, TV><<<grid, kBlock, 0, c->stream>>>(dims(B), F, V, st, di, m, sch[0], sch[1], sch[2], sch[3], B.lam);
    } else {
      Ptr4<__nv_bfloat16> st;
      Ptr4<float> di;
      for (int h = 0; h < kNH; ++h) { st.p[h] = (__nv_bfloat16*)B.st[h]; di.p[h] = (float*)B.dinv[h]; }
      ::p4d::count_launch(), k_level_combine<__nv_bfloat16, float, TV><<<grid, kBlock, 0, c->stream>>>(dims(B), F, V, st, di, m, sch[0], sch[1], sch[2], sch[3], B.lam);
    }
  }
  // coarsest: dense scaled operator and its inverse
  MGLevel& C = c->lev[c->nlev - 1];
  double* mats = C.inv;
  double* work = C.inv + (size_t)kNH * C.n * C.n;
  if (c->nlev == 1) {
    Ptr4<const uint8_t> m;
    for (int h = 0; h < kNH; ++h) m.p[h] = C.mask[h];
    ::p4d::count_launch(), k_dense0<<<dim3(nblocks(C.n), kNH), kBlock, 0, c->stream>>>(c->g, c->Jst, c->sfix, svar, m, sf[0], sf[1], sf[2],
                                                                 mats);
  } else {
    Ptr4<const double> F;
    Ptr4<const TV> V;
    for (int h = 0; h < kNH; ++h) {
      F.p[h] = C.Ffix + (size_t)h * 27 * C.n;
      V.p[h] = (const TV*)C.Vvar + (size_t)h * 27 * C.n;
    }
    ::p4d::count_launch(), k_dense<TV><<<dim3(nblocks(C.n), kNH), kBlock, 0, c->stream>>>(dims(C), F, V, sch[0], sch[1], sch[2], sch[3], mats);
  }
  P4D_TRYS(coarse_inverse(c, C, mats, work));
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status mg_update(p4d_ctx* c) {
  const int prec = c->prm.precision;
  const int64_t nn = c->g.nn;
  const double tau = (1.0 - c->prm.tplus) / c->prm.F;
  const double* sf = c->scale_f;
  const double sch[kNH] = {sf[0], sf[0], sf[1], sf[2]};
  double* svar = c->tmp;   // [3][nn] scratch (Krylov scratch is idle during an update)
  for (int l = 0; l < c->nlev; ++l) P4D_TRY(cudaMemsetAsync(c->lev[l].lam, 0, kNH * sizeof(double), c->stream));
  MGLevel& l0 = c->lev[0];
  if (prec == 0)
    ::p4d::count_launch(), k_level0_update<double, double><<<nblocks(nn), kBlock, 0, c->stream>>>(
        c->g, tau, c->sfix, c->offsum, c->absoff, c->label, c->eidx, c->Aj, c->ge, c->gc, c->zeta, sf[0], sf[1], sf[2],
        (double*)l0.st[0], (double*)l0.st[2], (double*)l0.st[3], (double*)l0.dinv[0], (double*)l0.dinv[2],
        (double*)l0.dinv[3], svar, l0.lam, (float2*)nullptr);
  else
    ::p4d::count_launch(), k_level0_update<float, float><<<nblocks(nn), kBlock, 0, c->stream>>>(
        c->g, tau, c->sfix, c->offsum, c->absoff, c->label, c->eidx, c->Aj, c->ge, c->gc, c->zeta, sf[0], sf[1], sf[2],
        (float*)l0.st[0], (float*)l0.st[2], (float*)l0.st[3], (float*)l0.dinv[0], (float*)l0.dinv[2],
        (float*)l0.dinv[3], svar, l0.lam, (float2*)c->mf_svs);
  if (prec == 0) P4D_TRYS(mg_update_levels<double>(c, svar, sch));
  else P4D_TRYS(mg_update_levels<float>(c, svar, sch));
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status mg_fetch_lam(p4d_ctx* c) {
  for (int l = 0; l < c->nlev; ++l)
    P4D_TRY(cudaMemcpyAsync(c->lam_pin + l * kNH, c->lev[l].lam, kNH * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
  P4D_TRY(cudaStreamSynchronize(c->stream));
  for (int l = 0; l < c->nlev; ++l)
    for (int h = 0; h < kNH; ++h) c->lam_h[l][h] = c->lam_pin[l * kNH + h];
  return cheb_upload(c);
}

// Chebyshev(degree d) coefficients on [lam/ratio, lam] of D^-1 A for every
// level, step and hierarchy (three-term recurrence of the shifted Chebyshev
// polynomials), copied to the device table.
p4d_status cheb_upload(p4d_ctx* c) {
  const double ratio = c->prm.cheb_ratio;
  double* t = c->cheb_pin;
  P4D_TRY(cudaStreamSynchronize(c->stream));   // the previous copy from t has completed
  for (int l = 0; l < c->nlev; ++l)
    for (int h = 0; h < kNH; ++h) {
      const double lm = c->lam_h[l][h] > 0 ? c->lam_h[l][h] : 1.0;
      const double alpha = lm / ratio, beta = lm;
      const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
      const double sigma = theta / delta;
      double rho = 1.0 / sigma, rho_new = rho;
      for (int st = 0; st < c->prm.cheb_degree && st < kMaxDeg; ++st) {
        if (st > 0) {
          rho = rho_new;
          rho_new = 1.0 / (2.0 * sigma - rho);
        }
        t[((l * kMaxDeg + st) * 3 + 0) * kNH + h] = 1.0 / theta;
        t[((l * kMaxDeg + st) * 3 + 1) * kNH + h] = rho_new * rho;
        t[((l * kMaxDeg + st) * 3 + 2) * kNH + h] = 2.0 * rho_new / delta;
      }
    }
  const size_t ne = (size_t)kMaxLevels * kMaxDeg * 3 * kNH;
  float* t32 = reinterpret_cast<float*>(t + ne);   // FP32 copy for the FP32 smoothers
  for (size_t q = 0; q < ne; ++q) t32[q] = (float)t[q];
  P4D_TRY(cudaMemcpyAsync(c->cheb_dev, t, sizeof(double) * ne, cudaMemcpyHostToDevice, c->stream));
  P4D_TRY(cudaMemcpyAsync(c->cheb_dev32, t32, sizeof(float) * ne, cudaMemcpyHostToDevice, c->stream));
  return P4D_OK;
}

p4d_status mg_vcycle(p4d_ctx* c, const int* hs, int nhs) {
  switch (c->prm.precision) {
    case 0: return vcycle_t<double, double, double>(c, hs, nhs);
    case 1: return vcycle_t<float, float, float>(c, hs, nhs);
    default: return vcycle_t<float, __nv_bfloat16, float>(c, hs, nhs);
  }
}

}  // namespace p4d
