// Right-preconditioned flexible GMRES(m) (Saad 1993) in FP64 on the scaled
// system s.J.s x^ = s.b (s_i = w_f / sqrt(J_ii)); the preconditioned
// directions are stored unscaled (z_k = P^-1 (s^-1 v_k)), so that
// x = x0 + sum_k y_k z_k and the operator is applied as s.(J z_k).
//
// Orthogonalisation: classical Gram-Schmidt; a second pass runs only when the
// first cancelled more than half of the vector ("twice is enough" with the
// Daniel-Gragg-Kaufman-Stewart test, decided on the device).  Each pass is a
// register-blocked multi-dot over the basis with a fixed-shape two-stage
// reduction (deterministic order).  The Hessenberg
// column, Givens rotations and residual estimate are updated on the device by
// one thread; the host reads one scalar per iteration.
#include <cmath>
#include <cstring>
#include "p4d_common.cuh"

namespace p4d {
namespace {

constexpr int kRedBlocks = 4 * 152;   // reduction grid: a multiple of the SM count
constexpr int kRedThreads = 256;

// Multi-dot, register blocked with a compile-time group size: each thread
// keeps one accumulator per dot of a group of NG dots (plus w.w) over all of
// its elements, so exactly NG FP64 FMAs run per element (a run-time group
// size with predicated FMAs issued all sixteen).  The warp stage is a
// transpose reduction: with P (a power of two >= NG + WW) values per lane,
// each butterfly step halves the values a lane keeps, P - 1 + log2(32/P)
// FP64 adds per lane instead of 5 per value (FP64 adds are as scarce as FP64
// FMAs on this GPU).
// partial[blk][g0 + i] = sum over the block's elements of V[g0 + i][n] * w[n];
// WW: partial[blk][kp1] = sum w[n]^2.
constexpr int kDotGroup = 16;

template <int X>
struct Pow2Up {
  static constexpr int v = X <= 1 ? 1 : (X <= 2 ? 2 : (X <= 4 ? 4 : (X <= 8 ? 8 : (X <= 16 ? 16 : 32))));
};
template <int X>
struct Log2 {
  static constexpr int v = X <= 1 ? 0 : 1 + Log2<X / 2>::v;
};
template <>
struct Log2<1> {
  static constexpr int v = 0;
};

// After the call, lane l holds in a[0] the warp total of value index
// l >> (5 - log2 P) (every lane of a group of 32/P lanes holds the same).
template <int P>
__device__ __forceinline__ void warp_transpose_reduce(double (&a)[P], int lane) {
#pragma unroll
  for (int c = P, o = 16; c > 1; c >>= 1, o >>= 1) {
    const bool upper = lane & o;
#pragma unroll
    for (int t = 0; t < c / 2; ++t) {
      const double send = upper ? a[t] : a[t + c / 2];
      const double keep = upper ? a[t + c / 2] : a[t];
      a[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 16 >> Log2<P>::v; o > 0; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
}

template <int NG, bool WW>
__global__ void __launch_bounds__(kRedThreads) k_mdot(const double* __restrict__ V, int64_t ldv, int g0, int kp1,
                                                      const double* __restrict__ w, int64_t len,
                                                      double* __restrict__ partial, int pstride,
                                                      const double* __restrict__ flag) {
  if (flag && *flag == 0.0) return;   // conditional pass not needed
  constexpr int NA = NG + (WW ? 1 : 0);
  constexpr int P = Pow2Up<NA>::v;
  __shared__ double red[kRedThreads / 32][P];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc[P];
#pragma unroll
  for (int i = 0; i < P; ++i) acc[i] = 0.0;
  const double* Vg = V + (int64_t)g0 * ldv;
  int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // two elements per trip, all their loads issued before the FMAs (twice the
  // loads in flight); each accumulator still takes n, n + stride, ... in order
  for (; n + stride < len; n += 2 * stride) {
    const double w0 = w[n], w1 = w[n + stride];
    double a0[NG > 0 ? NG : 1], a1[NG > 0 ? NG : 1];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      a0[i] = Vg[(int64_t)i * ldv + n];
      a1[i] = Vg[(int64_t)i * ldv + n + stride];
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      acc[i] = fma(a0[i], w0, acc[i]);
      acc[i] = fma(a1[i], w1, acc[i]);
    }
    if (WW) {
      acc[NG] = fma(w0, w0, acc[NG]);
      acc[NG] = fma(w1, w1, acc[NG]);
    }
  }
  for (; n < len; n += stride) {
    const double wn = w[n];
#pragma unroll
    for (int i = 0; i < NG; ++i) acc[i] = fma(Vg[(int64_t)i * ldv + n], wn, acc[i]);
    if (WW) acc[NG] = fma(wn, wn, acc[NG]);
  }
  warp_transpose_reduce<P>(acc, lane);
  constexpr int span = 32 / P;
  if ((lane & (span - 1)) == 0) red[warp][lane / span] = acc[0];
  __syncthreads();
  if (threadIdx.x < NA) {
    const int i = threadIdx.x;
    double sum = 0.0;
#pragma unroll
    for (int wv = 0; wv < kRedThreads / 32; ++wv) sum += red[wv][i];
    partial[(int64_t)blockIdx.x * pstride + (i < NG ? g0 + i : kp1)] = sum;
  }
}

// out[i] = sum over blocks of partial[b][i]: one block per dot, strided
// per-thread sums and a shared-memory tree (fixed order: deterministic).
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblk, int pstride, int nd,
                                  double* __restrict__ out, const double* __restrict__ flag, int zero_if_skipped) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  if (i >= nd) return;
  if (flag && *flag == 0.0) {
    if (zero_if_skipped && threadIdx.x == 0) out[i] = 0.0;
    return;
  }
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(int64_t)b * pstride + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}

// w[n] -= sum_i h[i] V[i][n]   (h on the device).  With `partial`, each
// block also writes the sum of the updated w[n]^2 over its elements.
__global__ void __launch_bounds__(kBlock) k_maxpy(const double* __restrict__ V, int64_t ldv, int kp1,
                                                  const double* __restrict__ h, double* __restrict__ w,
                                                  int64_t len, double sign, const double* __restrict__ flag,
                                                  double* __restrict__ partial) {
  if (flag && *flag == 0.0) return;
  __shared__ double hs[130];
  __shared__ double red[kBlock / 32];
  for (int i = threadIdx.x; i < kp1; i += blockDim.x) hs[i] = sign * h[i];
  __syncthreads();
  double ss = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < len; n += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[n];
    for (int i = 0; i < kp1; ++i) acc -= hs[i] * V[(int64_t)i * ldv + n];
    w[n] = acc;
    if (partial) ss = fma(acc, acc, ss);
  }
  if (!partial) return;
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) t += red[i];
    partial[blockIdx.x] = t;
  }
}

// y = x * f(*sp): mode 0 f = s, mode 1 f = 1/s, mode 2 f = 1/sqrt(s) (0 if
// s == 0); x and y may be the same vector (no __restrict__ on them).
__global__ void k_scale(const double* x, double* y, int64_t len, const double* __restrict__ sp, int mode) {
  // the factor once per block (an FP64 divide and square root per thread
  // cost more than the scaling itself on this GPU)
  __shared__ double sfac;
  if (threadIdx.x == 0) {
    const double v = *sp;
    sfac = mode == 0 ? v : (v != 0.0 ? (mode == 1 ? 1.0 / v : 1.0 / sqrt(v)) : 0.0);
  }
  __syncthreads();
  const double s = sfac;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < len; n += (int64_t)gridDim.x * blockDim.x)
    y[n] = x[n] * s;
}

// Per-field squared norms of (b / sqrt(d)) over the 4 fields (c_s optional),
// one contiguous range per field.
__global__ void k_field_norms(const double* __restrict__ b, const double* __restrict__ rsqd, int64_t nn, int64_t len,
                              double* __restrict__ partial) {
  double acc[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t lo = f * nn, hi = f < 3 ? (f + 1) * nn : len;
    acc[f] = hi > lo ? sumsq_share<true>(b + lo, rsqd + lo, hi - lo) : 0.0;
  }
  block_sum4(acc, partial);
}

// Field weights of the Krylov norm: w_f = 1 / max(||b~_f||, floor_f), b~ = b/sqrt(d).
// Forward solves: floor_f = (1e-14/rtol) ||(sqrt(d) u)_f|| with u the
// linearization state -- a field's right-hand side is balanced against the
// others unless it lies below the rounding level of the field's own terms
// (then FGMRES could never reduce its residual by rtol).  Adjoint solves:
// floor_f = 1e-2 ||b~|| (the adjoint variable has no state scale).
__device__ void weights_of(const double* s4, const double* __restrict__ unorm2, double floor_rel, int adjoint,
                           double* __restrict__ wf, double* __restrict__ iwf, double* bn2) {
  double all = 0.0;
  for (int f = 0; f < 4; ++f) all += s4[f];
  double tot = 0.0;
  for (int f = 0; f < 4; ++f) {
    const double fl = adjoint ? 1e-4 * all : floor_rel * floor_rel * unorm2[f];
    const double s = fmax(s4[f], fl);
    wf[f] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    iwf[f] = s > 0.0 ? sqrt(s) : 1.0;
    bn2[f] = s;
    tot += s > 0.0 ? s4[f] / s : 0.0;
  }
  bn2[4] = tot;
}

__global__ void k_weights(const double* __restrict__ partial, int nblk, const double* __restrict__ unorm2,
                          double floor_rel, int adjoint, double* __restrict__ wf, double* __restrict__ iwf,
                          double* bn2) {
  __shared__ double s4[4];
  sum4_warps(partial, nblk, s4);
  __syncthreads();
  if (threadIdx.x != 0) return;
  weights_of(s4, unorm2, floor_rel, adjoint, wf, iwf, bn2);
}

// The same from the four field sums already in sums[0..3] (bn2 may alias sums).
__global__ void k_weights_sums(const double* sums, const double* __restrict__ unorm2, double floor_rel,
                               double* __restrict__ wf, double* __restrict__ iwf, double* bn2) {
  if (threadIdx.x != 0) return;
  double s4[4];
  for (int f = 0; f < 4; ++f) s4[f] = sums[f];
  weights_of(s4, unorm2, floor_rel, 0, wf, iwf, bn2);
}

// dst = src when the second Gram-Schmidt pass ran (flag), else unchanged.
__global__ void k_take_if(double* dst, const double* __restrict__ src, const double* __restrict__ flag) {
  if (threadIdx.x == 0 && *flag != 0.0) *dst = *src;
}

// Per-field squared norms of an already scaled vector.
__global__ void k_field_norms_plain(const double* __restrict__ r, int64_t nn, int64_t len, double* __restrict__ partial) {
  double acc[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int64_t lo = f * nn, hi = f < 3 ? (f + 1) * nn : len;
    acc[f] = hi > lo ? sumsq_share<false>(r + lo, nullptr, hi - lo) : 0.0;
  }
  block_sum4(acc, partial);
}

__global__ void k_sum4(const double* __restrict__ partial, int nblk, double* out) { sum4_warps(partial, nblk, out); }

// Hessenberg layout in hs: H[(m+1) x m] column-major, cs[m], sn[m], g[m+1], y[m], misc
struct HLay {
  int m;
  int H, cs, sn, g, y, misc;
};
HLay hlay(int m) {
  HLay L;
  L.m = m;
  L.H = 0;
  L.cs = (m + 1) * m;
  L.sn = L.cs + m;
  L.g = L.sn + m;
  L.y = L.g + m + 1;
  L.misc = L.y + m;
  return L;
}
// misc: [0] h1 (m+1) ... we keep separate small arrays after misc:
//   misc+0 .. misc+m       : h1 (first-pass coefficients, then column)
//   misc+m+1 .. misc+2m+1  : h2 (second pass)
//   misc+2m+2              : ||w||^2 after the second pass (or first pass)
//   misc+2m+3              : residual estimate |g_{k+1}|
//   misc+2m+4              : status (0 ok, 1 breakdown, 2 nonfinite)
//   misc+2m+5              : beta (initial residual norm)

__global__ void k_init_cycle(double* hs, HLay L, int* kdev) {
  if (threadIdx.x != 0) return;
  *kdev = 0;   // Krylov column of the next preconditioner application
  const double* nrm2 = hs + L.misc + 2 * L.m + 2;
  const double beta = sqrt(*nrm2);
  for (int i = 0; i <= L.m; ++i) hs[L.g + i] = 0.0;
  hs[L.g] = beta;
  hs[L.misc + 2 * L.m + 5] = beta;
  hs[L.misc + 2 * L.m + 3] = beta;
}

// Column k: h = h1 + h2, h_{k+1,k} = ||w||, previous rotations, new rotation.
// refine = 0: no second Gram-Schmidt pass ran, h2 is not read.
__global__ void k_givens(double* hs, HLay L, int k, int* kdev, int refine) {
  if (threadIdx.x != 0) return;
  *kdev = k + 1;
  const int m = L.m;
  double* H = hs + L.H;
  double* cs = hs + L.cs;
  double* sn = hs + L.sn;
  double* g = hs + L.g;
  const double* h1 = hs + L.misc;
  const double* h2 = hs + L.misc + m + 1;
  const double nw = sqrt(hs[L.misc + 2 * m + 2]);
  double* col = H + (int64_t)k * (m + 1);
  for (int i = 0; i <= k; ++i) col[i] = refine ? h1[i] + h2[i] : h1[i];
  col[k + 1] = nw;
  for (int i = 0; i < k; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[k], col[k + 1]);
  double status = 0.0;
  if (!(den > 0.0) || !isfinite(den)) {
    cs[k] = 1.0; sn[k] = 0.0;
    status = isfinite(den) ? 1.0 : 2.0;
  } else {
    cs[k] = col[k] / den;
    sn[k] = col[k + 1] / den;
    col[k] = den;
    col[k + 1] = 0.0;
  }
  g[k + 1] = -sn[k] * g[k];
  g[k] = cs[k] * g[k];
  hs[L.misc + 2 * m + 3] = fabs(g[k + 1]);
  if (nw == 0.0 && status == 0.0) status = 1.0;   // happy breakdown: exact solution in the space
  if (!isfinite(g[k + 1])) status = 2.0;
  hs[L.misc + 2 * m + 4] = status;
}

// Reorthogonalise only when the first Gram-Schmidt pass cancelled more than
// half of the vector (||w_after|| < 0.7 ||w_before||, Daniel-Gragg-Kaufman-
// Stewart); count the passes in misc+2m+7.
// eta2 = 0.49: a second pass when ||w|| fell below 0.7 ||w_0||; eta2 = 2:
// always (||w|| never grows in a pass).
__global__ void k_reorth_flag(double* hs, HLay L, int k, double eta2) {
  if (threadIdx.x != 0) return;
  double* misc = hs + L.misc;
  const double before = misc[k + 1];
  const double after = misc[2 * L.m + 2];
  const double f = (after < eta2 * before) ? 1.0 : 0.0;
  misc[2 * L.m + 6] = f;
  misc[2 * L.m + 7] += f;
}

__global__ void k_backsolve(double* hs, HLay L, int kk) {
  if (threadIdx.x != 0) return;
  const int m = L.m;
  const double* H = hs + L.H;
  const double* g = hs + L.g;
  double* y = hs + L.y;
  for (int i = kk - 1; i >= 0; --i) {
    double s = g[i];
    for (int j = i + 1; j < kk; ++j) s -= H[(int64_t)j * (m + 1) + i] * y[j];
    const double d = H[(int64_t)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// Reduced-mode condensation / back-substitution helpers (per node).
__global__ void k_condense(Grid g, int nc, double tau, const int32_t* __restrict__ eidx,
                           const uint8_t* __restrict__ label, const double* __restrict__ Aj,
                           const double* __restrict__ Mj, const double* __restrict__ betaj,
                           const double* __restrict__ ge, const double* __restrict__ gc,
                           const double* __restrict__ gs, const double* __restrict__ b,
                           const double* __restrict__ yc, double* __restrict__ bm, int trans) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = g.nn;
  if (n >= nn) return;
  const int32_t e = eidx[n];
  double r0 = b[n], r1 = b[nn + n], r2 = b[2 * nn + n];
  if (e >= 0) {
    const bool act = label[n] & kLabActive;
    const double A = Aj[e];
    const double yN = yc[(int64_t)e * nc + nc - 1];
    if (!trans) {
      const double gsv = gs[e];
      if (act) r0 -= A * gsv * yN;
      r1 -= -A * gsv * yN;
      r2 -= -tau * A * gsv * yN;
    } else {
      const double mb = Mj[e] * betaj[e];
      if (act) r0 -= mb * ge[e] * yN;
      r1 -= mb * (-ge[e]) * yN;
      r2 -= mb * gc[e] * yN;
    }
  }
  bm[n] = r0;
  bm[nn + n] = r1;
  bm[2 * nn + n] = r2;
}

__global__ void k_surface_coupling(int64_t NE, double tau, const int32_t* __restrict__ enode, int64_t nn,
                                   const uint8_t* __restrict__ label, const double* __restrict__ Aj,
                                   const double* __restrict__ Mj, const double* __restrict__ betaj,
                                   const double* __restrict__ ge, const double* __restrict__ gc,
                                   const double* __restrict__ gs, const double* __restrict__ xm,
                                   double* __restrict__ tN, int trans) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= NE) return;
  const int64_t n = enode[e];
  const bool act = label[n] & kLabActive;
  if (!trans) {
    tN[e] = Mj[e] * betaj[e] * ((act ? ge[e] * xm[n] : 0.0) - ge[e] * xm[nn + n] + gc[e] * xm[2 * nn + n]);
  } else {
    const double A = Aj[e];
    tN[e] = gs[e] * ((act ? A * xm[n] : 0.0) - A * xm[nn + n] - tau * A * xm[2 * nn + n]);
  }
}

struct Reducer {
  p4d_ctx* c;
  int nblk(int64_t len) const {
    const int64_t want = (len + (int64_t)kRedThreads * 8 - 1) / ((int64_t)kRedThreads * 8);
    return (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, want));
  }
  // out[0..kp1) = V^T w, out[kp1] = w.w (optional)
  // flag (device, optional): the pass runs only if *flag != 0; otherwise out
  // is zeroed (zero_if_skipped) or left unchanged
  void mdot(const double* V, int64_t ldv, int kp1, const double* w, int64_t len, bool ww, double* out,
            const double* flag = nullptr, int zero_if_skipped = 0) {
    const int nb = nblk(len);
    const int ps = 132;
    if (kp1 == 0) launch_group<0>(ww, V, ldv, 0, kp1, w, len, nb, ps, flag);
    for (int g0 = 0; g0 < kp1; g0 += kDotGroup)
      dispatch(std::min(kDotGroup, kp1 - g0), ww && g0 == 0, V, ldv, g0, kp1, w, len, nb, ps, flag);
    ::p4d::count_launch(), k_reduce_partials<<<kp1 + (ww ? 1 : 0), 256, 0, c->stream>>>(c->part, nb, ps, kp1 + (ww ? 1 : 0), out, flag,
                                                                  zero_if_skipped);
  }
  template <int NG>
  void launch_group(bool ww, const double* V, int64_t ldv, int g0, int kp1, const double* w, int64_t len, int nb,
                    int ps, const double* flag) {
    if (ww) ::p4d::count_launch(), k_mdot<NG, true><<<nb, kRedThreads, 0, c->stream>>>(V, ldv, g0, kp1, w, len, c->part, ps, flag);
    else ::p4d::count_launch(), k_mdot<NG, false><<<nb, kRedThreads, 0, c->stream>>>(V, ldv, g0, kp1, w, len, c->part, ps, flag);
  }
  void dispatch(int ng, bool ww, const double* V, int64_t ldv, int g0, int kp1, const double* w, int64_t len, int nb,
                int ps, const double* flag) {
    switch (ng) {
#define P4D_MDOT_CASE(K) \
  case K: launch_group<K>(ww, V, ldv, g0, kp1, w, len, nb, ps, flag); break;
      P4D_MDOT_CASE(1) P4D_MDOT_CASE(2) P4D_MDOT_CASE(3) P4D_MDOT_CASE(4) P4D_MDOT_CASE(5) P4D_MDOT_CASE(6)
      P4D_MDOT_CASE(7) P4D_MDOT_CASE(8) P4D_MDOT_CASE(9) P4D_MDOT_CASE(10) P4D_MDOT_CASE(11) P4D_MDOT_CASE(12)
      P4D_MDOT_CASE(13) P4D_MDOT_CASE(14) P4D_MDOT_CASE(15) P4D_MDOT_CASE(16)
#undef P4D_MDOT_CASE
      default: break;
    }
  }
  // w -= V h over kp1 vectors; with norm_out, also norm_out = ||w_new||^2
  void maxpy(const double* V, int64_t ldv, int kp1, const double* h, double* w, int64_t len, double sign,
             const double* flag, double* norm_out, unsigned gb) {
    ::p4d::count_launch(), k_maxpy<<<gb, kBlock, 0, c->stream>>>(V, ldv, kp1, h, w, len, sign, flag,
                                                               norm_out ? c->part : nullptr);
    if (norm_out)
      ::p4d::count_launch(), k_reduce_partials<<<1, 256, 0, c->stream>>>(c->part, (int)gb, 1, 1, norm_out, flag, 0);
  }
};


}  // namespace

namespace {

// ---------------------------------------------------------------- FGMRES driver
// One solve advanced in phases: a launch phase issues work on c->stream and
// returns; its read phase runs after that stream has been synchronized.  The
// single-cell driver (fgmres) synchronizes after each launch phase; the
// batched driver (fgmres_batched) runs every cell's launch phase, then one
// synchronization for all, then every cell's read phase, with the Arnoldi
// steps of all cells in one graph per Krylov column.

// Status of Arnoldi step k into dst[0..1] (residual estimate, status): the
// batched step graphs gather every cell's pair in one device array.
__global__ void k_put_status(const double* __restrict__ src, double* __restrict__ dst) {
  if (threadIdx.x == 0) {
    dst[0] = src[0];
    dst[1] = src[1];
  }
}

// Condition of a cell's conditional (IF) node in a batched step graph.
__global__ void k_set_active(cudaGraphConditionalHandle h, const int* __restrict__ active) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, *active ? 1u : 0u);
}

// Device gate of a graph-driven restart cycle (in hs after the misc scalars):
// [0] stop, [1] steps run, [2] residual estimate and [3] status of the last
// step, [4] step limit of the cycle, [5] ||s.b_k||, [6] rtol.
constexpr int kGateOff = 48;

__global__ void k_gate(cudaGraphConditionalHandle h, const double* __restrict__ gate, int k) {
  if (threadIdx.x == 0) cudaGraphSetConditional(h, (gate[0] == 0.0 && (double)k < gate[4]) ? 1u : 0u);
}

// After Arnoldi step k (whose estimate and status k_put_status left in
// gate[2..3]): the cycle stops on a breakdown, a non-finite scalar or a
// converged estimate, the same tests the host applies to a step's status.
__global__ void k_step_done(double* gate, int k) {
  if (threadIdx.x != 0) return;
  gate[1] = k + 1;
  if (gate[3] != 0.0 || gate[2] / gate[5] <= gate[6]) gate[0] = 1.0;
}

struct FgRun;
void fg_release(FgRun& r);

struct FgRun {
  p4d_ctx* c = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  int trans = 0;
  bool full = false;
  int64_t nn = 0, len = 0;
  int m = 0;
  HLay L{};
  unsigned gb = 0;
  double tau = 0.0;
  const double* bk = nullptr;   // Krylov right-hand side (unscaled)
  double bnorm = 0.0, est = 1.0;
  int iters = 0, restarts = 0, kk = 0;
  p4d_status st = P4D_ERR_NOT_CONVERGED;
  bool stop = false;            // the solve ended at the start of a restart cycle
  bool cycle_done = true;       // no further Arnoldi step in the current cycle
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double* misc() const { return c->hs + L.misc; }
  bool active() const { return !stop && st == P4D_ERR_NOT_CONVERGED && iters < c->prm.maxit; }
  FgRun() = default;
  FgRun(const FgRun&) = delete;
  FgRun& operator=(const FgRun&) = delete;
  ~FgRun() { fg_release(*this); }   // the timing events, also on an early error return
};

void fg_release(FgRun& r) {
  if (r.ev0) cudaEventDestroy(r.ev0);
  if (r.ev1) cudaEventDestroy(r.ev1);
  r.ev0 = r.ev1 = nullptr;
}

// Field weights of the right-hand side, the particle condensation (REDUCED)
// and the norms of the Krylov right-hand side.
p4d_status fg_begin(FgRun& r, p4d_ctx* c, const double* b, double* x, int trans) {
  r.c = c;
  r.b = b;
  r.x = x;
  r.trans = trans;
  r.nn = c->g.nn;
  r.full = c->prm.mode == 0;
  r.len = r.full ? c->ndof : 3 * r.nn;
  r.m = std::min(c->prm.restart, c->mcap);
  r.L = hlay(c->mcap);
  r.tau = (1.0 - c->prm.tplus) / c->prm.F;
  r.gb = (unsigned)std::min<int64_t>(4 * 152 * 4, (int64_t)nblocks(r.len));
  const HLay& L = r.L;
  double* hs = c->hs;
  prof_reset(c);
  P4D_TRY(cudaEventCreate(&r.ev0));
  P4D_TRY(cudaEventCreate(&r.ev1));
  P4D_TRY(cudaEventRecord(r.ev0, c->stream));
  // per-field weights from the full right-hand side
  {
    const int nb = kRedBlocks;
    ::p4d::count_launch(), k_field_norms<<<nb, kRedThreads, 0, c->stream>>>(b, c->rsqd, r.nn, c->ndof, c->part);
    ::p4d::count_launch(), k_weights<<<1, 128, 0, c->stream>>>(c->part, nb, c->unorm2, 1e-14 / c->prm.rtol, trans,
                                                             c->wf, c->iwf, hs + L.misc + 2 * L.m + 8);
  }
  r.bk = b;
  if (!r.full) {
    // b_m' = b_m - A_mc T^-1 b_c
    P4D_TRYS(particle_solve64(c, b + 3 * r.nn, c->tmp + 3 * r.nn, nullptr, trans));
    ::p4d::count_launch(), k_condense<<<nblocks(r.nn), kBlock, 0, c->stream>>>(
        c->g, c->nc, r.tau, c->eidx, c->label, c->Aj, c->Mj, c->betaj, c->ge, c->gc, c->gs, b, c->tmp + 3 * r.nn,
        c->bred, trans);
    r.bk = c->bred;
  }
  ::p4d::count_launch(), k_field_norms<<<kRedBlocks, kRedThreads, 0, c->stream>>>(r.bk, c->rsqd, r.nn, r.len, c->part);
  ::p4d::count_launch(), k_sum4<<<1, 128, 0, c->stream>>>(c->part, kRedBlocks, hs + L.misc + 2 * L.m + 16);
  P4D_TRY(cudaMemcpyAsync(c->hs_h, hs + L.misc + 2 * L.m + 8, sizeof(double) * 12, cudaMemcpyDeviceToHost, c->stream));
  return P4D_OK;
}

// ||s.b_k|| = sqrt(sum_f w_f^2 ||(b_k / sqrt(d))_f||^2); b_k = 0 gives x = 0.
p4d_status fg_bnorm(FgRun& r) {
  p4d_ctx* c = r.c;
  const double* bn2 = c->hs_h;        // full-b field norms^2 (weights)
  const double* bk2 = c->hs_h + 8;    // Krylov-rhs field norms^2
  double bnorm = 0.0;
  for (int f = 0; f < (r.full ? 4 : 3); ++f) {
    const double wf = bn2[f] > 0 ? 1.0 / std::sqrt(bn2[f]) : 1.0;
    bnorm += wf * wf * bk2[f];
  }
  r.bnorm = std::sqrt(bnorm);
  if (r.bnorm == 0.0) {
    P4D_TRY(cudaMemsetAsync(r.x, 0, sizeof(double) * c->ndof, c->stream));
    r.st = P4D_OK;
    r.est = 0.0;
  }
  P4D_TRY(cudaMemsetAsync(r.misc() + 2 * r.L.m + 7, 0, sizeof(double), c->stream));
  return P4D_OK;
}

// Start of a restart cycle: V0 = s.(b_k - A x), beta = ||V0||, V0 /= beta.
p4d_status fg_cycle_launch(FgRun& r) {
  p4d_ctx* c = r.c;
  Reducer R{c};
  double* misc = r.misc();
  const HLay& L = r.L;
  ++r.restarts;
  if (r.full) P4D_TRYS(jvp_full(c, r.x, c->V, r.trans, r.bk, true));
  else P4D_TRYS(jvp_reduced(c, r.x, c->V, r.trans, r.bk, true));
  R.mdot(c->V, 0, 0, c->V, r.len, true, misc + 2 * L.m + 2);
  ::p4d::count_launch(), k_init_cycle<<<1, 1, 0, c->stream>>>(c->hs, L, c->kdev);
  ::p4d::count_launch(), k_scale<<<r.gb, kBlock, 0, c->stream>>>(c->V, c->V, r.len, misc + 2 * L.m + 5, 1);
  P4D_TRY(cudaMemcpyAsync(c->hs_h, misc + 2 * L.m + 5, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return P4D_OK;
}

void fg_cycle_read(FgRun& r) {
  const double beta = r.c->hs_h[0];
  r.est = beta / r.bnorm;
  r.kk = 0;
  r.cycle_done = false;
  if (!std::isfinite(beta)) {
    r.st = P4D_ERR_NONFINITE;
    r.stop = true;
  } else if (beta <= r.c->prm.rtol * r.bnorm) {
    r.st = P4D_OK;
    r.stop = true;
  }
  if (r.stop) r.cycle_done = true;
}

// Arnoldi step k: z_k = P^-1 (s^-1 v_k), w = s.J z_k, CGS (second pass only
// when needed), Givens, v_{k+1} = w / h_{k+1,k}; the residual estimate and
// status go to the host mirror (stat == nullptr) or to stat[0..1] (device).
p4d_status fg_step_body(FgRun& r, int k, bool graph_precond, double* stat) {
  p4d_ctx* c = r.c;
  Reducer R{c};
  double* misc = r.misc();
  const HLay& L = r.L;
  double* zk = c->Z + (int64_t)k * r.len;
  double* w = c->V + (int64_t)(k + 1) * r.len;
  prof_mark(c, 0);
  P4D_TRYS(precond_column(c, r.trans, graph_precond));   // k read from c->kdev
  prof_mark(c, 0);
  prof_mark(c, 1);
  if (r.full) P4D_TRYS(jvp_full(c, zk, w, r.trans, nullptr, true));
  else P4D_TRYS(jvp_reduced(c, zk, w, r.trans, nullptr, true));
  prof_mark(c, 1);
  prof_mark(c, 2);
  const double* flag = misc + 2 * L.m + 6;
  R.mdot(c->V, r.len, k + 1, w, r.len, true, misc);                                        // h1, ||w||^2 before
  R.maxpy(c->V, r.len, k + 1, misc, w, r.len, 1.0, nullptr, misc + 2 * L.m + 2, r.gb);     // ||w||^2 after
  if (c->prm.cgs_refine > 0) {
    ::p4d::count_launch(), k_reorth_flag<<<1, 1, 0, c->stream>>>(c->hs, L, k, c->prm.cgs_refine == 2 ? 2.0 : 0.49);
    R.mdot(c->V, r.len, k + 1, w, r.len, false, misc + L.m + 1, flag, 1);   // h2 (or 0)
    // ||w||^2 after the second pass (left unchanged when it is skipped)
    R.maxpy(c->V, r.len, k + 1, misc + L.m + 1, w, r.len, 1.0, flag, misc + 2 * L.m + 2, r.gb);
  }
  ::p4d::count_launch(), k_givens<<<1, 1, 0, c->stream>>>(c->hs, L, k, c->kdev, c->prm.cgs_refine);
  ::p4d::count_launch(), k_scale<<<r.gb, kBlock, 0, c->stream>>>(w, w, r.len, misc + 2 * L.m + 2, 2);
  prof_mark(c, 2);
  if (stat) ::p4d::count_launch(), k_put_status<<<1, 32, 0, c->stream>>>(misc + 2 * L.m + 3, stat);
  else P4D_TRY(cudaMemcpyAsync(c->hs_h, misc + 2 * L.m + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return P4D_OK;
}

// s2 = (residual estimate, status) of step k.
void fg_step_read(FgRun& r, int k, const double* s2) {
  ++r.iters;
  r.kk = k + 1;
  r.est = s2[0] / r.bnorm;
  const double stt = s2[1];
  if (stt == 2.0) r.st = P4D_ERR_NONFINITE;
  else if (r.est <= r.c->prm.rtol) r.st = P4D_OK;
  else if (stt == 1.0) r.st = P4D_OK;
  if (r.st != P4D_ERR_NOT_CONVERGED || r.kk >= r.m || r.iters >= r.c->prm.maxit) r.cycle_done = true;
}

// End of a cycle: x += Z y; when the estimate converged, the true residual.
p4d_status fg_cycle_end_launch(FgRun& r) {
  p4d_ctx* c = r.c;
  Reducer R{c};
  double* misc = r.misc();
  const HLay& L = r.L;
  if (r.kk > 0) {
    ::p4d::count_launch(), k_backsolve<<<1, 1, 0, c->stream>>>(c->hs, L, r.kk);
    // x += Z y  (k_maxpy computes w -= sum h_i V_i; use sign -1)
    R.maxpy(c->Z, r.len, r.kk, c->hs + L.y, r.x, r.len, -1.0, nullptr, nullptr, r.gb);
  }
  if (r.st == P4D_OK) {
    if (r.full) P4D_TRYS(jvp_full(c, r.x, c->V, r.trans, r.bk, true));
    else P4D_TRYS(jvp_reduced(c, r.x, c->V, r.trans, r.bk, true));
    R.mdot(c->V, 0, 0, c->V, r.len, true, misc + 2 * L.m + 2);
    P4D_TRY(cudaMemcpyAsync(c->hs_h, misc + 2 * L.m + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  return P4D_OK;
}

// Confirmation by the true residual (only after st == OK was launched).
void fg_cycle_end_read(FgRun& r) {
  if (r.st != P4D_OK) return;
  r.est = std::sqrt(r.c->hs_h[0]) / r.bnorm;
  if (!(r.est <= r.c->prm.rtol) && r.iters < r.c->prm.maxit) r.st = P4D_ERR_NOT_CONVERGED;
  if (!std::isfinite(r.est)) r.st = P4D_ERR_NONFINITE;
}

// Particle back-substitution (REDUCED) and the final true residual.
p4d_status fg_finish_launch(FgRun& r) {
  p4d_ctx* c = r.c;
  const HLay& L = r.L;
  const int64_t nn = r.nn;
  if (!r.full) {
    // x_c = T^-1 (b_c - A_cm x_m)
    ::p4d::count_launch(), k_surface_coupling<<<nblocks(std::max<int64_t>(1, c->NE)), kBlock, 0, c->stream>>>(
        c->NE, r.tau, c->enode, nn, c->label, c->Aj, c->Mj, c->betaj, c->ge, c->gc, c->gs, r.x, c->tloc, r.trans);
    P4D_TRYS(particle_solve64(c, r.b + 3 * nn, r.x + 3 * nn, c->tloc, r.trans));
  }
  // final true residual of the full system in the scaled norm
  P4D_TRYS(jvp_full(c, r.x, c->r0, r.trans, r.b, true));
  ::p4d::count_launch(), k_field_norms_plain<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->r0, nn, c->ndof, c->part);
  ::p4d::count_launch(), k_sum4<<<1, 128, 0, c->stream>>>(c->part, kRedBlocks, r.misc() + 2 * L.m + 24);
  // and unscaled: ||(b - J x)_f||^2 = ||(sqrt(d) r0)_f||^2 / w_f^2, ||b_f||^2
  ::p4d::count_launch(), k_field_norms<<<kRedBlocks, kRedThreads, 0, c->stream>>>(c->r0, c->sqd, nn, c->ndof, c->part);
  ::p4d::count_launch(), k_sum4<<<1, 128, 0, c->stream>>>(c->part, kRedBlocks, r.misc() + 2 * L.m + 32);
  ::p4d::count_launch(), k_field_norms_plain<<<kRedBlocks, kRedThreads, 0, c->stream>>>(r.b, nn, c->ndof, c->part);
  ::p4d::count_launch(), k_sum4<<<1, 128, 0, c->stream>>>(c->part, kRedBlocks, r.misc() + 2 * L.m + 36);
  P4D_TRY(cudaEventRecord(r.ev1, c->stream));
  P4D_TRY(cudaMemcpyAsync(c->hs_h, r.misc() + 2 * L.m + 7, sizeof(double) * 33, cudaMemcpyDeviceToHost, c->stream));
  return P4D_OK;
}

void fg_finish_read(FgRun& r, p4d_info* info) {
  p4d_ctx* c = r.c;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, r.ev0, r.ev1);
  fg_release(r);
  if (!info) return;
  std::memset(info, 0, sizeof(*info));
  info->iters = r.iters;
  info->restarts = r.restarts;
  info->status = r.st;
  info->reorth = (int)c->hs_h[0];
  const double* bn2 = c->hs_h + 1;      // field norms^2 of b/sqd (weights: 1/sqrt)
  const double* rr = c->hs_h + 17;      // field norms^2 of s.(b - Jx)
  double tot_r = 0.0;
  const double tot_b = bn2[4];          // ||s.b||^2
  for (int f = 0; f < 4; ++f) {
    info->rel_res_block[f] = std::sqrt(rr[f]);   // relative to the field's (floored) rhs norm
    tot_r += rr[f];
  }
  info->rel_res = tot_b > 0 ? std::sqrt(tot_r / tot_b) : std::sqrt(tot_r);
  const double* ru = c->hs_h + 25;      // field norms^2 of sqrt(d) s.(b - Jx)
  const double* bu = c->hs_h + 29;      // field norms^2 of b
  double ur = 0.0, ub = 0.0;
  for (int f = 0; f < 4; ++f) {
    const double rf = ru[f] * (bn2[f] > 0 ? bn2[f] : 1.0);   // 1 / w_f^2
    info->rel_res_block_unscaled[f] = bu[f] > 0 ? std::sqrt(rf / bu[f]) : std::sqrt(rf);
    ur += rf;
    ub += bu[f];
  }
  info->rel_res_unscaled = ub > 0 ? std::sqrt(ur / ub) : std::sqrt(ur);
  info->nsolves = 1;
  info->iters_total = r.iters;
  info->ms_total = ms;
  if (c->prm.profile) {
    int n = 0;
    info->ms_precond = prof_sum(c, 0, nullptr);
    info->ms_jvp = prof_sum(c, 1, &n);
    info->n_jvp = n;
    info->ms_ortho = prof_sum(c, 2, nullptr);
    info->ms_smooth0 = prof_sum(c, 3, &n);
    info->n_smooth0 = n;
  }
}

// What body() launches on c->stream, captured into a new (not instantiated)
// graph; kernels = its kernel launches.
template <typename F>
p4d_status capture_body(p4d_ctx* c, cudaGraph_t* out, long long* kernels, F&& body) {
  cudaStream_t user = c->stream;
  c->stream = c->cap_stream;
  *kernels = 0;
  capture_counter(kernels);
  *out = nullptr;
  p4d_status st = P4D_OK;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = P4D_ERR_CUDA;
  if (st == P4D_OK) {
    st = body();
    if (cudaStreamEndCapture(c->cap_stream, out) != cudaSuccess && st == P4D_OK) st = P4D_ERR_CUDA;
  }
  capture_counter(nullptr);
  c->stream = user;
  if (st != P4D_OK) {
    cudaGetLastError();
    if (*out) cudaGraphDestroy(*out);
    *out = nullptr;
  }
  return st;
}

// The restart cycle of r as one graph: for k < m, gate(k) -> IF { Arnoldi
// step k; its status into the gate }.
p4d_status cycle_graph(FgRun& r, p4d_ctx::CycleGraph*& out) {
  p4d_ctx* c = r.c;
  p4d_ctx::CycleGraph& cg = c->cyc[r.trans ? 1 : 0][r.full ? 1 : 0];
  out = &cg;
  if (cg.exec && cg.m == r.m) return P4D_OK;
  if (cg.exec) cudaGraphExecDestroy(cg.exec);
  cg.exec = nullptr;
  cg.kernels.assign(r.m, 0);
  double* gate = r.misc() + 2 * r.L.m + kGateOff;
  cudaGraph_t G = nullptr;
  P4D_TRY(cudaGraphCreate(&G, 0));
  p4d_status st = P4D_OK;
  cudaGraphNode_t prev = nullptr;
  for (int k = 0; k < r.m && st == P4D_OK; ++k) {
    cudaGraph_t step = nullptr;
    long long kc = 0;
    st = capture_body(c, &step, &kc, [&]() -> p4d_status {
      P4D_TRYS(fg_step_body(r, k, false, gate + 2));
      ::p4d::count_launch(), k_step_done<<<1, 32, 0, c->stream>>>(gate, k);
      return P4D_OK;
    });
    if (st != P4D_OK) break;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t kn = nullptr, cn = nullptr, ch = nullptr;
    const double* gc = gate;
    int kk = k;
    void* args[] = {&h, &gc, &kk};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_gate;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    if (cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault) != cudaSuccess ||
        cudaGraphAddKernelNode(&kn, G, prev ? &prev : nullptr, prev ? 1 : 0, &kp) != cudaSuccess)
      st = P4D_ERR_CUDA;
    cp.conditional.handle = h;
    if (st == P4D_OK && cudaGraphAddNode(&cn, G, &kn, nullptr, 1, &cp) != cudaSuccess) st = P4D_ERR_CUDA;
    if (st == P4D_OK && cudaGraphAddChildGraphNode(&ch, cp.conditional.phGraph_out[0], nullptr, 0, step) != cudaSuccess)
      st = P4D_ERR_CUDA;
    cudaGraphDestroy(step);
    prev = cn;
    cg.kernels[k] = kc;
  }
  if (st == P4D_OK && cudaGraphInstantiate(&cg.exec, G, 0) != cudaSuccess) st = P4D_ERR_CUDA;
  cudaGraphDestroy(G);
  if (st != P4D_OK) {
    cudaGetLastError();
    cg.exec = nullptr;
    return st;
  }
  cg.m = r.m;
  return P4D_OK;
}

// The Arnoldi steps of one restart cycle by its graph: the host uploads the
// gate, launches the graph, and reads the gate once at the end.
p4d_status fg_cycle_steps_graph(FgRun& r) {
  p4d_ctx* c = r.c;
  p4d_ctx::CycleGraph* cg = nullptr;
  P4D_TRYS(cycle_graph(r, cg));
  double* gate = r.misc() + 2 * r.L.m + kGateOff;
  double* stage = c->hs_h + kGateOff;
  stage[0] = 0.0;
  stage[1] = 0.0;
  stage[2] = 0.0;
  stage[3] = 0.0;
  stage[4] = (double)std::min(r.m, c->prm.maxit - r.iters);
  stage[5] = r.bnorm;
  stage[6] = c->prm.rtol;
  P4D_TRY(cudaMemcpyAsync(gate, stage, 7 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  P4D_TRY(cudaGraphLaunch(cg->exec, c->stream));
  P4D_TRY(cudaMemcpyAsync(c->hs_h, gate, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  P4D_TRY(cudaStreamSynchronize(c->stream));
  const int nrun = (int)c->hs_h[1];
  long long launched = cg->m;
  for (int k = 0; k < nrun; ++k) launched += cg->kernels[k];
  count_launches(launched);
  if (nrun < 1) return P4D_ERR_CUDA;   // the first step always runs (limit >= 1, no stop)
  const double s2[2] = {c->hs_h[2], c->hs_h[3]};
  r.iters += nrun - 1;
  fg_step_read(r, nrun - 1, s2);
  return P4D_OK;
}

}  // namespace

p4d_status fgmres(p4d_ctx* c, const double* b, double* x, p4d_info* info, int trans) {
  FgRun r;
  P4D_TRYS(fg_begin(r, c, b, x, trans));
  P4D_TRY(cudaStreamSynchronize(c->stream));
  P4D_TRYS(fg_bnorm(r));
  while (r.active()) {
    P4D_TRYS(fg_cycle_launch(r));
    P4D_TRY(cudaStreamSynchronize(c->stream));
    fg_cycle_read(r);
    if (r.stop) break;
    if (c->prm.profile) {
      // per-kernel events cannot sit inside a graph: step by step
      for (int k = 0; !r.cycle_done; ++k) {
        P4D_TRYS(fg_step_body(r, k, true, nullptr));
        P4D_TRY(cudaStreamSynchronize(c->stream));
        fg_step_read(r, k, c->hs_h);
      }
    } else {
      P4D_TRYS(fg_cycle_steps_graph(r));
    }
    P4D_TRYS(fg_cycle_end_launch(r));
    if (r.st == P4D_ERR_NONFINITE) break;
    if (r.st == P4D_OK) {
      P4D_TRY(cudaStreamSynchronize(c->stream));
      fg_cycle_end_read(r);
    }
  }
  P4D_TRYS(fg_finish_launch(r));
  P4D_TRY(cudaStreamSynchronize(c->stream));
  fg_finish_read(r, info);
  return r.st;
}

// ---------------------------------------------------------------- batched driver
namespace {


// The batched graph of Krylov column k: for every cell whose restart length
// exceeds k, set_active(cell) -> IF(cell active) { Arnoldi step k of the
// cell }.  The cells' chains are independent nodes, so the GPU runs them
// concurrently.
p4d_status batch_step_graph(p4d_batch_ctx* B, std::vector<FgRun>& R, int k, int trans) {
  auto& vec = B->gk[trans ? 1 : 0];
  if ((int)vec.size() <= k) vec.resize(k + 1);
  p4d_batch_ctx::StepGraph& sg = vec[k];
  if (sg.exec) return P4D_OK;
  const int n = (int)B->cells.size();
  sg.kernels.assign(n, 0);
  cudaGraph_t G = nullptr;
  P4D_TRY(cudaGraphCreate(&G, 0));
  p4d_status st = P4D_OK;
  for (int i = 0; i < n && st == P4D_OK; ++i) {
    FgRun& r = R[i];
    if (k >= r.m) continue;
    cudaGraph_t step = nullptr;
    long long kc = 0;
    st = capture_body(r.c, &step, &kc, [&]() { return fg_step_body(r, k, false, B->stat_dev + 2 * i); });
    if (st != P4D_OK) break;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t kn = nullptr, cn = nullptr, ch = nullptr;
    const int* act = B->active_dev + i;
    void* args[] = {&h, &act};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_set_active;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    if (cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault) != cudaSuccess ||
        cudaGraphAddKernelNode(&kn, G, nullptr, 0, &kp) != cudaSuccess)
      st = P4D_ERR_CUDA;
    cp.conditional.handle = h;
    if (st == P4D_OK && cudaGraphAddNode(&cn, G, &kn, nullptr, 1, &cp) != cudaSuccess) st = P4D_ERR_CUDA;
    if (st == P4D_OK && cudaGraphAddChildGraphNode(&ch, cp.conditional.phGraph_out[0], nullptr, 0, step) != cudaSuccess)
      st = P4D_ERR_CUDA;
    cudaGraphDestroy(step);
    sg.kernels[i] = kc;
  }
  if (st == P4D_OK && cudaGraphInstantiate(&sg.exec, G, 0) != cudaSuccess) st = P4D_ERR_CUDA;
  cudaGraphDestroy(G);
  if (st != P4D_OK) {
    cudaGetLastError();
    sg.exec = nullptr;
  }
  return st;
}

p4d_status sync_cells(p4d_batch_ctx* B) {
  for (size_t i = 0; i < B->cells.size(); ++i) {
    bool seen = false;
    for (size_t j = 0; j < i && !seen; ++j) seen = B->cells[j]->stream == B->cells[i]->stream;
    if (!seen) P4D_TRY(cudaStreamSynchronize(B->cells[i]->stream));
  }
  return P4D_OK;
}

}  // namespace

void batch_drop_graphs(p4d_batch_ctx* B) {
  for (auto& v : B->gk) {
    for (auto& g : v)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    v.clear();
  }
}

p4d_status fgmres_batched(p4d_batch_ctx* B, const double* const* b, double* const* x, p4d_info* info, int trans) {
  const int n = (int)B->cells.size();
  // step graphs captured before a cell's options changed are stale
  bool stale = (int)B->gen.size() != n;
  for (int i = 0; i < n && !stale; ++i) stale = B->gen[i] != B->cells[i]->graph_gen;
  if (stale) {
    batch_drop_graphs(B);
    B->gen.resize(n);
    for (int i = 0; i < n; ++i) B->gen[i] = B->cells[i]->graph_gen;
  }
  std::vector<FgRun> R(n);
  for (int i = 0; i < n; ++i) P4D_TRYS(fg_begin(R[i], B->cells[i], b[i], x[i], trans));
  P4D_TRYS(sync_cells(B));
  for (int i = 0; i < n; ++i) P4D_TRYS(fg_bnorm(R[i]));
  std::vector<int> cyc;
  while (true) {
    cyc.clear();
    for (int i = 0; i < n; ++i)
      if (R[i].active()) cyc.push_back(i);
    if (cyc.empty()) break;
    for (int i : cyc) P4D_TRYS(fg_cycle_launch(R[i]));
    P4D_TRYS(sync_cells(B));
    for (int i : cyc) fg_cycle_read(R[i]);
    // Arnoldi steps in lockstep; a cell leaves the cycle when its step says so
    for (int k = 0;; ++k) {
      bool any = false;
      for (int i = 0; i < n; ++i) {
        const bool a = !R[i].cycle_done && k < R[i].m;
        B->active_h[i] = a ? 1 : 0;
        any = any || a;
      }
      if (!any) break;
      P4D_TRYS(batch_step_graph(B, R, k, trans));
      const p4d_batch_ctx::StepGraph& sg = B->gk[trans ? 1 : 0][k];
      long long launched = 0;
      for (int i = 0; i < n; ++i)
        if (sg.kernels[i] > 0) launched += 1 + (B->active_h[i] ? sg.kernels[i] : 0);
      count_launches(launched);
      P4D_TRY(cudaMemcpyAsync(B->active_dev, B->active_h, sizeof(int) * n, cudaMemcpyHostToDevice, B->stream));
      P4D_TRY(cudaGraphLaunch(sg.exec, B->stream));
      P4D_TRY(cudaMemcpyAsync(B->stat_h, B->stat_dev, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, B->stream));
      P4D_TRY(cudaStreamSynchronize(B->stream));
      for (int i = 0; i < n; ++i)
        if (B->active_h[i]) fg_step_read(R[i], k, B->stat_h + 2 * i);
    }
    bool confirm = false;
    for (int i : cyc)
      if (!R[i].stop) {
        P4D_TRYS(fg_cycle_end_launch(R[i]));
        confirm = confirm || R[i].st == P4D_OK;
      }
    if (confirm) {
      P4D_TRYS(sync_cells(B));
      for (int i : cyc)
        if (!R[i].stop) fg_cycle_end_read(R[i]);
    }
  }
  for (int i = 0; i < n; ++i) P4D_TRYS(fg_finish_launch(R[i]));
  P4D_TRYS(sync_cells(B));
  p4d_status out = P4D_OK;
  for (int i = 0; i < n; ++i) {
    fg_finish_read(R[i], info ? info + i : nullptr);
    if (out == P4D_OK && R[i].st != P4D_OK) out = R[i].st;
  }
  return out;
}

// ---------------------------------------------------------------- slab-decomposed driver
// FGMRES over the z slabs of one cell (REDUCED mode, J x = b).  Every slab
// runs the single-cell steps on its own rows.  The Krylov vectors keep their
// ghost rows at zero, so an inner product is the allreduce of the slabs'
// partial sums, and every slab repeats the Givens update on the same reduced
// scalars (identical on all slabs).  The operator is the cell's J: before
// each application the ghost planes of its input receive the owners' values.
// The preconditioner of a slab is its own block preconditioner on the slab
// (block Jacobi across the slabs).
p4d_status fgmres_dd(p4d_dd_ctx* D, const double* const* b, double* const* x, p4d_info* info) {
  const int P = (int)D->parts.size();
  std::vector<FgRun> R(P);
  std::vector<double*> ptr(P), vec(P);
  auto reduce = [&](auto&& at, int n) -> p4d_status {
    for (int p = 0; p < P; ++p) ptr[p] = at(R[p]);
    return dd_allreduce(D, ptr.data(), n);
  };
  auto at_off = [](int64_t mult2m, int64_t add) {
    return [=](FgRun& r) { return r.misc() + mult2m * r.L.m + add; };
  };
  p4d_ctx* c0 = D->parts[0];
  FgRun& r0 = R[0];
  const int refine = c0->prm.cgs_refine;
  for (int p = 0; p < P; ++p) {
    FgRun& r = R[p];
    p4d_ctx* c = D->parts[p];
    r.c = c;
    r.b = D->bw[p];
    r.x = x[p];
    r.trans = 0;
    r.nn = c->g.nn;
    r.full = false;
    r.len = 3 * r.nn;
    r.m = std::min(c->prm.restart, c->mcap);
    r.L = hlay(c->mcap);
    r.tau = (1.0 - c->prm.tplus) / c->prm.F;
    r.gb = (unsigned)std::min<int64_t>(4 * 152 * 4, (int64_t)nblocks(r.len));
    prof_reset(c);
  }
  P4D_TRY(cudaEventCreate(&r0.ev0));
  P4D_TRY(cudaEventCreate(&r0.ev1));
  P4D_TRY(cudaEventRecord(r0.ev0, D->stream));
  // the right-hand side without its ghost rows
  for (int p = 0; p < P; ++p) {
    P4D_TRY(cudaMemcpyAsync(D->bw[p], b[p], sizeof(double) * D->parts[p]->ndof, cudaMemcpyDeviceToDevice, D->stream));
    P4D_TRYS(dd_zero_ghost(D, p, D->bw[p], true));
  }
  // field weights of the whole cell's right-hand side
  for (int p = 0; p < P; ++p) {
    p4d_ctx* c = D->parts[p];
    ::p4d::count_launch(), k_field_norms<<<kRedBlocks, kRedThreads, 0, D->stream>>>(D->bw[p], c->rsqd, R[p].nn, c->ndof,
                                                                                   c->part);
    ::p4d::count_launch(), k_sum4<<<1, 128, 0, D->stream>>>(c->part, kRedBlocks, R[p].misc() + 2 * R[p].L.m + 8);
  }
  P4D_TRYS(reduce(at_off(2, 8), 4));
  for (int p = 0; p < P; ++p) {
    p4d_ctx* c = D->parts[p];
    double* s4 = R[p].misc() + 2 * R[p].L.m + 8;
    ::p4d::count_launch(), k_weights_sums<<<1, 32, 0, D->stream>>>(s4, c->unorm2, 1e-14 / c->prm.rtol, c->wf, c->iwf, s4);
  }
  // particle condensation (node-local) and the norms of the Krylov right-hand side
  for (int p = 0; p < P; ++p) {
    FgRun& r = R[p];
    p4d_ctx* c = r.c;
    P4D_TRYS(particle_solve64(c, r.b + 3 * r.nn, c->tmp + 3 * r.nn, nullptr, 0));
    ::p4d::count_launch(), k_condense<<<nblocks(r.nn), kBlock, 0, D->stream>>>(
        c->g, c->nc, r.tau, c->eidx, c->label, c->Aj, c->Mj, c->betaj, c->ge, c->gc, c->gs, r.b, c->tmp + 3 * r.nn,
        c->bred, 0);
    r.bk = c->bred;
    ::p4d::count_launch(), k_field_norms<<<kRedBlocks, kRedThreads, 0, D->stream>>>(r.bk, c->rsqd, r.nn, r.len, c->part);
    ::p4d::count_launch(), k_sum4<<<1, 128, 0, D->stream>>>(c->part, kRedBlocks, r.misc() + 2 * r.L.m + 16);
  }
  P4D_TRYS(reduce(at_off(2, 16), 4));
  P4D_TRY(cudaMemcpyAsync(c0->hs_h, r0.misc() + 2 * r0.L.m + 8, sizeof(double) * 12, cudaMemcpyDeviceToHost, D->stream));
  P4D_TRY(cudaStreamSynchronize(D->stream));
  for (int p = 0; p < P; ++p) {
    if (p > 0) std::memcpy(D->parts[p]->hs_h, c0->hs_h, sizeof(double) * 12);
    P4D_TRYS(fg_bnorm(R[p]));
  }
  auto share_host = [&](int n) {
    for (int p = 1; p < P; ++p) std::memcpy(D->parts[p]->hs_h, c0->hs_h, sizeof(double) * n);
  };
  // V_0 = s.(b_k - J x), ||V_0|| and the true residual use the same sequence
  auto residual_norm = [&]() -> p4d_status {
    P4D_TRYS(dd_halo(D, x, false));
    for (int p = 0; p < P; ++p) {
      p4d_ctx* c = D->parts[p];
      P4D_TRYS(jvp_reduced(c, x[p], c->V, 0, R[p].bk, true));
      P4D_TRYS(dd_zero_ghost(D, p, c->V, false));
      Reducer{c}.mdot(c->V, 0, 0, c->V, R[p].len, true, R[p].misc() + 2 * R[p].L.m + 2);
    }
    return reduce(at_off(2, 2), 1);
  };
  while (r0.active()) {
    P4D_TRYS(residual_norm());
    for (int p = 0; p < P; ++p) {
      FgRun& r = R[p];
      p4d_ctx* c = r.c;
      ++r.restarts;
      ::p4d::count_launch(), k_init_cycle<<<1, 1, 0, D->stream>>>(c->hs, r.L, c->kdev);
      ::p4d::count_launch(), k_scale<<<r.gb, kBlock, 0, D->stream>>>(c->V, c->V, r.len, r.misc() + 2 * r.L.m + 5, 1);
    }
    P4D_TRY(cudaMemcpyAsync(c0->hs_h, r0.misc() + 2 * r0.L.m + 5, sizeof(double), cudaMemcpyDeviceToHost, D->stream));
    P4D_TRY(cudaStreamSynchronize(D->stream));
    share_host(1);
    for (int p = 0; p < P; ++p) fg_cycle_read(R[p]);
    if (r0.stop) break;
    for (int k = 0; !r0.cycle_done; ++k) {
      // z_k = P_slab^-1 (s^-1 v_k), then the owners' values in its ghost planes
      // restricted additive Schwarz: every slab preconditions v_k on its
      // owned and ghost rows (the owners' values) and keeps its owned rows.
      // With a single ghost plane, whose rows miss the elements beyond the
      // slab, its rows stay zero (block Jacobi across the slabs): fed the
      // owners' residual there the iteration counts grow several times.
      for (int p = 0; p < P; ++p) {
        vec[p] = D->parts[p]->Z + (int64_t)k * R[p].len;
        ptr[p] = D->parts[p]->V + (int64_t)k * R[p].len;
      }
      if (D->ghosts > 1) P4D_TRYS(dd_halo(D, ptr.data(), true));
      for (int p = 0; p < P; ++p) {
        P4D_TRYS(precond_column(D->parts[p], 0, true));
        P4D_TRYS(dd_zero_ghost(D, p, ptr[p], false));
      }
      // two-level: z_k += Z A_c^-1 Z^T (s^-1 v_k)
      {
        std::vector<const double*> vk(ptr.begin(), ptr.end());
        P4D_TRYS(dd_coarse_correct(D, vk.data(), vec.data()));
      }
      P4D_TRYS(dd_halo(D, vec.data(), false));
      // w = s.J z_k on the owned rows; h = V^T w, ||w||^2
      for (int p = 0; p < P; ++p) {
        p4d_ctx* c = D->parts[p];
        double* w = c->V + (int64_t)(k + 1) * R[p].len;
        P4D_TRYS(jvp_reduced(c, vec[p], w, 0, nullptr, true));
        P4D_TRYS(dd_zero_ghost(D, p, w, false));
        Reducer{c}.mdot(c->V, R[p].len, k + 1, w, R[p].len, true, R[p].misc());
      }
      P4D_TRYS(reduce(at_off(0, 0), k + 2));
      for (int p = 0; p < P; ++p) {
        p4d_ctx* c = D->parts[p];
        FgRun& r = R[p];
        Reducer{c}.maxpy(c->V, r.len, k + 1, r.misc(), c->V + (int64_t)(k + 1) * r.len, r.len, 1.0, nullptr,
                         r.misc() + 2 * r.L.m + 2, r.gb);
      }
      P4D_TRYS(reduce(at_off(2, 2), 1));
      if (refine > 0) {
        // second pass, decided on every slab from the same reduced norms
        for (int p = 0; p < P; ++p) {
          p4d_ctx* c = D->parts[p];
          FgRun& r = R[p];
          const double* flag = r.misc() + 2 * r.L.m + 6;
          ::p4d::count_launch(), k_reorth_flag<<<1, 1, 0, D->stream>>>(c->hs, r.L, k, refine == 2 ? 2.0 : 0.49);
          Reducer{c}.mdot(c->V, r.len, k + 1, c->V + (int64_t)(k + 1) * r.len, r.len, false, r.misc() + r.L.m + 1,
                          flag, 1);
        }
        P4D_TRYS(reduce(at_off(1, 1), k + 1));
        for (int p = 0; p < P; ++p) {
          p4d_ctx* c = D->parts[p];
          FgRun& r = R[p];
          const double* flag = r.misc() + 2 * r.L.m + 6;
          ::p4d::count_launch(), k_maxpy<<<r.gb, kBlock, 0, D->stream>>>(c->V, r.len, k + 1, r.misc() + r.L.m + 1,
                                                                         c->V + (int64_t)(k + 1) * r.len, r.len, 1.0,
                                                                         flag, c->part);
          ::p4d::count_launch(), k_reduce_partials<<<1, 256, 0, D->stream>>>(c->part, (int)r.gb, 1, 1,
                                                                             r.misc() + 2 * r.L.m + 44, flag, 1);
        }
        P4D_TRYS(reduce(at_off(2, 44), 1));
        for (int p = 0; p < P; ++p)
          ::p4d::count_launch(), k_take_if<<<1, 32, 0, D->stream>>>(R[p].misc() + 2 * R[p].L.m + 2,
                                                                    R[p].misc() + 2 * R[p].L.m + 44,
                                                                    R[p].misc() + 2 * R[p].L.m + 6);
      }
      for (int p = 0; p < P; ++p) {
        p4d_ctx* c = D->parts[p];
        FgRun& r = R[p];
        double* w = c->V + (int64_t)(k + 1) * r.len;
        ::p4d::count_launch(), k_givens<<<1, 1, 0, D->stream>>>(c->hs, r.L, k, c->kdev, refine);
        ::p4d::count_launch(), k_scale<<<r.gb, kBlock, 0, D->stream>>>(w, w, r.len, r.misc() + 2 * r.L.m + 2, 2);
      }
      P4D_TRY(cudaMemcpyAsync(c0->hs_h, r0.misc() + 2 * r0.L.m + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                              D->stream));
      P4D_TRY(cudaStreamSynchronize(D->stream));
      for (int p = 0; p < P; ++p) fg_step_read(R[p], k, c0->hs_h);
    }
    // x += Z y on every slab (the same y)
    for (int p = 0; p < P; ++p) {
      FgRun& r = R[p];
      p4d_ctx* c = r.c;
      if (r.kk > 0) {
        ::p4d::count_launch(), k_backsolve<<<1, 1, 0, D->stream>>>(c->hs, r.L, r.kk);
        Reducer{c}.maxpy(c->Z, r.len, r.kk, c->hs + r.L.y, r.x, r.len, -1.0, nullptr, nullptr, r.gb);
      }
    }
    if (r0.st == P4D_ERR_NONFINITE) break;
    if (r0.st == P4D_OK) {
      P4D_TRYS(residual_norm());
      P4D_TRY(cudaMemcpyAsync(c0->hs_h, r0.misc() + 2 * r0.L.m + 2, sizeof(double), cudaMemcpyDeviceToHost,
                              D->stream));
      P4D_TRY(cudaStreamSynchronize(D->stream));
      share_host(1);
      for (int p = 0; p < P; ++p) fg_cycle_end_read(R[p]);
    }
  }
  // particle back-substitution, then the true residual of the full system
  for (int p = 0; p < P; ++p) {
    FgRun& r = R[p];
    p4d_ctx* c = r.c;
    ::p4d::count_launch(), k_surface_coupling<<<nblocks(std::max<int64_t>(1, c->NE)), kBlock, 0, D->stream>>>(
        c->NE, r.tau, c->enode, r.nn, c->label, c->Aj, c->Mj, c->betaj, c->ge, c->gc, c->gs, r.x, c->tloc, 0);
    P4D_TRYS(particle_solve64(c, r.b + 3 * r.nn, r.x + 3 * r.nn, c->tloc, 0));
  }
  P4D_TRYS(dd_halo(D, x, false));
  for (int p = 0; p < P; ++p) {
    FgRun& r = R[p];
    p4d_ctx* c = r.c;
    double* m = r.misc() + 2 * r.L.m;
    P4D_TRYS(jvp_full(c, r.x, c->r0, 0, r.b, true));
    P4D_TRYS(dd_zero_ghost(D, p, c->r0, true));
    ::p4d::count_launch(), k_field_norms_plain<<<kRedBlocks, kRedThreads, 0, D->stream>>>(c->r0, r.nn, c->ndof, c->part);
    ::p4d::count_launch(), k_sum4<<<1, 128, 0, D->stream>>>(c->part, kRedBlocks, m + 24);
    ::p4d::count_launch(), k_field_norms<<<kRedBlocks, kRedThreads, 0, D->stream>>>(c->r0, c->sqd, r.nn, c->ndof, c->part);
    ::p4d::count_launch(), k_sum4<<<1, 128, 0, D->stream>>>(c->part, kRedBlocks, m + 32);
    ::p4d::count_launch(), k_field_norms_plain<<<kRedBlocks, kRedThreads, 0, D->stream>>>(r.b, r.nn, c->ndof, c->part);
    ::p4d::count_launch(), k_sum4<<<1, 128, 0, D->stream>>>(c->part, kRedBlocks, m + 36);
  }
  P4D_TRYS(reduce(at_off(2, 24), 4));
  P4D_TRYS(reduce(at_off(2, 32), 8));
  P4D_TRY(cudaEventRecord(r0.ev1, D->stream));
  P4D_TRY(cudaMemcpyAsync(c0->hs_h, r0.misc() + 2 * r0.L.m + 7, sizeof(double) * 33, cudaMemcpyDeviceToHost, D->stream));
  P4D_TRY(cudaStreamSynchronize(D->stream));
  fg_finish_read(r0, info);
  return r0.st;
}

}  // namespace p4d
