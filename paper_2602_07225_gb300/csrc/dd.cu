// Slab domain decomposition of one cell along z (the partitioning the
// paper's strong and weak scaling studies, section 5, run over MPI ranks):
// one handle per slab, consecutive slabs sharing one element layer, so that
// every interior interface has one ghost node plane on either side.  A
// stencil application (the JVP) needs the owners' values in the ghost
// planes (the halo exchange: pack on the owner, one transfer per message,
// unpack on the receiver); every inner product is a sum of the slabs'
// owned-row partial sums (the allreduce).  Here all slabs live on one GPU
// and one stream: a transfer is a device-to-device copy and the allreduce
// gathers the slabs' partial sums by copies, adds them in slab order and
// copies the sum back to every slab, which is what a send/recv pair and an
// allreduce over ranks do with one slab per rank.
#include <algorithm>
#include <cstring>
#include <new>

#include "p4d_common.cuh"

namespace p4d {
namespace {

constexpr int kDDThreads = 256;
constexpr int kDDBlocks = 2 * 152;

// buf[f][j] = x[f nn + off + j] (w: times w at the same row), j < len,
// f = phi_s, phi_e, c_e
__global__ void k_dd_pack(const double* __restrict__ x, const double* __restrict__ w, int64_t nn, int64_t off,
                          int64_t len, double* __restrict__ buf) {
  const int64_t n = 3 * len;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / len, row = f * nn + off + (i - f * len);
    buf[i] = w ? x[row] * w[row] : x[row];
  }
}

__global__ void k_dd_unpack(double* __restrict__ x, const double* __restrict__ w, int64_t nn, int64_t off,
                            int64_t len, const double* __restrict__ buf) {
  const int64_t n = 3 * len;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = i / len, row = f * nn + off + (i - f * len);
    x[row] = w ? buf[i] * w[row] : buf[i];
  }
}

// Zero the ghost rows of a slab vector: node rows [0, lo) and [hi, nn) of
// fields 0..2, and (cs_rows) the particle rows [3nn, 3nn + cs_lo nc) and
// [3nn + cs_hi nc, 3nn + ne nc) of the ghost planes' electrode nodes.
__global__ void k_dd_zero_ghost(double* __restrict__ v, int64_t nn, int64_t lo, int64_t hi, int cs_rows,
                                int64_t cs_lo, int64_t cs_hi, int64_t ne, int nc) {
  const int64_t nlo = lo, nhi = nn - hi;
  const int64_t nodes = 3 * (nlo + nhi);
  const int64_t clo = cs_rows ? cs_lo * nc : 0, chi = cs_rows ? (ne - cs_hi) * nc : 0;
  const int64_t total = nodes + clo + chi;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nodes) {
      const int64_t f = i / (nlo + nhi), j = i - f * (nlo + nhi);
      v[f * nn + (j < nlo ? j : hi + (j - nlo))] = 0.0;
    } else {
      const int64_t q = i - nodes;
      v[3 * nn + (q < clo ? q : cs_hi * nc + (q - clo))] = 0.0;
    }
  }
}

// Owned-row sums of squares of up to four ranges, (v w)^2 (w = null: 1),
// as block partials partial[block][4].
struct DDRanges {
  const double* v[4];
  const double* w[4];
  int64_t n[4];
};

__global__ void __launch_bounds__(kDDThreads) k_dd_sumsq(DDRanges r, double* __restrict__ partial) {
  double acc[4];
#pragma unroll
  for (int f = 0; f < 4; ++f)
    acc[f] = r.n[f] <= 0 ? 0.0 : (r.w[f] ? sumsq_share<true>(r.v[f], r.w[f], r.n[f])
                                         : sumsq_share<false>(r.v[f], nullptr, r.n[f]));
  block_sum4(acc, partial);
}

__global__ void k_dd_sum_blocks(const double* __restrict__ partial, int nblk, double* out) {
  sum4_warps(partial, nblk, out);
}

// out[i] = sum over slabs p (in order) of red[p n + i]
__global__ void k_dd_sum(const double* __restrict__ red, int nparts, int n, double* __restrict__ out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += red[(int64_t)p * n + i];
    out[i] = s;
  }
}

// Coarse bin of owned node n of field f (-1: phi_s not an unknown there):
// 2 g for the constant mode, 2 g + 1 for the linear one; g = 0 phi_s anode,
// 1 phi_s cathode, 2 phi_e, 3 c_e.
__device__ __forceinline__ int coarse_group(int f, uint8_t lab) {
  if (f > 0) return f + 1;
  if (!(lab & kLabActive)) return -1;
  return (lab & kLabAnode) ? 0 : 1;
}

// zeta of local node plane k among the owned planes [lo, hi): the cell
// centres of [-1, 1] cut into hi - lo equal parts
__device__ __forceinline__ double coarse_zeta(int k, int lo, int hi) {
  return (2.0 * (k - lo) + 1.0) / (double)(hi - lo) - 1.0;
}

// Block partials [block][8] of the coarse sums of a slab vector (fields
// 0..2): bin 2g += u, bin 2g + 1 += u zeta, u = v (sqd iwf_f when scaled:
// the unscaled s^-1 v of the Krylov space).
__global__ void __launch_bounds__(kDDThreads) k_dd_crestrict(const double* __restrict__ v,
                                                             const double* __restrict__ sqd,
                                                             const double* __restrict__ iwf,
                                                             const uint8_t* __restrict__ label, int64_t nn,
                                                             int64_t nxy, int lo, int hi,
                                                             double* __restrict__ partial) {
  double acc[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) acc[b] = 0.0;
  const int64_t nown = (int64_t)(hi - lo) * nxy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nown;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(i / nown);
    const int64_t n = (int64_t)lo * nxy + (i - f * nown);
    const int g = coarse_group(f, label[n]);
    if (g < 0) continue;
    const int64_t row = f * nn + n;
    const double u = sqd ? v[row] * sqd[row] * iwf[f] : v[row];
    const double z = coarse_zeta((int)(n / nxy), lo, hi);
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
      const bool on = gg == g;
      acc[2 * gg] += on ? u : 0.0;
      acc[2 * gg + 1] += on ? u * z : 0.0;
    }
  }
  double a4[4] = {acc[0], acc[1], acc[2], acc[3]};
  block_sum4(a4, partial);
  __syncthreads();
  double b4[4] = {acc[4], acc[5], acc[6], acc[7]};
  block_sum4(b4, partial + 4 * gridDim.x);
}

// bins[map[b]] = sum of the block partials of bin b (the other entries zero)
__global__ void k_dd_cbins(const double* __restrict__ partial, int nblk, const int* __restrict__ map, int nb,
                           double* __restrict__ bins) {
  __shared__ double s8[8];
  sum4_warps(partial, nblk, s8);
  sum4_warps(partial + 4 * nblk, nblk, s8 + 4);
  __syncthreads();
  for (int j = threadIdx.x; j < nb; j += blockDim.x) bins[j] = 0.0;
  __syncthreads();
  if (threadIdx.x < 8 && map[threadIdx.x] >= 0) bins[map[threadIdx.x]] = s8[threadIdx.x];
}

// y = A^-1 bins (dense nb x nb, column-major), one block
__global__ void k_dd_capply(const double* __restrict__ ainv, const double* __restrict__ bins, int nb,
                            double* __restrict__ y) {
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nb; ++j) s = fma(ainv[(int64_t)j * nb + i], bins[j], s);
    y[i] = s;
  }
}

// z += sum_b y[map[b]] basis_b over the slab's owned nodes (fields 0..2)
__global__ void k_dd_cprolong(double* __restrict__ z, const double* __restrict__ y, const int* __restrict__ map,
                              const uint8_t* __restrict__ label, int64_t nn, int64_t nxy, int lo, int hi) {
  const int64_t nown = (int64_t)(hi - lo) * nxy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nown;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(i / nown);
    const int64_t n = (int64_t)lo * nxy + (i - f * nown);
    const int g = coarse_group(f, label[n]);
    if (g < 0) continue;
    const int j0 = map[2 * g], j1 = map[2 * g + 1];
    double add = j0 >= 0 ? y[j0] : 0.0;
    if (j1 >= 0) add += y[j1] * coarse_zeta((int)(n / nxy), lo, hi);
    z[f * nn + n] += add;
  }
}

__global__ void k_dd_unit(double* __restrict__ y, int nb, int j) {
  for (int i = threadIdx.x; i < nb; i += blockDim.x) y[i] = i == j ? 1.0 : 0.0;
}

}  // namespace

p4d_status dd_halo(p4d_dd_ctx* D, double* const* v, bool scaled) {
  const int nmsg = (int)D->plan.size() / 4;
  const int64_t nxy = D->nxy, len = (int64_t)D->ghosts * nxy;
  const unsigned gb = std::min<unsigned>(nblocks(3 * len), 4 * 152);
  for (int m = 0; m < nmsg; ++m) {
    const int* q = &D->plan[4 * m];
    p4d_ctx* s = D->parts[q[0]];
    ::p4d::count_launch(), k_dd_pack<<<gb, kBlock, 0, D->stream>>>(v[q[0]], scaled ? s->sqd : nullptr, s->g.nn,
                                                                  q[1] * nxy, len, D->sbuf + m * 3 * len);
  }
  for (int m = 0; m < nmsg; ++m)
    P4D_TRY(cudaMemcpyAsync(D->rbuf + m * 3 * len, D->sbuf + m * 3 * len, sizeof(double) * 3 * len,
                            cudaMemcpyDeviceToDevice, D->stream));
  for (int m = 0; m < nmsg; ++m) {
    const int* q = &D->plan[4 * m];
    p4d_ctx* d = D->parts[q[2]];
    ::p4d::count_launch(), k_dd_unpack<<<gb, kBlock, 0, D->stream>>>(v[q[2]], scaled ? d->rsqd : nullptr, d->g.nn,
                                                                    q[3] * nxy, len, D->rbuf + m * 3 * len);
  }
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status dd_zero_ghost(p4d_dd_ctx* D, int p, double* v, bool cs_rows) {
  p4d_ctx* c = D->parts[p];
  const int64_t lo = (int64_t)D->own_lo[p] * D->nxy, hi = (int64_t)D->own_hi[p] * D->nxy;
  const int64_t rows = 3 * (lo + c->g.nn - hi) + (cs_rows ? (D->cs_lo[p] + c->NE - D->cs_hi[p]) * c->nc : 0);
  if (rows == 0) return P4D_OK;
  ::p4d::count_launch(), k_dd_zero_ghost<<<std::min<int64_t>(nblocks(rows), 4 * 152), kBlock, 0, D->stream>>>(
      v, c->g.nn, lo, hi, cs_rows ? 1 : 0, D->cs_lo[p], D->cs_hi[p], c->NE, c->nc);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status dd_allreduce(p4d_dd_ctx* D, double* const* ptrs, int n) {
  const int P = (int)D->parts.size();
  if (n <= 0) return P4D_OK;
  if (n > kDDRed) return P4D_ERR_INVALID_ARG;
  for (int p = 0; p < P; ++p)
    P4D_TRY(cudaMemcpyAsync(D->red + (int64_t)p * n, ptrs[p], sizeof(double) * n, cudaMemcpyDeviceToDevice,
                            D->stream));
  double* sum = D->red + (int64_t)P * kDDRed;
  ::p4d::count_launch(), k_dd_sum<<<1, 128, 0, D->stream>>>(D->red, P, n, sum);
  for (int p = 0; p < P; ++p)
    P4D_TRY(cudaMemcpyAsync(ptrs[p], sum, sizeof(double) * n, cudaMemcpyDeviceToDevice, D->stream));
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

// Owned-row sums of squares of (v w) per field of slab p: v laid out as the
// full system (fields 0..2 at f nn, particles at 3 nn), w the same layout
// or null; out[0..3] on the device.
p4d_status dd_owned_sumsq(p4d_dd_ctx* D, int p, const double* const* v, const double* w, double* out) {
  p4d_ctx* c = D->parts[p];
  const int64_t nn = c->g.nn, lo = (int64_t)D->own_lo[p] * D->nxy, hi = (int64_t)D->own_hi[p] * D->nxy;
  DDRanges r{};
  for (int f = 0; f < 3; ++f) {
    r.v[f] = v[f] + lo;
    r.w[f] = w ? w + f * nn + lo : nullptr;
    r.n[f] = hi - lo;
  }
  r.v[3] = v[3] ? v[3] + D->cs_lo[p] * c->nc : nullptr;
  r.w[3] = w ? w + 3 * nn + D->cs_lo[p] * c->nc : nullptr;
  r.n[3] = v[3] ? (D->cs_hi[p] - D->cs_lo[p]) * c->nc : 0;
  ::p4d::count_launch(), k_dd_sumsq<<<kDDBlocks, kDDThreads, 0, D->stream>>>(r, D->part);
  ::p4d::count_launch(), k_dd_sum_blocks<<<1, 128, 0, D->stream>>>(D->part, kDDBlocks, out);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

namespace {

// Coarse sums of slab p's vector v into row p of D->bins (scaled: of s^-1 v).
p4d_status dd_coarse_sums(p4d_dd_ctx* D, int p, const double* v, bool scaled) {
  p4d_ctx* c = D->parts[p];
  ::p4d::count_launch(), k_dd_crestrict<<<kDDBlocks, kDDThreads, 0, D->stream>>>(
      v, scaled ? c->sqd : nullptr, c->iwf, c->label, c->g.nn, D->nxy, D->own_lo[p], D->own_hi[p], D->cpart);
  ::p4d::count_launch(), k_dd_cbins<<<1, 128, 0, D->stream>>>(D->cpart, kDDBlocks, D->cmap_dev + 8 * p, D->nb,
                                                             D->bins + (int64_t)p * kDDRed);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

p4d_status dd_bins_allreduce(p4d_dd_ctx* D) {
  const int P = (int)D->parts.size();
  std::vector<double*> ptr(P);
  for (int p = 0; p < P; ++p) ptr[p] = D->bins + (int64_t)p * kDDRed;
  return dd_allreduce(D, ptr.data(), D->nb);
}

p4d_status dd_prolong(p4d_dd_ctx* D, int p, const double* y, double* z) {
  p4d_ctx* c = D->parts[p];
  const int64_t n = 3 * (int64_t)(D->own_hi[p] - D->own_lo[p]) * D->nxy;
  ::p4d::count_launch(), k_dd_cprolong<<<std::min<int64_t>(nblocks(n), 4 * 152), kBlock, 0, D->stream>>>(
      z, y, D->cmap_dev + 8 * p, c->label, c->g.nn, D->nxy, D->own_lo[p], D->own_hi[p]);
  P4D_TRY(cudaGetLastError());
  return P4D_OK;
}

// Inverse of the dense n x n column-major matrix a by Gauss-Jordan
// elimination with partial pivoting (FP64); false when a pivot vanishes.
bool dense_inverse(std::vector<double>& a, int n, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  auto A = [&](int i, int j) -> double& { return a[(size_t)j * n + i]; };
  auto I = [&](int i, int j) -> double& { return inv[(size_t)j * n + i]; };
  double amax = 0.0;
  for (double v : a) amax = std::max(amax, std::fabs(v));
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A(i, k)) > std::fabs(A(piv, k))) piv = i;
    if (!(std::fabs(A(piv, k)) > 1e-14 * amax)) return false;
    if (piv != k)
      for (int j = 0; j < n; ++j) {
        std::swap(A(k, j), A(piv, j));
        std::swap(I(k, j), I(piv, j));
      }
    const double d = 1.0 / A(k, k);
    for (int j = 0; j < n; ++j) {
      A(k, j) *= d;
      I(k, j) *= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = A(i, k);
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A(i, j) -= f * A(k, j);
        I(i, j) -= f * I(k, j);
      }
    }
  }
  return true;
}

// The coarse basis of the current linearization and A_c = Z^T J Z (REDUCED
// operator, unscaled), inverted on the host in FP64 and kept on the device.
p4d_status dd_coarse_build(p4d_dd_ctx* D) {
  const int P = (int)D->parts.size();
  D->nb = 0;
  if (D->coarse_modes == 0 || P < 2) return P4D_OK;
  // groups present on each slab (phi_s anode / cathode unknowns among the owned nodes)
  D->cmap.assign(8 * (size_t)P, -1);
  int nb = 0;
  for (int p = 0; p < P; ++p) {
    p4d_ctx* c = D->parts[p];
    std::vector<uint8_t> lab((size_t)c->g.nn);
    P4D_TRY(cudaMemcpy(lab.data(), c->label, lab.size(), cudaMemcpyDeviceToHost));
    bool has[4] = {false, false, true, true};
    for (int64_t n = (int64_t)D->own_lo[p] * D->nxy; n < (int64_t)D->own_hi[p] * D->nxy; ++n)
      if (lab[n] & kLabActive) has[(lab[n] & kLabAnode) ? 0 : 1] = true;
    const bool lin = D->coarse_modes >= 2 && D->own_hi[p] - D->own_lo[p] >= 2;
    for (int g = 0; g < 4; ++g) {
      if (!has[g]) continue;
      D->cmap[8 * p + 2 * g] = nb++;
      if (lin) D->cmap[8 * p + 2 * g + 1] = nb++;
    }
  }
  if (nb > kDDRed) return P4D_ERR_INVALID_ARG;   // cannot happen: at most 8 per slab, at most 32 slabs
  P4D_TRY(cudaMemcpyAsync(D->cmap_dev, D->cmap.data(), sizeof(int) * 8 * P, cudaMemcpyHostToDevice, D->stream));
  D->nb = nb;
  std::vector<double> ac((size_t)nb * nb), inv;
  for (int j = 0; j < nb; ++j) {
    // W = J Z_j over the slabs (halo exchange first), then Z^T W
    for (int p = 0; p < P; ++p) {
      p4d_ctx* c = D->parts[p];
      P4D_TRY(cudaMemsetAsync(D->wx[p], 0, sizeof(double) * 3 * c->g.nn, D->stream));
      ::p4d::count_launch(), k_dd_unit<<<1, 128, 0, D->stream>>>(D->cy + (int64_t)p * kDDRed, nb, j);
      P4D_TRYS(dd_prolong(D, p, D->cy + (int64_t)p * kDDRed, D->wx[p]));
    }
    P4D_TRYS(dd_halo(D, D->wx.data(), false));
    for (int p = 0; p < P; ++p) {
      P4D_TRYS(jvp_reduced(D->parts[p], D->wx[p], D->wy[p], 0, nullptr, false));
      P4D_TRYS(dd_zero_ghost(D, p, D->wy[p], false));
      P4D_TRYS(dd_coarse_sums(D, p, D->wy[p], false));
    }
    P4D_TRYS(dd_bins_allreduce(D));
    P4D_TRY(cudaMemcpyAsync(ac.data() + (size_t)j * nb, D->bins, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                            D->stream));
  }
  P4D_TRY(cudaStreamSynchronize(D->stream));
  if (!dense_inverse(ac, nb, inv)) {
    D->nb = 0;   // singular coarse matrix: one-level (block Jacobi) preconditioner
    return P4D_OK;
  }
  P4D_TRY(cudaMemcpyAsync(D->ainv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, D->stream));
  P4D_TRY(cudaStreamSynchronize(D->stream));
  return P4D_OK;
}

}  // namespace

p4d_status dd_coarse_correct(p4d_dd_ctx* D, const double* const* v, double* const* z) {
  if (D->nb == 0) return P4D_OK;
  const int P = (int)D->parts.size();
  for (int p = 0; p < P; ++p) P4D_TRYS(dd_coarse_sums(D, p, v[p], true));
  P4D_TRYS(dd_bins_allreduce(D));
  for (int p = 0; p < P; ++p) {
    double* y = D->cy + (int64_t)p * kDDRed;
    ::p4d::count_launch(), k_dd_capply<<<1, 256, 0, D->stream>>>(D->ainv, D->bins + (int64_t)p * kDDRed, D->nb, y);
    P4D_TRYS(dd_prolong(D, p, y, z[p]));
  }
  return P4D_OK;
}

// The slabs' kernels run on the current device with the slabs' memory.
bool dd_on_device(const p4d_dd_ctx* D) { return on_device(D->parts[0]); }

}  // namespace p4d

using namespace p4d;

extern "C" {

int32_t p4d_dd_halo_plan(int32_t nparts, const int32_t* nplanes, int32_t ghosts, int32_t* plan) {
  if (nparts < 1 || !nplanes || ghosts < 1) return -1;
  for (int p = 0; p < nparts; ++p) {
    const int ng = ghosts * ((p > 0) + (p < nparts - 1));
    // owned planes: at least one, and as many as a neighbour's ghost planes
    const int own = nplanes[p] - ng;
    if (own < 1 || (nparts > 1 && own < ghosts)) return -1;
  }
  int m = 0;
  for (int p = 0; p + 1 < nparts; ++p) {
    if (plan) {
      // the upper slab's lowest ghost planes <- the lower slab's last owned planes
      plan[4 * m + 0] = p; plan[4 * m + 1] = nplanes[p] - 2 * ghosts; plan[4 * m + 2] = p + 1; plan[4 * m + 3] = 0;
      // the lower slab's highest ghost planes <- the upper slab's first owned planes
      plan[4 * m + 4] = p + 1; plan[4 * m + 5] = ghosts; plan[4 * m + 6] = p; plan[4 * m + 7] = nplanes[p] - ghosts;
    }
    m += 2;
  }
  return m;
}

p4d_status p4d_dd_create(const p4d_handle* parts, int32_t nparts, int32_t ghosts, p4d_dd* out) {
  if (!out) return P4D_ERR_INVALID_ARG;
  *out = nullptr;
  if (!parts || nparts < 1 || nparts > 32) return P4D_ERR_INVALID_ARG;
  for (int i = 0; i < nparts; ++i) {
    if (!parts[i]) return P4D_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (parts[j] == parts[i]) return P4D_ERR_INVALID_ARG;
    const p4d_ctx* a = parts[0];
    const p4d_ctx* b = parts[i];
    if (b->device != a->device || b->stream != a->stream || b->g.nnx != a->g.nnx || b->g.nny != a->g.nny ||
        b->nc != a->nc)
      return P4D_ERR_INVALID_ARG;
  }
  std::vector<int32_t> nz1(nparts);
  for (int i = 0; i < nparts; ++i) nz1[i] = parts[i]->g.nnz;
  const int nmsg = p4d_dd_halo_plan(nparts, nz1.data(), ghosts, nullptr);
  if (nmsg < 0) return P4D_ERR_INVALID_ARG;
  p4d_dd_ctx* D = new (std::nothrow) p4d_dd_ctx;
  if (!D) return P4D_ERR_OOM;
  D->parts.assign(parts, parts + nparts);
  D->stream = parts[0]->stream;
  D->nxy = (int64_t)parts[0]->g.nnx * parts[0]->g.nny;
  D->plan.assign(4 * (size_t)nmsg, 0);
  D->ghosts = ghosts;
  p4d_dd_halo_plan(nparts, nz1.data(), ghosts, D->plan.data());
  for (int p = 0; p < nparts; ++p) {
    const p4d_ctx* c = parts[p];
    D->own_lo.push_back(p > 0 ? ghosts : 0);
    D->own_hi.push_back(p < nparts - 1 ? nz1[p] - ghosts : nz1[p]);
    // electrode nodes are numbered in node order, so a slab's owned ones are
    // one contiguous range of its list
    const int64_t lo = (int64_t)D->own_lo[p] * D->nxy, hi = (int64_t)D->own_hi[p] * D->nxy;
    const auto& en = c->enodes_h;
    D->cs_lo.push_back(std::lower_bound(en.begin(), en.end(), (int32_t)lo) - en.begin());
    D->cs_hi.push_back(std::lower_bound(en.begin(), en.end(), (int32_t)hi) - en.begin());
  }
  p4d_status st = P4D_OK;
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (cudaSetDevice(parts[0]->device) != cudaSuccess) st = P4D_ERR_CUDA;
  const size_t msg = (size_t)std::max(nmsg, 1) * 3 * ghosts * D->nxy;
  if (st == P4D_OK &&
      (cudaMalloc(&D->sbuf, sizeof(double) * msg) != cudaSuccess ||
       cudaMalloc(&D->rbuf, sizeof(double) * msg) != cudaSuccess ||
       cudaMalloc(&D->red, sizeof(double) * (size_t)(nparts + 1) * kDDRed) != cudaSuccess ||
       cudaMalloc(&D->part, sizeof(double) * 4 * kDDBlocks) != cudaSuccess ||
       cudaMalloc(&D->cpart, sizeof(double) * 8 * kDDBlocks) != cudaSuccess ||
       cudaMalloc(&D->cmap_dev, sizeof(int) * 8 * (size_t)nparts) != cudaSuccess ||
       cudaMalloc(&D->bins, sizeof(double) * (size_t)nparts * kDDRed) != cudaSuccess ||
       cudaMalloc(&D->cy, sizeof(double) * (size_t)nparts * kDDRed) != cudaSuccess ||
       cudaMalloc(&D->ainv, sizeof(double) * (size_t)kDDRed * kDDRed) != cudaSuccess))
    st = P4D_ERR_OOM;
  for (int p = 0; p < nparts && st == P4D_OK; ++p) {
    double *b = nullptr, *wx = nullptr, *wy = nullptr;
    const size_t n3 = 3 * (size_t)parts[p]->g.nn;
    if (cudaMalloc(&b, sizeof(double) * (size_t)parts[p]->ndof) != cudaSuccess ||
        cudaMalloc(&wx, sizeof(double) * n3) != cudaSuccess || cudaMalloc(&wy, sizeof(double) * n3) != cudaSuccess)
      st = P4D_ERR_OOM;
    D->bw.push_back(b);
    D->wx.push_back(wx);
    D->wy.push_back(wy);
  }
  if (dev_prev >= 0) cudaSetDevice(dev_prev);
  if (st != P4D_OK) {
    cudaGetLastError();
    p4d_dd_destroy(D);
    return st;
  }
  *out = D;
  return P4D_OK;
}

void p4d_dd_destroy(p4d_dd D) {
  if (!D) return;
  if (D->sbuf) cudaFree(D->sbuf);
  if (D->rbuf) cudaFree(D->rbuf);
  if (D->red) cudaFree(D->red);
  for (void* q : {(void*)D->part, (void*)D->cpart, (void*)D->cmap_dev, (void*)D->bins, (void*)D->cy,
                  (void*)D->ainv})
    if (q) cudaFree(q);
  for (auto* v : {&D->bw, &D->wx, &D->wy})
    for (double* b : *v)
      if (b) cudaFree(b);
  delete D;
}

p4d_status p4d_dd_jacobian_update(p4d_dd D, const p4d_state* states) {
  if (!D || !states) return P4D_ERR_INVALID_ARG;
  if (!dd_on_device(D)) return P4D_ERR_INVALID_ARG;
  const int P = (int)D->parts.size();
  for (int p = 0; p < P; ++p) P4D_TRYS(p4d_jacobian_update(D->parts[p], &states[p]));
  // the norm floor of the Krylov weights uses ||sqrt(d) u_f|| of the whole
  // cell: owned rows of every slab, summed over the slabs
  std::vector<double*> ptr(P);
  for (int p = 0; p < P; ++p) {
    const double* v[4] = {states[p].phis, states[p].phie, states[p].ce, states[p].cs};
    P4D_TRYS(dd_owned_sumsq(D, p, v, D->parts[p]->sqd, D->parts[p]->unorm2));
    ptr[p] = D->parts[p]->unorm2;
  }
  P4D_TRYS(dd_allreduce(D, ptr.data(), 4));
  P4D_TRYS(dd_coarse_build(D));
  P4D_TRY(cudaStreamSynchronize(D->stream));
  return P4D_OK;
}

p4d_status p4d_dd_set_coarse(p4d_dd D, int32_t modes) {
  if (!D || modes < 0 || modes > 2) return P4D_ERR_INVALID_ARG;
  D->coarse_modes = modes;
  D->nb = 0;   // rebuilt by the next p4d_dd_jacobian_update
  return P4D_OK;
}

p4d_status p4d_dd_jvp(p4d_dd D, double* const* x, double* const* y) {
  if (!D || !x || !y) return P4D_ERR_INVALID_ARG;
  if (!dd_on_device(D)) return P4D_ERR_INVALID_ARG;
  const int P = (int)D->parts.size();
  for (int p = 0; p < P; ++p)
    if (!x[p] || !y[p] || x[p] == y[p] || !D->parts[p]->linearized) return P4D_ERR_INVALID_ARG;
  P4D_TRYS(dd_halo(D, x, false));
  for (int p = 0; p < P; ++p) {
    P4D_TRYS(jvp_full(D->parts[p], x[p], y[p], 0, nullptr, false));
    P4D_TRYS(dd_zero_ghost(D, p, y[p], true));
  }
  return P4D_OK;
}

p4d_status p4d_dd_fgmres_solve(p4d_dd D, const double* const* b, double* const* x, p4d_info* info) {
  if (!D || !b || !x) return P4D_ERR_INVALID_ARG;
  if (!dd_on_device(D)) return P4D_ERR_INVALID_ARG;
  const int P = (int)D->parts.size();
  const p4d_params& p0 = D->parts[0]->prm;
  for (int p = 0; p < P; ++p) {
    const p4d_ctx* c = D->parts[p];
    if (!b[p] || !x[p] || b[p] == x[p] || !c->linearized || c->prm.profile || c->prm.mode != 1) return P4D_ERR_INVALID_ARG;
    if (c->prm.rtol != p0.rtol || c->prm.restart != p0.restart || c->prm.maxit != p0.maxit ||
        c->prm.cgs_refine != p0.cgs_refine)
      return P4D_ERR_INVALID_ARG;
  }
  return fgmres_dd(D, b, x, info);
}

}  // extern "C"
