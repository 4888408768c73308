// Internal declarations shared by the CUDA translation units of libp4d.
//
// Data layout in device memory (one handle = one cell):
//   node arrays      [nn]            x fastest (node (i,j,k) -> i + nnx*(j + nny*k))
//   element arrays   [nelem]
//   stencils         [27][nn]        SoA by offset o = (dx+1) + 3(dy+1) + 9(dz+1)
//   electrode nodes  [NE]            SoA per quantity, c_s vectors [NE][nc]
//   Krylov basis     [m+1][len]      FP64
// Multigrid stencils are kept in "difference form": slot 13 (the centre)
// holds the row sum s_n, the other 26 slots the off-diagonal entries, so that
// (A x)_n = sum_{o != 13} A_o (x_{n+o} - x_n) + s_n x_n.  The row sums carry
// the reaction/Schur terms that anchor the near-constant modes of the
// potential blocks; keeping them apart keeps those modes exact in FP32/BF16.
#pragma once
#include <cmath>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include "p4d.h"

#define P4D_TRY(x)                                   \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return P4D_ERR_CUDA;      \
  } while (0)

#define P4D_TRYS(x)                                  \
  do {                                               \
    p4d_status s_ = (x);                             \
    if (s_ != P4D_OK) return s_;                     \
  } while (0)

namespace p4d {

constexpr int kMaxNc = 32;
constexpr int kMaxDeg = 16;        // Chebyshev degree limit
constexpr int kMaxLevels = 16;
constexpr int kNH = 4;            // multigrid hierarchies: phi_s anode, phi_s cathode, phi_e, c_e
constexpr int kBlock = 256;

// device error flags (bits)
enum : unsigned {
  kFlagDomain = 1u,
  kFlagNonfinite = 2u,
};

// Node label bits
enum : uint8_t {
  kLabAnode = 1,       // node of an anode element
  kLabCathode = 2,     // node of a cathode element
  kLabDirichlet = 4,   // node of a grounded face (z = 0, gamma_n)
  kLabActive = 8,      // phi_s unknown (electrode node, not grounded)
};

// Small POD bundles passed to kernels by value.
struct Grid {
  int nnx, nny, nnz;
  int64_t nn;
};

template <typename T>
struct Ptr4 {
  T* p[kNH];
};

// Entry h of a per-hierarchy kernel-parameter array.  Indexing such an array
// with a run-time index makes the compiler copy the parameter block to the
// thread's stack; selecting among the four constant-index reads does not.
template <typename T>
__device__ __forceinline__ T pk(const T (&a)[kNH], int h) {
  return h == 0 ? a[0] : (h == 1 ? a[1] : (h == 2 ? a[2] : a[3]));
}

// One-dimensional interpolation tables between a fine node line and its
// coarsening (see mg.cu): per fine node up to two parents, per coarse node
// up to three support nodes, with weights.
struct Axis {
  const int* par;      // [nf][2] parent coarse nodes (-1: none)
  const double* parw;  // [nf][2]
  const int* sup;      // [nc][3] support fine nodes (-1: none)
  const double* supw;  // [nc][3]
  const float* parwf;  // FP32 copies of parw and supw (the weights are exact in FP32)
  const float* supwf;
};

// Interpolation weight tables in the precision T of a computation.
template <typename T> __device__ __forceinline__ const T* parw_t(const Axis& a);
template <typename T> __device__ __forceinline__ const T* supw_t(const Axis& a);
template <> __device__ __forceinline__ const double* parw_t<double>(const Axis& a) { return a.parw; }
template <> __device__ __forceinline__ const float* parw_t<float>(const Axis& a) { return a.parwf; }
template <> __device__ __forceinline__ const double* supw_t<double>(const Axis& a) { return a.supw; }
template <> __device__ __forceinline__ const float* supw_t<float>(const Axis& a) { return a.supwf; }
struct Xfer {
  Axis a[3];
};

struct MGLevel {
  int nnx = 0, nny = 0, nnz = 0;
  int64_t n = 0;
  int cx = 0, cy = 0, cz = 0;          // coarsen flags towards the next level
  Xfer X{};                            // interpolation tables towards the next level
  // FP64 fixed (linearization independent) operator, difference form [kNH][27][n]
  double* Ffix = nullptr;
  // linearization-dependent part (levels >= 1), difference form [kNH][27][n]:
  // FP64 for the FP64 preconditioner, FP32 otherwise
  void* Vvar = nullptr;
  // stencil in storage precision [kNH][27][n] (level 0: hierarchies 0/1 alias field phi_s)
  void* st[kNH] = {nullptr, nullptr, nullptr, nullptr};
  void* dinv[kNH] = {};                // [n] in compute precision
  uint8_t* mask[kNH] = {};             // [n]
  void* x[kNH] = {};                   // [n] compute precision (level 0: 0/1 alias)
  void* x2[kNH] = {};                  // double buffer
  void* b[kNH] = {};
  void* r[kNH] = {};
  void* d[kNH] = {};
  double* lam = nullptr;               // [kNH] Gershgorin bound of D^-1 A
  // stencil-kernel blocks holding rows of each hierarchy's mask: blocks
  // [blo, blo + bcnt) (set at planning; the masks do not change)
  int blo[kNH] = {};
  int bcnt[kNH] = {};
  // coarsest level only: dense inverse [kNH][n][n] FP64 (+ scratch), LU row permutation
  double* inv = nullptr;
  int* perm = nullptr;
};

}  // namespace p4d

struct p4d_ctx {
  // sizes
  int nx = 0, ny = 0, nz = 0;
  double len[3] = {0.0, 0.0, 0.0};     // axis lengths (element sizes summed in order)
  p4d::Grid g{};
  int64_t nelem = 0, NE = 0, ndof = 0;
  int nc = 0;
  p4d_params prm{};
  cudaStream_t stream = nullptr;
  int device = -1;                     // CUDA device current at p4d_setup (the handle's memory lives there)
  bool linearized = false;
  std::vector<int32_t> enodes_h;
  double scale_f[3] = {1, 1, 1};       // multigrid per-field scaling (FP32 range)
  double shell_p = 0.0, shell_n = 0.0; // collector-foil surface conductances on z = Lz / z = 0 (S)

  // owned allocations (freed in destroy)
  std::vector<void*> allocs;

  // mesh (device)
  double *hx = nullptr, *hy = nullptr, *hz = nullptr;
  uint8_t* label = nullptr;            // [nn]
  int32_t* eidx = nullptr;             // [nn] electrode index or -1
  int32_t* enode = nullptr;            // [NE] node index
  double* gpw = nullptr;               // [nn] Gamma_p lumped face weights
  double* Mj = nullptr;                // [NE] lumped electrode volume
  double* iMj = nullptr;               // [NE] 1 / Mj
  double* Aj = nullptr;                // [NE] 3 S_j / R_j
  double* kapj = nullptr;              // [NE] D_s / R_s^2
  double* betaj = nullptr;             // [NE] flux factor of eq. LR
  uint8_t* etype = nullptr;            // [NE] 0 anode, 1 cathode
  double* rref = nullptr;              // [3][nc] reference radial operator (R = D = 1): lo, di, up
  double beta_ref = 0.0;               // surface flux factor for R = 1
  uint8_t* region = nullptr;           // [nelem]
  double* eps_e = nullptr;             // [nelem] porosity
  double* epss_e = nullptr;            // [nelem] active-material fraction
  double* sig_e = nullptr;             // [nelem] bulk solid conductivity (region constants if not given)
  double* Rj = nullptr;                // [NE] particle radius
  double* nwork = nullptr;             // [4][ndof] Newton work (residual, step, trial state, trial residual)
  double gp_area = 0.0;                // area of Gamma_p
  double* nrm4 = nullptr;              // [4] device scratch for Newton field norms

  // fixed FP64 stencils [4][27][nn]: 0 K_sigma (lifted), 1 K_kappa, 2 C = M_eps/dt + K_D, 3 M_eps/dt
  double* Jst = nullptr;
  double* sfix = nullptr;              // [3][nn] fixed multigrid row sums per field
  double* offsum = nullptr;            // [3][nn] sum of the fixed off-diagonal entries per field
  double* absoff = nullptr;            // [3][nn] sum of their absolute values

  // linearization
  double* lnce = nullptr;              // [nn] ln c_e
  double* lnce_r = nullptr;            // [nn] ln c_e at the state of a residual evaluation
  double* rin = nullptr;               // [NE] i_n at the state of a residual evaluation
  double* gdc = nullptr;               // [nn] gamma / c_e
  double* in_ = nullptr;               // [NE] reaction current
  double* ge = nullptr;                // [NE]
  double* gc = nullptr;
  double* gs = nullptr;
  double* zj = nullptr;                // [NE] (T_j^-1)_NN
  double* zeta = nullptr;              // [NE] 1 - z_j g_s M_j beta_j
  double* tfac = nullptr;              // [2][nc][NE] LU of T_j/M_j: 1/pivot, multiplier
  double* tqfix = nullptr;             // [NE] last pivot of T_j/M_j without the surface term
  float* tfac32 = nullptr;             // FP32 copy of tfac (FP32 preconditioners)
  double* tloc = nullptr;              // [NE] node-local coupling scalar of the last operator application
  double* ujvp = nullptr;              // [nn] phi_e + gamma/c_e * c_e combination of a JVP input
  double* sqd = nullptr;               // [ndof] sqrt(|diag J|)
  double* rsqd = nullptr;              // [ndof] 1 / sqrt(|diag J|)
  double* iwf = nullptr;               // [4] 1 / w_f
  double* unorm2 = nullptr;            // [4] ||(sqrt(d) u)_f||^2 of the linearization state
  double* wf = nullptr;                // [4] per-field Krylov weights (device)
  unsigned* flags = nullptr;           // device error flags
  unsigned* flags_h = nullptr;         // pinned host mirror

  // multigrid
  int nlev = 0;
  p4d::MGLevel lev[p4d::kMaxLevels];
  double lam_h[p4d::kMaxLevels][p4d::kNH] = {};   // Gershgorin bounds (host copy, per Newton update)
  double* lam_pin = nullptr;           // pinned staging for lam
  void* yc = nullptr;                  // [NE][nc] particle solve work (compute precision)

  // concentration-dependent transport (transport.cu, transport_model 1)
  double kappa_fix = 0.0, De_fix = 0.0;  // bulk kappa, D_e of the fixed assembly and the preconditioner
  double* tr_coefL = nullptr;          // [4][nelem] kappa_eff, D_eff and derivatives at the linearization
  double* tr_GHL = nullptr;            // [16][nelem] K_e u_e, K_e c_e at the linearization
  double* tr_coefR = nullptr;          // the same at the state of the last residual evaluation
  double* tr_GHR = nullptr;
  double* tr_sc = nullptr;             // [2][nelem] per-element scalars of a Jacobian product
  double* tr_rows = nullptr;           // [2][nn] transport rows of the last residual evaluation

  // matrix-free level 0 (mf.cu), compute precision of the preconditioner
  void* mf_coef = nullptr;             // [3][nelem] float2 (stiffness, mass) per field: sc_0 sigma_eff,
                                       // sc_1 kappa_eff, (sc_2 D_eff, sc_2 eps/dt)
  void* mf_geo = nullptr;              // per-axis factors (2/h, h/2, h/6) [3][nx] / 8, [3][ny], [3][nz]
  void* mf_svs = nullptr;              // [3][nn] float2 (sc_f * variable node diagonal, 1/diag) (per linearization)
  int4* mf_items = nullptr;            // work items (field, tile, k0, k1), phi_s then phi_e then c_e
  int mf_off[3] = {0, 0, 0}, mf_cnt[3] = {0, 0, 0};
  int mf_ntx = 0, mf_nty = 0;          // node tiles per axis
  size_t mf_smem = 0;                  // dynamic shared memory per block
  bool mf_phis = false;                // phi_s matrix-free (no collector shells)

  // Krylov workspace
  int mcap = 0;                        // allocated restart capacity
  int64_t kry_len = 0;                 // allocated vector length
  double* V = nullptr;                 // [mcap+1][len]
  double* Z = nullptr;                 // [mcap][len]
  double* w = nullptr;                 // [len]
  double* r0 = nullptr;                // [ndof]
  double* tmp = nullptr;               // [ndof]
  double* bred = nullptr;              // [ndof] reduced right-hand side / scratch
  double* part = nullptr;              // [nparts][kry dots] partial sums
  double* hs = nullptr;                // device Hessenberg / Givens state
  double* hs_h = nullptr;              // pinned host mirror of small scalars

  // profiling (p4d_params.profile): event pairs per timed class, reused across solves
  struct Prof {
    std::vector<cudaEvent_t> ev[4];    // 0 precond, 1 jvp, 2 ortho, 3 level-0 stencil smoothing
    size_t used[4] = {0, 0, 0, 0};
  } prof;

  // CUDA graphs of the preconditioner applied to Krylov column k (k read on
  // the device from kdev), [transpose][full layout]; captured on cap_stream
  // at first use and dropped whenever the options change.
  struct PcGraph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;             // kernel nodes (added to the launch counter per launch)
  } pcg[2][2];
  // One FGMRES restart cycle as one graph, [transpose][full]: Arnoldi step k
  // inside a conditional (IF) node whose condition a one-thread kernel sets
  // from the device gate (no stop yet, k below the cycle's step limit).
  struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    int m = 0;                         // steps in the graph
    std::vector<long long> kernels;    // kernel launches of step k (gate kernels not included)
  } cyc[2][2];
  unsigned graph_gen = 0;              // incremented whenever the captured graphs are dropped
  cudaStream_t cap_stream = nullptr;
  int* kdev = nullptr;                 // current Krylov column (device)
  double* cheb_dev = nullptr;          // Chebyshev coefficients [kMaxLevels][kMaxDeg][3][kNH]
  float* cheb_dev32 = nullptr;         // the same in FP32
  double* cheb_pin = nullptr;          // pinned staging of cheb_dev and cheb_dev32
};

// Cells solved together by the lockstep FGMRES driver: one graph per Krylov
// column k holds every cell's Arnoldi step k inside a conditional (IF) node
// whose condition a one-thread kernel sets from active[cell]; the host
// launches one graph per column for the whole batch and reads every cell's
// residual estimate and status (stat[2 cell ...]) after it.
struct p4d_batch_ctx {
  std::vector<p4d_ctx*> cells;          // not owned
  cudaStream_t stream = nullptr;        // stream of the batched step graphs
  int* active_dev = nullptr;            // [n] cell takes step k
  int* active_h = nullptr;              // pinned mirror
  double* stat_dev = nullptr;           // [n][2] residual estimate, status of each cell's step
  double* stat_h = nullptr;             // pinned mirror
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> kernels;     // kernel launches of each cell's step (0: cell not in the graph)
  };
  std::vector<StepGraph> gk[2];         // [transpose][k]
  std::vector<unsigned> gen;            // cells' graph generations when gk was built
};

// Slab domain decomposition of one cell along z: parts[p] is the handle of
// slab p (bottom to top); consecutive slabs overlap by 2 ghosts - 1 element
// layers, so a slab's lowest `ghosts` node planes (above the bottom slab)
// and highest `ghosts` planes (below the top slab) are ghost planes owned
// by its neighbours.  Slab p owns
// its local node planes [own_lo, own_hi) and its electrode nodes
// [cs_lo, cs_hi) (node order).
constexpr int kDDRed = 256;   // largest allreduce (values)
struct p4d_dd_ctx {
  std::vector<p4d_ctx*> parts;          // not owned
  cudaStream_t stream = nullptr;        // the parts' common stream
  int64_t nxy = 0;                      // nodes per z plane
  int ghosts = 1;                       // ghost node planes per interior side
  std::vector<int32_t> plan;            // halo messages [n][4]: src slab, first src plane, dst slab, first dst plane
                                        // (ghosts consecutive planes each)
  std::vector<int> own_lo, own_hi;
  std::vector<int64_t> cs_lo, cs_hi;
  double* sbuf = nullptr;               // [n][3 ghosts nxy] packed planes (sender side)
  double* rbuf = nullptr;               // [n][3 ghosts nxy] received planes
  double* red = nullptr;                // [(P + 1)][kDDRed] allreduce staging; the sum in the last row
  double* part = nullptr;               // block partial sums
  std::vector<double*> bw;              // [P] right-hand sides with ghost rows zero
  // Two-level correction: coarse basis vectors per slab, field and group
  // (phi_s: anode and cathode unknowns; phi_e, c_e: all nodes) and mode
  // (constant, linear in z over the slab's owned planes); coarse bin b of a
  // slab (0..7: phi_s anode 1, z; phi_s cathode 1, z; phi_e 1, z; c_e 1, z)
  // is basis vector cmap[8 p + b] (-1: none).
  int coarse_modes = 2;                 // 0 none, 1 constants, 2 constants and linear in z
  int nb = 0;                           // coarse basis vectors (0: correction off)
  std::vector<int> cmap;                // [P][8]
  int* cmap_dev = nullptr;
  double* bins = nullptr;               // [P][kDDRed] coarse sums, one row per slab
  double* cy = nullptr;                 // [P][kDDRed] coarse solution, one row per slab
  double* ainv = nullptr;               // [kDDRed^2 / ...] inverse coarse matrix (nb x nb), FP64
  double* cpart = nullptr;              // block partials of the coarse sums
  std::vector<double*> wx, wy;          // [P] vectors of the coarse matrix build (3 nn)
};

// ---------------------------------------------------------------- helpers
namespace p4d {

p4d_status dalloc(p4d_ctx* c, void** p, size_t bytes);
template <typename T>
inline p4d_status dalloc_t(p4d_ctx* c, T** p, size_t count) {
  return dalloc(c, reinterpret_cast<void**>(p), count * sizeof(T));
}

inline unsigned nblocks(int64_t n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

// A handle's kernels run on the current device with the handle's memory:
// the calls that launch work refuse another device current.
inline bool on_device(const p4d_ctx* c) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev == c->device;
}

// Process-wide count of kernel launches issued by the library (every launch
// site is written "count_launch(), kernel<<<...>>>(...)").
void count_launch();

// This thread's grid-stride share of sum_i (a_i s_i)^2, i in [0, n)
// (SCALED = false: s_i = 1), with four independent loads in flight per
// step (one per step leaves the loop waiting on memory latency).
template <bool SCALED>
__device__ __forceinline__ double sumsq_share(const double* __restrict__ a, const double* __restrict__ s, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
  for (; i + 3 * stride < n; i += 4 * stride) {
    double v0 = a[i], v1 = a[i + stride], v2 = a[i + 2 * stride], v3 = a[i + 3 * stride];
    if (SCALED) {
      v0 *= s[i];
      v1 *= s[i + stride];
      v2 *= s[i + 2 * stride];
      v3 *= s[i + 3 * stride];
    }
    q0 = fma(v0, v0, q0);
    q1 = fma(v1, v1, q1);
    q2 = fma(v2, v2, q2);
    q3 = fma(v3, v3, q3);
  }
  for (; i < n; i += stride) {
    double v = a[i];
    if (SCALED) v *= s[i];
    q0 = fma(v, v, q0);
  }
  return (q0 + q1) + (q2 + q3);
}

// Block sums of four per-thread values into partial[blockIdx.x * 4 + f]
// (fixed order: warp shuffles, then the warps in order).  blockDim.x is a
// multiple of 32, at most 1024.
__device__ __forceinline__ void block_sum4(const double (&acc)[4], double* __restrict__ partial) {
  __shared__ double red[4][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    double a = acc[f];
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) red[f][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    partial[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// out[f] = sum_b partial[b * 4 + f] by warp f of a 128-thread block (fixed
// order: lanes stride over the blocks, then a butterfly).
__device__ __forceinline__ void sum4_warps(const double* __restrict__ partial, int nblk, double* out) {
  const int lane = threadIdx.x & 31, f = threadIdx.x >> 5;
  if (f >= 4) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[b * 4 + f];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[f] = s;
}


// While a thread captures a graph its launches are counted into *counter
// (the graph's kernel nodes) instead of the global launch counter.
void capture_counter(long long* counter);
void count_launches(long long n);

// A device vector chosen at run time: base + stride * (*k) (k == NULL: base).
struct VRef {
  double* base;
  int64_t stride;
  const int* k;
  __device__ __forceinline__ double* get() const { return k ? base + stride * (int64_t)(*k) : base; }
};

// ---- assembly / linearization (assemble.cu)
p4d_status assemble_fixed(p4d_ctx* c, const double* eps, const double* eps_s, const uint8_t* region);
p4d_status linearize(p4d_ctx* c, const p4d_state* st);
p4d_status residual(p4d_ctx* c, const p4d_state* st, double* r_out);
p4d_status check_flags(p4d_ctx* c);

// ---- operator application (jvp.cu)
// y[i] = sc_out[i] * ((b ? b[i] : 0) +/- (J x)[i]); sign = -1 with b for residual form.
p4d_status jvp_full(p4d_ctx* c, const double* x, double* y, int transpose, const double* b,
                    bool scaled);
p4d_status jvp_reduced(p4d_ctx* c, const double* x, double* y, int transpose, const double* b,
                       bool scaled);

// ---- particle elimination (particle.cu)
p4d_status particle_solve64(p4d_ctx* c, const double* rc, double* yc, const double* tN, int transpose);
p4d_status precond_full(p4d_ctx* c, const double* r, double* z, int transpose, bool scaled);
p4d_status precond_macro(p4d_ctx* c, const double* rm, double* zm, int transpose, bool scaled);
// Preconditioner applied to Krylov column *kdev of V into column *kdev of Z
// (scaled space), through a CUDA graph unless profiling.
p4d_status precond_column(p4d_ctx* c, int transpose, bool use_graph);

// Captures what body() launches on c->stream into g (on c->cap_stream,
// thread-local capture mode; launches are counted as g's kernel nodes).
template <typename F>
p4d_status capture_graph(p4d_ctx* c, p4d_ctx::PcGraph& g, F&& body) {
  cudaStream_t user = c->stream;
  c->stream = c->cap_stream;
  long long kernels = 0;
  capture_counter(&kernels);
  cudaGraph_t graph = nullptr;
  p4d_status st = P4D_OK;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = P4D_ERR_CUDA;
  if (st == P4D_OK) {
    st = body();
    if (cudaStreamEndCapture(c->cap_stream, &graph) != cudaSuccess && st == P4D_OK) st = P4D_ERR_CUDA;
  }
  capture_counter(nullptr);
  c->stream = user;
  if (st == P4D_OK && cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) st = P4D_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  if (st != P4D_OK) {
    cudaGetLastError();
    g.exec = nullptr;
    return st;
  }
  g.kernels = kernels;
  return P4D_OK;
}
void drop_graphs(p4d_ctx* c);
p4d_status cheb_upload(p4d_ctx* c);

// ---- multigrid (mg.cu)
p4d_status mg_plan(p4d_ctx* c);
p4d_status mg_setup_fixed(p4d_ctx* c);
p4d_status mg_update(p4d_ctx* c);
p4d_status mg_fetch_lam(p4d_ctx* c);
// run the V-cycles of the listed hierarchies on the level-0 right-hand sides already in place
p4d_status mg_vcycle(p4d_ctx* c, const int* hs, int nhs);
// matrix-free level 0 (mf.cu): setup after mg_setup_fixed; whether field f
// (0 phi_s, 1 phi_e, 2 c_e) is applied matrix-free; one launch over the
// fields in fmask: mode 0 Chebyshev step `step` (x -> x2, d), mode 1 r = b - A x
p4d_status mf_setup(p4d_ctx* c);
// The paper's bulk electrolyte conductivity kappa(c_e) (S/m) and diffusivity
// D_e(c_e) (m^2/s) (Appendix "Model Parameters", eqs. kappa_app and De_app,
// with their Arrhenius factors at temperature T) and their derivatives with
// respect to c_e (mol/m^3).
__host__ __device__ inline void transport_bulk(double ce, double T, double Rg, double& kap, double& dkap,
                                               double& De, double& dDe) {
  const double c = ce / 1000.0;
  const double ak = exp(34700.0 / Rg * (1.0 / 298.15 - 1.0 / T));
  const double ad = exp(37040.0 / Rg * (1.0 / 298.15 - 1.0 / T));
  kap = ak * (0.0911 + 1.9101 * c - 1.052 * c * c + 0.1554 * c * c * c);
  dkap = ak * (1.9101 - 2.104 * c + 0.4662 * c * c) / 1000.0;
  De = ad * 5.34e-10 * exp(-0.65 * c);
  dDe = -0.65e-3 * De;
}
// concentration-dependent transport (transport.cu); no-ops for transport_model 0
void transport_reference(const p4d_params& p, double* kap, double* De);
p4d_status transport_alloc(p4d_ctx* c);
p4d_status transport_linearize(p4d_ctx* c, const p4d_state* st);
const double* transport_residual_rows(p4d_ctx* c, const p4d_state* st, const double* lnce);
p4d_status transport_jvp(p4d_ctx* c, const double* x, double* y, int transpose, const double* b, bool scaled);
bool mf_field_on(const p4d_ctx* c, int f);
p4d_status mf_level0(p4d_ctx* c, int fmask, int mode, int step);
// level-0 rhs from an FP64 macro vector: b_h = scale * (r_f - corr)  (see mg.cu)
p4d_status mg_load_rhs(p4d_ctx* c, const double* rm, const double* sinv_m, const int* hs, int nhs);
p4d_status mg_store_out(p4d_ctx* c, const double* rm_unscaled_src, const double* sinv_m, double* zm,
                        const int* fields, int nf);

// ---- profiling: mark(c, cls, begin) records an event pair member when
// p4d_params.profile is set; prof_sum(c, cls) sums the pairs (after a sync)
void prof_mark(p4d_ctx* c, int cls);
double prof_sum(p4d_ctx* c, int cls, int* count);
void prof_reset(p4d_ctx* c);

// ---- Krylov (krylov.cu)
p4d_status fgmres(p4d_ctx* c, const double* b, double* x, p4d_info* info, int transpose);
// Lockstep FGMRES over the cells of a batch (see p4d_batch_ctx).
p4d_status fgmres_batched(p4d_batch_ctx* B, const double* const* b, double* const* x, p4d_info* info, int transpose);
void batch_drop_graphs(p4d_batch_ctx* B);

// ---- slab domain decomposition (dd.cu; the driver in krylov.cu)
// Ghost planes of fields 0..2 of every slab's vector v[p] <- the owners' planes
// (scaled: Krylov-space vectors s.u, rescaled by the rows' sqrt(diag J) of
// sender and receiver, so that the receiver holds s.u with its own s).
p4d_status dd_halo(p4d_dd_ctx* D, double* const* v, bool scaled);
// Zero slab p's ghost rows of v (fields 0..2; with cs_rows also the particle rows).
p4d_status dd_zero_ghost(p4d_dd_ctx* D, int p, double* v, bool cs_rows);
// ptrs[p][0..n) <- sum over the slabs of ptrs[q][0..n) (n <= kDDRed), on every slab.
p4d_status dd_allreduce(p4d_dd_ctx* D, double* const* ptrs, int n);
p4d_status dd_owned_sumsq(p4d_dd_ctx* D, int p, const double* const* v, const double* w, double* out);
p4d_status fgmres_dd(p4d_dd_ctx* D, const double* const* b, double* const* x, p4d_info* info);
// z_p += Z A_c^-1 Z^T (s^-1 v_p) on every slab (no-op when the correction is off).
p4d_status dd_coarse_correct(p4d_dd_ctx* D, const double* const* v, double* const* z);

}  // namespace p4d
