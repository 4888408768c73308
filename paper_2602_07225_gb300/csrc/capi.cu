// C ABI entry points, handle lifetime and host-side mesh bookkeeping.
//
// Setup classifies nodes and electrode particles on the host (one pass over
// the elements), builds the reference radial operator of eqs. L1, L2, L0,
// LR for R = D = 1 (the operator of a particle of radius R and diffusivity D
// is (D/R^2) times it; the flux factor is beta_ref/R), uploads everything and
// hands over to the device kernels for stencil assembly and the multigrid
// hierarchy.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include "p4d_common.cuh"

using namespace p4d;

namespace p4d {

static std::atomic<long long> g_launches{0};
static thread_local long long* t_capture = nullptr;
void count_launch() {
  if (t_capture) ++*t_capture;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void capture_counter(long long* counter) { t_capture = counter; }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

p4d_status dalloc(p4d_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return P4D_ERR_OOM;
  }
  c->allocs.push_back(*p);
  return P4D_OK;
}

void prof_mark(p4d_ctx* c, int cls) {
  if (!c->prm.profile) return;
  auto& P = c->prof;
  if (P.used[cls] >= P.ev[cls].size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
    P.ev[cls].push_back(e);
  }
  cudaEventRecord(P.ev[cls][P.used[cls]++], c->stream);
}

double prof_sum(p4d_ctx* c, int cls, int* count) {
  auto& P = c->prof;
  double ms = 0.0;
  int n = 0;
  for (size_t i = 0; i + 1 < P.used[cls]; i += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, P.ev[cls][i], P.ev[cls][i + 1]) == cudaSuccess) { ms += t; ++n; }
    else cudaGetLastError();
  }
  if (count) *count = n;
  return ms;
}

void prof_reset(p4d_ctx* c) {
  for (int k = 0; k < 4; ++k) c->prof.used[k] = 0;
}

p4d_status check_flags(p4d_ctx* c) {
  P4D_TRY(cudaMemcpyAsync(c->flags_h, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  P4D_TRY(cudaStreamSynchronize(c->stream));
  unsigned f = *c->flags_h;
  if (f & kFlagDomain) return P4D_ERR_DOMAIN;
  if (f & kFlagNonfinite) return P4D_ERR_NONFINITE;
  return P4D_OK;
}

}  // namespace p4d

namespace {

// Reference radial operator (R = 1, D = 1) on the node set rho[0..nc-1]:
// centre row eq. L0, interior rows eqs. L1 + L2 with the mesh ratio
// theta_i = dr_i / dr_{i-1}, surface row eq. LR (no-flux part); the flux
// enters the surface row as -beta * i_n with beta = 2 (1 + dr) / (F dr).
void radial_reference(const double* rho, int nc, double F, double* lo, double* di, double* up,
                      double* beta) {
  for (int i = 0; i < nc; ++i) lo[i] = di[i] = up[i] = 0.0;
  const double d1 = rho[1] - rho[0];
  di[0] = -6.0 / (d1 * d1);
  up[0] = 6.0 / (d1 * d1);
  for (int i = 1; i < nc - 1; ++i) {
    const double dp = rho[i + 1] - rho[i];   // dr_i
    const double dm = rho[i] - rho[i - 1];   // dr_{i-1}
    const double th = dp / dm;
    const double c1 = 2.0 / (rho[i] * dp * (1.0 + th));        // first-derivative term
    const double c2 = 2.0 / (dp * dm * (1.0 + th));            // second-derivative term
    up[i] = c1 + c2;
    lo[i] = -c1 * th * th + c2 * th;
    di[i] = -c1 * (1.0 - th * th) - c2 * (1.0 + th);
  }
  const double dN = rho[nc - 1] - rho[nc - 2];
  lo[nc - 1] = 2.0 / (dN * dN);
  di[nc - 1] = -2.0 / (dN * dN);
  *beta = 2.0 * (1.0 + dN / rho[nc - 1]) / (F * dN);
}

template <typename T>
p4d_status upload(p4d_ctx* c, T** dst, const T* src, size_t n) {
  P4D_TRYS(dalloc_t(c, dst, n));
  P4D_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return P4D_OK;
}

bool valid_params(const p4d_params* p) {
  if (!(p->dt > 0) || !(p->F > 0) || !(p->R > 0) || !(p->T > 0)) return false;
  if (p->precision < 0 || p->precision > 2) return false;
  if (p->combine < 0 || p->combine > 1) return false;
  if (p->mode < 0 || p->mode > 1) return false;
  if (p->restart < 1 || p->restart > 128 || p->maxit < 1) return false;
  if (p->cheb_degree < 1 || p->cheb_degree > 16 || !(p->cheb_ratio > 1.0)) return false;
  if (p->coarse_max < 8) return false;
  if (!(p->rtol > 0)) return false;
  if (!(p->alpha > 0 && p->alpha < 1)) return false;
  if (p->ocp_model < 0 || p->ocp_model > 1) return false;
  if (p->transport_model < 0 || p->transport_model > 1) return false;
  if (p->cgs_refine < 0 || p->cgs_refine > 2) return false;
  if (p->mf_zchunk < 0 || p->mf_zchunk > 64) return false;
  bool seen[3] = {false, false, false};
  for (int i = 0; i < 3; ++i) {
    if (p->order[i] < 0 || p->order[i] > 2 || seen[p->order[i]]) return false;
    seen[p->order[i]] = true;
  }
  return true;
}

p4d_status setup_impl(p4d_ctx* c, const p4d_mesh* m, const p4d_params* prm) {
  const int nx = m->nx, ny = m->ny, nz = m->nz;
  const int nnx = nx + 1, nny = ny + 1, nnz = nz + 1;
  const int64_t nn = (int64_t)nnx * nny * nnz;
  const int64_t nelem = (int64_t)nx * ny * nz;
  const int nc = m->nc;
  c->nx = nx; c->ny = ny; c->nz = nz;
  c->g = Grid{nnx, nny, nnz, nn};
  c->nelem = nelem;
  c->nc = nc;
  c->prm = *prm;
  if (!(m->shell_sigma_t_p >= 0.0) || !(m->shell_sigma_t_n >= 0.0) || !std::isfinite(m->shell_sigma_t_p) ||
      !std::isfinite(m->shell_sigma_t_n))
    return P4D_ERR_INVALID_ARG;
  c->shell_p = m->shell_sigma_t_p;
  c->shell_n = m->shell_sigma_t_n;

  // ---- node classification (host)
  std::vector<uint8_t> lab(nn, 0);
  auto node = [&](int i, int j, int k) { return (int64_t)i + nnx * ((int64_t)j + (int64_t)nny * k); };
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const uint8_t r = m->region[i + (int64_t)nx * (j + (int64_t)ny * k)];
        if (r > 3) return P4D_ERR_INVALID_ARG;
        uint8_t bit = r == 0 ? kLabAnode : (r == 2 ? kLabCathode : 0);
        if (!bit) continue;
        for (int l = 0; l < 8; ++l) lab[node(i + (l & 1), j + ((l >> 1) & 1), k + ((l >> 2) & 1))] |= bit;
      }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (m->gamma_n[i + (int64_t)nx * j])
        for (int l = 0; l < 4; ++l) lab[node(i + (l & 1), j + ((l >> 1) & 1), 0)] |= kLabDirichlet;
  std::vector<int32_t> eidx(nn, -1);
  c->enodes_h.clear();
  for (int64_t n = 0; n < nn; ++n) {
    const uint8_t e = lab[n] & (kLabAnode | kLabCathode);
    if (e == (kLabAnode | kLabCathode)) return P4D_ERR_INVALID_ARG;   // anode/cathode contact
    if (e) {
      eidx[n] = (int32_t)c->enodes_h.size();
      c->enodes_h.push_back((int32_t)n);
      if (!(lab[n] & kLabDirichlet)) lab[n] |= kLabActive;
    }
  }
  const int64_t NE = (int64_t)c->enodes_h.size();
  if (NE * nc >= (int64_t(1) << 31) || 27 * nn >= (int64_t(1) << 31)) return P4D_ERR_INVALID_ARG;   // 32-bit kernel indices
  c->NE = NE;
  c->ndof = 3 * nn + NE * nc;

  // ---- per electrode node: lumped volumes, particle constants
  std::vector<double> Mn(nn, 0.0), Sn(nn, 0.0), Dn(nn, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int64_t e = i + (int64_t)nx * (j + (int64_t)ny * k);
        const uint8_t r = m->region[e];
        if (r != 0 && r != 2) continue;
        const double v8 = m->hx[i] * m->hy[j] * m->hz[k] / 8.0;
        for (int l = 0; l < 8; ++l) {
          const int64_t n = node(i + (l & 1), j + ((l >> 1) & 1), k + ((l >> 2) & 1));
          Mn[n] += v8;
          Sn[n] += m->eps_s[e] * v8;
          if (m->Ds_e) Dn[n] += m->Ds_e[e] * v8;
        }
      }
  std::vector<double> rref(3 * nc);
  double beta_ref = 0.0;
  radial_reference(m->rgrid, nc, prm->F, rref.data(), rref.data() + nc, rref.data() + 2 * nc, &beta_ref);
  c->beta_ref = beta_ref;
  std::vector<double> Mj(NE), Aj(NE), kapj(NE), betaj(NE), Rj(NE);
  std::vector<uint8_t> et(NE);
  for (int64_t e = 0; e < NE; ++e) {
    const int64_t n = c->enodes_h[e];
    // D_s of the particle: the node value, or the volume-weighted mean of
    // the per-element values over the node's electrode elements
    const double R = m->Rs[n], D = m->Ds_e ? Dn[n] / Mn[n] : m->Ds[n];
    Rj[e] = R;
    if (!(R > 0) || !(D > 0)) return P4D_ERR_INVALID_ARG;
    Mj[e] = Mn[n];
    Aj[e] = 3.0 * Sn[n] / R;
    kapj[e] = D / (R * R);
    betaj[e] = beta_ref / R;
    et[e] = (lab[n] & kLabAnode) ? 0 : 1;
  }
  // ---- per-element bulk solid conductivity
  std::vector<double> sige(nelem, 0.0);
  for (int64_t e = 0; e < nelem; ++e) {
    const uint8_t r = m->region[e];
    if (r == 0 || r == 2) sige[e] = m->sigma_e ? m->sigma_e[e] : (r == 0 ? prm->sigma_n : prm->sigma_p);
  }
  // ---- Gamma_p face weights (bilinear face integral of N_j)
  std::vector<double> gpw(nn, 0.0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (m->gamma_p[i + (int64_t)nx * j]) {
        const double a4 = m->hx[i] * m->hy[j] / 4.0;
        for (int l = 0; l < 4; ++l) gpw[node(i + (l & 1), j + ((l >> 1) & 1), nz)] += a4;
      }

  // ---- axis lengths for the multigrid's coarsening rule
  {
    const double* hs[3] = {m->hx, m->hy, m->hz};
    const int ne[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
      double L = 0.0;
      for (int i = 0; i < ne[a]; ++i) L += hs[a][i];
      c->len[a] = L;
    }
  }

  // ---- upload
  P4D_TRYS(upload(c, &c->hx, m->hx, nx));
  P4D_TRYS(upload(c, &c->hy, m->hy, ny));
  P4D_TRYS(upload(c, &c->hz, m->hz, nz));
  P4D_TRYS(upload(c, &c->label, lab.data(), nn));
  P4D_TRYS(upload(c, &c->eidx, eidx.data(), nn));
  P4D_TRYS(upload(c, &c->enode, c->enodes_h.data(), NE));
  P4D_TRYS(upload(c, &c->gpw, gpw.data(), nn));
  P4D_TRYS(upload(c, &c->Mj, Mj.data(), NE));
  {
    std::vector<double> iM(NE);
    for (int64_t e = 0; e < NE; ++e) iM[e] = 1.0 / Mj[e];
    P4D_TRYS(upload(c, &c->iMj, iM.data(), NE));
  }
  P4D_TRYS(upload(c, &c->Aj, Aj.data(), NE));
  P4D_TRYS(upload(c, &c->kapj, kapj.data(), NE));
  P4D_TRYS(upload(c, &c->betaj, betaj.data(), NE));
  P4D_TRYS(upload(c, &c->etype, et.data(), NE));
  P4D_TRYS(upload(c, &c->rref, rref.data(), 3 * nc));
  P4D_TRYS(upload(c, &c->Rj, Rj.data(), NE));
  P4D_TRYS(upload(c, &c->region, m->region, nelem));
  P4D_TRYS(upload(c, &c->eps_e, m->eps, nelem));
  P4D_TRYS(upload(c, &c->epss_e, m->eps_s, nelem));
  P4D_TRYS(upload(c, &c->sig_e, sige.data(), nelem));
  double gp_area = 0.0;
  for (int64_t n = 0; n < nn; ++n) gp_area += gpw[n];
  c->gp_area = gp_area;

  // ---- linearization workspace
  P4D_TRYS(dalloc_t(c, &c->lnce, nn));
  P4D_TRYS(dalloc_t(c, &c->lnce_r, nn));
  P4D_TRYS(dalloc_t(c, &c->rin, NE));
  P4D_TRYS(dalloc_t(c, &c->gdc, nn));
  P4D_TRYS(dalloc_t(c, &c->in_, NE));
  P4D_TRYS(dalloc_t(c, &c->ge, NE));
  P4D_TRYS(dalloc_t(c, &c->gc, NE));
  P4D_TRYS(dalloc_t(c, &c->gs, NE));
  P4D_TRYS(dalloc_t(c, &c->zj, NE));
  P4D_TRYS(dalloc_t(c, &c->zeta, NE));
  P4D_TRYS(dalloc_t(c, &c->tloc, NE));
  P4D_TRYS(dalloc_t(c, &c->tfac, (size_t)2 * std::max<int64_t>(1, NE) * nc));
  if (prm->precision != 0) P4D_TRYS(dalloc_t(c, &c->tfac32, (size_t)2 * std::max<int64_t>(1, NE) * nc));
  P4D_TRYS(dalloc_t(c, &c->sqd, c->ndof));
  P4D_TRYS(dalloc_t(c, &c->rsqd, c->ndof));
  P4D_TRYS(dalloc_t(c, &c->iwf, 4));
  P4D_TRYS(dalloc_t(c, &c->unorm2, 4));
  P4D_TRYS(dalloc_t(c, &c->ujvp, nn));
  P4D_TRY(cudaMallocHost(&c->lam_pin, sizeof(double) * kMaxLevels * kNH));
  P4D_TRY(cudaMallocHost(&c->cheb_pin, 2 * sizeof(double) * kMaxLevels * kMaxDeg * 3 * kNH));
  P4D_TRYS(dalloc_t(c, &c->cheb_dev, (size_t)kMaxLevels * kMaxDeg * 3 * kNH));
  P4D_TRYS(dalloc_t(c, &c->cheb_dev32, (size_t)kMaxLevels * kMaxDeg * 3 * kNH));
  P4D_TRYS(dalloc_t(c, &c->kdev, 1));
  P4D_TRY(cudaMemset(c->kdev, 0, sizeof(int)));
  P4D_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  P4D_TRYS(dalloc_t(c, &c->wf, 4));
  P4D_TRYS(dalloc_t(c, &c->flags, 1));
  P4D_TRY(cudaMallocHost(&c->flags_h, sizeof(unsigned)));
  P4D_TRY(cudaMemset(c->flags, 0, sizeof(unsigned)));

  c->kappa_fix = prm->kappa;
  c->De_fix = prm->De;
  if (prm->transport_model == 1) transport_reference(*prm, &c->kappa_fix, &c->De_fix);
  P4D_TRYS(transport_alloc(c));
  P4D_TRYS(assemble_fixed(c, c->eps_e, c->epss_e, c->region));
  P4D_TRYS(mg_plan(c));
  P4D_TRYS(mg_setup_fixed(c));
  P4D_TRYS(mf_setup(c));

  // ---- Krylov workspace
  c->mcap = prm->restart;
  c->kry_len = prm->mode == 0 ? c->ndof : 3 * nn;
  P4D_TRYS(dalloc_t(c, &c->V, (size_t)(c->mcap + 1) * c->kry_len));
  P4D_TRYS(dalloc_t(c, &c->Z, (size_t)c->mcap * c->kry_len));
  P4D_TRYS(dalloc_t(c, &c->w, c->kry_len));
  P4D_TRYS(dalloc_t(c, &c->r0, c->ndof));
  P4D_TRYS(dalloc_t(c, &c->nwork, (size_t)5 * c->ndof));
  P4D_TRYS(dalloc_t(c, &c->nrm4, 4));
  P4D_TRYS(dalloc_t(c, &c->tmp, c->ndof));
  P4D_TRYS(dalloc_t(c, &c->bred, c->ndof));
  P4D_TRYS(dalloc_t(c, &c->part, (size_t)1024 * 136));
  P4D_TRYS(dalloc_t(c, &c->hs, (size_t)(c->mcap + 2) * (c->mcap + 8) + 64));
  P4D_TRY(cudaMallocHost(&c->hs_h, sizeof(double) * (size_t)(4 * c->mcap + 64)));
  P4D_TRY(cudaDeviceSynchronize());
  return P4D_OK;
}

void free_ctx(p4d_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (int k = 0; k < 4; ++k)
    for (cudaEvent_t e : c->prof.ev[k]) cudaEventDestroy(e);
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->cheb_pin) cudaFreeHost(c->cheb_pin);
  for (void* p : c->allocs) cudaFree(p);
  if (c->flags_h) cudaFreeHost(c->flags_h);
  if (c->lam_pin) cudaFreeHost(c->lam_pin);
  if (c->hs_h) cudaFreeHost(c->hs_h);
  delete c;
}

}  // namespace

extern "C" {

void p4d_params_default(p4d_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->F = 96485.33; p->R = 8.31446; p->T = 298.15; p->tplus = 0.4; p->brug = 1.5;
  p->De = 7.5e-10; p->kappa = 1.0; p->sigma_n = 100.0; p->sigma_p = 10.0;
  p->k_n = 2e-5; p->k_p = 6e-7; p->cmax_n = 2.5e4; p->cmax_p = 5.12e4; p->alpha = 0.5;
  p->ocp_n[0] = 0.229016; p->ocp_n[1] = -0.067279;
  p->ocp_p[0] = 4.948384; p->ocp_p[1] = -1.535617;
  p->dt = 10.0; p->i_app = -40.2022; p->diffpot_sign = 1.0;
  p->precision = 1; p->combine = 0; p->order[0] = 1; p->order[1] = 0; p->order[2] = 2;
  p->restart = 30; p->maxit = 500; p->mode = 1; p->cheb_degree = 2; p->coarse_max = 128;
  p->cheb_ratio = 10.0; p->rtol = 1e-8; p->profile = 0; p->ocp_model = 0; p->transport_model = 0;
  p->cgs_refine = 1;
  p->mf_zchunk = 0;
}

p4d_status p4d_setup(const p4d_mesh* m, const p4d_params* prm, const p4d_state* st, void* stream,
                     p4d_handle* out) {
  if (!m || !prm || !out) return P4D_ERR_INVALID_ARG;
  *out = nullptr;
  if (m->nx < 1 || m->ny < 1 || m->nz < 1 || m->nc < 3 || m->nc > kMaxNc) return P4D_ERR_INVALID_ARG;
  if (!m->hx || !m->hy || !m->hz || !m->region || !m->eps || !m->eps_s || !m->Rs || !m->Ds ||
      !m->gamma_p || !m->gamma_n || !m->rgrid)
    return P4D_ERR_INVALID_ARG;
  const double nnd = (double)(m->nx + 1) * (m->ny + 1) * (m->nz + 1);
  if (nnd * 27.0 * 4.0 > 9.0e18 || nnd > 2.0e9 / 27.0) return P4D_ERR_INVALID_ARG;
  for (int i = 0; i < m->nx; ++i) if (!(m->hx[i] > 0)) return P4D_ERR_INVALID_ARG;
  for (int i = 0; i < m->ny; ++i) if (!(m->hy[i] > 0)) return P4D_ERR_INVALID_ARG;
  for (int i = 0; i < m->nz; ++i) if (!(m->hz[i] > 0)) return P4D_ERR_INVALID_ARG;
  if (m->rgrid[0] != 0.0 || m->rgrid[m->nc - 1] != 1.0) return P4D_ERR_INVALID_ARG;
  for (int i = 1; i < m->nc; ++i) if (!(m->rgrid[i] > m->rgrid[i - 1])) return P4D_ERR_INVALID_ARG;
  if (!valid_params(prm)) return P4D_ERR_INVALID_ARG;
  p4d_ctx* c = new (std::nothrow) p4d_ctx();
  if (!c) return P4D_ERR_OOM;
  c->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return P4D_ERR_CUDA;
  }
  p4d_status s = setup_impl(c, m, prm);
  if (s == P4D_OK && st) s = p4d_jacobian_update(c, st);
  if (s != P4D_OK && s != P4D_ERR_DOMAIN) {
    free_ctx(c);
    return s;
  }
  *out = c;
  return s;
}

void p4d_destroy(p4d_handle h) { free_ctx(h); }

p4d_status p4d_get_sizes(p4d_handle h, int64_t* nnode, int64_t* nelec, int64_t* ndof, int32_t* nc) {
  if (!h) return P4D_ERR_INVALID_ARG;
  if (nnode) *nnode = h->g.nn;
  if (nelec) *nelec = h->NE;
  if (ndof) *ndof = h->ndof;
  if (nc) *nc = h->nc;
  return P4D_OK;
}

p4d_status p4d_electrode_nodes(p4d_handle h, int32_t* out) {
  if (!h || !out) return P4D_ERR_INVALID_ARG;
  std::memcpy(out, h->enodes_h.data(), h->enodes_h.size() * sizeof(int32_t));
  return P4D_OK;
}

p4d_status p4d_set_params(p4d_handle h, const p4d_params* p) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !p || !valid_params(p)) return P4D_ERR_INVALID_ARG;
  if (p->precision != h->prm.precision || p->coarse_max != h->prm.coarse_max || p->mf_zchunk != h->prm.mf_zchunk)
    return P4D_ERR_INVALID_ARG;
  if (p->profile != 0 && p->profile != 1) return P4D_ERR_INVALID_ARG;
  if (p->restart > h->mcap) return P4D_ERR_INVALID_ARG;
  // parameters baked into the assembled stencils, the particle factors and
  // the surface-flux factors at setup cannot change
  const p4d_params& o = h->prm;
  if (p->transport_model != o.transport_model) return P4D_ERR_INVALID_ARG;
  if (p->dt != o.dt || p->F != o.F || p->brug != o.brug || p->De != o.De || p->kappa != o.kappa ||
      p->sigma_n != o.sigma_n || p->sigma_p != o.sigma_p)
    return P4D_ERR_INVALID_ARG;
  if (p->mode == 0 && h->kry_len < h->ndof) return P4D_ERR_INVALID_ARG;
  const bool recoef = p->cheb_ratio != h->prm.cheb_ratio || p->cheb_degree != h->prm.cheb_degree;
  h->prm = *p;
  drop_graphs(h);
  if (recoef && h->linearized) return cheb_upload(h);
  return P4D_OK;
}

p4d_status p4d_residual(p4d_handle h, const p4d_state* st, double* r) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !st || !r || !st->phis || !st->phie || !st->ce || !st->cs || !st->ce_prev || !st->cs_prev)
    return P4D_ERR_INVALID_ARG;
  return residual(h, st, r);
}

p4d_status p4d_jacobian_update(p4d_handle h, const p4d_state* st) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !st || !st->phis || !st->phie || !st->ce || !st->cs || !st->ce_prev || !st->cs_prev)
    return P4D_ERR_INVALID_ARG;
  h->linearized = false;
  P4D_TRYS(linearize(h, st));
  P4D_TRYS(mg_update(h));
  P4D_TRYS(check_flags(h));
  P4D_TRYS(mg_fetch_lam(h));
  h->linearized = true;
  return P4D_OK;
}

p4d_status p4d_jvp(p4d_handle h, const double* x, double* y, int transpose) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !x || !y || x == y) return P4D_ERR_INVALID_ARG;
  if (!h->linearized) return P4D_ERR_INVALID_ARG;
  return jvp_full(h, x, y, transpose ? 1 : 0, nullptr, false);
}

p4d_status p4d_precond_apply(p4d_handle h, const double* r, double* z, int transpose) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !r || !z || r == z) return P4D_ERR_INVALID_ARG;
  if (!h->linearized) return P4D_ERR_INVALID_ARG;
  return precond_full(h, r, z, transpose ? 1 : 0, false);
}

p4d_status p4d_fgmres_solve(p4d_handle h, const double* b, double* x, p4d_info* info) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !b || !x || b == x) return P4D_ERR_INVALID_ARG;
  if (!h->linearized) return P4D_ERR_INVALID_ARG;
  return fgmres(h, b, x, info, 0);
}

p4d_status p4d_adjoint_solve(p4d_handle h, const double* g, double* lam, p4d_info* info) {
  if (h && !::p4d::on_device(h)) return P4D_ERR_INVALID_ARG;
  if (!h || !g || !lam || g == lam) return P4D_ERR_INVALID_ARG;
  if (!h->linearized) return P4D_ERR_INVALID_ARG;
  return fgmres(h, g, lam, info, 1);
}

void p4d_batch_destroy(p4d_batch B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  batch_drop_graphs(B);
  if (B->stream) cudaStreamDestroy(B->stream);
  if (B->active_dev) cudaFree(B->active_dev);
  if (B->stat_dev) cudaFree(B->stat_dev);
  if (B->active_h) cudaFreeHost(B->active_h);
  if (B->stat_h) cudaFreeHost(B->stat_h);
  delete B;
}

p4d_status p4d_batch_create(const p4d_handle* cells, int32_t ncells, p4d_batch* out) {
  if (!out) return P4D_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cells || ncells <= 0) return P4D_ERR_INVALID_ARG;
  for (int i = 0; i < ncells; ++i) {
    if (!cells[i]) return P4D_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (cells[j] == cells[i]) return P4D_ERR_INVALID_ARG;
  }
  p4d_batch_ctx* B = new (std::nothrow) p4d_batch_ctx;
  if (!B) return P4D_ERR_OOM;
  B->cells.assign(cells, cells + ncells);
  const size_t n = (size_t)ncells;
  p4d_status st = P4D_OK;
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) st = P4D_ERR_CUDA;
  if (st == P4D_OK && (cudaMalloc(&B->active_dev, sizeof(int) * n) != cudaSuccess ||
                       cudaMalloc(&B->stat_dev, sizeof(double) * 2 * n) != cudaSuccess))
    st = P4D_ERR_OOM;
  if (st == P4D_OK && (cudaMallocHost(&B->active_h, sizeof(int) * n) != cudaSuccess ||
                       cudaMallocHost(&B->stat_h, sizeof(double) * 2 * n) != cudaSuccess))
    st = P4D_ERR_OOM;
  if (st == P4D_OK && (cudaMemset(B->active_dev, 0, sizeof(int) * n) != cudaSuccess ||
                       cudaMemset(B->stat_dev, 0, sizeof(double) * 2 * n) != cudaSuccess))
    st = P4D_ERR_CUDA;
  if (st != P4D_OK) {
    cudaGetLastError();
    p4d_batch_destroy(B);
    return st;
  }
  std::memset(B->active_h, 0, sizeof(int) * n);
  std::memset(B->stat_h, 0, sizeof(double) * 2 * n);
  *out = B;
  return P4D_OK;
}

namespace {
p4d_status batch_solve(p4d_batch B, const double* const* b, double* const* x, p4d_info* info, int trans) {
  if (!B || !b || !x) return P4D_ERR_INVALID_ARG;
  for (size_t i = 0; i < B->cells.size(); ++i) {
    const p4d_ctx* c = B->cells[i];
    if (!b[i] || !x[i] || b[i] == x[i] || !c->linearized || c->prm.profile) return P4D_ERR_INVALID_ARG;
    if (!::p4d::on_device(c)) return P4D_ERR_INVALID_ARG;
  }
  return fgmres_batched(B, b, x, info, trans);
}
}  // namespace

p4d_status p4d_batch_fgmres_solve(p4d_batch B, const double* const* b, double* const* x, p4d_info* info) {
  return batch_solve(B, b, x, info, 0);
}

p4d_status p4d_batch_adjoint_solve(p4d_batch B, const double* const* g, double* const* lam, p4d_info* info) {
  return batch_solve(B, g, lam, info, 1);
}

long long p4d_launch_count(void) { return p4d::g_launches.load(std::memory_order_relaxed); }

}  // extern "C"

namespace p4d {
namespace {
// Sink of the FP64 rate probe (keeps its arithmetic live).
__device__ double g_fma_sink;

// Eight independent dependent-FMA chains per thread: the FP64 pipe is the
// only busy unit (no memory traffic inside the loop).
__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = 1.0 + 1e-3 * (threadIdx.x + q);
  for (int t = 0; t < iters; ++t) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == 12345.678) g_fma_sink = s;   // never true; the compiler cannot drop the chains
}
}  // namespace
}  // namespace p4d

extern "C" {

p4d_status p4d_fp64_fma_rate(double* tflops) {
  if (!tflops) return P4D_ERR_INVALID_ARG;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  P4D_TRY(cudaGetDevice(&dev));
  P4D_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  P4D_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return P4D_ERR_CUDA;
  }
  float best = 0.f;
  p4d_status st = P4D_OK;
  for (int rep = 0; rep < 4 && st == P4D_OK; ++rep) {
    cudaEventRecord(e0, 0);
    ::p4d::count_launch(), p4d::k_fp64_fma<<<blocks, threads>>>(iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = P4D_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;   // the first launch warms up
  }
  if (cudaGetLastError() != cudaSuccess) st = P4D_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == P4D_OK && best > 0.f) *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
  return st;
}

const char* p4d_status_string(p4d_status s) {
  switch (s) {
    case P4D_OK: return "ok";
    case P4D_ERR_INVALID_ARG: return "invalid argument";
    case P4D_ERR_CUDA: return "CUDA error";
    case P4D_ERR_OOM: return "out of device memory";
    case P4D_ERR_NOT_CONVERGED: return "not converged";
    case P4D_ERR_BREAKDOWN: return "Krylov breakdown";
    case P4D_ERR_NONFINITE: return "non-finite value";
    case P4D_ERR_DOMAIN: return "concentration outside the kinetics domain";
    case P4D_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

}  // extern "C"
