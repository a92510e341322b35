// C ABI of liblbm_fade: handle lifetime, parameter derivation (Algorithm 1's
// initialisation), graph-captured time stepping and host I/O.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.h"

#include <mutex>

namespace lbm {

int device_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < kMaxDev) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  if (dev >= 0 && dev < kMaxDev) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

cudaError_t dev_alloc(const lbm_s* h, void** p, size_t bytes) {
  if (h->mem.alloc) {
    *p = h->mem.alloc(bytes, h->stream, h->mem.ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

void dev_free(const lbm_s* h, void* p) {
  if (!p) return;
  if (h->mem.release) h->mem.release(p, h->mem.ctx);
  else cudaFree(p);
}

}  // namespace lbm

namespace {

thread_local char g_cuda_msg[256] = "";

int record_cuda(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s", what, cudaGetErrorString(e));
  return (e == cudaErrorMemoryAllocation) ? LBM_ENOMEM : LBM_ECUDA;
}

#define LBM_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return record_cuda(e_, #call);     \
  } while (0)

// Gauss-Jordan inverse of a small dense matrix (row-major, n <= 7). Returns false if singular.
bool invert(int n, const double* a, double* inv) {
  double m[7][14];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) m[i][j] = (j < n) ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[piv][c])) piv = r;
    if (std::fabs(m[piv][c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(m[c][j], m[piv][j]);
    const double d = m[c][c];
    for (int j = 0; j < 2 * n; ++j) m[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double fct = m[r][c];
      if (fct == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) m[r][j] -= fct * m[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i * n + j] = m[i][j + n];
  return true;
}

// Cholesky test for symmetric positive definiteness of a d x d matrix.
bool is_spd(int d, const double* a) {
  double l[3][3] = {{0}};
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j)
      if (std::fabs(a[i * d + j] - a[j * d + i]) > 1e-14 * (std::fabs(a[i * d + j]) + 1e-300)) return false;
  for (int j = 0; j < d; ++j) {
    double s = a[j * d + j];
    for (int k = 0; k < j; ++k) s -= l[j][k] * l[j][k];
    if (!(s > 0.0)) return false;
    l[j][j] = std::sqrt(s);
    for (int i = j + 1; i < d; ++i) {
      double t = a[i * d + j];
      for (int k = 0; k < j; ++k) t -= l[i][k] * l[j][k];
      l[i][j] = t / l[j][j];
    }
  }
  return true;
}

// MRT change of basis, Eq. (MatrixD2).
void moment_matrix(int d, double* M) {
  static const int m5[5][5] = {{1, 1, 1, 1, 1}, {0, 1, -1, 0, 0}, {0, 0, 0, 1, -1}, {4, -1, -1, -1, -1}, {0, 1, 1, -1, -1}};
  static const int m7[7][7] = {{1, 1, 1, 1, 1, 1, 1},      {0, 1, -1, 0, 0, 0, 0},    {0, 0, 0, 1, -1, 0, 0},
                               {0, 0, 0, 0, 0, 1, -1},     {6, -1, -1, -1, -1, -1, -1}, {0, 2, 2, -1, -1, -1, -1},
                               {0, 0, 0, 1, 1, -1, -1}};
  const int Q = (d == 2) ? 5 : 7;
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) M[i * Q + j] = (d == 2) ? m5[i][j] : m7[i][j];
}

struct Derived {
  lbm::StepParams sp;
  double h[3];  // BGK diagonal-D factors multiplying g_mu (end of Section 2.2)
};

int derive(const lbm_params* p, Derived* out) {
  if (!p) return LBM_EINVAL;
  if (p->lattice != LBM_D2Q5 && p->lattice != LBM_D3Q7) return LBM_EINVAL;
  if (p->collision != LBM_BGK && p->collision != LBM_MRT) return LBM_EINVAL;
  if (p->precision < LBM_FP64 || p->precision > LBM_FP32_BF16SPLIT6) return LBM_EINVAL;
  const int d = (p->lattice == LBM_D2Q5) ? 2 : 3;
  const int Q = 2 * d + 1;
  if (!(p->dx > 0.0) || !(p->dt > 0.0) || !std::isfinite(p->dx) || !std::isfinite(p->dt)) return LBM_EINVAL;
  if (!std::isfinite(p->C_wall)) return LBM_EINVAL;
  if (p->variant != LBM_VARIANT_FG && p->variant != LBM_VARIANT_CAPUTO) return LBM_EINVAL;
  for (int mu = 0; mu < 3; ++mu) {
    if (mu < d) {
      if (p->grid[mu] < 3) return LBM_EINVAL;
      if (!(p->alpha[mu] > 1.0 && p->alpha[mu] <= 2.0)) return LBM_EINVAL;
      if (!(p->p[mu] >= 0.0 && p->p[mu] <= 1.0)) return LBM_EINVAL;
      if (!(p->g[mu] > 0.0) || !std::isfinite(p->g[mu])) return LBM_EINVAL;
      if (!std::isfinite(p->u[mu])) return LBM_EINVAL;
    } else if (p->grid[mu] != 1) {
      return LBM_EINVAL;
    }
  }
  const long long nodes = (long long)p->grid[0] * p->grid[1] * p->grid[2];
  if (nodes > (1LL << 31)) return LBM_EINVAL;

  Derived D{};
  lbm::StepParams& sp = D.sp;
  for (int mu = 0; mu < 3; ++mu) sp.n[mu] = p->grid[mu];
  sp.nodes = nodes;
  const double e2 = (d == 2) ? 1.0 / 3.0 : 1.0 / 4.0;      // Fig. 1 caption
  sp.w0 = (d == 2) ? 1.0 / 3.0 : 1.0 / 4.0;
  sp.wi = (d == 2) ? 1.0 / 6.0 : 1.0 / 8.0;
  for (int mu = 0; mu < 3; ++mu) sp.adv[mu] = (mu < d) ? (p->dt / p->dx) * p->u[mu] / e2 : 0.0;
  sp.C_wall = p->C_wall;
  sp.ksum = 1;
  sp.pstride = 0;
  const double ratio = p->dt / (p->dx * p->dx);
  double Dm[9];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Dm[i * d + j] = p->D[3 * i + j];
  for (int i = 0; i < d; ++i)
    if (!(Dm[i * d + i] > 0.0) || !std::isfinite(Dm[i * d + i])) return LBM_EINVAL;
  for (int mu = 0; mu < 3; ++mu) D.h[mu] = 1.0;

  if (p->collision == LBM_BGK) {
    // D = e^2 (lambda - 1/2) dx^2/dt, Eq. (Diffusion_Coefficient_3D); a diagonal, non-spherical D
    // keeps one lambda (from the largest entry) and scales g_mu by h_mu = D_mumu / max D.
    double dmax = 0.0;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j)
        if (i != j && Dm[i * d + j] != 0.0) return LBM_EINVAL;
    for (int i = 0; i < d; ++i) dmax = std::fmax(dmax, Dm[i * d + i]);
    const double lam = dmax * ratio / e2 + 0.5;
    for (int i = 0; i < d; ++i) D.h[i] = Dm[i * d + i] / dmax;
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) sp.omega[i][j] = (i == j) ? 1.0 / lam : 0.0;
  } else {
    // Lambda^-1 = diag(lambda_0, lambdabar, 1/s_free), Eq. (MatrixS); lambdabar from Eq. (D_ab)
    double lambar[9];
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) lambar[i * d + j] = Dm[i * d + j] * ratio / e2 + (i == j ? 0.5 : 0.0);
    if (!is_spd(d, lambar)) return LBM_EINVAL;
    for (int k = 0; k < Q - d - 1; ++k)
      if (!(p->s_free[k] > 0.0 && p->s_free[k] < 2.0)) return LBM_EINVAL;
    for (int k = 0; k < Q - d - 1; ++k) sp.sfree[k] = p->s_free[k];
    double laminv[49] = {0}, lam[49], M[49], Minv[49], tmp[49];
    laminv[0] = 1.0;  // conserved moment: no effect
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) laminv[(1 + i) * Q + (1 + j)] = lambar[i * d + j];
    for (int k = 0; k < Q - d - 1; ++k) laminv[(d + 1 + k) * Q + (d + 1 + k)] = 1.0 / p->s_free[k];
    if (!invert(Q, laminv, lam)) return LBM_EINVAL;
    moment_matrix(d, M);
    // rows of M are orthogonal: M^-1 = M^T diag(1/|row|^2)
    for (int i = 0; i < Q; ++i) {
      double nrm = 0.0;
      for (int j = 0; j < Q; ++j) nrm += M[i * Q + j] * M[i * Q + j];
      for (int j = 0; j < Q; ++j) Minv[j * Q + i] = M[i * Q + j] / nrm;
    }
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += lam[i * Q + k] * M[k * Q + j];
        tmp[i * Q + j] = s;
      }
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += Minv[i * Q + k] * tmp[k * Q + j];
        sp.omega[i][j] = s;
      }
  }
  *out = D;
  return LBM_OK;
}

// dOmega/dD_mumu for MRT: Omega = M^-1 Lambda M, Lambda = (Lambda^-1)^-1 and
// dLambda^-1/dD_mumu = dt/(e^2 dx^2) at the flux entry (1+mu, 1+mu) (Eqs. MatrixS, D_ab),
// so dOmega/dD_mumu = -M^-1 Lambda E_mu Lambda M.
// Share of D_mumu in d(max_nu D_nunu): 1 for the unique largest entry, 1/k for each of k
// equal largest entries (the average of the one-sided derivatives at a tie), 0 otherwise.
void bgk_max_share(const lbm_params* p, int d, double share[3], double* dmax) {
  double m = 0.0;
  for (int i = 0; i < d; ++i) m = std::fmax(m, p->D[4 * i]);
  int k = 0;
  for (int i = 0; i < d; ++i) k += (p->D[4 * i] == m);
  for (int i = 0; i < 3; ++i) share[i] = (i < d && p->D[4 * i] == m) ? 1.0 / k : 0.0;
  *dmax = m;
}

int derive_dOmega(const lbm_params* p, double dOm[3][lbm::kMaxQ][lbm::kMaxQ]) {
  const int d = (p->lattice == LBM_D2Q5) ? 2 : 3;
  const int Q = 2 * d + 1;
  const double e2 = (d == 2) ? 1.0 / 3.0 : 1.0 / 4.0;
  const double ratio = p->dt / (p->dx * p->dx);
  if (p->collision == LBM_BGK) {
    // Omega = I / lambda, lambda = max D ratio / e^2 + 1/2 (Eq. Diffusion_Coefficient_3D):
    // dOmega/dD_mumu = -share_mu (ratio / e^2) / lambda^2 I
    double share[3], dmax;
    bgk_max_share(p, d, share, &dmax);
    const double lam = dmax * ratio / e2 + 0.5;
    for (int mu = 0; mu < 3; ++mu)
      for (int i = 0; i < lbm::kMaxQ; ++i)
        for (int j = 0; j < lbm::kMaxQ; ++j)
          dOm[mu][i][j] = (i == j && i < Q) ? -share[mu] * (ratio / e2) / (lam * lam) : 0.0;
    return LBM_OK;
  }
  double laminv[49] = {0}, lam[49], M[49], Minv[49];
  laminv[0] = 1.0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) laminv[(1 + i) * Q + (1 + j)] = p->D[3 * i + j] * ratio / e2 + (i == j ? 0.5 : 0.0);
  for (int k = 0; k < Q - d - 1; ++k) laminv[(d + 1 + k) * Q + (d + 1 + k)] = 1.0 / p->s_free[k];
  if (!invert(Q, laminv, lam)) return LBM_EINVAL;
  moment_matrix(d, M);
  for (int i = 0; i < Q; ++i) {
    double nrm = 0.0;
    for (int j = 0; j < Q; ++j) nrm += M[i * Q + j] * M[i * Q + j];
    for (int j = 0; j < Q; ++j) Minv[j * Q + i] = M[i * Q + j] / nrm;
  }
  for (int mu = 0; mu < 3; ++mu)
    for (int i = 0; i < lbm::kMaxQ; ++i)
      for (int j = 0; j < lbm::kMaxQ; ++j) dOm[mu][i][j] = 0.0;
  for (int mu = 0; mu < d; ++mu) {
    const int r = 1 + mu;
    double dL[49], t1[49];
    // dLambda = -Lambda[:, r] * ratio/e2 * Lambda[r, :]
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) dL[i * Q + j] = -lam[i * Q + r] * (ratio / e2) * lam[r * Q + j];
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += dL[i * Q + k] * M[k * Q + j];
        t1[i * Q + j] = s;
      }
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += Minv[i * Q + k] * t1[k * Q + j];
        dOm[mu][i][j] = s;
      }
  }
  return LBM_OK;
}

void drop_graphs(lbm_s* h) {
  for (int i = 0; i < 2; ++i) {
    if (h->graph_exec[i]) cudaGraphExecDestroy(h->graph_exec[i]);
    if (h->graph[i]) cudaGraphDestroy(h->graph[i]);
    h->graph_exec[i] = nullptr;
    h->graph[i] = nullptr;
  }
}

void free_all(lbm_s* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);  // nothing in flight uses the buffers
  drop_graphs(h);
  lbm::tc_release(h);
  lbm::cs_release(h);
  lbm::dev_free(h, h->fused_bar);
  h->fused_bar = nullptr;
  lbm::dev_free(h, h->cs_part);
  h->cs_part = nullptr;
  h->cs_part_cap = 0;
  for (void* p : {h->fld.coll, h->fld.advw, h->fld.g, h->fld.G, h->fld.src, h->fld.cw, (void*)h->fld.tf})
    lbm::dev_free(h, p);
  h->fld = lbm::FieldState{};
  void* ptrs[] = {h->dev.f[0], h->dev.f[1], h->dev.C,   h->dev.C0,  h->dev.F,   h->dev.K,   h->dev.KT,
                  h->dev.stage, h->dev.partials, h->dev.scalar, h->dev.flag, h->dev.Khi, h->dev.Klo, h->dev.Kl2,
                  h->dev.Chi,  h->dev.Clo, h->dev.Cl2};
  for (void* p : ptrs) lbm::dev_free(h, p);
  h->dev = lbm::DeviceState{};
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  h->stream = nullptr;
}

// Programmatic dependent launch between the operator and collide-stream kernels: only
// where both grids run in one wave (measured: with multi-wave 3-D grids the early CTAs
// cost ~30%) and no other launch sits between them (tf32: the regrouped operands come
// from the collide-stream kernel itself)
bool pdl_fits(const lbm_s* h) {
  if (h->is_batch()) return false;
  if (!h->tc) return h->elem == 4 && lbm::cs_one_wave(h) && lbm::simt_one_wave(h);  // FP32 SIMT operator
  const bool adjacent = lbm::bf16_parts(h->prm.precision) || lbm::cs_writes_T(h);
  // the field march's grid is not the one cs_one_wave describes: no early launch there
  return adjacent && !h->fld.on && lbm::cs_one_wave(h) && lbm::tc_one_wave(h);
}

int alloc_bytes(const lbm_s* h, void** p, size_t bytes) {
  const cudaError_t e = lbm::dev_alloc(h, p, bytes);
  if (e == cudaErrorMemoryAllocation) return LBM_ENOMEM;
  LBM_CUDA(e);
  return LBM_OK;
}

std::mutex g_mem_mutex;
DevMem g_mem;  // hooks for handles created from now on

DevMem current_hooks() {
  std::lock_guard<std::mutex> lock(g_mem_mutex);
  return g_mem;
}

bool uses_tc(const lbm_s* h) { return h->tc != nullptr; }

// F = fractional terms of the current C (the first stage of Algorithm 1's time step).  On the tensor-core
// path the hi/lo split of C is refreshed first (inside the time loop the fused
// collide-stream kernel writes it, so one_step skips this).
int run_frac(lbm_s* h, cudaStream_t s) {
  if (!uses_tc(h)) {
    if (h->fld.on) LBM_CUDA(lbm::launch_scale_fields(h, s));  // G_mu = g_mu(x) C
    LBM_CUDA(lbm::launch_frac_simt(h, h->dev.C, h->dev.F, s));
  } else {
    LBM_CUDA(lbm::launch_split_C(h, s));
    LBM_CUDA(lbm::launch_frac_tc(h, s));
  }
  return LBM_OK;
}

int one_step(lbm_s* h, int& cur, cudaStream_t s, int tk = 0) {
  if (h->is_batch()) {
    // grouped operator (or one SIMT operator per problem), then one grouped collide-stream
    if (h->batch_tc_blocks > 0) {
      LBM_CUDA(lbm::launch_frac_tc_batch(h, s));
    } else {
      for (lbm_s* p : h->subs) LBM_CUDA(lbm::launch_frac_simt(p, p->dev.C, p->dev.F, s));
    }
    LBM_CUDA(lbm::launch_collide_stream_batch(h, cur, s));
    cur ^= 1;
    return LBM_OK;
  }
  if (uses_tc(h)) {
    LBM_CUDA(lbm::launch_split_T_step(h, s));  // tf32: regrouped y/z operands of the current C
    LBM_CUDA(lbm::launch_frac_tc(h, s));
  } else if (h->fld.on) {
    // G_mu = g_mu(x) C of the current C: written by the previous collide-stream launch (or
    // by the re-initialisation)
    LBM_CUDA(lbm::launch_frac_simt(h, h->dev.C, h->dev.F, s));
  } else {
    int rc = run_frac(h, s);
    if (rc) return rc;
  }
  LBM_CUDA(lbm::launch_collide_stream(h, h->dev.f[cur], h->dev.f[cur ^ 1], h->dev.C, s, tk));
  cur ^= 1;
  return LBM_OK;
}

// time factors of the next n steps (from step t_steps) into the slots 0..n-1 read by the
// collide-stream launches of a source or of wall values that vary in time: exp(rate_S t) dt
// at each step's start and exp(rate_w (t + dt)) at its end.  A pageable copy: the host
// waits for the stream's earlier work (once per graph replay of 128 steps).
int upload_time(lbm_s* h, int n) {
  if (!h->fld.tf) return LBM_OK;
  std::vector<double> v(2 * (size_t)n);
  const double dt = h->prm.dt;
  for (int j = 0; j < n; ++j) {
    const double t = (double)(h->t_steps + j) * dt;
    v[2 * j] = std::exp(h->fld.src_rate * t) * dt;
    v[2 * j + 1] = std::exp(h->fld.cw_rate * (t + dt));
  }
  LBM_CUDA(cudaMemcpyAsync(h->fld.tf, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, h->stream));
  return LBM_OK;
}

// f = feq(C, F(C)), then C = <1|f> so that the first step sees the same C the populations carry.
int init_from_C(lbm_s* h) {
  h->mass_valid = false;  // C now comes from the re-initialisation, not from a step
  h->t_steps = 0;
  int rc = run_frac(h, h->stream);
  if (rc) return rc;
  LBM_CUDA(lbm::launch_init_equilibrium(h, h->dev.f[h->cur], h->stream));
  LBM_CUDA(lbm::launch_moment(h, h->dev.f[h->cur], h->dev.C, h->stream));
  if (uses_tc(h)) LBM_CUDA(lbm::launch_split_C(h, h->stream));
  if (h->fld.on) LBM_CUDA(lbm::launch_scale_fields(h, h->stream));
  return LBM_OK;
}

int latched(lbm_s* h) {
  if (h->mass_limit > 0.0 && h->mass_valid) LBM_CUDA(lbm::launch_step_mass(h, h->mass_limit, h->stream));
  int flag = 0;
  LBM_CUDA(cudaMemcpyAsync(&flag, h->dev.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (flag & 2) return LBM_ERR_TIMEOUT;
  return (flag & 1) ? LBM_ERR_UNSTABLE : LBM_OK;
}

int capture_graph(lbm_s* h, int parity) {
  cudaStream_t s = h->stream;
  LBM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int cur = parity;
  int rc = LBM_OK;
  for (int k = 0; k < h->graph_steps && rc == LBM_OK; ++k) rc = one_step(h, cur, s, k);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return record_cuda(e, "cudaStreamEndCapture");
  h->graph[parity] = g;
  LBM_CUDA(cudaGraphInstantiate(&h->graph_exec[parity], g, 0));
  return LBM_OK;
}

}  // namespace

// K_mu and K_mu^T (Section 2.4, Eqs. 1Dminus_discret, c+, c-) built in FP64 on the host and
// stored in the working precision; the scale carries g_mu h_mu, or 1 when g varies in space
// (then g_mu(x) multiplies C inside the integrals, Eq. Fg).  Kall receives the FP64 matrices.
static int upload_weights(lbm_s* h, const double* hfac, std::vector<std::vector<double>>* Kall) {
  const lbm_params* prm = &h->prm;
  const size_t E = h->elem;
  std::vector<double> K, KT;
  long long off = 0;
  for (int mu = 0; mu < h->d; ++mu) {
    const int side = prm->grid[mu];
    K.assign((size_t)side * side, 0.0);
    KT.assign((size_t)side * side, 0.0);
    // g multiplies C inside the integrals (SIMT operator with fields, or g(x) on the tensor
    // cores), or is folded into K
    const double scale = (h->fld.on && (!h->tc || h->fld.gvar)) ? 1.0 : prm->g[mu] * hfac[mu];
    lbm::build_frac_matrix(prm->alpha[mu], prm->p[mu], scale, side, prm->dx, prm->variant, K.data());
    for (int n = 0; n < side; ++n)
      for (int l = 0; l < side; ++l) KT[(size_t)l * side + n] = K[(size_t)n * side + l];
    const size_t cnt = (size_t)side * side;
    cudaError_t e = cudaMemcpyAsync(h->dev.stage, K.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = lbm::launch_convert_in(h->dev.stage, (char*)h->dev.K + off * E, h->elem, cnt, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dev.stage, KT.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = lbm::launch_convert_in(h->dev.stage, (char*)h->dev.KT + off * E, h->elem, cnt, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return record_cuda(e, "weight upload");
    off += (long long)cnt;
    if (Kall) Kall->push_back(K);
  }
  return LBM_OK;
}

extern "C" {

// One problem: validation, buffers, weights, initial state.  Sub-problems of a batch
// (batched = true) run their operator as part of a grouped launch: 128-wide column
// tiles, no k-split.
static int create_problem(const lbm_params* prm, const double* C0_host, void* stream, bool batched, lbm_t* out,
                          const DevMem* mem = nullptr) {
  if (!out || !C0_host) return LBM_EINVAL;
  *out = nullptr;
  Derived dv;
  int rc = derive(prm, &dv);
  if (rc) return rc;
  lbm_s* h = new (std::nothrow) lbm_s();
  if (!h) return LBM_ENOMEM;
  h->prm = *prm;
  h->d = (prm->lattice == LBM_D2Q5) ? 2 : 3;
  h->Q = 2 * h->d + 1;
  h->elem = (prm->precision == LBM_FP64) ? 8 : 4;
  h->sp = dv.sp;
  h->graph_steps = 128;  // steps per captured graph (even); longer graphs, fewer replay boundaries
  h->mem = mem ? *mem : current_hooks();
  cudaGetDevice(&h->device);
  auto fail = [&](int code) {
    free_all(h);
    delete h;
    return code;
  };
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(record_cuda(e, "cudaStreamCreateWithFlags"));
    h->own_stream = true;
  }
  const long long nodes = h->sp.nodes;
  const size_t E = h->elem;
  if (prm->precision == LBM_FP32 && !batched) {
    // small FP32 problems: the SIMT operator's contraction split (F holds the partials)
    h->sp.ksum = lbm::simt_ksplit(h);
    h->sp.pstride = h->sp.ksum > 1 ? (long long)h->d * nodes : 0;
  }
  long long ksz = 0;
  for (int mu = 0; mu < h->d; ++mu) ksz += (long long)prm->grid[mu] * prm->grid[mu];
  h->reduce_blocks = lbm::reduce_blocks_for(nodes);
  if ((rc = alloc_bytes(h, &h->dev.f[0], E * h->Q * nodes))) return fail(rc);
  if ((rc = alloc_bytes(h, &h->dev.f[1], E * h->Q * nodes))) return fail(rc);
  if ((rc = alloc_bytes(h, &h->dev.C, E * nodes))) return fail(rc);
  if ((rc = alloc_bytes(h, &h->dev.C0, E * nodes))) return fail(rc);
  if ((rc = alloc_bytes(h, &h->dev.F, E * h->d * nodes * h->sp.ksum))) return fail(rc);
  h->f_elems = (size_t)h->d * nodes * h->sp.ksum;
  if ((rc = alloc_bytes(h, &h->dev.K, E * ksz))) return fail(rc);
  if ((rc = alloc_bytes(h, &h->dev.KT, E * ksz))) return fail(rc);
  if ((rc = alloc_bytes(h, (void**)&h->dev.stage, sizeof(double) * (size_t)(nodes > ksz ? nodes : ksz)))) return fail(rc);
  if ((rc = alloc_bytes(h, (void**)&h->dev.partials, sizeof(double) * h->reduce_blocks))) return fail(rc);
  if ((rc = alloc_bytes(h, (void**)&h->dev.scalar, sizeof(double)))) return fail(rc);
  if ((rc = alloc_bytes(h, (void**)&h->dev.flag, sizeof(int)))) return fail(rc);
  // kMassSlots mass partials per collide-stream block: at most one block per 32 x 16 tile and plane
  h->cs_part_cap = (long long)((prm->grid[0] + 31) / 32) * ((prm->grid[1] + 15) / 16) * prm->grid[2];
  if ((rc = alloc_bytes(h, (void**)&h->cs_part, sizeof(double) * lbm::kMassSlots * h->cs_part_cap))) return fail(rc);
  if (cudaMemsetAsync(h->dev.flag, 0, sizeof(int), h->stream) != cudaSuccess) return fail(LBM_ECUDA);

  // weight matrices K_mu (Section 2.4) in FP64 on the host, then the working precision
  std::vector<std::vector<double>> Kall;
  if ((rc = upload_weights(h, dv.h, &Kall))) return fail(rc);
  if (lbm::bf16_parts(prm->precision) || prm->precision == LBM_FP32_TF32SPLIT) {
    if ((rc = lbm::tc_prepare(h, Kall, batched ? 128 : 0, batched ? 1 : 0))) return fail(rc);
    h->launches_per_step = 2;  // (lbm_launches_per_step counts the tf32 regrouping launches)
  } else {
    h->launches_per_step = 2;  // one SIMT operator launch over every axis, one collide-stream
  }
  if (!batched && (rc = lbm::cs_prepare(h))) return fail(rc);
  if (!batched) {
    h->pdl = pdl_fits(h);
    if (h->tc) lbm::tc_set_pdl(h, h->pdl);
  }
  *out = h;
  rc = lbm_set_C(h, C0_host);
  if (rc) {
    *out = nullptr;
    return fail(rc);
  }
  return LBM_OK;
}

int lbm_create(const lbm_params* prm, const double* C0_host, lbm_t* out, void* stream) {
  return create_problem(prm, C0_host, stream, false, out);
}

int lbm_create_batch(int nprob, const lbm_params* prms, const double* const* C0_host, lbm_t* out, void* stream) {
  if (!out || !prms || !C0_host || nprob < 1) return LBM_EINVAL;
  *out = nullptr;
  const lbm_params& p0 = prms[0];
  if (p0.precision != LBM_FP32 && !lbm::bf16_parts(p0.precision)) return LBM_ENOTSUP;
  for (int i = 0; i < nprob; ++i) {
    if (!C0_host[i]) return LBM_EINVAL;
    if (prms[i].lattice != p0.lattice || prms[i].collision != p0.collision || prms[i].precision != p0.precision)
      return LBM_EINVAL;
    Derived dv;
    int rc = derive(&prms[i], &dv);
    if (rc) return rc;
  }
  lbm_s* b = new (std::nothrow) lbm_s();
  if (!b) return LBM_ENOMEM;
  b->prm = p0;
  b->d = (p0.lattice == LBM_D2Q5) ? 2 : 3;
  b->Q = 2 * b->d + 1;
  b->elem = 4;
  b->graph_steps = 32;
  b->mem = current_hooks();
  cudaGetDevice(&b->device);
  auto fail = [&](int code) {
    lbm_destroy(b);
    return code;
  };
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return record_cuda(e, "cudaStreamCreateWithFlags");
    }
    b->own_stream = true;
  }
  for (int i = 0; i < nprob; ++i) {
    lbm_t sub = nullptr;
    int rc = create_problem(&prms[i], C0_host[i], b->stream, true, &sub);
    if (rc) return fail(rc);
    b->subs.push_back(sub);
  }
  int rc = LBM_OK;
  if (lbm::bf16_parts(p0.precision)) {
    if ((rc = lbm::tc_batch_prepare(b))) return fail(rc);
    b->launches_per_step = 2;
  } else {
    b->launches_per_step = nprob * b->d + 1;
  }
  if ((rc = lbm::cs_batch_prepare(b))) return fail(rc);
  *out = b;
  return LBM_OK;
}

int lbm_batch_size(lbm_t h, int* nprob) {
  if (!h || !nprob) return LBM_EINVAL;
  *nprob = h->is_batch() ? static_cast<int>(h->subs.size()) : 1;
  return LBM_OK;
}

int lbm_batch_set_C(lbm_t h, int prob, const double* C_host) {
  if (!h || !C_host) return LBM_EINVAL;
  if (!h->is_batch()) return prob == 0 ? lbm_set_C(h, C_host) : LBM_EINVAL;
  if (prob < 0 || prob >= static_cast<int>(h->subs.size())) return LBM_EINVAL;
  h->subs[prob]->cur = h->cur;
  return lbm_set_C(h->subs[prob], C_host);
}

int lbm_set_C(lbm_t h, const double* C_host) {
  if (!h || !C_host || h->is_batch()) return LBM_EINVAL;
  const long long nodes = h->sp.nodes;
  LBM_CUDA(cudaMemcpyAsync(h->dev.stage, C_host, sizeof(double) * nodes, cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(lbm::launch_convert_in(h->dev.stage, h->dev.C0, h->elem, nodes, h->stream));
  return lbm_reset(h);
}

int lbm_reset(lbm_t h) {
  if (!h) return LBM_EINVAL;
  if (h->is_batch()) {
    for (lbm_s* p : h->subs) {
      p->cur = h->cur;
      int rc = lbm_reset(p);
      if (rc) return rc;
    }
    return LBM_OK;
  }
  LBM_CUDA(cudaMemsetAsync(h->dev.flag, 0, sizeof(int), h->stream));  // a restart clears latched errors
  LBM_CUDA(cudaMemcpyAsync(h->dev.C, h->dev.C0, (size_t)h->elem * h->sp.nodes, cudaMemcpyDeviceToDevice,
                           h->stream));
  return init_from_C(h);
}

int lbm_profile(lbm_t h, int nsteps, double* ms) {
  if (!h || !ms || nsteps < 0 || nsteps > 4096) return LBM_EINVAL;
  ms[0] = ms[1] = 0.0;
  if (nsteps > 0) {
    h->mass_valid = true;
    for (lbm_s* p : h->subs) p->mass_valid = true;
  }
  // every step's three events are queued before the one synchronisation, so that the
  // intervals measure the kernels, not the host's submission of each launch
  std::vector<cudaEvent_t> ev(3 * (size_t)nsteps);
  int rc = LBM_OK;
  size_t made = 0;
  for (; made < ev.size(); ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  if (made < ev.size()) rc = record_cuda(cudaErrorMemoryAllocation, "lbm_profile");
  for (int k = 0; k < nsteps && rc == LBM_OK; ++k) {
    if ((rc = upload_time(h, 1))) break;
    cudaError_t e = cudaEventRecord(ev[3 * k], h->stream);
    if (e == cudaSuccess) {
      if (h->is_batch() && h->batch_tc_blocks > 0) e = lbm::launch_frac_tc_batch(h, h->stream);
      else if (h->is_batch())
        for (lbm_s* p : h->subs)
          if (e == cudaSuccess) e = lbm::launch_frac_simt(p, p->dev.C, p->dev.F, h->stream);
      if (!h->is_batch()) {
        if (uses_tc(h)) {
          e = lbm::launch_split_T_step(h, h->stream);
          if (e == cudaSuccess) e = lbm::launch_frac_tc(h, h->stream);
        }
        else rc = run_frac(h, h->stream);
      }
    }
    if (e == cudaSuccess && rc == LBM_OK) e = cudaEventRecord(ev[3 * k + 1], h->stream);
    if (e == cudaSuccess && rc == LBM_OK) {
      if (h->is_batch()) e = lbm::launch_collide_stream_batch(h, h->cur, h->stream);
      else e = lbm::launch_collide_stream(h, h->dev.f[h->cur], h->dev.f[h->cur ^ 1], h->dev.C, h->stream);
    }
    if (e == cudaSuccess && rc == LBM_OK) e = cudaEventRecord(ev[3 * k + 2], h->stream);
    if (e != cudaSuccess) rc = record_cuda(e, "lbm_profile");
    h->cur ^= 1;
    ++h->t_steps;
    for (lbm_s* p : h->subs) p->cur = h->cur;
  }
  if (rc == LBM_OK && nsteps > 0) {
    const cudaError_t e = cudaEventSynchronize(ev[3 * (size_t)nsteps - 1]);
    if (e != cudaSuccess) rc = record_cuda(e, "lbm_profile");
  }
  for (int k = 0; k < nsteps && rc == LBM_OK; ++k) {
    float a = 0.f, b = 0.f;
    cudaError_t e = cudaEventElapsedTime(&a, ev[3 * k], ev[3 * k + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * k + 1], ev[3 * k + 2]);
    if (e != cudaSuccess) rc = record_cuda(e, "lbm_profile");
    ms[0] += a;
    ms[1] += b;
  }
  for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

int lbm_step(lbm_t h, int nsteps) {
  if (!h || nsteps < 0) return LBM_EINVAL;
  int rc;
  if (nsteps > 0) {
    h->mass_valid = true;  // the collide-stream kernel leaves the new C's mass partials
    for (lbm_s* p : h->subs) p->mass_valid = true;
  }
  if (h->fused) {
    // one cooperative launch per (up to) 4096 steps; it flips the buffer parity per step
    while (nsteps > 0) {
      const int n = nsteps < 4096 ? nsteps : 4096;
      LBM_CUDA(lbm::launch_fused(h, n, h->stream));
      h->cur ^= (n & 1);
      nsteps -= n;
    }
    return LBM_OK;
  }
  while (nsteps >= h->graph_steps) {
    if (!h->graph_exec[h->cur] && (rc = capture_graph(h, h->cur))) return rc;
    if ((rc = upload_time(h, h->graph_steps))) return rc;
    LBM_CUDA(cudaGraphLaunch(h->graph_exec[h->cur], h->stream));
    nsteps -= h->graph_steps;  // even: the current buffer index is unchanged
    h->t_steps += h->graph_steps;
  }
  for (int k = 0; k < nsteps; ++k) {
    if ((rc = upload_time(h, 1)) || (rc = one_step(h, h->cur, h->stream))) return rc;
    ++h->t_steps;
  }
  for (lbm_s* p : h->subs) p->cur = h->cur;
  return LBM_OK;
}

// problem `prob` of a handle: the handle itself (single problem, prob 0) or a batch member
static lbm_s* member(lbm_t h, int prob) {
  if (!h) return nullptr;
  if (!h->is_batch()) return prob == 0 ? h : nullptr;
  if (prob < 0 || prob >= static_cast<int>(h->subs.size())) return nullptr;
  return h->subs[prob];
}

int lbm_read_C(lbm_t h, int prob, void* dst, int dst_is_device) {
  lbm_s* p = member(h, prob);
  if (!p || !dst) return LBM_EINVAL;
  const long long nodes = p->sp.nodes;
  if (dst_is_device) {
    // straight into the caller's device array, converted to FP64 on the way
    LBM_CUDA(lbm::launch_convert_out(p->dev.C, p->elem, static_cast<double*>(dst), nodes, h->stream));
  } else {
    LBM_CUDA(lbm::launch_convert_out(p->dev.C, p->elem, p->dev.stage, nodes, h->stream));
    LBM_CUDA(cudaMemcpyAsync(dst, p->dev.stage, sizeof(double) * nodes, cudaMemcpyDeviceToHost, h->stream));
  }
  return latched(p);
}

int lbm_read_F(lbm_t h, int mu, double* F_host) {
  if (!h || !F_host || mu < 0 || mu >= h->d) return LBM_EINVAL;
  if (h->is_batch()) return LBM_EINVAL;
  const long long nodes = h->sp.nodes;
  int rc = run_frac(h, h->stream);
  if (rc) return rc;
  if (h->sp.ksum > 1)  // split-K partial sums of the tensor-core operator (FP32 forms)
    LBM_CUDA(lbm::launch_sum_partials_out(static_cast<const float*>(h->dev.F) + (size_t)mu * nodes, h->sp.ksum,
                                          h->sp.pstride, h->dev.stage, nodes, h->stream));
  else
    LBM_CUDA(lbm::launch_convert_out((char*)h->dev.F + (size_t)mu * nodes * h->elem, h->elem, h->dev.stage, nodes,
                                     h->stream));
  LBM_CUDA(cudaMemcpyAsync(F_host, h->dev.stage, sizeof(double) * nodes, cudaMemcpyDeviceToHost, h->stream));
  return latched(h);
}

int lbm_read_f(lbm_t h, double* f_host) {
  if (!h || !f_host) return LBM_EINVAL;
  if (h->is_batch()) return LBM_EINVAL;
  const long long nodes = h->sp.nodes;
  for (int q = 0; q < h->Q; ++q) {
    LBM_CUDA(lbm::launch_convert_out((char*)h->dev.f[h->cur] + (size_t)q * nodes * h->elem, h->elem, h->dev.stage,
                                     nodes, h->stream));
    LBM_CUDA(cudaMemcpyAsync(f_host + (size_t)q * nodes, h->dev.stage, sizeof(double) * nodes,
                             cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
  }
  return latched(h);
}

int lbm_write_f(lbm_t h, const double* f_host) {
  if (!h || !f_host) return LBM_EINVAL;
  if (h->is_batch()) return LBM_EINVAL;
  const long long nodes = h->sp.nodes;
  for (int q = 0; q < h->Q; ++q) {
    LBM_CUDA(cudaMemcpyAsync(h->dev.stage, f_host + (size_t)q * nodes, sizeof(double) * nodes,
                             cudaMemcpyHostToDevice, h->stream));
    LBM_CUDA(lbm::launch_convert_in(h->dev.stage, (char*)h->dev.f[h->cur] + (size_t)q * nodes * h->elem, h->elem,
                                    nodes, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
  }
  LBM_CUDA(lbm::launch_moment(h, h->dev.f[h->cur], h->dev.C, h->stream));
  if (uses_tc(h)) LBM_CUDA(lbm::launch_split_C(h, h->stream));
  if (h->fld.on) LBM_CUDA(lbm::launch_scale_fields(h, h->stream));
  h->mass_valid = false;
  return latched(h);
}

namespace {

constexpr uint32_t kStateMagic = 0x464d424cu;  // "LBMF"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
  uint32_t magic, version;
  int32_t lattice, precision, nprob, pad;
  int64_t payload;  // bytes of populations after the header and the grid table
};

std::vector<lbm_s*> members(lbm_s* h) {
  if (h->is_batch()) return h->subs;
  return {h};
}

long long payload_bytes(lbm_s* h) {
  long long b = 0;
  for (lbm_s* p : members(h)) b += (long long)p->Q * p->sp.nodes * p->elem;
  return b;
}

long long state_bytes(lbm_s* h) {
  return (long long)sizeof(StateHeader) + 3LL * sizeof(int32_t) * (long long)members(h).size() + payload_bytes(h);
}

}  // namespace

long long lbm_state_size(lbm_t h) {
  if (!h) return LBM_EINVAL;
  return state_bytes(h);
}

int lbm_save(lbm_t h, void* dst_host, long long bytes) {
  if (!h || !dst_host || bytes < state_bytes(h)) return LBM_EINVAL;
  const std::vector<lbm_s*> ms = members(h);
  // the header's spare word carries the step counter (time of a source or wall values)
  StateHeader hd{kStateMagic, kStateVersion, h->prm.lattice, h->prm.precision, (int32_t)ms.size(),
                 (int32_t)std::min<long long>(h->t_steps, 0x7fffffff), payload_bytes(h)};
  char* out = static_cast<char*>(dst_host);
  std::memcpy(out, &hd, sizeof(hd));
  out += sizeof(hd);
  for (lbm_s* p : ms) {
    const int32_t g[3] = {p->sp.n[0], p->sp.n[1], p->sp.n[2]};
    std::memcpy(out, g, sizeof(g));
    out += sizeof(g);
  }
  for (lbm_s* p : ms) {
    const size_t b = (size_t)p->Q * p->sp.nodes * p->elem;
    LBM_CUDA(cudaMemcpyAsync(out, p->dev.f[h->cur], b, cudaMemcpyDeviceToHost, h->stream));
    out += b;
  }
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_load(lbm_t h, const void* src_host, long long bytes) {
  if (!h || !src_host || bytes < (long long)sizeof(StateHeader)) return LBM_EINVAL;
  const std::vector<lbm_s*> ms = members(h);
  StateHeader hd;
  const char* in = static_cast<const char*>(src_host);
  std::memcpy(&hd, in, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.lattice != h->prm.lattice ||
      hd.precision != h->prm.precision || hd.nprob != (int32_t)ms.size() || hd.payload != payload_bytes(h) ||
      bytes < state_bytes(h))
    return LBM_EINVAL;
  in += sizeof(hd);
  for (lbm_s* p : ms) {
    int32_t g[3];
    std::memcpy(g, in, sizeof(g));
    in += sizeof(g);
    if (g[0] != p->sp.n[0] || g[1] != p->sp.n[1] || g[2] != p->sp.n[2]) return LBM_EINVAL;
  }
  for (lbm_s* p : ms) {
    const size_t b = (size_t)p->Q * p->sp.nodes * p->elem;
    LBM_CUDA(cudaMemcpyAsync(p->dev.f[h->cur], in, b, cudaMemcpyHostToDevice, h->stream));
    in += b;
    LBM_CUDA(lbm::launch_moment(p, p->dev.f[h->cur], p->dev.C, h->stream));
    if (uses_tc(p)) LBM_CUDA(lbm::launch_split_C(p, h->stream));
    if (p->fld.on) LBM_CUDA(lbm::launch_scale_fields(p, h->stream));
    LBM_CUDA(cudaMemsetAsync(p->dev.flag, 0, sizeof(int), h->stream));
    p->mass_valid = false;
  }
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  h->t_steps = hd.pad;
  return LBM_OK;
}

namespace {

struct TuneCfg {
  int bn, ks, persist, chunk;
  int fused = 0;
};

// FP32 SIMT operator of a single problem: contraction split ks (1, 2, 4 or 8, at most
// the contraction blocks of 32 of the shortest axis); F grows to ks partial sums and the
// collide-stream tensor maps are re-encoded for it
int simt_replan(lbm_s* h, int ks) {
  if (!(ks == 1 || ks == 2 || ks == 4 || ks == 8)) return LBM_EINVAL;
  int kbmin = 1 << 30;
  for (int mu = 0; mu < h->d; ++mu) kbmin = std::min(kbmin, (h->sp.n[mu] + 31) / 32);
  if (ks > kbmin) return LBM_EINVAL;
  const size_t need = (size_t)ks * h->d * h->sp.nodes;
  if (need > h->f_elems) {
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    lbm::dev_free(h, h->dev.F);
    h->dev.F = nullptr;
    h->f_elems = 0;
    const int rc = alloc_bytes(h, &h->dev.F, need * sizeof(float));
    if (rc) return rc;
    h->f_elems = need;
  }
  h->sp.ksum = ks;
  h->sp.pstride = ks > 1 ? (long long)h->d * h->sp.nodes : 0;
  lbm::cs_release(h);
  return lbm::cs_prepare(h);
}

// the handle's launch configuration set to c (operator plan for tensor-core handles, the
// contraction split of the FP32 SIMT operator, collide-stream chunk for every handle);
// captured graphs are dropped
int apply_cfg(lbm_s* h, const TuneCfg& c) {
  int rc = LBM_OK;
  if (h->is_batch()) {
    h->cs_chunk = c.chunk;
    rc = lbm::cs_batch_prepare(h);
  } else {
    if (h->tc) {
      h->fused = false;
      if ((rc = lbm::tc_replan(h, c.bn, c.ks, c.persist))) return rc;
      lbm::cs_release(h);
      h->cs_chunk = c.chunk;
      if ((rc = lbm::cs_prepare(h))) return rc;
      h->pdl = pdl_fits(h);
      lbm::tc_set_pdl(h, h->pdl);
      if (c.fused) {
        if (h->fld.on) return LBM_EINVAL;  // the fused step runs the constant-coefficient march only
        if ((rc = lbm::fused_prepare(h))) return rc;
        h->fused = true;
      }
      // every operand copy of C current: the new plan may take the regrouped tf32 copies
      // from the collide-stream kernel, which the old one did not write
      LBM_CUDA(lbm::launch_split_C(h, h->stream));
    } else {
      h->cs_chunk = c.chunk;
      if (c.ks > 0 && h->elem == 4 && (rc = simt_replan(h, c.ks))) return rc;
      h->pdl = pdl_fits(h);
    }
  }
  drop_graphs(h);
  return rc;
}

// device time of one run of nsteps steps (graph replay)
int time_once(lbm_s* h, int nsteps, float* ms) {
  int rc = LBM_OK;
  cudaEvent_t e0, e1;
  LBM_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return record_cuda(cudaErrorMemoryAllocation, "lbm_autotune");
  }
  cudaError_t e = cudaEventRecord(e0, h->stream);
  if (e == cudaSuccess && (rc = lbm_step(h, nsteps)) == LBM_OK) {
    e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  return e == cudaSuccess ? LBM_OK : record_cuda(e, "lbm_autotune");
}

// device time of nsteps steps (graph replay), after as many warm-up steps; the faster of
// two timed runs
int time_steps(lbm_s* h, int nsteps, float* ms) {
  int rc = lbm_step(h, nsteps);  // captures the graphs
  if (rc) return rc;
  float best = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    float t = 0.f;
    if ((rc = time_once(h, nsteps, &t))) return rc;
    best = (rep == 0 || t < best) ? t : best;
  }
  *ms = best;
  return LBM_OK;
}


}  // namespace

int lbm_configure(lbm_t h, int bn, int ks, int persist, int chunk, int fused) {
  if (!h || chunk < 0) return LBM_EINVAL;
  TuneCfg c{0, 0, 0, chunk > 0 ? chunk : lbm::cs_chunk_default(h), fused ? 1 : 0};
  if (!h->is_batch() && h->tc) {
    lbm::tc_config(h, &c.bn, &c.ks, &c.persist);
    if (bn > 0) {
      c.bn = bn;
      c.ks = ks > 0 ? ks : 1;
      c.persist = persist ? 1 : 0;
    }
  } else if (!h->is_batch() && h->elem == 4 && bn == 0 && !persist && !fused) {
    c.ks = ks > 0 ? ks : h->sp.ksum;  // FP32 SIMT operator: its contraction split only
  } else if (bn > 0 || ks > 0 || persist || fused) {
    return LBM_EINVAL;  // no tensor-core operator to plan
  }
  return apply_cfg(h, c);
}

int lbm_autotune(lbm_t h, int nsteps, char* desc, int desc_len) {
  if (!h || nsteps < 2 || nsteps > 100000) return LBM_EINVAL;
  // whole graph replays, as lbm_step runs them (their length is even: buffer parity kept)
  nsteps = (nsteps + h->graph_steps - 1) / h->graph_steps * h->graph_steps;
  // the state is restored afterwards, bit for bit
  std::vector<char> state((size_t)state_bytes(h));
  int rc = lbm_save(h, state.data(), (long long)state.size());
  if (rc) return rc;
  TuneCfg cur{0, 0, 0, h->cs_chunk > 0 ? h->cs_chunk : lbm::cs_chunk_default(h), h->fused ? 1 : 0};
  if (!h->is_batch() && h->tc) lbm::tc_config(h, &cur.bn, &cur.ks, &cur.persist);
  const bool simt32 = !h->is_batch() && !h->tc && h->elem == 4;  // FP32 SIMT operator
  if (simt32) cur.ks = h->sp.ksum;
  // candidate chunks
  std::vector<int> chunks;
  if (h->is_batch()) {
    chunks = {2, 4, 8, 16};
  } else if (h->d == 2) {
    const int by = (h->sp.n[1] + 15) / 16;
    for (int c : {1, 2, 3, 4, 8}) if (c <= by) chunks.push_back(c);
  } else {
    const int d0 = lbm::cs_chunk_default(h);
    for (int c : {d0, d0 / 2, d0 + d0 / 2, d0 * 2, 1}) if (c >= 1 && c <= h->sp.n[2]) chunks.push_back(c);
  }
  if (std::find(chunks.begin(), chunks.end(), cur.chunk) == chunks.end()) chunks.push_back(cur.chunk);
  // candidate operator plans (tensor-core single problems; the FP32 SIMT split)
  std::vector<TuneCfg> ops;
  if (simt32)
    for (int ks : {1, 2, 4, 8}) {
      int kbmin = 1 << 30;
      for (int mu = 0; mu < h->d; ++mu) kbmin = std::min(kbmin, (h->sp.n[mu] + 31) / 32);
      if (ks <= kbmin) ops.push_back({0, ks, 0, cur.chunk});
    }
  if (!h->is_batch() && h->tc) {
    const int sms = lbm::device_sms();
    const int kbmin = lbm::tc_kbmin(h);
    // the forms with three weight parts take 64/128 columns
    const bool five = h->prm.precision == LBM_FP32_BF16SPLIT5 || h->prm.precision == LBM_FP32_BF16SPLIT6;
    for (int bn : {64, 128, 256})
      for (int ks : {1, 2, 4, 8}) {
        if (bn == 256 && (ks != 1 || five)) continue;
        if (ks > kbmin) continue;
        if (lbm::tc_count_tiles(h, bn) * ks > 2LL * sms) continue;  // at most two waves
        ops.push_back({bn, ks, 0, cur.chunk});
      }
    if (lbm::tc_count_tiles(h, 128) >= sms) ops.push_back({128, 1, 1, cur.chunk});
    if (!five && lbm::tc_count_tiles(h, 256) >= sms) ops.push_back({256, 1, 1, cur.chunk});
    // the fused step where the plan is one it covers (2-D bf16, 64/128 columns, split 2 or 4)
    const size_t nops = ops.size();
    for (size_t i = 0; i < nops; ++i)
      if (h->d == 2 && h->prm.precision == LBM_FP32_BF16SPLIT && !ops[i].persist && !h->fld.on &&
          (ops[i].bn == 64 || ops[i].bn == 128) && (ops[i].ks == 2 || ops[i].ks == 4)) {
        TuneCfg f = ops[i];
        f.fused = 1;
        ops.push_back(f);
      }
  }
  // coordinate search: operator plan with the current chunk, then the chunk.  Within a
  // stage every candidate is timed in two interleaved passes and keeps its faster time,
  // so that drift (clocks, caches) over the search does not favour late candidates.
  if ((rc = apply_cfg(h, cur)) || (rc = lbm_step(h, 4 * nsteps))) return rc;  // clocks up
  auto search = [&](std::vector<TuneCfg> cands, TuneCfg* winner, float* win_ms, float* first_ms) -> int {
    std::vector<float> t(cands.size(), -1.f);
    for (int pass = 0; pass < 2; ++pass)
      for (size_t i = 0; i < cands.size(); ++i) {
        float ms = 0.f;
        if (apply_cfg(h, cands[i]) != LBM_OK || time_steps(h, nsteps, &ms) != LBM_OK) continue;
        if (t[i] < 0.f || ms < t[i]) t[i] = ms;
      }
    int bi = -1;
    for (size_t i = 0; i < cands.size(); ++i)
      if (t[i] >= 0.f && (bi < 0 || t[i] < t[bi])) bi = static_cast<int>(i);
    if (bi < 0) return LBM_ECUDA;
    *winner = cands[bi];
    *win_ms = t[bi];
    if (first_ms) *first_ms = t[0];
    return LBM_OK;
  };
  std::vector<TuneCfg> stage1{cur};
  for (const TuneCfg& c : ops)
    if (!(c.bn == cur.bn && c.ks == cur.ks && c.persist == cur.persist && c.fused == cur.fused))
      stage1.push_back(c);
  TuneCfg best = cur;
  float best_ms = 0.f, base_ms = 0.f;
  if ((rc = search(stage1, &best, &best_ms, &base_ms))) return rc;
  std::vector<TuneCfg> stage2{best};
  for (int ch : chunks)
    if (ch != best.chunk) {
      TuneCfg c = best;
      c.chunk = ch;
      stage2.push_back(c);
    }
  if ((rc = search(stage2, &best, &best_ms, nullptr))) return rc;
  if ((rc = apply_cfg(h, best))) return rc;
  if ((rc = lbm_load(h, state.data(), (long long)state.size()))) return rc;
  if (desc && desc_len > 0) {
    if (h->tc && !h->is_batch())
      std::snprintf(desc, (size_t)desc_len,
                    "%soperator %s bn=%d ks=%d, collide chunk=%d: %.2f us/step (default %.2f)",
                    best.fused ? "fused step, " : "", best.persist ? "persistent" : "per-tile", best.bn, best.ks,
                    best.chunk, 1e3 * best_ms / nsteps, 1e3 * base_ms / nsteps);
    else if (simt32)
      std::snprintf(desc, (size_t)desc_len, "operator SIMT ks=%d, collide chunk=%d: %.2f us/step (default %.2f)",
                    best.ks, best.chunk, 1e3 * best_ms / nsteps, 1e3 * base_ms / nsteps);
    else
      std::snprintf(desc, (size_t)desc_len, "collide chunk=%d: %.2f us/step (default %.2f)", best.chunk,
                    1e3 * best_ms / nsteps, 1e3 * base_ms / nsteps);
  }
  return LBM_OK;
}

int lbm_mass(lbm_t h, int prob, double* mass) {
  lbm_s* p = member(h, prob);
  if (!p || !mass) return LBM_EINVAL;
  if (p->mass_valid)  // the latest step's warp partials: one small pass
    LBM_CUDA(lbm::launch_step_mass(p, 0.0, h->stream));
  else                // C from a re-initialisation: reduce C itself
    LBM_CUDA(lbm::launch_mass(p, p->dev.C, h->stream));
  LBM_CUDA(cudaMemcpyAsync(mass, p->dev.scalar, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return latched(p);
}

int lbm_set_mass_limit(lbm_t h, double limit) {
  if (!h || !(limit >= 0.0) || !std::isfinite(limit)) return LBM_EINVAL;
  h->mass_limit = limit;
  for (lbm_s* p : h->subs) p->mass_limit = limit;
  return LBM_OK;
}

// The per-node path's coefficient buffers from the arrays kept in fld (empty: the constants of
// lbm_params at every node), or freed when neither coefficients, a source nor wall values
// ask for that path; K_mu rebuilt accordingly; graphs dropped; re-initialised.
static int rebuild_fields(lbm_s* h) {
  const int d = h->d;
  const long long nodes = h->sp.nodes;
  const lbm_params& P = h->prm;
  const double e2 = (d == 2) ? 1.0 / 3.0 : 1.0 / 4.0, wi = h->sp.wi;
  const double ratio = P.dt / (P.dx * P.dx);
  const double* D_field = h->fld.D_host.empty() ? nullptr : h->fld.D_host.data();
  const double* g_field = h->fld.g_host.empty() ? nullptr : h->fld.g_host.data();
  const double* u_field = h->fld.u_host.empty() ? nullptr : h->fld.u_host.data();
  const bool on = D_field || g_field || u_field || h->fld.src || h->fld.cw;
  const int NC = (P.collision == LBM_MRT) ? d * (d + 1) / 2 : 1;
  std::vector<double> coll, advw, gv;
  if (on) {
    coll.assign((size_t)NC * nodes, 0.0);
    advw.assign((size_t)d * nodes, 0.0);
    gv.assign((size_t)d * nodes, 0.0);
    if (P.collision == LBM_BGK && !D_field) {
      // BGK keeps one relaxation time per node: the constant D must be spherical as well
      for (int a = 1; a < d; ++a)
        if (P.D[3 * a + a] != P.D[0]) return LBM_EINVAL;
    }
    for (long long i = 0; i < nodes; ++i) {
      double Dm[9];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) Dm[a * d + b] = D_field ? D_field[((size_t)a * d + b) * nodes + i] : P.D[3 * a + b];
      for (int k = 0; k < d * d; ++k)
        if (!std::isfinite(Dm[k])) return LBM_EINVAL;
      if (P.collision == LBM_BGK) {
        // one relaxation time per node: D(x) spherical (Eq. Diffusion_Coefficient_3D)
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b)
            if ((a == b && Dm[a * d + b] != Dm[0]) || (a != b && Dm[a * d + b] != 0.0)) return LBM_EINVAL;
        if (!(Dm[0] > 0.0)) return LBM_EINVAL;
        coll[i] = 1.0 / (Dm[0] * ratio / e2 + 0.5);
      } else {
        // flux block of Lambda^-1: lambdabar(x) = D(x) dt/(e^2 dx^2) + Id/2 (Eq. D_ab), SPD;
        // its inverse R(x) holds the rates of the flux moments (Eq. MatrixS)
        double lb[9], R[9];
        for (int a = 0; a < d; ++a)
          for (int b = 0; b < d; ++b) lb[a * d + b] = Dm[a * d + b] * ratio / e2 + (a == b ? 0.5 : 0.0);
        if (!is_spd(d, lb) || !invert(d, lb, R)) return LBM_EINVAL;
        int k = 0;
        for (int a = 0; a < d; ++a)
          for (int b = a; b < d; ++b) coll[(size_t)(k++) * nodes + i] = 0.5 * (R[a * d + b] + R[b * d + a]);
      }
      for (int mu = 0; mu < d; ++mu) {
        const double g = g_field ? g_field[(size_t)mu * nodes + i] : P.g[mu];
        const double u = u_field ? u_field[(size_t)mu * nodes + i] : P.u[mu];
        if (!(g > 0.0) || !std::isfinite(g) || !std::isfinite(u)) return LBM_EINVAL;
        gv[(size_t)mu * nodes + i] = g;
        advw[(size_t)mu * nodes + i] = (P.dt / P.dx) * u * wi / e2;
      }
    }
  }
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  drop_graphs(h);  // the captured launches take other kernels and arguments now
  for (void* p : {h->fld.coll, h->fld.advw, h->fld.g, h->fld.G}) lbm::dev_free(h, p);
  h->fld.coll = h->fld.advw = h->fld.g = h->fld.G = nullptr;
  h->fld.on = false;
  int rc = LBM_OK;
  if (on) {
    const size_t E = h->elem;
    if ((rc = alloc_bytes(h, &h->fld.coll, E * NC * nodes)) || (rc = alloc_bytes(h, &h->fld.advw, E * d * nodes)))
      return rc;
    // g(x) for the SIMT operator's input G = g C, or for the tensor-core operands of g_mu(x) C
    // (the tensor-core forms fold a uniform g into K and need neither); G itself for the
    // SIMT operator and for tf32, whose operands are regrouped from it
    const bool tf32 = h->prm.precision == LBM_FP32_TF32SPLIT;
    if ((!h->tc || g_field) && (rc = alloc_bytes(h, &h->fld.g, E * d * nodes))) return rc;
    if ((!h->tc || (g_field && tf32)) && (rc = alloc_bytes(h, &h->fld.G, E * d * nodes))) return rc;
    const std::pair<const std::vector<double>*, void*> ups[3] = {{&coll, h->fld.coll}, {&advw, h->fld.advw},
                                                                 {&gv, h->fld.g}};
    for (const auto& up : ups) {
      if (!up.second) continue;
      const std::vector<double>& v = *up.first;
      for (size_t off = 0; off < v.size(); off += (size_t)nodes) {  // one plane of nodes at a time
        LBM_CUDA(cudaMemcpyAsync(h->dev.stage, v.data() + off, sizeof(double) * nodes, cudaMemcpyHostToDevice,
                                 h->stream));
        LBM_CUDA(lbm::launch_convert_in(h->dev.stage, (char*)up.second + off * E, h->elem, nodes, h->stream));
        LBM_CUDA(cudaStreamSynchronize(h->stream));
      }
    }
    h->fld.on = true;
    h->fused = false;  // the fused step runs the constant-coefficient march only
  }
  h->pdl = pdl_fits(h);  // the march, and with tf32 whether the operands need a launch of their own
  if (h->tc) lbm::tc_set_pdl(h, h->pdl);
  h->fld.gvar = h->fld.on && g_field != nullptr;
  {  // g inside the integrals (K without g), or folded into K
    Derived dv;
    if ((rc = derive(&h->prm, &dv))) return rc;
    std::vector<std::vector<double>> Kall;
    if ((rc = upload_weights(h, dv.h, h->tc ? &Kall : nullptr))) return rc;
    if (h->tc && ((rc = lbm::tc_set_weights(h, Kall)) || (rc = lbm::tc_set_gfield(h, h->fld.gvar)))) return rc;
  }
  return lbm_reset(h);
}

// the per-node path applies to single problems in every form; the tensor-core forms fold a
// uniform g into K (as without fields) and need BGK's h_mu = 1 (a spherical constant D)
static int fields_supported(lbm_t h) {
  if (!h || h->is_batch()) return LBM_EINVAL;
  if (h->tc && h->prm.collision == LBM_BGK)
    for (int a = 1; a < h->d; ++a)
      if (h->prm.D[4 * a] != h->prm.D[0]) return LBM_ENOTSUP;
  return LBM_OK;
}

// host array of `count` nodes-long planes into a device array in the working precision
static int upload_planes(lbm_s* h, const double* host, int count, void** dst) {
  const long long nodes = h->sp.nodes;
  lbm::dev_free(h, *dst);
  *dst = nullptr;
  int rc = alloc_bytes(h, dst, (size_t)h->elem * count * nodes);
  if (rc) return rc;
  for (int k = 0; k < count; ++k) {
    LBM_CUDA(cudaMemcpyAsync(h->dev.stage, host + (size_t)k * nodes, sizeof(double) * nodes, cudaMemcpyHostToDevice,
                             h->stream));
    LBM_CUDA(lbm::launch_convert_in(h->dev.stage, (char*)*dst + (size_t)k * nodes * h->elem, h->elem, nodes,
                                    h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

// the slot table of the time factors exists while a source or wall values are set
static int ensure_time_table(lbm_s* h) {
  const bool want = h->fld.src || h->fld.cw;
  if (want && !h->fld.tf) {
    h->fld.tf_slots = h->graph_steps;
    return alloc_bytes(h, (void**)&h->fld.tf, sizeof(double) * 2 * h->fld.tf_slots);
  }
  if (!want && h->fld.tf) {
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    lbm::dev_free(h, h->fld.tf);
    h->fld.tf = nullptr;
    h->fld.tf_slots = 0;
  }
  return LBM_OK;
}

int lbm_set_fields(lbm_t h, const double* D_field, const double* g_field, const double* u_field) {
  int rc = fields_supported(h);
  if (rc) return rc;
  const size_t nodes = (size_t)h->sp.nodes, d = (size_t)h->d;
  // validate on a copy first: the handle stays unchanged when the arrays are rejected
  lbm::FieldState keep;
  keep.D_host.swap(h->fld.D_host);
  keep.g_host.swap(h->fld.g_host);
  keep.u_host.swap(h->fld.u_host);
  if (D_field) h->fld.D_host.assign(D_field, D_field + d * d * nodes);
  if (g_field) h->fld.g_host.assign(g_field, g_field + d * nodes);
  if (u_field) h->fld.u_host.assign(u_field, u_field + d * nodes);
  h->fld.coeff = D_field || g_field || u_field;
  rc = rebuild_fields(h);
  if (rc == LBM_EINVAL) {  // restore the previous arrays
    h->fld.D_host.swap(keep.D_host);
    h->fld.g_host.swap(keep.g_host);
    h->fld.u_host.swap(keep.u_host);
    h->fld.coeff = !h->fld.D_host.empty() || !h->fld.g_host.empty() || !h->fld.u_host.empty();
    const int rc2 = rebuild_fields(h);
    return rc2 ? rc2 : LBM_EINVAL;
  }
  return rc;
}

int lbm_set_params(lbm_t h, const lbm_params* prm) {
  if (!h || !prm || h->is_batch()) return LBM_EINVAL;
  const lbm_params& o = h->prm;
  if (prm->lattice != o.lattice || prm->collision != o.collision || prm->precision != o.precision ||
      prm->variant != o.variant)
    return LBM_EINVAL;
  for (int mu = 0; mu < 3; ++mu)
    if (prm->grid[mu] != o.grid[mu]) return LBM_EINVAL;
  Derived dv;
  int rc = derive(prm, &dv);
  if (rc) return rc;
  if (h->tc && h->fld.on && prm->collision == LBM_BGK)
    for (int a = 1; a < h->d; ++a)
      if (prm->D[4 * a] != prm->D[0]) return LBM_ENOTSUP;  // as lbm_set_fields
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  drop_graphs(h);  // the captured launches carry the old constants
  const lbm_params keep = h->prm;
  const lbm::StepParams keep_sp = h->sp;
  h->prm = *prm;
  lbm::StepParams sp = dv.sp;
  sp.ksum = keep_sp.ksum;  // the launch plan stays: its partial sums of F
  sp.pstride = keep_sp.pstride;
  h->sp = sp;
  if (h->fld.on) {
    rc = rebuild_fields(h);  // per-node rates, g and the weights from the new constants
  } else {
    std::vector<std::vector<double>> Kall;
    rc = upload_weights(h, dv.h, h->tc ? &Kall : nullptr);
    if (!rc && h->tc) rc = lbm::tc_set_weights(h, Kall);
    if (!rc) rc = lbm_reset(h);
  }
  if (rc == LBM_EINVAL) {  // e.g. a field no longer admissible with the new constants
    h->prm = keep;
    h->sp = keep_sp;
    if (h->fld.on) {
      rebuild_fields(h);
    } else {
      std::vector<std::vector<double>> Kall;
      Derived d0;
      if (!derive(&keep, &d0) && !upload_weights(h, d0.h, h->tc ? &Kall : nullptr) && h->tc)
        lbm::tc_set_weights(h, Kall);
      lbm_reset(h);
    }
  }
  return rc;
}

int lbm_set_source(lbm_t h, const double* S_field, double rate) {
  int rc = fields_supported(h);
  if (rc) return rc;
  if (!std::isfinite(rate)) return LBM_EINVAL;
  if (S_field)
    for (long long i = 0; i < h->sp.nodes; ++i)
      if (!std::isfinite(S_field[i])) return LBM_EINVAL;
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (S_field) {
    if ((rc = upload_planes(h, S_field, 1, &h->fld.src))) return rc;
  } else {
    lbm::dev_free(h, h->fld.src);
    h->fld.src = nullptr;
  }
  h->fld.src_rate = rate;
  if ((rc = ensure_time_table(h))) return rc;
  return rebuild_fields(h);
}

int lbm_set_wall_values(lbm_t h, const double* Cw_field, double rate) {
  int rc = fields_supported(h);
  if (rc) return rc;
  if (!std::isfinite(rate)) return LBM_EINVAL;
  if (Cw_field)
    for (long long i = 0; i < h->sp.nodes; ++i)
      if (!std::isfinite(Cw_field[i])) return LBM_EINVAL;
  LBM_CUDA(cudaStreamSynchronize(h->stream));
  if (Cw_field) {
    if ((rc = upload_planes(h, Cw_field, 1, &h->fld.cw))) return rc;
  } else {
    lbm::dev_free(h, h->fld.cw);
    h->fld.cw = nullptr;
  }
  h->fld.cw_rate = rate;
  if ((rc = ensure_time_table(h))) return rc;
  return rebuild_fields(h);
}

int lbm_sync(lbm_t h) {
  if (!h) return LBM_EINVAL;
  if (h->is_batch()) {
    int worst = LBM_OK;
    for (lbm_s* p : h->subs) {
      const int rc = latched(p);
      if (rc == LBM_ERR_TIMEOUT || rc == LBM_ECUDA || rc == LBM_ENOMEM) return rc;
      if (rc) worst = rc;
    }
    return worst;
  }
  return latched(h);
}

int lbm_get_stream(lbm_t h, void** stream) {
  if (!h || !stream) return LBM_EINVAL;
  *stream = h->stream;
  return LBM_OK;
}

int lbm_launches_per_step(lbm_t h, int* n) {
  if (!h || !n) return LBM_EINVAL;
  int k = h->launches_per_step;
  if (!h->is_batch() && uses_tc(h)) {
    if (h->fused) k = 0;  // one cooperative launch per lbm_step call (up to 4096 steps)
    else k = 2 + ((h->prm.precision == LBM_FP32_TF32SPLIT && !lbm::cs_writes_T(h)) ? h->d - 1 : 0);
  }
  *n = k;
  return LBM_OK;
}

int lbm_frac_matrix(const lbm_params* prm, int mu, double* K_host) {
  if (!K_host) return LBM_EINVAL;
  Derived dv;
  int rc = derive(prm, &dv);
  if (rc) return rc;
  const int d = (prm->lattice == LBM_D2Q5) ? 2 : 3;
  if (mu < 0 || mu >= d) return LBM_EINVAL;
  lbm::build_frac_matrix(prm->alpha[mu], prm->p[mu], prm->g[mu] * dv.h[mu], prm->grid[mu], prm->dx, prm->variant,
                         K_host);
  return LBM_OK;
}

static int reset_hook(lbm_s* h) { return lbm_reset(h); }
static int step_hook(lbm_s* h, int& cur, cudaStream_t s) { return one_step(h, cur, s); }

int lbm_grad(lbm_t h, int nsnap, const int* snap_steps, const double* obs, int ckpt_every, double* loss,
             double* grad) {
  if (!h || nsnap < 1 || !snap_steps || !obs || ckpt_every < 1 || !loss || !grad) return LBM_EINVAL;
  if (h->is_batch() || h->fld.on) return LBM_ENOTSUP;
  for (int k = 0; k < nsnap; ++k)
    if (snap_steps[k] < 0 || (k > 0 && snap_steps[k] <= snap_steps[k - 1])) return LBM_EINVAL;
  if (h->tc) {
    // split-precision forms: the adjoint of the plain FP32 scheme, which these forms follow
    // within their stated error, on an FP32 copy of the problem started from the handle's
    // initial concentration (same stream, same device-memory hooks)
    lbm_params p32 = h->prm;
    p32.precision = LBM_FP32;
    const long long nodes = h->sp.nodes;
    std::vector<double> C0((size_t)nodes);
    LBM_CUDA(lbm::launch_convert_out(h->dev.C0, h->elem, h->dev.stage, nodes, h->stream));
    LBM_CUDA(cudaMemcpyAsync(C0.data(), h->dev.stage, sizeof(double) * nodes, cudaMemcpyDeviceToHost, h->stream));
    LBM_CUDA(cudaStreamSynchronize(h->stream));
    lbm_t t = nullptr;
    int rc = create_problem(&p32, C0.data(), h->stream, false, &t, &h->mem);
    if (rc) return rc;
    rc = lbm_grad(t, nsnap, snap_steps, obs, ckpt_every, loss, grad);
    lbm_destroy(t);
    const int rc2 = lbm_reset(h);
    return rc ? rc : rc2;
  }
  double dOm[3][lbm::kMaxQ][lbm::kMaxQ];
  int rc = derive_dOmega(&h->prm, dOm);
  if (rc) return rc;
  Derived dv;
  if ((rc = derive(&h->prm, &dv))) return rc;
  const int d = h->d;
  const bool bgk = h->prm.collision == LBM_BGK;
  size_t gsz = 0;
  for (int mu = 0; mu < d; ++mu) gsz += (size_t)h->sp.n[mu] * h->sp.n[mu];
  std::vector<double> G(gsz), gsum(2 * d);
  const lbm::AdjHooks hooks{reset_hook, step_hook};
  rc = lbm::adjoint_grad(h, hooks, nsnap, snap_steps, obs, ckpt_every, dOm, loss, G.data(), gsum.data());
  const int rc2 = lbm_reset(h);  // the populations were overwritten by the recomputation
  if (rc) return rc;
  if (rc2) return rc2;
  size_t goff = 0;
  double KG[3] = {0.0, 0.0, 0.0};  // <K_mu, G_mu>, for BGK's h_mu = D_mumu / max D
  for (int mu = 0; mu < d; ++mu) {
    const int side = h->sp.n[mu];
    const double scale = h->prm.g[mu] * dv.h[mu];
    std::vector<double> da((size_t)side * side), dp((size_t)side * side), K;
    lbm::build_frac_matrix_grad(h->prm.alpha[mu], h->prm.p[mu], scale, side, h->prm.dx, h->prm.variant, da.data(),
                                dp.data());
    if (bgk) {
      K.resize((size_t)side * side);
      lbm::build_frac_matrix(h->prm.alpha[mu], h->prm.p[mu], scale, side, h->prm.dx, h->prm.variant, K.data());
    }
    double sa = 0.0, sp_ = 0.0, sk = 0.0;
    for (size_t i = 0; i < da.size(); ++i) {
      sa += da[i] * G[goff + i];
      sp_ += dp[i] * G[goff + i];
      if (bgk) sk += K[i] * G[goff + i];
    }
    KG[mu] = sk;
    grad[mu] = sa;
    grad[d + mu] = sp_;
    grad[2 * d + mu] = gsum[d + mu];
    grad[3 * d + mu] = gsum[mu];
    goff += (size_t)side * side;
  }
  if (bgk) {
    // K_nu is proportional to h_nu = D_nunu / max D (end of Section 2.2):
    // dK_nu/dD_mumu = K_nu (delta_nu,mu / D_nunu - share_mu / max D)
    double share[3], dmax;
    bgk_max_share(&h->prm, d, share, &dmax);
    for (int mu = 0; mu < d; ++mu) {
      double s = KG[mu] / h->prm.D[4 * mu];
      for (int nu = 0; nu < d; ++nu) s -= share[mu] / dmax * KG[nu];
      grad[2 * d + mu] += s;
    }
  }
  return LBM_OK;
}

int lbm_frac_matrix_grad(const lbm_params* prm, int mu, double* dK_dalpha, double* dK_dp) {
  if (!dK_dalpha || !dK_dp) return LBM_EINVAL;
  Derived dv;
  int rc = derive(prm, &dv);
  if (rc) return rc;
  const int d = (prm->lattice == LBM_D2Q5) ? 2 : 3;
  if (mu < 0 || mu >= d) return LBM_EINVAL;
  lbm::build_frac_matrix_grad(prm->alpha[mu], prm->p[mu], prm->g[mu] * dv.h[mu], prm->grid[mu], prm->dx, prm->variant,
                              dK_dalpha, dK_dp);
  return LBM_OK;
}

double lbm_digamma(double x) { return lbm::digamma_fn(x); }

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return LBM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mem_mutex);
  g_mem.alloc = alloc;
  g_mem.release = release;
  g_mem.ctx = alloc ? ctx : nullptr;
  return LBM_OK;
}

void lbm_destroy(lbm_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (lbm_s* p : h->subs) lbm_destroy(p);
  h->subs.clear();
  lbm::dev_free(h, h->batch_cs);
  lbm::dev_free(h, h->batch_cs_start);
  h->batch_cs = nullptr;
  h->batch_cs_start = nullptr;
  free_all(h);
  delete h;
}

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "device allocation failed";
    case LBM_ECUDA: return "CUDA runtime error";
    case LBM_ERR_UNSTABLE: return "non-finite concentration (numerical instability)";
    case LBM_ENOTSUP: return "not supported by this build";
    case LBM_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case LBM_ETOOBIG: return "input exceeds the static scratch capacity";
    default: return "unknown error";
  }
}

const char* lbm_last_cuda_error(void) { return g_cuda_msg; }

}  // extern "C"
