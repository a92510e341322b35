// Discrete adjoint of the time step and parameter gradients of a snapshot loss.
//
// With the parameters fixed, one time step of Algorithm 1 is linear in the
// populations f: C = <1|f>, F_mu = K_mu C along axis mu, feq = E(C, F) (Eqs. Feq,
// CoeffA_FADE3D), f* = f - Omega (f - feq) (Eqs. LBE_Ket / MRT-Coll), push streaming
// (Eq. Def_Translation) and the walls (Eq. Dirichlet_BC, affine).  Its transpose, in
// reverse order, with mu = dL/df(t+1):
//   walls      each known population b at a wall node z:  mu_b - (1/k) sum_{unknown u} mu_u
//   streaming  lambda*_q(y) = (walls^T mu)_q(y + e_q), 0 where y + e_q leaves the domain
//   collision  lambda_f = (I - Omega)^T lambda*,  lambda_feq = Omega^T lambda*
//   equilibrium lambda_C += lambda_feq_0 + sum_mu a_mu (lambda_feq_{2mu+1} - lambda_feq_{2mu+2})
//              lambda_F_mu = -w_0 lambda_feq_0 + w_i (lambda_feq_{2mu+1} + lambda_feq_{2mu+2})
//   operator   lambda_C += sum_mu K_mu^T lambda_F_mu   (the SIMT GEMM with K and K^T swapped)
//   moment     dL/df_q(t) = lambda_f_q + lambda_C (+ the snapshot residual 2 (C - obs)).
// Parameter gradients (sums over steps of lambda^T dA/dtheta f):
//   alpha_mu, p_mu : <dK_mu/dtheta, G_mu>,  G_mu[n][l] = sum_t sum_lines lambda_F(n) C_t(l)
//   D_mumu        : - sum lambda*^T (dOmega/dD_mumu) (f - feq)
//   u_mu          : sum (dt/dx)(w_i/e^2) C (lambda_feq_{2mu+1} - lambda_feq_{2mu+2})
// plus the initial condition f(0) = feq(C0, K C0).  Forward states are recomputed from
// checkpoints taken every `ckpt` steps.  Gradient sums are FP64; G_mu is one GEMM per
// checkpoint segment (FP32 forms: products summed in FP32 over 16 terms, then in FP64).
#include <cmath>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kThreads = 256;

template <typename real>
struct AdjConst {
  int n[3];
  long long nodes;
  real omT[kMaxQ][kMaxQ];       // Omega^T
  real dOm[3][kMaxQ][kMaxQ];    // dOmega / dD_mumu
  real w0, wi;
  real advw[3];                 // dfeq_{2mu+1}/dC = (dt/dx) u_mu w_i / e^2
  real cu;                      // dfeq_{2mu+1}/du_mu per unit C = (dt/dx) w_i / e^2
};

__device__ __forceinline__ void evec(int q, int& ex, int& ey, int& ez) {
  ex = (q == 1) - (q == 2);
  ey = (q == 3) - (q == 4);
  ez = (q == 5) - (q == 6);
}

// (1/k) sum of mu over the k unknown (wall-filled) populations of node (x, y, z); 0 inside
template <typename real, int D>
__device__ __forceinline__ real wall_nu(const AdjConst<real>& c, const real* __restrict__ lam, long long node, int x,
                                        int y, int z) {
  constexpr int Q = 2 * D + 1;
  real s = static_cast<real>(0);
  int k = 0;
#pragma unroll
  for (int q = 1; q < Q; ++q) {
    int ex, ey, ez;
    evec(q, ex, ey, ez);
    const int sx = x - ex, sy = y - ey, sz = z - ez;
    if (sx < 0 || sx >= c.n[0] || sy < 0 || sy >= c.n[1] || sz < 0 || sz >= c.n[2]) {
      s += lam[q * c.nodes + node];
      ++k;
    }
  }
  return k ? s / static_cast<real>(k) : static_cast<real>(0);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Adds the block's sums of v[0..K) to part[blockIdx.x * K + k] (fixed order, so repeated
// calls with the same grid accumulate deterministically).
template <int K>
__device__ __forceinline__ void block_accumulate(const double* v, double* __restrict__ part) {
  __shared__ double s[K][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double w = warp_sum(v[k]);
    if (lane == 0) s[k][wid] = w;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double acc = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) acc += s[threadIdx.x][i];
    part[blockIdx.x * K + threadIdx.x] += acc;
  }
}

template <typename real, int D>
__global__ void __launch_bounds__(kThreads)
adj_step_kernel(const AdjConst<real> c, const real* __restrict__ f, const real* __restrict__ F,
                const real* __restrict__ lam, real* __restrict__ lf, real* __restrict__ lcl, real* __restrict__ lF,
                long long lFs, double* __restrict__ part) {
  constexpr int Q = 2 * D + 1;
  const long long nodes = c.nodes;
  const long long node = blockIdx.x * (long long)kThreads + threadIdx.x;
  double g[2 * D];
#pragma unroll
  for (int k = 0; k < 2 * D; ++k) g[k] = 0.0;
  if (node < nodes) {
    const int n0 = c.n[0], n1 = c.n[1];
    const int x = static_cast<int>(node % n0);
    const int y = static_cast<int>((node / n0) % n1);
    const int z = static_cast<int>(node / ((long long)n0 * n1));
    // lambda* (adjoint of the post-collision populations of this node)
    real ls[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int ex, ey, ez;
      evec(q, ex, ey, ez);
      const int tx = x + ex, ty = y + ey, tz = z + ez;
      if (tx < 0 || tx >= n0 || ty < 0 || ty >= n1 || tz < 0 || tz >= c.n[2]) {
        ls[q] = static_cast<real>(0);
      } else {
        const long long t = tx + (long long)n0 * (ty + (long long)n1 * tz);
        ls[q] = lam[q * nodes + t] - wall_nu<real, D>(c, lam, t, tx, ty, tz);
      }
    }
    // forward state of this node
    real fv[Q], Fv[D];
#pragma unroll
    for (int q = 0; q < Q; ++q) fv[q] = f[q * nodes + node];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) Fv[mu] = F[mu * nodes + node];
    real C = fv[0];
#pragma unroll
    for (int q = 1; q < Q; ++q) C += fv[q];
    real sumF = Fv[0];
#pragma unroll
    for (int mu = 1; mu < D; ++mu) sumF += Fv[mu];
    real dl[Q];  // f - feq
    dl[0] = fv[0] - (C - c.w0 * sumF);
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const real a = c.wi * Fv[mu], b = c.advw[mu] * C;
      dl[2 * mu + 1] = fv[2 * mu + 1] - (a + b);
      dl[2 * mu + 2] = fv[2 * mu + 2] - (a - b);
    }
    // collision transpose
    real le[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      real acc = c.omT[i][0] * ls[0];
#pragma unroll
      for (int j = 1; j < Q; ++j) acc += c.omT[i][j] * ls[j];
      le[i] = acc;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) lf[q * nodes + node] = ls[q] - le[q];
    real lc = le[0];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) lc += c.advw[mu] * (le[2 * mu + 1] - le[2 * mu + 2]);
    lcl[node] = lc;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      lF[mu * lFs + node] = -c.w0 * le[0] + c.wi * (le[2 * mu + 1] + le[2 * mu + 2]);
      g[mu] = static_cast<double>(c.cu) * static_cast<double>(C) *
              static_cast<double>(le[2 * mu + 1] - le[2 * mu + 2]);
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        real row = static_cast<real>(0);
#pragma unroll
        for (int j = 0; j < Q; ++j) row += c.dOm[mu][i][j] * dl[j];
        acc += static_cast<double>(ls[i]) * static_cast<double>(row);
      }
      g[D + mu] = -acc;
    }
  }
  block_accumulate<2 * D>(g, part);
}

// f(0) = feq(C0, K C0): lambda_F of the initial fractional terms and the u-gradient part
template <typename real, int D>
__global__ void __launch_bounds__(kThreads)
adj_init_kernel(const AdjConst<real> c, const real* __restrict__ C0, const real* __restrict__ lam,
                real* __restrict__ lF, double* __restrict__ part) {
  const long long nodes = c.nodes;
  const long long node = blockIdx.x * (long long)kThreads + threadIdx.x;
  double g[2 * D];
#pragma unroll
  for (int k = 0; k < 2 * D; ++k) g[k] = 0.0;
  if (node < nodes) {
    const real l0 = lam[node];
    const real C = C0[node];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const real a = lam[(2 * mu + 1) * nodes + node], b = lam[(2 * mu + 2) * nodes + node];
      lF[mu * nodes + node] = -c.w0 * l0 + c.wi * (a + b);
      g[mu] = static_cast<double>(c.cu) * static_cast<double>(C) * static_cast<double>(a - b);
    }
  }
  block_accumulate<2 * D>(g, part);
}

// lambda(t) = lambda_f + lambda_C(local) + sum_mu K_mu^T lambda_F_mu (+ 2 (C - obs))
template <typename real, int D>
__global__ void adj_combine_kernel(long long nodes, const real* __restrict__ lf, const real* __restrict__ lcl,
                                   const real* __restrict__ lcf, const real* __restrict__ C,
                                   const real* __restrict__ obs, real* __restrict__ lam) {
  constexpr int Q = 2 * D + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
       i += (long long)gridDim.x * blockDim.x) {
    real r = lcl[i];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) r += lcf[mu * nodes + i];
    if (obs) r += static_cast<real>(2) * (C[i] - obs[i]);
#pragma unroll
    for (int q = 0; q < Q; ++q) lam[q * nodes + i] = lf[q * nodes + i] + r;
  }
}

// lambda = 2 (C - obs) on every population (the last snapshot)
template <typename real, int Q>
__global__ void adj_residual_kernel(long long nodes, const real* __restrict__ C, const real* __restrict__ obs,
                                    real* __restrict__ lam) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
       i += (long long)gridDim.x * blockDim.x) {
    const real r = static_cast<real>(2) * (C[i] - obs[i]);
#pragma unroll
    for (int q = 0; q < Q; ++q) lam[q * nodes + i] = r;
  }
}

// node index of (line o, position k along axis mu)
// G_mu[n][l] += sum_t sum_lines lambda_F_mu,t(line, n) C_t(line, l) over the steps of one
// checkpoint segment, as one SIMT GEMM whose reduction index runs over (step, line).
// The element (row n, reduction index jk = j * kin + k) of either operand sits at
// j * sj + n * ldn + k * ldk; the three axes map onto this as
//   x: ldn = 1,       ldk = n0, kin = steps * lines, nj = 1   (step stride nodes = lines * n0)
//   y: ldn = n0,      ldk = 1,  kin = n0, sj = n0 n1, nj = steps * n2
//   z: ldn = n0 n1,   ldk = 1,  kin = n0 n1, sj = nodes, nj = steps.
// Each block owns a 64x64 tile of G and one slice of the reduction index; partial sums go
// to their own FP64 slab and are added in slab order (deterministic).  FP32 operands are
// multiplied and summed in FP32 over one 16-deep slice, then added into FP64 accumulators.
struct GLayout {
  int side;
  long long kin, sj, ldn, ldk, ktotal, kchunk;
};

constexpr int GB = 64, GK = 16;

template <typename real, bool NCONTIG>
__global__ void __launch_bounds__(256)
adj_G_gemm(const GLayout L, const real* __restrict__ A, const real* __restrict__ B, double* __restrict__ part) {
  __shared__ real As[GK][GB + 4];
  __shared__ real Bs[GK][GB + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int n0 = blockIdx.y * GB, l0 = blockIdx.x * GB;
  const long long kb = blockIdx.z * L.kchunk;
  const long long ke = min(kb + L.kchunk, L.ktotal);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  constexpr int R = (GB * GK) / 256;
  // NCONTIG: consecutive threads walk the row index (contiguous); else the reduction index.
  // (j, k) of each loaded reduction index is stepped by GK per slice (no division in the loop)
  long long jj[R], kq[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = tid + r * 256;
    const long long jk = kb + (NCONTIG ? (e / GB) : (e % GK));
    jj[r] = jk / L.kin;
    kq[r] = jk - jj[r] * L.kin;
  }
  for (long long k0 = kb; k0 < ke; k0 += GK) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = tid + r * 256;
      const int rr = NCONTIG ? (e % GB) : (e / GK);
      const int kk = NCONTIG ? (e / GB) : (e % GK);
      real a = static_cast<real>(0), b = static_cast<real>(0);
      if (k0 + kk < ke) {
        const long long base = jj[r] * L.sj + kq[r] * L.ldk;
        if (n0 + rr < L.side) a = A[base + (long long)(n0 + rr) * L.ldn];
        if (l0 + rr < L.side) b = B[base + (long long)(l0 + rr) * L.ldn];
      }
      As[kk][rr] = a;
      Bs[kk][rr] = b;
      kq[r] += GK;
      while (kq[r] >= L.kin) {
        kq[r] -= L.kin;
        ++jj[r];
      }
    }
    __syncthreads();
    real sub[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sub[i][j] = static_cast<real>(0);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      real a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sub[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += static_cast<double>(sub[i][j]);
    __syncthreads();
  }
  double* slab = part + (size_t)blockIdx.z * L.side * L.side;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + ty + 16 * i;
    if (n >= L.side) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int l = l0 + tx + 16 * j;
      if (l < L.side) slab[(size_t)n * L.side + l] = acc[i][j];
    }
  }
}

__global__ void adj_G_reduce(long long count, int nslab, const double* __restrict__ part, double* __restrict__ G) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int z = 0; z < nslab; ++z) acc += part[(size_t)z * count + i];
    G[i] += acc;
  }
}

// slabs of the reduction split for one side x side G: about two blocks per SM, at least
// 1024 reduction indices per block, at most kMaxSlabs
constexpr int kMaxSlabs = 32;

int g_slabs(int side, long long ktotal) {
  const long long tiles = (long long)((side + GB - 1) / GB) * ((side + GB - 1) / GB);
  long long z = (304 + tiles - 1) / tiles;
  z = std::min<long long>(z, std::max<long long>(1, ktotal / 1024));
  return static_cast<int>(std::max<long long>(1, std::min<long long>(z, kMaxSlabs)));
}

// G_mu += sum over `steps` consecutive steps (operand step stride = nodes)
template <typename real>
cudaError_t accumulate_G(const lbm_s* h, int mu, int steps, const real* lF, const real* C, double* G, double* part,
                         cudaStream_t s) {
  const long long n0 = h->sp.n[0], n1 = h->sp.n[1], n2 = h->sp.n[2];
  const long long nodes = h->sp.nodes;
  GLayout L{};
  L.side = h->sp.n[mu];
  if (mu == 0) {
    L.ldn = 1; L.ldk = n0; L.kin = steps * (nodes / n0); L.sj = 0; L.ktotal = L.kin;
  } else if (mu == 1) {
    L.ldn = n0; L.ldk = 1; L.kin = n0; L.sj = n0 * n1; L.ktotal = n0 * (long long)steps * n2;
  } else {
    L.ldn = n0 * n1; L.ldk = 1; L.kin = n0 * n1; L.sj = nodes; L.ktotal = n0 * n1 * (long long)steps;
  }
  const int nslab = g_slabs(L.side, L.ktotal);
  L.kchunk = ((L.ktotal + nslab - 1) / nslab + GK - 1) / GK * GK;
  const int tiles = (L.side + GB - 1) / GB;
  dim3 grid(tiles, tiles, nslab);
  if (mu == 0)
    adj_G_gemm<real, true><<<grid, 256, 0, s>>>(L, lF, C, part);
  else
    adj_G_gemm<real, false><<<grid, 256, 0, s>>>(L, lF, C, part);
  const long long count = (long long)L.side * L.side;
  adj_G_reduce<<<static_cast<int>(std::min<long long>((count + 255) / 256, 1216)), 256, 0, s>>>(count, nslab, part, G);
  return cudaGetLastError();
}

// sum (C - obs)^2 into *out (FP64; partial sums per block then one block)
template <typename real>
__global__ void __launch_bounds__(kThreads)
adj_loss_partials(long long nodes, const real* __restrict__ C, const real* __restrict__ obs, double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < nodes; i += (long long)gridDim.x * kThreads) {
    const double r = static_cast<double>(C[i]) - static_cast<double>(obs[i]);
    acc += r * r;
  }
  double v[1] = {acc};
  // reuse the fixed-order block reduction on a zeroed slot
  if (threadIdx.x == 0) part[blockIdx.x] = 0.0;
  __syncthreads();
  block_accumulate<1>(v, part);
}

__global__ void adj_sum_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += part[i];
    *out = acc;
  }
}

template <typename real>
AdjConst<real> make_adj(const lbm_s* h, const double dOm[3][kMaxQ][kMaxQ]) {
  AdjConst<real> c{};
  for (int i = 0; i < 3; ++i) c.n[i] = h->sp.n[i];
  c.nodes = h->sp.nodes;
  for (int i = 0; i < kMaxQ; ++i)
    for (int j = 0; j < kMaxQ; ++j) {
      c.omT[i][j] = static_cast<real>(h->sp.omega[j][i]);
      for (int mu = 0; mu < 3; ++mu) c.dOm[mu][i][j] = static_cast<real>(dOm[mu][i][j]);
    }
  c.w0 = static_cast<real>(h->sp.w0);
  c.wi = static_cast<real>(h->sp.wi);
  for (int mu = 0; mu < 3; ++mu) c.advw[mu] = static_cast<real>(h->sp.adv[mu] * h->sp.wi);
  const double e2 = (h->d == 2) ? 1.0 / 3.0 : 1.0 / 4.0;
  c.cu = static_cast<real>((h->prm.dt / h->prm.dx) * h->sp.wi / e2);
  return c;
}

// the gradient's device buffers, from the handle's allocator, released on scope exit
// (after the handle's stream has drained)
struct Buffers {
  const lbm_s* h;
  std::vector<void*> ptrs;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (dev_alloc(h, &p, bytes) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
  ~Buffers() {
    if (!ptrs.empty() && h->stream) cudaStreamSynchronize(h->stream);
    for (void* p : ptrs) dev_free(h, p);
  }
};

template <typename real, int D>
int run_adjoint(lbm_s* h, const AdjHooks& hooks, int nsnap, const int* snaps, const double* obs_host, int ckpt,
                const double dOm[3][kMaxQ][kMaxQ], double* loss, double* G_host, double* gpart_host) {
  constexpr int Q = 2 * D + 1;
  cudaStream_t s = h->stream;
  const long long nodes = h->sp.nodes;
  const size_t E = sizeof(real);
  const int T = snaps[nsnap - 1];
  const int nck = T / ckpt + 1;
  const int seglen = ckpt < T ? ckpt : (T > 0 ? T : 1);
  const int nb = static_cast<int>((nodes + kThreads - 1) / kThreads);
  const int cb = std::min<long long>((nodes + kThreads - 1) / kThreads, 8LL * device_sms());
  Buffers B{h, {}};
  real* obs = static_cast<real*>(B.get(E * nodes * nsnap));
  real* ck = static_cast<real*>(B.get(E * Q * nodes * nck));
  real* sf = static_cast<real*>(B.get(E * Q * nodes * seglen));
  real* sF = static_cast<real*>(B.get(E * D * nodes * seglen));
  real* sC = static_cast<real*>(B.get(E * nodes * seglen));
  real* lam = static_cast<real*>(B.get(E * Q * nodes));
  real* lf = static_cast<real*>(B.get(E * Q * nodes));
  real* lcl = static_cast<real*>(B.get(E * nodes));
  // lambda_F of every step of a segment, [mu][step][node], for one G product per segment
  real* slF = static_cast<real*>(B.get(E * D * nodes * seglen));
  real* lcf = static_cast<real*>(B.get(E * D * nodes));
  size_t gsz = 0;
  for (int mu = 0; mu < D; ++mu) gsz += (size_t)h->sp.n[mu] * h->sp.n[mu];
  double* G = static_cast<double*>(B.get(sizeof(double) * gsz));
  int gmax = 0;
  for (int mu = 0; mu < D; ++mu) gmax = std::max(gmax, h->sp.n[mu]);
  double* Gpart = static_cast<double*>(B.get(sizeof(double) * kMaxSlabs * gmax * gmax));
  double* gpart = static_cast<double*>(B.get(sizeof(double) * nb * 2 * D));
  double* lpart = static_cast<double*>(B.get(sizeof(double) * nb));
  double* lossd = static_cast<double*>(B.get(sizeof(double) * nsnap));
  if (!obs || !ck || !sf || !sF || !sC || !lam || !lf || !lcl || !slF || !lcf || !G || !Gpart || !gpart || !lpart ||
      !lossd)
    return LBM_ENOMEM;
#define CK(x)                                    \
  do {                                           \
    if ((x) != cudaSuccess) return LBM_ECUDA;    \
  } while (0)
  // observations in the working precision
  for (int k = 0; k < nsnap; ++k) {
    CK(cudaMemcpyAsync(h->dev.stage, obs_host + (size_t)k * nodes, sizeof(double) * nodes, cudaMemcpyHostToDevice, s));
    CK(launch_convert_in(h->dev.stage, obs + (size_t)k * nodes, (int)E, nodes, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaMemsetAsync(G, 0, sizeof(double) * gsz, s));
  CK(cudaMemsetAsync(gpart, 0, sizeof(double) * nb * 2 * D, s));
  CK(cudaMemsetAsync(lossd, 0, sizeof(double) * nsnap, s));
  const AdjConst<real> c = make_adj<real>(h, dOm);
  auto snap_index = [&](int t) {
    for (int k = 0; k < nsnap; ++k)
      if (snaps[k] == t) return k;
    return -1;
  };
  auto loss_at = [&](int k, const real* C) -> cudaError_t {
    adj_loss_partials<real><<<nb, kThreads, 0, s>>>(nodes, C, obs + (size_t)k * nodes, lpart);
    adj_sum_kernel<<<1, 32, 0, s>>>(lpart, nb, lossd + k);
    return cudaGetLastError();
  };

  // ---- forward pass from the initial state, checkpoints every ckpt steps, losses
  int rc = hooks.reset(h);
  if (rc) return rc;
  int cur = h->cur;
  for (int t = 0; t < T; ++t) {
    if (t % ckpt == 0)
      CK(cudaMemcpyAsync(ck + (size_t)(t / ckpt) * Q * nodes, h->dev.f[cur], E * Q * nodes, cudaMemcpyDeviceToDevice, s));
    const int k0 = snap_index(t);
    if (k0 >= 0) CK(loss_at(k0, static_cast<const real*>(h->dev.C)));
    if ((rc = hooks.step(h, cur, s))) return rc;
  }
  {
    const int k = snap_index(T);
    CK(loss_at(k, static_cast<const real*>(h->dev.C)));
    // lambda(T) = 2 (C(T) - obs)
    adj_residual_kernel<real, Q><<<cb, kThreads, 0, s>>>(nodes, static_cast<const real*>(h->dev.C),
                                                          obs + (size_t)k * nodes, lam);
    CK(cudaGetLastError());
  }

  // ---- backward, segment by segment
  const int nseg = (T + ckpt - 1) / ckpt;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int t0 = seg * ckpt, t1 = std::min(t0 + ckpt, T);
    int c2 = 0;
    CK(cudaMemcpyAsync(h->dev.f[0], ck + (size_t)seg * Q * nodes, E * Q * nodes, cudaMemcpyDeviceToDevice, s));
    CK(launch_moment(h, h->dev.f[0], h->dev.C, s));
    for (int t = t0; t < t1; ++t) {
      const int i = t - t0;
      CK(cudaMemcpyAsync(sf + (size_t)i * Q * nodes, h->dev.f[c2], E * Q * nodes, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(sC + (size_t)i * nodes, h->dev.C, E * nodes, cudaMemcpyDeviceToDevice, s));
      CK(launch_frac_simt(h, h->dev.C, h->dev.F, s));
      if (h->sp.ksum > 1)  // the FP32 operator's partial sums, added as the collide-stream kernel adds them
        CK(launch_sum_partials(reinterpret_cast<const float*>(h->dev.F), h->sp.ksum, h->sp.pstride,
                               reinterpret_cast<float*>(sF + (size_t)i * D * nodes), (long long)D * nodes, s));
      else
        CK(cudaMemcpyAsync(sF + (size_t)i * D * nodes, h->dev.F, E * D * nodes, cudaMemcpyDeviceToDevice, s));
      CK(launch_collide_stream(h, h->dev.f[c2], h->dev.f[c2 ^ 1], h->dev.C, s));
      c2 ^= 1;
    }
    const long long lFs = (long long)seglen * nodes;
    for (int t = t1 - 1; t >= t0; --t) {
      const int i = t - t0;
      const real* Ct = sC + (size_t)i * nodes;
      real* lFi = slF + (size_t)i * nodes;
      adj_step_kernel<real, D><<<nb, kThreads, 0, s>>>(c, sf + (size_t)i * Q * nodes, sF + (size_t)i * D * nodes, lam,
                                                       lf, lcl, lFi, lFs, gpart);
      CK(cudaGetLastError());
      CK(launch_frac_simt_T(h, lFi, lFs, lcf, s));
      const int k = snap_index(t);
      adj_combine_kernel<real, D><<<cb, kThreads, 0, s>>>(nodes, lf, lcl, lcf, Ct,
                                                          k >= 0 ? obs + (size_t)k * nodes : nullptr, lam);
      CK(cudaGetLastError());
    }
    size_t goff = 0;
    for (int mu = 0; mu < D; ++mu) {
      CK(accumulate_G<real>(h, mu, t1 - t0, slF + (size_t)mu * lFs, sC, G + goff, Gpart, s));
      goff += (size_t)h->sp.n[mu] * h->sp.n[mu];
    }
  }
  // ---- the initial condition f(0) = feq(C0, K C0)
  adj_init_kernel<real, D><<<nb, kThreads, 0, s>>>(c, static_cast<const real*>(h->dev.C0), lam, slF, gpart);
  CK(cudaGetLastError());
  {
    size_t goff = 0;
    for (int mu = 0; mu < D; ++mu) {
      CK(accumulate_G<real>(h, mu, 1, slF + (size_t)mu * nodes, static_cast<const real*>(h->dev.C0), G + goff, Gpart,
                            s));
      goff += (size_t)h->sp.n[mu] * h->sp.n[mu];
    }
  }
  std::vector<double> lossv(nsnap);
  CK(cudaMemcpyAsync(lossv.data(), lossd, sizeof(double) * nsnap, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(G_host, G, sizeof(double) * gsz, cudaMemcpyDeviceToHost, s));
  std::vector<double> gp((size_t)nb * 2 * D);
  CK(cudaMemcpyAsync(gp.data(), gpart, sizeof(double) * gp.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
#undef CK
  double L = 0.0;
  for (double v : lossv) L += v;
  *loss = L;
  for (int k = 0; k < 2 * D; ++k) {
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += gp[(size_t)b * 2 * D + k];
    gpart_host[k] = acc;
  }
  return LBM_OK;
}

}  // namespace

int adjoint_grad(lbm_s* h, const AdjHooks& hooks, int nsnap, const int* snaps, const double* obs, int ckpt,
                 const double dOm[3][kMaxQ][kMaxQ], double* loss, double* G, double* gsum) {
  if (h->elem == 8) {
    return (h->d == 2) ? run_adjoint<double, 2>(h, hooks, nsnap, snaps, obs, ckpt, dOm, loss, G, gsum)
                       : run_adjoint<double, 3>(h, hooks, nsnap, snaps, obs, ckpt, dOm, loss, G, gsum);
  }
  return (h->d == 2) ? run_adjoint<float, 2>(h, hooks, nsnap, snaps, obs, ckpt, dOm, loss, G, gsum)
                     : run_adjoint<float, 3>(h, hooks, nsnap, snaps, obs, ckpt, dOm, loss, G, gsum);
}

}  // namespace lbm
