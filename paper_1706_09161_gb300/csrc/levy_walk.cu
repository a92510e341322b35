// Killed stable-Levy random walk on the GPU: the Monte-Carlo counterpart of the lattice
// Boltzmann scheme (Section 3.1 of the paper).
//
//   Eq. (RW_STABLE)  dX = u dt + D' dL, D'_mumu = (D_mumu g_mu)^(1/alpha_mu), independent axes
//   Eq. (distri)     each component of dL over dt ~ (-cos(pi alpha_mu / 2) dt)^(1/alpha_mu)
//                    S(alpha_mu, beta_mu), beta_mu = 2 p_mu - 1
//   Appendix A       S(alpha, beta) has the characteristic function
//                    exp(-|k|^alpha (1 - i beta sign(k) tan(pi alpha / 2)))
//   bounded domain   a path is killed at its first exit from the box (checked after every
//                    increment); the surviving positions sample the FADE with C = 0 on the walls
//
// One thread per path, the whole run in registers.  S(alpha, beta) comes from two uniforms by
// the formula of Chambers, Mallows & Stuck (1976) as given by Weron (1996).  The uniforms come
// from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC 2011), a counter-based generator: the
// draws of path i at step n depend only on (i, n, seed), so any run can be replayed and split
// across launches.  Counter (i mod 2^32, i div 2^32, n, call), key (seed mod 2^32, seed div
// 2^32); call 0 serves axes 0 and 1, call 1 axis 2; axis a takes output words 2(a mod 2) and
// 2(a mod 2) + 1.  FP64 form: uniforms (o + 1/2) 2^-32 and FP64 arithmetic; FP32 form: uniforms
// ((o >> 9) + 1/2) 2^-23 (exact in FP32, as are u - 1/2 and 1 - u; never 0 or 1) and FP32
// arithmetic.
#include <cmath>

#include "lbm_internal.h"

namespace lbm {
namespace {

struct WalkAxis {
  double cu;     // u dt
  double scale;  // (D g)^(1/alpha) (-cos(pi alpha / 2) dt)^(1/alpha)
  double alpha, one_m_alpha, inv_alpha, expo;  // alpha, 1 - alpha, 1/alpha, (1 - alpha) / alpha
  double Bpi, A;  // alpha B / pi = atan(beta tan(pi alpha / 2)) / pi and Weron's A
  double lo, hi;
};

struct WalkPrm {
  WalkAxis ax[3];
  unsigned int k0, k1;  // Philox key (the seed)
  long long n;
  unsigned int step0;
  int nsteps;
};

constexpr unsigned int kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr unsigned int kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// Philox4x32-10: ten rounds; the key is bumped between rounds
__device__ __forceinline__ void philox4x32_10(unsigned int c[4], unsigned int k0, unsigned int k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned int lo0 = kPhiloxM0 * c[0], hi0 = __umulhi(kPhiloxM0, c[0]);
    const unsigned int lo1 = kPhiloxM1 * c[2], hi1 = __umulhi(kPhiloxM1, c[2]);
    const unsigned int n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
}

template <typename real>
__device__ __forceinline__ real uniform_open(unsigned int o);
template <>
__device__ __forceinline__ double uniform_open<double>(unsigned int o) {
  return (static_cast<double>(o) + 0.5) * 0x1p-32;
}
template <>
__device__ __forceinline__ float uniform_open<float>(unsigned int o) {
  return (static_cast<float>(o >> 9) + 0.5f) * 0x1p-23f;
}

__device__ __forceinline__ double sin_pi(double x) { return sinpi(x); }
__device__ __forceinline__ float sin_pi(float x) { return sinpif(x); }
__device__ __forceinline__ double cos_pi(double x) { return cospi(x); }
__device__ __forceinline__ float cos_pi(float x) { return cospif(x); }

// S(alpha, beta) from uniforms u1, u2 (Weron 1996, alpha != 1).  With V = pi v, v = u1 - 1/2
// (exact for the generator's uniforms), the angles are taken in units of pi: sin(alpha (V + B))
// = sin(pi (alpha v + alpha B / pi)), cos(V - alpha (V + B)) = cos(pi ((1 - alpha) v -
// alpha B / pi)) and cos V = cos(pi v), which keeps cos V accurate as V -> +-pi/2.
template <typename real>
__device__ __forceinline__ real stable_sample(const WalkAxis& a, real u1, real u2) {
  const real v = u1 - static_cast<real>(0.5);
  const real W = -log(u2);
  const real Bp = static_cast<real>(a.Bpi);
  const real c = cos_pi(static_cast<real>(a.one_m_alpha) * v - Bp) / W;
  return static_cast<real>(a.A) * sin_pi(static_cast<real>(a.alpha) * v + Bp) /
         pow(cos_pi(v), static_cast<real>(a.inv_alpha)) *
         pow(c > static_cast<real>(0) ? c : static_cast<real>(0), static_cast<real>(a.expo));
}

// Advance every live path by nsteps increments (steps step0 .. step0 + nsteps - 1); X is
// [mu][n], alive 1 for a live path; a path that leaves the box keeps its exit position.
template <typename real, int D>
__global__ void __launch_bounds__(256) walk_kernel(const WalkPrm P, double* __restrict__ X,
                                                   unsigned char* __restrict__ alive) {
  const long long n = P.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!alive[i]) continue;
    real x[D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) x[mu] = static_cast<real>(X[mu * n + i]);
    bool ok = true;
    for (int j = 0; j < P.nsteps && ok; ++j) {
      const unsigned int step = P.step0 + static_cast<unsigned int>(j);
      unsigned int c[4] = {static_cast<unsigned int>(i), static_cast<unsigned int>(i >> 32), step, 0u};
      philox4x32_10(c, P.k0, P.k1);
      unsigned int c2[4] = {static_cast<unsigned int>(i), static_cast<unsigned int>(i >> 32), step, 1u};
      if (D == 3) philox4x32_10(c2, P.k0, P.k1);
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        const unsigned int o1 = mu < 2 ? c[2 * mu] : c2[0];
        const unsigned int o2 = mu < 2 ? c[2 * mu + 1] : c2[1];
        const WalkAxis& a = P.ax[mu];
        const real s = stable_sample<real>(a, uniform_open<real>(o1), uniform_open<real>(o2));
        x[mu] += static_cast<real>(a.cu) + static_cast<real>(a.scale) * s;
      }
#pragma unroll
      for (int mu = 0; mu < D; ++mu)
        ok = ok && x[mu] > static_cast<real>(P.ax[mu].lo) && x[mu] < static_cast<real>(P.ax[mu].hi);
    }
#pragma unroll
    for (int mu = 0; mu < D; ++mu) X[mu * n + i] = static_cast<double>(x[mu]);
    alive[i] = ok ? 1 : 0;
  }
}

// counts[node] += live paths in the cell of width dx centred at the node (nodes at lo + k dx)
__global__ void density_kernel(const double* __restrict__ X, const unsigned char* __restrict__ alive, long long n,
                               int d, int g0, int g1, int g2, double lo0, double lo1, double lo2, double dx,
                               unsigned int* __restrict__ counts) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (!alive[i]) continue;
    const int g[3] = {g0, g1, g2};
    const double lo[3] = {lo0, lo1, lo2};
    long long idx = 0, stride = 1;
    bool in = true;
    for (int mu = 0; mu < d; ++mu) {
      const long long k = static_cast<long long>(floor((X[mu * n + i] - lo[mu]) / dx + 0.5));
      in = in && k >= 0 && k < g[mu];
      idx += k * stride;
      stride *= g[mu];
    }
    if (in) atomicAdd(&counts[idx], 1u);
  }
}

int walk_setup(const lbm_walk_params* prm, WalkPrm* P) {
  if (!prm || (prm->d != 2 && prm->d != 3)) return LBM_EINVAL;
  if (prm->precision != LBM_FP64 && prm->precision != LBM_FP32) return LBM_EINVAL;
  if (!(prm->dt > 0.0) || !std::isfinite(prm->dt)) return LBM_EINVAL;
  const double pi = 3.14159265358979323846;
  for (int mu = 0; mu < prm->d; ++mu) {
    const double a = prm->alpha[mu], p = prm->p[mu], D = prm->D[mu], g = prm->g[mu];
    if (!(a > 1.0 && a <= 2.0) || !(p >= 0.0 && p <= 1.0) || !(D > 0.0) || !(g > 0.0)) return LBM_EINVAL;
    if (!std::isfinite(D) || !std::isfinite(g) || !std::isfinite(prm->u[mu])) return LBM_EINVAL;
    if (!(prm->lo[mu] < prm->hi[mu])) return LBM_EINVAL;
    const double beta = 2.0 * p - 1.0;
    const double t = beta * std::tan(pi * a / 2.0);
    WalkAxis& w = P->ax[mu];
    w.cu = prm->u[mu] * prm->dt;
    w.scale = std::pow(D * g, 1.0 / a) * std::pow(-std::cos(pi * a / 2.0) * prm->dt, 1.0 / a);
    w.alpha = a;
    w.one_m_alpha = 1.0 - a;
    w.inv_alpha = 1.0 / a;
    w.Bpi = std::atan(t) / pi;
    w.A = std::pow(1.0 + t * t, 1.0 / (2.0 * a));
    w.expo = (1.0 - a) / a;
    w.lo = prm->lo[mu];
    w.hi = prm->hi[mu];
  }
  P->k0 = static_cast<unsigned int>(prm->seed & 0xffffffffull);
  P->k1 = static_cast<unsigned int>(prm->seed >> 32);
  return LBM_OK;
}

int grid_blocks(long long n) {
  const long long b = (n + 255) / 256;
  const long long cap = 16LL * device_sms();
  return static_cast<int>(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_walk(const lbm_walk_params* prm, long long n, double* X, unsigned char* alive, long long step0,
                        int nsteps, void* stream) {
  lbm::WalkPrm P{};
  int rc = lbm::walk_setup(prm, &P);
  if (rc) return rc;
  if (n < 0 || nsteps < 0 || step0 < 0 || step0 + nsteps > 0xffffffffLL) return LBM_EINVAL;
  if (n > 0 && (!X || !alive)) return LBM_EINVAL;
  if (n == 0 || nsteps == 0) return LBM_OK;
  P.n = n;
  P.step0 = static_cast<unsigned int>(step0);
  P.nsteps = nsteps;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int g = lbm::grid_blocks(n);
  if (prm->precision == LBM_FP64) {
    if (prm->d == 2) lbm::walk_kernel<double, 2><<<g, 256, 0, s>>>(P, X, alive);
    else lbm::walk_kernel<double, 3><<<g, 256, 0, s>>>(P, X, alive);
  } else {
    if (prm->d == 2) lbm::walk_kernel<float, 2><<<g, 256, 0, s>>>(P, X, alive);
    else lbm::walk_kernel<float, 3><<<g, 256, 0, s>>>(P, X, alive);
  }
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_walk_density(const lbm_walk_params* prm, long long n, const double* X, const unsigned char* alive,
                                const int* grid, double dx, unsigned int* counts, void* stream) {
  if (!prm || (prm->d != 2 && prm->d != 3) || !grid || !counts || n < 0 || !(dx > 0.0)) return LBM_EINVAL;
  if (n > 0 && (!X || !alive)) return LBM_EINVAL;
  int g[3] = {1, 1, 1};
  for (int mu = 0; mu < prm->d; ++mu) {
    if (grid[mu] < 1) return LBM_EINVAL;
    g[mu] = grid[mu];
  }
  if (n == 0) return LBM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lbm::density_kernel<<<lbm::grid_blocks(n), 256, 0, s>>>(X, alive, n, prm->d, g[0], g[1], g[2], prm->lo[0],
                                                          prm->lo[1], prm->d == 3 ? prm->lo[2] : 0.0, dx, counts);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
