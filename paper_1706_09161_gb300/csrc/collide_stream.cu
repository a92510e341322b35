// Fused equilibrium + collision + streaming + Dirichlet walls + new concentration.
//
// One launch performs items 2-5 of Algorithm 1's time loop for every node:
//   item 2  equilibrium   feq = A + (C/e^2)(dt/dx) u_mu |e_mu w>            Eqs. (Feq), (CoeffA_FADE3D)
//           collision     f* = f - Omega (f - feq)                          Eqs. (LBE_Ket), (MRT-Coll)
//   item 3  streaming     f_i(x + e_i, t+dt) = f*_i(x, t)                   Eq. (Def_Translation)
//   item 4  walls         f_b = C_wall - sum_{i != b} f_i                   Eq. (Dirichlet_BC)
//   item 5  moment        C = <1|f>
// Populations are stored after streaming and boundary treatment, so a CTA
// collides its tile plus a one-node halo into shared memory, then gathers
// ("pulls") each population from the node it came from.  The halo nodes are
// collided redundantly by the neighbouring CTAs; their loads hit L2.
#include <cuda_bf16.h>

#include "lbm_internal.h"

namespace lbm {
namespace {

template <int D> struct Tile;
template <> struct Tile<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Tile<3> { static constexpr int X = 32, Y = 4, Z = 2; };

template <int D> struct Lat;
template <> struct Lat<2> { static constexpr int Q = 5; };
template <> struct Lat<3> { static constexpr int Q = 7; };

// Per-step constants in the working precision (no FP64 arithmetic per node on the
// FP32 forms; GB300's FP64 rate is a small fraction of its FP32 rate).
template <typename real>
struct KConst {
  int n[3];
  long long nodes;
  real omega[kMaxQ][kMaxQ];
  real w0, wi;
  real advw[3];  // (dt/dx) u_mu w_i / e^2
  real C_wall;
};

template <typename real>
KConst<real> make_const(const StepParams& sp) {
  KConst<real> k{};
  for (int i = 0; i < 3; ++i) k.n[i] = sp.n[i];
  k.nodes = sp.nodes;
  for (int i = 0; i < kMaxQ; ++i)
    for (int j = 0; j < kMaxQ; ++j) k.omega[i][j] = static_cast<real>(sp.omega[i][j]);
  k.w0 = static_cast<real>(sp.w0);
  k.wi = static_cast<real>(sp.wi);
  for (int i = 0; i < 3; ++i) k.advw[i] = static_cast<real>(sp.adv[i] * sp.wi);
  k.C_wall = static_cast<real>(sp.C_wall);
  return k;
}

// Equilibrium and collision of one node.  f: populations (in), fs: post-collision (out).
template <typename real, int D, bool MRT>
__device__ __forceinline__ void collide_node(const KConst<real>& sp, const real* f, const real* F, real* fs) {
  constexpr int Q = Lat<D>::Q;
  real C = f[0];
#pragma unroll
  for (int q = 1; q < Q; ++q) C += f[q];
  real sumF = F[0];
#pragma unroll
  for (int mu = 1; mu < D; ++mu) sumF += F[mu];
  real feq[Q];
  feq[0] = C - sp.w0 * sumF;
#pragma unroll
  for (int mu = 0; mu < D; ++mu) {
    const real a = sp.wi * F[mu];
    const real b = sp.advw[mu] * C;
    feq[2 * mu + 1] = a + b;
    feq[2 * mu + 2] = a - b;
  }
  if (!MRT) {
    const real om = sp.omega[0][0];
#pragma unroll
    for (int q = 0; q < Q; ++q) fs[q] = f[q] - om * (f[q] - feq[q]);
  } else {
    real dl[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) dl[q] = f[q] - feq[q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      real acc = sp.omega[i][0] * dl[0];
#pragma unroll
      for (int j = 1; j < Q; ++j) acc += sp.omega[i][j] * dl[j];
      fs[i] = f[i] - acc;
    }
  }
}

// velocity components of population q (Section 2.1 order)
__device__ __forceinline__ int ex_of(int q) { return q == 1 ? 1 : (q == 2 ? -1 : 0); }
__device__ __forceinline__ int ey_of(int q) { return q == 3 ? 1 : (q == 4 ? -1 : 0); }
__device__ __forceinline__ int ez_of(int q) { return q == 5 ? 1 : (q == 6 ? -1 : 0); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Operands of the split-precision fractional operator: C = hi + lo (+ residual), with
// hi, lo in bf16 (SPLIT = 1) or tf32 (SPLIT = 2), x-pitch ldp.
struct SplitOut {
  void* hi;
  void* lo;
  int ldp;
};

template <int SPLIT, typename real>
__device__ __forceinline__ void write_split(const SplitOut& so, long long o, real C) {
  const float c = static_cast<float>(C);
  if (SPLIT == 1) {
    const __nv_bfloat16 h = __float2bfloat16_rn(c);
    static_cast<__nv_bfloat16*>(so.hi)[o] = h;
    static_cast<__nv_bfloat16*>(so.lo)[o] = __float2bfloat16_rn(c - __bfloat162float(h));
  } else if (SPLIT == 2) {
    const float h = tf32_rna(c);
    static_cast<float*>(so.hi)[o] = h;
    static_cast<float*>(so.lo)[o] = tf32_rna(c - h);
  }
}

template <typename real, int D, bool MRT, int SPLIT>
__global__ void __launch_bounds__(256)
collide_stream_kernel(const KConst<real> sp, const real* __restrict__ f_in, const real* __restrict__ F,
                      real* __restrict__ f_out, real* __restrict__ C_out, int* __restrict__ flag, SplitOut so) {
  constexpr int Q = Lat<D>::Q;
  constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
  constexpr int EX = TX + 2, EY = TY + 2, EZ = (D == 3) ? TZ + 2 : 1;
  constexpr int EXT = EX * EY * EZ;
  __shared__ real s_f[Q][EXT];

  const int n0 = sp.n[0], n1 = sp.n[1], n2 = sp.n[2];
  const long long nodes = sp.nodes;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;

  // phase 1: collide tile + face halo into shared memory
  for (int e = threadIdx.x; e < EXT; e += blockDim.x) {
    const int ex = e % EX;
    const int ey = (e / EX) % EY;
    const int ez = (D == 3) ? e / (EX * EY) : 1;
    const int outx = (ex == 0 || ex == EX - 1), outy = (ey == 0 || ey == EY - 1);
    const int outz = (D == 3) ? (ez == 0 || ez == EZ - 1) : 0;
    if (outx + outy + outz > 1) continue;  // edge/corner of the halo: never read
    const int gx = x0 + ex - 1, gy = y0 + ey - 1, gz = (D == 3) ? z0 + ez - 1 : 0;
    if (gx < 0 || gx >= n0 || gy < 0 || gy >= n1 || gz < 0 || gz >= n2) continue;
    const long long node = gx + (long long)n0 * (gy + (long long)n1 * gz);
    real f[Q], Fv[D], fs[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) f[q] = f_in[q * nodes + node];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) Fv[mu] = F[mu * nodes + node];
    collide_node<real, D, MRT>(sp, f, Fv, fs);
#pragma unroll
    for (int q = 0; q < Q; ++q) s_f[q][e] = fs[q];
  }
  __syncthreads();

  // phase 2: pull-stream into the tile, impose the walls, new concentration
  for (int t = threadIdx.x; t < TX * TY * TZ; t += blockDim.x) {
    const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
    const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
    if (gx >= n0 || gy >= n1 || gz >= n2) continue;
    const long long node = gx + (long long)n0 * (gy + (long long)n1 * gz);
    real fv[Q];
    bool known[Q];
    real sum_known = static_cast<real>(0);
    int n_unknown = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int sx = gx - ex_of(q), sy = gy - ey_of(q), sz = gz - ez_of(q);
      known[q] = (sx >= 0 && sx < n0 && sy >= 0 && sy < n1 && sz >= 0 && sz < n2);
      if (known[q]) {
        const int e = (sx - x0 + 1) + EX * ((sy - y0 + 1) + EY * ((D == 3) ? (sz - z0 + 1) : 0));
        fv[q] = s_f[q][e];
        sum_known += fv[q];
      } else {
        fv[q] = static_cast<real>(0);
        ++n_unknown;
      }
    }
    real C = sum_known;
    if (n_unknown > 0) {
      // Eq. (Dirichlet_BC); with k unknown populations each takes 1/k of the deficit
      const real fill = (sp.C_wall - sum_known) / static_cast<real>(n_unknown);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (!known[q]) fv[q] = fill;
      C = fv[0];
#pragma unroll
      for (int q = 1; q < Q; ++q) C += fv[q];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) f_out[q * nodes + node] = fv[q];
    C_out[node] = C;
    if (SPLIT) write_split<SPLIT>(so, ((long long)gz * n1 + gy) * so.ldp + gx, C);
    if (!isfinite(C)) atomicOr(flag, 1);
  }
}

template <typename real, int D>
__global__ void init_equilibrium_kernel(const KConst<real> sp, const real* __restrict__ C, const real* __restrict__ F,
                                        real* __restrict__ f) {
  constexpr int Q = Lat<D>::Q;
  const long long nodes = sp.nodes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
       i += (long long)gridDim.x * blockDim.x) {
    const real c = C[i];
    real sumF = static_cast<real>(0);
    real Fv[D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      Fv[mu] = F[mu * nodes + i];
      sumF += Fv[mu];
    }
    f[i] = c - sp.w0 * sumF;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const real a = sp.wi * Fv[mu];
      const real b = sp.advw[mu] * c;
      f[(2 * mu + 1) * nodes + i] = a + b;
      f[(2 * mu + 2) * nodes + i] = a - b;
    }
  }
}

template <typename real, int Q>
__global__ void moment_kernel(long long nodes, const real* __restrict__ f, real* __restrict__ C) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
       i += (long long)gridDim.x * blockDim.x) {
    real c = f[i];
#pragma unroll
    for (int q = 1; q < Q; ++q) c += f[q * nodes + i];
    C[i] = c;
  }
}

template <typename real, int D, bool MRT>
cudaError_t launch_cs(const lbm_s* h, const void* f_in, void* f_out, void* C_out, cudaStream_t s) {
  constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
  const KConst<real> sp = make_const<real>(h->sp);
  dim3 grid((sp.n[0] + TX - 1) / TX, (sp.n[1] + TY - 1) / TY, (sp.n[2] + TZ - 1) / TZ);
  SplitOut so{h->dev.Chi, h->dev.Clo, tc_split_pitch(h)};
  const int split = (h->tc == nullptr) ? 0 : (h->prm.precision == LBM_FP32_BF16SPLIT ? 1 : 2);
  const real* fi = static_cast<const real*>(f_in);
  const real* F = static_cast<const real*>(h->dev.F);
  real* fo = static_cast<real*>(f_out);
  real* Co = static_cast<real*>(C_out);
  if (split == 0)
    collide_stream_kernel<real, D, MRT, 0><<<grid, 256, 0, s>>>(sp, fi, F, fo, Co, h->dev.flag, so);
  else if (split == 1)
    collide_stream_kernel<real, D, MRT, 1><<<grid, 256, 0, s>>>(sp, fi, F, fo, Co, h->dev.flag, so);
  else
    collide_stream_kernel<real, D, MRT, 2><<<grid, 256, 0, s>>>(sp, fi, F, fo, Co, h->dev.flag, so);
  return cudaGetLastError();
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_collide_stream(const lbm_s* h, const void* f_in, void* f_out, void* C_out, cudaStream_t s) {
  const bool mrt = h->prm.collision == LBM_MRT;
  if (h->elem == 8) {
    if (h->d == 2) return mrt ? launch_cs<double, 2, true>(h, f_in, f_out, C_out, s)
                              : launch_cs<double, 2, false>(h, f_in, f_out, C_out, s);
    return mrt ? launch_cs<double, 3, true>(h, f_in, f_out, C_out, s)
               : launch_cs<double, 3, false>(h, f_in, f_out, C_out, s);
  }
  if (h->d == 2) return mrt ? launch_cs<float, 2, true>(h, f_in, f_out, C_out, s)
                            : launch_cs<float, 2, false>(h, f_in, f_out, C_out, s);
  return mrt ? launch_cs<float, 3, true>(h, f_in, f_out, C_out, s)
             : launch_cs<float, 3, false>(h, f_in, f_out, C_out, s);
}

cudaError_t launch_init_equilibrium(const lbm_s* h, void* f, cudaStream_t s) {
  const int g = grid_for(h->sp.nodes);
  if (h->elem == 8) {
    if (h->d == 2)
      init_equilibrium_kernel<double, 2><<<g, 256, 0, s>>>(make_const<double>(h->sp), (const double*)h->dev.C, (const double*)h->dev.F, (double*)f);
    else
      init_equilibrium_kernel<double, 3><<<g, 256, 0, s>>>(make_const<double>(h->sp), (const double*)h->dev.C, (const double*)h->dev.F, (double*)f);
  } else {
    if (h->d == 2)
      init_equilibrium_kernel<float, 2><<<g, 256, 0, s>>>(make_const<float>(h->sp), (const float*)h->dev.C, (const float*)h->dev.F, (float*)f);
    else
      init_equilibrium_kernel<float, 3><<<g, 256, 0, s>>>(make_const<float>(h->sp), (const float*)h->dev.C, (const float*)h->dev.F, (float*)f);
  }
  return cudaGetLastError();
}

cudaError_t launch_moment(const lbm_s* h, const void* f, void* C, cudaStream_t s) {
  const int g = grid_for(h->sp.nodes);
  if (h->elem == 8) {
    if (h->Q == 5) moment_kernel<double, 5><<<g, 256, 0, s>>>(h->sp.nodes, (const double*)f, (double*)C);
    else moment_kernel<double, 7><<<g, 256, 0, s>>>(h->sp.nodes, (const double*)f, (double*)C);
  } else {
    if (h->Q == 5) moment_kernel<float, 5><<<g, 256, 0, s>>>(h->sp.nodes, (const float*)f, (float*)C);
    else moment_kernel<float, 7><<<g, 256, 0, s>>>(h->sp.nodes, (const float*)f, (float*)C);
  }
  return cudaGetLastError();
}

}  // namespace lbm
