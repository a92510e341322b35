// Fractional terms on CUDA cores (FP64 and plain-FP32 forms).
//
// Algorithm 1 (fractional terms) / Section 2.4, Eq. (XXminus_discret): along every
// lattice line of axis mu, F_mu[n] = sum_l K_mu[n][l] C[l].  Viewed over all
// lines this is one dense GEMM per axis:
//   axis x (fastest):  F[r][n] = sum_l C[r][l] K[n][l]     = C  * K^T   (rows r = other coords)
//   axis y, z:         F[b][n][c] = sum_l K[n][l] C[b][l][c] = K * C_b  (b = outer planes, c = inner)
// Both are written as a row-major NN GEMM D = A B (A: M x K, B: K x N), batched
// over b with strides; K^T is stored explicitly for the x axis.  One launch covers
// every axis: a table maps each block to (axis, batch, tile, contraction slice).  Small
// FP32 problems split the contraction over ks blocks per tile (enough blocks to fill
// the GPU twice); slice r writes its partial sum to F + r * pstride and the consumers
// add the ks partials in order, as for the tensor-core operator's split.
#include <algorithm>

#include "lbm_internal.h"

namespace lbm {
namespace {

struct GemmAxis {
  const void* A;
  const void* B;
  void* C;
  long long lda, sA, ldb, sB, ldc, sC;
  int M, N, K;
  int tm, tn;          // tiles along M and N
  long long begin;     // first block of this axis
};

struct GemmPlan {
  GemmAxis ax[3];
  int naxes;
  int ks;              // contraction slices per tile
  long long pstride;   // elements between the slices' partial outputs
  long long total;
  int early;           // one-wave grid: let the next kernel be scheduled at block start
};

// Block tile BM x BN, 256 threads with TM x TN outputs each, reduction slices of BK.
// A is staged as [m][k] (k contiguous, as it is read from global memory) and B as
// [k][n]; the next slice is fetched into registers while the current one is
// multiplied from the other shared-memory buffer.
template <typename real, int BM, int BN, int TM, int TN>
struct SimtCfg {
  static constexpr int BK = sizeof(real) == 8 ? 16 : 32;
  static constexpr int AL = BM * BK / 256;  // A elements per thread per slice
  static constexpr int BL = BK * BN / 256;
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
};

template <typename real, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256)
frac_simt_kernel(const GemmPlan P) {
  using G = SimtCfg<real, BM, BN, TM, TN>;
  constexpr int BK = G::BK;
  __shared__ real As[2][BM][BK + 1];
  __shared__ __align__(16) real Bs[2][BK][BN];
  // programmatic dependent launch: C (read) and F (written) belong to the previous kernel
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (P.early) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  long long b = blockIdx.x;
  int a = 0;
  while (a + 1 < P.naxes && b >= P.ax[a + 1].begin) ++a;
  const GemmAxis& X = P.ax[a];
  b -= X.begin;
  const int rank = static_cast<int>(b % P.ks);  // contraction slice
  b /= P.ks;
  const long long per = (long long)X.tm * X.tn;
  const long long bz = b / per;
  const int r = static_cast<int>(b - bz * per);
  const int m0 = (r / X.tn) * BM, n0 = (r % X.tn) * BN;
  const real* __restrict__ A = static_cast<const real*>(X.A) + bz * X.sA;
  const real* __restrict__ B = static_cast<const real*>(X.B) + bz * X.sB;
  real* __restrict__ Cm = static_cast<real*>(X.C) + bz * X.sC + rank * P.pstride;
  const int M = X.M, N = X.N;
  // slices of whole BK blocks: [kbeg, kend)
  const int nkb = (X.K + BK - 1) / BK;
  const int kbeg = (rank * nkb / P.ks) * BK;
  const int K = min(X.K, ((rank + 1) * nkb / P.ks) * BK);
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);

  real ra[G::AL], rb[G::BL];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int i = 0; i < G::AL; ++i) {
      const int e = tid + i * 256;
      const int mm = e / BK, kk = e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      ra[i] = (gm < M && gk < K) ? A[gm * X.lda + gk] : static_cast<real>(0);
    }
#pragma unroll
    for (int i = 0; i < G::BL; ++i) {
      const int e = tid + i * 256;
      const int kk = e / BN, nn = e % BN;
      const int gk = k0 + kk, gn = n0 + nn;
      rb[i] = (gk < K && gn < N) ? B[gk * X.ldb + gn] : static_cast<real>(0);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int i = 0; i < G::AL; ++i) {
      const int e = tid + i * 256;
      As[buf][e / BK][e % BK] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < G::BL; ++i) {
      const int e = tid + i * 256;
      Bs[buf][e / BN][e % BN] = rb[i];
    }
  };

  real acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = static_cast<real>(0);

  fetch(kbeg);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      real av[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) av[i] = As[buf][ty * TM + i][kk];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * bv[j];
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx * TN + j;
      if (gn < N) Cm[gm * X.ldc + gn] = acc[i][j];
    }
  }
  if (!P.early) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

void add_axis(GemmPlan& P, int BM, int BN, int M, int N, int K, int batch, const void* A, long long lda, long long sA,
              const void* B, long long ldb, long long sB, void* C, long long ldc, long long sC) {
  // (blocks of this axis = tiles x batch x P.ks)
  GemmAxis& X = P.ax[P.naxes++];
  X.A = A; X.B = B; X.C = C;
  X.lda = lda; X.sA = sA; X.ldb = ldb; X.sB = sB; X.ldc = ldc; X.sC = sC;
  X.M = M; X.N = N; X.K = K;
  X.tm = (M + BM - 1) / BM;
  X.tn = (N + BN - 1) / BN;
  X.begin = P.total;
  P.total += (long long)X.tm * X.tn * batch * P.ks;
}

// transpose = false: F_mu = K_mu applied along mu to C_mu, transpose = true: K_mu^T; the
// input of axis mu is the field at C + mu * cstride (cstride = 0: one input for every axis)
template <typename real, int BM, int BN>
GemmPlan make_plan(const lbm_s* h, const real* C, real* F, bool transpose, long long cstride, int ks = 1,
                   long long pstride = 0) {
  const int n0 = h->sp.n[0], n1 = h->sp.n[1], n2 = h->sp.n[2];
  const long long nodes = h->sp.nodes;
  const real* K = static_cast<const real*>(transpose ? h->dev.KT : h->dev.K);
  const real* KT = static_cast<const real*>(transpose ? h->dev.K : h->dev.KT);
  GemmPlan P{};
  P.ks = ks;
  P.pstride = pstride;
  long long koff = 0;
  // axis x: F_0 = C (rows x n0) * K_0^T
  add_axis(P, BM, BN, (int)(nodes / n0), n0, n0, 1, C, n0, 0, KT + koff, n0, 0, F, n0, 0);
  koff += (long long)n0 * n0;
  // axis y: for each z-plane b, F_1[b] = K_1 * C[b]  (C[b] is n1 x n0)
  add_axis(P, BM, BN, n1, n0, n1, n2, K + koff, n1, 0, C + cstride, n0, (long long)n1 * n0, F + nodes, n0,
           (long long)n1 * n0);
  koff += (long long)n1 * n1;
  // axis z: F_2 = K_2 * C  (C is n2 x (n1 n0))
  if (h->d == 3)
    add_axis(P, BM, BN, n2, n0 * n1, n2, 1, K + koff, n2, 0, C + 2 * cstride, (long long)n0 * n1, 0, F + 2 * nodes,
             (long long)n0 * n1, 0);
  return P;
}

// the grid of `blocks` blocks is resident at once (one wave)
template <typename real, int BM, int BN, int TM, int TN>
bool simt_blocks_fit(long long blocks) {
  static int per_sm = -1;
  if (per_sm < 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, frac_simt_kernel<real, BM, BN, TM, TN>, 256, 0) !=
          cudaSuccess)
    per_sm = 0;
  return blocks <= (long long)per_sm * device_sms();
}

// 64 x 64 tiles where they give two blocks per SM (with the handle's contraction split,
// forward operator only), else 32 x 32
template <typename real>
cudaError_t frac_all_axes(const lbm_s* h, const real* C, real* F, cudaStream_t s, bool transpose = false,
                          long long cstride = 0) {
  const int ks = transpose ? 1 : h->sp.ksum;
  // the forward operator of a handle with programmatic dependent launch overlaps the
  // previous collide-stream kernel's tail
  const bool pdl = !transpose && h->pdl;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  GemmPlan big = make_plan<real, 64, 64>(h, C, F, transpose, cstride, ks, ks > 1 ? h->sp.pstride : 0);
  if (big.total >= 2LL * device_sms() || ks > 1) {
    big.early = pdl && simt_blocks_fit<real, 64, 64, 4, 4>(big.total);
    cfg.gridDim = dim3(static_cast<unsigned>(big.total), 1, 1);
    return cudaLaunchKernelEx(&cfg, frac_simt_kernel<real, 64, 64, 4, 4>, big);
  }
  GemmPlan small = make_plan<real, 32, 32>(h, C, F, transpose, cstride);
  small.early = pdl && simt_blocks_fit<real, 32, 32, 2, 2>(small.total);
  cfg.gridDim = dim3(static_cast<unsigned>(small.total), 1, 1);
  return cudaLaunchKernelEx(&cfg, frac_simt_kernel<real, 32, 32, 2, 2>, small);
}

}  // namespace

bool simt_one_wave(const lbm_s* h) {
  if (h->elem != 4) return false;
  const float* C = static_cast<const float*>(h->dev.C);
  float* F = static_cast<float*>(h->dev.F);
  GemmPlan big = make_plan<float, 64, 64>(h, C, F, false, 0, h->sp.ksum, h->sp.pstride);
  if (big.total >= 2LL * device_sms() || h->sp.ksum > 1) return simt_blocks_fit<float, 64, 64, 4, 4>(big.total);
  GemmPlan small = make_plan<float, 32, 32>(h, C, F, false, 0);
  return simt_blocks_fit<float, 32, 32, 2, 2>(small.total);
}

int simt_ksplit(const lbm_s* h) {
  if (h->elem != 4) return 1;
  const long long n0 = h->sp.n[0], n1 = h->sp.n[1], n2 = h->sp.n[2];
  auto t64 = [](long long m, long long n) { return ((m + 63) / 64) * ((n + 63) / 64); };
  // 64 x 64 tiles of the forward plan: x (nodes / n0 x n0), y (n1 x n0, n2 of them), z (n2 x n0 n1)
  long long tiles = t64(h->sp.nodes / n0, n0) + t64(n1, n0) * n2;
  if (h->d == 3) tiles += t64(n2, n0 * n1);
  int kbmin = 1 << 30;
  for (int mu = 0; mu < h->d; ++mu) kbmin = std::min(kbmin, (h->sp.n[mu] + 31) / 32);  // BK = 32 (FP32)
  int ks = 1;
  const long long w = 2LL * device_sms();
  while (ks * 2 <= 8 && ks * 2 <= kbmin && tiles * ks < w) ks *= 2;
  return ks;
}

cudaError_t launch_frac_simt_T(const lbm_s* h, const void* in, long long in_stride, void* out, cudaStream_t s) {
  if (h->elem == 8)
    return frac_all_axes<double>(h, static_cast<const double*>(in), static_cast<double*>(out), s, true, in_stride);
  return frac_all_axes<float>(h, static_cast<const float*>(in), static_cast<float*>(out), s, true, in_stride);
}

cudaError_t launch_frac_simt(const lbm_s* h, const void* C, void* F, cudaStream_t s) {
  // spatially varying g: the input along mu is G_mu = g_mu(x) C (Eq. Fg), one field per axis
  const long long cs = (h->fld.on && h->fld.G) ? h->sp.nodes : 0;
  if (h->fld.on && h->fld.G) C = h->fld.G;
  if (h->elem == 8)
    return frac_all_axes<double>(h, static_cast<const double*>(C), static_cast<double*>(F), s, false, cs);
  return frac_all_axes<float>(h, static_cast<const float*>(C), static_cast<float*>(F), s, false, cs);
}

}  // namespace lbm
