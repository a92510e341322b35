// Fractional terms on CUDA cores (FP64 and plain-FP32 forms).
//
// Algorithm 1, loop item 1 / Section 2.4, Eq. (XXminus_discret): along every
// lattice line of axis mu, F_mu[n] = sum_l K_mu[n][l] C[l].  Viewed over all
// lines this is one dense GEMM per axis:
//   axis x (fastest):  F[r][n] = sum_l C[r][l] K[n][l]     = C  * K^T   (rows r = other coords)
//   axis y, z:         F[b][n][c] = sum_l K[n][l] C[b][l][c] = K * C_b  (b = outer planes, c = inner)
// Both are written as a row-major NN GEMM D = A B (A: M x K, B: K x N), batched
// over b with strides; K^T is stored explicitly for the x axis.
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

template <typename real>
__global__ void __launch_bounds__(256)
gemm_nn_kernel(int M, int N, int K, const real* __restrict__ A, long long lda, long long sA,
               const real* __restrict__ B, long long ldb, long long sB, real* __restrict__ Cm,
               long long ldc, long long sC) {
  __shared__ real As[BK][BM];
  __shared__ real Bs[BK][BN + 1];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  Cm += bz * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  real acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = static_cast<real>(0);

  for (int k0 = 0; k0 < K; k0 += BK) {
    // A tile: BM x BK, 4 elements per thread
#pragma unroll
    for (int r = 0; r < (BM * BK) / 256; ++r) {
      const int e = tid + r * 256;
      const int mm = e / BK, kk = e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[gm * lda + gk] : static_cast<real>(0);
    }
    // B tile: BK x BN
#pragma unroll
    for (int r = 0; r < (BK * BN) / 256; ++r) {
      const int e = tid + r * 256;
      const int kk = e / BN, nn = e % BN;
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? B[gk * ldb + gn] : static_cast<real>(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      real a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < N) Cm[gm * ldc + gn] = acc[i][j];
    }
  }
}

template <typename real>
cudaError_t gemm(int M, int N, int K, int batch, const real* A, long long lda, long long sA, const real* B,
                 long long ldb, long long sB, real* C, long long ldc, long long sC, cudaStream_t s) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  gemm_nn_kernel<real><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  return cudaGetLastError();
}

// transpose = false: F_mu = K_mu applied along mu to C (one input for every axis);
// transpose = true:  F_mu = K_mu^T applied along mu to C_mu (C holds one field per axis)
template <typename real>
cudaError_t frac_all_axes(const lbm_s* h, const real* C, real* F, cudaStream_t s, bool transpose = false) {
  const int n0 = h->sp.n[0], n1 = h->sp.n[1], n2 = h->sp.n[2];
  const long long nodes = h->sp.nodes;
  const real* K = static_cast<const real*>(transpose ? h->dev.KT : h->dev.K);
  const real* KT = static_cast<const real*>(transpose ? h->dev.K : h->dev.KT);
  const long long cstride = transpose ? nodes : 0;
  long long koff = 0;
  cudaError_t err;
  // axis x: F_0 = C (rows x n0) * K_0^T
  err = gemm<real>((int)(nodes / n0), n0, n0, 1, C, n0, 0, KT + koff, n0, 0, F, n0, 0, s);
  if (err != cudaSuccess) return err;
  koff += (long long)n0 * n0;
  // axis y: for each z-plane b, F_1[b] = K_1 * C[b]  (C[b] is n1 x n0)
  err = gemm<real>(n1, n0, n1, n2, K + koff, n1, 0, C + cstride, n0, (long long)n1 * n0, F + nodes, n0,
                   (long long)n1 * n0, s);
  if (err != cudaSuccess) return err;
  koff += (long long)n1 * n1;
  if (h->d == 3) {
    // axis z: F_2 = K_2 * C  (C is n2 x (n1 n0))
    err = gemm<real>(n2, n0 * n1, n2, 1, K + koff, n2, 0, C + 2 * cstride, (long long)n0 * n1, 0, F + 2 * nodes,
                     (long long)n0 * n1, 0, s);
  }
  return err;
}

}  // namespace

cudaError_t launch_frac_simt_T(const lbm_s* h, const void* in, void* out, cudaStream_t s) {
  if (h->elem == 8)
    return frac_all_axes<double>(h, static_cast<const double*>(in), static_cast<double*>(out), s, true);
  return frac_all_axes<float>(h, static_cast<const float*>(in), static_cast<float*>(out), s, true);
}

cudaError_t launch_frac_simt(const lbm_s* h, const void* C, void* F, cudaStream_t s) {
  if (h->elem == 8) return frac_all_axes<double>(h, static_cast<const double*>(C), static_cast<double*>(F), s);
  return frac_all_axes<float>(h, static_cast<const float*>(C), static_cast<float*>(F), s);
}

}  // namespace lbm
