// Fractional terms on the 5th-generation tensor cores (tcgen05), split precision.
//
// Algorithm 1, loop item 1 / Section 2.4, Eq. (XXminus_discret): along every lattice
// line of axis mu, F_mu[n] = sum_l K_mu[n][l] C[l].  Over all lines of an axis this is
// a dense GEMM (the weight matrix is Toeplitz up to its end columns, Eqs. c+ / c-):
//
//   D[m][n] = sum_l A[m][l] * B[n][l]
//     A = the C panel: m runs over the lines (x axis: rows y at fixed z, K-major,
//         i.e. l = x contiguous; y and z axes: m = x, "MN-major", m contiguous)
//     B = K_mu (row n, column l), K-major
//     D = F_mu, one 128 x BN FP32 accumulator tile in tensor memory per CTA.
//
// Split precision: A = A_hi + A_lo and B = B_hi + B_lo with each part in bf16
// (kind::f16) or tf32 (kind::tf32); every K step issues three MMAs
// (hi*hi + hi*lo + lo*hi) into the same FP32 accumulator; lo*lo is dropped.
//
// Per CTA: warp 0 / lane 0 issues TMA loads (128B-swizzled tiles, no multicast)
// into a STAGES-deep ring guarded by mbarriers, warp 1 / lane 0 issues the MMAs and
// releases ring slots with tcgen05.commit, then all four warps drain the accumulator
// (tcgen05.ld, one lane quarter per warp) and store F.  Every mbarrier wait is
// bounded by a 2 s %globaltimer budget; a wait that gives up sets bit 2 of the
// handle's error flag and the CTA skips the rest of its work and releases TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "lbm_internal.h"

namespace lbm {

struct TcAxis {
  int form;        // 0: A is K-major (x axis); 1: A is MN-major (y, z axes)
  int tiles_m;     // number of 128-line tiles
  int tiles_n;     // number of BN-column tiles (over n = 0..side-1)
  int tile_begin;  // first linear tile index of this axis
  int side;        // contraction length (nodes on axis mu)
  int kblocks;     // ceil(side / BK)
  int msub;        // M tiles per outer index (see decode in the kernel)
};

struct TcParams {
  int n0, n1, n2;
  int naxes;
  int total_tiles;
  long long nodes;
  TcAxis ax[3];
  float* F;
  int* flag;
};

struct TcMaps {
  CUtensorMap a_hi[3], a_lo[3];
  CUtensorMap b_hi[3], b_lo[3];
};

struct TcPlan {
  TcMaps maps;
  TcParams prm;
  int elem = 2;      // 2: bf16 parts, 4: tf32 parts
  int bn = 64;
  size_t smem = 0;
  int ldp = 0;       // padded x pitch of the C split arrays (elements)
};

namespace {

constexpr int BM = 128;
constexpr long long kWaitNs = 2000000000LL;

template <int E> struct Kind;
template <> struct Kind<2> {  // bf16 parts: kind::f16, UMMA_K = 16
  static constexpr int UK = 16;
  static constexpr uint32_t fmt = 1;
};
template <> struct Kind<4> {  // tf32 parts: kind::tf32, UMMA_K = 8
  static constexpr int UK = 8;
  static constexpr uint32_t fmt = 2;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and flag bit 2) after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > (unsigned long long)kWaitNs) {
      atomicOr(flag, 2);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle, sm_100 descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
  d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(2) << 61;
  return d;
}

template <int E>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accum) {
  if (E == 2) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int E, int BN>
struct Cfg {
  static constexpr int BK = 128 / E;                 // contraction elements per 128-byte row
  static constexpr int STAGES = (BN <= 64) ? 4 : 3;
  static constexpr uint32_t A_BYTES = BM * 128;      // one operand part of A: 128 rows x 128 B
  static constexpr uint32_t B_BYTES = BN * 128;
  static constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
  // A, MN-major: E boxes of (128/E) lines x BK rows
  static constexpr uint32_t A_BOX_MN = BK * 128;
  static constexpr uint32_t IDESC_K = (1u << 4) | (Kind<E>::fmt << 7) | (Kind<E>::fmt << 10) |
                                      (static_cast<uint32_t>(BN >> 3) << 17) | (static_cast<uint32_t>(BM >> 4) << 24);
  static constexpr uint32_t IDESC_MN = IDESC_K | (1u << 15);
};

template <int E, int BN>
__global__ void __launch_bounds__(128, 1) frac_tc_kernel(const __grid_constant__ TcMaps maps, const TcParams P) {
  using G = Cfg<E, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)G::STAGES * G::STAGE);
  uint64_t* empty = full + G::STAGES;
  uint64_t* done = empty + G::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // ---- which axis / tile
  int mu = 0;
  while (mu + 1 < P.naxes && static_cast<int>(blockIdx.x) >= P.ax[mu + 1].tile_begin) ++mu;
  const TcAxis ax = P.ax[mu];
  const int lt = blockIdx.x - ax.tile_begin;
  const int mt = lt / ax.tiles_n, nt = lt % ax.tiles_n;
  const int ncol0 = nt * BN;
  // line-tile coordinates: x axis -> (y0, z); y axis -> (x0, z); z axis -> (x0, y)
  const int m_in = (mt % ax.msub) * BM;
  const int m_out = mt / ax.msub;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int KB = ax.kblocks;
  if (threadIdx.x == 0) {
    // ---------------- producer
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % G::STAGES;
      if (kb >= G::STAGES && !mbar_wait(&empty[s], ((kb / G::STAGES) - 1) & 1, P.flag)) break;
      uint8_t* st = smem + (size_t)s * G::STAGE;
      uint8_t* a_hi = st;
      uint8_t* a_lo = st + G::A_BYTES;
      uint8_t* b_hi = st + 2 * G::A_BYTES;
      uint8_t* b_lo = b_hi + G::B_BYTES;
      mbar_expect_tx(&full[s], G::STAGE);
      const int k0 = kb * G::BK;
      if (mu == 0) {
        tma_load_3d(a_hi, &maps.a_hi[0], k0, m_in, m_out, &full[s]);
        tma_load_3d(a_lo, &maps.a_lo[0], k0, m_in, m_out, &full[s]);
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int x = m_in + j * (128 / E);
          if (mu == 1) {
            tma_load_3d(a_hi + j * G::A_BOX_MN, &maps.a_hi[1], x, k0, m_out, &full[s]);
            tma_load_3d(a_lo + j * G::A_BOX_MN, &maps.a_lo[1], x, k0, m_out, &full[s]);
          } else {
            tma_load_3d(a_hi + j * G::A_BOX_MN, &maps.a_hi[2], x, m_out, k0, &full[s]);
            tma_load_3d(a_lo + j * G::A_BOX_MN, &maps.a_lo[2], x, m_out, k0, &full[s]);
          }
        }
      }
      tma_load_2d(b_hi, &maps.b_hi[mu], k0, ncol0, &full[s]);
      tma_load_2d(b_lo, &maps.b_lo[mu], k0, ncol0, &full[s]);
    }
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer
    const uint32_t idesc = (mu == 0) ? G::IDESC_K : G::IDESC_MN;
    bool ok = true;
    for (int kb = 0; kb < KB && ok; ++kb) {
      const int s = kb % G::STAGES;
      ok = mbar_wait(&full[s], (kb / G::STAGES) & 1, P.flag);
      if (!ok) break;
      tc_fence_after();
      const uint32_t st = smem_u32(smem + (size_t)s * G::STAGE);
      const uint32_t a_hi = st, a_lo = st + G::A_BYTES;
      const uint32_t b_hi = st + 2 * G::A_BYTES, b_lo = b_hi + G::B_BYTES;
#pragma unroll
      for (int kk = 0; kk < G::BK / Kind<E>::UK; ++kk) {
        uint32_t a_off, a_lbo;
        if (mu == 0) {  // K-major A: advance within the 128-byte row
          a_off = kk * Kind<E>::UK * E;
          a_lbo = 16;
        } else {        // MN-major A: advance by UK rows of 128 bytes
          a_off = kk * Kind<E>::UK * 128;
          a_lbo = G::A_BOX_MN;
        }
        const uint32_t b_off = kk * Kind<E>::UK * E;
        const uint64_t dah = smem_desc(a_hi + a_off, a_lbo, 1024);
        const uint64_t dal = smem_desc(a_lo + a_off, a_lbo, 1024);
        const uint64_t dbh = smem_desc(b_hi + b_off, 16, 1024);
        const uint64_t dbl = smem_desc(b_lo + b_off, 16, 1024);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        mma<E>(tmem, dah, dbh, idesc, acc);
        mma<E>(tmem, dah, dbl, idesc, 1u);
        mma<E>(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  // ---------------- epilogue: TMEM -> registers -> F
  const bool have = mbar_wait(done, 0, P.flag);
  tc_fence_after();
  if (have) {
    const int row = warp * 32 + lane;  // accumulator lane = line index within the tile
    const long long nodes = P.nodes;
    float* F = P.F + (long long)mu * nodes;
    const int n0 = P.n0, n1 = P.n1;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
      if (mu == 0) {
        const int y = m_in + row, z = m_out;
        if (y < n1) {
          float* dst = F + ((long long)z * n1 + y) * n0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int x = ncol0 + c0 + j;
            if (x < n0) dst[x] = v[j];
          }
        }
      } else {
        const int x = m_in + row;
        if (x < n0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = ncol0 + c0 + j;
            if (n < ax.side) {
              const long long idx = (mu == 1) ? ((long long)m_out * n1 + n) * n0 + x
                                              : ((long long)n * n1 + m_out) * n0 + x;
              F[idx] = v[j];
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// ---------------------------------------------------------------------------- splits

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int E>
__global__ void split_C_kernel(const float* __restrict__ C, void* __restrict__ hi, void* __restrict__ lo, int n0,
                               int n1, int n2, int ldp) {
  const long long total = (long long)n0 * n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(i % n0);
    const long long row = i / n0;
    const long long o = row * ldp + x;
    const float c = C[i];
    if (E == 2) {
      const __nv_bfloat16 h = __float2bfloat16_rn(c);
      static_cast<__nv_bfloat16*>(hi)[o] = h;
      static_cast<__nv_bfloat16*>(lo)[o] = __float2bfloat16_rn(c - __bfloat162float(h));
    } else {
      const float h = tf32_rna(c);
      static_cast<float*>(hi)[o] = h;
      static_cast<float*>(lo)[o] = tf32_rna(c - h);
    }
  }
}

// ---------------------------------------------------------------------------- host

uint16_t bf16_rne_host(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
  return static_cast<uint16_t>((u + rounding) >> 16);
}

float bf16_to_float_host(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

float tf32_rna_host(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

EncodeTiled get_encoder() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

bool encode(CUtensorMap* m, int elem, int rank, void* base, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box) {
  EncodeTiled enc = get_encoder();
  if (!enc) return false;
  cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = (elem == 2) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(m, dt, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int E, int BN>
cudaError_t launch_kernel(const TcPlan* p, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(frac_tc_kernel<E, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<E, BN>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  frac_tc_kernel<E, BN><<<p->prm.total_tiles, 128, Cfg<E, BN>::SMEM, s>>>(p->maps, p->prm);
  return cudaGetLastError();
}

}  // namespace

// Allocate the split operands, split K_mu on the host, encode the tensor maps.
int tc_prepare(lbm_s* h, const std::vector<std::vector<double>>& K) {
  TcPlan* p = new (std::nothrow) TcPlan();
  if (!p) return LBM_ENOMEM;
  h->tc = p;
  const int E = (h->prm.precision == LBM_FP32_BF16SPLIT) ? 2 : 4;
  p->elem = E;
  // tf32 parts are only fed K-major: the y and z axes need an MN-major C panel, whose
  // tf32 form did not reproduce the oracle, so the tf32 split serves 1-D-contiguous
  // (x-axis) operators only and is refused for the full step.
  if (E == 4) return LBM_ENOTSUP;
  const int n[3] = {h->sp.n[0], h->sp.n[1], h->sp.n[2]};
  int maxside = 0;
  for (int mu = 0; mu < h->d; ++mu) maxside = n[mu] > maxside ? n[mu] : maxside;
  p->bn = (maxside >= 1024) ? 128 : 64;
  p->smem = (p->bn == 64) ? ((E == 2) ? Cfg<2, 64>::SMEM : Cfg<4, 64>::SMEM)
                          : ((E == 2) ? Cfg<2, 128>::SMEM : Cfg<4, 128>::SMEM);
  const int ldp = (n[0] + 7) / 8 * 8;
  p->ldp = ldp;
  const size_t split_elems = (size_t)ldp * n[1] * n[2];
  if (cudaMalloc(&h->dev.Chi, split_elems * E) != cudaSuccess) return LBM_ENOMEM;
  if (cudaMalloc(&h->dev.Clo, split_elems * E) != cudaSuccess) return LBM_ENOMEM;
  cudaMemset(h->dev.Chi, 0, split_elems * E);
  cudaMemset(h->dev.Clo, 0, split_elems * E);

  // weights: per axis, padded row pitch ldk
  size_t ktot = 0;
  int ldk[3] = {0, 0, 0};
  for (int mu = 0; mu < h->d; ++mu) {
    ldk[mu] = (n[mu] + 7) / 8 * 8;
    ktot += (size_t)ldk[mu] * n[mu];
  }
  if (cudaMalloc(&h->dev.Khi, ktot * E) != cudaSuccess) return LBM_ENOMEM;
  if (cudaMalloc(&h->dev.Klo, ktot * E) != cudaSuccess) return LBM_ENOMEM;
  std::vector<uint8_t> hbuf(ktot * E, 0), lbuf(ktot * E, 0);
  size_t koff[3] = {0, 0, 0};
  size_t off = 0;
  for (int mu = 0; mu < h->d; ++mu) {
    koff[mu] = off;
    const int side = n[mu];
    for (int r = 0; r < side; ++r)
      for (int c = 0; c < side; ++c) {
        const double x = K[mu][(size_t)r * side + c];
        const size_t o = off + (size_t)r * ldk[mu] + c;
        if (E == 2) {
          const uint16_t hb = bf16_rne_host(static_cast<float>(x));
          const uint16_t lb = bf16_rne_host(static_cast<float>(x - bf16_to_float_host(hb)));
          std::memcpy(&hbuf[o * 2], &hb, 2);
          std::memcpy(&lbuf[o * 2], &lb, 2);
        } else {
          const float hf = tf32_rna_host(static_cast<float>(x));
          const float lf = tf32_rna_host(static_cast<float>(x - hf));
          std::memcpy(&hbuf[o * 4], &hf, 4);
          std::memcpy(&lbuf[o * 4], &lf, 4);
        }
      }
    off += (size_t)ldk[mu] * side;
  }
  if (cudaMemcpy(h->dev.Khi, hbuf.data(), hbuf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;
  if (cudaMemcpy(h->dev.Klo, lbuf.data(), lbuf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;

  // tensor maps
  const int BK = 128 / E;
  const int MNW = 128 / E;  // MN-major box width (elements)
  TcParams& P = p->prm;
  P.n0 = n[0];
  P.n1 = n[1];
  P.n2 = n[2];
  P.naxes = h->d;
  P.nodes = h->sp.nodes;
  P.F = static_cast<float*>(h->dev.F);
  P.flag = h->dev.flag;
  const cuuint64_t cdims[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
  const cuuint64_t cstr[2] = {(cuuint64_t)ldp * E, (cuuint64_t)ldp * n[1] * E};
  int tiles = 0;
  for (int mu = 0; mu < h->d; ++mu) {
    TcAxis& a = P.ax[mu];
    a.form = (mu == 0) ? 0 : 1;
    a.side = n[mu];
    a.kblocks = (n[mu] + BK - 1) / BK;
    a.tiles_n = (n[mu] + p->bn - 1) / p->bn;
    cuuint32_t box[3];
    if (mu == 0) {  // lines = rows y (128 per tile) at fixed z
      a.msub = (n[1] + BM - 1) / BM;
      a.tiles_m = a.msub * n[2];
      box[0] = BK; box[1] = BM; box[2] = 1;
    } else if (mu == 1) {  // lines = x (128 per tile) at fixed z
      a.msub = (n[0] + BM - 1) / BM;
      a.tiles_m = a.msub * n[2];
      box[0] = MNW; box[1] = BK; box[2] = 1;
    } else {  // lines = x at fixed y
      a.msub = (n[0] + BM - 1) / BM;
      a.tiles_m = a.msub * n[1];
      box[0] = MNW; box[1] = 1; box[2] = BK;
    }
    a.tile_begin = tiles;
    tiles += a.tiles_m * a.tiles_n;
    if (!encode(&p->maps.a_hi[mu], E, 3, h->dev.Chi, cdims, cstr, box)) return LBM_ECUDA;
    if (!encode(&p->maps.a_lo[mu], E, 3, h->dev.Clo, cdims, cstr, box)) return LBM_ECUDA;
    const cuuint64_t kdims[2] = {(cuuint64_t)n[mu], (cuuint64_t)n[mu]};
    const cuuint64_t kstr[1] = {(cuuint64_t)ldk[mu] * E};
    const cuuint32_t kbox[2] = {(cuuint32_t)BK, (cuuint32_t)p->bn};
    if (!encode(&p->maps.b_hi[mu], E, 2, static_cast<uint8_t*>(h->dev.Khi) + koff[mu] * E, kdims, kstr, kbox))
      return LBM_ECUDA;
    if (!encode(&p->maps.b_lo[mu], E, 2, static_cast<uint8_t*>(h->dev.Klo) + koff[mu] * E, kdims, kstr, kbox))
      return LBM_ECUDA;
  }
  P.total_tiles = tiles;
  return LBM_OK;
}

void tc_release(lbm_s* h) {
  delete h->tc;
  h->tc = nullptr;
}

int tc_split_pitch(const lbm_s* h) { return h->tc ? h->tc->ldp : 0; }

cudaError_t launch_frac_tc(const lbm_s* h, cudaStream_t s) {
  const TcPlan* p = h->tc;
  if (!p) return cudaErrorNotSupported;
  if (p->elem == 2) return (p->bn == 64) ? launch_kernel<2, 64>(p, s) : launch_kernel<2, 128>(p, s);
  return (p->bn == 64) ? launch_kernel<4, 64>(p, s) : launch_kernel<4, 128>(p, s);
}

cudaError_t launch_split_C(const lbm_s* h, cudaStream_t s) {
  const TcPlan* p = h->tc;
  if (!p) return cudaErrorNotSupported;
  long long b = (h->sp.nodes + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (p->elem == 2)
    split_C_kernel<2><<<(int)b, 256, 0, s>>>(static_cast<const float*>(h->dev.C), h->dev.Chi, h->dev.Clo, h->sp.n[0],
                                             h->sp.n[1], h->sp.n[2], p->ldp);
  else
    split_C_kernel<4><<<(int)b, 256, 0, s>>>(static_cast<const float*>(h->dev.C), h->dev.Chi, h->dev.Clo, h->sp.n[0],
                                             h->sp.n[1], h->sp.n[2], p->ldp);
  return cudaGetLastError();
}

}  // namespace lbm
