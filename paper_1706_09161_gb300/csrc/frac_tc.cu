// Fractional terms on the 5th-generation tensor cores (tcgen05), split precision.
//
// Algorithm 1 (fractional terms) / Section 2.4, Eq. (XXminus_discret): along every lattice
// line of axis mu, F_mu[n] = sum_l K_mu[n][l] C[l].  Over all lines of an axis this is
// a dense GEMM (the weight matrix is Toeplitz up to its end columns, Eqs. c+ / c-):
//
//   D[m][n] = sum_l A[m][l] * B[n][l], accumulator lanes m always run along x so
//   that the epilogue stores are coalesced:
//     x axis:    A = K_x (m = output node x, K-major), B = C rows (n = y at fixed z,
//                K-major, l = x contiguous)
//     y, z axes: A = C panel (m = x, "MN-major": m contiguous), B = K_mu (n = output
//                node along mu, K-major)
//   one 128 x BN FP32 accumulator tile in tensor memory per CTA.
//
// Split precision: A = A_hi + A_lo and B = B_hi + B_lo with each part in bf16
// (kind::f16) or tf32 (kind::tf32); every K step issues three MMAs
// (hi*hi + hi*lo + lo*hi) into the same FP32 accumulator; lo*lo is dropped.
//
// Per CTA: warp 0 / lane 0 issues TMA loads (128B-swizzled tiles, no multicast)
// into a STAGES-deep ring guarded by mbarriers (the first loads leave before the
// accumulator is allocated), warp 1 / lane 0 issues the MMAs and releases ring slots
// with tcgen05.commit, then all four warps drain the accumulator (tcgen05.ld, one
// lane quarter per warp) into a shared [BN][128] tile that one TMA store writes to F.
// Small problems split the contraction over ksplit independent CTAs per tile: CTA
// `rank` contracts its k-range and stores its partial tile to slot `rank` of F, laid out
// [rank][axis][node]; the kernels that read F add the ksplit partials in rank order, so
// the result does not depend on timing (and no CTA waits for another).  Problems with many tiles use the persistent kernel further
// down (two TMEM accumulators, epilogue overlapping the next tile).  Every mbarrier wait is
// bounded by a 2 s %globaltimer budget; a wait that gives up sets bit 2 of the
// handle's error flag and the CTA skips the rest of its work and releases TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lbm_internal.h"
#include "tc_dev.cuh"

namespace lbm {
namespace {

// One output tile (or one k-slice of it when KS > 1) of one problem; `block` is the
// CTA's index among that problem's CTAs.  `maps` may live in parameter or global memory.
// per-tile operator: 4 warps (producer, MMA issuer, all four drain TMEM); tf32 adds warps 4-7,
// which with warps 2-3 split each stage's C into hi + lo and leave before the epilogue
constexpr int kTileSplitWarps = 6;
__host__ __device__ constexpr int tile_threads(int E) { return E == 4 ? 256 : 128; }

template <int E, int BN, int KS, int KP = 2>
__device__ __forceinline__ void frac_tc_tile(const TcMaps& maps, const TcParams& P, int block, uint8_t* smem_raw) {
  using G = Cfg<E, BN, KS, KP>;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::RING);
  uint64_t* empty = full + G::STAGES;
  uint64_t* done = empty + G::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  uint64_t* split = done + 2;  // tf32: the stage's C split into hi + lo by warps 2-7

  const int warp = threadIdx.x >> 5;

  // ---- which axis / tile / k-range: ksplit CTAs share a tile; CTA `rank` contracts
  // k-blocks [kb0, kb1)
  constexpr int ks = KS;
  const int cid = block / ks, rank = block % ks;
  const TileAt tl = decode_tile(P, cid, BN);
  const int mu = tl.mu, m_in = tl.m_in, m_out = tl.m_out, ncol0 = tl.ncol0;
  const TcAxis ax = P.ax[mu];
  const int kb0 = rank * ax.kblocks / ks, kb1 = (rank + 1) * ax.kblocks / ks;
  const int nkb = kb1 - kb0;
  const int nreg = acc_regions(nkb * ksteps<E>(), BN);  // TMEM accumulators, nreg * BN columns

  auto issue = [&](int i) {
    const int s = i % G::STAGES;
    mbar_expect_tx(&full[s], G::tx_bytes(mu));
    load_stage<E, BN, KP>(maps, tl, (kb0 + i) * G::BK, smem + (size_t)s * G::STAGE, &full[s]);
  };

  // ---- prologue: barrier setup and accumulator allocation overlap the previous kernel
  // (programmatic dependent launch); operand loads wait for its results
  if (threadIdx.x == 0) {
    for (int s = 0; s < G::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      if (E == 4) mbar_init(&split[s], kTileSplitWarps);  // one arrival per splitting warp
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the first stages' weight parts do not depend on the previous kernel
    const int pre = nkb < G::STAGES ? nkb : G::STAGES;
    for (int i = 0; i < pre; ++i) {
      mbar_expect_tx(&full[i], G::tx_bytes(mu));
      load_stage_weights<E, BN, KP>(maps, tl, (kb0 + i) * G::BK, smem + (size_t)i * G::STAGE, &full[i]);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int i = 0; i < pre; ++i)
      load_stage_conc<E, BN, KP>(maps, tl, (kb0 + i) * G::BK, smem + (size_t)i * G::STAGE, &full[i]);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(nreg * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  asm volatile("griddepcontrol.wait;" ::: "memory");  // F is written below
  // the next kernel may be scheduled now when this grid runs in one wave, else at the end
  if (P.early_trigger) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (threadIdx.x == 0) {
    // ---------------- producer (remaining k-blocks)
    for (int i = G::STAGES; i < nkb; ++i) {
      const int s = i % G::STAGES;
      if (!mbar_wait(&empty[s], ((i / G::STAGES) - 1) & 1, P.flag)) break;
      issue(i);
    }
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer (tf32: once the stage's C is split)
    const int amode = a_mode<E>(mu);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % G::STAGES;
      if (!mbar_wait(E == 4 ? &split[s] : &full[s], (i / G::STAGES) & 1, P.flag)) break;
      tc_fence_after();
      mma_stage<E, BN, KP>(tmem, i * ksteps<E>(), nreg, smem_u32(smem + (size_t)s * G::STAGE), amode);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  } else if (E == 4 && warp >= 2) {
    // ---------------- tf32: warps 2-7 split each stage's C into hi + lo
    for (int i = 0; i < nkb; ++i) {
      const int s = i % G::STAGES;
      int ok = 1;
      if ((threadIdx.x & 31) == 0) ok = mbar_wait(&full[s], (i / G::STAGES) & 1, P.flag) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);  // the lane's acquire, shared by the warp below
      if (!ok) break;
      __syncwarp();
      split_stage_tf32<E, BN, KP>(smem + (size_t)s * G::STAGE, mu, threadIdx.x - 64, 32 * kTileSplitWarps);
      __syncwarp();
      if ((threadIdx.x & 31) == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&split[s])) : "memory");
    }
  }
  __syncwarp();
  if (warp >= 4) return;  // tf32's extra splitting warps: the epilogue is warps 0-3

  // ---------------- epilogue
  bool have = mbar_wait(done, 0, P.flag);
  tc_fence_after();
  float* tile = reinterpret_cast<float*>(smem);  // the operand ring is idle once `done` fired
  const int row = threadIdx.x;                   // accumulator lane = x offset in the tile
  const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  int r0 = 0, r1 = BN;  // tile rows (output nodes n) this CTA writes
  // KS > 1: this CTA's partial sum over its k-range goes to partial slot `rank` of F
  // (F is [rank][axis][node]); the consumers add the KS partials in rank order
  const long long nodes = P.nodes;
  float* F = P.F + (long long)rank * P.naxes * nodes + (long long)mu * nodes;
  const int n0 = P.n0, n1 = P.n1;
  const int lim = (mu == 0) ? n1 : ax.side;  // output rows that exist
  // TMEM -> shared tile [BN][128] (lane = x), 32 rows at a time; with TMA stores each
  // 32-row chunk leaves by its own store as soon as it is in shared memory, so the stores
  // overlap the drain of the next chunk (each chunk has its own 16 KB of the tile)
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    float v[32], w[32];
    tmem_ld32(lane_addr + c0, v);
    for (int r = 1; r < nreg; ++r) {  // the regions, added in k order
      tmem_ld32(lane_addr + r * BN + c0, w);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += w[j];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[(c0 + j) * BM + row] = have ? v[j] : 0.0f;
    if (P.tma_store) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      named_sync128();  // warps 0-3 (tf32's extra warps have left)
      if (threadIdx.x == 0 && have && ncol0 + c0 < lim) {
        int c1, c2;
        if (mu == 2) {
          c1 = m_out;
          c2 = ncol0 + c0;
        } else {
          c1 = ncol0 + c0;
          c2 = m_out;
        }
        if (KS == 1)
          asm volatile(
              "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                  reinterpret_cast<uint64_t>(&maps.f[mu])),
              "r"(m_in), "r"(c1), "r"(c2), "r"(smem_u32(tile + c0 * BM))
              : "memory");
        else
          asm volatile(
              "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                  reinterpret_cast<uint64_t>(&maps.f[mu])),
              "r"(m_in), "r"(c1), "r"(c2), "r"(rank), "r"(smem_u32(tile + c0 * BM))
              : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
  }
  if (P.tma_store) {
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  } else {
    // rows of F that are not 16-byte aligned: plain stores, coalesced along x
    named_sync128();  // warps 0-3 (tf32's extra warps have left)
    const int x = m_in + row;
    if (have && x < n0) {
      for (int rr = r0; rr < r1; ++rr) {
        const int n = ncol0 + rr;  // x axis: row y at z = m_out; y/z axes: node along mu
        if (n >= lim) break;
        const long long idx = (mu == 2) ? ((long long)n * n1 + m_out) * n0 + x : ((long long)m_out * n1 + n) * n0 + x;
        F[idx] = tile[(rr - r0) * BM + row];
      }
    }
  }
  tc_fence_before();
  named_sync128();  // warps 0-3 (tf32's extra warps have left)
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nreg * BN) : "memory");
  }
  if (!P.early_trigger) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int E, int BN, int KS, int KP>
__global__ void __launch_bounds__(tile_threads(E), 1)
frac_tc_kernel(const __grid_constant__ TcMaps maps, const TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  frac_tc_tile<E, BN, KS, KP>(maps, P, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------- persistent form
// Problems with many tiles: one CTA per SM walks the tile list (tile t = first,
// first + stride, ...).  Warp 0 streams the k-blocks of consecutive tiles through the
// STAGES-deep operand ring without a break at tile boundaries, warp 1 issues each tile's
// MMAs into one of two TMEM accumulators (the i-th tile of the CTA into buffer i & 1),
// and warps 2-5 drain the other accumulator (tcgen05.ld, 32 columns at a time, through a
// double-buffered shared chunk and a TMA store), so a tile's epilogue overlaps the next
// tile's loads and MMAs.  With 128-column tiles each accumulator buffer has two regions:
// consecutive k-blocks alternate between them and the epilogue adds the two in FP32 (as
// the per-tile kernel's regions: shorter accumulation chains, smaller rounding error of
// the split forms).  Every wait is bounded as in the per-tile kernel; on a timeout
// the CTA stops issuing, waits (bounded) for its copies and MMAs in flight, releases
// TMEM and returns with bit 2 of the error flag set.
constexpr int PBN = 128;
constexpr int kPersistThreads = 192;
// tf32 adds eight warps (6-13) that split each stage's C into hi + lo
constexpr int kSplitWarps = 8;
__host__ __device__ constexpr int persist_threads(int E) { return E == 4 ? kPersistThreads + 32 * kSplitWarps : kPersistThreads; }

// BN = 128 (three ring stages; two with the weights in three parts) or 256 (two; the
// double accumulator then fills TMEM); KP = weight parts (2, or 3 for the five-product
// bf16 form, BN = 128 only)
template <int E, int BN = PBN, int KP = 2>
struct PCfg {
  using G = Cfg<E, BN, 1, KP>;
  static constexpr int STAGES = (BN == 128 && KP == 2) ? 3 : 2;
  static constexpr int NREG = (2 * 2 * BN <= 512) ? 2 : 1;  // accumulator regions per buffer
  static_assert(NREG <= ksteps<E>(), "every region is written by a tile's first k-block");
  static constexpr int TMEM_COLS = 2 * NREG * BN;
  static constexpr uint32_t CHUNK = 32 * BM * 4;  // 32 output rows x 128 x (FP32)
  static constexpr size_t RING = (size_t)STAGES * G::STAGE;
  static constexpr size_t SMEM = RING + 2 * CHUNK + 1024 /*align*/ + 256 /*barriers*/;
  static_assert(SMEM <= 232448, "persistent operator exceeds the shared memory of one CTA");
  static_assert(KP == 2 || BN == 128, "three weight parts: 128-column tiles only");
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Locate(t, maps, prm, cid): the problem and local tile index of global tile t
template <int E, int BN, int KP, class Locate>
__device__ __forceinline__ void persist_body(const Locate& locate, int ntiles, int* flag, uint8_t* smem_raw) {
  using C = PCfg<E, BN, KP>;
  using G = typename C::G;
  constexpr int STAGES = C::STAGES;
  constexpr int NREG = C::NREG;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* stage_out = reinterpret_cast<float*>(smem + C::RING);  // [2][32][128]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::RING + 2 * C::CHUNK);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;  // [2]
  uint64_t* tempty = tfull + 2;      // [2]
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  int* s_ok = reinterpret_cast<int*>(tmem_slot + 1);
  uint64_t* split = drain + 2;  // [STAGES] tf32: the stage's C split into hi + lo by warps 6-13

  const int warp = threadIdx.x >> 5;
  const int first = blockIdx.x, stride = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      if (E == 4) mbar_init(&split[s], kSplitWarps);  // one arrival per splitting warp
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 1);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // programmatic dependent launch: C (loaded) and F (stored) belong to the previous kernels
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (threadIdx.x == 0) {
    // ---------------- producer
    int r = 0;
    bool ok = true;
    for (int t = first; t < ntiles && ok; t += stride) {
      const TcMaps* maps;
      const TcParams* P;
      int cid;
      locate(t, maps, P, cid);
      const TileAt tl = decode_tile(*P, cid, BN);
      const int nkb = P->ax[tl.mu].kblocks;
      for (int kb = 0; kb < nkb; ++kb, ++r) {
        const int s = r % STAGES;
        if (r >= STAGES && !mbar_wait(&empty[s], ((r / STAGES) - 1) & 1, flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full[s], G::tx_bytes(tl.mu));
        load_stage<E, BN, KP>(*maps, tl, kb * G::BK, smem + (size_t)s * G::STAGE, &full[s]);
      }
    }
    // every issued copy has landed before the CTA may leave (bounded)
    for (int q = (r > STAGES ? r - STAGES : 0); q < r; ++q) mbar_wait(&full[q % STAGES], (q / STAGES) & 1, flag);
  } else if (threadIdx.x == 32) {
    // ---------------- MMA issuer
    int r = 0, i = 0;
    bool ok = true;
    for (int t = first; t < ntiles && ok; t += stride, ++i) {
      const TcMaps* maps;
      const TcParams* P;
      int cid;
      locate(t, maps, P, cid);
      const TileAt tl = decode_tile(*P, cid, BN);
      const int nkb = P->ax[tl.mu].kblocks;
      const int b = i & 1;
      if (i >= 2 && !mbar_wait(&tempty[b], ((i >> 1) - 1) & 1, flag)) break;
      tc_fence_after();
      const uint32_t d = tmem + b * NREG * BN;
      const int amode = a_mode<E>(tl.mu);
      for (int kb = 0; kb < nkb; ++kb, ++r) {
        const int s = r % STAGES;
        if (!mbar_wait(E == 4 ? &split[s] : &full[s], (r / STAGES) & 1, flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // k-step c = kb * ksteps + kk accumulates into region c % NREG of this buffer
        mma_stage<E, BN, KP>(d, kb * ksteps<E>(), NREG, smem_u32(smem + (size_t)s * G::STAGE), amode);
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(&tfull[b]);
    }
    mma_commit(drain);  // fires once every MMA issued above has completed
  } else if (E == 4 && warp >= 6) {
    // ---------------- tf32: warps 6-13 split each stage's C into hi + lo
    int r = 0;
    bool ok = true;
    for (int t = first; t < ntiles && ok; t += stride) {
      const TcMaps* maps;
      const TcParams* P;
      int cid;
      locate(t, maps, P, cid);
      const TileAt tl = decode_tile(*P, cid, BN);
      const int nkb = P->ax[tl.mu].kblocks;
      for (int kb = 0; kb < nkb; ++kb, ++r) {
        const int s = r % STAGES;
        int got = 1;
        if ((threadIdx.x & 31) == 0) got = mbar_wait(&full[s], (r / STAGES) & 1, flag) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);  // the lane's acquire, shared by the warp below
        if (!got) {
          ok = false;
          break;
        }
        __syncwarp();
        split_stage_tf32<E, BN, KP>(smem + (size_t)s * G::STAGE, tl.mu, threadIdx.x - kPersistThreads,
                                    32 * kSplitWarps);
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&split[s]);
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: 128 threads, TMEM lane quarter = warp % 4
    const int et = threadIdx.x - 64;
    const int q = warp & 3;
    const int row = q * 32 + (threadIdx.x & 31);  // accumulator lane = x offset in the tile
    int i = 0, chunk = 0;
    for (int t = first; t < ntiles; t += stride, ++i) {
      const TcMaps* maps;
      const TcParams* P;
      int cid;
      locate(t, maps, P, cid);
      const TileAt tl = decode_tile(*P, cid, BN);
      const int b = i & 1;
      if (et == 0) *s_ok = mbar_wait(&tfull[b], (i >> 1) & 1, flag) ? 1 : 0;
      epi_sync();
      if (!*s_ok) break;
      tc_fence_after();
      const long long nodes = P->nodes;
      float* F = P->F + (long long)tl.mu * nodes;
      const int n0 = P->n0, n1 = P->n1;
      const int lim = (tl.mu == 0) ? n1 : P->ax[tl.mu].side;  // output rows that exist
      // regions written by this tile (every one: a k-block has ksteps >= NREG k-steps)
      const int nreg = NREG;
      for (int c0 = 0; c0 < BN; c0 += 32, ++chunk) {
        float v[32];
        const uint32_t abase = tmem + b * NREG * BN + (static_cast<uint32_t>(q * 32) << 16) + c0;
        tmem_ld32(abase, v);
        for (int rg = 1; rg < nreg; ++rg) {  // the regions, added in k order
          float w[32];
          tmem_ld32(abase + rg * BN, w);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] += w[j];
        }
        if (c0 + 32 >= BN) {
          // the accumulator is drained: hand it back to the MMA warp
          tc_fence_before();
        }
        if (P->tma_store) {
          float* sb = stage_out + (chunk & 1) * (32 * BM);
          if (et == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          epi_sync();  // the store that last read this buffer is done with it
#pragma unroll
          for (int j = 0; j < 32; ++j) sb[j * BM + row] = v[j];
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          epi_sync();
          if (et == 0) {
            if (c0 + 32 >= BN) mbar_arrive(&tempty[b]);
            if (tl.ncol0 + c0 < lim) {
              int c1, c2;
              if (tl.mu == 2) {
                c1 = tl.m_out;
                c2 = tl.ncol0 + c0;
              } else {
                c1 = tl.ncol0 + c0;
                c2 = tl.m_out;
              }
              asm volatile(
                  "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                      reinterpret_cast<uint64_t>(&maps->f[tl.mu])),
                  "r"(tl.m_in), "r"(c1), "r"(c2), "r"(smem_u32(sb))
                  : "memory");
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        } else {
          // rows of F that are not 16-byte aligned: plain stores, coalesced along x
          const int x = tl.m_in + row;
          if (x < n0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int n = tl.ncol0 + c0 + j;
              const long long idx = (tl.mu == 2) ? ((long long)n * n1 + tl.m_out) * n0 + x
                                                 : ((long long)tl.m_out * n1 + n) * n0 + x;
              if (n < lim) F[idx] = v[j];
            }
          }
          if (c0 + 32 >= BN) {
            epi_sync();
            if (et == 0) mbar_arrive(&tempty[b]);
          }
        }
      }
    }
    if (et == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    if (threadIdx.x == 32) mbar_wait(drain, 0, flag);
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

struct LocateOne {
  const TcMaps* maps;
  const TcParams* prm;
  __device__ __forceinline__ void operator()(int t, const TcMaps*& m, const TcParams*& p, int& cid) const {
    m = maps;
    p = prm;
    cid = t;
  }
};

struct LocateBatch {
  const TcMaps* maps;
  const TcParams* prm;
  const int* start;
  int nprob;
  __device__ __forceinline__ void operator()(int t, const TcMaps*& m, const TcParams*& p, int& cid) const {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&start[mid]) <= t) lo = mid;
      else hi = mid - 1;
    }
    m = maps + lo;
    p = prm + lo;
    cid = t - __ldg(&start[lo]);
  }
};

template <int E, int BN, int KP>
__global__ void __launch_bounds__(persist_threads(E), 1)
frac_tc_persist_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  persist_body<E, BN, KP>(LocateOne{&maps, &P}, P.total_tiles, P.flag, smem_raw);
}

template <int E, int KP>
__global__ void __launch_bounds__(kPersistThreads, 1)
frac_tc_persist_batch_kernel(const TcMaps* __restrict__ maps, const TcParams* __restrict__ prm,
                             const int* __restrict__ start, int nprob, int ntiles, int* flag) {
  extern __shared__ uint8_t smem_raw[];
  persist_body<E, PBN, KP>(LocateBatch{maps, prm, start, nprob}, ntiles, flag, smem_raw);
}

// ---------------------------------------------------------------------------- splits

template <int E>
__global__ void split_C_kernel(const float* __restrict__ C, void* __restrict__ hi, void* __restrict__ lo,
                               void* __restrict__ lo2, int n0, int n1, int n2, int ldp) {
  const long long total = (long long)n0 * n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(i % n0);
    const long long row = i / n0;
    const long long o = row * ldp + x;
    const float c = C[i];
    if (E == 2) {
      // each part the bf16 rounding of what the previous ones left (exact FP32 residuals)
      const __nv_bfloat16 h = __float2bfloat16_rn(c);
      const float r1 = c - __bfloat162float(h);
      const __nv_bfloat16 l = __float2bfloat16_rn(r1);
      static_cast<__nv_bfloat16*>(hi)[o] = h;
      static_cast<__nv_bfloat16*>(lo)[o] = l;
      if (lo2) static_cast<__nv_bfloat16*>(lo2)[o] = __float2bfloat16_rn(r1 - __bfloat162float(l));
    } else {
      static_cast<float*>(hi)[o] = c;  // tf32: the operator splits C in shared memory
    }
  }
}

// bf16 forms with g(x): for every axis mu the parts of g_mu(x) C (g_mu at g[mu * nodes + i]),
// each the bf16 rounding of what the previous ones left, at gp.p[mu][part] (pitch ldp)
struct GParts {
  void* p[3][3];
};
__global__ void split_G_kernel(const float* __restrict__ C, const float* __restrict__ g, GParts gp, int d, int cparts,
                               int n0, int n1, int n2, int ldp) {
  const long long total = (long long)n0 * n1 * n2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = static_cast<int>(i % n0);
    const long long o = (i / n0) * ldp + x;
    const float c = C[i];
    for (int mu = 0; mu < d; ++mu) {
      const float v = g[mu * total + i] * c;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(h);
      const __nv_bfloat16 l = __float2bfloat16_rn(r1);
      static_cast<__nv_bfloat16*>(gp.p[mu][0])[o] = h;
      static_cast<__nv_bfloat16*>(gp.p[mu][1])[o] = l;
      if (cparts == 3) static_cast<__nv_bfloat16*>(gp.p[mu][2])[o] = __float2bfloat16_rn(r1 - __bfloat162float(l));
    }
  }
}

// tf32: C regrouped along axis mu (1: y, 2: z) in groups of 4 (layout at TcPlan::ct_hi):
// one thread per (x, group, remaining axis) reads the group's 4 values (coalesced over x)
// and writes one 16-byte group (coalesced over x); values past the end of the axis are zero.
__global__ void split_T_kernel(const float* __restrict__ C, float* __restrict__ out, int n0, int n1, int n2, int mu,
                               int tg, int tpx) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = blockIdx.y;   // group along mu
  const int r = blockIdx.z;   // remaining axis: z for the y copy, y for the z copy
  if (x >= n0) return;
  const long long plane = (long long)n0 * n1;
  const int side = mu == 1 ? n1 : n2;
  const long long step = mu == 1 ? n0 : plane;  // distance between consecutive mu
  const long long base = mu == 1 ? (long long)r * plane + x : (long long)r * n0 + x;
  float v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = (4 * g + k < side) ? C[base + (4 * g + k) * step] : 0.0f;
  const long long o = mu == 1 ? (((long long)r * tg + g) * tpx + x) * 4 : (((long long)g * n1 + r) * tpx + x) * 4;
  *reinterpret_cast<float4*>(out + o) = make_float4(v[0], v[1], v[2], v[3]);
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
            const cuuint32_t* box, bool swizzle = true) {
  EncodeTiled enc = get_encoder();
  if (!enc) return false;
  cuuint32_t es[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = (elem == 2) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(m, dt, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int E, int BN, int KS, int KP = 2>
cudaError_t launch_kernel(const TcPlan* p, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, frac_tc_kernel<E, BN, KS, KP>, (int)Cfg<E, BN, KS, KP>::SMEM); e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p->prm.total_tiles * KS, 1, 1);
  cfg.blockDim = dim3(tile_threads(E), 1, 1);
  cfg.dynamicSmemBytes = Cfg<E, BN, KS, KP>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = p->pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, frac_tc_kernel<E, BN, KS, KP>, p->maps, p->prm);
}

template <int E, int BN, int KP = 2>
cudaError_t launch_bn(const TcPlan* p, cudaStream_t s) {
  switch (p->prm.ksplit) {
    case 1: return launch_kernel<E, BN, 1, KP>(p, s);
    case 2: return launch_kernel<E, BN, 2, KP>(p, s);
    case 4: return launch_kernel<E, BN, 4, KP>(p, s);
    default: return launch_kernel<E, BN, 8, KP>(p, s);
  }
}


template <int E, int BN, int KP = 2>
cudaError_t launch_persist(const TcPlan* p, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, frac_tc_persist_kernel<E, BN, KP>, (int)PCfg<E, BN, KP>::SMEM);
      e != cudaSuccess)
    return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(p->prm.total_tiles, device_sms()), 1, 1);  // one CTA per SM
  cfg.blockDim = dim3(persist_threads(E), 1, 1);
  cfg.dynamicSmemBytes = PCfg<E, BN, KP>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = p->pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, frac_tc_persist_kernel<E, BN, KP>, p->maps, p->prm);
}

}  // namespace

// Split K_mu (FP64, row-major side x side) into the plan's parts on the host and upload
// them (rows padded to ldk[mu], axis blocks at koff[mu]); each part rounds what the previous
// ones left.
int tc_set_weights(lbm_s* h, const std::vector<std::vector<double>>& K) {
  TcPlan* p = h->tc;
  if (!p) return LBM_EINVAL;
  const int E = p->elem;
  const int n[3] = {h->sp.n[0], h->sp.n[1], h->sp.n[2]};
  size_t ktot = 0;
  for (int mu = 0; mu < h->d; ++mu) ktot += (size_t)p->ldk[mu] * n[mu];
  std::vector<uint8_t> hbuf(ktot * E, 0), lbuf(ktot * E, 0), l2buf(p->kparts == 3 ? ktot * E : 0, 0);
  for (int mu = 0; mu < h->d; ++mu) {
    const size_t off = p->koff[mu];
    const int side = n[mu];
    for (int r = 0; r < side; ++r)
      for (int c = 0; c < side; ++c) {
        const double x = K[mu][(size_t)r * side + c];
        const size_t o = off + (size_t)r * p->ldk[mu] + c;
        if (E == 2) {
          const uint16_t hb = bf16_rne_host(static_cast<float>(x));
          const double r1 = x - bf16_to_float_host(hb);
          const uint16_t lb = bf16_rne_host(static_cast<float>(r1));
          std::memcpy(&hbuf[o * 2], &hb, 2);
          std::memcpy(&lbuf[o * 2], &lb, 2);
          if (p->kparts == 3) {
            const uint16_t l2 = bf16_rne_host(static_cast<float>(r1 - bf16_to_float_host(lb)));
            std::memcpy(&l2buf[o * 2], &l2, 2);
          }
        } else {
          const float hf = tf32_rna_host(static_cast<float>(x));
          const float lf = tf32_rna_host(static_cast<float>(x - hf));
          std::memcpy(&hbuf[o * 4], &hf, 4);
          std::memcpy(&lbuf[o * 4], &lf, 4);
        }
      }
  }
  if (cudaMemcpy(h->dev.Khi, hbuf.data(), hbuf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;
  if (cudaMemcpy(h->dev.Klo, lbuf.data(), lbuf.size(), cudaMemcpyHostToDevice) != cudaSuccess) return LBM_ECUDA;
  if (p->kparts == 3 &&
      cudaMemcpy(h->dev.Kl2, l2buf.data(), l2buf.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return LBM_ECUDA;
  return LBM_OK;
}

// Allocate the split operands, split K_mu on the host, encode the tensor maps.
int tc_prepare(lbm_s* h, const std::vector<std::vector<double>>& K, int force_bn, int force_ks) {
  TcPlan* p = new (std::nothrow) TcPlan();
  if (!p) return LBM_ENOMEM;
  h->tc = p;
  const int E = bf16_parts(h->prm.precision) ? 2 : 4;
  p->elem = E;
  p->kparts = (h->prm.precision == LBM_FP32_BF16SPLIT5 || h->prm.precision == LBM_FP32_BF16SPLIT6) ? 3 : 2;
  p->cparts = (h->prm.precision == LBM_FP32_BF16SPLIT6) ? 3 : 2;
  // tf32 parts are fed K-major on every axis: the y and z axes read copies of the C split
  // regrouped along y (resp. z), written each step by the collide-stream kernel (TMA-fed
  // marches) or by split_T_kernel.
  const int n[3] = {h->sp.n[0], h->sp.n[1], h->sp.n[2]};
  int maxside = 0;
  for (int mu = 0; mu < h->d; ++mu) maxside = n[mu] > maxside ? n[mu] : maxside;
  (void)maxside;
  const int ldp = (n[0] + 7) / 8 * 8;
  p->ldp = ldp;
  const size_t split_elems = (size_t)ldp * n[1] * n[2];
  // bf16: the parts of C; tf32: C itself (FP32), split into hi + lo by the operator
  if (dev_alloc(h, (void**)&h->dev.Chi, split_elems * E) != cudaSuccess) return LBM_ENOMEM;
  cudaMemset(h->dev.Chi, 0, split_elems * E);
  if (E == 2) {
    if (dev_alloc(h, (void**)&h->dev.Clo, split_elems * E) != cudaSuccess) return LBM_ENOMEM;
    cudaMemset(h->dev.Clo, 0, split_elems * E);
  }
  if (p->cparts == 3) {
    if (dev_alloc(h, (void**)&h->dev.Cl2, split_elems * E) != cudaSuccess) return LBM_ENOMEM;
    cudaMemset(h->dev.Cl2, 0, split_elems * E);
  }
  if (E == 4) {
    p->tpx = (n[0] + 15) / 16 * 16;
    for (int mu = 1; mu < h->d; ++mu) {
      p->tg[mu] = (n[mu] + 3) / 4;
      const size_t cnt = (size_t)4 * p->tg[mu] * p->tpx * (h->sp.nodes / n[0] / n[mu]);
      if (dev_alloc(h, &p->ct_hi[mu], cnt * 4) != cudaSuccess) return LBM_ENOMEM;
      cudaMemset(p->ct_hi[mu], 0, cnt * 4);
    }
  }

  // weights: per axis, padded row pitch ldk
  size_t ktot = 0;
  int ldk[3] = {0, 0, 0};
  for (int mu = 0; mu < h->d; ++mu) {
    ldk[mu] = (n[mu] + 7) / 8 * 8;
    ktot += (size_t)ldk[mu] * n[mu];
  }
  if (dev_alloc(h, (void**)&h->dev.Khi, ktot * E) != cudaSuccess) return LBM_ENOMEM;
  if (dev_alloc(h, (void**)&h->dev.Klo, ktot * E) != cudaSuccess) return LBM_ENOMEM;
  if (p->kparts == 3 && dev_alloc(h, (void**)&h->dev.Kl2, ktot * E) != cudaSuccess) return LBM_ENOMEM;
  size_t koff[3] = {0, 0, 0};
  size_t off = 0;
  for (int mu = 0; mu < h->d; ++mu) {
    koff[mu] = off;
    off += (size_t)ldk[mu] * n[mu];
  }
  for (int mu = 0; mu < h->d; ++mu) {
    p->ldk[mu] = ldk[mu];
    p->koff[mu] = koff[mu];
  }
  if (int rc = tc_set_weights(h, K)) return rc;
  p->f_elems = (size_t)h->d * h->sp.nodes;

  // default plan: column tiles of 128 (an M = 128 MMA costs the same for any N <= 128)
  // or 256 when that still fills the GPU; small problems split the contraction over up
  // to 8 CTAs per tile so that about one CTA per SM is busy; many tiles: the persistent
  // kernel (128-column tiles, no split); batched handles always use it
  const int kSMs = device_sms();
  int bn = (p->kparts == 2 && tc_count_tiles(h, 256) >= kSMs) ? 256 : 128;
  const int kbmin = tc_kbmin(h);
  int ks = 1;
  const long long nt = tc_count_tiles(h, bn);
  while (ks * 2 <= 8 && ks * 2 <= kbmin && nt * ks * 2 <= kSMs) ks *= 2;
  bool persist = false;
  if (force_bn > 0) {
    bn = force_bn;
    ks = std::max(1, force_ks);
    persist = (force_bn == PBN && ks == 1);
  } else if (tc_count_tiles(h, PBN) >= 2 * kSMs) {
    persist = true;
    bn = PBN;
    ks = 1;
  }
  return tc_replan(h, bn, ks, persist ? 1 : 0);
}

long long tc_count_tiles(const lbm_s* h, int bn) {
  const int n[3] = {h->sp.n[0], h->sp.n[1], h->sp.n[2]};
  long long t = 0;
  for (int mu = 0; mu < h->d; ++mu) {
    const long long msub = (n[0] + BM - 1) / BM;
    const long long outer = (mu == 0 || mu == 1) ? n[2] : n[1];
    const long long ncols = (mu == 0) ? n[1] : n[mu];
    t += msub * outer * ((ncols + bn - 1) / bn);
  }
  return t;
}

int tc_kbmin(const lbm_s* h) {
  const int BK = 128 / (bf16_parts(h->prm.precision) ? 2 : 4);
  int kbmin = 1 << 30;
  for (int mu = 0; mu < h->d; ++mu) kbmin = std::min(kbmin, (h->sp.n[mu] + BK - 1) / BK);
  return kbmin;
}

// (Re)plan the operator: column tile width bn, contraction split ks, persistent or per
// tile; re-encodes every tensor map and grows the F buffer when the split needs it.
int tc_replan(lbm_s* h, int bn, int ks, int persist) {
  TcPlan* p = h->tc;
  if (!p) return LBM_EINVAL;
  if (!(bn == 64 || bn == 128 || bn == 256) || !(ks == 1 || ks == 2 || ks == 4 || ks == 8)) return LBM_EINVAL;
  if ((persist && ((bn != PBN && bn != 256) || ks != 1)) || (bn == 256 && ks != 1) || ks > tc_kbmin(h))
    return LBM_EINVAL;
  // the five- and six-product forms keep third parts per stage: 64 or 128 columns
  if (p->kparts == 3 && bn == 256) return LBM_EINVAL;
  const int E = p->elem;
  const int n[3] = {h->sp.n[0], h->sp.n[1], h->sp.n[2]};
  const int ldp = p->ldp;
  const int* ldk = p->ldk;
  const size_t* koff = p->koff;
  p->bn = bn;
  p->persist = persist != 0;
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
  const int kSMs = device_sms();
  P.ksplit = ks;
  P.tma_store = (n[0] % 4 == 0) ? 1 : 0;
  int tiles = 0;
  for (int mu = 0; mu < h->d; ++mu) {
    TcAxis& a = P.ax[mu];
    a.form = (mu == 0) ? 0 : 1;
    a.side = n[mu];
    a.kblocks = (n[mu] + BK - 1) / BK;
    a.msub = (n[0] + BM - 1) / BM;  // 128-wide x tiles on every axis
    cuuint32_t box[3];
    if (mu == 0) {  // B = C rows: BN rows y at fixed z
      a.tiles_m = a.msub * n[2];
      a.tiles_n = (n[1] + p->bn - 1) / p->bn;
      box[0] = BK; box[1] = p->bn; box[2] = 1;
    } else if (mu == 1) {  // A = C panel, lines = x at fixed z
      a.tiles_m = a.msub * n[2];
      a.tiles_n = (n[1] + p->bn - 1) / p->bn;
      box[0] = MNW; box[1] = BK; box[2] = 1;
    } else {  // lines = x at fixed y
      a.tiles_m = a.msub * n[1];
      a.tiles_n = (n[2] + p->bn - 1) / p->bn;
      box[0] = MNW; box[1] = 1; box[2] = BK;
    }
    a.tile_begin = tiles;
    tiles += a.tiles_m * a.tiles_n;
    if (E == 4 && mu > 0) {
      // regrouped copy, no swizzle, rows of 16 x-groups (256 bytes): y copy dims (64, x
      // blocks, y groups, z), box (64, 8, BK / 4, 1); z copy dims (64, x blocks, y, z
      // groups), box (64, 8, 1, BK / 4)
      const cuuint64_t g = (cuuint64_t)p->tg[mu], xb = (cuuint64_t)p->tpx / 16;
      const cuuint64_t tdims[4] = {64, xb, mu == 1 ? g : (cuuint64_t)n[1], mu == 1 ? (cuuint64_t)n[2] : g};
      const cuuint64_t tstr[3] = {256, (cuuint64_t)16 * p->tpx, (cuuint64_t)16 * p->tpx * tdims[2]};
      const cuuint32_t tbox[4] = {64, (cuuint32_t)BM / 16, mu == 1 ? (cuuint32_t)(BK / 4) : 1u,
                                  mu == 1 ? 1u : (cuuint32_t)(BK / 4)};
      if (!encode(&p->maps.c_hi[mu], E, 4, p->ct_hi[mu], tdims, tstr, tbox, false)) return LBM_ECUDA;
    } else {
      // the split of C, or with g(x) the bf16 split of this axis's g_mu(x) C (tf32: Chi holds
      // G_0 then)
      const bool gparts = p->gvar && E == 2;
      void* c0 = gparts ? p->gp[mu][0] : h->dev.Chi;
      void* c1 = gparts ? p->gp[mu][1] : h->dev.Clo;
      void* c2 = gparts ? p->gp[mu][2] : h->dev.Cl2;
      if (!encode(&p->maps.c_hi[mu], E, 3, c0, cdims, cstr, box)) return LBM_ECUDA;
      if (E == 2 && !encode(&p->maps.c_lo[mu], E, 3, c1, cdims, cstr, box)) return LBM_ECUDA;
      if (p->cparts == 3 && !encode(&p->maps.c_l2[mu], E, 3, c2, cdims, cstr, box)) return LBM_ECUDA;
    }
    const cuuint64_t kdims[2] = {(cuuint64_t)n[mu], (cuuint64_t)n[mu]};
    const cuuint64_t kstr[1] = {(cuuint64_t)ldk[mu] * E};
    const cuuint32_t kbox[2] = {(cuuint32_t)BK, (cuuint32_t)(mu == 0 ? BM : p->bn)};
    if (!encode(&p->maps.k_hi[mu], E, 2, static_cast<uint8_t*>(h->dev.Khi) + koff[mu] * E, kdims, kstr, kbox))
      return LBM_ECUDA;
    if (!encode(&p->maps.k_lo[mu], E, 2, static_cast<uint8_t*>(h->dev.Klo) + koff[mu] * E, kdims, kstr, kbox))
      return LBM_ECUDA;
    if (p->kparts == 3 &&
        !encode(&p->maps.k_l2[mu], E, 2, static_cast<uint8_t*>(h->dev.Kl2) + koff[mu] * E, kdims, kstr, kbox))
      return LBM_ECUDA;
  }
  // split contraction: F holds one partial sum per rank, [rank][axis][node]; the
  // kernels that read F add them in rank order
  const size_t need = (size_t)ks * h->d * h->sp.nodes;
  if (need > p->f_elems) {
    dev_free(h, h->dev.F);
    h->dev.F = nullptr;
    p->f_elems = 0;
    if (dev_alloc(h, (void**)&h->dev.F, need * 4) != cudaSuccess) return LBM_ENOMEM;
    p->f_elems = need;
  }
  P.F = static_cast<float*>(h->dev.F);
  h->sp.ksum = ks;
  h->sp.pstride = (ks > 1) ? (long long)h->d * h->sp.nodes : 0;
  if (P.tma_store) {
    for (int mu = 0; mu < h->d; ++mu) {
      // 32-row chunks of an output tile (per tile: of one rank's partial when ks > 1)
      const cuuint32_t rows = 32u;
      const cuuint64_t fd[4] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2], (cuuint64_t)ks};
      const cuuint64_t fs[3] = {(cuuint64_t)n[0] * 4, (cuuint64_t)n[0] * n[1] * 4,
                                (cuuint64_t)h->d * h->sp.nodes * 4};
      const cuuint32_t fb[4] = {BM, mu == 2 ? 1u : rows, mu == 2 ? rows : 1u, 1u};
      const cuuint32_t es[4] = {1, 1, 1, 1};
      EncodeTiled enc = get_encoder();
      if (!enc) return LBM_ECUDA;
      CUresult r = enc(&p->maps.f[mu], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, ks > 1 ? 4 : 3,
                       static_cast<float*>(h->dev.F) + (size_t)mu * h->sp.nodes, fd, fs, fb, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return LBM_ECUDA;
    }
  }
  P.total_tiles = tiles;
  P.early_trigger = (tiles * ks <= kSMs) ? 1 : 0;
  return LBM_OK;
}

void tc_release(lbm_s* h) {
  if (h->tc)
    for (int mu = 0; mu < 3; ++mu) {
      dev_free(h, h->tc->ct_hi[mu]);
      for (int k = 0; k < 3; ++k) dev_free(h, h->tc->gp[mu][k]);
    }
  delete h->tc;
  h->tc = nullptr;
  dev_free(h, h->batch_tc_maps);
  dev_free(h, h->batch_tc_prm);
  dev_free(h, h->batch_tc_start);
  h->batch_tc_maps = h->batch_tc_prm = nullptr;
  h->batch_tc_start = nullptr;
}

int tc_batch_prepare(lbm_s* b) {
  const int P = static_cast<int>(b->subs.size());
  std::vector<TcMaps> maps(P);
  std::vector<TcParams> prm(P);
  std::vector<int> start(P);
  int total = 0;
  for (int i = 0; i < P; ++i) {
    const TcPlan* t = b->subs[i]->tc;
    if (!t || !t->persist || t->prm.ksplit != 1 || t->elem != 2 || t->kparts != b->subs[0]->tc->kparts ||
        t->cparts != b->subs[0]->tc->cparts)
      return LBM_EINVAL;
    maps[i] = t->maps;
    prm[i] = t->prm;
    start[i] = total;
    total += t->prm.total_tiles;
  }
  if (dev_alloc(b, (void**)&b->batch_tc_maps, sizeof(TcMaps) * P) != cudaSuccess) return LBM_ENOMEM;
  if (dev_alloc(b, (void**)&b->batch_tc_prm, sizeof(TcParams) * P) != cudaSuccess) return LBM_ENOMEM;
  if (dev_alloc(b, (void**)&b->batch_tc_start, sizeof(int) * P) != cudaSuccess) return LBM_ENOMEM;
  if (cudaMemcpy(b->batch_tc_maps, maps.data(), sizeof(TcMaps) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->batch_tc_prm, prm.data(), sizeof(TcParams) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->batch_tc_start, start.data(), sizeof(int) * P, cudaMemcpyHostToDevice) != cudaSuccess)
    return LBM_ECUDA;
  b->batch_tc_blocks = total;
  return LBM_OK;
}

template <int KP>
cudaError_t launch_batch_kp(const lbm_s* b, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, frac_tc_persist_batch_kernel<2, KP>, (int)PCfg<2, PBN, KP>::SMEM);
      e != cudaSuccess)
    return e;
  const int grid = std::min(b->batch_tc_blocks, device_sms());  // one CTA per SM
  frac_tc_persist_batch_kernel<2, KP><<<grid, kPersistThreads, PCfg<2, PBN, KP>::SMEM, s>>>(
      static_cast<const TcMaps*>(b->batch_tc_maps), static_cast<const TcParams*>(b->batch_tc_prm), b->batch_tc_start,
      static_cast<int>(b->subs.size()), b->batch_tc_blocks, b->dev.flag);
  return cudaGetLastError();
}

cudaError_t launch_frac_tc_batch(const lbm_s* b, cudaStream_t s) {
  const TcPlan* t = b->subs[0]->tc;
  if (t->cparts == 3) return launch_batch_kp<6>(b, s);
  return t->kparts == 3 ? launch_batch_kp<3>(b, s) : launch_batch_kp<2>(b, s);
}

int tc_split_pitch(const lbm_s* h) { return h->tc ? h->tc->ldp : 0; }

bool encode_f32_map(void* map, int rank, void* base, const unsigned long long* dims,
                    const unsigned long long* strides_bytes, const unsigned int* box) {
  EncodeTiled enc = get_encoder();
  if (!enc || rank < 1 || rank > 5) return false;
  cuuint64_t d[5];
  cuuint64_t st[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = strides_bytes[i];
  }
  const CUresult r = enc(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, d, st, b, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_tma_store(const lbm_s* h) { return h->tc && h->tc->prm.tma_store; }

void tc_config(const lbm_s* h, int* bn, int* ks, int* persist) {
  const TcPlan* p = h->tc;
  *bn = p ? p->bn : 0;
  *ks = p ? p->prm.ksplit : 0;
  *persist = (p && p->persist) ? 1 : 0;
}

bool tc_one_wave(const lbm_s* h) {
  const TcPlan* p = h->tc;
  return p && (p->persist || (long long)p->prm.total_tiles * p->prm.ksplit <= device_sms());
}

void tc_set_pdl(lbm_s* h, bool on) {
  if (h->tc) h->tc->pdl = on;
}

cudaError_t launch_frac_tc(const lbm_s* h, cudaStream_t s) {
  const TcPlan* p = h->tc;
  if (!p) return cudaErrorNotSupported;
  if (p->kparts == 3) {  // five- and six-product bf16 forms: 64 or 128 columns, per tile or persistent (128)
    if (p->elem != 2 || p->bn == 256 || (p->persist && p->bn != PBN)) return cudaErrorInvalidConfiguration;
    if (p->cparts == 3) {
      if (p->persist) return launch_persist<2, PBN, 6>(p, s);
      return (p->bn == 64) ? launch_bn<2, 64, 6>(p, s) : launch_bn<2, 128, 6>(p, s);
    }
    if (p->persist) return launch_persist<2, PBN, 3>(p, s);
    return (p->bn == 64) ? launch_bn<2, 64, 3>(p, s) : launch_bn<2, 128, 3>(p, s);
  }
  if (p->persist) {
    if (p->bn == 256) return (p->elem == 2) ? launch_persist<2, 256>(p, s) : launch_persist<4, 256>(p, s);
    return (p->elem == 2) ? launch_persist<2, 128>(p, s) : launch_persist<4, 128>(p, s);
  }
  // 256-column tiles are chosen only when they alone fill the GPU: never split
  if (p->bn == 256 && p->prm.ksplit != 1) return cudaErrorInvalidConfiguration;
  if (p->elem == 2) {
    if (p->bn == 64) return launch_bn<2, 64>(p, s);
    return (p->bn == 128) ? launch_bn<2, 128>(p, s) : launch_kernel<2, 256, 1>(p, s);
  }
  if (p->bn == 64) return launch_bn<4, 64>(p, s);
  return (p->bn == 128) ? launch_bn<4, 128>(p, s) : launch_kernel<4, 256, 1>(p, s);
}

cudaError_t launch_split_T(const lbm_s* h, cudaStream_t s) {
  const TcPlan* p = h->tc;
  if (!p || p->elem != 4) return cudaSuccess;
  const int n0 = h->sp.n[0], n1 = h->sp.n[1], n2 = h->sp.n[2];
  const long long nodes = h->sp.nodes;
  // the operator's input along mu: C, or with g(x) G_mu = g_mu(x) C (the collide-stream
  // kernel's or launch_scale_fields' FP32 fields); the x operand is then G_0 at pitch ldp
  const float* C = static_cast<const float*>(h->dev.C);
  const float* G = static_cast<const float*>(h->fld.G);
  if (p->gvar) {
    long long b = (nodes + 255) / 256;
    const long long cap = 16LL * device_sms();
    if (b > cap) b = cap;
    split_C_kernel<4><<<(int)b, 256, 0, s>>>(G, h->dev.Chi, nullptr, nullptr, n0, n1, n2, p->ldp);
  }
  for (int mu = 1; mu < h->d; ++mu)
    split_T_kernel<<<dim3((n0 + 127) / 128, p->tg[mu], mu == 1 ? n2 : n1), 128, 0, s>>>(
        p->gvar ? G + mu * nodes : C, static_cast<float*>(p->ct_hi[mu]), n0, n1, n2, mu, p->tg[mu], p->tpx);
  return cudaGetLastError();
}

cudaError_t launch_split_T_step(const lbm_s* h, cudaStream_t s) {
  return cs_writes_T(h) ? cudaSuccess : launch_split_T(h, s);
}

// g(x) on the tensor cores: the bf16 forms keep operand parts of g_mu(x) C for every axis
// mu; tf32 takes its operands from the FP32 fields G_mu = g_mu(x) C (launch_split_T)
int tc_set_gfield(lbm_s* h, bool on) {
  TcPlan* p = h->tc;
  if (!p) return LBM_EINVAL;
  if (on == p->gvar) return LBM_OK;
  if (p->elem == 4) {  // tf32: the operands come from the FP32 fields G_mu (launch_split_T)
    p->gvar = on;
    return LBM_OK;
  }
  for (int mu = 0; mu < 3; ++mu)
    for (int k = 0; k < 3; ++k) {
      dev_free(h, p->gp[mu][k]);
      p->gp[mu][k] = nullptr;
    }
  p->gvar = false;
  if (on) {
    const size_t bytes = (size_t)p->ldp * h->sp.n[1] * h->sp.n[2] * p->elem;
    for (int mu = 0; mu < h->d; ++mu)
      for (int k = 0; k < p->cparts; ++k) {
        if (dev_alloc(h, &p->gp[mu][k], bytes) != cudaSuccess) return LBM_ENOMEM;
        if (cudaMemset(p->gp[mu][k], 0, bytes) != cudaSuccess) return LBM_ECUDA;
      }
    p->gvar = true;
  }
  return tc_replan(h, p->bn, p->prm.ksplit, p->persist ? 1 : 0);  // re-encodes the operand maps
}

cudaError_t launch_split_C(const lbm_s* h, cudaStream_t s) {
  const TcPlan* p = h->tc;
  if (!p) return cudaErrorNotSupported;
  long long b = (h->sp.nodes + 255) / 256;
  const long long cap = 16LL * device_sms();
  if (b > cap) b = cap;
  if (p->gvar && p->elem == 4) {  // tf32 with g(x): G = g C, then the operands from G
    cudaError_t e = launch_scale_fields(h, s);
    if (e != cudaSuccess) return e;
    return launch_split_T(h, s);
  }
  if (p->gvar) {
    GParts gp{};
    for (int mu = 0; mu < 3; ++mu)
      for (int k = 0; k < 3; ++k) gp.p[mu][k] = p->gp[mu][k];
    split_G_kernel<<<(int)b, 256, 0, s>>>(static_cast<const float*>(h->dev.C), static_cast<const float*>(h->fld.g), gp,
                                          h->d, p->cparts, h->sp.n[0], h->sp.n[1], h->sp.n[2], p->ldp);
    return cudaGetLastError();
  }
  if (p->elem == 2)
    split_C_kernel<2><<<(int)b, 256, 0, s>>>(static_cast<const float*>(h->dev.C), h->dev.Chi, h->dev.Clo,
                                             p->cparts == 3 ? h->dev.Cl2 : nullptr, h->sp.n[0], h->sp.n[1],
                                             h->sp.n[2], p->ldp);
  else
    split_C_kernel<4><<<(int)b, 256, 0, s>>>(static_cast<const float*>(h->dev.C), h->dev.Chi, h->dev.Clo, nullptr,
                                             h->sp.n[0], h->sp.n[1], h->sp.n[2], p->ldp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_split_T(h, s);
}

}  // namespace lbm
