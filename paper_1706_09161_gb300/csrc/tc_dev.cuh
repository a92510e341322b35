// Device-side building blocks of the tcgen05 split-precision fractional operator:
// plan structures, PTX wrappers (TMA, mbarrier, tcgen05), the per-k-block operand loads
// and MMAs.  Shared by the operator kernels and the fused small-problem step kernel.
// Section 2.4, Eq. (XXminus_discret): along every lattice line of axis mu,
// F_mu[n] = sum_l K_mu[n][l] C[l], a GEMM per axis over all lines.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdint>

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
  int ksplit;     // CTAs per output tile, each contracting a k-range into its own partial
  int tma_store;  // F rows are 16-byte aligned (n0 % 4 == 0): store tiles with TMA
  int early_trigger;  // the per-tile grid fits in one wave: release dependents after the prologue
  long long nodes;
  TcAxis ax[3];
  float* F;
  int* flag;
};

struct TcMaps {
  CUtensorMap c_hi[3], c_lo[3];  // C split; box per axis (x: B rows; y, z: MN-major A)
  CUtensorMap c_l2[3];           // third part of C (six-product bf16 form only)
  CUtensorMap k_hi[3], k_lo[3];  // K_mu split; box BK x 128 for the x axis (A), BK x BN else (B)
  CUtensorMap k_l2[3];           // third part of K_mu (five- and six-product bf16 forms)
  CUtensorMap f[3];              // F_mu (FP32), box 128 x (BN / ksplit) output rows
};

struct TcPlan {
  TcMaps maps;
  TcParams prm;
  int elem = 2;      // 2: bf16 parts, 4: tf32 parts
  int kparts = 2;    // parts of K_mu: 2 (three products) or 3 (bf16, five or six products)
  int cparts = 2;    // parts of C: 2, or 3 (bf16, six products)
  int bn = 64;
  bool persist = false;  // one CTA per SM walking the tile list (frac_tc_persist_kernel)
  bool pdl = false;      // launch with programmatic stream serialization (the handle's choice)
  int ldk[3] = {0, 0, 0};     // padded row pitch of K_mu's split parts (elements)
  size_t koff[3] = {0, 0, 0}; // offset of K_mu's split parts (elements)
  size_t f_elems = 0;         // capacity of the F buffer (floats)
  size_t smem = 0;
  int ldp = 0;       // padded x pitch of the C split arrays (elements)
  // tf32 only: C (FP32, split into tf32 hi + lo by the operator in shared memory) regrouped
  // so that axis mu (1: y, 2: z) is the contraction of a K-major operand, in groups of 4
  // along mu (16 bytes) with x next (pitch tpx):
  //   y copy  element (x, y, z) at ((z * tg[1] + y / 4) * tpx + x) * 4 + y % 4
  //   z copy  element (x, y, z) at ((z / 4 * n1 + y) * tpx + x) * 4 + z % 4
  // Entries past the end of an axis are zero.  A TMA box of (16 x, 4) x 8 x-blocks x 8
  // groups (256-byte rows) lands as the tensor cores' no-swizzle K-major layout (8-row x
  // 16-byte core matrices), and the collide-stream kernels write whole 16-byte groups of
  // consecutive x.
  void* ct_hi[3] = {nullptr, nullptr, nullptr};
  int tg[3] = {0, 0, 0};  // groups of 4 along axis mu: ceil(n_mu / 4)
  int tpx = 0;            // x pitch of the regrouped copies: n0 rounded up to 16
  // bf16 forms with g varying in space: the operand of axis mu is g_mu(x) C, split into
  // cparts parts gp[mu][k] (layout of the C split, pitch ldp); K_mu then carries no g
  bool gvar = false;
  void* gp[3][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
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

// Bounded wait on an mbarrier phase; false (and flag bit 2) after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag, long long limit_ns = kWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > (unsigned long long)limit_ns) {
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

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor, sm_100 descriptor version 1; layout 2 = 128-byte
// swizzle, 0 = no swizzle (8-row x 16-byte core matrices: lbo = stride between core
// matrices along K, sbo = stride between groups of 8 rows).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout = 2) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
  d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(layout) << 61;
  return d;
}

// Layout of the A operand (the 128-line side) in a ring stage
enum AMode : int {
  kAKSw128 = 0,  // K-major, 128-byte swizzle (x axis: K_x rows)
  kAMNSw128 = 1, // MN-major, 128-byte swizzle (bf16 y, z axes: the C panel, x contiguous)
  kAKGroup4 = 2  // K-major, no swizzle, [k/4][128 lines][4] (tf32 y, z axes: regrouped C)
};

template <int E>
__device__ __forceinline__ int a_mode(int mu) {
  return mu == 0 ? kAKSw128 : (E == 4 ? kAKGroup4 : kAMNSw128);
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

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Split forms, by KP: 2 = weights and C in two parts (hi*hi + hi*lo + lo*hi); 3 = the
// weights in three bf16 parts, C in two (five products); 6 = both in three bf16 parts
// (six products: every pair of parts whose orders sum to at most 2).
__host__ __device__ constexpr int k_parts(int KP) { return KP == 2 ? 2 : 3; }
__host__ __device__ constexpr int c_parts(int KP) { return KP == 6 ? 3 : 2; }

// E: operand bytes; BN: output columns per tile; KS: contraction split; KP: split form
// (above).  A ring stage holds k_parts(KP) slots of A (from st) and as many of B (from
// st + k_parts(KP) * A_BYTES); C fills two or three of its operand's slots.
template <int E, int BN, int KS = 1, int KP = 2>
struct Cfg {
  static constexpr int BK = 128 / E;                 // contraction elements per 128-byte row
  static constexpr int NP = k_parts(KP);             // operand slots per side
  static constexpr int STAGES = NP == 2 ? ((BN <= 64) ? 4 : (BN <= 128 ? 3 : 2)) : (BN <= 64 ? 3 : 2);
  static constexpr uint32_t A_BYTES = BM * 128;      // one operand part of A: 128 rows x 128 B
  static constexpr uint32_t B_BYTES = BN * 128;
  static constexpr uint32_t STAGE = NP * A_BYTES + NP * B_BYTES;
  // parts of C one k-block loads: bf16 c_parts(KP); tf32 one (C itself, split on chip)
  static constexpr int CL = E == 4 ? 1 : c_parts(KP);
  // bytes one k-block of axis mu loads: the weights in k_parts, C in CL parts
  __host__ __device__ static constexpr uint32_t tx_bytes(int mu) {
    return mu == 0 ? k_parts(KP) * A_BYTES + CL * B_BYTES : CL * A_BYTES + k_parts(KP) * B_BYTES;
  }
  static constexpr size_t RING = (size_t)STAGES * STAGE;
  static constexpr size_t SMEM = RING + 1024 /*align*/ + 256 /*barriers*/;
  // A, MN-major: E boxes of (128/E) lines x BK rows
  static constexpr uint32_t A_BOX_MN = BK * 128;
  static constexpr uint32_t IDESC_K = (1u << 4) | (Kind<E>::fmt << 7) | (Kind<E>::fmt << 10) |
                                      (static_cast<uint32_t>(BN >> 3) << 17) | (static_cast<uint32_t>(BM >> 4) << 24);
  static constexpr uint32_t IDESC_MN = IDESC_K | (1u << 15);
};

// Tile `cid` of a problem: axis mu, first x of the tile (m_in), outer coordinate
// (m_out: z for the x and y axes, y for the z axis) and first output column (ncol0).
struct TileAt {
  int mu, m_in, m_out, ncol0;
};

__device__ __forceinline__ TileAt decode_tile(const TcParams& P, int cid, int bn) {
  int mu = 0;
  while (mu + 1 < P.naxes && cid >= P.ax[mu + 1].tile_begin) ++mu;
  const TcAxis& ax = P.ax[mu];
  const int lt = cid - ax.tile_begin;
  const int mt = lt / ax.tiles_n, nt = lt % ax.tiles_n;
  return TileAt{mu, (mt % ax.msub) * BM, mt / ax.msub, nt * bn};
}

// TMA loads of one k-block (contraction offset k0) of tile `t` into ring stage `st`,
// completing on `bar` (whose expected byte count the caller has set).  The weight
// parts (K_mu, fixed for the whole run) and the concentration parts (C, written by the
// previous step) are issued separately, so the former can leave before the previous
// kernel has finished.
template <int E, int BN, int KP = 2>
__device__ __forceinline__ void load_stage_weights(const TcMaps& maps, const TileAt& t, int k0, uint8_t* st,
                                                   uint64_t* bar) {
  using G = Cfg<E, BN, 1, KP>;
  if (t.mu == 0) {
    // A = K_x rows n = m_in..
    tma_load_2d(st, &maps.k_hi[0], k0, t.m_in, bar);
    tma_load_2d(st + G::A_BYTES, &maps.k_lo[0], k0, t.m_in, bar);
    if (k_parts(KP) == 3) tma_load_2d(st + 2 * G::A_BYTES, &maps.k_l2[0], k0, t.m_in, bar);
  } else {
    // B = K_mu rows n = ncol0..
    uint8_t* b_hi = st + G::NP * G::A_BYTES;
    tma_load_2d(b_hi, &maps.k_hi[t.mu], k0, t.ncol0, bar);
    tma_load_2d(b_hi + G::B_BYTES, &maps.k_lo[t.mu], k0, t.ncol0, bar);
    if (k_parts(KP) == 3) tma_load_2d(b_hi + 2 * G::B_BYTES, &maps.k_l2[t.mu], k0, t.ncol0, bar);
  }
}

template <int E, int BN, int KP = 2>
__device__ __forceinline__ void load_stage_conc(const TcMaps& maps, const TileAt& t, int k0, uint8_t* st,
                                                uint64_t* bar) {
  using G = Cfg<E, BN, 1, KP>;
  uint8_t* a_hi = st;
  uint8_t* a_lo = st + G::A_BYTES;
  uint8_t* b_hi = st + G::NP * G::A_BYTES;
  uint8_t* b_lo = b_hi + G::B_BYTES;
  if (t.mu == 0) {
    // B = C rows y = ncol0.. at z = m_out (tf32: C itself into the hi slot)
    tma_load_3d(b_hi, &maps.c_hi[0], k0, t.ncol0, t.m_out, bar);
    if (E == 2) tma_load_3d(b_lo, &maps.c_lo[0], k0, t.ncol0, t.m_out, bar);
    if (c_parts(KP) == 3) tma_load_3d(b_lo + G::B_BYTES, &maps.c_l2[0], k0, t.ncol0, t.m_out, bar);
  } else if (E == 4) {
    // tf32: A = C regrouped (contraction in groups of 4) into the hi slot, 128 x-lines
    // (8 blocks of 16), BK / 4 groups: dims (64, x blocks, y groups or y, z or z groups)
    (void)a_lo;
    if (t.mu == 1) tma_load_4d(a_hi, &maps.c_hi[1], 0, t.m_in / 16, k0 / 4, t.m_out, bar);
    else tma_load_4d(a_hi, &maps.c_hi[2], 0, t.m_in / 16, t.m_out, k0 / 4, bar);
  } else {
    // bf16 parts: A = the C panel, MN-major (x contiguous), E boxes of 128/E lines
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int x = t.m_in + j * (128 / E);
      if (t.mu == 1) {
        tma_load_3d(a_hi + j * G::A_BOX_MN, &maps.c_hi[1], x, k0, t.m_out, bar);
        tma_load_3d(a_lo + j * G::A_BOX_MN, &maps.c_lo[1], x, k0, t.m_out, bar);
        if (c_parts(KP) == 3)
          tma_load_3d(a_lo + G::A_BYTES + j * G::A_BOX_MN, &maps.c_l2[1], x, k0, t.m_out, bar);
      } else {
        tma_load_3d(a_hi + j * G::A_BOX_MN, &maps.c_hi[2], x, t.m_out, k0, bar);
        tma_load_3d(a_lo + j * G::A_BOX_MN, &maps.c_lo[2], x, t.m_out, k0, bar);
        if (c_parts(KP) == 3)
          tma_load_3d(a_lo + G::A_BYTES + j * G::A_BOX_MN, &maps.c_l2[2], x, t.m_out, k0, bar);
      }
    }
  }
}

template <int E, int BN, int KP = 2>
__device__ __forceinline__ void load_stage(const TcMaps& maps, const TileAt& t, int k0, uint8_t* st, uint64_t* bar) {
  load_stage_weights<E, BN, KP>(maps, t, k0, st, bar);
  load_stage_conc<E, BN, KP>(maps, t, k0, st, bar);
}

// tf32 forms: C arrives in FP32 in the hi slot of its operand; before the MMAs the splitting
// warps (nthr threads, this one numbered tid) replace it by its tf32 rounding and write the
// rounding of the remainder to the lo slot, element by element, so the staged layout
// (swizzled rows or regrouped core matrices) is kept as it landed.  Rounding: to nearest,
// ties away from zero, on the magnitude bits (add half a unit of the 10-bit mantissa, clear
// the 13 bits below it; finite values); two integer operations per element.  The writes are
// made visible to the tensor cores' async proxy before the caller signals the MMA thread.
__device__ __forceinline__ float tc_tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <int E, int BN, int KP = 2>
__device__ __forceinline__ void split_stage_tf32(uint8_t* st, int mu, int tid, int nthr) {
  using G = Cfg<E, BN, 1, KP>;
  const uint32_t bytes = mu == 0 ? G::B_BYTES : G::A_BYTES;
  float4* hi = reinterpret_cast<float4*>(mu == 0 ? st + G::NP * G::A_BYTES : st);
  float4* lo = hi + bytes / 16;
  for (uint32_t i = tid; i < bytes / 16; i += nthr) {
    const float4 v = hi[i];
    float4 h, l;
    h.x = tc_tf32_rna(v.x); l.x = tc_tf32_rna(v.x - h.x);
    h.y = tc_tf32_rna(v.y); l.y = tc_tf32_rna(v.y - h.y);
    h.z = tc_tf32_rna(v.z); l.z = tc_tf32_rna(v.z - h.z);
    h.w = tc_tf32_rna(v.w); l.w = tc_tf32_rna(v.w - h.w);
    hi[i] = h;
    lo[i] = l;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The split products of one k-block from ring stage `st` into accumulator `d` (first =
// no previous contribution in d).  With KP = 2: hi*hi, hi*lo, lo*hi.  With KP = 3 (the
// weights in parts k1 + k2 + k3, C in c1 + c2) every product whose part orders sum to at
// most 2 that the parts allow: k1 c1, k1 c2, k2 c1, k2 c2, k3 c1; KP = 6 (C in c1 + c2 +
// c3 too) adds k1 c3.
//
// Accumulation chains: the k-steps of a CTA's contraction are numbered c = chain0 + kk
// (kk = 0..BK/UK-1 within this k-block) and k-step c accumulates into TMEM region c % nreg
// (BN columns each, from tmem); the first k-step of a region overwrites it.  The tensor
// cores round each accumulation at the accumulator's own scale, so the error of a long
// chain grows with its length (measured as a drift of the split forms over many time
// steps); short chains, added in FP32 by the epilogue, keep it at the FP32 level.
template <int E, int BN, int KP = 2>
__device__ __forceinline__ void mma_stage(uint32_t tmem, int chain0, int nreg, uint32_t st, int amode) {
  using G = Cfg<E, BN, 1, KP>;
  const uint32_t idesc = amode == kAMNSw128 ? G::IDESC_MN : G::IDESC_K;
  const uint32_t a_hi = st, a_lo = st + G::A_BYTES;
  const uint32_t b_hi = st + G::NP * G::A_BYTES, b_lo = b_hi + G::B_BYTES;
#pragma unroll
  for (int kk = 0; kk < G::BK / Kind<E>::UK; ++kk) {
    uint32_t a_off, a_lbo, a_sbo = 1024, a_lay = 2;
    if (amode == kAKSw128) {  // K-major A: advance within the 128-byte row
      a_off = kk * Kind<E>::UK * E;
      a_lbo = 16;
    } else if (amode == kAMNSw128) {  // MN-major A: advance by UK rows of 128 bytes
      a_off = kk * Kind<E>::UK * 128;
      a_lbo = G::A_BOX_MN;
    } else {  // grouped K-major A: 16-byte groups of K, 128 lines each (2 KB apart)
      constexpr uint32_t kGroup = BM * 16;
      a_off = kk * (Kind<E>::UK * E / 16) * kGroup;
      a_lbo = kGroup;
      a_sbo = 8 * 16;
      a_lay = 0;
    }
    const uint32_t b_off = kk * Kind<E>::UK * E;
    const uint64_t dah = smem_desc(a_hi + a_off, a_lbo, a_sbo, a_lay);
    const uint64_t dal = smem_desc(a_lo + a_off, a_lbo, a_sbo, a_lay);
    const uint64_t dbh = smem_desc(b_hi + b_off, 16, 1024);
    const uint64_t dbl = smem_desc(b_lo + b_off, 16, 1024);
    const int c = chain0 + kk;
    const uint32_t d = tmem + (uint32_t)((c % nreg) * BN);
    mma<E>(d, dah, dbh, idesc, c >= nreg ? 1u : 0u);
    mma<E>(d, dah, dbl, idesc, 1u);
    mma<E>(d, dal, dbh, idesc, 1u);
    if (KP >= 3) {
      mma<E>(d, dal, dbl, idesc, 1u);
      if (amode == kAKSw128) {  // A = the weights: k3 c1
        mma<E>(d, smem_desc(a_hi + 2 * G::A_BYTES + a_off, a_lbo, a_sbo, a_lay), dbh, idesc, 1u);
      } else {                  // B = the weights: c1 k3
        mma<E>(d, dah, smem_desc(b_hi + 2 * G::B_BYTES + b_off, 16, 1024), idesc, 1u);
      }
    }
    if (KP == 6) {
      if (amode == kAKSw128) {  // B = C: k1 c3
        mma<E>(d, dah, smem_desc(b_hi + 2 * G::B_BYTES + b_off, 16, 1024), idesc, 1u);
      } else {                  // A = C: c3 k1
        mma<E>(d, smem_desc(a_hi + 2 * G::A_BYTES + a_off, a_lbo, a_sbo, a_lay), dbh, idesc, 1u);
      }
    }
  }
}

__device__ __forceinline__ void named_sync128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// MMA k-steps per k-block (128-byte rows of UK-element MMAs): 4 for bf16 and tf32
template <int E>
__host__ __device__ constexpr int ksteps() {
  return (128 / E) / Kind<E>::UK;
}

// Accumulator regions of a CTA that runs `chains` k-steps into BN columns: the largest power
// of two up to 8 regions, 512 TMEM columns and the number of k-steps; the epilogue adds the
// regions in FP32, in order.  A tensor-core accumulator rounds each update at its own scale
// (measured: the error of the result grows with the number of MMAs into one accumulator),
// so shorter chains make the split forms more accurate at no extra MMA work.
__host__ __device__ constexpr int acc_regions(int chains, int bn) {
  int r = 1;
  while (r < 8 && 2 * r <= chains && 2 * r * bn <= 512) r *= 2;
  return r;
}

// One operator work item (tile item / KS, contraction slice item % KS) run by threads
// 0..127 (tid, warps 0-3) of a larger block: the per-tile kernel's pipeline with named
// barrier 1 in place of block barriers and a TMEM accumulator of BN columns allocated by
// the caller.  The item's partial tile goes to its slot of F by one TMA store (the plan
// must have tma_store set).  Every wait is bounded; a wait that gives up sets bit 2 of
// the flag and the item stores nothing.  `tmem` holds acc_regions(nkb k-steps, BN) * BN
// columns (at most 512; the caller allocates 512).
template <int E, int BN, int KS>
__device__ __forceinline__ void op_item(const TcMaps& maps, const TcParams& P, int item, uint8_t* smem, uint32_t tmem,
                                        int tid) {
  using G = Cfg<E, BN, KS>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + G::RING);
  uint64_t* empty = full + G::STAGES;
  uint64_t* done = empty + G::STAGES;
  const int warp = tid >> 5;
  const int cid = item / KS, rank = item % KS;
  const TileAt tl = decode_tile(P, cid, BN);
  const TcAxis& ax = P.ax[tl.mu];
  const int kb0 = rank * ax.kblocks / KS, kb1 = (rank + 1) * ax.kblocks / KS;
  const int nkb = kb1 - kb0;
  const int nreg = acc_regions(nkb * ksteps<E>(), BN);
  auto issue = [&](int i) {
    const int s = i % G::STAGES;
    mbar_expect_tx(&full[s], G::STAGE);
    load_stage<E, BN>(maps, tl, (kb0 + i) * G::BK, smem + (size_t)s * G::STAGE, &full[s]);
  };
  if (tid == 0) {
    for (int s = 0; s < G::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");  // operands written before the grid barrier
    for (int i = 0; i < G::STAGES && i < nkb; ++i) issue(i);
  }
  named_sync128();
  if (tid == 0) {
    for (int i = G::STAGES; i < nkb; ++i) {
      const int s = i % G::STAGES;
      if (!mbar_wait(&empty[s], ((i / G::STAGES) - 1) & 1, P.flag)) break;
      issue(i);
    }
  } else if (tid == 32) {
    const int amode = a_mode<E>(tl.mu);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % G::STAGES;
      if (!mbar_wait(&full[s], (i / G::STAGES) & 1, P.flag)) break;
      tc_fence_after();
      mma_stage<E, BN>(tmem, i * ksteps<E>(), nreg, smem_u32(smem + (size_t)s * G::STAGE), amode);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  const bool have = mbar_wait(done, 0, P.flag);
  tc_fence_after();
  float* tile = reinterpret_cast<float*>(smem);  // the ring is idle once `done` fired
  const int row = tid;                            // accumulator lane = x offset in the tile
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    float v[32], w[32];
    tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
    for (int r = 1; r < nreg; ++r) {
      tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + r * BN + c0, w);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += w[j];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[(c0 + j) * BM + row] = have ? v[j] : 0.0f;
  }
  tc_fence_before();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  named_sync128();
  if (tid == 0) {
    // every copy this item issued has landed (bounded) before the ring is reused
    for (int i = (nkb > G::STAGES ? nkb - G::STAGES : 0); i < nkb; ++i)
      mbar_wait(&full[i % G::STAGES], (i / G::STAGES) & 1, P.flag);
    if (have) {
      // the tile in 32-row chunks (the box of the F maps); chunks past the last output row
      // are not stored
      const int lim = (tl.mu == 0) ? P.n1 : P.ax[tl.mu].side;
      for (int c0 = 0; c0 < BN && tl.ncol0 + c0 < lim; c0 += 32) {
        int c1, c2;
        if (tl.mu == 2) {
          c1 = tl.m_out;
          c2 = tl.ncol0 + c0;
        } else {
          c1 = tl.ncol0 + c0;
          c2 = tl.m_out;
        }
        if (KS == 1)
          asm volatile(
              "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                  reinterpret_cast<uint64_t>(&maps.f[tl.mu])),
              "r"(tl.m_in), "r"(c1), "r"(c2), "r"(smem_u32(tile + c0 * BM))
              : "memory");
        else
          asm volatile(
              "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                  reinterpret_cast<uint64_t>(&maps.f[tl.mu])),
              "r"(tl.m_in), "r"(c1), "r"(c2), "r"(rank), "r"(smem_u32(tile + c0 * BM))
              : "memory");
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");  // F visible past the grid barrier
    }
  }
  named_sync128();
  if (tid == 0) {  // the barrier words may hold other data before the next item
    for (int s = 0; s < G::STAGES; ++s) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(done)) : "memory");
  }
}

}  // namespace
}  // namespace lbm
