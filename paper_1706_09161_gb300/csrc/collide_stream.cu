// Fused equilibrium + collision + streaming + Dirichlet walls + new concentration.
//
// One launch performs the rest of Algorithm 1's time step after the fractional terms:
//           equilibrium   feq = A + (C/e^2)(dt/dx) u_mu |e_mu w>            Eqs. (Feq), (CoeffA_FADE3D)
//           collision     f* = f - Omega (f - feq)                          Eqs. (LBE_Ket), (MRT-Coll)
//           streaming     f_i(x + e_i, t+dt) = f*_i(x, t)                   Eq. (Def_Translation)
//           walls         f_b = C_wall - sum_{i != b} f_i                   Eq. (Dirichlet_BC)
//           moment        C = <1|f>
// Populations are stored after streaming and boundary treatment, so a CTA
// collides its nodes plus a one-node ring and gathers ("pulls") each population
// from the node it came from; the ring's collisions are recomputed by the
// neighbouring CTAs and their loads mostly hit L2.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "lbm_internal.h"
#include "tc_dev.cuh"

namespace lbm {
namespace {

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
  int ksum;           // F holds ksum partial sums (split-K operator), added in order
  long long pstride;  // elements between partial sums
  real sfree[3];      // MRT rates of the free moments d+1..Q-1 (spatially varying coefficients)
};

// Coefficients that vary from node to node (lbm_set_fields), working precision, [k][node]:
//   coll: BGK 1/lambda(x); MRT the symmetric rate block R(x) = lambdabar(x)^-1 of the flux
//         moments, entries (00, 01, 11) in 2-D, (00, 01, 02, 11, 12, 22) in 3-D
//   advw: (dt/dx) u_mu(x) w_i / e^2, the advective factor of Eq. (Feq)
//   g:    g_mu(x); the kernel writes G_mu = g_mu(x) C(x), the operator's input along mu
//   src:  S(x) of a source S_c(x, t) = S(x) exp(rate t) (or null), added after the collision
//         as w_i S_c dt (Eq. LBE_Ket); cw: wall values C_w(x) of C_0(x, t) = C_w(x) exp(rate t)
//         (or null: the constant C_wall); tf: this launch's time factors, tf[0] =
//         exp(rate_S t) dt at the step's start t, tf[1] = exp(rate_w (t + dt)) at its end.
template <typename real>
struct FieldPtrs {
  const real* coll;
  const real* advw;
  const real* g;
  real* G;
  const real* src;
  const real* cw;
  const double* tf;
  // tensor-core forms with g(x): the operand parts of g_mu(x) C per axis ([mu][part], pitch
  // gldp), written in place of those of C
  void* gs[3][3];
  int gsplit;
  int gldp;
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
  k.ksum = sp.ksum;
  k.pstride = sp.pstride;
  for (int i = 0; i < 3; ++i) k.sfree[i] = static_cast<real>(sp.sfree[i]);
  return k;
}

// F_mu at `node`: the sum of the operator's ksum partial sums, in order
template <typename real>
__device__ __forceinline__ real frac_term(const KConst<real>& sp, const real* __restrict__ F, int mu, long long node) {
  const real* p = F + (long long)mu * sp.nodes + node;
  real acc = p[0];
  for (int s = 1; s < sp.ksum; ++s) acc += p[s * sp.pstride];
  return acc;
}

// The FP32 collision matrix of a block's problem in shared memory, rows padded to 8: the
// grouped (batched) 2-D kernels stage it here and read each row in 128-bit loads
// (collide_node<float, 2, true, KS = true>).
__shared__ float4 s_om_rows[kMaxQ][2];

// Equilibrium and collision of one node.  f: populations (in), fs: post-collision (out).
// KS: the matrix is read from s_om_rows (same products in the same order: bit-identical).
template <typename real, int D, bool MRT, bool KS = false>
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
      real acc;
      if constexpr (KS && sizeof(real) == 4) {
        const float4 a = s_om_rows[i][0];
        acc = a.x * dl[0];
        acc += a.y * dl[1];
        acc += a.z * dl[2];
        acc += a.w * dl[3];
        if constexpr (Q == 5) {
          acc += s_om_rows[i][1].x * dl[4];
        } else {
          const float4 b = s_om_rows[i][1];
          acc += b.x * dl[4];
          acc += b.y * dl[5];
          acc += b.z * dl[6];
        }
      } else {
        acc = sp.omega[i][0] * dl[0];
#pragma unroll
        for (int j = 1; j < Q; ++j) acc += sp.omega[i][j] * dl[j];
      }
      fs[i] = f[i] - acc;
    }
  }
}

// MRT change of basis, Eq. (MatrixD2): entry (i, q) of M for D2Q5 (D = 2) or D3Q7 (D = 3),
// and the squared norm of row i (the rows are orthogonal: M^-1 = M^T diag(1 / norm))
__host__ __device__ constexpr int mom(int D, int i, int q) {
  if (i == 0) return 1;
  if (i <= D) return q == 2 * i - 1 ? 1 : (q == 2 * i ? -1 : 0);  // flux moments
  if (D == 2) return i == 3 ? (q == 0 ? 4 : -1) : (q == 0 ? 0 : (q <= 2 ? 1 : -1));
  if (i == 4) return q == 0 ? 6 : -1;
  if (i == 5) return q == 0 ? 0 : (q <= 2 ? 2 : -1);
  return (q == 0 || q <= 2) ? 0 : (q <= 4 ? 1 : -1);
}
__host__ __device__ constexpr int mom_norm(int D, int i) {
  int n = 0;
  for (int q = 0; q < 2 * D + 1; ++q) n += mom(D, i, q) * mom(D, i, q);
  return n;
}
static_assert(mom_norm(2, 3) == 20 && mom_norm(3, 4) == 42 && mom_norm(3, 5) == 12 && mom_norm(3, 6) == 4,
              "moment rows of Eq. (MatrixD2)");

template <typename real, int D>
__device__ __forceinline__ void collide_moments(const KConst<real>& sp, const FieldPtrs<real>& fp, long long node,
                                                const real* f, const real* dl, real* fs);

// Equilibrium and collision of one node with coefficients of that node (FieldPtrs):
// Eq. (Feq) with u(x); BGK f* = f - (f - feq)/lambda(x); MRT in moment space
// f* = f - M^-1 Lambda(x) M (f - feq), Lambda(x) = diag(1, R(x), s_free) (Eqs. MRT-Coll,
// MatrixS, D_ab with lambda_{mu nu}(x)).
template <typename real, int D, bool MRT>
__device__ __forceinline__ void collide_node_field(const KConst<real>& sp, const FieldPtrs<real>& fp, long long node,
                                                   const real* f, const real* F, real* fs) {
  constexpr int Q = Lat<D>::Q;
  const long long nodes = sp.nodes;
  real C = f[0];
#pragma unroll
  for (int q = 1; q < Q; ++q) C += f[q];
  real sumF = F[0];
#pragma unroll
  for (int mu = 1; mu < D; ++mu) sumF += F[mu];
  real dl[Q];
  dl[0] = f[0] - (C - sp.w0 * sumF);
#pragma unroll
  for (int mu = 0; mu < D; ++mu) {
    const real a = sp.wi * F[mu];
    const real b = fp.advw[mu * nodes + node] * C;
    dl[2 * mu + 1] = f[2 * mu + 1] - (a + b);
    dl[2 * mu + 2] = f[2 * mu + 2] - (a - b);
  }
  if (!MRT) {
    const real om = fp.coll[node];
#pragma unroll
    for (int q = 0; q < Q; ++q) fs[q] = f[q] - om * dl[q];
  } else {
    collide_moments<real, D>(sp, fp, node, f, dl, fs);
  }
  if (fp.src) {  // |w> S_c(x, t) dt, Eq. (LBE_Ket)
    const real sv = fp.src[node] * static_cast<real>(fp.tf[0]);
    fs[0] += sp.w0 * sv;
#pragma unroll
    for (int q = 1; q < Q; ++q) fs[q] += sp.wi * sv;
  }
}

// MRT collision in moment space with the rates of the node: f* = f - M^-1 Lambda(x) M dl,
// dl = f - feq, Lambda(x) = diag(1, R(x), s_free) (Eqs. MRT-Coll, MatrixS, D_ab)
template <typename real, int D>
__device__ __forceinline__ void collide_moments(const KConst<real>& sp, const FieldPtrs<real>& fp, long long node,
                                                const real* f, const real* dl, real* fs) {
  constexpr int Q = Lat<D>::Q;
  const long long nodes = sp.nodes;
  real dm[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    real acc = static_cast<real>(mom(D, i, 0)) * dl[0];
#pragma unroll
    for (int q = 1; q < Q; ++q)
      if (mom(D, i, q) != 0) acc += static_cast<real>(mom(D, i, q)) * dl[q];
    dm[i] = acc;
  }
  real R[D][D];
  if (D == 2) {
    R[0][0] = fp.coll[node];
    R[0][1] = R[1][0] = fp.coll[nodes + node];
    R[1][1] = fp.coll[2 * nodes + node];
  } else {
    int k = 0;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) {
        R[a][b] = R[b][a] = fp.coll[k * nodes + node];
        ++k;
      }
  }
  real dmp[Q];
  dmp[0] = dm[0];  // conserved moment: rate 1, no effect (dm[0] = 0 up to rounding)
#pragma unroll
  for (int a = 0; a < D; ++a) {
    real acc = R[a][0] * dm[1];
#pragma unroll
    for (int b = 1; b < D; ++b) acc += R[a][b] * dm[1 + b];
    dmp[1 + a] = acc;
  }
#pragma unroll
  for (int k = D + 1; k < Q; ++k) dmp[k] = sp.sfree[k - D - 1] * dm[k];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    real acc = static_cast<real>(0);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (mom(D, i, q) != 0) acc += static_cast<real>(mom(D, i, q)) * dmp[i] / static_cast<real>(mom_norm(D, i));
    fs[q] = f[q] - acc;
  }
}

// Operands of the split-precision fractional operator, x-pitch ldp: bf16 parts C = hi + lo
// (SPLIT = 1) or hi + lo + lo2 (SPLIT = 3); tf32 (SPLIT = 2): C itself in hi (FP32).
struct SplitOut {
  void* hi;
  void* lo;
  int ldp;
  // tf32 on the TMA-fed marches: C again (FP32), regrouped along y (index 0) and z (index 1)
  // in groups of 4, the K-major operands of the y and z axes: element (x, y, z) at
  // thi[0][((z tg1 + y/4) tpx + x) 4 + y%4] and thi[1][((z/4 n1 + y) tpx + x) 4 + z%4]
  float* thi[2];
  int tg1;  // groups of 4 along y
  int tpx;  // x pitch (n0 rounded up to 16)
  void* lo2;  // bf16 with C in three parts (SPLIT = 3): the third part
};

// Per-problem entry of a grouped (batched) collide-stream launch.
struct BatchCS {
  CUtensorMap mf[2];  // 2-D members with n0 % 4 == 0: population windows (see march2_tma)
  CUtensorMap mF;     //   and fractional-term windows
  KConst<float> k;
  const float* f[2];  // population buffers; the launch's parity picks input and output
  const float* F;
  float* C;
  SplitOut so;
  int* flag;
  double* mpart;       // the problem's mass partials, one per block of it
  int bx, by, zchunk;  // blocks in x, y and the z chunk length (2-D: tile rows per block)
  int tma;             // the maps above are valid
};

// SPLIT: 1 = bf16 hi + lo, 3 = bf16 in three parts (each the rounding of what the previous
// ones left: the three add up to C exactly), 2 = tf32: C itself in FP32 (the operator splits
// it into tf32 hi + lo in shared memory)
template <int SPLIT, typename real>
__device__ __forceinline__ void write_split(const SplitOut& so, long long o, real C) {
  const float c = static_cast<float>(C);
  if (SPLIT == 1 || SPLIT == 3) {
    const __nv_bfloat16 h = __float2bfloat16_rn(c);
    const float r1 = c - __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(r1);
    static_cast<__nv_bfloat16*>(so.hi)[o] = h;
    static_cast<__nv_bfloat16*>(so.lo)[o] = l;
    if (SPLIT == 3) static_cast<__nv_bfloat16*>(so.lo2)[o] = __float2bfloat16_rn(r1 - __bfloat162float(l));
  } else if (SPLIT == 2) {
    static_cast<float*>(so.hi)[o] = c;
  }
}

// Mass of the new concentration (the moment C = <1|f> of Algorithm 1), as a by-product of the step.
// Every thread adds the C it wrote; each warp reduces its threads' sums in a fixed order
// (xor shuffles: every lane ends with the same value) and lane 0 stores the warp's partial
// at part[slot * kMassSlots + warp]; the handle adds the partials of the latest step in one
// small fixed-order FP64 pass when asked (lbm_mass).  FP32 concentrations are carried as an
// unevaluated sum hi + lo of two floats, combined by TwoSum (Knuth), which keeps the sum
// exact up to the rounding of lo (of order u^2 per addition, u = 2^-24) without FP64
// arithmetic, and the partial is stored as the pair (hi, lo) in the 8-byte slot: the final
// pass forms hi + lo in FP64.  The FP64 pipe is narrow (a warp instruction on it holds an
// SM sub-partition for tens of cycles): the FP64 per-node sum had cost 3-12% of the
// collide-stream kernels, and even the three FP64 operations per warp of a double partial
// kept that pipe 11% busy at the tail of the 512^2 kernel.  FP64 concentrations are summed
// and stored in FP64.  No block-wide barrier.  part may be null (no partial wanted).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

template <typename real>
struct MassAcc;
template <>
struct MassAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  __device__ __forceinline__ void store(double* slot) const { *slot = s; }
};
template <>
struct MassAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float t, e;
    two_sum(hi, x, t, e);
    hi = t;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
      float t, e;
      two_sum(hi, oh, t, e);
      hi = t;
      lo = __fadd_rn(__fadd_rn(lo, ol), e);
    }
  }
  // the pair (hi, lo) in the slot's 8 bytes; the final pass adds hi + lo in FP64
  __device__ __forceinline__ void store(double* slot) const { *reinterpret_cast<float2*>(slot) = make_float2(hi, lo); }
};

template <typename real>
__device__ __forceinline__ void block_mass(MassAcc<real>& macc, double* part, int slot) {
  macc.warp_reduce();
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  if ((tid & 31) == 0 && part) macc.store(part + (long long)slot * kMassSlots + (tid >> 5));
}

// Thread block: 16 warps own a 32 x 16 tile of nodes (one node per thread, full
// 128-byte rows), and three more warps collide the one-node ring the pull needs: the
// x-ring (16 + 16 nodes, one warp) and the rows below and above (one warp each).
// The block marches along z through a chunk of planes, colliding every plane once; the
// in-plane movers (e_1..e_4) of the current plane go through shared memory, the z
// movers (e_5, e_6) stay in registers (previous plane's f*_5, next plane's f*_6).
// In 2-D the block handles one plane.  Each node is loaded ~1.19 times per step.
constexpr int TX = 32, TY = 16, HALO_WARPS = 3;
static_assert(kMassSlots * 32 == TX * (TY + HALO_WARPS), "one mass partial per warp of a block");

template <typename real, int D, bool MRT, bool FLD = false, bool KS = false>
__device__ __forceinline__ void collide_at(const KConst<real>& sp, const real* __restrict__ f_in,
                                           const real* __restrict__ F, bool inside, long long node, real* fs,
                                           const FieldPtrs<real>& fp) {
  constexpr int Q = Lat<D>::Q;
  if (!inside) {
#pragma unroll
    for (int q = 0; q < Q; ++q) fs[q] = static_cast<real>(0);
    return;
  }
  const long long nodes = sp.nodes;
  real f[Q], Fv[D];
#pragma unroll
  for (int q = 0; q < Q; ++q) f[q] = f_in[q * nodes + node];
#pragma unroll
  for (int mu = 0; mu < D; ++mu) Fv[mu] = frac_term(sp, F, mu, node);
  if (FLD) collide_node_field<real, D, MRT>(sp, fp, node, f, Fv, fs);
  else collide_node<real, D, MRT, KS>(sp, f, Fv, fs);
}

// Asynchronous prefetch of the 2-D march (FP32): every thread copies the populations and
// fractional terms of its node in the next two tiles into its own column of a
// shared-memory ring (cp.async, 4 bytes each), so the loads of later tiles are in
// flight while the current one is processed.
constexpr int NT = TX * (TY + HALO_WARPS);
constexpr int PIPE_STAGES = 3;
constexpr int PIPE_VALS = 7;  // D2Q5: 5 populations + 2 fractional terms
constexpr int PIPE_SMEM = PIPE_STAGES * PIPE_VALS * NT * 4;

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}

// Programmatic dependent launch: let the next kernel of the stream be scheduled.  A grid
// that fits in one wave does this at block start (its dependents' prologues overlap it);
// a longer grid does it at block end, so that early dependents do not take SMs that its
// later waves need.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One block's column (tile bx, by; planes z0 .. z1-1) of one problem.
template <typename real, int D, bool MRT, int SPLIT, bool FLD = false, bool KS = false>
__device__ __forceinline__ void march_body(const KConst<real>& sp, const real* __restrict__ f_in,
                                           const real* __restrict__ F, real* __restrict__ f_out,
                                           real* __restrict__ C_out, int* __restrict__ flag, const SplitOut& so,
                                           int bx, int by, int z0, int z1, double* mpart, int mslot,
                                           const FieldPtrs<real> fp = FieldPtrs<real>{}) {
  constexpr int Q = Lat<D>::Q;
  // movers of the current plane on the tile plus ring: [buffer][mover 1..4][y+1][x+1]
  __shared__ real s_m[2][4][TY + 2][TX + 2];
  const int n0 = sp.n[0], n1 = sp.n[1], n2 = sp.n[2];
  const long long nodes = sp.nodes;
  const long long plane = (long long)n0 * n1;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int x0 = bx * TX, y0 = by * TY;

  // the node this thread collides every plane, and where its movers go
  int gx, gy, sx, sy;
  const bool owner = wy < TY;
  if (owner) {
    gx = x0 + lane;
    gy = y0 + wy;
  } else if (wy == TY) {  // x-ring: left column (lanes 0-15), right column (16-31)
    gx = (lane < 16) ? x0 - 1 : x0 + TX;
    gy = y0 + (lane & 15);
  } else {                // rows below (wy = TY+1) and above (wy = TY+2)
    gx = x0 + lane;
    gy = (wy == TY + 1) ? y0 - 1 : y0 + TY;
  }
  sx = gx - x0 + 1;
  sy = gy - y0 + 1;
  // programmatic dependent launch: the operator's F (and the previous step's f) must be
  // complete before any load
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool in_xy = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
  const long long col = gx + (long long)n0 * gy;
  bool bad = false;
  MassAcc<real> macc;

  real cur[Q], nxt[Q];
  real prev5 = static_cast<real>(0);
  if (owner) {
    if (D == 3) {
      real t[Q];
      collide_at<real, D, MRT, FLD, KS>(sp, f_in, F, in_xy && z0 > 0, col + (z0 - 1) * plane, t, fp);
      prev5 = t[5];
    }
    collide_at<real, D, MRT, FLD, KS>(sp, f_in, F, in_xy, col + z0 * plane, cur, fp);
  }
  int buf = 0;
  for (int z = z0; z < z1; ++z) {
    if (owner) {
      if (D == 3) collide_at<real, D, MRT, FLD, KS>(sp, f_in, F, in_xy && z + 1 < n2, col + (z + 1) * plane, nxt, fp);
      s_m[buf][0][sy][sx] = cur[1];
      s_m[buf][1][sy][sx] = cur[2];
      s_m[buf][2][sy][sx] = cur[3];
      s_m[buf][3][sy][sx] = cur[4];
    } else {
      real h[Q];
      collide_at<real, D, MRT, FLD, KS>(sp, f_in, F, in_xy, col + z * plane, h, fp);
      if (wy == TY) {
        if (lane < 16) s_m[buf][0][sy][sx] = h[1];  // moves +x into the tile
        else s_m[buf][1][sy][sx] = h[2];            // moves -x into the tile
      } else if (wy == TY + 1) {
        s_m[buf][2][sy][sx] = h[3];                 // moves +y into the tile
      } else {
        s_m[buf][3][sy][sx] = h[4];                 // moves -y into the tile
      }
    }
    __syncthreads();
    if (owner && in_xy) {
      real fv[Q];
      bool known[Q];
      fv[0] = cur[0];
      known[0] = true;
      known[1] = gx > 0;
      known[2] = gx + 1 < n0;
      known[3] = gy > 0;
      known[4] = gy + 1 < n1;
      fv[1] = s_m[buf][0][sy][sx - 1];
      fv[2] = s_m[buf][1][sy][sx + 1];
      fv[3] = s_m[buf][2][sy - 1][sx];
      fv[4] = s_m[buf][3][sy + 1][sx];
      if (D == 3) {
        known[5] = z > 0;
        known[6] = z + 1 < n2;
        fv[5] = prev5;
        fv[6] = nxt[6];
      }
      real sum_known = static_cast<real>(0);
      int n_unknown = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (known[q]) {
          sum_known += fv[q];
        } else {
          fv[q] = static_cast<real>(0);
          ++n_unknown;
        }
      }
      real C = sum_known;
      if (n_unknown > 0) {
        // Eq. (Dirichlet_BC); with k unknown populations each takes 1/k of the deficit; the
        // wall value varies with position and time when given (Section 2.5)
        real cwall = sp.C_wall;
        if (FLD && fp.cw) cwall = fp.cw[col + z * plane] * static_cast<real>(fp.tf[1]);
        const real fill = (cwall - sum_known) / static_cast<real>(n_unknown);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (!known[q]) fv[q] = fill;
        C = fv[0];
#pragma unroll
        for (int q = 1; q < Q; ++q) C += fv[q];
      }
      const long long node = col + z * plane;
#pragma unroll
      for (int q = 0; q < Q; ++q) f_out[q * nodes + node] = fv[q];
      C_out[node] = C;
      if (SPLIT && FLD && fp.gsplit) {
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
          SplitOut sm{};
          sm.hi = fp.gs[mu][0];
          sm.lo = fp.gs[mu][1];
          sm.lo2 = fp.gs[mu][2];
          write_split<SPLIT>(sm, ((long long)z * n1 + gy) * fp.gldp + gx, fp.g[mu * nodes + node] * C);
        }
      } else if (SPLIT) {
        write_split<SPLIT>(so, ((long long)z * n1 + gy) * so.ldp + gx, C);
      }
      if (FLD && fp.G) {  // the SIMT operator's inputs of the next step: g_mu(x) C, one field per axis
#pragma unroll
        for (int mu = 0; mu < D; ++mu) fp.G[mu * nodes + node] = fp.g[mu * nodes + node] * C;
      }
      bad |= !isfinite(C);
      macc.add(C);
    }
    if (owner && D == 3) {
      prev5 = cur[5];
#pragma unroll
      for (int q = 0; q < Q; ++q) cur[q] = nxt[q];
    }
    buf ^= 1;
  }
  // one flag update per warp at most
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1);
  block_mass(macc, mpart, mslot);
}

// movers of the current tile plus ring for the 2-D FP32 marches: [buffer][mover 1..4][y+1][x+1]
// (one array per kernel, whichever 2-D march it runs)
__shared__ float s_m2[2][4][TY + 2][TX + 2];

// 2-D FP32: the block walks `ychunk` consecutive 32 x 16 tiles up the y axis (tile
// rows tr0 .. tr0 + ychunk - 1 of column bx), each thread prefetching its node of the
// next two tiles through the cp.async ring while the current tile is collided.  The
// per-tile work is that of march_body with one plane.
template <bool MRT, int SPLIT, bool KS = false>
__device__ __forceinline__ void march2_pipe(const KConst<float>& sp, const float* __restrict__ f_in,
                                            const float* __restrict__ F, float* __restrict__ f_out,
                                            float* __restrict__ C_out, int* __restrict__ flag, const SplitOut& so,
                                            int ychunk, int bx, int byc, float* stage, double* mpart, int mslot) {
  constexpr int D = 2, Q = 5;
  auto& s_m = s_m2;
  const int n0 = sp.n[0], n1 = sp.n[1];
  const long long nodes = sp.nodes;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int tid = wy * TX + lane;
  const int tr0 = byc * ychunk;
  const int tr1 = min(tr0 + ychunk, (n1 + TY - 1) / TY);
  // this thread's node relative to the tile origin: owners, x-ring, rows below / above
  const bool owner = wy < TY;
  int dx, dy;
  if (owner) {
    dx = lane;
    dy = wy;
  } else if (wy == TY) {
    dx = (lane < 16) ? -1 : TX;
    dy = lane & 15;
  } else {
    dx = lane;
    dy = (wy == TY + 1) ? -1 : TY;
  }
  const int gx = bx * TX + dx;
  const int sx = dx + 1, sy = dy + 1;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool in_x = gx >= 0 && gx < n0;
  auto issue = [&](int tr, int slot) {
    const int gy = tr * TY + dy;
    if (in_x && gy >= 0 && gy < n1) {
      const long long node = gx + (long long)n0 * gy;
      float* st = stage + (size_t)slot * PIPE_VALS * NT + tid;
#pragma unroll
      for (int q = 0; q < Q; ++q) cp_async4(st + q * NT, f_in + q * nodes + node);
      if (sp.ksum == 1) {
#pragma unroll
        for (int mu = 0; mu < D; ++mu) cp_async4(st + (Q + mu) * NT, F + mu * nodes + node);
      }
    }
    cp_async_commit();
  };
  issue(tr0, 0);
  if (tr0 + 1 < tr1) issue(tr0 + 1, 1); else cp_async_commit();
  bool bad = false;
  MassAcc<float> macc;
  int buf = 0;
  for (int tr = tr0; tr < tr1; ++tr) {
    const int slot = (tr - tr0) % PIPE_STAGES;
    if (tr + 2 < tr1) issue(tr + 2, (tr - tr0 + 2) % PIPE_STAGES); else cp_async_commit();
    cp_async_wait<2>();  // this thread's copies for tile row tr have landed
    const int gy = tr * TY + dy;
    const bool inside = in_x && gy >= 0 && gy < n1;
    float fs[Q];
    if (inside) {
      const float* st = stage + (size_t)slot * PIPE_VALS * NT + tid;
      float fv[Q], Fv[D];
#pragma unroll
      for (int q = 0; q < Q; ++q) fv[q] = st[q * NT];
      if (sp.ksum == 1) {
#pragma unroll
        for (int mu = 0; mu < D; ++mu) Fv[mu] = st[(Q + mu) * NT];
      } else {  // split-K partials: summed here, in order
#pragma unroll
        for (int mu = 0; mu < D; ++mu) Fv[mu] = frac_term(sp, F, mu, gx + (long long)n0 * gy);
      }
      collide_node<float, D, MRT, KS>(sp, fv, Fv, fs);
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) fs[q] = 0.f;
    }
    if (owner) {
      s_m[buf][0][sy][sx] = fs[1];
      s_m[buf][1][sy][sx] = fs[2];
      s_m[buf][2][sy][sx] = fs[3];
      s_m[buf][3][sy][sx] = fs[4];
    } else if (wy == TY) {
      if (lane < 16) s_m[buf][0][sy][sx] = fs[1];  // moves +x into the tile
      else s_m[buf][1][sy][sx] = fs[2];            // moves -x into the tile
    } else if (wy == TY + 1) {
      s_m[buf][2][sy][sx] = fs[3];                 // moves +y into the tile
    } else {
      s_m[buf][3][sy][sx] = fs[4];                 // moves -y into the tile
    }
    __syncthreads();
    if (owner && inside) {
      float fv[Q];
      bool known[Q];
      fv[0] = fs[0];
      known[0] = true;
      known[1] = gx > 0;
      known[2] = gx + 1 < n0;
      known[3] = gy > 0;
      known[4] = gy + 1 < n1;
      fv[1] = s_m[buf][0][sy][sx - 1];
      fv[2] = s_m[buf][1][sy][sx + 1];
      fv[3] = s_m[buf][2][sy - 1][sx];
      fv[4] = s_m[buf][3][sy + 1][sx];
      float sum_known = 0.f;
      int n_unknown = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (known[q]) {
          sum_known += fv[q];
        } else {
          fv[q] = 0.f;
          ++n_unknown;
        }
      }
      float C = sum_known;
      if (n_unknown > 0) {
        // Eq. (Dirichlet_BC); with k unknown populations each takes 1/k of the deficit
        const float fill = (sp.C_wall - sum_known) / static_cast<float>(n_unknown);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (!known[q]) fv[q] = fill;
        C = fv[0];
#pragma unroll
        for (int q = 1; q < Q; ++q) C += fv[q];
      }
      const long long node = gx + (long long)n0 * gy;
#pragma unroll
      for (int q = 0; q < Q; ++q) f_out[q * nodes + node] = fv[q];
      C_out[node] = C;
      if (SPLIT) write_split<SPLIT>(so, (long long)gy * so.ldp + gx, C);
      bad |= !isfinite(C);
      macc.add(C);
    }
    buf ^= 1;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1);
  block_mass(macc, mpart, mslot);
}

// linear index of this block in its grid (the slot of its mass partial)
__device__ __forceinline__ int block_linear() {
  return static_cast<int>(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

template <bool MRT, int SPLIT>
__global__ void __launch_bounds__(TX*(TY + HALO_WARPS), 2)
collide_stream_march2_kernel(const KConst<float> sp, const float* __restrict__ f_in, const float* __restrict__ F,
                             float* __restrict__ f_out, float* __restrict__ C_out, int* __restrict__ flag,
                             SplitOut so, int ychunk, int early, double* mpart) {
  extern __shared__ __align__(16) float pipe_stage[];
  if (early) pdl_trigger();
  march2_pipe<MRT, SPLIT>(sp, f_in, F, f_out, C_out, flag, so, ychunk, blockIdx.x, blockIdx.y, pipe_stage, mpart,
                          block_linear());
  if (!early) pdl_trigger();
}

template <typename real, int D, bool MRT, int SPLIT, bool FLD = false>
__global__ void __launch_bounds__(TX*(TY + HALO_WARPS), 2)
collide_stream_march_kernel(const KConst<real> sp, const real* __restrict__ f_in, const real* __restrict__ F,
                            real* __restrict__ f_out, real* __restrict__ C_out, int* __restrict__ flag, SplitOut so,
                            int nz, int early, double* mpart, const FieldPtrs<real> fp = FieldPtrs<real>{}) {
  // z chunk blockIdx.z of nz (boundaries bz * n2 / nz): concurrent blocks march the same
  // z window, so the ring loads of neighbouring columns hit L2
  const int n2 = sp.n[2];
  const int bz = blockIdx.z;
  const int z0 = static_cast<int>((long long)bz * n2 / nz), z1 = static_cast<int>((long long)(bz + 1) * n2 / nz);
  if (early) pdl_trigger();
  march_body<real, D, MRT, SPLIT, FLD>(sp, f_in, F, f_out, C_out, flag, so, blockIdx.x, blockIdx.y, z0, z1, mpart,
                                       block_linear(), fp);
  if (!early) pdl_trigger();
}

// ---------------------------------------------------------------------------- TMA-fed 3-D march
// FP32 forms with n0 % 4 == 0: per plane, one thread loads the block's 40 x 18 window of
// all Q populations and all d fractional terms (tile, one-node ring, x aligned down to a
// 16-byte boundary) with two 4-D TMA box loads into a 3-stage shared-memory ring, two
// planes ahead of the plane being collided; every thread then reads its node (owners)
// or ring node (the three halo warps) from shared memory.  Nodes outside the domain
// arrive as zeros (TMA out-of-bounds fill), which the collision maps to zero movers,
// exactly as the plain march treats them.  The march itself (movers through shared
// memory, z movers in registers, walls, moment, split) is that of march_body.
constexpr int TW = TX + 8, TH = TY + 2;  // staged window: x from x0 - 4, y from y0 - 1
constexpr int TCP = TX;  // row pitch of the tf32 C ring
constexpr int TMA_STAGES = 3;
constexpr uint32_t TMA_F_BYTES = 7u * TH * TW * 4;   // D3Q7 populations
constexpr uint32_t TMA_FF_BYTES = 3u * TH * TW * 4;  // fractional terms
constexpr uint32_t TMA_TX = TMA_F_BYTES + TMA_FF_BYTES;  // bytes landing per plane
constexpr uint32_t TMA_FF_OFF = (TMA_F_BYTES + 127) / 128 * 128;  // 128-byte aligned box starts
constexpr uint32_t TMA_STAGE = (TMA_FF_OFF + TMA_FF_BYTES + 127) / 128 * 128;
constexpr size_t TMA_SMEM = (size_t)TMA_STAGES * TMA_STAGE + 128 /*align*/ + 64 /*barriers*/;
constexpr long long kTmaWaitNs = 2000000000LL;

struct CsPlan {
  CUtensorMap f[2];  // populations, dims (n0, n1, n2, Q), box (TW, TH, 1, Q)
  CUtensorMap F;     // fractional terms, dims (n0, n1, n2, d), box (TW, TH, 1, d)
};

__device__ __forceinline__ uint32_t cs_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool cs_mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(cs_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false (and bit 2 of the flag) after kTmaWaitNs of %globaltimer
__device__ __forceinline__ bool cs_mbar_wait(uint64_t* bar, uint32_t parity, int* flag) {
  if (cs_mbar_try(bar, parity)) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (cs_mbar_try(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > (unsigned long long)kTmaWaitNs) {
      atomicOr(flag, 2);
      return false;
    }
  }
}

__device__ __forceinline__ void cs_tma_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(cs_smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(cs_smem_u32(bar))
      : "memory");
}

template <bool MRT, int SPLIT>
__global__ void __launch_bounds__(TX*(TY + HALO_WARPS), 2)
collide_stream_tma3_kernel(const KConst<float> sp, const __grid_constant__ CUtensorMap map_f,
                           const __grid_constant__ CUtensorMap map_F, float* __restrict__ f_out,
                           float* __restrict__ C_out, int* __restrict__ flag, SplitOut so, int nz, int early,
                           double* mpart) {
  constexpr int D = 3, Q = 7;
  extern __shared__ uint8_t cs_raw[];
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(cs_raw) + 127) & ~uintptr_t(127));
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)TMA_STAGES * TMA_STAGE);
  __shared__ float s_m[2][4][TY + 2][TX + 2];
  // tf32: C of the last four planes (slot z & 3), the source of the regrouped split
  __shared__ float s_c[SPLIT == 2 ? 4 * TY * TCP : 1];
  const bool wT = SPLIT == 2 && so.thi[0] != nullptr;
  const int n0 = sp.n[0], n1 = sp.n[1], n2 = sp.n[2];
  const long long nodes = sp.nodes;
  const long long plane = (long long)n0 * n1;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int tid = wy * TX + lane;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int bz = blockIdx.z;
  const int z0 = static_cast<int>((long long)bz * n2 / nz), z1 = static_cast<int>((long long)(bz + 1) * n2 / nz);
  if (early) pdl_trigger();

  int gx, gy, sx, sy;
  const bool owner = wy < TY;
  if (owner) {
    gx = x0 + lane;
    gy = y0 + wy;
  } else if (wy == TY) {
    gx = (lane < 16) ? x0 - 1 : x0 + TX;
    gy = y0 + (lane & 15);
  } else {
    gx = x0 + lane;
    gy = (wy == TY + 1) ? y0 - 1 : y0 + TY;
  }
  sx = gx - x0 + 1;
  sy = gy - y0 + 1;
  const int lx = gx - (x0 - 4), ly = gy - (y0 - 1);  // position in the staged window
  const bool in_xy = gx >= 0 && gx < n0 && gy >= 0 && gy < n1;
  const long long col = gx + (long long)n0 * gy;

  // plane p lives in stage (p - z0 + 1) % 3; its k-th use of that stage completes phase k
  auto stage_of = [&](int p) { return (p - z0 + 1) % TMA_STAGES; };
  auto parity_of = [&](int p) { return static_cast<uint32_t>(((p - z0 + 1) / TMA_STAGES) & 1); };
  auto issue = [&](int p) {
    const int s = stage_of(p);
    uint8_t* st = ring + (size_t)s * TMA_STAGE;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cs_smem_u32(&full[s])),
                 "r"(TMA_TX)
                 : "memory");
    cs_tma_4d(st, &map_f, x0 - 4, y0 - 1, p, 0, &full[s]);
    cs_tma_4d(st + TMA_FF_OFF, &map_F, x0 - 4, y0 - 1, p, 0, &full[s]);
  };
  auto collide_staged = [&](int p, float* fs) {
    cs_mbar_wait(&full[stage_of(p)], parity_of(p), flag);
    const float* st = reinterpret_cast<const float*>(ring + (size_t)stage_of(p) * TMA_STAGE);
    float fv[Q], Fv[D];
#pragma unroll
    for (int q = 0; q < Q; ++q) fv[q] = st[(q * TH + ly) * TW + lx];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) Fv[mu] = st[TMA_FF_OFF / 4 + (mu * TH + ly) * TW + lx];
    collide_node<float, D, MRT>(sp, fv, Fv, fs);
  };

  // tf32: planes (ge & ~3 or z0) .. ge of the ring to the regrouped copies.  y copy:
  // owner warp (plane ge & ~3 + (wy & 3), y group wy >> 2) writes 32 x 16-byte groups
  // (512 contiguous bytes); z copy: each owner writes its own column's z group.
  auto flush_T = [&](int ge) {
    const int gs = max(ge & ~3, z0), cnt = ge - gs + 1;
    const int zz = (ge & ~3) + (wy & 3), yq = 4 * (wy >> 2);
    if (zz >= gs && zz <= ge && gx < n0 && y0 + yq < n1) {
      const float* r = &s_c[((zz & 3) * TY + yq) * TCP + lane];
      const long long o = (((long long)zz * so.tg1 + ((y0 + yq) >> 2)) * so.tpx + gx) * 4;
      *reinterpret_cast<float4*>(so.thi[0] + o) = make_float4(r[0], r[TCP], r[2 * TCP], r[3 * TCP]);
    }
    if (in_xy) {
      const long long o = (((long long)(gs >> 2) * n1 + gy) * so.tpx + gx) * 4 + (gs & 3);
      if (cnt == 4) {
        *reinterpret_cast<float4*>(so.thi[1] + o) =
            make_float4(s_c[(0 * TY + wy) * TCP + lane], s_c[(1 * TY + wy) * TCP + lane],
                        s_c[(2 * TY + wy) * TCP + lane], s_c[(3 * TY + wy) * TCP + lane]);
      } else {
        for (int k = 0; k < cnt; ++k) so.thi[1][o + k] = s_c[(((gs + k) & 3) * TY + wy) * TCP + lane];
      }
    }
  };

  if (tid == 0) {
    for (int s = 0; s < TMA_STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cs_smem_u32(&full[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // programmatic dependent launch: f and F come from the previous kernels
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tid == 0) {
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);  // z0 + 1 <= z1: needed by the owners' first iteration
  }
  bool bad = false;
  MassAcc<float> macc;
  float cur[Q], nxt[Q];
  float prev5 = 0.f;
  if (owner) {
    float t[Q];
    collide_staged(z0 - 1, t);
    prev5 = t[5];
    collide_staged(z0, cur);
  }
  __syncthreads();  // plane z0 - 1 is read: its stage takes plane z0 + 2
  if (tid == 0 && z0 + 2 <= z1) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(z0 + 2);
  }
  int buf = 0;
  for (int z = z0; z < z1; ++z) {
    if (owner) {
      collide_staged(z + 1, nxt);
      s_m[buf][0][sy][sx] = cur[1];
      s_m[buf][1][sy][sx] = cur[2];
      s_m[buf][2][sy][sx] = cur[3];
      s_m[buf][3][sy][sx] = cur[4];
    } else {
      float h[Q];
      collide_staged(z, h);
      if (wy == TY) {
        if (lane < 16) s_m[buf][0][sy][sx] = h[1];  // moves +x into the tile
        else s_m[buf][1][sy][sx] = h[2];            // moves -x into the tile
      } else if (wy == TY + 1) {
        s_m[buf][2][sy][sx] = h[3];                 // moves +y into the tile
      } else {
        s_m[buf][3][sy][sx] = h[4];                 // moves -y into the tile
      }
    }
    __syncthreads();
    // plane z is read by everyone: its stage takes plane z + 3
    if (tid == 0 && z + 3 <= z1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(z + 3);
    }
    if (SPLIT == 2 && wT && z > z0 && ((z - 1) & 3) == 3) {
      if (owner) flush_T(z - 1);
      __syncthreads();  // slot z & 3 is rewritten below
    }
    float Cn = 0.f;
    if (owner && in_xy) {
      float fv[Q];
      bool known[Q];
      fv[0] = cur[0];
      known[0] = true;
      known[1] = gx > 0;
      known[2] = gx + 1 < n0;
      known[3] = gy > 0;
      known[4] = gy + 1 < n1;
      known[5] = z > 0;
      known[6] = z + 1 < n2;
      fv[1] = s_m[buf][0][sy][sx - 1];
      fv[2] = s_m[buf][1][sy][sx + 1];
      fv[3] = s_m[buf][2][sy - 1][sx];
      fv[4] = s_m[buf][3][sy + 1][sx];
      fv[5] = prev5;
      fv[6] = nxt[6];
      float sum_known = 0.f;
      int n_unknown = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (known[q]) {
          sum_known += fv[q];
        } else {
          fv[q] = 0.f;
          ++n_unknown;
        }
      }
      float C = sum_known;
      if (n_unknown > 0) {
        // Eq. (Dirichlet_BC); with k unknown populations each takes 1/k of the deficit
        const float fill = (sp.C_wall - sum_known) / static_cast<float>(n_unknown);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (!known[q]) fv[q] = fill;
        C = fv[0];
#pragma unroll
        for (int q = 1; q < Q; ++q) C += fv[q];
      }
      const long long node = col + z * plane;
#pragma unroll
      for (int q = 0; q < Q; ++q) f_out[q * nodes + node] = fv[q];
      C_out[node] = C;
      if (SPLIT) write_split<SPLIT>(so, ((long long)z * n1 + gy) * so.ldp + gx, C);
      bad |= !isfinite(C);
      macc.add(C);
      Cn = C;
    }
    if (owner) {
      if (SPLIT == 2 && wT) s_c[((z & 3) * TY + wy) * TCP + lane] = Cn;  // zero outside the domain
      prev5 = cur[5];
#pragma unroll
      for (int q = 0; q < Q; ++q) cur[q] = nxt[q];
    }
    buf ^= 1;
  }
  if (SPLIT == 2 && wT) {
    __syncthreads();
    if (owner) flush_T(z1 - 1);
  }
  // every issued plane (up to z1) was waited for by the owners; after a timeout make sure
  // no copy is still in flight into this block's shared memory before it exits
  if (tid == 0)
    for (int p = (z1 - 2 > z0 - 1 ? z1 - 2 : z0 - 1); p <= z1; ++p) cs_mbar_wait(&full[stage_of(p)], parity_of(p), flag);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1);
  block_mass(macc, mpart, block_linear());
  if (!early) pdl_trigger();
}

// ---------------------------------------------------------------------------- TMA-fed 2-D march
// FP32 forms with n0 % 4 == 0: the block walks `ychunk` tiles up y; per tile one thread
// loads the 40 x 18 window of the 5 populations and the 2 fractional terms with two 3-D
// TMA box loads into a 3-stage ring, two tiles ahead.  Otherwise as march2_pipe.
constexpr uint32_t TMA2_F_BYTES = 5u * TH * TW * 4;
constexpr uint32_t TMA2_FF_BYTES = 2u * TH * TW * 4;
constexpr uint32_t TMA2_TX = TMA2_F_BYTES + TMA2_FF_BYTES;
constexpr uint32_t TMA2_FF_OFF = (TMA2_F_BYTES + 127) / 128 * 128;
constexpr uint32_t TMA2_STAGE = (TMA2_FF_OFF + TMA2_FF_BYTES + 127) / 128 * 128;
constexpr size_t TMA2_SMEM = (size_t)TMA_STAGES * TMA2_STAGE + 128 /*align*/ + 64 /*barriers*/;
// with ks split-K partial sums the fractional-term window holds 2 ks planes; two stages
// then (the ring must leave room for two blocks per SM up to ks = 4)
__host__ __device__ constexpr uint32_t tma2_ff_bytes(int ks) { return 2u * ks * TH * TW * 4; }
__host__ __device__ constexpr uint32_t tma2_stage(int ks) {
  return (TMA2_FF_OFF + tma2_ff_bytes(ks) + 127) / 128 * 128;
}
__host__ __device__ constexpr int tma2_nst(int ks) { return ks > 1 ? 2 : TMA_STAGES; }
__host__ __device__ constexpr size_t tma2_smem(int ks) {
  return (size_t)tma2_nst(ks) * tma2_stage(ks) + 128 /*align*/ + 64 /*barriers*/;
}

__device__ __forceinline__ void cs_tma_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(cs_smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(cs_smem_u32(bar))
      : "memory");
}

// tf32: C of the last two tile rows (slot t & 1), the source of the y-contiguous split
__shared__ float s_c2[2 * TY * TCP];

template <bool MRT, int SPLIT, bool KS = false>
__device__ __forceinline__ void march2_tma(const KConst<float>& sp, const CUtensorMap* map_f,
                                           const CUtensorMap* map_F, float* __restrict__ f_out,
                                           float* __restrict__ C_out, int* __restrict__ flag, const SplitOut& so,
                                           int ychunk, int bx, int byc, uint8_t* raw, double* mpart, int mslot) {
  constexpr int D = 2, Q = 5;
  auto& s_m = s_m2;
  float* s_c = nullptr;
  if constexpr (SPLIT == 2) s_c = s_c2;
  const bool wT = SPLIT == 2 && so.thi[0] != nullptr;
  uint8_t* ring = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
  const int ks = sp.ksum;
  const int nst = tma2_nst(ks);
  const uint32_t stg = tma2_stage(ks);
  const uint32_t tx = TMA2_F_BYTES + tma2_ff_bytes(ks);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)nst * stg);
  const int n0 = sp.n[0], n1 = sp.n[1];
  const long long nodes = sp.nodes;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int tid = wy * TX + lane;
  const int x0 = bx * TX;
  const int tr0 = byc * ychunk;
  const int tr1 = min(tr0 + ychunk, (n1 + TY - 1) / TY);
  const bool owner = wy < TY;
  int dx, dy;
  if (owner) {
    dx = lane;
    dy = wy;
  } else if (wy == TY) {
    dx = (lane < 16) ? -1 : TX;
    dy = lane & 15;
  } else {
    dx = lane;
    dy = (wy == TY + 1) ? -1 : TY;
  }
  const int gx = x0 + dx;
  const int sx = dx + 1, sy = dy + 1;
  const int lx = dx + 4, ly = dy + 1;  // position in the staged window
  const bool in_x = gx >= 0 && gx < n0;
  auto stage_of = [&](int t) { return (t - tr0) % nst; };
  auto parity_of = [&](int t) { return static_cast<uint32_t>(((t - tr0) / nst) & 1); };
  // tile row t to the y copy (element (x, y) at thi[0][(y/4 tpx + x) 4 + y%4]): warp w < 4
  // writes y group 4t + w for the tile's 32 x (512 contiguous bytes)
  auto flush_T = [&](int t) {
    const int xi = lane, yq = 4 * wy;
    if (wy < 4 && x0 + xi < n0 && t * TY + yq < n1) {
      const float* r = &s_c[((t & 1) * TY + yq) * TCP + xi];
      const long long o = ((long long)((t * TY + yq) >> 2) * so.tpx + x0 + xi) * 4;
      *reinterpret_cast<float4*>(so.thi[0] + o) = make_float4(r[0], r[TCP], r[2 * TCP], r[3 * TCP]);
    }
  };
  auto issue = [&](int t) {
    const int s = stage_of(t);
    uint8_t* st = ring + (size_t)s * stg;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cs_smem_u32(&full[s])), "r"(tx)
                 : "memory");
    cs_tma_3d(st, map_f, x0 - 4, t * TY - 1, 0, &full[s]);
    cs_tma_3d(st + TMA2_FF_OFF, map_F, x0 - 4, t * TY - 1, 0, &full[s]);
  };
  if (tid == 0) {
    for (int s = 0; s < nst; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cs_smem_u32(&full[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("griddepcontrol.wait;" ::: "memory");  // f and F come from the previous kernels
  if (tid == 0)
    for (int t = tr0; t < tr1 && t < tr0 + nst; ++t) issue(t);
  bool bad = false;
  MassAcc<float> macc;
  int buf = 0;
  for (int tr = tr0; tr < tr1; ++tr) {
    cs_mbar_wait(&full[stage_of(tr)], parity_of(tr), flag);
    const float* st = reinterpret_cast<const float*>(ring + (size_t)stage_of(tr) * stg);
    float fs[Q];
    {
      float fv[Q], Fv[D];
#pragma unroll
      for (int q = 0; q < Q; ++q) fv[q] = st[(q * TH + ly) * TW + lx];
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        // planes of the window: partial s of axis mu at plane s * D + mu, added in order of s
        float acc = st[TMA2_FF_OFF / 4 + (mu * TH + ly) * TW + lx];
        for (int k = 1; k < ks; ++k) acc += st[TMA2_FF_OFF / 4 + ((k * D + mu) * TH + ly) * TW + lx];
        Fv[mu] = acc;
      }
      collide_node<float, D, MRT, KS>(sp, fv, Fv, fs);
    }
    if (owner) {
      s_m[buf][0][sy][sx] = fs[1];
      s_m[buf][1][sy][sx] = fs[2];
      s_m[buf][2][sy][sx] = fs[3];
      s_m[buf][3][sy][sx] = fs[4];
    } else if (wy == TY) {
      if (lane < 16) s_m[buf][0][sy][sx] = fs[1];  // moves +x into the tile
      else s_m[buf][1][sy][sx] = fs[2];            // moves -x into the tile
    } else if (wy == TY + 1) {
      s_m[buf][2][sy][sx] = fs[3];                 // moves +y into the tile
    } else {
      s_m[buf][3][sy][sx] = fs[4];                 // moves -y into the tile
    }
    __syncthreads();
    // tile row tr is read by everyone: its stage takes tile row tr + nst
    if (tid == 0 && tr + nst < tr1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(tr + nst);
    }
    if (wT && tr > tr0) flush_T(tr - 1);  // its slot is rewritten only after the next barrier
    const int gy = tr * TY + dy;
    if (SPLIT == 2 && wT && owner && !(in_x && gy < n1)) s_c[((tr & 1) * TY + dy) * TCP + dx] = 0.f;
    if (owner && in_x && gy < n1) {
      float fv[Q];
      bool known[Q];
      fv[0] = fs[0];
      known[0] = true;
      known[1] = gx > 0;
      known[2] = gx + 1 < n0;
      known[3] = gy > 0;
      known[4] = gy + 1 < n1;
      fv[1] = s_m[buf][0][sy][sx - 1];
      fv[2] = s_m[buf][1][sy][sx + 1];
      fv[3] = s_m[buf][2][sy - 1][sx];
      fv[4] = s_m[buf][3][sy + 1][sx];
      float C = 0.f;
      if (x0 > 0 && x0 + TX < n0 && tr * TY > 0 && tr * TY + TY < n1) {  // no wall within reach (block-uniform)
#pragma unroll
        for (int q = 0; q < Q; ++q) C += fv[q];
      } else {
        int n_unknown = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          if (known[q]) {
            C += fv[q];
          } else {
            fv[q] = 0.f;
            ++n_unknown;
          }
        }
        if (n_unknown > 0) {
          // Eq. (Dirichlet_BC); with k unknown populations each takes 1/k of the deficit
          const float fill = (sp.C_wall - C) / static_cast<float>(n_unknown);
#pragma unroll
          for (int q = 0; q < Q; ++q)
            if (!known[q]) fv[q] = fill;
          C = fv[0];
#pragma unroll
          for (int q = 1; q < Q; ++q) C += fv[q];
        }
      }
      const long long node = gx + (long long)n0 * gy;
#pragma unroll
      for (int q = 0; q < Q; ++q) f_out[q * nodes + node] = fv[q];
      C_out[node] = C;
      if (SPLIT) write_split<SPLIT>(so, (long long)gy * so.ldp + gx, C);
      if (SPLIT == 2 && wT) s_c[((tr & 1) * TY + dy) * TCP + dx] = C;
      bad |= !isfinite(C);
      macc.add(C);
    }
    buf ^= 1;
  }
  if (wT) {
    __syncthreads();
    flush_T(tr1 - 1);
  }
  // after a timeout no copy may still be landing in this block's shared memory
  if (tid == 0) {
    for (int t = (tr1 - nst > tr0 ? tr1 - nst : tr0); t < tr1; ++t)
      cs_mbar_wait(&full[stage_of(t)], parity_of(t), flag);
    for (int s = 0; s < nst; ++s)  // the barrier words may hold other data afterwards
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(cs_smem_u32(&full[s])) : "memory");
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1);
  block_mass(macc, mpart, mslot);
}

template <bool MRT, int SPLIT>
__global__ void __launch_bounds__(TX*(TY + HALO_WARPS), 2)
collide_stream_tma2_kernel(const KConst<float> sp, const __grid_constant__ CUtensorMap map_f,
                           const __grid_constant__ CUtensorMap map_F, float* __restrict__ f_out,
                           float* __restrict__ C_out, int* __restrict__ flag, SplitOut so, int ychunk, int early,
                           double* mpart) {
  extern __shared__ uint8_t cs_raw2[];
  if (early) pdl_trigger();
  march2_tma<MRT, SPLIT>(sp, &map_f, &map_F, f_out, C_out, flag, so, ychunk, blockIdx.x, blockIdx.y, cs_raw2, mpart,
                         block_linear());
  if (!early) pdl_trigger();
}

int ychunk_for(long long tiles, int by);

// ---------------------------------------------------------------------------- fused 2-D step
// Small 2-D problems on the bf16 split: one cooperative launch runs many whole steps.
// Every block of (32, 19) threads is resident (one per SM); per step
//   phase A  warps 0-3 run operator work items (tile, contraction slice) of the per-tile
//            plan, storing partial tiles of F (op_item);
//   barrier  all blocks;
//   phase B  the block runs TMA-fed collide-stream items (tile column, tile rows), which
//            add the partial tiles in rank order (march2_tma);
//   barrier  all blocks.
// The arithmetic is that of the two-kernel step with the same plan, so the results are
// identical; the kernel boundaries (completion, flush, launch of the next grid) become
// grid barriers.  A barrier wait is bounded: after 2 s it sets bit 2 of the flag and the
// block continues, so every block reaches the end.
__device__ __forceinline__ void grid_sync(unsigned int* gbar, unsigned int target, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    atomicAdd(gbar, 1u);
    unsigned int v;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(gbar) : "memory");
      if (v >= target) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > (unsigned long long)kTmaWaitNs) {
        atomicOr(flag, 2);
        break;
      }
    }
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");  // this block's next TMA reads
  }
  __syncthreads();
}

template <int BN, int KS, bool MRT>
__global__ void __launch_bounds__(NT, 1)
lbm_fused2_kernel(const __grid_constant__ TcMaps maps, const __grid_constant__ TcParams P, const KConst<float> sp,
                  const __grid_constant__ CUtensorMap mf0, const __grid_constant__ CUtensorMap mf1,
                  const __grid_constant__ CUtensorMap mF, float* f0, float* f1, float* C, SplitOut so, int ychunk,
                  int nsteps, int parity, unsigned int* gbar, int* flag, double* mpart) {
  extern __shared__ uint8_t fused_raw[];
  __shared__ uint32_t tmem_slot;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(fused_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.y * TX + threadIdx.x;
  if (threadIdx.y == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)  // op_item's accumulator regions (at most 512 columns)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int G = gridDim.x;
  const int op_items = P.total_tiles * KS;
  const int bxn = (sp.n[0] + TX - 1) / TX, byn = (sp.n[1] + TY - 1) / TY;
  const int cs_items = bxn * ((byn + ychunk - 1) / ychunk);
  unsigned int target = 0;
  for (int st = 0; st < nsteps; ++st) {
    if (tid < 128)
      for (int it = blockIdx.x; it < op_items; it += G) op_item<2, BN, KS>(maps, P, it, smem, tmem, tid);
    target += G;
    grid_sync(gbar, target, flag);
    const int par = parity ^ (st & 1);
    const CUtensorMap* mf = par ? &mf1 : &mf0;
    float* fo = par ? f0 : f1;
    for (int it = blockIdx.x; it < cs_items; it += G) {
      march2_tma<MRT, 1>(sp, mf, &mF, fo, C, flag, so, ychunk, it % bxn, it / bxn, smem, mpart, it);
      __syncthreads();
    }
    target += G;
    grid_sync(gbar, target, flag);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.y == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

template <int BN, int KS>
size_t fused_smem() {
  const size_t a = Cfg<2, BN, KS>::SMEM, b = tma2_smem(KS);
  return (a > b ? a : b) + 1024;
}

template <int BN, int KS, bool MRT>
cudaError_t fused_attr(int* blocks_per_sm) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, lbm_fused2_kernel<BN, KS, MRT>, (int)fused_smem<BN, KS>()); e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, lbm_fused2_kernel<BN, KS, MRT>, NT,
                                                       fused_smem<BN, KS>());
}

template <int BN, int KS, bool MRT>
cudaError_t fused_launch(const lbm_s* h, int nsteps, int grid, cudaStream_t s) {
  const TcPlan* p = h->tc;
  const CsPlan* pl = static_cast<const CsPlan*>(h->cs_plan);
  const KConst<float> sp = make_const<float>(h->sp);
  SplitOut so{h->dev.Chi, h->dev.Clo, tc_split_pitch(h)};
  const int bx = (h->sp.n[0] + TX - 1) / TX, by = (h->sp.n[1] + TY - 1) / TY;
  const int ychunk = h->cs_chunk > 0 ? std::min(h->cs_chunk, by) : ychunk_for((long long)bx * by, by);
  h->cs_nparts = bx * ((by + ychunk - 1) / ychunk);  // kMassSlots mass partials per collide-stream item
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(TX, TY + HALO_WARPS);
  cfg.dynamicSmemBytes = fused_smem<BN, KS>();
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lbm_fused2_kernel<BN, KS, MRT>, p->maps, p->prm, sp, pl->f[0], pl->f[1], pl->F,
                            static_cast<float*>(h->dev.f[0]), static_cast<float*>(h->dev.f[1]),
                            static_cast<float*>(h->dev.C), so, ychunk, nsteps, h->cur, h->fused_bar, h->dev.flag,
                            h->cs_part);
}

// 2-D batch blocks run either march (per problem): room for the larger ring
constexpr int BATCH2_SMEM = (int)(TMA2_SMEM > (size_t)PIPE_SMEM ? TMA2_SMEM : (size_t)PIPE_SMEM);

// Grouped form for a batch of independent problems: one launch covers every block of
// every problem; block_map[b] = (problem, block within it), one load per block.  The
// problem's constants are staged in shared memory.
template <int D, bool MRT, int SPLIT>
__global__ void __launch_bounds__(TX*(TY + HALO_WARPS), 2)
collide_stream_batch_kernel(const BatchCS* __restrict__ tab, const int2* __restrict__ block_map, int parity) {
  __shared__ KConst<float> s_k;
  const int2 pb = __ldg(&block_map[blockIdx.x]);
  const BatchCS& e = tab[pb.x];
  const int tid = threadIdx.y * TX + threadIdx.x;
  constexpr int words = sizeof(KConst<float>) / sizeof(int);
  for (int i = tid; i < words; i += TX * (TY + HALO_WARPS))
    reinterpret_cast<int*>(&s_k)[i] = reinterpret_cast<const int*>(&e.k)[i];
  if (D == 2 && MRT && tid < kMaxQ * 8) {
    const int r = tid >> 3, c = tid & 7;
    reinterpret_cast<float*>(&s_om_rows[r][0])[c] = c < kMaxQ ? e.k.omega[r][c] : 0.0f;
  }
  __syncthreads();
  const int lb = pb.y;
  const int bx = lb % e.bx, rest = lb / e.bx;
  if constexpr (D == 2) {
    extern __shared__ __align__(128) uint8_t batch_raw[];
    if (e.tma)
      march2_tma<MRT, SPLIT, true>(s_k, &e.mf[parity], &e.mF, const_cast<float*>(e.f[parity ^ 1]), e.C, e.flag, e.so,
                             e.zchunk, bx, rest, batch_raw, e.mpart, lb);
    else
      march2_pipe<MRT, SPLIT, true>(s_k, e.f[parity], e.F, const_cast<float*>(e.f[parity ^ 1]), e.C, e.flag, e.so,
                              e.zchunk, bx, rest, reinterpret_cast<float*>(batch_raw), e.mpart, lb);
  } else {
    march_body<float, D, MRT, SPLIT>(s_k, e.f[parity], e.F, const_cast<float*>(e.f[parity ^ 1]), e.C, e.flag, e.so,
                                     bx, rest, 0, e.k.n[2], e.mpart, lb);
  }
}

template <typename real, int D>
__global__ void init_equilibrium_kernel(const KConst<real> sp, const real* __restrict__ C, const real* __restrict__ F,
                                        real* __restrict__ f, const real* __restrict__ advw) {
  const long long nodes = sp.nodes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
       i += (long long)gridDim.x * blockDim.x) {
    const real c = C[i];
    real sumF = static_cast<real>(0);
    real Fv[D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      Fv[mu] = frac_term(sp, F, mu, i);
      sumF += Fv[mu];
    }
    f[i] = c - sp.w0 * sumF;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const real a = sp.wi * Fv[mu];
      const real b = (advw ? advw[mu * nodes + i] : sp.advw[mu]) * c;  // u(x) when it varies
      f[(2 * mu + 1) * nodes + i] = a + b;
      f[(2 * mu + 2) * nodes + i] = a - b;
    }
  }
}

// G_mu = g_mu(x) C, the operator's inputs when g varies in space
template <typename real>
__global__ void scale_fields_kernel(long long nodes, int d, const real* __restrict__ C, const real* __restrict__ g,
                                    real* __restrict__ G) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
       i += (long long)gridDim.x * blockDim.x)
    for (int mu = 0; mu < d; ++mu) G[mu * nodes + i] = g[mu * nodes + i] * C[i];
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

template <bool MRT, int SPLIT>
cudaError_t launch_tma3(const cudaLaunchConfig_t& cfg, const KConst<float>& sp, const CUtensorMap& mf,
                        const CUtensorMap& mF, float* fo, float* Co, int* flag, const SplitOut& so, int nz,
                        int early, double* mpart) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, collide_stream_tma3_kernel<MRT, SPLIT>, (int)TMA_SMEM); e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, collide_stream_tma3_kernel<MRT, SPLIT>, sp, mf, mF, fo, Co, flag, so, nz, early,
                            mpart);
}

template <bool MRT, int SPLIT>
cudaError_t launch_tma2(const cudaLaunchConfig_t& cfg, const KConst<float>& sp, const CUtensorMap& mf,
                        const CUtensorMap& mF, float* fo, float* Co, int* flag, const SplitOut& so, int ychunk,
                        int early, double* mpart) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, collide_stream_tma2_kernel<MRT, SPLIT>, (int)tma2_smem(8)); e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, collide_stream_tma2_kernel<MRT, SPLIT>, sp, mf, mF, fo, Co, flag, so, ychunk,
                            early, mpart);
}

// at most two blocks per SM resident: the grid runs in one wave
bool one_wave(const dim3& g) { return (long long)g.x * g.y * g.z <= 2LL * device_sms(); }

template <bool MRT, int SPLIT>
cudaError_t launch_march2(const cudaLaunchConfig_t& cfg, const KConst<float>& sp, const float* fi, const float* F,
                          float* fo, float* Co, int* flag, const SplitOut& so, int ychunk, int early, double* mpart) {
  static std::atomic<unsigned long long> attr{0};
  if (const cudaError_t e = smem_attr_once(attr, collide_stream_march2_kernel<MRT, SPLIT>, PIPE_SMEM); e != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, collide_stream_march2_kernel<MRT, SPLIT>, sp, fi, F, fo, Co, flag, so, ychunk,
                            early, mpart);
}

// z chunks of the 3-D march over `cols` tile columns: the count that maximises the wave
// efficiency (blocks / 304 over its ceiling, two blocks per SM) per plane collided,
// each chunk re-colliding two planes at its start; chunks of at least 16 planes
int z_chunks(long long cols, int n2) {
  if (n2 < 32) return 1;
  const int sms = device_sms();
  int best = 1;
  double best_eff = 0.0;
  for (int nz = 1; nz <= n2 / 16; ++nz) {
    const double waves = static_cast<double>(cols * nz) / (2 * sms);
    const double eff = waves / std::ceil(waves);
    const double zc = static_cast<double>(n2) / nz;
    const double score = eff * zc / (zc + 2.0);
    if (score > best_eff + 1e-9) {
      best_eff = score;
      best = nz;
    }
  }
  return best;
}

// tile rows per 2-D block: ceil(tiles / 304) (one wave of two blocks per SM), at most by
int ychunk_for(long long tiles, int by) {
  const long long w = 2LL * device_sms();
  const long long c = (tiles + w - 1) / w;
  return static_cast<int>(std::max<long long>(1, std::min<long long>(c, by)));
}

// which operand split of the new C the collide-stream kernel writes (write_split codes)
int cs_split_code(const lbm_s* h) {
  if (h->tc == nullptr) return 0;
  if (!bf16_parts(h->prm.precision)) return 2;
  return h->prm.precision == LBM_FP32_BF16SPLIT6 ? 3 : 1;
}

template <typename real, int D, bool MRT>
cudaError_t launch_cs(const lbm_s* h, const void* f_in, void* f_out, void* C_out, cudaStream_t s, int tk) {
  const KConst<real> sp = make_const<real>(h->sp);
  SplitOut so{h->dev.Chi, h->dev.Clo, tc_split_pitch(h)};
  so.lo2 = h->dev.Cl2;
  const int split = cs_split_code(h);
  const real* fi = static_cast<const real*>(f_in);
  const real* F = static_cast<const real*>(h->dev.F);
  real* fo = static_cast<real*>(f_out);
  real* Co = static_cast<real*>(C_out);
  int* flag = h->dev.flag;
  double* mp = h->cs_part;
  const int bx = (sp.n[0] + TX - 1) / TX, by = (sp.n[1] + TY - 1) / TY;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TX, TY + HALO_WARPS);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = h->pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (h->fld.on) {
    // coefficients per node: the plain march with the per-node collision (2-D: one plane)
    const int nz = (D == 2) ? 1 : (h->cs_chunk > 0 ? std::min(h->cs_chunk, sp.n[2]) : z_chunks((long long)bx * by, sp.n[2]));
    cfg.gridDim = dim3(bx, by, nz);
    h->cs_nparts = bx * by * nz;
    const int early = one_wave(cfg.gridDim) ? 1 : 0;
    FieldPtrs<real> fp{static_cast<const real*>(h->fld.coll), static_cast<const real*>(h->fld.advw),
                       static_cast<const real*>(h->fld.g),    static_cast<real*>(h->fld.G),
                       static_cast<const real*>(h->fld.src),  static_cast<const real*>(h->fld.cw),
                       h->fld.tf ? h->fld.tf + 2 * tk : nullptr, {}, 0, 0};
    if (h->tc && h->tc->gvar && h->tc->elem == 2) {  // bf16: the parts of g_mu(x) C per axis
      fp.gsplit = 1;
      fp.gldp = h->tc->ldp;
      for (int mu = 0; mu < 3; ++mu)
        for (int k = 0; k < 3; ++k) fp.gs[mu][k] = h->tc->gp[mu][k];
    }
    if constexpr (sizeof(real) == 4) {
      // tensor-core forms: the march also writes the operator's operands of the new C
      if (split == 1)
        return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 1, true>, sp, fi, F, fo, Co, flag, so,
                                  nz, early, mp, fp);
      if (split == 2)
        return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 2, true>, sp, fi, F, fo, Co, flag, so,
                                  nz, early, mp, fp);
      if (split == 3)
        return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 3, true>, sp, fi, F, fo, Co, flag, so,
                                  nz, early, mp, fp);
    }
    return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 0, true>, sp, fi, F, fo, Co, flag, so,
                              nz, early, mp, fp);
  }
  if constexpr (D == 2 && sizeof(real) == 4) {
    // tile rows per block: about one wave of two blocks per SM, unless tuned
    const int ychunk = h->cs_chunk > 0 ? std::min(h->cs_chunk, by) : ychunk_for((long long)bx * by, by);
    cfg.gridDim = dim3(bx, (by + ychunk - 1) / ychunk, 1);
    h->cs_nparts = static_cast<int>(cfg.gridDim.x * cfg.gridDim.y);
    const int early = one_wave(cfg.gridDim) ? 1 : 0;
    if (h->cs_plan) {
      const CsPlan* pl = static_cast<const CsPlan*>(h->cs_plan);
      const CUtensorMap& mf = pl->f[f_in == h->dev.f[0] ? 0 : 1];
      cfg.dynamicSmemBytes = tma2_smem(h->sp.ksum);
      if (split == 0) return launch_tma2<MRT, 0>(cfg, sp, mf, pl->F, fo, Co, flag, so, ychunk, early, mp);
      if (split == 1) return launch_tma2<MRT, 1>(cfg, sp, mf, pl->F, fo, Co, flag, so, ychunk, early, mp);
      if (split == 3) return launch_tma2<MRT, 3>(cfg, sp, mf, pl->F, fo, Co, flag, so, ychunk, early, mp);
      so.thi[0] = static_cast<float*>(h->tc->ct_hi[1]);  // the y operand of the tf32 operator
      so.tg1 = h->tc->tg[1];
      so.tpx = h->tc->tpx;
      return launch_tma2<MRT, 2>(cfg, sp, mf, pl->F, fo, Co, flag, so, ychunk, early, mp);
    }
    cfg.dynamicSmemBytes = PIPE_SMEM;
    if (split == 0) return launch_march2<MRT, 0>(cfg, sp, fi, F, fo, Co, flag, so, ychunk, early, mp);
    if (split == 1) return launch_march2<MRT, 1>(cfg, sp, fi, F, fo, Co, flag, so, ychunk, early, mp);
    if (split == 3) return launch_march2<MRT, 3>(cfg, sp, fi, F, fo, Co, flag, so, ychunk, early, mp);
    return launch_march2<MRT, 2>(cfg, sp, fi, F, fo, Co, flag, so, ychunk, early, mp);
  }
  const int nz = h->cs_chunk > 0 ? std::min(h->cs_chunk, sp.n[2]) : z_chunks((long long)bx * by, sp.n[2]);
  cfg.gridDim = dim3(bx, by, nz);
  h->cs_nparts = bx * by * nz;
  const int early = one_wave(cfg.gridDim) ? 1 : 0;
  if constexpr (D == 3 && sizeof(real) == 4) {
    if (h->cs_plan) {
      // TMA-fed march: the map of whichever population buffer is the input
      const CsPlan* pl = static_cast<const CsPlan*>(h->cs_plan);
      const CUtensorMap& mf = pl->f[f_in == h->dev.f[0] ? 0 : 1];
      cfg.dynamicSmemBytes = TMA_SMEM;
      if (split == 0) return launch_tma3<MRT, 0>(cfg, sp, mf, pl->F, fo, Co, flag, so, nz, early, mp);
      if (split == 1) return launch_tma3<MRT, 1>(cfg, sp, mf, pl->F, fo, Co, flag, so, nz, early, mp);
      if (split == 3) return launch_tma3<MRT, 3>(cfg, sp, mf, pl->F, fo, Co, flag, so, nz, early, mp);
      for (int a = 0; a < 2; ++a) {  // the y and z operands of the tf32 operator
        so.thi[a] = static_cast<float*>(h->tc->ct_hi[a + 1]);
      }
      so.tg1 = h->tc->tg[1];
      so.tpx = h->tc->tpx;
      return launch_tma3<MRT, 2>(cfg, sp, mf, pl->F, fo, Co, flag, so, nz, early, mp);
    }
  }
  if (split == 0)
    return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 0>, sp, fi, F, fo, Co, flag, so, nz,
                              early, mp, FieldPtrs<real>{});
  if (split == 1)
    return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 1>, sp, fi, F, fo, Co, flag, so, nz,
                              early, mp, FieldPtrs<real>{});
  if (split == 3)
    return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 3>, sp, fi, F, fo, Co, flag, so, nz,
                              early, mp, FieldPtrs<real>{});
  return cudaLaunchKernelEx(&cfg, collide_stream_march_kernel<real, D, MRT, 2>, sp, fi, F, fo, Co, flag, so, nz,
                            early, mp, FieldPtrs<real>{});
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 16LL * device_sms();
  if (b > cap) b = cap;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

// tf32 handles on the TMA-fed marches: the collide-stream kernel writes the regrouped split
bool cs_writes_T(const lbm_s* h) {
  return !h->is_batch() && h->elem == 4 && h->cs_plan != nullptr && h->tc != nullptr && h->tc->elem == 4 &&
         h->prm.precision == LBM_FP32_TF32SPLIT && !h->fld.on;  // the field march writes x-major operands only
}

cudaError_t launch_collide_stream(const lbm_s* h, const void* f_in, void* f_out, void* C_out, cudaStream_t s,
                                  int tk) {
  const bool mrt = h->prm.collision == LBM_MRT;
  if (h->elem == 8) {
    if (h->d == 2) return mrt ? launch_cs<double, 2, true>(h, f_in, f_out, C_out, s, tk)
                              : launch_cs<double, 2, false>(h, f_in, f_out, C_out, s, tk);
    return mrt ? launch_cs<double, 3, true>(h, f_in, f_out, C_out, s, tk)
               : launch_cs<double, 3, false>(h, f_in, f_out, C_out, s, tk);
  }
  if (h->d == 2) return mrt ? launch_cs<float, 2, true>(h, f_in, f_out, C_out, s, tk)
                            : launch_cs<float, 2, false>(h, f_in, f_out, C_out, s, tk);
  return mrt ? launch_cs<float, 3, true>(h, f_in, f_out, C_out, s, tk)
             : launch_cs<float, 3, false>(h, f_in, f_out, C_out, s, tk);
}

constexpr int kBatchYChunk = 16;  // tile rows per block (the autotuner's usual choice on mixed batches)

// window maps of a 2-D handle: populations (n0, n1, 5) and fractional terms (n0, n1, 2)
bool encode_2d_maps(const lbm_s* h, CUtensorMap* mf, CUtensorMap* mF) {
  const unsigned long long n0 = h->sp.n[0], n1 = h->sp.n[1];
  const unsigned long long nodes = h->sp.nodes;
  const unsigned long long strides[2] = {n0 * 4, nodes * 4};
  const unsigned long long ks = (unsigned long long)h->sp.ksum;  // F: [partial][axis][node]
  const unsigned long long df[3] = {n0, n1, 5};
  const unsigned long long dF[3] = {n0, n1, 2 * ks};
  const unsigned int bf[3] = {TW, TH, 5};
  const unsigned int bF[3] = {TW, TH, (unsigned int)(2 * ks)};
  return encode_f32_map(&mf[0], 3, h->dev.f[0], df, strides, bf) &&
         encode_f32_map(&mf[1], 3, h->dev.f[1], df, strides, bf) &&
         encode_f32_map(mF, 3, h->dev.F, dF, strides, bF);
}

// the fused step for this handle's plan: 0 (not covered) or the blocks per SM it gets
namespace {
template <int BN, int KS>
cudaError_t fused_call(lbm_s* h, int nsteps, int grid, cudaStream_t s, int* occ) {
  const bool mrt = h->prm.collision == LBM_MRT;
  if (occ) return mrt ? fused_attr<BN, KS, true>(occ) : fused_attr<BN, KS, false>(occ);
  return mrt ? fused_launch<BN, KS, true>(h, nsteps, grid, s) : fused_launch<BN, KS, false>(h, nsteps, grid, s);
}

cudaError_t fused_any(lbm_s* h, int nsteps, int grid, cudaStream_t s, int* occ) {
  int bn = 0, ks = 0, persist = 0;
  tc_config(h, &bn, &ks, &persist);
  if (persist) return cudaErrorNotSupported;
  if (bn == 64 && ks == 2) return fused_call<64, 2>(h, nsteps, grid, s, occ);
  if (bn == 64 && ks == 4) return fused_call<64, 4>(h, nsteps, grid, s, occ);
  if (bn == 128 && ks == 2) return fused_call<128, 2>(h, nsteps, grid, s, occ);
  if (bn == 128 && ks == 4) return fused_call<128, 4>(h, nsteps, grid, s, occ);
  return cudaErrorNotSupported;
}
}  // namespace

int fused_prepare(lbm_s* h) {
  h->fused_grid = 0;
  if (h->is_batch() || h->d != 2 || h->prm.precision != LBM_FP32_BF16SPLIT || !h->tc || !h->cs_plan) return LBM_ENOTSUP;
  if (!tc_tma_store(h)) return LBM_ENOTSUP;
  int occ = 0;
  if (fused_any(h, 0, 0, nullptr, &occ) != cudaSuccess || occ < 1) return LBM_ENOTSUP;
  if (!h->fused_bar && dev_alloc(h, (void**)&h->fused_bar, sizeof(unsigned int)) != cudaSuccess) return LBM_ENOMEM;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  h->fused_grid = sms * occ;
  return LBM_OK;
}

cudaError_t launch_fused(lbm_s* h, int nsteps, cudaStream_t s) {
  if (h->fused_grid < 1) return cudaErrorNotSupported;
  const cudaError_t e = cudaMemsetAsync(h->fused_bar, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  return fused_any(h, nsteps, h->fused_grid, s, nullptr);
}

int cs_prepare(lbm_s* h) {
  if (h->elem != 4 || h->sp.n[0] % 4 != 0) return LBM_OK;
  if (h->d == 3 && h->sp.ksum != 1) return LBM_OK;  // the plain 3-D march sums the partials
  CsPlan* pl = new (std::nothrow) CsPlan();
  if (!pl) return LBM_ENOMEM;
  if (h->d == 2) {
    if (encode_2d_maps(h, pl->f, &pl->F)) h->cs_plan = pl;
    else delete pl;  // the cp.async march serves the handle
    return LBM_OK;
  }
  const unsigned long long n0 = h->sp.n[0], n1 = h->sp.n[1], n2 = h->sp.n[2];
  const unsigned long long nodes = h->sp.nodes;
  const unsigned long long strides[3] = {n0 * 4, n0 * n1 * 4, nodes * 4};
  const unsigned long long df[4] = {n0, n1, n2, 7};
  const unsigned long long dF[4] = {n0, n1, n2, 3};
  const unsigned int bf[4] = {TW, TH, 1, 7};
  const unsigned int bF[4] = {TW, TH, 1, 3};
  bool ok = encode_f32_map(&pl->f[0], 4, h->dev.f[0], df, strides, bf) &&
            encode_f32_map(&pl->f[1], 4, h->dev.f[1], df, strides, bf) &&
            encode_f32_map(&pl->F, 4, h->dev.F, dF, strides, bF);
  if (!ok) {
    delete pl;
    return LBM_OK;  // the plain march serves the handle
  }
  h->cs_plan = pl;
  return LBM_OK;
}

void cs_release(lbm_s* h) {
  delete static_cast<CsPlan*>(h->cs_plan);
  h->cs_plan = nullptr;
}

bool cs_one_wave(const lbm_s* h) {
  const int bx = (h->sp.n[0] + TX - 1) / TX, by = (h->sp.n[1] + TY - 1) / TY;
  if (h->d == 2 && h->elem == 4) {
    const int ychunk = h->cs_chunk > 0 ? std::min(h->cs_chunk, by) : ychunk_for((long long)bx * by, by);
    return one_wave(dim3(bx, (by + ychunk - 1) / ychunk, 1));
  }
  if (h->d == 2) return one_wave(dim3(bx, by, 1));
  const int nz = h->cs_chunk > 0 ? std::min(h->cs_chunk, h->sp.n[2]) : z_chunks((long long)bx * by, h->sp.n[2]);
  return one_wave(dim3(bx, by, nz));
}

int cs_chunk_default(const lbm_s* h) {
  const int bx = (h->sp.n[0] + TX - 1) / TX, by = (h->sp.n[1] + TY - 1) / TY;
  if (h->is_batch()) return kBatchYChunk;
  if (h->d == 2) return h->elem == 4 ? ychunk_for((long long)bx * by, by) : 1;
  return z_chunks((long long)bx * by, h->sp.n[2]);
}

int cs_batch_prepare(lbm_s* b) {
  const int P = static_cast<int>(b->subs.size());
  std::vector<BatchCS> tab(P);
  std::vector<int2> map;
  int total = 0;
  for (int i = 0; i < P; ++i) {
    lbm_s* h = b->subs[i];
    if (h->elem != 4) return LBM_EINVAL;
    BatchCS& e = tab[i];
    e.k = make_const<float>(h->sp);
    e.f[0] = static_cast<const float*>(h->dev.f[0]);
    e.f[1] = static_cast<const float*>(h->dev.f[1]);
    e.F = static_cast<const float*>(h->dev.F);
    e.C = static_cast<float*>(h->dev.C);
    e.so = SplitOut{h->dev.Chi, h->dev.Clo, tc_split_pitch(h)};
    e.so.lo2 = h->dev.Cl2;
    e.flag = h->dev.flag;
    e.mpart = h->cs_part;
    e.tma = (h->d == 2 && h->sp.n[0] % 4 == 0 && encode_2d_maps(h, e.mf, &e.mF)) ? 1 : 0;
    e.bx = (h->sp.n[0] + TX - 1) / TX;
    e.by = (h->sp.n[1] + TY - 1) / TY;
    // 2-D: tile rows per block (the pipelined y-march); 3-D: the whole z extent
    e.zchunk = (h->d == 2) ? std::min(e.by, b->cs_chunk > 0 ? b->cs_chunk : kBatchYChunk) : h->sp.n[2];
    h->cs_nparts = e.bx * ((h->d == 2) ? (e.by + e.zchunk - 1) / e.zchunk : e.by);
    for (int k = 0; k < h->cs_nparts; ++k) map.push_back(make_int2(i, k));
    total += h->cs_nparts;
  }
  dev_free(b, b->batch_cs);
  dev_free(b, b->batch_cs_start);
  b->batch_cs = nullptr;
  b->batch_cs_start = nullptr;
  if (dev_alloc(b, &b->batch_cs, sizeof(BatchCS) * P) != cudaSuccess) return LBM_ENOMEM;
  if (dev_alloc(b, (void**)&b->batch_cs_start, sizeof(int2) * total) != cudaSuccess) return LBM_ENOMEM;
  if (cudaMemcpy(b->batch_cs, tab.data(), sizeof(BatchCS) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->batch_cs_start, map.data(), sizeof(int2) * total, cudaMemcpyHostToDevice) != cudaSuccess)
    return LBM_ECUDA;
  b->batch_cs_blocks = total;
  return LBM_OK;
}

cudaError_t launch_collide_stream_batch(const lbm_s* b, int parity, cudaStream_t s) {
  const lbm_s* h0 = b->subs[0];
  const bool mrt = h0->prm.collision == LBM_MRT;
  const int split = cs_split_code(h0);  // 0, 1 or 3 (batches have no tf32 form)
  const BatchCS* tab = static_cast<const BatchCS*>(b->batch_cs);
  const int P = static_cast<int>(b->subs.size());
  dim3 block(TX, TY + HALO_WARPS);
  const int g = b->batch_cs_blocks;
  const int smem = (h0->d == 2) ? BATCH2_SMEM : 0;
  if (h0->d == 2) {
    static std::atomic<unsigned long long> attr[2][4] = {{{0}, {0}, {0}, {0}}, {{0}, {0}, {0}, {0}}};
    cudaError_t e;
    if (mrt) e = split == 3 ? smem_attr_once(attr[1][3], collide_stream_batch_kernel<2, true, 3>, BATCH2_SMEM)
                 : split    ? smem_attr_once(attr[1][1], collide_stream_batch_kernel<2, true, 1>, BATCH2_SMEM)
                            : smem_attr_once(attr[1][0], collide_stream_batch_kernel<2, true, 0>, BATCH2_SMEM);
    else e = split == 3 ? smem_attr_once(attr[0][3], collide_stream_batch_kernel<2, false, 3>, BATCH2_SMEM)
             : split    ? smem_attr_once(attr[0][1], collide_stream_batch_kernel<2, false, 1>, BATCH2_SMEM)
                        : smem_attr_once(attr[0][0], collide_stream_batch_kernel<2, false, 0>, BATCH2_SMEM);
    if (e != cudaSuccess) return e;
  }
#define LBM_CSB(D_, M_, S_) \
  collide_stream_batch_kernel<D_, M_, S_><<<g, block, smem, s>>>(tab, reinterpret_cast<const int2*>(b->batch_cs_start), parity)
  if (h0->d == 2) {
    if (mrt) { if (split == 3) LBM_CSB(2, true, 3); else if (split) LBM_CSB(2, true, 1); else LBM_CSB(2, true, 0); }
    else { if (split == 3) LBM_CSB(2, false, 3); else if (split) LBM_CSB(2, false, 1); else LBM_CSB(2, false, 0); }
  } else {
    if (mrt) { if (split == 3) LBM_CSB(3, true, 3); else if (split) LBM_CSB(3, true, 1); else LBM_CSB(3, true, 0); }
    else { if (split == 3) LBM_CSB(3, false, 3); else if (split) LBM_CSB(3, false, 1); else LBM_CSB(3, false, 0); }
  }
#undef LBM_CSB
  return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(const lbm_s* h, void* f, cudaStream_t s) {
  const int g = grid_for(h->sp.nodes);
  const void* aw = h->fld.on ? h->fld.advw : nullptr;
  if (h->elem == 8) {
    if (h->d == 2)
      init_equilibrium_kernel<double, 2><<<g, 256, 0, s>>>(make_const<double>(h->sp), (const double*)h->dev.C, (const double*)h->dev.F, (double*)f, (const double*)aw);
    else
      init_equilibrium_kernel<double, 3><<<g, 256, 0, s>>>(make_const<double>(h->sp), (const double*)h->dev.C, (const double*)h->dev.F, (double*)f, (const double*)aw);
  } else {
    if (h->d == 2)
      init_equilibrium_kernel<float, 2><<<g, 256, 0, s>>>(make_const<float>(h->sp), (const float*)h->dev.C, (const float*)h->dev.F, (float*)f, (const float*)aw);
    else
      init_equilibrium_kernel<float, 3><<<g, 256, 0, s>>>(make_const<float>(h->sp), (const float*)h->dev.C, (const float*)h->dev.F, (float*)f, (const float*)aw);
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_fields(const lbm_s* h, cudaStream_t s) {
  if (!h->fld.G) return cudaSuccess;  // tensor-core forms: g is uniform and folded into K
  const int g = grid_for(h->sp.nodes);
  if (h->elem == 8)
    scale_fields_kernel<double><<<g, 256, 0, s>>>(h->sp.nodes, h->d, (const double*)h->dev.C, (const double*)h->fld.g,
                                                  (double*)h->fld.G);
  else
    scale_fields_kernel<float><<<g, 256, 0, s>>>(h->sp.nodes, h->d, (const float*)h->dev.C, (const float*)h->fld.g,
                                                 (float*)h->fld.G);
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
