// Internal declarations shared by the translation units of liblbm_fade.so.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <vector>

#include "lbm_fade.h"

namespace lbm {

constexpr int kMaxQ = 7;
// mass partials per collide-stream block: one per warp of its 32 x (16 + 3) threads
constexpr int kMassSlots = 19;
struct TcPlan;  // tensor-core plan (frac_tc.cu)

// Per-problem constants of one time step, passed by value to the kernels.
// Derived on the host in FP64 from lbm_params (Algorithm 1, initialisation).
struct StepParams {
  int n[3];                  // nodes per axis (unused axes: 1)
  long long nodes;           // n[0]*n[1]*n[2]
  double omega[kMaxQ][kMaxQ];// collision matrix: f* = f - omega (f - feq)
                             //   BGK: omega = I/lambda; MRT: M^-1 Lambda M (Eq. MRT-Coll)
  double w0, wi;             // lattice weights: rest and moving (Fig. 1 caption)
  double adv[3];             // (dt/dx) u_mu / e^2: advective factor of Eq. (Feq)
  double C_wall;             // Dirichlet value (Eq. Dirichlet_BC)
  // fractional terms held as ksum partial sums over the contraction (split-K operator):
  // F_mu(node) = sum_{s < ksum} F[s * pstride + mu * nodes + node], added in order of s
  int ksum;
  long long pstride;
  double sfree[3];           // MRT rates of the free moments (Eq. MatrixS)
};

// Coefficients that vary from node to node (lbm_set_fields); device arrays in the working
// precision, [k][node].  coll: BGK 1/lambda(x), MRT the symmetric flux-block rates
// R(x) = lambdabar(x)^-1 (d(d+1)/2 entries); advw: (dt/dx) u_mu(x) w_i / e^2; g: g_mu(x);
// G: g_mu(x) C, the operator's input along mu.
struct FieldState {
  bool on = false;     // the per-node kernel path runs (coefficients, source or wall values)
  bool coeff = false;  // D, g or u vary (lbm_set_fields)
  bool gvar = false;   // g varies (the operator's input is g_mu(x) C, K_mu without g)
  void* coll = nullptr;
  void* advw = nullptr;
  void* g = nullptr;
  void* G = nullptr;
  // the coefficient arrays last given to lbm_set_fields (empty: the constants)
  std::vector<double> D_host, g_host, u_host;
  // source S_c(x, t) = S(x) exp(src_rate t) and wall values C_w(x) exp(cw_rate t) (null: none /
  // the constant C_wall), working precision [node]; tf: per-launch time factors [slot][2]
  void* src = nullptr;
  double src_rate = 0.0;
  void* cw = nullptr;
  double cw_rate = 0.0;
  double* tf = nullptr;
  int tf_slots = 0;
};

// Device-side buffers of one problem.
struct DeviceState {
  void* f[2] = {nullptr, nullptr};  // populations [q][node], double-buffered
  void* C = nullptr;                 // concentration [node]
  void* C0 = nullptr;                // initial concentration kept for lbm_reset [node]
  void* F = nullptr;                 // fractional terms [mu][node]
  void* K = nullptr;                 // K_mu, [mu][side_mu^2] row-major (n, l)
  void* KT = nullptr;                // K_mu transposed, [mu][side_mu^2] row-major (l, n)
  double* stage = nullptr;           // FP64 staging [node] / [q][node] for host I/O
  double* partials = nullptr;        // FP64 block partial sums (mass reduction)
  double* scalar = nullptr;          // FP64 reduction result
  int* flag = nullptr;               // latched device error bits (1 = non-finite C)
  // split operands for the tensor-core fractional operator
  void* Khi = nullptr;               // [mu][side^2] hi part of K (bf16 or tf32-in-fp32)
  void* Klo = nullptr;               // [mu][side^2] lo part of K
  void* Kl2 = nullptr;               // [mu][side^2] third part of K (five-product bf16 form)
  void* Chi = nullptr;               // [node] hi part of C
  void* Clo = nullptr;               // [node] lo part of C
  void* Cl2 = nullptr;               // [node] third part of C (six-product bf16 form)
};

}  // namespace lbm

// device-memory hooks a handle was created with (lbm_set_allocator; null: cudaMalloc)
struct DevMem {
  lbm_alloc_fn alloc = nullptr;
  lbm_free_fn release = nullptr;
  void* ctx = nullptr;
};

struct lbm_s {
  lbm_params prm;
  DevMem mem;
  int d = 2, Q = 5;
  int elem = 8;                        // bytes per real (8 FP64, 4 FP32 forms)
  lbm::StepParams sp;
  lbm::DeviceState dev;
  lbm::FieldState fld;
  long long t_steps = 0;               // steps since the last (re-)initialisation: t = t_steps dt
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int cur = 0;                         // index of the current population buffer
  int reduce_blocks = 0;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int graph_steps = 0;                 // steps per captured graph (even)
  int launches_per_step = 0;
  size_t f_elems = 0;                  // capacity of dev.F (elements) for the SIMT operator's partials
  // programmatic dependent launch between the operator and collide-stream: only when both
  // grids run in a single wave (measured: with multi-wave 3-D grids it costs ~30%)
  bool pdl = false;
  // collide-stream work per block: 2-D tile rows, 3-D z chunks (0: the built-in choice)
  int cs_chunk = 0;
  // fused small-problem step (one cooperative launch runs many steps), if selected
  bool fused = false;
  int fused_grid = 0;
  unsigned int* fused_bar = nullptr;   // grid-barrier counter
  int device = 0;
  // FP64 warp partials of the mass of the concentration each collide-stream launch writes
  // (kMassSlots per block of its grid: cs_nparts blocks, at most cs_part_cap); mass_valid when the
  // latest C came from a step (not from a re-initialisation); mass_limit > 0 turns a mass of
  // larger magnitude (or a non-finite one) into LBM_ERR_UNSTABLE at the next synchronising call
  double* cs_part = nullptr;
  long long cs_part_cap = 0;
  mutable int cs_nparts = 0;
  bool mass_valid = false;
  double mass_limit = 0.0;
  lbm::TcPlan* tc = nullptr;           // split-precision tensor-core operator, if used
  void* cs_plan = nullptr;             // TMA-fed 3-D collide-stream (tensor maps), if used
  // batch of independent problems: one sub-handle per problem (each owns its buffers)
  std::vector<lbm_s*> subs;
  void* batch_tc_maps = nullptr;       // device table of per-problem tensor maps
  void* batch_tc_prm = nullptr;        // device table of per-problem operator parameters
  int* batch_tc_start = nullptr;       // first CTA of each problem (grouped operator)
  int batch_tc_blocks = 0;
  void* batch_cs = nullptr;            // device table of per-problem collide-stream entries
  int* batch_cs_start = nullptr;       // (problem, block within it) per block, int2 pairs (grouped collide-stream)
  int batch_cs_blocks = 0;
  bool is_batch() const { return !subs.empty(); }
};

namespace lbm {

// streaming multiprocessors of the current device (queried once per device)
int device_sms();

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per device for one kernel:
// `done` is a static of the calling launcher (one per kernel instantiation), bit d of it
// stands for device d.
template <typename Kernel>
cudaError_t smem_attr_once(std::atomic<unsigned long long>& done, Kernel k, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// a handle's device memory: through its hooks, else cudaMalloc / cudaFree
cudaError_t dev_alloc(const lbm_s* h, void** p, size_t bytes);
void dev_free(const lbm_s* h, void* p);

// ---- kernels (launchers return cudaGetLastError of the launch)
// fractional operator, SIMT: F_mu = K_mu applied along axis mu, for all mu
cudaError_t launch_frac_simt(const lbm_s* h, const void* C, void* F, cudaStream_t s);
// contraction split of the FP32 SIMT operator for a single problem: F then holds that
// many partial sums ([rank][axis][node], like the tensor-core split), 1 for FP64
int simt_ksplit(const lbm_s* h);
// the FP32 SIMT operator's grid is resident at once (programmatic dependent launch)
bool simt_one_wave(const lbm_s* h);
// tensor-core split-precision fractional operator (tcgen05); returns
// cudaErrorNotSupported when the handle's shape is not covered
cudaError_t launch_frac_tc(const lbm_s* h, cudaStream_t s);
// fused equilibrium + collision + streaming + Dirichlet + new concentration; on the
// tensor-core path it also writes the hi/lo split of the new concentration
cudaError_t launch_collide_stream(const lbm_s* h, const void* f_in, void* f_out, void* C_out,
                                  cudaStream_t s, int tk = 0);
// f = feq(C, F) (with u(x) when the coefficients vary)
cudaError_t launch_init_equilibrium(const lbm_s* h, void* f, cudaStream_t s);
// G_mu = g_mu(x) C (spatially varying coefficients only)
cudaError_t launch_scale_fields(const lbm_s* h, cudaStream_t s);
// C = sum_q f_q
cudaError_t launch_moment(const lbm_s* h, const void* f, void* C, cudaStream_t s);
// conversions between the FP64 staging buffer and the working precision
cudaError_t launch_convert_in(const void* src_f64, void* dst, int elem, long long n, cudaStream_t s);
cudaError_t launch_convert_out(const void* src, int elem, double* dst_f64, long long n, cudaStream_t s);
// dst_f64[i] = sum_{s < k} src[s * stride + i], FP32 partials added in order of s
cudaError_t launch_sum_partials_out(const float* src, int k, long long stride, double* dst_f64, long long n,
                                    cudaStream_t s);
// dst[i] = sum_{s < k} src[s * stride + i] in FP32, in order of s (as the collide-stream
// kernels add the operator's partial sums)
cudaError_t launch_sum_partials(const float* src, int k, long long stride, float* dst, long long n, cudaStream_t s);
// mass reduction: partials then final
cudaError_t launch_mass(const lbm_s* h, const void* C, cudaStream_t s);
// mass of the latest step from the collide-stream kernel's warp partials (one small pass,
// fixed order) into dev.scalar; with limit > 0 a mass that is not within [-limit, limit]
// sets the instability bit of the handle's flag
cudaError_t launch_step_mass(const lbm_s* h, double limit, cudaStream_t s);
// split C into hi/lo operands for the tensor-core path (tf32: also the regrouped copies)
cudaError_t launch_split_C(const lbm_s* h, cudaStream_t s);
// tf32 only: the transposed copies of the split of the current C (no-op otherwise)
cudaError_t launch_split_T(const lbm_s* h, cudaStream_t s);
// launch_split_T inside the time loop: a no-op where the collide-stream kernel writes the
// transposed split itself (cs_writes_T: tf32, 3-D, TMA-fed march)
cudaError_t launch_split_T_step(const lbm_s* h, cudaStream_t s);
bool cs_writes_T(const lbm_s* h);
// the tensor-core forms with bf16 parts (three, five or six products)
inline bool bf16_parts(int precision) {
  return precision == LBM_FP32_BF16SPLIT || precision == LBM_FP32_BF16SPLIT5 || precision == LBM_FP32_BF16SPLIT6;
}
int reduce_blocks_for(long long n);
// tensor-core plan: split K_mu (row-major FP64 per axis), allocate split C, encode TMA maps
// force_bn / force_ks (> 0) fix the column-tile width and k-split (grouped batches use 128 / 1)
int tc_prepare(lbm_s* h, const std::vector<std::vector<double>>& K, int force_bn, int force_ks);
// operator plan: column tile width bn (64, 128, 256), contraction split ks (1, 2, 4, 8),
// persistent kernel or one CTA per tile; re-encodes the tensor maps (LBM_EINVAL for a
// combination the kernels do not cover).  Captured graphs must be dropped afterwards.
int tc_replan(lbm_s* h, int bn, int ks, int persist);
long long tc_count_tiles(const lbm_s* h, int bn);  // output tiles of bn columns, all axes
int tc_kbmin(const lbm_s* h);                      // fewest contraction blocks of any axis
void tc_config(const lbm_s* h, int* bn, int* ks, int* persist);
// grouped launches over the sub-problems of a batch handle
int tc_batch_prepare(lbm_s* b);
cudaError_t launch_frac_tc_batch(const lbm_s* b, cudaStream_t s);
int cs_batch_prepare(lbm_s* b);
// TMA-fed 3-D collide-stream: tensor maps of the population and fractional-term buffers
// (FP32 forms with n0 % 4 == 0); no-op otherwise.  cs_release frees them.
int cs_prepare(lbm_s* h);
void cs_release(lbm_s* h);
// tensor map of an FP32 array (no swizzle, zero fill out of bounds); false on failure
bool encode_f32_map(void* map, int rank, void* base, const unsigned long long* dims,
                    const unsigned long long* strides_bytes, const unsigned int* box);
bool cs_one_wave(const lbm_s* h);  // the collide-stream grid fits in one wave
int cs_chunk_default(const lbm_s* h);  // the built-in tile rows (2-D) / z chunks (3-D)
// fused 2-D step (bf16 split, per-tile plan with 64/128-column tiles and a split of 2 or
// 4): LBM_OK if this handle can run it (sets fused_grid), LBM_ENOTSUP otherwise
int fused_prepare(lbm_s* h);
cudaError_t launch_fused(lbm_s* h, int nsteps, cudaStream_t s);
bool tc_tma_store(const lbm_s* h);  // the operator stores F tiles with TMA
bool tc_one_wave(const lbm_s* h);  // the tensor-core operator grid fits in one wave
void tc_set_pdl(lbm_s* h, bool on);
cudaError_t launch_collide_stream_batch(const lbm_s* b, int parity, cudaStream_t s);
void tc_release(lbm_s* h);
int tc_set_weights(lbm_s* h, const std::vector<std::vector<double>>& K);  // re-split K_mu (plan kept)
int tc_set_gfield(lbm_s* h, bool on);  // bf16 forms: operands g_mu(x) C per axis (or C)
int tc_split_pitch(const lbm_s* h);

// host-side weight build (FP64), K row-major [n][l] for one axis
void build_frac_matrix(double alpha, double p, double scale_g, int side, double dx, int variant, double* K);
// its derivatives dK/dalpha and dK/dp (FP64, same layout)
void build_frac_matrix_grad(double alpha, double p, double scale_g, int side, double dx, int variant, double* dKda,
                            double* dKdp);
double digamma_fn(double x);

// adjoint driver (adjoint.cu); the handle's own reset and step are passed in
struct AdjHooks {
  int (*reset)(lbm_s*);
  int (*step)(lbm_s*, int&, cudaStream_t);
};
int adjoint_grad(lbm_s* h, const AdjHooks& hooks, int nsnap, const int* snaps, const double* obs, int ckpt,
                 const double dOm[3][kMaxQ][kMaxQ], double* loss, double* G, double* gsum);
// transpose of the SIMT fractional operator: out_mu = K_mu^T applied along axis mu to in_mu
// out_mu = K_mu^T applied along mu to the field at in + mu * in_stride (elements)
cudaError_t launch_frac_simt_T(const lbm_s* h, const void* in, long long in_stride, void* out, cudaStream_t s);

}  // namespace lbm
