/*
 * lbm_fade.h -- C ABI of the GB300 (sm_103a) time step of the BGK/MRT lattice
 * Boltzmann scheme for the space-fractional advection-diffusion equation
 *
 *   dC/dt + div(u C) = div( D F(C) ),
 *   F_mu(C) = d/dx_mu [ p_mu I+^{2-alpha_mu}(g_mu C) + (1-p_mu) I-^{2-alpha_mu}(g_mu C) ]
 *
 * of Cartalade, Younsi & Neel, "Multiple-Relaxation-Time Lattice Boltzmann
 * scheme for Fractional Advection-Diffusion Equation" (arXiv:1706.09161),
 * Eqs. (FADE_moreGeneral) and (Fg).
 *
 * One handle = one problem (or one batch of independent problems) on one GPU.
 * The handle owns every device buffer it uses (populations, concentration,
 * fractional terms, weight matrices, tables, adjoint checkpoints).  It takes them,
 * in lbm_create / lbm_create_batch (and lbm_grad for the checkpoints), from the
 * device-memory hooks installed by lbm_set_allocator when the handle was created
 * (for example PyTorch's caching allocator), otherwise from cudaMalloc, and gives
 * them back the same way in lbm_destroy.  The caller owns every array passed in
 * (host or device); the library copies from / into it during the call and keeps
 * no pointer to it.
 *
 * Conventions
 *   - Grid: grid[mu] = nodes on axis mu including both wall nodes, so the axis
 *     spans n = 0..N_mu with N_mu = grid[mu]-1 (Section 2.4, Eq. XXminus_discret).
 *     Unused axes (3rd axis in 2-D) must be 1.
 *   - Field layout (host and device): axis 0 (x) fastest, i.e. index
 *     x + grid[0]*(y + grid[1]*z).  Population arrays are [q][node] (SoA),
 *     q = 0..Q-1 in the velocity order of Section 2.1: e_0 = 0, e_{1,2} = +-x,
 *     e_{3,4} = +-y, e_{5,6} = +-z.
 *   - All host-side numbers are double precision.
 *
 * Errors: every function returns 0 (LBM_OK) or a negative code; nothing aborts
 * the process.  Launches are asynchronous on the handle's stream; errors raised
 * on the device (non-finite concentration, a bounded wait that gave up) are latched
 * and returned by the next synchronising call (lbm_sync, lbm_read_*, lbm_mass).
 *
 * Problems: a handle made by lbm_create holds one problem (index 0); one made by
 * lbm_create_batch holds nprob problems (indices 0..nprob-1).  The accessors that
 * take `prob` (lbm_read_C, lbm_mass, lbm_batch_set_C) return LBM_EINVAL for an index
 * outside that range.
 */
#ifndef LBM_FADE_H
#define LBM_FADE_H

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK            0
#define LBM_EINVAL       -1  /* invalid argument: see lbm_create for the admissible ranges */
#define LBM_ENOMEM       -2  /* device allocation failed */
#define LBM_ECUDA        -3  /* a CUDA runtime call failed (message via lbm_last_cuda_error) */
#define LBM_ERR_UNSTABLE -4  /* a non-finite concentration appeared during lbm_step */
#define LBM_ENOTSUP      -5  /* combination not supported by this build */
#define LBM_ERR_TIMEOUT  -6  /* a bounded device-side wait (tensor-core pipeline) gave up */
#define LBM_ETOOBIG      -7  /* input larger than a fixed-capacity (static) scratch area */

typedef struct lbm_s* lbm_t;

enum { LBM_D2Q5 = 0, LBM_D3Q7 = 1 };                 /* lattices of Section 2.1 */
enum { LBM_BGK = 0, LBM_MRT = 1 };                   /* Eq. (LBE_Ket) / Eq. (MRT-Coll) */
enum {
  LBM_FP64 = 0,            /* every stage in FP64 */
  LBM_FP32 = 1,            /* FP32 collision/streaming, FP32 fractional operator */
  LBM_FP32_BF16SPLIT = 2,  /* FP32 collision, fractional operator on tensor cores with
                              bf16 hi+lo operands (3 products), FP32 accumulation */
  LBM_FP32_TF32SPLIT = 3,  /* FP32 collision, fractional operator on tensor cores with
                              tf32 hi+lo operands (3 products; the operator splits C
                              into hi + lo in shared memory), FP32 accumulation */
  LBM_FP32_BF16SPLIT5 = 4, /* as LBM_FP32_BF16SPLIT with K_mu in three bf16 parts
                              k1+k2+k3 and C in two, five products (k1c1, k1c2, k2c1,
                              k2c2, k3c1): the weights' rounding, which the three-product
                              form carries into every step, drops to the FP32 level.
                              Operator plans with 64- or 128-column tiles (per tile, or
                              persistent with 128); single problems and batches. */
  LBM_FP32_BF16SPLIT6 = 5  /* as LBM_FP32_BF16SPLIT5 with C in three bf16 parts as well
                              (c1+c2+c3 = C exactly in FP32), six products (adds k1c3):
                              the operator's operands carry FP32's precision, so the form
                              matches the plain FP32 form's accuracy.  Same plans as
                              LBM_FP32_BF16SPLIT5. */
};

enum { LBM_VARIANT_FG = 0, LBM_VARIANT_CAPUTO = 1 };  /* Eq. (Fg) / Eq. (Fg2) */

typedef struct {
  int lattice;        /* LBM_D2Q5 or LBM_D3Q7 */
  int collision;      /* LBM_BGK or LBM_MRT */
  int precision;      /* LBM_FP64, LBM_FP32, LBM_FP32_BF16SPLIT, LBM_FP32_TF32SPLIT,
                         LBM_FP32_BF16SPLIT5, LBM_FP32_BF16SPLIT6 */
  int grid[3];        /* nodes per axis incl. walls, >= 3 on used axes, 1 on unused axes */
  double alpha[3];    /* fractional order per axis, in ]1,2] (Eq. FADE_moreGeneral) */
  double p[3];        /* weight of the left integral I+, in [0,1] (Eq. Fg) */
  double g[3];        /* positive constant factor g_mu (Eq. Fg) */
  double D[9];        /* d x d diffusion tensor, row-major (stride 3 in memory: D[3*i+j]).
                         BGK: diagonal (non-spherical handled by h_mu, end of Section 2.2);
                         MRT: symmetric, lambdabar = D dt/(e^2 dx^2) + Id/2 must be SPD (Eq. D_ab) */
  double u[3];        /* advection velocity (physical units; the scheme uses u dt/dx, Eq. Feq) */
  double s_free[3];   /* MRT relaxation rates 1/lambda_k of the free moments k = d+1..Q-1
                         (Eq. MatrixS; D2Q5 uses 2, D3Q7 uses 3), each in ]0,2[ */
  double dx, dt;      /* space and time steps (> 0) */
  double C_wall;      /* Dirichlet concentration imposed on every wall node (Eq. Dirichlet_BC) */
  int variant;        /* LBM_VARIANT_FG: equilibrium moment F of Eq. (Fg), the Riemann-Liouville
                         form; LBM_VARIANT_CAPUTO: F~ of Eq. (Fg2) (Section 3.5), each integral
                         less its boundary term f(end) (distance)^gamma / Gamma(1+gamma), which
                         gives the Caputo-type FADE of Eq. (Fg22) and admits uniform equilibria.
                         Zero-initialised parameters select LBM_VARIANT_FG. */
} lbm_params;

/* Create a problem and initialise it from C0.
 *   prm      : problem description (copied).
 *   C0_host  : initial concentration, grid[0]*grid[1]*grid[2] doubles (host).
 *   out      : receives the handle.
 *   stream   : cudaStream_t to run on, or NULL to let the handle create its own
 *              non-blocking stream (destroyed with the handle).
 * The initial populations are the equilibrium of C0 (Algorithm 1, initialisation;
 * f(x,0) is not stated by the paper, this is the reading taken).
 * Weight matrices (Section 2.4, Eqs. c+ and c-) are built on the host in FP64.
 * Returns LBM_EINVAL for alpha outside ]1,2], p outside [0,1], g <= 0, dx or dt <= 0,
 * a grid axis < 3, BGK with off-diagonal D, a non-SPD lambdabar, free rates outside
 * ]0,2[; LBM_ENOMEM / LBM_ECUDA on device failures (no handle is returned then). */
int lbm_create(const lbm_params* prm, const double* C0_host, lbm_t* out, void* stream);

/* Device-memory hooks.  A handle created after this call takes every device buffer it
 * owns (populations, C, F, operands, weights, tables, adjoint checkpoints) from
 * alloc(bytes, stream, ctx), with `stream` the handle's stream, and returns it through
 * release(ptr, ctx) when it no longer needs it (after synchronising its stream).  alloc
 * returns NULL when it cannot serve the request (the creating or stepping call then
 * returns LBM_ENOMEM) and a pointer aligned to at least 256 bytes otherwise.  Each
 * handle keeps the hooks it was created with.  Both NULL restores cudaMalloc/cudaFree;
 * exactly one NULL returns LBM_EINVAL.  Process-wide; the hooks must stay callable until
 * the last handle created with them is destroyed.  This is how a host framework that
 * owns the GPU memory (e.g. PyTorch's caching allocator) lends it to the library. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*lbm_free_fn)(void* ptr, void* ctx);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void* ctx);

/* A batch of nprob independent problems advanced together (each one is the scheme of
 * Algorithm 1, exactly as lbm_create would run it).  All problems share lattice,
 * collision and precision (LBM_FP32 or a bf16 split form: LBM_FP32_BF16SPLIT, _BF16SPLIT5,
 * _BF16SPLIT6); grids and every other
 * parameter may differ.  prms[i] and C0_host[i] (host array of the problem's nodes)
 * describe problem i.  One time step is one grouped tensor-core launch covering every
 * problem's tiles (FP32: one SIMT launch per problem and axis) and one grouped
 * collide-stream launch covering every problem's nodes.  On a batch handle lbm_step,
 * lbm_reset, lbm_sync, lbm_profile, lbm_get_stream, lbm_launches_per_step and
 * lbm_destroy act on all problems; lbm_read_C, lbm_mass and lbm_batch_set_C take the
 * problem's index; the other single-problem accessors return LBM_EINVAL.
 * Errors: LBM_EINVAL for mixed lattices/collisions/precisions or any invalid problem,
 * LBM_ENOTSUP for other precisions, LBM_ENOMEM / LBM_ECUDA as lbm_create. */
int lbm_create_batch(int nprob, const lbm_params* prms, const double* const* C0_host, lbm_t* out, void* stream);

/* Number of problems of a handle (1 for a single-problem handle). */
int lbm_batch_size(lbm_t h, int* nprob);

/* Re-initialise problem `prob` from a new concentration (host doubles), as lbm_set_C. */
int lbm_batch_set_C(lbm_t h, int prob, const double* C_host);

/* Re-initialise the populations from a new concentration field (host, same layout
 * as lbm_create): f = feq(C, F(C)); clears any latched device error.  Asynchronous w.r.t. the device; the host
 * array may be reused as soon as the call returns. */
int lbm_set_C(lbm_t h, const double* C_host);

/* Restart from the concentration last given to lbm_create or lbm_set_C, which the
 * handle keeps on the device: f = feq(C0, F(C0)), and clear any latched device
 * error.  No host transfer; asynchronous. */
int lbm_reset(lbm_t h);

/* Advance nsteps >= 0 time steps (Algorithm 1's time loop): fractional
 * terms F_mu (Section 2.4), equilibrium (Eqs. Feq, CoeffA_FADE3D), BGK/MRT collision
 * (Eqs. LBE_Ket, MRT-Coll), push streaming (Eq. Def_Translation), Dirichlet walls
 * (Eq. Dirichlet_BC; k unknown populations at edges/corners share the deficit
 * equally), new concentration C = <1|f>.  Asynchronous; steps are replayed from
 * captured CUDA graphs. */
int lbm_step(lbm_t h, int nsteps);

/* Current concentration C = <1|f> of problem `prob` (the moment of Algorithm 1's time step), as
 * that problem's grid[0]*grid[1]*grid[2] doubles in the field layout above, written to
 * dst: a host array (dst_is_device = 0) or a device array of the handle's GPU
 * (dst_is_device != 0; converted to FP64 on the device, no host round trip), owned by
 * the caller.  Synchronises the handle's stream; returns that problem's latched
 * LBM_ERR_UNSTABLE or LBM_ERR_TIMEOUT if one was raised (the data is copied even then);
 * LBM_EINVAL for a null dst or a bad problem index. */
int lbm_read_C(lbm_t h, int prob, void* dst, int dst_is_device);

/* Fractional term F_mu (mu = 0..d-1) of the current concentration,
 * F_mu = p I+(g h C) + (1-p) I-(g h C) discretised by Eq. (XXminus_discret),
 * recomputed by the step's own operator and copied to F_host (nodes doubles).
 * Synchronises. */
int lbm_read_F(lbm_t h, int mu, double* F_host);

/* Copy / overwrite the populations, Q*nodes doubles laid out [q][node] (host).
 * lbm_write_f also recomputes C = <1|f> (and the split operands of the tensor-core
 * forms).  Both synchronise. */
int lbm_read_f(lbm_t h, double* f_host);
int lbm_write_f(lbm_t h, const double* f_host);

/* Checkpoint and resume.  The paper has no counterpart: by Algorithm 1 the
 * populations f alone determine the rest of a run, so the state is the current f of
 * every problem of the handle (single or batched), bit for bit in the working
 * precision, after a header (magic, version, lattice, precision, problem count and
 * grids).
 *   lbm_state_size: bytes that lbm_save writes (> 0), or LBM_EINVAL for a null handle.
 *   lbm_save: writes the state into dst_host (caller-owned, `bytes` long; LBM_EINVAL
 *             if smaller than lbm_state_size).  Synchronises.
 *   lbm_load: restores a state saved from a handle with the same lattice, precision
 *             and grids (LBM_EINVAL otherwise, handle unchanged); recomputes C and the
 *             split operands and clears the latched instability flag.  Synchronises.
 * Saving, stepping k times, loading and stepping k times again gives bit-identical
 * populations. */
/* Launch-configuration autotuning (no counterpart in the paper): times nsteps steps
 * (graph replay, after nsteps warm-up steps) of each candidate configuration on the
 * handle's own data and keeps the fastest:
 *   tensor-core forms, single problem: the operator's column tile width (64, 128, 256),
 *     its contraction split (1, 2, 4, 8 partial sums) or the persistent kernel;
 *   FP32 form, single problem: the SIMT operator's contraction split (1, 2, 4, 8);
 *   every handle: collide-stream tile rows per block (2-D) or z chunks (3-D);
 *   batches: tile rows per block of every 2-D member.
 * The operator plan is searched first with the current collide-stream setting, then the
 * collide-stream setting with the best plan; 2-D bf16 plans are also tried as a fused
 * step (operator and collide-stream phases of many steps in one cooperative launch,
 * separated by bounded grid barriers).  The populations are restored bit for bit
 * afterwards (as lbm_save / lbm_load), so tuning does not advance the run.  desc, if
 * not NULL, receives up to desc_len bytes describing the choice.  nsteps in
 * [2, 100000] (rounded up to whole graph replays: 128 steps, 32 for batches), else
 * LBM_EINVAL.  Synchronises. */
int lbm_autotune(lbm_t h, int nsteps, char* desc, int desc_len);

/* Apply a launch configuration directly (for example one lbm_autotune found before):
 * bn > 0 sets the tensor-core operator plan (bn in {64, 128, 256}, ks in {1, 2, 4, 8},
 * persist 0/1; combinations the kernels do not cover give LBM_EINVAL), bn = 0 keeps it;
 * chunk > 0 sets the collide-stream tile rows (2-D) or z chunks (3-D), 0 the built-in
 * choice; fused = 1 runs whole steps in one cooperative kernel (2-D bf16 split with a
 * per-tile plan of 64/128 columns split 2 or 4, rows TMA can address; LBM_ENOTSUP
 * otherwise).  FP32 single problems take ks > 0 as the SIMT operator's contraction split
 * (1, 2, 4, 8, at most the 32-wide contraction blocks of the shortest axis) with
 * bn = persist = fused = 0; other non-tensor-core handles accept only
 * bn = ks = persist = fused = 0.  Synchronises when the split needs a larger F. */
int lbm_configure(lbm_t h, int bn, int ks, int persist, int chunk, int fused);

long long lbm_state_size(lbm_t h);
int lbm_save(lbm_t h, void* dst_host, long long bytes);
int lbm_load(lbm_t h, const void* src_host, long long bytes);

/* Total mass sum_x C(x) of problem `prob`'s current concentration (the moment of
 * Algorithm 1's time step), in FP64, into the host double *mass.  After a step the mass is a by-product
 * of the collide-stream kernel: each warp of its blocks sums the concentrations it wrote
 * (FP32 forms: per thread and across the warp as a compensated two-float sum, stored as
 * that pair; FP64: in FP64) and stores one partial; this call adds the partials of the
 * latest step in FP64 in one small pass (a fixed order: the same result every time).  Right after lbm_create,
 * lbm_set_C, lbm_reset, lbm_write_f or lbm_load it reduces C itself (block partials,
 * then one final pass).  Synchronises; returns the problem's latched error as
 * lbm_read_C does. */
int lbm_mass(lbm_t h, int prob, double* mass);

/* Mass check for instability detection (the paper has no counterpart; Section 3.3
 * reports the scheme's instability at high Peclet number).  With limit > 0, every
 * synchronising call (lbm_sync, lbm_read_*, lbm_mass) first adds the latest step's mass
 * partials and latches LBM_ERR_UNSTABLE when that mass is not finite or its magnitude
 * exceeds `limit` (a run whose mass explodes, positive or negative); the check costs one
 * small launch per synchronising call and nothing per step.  limit = 0 (the default)
 * turns the check off; a non-finite concentration is latched in any case.  Applies to
 * every problem of the handle.  LBM_EINVAL for a negative or non-finite limit. */
int lbm_set_mass_limit(lbm_t h, double limit);

/* Coefficients that vary in space (Section 1: the scheme is meant for a diffusion tensor D
 * and factors g that depend on x; Eq. (Fg) with g_mu(x) multiplying C inside the integrals,
 * Eqs. (MatrixS), (D_ab) with lambda_{mu nu}(x), Eq. (Feq) with u(x)).  Each argument is a
 * host array of the handle's nodes (field layout above), or NULL for the constant value of
 * lbm_params at every node:
 *   D_field: d*d*nodes doubles, entry (a, b) of node i at D_field[(a*d + b)*nodes + i];
 *            symmetric, lambdabar(x) = D(x) dt/(e^2 dx^2) + Id/2 SPD at every node (MRT);
 *            BGK needs D(x) spherical at every node (one relaxation time lambda(x), Eq.
 *            Diffusion_Coefficient_3D; the constant-D h_mu trick does not apply);
 *   g_field: d*nodes doubles (g_mu(x) > 0 at g_field[mu*nodes + i]);
 *   u_field: d*nodes doubles (u_mu(x), physical units).
 * All three NULL returns to the constant coefficients.  The step then collides in moment
 * space with the rates of each node and the operator contracts g_mu(x) C along each axis;
 * the handle re-initialises from its initial concentration (as lbm_reset).  The arrays are
 * copied.  Single-problem handles (LBM_EINVAL for batches) in every precision form.  On the
 * tensor cores g(x) enters as one operand g_mu(x) C per axis (K_mu then without g): bf16
 * parts of it, or for tf32 the FP32 product (split into hi + lo by the operator); a
 * uniform g stays folded into K_mu; with BGK the tensor-core forms need a spherical
 * constant D (LBM_ENOTSUP).
 * LBM_EINVAL for a non-finite entry, g <= 0 or a D that breaks the conditions above (the
 * handle is unchanged then).  lbm_grad returns LBM_ENOTSUP on a handle with varying
 * coefficients.  Synchronises. */
int lbm_set_fields(lbm_t h, const double* D_field, const double* g_field, const double* u_field);

/* Source term S_c(x, t) = S(x) exp(rate t) of Eq. (FADE_moreGeneral), added after the collision
 * as w_i S_c(x, t) dt (Eqs. LBE_FADE, LBE_Ket, MRT-Coll) with t the time at the start of the
 * step (t = n dt after n steps since the last re-initialisation; the exponential form covers
 * Section 3.4's exact solution, S_c = -(d+1) exp(-t) prod x_mu^a_mu).  S_field: host array of
 * the handle's nodes (copied), or NULL to remove the source.  rate finite.  Runs the step on
 * the per-node path (as lbm_set_fields, constant coefficients unless set), re-initialises from
 * the initial concentration (as lbm_reset, time 0).  The time is carried by the step counter
 * (lbm_save / lbm_load keep it).  Single problems in every precision form (LBM_EINVAL for
 * batches; the tensor-core forms as for lbm_set_fields); LBM_EINVAL for a non-finite value.
 * Synchronises; every
 * lbm_step call of a handle with a time-dependent source or wall values waits for the
 * handle's earlier work once per 128 steps (it copies that range's time factors). */
int lbm_set_source(lbm_t h, const double* S_field, double rate);

/* Dirichlet values that vary with position and time, C_0(x, t) = C_w(x) exp(rate t) on every
 * wall node (Eq. Dirichlet_BC, Section 2.5: the same update with C_0 depending on x and t;
 * Section 3.4 takes them from the exact solution), imposed after the step that ends at time t.
 * Cw_field: host array of the handle's nodes (only the wall nodes are read), or NULL for the
 * constant C_wall of lbm_params.  Otherwise as lbm_set_source. */
int lbm_set_wall_values(lbm_t h, const double* Cw_field, double rate);

/* New constant parameters for an existing single-problem handle: alpha, p, g, D, u, s_free,
 * dx, dt and C_wall may change; lattice, collision, precision, grid and variant may not
 * (LBM_EINVAL).  The weights (Section 2.4) and the collision constants (Eqs. MatrixS, D_ab,
 * Diffusion_Coefficient_3D) are rebuilt in place, the device buffers, the launch plan and any
 * coefficient fields, source or wall values are kept, and the handle re-initialises from its
 * initial concentration (as lbm_reset).  This is how a fit of the parameters (lbm_grad in a
 * loop) avoids a new handle per evaluation.  LBM_EINVAL for inadmissible parameters (as
 * lbm_create; the handle keeps the old ones then), LBM_ENOTSUP as lbm_set_fields for the
 * tensor-core forms.  Synchronises. */
int lbm_set_params(lbm_t h, const lbm_params* prm);

/* Killed stable-Levy random walk (Section 3.1: Eqs. RW_STABLE and distri; the bounded-domain
 * subsection: a path is killed at its first exit from the box), the paper's Monte-Carlo
 * counterpart of the scheme.  The density of the live paths solves the FADE with
 * D'_mumu = (D_mumu g_mu)^(1/alpha_mu), beta_mu = 2 p_mu - 1 and C = 0 on the box's walls. */
typedef struct {
  int d;                    /* 2 or 3 */
  int precision;            /* LBM_FP64: FP64 arithmetic, uniforms (o + 1/2) 2^-32;
                               LBM_FP32: FP32 arithmetic, uniforms ((o >> 9) + 1/2) 2^-23
                               (exact in FP32) */
  double alpha[3];          /* ]1,2] per axis */
  double p[3];              /* [0,1] per axis (skewness beta = 2p - 1) */
  double D[3], g[3];        /* > 0 per axis */
  double u[3];              /* drift per axis */
  double lo[3], hi[3];      /* the box ]lo, hi[ */
  double dt;                /* > 0 */
  unsigned long long seed;  /* Philox4x32-10 key */
} lbm_walk_params;

/* Advance n paths by nsteps increments, steps step0 .. step0 + nsteps - 1 of their draws
 * (Philox4x32-10, counter (i mod 2^32, i div 2^32, step, call), key = seed: a run split over
 * several calls gives the same paths as one call).  S(alpha, beta) from two uniforms by
 * Chambers-Mallows-Stuck / Weron (1996).
 *   X:     device array of d*n doubles, [mu][i] (in/out); a killed path keeps its exit position
 *   alive: device array of n bytes (in/out): paths with 0 are not moved; a path that leaves the
 *          box gets 0
 * Both caller-owned (the call allocates nothing).  Asynchronous on `stream` (NULL: legacy
 * default).  LBM_EINVAL for parameters outside the ranges above, n < 0, nsteps < 0, step0 < 0
 * or step0 + nsteps > 2^32 - 1; LBM_ECUDA if the launch fails. */
int lbm_walk(const lbm_walk_params* prm, long long n, double* X, unsigned char* alive, long long step0, int nsteps,
             void* stream);

/* Histogram of the live paths on a lattice: counts[node] (device, caller-owned, not cleared)
 * += the live paths whose position lies in the cell of width dx centred at the node, nodes at
 * lo + k dx, k = 0..grid[mu]-1, node index x fastest (field layout above).  With n paths the
 * density at a node is counts / (n dx^d).  Asynchronous; LBM_EINVAL for bad arguments. */
int lbm_walk_density(const lbm_walk_params* prm, long long n, const double* X, const unsigned char* alive,
                     const int* grid, double dx, unsigned int* counts, void* stream);

/* Wait for all work of the handle; return a latched device error if any. */
int lbm_sync(lbm_t h);

/* The cudaStream_t the handle runs on (for event timing by the caller). */
int lbm_get_stream(lbm_t h, void** stream);

/* Run nsteps time steps (0 <= nsteps <= 4096) with one-kernel launches bracketed by
 * CUDA events on the handle's stream and accumulate the device time of each kernel
 * class:
 *   ms[0] = fractional operator (all axes),
 *   ms[1] = fused collide/stream/walls/moment.
 * All steps are queued before one synchronisation, so the intervals exclude the host's
 * submission of each launch.  Divide by nsteps for the mean duration per launch.
 * LBM_EINVAL for nsteps outside that range.  Synchronises. */
int lbm_profile(lbm_t h, int nsteps, double* ms);

/* Number of kernel launches one time step issues (per problem batch) under the current
 * launch configuration; 0 for the fused small-problem step, which issues one launch
 * per lbm_step call of up to 4096 steps. */
int lbm_launches_per_step(lbm_t h, int* n);

/* Host-only: the (grid[mu])^2 FP64 matrix K_mu, row-major K[n*side + l], such that
 * F_mu[n] = sum_l K[n][l] C[l] along each lattice line of axis mu, i.e.
 * K = g h dx^gamma / Gamma(2+gamma) * (p W+ + (1-p) W-) with gamma = 2 - alpha
 * (Eqs. 1Dminus_discret, c+, c-).  W+ and W- hold 1 on the diagonal except at the
 * line's own end (W+ at n = 0, W- at n = N), where the integral runs over an empty
 * interval and the entry is 0 for alpha < 2.  With variant LBM_VARIANT_CAPUTO the
 * matrix is K - B (Section 3.5, Eqs. PSRLdD-a/b, Fg22): column 0 loses
 * g h p (n dx)^gamma / Gamma(1+gamma) and column N loses
 * g h (1-p) ((N-n) dx)^gamma / Gamma(1+gamma), so K~ maps constants to 0.  Needs no GPU. */
int lbm_frac_matrix(const lbm_params* prm, int mu, double* K_host);

/* FP64 sum of n device values (elem_bytes 4: float, 8: double) written to *sum_dev,
 * a caller-owned device double, asynchronously on `stream` (NULL: legacy default).
 * The paper has no counterpart: this is the lbm_mass reduction for callers that
 * cannot allocate device memory -- plug-ins running inside a host framework that
 * owns all GPU memory and hands out only pointers, and code that must not call
 * cudaMalloc because an allocation can synchronise the device.  It calls no
 * cudaMalloc, cudaFree or allocating library routine: its partial sums live in a
 * static device array of 65,536 doubles (512 KiB) that every GPU which loads this
 * library holds until the process exits.  n may be at most 67,108,864
 * (65,536 partials of 1,024 elements); larger n returns LBM_ETOOBIG, n < 0 or a
 * bad pointer / elem_bytes returns LBM_EINVAL.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is cached for the
 * life of the process: after a cudaDeviceReset of that device in the same process
 * the cached address is stale and the entry point must not be called again.  All
 * calls share the one
 * array, which keeps the last call's partials: each call overwrites every
 * partial it reads, and calls that overlap on the GPU (different streams, no
 * ordering between them) race on it and must be serialised by the caller. */
int lbm_mass_static(const void* x_dev, int elem_bytes, long long n, double* sum_dev, void* stream);

/* Check of the bounded device-side wait behind LBM_ERR_TIMEOUT (the paper has no
 * counterpart).  Every pipelined kernel waits on shared-memory barrier phases (TMA
 * completions, MMA commits, the fused step's grid barrier) with a %globaltimer limit;
 * a wait that gives up sets the timeout bit of the handle's status word and the kernel
 * runs to its end, so the next synchronising call returns LBM_ERR_TIMEOUT and the CUDA
 * context stays usable.  This runs that same wait, in one block on `stream` (NULL:
 * legacy default), on a barrier whose phase is completed first (complete != 0: returns
 * LBM_OK) or never (complete == 0: the wait gives up after limit_us microseconds and
 * the call returns LBM_ERR_TIMEOUT).  limit_us in [1, 1000000], else LBM_EINVAL.
 * Allocates and frees one device int; synchronises the stream. */
int lbm_wait_check(int complete, int limit_us, void* stream);

/* Loss and gradient of a snapshot misfit (the inverse problem):
 *   L(theta) = sum_k sum_x ( C(x, t_k) - obs_k(x) )^2,
 * C from the scheme started at the handle's initial concentration (lbm_create /
 * lbm_set_C) with the handle's parameters theta; grad receives 4d doubles,
 * dL/d[alpha_1..d, p_1..d, D_11..D_dd, u_1..d] (D: diagonal entries, physical units).
 * Computed with the discrete adjoint of the step (the exact transpose of Algorithm 1's
 * time step for fixed theta: walls, streaming, collision, equilibrium, K_mu^T),
 * parameter derivatives of K_mu (lbm_frac_matrix_grad), of Omega (Eqs. MatrixS, D_ab)
 * and of the advective equilibrium term (Eq. Feq), including the initial populations
 * feq(C0, K C0).  Forward states are recomputed from checkpoints taken every
 * ckpt_every steps (memory: ckpt_every + T/ckpt_every states); sums are FP64.
 *   snap_steps : nsnap strictly increasing step indices >= 0 (the last one is T)
 *   obs        : nsnap x nodes host doubles (field layout as lbm_create)
 * BGK and MRT single-problem handles with constant coefficients (LBM_ENOTSUP for batches and
 * lbm_set_fields / lbm_set_source handles).  On the split-precision forms the gradient is
 * that of the plain FP32 scheme (which those forms follow within their stated error),
 * computed on an FP32 copy of the problem that the call creates and frees (same stream and
 * device-memory hooks, started from the handle's initial concentration).  BGK:
 * Omega = I / lambda with lambda from the largest D_mumu and K_mu scaled by
 * h_mu = D_mumu / max D (end of Section 2.2), so dL/dD_mumu includes both dependences;
 * where several D_mumu share the maximum, each takes an equal part of d(max D) (the
 * average of the one-sided derivatives).  Synchronises; leaves the handle reset to its
 * initial state. */
int lbm_grad(lbm_t h, int nsnap, const int* snap_steps, const double* obs, int ckpt_every, double* loss,
             double* grad);

/* Host-only: derivatives of K_mu (as lbm_frac_matrix) with respect to alpha_mu and
 * p_mu, FP64, row-major (grid[mu])^2 each.  With gamma = 2 - alpha:
 * dK/dp = s (W+ - W-), dK/dalpha = -d/dgamma [ s (p W+ + (1-p) W-) ],
 * s = g h dx^gamma / Gamma(2+gamma), ds/dgamma = s (ln dx - psi(2+gamma))
 * (Eqs. 1Dminus_discret, c+, c- differentiated in gamma); with LBM_VARIANT_CAPUTO the
 * boundary terms' derivatives are included (d/dgamma of x^gamma / Gamma(1+gamma) is
 * x^gamma (ln x - psi(1+gamma)) / Gamma(1+gamma)).  Needs no GPU. */
int lbm_frac_matrix_grad(const lbm_params* prm, int mu, double* dK_dalpha, double* dK_dp);

/* Host-only: digamma psi(x), x > 0 (recurrence + asymptotic series, Abramowitz &
 * Stegun 6.3.5 / 6.3.18), used by lbm_frac_matrix_grad. */
double lbm_digamma(double x);

/* Release every device buffer, graph and (if created by the handle) stream. */
void lbm_destroy(lbm_t h);

/* Static description of an error code. */
const char* lbm_strerror(int code);

/* Text of the last CUDA error seen by this thread's library calls ("" if none). */
const char* lbm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_FADE_H */
