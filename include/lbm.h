/*
 * lbm.h -- C ABI of the GB300 pseudo-potential wetting lattice-Boltzmann engine.
 *
 * The engine advances the mesoscopic wetting model of Colosqui, Kavousanakis,
 * Papathanasiou & Kevrekidis (arXiv:1202.6130), Sec. II: per time step and per
 * lattice node it pulls the populations (streaming), forms rho and j
 * (Eqs. M0, M1), the pseudo-potential psi (Eq. EOS or the exponential form),
 * the fluid-fluid force (Eq. force_SC), the long-range fluid-solid force and
 * the short-range wall momentum exchange weighted by the wall probability
 * (Eqs. force_SC_FS, pseudopotential, wall_shift), then relaxes with BGK plus
 * the exact-difference-method forcing (Eq. BE-BGK, Sec. II B).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an int status (LBM_OK or a negative LBM_E* code) and
 *     never throws across the ABI.  After LBM_ECUDA the context is poisoned:
 *     later calls except lbm_destroy / lbm_last_error return LBM_ESTATE.
 *   - Host arrays are row-major [y][x] (x fastest, y = 0 at the bottom) in
 *     FP64; population arrays are [i][y][x] with i in the lattice table order
 *     (D2Q9: rest, (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1);
 *     D2Q21: Table I order, states 1-4 axes speed 1, 5-8 diagonals, 9-12 axes
 *     speed 2, 13-16 (+-2,+-2), 17-20 axes speed 3, 21 rest; counter-clockwise
 *     from +x inside each group).
 *   - The caller owns every host buffer; the engine copies what it needs
 *     during the call and keeps no pointer to it.  The context owns all device
 *     memory, obtained from the caller's lbm_allocator if one is given, else
 *     from cudaMalloc.
 *   - The lattice is fully periodic in x and y.  The solid exists only through
 *     the wall fields of lbm_set_wall (a wall "at y = 0" is a slab across the
 *     periodic seam).
 *   - A population f_i(x, t) given to or returned by the engine is the value
 *     just after streaming, before collision, at time t.
 *   - Work is enqueued on the context's CUDA stream.  lbm_step returns after
 *     enqueueing (unless a periodic check is due); calls that fill host
 *     buffers synchronise the stream.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Device-memory provider.  alloc returns a device pointer aligned to at least
 * 256 bytes, or NULL on failure (the engine then returns LBM_ENOMEM); free
 * releases it.  Both may be called from any engine entry point. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} lbm_allocator;

enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,     /* bad argument: null pointer, size, tau <= 0.5, ... */
  LBM_ENOMEM = -2,     /* the allocator returned NULL */
  LBM_ECUDA = -3,      /* a CUDA call failed; the context is poisoned */
  LBM_ESTATE = -4,     /* call not valid in this state (poisoned, no populations) */
  LBM_ENONFINITE = -5, /* a periodic check found a non-finite density */
  LBM_ETIMEOUT = -6    /* a bounded device-side wait gave up */
};

enum { LBM_D2Q9 = 9, LBM_D2Q21 = 21 };

/* Population storage.  FP16S / BF16S store the deviation from the shift
 * w_i rho_s in 16 bits, h_i = sigma (f_i - w_i rho_s), where rho_s is
 * shift_rho rounded to FP32 and sigma = 2^8 for FP16S (|f_i - w_i rho_s| < 256,
 * beyond which the stored value becomes inf and the non-finite check reports
 * it) and 1 for BF16S.  All arithmetic of the step is FP32 and works on h
 * directly (rho = sum_i h_i / sigma + rho_s, j = sum_i h_i c_i / sigma; the
 * collision maps deviations to deviations); set-up and read-out convert
 * between f and h in FP64.  The step rounds
 * the stored deviations stochastically by default (LBM_ROUND_STOCHASTIC: the
 * expectation of the stored value is the FP32 value; the random bits are a
 * counter-based hash of the node and the step, so runs are reproducible and a
 * lattice gives the same bits alone and in a batch) or to nearest-even
 * (LBM_ROUND_NEAREST).  Initial populations are encoded to nearest-even. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16S = 2, LBM_BF16S = 3 };
enum { LBM_ROUND_STOCHASTIC = 0, LBM_ROUND_NEAREST = 1 };

/* Pseudo-potential psi(rho):
 *   LBM_PSI_EXP: rho0 * (1 - exp(-rho / rho0))          (Shan-Chen form)
 *   LBM_PSI_EOS: sqrt(2 (rho theta - p_EOS(rho)))       (Sec. II, Eq. EOS)  */
enum { LBM_PSI_EXP = 0, LBM_PSI_EOS = 1 };

/* The problem statement of Sec. II: lattice, relaxation time tau (Eq. BE-BGK),
 * fluid-fluid coupling, equation of state, body force.  The fluid-fluid force
 * is F_FF = -G psi(x) sum_i w_i psi(x + r_i) r_i (Eq. force_SC); the paper's
 * EOS fluid corresponds to G = -1/theta. */
typedef struct {
  int32_t nx, ny;        /* lattice size, >= 1 each */
  int32_t lattice;       /* LBM_D2Q9 or LBM_D2Q21 */
  int32_t storage;       /* LBM_FP64 .. LBM_BF16S */
  int32_t psi_kind;      /* LBM_PSI_EXP or LBM_PSI_EOS */
  int32_t project;       /* 1: projection step (Sec. II, after Eq. f2) before collision */
  double tau;            /* > 0.5 */
  double G;              /* fluid-fluid coupling */
  double rho0;           /* LBM_PSI_EXP scale, > 0 */
  double eos_theta_v;    /* Eq. EOS slopes (absolute, not divided by theta) */
  double eos_theta_u;
  double eos_theta_l;
  double eos_rho1;       /* Eq. EOS knots rho_1 < rho_2 */
  double eos_rho2;
  double body_force[2];  /* uniform force density added on every node */
  double shift_rho;      /* FP16S/BF16S shift; <= 0: mean initial density */
  int32_t check_every;   /* lbm_step checks for non-finite rho every K steps; 0 = never */
  int32_t tile_rows;     /* rows per CTA strip segment; 0 = chosen by the engine */
  int32_t rounding;      /* FP16S/BF16S: LBM_ROUND_STOCHASTIC (default) or LBM_ROUND_NEAREST */
  int32_t reserved;      /* 0 */
} lbm_params;

/* Fills *p with defaults: D2Q9, FP32, exponential psi, tau 1, G -5.5, rho0 1,
 * the paper's EOS parameters scaled by theta = 1/3, no body force. */
int lbm_params_default(lbm_params* p);

/* Creates a context for one lattice with the problem statement of Sec. II
 * (lattice and its Table I weights, tau of Eq. BE-BGK, the fluid-fluid coupling
 * of Eq. force_SC, Eq. EOS, a uniform body force as in Sec. III A).  a may be
 * NULL (cudaMalloc is used); stream may be NULL (the legacy default stream).
 * The population state is undefined until lbm_set_populations or
 * lbm_set_equilibrium succeeds.  *out is NULL on error.  Errors: LBM_EINVAL
 * (p NULL, a size < 1, tau <= 0.5, an unknown lattice, storage, psi kind or
 * rounding), LBM_ENOMEM (the allocator returned NULL; every block already
 * obtained is returned to it), LBM_ECUDA. */
int lbm_create(const lbm_params* p, const lbm_allocator* a, void* cuda_stream, lbm_ctx** out);

/* Replaces the CUDA stream on which later calls enqueue work. */
int lbm_set_stream(lbm_ctx* c, void* cuda_stream);

/* Static wall fields (Sec. II "Fluid-Solid interactions", Eqs. force_SC_FS,
 * pseudopotential, wall_shift).  phi_s: wall probability phi_S; psi_r, psi_a:
 * the repulsive and attractive potentials psi_R-bar, psi_A-bar; each [ny][nx],
 * NULL meaning identically 0.  The fluid-solid pseudo-potential is
 * psi_FS = G_A psi_A-bar - G_R psi_R-bar (G_R, G_A >= 0 are strengths: the core
 * repels, the tail attracts).  epsilon >= 1 is the exponent of phi_S^epsilon.
 * u_wall: [2][ny][nx] wall velocity (x plane then y plane) or NULL (solid at rest).
 * The engine precomputes phi_S^epsilon and S(x) = sum_i w_i psi_FS(x + r_i) r_i
 * on the device; the long-range force is then rho(x) S(x). */
int lbm_set_wall(lbm_ctx* c, const double* phi_s, const double* psi_r, const double* psi_a,
                 double G_R, double G_A, double epsilon, const double* u_wall);

/* Sets the populations f_i(x, t) from a host array [Q][ny][nx]. */
int lbm_set_populations(lbm_ctx* c, const double* f);

/* Sets f_i = f_i^eq(rho, u) (Eq. feqc, second-order Hermite form) plus an
 * optional perturbation dfi [Q][ny][nx] (NULL = none).  rho, ux, uy: [ny][nx]. */
int lbm_set_equilibrium(lbm_ctx* c, const double* rho, const double* ux, const double* uy,
                        const double* dfi);

/* Advances nsteps >= 0 time steps (one fused kernel launch per step): the
 * update of Sec. II per node -- streaming, Eqs. M0 and M1, psi (Eq. EOS or
 * the exponential form), F_FF (Eq. force_SC), F_FS and Delta F_S (Eqs.
 * force_SC_FS, wall_shift), the optional projection (after Eq. f2) and the
 * EDM-BGK collision (Eq. BE-BGK with the shifted-velocity equilibrium of
 * Sec. II B).  Returns after enqueueing, or LBM_ENONFINITE when check_every > 0
 * and a check found a non-finite density (the state is then kept as it was
 * after that step), or LBM_ETIMEOUT when a bounded device wait gave up.
 * Errors: LBM_EINVAL (nsteps < 0), LBM_ESTATE (no populations set yet, or a
 * poisoned context), LBM_ECUDA. */
int lbm_step(lbm_ctx* c, int64_t nsteps);

/* Reads rho (Eq. M0) and the reported velocity u = (j + F/2) / rho (j of Eq.
 * M1, F the total force of the step) of the current state into host arrays
 * [ny][nx] (any may be NULL).  Synchronises the stream.  Errors: LBM_ESTATE,
 * LBM_ECUDA. */
int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy);

/* As lbm_moments, but into DEVICE arrays of ny*nx doubles, enqueued on the
 * stream without synchronising. */
int lbm_moments_device(lbm_ctx* c, double* d_rho, double* d_ux, double* d_uy);

/* Reads the populations f_i(x, t) into a host array [Q][ny][nx].  Synchronises. */
int lbm_get_populations(lbm_ctx* c, double* f);

/* out[0] = sum rho, out[1..2] = sum (j + F/2) over the lattice, FP64 with
 * compensated (Neumaier) summation per thread.  Synchronises. */
int lbm_totals(lbm_ctx* c, double out[3]);

/* Steps taken since the populations were last set. */
int lbm_steps_done(const lbm_ctx* c, int64_t* out);

/* The context's clock, for checkpoint and resume: the steps taken since the
 * populations were last set, and the counter from which stochastic rounding
 * draws the random bits of the next step (16-bit storage: the bits are a hash
 * of the node and this counter).  lbm_get_clock also reports the shift
 * density rho_s of 16-bit storage (0 otherwise; rho_s may be NULL).  A
 * checkpoint is the populations (lbm_get_populations) plus these numbers.  To
 * resume, create a context with the same parameters and shift_rho = rho_s,
 * then lbm_set_populations and lbm_set_clock: it steps on bit for bit as the
 * original would have, in every storage (16-bit values survive the FP64 round
 * trip exactly).  No paper passage: state management of the library.
 * lbm_get_clock synchronises the stream.  Errors: LBM_EINVAL (null steps or
 * counter output, negative steps), LBM_ESTATE (no populations set),
 * LBM_ECUDA. */
int lbm_get_clock(lbm_ctx* c, int64_t* steps, uint32_t* rounding_counter, double* rho_s);
int lbm_set_clock(lbm_ctx* c, int64_t steps, uint32_t rounding_counter);

/* Waits for all work enqueued by this context. */
int lbm_sync(lbm_ctx* c);

/* Frees the context and its device memory (returned through the allocator it
 * came from); NULL is accepted.  Always LBM_OK.  No paper passage: resource
 * management of the library. */
int lbm_destroy(lbm_ctx* c);

/* Human-readable description of the last error on c ("" if none), owned by c.
 * lbm_last_error(NULL) reports errors of calls that had no context yet. */
const char* lbm_last_error(const lbm_ctx* c);

/* ---- test hook (failure detection; not part of the modelling API) -------- */

/* Test hook for failure detection: arms the next lbm_step so that every
 * shared-memory stage of its kernel expects 16 bytes more than its copies
 * deliver.  The stage waits then run out after wait_ms milliseconds (instead
 * of the normal 2 s bound), the kernel records a timeout in the context's
 * status word and returns, and lbm_sync (or a periodic check) reports
 * LBM_ETIMEOUT.  Nothing faults and the context stays usable; the populations
 * of that step are not valid, so set them again.  Covers one step. */
int lbm_debug_stall_next_step(lbm_ctx* c, int32_t wait_ms);

/* Layout facts for measurement: bytes per node per step that the population
 * traffic needs (2 Q s), the padded row pitch in elements, and the launch shape
 * (strip width, rows per CTA, grid) of the fused step. */
typedef struct {
  int64_t bytes_per_node;
  int64_t pitch;
  int32_t strip_width;
  int32_t tile_rows;
  int32_t grid_x, grid_y;
  int32_t stages;
  int32_t ghost_x, ghost_y;
  int64_t device_bytes;
} lbm_layout;
int lbm_get_layout(const lbm_ctx* c, lbm_layout* out);

/* ---- wall-function helpers (initialisation; FP64) ------------------------ */

/* Recursive Gaussian filter of the Appendix (Eq. iteration): G^(0) = 1 on the
 * solid nodes (solid[y*nx+x] != 0) and 0 elsewhere; each pass sets
 * G^(n)(x) = sum_i w_i G^(n-1)(x + r_i) on the periodic lattice and resets G to 1
 * on the solid nodes.  Outputs phi_S = G^(n_att), psi_R-bar = G^(n_rep),
 * psi_A-bar = G^(n_att) - G^(n_rep), each [ny][nx] host (any may be NULL).
 * Runs on the current CUDA device; 0 <= n_rep <= n_att. */
int lbm_wall_gaussian_filter(int32_t nx, int32_t ny, int32_t lattice, const uint8_t* solid,
                             int32_t n_rep, int32_t n_att, double* phi_s, double* psi_r,
                             double* psi_a);

/* Closed-form wall fields from a distance-to-solid map dist [ny][nx] and a
 * thickness per column (thickness[x], nx entries): phi_S = (1 - tanh((d - T/2)
 * / (T/4))) / 2, zeroed below phi_cut; psi_R-bar = exp(-d / lambda) -
 * exp(-core_cut / lambda) for d < core_cut, else 0; psi_A-bar = (1 + d)^-p -
 * (1 + tail_cut)^-p for d < tail_cut, else 0.  Host-only. */
int lbm_wall_core_tail(int32_t nx, int32_t ny, const double* dist, const double* thickness,
                       double core_lambda, double core_cut, double tail_exp, double tail_cut,
                       double phi_cut, double* phi_s, double* psi_r, double* psi_a);

/* ---- batches: many lattices advanced by shared launches --------------------- */

/* A batch advances several contexts (its members) together: every time step is
 * one launch of one fused kernel per chunk of up to 64 members (32 with FP64
 * storage), whose CTAs march
 * the chunk's (member, strip, segment) tiles, each launched as a programmatic
 * dependent of the chunk's previous step; the chunks run on streams forked
 * from the batch stream, and runs of 16 and of 2 consecutive steps are
 * captured once in CUDA graphs and replayed (the chunk streams join at the end
 * of each replay).  Members must share lattice and storage but may
 * differ in size and in every physical parameter.  Members stay owned by the
 * caller (destroy a member only after removing it), keep their own device
 * memory, and can still be read with lbm_moments and friends between batch
 * steps.  Stepping a member on its own, or changing its wall or stream,
 * between batch steps is allowed; the batch notices and rebuilds its tile
 * list.  The batch's own small descriptor arrays come from a (nullable)
 * allocator.  Graph capture needs a non-default stream; with a NULL stream
 * every step is a plain launch.  lbm_batch_step orders itself with the
 * members' own streams by events: it starts after work already enqueued on
 * them, and work enqueued on them afterwards waits for it.  Errors are
 * reported by lbm_batch_last_error. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(const lbm_allocator* a, void* cuda_stream, lbm_batch** out);
/* Adds c (populations set; same lattice and storage as the other members). */
int lbm_batch_add(lbm_batch* b, lbm_ctx* c);
int lbm_batch_remove(lbm_batch* b, lbm_ctx* c);
int lbm_batch_size(const lbm_batch* b, int32_t* n);
/* Kernel launches per batch time step: the number of member chunks (members
 * divided by 64, or by 32 with FP64 storage, rounded up; 0 for an empty
 * batch). */
int lbm_batch_launches_per_step(const lbm_batch* b, int32_t* n);
/* Tile shape: tile_rows rows per segment (0: each member's own choice) and
 * ctas persistent CTAs that deal the tiles round-robin (0: one CTA per tile). */
int lbm_batch_set_tiling(lbm_batch* b, int32_t tile_rows, int32_t ctas);
/* Advances every member by nsteps time steps; enqueued on the batch stream. */
int lbm_batch_step(lbm_batch* b, int64_t nsteps);
/* Times each candidate tiling (rows 4..64 x {one CTA per tile, one persistent
 * wave}) for steps_per_trial steps (plus 18 warm-up steps) on the members
 * themselves -- so they advance by those steps -- keeps the fastest, and
 * records it for the batch's size class (see lbm_batch_use_tuned).
 * Outputs may be NULL.  Synchronises the stream. */
int lbm_batch_autotune(lbm_batch* b, int32_t steps_per_trial, int32_t* best_tile_rows,
                       int32_t* best_ctas, double* best_ms_per_step);
/* The tiling lbm_batch_autotune last chose for a batch of the same lattice,
 * storage and size class (floor(log2) of the total node count and of the
 * member count), kept process-wide: when there is one, it becomes b's tiling
 * and *found = 1; otherwise b is unchanged and *found = 0.  Advances nothing,
 * so a batch whose members must not take extra steps (a serving loop) can use
 * a tiling tuned earlier on a similar batch.  Errors: LBM_EINVAL (found
 * NULL). */
int lbm_batch_use_tuned(lbm_batch* b, int32_t* found);
int lbm_batch_destroy(lbm_batch* b); /* NULL ok; members are untouched */
const char* lbm_batch_last_error(const lbm_batch* b);

/* ---- allocation-free reduction ------------------------------------------ */

/* Compensated (Neumaier) FP64 sums of up to three DEVICE arrays of n doubles
 * each (a, b, c; a NULL array sums to 0), written to the DEVICE array out[3]:
 * the same reduction lbm_totals applies to rho and j + F/2, offered to callers
 * that must not allocate device memory while they run: a real-time loop with a
 * fixed memory budget, code working inside a memory pool it does not own, or a
 * host framework that forbids cudaMalloc after start-up.  The paper has no
 * counterpart; this is a service of the library.
 *
 * It runs the kernels and block partition of lbm_totals (1024 blocks, merged
 * in block order), so the same arrays give the same bits, and it calls no
 * cudaMalloc / cudaFree and no allocating library routine: its partial sums
 * live in one fixed 48 KiB array in device memory, which every GPU that loads
 * the library holds until the process exits.  n has no limit beyond int64_t.
 * The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) once, with the device
 * current; with CUDA's default lazy module loading that first call is also
 * when the array and these kernels are loaded onto the device, which takes
 * device memory.  So make the first call on every device during start-up
 * (a call with n = 0 does it and writes zeros), before any stream capture and
 * before the point after which the caller may not allocate.  The cached
 * address belongs to the device's primary context: after that context is
 * reset (cudaDeviceReset or a primary-context reset by any component of the
 * process) this entry point must not be called again.  Work is enqueued
 * on cuda_stream (NULL = legacy default stream) and the call returns without
 * synchronising.  Every call on a device shares the one array, so calls whose
 * kernels overlap on the GPU (different streams, no ordering between them)
 * race and give wrong sums; calls on one stream are safe.  Errors: LBM_EINVAL
 * (out NULL or n < 0), LBM_ECUDA (launch failure). */
int lbm_reduce3_noalloc(const double* d_a, const double* d_b, const double* d_c, int64_t n,
                        double* d_out3, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
