/*
 * gbpme.h -- C ABI of the GB300 charge+dipole particle-mesh Ewald library (libgbpme.so).
 *
 * The library evaluates, for one periodic frame of N point charges q_i and point dipoles
 * mu_i at positions r_i, the electrostatic energy of the Ewald-split Coulomb interaction
 *
 *   E = E_recip + E_pair + E_self + E_background                                  (1)
 *
 *   E_recip      particle-mesh reciprocal energy, Section 2.3 of the paper:
 *                spline assignment of q and of the dipole bound charge (Eq.
 *                charge_dipole_assign), R2C FFT (Eq. fft), deconvolved Green's function
 *                G(k) C(n) (Eqs. green, Bk, influence), energy (Eq. energy_recip);
 *   E_pair       real-space erfc(alpha r)/r charge-charge, charge-dipole and
 *                dipole-dipole pair term over every periodic image within rcut (the
 *                conventional-Ewald complement of the mesh term);
 *   E_self       Eqs. self_q and self_mu;
 *   E_background -pi Q^2 / (2 V alpha^2), Q = sum q (zero for neutral frames).
 *
 * and its derivatives, and the vector-Jacobian product (adjoint) of those derivatives that
 * a force-matching loss (Eq. loss) needs. pme_forward_quad / pme_backward_quad and their batch
 * forms add point quadrupoles (the rank-2 channel), documented at their declarations.
 *
 * Conventions
 *   - Lengths in the caller's unit (Angstrom in the tests), charges in e, dipoles in e*length.
 *     Every energy and derivative is multiplied by opts.coulomb_k (default 1: Gaussian units).
 *   - box[9] is row-major with ROWS the lattice vectors a_x, a_y, a_z (Section 2.3.1).
 *   - Per-ion arrays are contiguous, in the caller's ion order: pos/mu/force/field [n][3]
 *     float32, q/phi [n] float32, field_grad [n][6] float32 ordered xx, yy, zz, xy, xz, yz.
 *   - Outputs are WRITTEN, never accumulated into.
 *   - Pointers to per-ion arrays and to energies may be device pointers or host pointers
 *     (pinned or pageable); the library asks the CUDA runtime which one it is and stages
 *     host arrays through plan-owned device buffers with cudaMemcpyAsync on the call's
 *     stream. Host outputs are complete when the stream is synchronised.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *     Calls are asynchronous on that stream. A plan must not be used by two calls that
 *     overlap in time (its scratch buffers are shared); use one plan per stream.
 *   - The plan owns all scratch (sorted ion records, meshes, spectra, cuFFT plans when it
 *     uses cuFFT), sized at creation for opts.max_ions ions. Nothing is allocated on the
 *     device by the compute calls.
 *
 * Errors: every function returns a pme_status. No exception crosses the ABI. The text of
 * the last error of a plan is returned by pme_last_error(). Non-finite inputs are detected
 * on the device and reported by pme_sync_status().
 */
#ifndef GBPME_H
#define GBPME_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PME_OK = 0,
  PME_ERR_ARG = 1,          /* invalid argument: null handle, n > max_ions, order not in
                               1..7, alpha <= 0, singular box, mesh dimension < order ... */
  PME_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
  PME_ERR_CUFFT = 3,        /* a cuFFT call failed */
  PME_ERR_NONFINITE = 4,    /* a NaN or Inf appeared in pos, q, mu or theta (device flag) */
  PME_ERR_UNSUPPORTED = 5,  /* option combination not implemented (e.g. finite surface eps) */
  PME_ERR_TIMEOUT = 6,      /* a bounded device-side wait expired */
  PME_ERR_NOMEM = 7,        /* device allocation failed at plan creation */
  PME_ERR_BOUNDS = 8        /* index-checking build only: a kernel's index check failed */
} pme_status;

typedef struct pme_plan_s* pme_plan_t;

/* Options of a plan. Fill with pme_opts_default() and change what you need. */
typedef struct {
  double influence_power;  /* gamma of Eq. influence, C(n) = 1/|B(n)|^(2 gamma); default 1 */
  int deconvolution;       /* 1: apply C(n) (default); 0: plain G(k) (the paper's ablation) */
  double coulomb_k;        /* scale of every energy and derivative; 1 = Gaussian units,
                              14.3996454784 for eV with Angstrom and e */
  int include_pair;        /* 1: real-space erfc pair term (default); 0: mesh + self only */
  int include_self;        /* 1: self terms (default) */
  int include_background;  /* 1: neutralising background term (default) */
  int max_ions;            /* capacity; default 1<<18, at most 1<<27 (PME_ERR_UNSUPPORTED) */
  int brick[3];            /* spread brick edge in mesh points, x y z: one of the built shapes
                              8x8x16 (the default), 8x8x32, 16x8x16, 16x16x16, 4x8x16
                              (PME_ERR_UNSUPPORTED otherwise); {0,0,0} = automatic: the
                              autotuner's choice when opts.autotune is set (single-frame
                              plans), the default shape otherwise */
  int overlap_pair;        /* 1: run the pair term on a plan-owned side stream, concurrently
                              with the mesh stages (default); 0: everything on the call's
                              stream, one stage after the other (per-kernel timing) */
  int recip_method;        /* 0: particle mesh (default). 1: explicit Ewald k-sum over the half
                              space |k| <= ewald_kmax instead of the mesh (the conventional
                              baseline of the paper's timing crossover; forward only) */
  double ewald_kmax;       /* |k| cutoff in 1/length for recip_method 1; <= 0 selects
                              2 alpha sqrt(ln 1e8), where exp(-k^2/4 alpha^2) = 1e-8 */
  int influence_kind;      /* 0: G(k) C(n), the sinc deconvolution of Eq. influence (default).
                              1: the P3M influence function that minimises the mean-square
                              force error for analytical differentiation (Hockney-Eastwood
                              least squares), with alias sums |m| <= 2: G(n) = sum_m k_m^2 U_m
                              phi(k_m) / [(sum_m U_m)(sum_m k_m^2 U_m)], U_m = prod sinc^(2p);
                              deconvolution and influence_power are then unused, and
                              pme_forward_virial reports PME_ERR_UNSUPPORTED */
  int fft;                 /* transforms of the mesh convolution. The library's own apply when
                              every mesh axis of every frame is 2,3,5-smooth and at most 256
                              long and a mesh plane fits in one block's shared memory; when
                              every axis of every frame is 64 or 128 points they run as
                              power-of-two kernels (compile-time four-step transforms).
                              0 (default): automatic, the library's own when every frame's
                              mesh takes the power-of-two kernels, or for batched plans whose
                              meshes have no axis above 64 points (one launch per pass for
                              all frames; faster there on GB300), cuFFT otherwise.
                              1: always cuFFT. 2: always the library's own
                              (PME_ERR_UNSUPPORTED where they do not apply). 3: the library's
                              own without the power-of-two kernels. With the own transforms
                              the stage timers' "FFT R2C" and "FFT C2R" stages are the z/y
                              passes and "influence" includes the x transforms */
  int autotune;            /* 1 (default): with brick {0,0,0}, pme_plan_create times every
                              built brick shape once for this (device, mesh, order, max_ions
                              rounded up to a power of two) on synthetic uniform ions -- the
                              forward + backward of the mesh part, CUDA events, median of 5 --
                              and keeps the fastest (the default shape unless another is more
                              than 2 % faster); the choice is cached for the process (and in the
                              file named by the environment variable GBPME_TUNE_CACHE, if set).
                              0: no tuning. Batched plans are not tuned. */
  int reserved[3];
} pme_opts;

void pme_opts_default(pme_opts* opts);

/* Mesh-size rules of Section 2.3.1. rule 0: N = ceil(2 |a| / spacing + 1) (Eq. mesh_target
 * as printed); rule 1: N = ceil(|a| / spacing). strategy 0: power of two; 1: smallest
 * 2,3,5-smooth integer >= target (the paper's default); 2: the target itself. clamp_lo /
 * clamp_hi bound the result when > 0. Writes mesh[3]. Host only; no GPU needed. */
int pme_mesh_dims(const double box[9], double spacing, int rule, int strategy,
                  int clamp_lo, int clamp_hi, int mesh[3]);

/* Create a plan for one box, mesh, spline order p (1..7), Ewald alpha (> 0) and real-space
 * cutoff rcut (> 0; ignored when include_pair = 0). mesh[3] = {Nx, Ny, Nz}, each >= order.
 * opts may be NULL (defaults). Allocates all device scratch on the current CUDA device.
 * Section 2.3.1 (cell, reciprocal basis, mesh), 2.3.3 (deconvolution). */
int pme_plan_create(pme_plan_t* out, const double box[9], const int mesh[3], int order,
                    double alpha, double rcut, const pme_opts* opts);

/* Replace the box of an existing plan (same mesh, order, alpha, rcut). Not stream-ordered:
 * the caller must make sure no call on the plan is in flight. */
int pme_plan_set_box(pme_plan_t plan, const double box[9]);

int pme_plan_destroy(pme_plan_t plan);

/* Which transforms the plan's mesh convolution uses: *kind = 0 for the library's own
 * (Stockham transforms in shared memory, the x transform fused with the influence multiply),
 * 1 for cuFFT, 2 for the library's own power-of-two kernels (every axis 64 or 128). */
int pme_plan_fft_kind(pme_plan_t plan, int* kind);

/* The spread brick shape the plan uses (explicit, tuned or default): brick[3] = x, y, z edges. */
int pme_plan_brick(pme_plan_t plan, int brick[3]);

/* Text of the last error recorded on the plan (never NULL). */
const char* pme_last_error(pme_plan_t plan);
const char* pme_status_string(int status);

/* Synchronise `stream` and report device-detected errors (PME_ERR_NONFINITE, PME_ERR_TIMEOUT)
 * raised since the previous pme_sync_status, clearing them. */
int pme_sync_status(pme_plan_t plan, void* stream);

/* Repeated calls. pme_forward, pme_backward and their pme_batch_* forms keep one CUDA graph
 * per pass kind: the second call with the same n and the same pointers (host arguments count
 * by the plan's staging buffers, so any host pointers qualify) records the pass once on a
 * plan-owned stream, and that call and every later identical call launch the recorded graph
 * on `stream`, with the same results. A different call runs directly; pme_plan_set_box drops
 * the graphs, and calls made while the stage timers are on always run directly. */

/* Forward: energy and derivatives of Eq. (1).
 *   energy     [1] float64: E                     (may be NULL)
 *   force      [n][3]: F_i = -dE/dr_i             (may be NULL)
 *   phi        [n]:    dE/dq_i                    (may be NULL)
 *   field      [n][3]: -dE/dmu_i, the field of all other sources at r_i   (may be NULL)
 *   field_grad [n][6]: gradient of that field at r_i (xx,yy,zz,xy,xz,yz)   (may be NULL)
 * so that F_i = q_i field_i + field_grad_i mu_i. mu may be NULL (charges only).
 * Forces follow Eq. forces (analytic derivative of the discrete mesh energy). */
int pme_forward(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
                const float* mu, double* energy, float* force, float* phi, float* field,
                float* field_grad);

/* With opts.recip_method = 1 the reciprocal part is the explicit Ewald sum
 *   E_recip = (2 pi / V) sum_{0 < |k| <= kmax} exp(-k^2/4 alpha^2)/k^2 |sum_j (q_j + i mu_j.k) e^{i k.r_j}|^2
 * (O(N K) work) and every output keeps its meaning; pme_backward then returns
 * PME_ERR_UNSUPPORTED. */

/* Backward: vector-Jacobian product of the map (pos, q, mu) -> (E, force, phi, field) of
 * pme_forward, for cotangents g_energy [1] float64, g_force [n][3], g_phi [n], g_field [n][3]
 * (each may be NULL = zero):
 *   grad_pos = g_E dE/dr + H v,  grad_q = g_E dE/dq + H v,  grad_mu = g_E dE/dmu + H v,
 * with H the Hessian of E in (r, q, mu) and v = (-g_force, g_phi, -g_field). This is the
 * double backward through Eq. forces that the force-matching loss of Eq. loss needs; it
 * recomputes the mesh potential instead of storing it. Outputs may be NULL. */
int pme_backward(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
                 const float* mu, const double* g_energy, const float* g_force,
                 const float* g_phi, const float* g_field, float* grad_pos, float* grad_q,
                 float* grad_mu);

/* Forward plus the virial (an extension of the paper's outputs, for stress / NPT training):
 *   virial [9] float64, row-major, W_ab = -dE/d(eps_ab) for the homogeneous strain
 *   r -> (I + eps) r of the positions and the lattice vectors with the dipoles held fixed:
 *   W = k (E_rec I - (1/V) sum_n G C |rho_hat|^2 (1/k^2 + 1/(4 alpha^2)) k (x) k
 *          + sum_i (grad phi_mesh)_i (x) mu_i + 1/2 sum_(i,j) F_ij (x) r_ij + E_bg I)
 *   (not symmetric when dipoles are present). energy and virial are required (device or
 *   host pointers); the other outputs as in pme_forward.
 * Needs the particle-mesh reciprocal method and, with the pair term on, the plan's pair-hit
 * lists (PME_ERR_UNSUPPORTED for a plan too large to hold them). If a list overflows at run
 * time the pair part of the virial cannot be formed: the next pme_sync_status reports
 * PME_ERR_UNSUPPORTED. */
int pme_forward_virial(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
                       const float* mu, double* energy, float* force, float* phi, float* field,
                       float* field_grad, double* virial);

/* Forward with point quadrupoles: the rank-2 multipole channel the paper's concluding
 * section names as the next extension of its PME layer (an extension beyond the paper's
 * equations; the readings below are the library's). Each ion carries a symmetric Cartesian
 * quadrupole Theta, theta [n][6] float32 = (xx, yy, zz, xy, xz, yz), not made traceless,
 * entering the multipole operator q + mu . grad + Theta : grad grad: the energy of an ion in a
 * potential phi is q phi + mu . grad phi + Theta : grad grad phi, and a cluster of charges q_c
 * at offsets d_c with zero net charge and dipole has Theta = 1/2 sum_c q_c d_c d_c. The mesh
 * density adds Theta : grad grad W (second derivatives of the spline weights, the derivative
 * terms of Eq. charge_dipole_assign taken one order further), the pair term adds the
 * quadrupole contractions of grad^2..grad^5 erfc(alpha r)/r, and the self energy adds the
 * quadrupole parts of the Gaussian-cloud self interaction
 *   -(alpha/sqrt(pi)) [-(4 alpha^2/3) q tr Theta + (4 alpha^4/5)((tr Theta)^2 + 2 Theta:Theta)].
 * Outputs as pme_forward, except field_grad = -dE/dTheta (the symmetric matrix G with
 * dE = -G : dTheta for symmetric dTheta; equal to pme_forward's field gradient when Theta = 0)
 * and force = -dE/dr including Theta : grad^3 phi. Plans with recip_method 0 (batched plans:
 * pme_batch_forward_quad); no CUDA graph and no virial; the backward is pme_backward_quad. Pointers follow pme_forward's host/device rule. theta may
 * be NULL only when n = 0. */
int pme_forward_quad(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
                     const float* mu, const float* theta, double* energy, float* force, float* phi,
                     float* field, float* field_grad);

/* Backward with point quadrupoles: the vector-Jacobian product of the map
 * (pos, q, mu, theta) -> (E, force, phi, field) of pme_forward_quad for cotangents g_energy [1]
 * float64, g_force [n][3], g_phi [n], g_field [n][3] (each may be NULL = zero; there is no
 * cotangent on the -dE/dTheta output):
 *   grad = g_E dE + H v  in (r, q, mu, Theta),  v = (-g_force, g_phi, -g_field, 0),
 * with H the Hessian of E. grad_theta [n][6] (xx, yy, zz, xy, xz, yz) is the symmetric matrix G
 * with dL = G : dTheta for symmetric dTheta. This is the double backward through the forces
 * that a force-matching loss (Eq. loss) needs when the quadrupole channel is trained: the mesh
 * part spreads the tangent density (Theta : grad grad)(dr . grad) W with third spline
 * derivatives and gathers Phi to fourth and d Phi to third order; the pair part evaluates the
 * quadrupole pair sums in dual numbers (value and directional derivative). Needs spline order
 * >= 4 and, with the pair term, the plan's pair-hit lists (PME_ERR_UNSUPPORTED otherwise; a
 * list that overflows at run time is reported by pme_sync_status as PME_ERR_UNSUPPORTED).
 * Recomputes everything from its own inputs (no reuse of a forward, no CUDA graph). Pointers
 * follow pme_forward's host/device rule; outputs may be NULL. */
int pme_backward_quad(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
                      const float* mu, const float* theta, const double* g_energy,
                      const float* g_force, const float* g_phi, const float* g_field,
                      float* grad_pos, float* grad_q, float* grad_mu, float* grad_theta);

/* ---- batched frames ----------------------------------------------------------------------
 * One plan over F frames stored back to back in the per-ion arrays: frame f owns ions
 * [offsets[f], offsets[f+1]) (offsets[0] = 0, host array of F+1), with its own box
 * (boxes + 9 f, rows = lattice vectors), mesh (meshes + 3 f) and spline order (orders[f]);
 * alpha, rcut and opts are shared (opts.max_ions is ignored: the plan holds offsets[F] ions;
 * opts.recip_method must be 0). Every stage runs as one launch over the whole batch (spread
 * and gather: one launch per distinct spline order; the transforms: one launch per pass on
 * the library's own transforms, or one batched cuFFT call per distinct mesh shape; see
 * opts.fft), so a batch of small frames costs a handful of launches instead of a handful
 * per frame. The handle is a pme_plan_t: destroy it with pme_plan_destroy; the
 * single-frame calls reject it and the batch calls reject single-frame plans. */
int pme_batch_create(pme_plan_t* out, int nframes, const int* offsets, const double* boxes,
                     const int* meshes, const int* orders, double alpha, double rcut,
                     const pme_opts* opts);
int pme_batch_frames(pme_plan_t plan);

/* As pme_forward for every frame: energy [F] float64 (per frame), per-ion outputs over all
 * offsets[F] ions in the caller's order. Pointers follow the same host/device rule. */
int pme_batch_forward(pme_plan_t plan, void* stream, const float* pos, const float* q,
                      const float* mu, double* energy, float* force, float* phi, float* field,
                      float* field_grad);

/* As pme_forward_virial for every frame: virial [F][9] float64. */
int pme_batch_forward_virial(pme_plan_t plan, void* stream, const float* pos, const float* q,
                             const float* mu, double* energy, float* force, float* phi,
                             float* field, float* field_grad, double* virial);

/* As pme_forward_quad for every frame: theta [offsets[F]][6], energy [F] float64. */
int pme_batch_forward_quad(pme_plan_t plan, void* stream, const float* pos, const float* q,
                           const float* mu, const float* theta, double* energy, float* force,
                           float* phi, float* field, float* field_grad);

/* As pme_backward_quad for every frame: theta [offsets[F]][6], g_energy [F] float64. */
int pme_batch_backward_quad(pme_plan_t plan, void* stream, const float* pos, const float* q,
                            const float* mu, const float* theta, const double* g_energy,
                            const float* g_force, const float* g_phi, const float* g_field,
                            float* grad_pos, float* grad_q, float* grad_mu, float* grad_theta);

/* As pme_backward for every frame; g_energy is [F] float64 (one cotangent per frame). */
int pme_batch_backward(pme_plan_t plan, void* stream, const float* pos, const float* q,
                       const float* mu, const double* g_energy, const float* g_force,
                       const float* g_phi, const float* g_field, float* grad_pos, float* grad_q,
                       float* grad_mu);

/* ---- stage-level entry points (each runs one step of the pipeline on its own) ---------- */

/* Mesh density rho_mesh of Eq. charge_dipole_assign, written to rho [Nx][Ny][Nz] float32
 * (z fastest). Ions are sorted into mesh bricks and every mesh point is written once. */
int pme_spread(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
               const float* mu, float* rho);

/* Potential mesh Phi = (1/V) IFFT_unnormalised[ G C FFT[rho] ] (Eqs. fft, potential_k, ifft)
 * and E_recip = 1/2 sum rho Phi evaluated on the half spectrum in float64 (Eq.
 * energy_recip), both WITHOUT the coulomb_k factor. rho is not modified. */
int pme_solve(pme_plan_t plan, void* stream, const float* rho, float* phi_mesh,
              double* e_recip);

/* Interpolated potential of a mesh at the ions: out [n][10] = phi, d phi/dr (3),
 * d^2 phi/dr dr (xx,yy,zz,xy,xz,yz), with the same assignment weights as the spread. */
int pme_gather(pme_plan_t plan, void* stream, int n, const float* pos, const float* phi_mesh,
               float* out);

/* Real-space pair term alone: out [n][10] = pair potential at each ion and its first and
 * second spatial derivatives (as pme_gather), e_pair [1] float64 = E_pair. No coulomb_k. */
int pme_pair(pme_plan_t plan, void* stream, int n, const float* pos, const float* q,
             const float* mu, float* out, double* e_pair);

/* The brick autotuner on its own (what pme_plan_create does with opts.autotune): times the
 * forward + backward of the mesh part (pair term off) of a plan with each built brick shape on
 * n_ions synthetic uniform ions in `box` and writes the fastest shape to brick_out[3] and, if
 * ms_out is not NULL, the median milliseconds of each shape in the order 8x8x16, 8x8x32,
 * 16x8x16, 16x16x16, 4x8x16 (a negative value: that shape does not fit this mesh and order).
 * opts (may be NULL) supplies the remaining options. Allocates its own device buffers and
 * temporary plans on the current device; uses the process-wide cache. No counterpart in the
 * paper (its kernels are PyTorch operations with no launch parameters to choose). */
int pme_autotune_brick(const double box[9], const int mesh[3], int order, double alpha, double rcut,
                       int n_ions, const pme_opts* opts, int brick_out[3], double* ms_out);

/* Index-checking build. Compiled with -DGBPME_BOUNDS (libgbpme_bounds.so, built on request),
 * the sort, spread, gather, pair-list and combine kernels test every array index they derive
 * (sorted slots, mesh offsets, pair-list slots and partner indices) against its array's size
 * before the access; a failed test skips the access and sets a device flag -- it never traps,
 * so the context stays usable. pme_sync_status then reports PME_ERR_BOUNDS.
 * pme_bounds_flags() returns and clears the flags of all kernels (bit 0 spread, 1 gather,
 * 2 pair, 3 combine, 4 sort; always 0 in the normal build) and pme_bounds_checking() tells
 * which build is loaded (1 = index-checking). No counterpart in the paper: a debugging aid
 * for memory races and indexing errors, in place of compute-sanitizer. */
int pme_bounds_flags(void);
int pme_bounds_checking(void);

/* Number of the library's own kernels launched since the library was loaded (cuFFT's
 * kernels are not counted). */
long long pme_launch_count(void);

/* ---- stage timers ------------------------------------------------------------------------
 * When enabled, every stage of pme_forward / pme_backward is bracketed by CUDA events on
 * the stream it runs on (the pair term runs on the plan's side stream). Stage index =
 * stage + PME_STAGES_PER_PASS * pass, pass 0 = forward, 1 = backward, with stage
 * 0 sort, 1 spread, 2 FFT R2C, 3 influence, 4 FFT C2R, 5 gather, 6 pair (all of it),
 * 7 combine (with the forward's energy reduction), 8 pair evaluation from the hit lists
 * alone (a part of stage 6). At most 4096 stage executions are recorded between two reads.
 * While the timers are on, each timed stage is also an NVTX range named "fwd.spread" etc.,
 * for timeline profilers. */
#define PME_STAGES_PER_PASS 9
#define PME_NUM_STAGES 18
int pme_profile_enable(pme_plan_t plan, int enable);
/* Synchronises the plan's device, writes the summed milliseconds and the number of
 * executions of each stage since the last read into ms[PME_NUM_STAGES] and
 * calls[PME_NUM_STAGES] (either may be NULL), and resets the timers. */
int pme_profile_read(pme_plan_t plan, double* ms, long long* calls);

/* ---- allocation-free spread ----------------------------------------------------------------
 * No counterpart in the paper: a deployment variant of pme_spread for callers that cannot
 * call cudaMalloc when they need the mesh density -- typically code embedded in a host
 * framework that has already reserved the whole device for its own memory pool (so a new
 * cudaMalloc fails), or a simulation loop that must not allocate or free because
 * cudaMalloc / cudaFree can synchronise the device. It computes the same rho_mesh as
 * pme_spread with the same kernels in the same order, so the result is bitwise that of a
 * plan's pme_spread with the same box, mesh and order and the default brick (8 x 8 x 16, which
 * this entry point always uses), but it needs no plan and allocates
 * nothing: all of its sort scratch lives in ONE static device array of
 * PME_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that loads the library
 * keeps until the process exits.
 *   box[9], mesh[3], order: as for pme_plan_create. pos [n][3], q [n], mu [n][3] (may be NULL)
 *     and rho [Nx][Ny][Nz] are DEVICE pointers owned by the caller; rho is written.
 *   status (DEVICE pointer to one int, may be NULL): written on the stream after the spread,
 *     PME_ERR_NONFINITE when pos, q or mu held a NaN or Inf (rho is then not meaningful),
 *     PME_OK otherwise. The return value cannot report this: it is known only on the device.
 *   Limits: 0 <= n <= PME_NOALLOC_MAX_IONS and order <= mesh[a] <= PME_NOALLOC_MAX_MESH;
 *     anything larger returns PME_ERR_ARG without touching the device.
 *   The first call on a device looks up the device address of the array (with that device
 *     current) and caches it; make that first call before any stream capture on the device.
 *   Every call uses the same array and leaves its contents behind; what must start at zero
 *     (counters, the error flag) and the candidate-brick table are rewritten on the call's
 *     stream at the start of each call, by kernels and a memset (nothing is copied from host
 *     memory). Calls whose execution overlaps on the GPU (other streams, other host threads)
 *     race on the array and give wrong results: serialise them.
 *   Returns PME_OK, PME_ERR_ARG, PME_ERR_UNSUPPORTED or PME_ERR_CUDA. */
#define PME_NOALLOC_MAX_IONS 32768
#define PME_NOALLOC_MAX_MESH 128
#define PME_NOALLOC_SCRATCH_BYTES 2396672
int pme_spread_noalloc(void* stream, const double box[9], const int mesh[3], int order, int n,
                       const float* pos, const float* q, const float* mu, float* rho, int* status);

#ifdef __cplusplus
}
#endif

#endif /* GBPME_H */
