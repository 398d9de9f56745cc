// Host-side launchers of the libgbpme kernels (one translation unit per pipeline stage).
#pragma once

#include <vector>

#include "common.cuh"

namespace gbpme {

// Ion inputs in the caller's order. Tangent cotangents are only read by the backward pass.
struct IonInputs {
  const float* pos;     // [n][3]
  const float* q;       // [n]
  const float* mu;      // [n][3] or null
  const float* gforce;  // [n][3] or null: dr = -g_force
  const float* gphi;    // [n] or null:    dq = g_phi
  const float* gfield;  // [n][3] or null: dmu = -g_field
  const float* theta;   // [n][6] point quadrupoles (xx yy zz xy xz yz) or null (forward only)
  int n;
};

// sort.cu: brick and pair-cell counting sorts (4 kernels), records in both orders.
// reuse (nullable): when *reuse == 0 the plan's sorted order and primal records are those of
// these inputs (a forward on them) and are kept; only charge sums and tangent records are
// formed. A sort without reuse clears the plan's saved-forward state.
// save (nullable): the binning pass also copies the inputs there (positions at 0, charges at
// 3 max_ions, dipoles at 4 max_ions) for a later backward's comparison.
// The count arrays must be zero unless p->counts_clean is false (then they are cleared here).
int launch_sort(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool tangent, bool need_mesh,
                bool need_pair, const int* reuse, float* save = nullptr);
// *in_diff = 1 unless the inputs equal the saved ones bit for bit; *cache_bad = 1 when
// *in_diff or (with_lists) a recorded pair list overflowed; both 0 otherwise.
int launch_input_check(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool with_lists);

// spread.cu: owner-computes spread of rho (and, with tangent, of the tangent density) of every
// frame; frame f writes mesh + mesh_off (and mesh + tmesh_off).
// keep_rho (tangent pass, nullable): *keep_rho == 0 means rho is in place from the forward on
// the same inputs; only d rho is formed and written.
int launch_spread(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh, const int* keep_rho = nullptr);
// Quadrupole forward: rho of charges, dipoles and point quadrupoles theta [caller index][6]
// into mesh + mesh_off of every frame.
int launch_spread_quad(pme_plan_t p, cudaStream_t s, const float* theta, float* mesh);
// Quadrupole Hessian-vector product: the tangent density d rho of charges, dipoles and
// quadrupoles along (dr, dq, dmu) into mesh + tmesh_off of every frame.
int launch_spread_quad_tangent(pme_plan_t p, cudaStream_t s, const float* theta, float* mesh);

// influence.cu: in-place G C / V multiply of every frame's spectrum (and tangent spectrum)
// and the float64 energy partials (one per block, blocks grouped by frame).
int launch_influence(pme_plan_t p, cudaStream_t s, cufftComplex* spec, bool tangent,
                     double* partials, double* vparts = nullptr);
// Per-frame energies: out[f] = k (recip_coef(f) * sum of f's block partials + sum of f's
// per-ion energies e_ion + background(Q_f)); recip_coef = 1/(2V) for the mesh, 4 pi / V for
// the explicit k-sum, 0 without a reciprocal part.
int launch_energy_final(pme_plan_t p, cudaStream_t s, const double* parts, int recip_kind,
                        bool with_ions, bool with_bg, double scale, int n_single, double* out);
int influence_blocks(const Geometry& g);
// Fill the P3M influence table of every frame (influence_kind 1; plan creation, set_box).
int launch_p3m_tables(pme_plan_t p, cudaStream_t s);
// Fill every frame's influence table for the plan's kind (G C for kind 0, P3M for kind 1):
// plan creation and set_box; the multiply passes read it.
int launch_influence_tables(pme_plan_t p, cudaStream_t s);
void spread_brick_shape(int shape[3]);   // the default brick
// Brick shapes the spread kernels are built for (the autotuner chooses among them).
constexpr int kNumSpreadShapes = 5;
constexpr int kSpreadShapes[kNumSpreadShapes][3] = {{8, 8, 16}, {8, 8, 32}, {16, 8, 16}, {16, 16, 16}, {4, 8, 16}};
bool spread_shape_supported(const int shape[3]);
// tune.cu: the brick autotuner (pme_autotune_brick); use_cache: answer from the cache when the
// key is known (ms_out then stays untouched)
int autotune_brick(const double box[9], const int mesh[3], int order, double alpha, double rcut, int n,
                   const pme_opts& base, int out[3], double* ms_out, bool use_cache);
// one launcher per brick shape (spread.cu, spread_shapes_*.cu); mode 0 forward, 1 tangent,
// 2 quadrupole forward
#define GBPME_SPREAD_SHAPE(tag)                                                                      \
  int launch_spread_##tag(pme_plan_t p, cudaStream_t s, int mode, float* mesh, const int* keep_rho, \
                          const float* theta);
GBPME_SPREAD_SHAPE(8x8x16)
GBPME_SPREAD_SHAPE(8x8x32)
GBPME_SPREAD_SHAPE(16x8x16)
GBPME_SPREAD_SHAPE(16x16x16)
GBPME_SPREAD_SHAPE(4x8x16)
#undef GBPME_SPREAD_SHAPE

// conv.cu: the mesh convolution by hand-written transforms (meshes whose axes are all
// 2,3,5-smooth and at most kConvMaxLen long, planes within shared memory).
//   forward: R2C of every rho (and, tangent, d rho) in mesh into the plan's spectra
//   influence: x transform, G C / V multiply with the energy (virial) partials, inverse x
//   inverse: C2R of the spectra into mesh (Phi, and d Phi)
constexpr int kConvMaxLen = 256;
bool conv_axis_ok(int L);
// the power-of-two kernels: every axis 64 or 128 points; their shared memory per plane block
// (pass A / C, kP2PlaneThreads threads) and per pass-B block
bool conv_p2_ok(const int N[3]);
size_t conv_p2_plane_smem(const int N[3]);
size_t conv_p2_x_smem(const int N[3]);
void conv_tiles(const int N[3], int* ntile, int* cols);
int conv_planes_per_block(const int N[3]);
size_t conv_plane_cap(const int N[3]);
size_t conv_plane_smem(const int N[3], size_t cap);
size_t conv_x_smem(const int N[3]);
void conv_twiddles(int L, std::vector<float2>& out);
// keep (tangent passes, nullable): *keep == 0 means the plan's rho and Phi are those of the
// forward on the same inputs; the passes then skip them and transform the tangent mesh only.
int launch_conv_forward(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh, const int* keep = nullptr);
int launch_conv_influence(pme_plan_t p, cudaStream_t s, bool tangent, double* partials,
                          double* vparts = nullptr, const int* keep = nullptr);
int launch_conv_inverse(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh, const int* keep = nullptr);

// The backward pass's final per-ion assembly (the pair term's tangent sums, the self and
// background terms, coulomb_k), done in the tangent gather's epilogue so that the backward
// needs no separate combine launch.
struct BackwardFinish {
  const float* pair_out;   // [n][8] tangent pair sums in caller order (null: no pair term)
  const float* q;          // [n]
  const float* mu;         // [n][3] or null
  const float* gphi;       // [n] or null: dq
  const float* gfield;     // [n][3] or null: dmu = -g_field
  const double* qsum;      // Q, dQ per frame
  float* grad_pos;         // [n][3] or null
  float* grad_q;           // [n] or null
  float* grad_mu;          // [n][3] or null
  float k, self_phi, self_c;
  int with_bg;
};
// combine.cu: the constants and pointers of the assembly for these inputs and outputs.
BackwardFinish backward_finish_args(pme_plan_t p, const IonInputs& in, float* grad_pos, float* grad_q,
                                    float* grad_mu);

// gather.cu: per-ion interpolation of the potential mesh(es).
//   forward: out[orig][10] = phi, dphi/dr (3), d2phi/drdr (6)
//   tangent: out[orig][8]  = mesh part of (grad_r (3), grad_q, grad_mu (3)) of the backward
int launch_gather(pme_plan_t p, cudaStream_t s, int n, const float* mesh, bool tangent,
                  const double* g_energy, float* out);
// Tangent gather that also does the backward's final assembly (fin) and writes the gradients
// in place of the mesh part; the pair term's results must be complete when it runs.
int launch_gather_finish(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const double* g_energy,
                         const BackwardFinish& fin);
// Quadrupole Hessian-vector product, mesh part: the 13 gathered values of the quadrupole
// forward and their tangents along (dr, d Phi) at out[orig][26] (Phi at mesh_off, d Phi at
// tmesh_off of mesh).
int launch_gather_qdual(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const float* theta, float* out);
// Quadrupole forward: the forward layout in out, and Theta_i : grad^3 phi at qout[orig][0..2].
int launch_gather_quad(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const float* theta,
                       float* out, float* qout);

// quad.cu: real-space pair term with point quadrupoles (every frame): the forward layout of
// the pair potential of every source in out, Theta_i : grad^3 phi at qout[orig][4..6].
// skip (nullable): return at once when *skip == 0 (the hit lists hold).
int launch_pair_quad(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out, float* qout,
                     const int* skip = nullptr);
// Quadrupole Hessian-vector product: the 13 per-ion pair sums and their tangents along
// (dr, dq, dmu) from the hit lists, out[caller index][26] (runs only when *flag == 0).
int launch_pair_quad_dual(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out, const int* flag);
// The same from the plan's hit lists (runs only when *flag == 0).
int launch_pair_quad_listed(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out,
                            float* qout, const int* flag);

// pair.cu: real-space erfc pair term over the cell list, same output layouts as gather.
// The fused pass; skip (nullable): return at once when *skip == 0.
// virial (forward): the fused pass cannot form the pair virial and sets the lost-virial flag.
int launch_pair(pme_plan_t p, cudaStream_t s, int n, bool tangent, const IonInputs& in,
                const double* g_energy, float* out, const int* skip, bool virial = false);
// Write every ion's hits to the plan's pair lists; *overflow = 1 when a list is too short.
int launch_pair_build(pme_plan_t p, cudaStream_t s, int n, int* overflow);
// Pair term from the lists (runs only when *flag == 0).
// virial (forward): also each ion's 1/2 sum_j F_ij (x) r_ij into the plan's pvir [n][9].
int launch_pair_listed(pme_plan_t p, cudaStream_t s, int n, bool tangent, const double* g_energy,
                       float* out, const int* flag, bool virial = false);

// combine.cu: add the parts, the self and background terms, apply coulomb_k, write outputs;
// with energy non-null also the frame energies, as launch_energy_final with the per-ion
// energies of this pass (recip_kind as there).
// virial (nullable, needs energy): also the frame virials [9] per frame from the plan's
// k-space sums (vpart) and per-ion pair virials (pvir).
// With in.theta the quadrupole terms are added (quad_out: the gather's and the pair
// kernel's Theta : grad^3 phi; no virial).
int launch_combine_forward(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool with_mesh,
                           bool with_pair, float* force, float* phi, float* field,
                           float* field_grad, double* energy, int recip_kind,
                           double* virial = nullptr, const float* quad_out = nullptr);
// Quadrupole Hessian-vector product: grads in (r, q, mu, Theta) from the mesh and pair parts'
// 26-value dual outputs (qmesh, qpair: [n][26]).
int launch_combine_backward_quad(pme_plan_t p, cudaStream_t s, const IonInputs& in, const double* g_energy,
                                 const float* qmesh, const float* qpair, float* grad_pos, float* grad_q,
                                 float* grad_mu, float* grad_theta);
// ewald.cu: explicit Ewald reciprocal sum (structure factor, then per-ion potential
// derivatives in the gather's [n][10] layout); energy partials sum A |S|^2 over the half space.
int ewald_build_kvectors(pme_plan_t p, std::vector<int4>& kn, std::vector<float4>& kv);
int launch_ewald_recip(pme_plan_t p, cudaStream_t s, const IonInputs& in, double* partials,
                       float* out);
int ewald_partial_blocks(pme_plan_t p);

// Sum of per-ion pair energies 1/2 (q phi + mu . dphi/dr) of a pair_out buffer.
int launch_pair_energy(pme_plan_t p, cudaStream_t s, int n, const IonInputs& in,
                       const float* pair_out);

}  // namespace gbpme
