/*
 * gbnet.h -- C ABI of the learned charge/dipole network of libgbpme.so.
 *
 * The paper's long-range channel takes its charges and dipoles from readout heads of a
 * Cartesian-tensor message-passing network (Section 2.1; Eqs. charge_pred, dipole_pred and
 * site_energy of Section 2.2) and trains them, without direct supervision, through the
 * differentiable PME on energies and forces (Section 2.4, Eqs. E_total, forces, loss). This
 * header exposes the library's own small network of that family and its training step:
 *
 *   inputs    positions r_i, species s_i in {0, 1} of F periodic frames;
 *   edges     every ordered pair (i, j) of a frame with 0 < |d| < GBNET_CUTOFF,
 *             d = r_j - r_i + (lattice vector), the nearest periodic image;
 *   basis     e_k(r) = sqrt(2/r_c) sin(k pi r/r_c)/r * u(r/r_c), k = 1..8,
 *             u(x) = 1 - 21 x^5 + 35 x^6 - 15 x^7;
 *   features  32 scalar channels h^s (start: the species embedding), 16 vector channels h^v
 *             (3 x 16, start: zero);
 *   layer     A = h^s WA, B = h^v WB (per Cartesian component), R = e WR per edge, split
 *             into R_ss (32), R_sv (16), R_vs (16), R_vv (16); messages summed over the
 *             edges of i and divided by 16:
 *               m^s_c = sum R_ss,c A_j,c;  m^s_(32+c) = sum R_sv,c (d^ . B_j,c);
 *               m^v_c = sum R_vs,c d^ A_j,(32+c);  m^v_(16+c) = sum R_vv,c B_j,(16+c);
 *             U = m^s WU, Y = m^v WY; h^s += SiLU(U_(0..31)),
 *             h^v += sigmoid(U_(32..47)) * Y (one gate per vector channel);
 *   readouts  H = h^s Wh + bh; q~ = wq . SiLU(H_(0..31)) + bq, q = q~ - mean over the frame
 *             (neutral charges); mu = sum_c wmu_c h^v_c; site energy wE . SiLU(H_(32..63)) + bE;
 *             E_sr = sum of site energies of the frame.
 *   model     E_b = E_sr,b + E_PME,b(r, q(r), mu(r)), forces F = -dE/dr through every path.
 *
 * The five channel-mixing products (WA, WB, WU, WY, Wh) run on the tensor cores (tcgen05,
 * bfloat16 weights, float32 accumulation; activations are split into two bfloat16 parts, so
 * the products keep about 16 significant bits); everything else is float32 in the library's
 * own kernels. Gradients of the force-matching loss with respect to the parameters are
 * formed by one forward and one backward pass carrying a tangent along the force residual
 * (forward-over-reverse differentiation), with the PME's own Hessian-vector product
 * (pme_batch_backward) for the long-range part.
 *
 * Parameter vector: GBNET_NUM_PARAMS float32 values, the blocks below in this order, each
 * row-major with shape (rows, cols) = (fan_in, fan_out) for the matrices:
 *   emb (2, 32); for layer t = 0, 1: WA_t (32, 48), WB_t (16, 32), WR_t (8, 80),
 *   WU_t (48, 48), WY_t (32, 16); Wh (32, 64); bh (64); wq (32); bq (1); wE (32); bE (1);
 *   wmu (16).
 * The library keeps a float32 master copy; the tensor cores use its bfloat16 rounding
 * (nearest, ties to even) of WA, WB, WU, WY and Wh.
 *
 * Conventions as in gbpme.h: every pointer argument is a DEVICE pointer unless it is said to
 * be a host array; calls are asynchronous on `stream` (a cudaStream_t as void*, NULL = the
 * legacy default stream); a handle must not be used by two calls that overlap in time.
 * Errors: every function returns a pme_status; gbnet_last_error() gives the text.
 */
#ifndef GBNET_H
#define GBNET_H

#include "gbpme.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GBNET_SCALARS 32
#define GBNET_VECTORS 16
#define GBNET_RADIAL 8
#define GBNET_LAYERS 2
#define GBNET_CUTOFF 5.0
#define GBNET_MAX_NEIGHBOURS 64
#define GBNET_NUM_PARAMS 13266

typedef struct gbnet_s* gbnet_t;

/* Create a network handle for batches of at most max_ions ions in at most max_frames frames
 * (all scratch is allocated here, on the current device; the compute calls allocate
 * nothing). Parameters start at zero: set them with gbnet_set_params. */
int gbnet_create(gbnet_t* out, int max_ions, int max_frames);
int gbnet_destroy(gbnet_t net);
const char* gbnet_last_error(gbnet_t net);

/* The frames of the following calls: offsets (host, [nframes + 1], offsets[0] = 0), boxes
 * (host, [nframes][9], rows = lattice vectors), species (device int32 [offsets[nframes]],
 * 0 or 1). Each box must be at least 2 GBNET_CUTOFF wide across every pair of faces (then
 * each pair of ions has at most one image within the cutoff); PME_ERR_ARG otherwise. */
int gbnet_set_frames(gbnet_t net, void* stream, int nframes, const int* offsets,
                     const double* boxes, const int* species);

/* Copy GBNET_NUM_PARAMS float32 parameters in (params: device) and reset the optimiser
 * state (Adam moments and step count), or copy the float32 master parameters out. */
int gbnet_set_params(gbnet_t net, void* stream, const float* params);
int gbnet_get_params(gbnet_t net, void* stream, float* params);

/* Forward pass of the network on positions pos [n][3]: charges q [n], dipoles mu [n][3],
 * per-frame short-range energies e_sr [nframes] float64 (each may be NULL). The neighbour
 * lists are rebuilt from pos. Activations are kept for gbnet_backward. */
int gbnet_forward(gbnet_t net, void* stream, const float* pos, float* q, float* mu, double* e_sr);

/* Vector-Jacobian product of the last gbnet_forward, (r, theta) -> (q, mu, E_sr), for
 * cotangents g_q [n], g_mu [n][3], g_esr [nframes] float64 (each may be NULL = zero):
 * g_pos [n][3] = sum g . d(q, mu, E_sr)/dr and g_params [GBNET_NUM_PARAMS] the same with
 * respect to the parameters (each output may be NULL; outputs are written). */
int gbnet_backward(gbnet_t net, void* stream, const float* g_q, const float* g_mu,
                   const double* g_esr, float* g_pos, float* g_params);

/* Loss of Eq. loss over the frames and its gradient with respect to the parameters:
 *   L = lambda_e / F sum_b ((E_b - e_ref_b) / N_b)^2 + lambda_f / (3 sum_b N_b) sum |F - f_ref|^2
 * with E_b = E_sr,b + E_PME,b and F = -dE/dr of the model. pme is a batched plan
 * (pme_batch_create) over the same frames (offsets, boxes), whose options define E_PME.
 * e_ref [nframes] float64, f_ref [n][3]. loss [3] float64 = (L, its energy term, its force
 * term), the lambda-weighted parts, which add up to L; force [n][3] (may be NULL) = the
 * model's forces; grad [GBNET_NUM_PARAMS] = dL/dtheta, written, or added to when
 * accumulate != 0. */
int gbnet_loss_grad(gbnet_t net, pme_plan_t pme, void* stream, const float* pos,
                    const double* e_ref, const float* f_ref, double lambda_e, double lambda_f,
                    double* loss, float* force, float* grad, int accumulate);

/* Adam update of the master parameters with gradient grad [GBNET_NUM_PARAMS]:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, theta -= lr m^ / (sqrt(v^) + eps) with the
 * bias-corrected moments of step t (counted by the handle); refreshes the bfloat16 copies. */
int gbnet_adam(gbnet_t net, void* stream, const float* grad, double lr, double beta1,
               double beta2, double eps);

/* One training step: gbnet_loss_grad into the handle's own gradient buffer, then gbnet_adam. */
int gbnet_train_step(gbnet_t net, pme_plan_t pme, void* stream, const float* pos,
                     const double* e_ref, const float* f_ref, double lambda_e, double lambda_f,
                     double lr, double* loss);

/* Stage-level entry point of the channel mixing: Y [M][nout] (+)= X [M][k] W on the tensor
 * cores, W given transposed as wt [nout][k] bfloat16 bits (uint16). Supported (k, nout):
 * (32,48), (16,32), (48,48), (32,16), (32,64), (48,32), (64,32); X, Y float32, 16-byte
 * aligned. err (device int, may be NULL): bit 0 set if a bounded wait on the tensor cores
 * gave up (the affected rows are then not written). */
int gbnet_mix(void* stream, int M, int k, int nout, const float* X, const unsigned short* wt,
              float* Y, int accumulate, int* err);

/* Synchronise `stream` and report device-detected errors of the handle since the last call
 * (PME_ERR_TIMEOUT: a tensor-core wait gave up; PME_ERR_ARG: an ion had more than
 * GBNET_MAX_NEIGHBOURS neighbours; PME_ERR_NONFINITE: a non-finite position), clearing them. */
int gbnet_sync_status(gbnet_t net, void* stream);

/* Number of the network's kernels launched by the last gbnet_loss_grad / gbnet_train_step
 * (the PME calls inside them not counted). */
long long gbnet_last_launches(gbnet_t net);

#ifdef __cplusplus
}
#endif

#endif /* GBNET_H */
