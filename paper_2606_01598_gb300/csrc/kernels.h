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
  int n;
};

// sort.cu: brick and pair-cell counting sorts (4 kernels), records in both orders.
int launch_sort(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool tangent, bool need_mesh,
                bool need_pair);

// spread.cu: owner-computes spread of rho (and, with tangent, of the tangent density).
int launch_spread(pme_plan_t p, cudaStream_t s, int n, bool tangent, float* rho_out,
                  float* drho_out);

// influence.cu: in-place G C / V multiply of nspec half spectra and the float64 energy
// partials of the first; energy_final reduces all partials into one float64 value.
int launch_influence(pme_plan_t p, cudaStream_t s, cufftComplex* spec, int nspec,
                     double* partials);
// out = scale * (coef_a * sum parts[0, na) + sum parts[na, na + nb) + bgfac * Q^2)
int launch_energy_final(pme_plan_t p, cudaStream_t s, const double* parts, int na, int nb,
                        double coef_a, double scale, double bgfac, const double* qsum,
                        double* out);
int influence_grid(pme_plan_t p);
void spread_brick_shape(int shape[3]);
int combine_blocks(int n);

// gather.cu: per-ion interpolation of the potential mesh(es).
//   forward: out[orig][10] = phi, dphi/dr (3), d2phi/drdr (6)
//   tangent: out[orig][8]  = mesh part of (grad_r (3), grad_q, grad_mu (3)) of the backward
int launch_gather(pme_plan_t p, cudaStream_t s, int n, const float* phi_mesh,
                  const float* dphi_mesh, bool tangent, const IonInputs& in,
                  const double* g_energy, float* out);

// pair.cu: real-space erfc pair term over the cell list, same output layouts as gather.
int launch_pair(pme_plan_t p, cudaStream_t s, int n, bool tangent, const IonInputs& in,
                const double* g_energy, float* out);

// combine.cu: add the parts, the self and background terms, apply coulomb_k, write outputs.
int launch_combine_forward(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool with_mesh,
                           bool with_pair, double* e_parts, float* force, float* phi,
                           float* field, float* field_grad);
int launch_combine_backward(pme_plan_t p, cudaStream_t s, const IonInputs& in,
                            const double* g_energy, float* grad_pos, float* grad_q,
                            float* grad_mu);
// ewald.cu: explicit Ewald reciprocal sum (structure factor, then per-ion potential
// derivatives in the gather's [n][10] layout); energy partials sum A |S|^2 over the half space.
int ewald_build_kvectors(pme_plan_t p, std::vector<int4>& kn, std::vector<float4>& kv);
int launch_ewald_recip(pme_plan_t p, cudaStream_t s, const IonInputs& in, double* partials,
                       float* out);
int ewald_partial_blocks(pme_plan_t p);

// Sum of per-ion pair energies 1/2 (q phi + mu . dphi/dr) of a pair_out buffer.
int launch_pair_energy(pme_plan_t p, cudaStream_t s, int n, const IonInputs& in,
                       const float* pair_out, double* e_pair);

}  // namespace gbpme
