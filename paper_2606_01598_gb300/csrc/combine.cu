// Per-ion assembly of the outputs from the mesh and pair parts, plus the self terms
// (Eqs. self_q, self_mu) and the neutralising background -pi Q^2 / (2 V alpha^2).
//
// Forward, per ion (k = coulomb_k, c = 4 alpha^3 / (3 sqrt(pi))):
//   phi        = k (phi_mesh + phi_pair - 2 alpha q / sqrt(pi) - pi Q / (V alpha^2))
//   field      = k (-grad phi_mesh - grad phi_pair + c mu)              (= -dE/dmu)
//   field_grad = k (-hess phi_mesh - hess phi_pair - c q I)
//   force      = q field + field_grad mu                               (= -dE/dr)
// where the c terms remove the ion's own screening cloud (for mu they are the derivative of
// Eq. self_mu; for the field gradient the analogous part of the reciprocal sum), so field
// and field_grad are those of all other sources. The per-ion float64 energy contributions
// 1/2 (q phi_pair + mu . grad phi_pair) + self energies are summed per reduction item (one
// block of kRedItem ions), and the item of each frame that finishes last adds the item sums,
// the frame's reciprocal-space partials and the background energy in a fixed order.
//
// With point quadrupoles Theta (the rank-2 channel; in.theta non-null) the forward also adds
// the quadrupole self terms: with c5 = 8 alpha^5 / (5 sqrt(pi)),
//   phi        += k c tr Theta
//   field_grad  = k (-hess phi_mesh - hess phi_pair - c q I + c5 (tr Theta I + 2 Theta))
//                                                                      (= -dE/dTheta)
//   force       = -k (q grad phi + (hess phi) mu + Theta : grad^3 phi)    (mesh + pair parts)
// and the per-ion energy 1/2 Theta : hess phi_pair + c q tr Theta
// - (4 alpha^5 / (5 sqrt(pi))) ((tr Theta)^2 + 2 Theta : Theta).
//
// Backward, per ion: grad = k (mesh part + pair part) + the self and background terms of
// the g_E-weighted gradient and of the Hessian-vector product.
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kCombThreads = kRedItem;   // one block per reduction item

struct CombineArgs {
  FrameDesc one;
  FrameMaps maps;
  const float* mesh_out;
  const float* pair_out;
  int with_mesh, with_pair;
  IonInputs in;
  const double* qsum;       // Q, dQ per frame
  const double* g_energy;   // per frame
  double* e_ion;            // per-ion energy contributions (forward)
  float* force;
  float* phi;
  float* field;
  float* field_grad;
  float* grad_pos;
  float* grad_q;
  float* grad_mu;
  float k;
  float self_phi;     // 2 alpha / sqrt(pi)     (0 when self terms are off)
  float self_c;       // 4 alpha^3 / (3 sqrt(pi))
  int with_bg;        // background term on
  double e_self_q;    // alpha / sqrt(pi)
  double e_self_mu;   // 2 alpha^3 / (3 sqrt(pi))
  // quadrupoles (forward; null: none)
  const float* qout;  // [n][8]: Theta : grad^3 phi of the mesh at 0..2, of the pair term at 4..6
  float self_c5;      // 8 alpha^5 / (5 sqrt(pi))
  double e_self_t1;   // 4 alpha^3 / (3 sqrt(pi))
  double e_self_t2;   // 4 alpha^5 / (5 sqrt(pi))
  // frame energies (forward; energy_out null: not wanted)
  double* energy_out;
  const double* recip_parts;
  int recip_kind;     // 0 none, 1 mesh (1/2V), 2 explicit k-sum (4 pi / V)
  double kd;          // coulomb_k
  double* eitem;
  int* ecount;
  // frame virials (forward; virial_out null: not wanted), row-major [9] per frame:
  // W = k (E_rec I - S / V + sum_i grad phi_mesh,i (x) mu_i + W_pair + E_bg I)
  double* virial_out;
  const double* vparts;   // [6 * influence blocks] S_ab (xx yy zz xy xz yz)
  const float* pvir;      // [n][9] per-ion pair virial (null without the pair term)
  double* vitem;          // [9 * items]
};

// pi / (V alpha^2) of the ion's frame, or 0 without the background term
__device__ __forceinline__ float bg_factor(const CombineArgs& a, const FrameDesc& F) {
  return a.with_bg ? F.g.bg_fac : 0.f;
}

template <bool BATCH>
__global__ void __launch_bounds__(kCombThreads) k_combine_forward(CombineArgs a) {
  pdl_begin();
  static_assert(kRedItem == kCombThreads, "one ion per thread");
  const int item = blockIdx.x;
  const int f = BATCH ? a.maps.item_frame[item] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, f);
  int lo, hi;
  item_range(F, item, lo, hi);
  const int i = lo + int(threadIdx.x);
  double e_i = 0.0;   // quadrupole terms (float64)
  float e_f = 0.f;    // pair and self terms
  float vi[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // virial terms of ion i
  if (i < hi && index_ok(i, a.in.n)) {
    const float bg = bg_factor(a, F);
    float qi = a.in.q[i];
    float mu[3] = {0.f, 0.f, 0.f};
    if (a.in.mu) {
      mu[0] = a.in.mu[3 * i];
      mu[1] = a.in.mu[3 * i + 1];
      mu[2] = a.in.mu[3 * i + 2];
    }
    float v[10], w[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      v[t] = a.with_mesh ? a.mesh_out[size_t(i) * 10 + t] : 0.f;
      w[t] = a.with_pair ? a.pair_out[size_t(i) * 10 + t] : 0.f;
    }
    const float Q = float(a.qsum[2 * f]);
    const float k = a.k;
    const float ph = k * (v[0] + w[0] - a.self_phi * qi - bg * Q);
    float fld[3], fg[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) fld[c] = k * (-(v[1 + c] + w[1 + c]) + a.self_c * mu[c]);
#pragma unroll
    for (int c = 0; c < 6; ++c) fg[c] = k * (-(v[4 + c] + w[4 + c]) - (c < 3 ? a.self_c * qi : 0.f));
    // force = q field + field_grad mu ; field_grad order xx yy zz xy xz yz
    const float F0 = qi * fld[0] + fg[0] * mu[0] + fg[3] * mu[1] + fg[4] * mu[2];
    const float F1 = qi * fld[1] + fg[3] * mu[0] + fg[1] * mu[1] + fg[5] * mu[2];
    const float F2 = qi * fld[2] + fg[4] * mu[0] + fg[5] * mu[1] + fg[2] * mu[2];
    float F0q = 0.f, F1q = 0.f, F2q = 0.f;
    float ph_q = ph;
    if (a.in.theta) {
      const float* th = a.in.theta + size_t(i) * 6;
      const float T[6] = {th[0], th[1], th[2], th[3], th[4], th[5]};
      const float trT = T[0] + T[1] + T[2];
      ph_q = ph + k * a.self_c * trT;
#pragma unroll
      for (int c = 0; c < 6; ++c) fg[c] += k * a.self_c5 * ((c < 3 ? trT : 0.f) + 2.f * T[c]);
      float g[3], H[6], t3[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        g[c] = v[1 + c] + w[1 + c];
        t3[c] = (a.with_mesh ? a.qout[size_t(i) * 8 + c] : 0.f) + (a.with_pair ? a.qout[size_t(i) * 8 + 4 + c] : 0.f);
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) H[c] = v[4 + c] + w[4 + c];
      F0q = -k * (qi * g[0] + H[0] * mu[0] + H[3] * mu[1] + H[4] * mu[2] + t3[0]);
      F1q = -k * (qi * g[1] + H[3] * mu[0] + H[1] * mu[1] + H[5] * mu[2] + t3[1]);
      F2q = -k * (qi * g[2] + H[4] * mu[0] + H[5] * mu[1] + H[2] * mu[2] + t3[2]);
      const double TW = double(T[0]) * w[4] + double(T[1]) * w[5] + double(T[2]) * w[6] +
                        2.0 * (double(T[3]) * w[7] + double(T[4]) * w[8] + double(T[5]) * w[9]);
      const double TT = double(T[0]) * T[0] + double(T[1]) * T[1] + double(T[2]) * T[2] +
                        2.0 * (double(T[3]) * T[3] + double(T[4]) * T[4] + double(T[5]) * T[5]);
      e_i += 0.5 * TW + a.e_self_t1 * double(qi) * trT - a.e_self_t2 * (double(trT) * trT + 2.0 * TT);
    }
    if (a.phi) a.phi[i] = ph_q;
    if (a.field) {
      a.field[3 * i] = fld[0];
      a.field[3 * i + 1] = fld[1];
      a.field[3 * i + 2] = fld[2];
    }
    if (a.field_grad) {
#pragma unroll
      for (int c = 0; c < 6; ++c) a.field_grad[6 * i + c] = fg[c];
    }
    if (a.force) {
      a.force[3 * i] = a.in.theta ? F0q : F0;
      a.force[3 * i + 1] = a.in.theta ? F1q : F1;
      a.force[3 * i + 2] = a.in.theta ? F2q : F2;
    }
    // the ion's pair and self energy in float32 (float64 across the block's warps below; the
    // per-ion float64 arithmetic kept the float64 pipe a third busy)
    const float mu2 = mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2];
    e_f = 0.5f * (qi * w[0] + mu[0] * w[1] + mu[1] * w[2] + mu[2] * w[3]) - float(a.e_self_q) * qi * qi -
          float(a.e_self_mu) * mu2;
    if (a.virial_out) {
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          vi[3 * r + c] = v[1 + r] * mu[c] + (a.pvir ? a.pvir[size_t(i) * 9 + 3 * r + c] : 0.f);
    }
  }
  if (a.virial_out) {
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      const double t = block_sum_f(vi[c]);
      if (threadIdx.x == 0) a.vitem[9 * item + c] = t;
    }
  }
  if (!a.energy_out) return;   // uniform
  const double e_item = block_sum_f(e_f) + (a.in.theta ? block_sum_d(e_i) : 0.0);
  if (threadIdx.x == 0) a.eitem[item] = e_item;
  if (!last_item_done(a.ecount + f, F.nitems)) return;
  // the frame's reciprocal and per-item partials, both sums at once (the last block's float64
  // chain is what this kernel's duration is made of)
  double rp, ep;
  strided_sum2_d(a.recip_parts + F.infl_blk_off, a.recip_kind ? F.infl_nblk : 0, 1, a.eitem + F.item_off,
                 F.nitems, 1, rp, ep);
  block_sum2_d(rp, ep);
  double W[9], S[6];
  if (a.virial_out) {
#pragma unroll
    for (int c = 0; c < 9; ++c) W[c] = block_sum_d(strided_sum_d(a.vitem + 9 * F.item_off + c, F.nitems, 9));
#pragma unroll
    for (int c = 0; c < 6; ++c) S[c] = block_sum_d(strided_sum_d(a.vparts + 6 * F.infl_blk_off + c, F.infl_nblk, 6));
  }
  if (threadIdx.x == 0) {
    const double V = F.g.volume;
    const double coef = a.recip_kind == 1 ? F.g.e_mesh_coef : (a.recip_kind == 2 ? F.g.e_ewald_coef : 0.0);
    double e_bg = 0.0;
    if (a.with_bg) {
      const double Q = a.qsum[2 * f];
      e_bg = -(Q * Q) * F.g.e_bg_coef;
    }
    a.energy_out[f] = a.kd * (coef * rp + ep + e_bg);
    if (a.virial_out) {
      const int sidx[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};   // S_ab from xx yy zz xy xz yz
      const double diag = coef * rp + e_bg;
      for (int c = 0; c < 9; ++c)
        a.virial_out[9 * f + c] = a.kd * (W[c] - S[sidx[c]] / V + ((c % 4) == 0 ? diag : 0.0));
    }
    a.ecount[f] = 0;
  }
}

// Quadrupole Hessian-vector product, per ion: from the mesh and pair parts' 13 gathered values
// and their tangents (out[26]: phi, grad phi, grad^2 phi, Theta : grad^3 phi), the gradient of
// E in (r, q, mu, Theta) and its directional derivative along v = (dr, dq, dmu) = (-g_force,
// g_phi, -g_field), grad = g_E dE + d(dE):
//   dE/dr     = k (q g + H mu + t3)
//   dE/dq     = k (phi - c_phi q - bg Q + c tr Theta)
//   dE/dmu    = k (g - c mu)
//   dE/dTheta = k (H + c q I - c5 (tr Theta I + 2 Theta))
// (c_phi = 2 alpha / sqrt(pi), c = 4 alpha^3 / (3 sqrt(pi)), c5 = 8 alpha^5 / (5 sqrt(pi)), bg =
// pi / (V alpha^2)), and their tangents k (dq g + q dg + dH mu + H dmu + dt3),
// k (dphi - c_phi dq - bg dQ), k (dg - c dmu), k (dH + c dq I).
template <bool BATCH>
__global__ void __launch_bounds__(kCombThreads) k_combine_backward_quad(CombineArgs a, const float* qm,
                                                                      const float* qp, float* grad_theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.in.n) return;
  const int f = BATCH ? a.maps.ion_frame[i] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, f);
  const float bg = bg_factor(a, F);
  const float qi = a.in.q[i];
  float mu[3] = {0.f, 0.f, 0.f}, dmu[3] = {0.f, 0.f, 0.f};
  if (a.in.mu)
    for (int c = 0; c < 3; ++c) mu[c] = a.in.mu[3 * i + c];
  if (a.in.gfield)
    for (int c = 0; c < 3; ++c) dmu[c] = -a.in.gfield[3 * i + c];
  const float dq = a.in.gphi ? a.in.gphi[i] : 0.f;
  const float gE = a.g_energy ? float(a.g_energy[f]) : 0.f;
  float v[26];
#pragma unroll
  for (int t = 0; t < 26; ++t) v[t] = qm[size_t(i) * 26 + t] + (a.with_pair ? qp[size_t(i) * 26 + t] : 0.f);
  const float* P = v;          // phi, g (3), H (6: xx yy zz xy xz yz), t3 (3)
  const float* T = v + 13;     // their tangents
  const float* th = a.in.theta + size_t(i) * 6;
  const float trT = th[0] + th[1] + th[2];
  const float Q = float(a.qsum[2 * f]), dQ = float(a.qsum[2 * f + 1]);
  const float k = a.k;
  // H mu and dH mu, H dmu (symmetric 6-vectors)
  auto hv = [](const float* H, const float* x, float* y) {
    y[0] = H[0] * x[0] + H[3] * x[1] + H[4] * x[2];
    y[1] = H[3] * x[0] + H[1] * x[1] + H[5] * x[2];
    y[2] = H[4] * x[0] + H[5] * x[1] + H[2] * x[2];
  };
  float Hm[3], dHm[3], Hdm[3];
  hv(P + 4, mu, Hm);
  hv(T + 4, mu, dHm);
  hv(P + 4, dmu, Hdm);
  if (a.grad_pos) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float Er = qi * P[1 + c] + Hm[c] + P[10 + c];
      const float dEr = dq * P[1 + c] + qi * T[1 + c] + dHm[c] + Hdm[c] + T[10 + c];
      a.grad_pos[3 * i + c] = k * (gE * Er + dEr);
    }
  }
  if (a.grad_q) {
    const float Eq = P[0] - a.self_phi * qi - bg * Q + a.self_c * trT;
    const float dEq = T[0] - a.self_phi * dq - bg * dQ;
    a.grad_q[i] = k * (gE * Eq + dEq);
  }
  if (a.grad_mu) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.grad_mu[3 * i + c] = k * (gE * (P[1 + c] - a.self_c * mu[c]) + T[1 + c] - a.self_c * dmu[c]);
  }
  if (grad_theta) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const float diag = c < 3 ? 1.f : 0.f;
      const float Et = P[4 + c] + a.self_c * qi * diag - a.self_c5 * (trT * diag + 2.f * th[c]);
      const float dEt = T[4 + c] + a.self_c * dq * diag;
      grad_theta[6 * i + c] = k * (gE * Et + dEt);
    }
  }
}

__global__ void __launch_bounds__(kCombThreads)
k_pair_energy(int n, const float* q, const float* mu, const float* pair_out, double* e_ion) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* w = pair_out + size_t(i) * 10;
  double e = 0.5 * double(q[i]) * w[0];
  if (mu)
    e += 0.5 * (double(mu[3 * i]) * w[1] + double(mu[3 * i + 1]) * w[2] + double(mu[3 * i + 2]) * w[3]);
  e_ion[i] = e;
}

CombineArgs base_args(pme_plan_t p, const IonInputs& in) {
  CombineArgs a = {};
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.in = in;
  a.qsum = p->sb.qsum;
  a.e_ion = p->e_ion;
  a.k = float(p->opts.coulomb_k);
  const double sp = 1.7724538509055160273;
  const double al = p->alpha;
  const bool self = p->opts.include_self != 0;
  a.self_phi = self ? float(2.0 * al / sp) : 0.f;
  a.self_c = self ? float(4.0 * al * al * al / (3.0 * sp)) : 0.f;
  a.with_bg = p->opts.include_background ? 1 : 0;
  a.e_self_q = self ? al / sp : 0.0;
  a.e_self_mu = self ? 2.0 * al * al * al / (3.0 * sp) : 0.0;
  a.self_c5 = self ? float(8.0 * std::pow(al, 5) / (5.0 * sp)) : 0.f;
  a.e_self_t1 = self ? 4.0 * al * al * al / (3.0 * sp) : 0.0;
  a.e_self_t2 = self ? 4.0 * std::pow(al, 5) / (5.0 * sp) : 0.0;
  return a;
}

}  // namespace

int launch_combine_forward(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool with_mesh,
                           bool with_pair, float* force, float* phi, float* field,
                           float* field_grad, double* energy, int recip_kind, double* virial,
                           const float* quad_out) {
  CombineArgs a = base_args(p, in);
  a.qout = quad_out;
  a.mesh_out = p->mesh_out;
  a.pair_out = p->pair_out;
  a.with_mesh = with_mesh;
  a.with_pair = with_pair;
  a.force = force;
  a.phi = phi;
  a.field = field;
  a.field_grad = field_grad;
  a.energy_out = energy;
  a.recip_parts = p->epart;
  a.recip_kind = recip_kind;
  a.kd = p->opts.coulomb_k;
  a.eitem = p->eitem;
  a.ecount = p->ecount;
  a.virial_out = (virial && energy) ? virial : nullptr;
  a.vparts = p->vpart;
  a.pvir = with_pair ? p->pvir : nullptr;
  a.vitem = p->vitem;
  int items;
  if (p->batch) {
    items = p->total_items;
  } else {
    a.one.n = in.n;
    a.one.item_off = 0;
    a.one.nitems = std::max(1, (in.n + kRedItem - 1) / kRedItem);
    items = a.one.nitems;
  }
  if (p->batch) pdl_launch(k_combine_forward<true>, items, kCombThreads, 0, s, a);
  else pdl_launch(k_combine_forward<false>, items, kCombThreads, 0, s, a);
  count_launch();
  return check_launch(p, "k_combine_forward");
}

BackwardFinish backward_finish_args(pme_plan_t p, const IonInputs& in, float* grad_pos, float* grad_q,
                                    float* grad_mu) {
  const CombineArgs a = base_args(p, in);
  BackwardFinish f = {};
  f.pair_out = p->opts.include_pair ? p->pair_out : nullptr;
  f.q = in.q;
  f.mu = in.mu;
  f.gphi = in.gphi;
  f.gfield = in.gfield;
  f.qsum = a.qsum;
  f.grad_pos = grad_pos;
  f.grad_q = grad_q;
  f.grad_mu = grad_mu;
  f.k = a.k;
  f.self_phi = a.self_phi;
  f.self_c = a.self_c;
  f.with_bg = a.with_bg;
  return f;
}

int launch_combine_backward_quad(pme_plan_t p, cudaStream_t s, const IonInputs& in, const double* g_energy,
                                 const float* qmesh, const float* qpair, float* grad_pos, float* grad_q,
                                 float* grad_mu, float* grad_theta) {
  CombineArgs a = base_args(p, in);
  a.with_mesh = 1;
  a.with_pair = p->opts.include_pair != 0;
  a.g_energy = g_energy;
  a.grad_pos = grad_pos;
  a.grad_q = grad_q;
  a.grad_mu = grad_mu;
  const int grid = (in.n + kCombThreads - 1) / kCombThreads;
  if (grid == 0) return PME_OK;
  if (p->batch) k_combine_backward_quad<true><<<grid, kCombThreads, 0, s>>>(a, qmesh, qpair, grad_theta);
  else k_combine_backward_quad<false><<<grid, kCombThreads, 0, s>>>(a, qmesh, qpair, grad_theta);
  count_launch();
  return check_launch(p, "k_combine_backward_quad");
}

int launch_pair_energy(pme_plan_t p, cudaStream_t s, int n, const IonInputs& in,
                       const float* pair_out) {
  const int grid = (n + kCombThreads - 1) / kCombThreads;
  if (grid == 0) return PME_OK;
  k_pair_energy<<<grid, kCombThreads, 0, s>>>(n, in.q, in.mu, pair_out, p->e_ion);
  count_launch();
  return check_launch(p, "k_pair_energy");
}


GBPME_BOUNDS_READER(bounds_hit_combine)

}  // namespace gbpme
