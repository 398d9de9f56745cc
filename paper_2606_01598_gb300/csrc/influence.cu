// Influence multiply and reciprocal energy (Sections 2.3.3-2.3.4, Eqs. Bk, influence, green,
// potential_k, energy_recip).
//
// One pass over each frame's R2C half spectrum [Nx][Ny][Nz/2+1]. For every signed frequency
// n, k = n_x b_x + n_y b_y + n_z b_z, G(k) = 4 pi exp(-k^2 / 4 alpha^2) / k^2 (G(0) = 0) and
// the separable deconvolution C(n) = prod_a 1/sinc^(2 p gamma)(n_a / N_a) (per-axis tables
// built on the host). The energy (1/2V) sum_{n != 0} G C |rho_hat|^2 over the full spectrum
// is accumulated on the half spectrum with weight 2 for the planes that stand for their
// mirror images (0 < n_z < Nz/2) and 1 otherwise; per-thread float sums go to float64 block
// partials. Each spectrum (and, in the backward pass, the tangent spectrum) is then multiplied
// in place by G C / V, so the C2R transform that follows yields Phi with
// E_recip = 1/2 sum_m rho(m) Phi(m). A batched plan gives every frame its own run of blocks.
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kInflThreads = 256;
constexpr int kInflMaxBlocks = 152 * 8;

template <bool BATCH>
__global__ void __launch_bounds__(kInflThreads)
k_influence(FrameDesc one, FrameMaps maps, float2* spec, int tangent, const float* dconv,
            float inv4a2, double* partials) {
  const FrameDesc& F = frame_at<BATCH>(one, maps, BATCH ? maps.blk_frame[blockIdx.x] : 0);
  const Geometry& g = F.g;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int Nzh = N2 / 2 + 1;
  const long long Mh = (long long)N0 * N1 * Nzh;
  float b[9];   // rows b_x, b_y, b_z of 2 pi C^{-T}: b_r[c] = 2 pi cinv[c][r]
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) b[r * 3 + c] = float(2.0 * kPi * g.cinv[c * 3 + r]);
  const float inv_volume = float(1.0 / g.volume);
  const float* cx = dconv + F.dconv_off;
  const float* cy = cx + N0;
  const float* cz = cy + N1;
  float2* sp = spec + F.spec_off;
  float2* tp = spec + F.tspec_off;
  float e = 0.f;
  const long long step = (long long)F.infl_nblk * blockDim.x;
  for (long long idx = (long long)(blockIdx.x - F.infl_blk_off) * blockDim.x + threadIdx.x; idx < Mh;
       idx += step) {
    const int iz = int(idx % Nzh);
    const long long r = idx / Nzh;
    const int iy = int(r % N1);
    const int ix = int(r / N1);
    const float nx = float(ix <= N0 / 2 ? ix : ix - N0);
    const float ny = float(iy <= N1 / 2 ? iy : iy - N1);
    const float nz = float(iz);
    const float kx = nx * b[0] + ny * b[3] + nz * b[6];
    const float ky = nx * b[1] + ny * b[4] + nz * b[7];
    const float kz = nx * b[2] + ny * b[5] + nz * b[8];
    const float k2 = kx * kx + ky * ky + kz * kz;
    float gc = 0.f;
    if (k2 > 0.f) gc = 4.f * 3.14159265358979f * expf(-k2 * inv4a2) / k2 * cx[ix] * cy[iy] * cz[iz];
    const float2 v = sp[idx];
    const float w = (iz == 0 || (2 * iz == N2)) ? 1.f : 2.f;
    e += w * gc * (v.x * v.x + v.y * v.y);
    const float f = gc * inv_volume;
    sp[idx] = make_float2(v.x * f, v.y * f);
    if (tangent) {
      const float2 u = tp[idx];
      tp[idx] = make_float2(u.x * f, u.y * f);
    }
  }
  const double t = block_sum_d(double(e));
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// One block per frame: reciprocal partials, per-ion energies and background, times k.
template <bool BATCH>
__global__ void __launch_bounds__(1024)
k_energy_final(FrameDesc one, FrameMaps maps, const double* parts, int recip_kind,
               const double* e_ion, const double* qsum, int with_bg, double alpha, double scale,
               double* out) {
  const FrameDesc& F = frame_at<BATCH>(one, maps, blockIdx.x);
  double a = 0.0, b = 0.0;
  if (recip_kind)
    for (int k = threadIdx.x; k < F.infl_nblk; k += blockDim.x) a += parts[F.infl_blk_off + k];
  if (e_ion)
    for (int k = threadIdx.x; k < F.n; k += blockDim.x) b += e_ion[F.ion_off + k];
  a = block_sum_d(a);
  b = block_sum_d(b);
  if (threadIdx.x == 0) {
    const double V = F.g.volume;
    const double coef = recip_kind == 1 ? 0.5 / V : (recip_kind == 2 ? 4.0 * kPi / V : 0.0);
    double bg = 0.0;
    if (with_bg) {
      const double Q = qsum[2 * blockIdx.x];
      bg = -kPi * Q * Q / (2.0 * V * alpha * alpha);
    }
    out[blockIdx.x] = scale * (coef * a + b + bg);
  }
}

}  // namespace

int influence_blocks(const Geometry& g) {
  const long long Mh = (long long)g.N[0] * g.N[1] * (g.N[2] / 2 + 1);
  const long long want = (Mh + kInflThreads - 1) / kInflThreads;
  return int(want < kInflMaxBlocks ? (want > 0 ? want : 1) : kInflMaxBlocks);
}

int launch_influence(pme_plan_t p, cudaStream_t s, cufftComplex* spec, bool tangent,
                     double* partials) {
  const float inv4a2 = float(1.0 / (4.0 * p->alpha * p->alpha));
  FrameDesc one = p->frames_h[0];
  if (p->batch)
    k_influence<true><<<p->total_blocks, kInflThreads, 0, s>>>(one, p->maps, reinterpret_cast<float2*>(spec),
                                                              tangent ? 1 : 0, p->dconv_all, inv4a2, partials);
  else
    k_influence<false><<<one.infl_nblk, kInflThreads, 0, s>>>(one, p->maps, reinterpret_cast<float2*>(spec),
                                                             tangent ? 1 : 0, p->dconv_all, inv4a2, partials);
  count_launch();
  return check_launch(p, "k_influence");
}

int launch_energy_final(pme_plan_t p, cudaStream_t s, const double* parts, int recip_kind,
                        bool with_ions, bool with_bg, double scale, int n_single, double* out) {
  FrameDesc one = p->frames_h[0];
  if (!p->batch) one.n = n_single;
  const double* e_ion = with_ions ? p->e_ion : nullptr;
  if (p->batch)
    k_energy_final<true><<<p->nframes, 1024, 0, s>>>(one, p->maps, parts, recip_kind, e_ion, p->sb.qsum,
                                                     with_bg ? 1 : 0, p->alpha, scale, out);
  else
    k_energy_final<false><<<1, 1024, 0, s>>>(one, p->maps, parts, recip_kind, e_ion, p->sb.qsum,
                                             with_bg ? 1 : 0, p->alpha, scale, out);
  count_launch();
  return check_launch(p, "k_energy_final");
}

}  // namespace gbpme
