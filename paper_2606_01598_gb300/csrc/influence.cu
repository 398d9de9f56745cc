// Influence multiply and reciprocal energy (Sections 2.3.3-2.3.4, Eqs. Bk, influence, green,
// potential_k, energy_recip).
//
// One pass over each frame's R2C half spectrum [Nx][Ny][Nz/2+1]. For every signed frequency
// n, k = n_x b_x + n_y b_y + n_z b_z, G(k) = 4 pi exp(-k^2 / 4 alpha^2) / k^2 (G(0) = 0) and
// the separable deconvolution C(n) = prod_a 1/sinc^(2 p gamma)(n_a / N_a) (per-axis tables
// built on the host); G C itself depends only on the GPU machine and the mesh, so the plan keeps it
// as a table per frame (k_gc_table, rebuilt when the box changes) and the pass reads it. The energy (1/2V) sum_{n != 0} G C |rho_hat|^2 over the full spectrum
// is accumulated on the half spectrum with weight 2 for the planes that stand for their
// mirror images (0 < n_z < Nz/2) and 1 otherwise; compensated (Neumaier) float sums per
// thread and per warp go to float64 block partials. Each spectrum (and, in the backward pass,
// the tangent spectrum) is then multiplied in place by G C / V, so the C2R transform that
// follows yields Phi with E_recip = 1/2 sum_m rho(m) Phi(m). A batched plan gives every frame
// its own run of blocks. All per-element arithmetic is float32 (the float64 rate of the part
// is a small fraction of its float32 rate), with the constants precomputed on the host.
#include <algorithm>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kInflThreads = 256;

// Neumaier-compensated float accumulation (sum s, running correction c)
__device__ __forceinline__ void comp_add(float& s, float& c, float v) {
  const float t = s + v;
  c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
  s = t;
}

// VIR: also the virial sums S_ab = sum_n w G C |rho_hat|^2 (1/k^2 + 1/(4 alpha^2)) k_a k_b
// (xx yy zz xy xz yz) into vparts[6 * block + c].
template <bool BATCH, bool VIR>
__global__ void __launch_bounds__(kInflThreads)
k_influence(FrameDesc one, FrameMaps maps, float2* spec, int tangent, const float* dconv,
            float inv4a2, double* partials, double* vparts, const float* gtab) {
  pdl_begin();
  const FrameDesc& F = frame_at<BATCH>(one, maps, BATCH ? maps.blk_frame[blockIdx.x] : 0);
  const Geometry& g = F.g;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int Nzh = N2 / 2 + 1;
  const int Mh = N0 * N1 * Nzh;   // < 2^30 (checked when the plan is made)
  const float* cx = dconv + F.dconv_off;
  const float* cy = cx + N0;
  const float* cz = cy + N1;
  const float four_pi = 12.566370614359172f;
  float2* sp = spec + F.spec_off;
  float2* tp = spec + F.tspec_off;
  float e = 0.f, ec = 0.f;
  float sv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, sc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int step = F.infl_nblk * blockDim.x;
  for (int idx = (blockIdx.x - F.infl_blk_off) * blockDim.x + threadIdx.x; idx < Mh; idx += step) {
    const int r = fdiv(idx, F.div_zh);
    const int iz = idx - r * Nzh;
    const int ix = fdiv(r, F.div_y);
    const int iy = r - ix * N1;
    const float nx = float(ix <= N0 / 2 ? ix : ix - N0);
    const float ny = float(iy <= N1 / 2 ? iy : iy - N1);
    const float nz = float(iz);
    const float kx = nx * g.bk[0] + ny * g.bk[3] + nz * g.bk[6];
    const float ky = nx * g.bk[1] + ny * g.bk[4] + nz * g.bk[7];
    const float kz = nx * g.bk[2] + ny * g.bk[5] + nz * g.bk[8];
    const float k2 = kx * kx + ky * ky + kz * kz;
    float gc = 0.f;
    if (gtab) gc = gtab[F.gtab_off + idx];
    else if (k2 > 0.f) gc = four_pi * expf(-k2 * inv4a2) / k2 * cx[ix] * cy[iy] * cz[iz];
    const float2 v = sp[idx];
    const float w = (iz == 0 || (2 * iz == N2)) ? 1.f : 2.f;
    const float eg = w * gc * (v.x * v.x + v.y * v.y);
    comp_add(e, ec, eg);
    if (VIR && k2 > 0.f) {
      const float t = eg * (1.f / k2 + inv4a2);
      comp_add(sv[0], sc[0], t * kx * kx);
      comp_add(sv[1], sc[1], t * ky * ky);
      comp_add(sv[2], sc[2], t * kz * kz);
      comp_add(sv[3], sc[3], t * kx * ky);
      comp_add(sv[4], sc[4], t * kx * kz);
      comp_add(sv[5], sc[5], t * ky * kz);
    }
    const float f = gc * g.inv_volume;
    sp[idx] = make_float2(v.x * f, v.y * f);
    if (tangent) {
      const float2 u = tp[idx];
      tp[idx] = make_float2(u.x * f, u.y * f);
    }
  }
  // warp sums of the compensated pairs in float, then float64 over the block's warps
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, ec, o);
    ec += c2;
    comp_add(e, ec, e2);
  }
  __shared__ double wsum[kInflThreads / 32];
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = double(e) + double(ec);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kInflThreads / 32; ++w) t += wsum[w];
    partials[blockIdx.x] = t;
  }
  if (VIR) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float v = sv[c], cc = sc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, cc, o);
        cc += c2;
        comp_add(v, cc, v2);
      }
      __syncthreads();
      if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = double(v) + double(cc);
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kInflThreads / 32; ++w) t += wsum[w];
        vparts[6 * blockIdx.x + c] = t;
      }
    }
  }
}

// Frame energies: one block per reduction item sums the item's per-ion energies; the last item
// of each frame to finish adds the reciprocal partials, the item partials (both in a fixed
// order) and the background term, times k.
constexpr int kEnergyThreads = 256;

template <bool BATCH>
__global__ void __launch_bounds__(kEnergyThreads)
k_energy_final(FrameDesc one, FrameMaps maps, const double* parts, int recip_kind,
               const double* e_ion, const double* qsum, int with_bg, double alpha, double scale,
               double* eitem, int* ecount, double* out) {
  pdl_begin();
  const int item = blockIdx.x;
  const int f = BATCH ? maps.item_frame[item] : 0;
  const FrameDesc& F = frame_at<BATCH>(one, maps, f);
  int lo, hi;
  item_range(F, item, lo, hi);
  double b = 0.0;
  if (e_ion)
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) b += e_ion[i];
  b = block_sum_d(b);
  if (threadIdx.x == 0) eitem[item] = b;
  if (!last_item_done(ecount + f, F.nitems)) return;
  double a, e;
  strided_sum2_d(parts + F.infl_blk_off, recip_kind ? F.infl_nblk : 0, 1, eitem + F.item_off, F.nitems, 1, a, e);
  block_sum2_d(a, e);
  if (threadIdx.x == 0) {
    const double V = F.g.volume;
    const double coef = recip_kind == 1 ? 0.5 / V : (recip_kind == 2 ? 4.0 * kPi / V : 0.0);
    double bg = 0.0;
    if (with_bg) {
      const double Q = qsum[2 * f];
      bg = -kPi * Q * Q / (2.0 * V * alpha * alpha);
    }
    out[f] = scale * (coef * a + e + bg);
    ecount[f] = 0;
  }
}

// P3M influence table of one frame (influence_kind 1): for every half-spectrum point,
// G(n) = sum_m k_m^2 U_m phi(k_m) / [(sum_m U_m)(sum_m k_m^2 U_m)] with U_m = prod_a
// sinc^(2p)(n_a / N_a + m_a), |m_a| <= kAlias, phi(k) = 4 pi e^{-k^2/4 alpha^2}/k^2 (so
// k_m^2 phi(k_m) = 4 pi e^{-k_m^2/4 alpha^2}); G(0) = 0. Float32 sums of positive terms.
constexpr int kAlias = 2;

__device__ __forceinline__ float sinc_pow2p(float x, int p) {
  const float s = (x == 0.f) ? 1.f : sinpif(x) / (3.14159265358979f * x);
  const float s2 = s * s;
  float r = 1.f;
  for (int k = 0; k < p; ++k) r *= s2;
  return r;
}

__global__ void __launch_bounds__(kInflThreads) k_p3m_table(FrameDesc F, float inv4a2, float* tab) {
  const Geometry& g = F.g;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int Nzh = N2 / 2 + 1;
  const int Mh = N0 * N1 * Nzh;
  const float four_pi = 12.566370614359172f;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Mh; idx += gridDim.x * blockDim.x) {
    const int r = fdiv(idx, F.div_zh);
    const int iz = idx - r * Nzh;
    const int ix = fdiv(r, F.div_y);
    const int iy = r - ix * N1;
    const int n[3] = {ix <= N0 / 2 ? ix : ix - N0, iy <= N1 / 2 ? iy : iy - N1, iz};
    float U[3][2 * kAlias + 1];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int m = -kAlias; m <= kAlias; ++m) U[a][m + kAlias] = sinc_pow2p(float(n[a]) / float(g.N[a]) + float(m), g.order);
    float num = 0.f, s1 = 0.f, s2 = 0.f;
    for (int mx = -kAlias; mx <= kAlias; ++mx)
      for (int my = -kAlias; my <= kAlias; ++my)
        for (int mz = -kAlias; mz <= kAlias; ++mz) {
          const float u = U[0][mx + kAlias] * U[1][my + kAlias] * U[2][mz + kAlias];
          const float fx = float(n[0] + mx * N0), fy = float(n[1] + my * N1), fz = float(n[2] + mz * N2);
          const float kx = fx * g.bk[0] + fy * g.bk[3] + fz * g.bk[6];
          const float ky = fx * g.bk[1] + fy * g.bk[4] + fz * g.bk[7];
          const float kz = fx * g.bk[2] + fy * g.bk[5] + fz * g.bk[8];
          const float k2 = kx * kx + ky * ky + kz * kz;
          num += u * four_pi * expf(-k2 * inv4a2);
          s1 += u;
          s2 += u * k2;
        }
    tab[F.gtab_off + idx] = (idx == 0 || s2 <= 0.f) ? 0.f : num / (s1 * s2);
  }
}

// Influence table of one frame for the default kind: G(k) C(n) at every half-spectrum point,
// the same float expression the multiply would evaluate (G(0) = 0). It depends on the box and
// the mesh only, so the plan builds it once (and again when the box changes) and the
// multiply reads it instead of evaluating exp and a division per point on every call.
__global__ void __launch_bounds__(kInflThreads) k_gc_table(FrameDesc F, const float* dconv, float inv4a2,
                                                           float* tab) {
  const Geometry& g = F.g;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2];
  const int Nzh = N2 / 2 + 1;
  const int Mh = N0 * N1 * Nzh;
  const float* cx = dconv + F.dconv_off;
  const float* cy = cx + N0;
  const float* cz = cy + N1;
  const float four_pi = 12.566370614359172f;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Mh; idx += gridDim.x * blockDim.x) {
    const int r = fdiv(idx, F.div_zh);
    const int iz = idx - r * Nzh;
    const int ix = fdiv(r, F.div_y);
    const int iy = r - ix * N1;
    const float nx = float(ix <= N0 / 2 ? ix : ix - N0);
    const float ny = float(iy <= N1 / 2 ? iy : iy - N1);
    const float nz = float(iz);
    const float kx = nx * g.bk[0] + ny * g.bk[3] + nz * g.bk[6];
    const float ky = nx * g.bk[1] + ny * g.bk[4] + nz * g.bk[7];
    const float kz = nx * g.bk[2] + ny * g.bk[5] + nz * g.bk[8];
    const float k2 = kx * kx + ky * ky + kz * kz;
    float gc = 0.f;
    if (k2 > 0.f) gc = four_pi * expf(-k2 * inv4a2) / k2 * cx[ix] * cy[iy] * cz[iz];
    tab[F.gtab_off + idx] = gc;
  }
}

}  // namespace

int launch_influence_tables(pme_plan_t p, cudaStream_t s) {
  if (p->opts.influence_kind == 1) return launch_p3m_tables(p, s);
  const float inv4a2 = float(1.0 / (4.0 * p->alpha * p->alpha));
  for (int f = 0; f < p->nframes; ++f) {
    const FrameDesc& F = p->frames_h[f];
    const long long Mh = (long long)F.g.N[0] * F.g.N[1] * (F.g.N[2] / 2 + 1);
    const int grid = int(std::min<long long>((Mh + kInflThreads - 1) / kInflThreads, 8LL * device_sm_count()));
    k_gc_table<<<grid, kInflThreads, 0, s>>>(F, p->dconv_all, inv4a2, p->gtab);
    const int st = check_launch(p, "k_gc_table");
    if (st) return st;
  }
  return PME_OK;
}

int launch_p3m_tables(pme_plan_t p, cudaStream_t s) {
  const float inv4a2 = float(1.0 / (4.0 * p->alpha * p->alpha));
  for (int f = 0; f < p->nframes; ++f) {
    const FrameDesc& F = p->frames_h[f];
    const long long Mh = (long long)F.g.N[0] * F.g.N[1] * (F.g.N[2] / 2 + 1);
    const int grid = int(std::min<long long>((Mh + kInflThreads - 1) / kInflThreads, 8LL * device_sm_count()));
    k_p3m_table<<<grid, kInflThreads, 0, s>>>(F, inv4a2, p->gtab);
    const int st = check_launch(p, "k_p3m_table");
    if (st) return st;
  }
  return PME_OK;
}

int influence_blocks(const Geometry& g) {
  const long long Mh = (long long)g.N[0] * g.N[1] * (g.N[2] / 2 + 1);
  const long long want = (Mh + kInflThreads - 1) / kInflThreads;
  const long long cap = 4LL * device_sm_count();
  return int(want < cap ? (want > 0 ? want : 1) : cap);
}

int launch_influence(pme_plan_t p, cudaStream_t s, cufftComplex* spec, bool tangent,
                     double* partials, double* vparts) {
  const float inv4a2 = float(1.0 / (4.0 * p->alpha * p->alpha));
  FrameDesc one = p->frames_h[0];
  float2* sp = reinterpret_cast<float2*>(spec);
  const int grid = p->batch ? p->total_blocks : one.infl_nblk;
  const int tg = tangent ? 1 : 0;
  if (p->batch) {
    if (vparts) pdl_launch(k_influence<true, true>, grid, kInflThreads, 0, s, one, p->maps, sp, tg, p->dconv_all, inv4a2, partials, vparts, p->gtab);
    else pdl_launch(k_influence<true, false>, grid, kInflThreads, 0, s, one, p->maps, sp, tg, p->dconv_all, inv4a2, partials, vparts, p->gtab);
  } else {
    if (vparts) pdl_launch(k_influence<false, true>, grid, kInflThreads, 0, s, one, p->maps, sp, tg, p->dconv_all, inv4a2, partials, vparts, p->gtab);
    else pdl_launch(k_influence<false, false>, grid, kInflThreads, 0, s, one, p->maps, sp, tg, p->dconv_all, inv4a2, partials, vparts, p->gtab);
  }
  count_launch();
  return check_launch(p, "k_influence");
}

int launch_energy_final(pme_plan_t p, cudaStream_t s, const double* parts, int recip_kind,
                        bool with_ions, bool with_bg, double scale, int n_single, double* out) {
  FrameDesc one = p->frames_h[0];
  if (!p->batch) {
    one.n = n_single;
    one.item_off = 0;
    one.nitems = n_single > kRedItem ? (n_single + kRedItem - 1) / kRedItem : 1;
  }
  const double* e_ion = with_ions ? p->e_ion : nullptr;
  const int items = p->batch ? p->total_items : one.nitems;
  if (p->batch)
    pdl_launch(k_energy_final<true>, items, kEnergyThreads, 0, s, one, p->maps, parts, recip_kind, e_ion, p->sb.qsum,
                                                          with_bg ? 1 : 0, p->alpha, scale, p->eitem,
                                                          p->ecount, out);
  else
    pdl_launch(k_energy_final<false>, items, kEnergyThreads, 0, s, one, p->maps, parts, recip_kind, e_ion, p->sb.qsum,
                                                           with_bg ? 1 : 0, p->alpha, scale, p->eitem,
                                                           p->ecount, out);
  count_launch();
  return check_launch(p, "k_energy_final");
}

}  // namespace gbpme
