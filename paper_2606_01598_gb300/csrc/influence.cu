// Influence multiply and reciprocal energy (Sections 2.3.3-2.3.4, Eqs. Bk, influence, green,
// potential_k, energy_recip).
//
// One pass over the R2C half spectrum [Nx][Ny][Nz/2+1]. For every signed frequency n,
// k = n_x b_x + n_y b_y + n_z b_z, G(k) = 4 pi exp(-k^2 / 4 alpha^2) / k^2 (G(0) = 0) and the
// separable deconvolution C(n) = prod_a 1/sinc^(2 p gamma)(n_a / N_a) (per-axis tables built
// on the host). The energy (1/2V) sum_{n != 0} G C |rho_hat|^2 over the full spectrum is
// accumulated on the half spectrum with weight 2 for the planes that stand for their mirror
// images (0 < n_z < Nz/2) and 1 otherwise; per-thread float sums go to float64 block
// partials. Each spectrum is then multiplied in place by G C / V, so the C2R transform that
// follows yields Phi with E_recip = 1/2 sum_m rho(m) Phi(m).
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kInflThreads = 256;

struct InflArgs {
  int N[3];
  int Nzh;
  long long Mh;
  float b[9];          // rows b_x, b_y, b_z
  float inv4a2;        // 1 / (4 alpha^2)
  float inv_volume;
  const float* cx;
  const float* cy;
  const float* cz;
};

__global__ void __launch_bounds__(kInflThreads)
k_influence(InflArgs a, float2* spec, int nspec, long long stride, double* partials) {
  float e = 0.f;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.Mh; idx += step) {
    const int iz = int(idx % a.Nzh);
    const long long r = idx / a.Nzh;
    const int iy = int(r % a.N[1]);
    const int ix = int(r / a.N[1]);
    const float nx = float(ix <= a.N[0] / 2 ? ix : ix - a.N[0]);
    const float ny = float(iy <= a.N[1] / 2 ? iy : iy - a.N[1]);
    const float nz = float(iz);
    const float kx = nx * a.b[0] + ny * a.b[3] + nz * a.b[6];
    const float ky = nx * a.b[1] + ny * a.b[4] + nz * a.b[7];
    const float kz = nx * a.b[2] + ny * a.b[5] + nz * a.b[8];
    const float k2 = kx * kx + ky * ky + kz * kz;
    float gc = 0.f;
    if (k2 > 0.f) gc = 4.f * 3.14159265358979f * expf(-k2 * a.inv4a2) / k2 * a.cx[ix] * a.cy[iy] * a.cz[iz];
    const float2 v = spec[idx];
    const float w = (iz == 0 || (2 * iz == a.N[2])) ? 1.f : 2.f;
    e += w * gc * (v.x * v.x + v.y * v.y);
    const float f = gc * a.inv_volume;
    spec[idx] = make_float2(v.x * f, v.y * f);
    for (int s = 1; s < nspec; ++s) {
      const float2 u = spec[idx + s * stride];
      spec[idx + s * stride] = make_float2(u.x * f, u.y * f);
    }
  }
  const double t = block_sum_d(double(e));
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Final float64 energy: out = scale * (coef_a * sum parts[0, na) + sum parts[na, na + nb))
//                              + background(Q) where background = bgfac * Q^2.
__global__ void __launch_bounds__(1024)
k_energy_final(const double* parts, int na, int nb, double coef_a, double scale,
               double bgfac, const double* qsum, double* out) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < na; k += blockDim.x) a += parts[k];
  for (int k = threadIdx.x; k < nb; k += blockDim.x) b += parts[na + k];
  a = block_sum_d(a);
  b = block_sum_d(b);
  if (threadIdx.x == 0) {
    double q = qsum ? qsum[0] : 0.0;
    out[0] = scale * (coef_a * a + b + bgfac * q * q);
  }
}

}  // namespace

int influence_grid(pme_plan_t p) {
  long long want = (p->Mh + kInflThreads - 1) / kInflThreads;
  long long cap = 152 * 8;
  return int(want < cap ? (want > 0 ? want : 1) : cap);
}

int launch_influence(pme_plan_t p, cudaStream_t s, cufftComplex* spec, int nspec,
                     double* partials) {
  InflArgs a;
  for (int d = 0; d < 3; ++d) a.N[d] = p->g.N[d];
  a.Nzh = p->g.N[2] / 2 + 1;
  a.Mh = p->Mh;
  // b rows = 2 pi C^{-T} rows: b_a[c] = 2 pi cinv[c][a]
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) a.b[r * 3 + c] = float(2.0 * kPi * p->g.cinv[c * 3 + r]);
  a.inv4a2 = float(1.0 / (4.0 * p->alpha * p->alpha));
  a.inv_volume = float(1.0 / p->g.volume);
  a.cx = p->dconv[0];
  a.cy = p->dconv[1];
  a.cz = p->dconv[2];
  const int grid = influence_grid(p);
  k_influence<<<grid, kInflThreads, 0, s>>>(a, reinterpret_cast<float2*>(spec), nspec, p->Mh,
                                            partials);
  count_launch();
  return check_launch(p, "k_influence");
}

int launch_energy_final(pme_plan_t p, cudaStream_t s, const double* parts, int na, int nb,
                        double coef_a, double scale, double bgfac, const double* qsum,
                        double* out) {
  k_energy_final<<<1, 1024, 0, s>>>(parts, na, nb, coef_a, scale, bgfac, qsum, out);
  count_launch();
  return check_launch(p, "k_energy_final");
}

}  // namespace gbpme
