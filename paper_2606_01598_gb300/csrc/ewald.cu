// Explicit Ewald reciprocal sum on the GPU (the conventional baseline the paper times PME
// against; Results, Example 2, timing crossover).
//
//   S(k)      = sum_j (q_j + i mu_j . k) exp(i k . r_j)
//   E_recip   = (2 pi / V) sum_{k != 0} A(k) |S(k)|^2,   A(k) = exp(-k^2 / 4 alpha^2) / k^2
// over the half space of k = n_x b_x + n_y b_y + n_z b_z with |k| <= kmax (each k stands for
// itself and -k), and per ion, with t = A(k) exp(i k . r_i) S*(k),
//   phi_i = (8 pi / V) sum_half Re t,  grad phi_i = -(8 pi / V) sum_half k Im t,
//   grad grad phi_i = -(8 pi / V) sum_half k k^T Re t,
// i.e. the same "potential of the smooth long-range part at the ion" that the mesh gather
// produces, so the pair, self, background and combine stages are shared with the mesh path.
//
// Phases are exact: fractional coordinates are stored as 32-bit fixed point
// u = round(2^32 s), so (n . s mod 1) is the wrapping integer n_x u_x + n_y u_y + n_z u_z and
// the phase 2 pi t, t in [-1/2, 1/2), is evaluated with sincospif at any box size.
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kKThreads = 256;

__global__ void __launch_bounds__(kKThreads)
k_fixed_coords(Geometry g, IonInputs in, uint4* fx, float4* qm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= in.n) return;
  double s[3];
  frac_coords(g, in.pos[3 * i], in.pos[3 * i + 1], in.pos[3 * i + 2], s);
  unsigned u[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    // s in [0,1): round to 32-bit fixed point, wrapping 2^32 to 0
    const double v = floor(s[b] * 4294967296.0 + 0.5);
    u[b] = (v >= 4294967296.0) ? 0u : unsigned(v);
  }
  fx[i] = make_uint4(u[0], u[1], u[2], 0u);
  float q = in.q ? in.q[i] : 0.f;
  float mx = 0.f, my = 0.f, mz = 0.f;
  if (in.mu) {
    mx = in.mu[3 * i];
    my = in.mu[3 * i + 1];
    mz = in.mu[3 * i + 2];
  }
  if (!isfinite(q)) q = 0.f;
  qm[i] = make_float4(q, isfinite(mx) ? mx : 0.f, isfinite(my) ? my : 0.f, isfinite(mz) ? mz : 0.f);
}

__device__ __forceinline__ float phase_frac(int nx, int ny, int nz, uint4 u) {
  const unsigned w = unsigned(nx) * u.x + unsigned(ny) * u.y + unsigned(nz) * u.z;
  return float(int(w)) * 2.3283064365386963e-10f;   // 2^-32, t in [-1/2, 1/2)
}

// One thread per k-vector; ions staged through shared memory in tiles.
__global__ void __launch_bounds__(kKThreads)
k_structure_factor(int K, const int4* kn, const float4* kv, int n, const uint4* fx,
                   const float4* qm, float2* S, double* partials) {
  __shared__ uint4 su[kKThreads];
  __shared__ float4 sq[kKThreads];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int4 nn = make_int4(0, 0, 0, 0);
  float4 kk = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k < K) {
    nn = kn[k];
    kk = kv[k];
  }
  double re = 0.0, im = 0.0;
  for (int base = 0; base < n; base += kKThreads) {
    const int j = base + threadIdx.x;
    __syncthreads();
    if (j < n) {
      su[threadIdx.x] = fx[j];
      sq[threadIdx.x] = qm[j];
    }
    __syncthreads();
    const int m = min(kKThreads, n - base);
    float tr = 0.f, ti = 0.f;
    for (int l = 0; l < m; ++l) {
      const uint4 u = su[l];
      const float4 c = sq[l];
      float sn, cs;
      sincospif(2.f * phase_frac(nn.x, nn.y, nn.z, u), &sn, &cs);
      const float mk = c.y * kk.x + c.z * kk.y + c.w * kk.z;   // mu . k
      tr += c.x * cs - mk * sn;
      ti += c.x * sn + mk * cs;
    }
    re += tr;
    im += ti;
  }
  double e = 0.0;
  if (k < K) {
    S[k] = make_float2(float(re), float(im));
    e = double(__int_as_float(nn.w)) * (re * re + im * im);   // A |S|^2
  }
  const double t = block_sum_d(e);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// One thread per ion; (n, k, A S*) staged through shared memory in tiles.
__global__ void __launch_bounds__(kKThreads)
k_kspace_gather(int K, const int4* kn, const float4* kv, const float2* S, int n, const uint4* fx,
                double pref, float* out) {
  __shared__ int4 sn_[kKThreads];
  __shared__ float4 sk[kKThreads];
  __shared__ float2 ss[kKThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint4 u = (i < n) ? fx[i] : make_uint4(0u, 0u, 0u, 0u);
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int base = 0; base < K; base += kKThreads) {
    const int k = base + threadIdx.x;
    __syncthreads();
    if (k < K) {
      const int4 nn = kn[k];
      const float A = __int_as_float(nn.w);
      const float2 s = S[k];
      sn_[threadIdx.x] = nn;
      sk[threadIdx.x] = kv[k];
      ss[threadIdx.x] = make_float2(A * s.x, -A * s.y);   // A S*
    }
    __syncthreads();
    const int m = min(kKThreads, K - base);
    float a[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int l = 0; l < m; ++l) {
      const int4 nn = sn_[l];
      const float4 kk = sk[l];
      const float2 as = ss[l];
      float sn, cs;
      sincospif(2.f * phase_frac(nn.x, nn.y, nn.z, u), &sn, &cs);
      const float tr = cs * as.x - sn * as.y;   // Re[e^{ik r} A S*]
      const float ti = cs * as.y + sn * as.x;   // Im[...]
      a[0] += tr;
      a[1] -= kk.x * ti;
      a[2] -= kk.y * ti;
      a[3] -= kk.z * ti;
      a[4] -= kk.x * kk.x * tr;
      a[5] -= kk.y * kk.y * tr;
      a[6] -= kk.z * kk.z * tr;
      a[7] -= kk.x * kk.y * tr;
      a[8] -= kk.x * kk.z * tr;
      a[9] -= kk.y * kk.z * tr;
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] += a[c];
  }
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 10; ++c) out[size_t(i) * 10 + c] = float(pref * acc[c]);
  }
}

}  // namespace

// Half-space reciprocal vectors with 0 < |k| <= kmax: n (with A(k) in .w) and k.
int ewald_build_kvectors(pme_plan_t p, std::vector<int4>& kn, std::vector<float4>& kv) {
  const double kmax = p->opts_kmax;
  double b[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) b[r * 3 + c] = 2.0 * kPi * p->g.cinv[c * 3 + r];
  int nmax[3];
  for (int a = 0; a < 3; ++a) {
    const double L = std::sqrt(p->box[3 * a] * p->box[3 * a] + p->box[3 * a + 1] * p->box[3 * a + 1] +
                               p->box[3 * a + 2] * p->box[3 * a + 2]);
    nmax[a] = int(std::ceil(kmax * L / (2.0 * kPi))) + 1;
  }
  kn.clear();
  kv.clear();
  const double a4 = 1.0 / (4.0 * p->alpha * p->alpha);
  for (int x = -nmax[0]; x <= nmax[0]; ++x)
    for (int y = -nmax[1]; y <= nmax[1]; ++y)
      for (int z = -nmax[2]; z <= nmax[2]; ++z) {
        const bool half = (x > 0) || (x == 0 && y > 0) || (x == 0 && y == 0 && z > 0);
        if (!half) continue;
        const double k0 = x * b[0] + y * b[3] + z * b[6];
        const double k1 = x * b[1] + y * b[4] + z * b[7];
        const double k2 = x * b[2] + y * b[5] + z * b[8];
        const double kk = k0 * k0 + k1 * k1 + k2 * k2;
        if (kk > kmax * kmax) continue;
        const float A = float(std::exp(-kk * a4) / kk);
        int4 e;
        e.x = x;
        e.y = y;
        e.z = z;
        std::memcpy(&e.w, &A, sizeof(float));
        kn.push_back(e);
        kv.push_back(make_float4(float(k0), float(k1), float(k2), 0.f));
      }
  return PME_OK;
}

int launch_ewald_recip(pme_plan_t p, cudaStream_t s, const IonInputs& in, double* partials,
                       float* out) {
  const int n = in.n;
  int st;
  if (n > 0) {
    k_fixed_coords<<<(n + kKThreads - 1) / kKThreads, kKThreads, 0, s>>>(p->g, in, p->ew_fx, p->ew_qm);
    count_launch();
    if ((st = check_launch(p, "k_fixed_coords"))) return st;
  }
  const int kb = (p->ew_K + kKThreads - 1) / kKThreads;
  if (kb > 0) {
    k_structure_factor<<<kb, kKThreads, 0, s>>>(p->ew_K, p->ew_kn, p->ew_kv, n, p->ew_fx, p->ew_qm,
                                                p->ew_S, partials);
    count_launch();
    if ((st = check_launch(p, "k_structure_factor"))) return st;
  }
  if (n > 0) {
    k_kspace_gather<<<(n + kKThreads - 1) / kKThreads, kKThreads, 0, s>>>(
        p->ew_K, p->ew_kn, p->ew_kv, p->ew_S, n, p->ew_fx, 8.0 * kPi / p->g.volume, out);
    count_launch();
    if ((st = check_launch(p, "k_kspace_gather"))) return st;
  }
  return PME_OK;
}

int ewald_partial_blocks(pme_plan_t p) { return (p->ew_K + kKThreads - 1) / kKThreads; }

}  // namespace gbpme
