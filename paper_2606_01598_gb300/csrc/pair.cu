// Real-space pair term of the Ewald split for point charges and point dipoles.
//
// The interaction of multipoles (q_i, mu_i) and (q_j, mu_j) at r = r_i - r_j + n is
// (q_i + mu_i . grad_i)(q_j + mu_j . grad_j) psi(|r|), psi = erfc(alpha r)/r, the short-range
// complement of the Gaussian-screened mesh term (Eq. green). Its radial derivative functions
// B_0 = psi, B_l = [(2l - 1) B_{l-1} + (2 alpha^2)^l exp(-alpha^2 r^2) / (alpha sqrt(pi))] / r^2
// give the derivative tensors of psi; with g1 = -r B1 and, for vectors u, v, w,
//   g2(u)       = -u B1 + r (r.u) B2
//   g3(u,v)     = (u (v.r) + v (u.r) + (u.v) r) B2 - r (u.r)(v.r) B3
//   g4(u,v,w)   = (u (v.w) + v (u.w) + w (u.v)) B2
//                 - (u (v.r)(w.r) + v (u.r)(w.r) + w (u.r)(v.r)
//                    + r ((u.v)(w.r) + (u.w)(v.r) + (v.w)(u.r))) B3 + r (u.r)(v.r)(w.r) B4
// (the contractions of grad^k psi). The potential at i of source j is q_j psi - mu_j . grad psi.
//
// Ions are sorted into cells at least rcut/2 wide; each thread owns one ion and visits the
// 5 x 5 x 5 neighbouring cells (or, along an axis too short for five cells, every periodic
// image within rcut). Displacements are formed from in-cell offsets, which keeps them exact
// to float rounding of a few Angstrom. Every pair is visited from both sides (no atomics);
// per-thread sums are written once per ion.
//
// Forward: out[orig][10] = phi, grad phi (3), grad grad phi (6) of the pair potential.
// Tangent: out[orig][8] = pair part of the backward (grad_r, grad_q, grad_mu), i.e. the
// g_E-weighted gradient plus the Hessian-vector product along (dr, dq, dmu), assembled from
// the potential of the primal sources (q_j, mu_j) up to third derivatives and the potential
// of the tangent sources (dq_j, dmu_j + q_j dr_j, mu_j (x) dr_j) up to second derivatives.
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kPairThreads = 128;

struct PairArgs {
  Geometry g;
  PairRecords pr;
  const int* start_c;
  const double* g_energy;
  float* out;
  int n;
  float c1, c2, c3, c4;   // (2 alpha^2)^l / (alpha sqrt(pi)), l = 1..4
};

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 mk(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return mk(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ void acc(V3& a, V3 b) { a.x += b.x; a.y += b.y; a.z += b.z; }

template <bool TAN>
__global__ void __launch_bounds__(kPairThreads) k_pair(PairArgs a) {
  const Geometry& g = a.g;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int4 ci = a.pr.idx[i];
  const float4 fi = a.pr.fq[i];
  const float4 mi4 = a.pr.mu[i];
  const V3 mu_i = mk(mi4.x, mi4.y, mi4.z);
  const float q_i = fi.w;
  const float alpha = g.alpha;

  float phi = 0.f;
  V3 gphi = mk(0.f, 0.f, 0.f);
  // forward: Hessian of phi, xx yy zz xy xz yz
  float h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // tangent accumulators
  V3 Hdr = mk(0.f, 0.f, 0.f), Hw = mk(0.f, 0.f, 0.f), T3 = mk(0.f, 0.f, 0.f);
  float dphi = 0.f;
  V3 gdphi = mk(0.f, 0.f, 0.f), Hdmu = mk(0.f, 0.f, 0.f);
  V3 dr_i = mk(0.f, 0.f, 0.f), w_i = mk(0.f, 0.f, 0.f);
  float dq_i = 0.f, gE = 0.f;
  if (TAN) {
    const float4 t = a.pr.tq[i];
    const float4 d = a.pr.dr[i];
    gE = a.g_energy ? float(*a.g_energy) : 0.f;
    dq_i = t.x;
    dr_i = mk(d.x, d.y, d.z);
    const V3 dp = mk(t.y, t.z, t.w);   // dmu + q dr
    w_i = gE * mu_i + dp;              // gE mu + dmu + q dr
  }

  for (int ox = -g.kimg[0]; ox <= g.kimg[0]; ++ox) {
    int cx = ci.x + ox;
    cx = ((cx % g.ncell[0]) + g.ncell[0]) % g.ncell[0];
    for (int oy = -g.kimg[1]; oy <= g.kimg[1]; ++oy) {
      int cy = ci.y + oy;
      cy = ((cy % g.ncell[1]) + g.ncell[1]) % g.ncell[1];
      for (int oz = -g.kimg[2]; oz <= g.kimg[2]; ++oz) {
        int cz = ci.z + oz;
        cz = ((cz % g.ncell[2]) + g.ncell[2]) % g.ncell[2];
        const int key = (cx * g.ncell[1] + cy) * g.ncell[2] + cz;
        const int lo = a.start_c[key], hi = a.start_c[key + 1];
        const bool center = (ox == 0) && (oy == 0) && (oz == 0);
        for (int j = lo; j < hi; ++j) {
          if (center && j == i) continue;
          const float4 fj = a.pr.fq[j];
          const float ux = fi.x - fj.x - float(ox);
          const float uy = fi.y - fj.y - float(oy);
          const float uz = fi.z - fj.z - float(oz);
          const V3 r = mk(ux * g.H[0] + uy * g.H[3] + uz * g.H[6],
                          ux * g.H[1] + uy * g.H[4] + uz * g.H[7],
                          ux * g.H[2] + uy * g.H[5] + uz * g.H[8]);
          const float r2 = dot(r, r);
          if (r2 >= g.rcut2) continue;
          const float rinv2 = 1.f / r2;
          const float rr = sqrtf(r2);
          const float ex = expf(-alpha * alpha * r2);
          const float B0 = erfcf(alpha * rr) / rr;
          const float B1 = (B0 + a.c1 * ex) * rinv2;
          const float B2 = (3.f * B1 + a.c2 * ex) * rinv2;
          const float B3 = (5.f * B2 + a.c3 * ex) * rinv2;
          const float4 mj4 = a.pr.mu[j];
          const V3 d = mk(mj4.x, mj4.y, mj4.z);
          const float c = fj.w;
          const float dr_ = dot(d, r);
          phi += c * B0 + dr_ * B1;
          // grad phi = c g1 - g2(d) = -(c B1 + (d.r) B2) r + B1 d
          acc(gphi, (-c * B1 - dr_ * B2) * r + B1 * d);
          if (!TAN) {
            // grad grad phi = c (-I B1 + r r B2) - [(I (d.r) + r d + d r) B2 - r r (d.r) B3]
            const float s_rr = c * B2 + dr_ * B3;
            const float s_I = -c * B1 - dr_ * B2;
            h[0] += s_I + s_rr * r.x * r.x - 2.f * B2 * d.x * r.x;
            h[1] += s_I + s_rr * r.y * r.y - 2.f * B2 * d.y * r.y;
            h[2] += s_I + s_rr * r.z * r.z - 2.f * B2 * d.z * r.z;
            h[3] += s_rr * r.x * r.y - B2 * (r.x * d.y + d.x * r.y);
            h[4] += s_rr * r.x * r.z - B2 * (r.x * d.z + d.x * r.z);
            h[5] += s_rr * r.y * r.z - B2 * (r.y * d.z + d.y * r.z);
          } else {
            const float B4 = (7.f * B3 + a.c4 * ex) * rinv2;
            const float4 tj = a.pr.tq[j];
            const float4 drj4 = a.pr.dr[j];
            const float cp = tj.x;
            const V3 dp = mk(tj.y, tj.z, tj.w);
            const V3 drj = mk(drj4.x, drj4.y, drj4.z);
            // helpers (see file header)
            auto g2 = [&](V3 u) { return (-B1) * u + (dot(r, u) * B2) * r; };
            auto g3 = [&](V3 u, V3 v) {
              const float ur = dot(u, r), vr = dot(v, r);
              return B2 * (vr * u + ur * v + dot(u, v) * r) - (ur * vr * B3) * r;
            };
            auto g4 = [&](V3 u, V3 v, V3 w) {
              const float ur = dot(u, r), vr = dot(v, r), wr = dot(w, r);
              const float uv = dot(u, v), uw = dot(u, w), vw = dot(v, w);
              V3 o = B2 * (vw * u + uw * v + uv * w);
              o = o - B3 * ((vr * wr) * u + (ur * wr) * v + (ur * vr) * w +
                            (uv * wr + uw * vr + vw * ur) * r);
              return o + (B4 * ur * vr * wr) * r;
            };
            // primal potential: third-derivative and Hessian contractions
            acc(Hdr, c * g2(dr_i) - g3(d, dr_i));
            acc(Hw, c * g2(w_i) - g3(d, w_i));
            acc(T3, c * g3(mu_i, dr_i) - g4(d, mu_i, dr_i));
            // tangent potential: sources cp, dp, mu_j (x) dr_j
            const float mjr = dot(d, r), djr = dot(drj, r);
            dphi += cp * B0 + dot(dp, r) * B1 - dot(d, drj) * B1 + mjr * djr * B2;
            acc(gdphi, (-cp * B1) * r - g2(dp) + g3(d, drj));
            acc(Hdmu, cp * g2(mu_i) - g3(dp, mu_i) + g4(d, drj, mu_i));
          }
        }
      }
    }
  }
  const int orig = ci.w;
  if (!TAN) {
    float* o = a.out + size_t(orig) * 10;
    o[0] = phi;
    o[1] = gphi.x;
    o[2] = gphi.y;
    o[3] = gphi.z;
#pragma unroll
    for (int k = 0; k < 6; ++k) o[4 + k] = h[k];
  } else {
    // grad_q = gE phi + dphi + grad phi . dr ; grad_mu = gE grad phi + grad dphi + H dr
    // grad_r = (gE q + dq) grad phi + H w + q grad dphi + (grad grad dphi) mu + T3[mu, dr]
    const float gq = gE * phi + dphi + dot(gphi, dr_i);
    const V3 gm = gE * gphi + gdphi + Hdr;
    const V3 gr = (gE * q_i + dq_i) * gphi + Hw + q_i * gdphi + Hdmu + T3;
    float* o = a.out + size_t(orig) * 8;
    o[0] = gr.x;
    o[1] = gr.y;
    o[2] = gr.z;
    o[3] = gq;
    o[4] = gm.x;
    o[5] = gm.y;
    o[6] = gm.z;
    o[7] = 0.f;
  }
}

}  // namespace

int launch_pair(pme_plan_t p, cudaStream_t s, int n, bool tangent, const IonInputs& in,
                const double* g_energy, float* out) {
  (void)in;
  if (n == 0) return PME_OK;
  PairArgs a;
  a.g = p->g;
  a.pr = p->pr;
  a.start_c = p->sb.start_c;
  a.g_energy = g_energy;
  a.out = out;
  a.n = n;
  const double al = p->alpha;
  const double sp = 1.7724538509055160273;   // sqrt(pi)
  double t = 1.0 / (al * sp);
  double cl[5];
  for (int l = 1; l <= 4; ++l) {
    t *= 2.0 * al * al;
    cl[l] = t;
  }
  a.c1 = float(cl[1]);
  a.c2 = float(cl[2]);
  a.c3 = float(cl[3]);
  a.c4 = float(cl[4]);
  const int grid = (n + kPairThreads - 1) / kPairThreads;
  if (tangent)
    k_pair<true><<<grid, kPairThreads, 0, s>>>(a);
  else
    k_pair<false><<<grid, kPairThreads, 0, s>>>(a);
  count_launch();
  return check_launch(p, "k_pair");
}

}  // namespace gbpme
