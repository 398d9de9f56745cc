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
// Work split: one warp per ion (ions in pair-cell order, cells at least rcut/2 wide, so a
// partner is at most kimg = ceil(rcut / cell width) cells away per axis). Its candidates are
// the (2 kimg + 1)^2 neighbouring (x, y) cell columns, each holding the contiguous run of the
// 2 kimg + 1 z-cells around the ion (one or two ranges at the periodic wrap); when an axis has
// too few cells for distinct offsets, each offset is its own segment and stands for its own
// periodic image. The lanes describe the columns in
// parallel and a warp scan turns them into one dense candidate stream, tested 32 at a time;
// candidates inside rcut are compacted (ballot + popc) into a per-warp shared-memory buffer
// and evaluated with all lanes busy once 32 or more are waiting. Each lane accumulates its share,
// and a warp-shuffle reduction gives the ion's sums. Every pair is visited from both sides
// (no atomics). Displacements are formed from in-cell offsets, which keeps them exact to float
// rounding of a few Angstrom.
//
// Forward: out[orig][10] = phi, grad phi (3), grad grad phi (6) of the pair potential.
// Tangent: out[orig][8] = pair part of the backward (grad_r, grad_q, grad_mu), i.e. the
// g_E-weighted gradient plus the Hessian-vector product along (dr, dq, dmu), assembled from
// the potential of the primal sources (q_j, mu_j) up to third derivatives and the potential
// of the tangent sources (dq_j, dmu_j + q_j dr_j, mu_j (x) dr_j) up to second derivatives;
// every term is linear in the per-pair contributions, so each lane folds its pairs straight
// into the seven outputs before the reduction.
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kPairWarps = 4;
constexpr int kPairThreads = kPairWarps * 32;
constexpr int kHitCap = 96;   // compacted hits buffered per warp

struct PairArgs {
  FrameDesc one;
  FrameMaps maps;
  PairRecords pr;
  const int* start_c;
  const double* g_energy;   // per frame
  float* out;
  int n;
  float alpha;
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

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-lane state of one ion's sums.
template <bool TAN>
struct Acc;

template <>
struct Acc<false> {
  float phi = 0.f;
  V3 g = {0.f, 0.f, 0.f};
  float h[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // xx yy zz xy xz yz
};

template <>
struct Acc<true> {
  float gq = 0.f;
  V3 gm = {0.f, 0.f, 0.f}, gr = {0.f, 0.f, 0.f};
};

// Ion-side data the pair contributions need.
struct Ion {
  V3 mu, dr, w;   // mu_i, dr_i, w_i = gE mu_i + dmu_i + q_i dr_i
  float q, dq, gE;
};

template <bool TAN>
__device__ __forceinline__ void interact(const PairArgs& a, const Ion& I, int j, V3 r, Acc<TAN>& A) {
  const float r2 = dot(r, r);
  const float rinv2 = 1.f / r2;
  const float rr = sqrtf(r2);
  const float alpha = a.alpha;
  const float ex = expf(-alpha * alpha * r2);
  const float B0 = erfcf(alpha * rr) / rr;
  const float B1 = (B0 + a.c1 * ex) * rinv2;
  const float B2 = (3.f * B1 + a.c2 * ex) * rinv2;
  const float B3 = (5.f * B2 + a.c3 * ex) * rinv2;
  const float4 fj = a.pr.fq[j];
  const float4 mj4 = a.pr.mu[j];
  const V3 d = mk(mj4.x, mj4.y, mj4.z);
  const float c = fj.w;
  const float dr_ = dot(d, r);
  const float phi = c * B0 + dr_ * B1;
  // grad phi = c g1 - g2(d) = -(c B1 + (d.r) B2) r + B1 d
  const V3 gphi = (-c * B1 - dr_ * B2) * r + B1 * d;
  if constexpr (!TAN) {
    A.phi += phi;
    acc(A.g, gphi);
    // grad grad phi = c (-I B1 + r r B2) - [(I (d.r) + r d + d r) B2 - r r (d.r) B3]
    const float s_rr = c * B2 + dr_ * B3;
    const float s_I = -c * B1 - dr_ * B2;
    A.h[0] += s_I + s_rr * r.x * r.x - 2.f * B2 * d.x * r.x;
    A.h[1] += s_I + s_rr * r.y * r.y - 2.f * B2 * d.y * r.y;
    A.h[2] += s_I + s_rr * r.z * r.z - 2.f * B2 * d.z * r.z;
    A.h[3] += s_rr * r.x * r.y - B2 * (r.x * d.y + d.x * r.y);
    A.h[4] += s_rr * r.x * r.z - B2 * (r.x * d.z + d.x * r.z);
    A.h[5] += s_rr * r.y * r.z - B2 * (r.y * d.z + d.y * r.z);
  } else {
    const float B4 = (7.f * B3 + a.c4 * ex) * rinv2;
    const float4 tj = a.pr.tq[j];
    const float4 drj4 = a.pr.dr[j];
    const float cp = tj.x;
    const V3 dp = mk(tj.y, tj.z, tj.w);
    const V3 drj = mk(drj4.x, drj4.y, drj4.z);
    auto g2 = [&](V3 u) { return (-B1) * u + (dot(r, u) * B2) * r; };
    auto g3 = [&](V3 u, V3 v) {
      const float ur = dot(u, r), vr = dot(v, r);
      return B2 * (vr * u + ur * v + dot(u, v) * r) - (ur * vr * B3) * r;
    };
    auto g4 = [&](V3 u, V3 v, V3 w) {
      const float ur = dot(u, r), vr = dot(v, r), wr = dot(w, r);
      const float uv = dot(u, v), uw = dot(u, w), vw = dot(v, w);
      V3 o = B2 * (vw * u + uw * v + uv * w);
      o = o - B3 * ((vr * wr) * u + (ur * wr) * v + (ur * vr) * w + (uv * wr + uw * vr + vw * ur) * r);
      return o + (B4 * ur * vr * wr) * r;
    };
    // primal potential: Hessian and third-derivative contractions
    const V3 Hdr = c * g2(I.dr) - g3(d, I.dr);
    const V3 Hw = c * g2(I.w) - g3(d, I.w);
    const V3 T3 = c * g3(I.mu, I.dr) - g4(d, I.mu, I.dr);
    // tangent potential of sources cp, dp, mu_j (x) dr_j
    const float djr = dot(drj, r);
    const float dphi = cp * B0 + dot(dp, r) * B1 - dot(d, drj) * B1 + dr_ * djr * B2;
    const V3 gdphi = (-cp * B1) * r - g2(dp) + g3(d, drj);
    const V3 Hdmu = cp * g2(I.mu) - g3(dp, I.mu) + g4(d, drj, I.mu);
    // grad_q = gE phi + dphi + grad phi . dr ; grad_mu = gE grad phi + grad dphi + H dr
    // grad_r = (gE q + dq) grad phi + H w + q grad dphi + (grad grad dphi) mu + T3[mu, dr]
    A.gq += I.gE * phi + dphi + dot(gphi, I.dr);
    acc(A.gm, I.gE * gphi + gdphi + Hdr);
    acc(A.gr, (I.gE * I.q + I.dq) * gphi + Hw + I.q * gdphi + Hdmu + T3);
  }
}

template <bool TAN, bool BATCH>
__global__ void __launch_bounds__(kPairThreads) k_pair(PairArgs a) {
  __shared__ int s_j[kPairWarps][kHitCap];
  __shared__ float s_r[kPairWarps][3][kHitCap];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kPairWarps + w;
  if (i >= a.n) return;   // uniform per warp
  const int frame = BATCH ? a.maps.sorted_frame[i] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, frame);
  const Geometry& g = F.g;
  const int4 ci = a.pr.idx[i];
  const float4 fi = a.pr.fq[i];
  const float4 mi4 = a.pr.mu[i];
  Ion I;
  I.mu = mk(mi4.x, mi4.y, mi4.z);
  I.q = fi.w;
  I.dq = 0.f;
  I.gE = 0.f;
  I.dr = mk(0.f, 0.f, 0.f);
  I.w = mk(0.f, 0.f, 0.f);
  if (TAN) {
    const float4 t = a.pr.tq[i];
    const float4 d = a.pr.dr[i];
    I.gE = a.g_energy ? float(a.g_energy[frame]) : 0.f;
    I.dq = t.x;
    I.dr = mk(d.x, d.y, d.z);
    I.w = I.gE * I.mu + mk(t.y, t.z, t.w);   // gE mu + dmu + q dr
  }
  Acc<TAN> A;
  int cnt = 0;
  int* sj = s_j[w];
  float* sx = s_r[w][0];
  float* sy = s_r[w][1];
  float* sz = s_r[w][2];

  auto flush = [&]() {
    __syncwarp();
    for (int k = lane; k < cnt; k += 32) interact<TAN>(a, I, sj[k], mk(sx[k], sy[k], sz[k]), A);
    __syncwarp();
    cnt = 0;
  };
  // test candidate j (valid lanes only) with cell offsets (ox, oy, oz); append the hits
  auto test = [&](bool valid, int j, int ox, int oy, int oz) {
    bool hit = false;
    V3 r = mk(0.f, 0.f, 0.f);
    if (valid) {
      const float4 fj = a.pr.fq[j];
      const float ux = fi.x - fj.x - float(ox);
      const float uy = fi.y - fj.y - float(oy);
      const float uz = fi.z - fj.z - float(oz);
      r = mk(ux * g.H[0] + uy * g.H[3] + uz * g.H[6], ux * g.H[1] + uy * g.H[4] + uz * g.H[7],
             ux * g.H[2] + uy * g.H[5] + uz * g.H[8]);
      hit = dot(r, r) < g.rcut2 && !(j == i && ox == 0 && oy == 0 && oz == 0);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int k = cnt + __popc(bal & ((1u << lane) - 1u));
      sj[k] = j;
      sx[k] = r.x;
      sy[k] = r.y;
      sz[k] = r.z;
    }
    cnt += __popc(bal);
    if (cnt > kHitCap - 32) flush();
  };

  // ---- dense candidate stream ---------------------------------------------------------
  // A segment is one (ox, oy[, oz]) neighbour column: the ions of one or two contiguous
  // ranges of the cell order. Lane l describes segment (32 g + l) of group g; a warp scan of
  // the lengths lets every lane pick its candidate c = base + lane of the group's
  // concatenated ranges by a 5-step shuffle search, so each 32-wide chunk holds 32 candidates.
  const int ncx = g.ncell[0], ncy = g.ncell[1], ncz = g.ncell[2];
  const int kx = g.kimg[0], ky = g.kimg[1], kz = g.kimg[2];
  const bool zrun = ncz >= 2 * kz + 1;              // the z-cells of a column are distinct:
                                                    // z offsets come from the candidate's cell
  const int nzs = zrun ? 1 : 2 * kz + 1;            // segments per (ox, oy) column
  const int nseg = (2 * kx + 1) * (2 * ky + 1) * nzs;
  for (int g0 = 0; g0 < nseg; g0 += 32) {
    const int sidx = g0 + lane;
    int loA = 0, lenA = 0, loB = 0, lenB = 0, code = 0;
    if (sidx < nseg) {
      const int oz = zrun ? 0 : (sidx % nzs) - kz;
      const int t = sidx / nzs;
      const int oy = (t % (2 * ky + 1)) - ky;
      const int ox = (t / (2 * ky + 1)) - kx;
      int cx = (ci.x + ox) % ncx, cy = (ci.y + oy) % ncy;
      if (cx < 0) cx += ncx;
      if (cy < 0) cy += ncy;
      const int row = F.cell_off + (cx * ncy + cy) * ncz;
      if (zrun) {
        const int z0 = ci.z - kz, z1 = ci.z + kz;
        if (z0 < 0) {
          loA = a.start_c[row + z0 + ncz]; lenA = a.start_c[row + ncz] - loA;
          loB = a.start_c[row]; lenB = a.start_c[row + z1 + 1] - loB;
        } else if (z1 >= ncz) {
          loA = a.start_c[row + z0]; lenA = a.start_c[row + ncz] - loA;
          loB = a.start_c[row]; lenB = a.start_c[row + z1 - ncz + 1] - loB;
        } else {
          loA = a.start_c[row + z0]; lenA = a.start_c[row + z1 + 1] - loA;
        }
      } else {
        int cz = (ci.z + oz) % ncz;
        if (cz < 0) cz += ncz;
        loA = a.start_c[row + cz]; lenA = a.start_c[row + cz + 1] - loA;
      }
      // offsets packed in one int: 10 bits each, biased by 512
      code = ((ox + 512) << 20) | ((oy + 512) << 10) | (oz + 512);
    }
    const int len = lenA + lenB;
    int pre = len;   // inclusive scan over the group's segments
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += u;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    for (int base = 0; base < total; base += 32) {
      const int c = base + lane;
      // smallest segment s with pre[s] > c
      int sl = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, pre, sl + step - 1);
        if (v <= c) sl += step;
      }
      const int sp = __shfl_sync(0xffffffffu, pre, sl);
      const int sl_len = __shfl_sync(0xffffffffu, len, sl);
      const int sa = __shfl_sync(0xffffffffu, loA, sl);
      const int sla = __shfl_sync(0xffffffffu, lenA, sl);
      const int sb = __shfl_sync(0xffffffffu, loB, sl);
      const int scode = __shfl_sync(0xffffffffu, code, sl);
      const bool valid = c < total;
      const int off = c - (sp - sl_len);
      const int j = valid ? ((off < sla) ? sa + off : sb + (off - sla)) : 0;
      const int ox = ((scode >> 20) & 1023) - 512;
      const int oy = ((scode >> 10) & 1023) - 512;
      int oz = (scode & 1023) - 512;
      if (zrun && valid) {
        oz = a.pr.cz[j] - ci.z;
        if (oz > kz) oz -= ncz;
        else if (oz < -kz) oz += ncz;
      }
      test(valid, j, ox, oy, oz);
    }
  }
  if (cnt > 0) flush();

  const int orig = ci.w;
  if constexpr (!TAN) {
    const float phi = warp_sum(A.phi);
    const float gx = warp_sum(A.g.x), gy = warp_sum(A.g.y), gz = warp_sum(A.g.z);
    float h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = warp_sum(A.h[k]);
    if (lane == 0) {
      float* o = a.out + size_t(orig) * 10;
      o[0] = phi;
      o[1] = gx;
      o[2] = gy;
      o[3] = gz;
#pragma unroll
      for (int k = 0; k < 6; ++k) o[4 + k] = h[k];
    }
  } else {
    const float rx = warp_sum(A.gr.x), ry = warp_sum(A.gr.y), rz = warp_sum(A.gr.z);
    const float q = warp_sum(A.gq);
    const float mx = warp_sum(A.gm.x), my = warp_sum(A.gm.y), mz = warp_sum(A.gm.z);
    if (lane == 0) {
      float* o = a.out + size_t(orig) * 8;
      o[0] = rx;
      o[1] = ry;
      o[2] = rz;
      o[3] = q;
      o[4] = mx;
      o[5] = my;
      o[6] = mz;
      o[7] = 0.f;
    }
  }
}

}  // namespace

int launch_pair(pme_plan_t p, cudaStream_t s, int n, bool tangent, const IonInputs& in,
                const double* g_energy, float* out) {
  (void)in;
  if (n == 0) return PME_OK;
  PairArgs a;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.alpha = float(p->alpha);
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
  const int grid = (n + kPairWarps - 1) / kPairWarps;
  if (p->batch) {
    if (tangent) k_pair<true, true><<<grid, kPairThreads, 0, s>>>(a);
    else k_pair<false, true><<<grid, kPairThreads, 0, s>>>(a);
  } else {
    if (tangent) k_pair<true, false><<<grid, kPairThreads, 0, s>>>(a);
    else k_pair<false, false><<<grid, kPairThreads, 0, s>>>(a);
  }
  count_launch();
  return check_launch(p, "k_pair");
}

}  // namespace gbpme
