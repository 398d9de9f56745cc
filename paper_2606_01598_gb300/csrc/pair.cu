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
// Work split: one warp per pair cell (cells at least rcut/2 wide, so a partner is at most
// kimg = ceil(rcut / cell width) cells away per axis); the warp handles the cell's ions a few
// at a time (four in the fused pass, eight in the list pass), and they share one candidate
// stream. The candidates are the
// (2 kimg + 1)^2 neighbouring (x, y) cell columns, each holding the contiguous run of the
// 2 kimg + 1 z-cells around the cell (one or two ranges at the periodic wrap); when an axis
// has too few cells for distinct offsets, each offset is its own segment and stands for its
// own periodic image. The lanes describe the columns in parallel and a warp scan turns them
// into one dense candidate stream, loaded 32 at a time; each candidate is tested against
// every ion of the group, and the ones inside rcut are compacted (ballot + popc) into that
// ion's shared-memory hit list. Whenever a list holds 32 hits they are evaluated with all
// lanes busy (the remainder waits for the next chunk). Each lane accumulates its share and a
// warp-shuffle reduction gives each ion's sums. Every pair is visited from both sides (no
// atomics), and every sum runs in a fixed order. Displacements are formed from in-cell
// offsets, which keeps them exact to float rounding of a few Angstrom.
//
// Forward: out[orig][10] = phi, grad phi (3), grad grad phi (6) of the pair potential.
// Tangent: out[orig][8] = pair part of the backward (grad_r, grad_q, grad_mu), i.e. the
// g_E-weighted gradient plus the Hessian-vector product along (dr, dq, dmu), assembled from
// the potential of the primal sources (q_j, mu_j) up to third derivatives and the potential
// of the tangent sources (dq_j, dmu_j + q_j dr_j, mu_j (x) dr_j) up to second derivatives;
// every term is linear in the per-pair contributions, so each lane folds its pairs straight
// into the seven outputs before the reduction.
//
// Rounding: this file is compiled with -fmad=false, so a multiply and an add fuse only where
// fmaf_ below says so. The fused and the list-driven kernels inline the same pair expressions
// into different code; with contraction left to the compiler, the two could round a term
// differently (the choice depends on the surrounding code), and the two paths would no longer
// agree bit for bit.
#include <algorithm>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kPairWarps = 4;
constexpr int kPairThreads = kPairWarps * 32;
constexpr int kSlots = 4;      // ions of one cell sharing a candidate stream
constexpr int kSlotCap = 64;   // buffered hits per ion (< 32 wait between chunks)
constexpr int kCandCap = 512;  // candidates listed per warp at a time
constexpr int kSegShift = 27;  // candidate entry: (segment lane << 27) | sorted index

struct PairArgs {
  FrameDesc one;
  FrameMaps maps;
  PairRecords pr;
  const int* start_c;
  const double* g_energy;   // per frame
  float* out;
  int cell_lo, ncells;      // global cell keys handled by this launch
  // per-ion hit lists (r, j) in stream order, pair-cell order; list_cnt = hits, or -1 when
  // more than list_cap
  float4* list;
  int* list_cnt;
  int list_cap;
  // *cache_bad == 0: the lists hold for this pass -- the fused kernel returns at once and
  // the list-driven one runs (fused kernel: null means always run)
  const int* cache_bad;
  // virial: per-ion 1/2 sum_j F_ij (x) r_ij [9] (caller order), forward list pass only
  float* vir_out;
  // fused fallback of a virial pass: it cannot form the pair virial, so it reports
  int* vir_lost;
  float alpha;
  float c1, c2, c3, c4;   // (2 alpha^2)^l / (alpha sqrt(pi)), l = 1..4
};

struct V3 {
  float x, y, z;
};
__device__ __forceinline__ V3 mk(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ float fmaf_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf_(a.x, b.x, fmaf_(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
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
// vir (forward only, nullable): adds 1/2 F_ij (x) r_ij, with F_ij = -(q_i grad phi_ij +
// (grad grad phi_ij) mu_i) the force on i from j, row-major [9].
__device__ __forceinline__ void interact(const PairArgs& a, const Ion& I, int j, V3 r, Acc<TAN>& A,
                                         float* vir = nullptr) {
  const float r2 = dot(r, r);
  const float rinv = rsqrtf(r2);
  const float rinv2 = rinv * rinv;
  const float rr = r2 * rinv;
  const float alpha = a.alpha;
  const float ex = expf(-alpha * alpha * r2);
  const float B0 = erfcf(alpha * rr) * rinv;
  const float B1 = fmaf_(a.c1, ex, B0) * rinv2;
  const float B2 = fmaf_(a.c2, ex, 3.f * B1) * rinv2;
  const float B3 = fmaf_(a.c3, ex, 5.f * B2) * rinv2;
  const float4 mj4 = a.pr.mu[j];
  const V3 d = mk(mj4.x, mj4.y, mj4.z);
  const float c = mj4.w;
  const float rd = dot(d, r);
  const float phi = fmaf_(c, B0, rd * B1);
  // grad phi = c g1 - g2(d) = -(c B1 + (d.r) B2) r + B1 d = al r + B1 d
  const float al = -fmaf_(c, B1, rd * B2);
  const V3 gphi = mk(fmaf_(al, r.x, B1 * d.x), fmaf_(al, r.y, B1 * d.y), fmaf_(al, r.z, B1 * d.z));
  // s_rr = c B2 + (d.r) B3, the coefficient of r r in grad grad phi
  const float s_rr = fmaf_(c, B2, rd * B3);
  if constexpr (!TAN) {
    A.phi += phi;
    acc(A.g, gphi);
    // grad grad phi = c (-I B1 + r r B2) - [(I (d.r) + r d + d r) B2 - r r (d.r) B3]
    //               = al I + s_rr r r - B2 (r d + d r)
    const V3 u = s_rr * r, b = B2 * d;
    float h[6];
    h[0] = fmaf_(fmaf_(-2.f, b.x, u.x), r.x, al);
    h[1] = fmaf_(fmaf_(-2.f, b.y, u.y), r.y, al);
    h[2] = fmaf_(fmaf_(-2.f, b.z, u.z), r.z, al);
    h[3] = fmaf_(u.x, r.y, -fmaf_(r.x, b.y, b.x * r.y));
    h[4] = fmaf_(u.x, r.z, -fmaf_(r.x, b.z, b.x * r.z));
    h[5] = fmaf_(u.y, r.z, -fmaf_(r.y, b.z, b.y * r.z));
#pragma unroll
    for (int k = 0; k < 6; ++k) A.h[k] += h[k];
    if (vir) {
      const V3 m = I.mu;
      const float Fx = -fmaf_(I.q, gphi.x, fmaf_(h[0], m.x, fmaf_(h[3], m.y, h[4] * m.z)));
      const float Fy = -fmaf_(I.q, gphi.y, fmaf_(h[3], m.x, fmaf_(h[1], m.y, h[5] * m.z)));
      const float Fz = -fmaf_(I.q, gphi.z, fmaf_(h[4], m.x, fmaf_(h[5], m.y, h[2] * m.z)));
      const float hx = 0.5f * Fx, hy = 0.5f * Fy, hz = 0.5f * Fz;
      vir[0] = fmaf_(hx, r.x, vir[0]);
      vir[1] = fmaf_(hx, r.y, vir[1]);
      vir[2] = fmaf_(hx, r.z, vir[2]);
      vir[3] = fmaf_(hy, r.x, vir[3]);
      vir[4] = fmaf_(hy, r.y, vir[4]);
      vir[5] = fmaf_(hy, r.z, vir[5]);
      vir[6] = fmaf_(hz, r.x, vir[6]);
      vir[7] = fmaf_(hz, r.y, vir[7]);
      vir[8] = fmaf_(hz, r.z, vir[8]);
    }
  } else {
    const float B4 = fmaf_(a.c4, ex, 7.f * B3) * rinv2;
    const float4 tj = a.pr.tq[j];
    const float4 drj4 = a.pr.dr[j];
    const float cp = tj.x;                       // tangent charge of j
    const V3 dp = mk(tj.y, tj.z, tj.w);          // tangent dipole d'_j = dmu_j + q_j dr_j
    const V3 drj = mk(drj4.x, drj4.y, drj4.z);   // dr_j
    const V3 m = I.mu, t = I.dr, w = I.w;
    // Every term below is a contraction of grad^k psi (k <= 4) with the vectors r, d = mu_j,
    // d', dr_j, mu_i, dr_i, w_i; it is written as a combination of those vectors with scalar
    // coefficients built from their dot products:
    //   H(u)      = (grad grad phi) u            = al u + (ru s_rr - B2 du) r - B2 ru d
    //   T3        = (grad^3 phi)[mu_i, dr_i]
    //   gdphi     = grad of the potential of the tangent sources (cp, d', mu_j (x) dr_j)
    //   Hdmu      = (grad grad dphi) mu_i
    // with al = -(c B1 + rd B2), s_rr = c B2 + rd B3 (the coefficients of g2 / g3 / g4
    // contractions of the header, expanded).
    const float rm = dot(r, m), rt = dot(r, t), rw = dot(r, w);
    const float rdp = dot(r, dp), rdj = dot(r, drj);
    const float d_t = dot(d, t), d_w = dot(d, w), d_m = dot(d, m), m_t = dot(m, t);
    const float dp_m = dot(dp, m), dj_m = dot(drj, m), d_dj = dot(d, drj);
    const float rd_rdj = rd * rdj;
    // dphi = cp B0 + (rdp - d_dj) B1 + rd rdj B2
    const float dphi = fmaf_(cp, B0, fmaf_(rdp - d_dj, B1, rd_rdj * B2));
    // gdphi = gd_r r + B1 d' + B2 rdj d + B2 rd dr_j, gd_r = -cp B1 + (d_dj - rdp) B2 - rd rdj B3;
    // gd_r is also the coefficient of m in Hdmu
    const float gd_r = fmaf_(-cp, B1, fmaf_(d_dj - rdp, B2, -(rd_rdj * B3)));
    // T3 on m, t, d, r
    const float T_m = fmaf_(s_rr, rt, -(B2 * d_t));
    const float T_t = fmaf_(s_rr, rm, -(B2 * d_m));
    const float rm_rt = rm * rt;
    const float T_d = fmaf_(B3, rm_rt, -(B2 * m_t));
    // T_r = c B2 m_t + B3 (d_m rt + d_t rm + m_t rd - c rm rt) - B4 rd rm rt
    const float T_in = fmaf_(d_m, rt, fmaf_(d_t, rm, fmaf_(m_t, rd, -(c * rm_rt))));
    const float T_r = fmaf_(c * B2, m_t, fmaf_(B3, T_in, -(B4 * rd * rm_rt)));
    // Hdmu on r, d', d, dr_j:
    // D_r = B2 (cp rm - dp_m) + B3 ((rdp - d_dj) rm - d_m rdj - dj_m rd) + B4 rd rdj rm
    const float D_in = fmaf_(rdp - d_dj, rm, -fmaf_(d_m, rdj, dj_m * rd));
    const float D_r = fmaf_(B2, fmaf_(cp, rm, -dp_m), fmaf_(B3, D_in, B4 * rd_rdj * rm));
    const float D_dp = -(B2 * rm);
    const float D_d = fmaf_(B2, dj_m, -(B3 * rdj * rm));
    const float D_dj = fmaf_(B2, d_m, -(B3 * rd * rm));
    // grad_q = gE phi + dphi + gphi . dr_i
    A.gq += fmaf_(I.gE, phi, fmaf_(al, rt, fmaf_(B1, d_t, dphi)));
    // grad_mu = gE gphi + gdphi + H(dr_i)
    {
      const float cr = fmaf_(I.gE, al, gd_r + T_m);
      const float cd = fmaf_(I.gE, B1, B2 * (rdj - rt));
      const float cdp = B1, cdj = B2 * rd, ct = al;
      A.gm.x += fmaf_(cr, r.x, fmaf_(cd, d.x, fmaf_(cdp, dp.x, fmaf_(cdj, drj.x, ct * t.x))));
      A.gm.y += fmaf_(cr, r.y, fmaf_(cd, d.y, fmaf_(cdp, dp.y, fmaf_(cdj, drj.y, ct * t.y))));
      A.gm.z += fmaf_(cr, r.z, fmaf_(cd, d.z, fmaf_(cdp, dp.z, fmaf_(cdj, drj.z, ct * t.z))));
    }
    // grad_r = (gE q + dq) gphi + H(w_i) + q gdphi + Hdmu + T3
    {
      const float k1 = fmaf_(I.gE, I.q, I.dq);
      const float cr = fmaf_(k1, al, fmaf_(rw, s_rr, fmaf_(-B2, d_w, fmaf_(I.q, gd_r, D_r + T_r))));
      const float cd = fmaf_(k1, B1, fmaf_(B2, fmaf_(I.q, rdj, -rw), D_d + T_d));
      const float cw = al;
      const float cdp = fmaf_(I.q, B1, D_dp);
      const float cdj = fmaf_(I.q * B2, rd, D_dj);
      const float cm = gd_r + T_m;
      const float ct = T_t;
      A.gr.x += fmaf_(cr, r.x, fmaf_(cd, d.x, fmaf_(cw, w.x, fmaf_(cdp, dp.x, fmaf_(cdj, drj.x, fmaf_(cm, m.x, ct * t.x))))));
      A.gr.y += fmaf_(cr, r.y, fmaf_(cd, d.y, fmaf_(cw, w.y, fmaf_(cdp, dp.y, fmaf_(cdj, drj.y, fmaf_(cm, m.y, ct * t.y))))));
      A.gr.z += fmaf_(cr, r.z, fmaf_(cd, d.z, fmaf_(cw, w.z, fmaf_(cdp, dp.z, fmaf_(cdj, drj.z, fmaf_(cm, m.z, ct * t.z))))));
    }
  }
}

// Accumulator floats per ion: phi, grad phi, grad grad phi (forward); grad_r, grad_q, grad_mu
// (tangent).
template <bool TAN>
constexpr int kAccN = TAN ? 7 : 10;

template <bool TAN>
__device__ __forceinline__ void acc_load(Acc<TAN>& A, const float* p) {
  if constexpr (!TAN) {
    A.phi = p[0];
    A.g = mk(p[32], p[64], p[96]);
#pragma unroll
    for (int k = 0; k < 6; ++k) A.h[k] = p[32 * (4 + k)];
  } else {
    A.gr = mk(p[0], p[32], p[64]);
    A.gq = p[96];
    A.gm = mk(p[128], p[160], p[192]);
  }
}

template <bool TAN>
__device__ __forceinline__ void acc_store(const Acc<TAN>& A, float* p) {
  if constexpr (!TAN) {
    p[0] = A.phi;
    p[32] = A.g.x;
    p[64] = A.g.y;
    p[96] = A.g.z;
#pragma unroll
    for (int k = 0; k < 6; ++k) p[32 * (4 + k)] = A.h[k];
  } else {
    p[0] = A.gr.x;
    p[32] = A.gr.y;
    p[64] = A.gr.z;
    p[96] = A.gq;
    p[128] = A.gm.x;
    p[160] = A.gm.y;
    p[192] = A.gm.z;
  }
}

__device__ __forceinline__ unsigned pack_counts(const int (&c)[kSlots]) {
  unsigned p = 0;
#pragma unroll
  for (int s = 0; s < kSlots; ++s) p |= unsigned(c[s]) << (8 * s);
  return p;
}

__device__ __forceinline__ void unpack_counts(unsigned p, int (&c)[kSlots]) {
#pragma unroll
  for (int s = 0; s < kSlots; ++s) c[s] = int((p >> (8 * s)) & 0xffu);
}

// Geometry of one pair cell and its neighbourhood.
struct CellCtx {
  int cix, ciy, ciz;         // the cell
  int ncx, ncy, ncz;         // cells per axis
  int kx, ky, kz;            // neighbour range per axis
  bool zrun;                 // the z-cells of a column are distinct: z offsets come from the
                             // candidate's own cell
  int nzs, nseg;             // segments per (ox, oy) column, segments in all
  int cell_off;              // first global cell key of the frame
};

__device__ __forceinline__ CellCtx cell_ctx(const Geometry& g, int lc, int cell_off) {
  CellCtx c;
  c.ncx = g.ncell[0];
  c.ncy = g.ncell[1];
  c.ncz = g.ncell[2];
  c.kx = g.kimg[0];
  c.ky = g.kimg[1];
  c.kz = g.kimg[2];
  c.ciz = lc % c.ncz;
  c.ciy = (lc / c.ncz) % c.ncy;
  c.cix = lc / (c.ncz * c.ncy);
  c.zrun = c.ncz >= 2 * c.kz + 1;
  c.nzs = c.zrun ? 1 : 2 * c.kz + 1;
  c.nseg = (2 * c.kx + 1) * (2 * c.ky + 1) * c.nzs;
  c.cell_off = cell_off;
  return c;
}

// The dense candidate stream of one cell, 32 candidates at a time. A segment is one
// (ox, oy[, oz]) neighbour column: the ions of one or two contiguous ranges of the cell order.
// Lane l describes segment (32 g + l) of group g; a warp scan of the lengths places the
// segments back to back, each lane lists its own segment's ions (tagged with the lane) in
// shared memory (cand: this warp's kCandCap entries, code: its 32 segment codes), and the warp
// walks the list, loading the next chunk's records while fn(valid, j, bx, by, bz, self_cell)
// handles the current one: candidate j (sorted index), b = -(offset of j) - (cell offset) in
// cell units, self_cell when the offset is zero. fn is called by the whole warp.
template <class Fn>
__device__ __forceinline__ void walk_candidates(const PairArgs& a, const CellCtx& c, unsigned* cand,
                                                int* code_s, int lane, Fn&& fn) {
  for (int g0 = 0; g0 < c.nseg; g0 += 32) {
    const int sidx = g0 + lane;
    int loA = 0, lenA = 0, loB = 0, lenB = 0, code = 0;
    if (sidx < c.nseg) {
      const int oz = c.zrun ? 0 : (sidx % c.nzs) - c.kz;
      const int t = sidx / c.nzs;
      const int oy = (t % (2 * c.ky + 1)) - c.ky;
      const int ox = (t / (2 * c.ky + 1)) - c.kx;
      int cx = (c.cix + ox) % c.ncx, cy = (c.ciy + oy) % c.ncy;
      if (cx < 0) cx += c.ncx;
      if (cy < 0) cy += c.ncy;
      const int row = c.cell_off + (cx * c.ncy + cy) * c.ncz;
      if (c.zrun) {
        const int z0 = c.ciz - c.kz, z1 = c.ciz + c.kz;
        if (z0 < 0) {
          loA = a.start_c[row + z0 + c.ncz]; lenA = a.start_c[row + c.ncz] - loA;
          loB = a.start_c[row]; lenB = a.start_c[row + z1 + 1] - loB;
        } else if (z1 >= c.ncz) {
          loA = a.start_c[row + z0]; lenA = a.start_c[row + c.ncz] - loA;
          loB = a.start_c[row]; lenB = a.start_c[row + z1 - c.ncz + 1] - loB;
        } else {
          loA = a.start_c[row + z0]; lenA = a.start_c[row + z1 + 1] - loA;
        }
      } else {
        int cz = (c.ciz + oz) % c.ncz;
        if (cz < 0) cz += c.ncz;
        loA = a.start_c[row + cz]; lenA = a.start_c[row + cz + 1] - loA;
      }
      // offsets packed in one int: 10 bits each, biased by 512
      code = ((ox + 512) << 20) | ((oy + 512) << 10) | (oz + 512);
    }
    code_s[lane] = code;
    const int len = lenA + lenB;
    int pre = len;   // inclusive scan over the group's segments
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += u;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    for (int piece = 0; piece < total; piece += kCandCap) {
      const int npc = min(kCandCap, total - piece);
      {
        const int first = pre - len;
        const int lo = max(first, piece), hi = min(pre, piece + kCandCap);
        const unsigned tag = unsigned(lane) << kSegShift;
        for (int q = lo; q < hi; ++q) {
          const int off = q - first;
          cand[q - piece] = tag | unsigned(off < lenA ? loA + off : loB + (off - lenA));
        }
      }
      __syncwarp();
      constexpr unsigned kIdx = (1u << kSegShift) - 1u;
      unsigned e = lane < npc ? cand[lane] : 0u;
      float4 fj = lane < npc ? a.pr.fq[e & kIdx] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int base = 0; base < npc; base += 32) {
        // records of the next chunk, in flight while this one is tested
        const int kn = base + 32 + lane;
        const unsigned en = kn < npc ? cand[kn] : 0u;
        const float4 fjn = kn < npc ? a.pr.fq[en & kIdx] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool valid = base + lane < npc;
        const int j = int(e & kIdx);
        const int scode = code_s[e >> kSegShift];
        const int ox = ((scode >> 20) & 1023) - 512;
        const int oy = ((scode >> 10) & 1023) - 512;
        int oz = (scode & 1023) - 512;
        if (c.zrun) {
          oz = __float_as_int(fj.w) - c.ciz;
          if (oz > c.kz) oz -= c.ncz;
          else if (oz < -c.kz) oz += c.ncz;
        }
        fn(valid, j, -fj.x - float(ox), -fj.y - float(oy), -fj.z - float(oz), ox == 0 && oy == 0 && oz == 0);
        e = en;
        fj = fjn;
      }
      __syncwarp();
    }
  }
}

// r = u . H for u = (offset of i) + b in cell units; ORTHO: diagonal cell matrix
template <bool ORTHO>
__device__ __forceinline__ V3 cell_to_r(const Geometry& g, float ux, float uy, float uz) {
  if constexpr (ORTHO) {
    return mk(ux * g.H[0], uy * g.H[4], uz * g.H[8]);
  } else {
    return mk(ux * g.H[0] + uy * g.H[3] + uz * g.H[6], ux * g.H[1] + uy * g.H[4] + uz * g.H[7],
              ux * g.H[2] + uy * g.H[5] + uz * g.H[8]);
  }
}

// Ion-side data of sorted ion i for pair contributions.
template <bool TAN>
__device__ __forceinline__ Ion load_ion(const PairArgs& a, int i, float gE) {
  Ion I;
  const float4 mi4 = a.pr.mu[i];
  I.mu = mk(mi4.x, mi4.y, mi4.z);
  I.q = mi4.w;
  I.dq = 0.f;
  I.gE = gE;
  I.dr = mk(0.f, 0.f, 0.f);
  I.w = mk(0.f, 0.f, 0.f);
  if (TAN) {
    const float4 t = a.pr.tq[i];
    const float4 d = a.pr.dr[i];
    I.dq = t.x;
    I.dr = mk(d.x, d.y, d.z);
    I.w = gE * I.mu + mk(t.y, t.z, t.w);   // gE mu + dmu + q dr
  }
  return I;
}

// Fused pass (used when no valid lists exist): one warp per pair cell; the cell's ions
// (kSlots at a time) share the candidate stream, each keeps its own hit list in shared memory,
// evaluated whenever it holds 32 hits (the remainder waits for the next chunk).
// skip (nullable): return at once when *skip == 0 (the list-driven kernels do the work).
template <bool TAN, bool BATCH, bool ORTHO>
__global__ void __launch_bounds__(kPairThreads) k_pair(PairArgs a) {
  constexpr int NA = kAccN<TAN>;
  __shared__ float4 s_hit[kPairWarps][kSlots][kSlotCap];   // r (x, y, z), w = j (int bits)
  __shared__ float s_acc[kPairWarps][kSlots][NA][32];   // per-lane partial sums of each ion
  __shared__ float4 s_fi[kPairWarps][kSlots];          // in-cell offsets, w = sorted index bits
  __shared__ unsigned s_cand[kPairWarps][kCandCap];     // candidate stream of the segment group
  __shared__ int s_code[kPairWarps][32];                // packed (ox, oy, oz) of each segment
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (a.cache_bad && *a.cache_bad == 0) return;
  if (a.vir_lost && blockIdx.x == 0 && w == 0 && lane == 0) atomicOr(a.vir_lost, kFlagVirialLost);
  // grid-stride over the cells (the launch may be capped: as a fallback it mostly exits here)
  for (int cidx = blockIdx.x * kPairWarps + w; cidx < a.ncells; cidx += gridDim.x * kPairWarps) {
    const int cell = a.cell_lo + cidx;
    const int c_lo = a.start_c[cell], c_hi = a.start_c[cell + 1];
    if (c_lo == c_hi) continue;   // uniform per warp
    const int frame = BATCH ? a.maps.sorted_frame[c_lo] : 0;
    const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, frame);
    const Geometry& g = F.g;
    const CellCtx cc = cell_ctx(g, cell - F.cell_off, F.cell_off);
    const unsigned lane_lt = (1u << lane) - 1u;
    const float gE = (TAN && a.g_energy) ? float(a.g_energy[frame]) : 0.f;

    for (int i0 = c_lo; i0 < c_hi; i0 += kSlots) {
      const int ni = min(kSlots, c_hi - i0);
      if (lane < ni) {
        const float4 f = a.pr.fq[i0 + lane];
        s_fi[w][lane] = make_float4(f.x, f.y, f.z, __int_as_float(i0 + lane));
      }
#pragma unroll
      for (int s = 0; s < kSlots; ++s)
#pragma unroll
        for (int k = 0; k < NA; ++k) s_acc[w][s][k][lane] = 0.f;
      __syncwarp();
      int cnt[kSlots];     // hits waiting per slot (< 64)
#pragma unroll
      for (int s = 0; s < kSlots; ++s) cnt[s] = 0;
      unsigned cnts = 0;   // the same, packed 8 bits per slot, for the flush loop

      // Evaluate, for every slot, its waiting hits in whole 32-wide chunks (all of them when
      // `last`), keeping the remainder at the front of the list.
      auto flush = [&](bool last) {
        for (int s = 0; s < ni; ++s) {
          const int c = int((cnts >> (8 * s)) & 0xffu);
          const int upto = last ? c : (c & ~31);
          if (upto == 0) continue;   // uniform
          const Ion I = load_ion<TAN>(a, i0 + s, gE);
          Acc<TAN> A;
          float* ap = &s_acc[w][s][0][lane];
          acc_load<TAN>(A, ap);
          for (int k = lane; k < upto; k += 32) {
            const float4 h = s_hit[w][s][k];
            interact<TAN>(a, I, __float_as_int(h.w), mk(h.x, h.y, h.z), A);
          }
          acc_store<TAN>(A, ap);
          __syncwarp();
          const int rest = c - upto;
          if (lane < rest)   // [0, rest) and [upto, c) do not overlap: upto >= 32 > rest
            s_hit[w][s][lane] = s_hit[w][s][upto + lane];
          __syncwarp();
          cnts = (cnts & ~(0xffu << (8 * s))) | (unsigned(rest) << (8 * s));
        }
      };

      walk_candidates(a, cc, s_cand[w], s_code[w], lane,
                      [&](bool valid, int j, float bx, float by, float bz, bool self_cell) {
        bool any_full = false;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          if (s >= ni) break;   // uniform per warp
          const float4 fi = s_fi[w][s];
          const V3 r = cell_to_r<ORTHO>(g, fi.x + bx, fi.y + by, fi.z + bz);
          const bool hit = valid && dot(r, r) < g.rcut2 && !(self_cell && j == __float_as_int(fi.w));
          const unsigned bal = __ballot_sync(0xffffffffu, hit);
          if (hit) s_hit[w][s][cnt[s] + __popc(bal & lane_lt)] = make_float4(r.x, r.y, r.z, __int_as_float(j));
          cnt[s] += __popc(bal);
          any_full |= cnt[s] >= 32;
        }
        if (any_full) {
          __syncwarp();
          cnts = pack_counts(cnt);
          flush(false);
          unpack_counts(cnts, cnt);
        }
      });
      __syncwarp();
      cnts = pack_counts(cnt);
      flush(true);

      for (int s = 0; s < ni; ++s) {
        const int orig = a.pr.idx[i0 + s].w;
        const float* ap = &s_acc[w][s][0][0];
        float v[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) v[k] = warp_sum(ap[32 * k + lane]);
        if (lane == 0) {
          float* o = a.out + size_t(orig) * (TAN ? 8 : 10);
#pragma unroll
          for (int k = 0; k < NA; ++k) o[k] = v[k];
          if (TAN) o[7] = 0.f;
        }
      }
      __syncwarp();
    }
  }
}

// List pass: one warp per pair cell walks the same candidate stream and writes every ion's
// hits (r, j), in stream order, to its list in global memory; list_cnt = hits, or -1 (and
// *overflow = 1) when an ion has more than list_cap.
// (ions of a cell sharing one candidate stream in the list pass: up to eight, so that most
// cells walk their stream once; slots past the cell's last ion are skipped, warp-uniformly)
constexpr int kBuildSlots = 8;

template <bool BATCH, bool ORTHO>
__global__ void __launch_bounds__(kPairThreads) k_pair_build(PairArgs a, int* overflow) {
  constexpr int kSlots = kBuildSlots;
  __shared__ float4 s_fi[kPairWarps][kSlots];
  __shared__ unsigned s_cand[kPairWarps][kCandCap];
  __shared__ int s_code[kPairWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cidx = blockIdx.x * kPairWarps + w;
  if (cidx >= a.ncells) return;   // uniform per warp
  const int cell = a.cell_lo + cidx;
  const int c_lo = a.start_c[cell], c_hi = a.start_c[cell + 1];
  if (c_lo == c_hi) return;
  const int frame = BATCH ? a.maps.sorted_frame[c_lo] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, frame);
  const Geometry& g = F.g;
  const CellCtx cc = cell_ctx(g, cell - F.cell_off, F.cell_off);
  const unsigned lane_lt = (1u << lane) - 1u;
  const int cap = a.list_cap;
  for (int i0 = c_lo; i0 < c_hi; i0 += kSlots) {
    const int ni = min(kSlots, c_hi - i0);
    if (lane < ni) {
      const float4 f = a.pr.fq[i0 + lane];
      s_fi[w][lane] = make_float4(f.x, f.y, f.z, __int_as_float(i0 + lane));
    }
    __syncwarp();
    int cnt[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) cnt[s] = 0;
    walk_candidates(a, cc, s_cand[w], s_code[w], lane,
                    [&](bool valid, int j, float bx, float by, float bz, bool self_cell) {
#pragma unroll
      for (int s = 0; s < kSlots; ++s) {
        if (s >= ni) break;   // uniform per warp
        const float4 fi = s_fi[w][s];
        const V3 r = cell_to_r<ORTHO>(g, fi.x + bx, fi.y + by, fi.z + bz);
        const bool hit = valid && dot(r, r) < g.rcut2 && !(self_cell && j == __float_as_int(fi.w));
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const int k = cnt[s] + __popc(bal & lane_lt);
        if (hit && k < cap && index_ok(k, cap))
          a.list[size_t(i0 + s) * cap + k] = make_float4(r.x, r.y, r.z, __int_as_float(j));
        cnt[s] += __popc(bal);
      }
    });
    if (lane < ni) {
      int c = 0;
#pragma unroll
      for (int s = 0; s < kSlots; ++s) c = (s == lane) ? cnt[s] : c;
      a.list_cnt[i0 + lane] = c <= cap ? c : -1;
      if (c > cap) atomicOr(overflow, 1);
    }
    __syncwarp();
  }
}

// Pair term from the lists: one warp per ion (pair-cell order); lane l takes hits l, l + 32,
// ... in order -- the same per-lane order as the fused kernel, so the two paths give bitwise
// equal results. Runs only when *cache_bad == 0.
template <bool TAN, bool BATCH, bool VIR = false>
__global__ void __launch_bounds__(kPairThreads) k_pair_listed(PairArgs a, int n) {
  if (*a.cache_bad != 0) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * kPairWarps + w;
  if (i >= n) return;   // uniform per warp
  const int frame = BATCH ? a.maps.sorted_frame[i] : 0;
  const float gE = (TAN && a.g_energy) ? float(a.g_energy[frame]) : 0.f;
  const Ion I = load_ion<TAN>(a, i, gE);
  Acc<TAN> A;
  float vir[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int c = a.list_cnt[i];
  const float4* li = a.list + size_t(i) * a.list_cap;
  for (int k = lane; k < c; k += 32) {
    if (!index_ok(k, a.list_cap)) break;
    const float4 h = li[k];
    if (!index_ok(__float_as_int(h.w), n)) continue;
    interact<TAN>(a, I, __float_as_int(h.w), mk(h.x, h.y, h.z), A, VIR ? vir : nullptr);
  }
  if (VIR) {
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = warp_sum(vir[k]);
    if (lane == 0) {
      float* o = a.vir_out + size_t(a.pr.idx[i].w) * 9;
#pragma unroll
      for (int k = 0; k < 9; ++k) o[k] = vir[k];
    }
  }
  constexpr int NA = kAccN<TAN>;
  float v[NA];
  if constexpr (!TAN) {
    v[0] = A.phi;
    v[1] = A.g.x;
    v[2] = A.g.y;
    v[3] = A.g.z;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[4 + k] = A.h[k];
  } else {
    v[0] = A.gr.x;
    v[1] = A.gr.y;
    v[2] = A.gr.z;
    v[3] = A.gq;
    v[4] = A.gm.x;
    v[5] = A.gm.y;
    v[6] = A.gm.z;
  }
#pragma unroll
  for (int k = 0; k < NA; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
    float* o = a.out + size_t(a.pr.idx[i].w) * (TAN ? 8 : 10);
#pragma unroll
    for (int k = 0; k < NA; ++k) o[k] = v[k];
    if (TAN) o[7] = 0.f;
  }
}

template <bool TAN, bool BATCH>
void launch_k(bool ortho, int grid, cudaStream_t s, const PairArgs& a) {
  if (ortho) k_pair<TAN, BATCH, true><<<grid, kPairThreads, 0, s>>>(a);
  else k_pair<TAN, BATCH, false><<<grid, kPairThreads, 0, s>>>(a);
}

// Arguments shared by the pair launches.
PairArgs pair_args(pme_plan_t p, const double* g_energy, float* out) {
  PairArgs a = {};
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.alpha = float(p->alpha);
  a.pr = p->pr;
  a.start_c = p->sb.start_c;
  a.g_energy = g_energy;
  a.out = out;
  if (p->batch) {
    a.cell_lo = 0;
    a.ncells = p->total_cells;
  } else {
    a.cell_lo = p->frames_h[0].cell_off;
    a.ncells = p->frames_h[0].ncells;
  }
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
  a.list = p->plist;
  a.list_cnt = p->plist_cnt;
  a.list_cap = p->plist_cap;
  return a;
}

}  // namespace

// every frame of the plan has a diagonal cell matrix
static bool plan_ortho(pme_plan_t p) {
  for (int f = 0; f < p->nframes; ++f) {
    const float* H = p->frames_h[f].g.H;
    if (!(H[1] == 0.f && H[2] == 0.f && H[3] == 0.f && H[5] == 0.f && H[6] == 0.f && H[7] == 0.f))
      return false;
  }
  return true;
}

int launch_pair(pme_plan_t p, cudaStream_t s, int n, bool tangent, const IonInputs& in,
                const double* g_energy, float* out, const int* skip, bool virial) {
  (void)in;
  if (n == 0) return PME_OK;
  PairArgs a = pair_args(p, g_energy, out);
  a.cache_bad = skip;
  if (virial && !tangent) a.vir_lost = p->flags;
  int grid = (a.ncells + kPairWarps - 1) / kPairWarps;
  if (grid == 0) return PME_OK;
  // as the fallback of the list path (skip non-null) it normally exits at once: a small grid
  // keeps that cheap; the cells are walked grid-stride when it does run
  if (skip) grid = std::min(grid, 2 * device_sm_count());
  const bool ortho = plan_ortho(p);
  if (p->batch) {
    if (tangent) launch_k<true, true>(ortho, grid, s, a);
    else launch_k<false, true>(ortho, grid, s, a);
  } else {
    if (tangent) launch_k<true, false>(ortho, grid, s, a);
    else launch_k<false, false>(ortho, grid, s, a);
  }
  count_launch();
  return check_launch(p, "k_pair");
}

int launch_pair_build(pme_plan_t p, cudaStream_t s, int n, int* overflow) {
  int st = check_cuda(p, cudaMemsetAsync(overflow, 0, sizeof(int), s), "memset");
  if (st || n == 0) return st;
  PairArgs a = pair_args(p, nullptr, nullptr);
  const int grid = (a.ncells + kPairWarps - 1) / kPairWarps;
  if (grid == 0) return PME_OK;
  const bool ortho = plan_ortho(p);
  if (p->batch) {
    if (ortho) k_pair_build<true, true><<<grid, kPairThreads, 0, s>>>(a, overflow);
    else k_pair_build<true, false><<<grid, kPairThreads, 0, s>>>(a, overflow);
  } else {
    if (ortho) k_pair_build<false, true><<<grid, kPairThreads, 0, s>>>(a, overflow);
    else k_pair_build<false, false><<<grid, kPairThreads, 0, s>>>(a, overflow);
  }
  count_launch();
  return check_launch(p, "k_pair_build");
}

int launch_pair_listed(pme_plan_t p, cudaStream_t s, int n, bool tangent, const double* g_energy,
                       float* out, const int* flag, bool virial) {
  if (n == 0) return PME_OK;
  PairArgs a = pair_args(p, g_energy, out);
  a.cache_bad = flag;
  a.vir_out = p->pvir;
  const int grid = (n + kPairWarps - 1) / kPairWarps;
  const bool vir = virial && !tangent;
  if (p->batch) {
    if (tangent) k_pair_listed<true, true><<<grid, kPairThreads, 0, s>>>(a, n);
    else if (vir) k_pair_listed<false, true, true><<<grid, kPairThreads, 0, s>>>(a, n);
    else k_pair_listed<false, true><<<grid, kPairThreads, 0, s>>>(a, n);
  } else {
    if (tangent) k_pair_listed<true, false><<<grid, kPairThreads, 0, s>>>(a, n);
    else if (vir) k_pair_listed<false, false, true><<<grid, kPairThreads, 0, s>>>(a, n);
    else k_pair_listed<false, false><<<grid, kPairThreads, 0, s>>>(a, n);
  }
  count_launch();
  return check_launch(p, "k_pair_listed");
}

GBPME_BOUNDS_READER(bounds_hit_pair)

}  // namespace gbpme
