// Real-space pair term with point quadrupoles (every frame of the plan): the rank-2 channel of
// the multipole operator L_i = q_i + mu_i . grad + Theta_i : grad grad (an extension; the paper
// names quadrupolar channels as future work).
//
// For a source j = (c, d, B) = (q_j, mu_j, Theta_j) at r = r_i - r_j + n, the potential at i
// is phi = (c - d . grad + B : grad grad) psi(r), psi = erfc(alpha r)/r. With the radial
// functions B_0 = psi, B_l = [(2l - 1) B_{l-1} + (2 alpha^2)^l exp(-alpha^2 r^2)/(alpha sqrt(pi))]/r^2
// (d/dr_a B_l = -r_a B_{l+1}), and for the field point's own quadrupole A = Theta_i, the
// contractions of grad^n psi give, with dr = d.r, Br = B r, rBr = r.B.r, Ar = A r, rAr = r.A.r:
//   phi        = c B0 + dr B1 - tr B B1 + rBr B2
//   grad phi   = r (-c B1 - dr B2 + tr B B2 - rBr B3) + d B1 + 2 Br B2
//   grad^2 phi = I (-c B1 - dr B2 + tr B B2 - rBr B3) + r r (c B2 + dr B3 - tr B B3 + rBr B4)
//                - B2 (d r + r d) - 2 B3 (Br r + r Br) + 2 B2 B
//   A : grad^3 phi = r [c tr A B2 - c rAr B3 + tr A dr B3 + 2 (Ar . d) B3 - rAr dr B4
//                       - (tr A tr B + 2 A:B) B3 + (tr A rBr + tr B rAr + 4 Ar . Br) B4
//                       - rAr rBr B5]
//                    + Ar (2 c B2 + 2 dr B3 - 2 tr B B3 + 2 rBr B4) + Br (-2 tr A B3 + 2 rAr B4)
//                    + d (-tr A B2 + rAr B3) - 2 B2 A d - 4 B3 (B A r + A B r)
//
// Work split: one warp per ion (pair-cell order). The neighbouring cells are the
// (2 kimg + 1)^2 (x, y) columns, each the contiguous run of the 2 kimg + 1 z-cells around the
// ion's cell (one or two ranges at the periodic wrap; a candidate's z offset follows from its
// own cell), or, when an axis has too few cells for distinct offsets, every offset of the
// [-kimg, kimg]^3 cube on its own (each then one periodic image of the cell it wraps to). The
// lanes describe 32 such segments at a time and a warp scan lays their candidates out as one
// dense stream in shared memory; the lanes test 32 candidates at a time, forming
// r = (f_i - f_j - o) H from the in-cell offsets, and append the hits inside rcut, in order, to
// the warp's hit list (ballot + popc); each time the list holds 32 hits all lanes evaluate one
// each. Per-lane sums are reduced with warp shuffles in a fixed order, so the result is
// reproducible. Output in caller order: out[10] = phi, grad phi, grad^2 phi (xx yy zz xy xz
// yz); qout[4..6] = A : grad^3 phi.
//
// When the plan keeps pair-hit lists, the forward builds them with the charge-dipole list pass
// (k_pair_build: the ions of a cell share one candidate stream) and k_pair_quad_listed
// evaluates each ion's list; the cell-walking kernel then runs only if a list overflowed.
#include <cmath>

#include "dual.cuh"
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kQuadThreads = 128;

struct QuadPairArgs {
  FrameDesc one;
  FrameMaps maps;
  PairRecords pr;
  const int* start_c;
  const float* theta;   // [caller index][6]
  float* out;           // [caller index][10]
  float* qout;          // [caller index][8], this kernel writes 4..6
  int n;
  float alpha;
  // hit lists of the list pass (k_pair_build): per ion (r, j) in stream order, list_cnt hits
  // or -1 when more than list_cap; flag = that pass's overflow flag: the list-driven kernel
  // runs when *flag == 0, the cell-walking kernel when *flag != 0 (or flag null)
  const float4* list;
  const int* list_cnt;
  int list_cap;
  const int* flag;
  float c[6];           // (2 alpha^2)^l / (alpha sqrt(pi)), l = 1..5 at c[l]
};

struct Sym {
  float xx, yy, zz, xy, xz, yz;
};

__device__ __forceinline__ Sym load_sym(const float* t) { return Sym{t[0], t[1], t[2], t[3], t[4], t[5]}; }

template <typename T>
__device__ __forceinline__ void mul(const Sym& A, T x, T y, T z, T& ox, T& oy, T& oz) {
  ox = A.xx * x + A.xy * y + A.xz * z;
  oy = A.xy * x + A.yy * y + A.yz * z;
  oz = A.xz * x + A.yz * y + A.zz * z;
}

template <typename T>
struct QuadAcc {
  T phi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  T hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
  T tx = 0.f, ty = 0.f, tz = 0.f;
};

// One pair: source j = (c, d, B) at displacement r from the field point with quadrupole A
// (trace trA). Written once over the scalar type T: float for the forward; Dual for the
// Hessian-vector product, where r, c and d carry their tangents along (dr, dq, dmu) and every
// output its directional derivative (the quadrupoles have none).
template <typename T>
__device__ __forceinline__ void quad_pair(const QuadPairArgs& a, const Sym& A, float trA, int j, T rx, T ry, T rz,
                                          T c, T dx, T dy, T dz, QuadAcc<T>& S) {
  const float al = a.alpha;
  const T r2 = rx * rx + ry * ry + rz * rz;
  const T rinv = rsqrtT(r2);
  const T rinv2 = rinv * rinv;
  const T ex = expT(-(al * al) * r2);
  const T B0 = erfcT(al * (r2 * rinv)) * rinv;
  const T B1 = (B0 + a.c[1] * ex) * rinv2;
  const T B2 = (3.f * B1 + a.c[2] * ex) * rinv2;
  const T B3 = (5.f * B2 + a.c[3] * ex) * rinv2;
  const T B4 = (7.f * B3 + a.c[4] * ex) * rinv2;
  const T B5 = (9.f * B4 + a.c[5] * ex) * rinv2;
  const Sym Bm = load_sym(a.theta + size_t(a.pr.idx[j].w) * 6);
  const float trB = Bm.xx + Bm.yy + Bm.zz;
  T Brx, Bry, Brz, Arx, Ary, Arz;
  mul(Bm, rx, ry, rz, Brx, Bry, Brz);
  mul(A, rx, ry, rz, Arx, Ary, Arz);
  const T dr = dx * rx + dy * ry + dz * rz;
  const T rBr = Brx * rx + Bry * ry + Brz * rz;
  const T rAr = Arx * rx + Ary * ry + Arz * rz;
  // potential, gradient, Hessian
  const T sI = -(c * B1) - dr * B2 + trB * B2 - rBr * B3;
  const T srr = c * B2 + dr * B3 - trB * B3 + rBr * B4;
  S.phi += c * B0 + dr * B1 - trB * B1 + rBr * B2;
  S.gx += sI * rx + B1 * dx + 2.f * B2 * Brx;
  S.gy += sI * ry + B1 * dy + 2.f * B2 * Bry;
  S.gz += sI * rz + B1 * dz + 2.f * B2 * Brz;
  S.hxx += sI + srr * rx * rx - 2.f * B2 * dx * rx - 4.f * B3 * Brx * rx + 2.f * Bm.xx * B2;
  S.hyy += sI + srr * ry * ry - 2.f * B2 * dy * ry - 4.f * B3 * Bry * ry + 2.f * Bm.yy * B2;
  S.hzz += sI + srr * rz * rz - 2.f * B2 * dz * rz - 4.f * B3 * Brz * rz + 2.f * Bm.zz * B2;
  S.hxy += srr * rx * ry - B2 * (dx * ry + rx * dy) - 2.f * B3 * (Brx * ry + rx * Bry) + 2.f * Bm.xy * B2;
  S.hxz += srr * rx * rz - B2 * (dx * rz + rx * dz) - 2.f * B3 * (Brx * rz + rx * Brz) + 2.f * Bm.xz * B2;
  S.hyz += srr * ry * rz - B2 * (dy * rz + ry * dz) - 2.f * B3 * (Bry * rz + ry * Brz) + 2.f * Bm.yz * B2;
  // A : grad^3 phi
  const float AB = A.xx * Bm.xx + A.yy * Bm.yy + A.zz * Bm.zz + 2.f * (A.xy * Bm.xy + A.xz * Bm.xz + A.yz * Bm.yz);
  const T Ard = Arx * dx + Ary * dy + Arz * dz;
  const T ArBr = Arx * Brx + Ary * Bry + Arz * Brz;
  T Adx, Ady, Adz, BArx, BAry, BArz, ABrx, ABry, ABrz;
  mul(A, dx, dy, dz, Adx, Ady, Adz);
  mul(Bm, Arx, Ary, Arz, BArx, BAry, BArz);
  mul(A, Brx, Bry, Brz, ABrx, ABry, ABrz);
  const T s_r = trA * (c * B2) - c * rAr * B3 + trA * (dr * B3) + 2.f * (Ard * B3) - rAr * dr * B4 -
                (trA * trB + 2.f * AB) * B3 + (trA * rBr + trB * rAr + 4.f * ArBr) * B4 - rAr * rBr * B5;
  const T s_Ar = 2.f * (c * B2) + 2.f * (dr * B3) - (2.f * trB) * B3 + 2.f * (rBr * B4);
  const T s_Br = -(2.f * trA) * B3 + 2.f * (rAr * B4);
  const T s_d = -trA * B2 + rAr * B3;
  S.tx += s_r * rx + s_Ar * Arx + s_Br * Brx + s_d * dx - 2.f * B2 * Adx - 4.f * B3 * (BArx + ABrx);
  S.ty += s_r * ry + s_Ar * Ary + s_Br * Bry + s_d * dy - 2.f * B2 * Ady - 4.f * B3 * (BAry + ABry);
  S.tz += s_r * rz + s_Ar * Arz + s_Br * Brz + s_d * dz - 2.f * B2 * Adz - 4.f * B3 * (BArz + ABrz);
}

// forward call: the source's charge and dipole from the pair records
__device__ __forceinline__ void quad_pair(const QuadPairArgs& a, const Sym& A, float trA, int j, float rx, float ry,
                                          float rz, QuadAcc<float>& S) {
  const float4 mj = a.pr.mu[j];
  quad_pair<float>(a, A, trA, j, rx, ry, rz, mj.w, mj.x, mj.y, mj.z, S);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kWarps = kQuadThreads / 32;
constexpr int kHitCap = 64;   // < 32 carried over + 32 appended per test round
constexpr int kCandCap = 512; // candidates listed per warp at a time
constexpr int kSegShift = 27; // candidate entry: (segment lane << 27) | sorted index

template <bool BATCH>
__global__ void __launch_bounds__(kQuadThreads) k_pair_quad(QuadPairArgs a) {
  __shared__ float4 s_hit[kWarps][kHitCap];   // r (x, y, z), source j (int bits)
  __shared__ unsigned s_cand[kWarps][kCandCap];
  if (a.flag && *a.flag == 0) return;   // the lists hold: the list-driven kernel does the work
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + wid;
  if (i >= a.n) return;   // warp-uniform
  float4* hits = s_hit[wid];
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, BATCH ? a.maps.sorted_frame[i] : 0);
  const Geometry& g = F.g;
  const int4 ci = a.pr.idx[i];
  const float4 fi = a.pr.fq[i];
  const Sym A = load_sym(a.theta + size_t(ci.w) * 6);
  const float trA = A.xx + A.yy + A.zz;
  const float rc2 = g.rcut2;
  const int kx = g.kimg[0], ky = g.kimg[1], kz = g.kimg[2];
  const int ncx = g.ncell[0], ncy = g.ncell[1], ncz = g.ncell[2];
  const bool zrun = ncz >= 2 * kz + 1;
  QuadAcc<float> S;
  int nh = 0;   // hits in the list (the same in every lane)
  unsigned* cand = s_cand[wid];
  const int nzs = zrun ? 1 : 2 * kz + 1;
  const int nseg = (2 * kx + 1) * (2 * ky + 1) * nzs;
  for (int g0 = 0; g0 < nseg; g0 += 32) {
    // lane l describes segment g0 + l: one or two contiguous ranges of the cell order, with
    // the segment's cell offset folded into (fxo, fyo) and, outside z-runs, its z offset
    const int sidx = g0 + lane;
    int loA = 0, lenA = 0, loB = 0, lenB = 0, ozs = 0, zxy = 0;
    float fxo = 0.f, fyo = 0.f;
    if (sidx < nseg) {
      ozs = zrun ? 0 : (sidx % nzs) - kz;
      const int t = sidx / nzs;
      const int oy = (t % (2 * ky + 1)) - ky;
      const int ox = (t / (2 * ky + 1)) - kx;
      int cx = (ci.x + ox) % ncx, cy = (ci.y + oy) % ncy;
      if (cx < 0) cx += ncx;
      if (cy < 0) cy += ncy;
      fxo = fi.x - float(ox);
      fyo = fi.y - float(oy);
      zxy = ox == 0 && oy == 0;
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
        int cz = (ci.z + ozs) % ncz;
        if (cz < 0) cz += ncz;
        loA = a.start_c[row + cz]; lenA = a.start_c[row + cz + 1] - loA;
      }
    }
    // segments back to back: one dense candidate stream
    const int len = lenA + lenB;
    int pre = len;
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
        for (int q = lo; q < hi; ++q) {
          const int off = q - first;
          cand[q - piece] = (unsigned(lane) << kSegShift) | unsigned(off < lenA ? loA + off : loB + (off - lenA));
        }
      }
      __syncwarp();
      for (int base = 0; base < npc; base += 32) {
        const int k = base + lane;
        const bool valid = k < npc;
        const unsigned e = valid ? cand[k] : 0u;
        const int src = int(e >> kSegShift);
        const float sfx = __shfl_sync(0xffffffffu, fxo, src);
        const float sfy = __shfl_sync(0xffffffffu, fyo, src);
        const int soz = __shfl_sync(0xffffffffu, ozs, src);
        const int szxy = __shfl_sync(0xffffffffu, zxy, src);
        bool hit = false;
        float rx = 0.f, ry = 0.f, rz = 0.f;
        int j = 0;
        if (valid) {
          j = int(e & ((1u << kSegShift) - 1u));
          const float4 fj = a.pr.fq[j];
          int oz = soz;
          if (zrun) {
            oz = __float_as_int(fj.w) - ci.z;
            if (oz > kz) oz -= ncz;
            else if (oz < -kz) oz += ncz;
          }
          const float ux = sfx - fj.x, uy = sfy - fj.y, uz = fi.z - float(oz) - fj.z;
          rx = ux * g.H[0] + uy * g.H[3] + uz * g.H[6];
          ry = ux * g.H[1] + uy * g.H[4] + uz * g.H[7];
          rz = ux * g.H[2] + uy * g.H[5] + uz * g.H[8];
          const float r2 = rx * rx + ry * ry + rz * rz;
          hit = r2 < rc2 && !(j == i && szxy && oz == 0);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) hits[nh + __popc(bal & ((1u << lane) - 1u))] = make_float4(rx, ry, rz, __int_as_float(j));
        nh += __popc(bal);
        __syncwarp();
        if (nh >= 32) {
          const float4 h = hits[lane];
          quad_pair(a, A, trA, __float_as_int(h.w), h.x, h.y, h.z, S);
          __syncwarp();
          if (lane < nh - 32) hits[lane] = hits[32 + lane];
          nh -= 32;
          __syncwarp();
        }
      }
      __syncwarp();
    }
  }
  if (lane < nh) {
    const float4 h = hits[lane];
    quad_pair(a, A, trA, __float_as_int(h.w), h.x, h.y, h.z, S);
  }
  const float v[13] = {warp_sum_f(S.phi), warp_sum_f(S.gx), warp_sum_f(S.gy), warp_sum_f(S.gz),
                       warp_sum_f(S.hxx), warp_sum_f(S.hyy), warp_sum_f(S.hzz), warp_sum_f(S.hxy),
                       warp_sum_f(S.hxz), warp_sum_f(S.hyz), warp_sum_f(S.tx), warp_sum_f(S.ty),
                       warp_sum_f(S.tz)};
  if (lane == 0) {
    float* o = a.out + size_t(ci.w) * 10;
#pragma unroll
    for (int c = 0; c < 10; ++c) o[c] = v[c];
    float* qo = a.qout + size_t(ci.w) * 8;
    qo[4] = v[10];
    qo[5] = v[11];
    qo[6] = v[12];
  }
}

// The same sums from the hit lists of the list pass: one warp per ion, lane l takes hits
// l, l + 32, ... in order; shuffle reduction in a fixed order.
template <bool BATCH>
__global__ void __launch_bounds__(kQuadThreads) k_pair_quad_listed(QuadPairArgs a) {
  if (*a.flag != 0) return;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + wid;
  if (i >= a.n) return;   // warp-uniform
  const int4 ci = a.pr.idx[i];
  const Sym A = load_sym(a.theta + size_t(ci.w) * 6);
  const float trA = A.xx + A.yy + A.zz;
  QuadAcc<float> S;
  const int c = a.list_cnt[i];
  const float4* li = a.list + size_t(i) * a.list_cap;
  for (int k = lane; k < c; k += 32) {
    const float4 h = li[k];
    quad_pair(a, A, trA, __float_as_int(h.w), h.x, h.y, h.z, S);
  }
  const float v[13] = {warp_sum_f(S.phi), warp_sum_f(S.gx), warp_sum_f(S.gy), warp_sum_f(S.gz),
                       warp_sum_f(S.hxx), warp_sum_f(S.hyy), warp_sum_f(S.hzz), warp_sum_f(S.hxy),
                       warp_sum_f(S.hxz), warp_sum_f(S.hyz), warp_sum_f(S.tx), warp_sum_f(S.ty),
                       warp_sum_f(S.tz)};
  if (lane == 0) {
    float* o = a.out + size_t(ci.w) * 10;
#pragma unroll
    for (int k = 0; k < 10; ++k) o[k] = v[k];
    float* qo = a.qout + size_t(ci.w) * 8;
    qo[4] = v[10];
    qo[5] = v[11];
    qo[6] = v[12];
  }
}

// Tangent of the per-ion pair sums along (dr, dq, dmu) (the quadrupole Hessian-vector
// product): the list-driven evaluation in dual numbers. For hit (j, r = r_i - r_j + n) the
// displacement's tangent is dr_i - dr_j and the source's charge and dipole carry dq_j and
// dmu_j = d'_j - q_j dr_j (the pair records hold d' = dmu + q dr). Output in caller order:
// out[26] = the 13 sums (phi, grad phi, grad^2 phi, A : grad^3 phi) and their 13 tangents.
// Needs the hit lists (runs when *flag == 0; the caller reports a lost list otherwise).
template <bool BATCH>
__global__ void __launch_bounds__(kQuadThreads) k_pair_quad_dual(QuadPairArgs a) {
  if (*a.flag != 0) return;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + wid;
  if (i >= a.n) return;   // warp-uniform
  const int4 ci = a.pr.idx[i];
  const Sym A = load_sym(a.theta + size_t(ci.w) * 6);
  const float trA = A.xx + A.yy + A.zz;
  const float4 dri = a.pr.dr[i];
  QuadAcc<Dual> S;
  const int c = a.list_cnt[i];
  const float4* li = a.list + size_t(i) * a.list_cap;
  for (int k = lane; k < c; k += 32) {
    if (!index_ok(k, a.list_cap)) break;
    const float4 h = li[k];
    const int j = __float_as_int(h.w);
    if (!index_ok(j, a.n)) continue;
    const float4 mj = a.pr.mu[j], tj = a.pr.tq[j], drj = a.pr.dr[j];
    const Dual rx(h.x, dri.x - drj.x), ry(h.y, dri.y - drj.y), rz(h.z, dri.z - drj.z);
    const Dual cj(mj.w, tj.x);
    const Dual dx(mj.x, tj.y - mj.w * drj.x), dy(mj.y, tj.z - mj.w * drj.y), dz(mj.z, tj.w - mj.w * drj.z);
    quad_pair<Dual>(a, A, trA, j, rx, ry, rz, cj, dx, dy, dz, S);
  }
  const Dual v[13] = {S.phi, S.gx, S.gy, S.gz, S.hxx, S.hyy, S.hzz, S.hxy, S.hxz, S.hyz, S.tx, S.ty, S.tz};
  float o[26];
#pragma unroll
  for (int k = 0; k < 13; ++k) {
    o[k] = warp_sum_f(v[k].v);
    o[13 + k] = warp_sum_f(v[k].d);
  }
  if (lane == 0) {
    float* out = a.out + size_t(ci.w) * 26;
#pragma unroll
    for (int k = 0; k < 26; ++k) out[k] = o[k];
  }
}

__global__ void k_flag_if_set(const int* cond, int* flags, int bit) {
  if (threadIdx.x == 0 && *cond != 0) atomicOr(flags, bit);
}

QuadPairArgs quad_args(pme_plan_t p, int n, const float* theta, float* out, float* qout, const int* flag) {
  QuadPairArgs a;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.pr = p->pr;
  a.start_c = p->sb.start_c;
  a.theta = theta;
  a.out = out;
  a.qout = qout;
  a.n = n;
  a.alpha = float(p->alpha);
  const double al = p->alpha;
  for (int l = 0; l < 6; ++l) a.c[l] = float(std::pow(2.0 * al * al, l) / (al * std::sqrt(kPi)));
  a.list = p->plist;
  a.list_cnt = p->plist_cnt;
  a.list_cap = p->plist_cap;
  a.flag = flag;
  return a;
}

}  // namespace

int launch_pair_quad_listed(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out,
                            float* qout, const int* flag) {
  if (n <= 0) return PME_OK;
  const QuadPairArgs a = quad_args(p, n, theta, out, qout, flag);
  const int grid = (n + kWarps - 1) / kWarps;
  if (p->batch) k_pair_quad_listed<true><<<grid, kQuadThreads, 0, s>>>(a);
  else k_pair_quad_listed<false><<<grid, kQuadThreads, 0, s>>>(a);
  count_launch();
  return check_launch(p, "k_pair_quad_listed");
}

int launch_pair_quad_dual(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out, const int* flag) {
  if (n <= 0) return PME_OK;
  const QuadPairArgs a = quad_args(p, n, theta, out, nullptr, flag);
  const int grid = (n + kWarps - 1) / kWarps;
  if (p->batch) k_pair_quad_dual<true><<<grid, kQuadThreads, 0, s>>>(a);
  else k_pair_quad_dual<false><<<grid, kQuadThreads, 0, s>>>(a);
  count_launch();
  int st = check_launch(p, "k_pair_quad_dual");
  if (st) return st;
  // an overflowed list leaves the pair part out: flag it for pme_sync_status
  k_flag_if_set<<<1, 32, 0, s>>>(flag, p->flags, kFlagQuadLost);
  count_launch();
  return check_launch(p, "k_flag_if_set");
}

int launch_pair_quad(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out, float* qout,
                     const int* skip) {
  if (n <= 0) return PME_OK;
  if (n >= (1 << 27)) return set_error(p, PME_ERR_UNSUPPORTED, "quadrupole pair term: more than 2^27 ions");
  const QuadPairArgs a = quad_args(p, n, theta, out, qout, skip);
  const int grid = (n + kWarps - 1) / kWarps;
  if (p->batch) k_pair_quad<true><<<grid, kQuadThreads, 0, s>>>(a);
  else k_pair_quad<false><<<grid, kQuadThreads, 0, s>>>(a);
  count_launch();
  return check_launch(p, "k_pair_quad");
}

}  // namespace gbpme
