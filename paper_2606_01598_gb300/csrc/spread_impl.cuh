// Spread kernel template (Section 2.3.2, Eq. charge_dipole_assign): included once per brick
// shape by the spread_*.cu translation units; the design is described in spread.cu.
#pragma once

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int ZS = 8;                     // z points per thread
constexpr int kMaxCand = kMaxCandPerDim * kMaxCandPerDim * kMaxCandPerDim;

// A brick shape: BX x BY x BZ mesh points per CTA, one thread per z-segment of ZS points of
// one (X, Y) column.
template <int BX_, int BY_, int BZ_>
struct Shape {
  static constexpr int BX = BX_, BY = BY_, BZ = BZ_;
  static constexpr int NSEG = BZ / ZS;              // z-segments per column
  static constexpr int NT = BX * BY * NSEG;         // threads
  static constexpr int CAP = NT / 2 < 128 ? NT / 2 : 128;   // ions staged at once
  static constexpr int NW = CAP / 32;               // mask words
  static constexpr int SL = 2 * NT;                 // listed (overlapping) ions held before staging
  static_assert(NSEG == 1 || NSEG == 2 || NSEG == 4, "z-segments per column: 1, 2 or 4");
  static_assert(NT >= kMaxCand && NW >= 1 && NW <= NT / 32, "64 <= threads, at least one mask word");
};

struct SpreadArgs {
  const float* theta;   // quadrupole mode: Theta [caller index][6] (xx yy zz xy xz yz)
  FrameDesc one;
  FrameMaps maps;
  int key_lo;           // first global brick of this launch
  MeshRecords mr;
  const int* start_b;
  const int* cand;      // base of the candidate tables
  float* mesh;          // base of the meshes: rho at mesh_off, d rho at tmesh_off
  // tangent pass: *keep_rho == 0 means rho is still in place from the forward on the same
  // inputs, so only d rho is formed and written (null: form both)
  const int* keep_rho;
};

// Shared-memory record of one staged ion (floats), DW = weight-derivative orders kept
// (quadrupole tangent mode: orders 0..3, the x table holding per column the ten sums
// u_(ny,nz) = sum_nx C_(nx,ny,nz) W_x^(nx) for ny + nz <= 3, the y table W_y^(0..3)):
//   [ZOFF, ...)  z windows: for segment g and order d, 8 floats at ZOFF + g ZSEG + 8 d (ZSEG
//                = 8 DW, plus 4 in the forward record: the four segments of one ion start in
//                different banks)
//   [XOFF, ...)  per brick column X, NXV floats at XOFF + X NXV:
//                forward: (u, v, b, 0), A = u wy0 + v wy1 and B = b wy0 being the
//                coefficients of W_z and W'_z in rho;
//                tangent: (p0, p1, p2, q0, q1, r0, u, v, b), the coefficients of W_z, W'_z,
//                W''_z in d rho being A0 = p0 wy0 + p1 wy1 + p2 wy2, A1 = q0 wy0 + q1 wy1,
//                A2 = r0 wy0 (and A, B as above for rho)
//   [YOFF, ...)  per brick row Y, the y weights wy0, wy1 (and wy2), NYV floats
// The stride is a multiple of 4 with an odd quotient, so 16-byte reads of different ions
// spread over the banks.
template <class SH, int RK>
struct Rec {
  static constexpr int BX = SH::BX, BY = SH::BY, NSEG = SH::NSEG;
  static constexpr bool TAN = RK != 0;
  static constexpr int DW = RK == 0 ? 2 : (RK == 1 ? 3 : 4);
  static constexpr int ZOFF = 0;
  static constexpr int ZSEG = DW * ZS + (RK == 0 ? 4 : 0);   // 64 B apart would share banks
  static constexpr int XOFF = NSEG * ZSEG;
  static constexpr int NXV = RK == 0 ? 4 : (RK == 1 ? 9 : 10);
  static constexpr int YOFF = XOFF + BX * NXV;
  static constexpr int NYV = DW;
  static constexpr int LEN = YOFF + BY * NYV;
  static constexpr int STR = ((LEN + 3) / 4) % 2 == 0 ? (LEN + 3) / 4 * 4 + 4 : (LEN + 3) / 4 * 4;
};

// record kind of a mode: 0 forward (orders <= 1), 1 tangent / quadrupole forward (<= 2),
// 2 quadrupole tangent (<= 3)
template <int MODE>
__host__ __device__ constexpr int rec_kind() {
  return MODE == 0 ? 0 : (MODE == 3 ? 2 : 1);
}

template <class SH, int P, int RK>
constexpr int spread_smem_bytes() {
  return SH::CAP * Rec<SH, RK>::STR * 4 + SH::SL * (4 + 8);
}
static_assert(spread_smem_bytes<Shape<16, 16, 16>, 7, 2>() <= 200 * 1024, "staging fits in shared memory");

// distance from a to b going up the periodic axis of length n (a, b in [0, n))
__device__ __forceinline__ int up_dist(int a, int b, int n) {
  const int d = b - a;
  return d < 0 ? d + n : d;
}

// MODE: 0 forward, 1 tangent, 2 quadrupole forward, 3 quadrupole tangent (d rho only)
template <class SH, int P, int MODE, bool BATCH>
__global__ void __launch_bounds__(SH::NT) k_spread(SpreadArgs a) {
  pdl_begin();
  constexpr int BX = SH::BX, BY = SH::BY, BZ = SH::BZ, NSEG = SH::NSEG, NT = SH::NT, CAP = SH::CAP,
                NW = SH::NW, SL = SH::SL;
  constexpr bool TAN = MODE != 0;   // a second accumulator (d rho, or rho of the quadrupole modes)
  using RC = Rec<SH, rec_kind<MODE>()>;
  constexpr int DW = RC::DW;                      // weight derivative orders kept

  extern __shared__ __align__(16) float dyn[];
  float* sw = dyn;                                        // [CAP][RC::STR] staged records
  int2* srel = reinterpret_cast<int2*>(sw + CAP * RC::STR);   // [SL] stencil index of the brick
                                                              // origin: x | y << 16, z
  int* slist = reinterpret_cast<int*>(srel + SL);         // [SL] listed ions
  __shared__ unsigned xmask[BX][NW], ymask[BY][NW], zmask[NSEG][NW];
  __shared__ int cand_lo[kMaxCand];
  __shared__ int cand_cnt[kMaxCand];
  __shared__ int cand_cum[kMaxCand + 1];
  __shared__ int warp_cnt[NT / 32];

  const int gkey = a.key_lo + blockIdx.x;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, BATCH ? a.maps.brick_frame[gkey] : 0);
  const Geometry& g = F.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int bkey = gkey - F.brick_off;
  const int bz = bkey % g.nb[2];
  const int by = (bkey / g.nb[2]) % g.nb[1];
  const int bx = bkey / (g.nb[2] * g.nb[1]);
  const int b0x = bx * BX, b0y = by * BY, b0z = bz * BZ;
  const int ex = min(BX, g.N[0] - b0x), ey = min(BY, g.N[1] - b0y), ez = min(BZ, g.N[2] - b0z);
  const int Nx = g.N[0], Ny = g.N[1], Nz = g.N[2];
  const bool with_rho = MODE == 0 || (MODE == 1 && (!a.keep_rho || *a.keep_rho != 0));

  // ---- (1) candidate source bricks: product of the per-axis lists, in a fixed order ----
  const int* ct = a.cand + F.cand_off;
  const int* cx = ct + (0 * F.max_nb + bx) * (1 + kMaxCandPerDim);
  const int* cy = ct + (1 * F.max_nb + by) * (1 + kMaxCandPerDim);
  const int* cz = ct + (2 * F.max_nb + bz) * (1 + kMaxCandPerDim);
  const int ncx = cx[0], ncy = cy[0], ncz = cz[0];
  const int ncand = ncx * ncy * ncz;
  if (tid < kMaxCand) {
    int lo = 0, c = 0;
    if (tid < ncand) {
      const int iz = tid % ncz, iy = (tid / ncz) % ncy, ix = tid / (ncz * ncy);
      const int key = F.brick_off + (cx[1 + ix] * g.nb[1] + cy[1 + iy]) * g.nb[2] + cz[1 + iz];
      lo = a.start_b[key];
      c = a.start_b[key + 1] - lo;
    }
    cand_lo[tid] = lo;
    cand_cnt[tid] = c;
  }
  __syncthreads();
  if (wid == 0) {
    // exclusive scan of the 64 counts, two per lane
    const int c0 = cand_cnt[2 * lane], c1 = cand_cnt[2 * lane + 1];
    int v = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    const int excl = v - c0 - c1;
    cand_cum[2 * lane] = excl;
    cand_cum[2 * lane + 1] = excl + c0;
    if (lane == 31) cand_cum[kMaxCand] = v;
  }
  __syncthreads();
  const int total = cand_cum[kMaxCand];

  // this thread's points: column (X, Y), z-segment seg
  const int seg = tid & (NSEG - 1), col = tid / NSEG;
  const int X = col / BY, Y = col % BY;
  const int gx = b0x + X, gy = b0y + Y, zs0 = b0z + seg * ZS;
  float acc[ZS], dacc[TAN ? ZS : 1];
#pragma unroll
  for (int z = 0; z < ZS; ++z) acc[z] = 0.f;
#pragma unroll
  for (int z = 0; z < (TAN ? ZS : 1); ++z) dacc[z] = 0.f;

  int cnt = 0;
  for (int cursor = 0; cursor < total; cursor += NT) {
    // ---- (2) test NT candidates, append the overlapping ones in order -----------------
    const int gi = cursor + tid;
    bool take = false;
    int ion = 0;
    int4 m = make_int4(0, 0, 0, 0);
    if (gi < total) {
      int k = 0;
#pragma unroll
      for (int st = 32; st >= 1; st >>= 1)
        if (k + st < ncand && cand_cum[k + st] <= gi) k += st;
      ion = cand_lo[k] + (gi - cand_cum[k]);
      m = a.mr.idx[ion];
      const int dx = up_dist(m.x, b0x, Nx), dy = up_dist(m.y, b0y, Ny), dz = up_dist(m.z, b0z, Nz);
      take = (dx <= P - 1 || dx >= Nx - ex + 1) && (dy <= P - 1 || dy >= Ny - ey + 1) &&
             (dz <= P - 1 || dz >= Nz - ez + 1);
      m = make_int4(dx, dy, dz, 0);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
      before += (w < wid) ? warp_cnt[w] : 0;
      tot += warp_cnt[w];
    }
    if (take) {
      const int l = cnt + before + __popc(bal & ((1u << lane) - 1u));
      slist[l] = ion;
      srel[l] = make_int2(m.x | (m.y << 16), m.z);
    }
    cnt += tot;
    __syncthreads();
    if (cnt <= SL - NT && cursor + NT < total) continue;

    for (int base = 0; base < cnt; base += CAP) {
      const int nst = min(CAP, cnt - base);
      // ---- (3) stage: threads [0, CAP) the x / y tables, [CAP, 2 CAP) the z windows ----
      if (tid < CAP && tid < nst) {
        const int l = base + tid;
        const int src = slist[l];
        const int2 rl = srel[l];
        const int rx = rl.x & 0xffff, ry = rl.x >> 16;
        const float4 fq = a.mr.fq[src];
        const float4 dm = a.mr.dm[src];
        float* rec = sw + tid * RC::STR;
        float w[DW][P];
        spline_weights<P, DW - 1>(fq.x, w);
        const float q = fq.w, mx = dm.x, my = dm.y, mz = dm.z;
        float c4 = 0.f, c5 = 0.f, c6 = 0.f, c7 = 0.f, tx = 0.f, ty = 0.f, tz = 0.f;
        // quadrupole mode: Theta' = D^T Theta D (mesh coordinates) as xx, 2 xy, yy, 2 xz, 2 yz, zz
        float t_xx = 0.f, t_xy = 0.f, t_yy = 0.f, t_xz = 0.f, t_yz = 0.f, t_zz = 0.f;
        // quadrupole tangent mode: coefficients C_(nx,ny,nz) of d rho (mesh coordinates)
        float C[4][4][4];
        if (MODE == 3) {
#pragma unroll
          for (int i0 = 0; i0 < 4; ++i0)
#pragma unroll
            for (int i1 = 0; i1 < 4; ++i1)
#pragma unroll
              for (int i2 = 0; i2 < 4; ++i2) C[i0][i1][i2] = 0.f;
          const float4 tq = a.mr.tq[src];
          const float4 tt = a.mr.tt[src];
          const float t0 = tt.x, t1 = tt.y, t2 = tt.z;
          const float* th = a.theta + size_t(a.mr.idx[src].w) * 6;
          const float T[3][3] = {{th[0], th[3], th[4]}, {th[3], th[1], th[5]}, {th[4], th[5], th[2]}};
          const float* D = F.g.D;
          float TD[3][3], Tp[3][3];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              TD[r][c] = T[r][0] * D[0 * 3 + c] + T[r][1] * D[1 * 3 + c] + T[r][2] * D[2 * 3 + c];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              Tp[r][c] = D[0 * 3 + r] * TD[0][c] + D[1 * 3 + r] * TD[1][c] + D[2 * 3 + r] * TD[2][c];
          // dq W + d' . grad W + (mu' . grad)(t . grad) W + (Theta' : grad grad)(t . grad) W
          C[0][0][0] = tq.x;
          C[1][0][0] = tq.y;
          C[0][1][0] = tq.z;
          C[0][0][1] = tq.w;
          C[2][0][0] = mx * t0;
          C[0][2][0] = my * t1;
          C[0][0][2] = mz * t2;
          C[1][1][0] = mx * t1 + my * t0;
          C[1][0][1] = mx * t2 + mz * t0;
          C[0][1][1] = my * t2 + mz * t1;
          C[3][0][0] = Tp[0][0] * t0;
          C[0][3][0] = Tp[1][1] * t1;
          C[0][0][3] = Tp[2][2] * t2;
          C[2][1][0] = Tp[0][0] * t1 + 2.f * Tp[0][1] * t0;
          C[2][0][1] = Tp[0][0] * t2 + 2.f * Tp[0][2] * t0;
          C[1][2][0] = Tp[1][1] * t0 + 2.f * Tp[0][1] * t1;
          C[0][2][1] = Tp[1][1] * t2 + 2.f * Tp[1][2] * t1;
          C[1][0][2] = Tp[2][2] * t0 + 2.f * Tp[0][2] * t2;
          C[0][1][2] = Tp[2][2] * t1 + 2.f * Tp[1][2] * t2;
          C[1][1][1] = 2.f * (Tp[0][1] * t2 + Tp[0][2] * t1 + Tp[1][2] * t0);
        }
        if (MODE == 2) {
          const float* th = a.theta + size_t(a.mr.idx[src].w) * 6;
          const float T[3][3] = {{th[0], th[3], th[4]}, {th[3], th[1], th[5]}, {th[4], th[5], th[2]}};
          const float* D = F.g.D;
          float TD[3][3];   // Theta D
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              TD[r][c] = T[r][0] * D[0 * 3 + c] + T[r][1] * D[1 * 3 + c] + T[r][2] * D[2 * 3 + c];
          float Tp[3][3];   // D^T Theta D
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              Tp[r][c] = D[0 * 3 + r] * TD[0][c] + D[1 * 3 + r] * TD[1][c] + D[2 * 3 + r] * TD[2][c];
          c4 = q;
          c5 = mx;
          c6 = my;
          c7 = mz;
          t_xx = Tp[0][0];
          t_yy = Tp[1][1];
          t_zz = Tp[2][2];
          t_xy = Tp[0][1] + Tp[1][0];
          t_xz = Tp[0][2] + Tp[2][0];
          t_yz = Tp[1][2] + Tp[2][1];
        } else if (TAN) {
          const float4 tq = a.mr.tq[src];
          const float4 tt = a.mr.tt[src];
          c4 = tq.x;
          c5 = tq.y;
          c6 = tq.z;
          c7 = tq.w;
          tx = tt.x;
          ty = tt.y;
          tz = tt.z;
        }
        // stencil index j sits in brick column (j - rx) mod Nx. Only the columns (and rows) the
        // ion's stencil covers are written: the accumulation reads an entry only for an ion
        // whose coverage bit of that column (row) is set
#pragma unroll
        for (int j = 0; j < P; ++j) {
          int X = j - rx;
          if (X < 0) X += Nx;
          if (X < BX) {
            const float w0 = w[0][j], w1 = w[1][j];
            float* e = rec + RC::XOFF + X * RC::NXV;
            if (MODE == 3) {
              // u_(ny,nz) = sum_nx C_(nx,ny,nz) W_x^(nx), order (ny,nz): 00 10 01 20 11 02 30 21 12 03
              const float w2 = w[2][j], w3 = w[DW - 1][j];
              e[0] = C[0][0][0] * w0 + C[1][0][0] * w1 + C[2][0][0] * w2 + C[3][0][0] * w3;
              e[1] = C[0][1][0] * w0 + C[1][1][0] * w1 + C[2][1][0] * w2;
              e[2] = C[0][0][1] * w0 + C[1][0][1] * w1 + C[2][0][1] * w2;
              e[3] = C[0][2][0] * w0 + C[1][2][0] * w1;
              e[4] = C[0][1][1] * w0 + C[1][1][1] * w1;
              e[5] = C[0][0][2] * w0 + C[1][0][2] * w1;
              e[6] = C[0][3][0] * w0;
              e[7] = C[0][2][1] * w0;
              e[8] = C[0][1][2] * w0;
              e[9] = C[0][0][3] * w0;
            } else if (MODE == 2) {
              const float w2 = w[DW - 1][j];
              e[0] = c4 * w0 + c5 * w1 + t_xx * w2;
              e[1] = c6 * w0 + t_xy * w1;
              e[2] = t_yy * w0;
              e[3] = c7 * w0 + t_xz * w1;
              e[4] = t_yz * w0;
              e[5] = t_zz * w0;
            } else if (TAN) {
              const float w2 = w[DW - 1][j];
              e[0] = c4 * w0 + c5 * w1 + mx * tx * w2;
              e[1] = c6 * w0 + (mx * ty + my * tx) * w1;
              e[2] = my * ty * w0;
              e[3] = c7 * w0 + (mx * tz + mz * tx) * w1;
              e[4] = (my * tz + mz * ty) * w0;
              e[5] = mz * tz * w0;
              e[6] = q * w0 + mx * w1;
              e[7] = my * w0;
              e[8] = mz * w0;
            } else {
              *reinterpret_cast<float4*>(e) = make_float4(q * w0 + mx * w1, my * w0, mz * w0, 0.f);
            }
          }
        }
        spline_weights<P, DW - 1>(fq.y, w);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          int Yr = j - ry;
          if (Yr < 0) Yr += Ny;
          if (Yr < BY) {
            float* e = rec + RC::YOFF + Yr * RC::NYV;
#pragma unroll
            for (int d = 0; d < DW; ++d) e[d] = w[d][j];
          }
        }
      } else if (tid >= CAP && tid - CAP < nst) {
        const int k = tid - CAP;
        const int l = base + k;
        const int rz = srel[l].y;
        const float4 fq = a.mr.fq[slist[l]];
        float* rec = sw + k * RC::STR;
        float w[DW][P];
        spline_weights<P, DW - 1>(fq.z, w);
#pragma unroll
        for (int u = 0; u < NSEG * RC::ZSEG; u += 4)
          *reinterpret_cast<float4*>(rec + RC::ZOFF + u) = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int g = 0; g < NSEG; ++g) {
          // stencil index of the segment's first point; stencil index j lands on point
          // (j - j0) mod Nz of the segment
          const int j0 = (rz + g * ZS) % Nz;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            int z = j - j0;
            if (z < 0) z += Nz;
            if (z < ZS) {
#pragma unroll
              for (int d = 0; d < DW; ++d) rec[RC::ZOFF + g * RC::ZSEG + d * ZS + z] = w[d][j];
            }
          }
        }
      }
      // ---- (4) coverage masks: warp w builds word w -----------------------------------
      if (wid < NW) {
        const int l = base + wid * 32 + lane;
        const bool in = wid * 32 + lane < nst;
        const int2 rl = in ? srel[l] : make_int2(0, 0);
        const int rx = rl.x & 0xffff, ry = rl.x >> 16, rz = rl.y;
#pragma unroll
        for (int t = 0; t < BX; ++t) {
          int d = rx + t;
          if (d >= Nx) d -= Nx;
          const unsigned b = __ballot_sync(0xffffffffu, in && t < ex && d < P);
          if (lane == 0) xmask[t][wid] = b;
        }
#pragma unroll
        for (int t = 0; t < BY; ++t) {
          int d = ry + t;
          if (d >= Ny) d -= Ny;
          const unsigned b = __ballot_sync(0xffffffffu, in && t < ey && d < P);
          if (lane == 0) ymask[t][wid] = b;
        }
#pragma unroll
        for (int t = 0; t < NSEG; ++t) {
          // stencil index of the segment's first point, and the segment start's distance to
          // the ion's first point
          const int ext = min(ZS, ez - t * ZS);
          int d = (rz + t * ZS) % Nz;
          const int back = d == 0 ? 0 : Nz - d;
          const unsigned b = __ballot_sync(0xffffffffu, in && ext > 0 && (d < P || back < ext));
          if (lane == 0) zmask[t][wid] = b;
        }
      }
      __syncthreads();
      // ---- accumulate this thread's points over the ions that touch them --------------
      const int nw = (nst + 31) >> 5;
      const int xo = RC::XOFF + X * RC::NXV, yo = RC::YOFF + Y * RC::NYV, zo = RC::ZOFF + seg * RC::ZSEG;
      for (int w = 0; w < nw; ++w) {
        unsigned bits = xmask[X][w] & ymask[Y][w] & zmask[seg][w];
        while (bits) {
          const int t = w * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const float* rec = sw + t * RC::STR;
          const float4* wz = reinterpret_cast<const float4*>(rec + zo);
          if (MODE == 3) {
            const float* xe = rec + xo;
            const float4 ye = *reinterpret_cast<const float4*>(rec + yo);
            const float A0 = xe[0] * ye.x + xe[1] * ye.y + xe[3] * ye.z + xe[6] * ye.w;
            const float A1 = xe[2] * ye.x + xe[4] * ye.y + xe[7] * ye.z;
            const float A2 = xe[5] * ye.x + xe[8] * ye.y;
            const float A3 = xe[9] * ye.x;
#pragma unroll
            for (int z = 0; z < ZS; z += 4) {
              const float4 w0 = wz[z / 4], w1 = wz[2 + z / 4], w2 = wz[4 + z / 4], w3 = wz[6 + z / 4];
              dacc[z] += A0 * w0.x + A1 * w1.x + A2 * w2.x + A3 * w3.x;
              dacc[z + 1] += A0 * w0.y + A1 * w1.y + A2 * w2.y + A3 * w3.y;
              dacc[z + 2] += A0 * w0.z + A1 * w1.z + A2 * w2.z + A3 * w3.z;
              dacc[z + 3] += A0 * w0.w + A1 * w1.w + A2 * w2.w + A3 * w3.w;
            }
          } else if (TAN) {
            const float* xe = rec + xo;
            const float* ye = rec + yo;
            const float wy0 = ye[0], wy1 = ye[1], wy2 = ye[2];
            const float A0 = xe[0] * wy0 + xe[1] * wy1 + xe[2] * wy2;
            const float A1 = xe[3] * wy0 + xe[4] * wy1;
            const float A2 = xe[5] * wy0;
            const float4 z0a = wz[0], z0b = wz[1], z1a = wz[2], z1b = wz[3], z2a = wz[4], z2b = wz[5];
            const float W0[ZS] = {z0a.x, z0a.y, z0a.z, z0a.w, z0b.x, z0b.y, z0b.z, z0b.w};
            const float W1[ZS] = {z1a.x, z1a.y, z1a.z, z1a.w, z1b.x, z1b.y, z1b.z, z1b.w};
            const float W2[ZS] = {z2a.x, z2a.y, z2a.z, z2a.w, z2b.x, z2b.y, z2b.z, z2b.w};
#pragma unroll
            for (int z = 0; z < ZS; ++z) dacc[z] += A0 * W0[z] + A1 * W1[z] + A2 * W2[z];
            if (with_rho) {
              const float A = xe[6] * wy0 + xe[7] * wy1, B = xe[8] * wy0;
#pragma unroll
              for (int z = 0; z < ZS; ++z) acc[z] += A * W0[z] + B * W1[z];
            }
          } else {
            const float4 xe = *reinterpret_cast<const float4*>(rec + xo);
            const float2 ye = *reinterpret_cast<const float2*>(rec + yo);
            const float A = xe.x * ye.x + xe.y * ye.y, B = xe.z * ye.x;
            const float4 z0a = wz[0], z0b = wz[1], z1a = wz[2], z1b = wz[3];
            const float W0[ZS] = {z0a.x, z0a.y, z0a.z, z0a.w, z0b.x, z0b.y, z0b.z, z0b.w};
            const float W1[ZS] = {z1a.x, z1a.y, z1a.z, z1a.w, z1b.x, z1b.y, z1b.z, z1b.w};
#pragma unroll
            for (int z = 0; z < ZS; ++z) acc[z] += A * W0[z] + B * W1[z];
          }
        }
      }
      __syncthreads();
    }
    cnt = 0;
  }

  // ---- (5) write: every owned mesh point exactly once ---------------------------------
  if (X < ex && Y < ey) {
    const size_t off = (size_t(gx) * Ny + gy) * Nz + zs0;
    float* rho = a.mesh + F.mesh_off + off;
    float* drho = a.mesh + (MODE == 2 ? F.mesh_off : F.tmesh_off) + off;
    const int nz = min(ZS, ez - seg * ZS);
    const long long M = (long long)Nx * Ny * Nz;
#pragma unroll
    for (int z = 0; z < ZS; ++z)
      if (z < nz && index_ok((long long)(off + z), M)) {
        if (with_rho) rho[z] = acc[z];
        if (TAN) drho[z] = dacc[z];
      }
  }
}

// One instantiation's launch; the first use on a device raises its dynamic shared-memory limit.
template <class SH, int P, int MODE, bool BATCH>
int launch_order(pme_plan_t p, cudaStream_t s, int grid, const SpreadArgs& a) {
  constexpr int bytes = spread_smem_bytes<SH, P, rec_kind<MODE>()>();
  static int done_mask = 0;   // devices 0..31 already configured (idempotent if raced)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 32 || !(done_mask & (1 << dev))) {
    const int st = check_cuda(p, cudaFuncSetAttribute(k_spread<SH, P, MODE, BATCH>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
                              "cudaFuncSetAttribute");
    if (st) return st;
    if (dev < 32) done_mask |= 1 << dev;
  }
  pdl_launch(k_spread<SH, P, MODE, BATCH>, grid, SH::NT, bytes, s, a);
  count_launch();
  return PME_OK;
}

template <class SH, int MODE, bool BATCH>
int launch_t(pme_plan_t p, cudaStream_t s, float* mesh, const int* keep_rho, const float* theta = nullptr) {
  SpreadArgs a;
  a.theta = theta;
  a.keep_rho = MODE == 1 ? keep_rho : nullptr;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.mr = p->mr;
  a.start_b = p->sb.start_b;
  a.cand = p->cand;
  a.mesh = mesh;
  for (int gi = 0; gi < p->nogroups; ++gi) {
    const OrderGroup& G = p->ogroups[gi];
    const int grid = G.brick_hi - G.brick_lo;
    if (grid <= 0) continue;
    a.key_lo = G.brick_lo;
    int st = PME_OK;
    switch (G.order) {
      case 1: st = launch_order<SH, 1, MODE, BATCH>(p, s, grid, a); break;
      case 2: st = launch_order<SH, 2, MODE, BATCH>(p, s, grid, a); break;
      case 3: st = launch_order<SH, 3, MODE, BATCH>(p, s, grid, a); break;
      case 4: st = launch_order<SH, 4, MODE, BATCH>(p, s, grid, a); break;
      case 5: st = launch_order<SH, 5, MODE, BATCH>(p, s, grid, a); break;
      case 6: st = launch_order<SH, 6, MODE, BATCH>(p, s, grid, a); break;
      case 7: st = launch_order<SH, 7, MODE, BATCH>(p, s, grid, a); break;
      default: return set_error(p, PME_ERR_ARG, "spline order out of range");
    }
    if (st) return st;
    if ((st = check_launch(p, "k_spread"))) return st;
  }
  return PME_OK;
}

}  // namespace

// Every mode of one brick shape (one translation unit per shape, so they compile in parallel).
template <class SH>
int launch_spread_shape(pme_plan_t p, cudaStream_t s, int mode, float* mesh, const int* keep_rho,
                        const float* theta) {
  if (p->batch) {
    if (mode == 0) return launch_t<SH, 0, true>(p, s, mesh, keep_rho);
    if (mode == 1) return launch_t<SH, 1, true>(p, s, mesh, keep_rho);
    if (mode == 3) return launch_t<SH, 3, true>(p, s, mesh, nullptr, theta);
    return launch_t<SH, 2, true>(p, s, mesh, nullptr, theta);
  }
  if (mode == 0) return launch_t<SH, 0, false>(p, s, mesh, keep_rho);
  if (mode == 1) return launch_t<SH, 1, false>(p, s, mesh, keep_rho);
  if (mode == 3) return launch_t<SH, 3, false>(p, s, mesh, nullptr, theta);
  return launch_t<SH, 2, false>(p, s, mesh, nullptr, theta);
}

}  // namespace gbpme
