// Spread of charges and dipoles onto the mesh (Section 2.3.2, Eq. charge_dipole_assign).
//
// Owner-computes design: one CTA owns one brick of BX x BY x BZ mesh points of one frame and
// is the only writer of those points, so the mesh needs no zeroing and no global atomics.
// One launch covers every brick of every frame of one spline order. The CTA walks
// the ions of the few bricks whose ions' stencils can reach it (ions are sorted by the brick
// of their first stencil point), keeps those whose p^3 stencil really overlaps it (an
// order-preserving compaction), stages their 1D spline weights in shared memory, and then
// each thread accumulates the z-column (X, Y) it owns inside a shared-memory tile. Ions are
// visited in a fixed order, so the result is bitwise reproducible. The finished tile is
// flushed with coalesced stores along z (the fastest mesh axis).
//
// Tangent mode (backward pass) spreads, in the same sweep, the tangent density
//   d rho = sum_i [dq_i + (dmu_i + q_i dr_i) . grad + (mu_i . grad)(dr_i . grad)] W(x_i - m)
// (gradients with respect to the source position), the directional derivative of rho_mesh
// along the cotangent direction.
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int BX = 8, BY = 8, BZ = 32;
constexpr int NT = BX * BY;           // one thread per owned column
constexpr int kMaxCand = kMaxCandPerDim * kMaxCandPerDim * kMaxCandPerDim;

struct SpreadArgs {
  FrameDesc one;
  FrameMaps maps;
  int key_lo;           // first global brick of this launch
  MeshRecords mr;
  const int* start_b;
  const int* cand;      // base of the candidate tables
  float* mesh;          // base of the meshes: rho at mesh_off, d rho at tmesh_off
};

template <int P, bool TAN, bool BATCH>
__global__ void __launch_bounds__(NT) k_spread(SpreadArgs a) {
  constexpr int DW = TAN ? 3 : 2;                 // weight derivative orders kept
  constexpr int CAP = TAN ? NT : 2 * NT;          // staged ions per batch
  constexpr int WSTRIDE = 3 * DW * P;             // floats of weights per staged ion
  constexpr int NC = TAN ? 11 : 4;                // coefficients per staged ion

  __shared__ float tile[BZ][NT + 1];
  __shared__ float dtile[TAN ? BZ : 1][NT + 1];
  __shared__ float sw[CAP * WSTRIDE];
  __shared__ float sc[CAP * NC];
  __shared__ int sm0[CAP * 3];
  __shared__ int slist[CAP];
  __shared__ int cand_lo[kMaxCand];
  __shared__ int cand_cum[kMaxCand + 1];
  __shared__ int warp_cnt[NT / 32];
  __shared__ int ncand_s;

  const int gkey = a.key_lo + blockIdx.x;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, BATCH ? a.maps.brick_frame[gkey] : 0);
  const Geometry& g = F.g;
  const int tid = threadIdx.x;
  const int bkey = gkey - F.brick_off;
  const int bz = bkey % g.nb[2];
  const int by = (bkey / g.nb[2]) % g.nb[1];
  const int bx = bkey / (g.nb[2] * g.nb[1]);
  const int b0x = bx * BX, b0y = by * BY, b0z = bz * BZ;
  const int ex = min(BX, g.N[0] - b0x), ey = min(BY, g.N[1] - b0y), ez = min(BZ, g.N[2] - b0z);

  for (int e = tid; e < BZ * (NT + 1); e += NT) {
    (&tile[0][0])[e] = 0.f;
    if (TAN) (&dtile[0][0])[e] = 0.f;
  }
  // candidate source bricks: product of the per-axis lists, in a fixed order
  if (tid == 0) {
    const int* ct = a.cand + F.cand_off;
    const int* cx = ct + (0 * F.max_nb + bx) * (1 + kMaxCandPerDim);
    const int* cy = ct + (1 * F.max_nb + by) * (1 + kMaxCandPerDim);
    const int* cz = ct + (2 * F.max_nb + bz) * (1 + kMaxCandPerDim);
    int k = 0, cum = 0;
    for (int ix = 0; ix < cx[0]; ++ix)
      for (int iy = 0; iy < cy[0]; ++iy)
        for (int iz = 0; iz < cz[0]; ++iz) {
          const int key = F.brick_off + (cx[1 + ix] * g.nb[1] + cy[1 + iy]) * g.nb[2] + cz[1 + iz];
          const int lo = a.start_b[key], hi = a.start_b[key + 1];
          cand_lo[k] = lo;
          cand_cum[k] = cum;
          cum += hi - lo;
          ++k;
        }
    cand_cum[k] = cum;
    ncand_s = k;
  }
  __syncthreads();
  const int ncand = ncand_s;
  const int total = cand_cum[ncand];

  const int X = tid / BY, Y = tid % BY;
  const bool own = (X < ex) && (Y < ey);
  const int gx = b0x + X, gy = b0y + Y;
  const int lane = tid & 31, wid = tid >> 5;

  int cnt = 0;
  for (int cursor = 0; cursor < total; cursor += NT) {
    // ---- fill: test NT candidates, append the overlapping ones in order --------------
    const int gi = cursor + tid;
    int ion = -1;
    bool take = false;
    if (gi < total) {
      int k = 0;
      while (k + 1 < ncand && cand_cum[k + 1] <= gi) ++k;
      ion = cand_lo[k] + (gi - cand_cum[k]);
      const int4 m = a.mr.idx[ion];
      int d;
      d = b0x - m.x; if (d < 0) d += g.N[0];
      const bool okx = (d <= P - 1) || (d >= g.N[0] - ex + 1);
      d = b0y - m.y; if (d < 0) d += g.N[1];
      const bool oky = (d <= P - 1) || (d >= g.N[1] - ey + 1);
      d = b0z - m.z; if (d < 0) d += g.N[2];
      const bool okz = (d <= P - 1) || (d >= g.N[2] - ez + 1);
      take = okx && oky && okz;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
      if (w < wid) before += warp_cnt[w];
      tot += warp_cnt[w];
    }
    if (take) slist[cnt + before + __popc(bal & ((1u << lane) - 1u))] = ion;
    cnt += tot;
    __syncthreads();
    const bool last = cursor + NT >= total;
    if (cnt > CAP - NT || last) {
      // ---- stage weights and coefficients of the listed ions -----------------------
      for (int l = tid; l < cnt; l += NT) {
        const int src = slist[l];
        const int4 m = a.mr.idx[src];
        const float4 fq = a.mr.fq[src];
        const float4 dm = a.mr.dm[src];
        float w[DW][P];
        float* dst = sw + l * WSTRIDE;
        spline_weights<P, DW - 1>(fq.x, w);
#pragma unroll
        for (int d = 0; d < DW; ++d)
#pragma unroll
          for (int j = 0; j < P; ++j) dst[(0 * DW + d) * P + j] = w[d][j];
        spline_weights<P, DW - 1>(fq.y, w);
#pragma unroll
        for (int d = 0; d < DW; ++d)
#pragma unroll
          for (int j = 0; j < P; ++j) dst[(1 * DW + d) * P + j] = w[d][j];
        spline_weights<P, DW - 1>(fq.z, w);
#pragma unroll
        for (int d = 0; d < DW; ++d)
#pragma unroll
          for (int j = 0; j < P; ++j) dst[(2 * DW + d) * P + j] = w[d][j];
        sm0[3 * l] = m.x;
        sm0[3 * l + 1] = m.y;
        sm0[3 * l + 2] = m.z;
        float* c = sc + l * NC;
        c[0] = fq.w;
        c[1] = dm.x;
        c[2] = dm.y;
        c[3] = dm.z;
        if (TAN) {
          const float4 tq = a.mr.tq[src];
          const float4 tt = a.mr.tt[src];
          c[4] = tq.x;
          c[5] = tq.y;
          c[6] = tq.z;
          c[7] = tq.w;
          c[8] = tt.x;
          c[9] = tt.y;
          c[10] = tt.z;
        }
      }
      __syncthreads();
      // ---- accumulate the owned column ----------------------------------------------
      if (own) {
        for (int l = 0; l < cnt; ++l) {
          int dx = gx - sm0[3 * l];
          if (dx < 0) dx += g.N[0];
          if (dx >= P) continue;
          int dy = gy - sm0[3 * l + 1];
          if (dy < 0) dy += g.N[1];
          if (dy >= P) continue;
          const float* w = sw + l * WSTRIDE;
          const float* c = sc + l * NC;
          const float wx = w[(0 * DW + 0) * P + dx], wx1 = w[(0 * DW + 1) * P + dx];
          const float wy = w[(1 * DW + 0) * P + dy], wy1 = w[(1 * DW + 1) * P + dy];
          const float wxy = wx * wy;
          // rho: coefficient of W_z and of W'_z
          const float A = c[0] * wxy + c[1] * wx1 * wy + c[2] * wx * wy1;
          const float B = c[3] * wxy;
          float A0 = 0.f, A1 = 0.f, A2 = 0.f;
          if (TAN) {
            const float wx2 = w[(0 * DW + 2) * P + dx], wy2 = w[(1 * DW + 2) * P + dy];
            const float mx = c[1], my = c[2], mz = c[3];
            const float tx = c[8], ty = c[9], tz = c[10];
            A0 = c[4] * wxy + c[5] * wx1 * wy + c[6] * wx * wy1 + mx * tx * wx2 * wy +
                 my * ty * wx * wy2 + (mx * ty + my * tx) * wx1 * wy1;
            A1 = c[7] * wxy + (mx * tz + mz * tx) * wx1 * wy + (my * tz + mz * ty) * wx * wy1;
            A2 = mz * tz * wxy;
          }
          const int mz0 = sm0[3 * l + 2];
#pragma unroll
          for (int jz = 0; jz < P; ++jz) {
            int Z = mz0 + jz - b0z;
            if (Z < 0) Z += g.N[2];
            else if (Z >= g.N[2]) Z -= g.N[2];
            if (Z < ez) {
              const float wz = w[(2 * DW + 0) * P + jz], wz1 = w[(2 * DW + 1) * P + jz];
              tile[Z][tid] += A * wz + B * wz1;
              if (TAN) {
                const float wz2 = w[(2 * DW + 2) * P + jz];
                dtile[Z][tid] += A0 * wz + A1 * wz1 + A2 * wz2;
              }
            }
          }
        }
      }
      __syncthreads();
      cnt = 0;
    }
  }
  __syncthreads();
  // ---- flush: every owned mesh point written exactly once, z fastest ----------------
  const int Ny = g.N[1], Nz = g.N[2];
  float* rho = a.mesh + F.mesh_off;
  float* drho = a.mesh + F.tmesh_off;
  for (int e = tid; e < NT * BZ; e += NT) {
    const int Z = e % BZ, col = e / BZ;
    const int x = col / BY, y = col % BY;
    if (x < ex && y < ey && Z < ez) {
      const size_t off = (size_t(b0x + x) * Ny + (b0y + y)) * Nz + (b0z + Z);
      rho[off] = tile[Z][col];
      if (TAN) drho[off] = dtile[Z][col];
    }
  }
}

template <bool TAN, bool BATCH>
int launch_t(pme_plan_t p, cudaStream_t s, float* mesh) {
  SpreadArgs a;
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
    switch (G.order) {
      case 1: k_spread<1, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      case 2: k_spread<2, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      case 3: k_spread<3, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      case 4: k_spread<4, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      case 5: k_spread<5, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      case 6: k_spread<6, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      case 7: k_spread<7, TAN, BATCH><<<grid, NT, 0, s>>>(a); break;
      default: return set_error(p, PME_ERR_ARG, "spline order out of range");
    }
    count_launch();
    int st = check_launch(p, "k_spread");
    if (st) return st;
  }
  return PME_OK;
}

}  // namespace

void spread_brick_shape(int shape[3]) {
  shape[0] = BX;
  shape[1] = BY;
  shape[2] = BZ;
}

int launch_spread(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh) {
  if (p->batch)
    return tangent ? launch_t<true, true>(p, s, mesh) : launch_t<false, true>(p, s, mesh);
  return tangent ? launch_t<true, false>(p, s, mesh) : launch_t<false, false>(p, s, mesh);
}

}  // namespace gbpme
