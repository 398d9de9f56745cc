// Gather of the potential mesh at the ions (the interpolation that is the adjoint of the
// spread of Eq. charge_dipole_assign; forces follow Eq. forces).
//
// For an ion with first stencil point m0 and offsets f, the interpolated potential
// phi(x) = sum_m W(x - m) Phi(m) has mesh-coordinate derivatives
//   M_abc = sum_{jx,jy,jz} Phi(m0 + j) W^(a)(t_jx) W^(b)(t_jy) W^(c)(t_jz),
// and r-space derivatives follow with D[a][b] = N_b C^{-1}[a][b] (d/dr = D d/dx).
//
// One launch per spline order covers the ions of every frame of that order, one block per
// mesh brick (the bricks of the sort: an ion belongs to the brick holding its first stencil
// point). The block loads the brick's tile of Phi (and d Phi) -- the brick plus p - 1 points
// on the upper side of each axis, wrapped periodically -- into shared memory, eight loads in
// flight per thread, and then evaluates the brick's ions from it, 32 at a time.
// Work split: a group of 8 lanes per ion, lane l owning stencil z-offset l (l < p), so each
// tile row segment is read by consecutive lanes. Each lane forms the y- and x-moments of its
// z-column, scales them by its own z-weights, and the group sums the moments with warp
// shuffles. Forward mode keeps orders <= 2 (potential, gradient, Hessian). Tangent mode
// (backward pass) keeps orders <= 3 of Phi and <= 2 of the tangent potential dPhi and
// evaluates the mesh part of the Hessian-vector product in mesh coordinates.
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kGatherThreads = 256;
constexpr int kGroup = 8;
constexpr int kTileLoads = 8;   // tile loads a thread keeps in flight
constexpr int GBX = 8, GBY = 8, GBZ = 32;   // the sort's brick shape

struct GatherArgs {
  FrameDesc one;
  FrameMaps maps;
  MeshRecords mr;
  const int* start_b;     // sorted segment of each global brick
  const float* mesh;      // Phi of frame f at mesh_off, d Phi at tmesh_off
  const double* g_energy; // per frame
  float* out;
  int key_lo;             // first global brick of this launch
};

template <int P>
struct Tile {
  static constexpr int X = GBX + P - 1, Y = GBY + P - 1, Z = GBZ + P - 1, N = X * Y * Z;
};

template <int P, bool TAN>
constexpr int gather_smem_bytes() {
  return Tile<P>::N * (TAN ? 2 : 1) * 4;
}

__device__ __forceinline__ float group_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// y = D x
__device__ __forceinline__ void apply_D(const float* D, const float x[3], float y[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) y[a] = D[a * 3 + 0] * x[0] + D[a * 3 + 1] * x[1] + D[a * 3 + 2] * x[2];
}

template <int P, bool TAN, bool BATCH>
__global__ void __launch_bounds__(kGatherThreads) k_gather(GatherArgs a) {
  constexpr int DM = TAN ? 3 : 2;
  using TL = Tile<P>;
  extern __shared__ __align__(16) float tile[];   // [TL::N] Phi, then [TL::N] d Phi
  const int gkey = a.key_lo + blockIdx.x;
  const int lo_ion = a.start_b[gkey], hi_ion = a.start_b[gkey + 1];
  if (lo_ion == hi_ion) return;   // uniform: no ion starts its stencil in this brick
  const int frame = BATCH ? a.maps.brick_frame[gkey] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, frame);
  const Geometry& g = F.g;
  const int Nx = g.N[0], Ny = g.N[1], Nz = g.N[2];
  const int bkey = gkey - F.brick_off;
  const int b0z = (bkey % g.nb[2]) * GBZ;
  const int b0y = ((bkey / g.nb[2]) % g.nb[1]) * GBY;
  const int b0x = (bkey / (g.nb[2] * g.nb[1])) * GBX;
  {
    const float* phi_mesh = a.mesh + F.mesh_off;
    const float* dphi_mesh = a.mesh + F.tmesh_off;
    for (int t0 = threadIdx.x; t0 < TL::N; t0 += kTileLoads * blockDim.x) {
      float v[kTileLoads], dv[kTileLoads];
#pragma unroll
      for (int u = 0; u < kTileLoads; ++u) {
        const int t = t0 + u * blockDim.x;
        v[u] = 0.f;
        dv[u] = 0.f;
        if (t < TL::N) {
          const int tz = t % TL::Z, r = t / TL::Z;
          const int ty = r % TL::Y, tx = r / TL::Y;
          int x = b0x + tx, y = b0y + ty, z = b0z + tz;
          while (x >= Nx) x -= Nx;
          while (y >= Ny) y -= Ny;
          while (z >= Nz) z -= Nz;
          const size_t off = (size_t(x) * Ny + y) * Nz + z;
          v[u] = __ldg(phi_mesh + off);
          if (TAN) dv[u] = __ldg(dphi_mesh + off);
        }
      }
#pragma unroll
      for (int u = 0; u < kTileLoads; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < TL::N) {
          tile[t] = v[u];
          if (TAN) tile[TL::N + t] = dv[u];
        }
      }
    }
  }
  __syncthreads();
  const float* dtile = tile + TL::N;
  const int l = threadIdx.x & (kGroup - 1);
  for (int base = lo_ion; base < hi_ion; base += kGatherThreads / kGroup) {
  const int gid = base + int(threadIdx.x) / kGroup;
  const bool valid = gid < hi_ion;
  const int ion = valid ? gid : lo_ion;
  const int4 m = a.mr.idx[ion];
  const float4 fq = a.mr.fq[ion];
  float wx[DM + 1][P], wy[DM + 1][P], wzall[DM + 1][P];
  spline_weights<P, DM>(fq.x, wx);
  spline_weights<P, DM>(fq.y, wy);
  spline_weights<P, DM>(fq.z, wzall);
  const bool act = valid && (l < P);
  float wz[DM + 1];
#pragma unroll
  for (int c = 0; c <= DM; ++c) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) v = (j == l) ? wzall[c][j] : v;
    wz[c] = act ? v : 0.f;
  }
  // the ion's first stencil point lies in this brick: its stencil is inside the tile
  const int lx = m.x - b0x, ly = m.y - b0y, lz = m.z - b0z + l;

  // S[a][b]: sum over (jx, jy) of Phi * W^(a)_x * W^(b)_y for this lane's z, a + b <= DM
  float S[DM + 1][DM + 1];
  float T[3][3];   // same for the tangent mesh, a + b <= 2
#pragma unroll
  for (int i = 0; i <= DM; ++i)
#pragma unroll
    for (int j = 0; j <= DM; ++j) S[i][j] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) T[i][j] = 0.f;

  if (act) {
#pragma unroll
    for (int jx = 0; jx < P; ++jx) {
      float r[DM + 1], rt[3];
#pragma unroll
      for (int b = 0; b <= DM; ++b) r[b] = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) rt[b] = 0.f;
#pragma unroll
      for (int jy = 0; jy < P; ++jy) {
        const int off = ((lx + jx) * TL::Y + (ly + jy)) * TL::Z + lz;
        const float v = tile[off];
#pragma unroll
        for (int b = 0; b <= DM; ++b) r[b] += v * wy[b][jy];
        if (TAN) {
          const float dv = dtile[off];
#pragma unroll
          for (int b = 0; b < 3; ++b) rt[b] += dv * wy[b][jy];
        }
      }
#pragma unroll
      for (int ia = 0; ia <= DM; ++ia)
#pragma unroll
        for (int ib = 0; ib <= DM; ++ib)
          if (ia + ib <= DM) S[ia][ib] += r[ib] * wx[ia][jx];
      if (TAN) {
#pragma unroll
        for (int ia = 0; ia < 3; ++ia)
#pragma unroll
          for (int ib = 0; ib < 3; ++ib)
            if (ia + ib <= 2) T[ia][ib] += rt[ib] * wx[ia][jx];
      }
    }
  }
  // moments M_abc, reduced over the group's z-lanes
#define MOM(ia, ib, ic) group_sum(S[ia][ib] * wz[ic])
#define TMOM(ia, ib, ic) group_sum(T[ia][ib] * wz[ic])
  const float m000 = MOM(0, 0, 0);
  const float m100 = MOM(1, 0, 0), m010 = MOM(0, 1, 0), m001 = MOM(0, 0, 1);
  const float m200 = MOM(2, 0, 0), m020 = MOM(0, 2, 0), m002 = MOM(0, 0, 2);
  const float m110 = MOM(1, 1, 0), m101 = MOM(1, 0, 1), m011 = MOM(0, 1, 1);
  if (!TAN) {
    if (!valid || l != 0) continue;
    const float gx[3] = {m100, m010, m001};
    const float Hx[3][3] = {{m200, m110, m101}, {m110, m020, m011}, {m101, m011, m002}};
    float gr[3];
    apply_D(g.D, gx, gr);
    float HD[3][3];   // Hx D^T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        HD[i][b] = Hx[i][0] * g.D[b * 3 + 0] + Hx[i][1] * g.D[b * 3 + 1] + Hx[i][2] * g.D[b * 3 + 2];
    float Hr[3][3];   // D Hx D^T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Hr[i][b] = g.D[i * 3 + 0] * HD[0][b] + g.D[i * 3 + 1] * HD[1][b] + g.D[i * 3 + 2] * HD[2][b];
    float* o = a.out + size_t(m.w) * 10;
    o[0] = m000;
    o[1] = gr[0];
    o[2] = gr[1];
    o[3] = gr[2];
    o[4] = Hr[0][0];
    o[5] = Hr[1][1];
    o[6] = Hr[2][2];
    o[7] = Hr[0][1];
    o[8] = Hr[0][2];
    o[9] = Hr[1][2];
    continue;
  }
  if constexpr (TAN) {
    const float m300 = MOM(3, 0, 0), m030 = MOM(0, 3, 0), m003 = MOM(0, 0, 3);
    const float m210 = MOM(2, 1, 0), m201 = MOM(2, 0, 1), m120 = MOM(1, 2, 0);
    const float m021 = MOM(0, 2, 1), m102 = MOM(1, 0, 2), m012 = MOM(0, 1, 2);
    const float m111 = MOM(1, 1, 1);
    const float t000 = TMOM(0, 0, 0);
    const float t100 = TMOM(1, 0, 0), t010 = TMOM(0, 1, 0), t001 = TMOM(0, 0, 1);
    const float t200 = TMOM(2, 0, 0), t020 = TMOM(0, 2, 0), t002 = TMOM(0, 0, 2);
    const float t110 = TMOM(1, 1, 0), t101 = TMOM(1, 0, 1), t011 = TMOM(0, 1, 1);
    if (!valid || l != 0) continue;
    const float gE = a.g_energy ? float(a.g_energy[frame]) : 0.f;
    const float4 dm = a.mr.dm[ion];   // m = D^T mu
    const float4 tq = a.mr.tq[ion];   // dq, dd = D^T (dmu + q dr)
    const float4 tt = a.mr.tt[ion];   // t = D^T dr
    const float q = fq.w, dq = tq.x;
    const float mv[3] = {dm.x, dm.y, dm.z};
    const float dd[3] = {tq.y, tq.z, tq.w};
    const float tv[3] = {tt.x, tt.y, tt.z};
    const float gx[3] = {m100, m010, m001};
    const float Hx[3][3] = {{m200, m110, m101}, {m110, m020, m011}, {m101, m011, m002}};
    const float dgx[3] = {t100, t010, t001};
    const float dHx[3][3] = {{t200, t110, t101}, {t110, t020, t011}, {t101, t011, t002}};
    // third-derivative tensor T3[a][b][c] of the potential in mesh coordinates
    float T3[3][3][3];
    T3[0][0][0] = m300; T3[1][1][1] = m030; T3[2][2][2] = m003;
    T3[0][0][1] = T3[0][1][0] = T3[1][0][0] = m210;
    T3[0][0][2] = T3[0][2][0] = T3[2][0][0] = m201;
    T3[0][1][1] = T3[1][0][1] = T3[1][1][0] = m120;
    T3[1][1][2] = T3[1][2][1] = T3[2][1][1] = m021;
    T3[0][2][2] = T3[2][0][2] = T3[2][2][0] = m102;
    T3[1][2][2] = T3[2][1][2] = T3[2][2][1] = m012;
    T3[0][1][2] = T3[0][2][1] = T3[1][0][2] = T3[1][2][0] = T3[2][0][1] = T3[2][1][0] = m111;
    // D^T w with w = gE mu + dmu + q dr  ->  gE m + dd
    const float wv[3] = {gE * mv[0] + dd[0], gE * mv[1] + dd[1], gE * mv[2] + dd[2]};
    float xr[3], xm[3];
    const float cq = gE * q + dq;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float Hw = 0.f, Ht = 0.f, dHm = 0.f, T3mt = 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Hw += Hx[i][j] * wv[j];
        Ht += Hx[i][j] * tv[j];
        dHm += dHx[i][j] * mv[j];
#pragma unroll
        for (int k = 0; k < 3; ++k) T3mt += T3[i][j][k] * mv[j] * tv[k];
      }
      // grad_r (mesh coords) = (gE q + dq) g + H w + q dg + dH m + T3[m, t]
      xr[i] = cq * gx[i] + Hw + q * dgx[i] + dHm + T3mt;
      // grad_mu (mesh coords) = gE g + dg + H t
      xm[i] = gE * gx[i] + dgx[i] + Ht;
    }
    float gr[3], gm[3];
    apply_D(g.D, xr, gr);
    apply_D(g.D, xm, gm);
    // grad_q = gE phi + dphi + g . t
    const float gq = gE * m000 + t000 + gx[0] * tv[0] + gx[1] * tv[1] + gx[2] * tv[2];
    float* o = a.out + size_t(m.w) * 8;
    o[0] = gr[0];
    o[1] = gr[1];
    o[2] = gr[2];
    o[3] = gq;
    o[4] = gm[0];
    o[5] = gm[1];
    o[6] = gm[2];
    o[7] = 0.f;
  }
  }   // ions of the brick
#undef MOM
#undef TMOM
}

// One instantiation's launch; the first use on a device raises its dynamic shared-memory limit.
template <int P, bool TAN, bool BATCH>
int launch_order(pme_plan_t p, cudaStream_t s, int grid, const GatherArgs& a) {
  constexpr int bytes = gather_smem_bytes<P, TAN>();
  static unsigned done_mask = 0;   // devices 0..31 already configured (idempotent if raced)
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 32 || !(done_mask & (1u << dev))) {
    const int st = check_cuda(p, cudaFuncSetAttribute(k_gather<P, TAN, BATCH>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
                              "cudaFuncSetAttribute");
    if (st) return st;
    if (dev < 32) done_mask |= 1u << dev;
  }
  k_gather<P, TAN, BATCH><<<grid, kGatherThreads, bytes, s>>>(a);
  return PME_OK;
}

template <bool TAN, bool BATCH>
int launch_t(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const double* g_energy,
             float* out) {
  GatherArgs a;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.mr = p->mr;
  a.start_b = p->sb.start_b;
  a.mesh = mesh;
  a.g_energy = g_energy;
  a.out = out;
  if (n <= 0 && !BATCH) return PME_OK;
  for (int gi = 0; gi < p->nogroups; ++gi) {
    const OrderGroup& G = p->ogroups[gi];
    const int grid = G.brick_hi - G.brick_lo;
    if (grid <= 0) continue;
    a.key_lo = G.brick_lo;
    int st = PME_OK;
    switch (G.order) {
      case 1: st = launch_order<1, TAN, BATCH>(p, s, grid, a); break;
      case 2: st = launch_order<2, TAN, BATCH>(p, s, grid, a); break;
      case 3: st = launch_order<3, TAN, BATCH>(p, s, grid, a); break;
      case 4: st = launch_order<4, TAN, BATCH>(p, s, grid, a); break;
      case 5: st = launch_order<5, TAN, BATCH>(p, s, grid, a); break;
      case 6: st = launch_order<6, TAN, BATCH>(p, s, grid, a); break;
      case 7: st = launch_order<7, TAN, BATCH>(p, s, grid, a); break;
      default: return set_error(p, PME_ERR_ARG, "spline order out of range");
    }
    if (st) return st;
    count_launch();
    if ((st = check_launch(p, "k_gather"))) return st;
  }
  return PME_OK;
}

}  // namespace

int launch_gather(pme_plan_t p, cudaStream_t s, int n, const float* mesh, bool tangent,
                  const double* g_energy, float* out) {
  if (p->batch)
    return tangent ? launch_t<true, true>(p, s, n, mesh, g_energy, out)
                   : launch_t<false, true>(p, s, n, mesh, nullptr, out);
  return tangent ? launch_t<true, false>(p, s, n, mesh, g_energy, out)
                 : launch_t<false, false>(p, s, n, mesh, nullptr, out);
}

}  // namespace gbpme
