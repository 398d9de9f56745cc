// Gather of the potential mesh at the ions (the interpolation that is the adjoint of the
// spread of Eq. charge_dipole_assign; forces follow Eq. forces).
//
// For an ion with first stencil point m0 and offsets f, the interpolated potential
// phi(x) = sum_m W(x - m) Phi(m) has mesh-coordinate derivatives
//   M_abc = sum_{jx,jy,jz} Phi(m0 + j) W^(a)(t_jx) W^(b)(t_jy) W^(c)(t_jz),
// and r-space derivatives follow with D[a][b] = N_b C^{-1}[a][b] (d/dr = D d/dx).
//
// One launch per spline order covers the ions of every frame of that order.
// Work split: a group of 8 lanes per ion, lane l owning stencil z-offset l (l < p), so each
// mesh row segment is read by consecutive lanes. Each lane forms the y- and x-moments of its
// z-column, scales them by its own z-weights, and the group sums the moments with warp
// shuffles. Forward mode keeps orders <= 2 (potential, gradient, Hessian). Tangent mode
// (backward pass) keeps orders <= 3 of Phi and <= 2 of the tangent potential dPhi and
// evaluates the mesh part of the Hessian-vector product in mesh coordinates. Quadrupole mode
// (the rank-2 channel) writes the forward outputs and, from the orders-3 moments, the
// contraction Theta_i : grad^3 phi that the force on a point quadrupole needs:
// sum_ab Theta_ab d_a d_b d_c phi = (D v)_c with v_k = sum_ij Theta'_ij M_ijk, Theta' = D^T Theta D.
#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kGatherThreads = 128;
constexpr int kGroup = 8;

struct GatherArgs {
  FrameDesc one;
  FrameMaps maps;
  MeshRecords mr;
  const float* mesh;      // Phi of frame f at mesh_off, d Phi at tmesh_off
  const double* g_energy; // per frame
  float* out;
  const float* theta;     // quadrupole mode: Theta [caller index][6] (xx yy zz xy xz yz)
  float* qout;            // quadrupole mode: Theta : grad^3 phi at [caller index * 8 + 0..2]
  int t_lo, t_hi;         // sorted positions of this launch
};

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

// MODE: 0 forward, 1 tangent, 2 quadrupole forward
template <int P, int MODE, bool BATCH>
__global__ void __launch_bounds__(kGatherThreads) k_gather(GatherArgs a) {
  constexpr bool TAN = MODE == 1;
  constexpr int DM = MODE == 0 ? 2 : 3;
  const int gid = a.t_lo + (blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
  const int l = threadIdx.x & (kGroup - 1);
  const bool valid = gid < a.t_hi;
  const int ion = valid ? gid : a.t_lo;
  const int frame = BATCH ? a.maps.sorted_frame[ion] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, frame);
  const Geometry& g = F.g;
  const float* phi_mesh = a.mesh + F.mesh_off;
  const float* dphi_mesh = a.mesh + F.tmesh_off;
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
  int z = m.z + l;
  if (z >= g.N[2]) z -= g.N[2];
  const int Ny = g.N[1], Nz = g.N[2];

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
      int x = m.x + jx;
      if (x >= g.N[0]) x -= g.N[0];
      float r[DM + 1], rt[3];
#pragma unroll
      for (int b = 0; b <= DM; ++b) r[b] = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) rt[b] = 0.f;
#pragma unroll
      for (int jy = 0; jy < P; ++jy) {
        int y = m.y + jy;
        if (y >= Ny) y -= Ny;
        const size_t off = (size_t(x) * Ny + y) * Nz + z;
        const bool in_mesh = index_ok((long long)off, (long long)g.N[0] * Ny * Nz);
        const float v = in_mesh ? __ldg(phi_mesh + off) : 0.f;
#pragma unroll
        for (int b = 0; b <= DM; ++b) r[b] += v * wy[b][jy];
        if (TAN) {
          const float dv = in_mesh ? __ldg(dphi_mesh + off) : 0.f;
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
    float m3[10];   // quadrupole mode: 300 030 003 210 201 120 021 102 012 111
    if constexpr (MODE == 2) {
      m3[0] = MOM(3, 0, 0); m3[1] = MOM(0, 3, 0); m3[2] = MOM(0, 0, 3);
      m3[3] = MOM(2, 1, 0); m3[4] = MOM(2, 0, 1); m3[5] = MOM(1, 2, 0);
      m3[6] = MOM(0, 2, 1); m3[7] = MOM(1, 0, 2); m3[8] = MOM(0, 1, 2);
      m3[9] = MOM(1, 1, 1);
    }
    if (!valid || l != 0) return;
    if constexpr (MODE == 2) {
      const float* th = a.theta + size_t(m.w) * 6;
      const float T[3][3] = {{th[0], th[3], th[4]}, {th[3], th[1], th[5]}, {th[4], th[5], th[2]}};
      float TD[3][3], Tp[3][3];   // Theta D, D^T Theta D
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          TD[r][c] = T[r][0] * g.D[0 * 3 + c] + T[r][1] * g.D[1 * 3 + c] + T[r][2] * g.D[2 * 3 + c];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          Tp[r][c] = g.D[0 * 3 + r] * TD[0][c] + g.D[1 * 3 + r] * TD[1][c] + g.D[2 * 3 + r] * TD[2][c];
      const float sxy = Tp[0][1] + Tp[1][0], sxz = Tp[0][2] + Tp[2][0], syz = Tp[1][2] + Tp[2][1];
      // v_k = sum_ij Theta'_ij M_ijk
      float v[3];
      v[0] = Tp[0][0] * m3[0] + Tp[1][1] * m3[5] + Tp[2][2] * m3[7] + sxy * m3[3] + sxz * m3[4] + syz * m3[9];
      v[1] = Tp[0][0] * m3[3] + Tp[1][1] * m3[1] + Tp[2][2] * m3[8] + sxy * m3[5] + sxz * m3[9] + syz * m3[6];
      v[2] = Tp[0][0] * m3[4] + Tp[1][1] * m3[6] + Tp[2][2] * m3[2] + sxy * m3[9] + sxz * m3[7] + syz * m3[8];
      float tr[3];
      apply_D(g.D, v, tr);
      float* qo = a.qout + size_t(m.w) * 8;
      qo[0] = tr[0];
      qo[1] = tr[1];
      qo[2] = tr[2];
    }
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
    return;
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
    if (!valid || l != 0) return;
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
#undef MOM
#undef TMOM
}

template <int MODE, bool BATCH>
int launch_t(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const double* g_energy,
             float* out, const float* theta = nullptr, float* qout = nullptr) {
  GatherArgs a;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.mr = p->mr;
  a.mesh = mesh;
  a.g_energy = g_energy;
  a.out = out;
  a.theta = theta;
  a.qout = qout;
  for (int gi = 0; gi < p->nogroups; ++gi) {
    const OrderGroup& G = p->ogroups[gi];
    a.t_lo = BATCH ? G.sorted_lo : 0;
    a.t_hi = BATCH ? G.sorted_hi : n;
    const int grid = int((size_t(a.t_hi - a.t_lo) * kGroup + kGatherThreads - 1) / kGatherThreads);
    if (grid <= 0) continue;
    switch (G.order) {
      case 1: k_gather<1, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      case 2: k_gather<2, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      case 3: k_gather<3, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      case 4: k_gather<4, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      case 5: k_gather<5, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      case 6: k_gather<6, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      case 7: k_gather<7, MODE, BATCH><<<grid, kGatherThreads, 0, s>>>(a); break;
      default: return set_error(p, PME_ERR_ARG, "spline order out of range");
    }
    count_launch();
    int st = check_launch(p, "k_gather");
    if (st) return st;
  }
  return PME_OK;
}

}  // namespace

int launch_gather(pme_plan_t p, cudaStream_t s, int n, const float* mesh, bool tangent,
                  const double* g_energy, float* out) {
  if (p->batch)
    return tangent ? launch_t<1, true>(p, s, n, mesh, g_energy, out)
                   : launch_t<0, true>(p, s, n, mesh, nullptr, out);
  return tangent ? launch_t<1, false>(p, s, n, mesh, g_energy, out)
                 : launch_t<0, false>(p, s, n, mesh, nullptr, out);
}

int launch_gather_quad(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const float* theta,
                       float* out, float* qout) {
  if (p->batch) return launch_t<2, true>(p, s, n, mesh, nullptr, out, theta, qout);
  return launch_t<2, false>(p, s, n, mesh, nullptr, out, theta, qout);
}

GBPME_BOUNDS_READER(bounds_hit_gather)

}  // namespace gbpme
