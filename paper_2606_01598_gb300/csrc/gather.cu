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
  int finish;             // tangent mode: write the backward's gradients (fin), not out
  BackwardFinish fin;
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

// Lanes per ion of k_gather: P (one per stencil z-offset), 32 / P ions per warp (the last
// 32 mod P lanes idle).
template <int P>
__host__ __device__ constexpr int gather_ions_per_warp() {
  return 32 / P;
}

// Sum over the P lanes of a group (lane l of the group holds v); valid in lane 0 of the group.
template <int P>
__device__ __forceinline__ float group_sum_p(float v, int l) {
#pragma unroll
  for (int off = 1; off < P; off <<= 1) {
    const float t = __shfl_down_sync(0xffffffffu, v, off);
    if ((l & (2 * off - 1)) == 0 && l + off < P) v += t;
  }
  return v;
}

// Per-group weight tables in shared memory: [axis][stencil index][order], orders padded to
// 4; the groups of a warp lie an odd number of 16-byte units apart, so that the same entry of
// every group falls in distinct banks.
template <int P>
__host__ __device__ constexpr int gather_tab_floats() {
  return 4 * ((3 * P + 1) | 1);
}

// MODE: 0 forward, 1 tangent, 2 quadrupole forward
template <int P, int MODE, bool BATCH>
__global__ void __launch_bounds__(kGatherThreads) k_gather(GatherArgs a) {
  pdl_begin();
  constexpr bool TAN = MODE == 1;
  constexpr int DM = MODE == 0 ? 2 : 3;
  constexpr int IPW = gather_ions_per_warp<P>();
  constexpr int TABF = gather_tab_floats<P>();
  static_assert(DM <= 3, "orders fit the table");
  __shared__ __align__(16) float tabs[kGatherThreads / 32][IPW][TABF];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane / P, l = lane - grp * P;
  const int gid = a.t_lo + (blockIdx.x * (kGatherThreads / 32) + wid) * IPW + grp;
  const bool valid = grp < IPW && gid < a.t_hi;
  const int ion = valid ? gid : a.t_lo;
  const int frame = BATCH ? a.maps.sorted_frame[ion] : 0;
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, frame);
  const Geometry& g = F.g;
  const float* phi_mesh = a.mesh + F.mesh_off;
  const float* dphi_mesh = a.mesh + F.tmesh_off;
  const int4 m = a.mr.idx[ion];
  const float4 fq = a.mr.fq[ion];
  // the weights of each axis once per ion: lanes 0, 1, 2 of the group take x, y, z and put
  // them in the group's table
  float* tab = tabs[wid][grp < IPW ? grp : 0];
  auto put = [&](int ax, const float (&w)[DM + 1][P]) {
#pragma unroll
    for (int j = 0; j < P; ++j)
      *reinterpret_cast<float4*>(tab + (ax * P + j) * 4) =
          make_float4(w[0][j], w[1][j], w[2][j], DM >= 3 ? w[DM][j] : 0.f);
  };
  if constexpr (P >= 3) {
    const float f = l == 0 ? fq.x : (l == 1 ? fq.y : fq.z);
    float w[DM + 1][P];
    spline_weights<P, DM>(f, w);
    if (valid && l < 3) put(l, w);
  } else {   // fewer than three lanes: lane 0 forms all three
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      float w[DM + 1][P];
      spline_weights<P, DM>(ax == 0 ? fq.x : (ax == 1 ? fq.y : fq.z), w);
      if (valid && l == 0) put(ax, w);
    }
  }
  __syncwarp();
  const bool act = valid;
  float wz[DM + 1];
  {
    const float4 t = *reinterpret_cast<const float4*>(tab + (2 * P + l) * 4);
    const float tz[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int c = 0; c <= DM; ++c) wz[c] = act ? tz[c] : 0.f;
  }
  float wy[P][DM + 1];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const float4 t = *reinterpret_cast<const float4*>(tab + (1 * P + j) * 4);
    const float ty[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int c = 0; c <= DM; ++c) wy[j][c] = ty[c];
  }
  const int Nx = g.N[0], Ny = g.N[1], Nz = g.N[2];
  int z = m.z + l;
  if (z >= Nz) z -= Nz;
  int yo[P];
#pragma unroll
  for (int jy = 0; jy < P; ++jy) {
    int y = m.y + jy;
    if (y >= Ny) y -= Ny;
    yo[jy] = y * Nz + z;
  }
  const int plane = Ny * Nz;
  const long long Mtot = (long long)Nx * plane;

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
      if (x >= Nx) x -= Nx;
      const int xo = x * plane;
      float r[DM + 1], rt[3];
#pragma unroll
      for (int b = 0; b <= DM; ++b) r[b] = 0.f;
#pragma unroll
      for (int b = 0; b < 3; ++b) rt[b] = 0.f;
#pragma unroll
      for (int jy = 0; jy < P; ++jy) {
        const int off = xo + yo[jy];
        const bool in_mesh = index_ok((long long)off, Mtot);
        const float v = in_mesh ? __ldg(phi_mesh + off) : 0.f;
#pragma unroll
        for (int b = 0; b <= DM; ++b) r[b] += v * wy[jy][b];
        if (TAN) {
          const float dv = in_mesh ? __ldg(dphi_mesh + off) : 0.f;
#pragma unroll
          for (int b = 0; b < 3; ++b) rt[b] += dv * wy[jy][b];
        }
      }
      const float4 t = *reinterpret_cast<const float4*>(tab + jx * 4);
      const float wxj[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int ia = 0; ia <= DM; ++ia)
#pragma unroll
        for (int ib = 0; ib <= DM; ++ib)
          if (ia + ib <= DM) S[ia][ib] += r[ib] * wxj[ia];
      if (TAN) {
#pragma unroll
        for (int ia = 0; ia < 3; ++ia)
#pragma unroll
          for (int ib = 0; ib < 3; ++ib)
            if (ia + ib <= 2) T[ia][ib] += rt[ib] * wxj[ia];
      }
    }
  }
  // moments M_abc, reduced over the group's z-lanes
#define MOM(ia, ib, ic) group_sum_p<P>(S[ia][ib] * wz[ic], l)
#define TMOM(ia, ib, ic) group_sum_p<P>(T[ia][ib] * wz[ic], l)
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
    if (a.finish) {
      // the backward's final assembly: mesh part + pair part, self and background terms,
      // coulomb_k
      const BackwardFinish& fn = a.fin;
      const int i = m.w;
      const float v[7] = {gr[0], gr[1], gr[2], gq, gm[0], gm[1], gm[2]};
      float w[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (fn.pair_out) {
#pragma unroll
        for (int c = 0; c < 7; ++c) w[c] = fn.pair_out[size_t(i) * 8 + c];
      }
      const float qi = fn.q[i];
      float mu_i[3] = {0.f, 0.f, 0.f}, dmu[3] = {0.f, 0.f, 0.f};
      if (fn.mu) {
#pragma unroll
        for (int c = 0; c < 3; ++c) mu_i[c] = fn.mu[3 * i + c];
      }
      if (fn.gfield) {
#pragma unroll
        for (int c = 0; c < 3; ++c) dmu[c] = -fn.gfield[3 * i + c];
      }
      const float dqi = fn.gphi ? fn.gphi[i] : 0.f;
      const float bg = fn.with_bg ? g.bg_fac : 0.f;
      const float Q = float(fn.qsum[2 * frame]), dQ = float(fn.qsum[2 * frame + 1]);
      const float k = fn.k;
      if (fn.grad_pos) {
#pragma unroll
        for (int c = 0; c < 3; ++c) fn.grad_pos[3 * i + c] = k * (v[c] + w[c]);
      }
      if (fn.grad_q) fn.grad_q[i] = k * (v[3] + w[3] - fn.self_phi * (gE * qi + dqi) - bg * (gE * Q + dQ));
      if (fn.grad_mu) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          fn.grad_mu[3 * i + c] = k * (v[4 + c] + w[4 + c] - fn.self_c * (gE * mu_i[c] + dmu[c]));
      }
    } else {
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
  }
#undef MOM
#undef TMOM
}

// Quadrupole Hessian-vector product, mesh part: for each ion the 13 gathered quantities of the
// quadrupole forward -- phi, grad phi, grad^2 phi and Theta_i : grad^3 phi -- and their
// directional derivatives along the ion's displacement dr and the tangent mesh d Phi (the
// potential of d rho): with t = D^T dr, M the moments of Phi and N those of d Phi (mesh
// coordinates),
//   d phi = N_0 + M_1 . t,  d grad phi = D (N_1 + M_2 t),  d grad^2 phi = D (N_2 + M_3[t]) D^T,
//   d (Theta : grad^3 phi) = D (Theta' : N_3 + Theta' : M_4[t]),  Theta' = D^T Theta D,
// which needs the moments of Phi up to order 4 and of d Phi up to order 3. Output
// out[caller index][26]: the 13 values, then their 13 tangents.
template <int P, bool BATCH>
__global__ void __launch_bounds__(kGatherThreads) k_gather_qdual(GatherArgs a) {
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
  float wx[5][P], wy[5][P], wzall[5][P];
  spline_weights<P, 4>(fq.x, wx);
  spline_weights<P, 4>(fq.y, wy);
  spline_weights<P, 4>(fq.z, wzall);
  const bool act = valid && (l < P);
  float wz[5];
#pragma unroll
  for (int c = 0; c <= 4; ++c) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) v = (j == l) ? wzall[c][j] : v;
    wz[c] = act ? v : 0.f;
  }
  int z = m.z + l;
  if (z >= g.N[2]) z -= g.N[2];
  const int Ny = g.N[1], Nz = g.N[2];
  const long long Mtot = (long long)g.N[0] * Ny * Nz;
  float S[5][5], T[4][4];   // S[a][b]: sum over (jx, jy) of Phi W_x^(a) W_y^(b), a + b <= 4
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) S[i][j] = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) T[i][j] = 0.f;
  if (act) {
#pragma unroll
    for (int jx = 0; jx < P; ++jx) {
      int x = m.x + jx;
      if (x >= g.N[0]) x -= g.N[0];
      float r[5], rt[4];
#pragma unroll
      for (int b = 0; b < 5; ++b) r[b] = 0.f;
#pragma unroll
      for (int b = 0; b < 4; ++b) rt[b] = 0.f;
#pragma unroll
      for (int jy = 0; jy < P; ++jy) {
        int y = m.y + jy;
        if (y >= Ny) y -= Ny;
        const size_t off = (size_t(x) * Ny + y) * Nz + z;
        const bool in_mesh = index_ok((long long)off, Mtot);
        const float v = in_mesh ? __ldg(phi_mesh + off) : 0.f;
        const float dv = in_mesh ? __ldg(dphi_mesh + off) : 0.f;
#pragma unroll
        for (int b = 0; b < 5; ++b) r[b] += v * wy[b][jy];
#pragma unroll
        for (int b = 0; b < 4; ++b) rt[b] += dv * wy[b][jy];
      }
#pragma unroll
      for (int ia = 0; ia < 5; ++ia)
#pragma unroll
        for (int ib = 0; ib < 5; ++ib)
          if (ia + ib <= 4) S[ia][ib] += r[ib] * wx[ia][jx];
#pragma unroll
      for (int ia = 0; ia < 4; ++ia)
#pragma unroll
        for (int ib = 0; ib < 4; ++ib)
          if (ia + ib <= 3) T[ia][ib] += rt[ib] * wx[ia][jx];
    }
  }
  // moments M[a][b][c] (a + b + c <= 4) and N[a][b][c] (<= 3), reduced over the z-lanes
  float M[5][5][5], N[4][4][4];
#pragma unroll
  for (int ia = 0; ia < 5; ++ia)
#pragma unroll
    for (int ib = 0; ib < 5; ++ib)
#pragma unroll
      for (int ic = 0; ic < 5; ++ic) M[ia][ib][ic] = (ia + ib + ic <= 4) ? group_sum(S[ia][ib] * wz[ic]) : 0.f;
#pragma unroll
  for (int ia = 0; ia < 4; ++ia)
#pragma unroll
    for (int ib = 0; ib < 4; ++ib)
#pragma unroll
      for (int ic = 0; ic < 4; ++ic) N[ia][ib][ic] = (ia + ib + ic <= 3) ? group_sum(T[ia][ib] * wz[ic]) : 0.f;
  if (!valid || l != 0) return;
  const float4 tt = a.mr.tt[ion];
  const float tv[3] = {tt.x, tt.y, tt.z};
  // Theta' = D^T Theta D
  const float* th = a.theta + size_t(m.w) * 6;
  const float Th[3][3] = {{th[0], th[3], th[4]}, {th[3], th[1], th[5]}, {th[4], th[5], th[2]}};
  float TD[3][3], Tp[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      TD[r][c] = Th[r][0] * g.D[0 * 3 + c] + Th[r][1] * g.D[1 * 3 + c] + Th[r][2] * g.D[2 * 3 + c];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Tp[r][c] = g.D[0 * 3 + r] * TD[0][c] + g.D[1 * 3 + r] * TD[1][c] + g.D[2 * 3 + r] * TD[2][c];
  // moment of a multi-index given as axis list: e1 = unit steps
  auto mom = [&](int i0, int i1, int i2) { return M[i0][i1][i2]; };
  auto nmom = [&](int i0, int i1, int i2) { return N[i0][i1][i2]; };
  (void)mom;
  (void)nmom;
  // first-, second-, third-order tensors in mesh coordinates
  const int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  float m1[3], n1[3], m2[3][3], n2[3][3], m2t[3], m3t[3][3], n3th[3], m4t[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    m1[i] = M[e[i][0]][e[i][1]][e[i][2]];
    n1[i] = N[e[i][0]][e[i][1]][e[i][2]];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      m2[i][j] = M[e[i][0] + e[j][0]][e[i][1] + e[j][1]][e[i][2] + e[j][2]];
      n2[i][j] = N[e[i][0] + e[j][0]][e[i][1] + e[j][1]][e[i][2] + e[j][2]];
    }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s2 += m2[i][j] * tv[j];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int a0 = e[i][0] + e[j][0] + e[k][0], a1 = e[i][1] + e[j][1] + e[k][1], a2 = e[i][2] + e[j][2] + e[k][2];
        // Theta'_jk N_jki and Theta'_jk sum_l M_jkil t_l
        s3 += Tp[j][k] * N[a0][a1][a2];
        float s = 0.f;
#pragma unroll
        for (int l2 = 0; l2 < 3; ++l2) s += M[a0 + e[l2][0]][a1 + e[l2][1]][a2 + e[l2][2]] * tv[l2];
        s4 += Tp[j][k] * s;
      }
    }
    m2t[i] = s2;
    n3th[i] = s3;
    m4t[i] = s4;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        s += M[e[i][0] + e[j][0] + e[k][0]][e[i][1] + e[j][1] + e[k][1]][e[i][2] + e[j][2] + e[k][2]] * tv[k];
      m3t[i][j] = s;
    }
  // Theta' : M_3 (the forward's third-order contraction)
  float v3[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        s += Tp[j][k] * M[e[i][0] + e[j][0] + e[k][0]][e[i][1] + e[j][1] + e[k][1]][e[i][2] + e[j][2] + e[k][2]];
    v3[i] = s;
  }
  // r-space: vectors D x, matrices D X D^T
  float gr[3], dgr[3], t3r[3], dt3r[3];
  {
    float a1[3], a2[3], a3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a1[i] = n1[i] + m2t[i];
      a2[i] = n3th[i] + m4t[i];
      a3[i] = m1[i];
    }
    apply_D(g.D, a3, gr);
    apply_D(g.D, a1, dgr);
    apply_D(g.D, v3, t3r);
    apply_D(g.D, a2, dt3r);
  }
  float Hr[3][3], dHr[3][3];
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    float X[3][3], XD[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) X[i][j] = pass == 0 ? m2[i][j] : n2[i][j] + m3t[i][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int b = 0; b < 3; ++b) XD[i][b] = X[i][0] * g.D[b * 3 + 0] + X[i][1] * g.D[b * 3 + 1] + X[i][2] * g.D[b * 3 + 2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float v = g.D[i * 3 + 0] * XD[0][b] + g.D[i * 3 + 1] * XD[1][b] + g.D[i * 3 + 2] * XD[2][b];
        if (pass == 0) Hr[i][b] = v;
        else dHr[i][b] = v;
      }
  }
  const float dphi = N[0][0][0] + m1[0] * tv[0] + m1[1] * tv[1] + m1[2] * tv[2];
  float* o = a.out + size_t(m.w) * 26;
  const float vals[26] = {M[0][0][0], gr[0], gr[1], gr[2], Hr[0][0], Hr[1][1], Hr[2][2], Hr[0][1], Hr[0][2], Hr[1][2],
                          t3r[0], t3r[1], t3r[2],
                          dphi, dgr[0], dgr[1], dgr[2], dHr[0][0], dHr[1][1], dHr[2][2], dHr[0][1], dHr[0][2],
                          dHr[1][2], dt3r[0], dt3r[1], dt3r[2]};
#pragma unroll
  for (int k = 0; k < 26; ++k) o[k] = vals[k];
}

template <int MODE, bool BATCH>
int launch_t(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const double* g_energy,
             float* out, const float* theta = nullptr, float* qout = nullptr,
             const BackwardFinish* fin = nullptr) {
  GatherArgs a;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.mr = p->mr;
  a.mesh = mesh;
  a.g_energy = g_energy;
  a.out = out;
  a.theta = theta;
  a.qout = qout;
  a.finish = fin ? 1 : 0;
  a.fin = fin ? *fin : BackwardFinish{};
  for (int gi = 0; gi < p->nogroups; ++gi) {
    const OrderGroup& G = p->ogroups[gi];
    a.t_lo = BATCH ? G.sorted_lo : 0;
    a.t_hi = BATCH ? G.sorted_hi : n;
    const size_t nion = size_t(a.t_hi - a.t_lo);
    if (nion == 0) continue;
    // blocks of kGatherThreads / 32 warps, gather_ions_per_warp<P>() ions per warp
#define GBPME_GATHER(PP)                                                                        \
  case PP: {                                                                                    \
    const size_t per_block = size_t(kGatherThreads / 32) * gather_ions_per_warp<PP>();          \
    const int grid = int((nion + per_block - 1) / per_block);                                   \
    pdl_launch(k_gather<PP, MODE, BATCH>, grid, kGatherThreads, 0, s, a);                               \
    break;                                                                                      \
  }
    switch (G.order) {
      GBPME_GATHER(1)
      GBPME_GATHER(2)
      GBPME_GATHER(3)
      GBPME_GATHER(4)
      GBPME_GATHER(5)
      GBPME_GATHER(6)
      GBPME_GATHER(7)
      default: return set_error(p, PME_ERR_ARG, "spline order out of range");
    }
#undef GBPME_GATHER
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

int launch_gather_finish(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const double* g_energy,
                         const BackwardFinish& fin) {
  if (p->batch) return launch_t<1, true>(p, s, n, mesh, g_energy, nullptr, nullptr, nullptr, &fin);
  return launch_t<1, false>(p, s, n, mesh, g_energy, nullptr, nullptr, nullptr, &fin);
}

int launch_gather_quad(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const float* theta,
                       float* out, float* qout) {
  if (p->batch) return launch_t<2, true>(p, s, n, mesh, nullptr, out, theta, qout);
  return launch_t<2, false>(p, s, n, mesh, nullptr, out, theta, qout);
}

int launch_gather_qdual(pme_plan_t p, cudaStream_t s, int n, const float* mesh, const float* theta, float* out) {
  GatherArgs a;
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.mr = p->mr;
  a.mesh = mesh;
  a.g_energy = nullptr;
  a.out = out;
  a.theta = theta;
  a.qout = nullptr;
  a.finish = 0;
  a.fin = BackwardFinish{};
  for (int gi = 0; gi < p->nogroups; ++gi) {
    const OrderGroup& G = p->ogroups[gi];
    a.t_lo = p->batch ? G.sorted_lo : 0;
    a.t_hi = p->batch ? G.sorted_hi : n;
    const int grid = int((size_t(a.t_hi - a.t_lo) * kGroup + kGatherThreads - 1) / kGatherThreads);
    if (grid <= 0) continue;
#define GBPME_QDUAL(PP)                                                                   \
  case PP:                                                                                \
    if (p->batch) k_gather_qdual<PP, true><<<grid, kGatherThreads, 0, s>>>(a);            \
    else k_gather_qdual<PP, false><<<grid, kGatherThreads, 0, s>>>(a);                    \
    break;
    switch (G.order) {
      GBPME_QDUAL(4)
      GBPME_QDUAL(5)
      GBPME_QDUAL(6)
      GBPME_QDUAL(7)
      default: return set_error(p, PME_ERR_UNSUPPORTED, "quadrupole backward: spline order below 4");
    }
#undef GBPME_QDUAL
    count_launch();
    const int st = check_launch(p, "k_gather_qdual");
    if (st) return st;
  }
  return PME_OK;
}

GBPME_BOUNDS_READER(bounds_hit_gather)

}  // namespace gbpme
