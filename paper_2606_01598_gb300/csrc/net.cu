// The learned charge/dipole network and its force-matching training step (gbnet.h).
//
// Sections 2.1-2.2 of the paper: latent charges from the scalar features (Eq. charge_pred),
// dipoles from the vector features (Eq. dipole_pred) and site energies (Eq. site_energy) of a
// Cartesian-tensor message-passing net; Section 2.4: the model energy E_sr + E_PME, forces
// by differentiation through every path (Eq. forces) and the loss of Eq. loss, whose
// parameter gradient needs the derivative of the forces (a second derivative of E).
//
// Differentiation. Every kernel is written once over a scalar type T: float for a plain
// pass, Dual (value + tangent) for a pass that also carries the directional derivative
// along a position tangent r' (forward mode). Running the reverse pass (the backward
// kernels) in Dual arithmetic gives d/de [dE/dtheta (r + e r')], i.e. forward-over-reverse.
// The gradient of the force term of Eq. loss is exactly that with r' = -w,
// w = 2 lambda_f / (3 sum N) (F - F_ref); seeding the energy cotangent as 1 + e c_b,
// c_b = 2 lambda_e (E_b - E_ref,b) / (F N_b^2), adds the energy term, so the tangent part of
// one Dual backward is dL/dtheta. The PME's part of that tangent is its Hessian-vector
// product, which pme_batch_backward evaluates.
//
// Layout: every activation buffer holds two planes, [value][rows][C] then [tangent][rows][C];
// a Dual pass reads and writes both, a plain pass the first. The tensor-core products
// (net_mix.cu) treat the two planes as one matrix of 2 rows x C rows, since the tangent of
// X W is X' W. Per-ion work is one warp per ion with lane = channel; edges come from
// per-ion neighbour lists (symmetric, so the reverse-mode scatter onto senders is done as a
// gather over the receiver's own list); parameter gradients are reduced over fixed
// per-block partials (deterministic, no atomics).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dual.cuh"
#include "net.cuh"

namespace gbnet {

using gbpme::Dual;
using gbpme::rcpT;
using gbpme::sqrtT;
using gbpme::sincosT;
using gbpme::sigmoidT;
using gbpme::siluT;
using gbpme::dsiluT;
using gbpme::shfl_xor;
using gbpme::warp_sum;

namespace {

constexpr int S = GBNET_SCALARS, V = GBNET_VECTORS, NR = GBNET_RADIAL;
constexpr int kMaxNbr = GBNET_MAX_NEIGHBOURS;
constexpr float kRc = float(GBNET_CUTOFF);
constexpr float kInvAvg = 1.0f / 16.0f;    // message normalisation: mean neighbour count
constexpr int kWarps = 8;                  // warps per block of the per-ion kernels
constexpr int NCOL = S + 3 * V;            // radial weight columns: ss 32, sv 16, vs 16, vv 16

// parameter offsets (floats) of the layout documented in gbnet.h
constexpr int kLayerSize = S * (S + V) + V * 2 * V + NR * NCOL + (S + V) * (S + V) + 2 * V * V;
constexpr int oEmb = 0;
constexpr int oLayer0 = 2 * S;
constexpr int oWA = 0, oWB = oWA + S * (S + V), oWR = oWB + V * 2 * V, oWU = oWR + NR * NCOL,
              oWY = oWU + (S + V) * (S + V);
constexpr int oWh = oLayer0 + 2 * kLayerSize;
constexpr int oBh = oWh + S * 2 * S;
constexpr int oWq = oBh + 2 * S;
constexpr int oBq = oWq + S;
constexpr int oWE = oBq + 1;
constexpr int oBE = oWE + S;
constexpr int oWmu = oBE + 1;
constexpr int kParams = oWmu + V;
static_assert(kParams == GBNET_NUM_PARAMS, "parameter layout");
constexpr int kReadoutW = S + S + 2 * S + 1 + 1 + V;   // wq, wE, bh, bq, bE, wmu partials

// the nine channel-mixing matrices (param offset, K = fan-in, N = fan-out)
struct MixW {
  int off, K, N;
};
constexpr int kNumMix = 9;
__host__ __device__ constexpr MixW mix_w(int w) {
  return w == 8 ? MixW{oWh, S, 2 * S}
                : (w % 4 == 0 ? MixW{oLayer0 + (w / 4) * kLayerSize + oWA, S, S + V}
                   : w % 4 == 1 ? MixW{oLayer0 + (w / 4) * kLayerSize + oWB, V, 2 * V}
                   : w % 4 == 2 ? MixW{oLayer0 + (w / 4) * kLayerSize + oWU, S + V, S + V}
                                : MixW{oLayer0 + (w / 4) * kLayerSize + oWY, 2 * V, V});
}

template <typename T> __device__ __forceinline__ T mk(float v, float d);
template <> __device__ __forceinline__ float mk<float>(float v, float) { return v; }
template <> __device__ __forceinline__ Dual mk<Dual>(float v, float d) { return Dual(v, d); }
__device__ __forceinline__ float val(float x) { return x; }
__device__ __forceinline__ float val(Dual x) { return x.v; }
__device__ __forceinline__ float tan_(float) { return 0.f; }
__device__ __forceinline__ float tan_(Dual x) { return x.d; }

// two-plane loads and stores: plane = floats per plane
__device__ __forceinline__ void ldv(const float* p, size_t i, size_t, float& o) { o = p[i]; }
__device__ __forceinline__ void ldv(const float* p, size_t i, size_t pl, Dual& o) { o = Dual(p[i], p[i + pl]); }
template <typename T> __device__ __forceinline__ T ldT(const float* p, size_t i, size_t pl) {
  T x;
  ldv(p, i, pl, x);
  return x;
}
__device__ __forceinline__ void stT(float* p, size_t i, size_t, float v) { p[i] = v; }
__device__ __forceinline__ void stT(float* p, size_t i, size_t pl, Dual v) { p[i] = v.v; p[i + pl] = v.d; }
// positions: value array and (Dual) tangent array
__device__ __forceinline__ void ldpos(const float* p, const float*, size_t i, float& o) { o = p[i]; }
__device__ __forceinline__ void ldpos(const float* p, const float* dp, size_t i, Dual& o) { o = Dual(p[i], dp[i]); }

template <typename T> struct Vec3 { T x, y, z; };
template <typename T> __device__ __forceinline__ T dot3(const Vec3<T>& a, const Vec3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// ---------------------------------------------------------------------------------------
// frames and neighbour lists
// ---------------------------------------------------------------------------------------
struct NetFrame {
  int off, n;
  float C[9];     // rows = lattice vectors
  float Ci[9];    // C^{-1}
  int ortho;      // orthorhombic box: the rounded fractional difference is the nearest image
};

struct Nbr {
  const int* cnt;     // [n]
  const int* j;       // [n][kMaxNbr]
  const float4* sh;   // [n][kMaxNbr]: lattice shift of the image (d = r_j - r_i + sh)
};

// One warp per ion: every other ion of the frame within r_c (nearest image), compacted in
// increasing j order.
__global__ void k_nbr(const NetFrame* __restrict__ frames, const int* __restrict__ frame_of,
                      const float* __restrict__ pos, int n, int* cnt, int* nj, float4* nsh, int* flags) {
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  const NetFrame F = frames[frame_of[i]];
  const float xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
  if (!(isfinite(xi) && isfinite(yi) && isfinite(zi)) && lane == 0) atomicOr(flags, kNetFlagNonFinite);
  const float rc2 = kRc * kRc;
  int c = 0;
  for (int j0 = F.off; j0 < F.off + F.n; j0 += 32) {
    const int j = j0 + lane;
    bool hit = false;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (j < F.off + F.n && j != i) {
      const float dx = pos[3 * j] - xi, dy = pos[3 * j + 1] - yi, dz = pos[3 * j + 2] - zi;
      // fractional difference, wrapped to the nearest cell
      const float fa = rintf(dx * F.Ci[0] + dy * F.Ci[3] + dz * F.Ci[6]);
      const float fb = rintf(dx * F.Ci[1] + dy * F.Ci[4] + dz * F.Ci[7]);
      const float fc = rintf(dx * F.Ci[2] + dy * F.Ci[5] + dz * F.Ci[8]);
      const int rng = F.ortho ? 0 : 1;
      for (int a = -rng; a <= rng && !hit; ++a)
        for (int b = -rng; b <= rng && !hit; ++b)
          for (int cc = -rng; cc <= rng && !hit; ++cc) {
            const float na = -fa + a, nb = -fb + b, nc = -fc + cc;
            const float tx = na * F.C[0] + nb * F.C[3] + nc * F.C[6];
            const float ty = na * F.C[1] + nb * F.C[4] + nc * F.C[7];
            const float tz = na * F.C[2] + nb * F.C[5] + nc * F.C[8];
            const float ex = dx + tx, ey = dy + ty, ez = dz + tz;
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rc2 && r2 > 0.f) {
              hit = true;
              sx = tx; sy = ty; sz = tz;
            }
          }
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int slot = c + __popc(m & ((1u << lane) - 1u));
    if (hit && slot < kMaxNbr) {
      nj[size_t(i) * kMaxNbr + slot] = j;
      nsh[size_t(i) * kMaxNbr + slot] = make_float4(sx, sy, sz, 0.f);
    }
    c += __popc(m);
  }
  if (lane == 0) {
    if (c > kMaxNbr) atomicOr(flags, kNetFlagNbrFull);
    cnt[i] = min(c, kMaxNbr);
  }
}

// Edge geometry along one neighbour: d, r, d^, the basis e_k and de_k/dr (k = 1..8).
template <typename T>
__device__ __forceinline__ void edge_basis(const Vec3<T>& d, T& r, Vec3<T>& dh, T (&e)[NR], T (&de)[NR]) {
  const T r2 = dot3(d, d);
  r = sqrtT(r2);
  const T ri = rcpT(r);
  dh = Vec3<T>{d.x * ri, d.y * ri, d.z * ri};
  const float w = float(gbpme::kPi) / kRc;
  T s1, c1;
  sincosT(r * w, s1, c1);
  // envelope u(x) = 1 - 21 x^5 + 35 x^6 - 15 x^7 and u'(x)
  const T x = r * (1.f / kRc);
  const T x2 = x * x, x4 = x2 * x2;
  const T u = 1.f + x4 * x * (-21.f + x * (35.f - 15.f * x));
  const T du = x4 * (-105.f + x * (210.f - 105.f * x)) * (1.f / kRc);
  const float nrm = sqrtf(2.f / kRc);
  // sin(k w r) and cos(k w r) by the angle-addition recurrence
  T sk = s1, ck = c1;
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    const float kw = float(k + 1) * w;
    const T a = nrm * sk * ri;                               // sqrt(2/rc) sin(k w r) / r
    const T da = nrm * (kw * ck * ri - sk * ri * ri);        // its r-derivative
    e[k] = a * u;
    de[k] = da * u + a * du;
    const T sn = sk * c1 + ck * s1, cn = ck * c1 - sk * s1;
    sk = sn;
    ck = cn;
  }
}

struct MsgArgs {
  const NetFrame* frames;
  const int* frame_of;
  Nbr nb;
  const float* pos;    // [n][3]
  const float* dpos;   // [n][3] tangent (Dual passes)
  const float* WR;     // [8][80] of this layer (float32 master)
  int n;
  size_t plS, plV;     // plane sizes: n * 48 (scalar-shaped 48) and n * 96 (vector-shaped 3 x 32)
};

// Messages of one layer: ms [n][48], mv [n][3][32] from A [n][48], B [n][3][32].
template <typename T>
__global__ void __launch_bounds__(32 * kWarps) k_msg_fwd(MsgArgs a, const float* __restrict__ A,
                                                       const float* __restrict__ B, float* ms, float* mv) {
  __shared__ float sW[NR * NCOL];
  for (int k = threadIdx.x; k < NR * NCOL; k += blockDim.x) sW[k] = a.WR[k];
  __syncthreads();
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5), c = threadIdx.x & 31;
  if (i >= a.n) return;
  const bool lo = c < V;
  Vec3<T> ri;
  ldpos(a.pos, a.dpos, 3 * i, ri.x);
  ldpos(a.pos, a.dpos, 3 * i + 1, ri.y);
  ldpos(a.pos, a.dpos, 3 * i + 2, ri.z);
  T acc_s = 0.f, acc_s2 = 0.f;
  Vec3<T> acc_v{T(0.f), T(0.f), T(0.f)};
  const int ne = a.nb.cnt[i];
  for (int q = 0; q < ne; ++q) {
    const int j = a.nb.j[size_t(i) * kMaxNbr + q];
    const float4 sh = a.nb.sh[size_t(i) * kMaxNbr + q];
    Vec3<T> rj;
    ldpos(a.pos, a.dpos, 3 * j, rj.x);
    ldpos(a.pos, a.dpos, 3 * j + 1, rj.y);
    ldpos(a.pos, a.dpos, 3 * j + 2, rj.z);
    const Vec3<T> d{rj.x - ri.x + sh.x, rj.y - ri.y + sh.y, rj.z - ri.z + sh.z};
    T r, e[NR], de[NR];
    Vec3<T> dh;
    edge_basis(d, r, dh, e, de);
    T Rss = 0.f, R2 = 0.f, R3 = 0.f;   // lo lanes: R_ss, R_sv, R_vs;  hi lanes: R_ss, R_vv
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      Rss += e[k] * sW[k * NCOL + c];
      if (lo) {
        R2 += e[k] * sW[k * NCOL + S + c];
        R3 += e[k] * sW[k * NCOL + S + V + c];
      } else {
        R2 += e[k] * sW[k * NCOL + S + 2 * V + (c - V)];
      }
    }
    acc_s += Rss * ldT<T>(A, size_t(j) * (S + V) + c, a.plS);
    const Vec3<T> Bj{ldT<T>(B, (size_t(j) * 3 + 0) * 2 * V + c, a.plV), ldT<T>(B, (size_t(j) * 3 + 1) * 2 * V + c, a.plV),
                     ldT<T>(B, (size_t(j) * 3 + 2) * 2 * V + c, a.plV)};
    if (lo) {
      acc_s2 += R2 * dot3(dh, Bj);
      const T t = R3 * ldT<T>(A, size_t(j) * (S + V) + S + c, a.plS);
      acc_v.x += t * dh.x;
      acc_v.y += t * dh.y;
      acc_v.z += t * dh.z;
    } else {
      acc_v.x += R2 * Bj.x;
      acc_v.y += R2 * Bj.y;
      acc_v.z += R2 * Bj.z;
    }
  }
  stT(ms, size_t(i) * (S + V) + c, a.plS, acc_s * kInvAvg);
  if (lo) stT(ms, size_t(i) * (S + V) + S + c, a.plS, acc_s2 * kInvAvg);
  stT(mv, (size_t(i) * 3 + 0) * 2 * V + c, a.plV, acc_v.x * kInvAvg);
  stT(mv, (size_t(i) * 3 + 1) * 2 * V + c, a.plV, acc_v.y * kInvAvg);
  stT(mv, (size_t(i) * 3 + 2) * 2 * V + c, a.plV, acc_v.z * kInvAvg);
}

// Reverse pass of the messages. Inputs: the layer's A, B and the cotangents g_ms [n][48],
// g_mv [n][3][32] of its messages. Outputs: g_A [n][48], g_B [n][3][32] (written),
// g_pos [n][3] (added), and per-block partials of dL/dWR [8][80] (two planes for Dual).
template <typename T>
__global__ void __launch_bounds__(32 * kWarps) k_msg_bwd(MsgArgs a, const float* __restrict__ A,
                                                       const float* __restrict__ B, const float* __restrict__ gms,
                                                       const float* __restrict__ gmv, float* gA_out, float* gB_out,
                                                       float* gpos, float* wr_part) {
  __shared__ float sW[NR * NCOL];
  __shared__ float sG[kWarps][2][NR * NCOL];
  for (int k = threadIdx.x; k < NR * NCOL; k += blockDim.x) sW[k] = a.WR[k];
  __syncthreads();
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + w;
  const bool lo = c < V;
  // per-lane partials of dL/dWR for this lane's columns: cols c, and (lo) S + c, S + V + c,
  // (hi) S + 2V + c - V
  T gw0[NR], gw1[NR], gw2[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) gw0[k] = gw1[k] = gw2[k] = 0.f;
  if (i < a.n) {
    Vec3<T> ri;
    ldpos(a.pos, a.dpos, 3 * i, ri.x);
    ldpos(a.pos, a.dpos, 3 * i + 1, ri.y);
    ldpos(a.pos, a.dpos, 3 * i + 2, ri.z);
    const size_t iS = size_t(i) * (S + V);
    const T Gs_i = ldT<T>(gms, iS + c, a.plS) * kInvAvg;
    const T Gs2_i = lo ? ldT<T>(gms, iS + S + c, a.plS) * kInvAvg : T(0.f);
    const Vec3<T> Gv_i{ldT<T>(gmv, (size_t(i) * 3 + 0) * 2 * V + c, a.plV) * kInvAvg,
                       ldT<T>(gmv, (size_t(i) * 3 + 1) * 2 * V + c, a.plV) * kInvAvg,
                       ldT<T>(gmv, (size_t(i) * 3 + 2) * 2 * V + c, a.plV) * kInvAvg};
    const T A_i = ldT<T>(A, iS + c, a.plS);
    const T A2_i = lo ? ldT<T>(A, iS + S + c, a.plS) : T(0.f);
    const Vec3<T> B_i{ldT<T>(B, (size_t(i) * 3 + 0) * 2 * V + c, a.plV), ldT<T>(B, (size_t(i) * 3 + 1) * 2 * V + c, a.plV),
                      ldT<T>(B, (size_t(i) * 3 + 2) * 2 * V + c, a.plV)};
    T gA = 0.f, gA2 = 0.f;
    Vec3<T> gBv{T(0.f), T(0.f), T(0.f)}, gp{T(0.f), T(0.f), T(0.f)};
    const int ne = a.nb.cnt[i];
    for (int q = 0; q < ne; ++q) {
      const int j = a.nb.j[size_t(i) * kMaxNbr + q];
      const float4 sh = a.nb.sh[size_t(i) * kMaxNbr + q];
      Vec3<T> rj;
      ldpos(a.pos, a.dpos, 3 * j, rj.x);
      ldpos(a.pos, a.dpos, 3 * j + 1, rj.y);
      ldpos(a.pos, a.dpos, 3 * j + 2, rj.z);
      const Vec3<T> d{rj.x - ri.x + sh.x, rj.y - ri.y + sh.y, rj.z - ri.z + sh.z};
      T r, e[NR], de[NR];
      Vec3<T> dh;
      edge_basis(d, r, dh, e, de);
      const T rinv = rcpT(r);
      T R0 = 0.f, R1 = 0.f, R2 = 0.f, dR0 = 0.f, dR1 = 0.f, dR2 = 0.f;
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const float w0 = sW[k * NCOL + c];
        R0 += e[k] * w0;
        dR0 += de[k] * w0;
        if (lo) {
          const float w1 = sW[k * NCOL + S + c], w2 = sW[k * NCOL + S + V + c];
          R1 += e[k] * w1;
          dR1 += de[k] * w1;
          R2 += e[k] * w2;
          dR2 += de[k] * w2;
        } else {
          const float w1 = sW[k * NCOL + S + 2 * V + (c - V)];
          R1 += e[k] * w1;
          dR1 += de[k] * w1;
        }
      }
      // neighbour's data
      const size_t jS = size_t(j) * (S + V);
      const T A_j = ldT<T>(A, jS + c, a.plS);
      const Vec3<T> B_j{ldT<T>(B, (size_t(j) * 3 + 0) * 2 * V + c, a.plV), ldT<T>(B, (size_t(j) * 3 + 1) * 2 * V + c, a.plV),
                        ldT<T>(B, (size_t(j) * 3 + 2) * 2 * V + c, a.plV)};
      const T Gs_j = ldT<T>(gms, jS + c, a.plS) * kInvAvg;
      const Vec3<T> Gv_j{ldT<T>(gmv, (size_t(j) * 3 + 0) * 2 * V + c, a.plV) * kInvAvg,
                         ldT<T>(gmv, (size_t(j) * 3 + 1) * 2 * V + c, a.plV) * kInvAvg,
                         ldT<T>(gmv, (size_t(j) * 3 + 2) * 2 * V + c, a.plV) * kInvAvg};
      // --- forward direction: receiver i, sender j (d) ---
      // scalar-type terms: Phi += R s, dPhi/dd = R' s d^; vector-type terms: Phi += R (d^.t),
      // dPhi/dd = R' (d^.t) d^ + R (t - (d^.t) d^) / r
      T sc = 0.f, vcoef = 0.f;            // sum R' s + sum R' (d^.t) ; and the t-terms below
      Vec3<T> tv{T(0.f), T(0.f), T(0.f)}; // sum R t / r
      T dtv = 0.f;                        // sum R (d^.t) / r
      {
        const T s0 = Gs_i * A_j;          // ss
        sc += dR0 * s0;
#pragma unroll
        for (int k = 0; k < NR; ++k) gw0[k] += e[k] * s0;
        if (lo) {
          const T g2 = Gs2_i;
          const Vec3<T> t1{g2 * B_j.x, g2 * B_j.y, g2 * B_j.z};    // sv
          const T p1 = dot3(dh, t1);
          const T A2_j = ldT<T>(A, jS + S + c, a.plS);
          const Vec3<T> t2{A2_j * Gv_i.x, A2_j * Gv_i.y, A2_j * Gv_i.z};   // vs
          const T p2 = dot3(dh, t2);
          vcoef += dR1 * p1 + dR2 * p2;
          const T f1 = R1 * rinv, f2 = R2 * rinv;
          tv.x += f1 * t1.x + f2 * t2.x;
          tv.y += f1 * t1.y + f2 * t2.y;
          tv.z += f1 * t1.z + f2 * t2.z;
          dtv += f1 * p1 + f2 * p2;
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            gw1[k] += e[k] * p1;
            gw2[k] += e[k] * p2;
          }
        } else {
          const T s1 = dot3(Gv_i, B_j);   // vv
          sc += dR1 * s1;
#pragma unroll
          for (int k = 0; k < NR; ++k) gw1[k] += e[k] * s1;
        }
      }
      const T radial = sc + vcoef - dtv;
      // V_ij = radial d^ + tv ; g_pos_i -= V_ij
      gp.x -= radial * dh.x + tv.x;
      gp.y -= radial * dh.y + tv.y;
      gp.z -= radial * dh.z + tv.z;
      // --- reverse direction: receiver j, sender i (d' = -d, d^' = -d^) ---
      gA += R0 * Gs_j;
      T sc2 = dR0 * (Gs_j * A_i), vcoef2 = 0.f, dtv2 = 0.f;
      Vec3<T> tv2{T(0.f), T(0.f), T(0.f)};
      if (lo) {
        const T Gs2_j = ldT<T>(gms, jS + S + c, a.plS) * kInvAvg;
        // g_A_i[32+c] += R_vs (d^' . Gv_j),  g_B_i[:,c] += R_sv d^' Gs_j[32+c]
        gA2 -= R2 * dot3(dh, Gv_j);
        gBv.x -= R1 * Gs2_j * dh.x;
        gBv.y -= R1 * Gs2_j * dh.y;
        gBv.z -= R1 * Gs2_j * dh.z;
        const Vec3<T> t1{Gs2_j * B_i.x, Gs2_j * B_i.y, Gs2_j * B_i.z};
        const Vec3<T> t2{A2_i * Gv_j.x, A2_i * Gv_j.y, A2_i * Gv_j.z};
        const T p1 = -dot3(dh, t1), p2 = -dot3(dh, t2);        // d^' . t
        vcoef2 += dR1 * p1 + dR2 * p2;
        const T f1 = R1 * rinv, f2 = R2 * rinv;
        tv2.x += f1 * t1.x + f2 * t2.x;
        tv2.y += f1 * t1.y + f2 * t2.y;
        tv2.z += f1 * t1.z + f2 * t2.z;
        dtv2 += f1 * p1 + f2 * p2;
      } else {
        gBv.x += R1 * Gv_j.x;
        gBv.y += R1 * Gv_j.y;
        gBv.z += R1 * Gv_j.z;
        sc2 += dR1 * dot3(Gv_j, B_i);
      }
      // V_ji = radial' d^' + tv2 ; g_pos_i += V_ji
      const T radial2 = sc2 + vcoef2 - dtv2;
      gp.x += tv2.x - radial2 * dh.x;
      gp.y += tv2.y - radial2 * dh.y;
      gp.z += tv2.z - radial2 * dh.z;
    }
    stT(gA_out, iS + c, a.plS, gA);
    if (lo) stT(gA_out, iS + S + c, a.plS, gA2);
    stT(gB_out, (size_t(i) * 3 + 0) * 2 * V + c, a.plV, gBv.x);
    stT(gB_out, (size_t(i) * 3 + 1) * 2 * V + c, a.plV, gBv.y);
    stT(gB_out, (size_t(i) * 3 + 2) * 2 * V + c, a.plV, gBv.z);
    gp.x = warp_sum(gp.x);
    gp.y = warp_sum(gp.y);
    gp.z = warp_sum(gp.z);
    if (c == 0) {
      const size_t pl = size_t(a.n) * 3;
      stT(gpos, 3 * size_t(i), pl, ldT<T>(gpos, 3 * size_t(i), pl) + gp.x);
      stT(gpos, 3 * size_t(i) + 1, pl, ldT<T>(gpos, 3 * size_t(i) + 1, pl) + gp.y);
      stT(gpos, 3 * size_t(i) + 2, pl, ldT<T>(gpos, 3 * size_t(i) + 2, pl) + gp.z);
    }
  }
  // block partials of dL/dWR: [block][plane][NR][NCOL]
  const int col1 = lo ? S + c : S + 2 * V + (c - V);
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    sG[w][0][k * NCOL + c] = val(gw0[k]);
    sG[w][1][k * NCOL + c] = tan_(gw0[k]);
    sG[w][0][k * NCOL + col1] = val(gw1[k]);
    sG[w][1][k * NCOL + col1] = tan_(gw1[k]);
    if (lo) {
      sG[w][0][k * NCOL + S + V + c] = val(gw2[k]);
      sG[w][1][k * NCOL + S + V + c] = tan_(gw2[k]);
    }
  }
  __syncthreads();
  constexpr int kPlanes = sizeof(T) / sizeof(float);
  for (int t = threadIdx.x; t < kPlanes * NR * NCOL; t += blockDim.x) {
    const int pl = t / (NR * NCOL), k = t % (NR * NCOL);
    float acc = 0.f;
    for (int ww = 0; ww < kWarps; ++ww) acc += sG[ww][pl][k];
    wr_part[(size_t(blockIdx.x) * kPlanes + pl) * NR * NCOL + k] = acc;
  }
}

// ---------------------------------------------------------------------------------------
// per-ion elementwise stages
// ---------------------------------------------------------------------------------------

// h^s = emb[species]; h^v = 0 (both planes: the embedding has no position tangent)
__global__ void k_embed(const float* __restrict__ P, const int* __restrict__ species, int n, float* hs, float* hv,
                        size_t plS, size_t plV, int planes) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < size_t(n) * S) {
    const int i = int(t / S), c = int(t % S);
    hs[t] = P[oEmb + species[i] * S + c];
    if (planes > 1) hs[t + plS] = 0.f;
  }
  if (t < size_t(n) * 3 * V) {
    hv[t] = 0.f;
    if (planes > 1) hv[t + plV] = 0.f;
  }
}

// h^s_out = h^s_in + SiLU(U[:, :32]);  h^v_out = h^v_in + sigmoid(U[:, 32:]) * Y.
// One thread per (ion, scalar channel); the first 16 also do the vector channel.
template <typename T>
__global__ void k_update_fwd(int n, const float* __restrict__ U, const float* __restrict__ Y,
                             const float* __restrict__ hs_in, const float* __restrict__ hv_in, float* hs_out,
                             float* hv_out, size_t plU, size_t plY, size_t plS, size_t plV) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= size_t(n) * S) return;
  const size_t i = t / S;
  const int c = int(t % S);
  stT(hs_out, t, plS, ldT<T>(hs_in, t, plS) + siluT(ldT<T>(U, i * (S + V) + c, plU)));
  if (c < V) {
    const T g = sigmoidT(ldT<T>(U, i * (S + V) + S + c, plU));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t k = (i * 3 + a) * V + c;
      stT(hv_out, k, plV, ldT<T>(hv_in, k, plV) + g * ldT<T>(Y, k, plY));
    }
  }
}

// Reverse of k_update_fwd: g_U [n][48], g_Y [n][3][16] from the output cotangents g_hs, g_hv
// (which also pass unchanged to the layer input through the residual).
template <typename T>
__global__ void k_update_bwd(int n, const float* __restrict__ U, const float* __restrict__ Y,
                             const float* __restrict__ ghs, const float* __restrict__ ghv, float* gU, float* gY,
                             size_t plU, size_t plY, size_t plS, size_t plV) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= size_t(n) * S) return;
  const size_t i = t / S;
  const int c = int(t % S);
  stT(gU, i * (S + V) + c, plU, ldT<T>(ghs, t, plS) * dsiluT(ldT<T>(U, i * (S + V) + c, plU)));
  if (c < V) {
    const T g = sigmoidT(ldT<T>(U, i * (S + V) + S + c, plU));
    T acc = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t k = (i * 3 + a) * V + c;
      const T gh = ldT<T>(ghv, k, plV);
      acc += gh * ldT<T>(Y, k, plY);
      stT(gY, k, plY, gh * g);
    }
    stT(gU, i * (S + V) + S + c, plU, acc * (g * (1.f - g)));
  }
}

// Readouts of one warp per ion: q~ (before neutralisation), site energy, dipole.
template <typename T>
__global__ void k_readout_fwd(int n, const float* __restrict__ P, const float* __restrict__ H,
                              const float* __restrict__ hv, float* qt, float* ei, float* mu, size_t plH,
                              size_t plV, size_t pln) {
  const int i = blockIdx.x * kWarps + (threadIdx.x >> 5), c = threadIdx.x & 31;
  if (i >= n) return;
  const T hq = ldT<T>(H, size_t(i) * 2 * S + c, plH) + P[oBh + c];
  const T he = ldT<T>(H, size_t(i) * 2 * S + S + c, plH) + P[oBh + S + c];
  T sq = P[oWq + c] * siluT(hq);
  T se = P[oWE + c] * siluT(he);
  T m[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) m[a] = c < V ? ldT<T>(hv, (size_t(i) * 3 + a) * V + c, plV) * P[oWmu + c] : T(0.f);
  sq = warp_sum(sq);
  se = warp_sum(se);
#pragma unroll
  for (int a = 0; a < 3; ++a) m[a] = warp_sum(m[a]);
  if (c == 0) {
    stT(qt, i, pln, sq + P[oBq]);
    stT(ei, i, pln, se + P[oBE]);
#pragma unroll
    for (int a = 0; a < 3; ++a) stT(mu, 3 * size_t(i) + a, 3 * pln, m[a]);
  }
}

// One block per frame: q = q~ - mean(q~) (both planes for Dual) and E_sr = sum of site
// energies (float64, value only).
template <typename T>
__global__ void k_frame_fwd(const NetFrame* __restrict__ frames, const float* __restrict__ qt,
                            const float* __restrict__ ei, float* q, double* esr, size_t pln) {
  const NetFrame F = frames[blockIdx.x];
  double sq = 0.0, sqd = 0.0, se = 0.0;
  for (int i = F.off + threadIdx.x; i < F.off + F.n; i += blockDim.x) {
    const T x = ldT<T>(qt, i, pln);
    sq += double(val(x));
    sqd += double(tan_(x));
    se += double(val(ldT<T>(ei, i, pln)));
  }
  __shared__ double red[3][32];
  sq = gbpme::warp_sum_d(sq);
  sqd = gbpme::warp_sum_d(sqd);
  se = gbpme::warp_sum_d(se);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sq;
    red[1][threadIdx.x >> 5] = sqd;
    red[2][threadIdx.x >> 5] = se;
  }
  __syncthreads();
  __shared__ float mean[2];
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, e = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      e += red[2][w];
    }
    mean[0] = F.n ? float(a / F.n) : 0.f;
    mean[1] = F.n ? float(b / F.n) : 0.f;
    if (esr) esr[blockIdx.x] = e;
  }
  __syncthreads();
  for (int i = F.off + threadIdx.x; i < F.off + F.n; i += blockDim.x) {
    q[i] = qt[i] - mean[0];
    if (sizeof(T) > sizeof(float)) q[i + pln] = qt[i + pln] - mean[1];
  }
}

// Per-frame mean of the charge cotangent (both planes): the reverse of the neutralisation.
template <typename T>
__global__ void k_frame_mean(const NetFrame* __restrict__ frames, const float* __restrict__ g, float* mean,
                             size_t pln) {
  const NetFrame F = frames[blockIdx.x];
  double a = 0.0, b = 0.0;
  for (int i = F.off + threadIdx.x; i < F.off + F.n; i += blockDim.x) {
    const T x = ldT<T>(g, i, pln);
    a += double(val(x));
    b += double(tan_(x));
  }
  a = gbpme::block_sum_d(a);
  __syncthreads();
  b = gbpme::block_sum_d(b);
  if (threadIdx.x == 0) {
    mean[2 * blockIdx.x] = F.n ? float(a / F.n) : 0.f;
    mean[2 * blockIdx.x + 1] = F.n ? float(b / F.n) : 0.f;
  }
}

struct ReadoutBwdArgs {
  const float* P;
  const int* frame_of;
  const float* H;       // [n][64] (before the bias)
  const float* hv;      // [n][3][16] final vector features
  const float* gq;      // [n] cotangent of q (may be null)
  const float* gq_mean; // [F][2]
  const float* gmu;     // [n][3] (may be null)
  const float* gesr;    // [F] value and tangent: gesr[2 f], gesr[2 f + 1] (may be null)
  float* gH;            // [n][64]
  float* ghv;           // [n][3][16] (written)
  float* part;          // [block][planes][kReadoutW]
  int n;
  size_t pln, plH, plV;
};

template <typename T>
__global__ void __launch_bounds__(32 * kWarps) k_readout_bwd(ReadoutBwdArgs a) {
  __shared__ float sp[kWarps][2][kReadoutW];
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int i = blockIdx.x * kWarps + w;
  for (int k = c; k < kReadoutW; k += 32) sp[w][0][k] = sp[w][1][k] = 0.f;
  __syncwarp();
  if (i < a.n) {
    const int f = a.frame_of[i];
    T gqt = 0.f;
    if (a.gq) gqt = ldT<T>(a.gq, i, a.pln) - mk<T>(a.gq_mean[2 * f], a.gq_mean[2 * f + 1]);
    const T ge = a.gesr ? mk<T>(a.gesr[2 * f], a.gesr[2 * f + 1]) : T(0.f);
    const T hq = ldT<T>(a.H, size_t(i) * 2 * S + c, a.plH) + a.P[oBh + c];
    const T he = ldT<T>(a.H, size_t(i) * 2 * S + S + c, a.plH) + a.P[oBh + S + c];
    const T gHq = gqt * a.P[oWq + c] * dsiluT(hq);
    const T gHe = ge * a.P[oWE + c] * dsiluT(he);
    stT(a.gH, size_t(i) * 2 * S + c, a.plH, gHq);
    stT(a.gH, size_t(i) * 2 * S + S + c, a.plH, gHe);
    const T pwq = gqt * siluT(hq), pwe = ge * siluT(he);
    sp[w][0][c] = val(pwq);                 sp[w][1][c] = tan_(pwq);
    sp[w][0][S + c] = val(pwe);             sp[w][1][S + c] = tan_(pwe);
    sp[w][0][2 * S + c] = val(gHq);         sp[w][1][2 * S + c] = tan_(gHq);
    sp[w][0][3 * S + c] = val(gHe);         sp[w][1][3 * S + c] = tan_(gHe);
    if (c == 0) {
      sp[w][0][4 * S] = val(gqt);           sp[w][1][4 * S] = tan_(gqt);
      sp[w][0][4 * S + 1] = val(ge);        sp[w][1][4 * S + 1] = tan_(ge);
    }
    if (c < V) {
      T gw = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T gm = a.gmu ? ldT<T>(a.gmu, 3 * size_t(i) + d, 3 * a.pln) : T(0.f);
        const size_t k = (size_t(i) * 3 + d) * V + c;
        stT(a.ghv, k, a.plV, gm * a.P[oWmu + c]);
        gw += gm * ldT<T>(a.hv, k, a.plV);
      }
      sp[w][0][4 * S + 2 + c] = val(gw);
      sp[w][1][4 * S + 2 + c] = tan_(gw);
    }
  }
  __syncthreads();
  constexpr int kPlanes = sizeof(T) / sizeof(float);
  for (int t = threadIdx.x; t < kPlanes * kReadoutW; t += blockDim.x) {
    const int pl = t / kReadoutW, k = t % kReadoutW;
    float acc = 0.f;
    for (int ww = 0; ww < kWarps; ++ww) acc += sp[ww][pl][k];
    a.part[(size_t(blockIdx.x) * kPlanes + pl) * kReadoutW + k] = acc;
  }
}

// Per-block partials of dL/d emb [2][32] from the layer-0 input cotangent g_hs.
template <typename T>
__global__ void k_emb_bwd(int n, const int* __restrict__ species, const float* __restrict__ ghs, size_t plS,
                          float* part) {
  // block of 256 threads = 8 ion slots x 32 channels; each block covers 8 * 64 ions
  __shared__ float sp[8][2][2 * S];
  const int slot = threadIdx.x >> 5, c = threadIdx.x & 31;
  T a0 = 0.f, a1 = 0.f;
  for (int i = blockIdx.x * 512 + slot; i < min(n, int(blockIdx.x + 1) * 512); i += 8) {
    const T g = ldT<T>(ghs, size_t(i) * S + c, plS);
    if (species[i] == 0) a0 += g;
    else a1 += g;
  }
  sp[slot][0][c] = val(a0);      sp[slot][1][c] = tan_(a0);
  sp[slot][0][S + c] = val(a1);  sp[slot][1][S + c] = tan_(a1);
  __syncthreads();
  constexpr int kPlanes = sizeof(T) / sizeof(float);
  for (int t = threadIdx.x; t < kPlanes * 2 * S; t += blockDim.x) {
    const int pl = t / (2 * S), k = t % (2 * S);
    float acc = 0.f;
    for (int s2 = 0; s2 < 8; ++s2) acc += sp[s2][pl][k];
    part[(size_t(blockIdx.x) * kPlanes + pl) * 2 * S + k] = acc;
  }
}

// Per-block partials of the weight gradient G[K][N] = sum_rows X[r][k] Gy[r][n] over 128-row
// chunks (X: [rows][K], Gy: [rows][N]), staged 32 rows at a time; for Dual also the tangent
// sum X' Gy + X Gy'.
constexpr int kWgRows = 128;
constexpr int kWgSub = 32;
template <typename T, int K, int N>
__global__ void __launch_bounds__(256) k_wgrad(int rows, const float* __restrict__ X, const float* __restrict__ Gy,
                                              size_t plX, size_t plG, float* part) {
  constexpr int kPlanes = sizeof(T) / sizeof(float);
  constexpr int kOut = (K * N + 255) / 256;
  __shared__ float sX[kPlanes][kWgSub][K];
  __shared__ float sGy[kPlanes][kWgSub][N + 1];
  float a[kOut], b[kOut];
#pragma unroll
  for (int u = 0; u < kOut; ++u) a[u] = b[u] = 0.f;
  for (int r0 = blockIdx.x * kWgRows; r0 < min(rows, int(blockIdx.x + 1) * kWgRows); r0 += kWgSub) {
    __syncthreads();
    for (int t = threadIdx.x; t < kWgSub * K; t += blockDim.x) {
      const int r = t / K, k = t % K;
      const bool ok = r0 + r < rows;
      sX[0][r][k] = ok ? X[size_t(r0 + r) * K + k] : 0.f;
      if (kPlanes > 1) sX[kPlanes - 1][r][k] = ok ? X[size_t(r0 + r) * K + k + plX] : 0.f;
    }
    for (int t = threadIdx.x; t < kWgSub * N; t += blockDim.x) {
      const int r = t / N, k = t % N;
      const bool ok = r0 + r < rows;
      sGy[0][r][k] = ok ? Gy[size_t(r0 + r) * N + k] : 0.f;
      if (kPlanes > 1) sGy[kPlanes - 1][r][k] = ok ? Gy[size_t(r0 + r) * N + k + plG] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int o = threadIdx.x + 256 * u;
      if (o < K * N) {
        const int k = o / N, nn = o % N;
        for (int r = 0; r < kWgSub; ++r) {
          a[u] += sX[0][r][k] * sGy[0][r][nn];
          if (kPlanes > 1) b[u] += sX[kPlanes - 1][r][k] * sGy[0][r][nn] + sX[0][r][k] * sGy[kPlanes - 1][r][nn];
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int o = threadIdx.x + 256 * u;
    if (o < K * N) {
      part[(size_t(blockIdx.x) * kPlanes) * K * N + o] = a[u];
      if (kPlanes > 1) part[(size_t(blockIdx.x) * kPlanes + 1) * K * N + o] = b[u];
    }
  }
}

// out[plane][w] (+)= sum over blocks b of part[b][plane][w] (fixed order); planes selected by
// plane_out: the value plane goes to out_v, the tangent plane to out_t (either may be null).
__global__ void k_reduce_parts(const float* __restrict__ part, int nblk, int planes, int width, float* out_v,
                               float* out_t, int accumulate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= planes * width) return;
  const int pl = t / width, k = t % width;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[(size_t(b) * planes + pl) * width + k];
  float* out = pl == 0 ? out_v : out_t;
  if (!out) return;
  out[k] = accumulate ? out[k] + float(acc) : float(acc);
}

// Scatter the readout partial sums (wq, wE, bh, bq, bE, wmu) into a parameter-gradient
// vector: reduced[w] -> param index.
__device__ __forceinline__ int readout_param(int k) {
  if (k < S) return oWq + k;
  if (k < 2 * S) return oWE + (k - S);
  if (k < 4 * S) return oBh + (k - 2 * S);
  if (k == 4 * S) return oBq;
  if (k == 4 * S + 1) return oBE;
  return oWmu + (k - 4 * S - 2);
}
__global__ void k_reduce_readout(const float* __restrict__ part, int nblk, int planes, float* out_v, float* out_t,
                                 int accumulate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= planes * kReadoutW) return;
  const int pl = t / kReadoutW, k = t % kReadoutW;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[(size_t(b) * planes + pl) * kReadoutW + k];
  float* out = pl == 0 ? out_v : out_t;
  if (!out) return;
  const int o = readout_param(k);
  out[o] = accumulate ? out[o] + float(acc) : float(acc);
}

// ---------------------------------------------------------------------------------------
// loss, optimiser, weights
// ---------------------------------------------------------------------------------------

// Per frame (one block each): E_b = E_pme,b + E_sr,b; energy cotangent c_b; per ion: the
// model force F = F_pme - g_pos(net), the force residual and the position tangent r' = -w.
// part[f] = (L_E, L_F) contributions of frame f (float64).
__global__ void k_loss(const NetFrame* __restrict__ frames, int nframes, int ntot, const double* __restrict__ e_pme,
                       const double* __restrict__ e_sr, const double* __restrict__ e_ref,
                       const float* __restrict__ f_pme, const float* __restrict__ gpos_net,
                       const float* __restrict__ f_ref, double lambda_e, double lambda_f, double* cvec,
                       float* force, float* dpos, float* wneg, double* part) {
  const NetFrame F = frames[blockIdx.x];
  const double wf = 2.0 * lambda_f / (3.0 * double(ntot));
  double lf = 0.0;
  for (int t = threadIdx.x; t < 3 * F.n; t += blockDim.x) {
    const size_t k = 3 * size_t(F.off) + t;
    const float Fm = f_pme[k] - gpos_net[k];
    const float res = Fm - f_ref[k];
    if (force) force[k] = Fm;
    lf += double(res) * double(res);
    const float wv = float(wf * double(res));
    dpos[k] = -wv;
    wneg[k] = wv;     // g_force of the PME Hessian-vector product: -r' = w
  }
  lf = gbpme::block_sum_d(lf);
  if (threadIdx.x == 0) {
    const double E = e_pme[blockIdx.x] + e_sr[blockIdx.x];
    const double dE = (E - e_ref[blockIdx.x]) / double(max(F.n, 1));
    cvec[blockIdx.x] = F.n ? 2.0 * lambda_e * dE / (double(nframes) * double(F.n)) : 0.0;
    part[2 * blockIdx.x] = lambda_e * dE * dE / double(nframes);
    part[2 * blockIdx.x + 1] = lambda_f * lf / (3.0 * double(ntot));
  }
}

__global__ void k_loss_total(const double* __restrict__ part, int nframes, double* loss) {
  double le = 0.0, lf = 0.0;
  for (int f = threadIdx.x; f < nframes; f += blockDim.x) {
    le += part[2 * f];
    lf += part[2 * f + 1];
  }
  le = gbpme::block_sum_d(le);
  __syncthreads();
  lf = gbpme::block_sum_d(lf);
  if (threadIdx.x == 0) {
    loss[0] = le + lf;
    loss[1] = le;
    loss[2] = lf;
  }
}

// energy cotangent seeds of the Dual backward: gesr[2 f] = 1, gesr[2 f + 1] = c_f
__global__ void k_seed_esr(int nframes, const double* __restrict__ cvec, float* gesr, int with_tangent) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nframes) return;
  gesr[2 * f] = 1.f;
  gesr[2 * f + 1] = with_tangent ? float(cvec[f]) : 0.f;
}

// dst[k] = s * src[k] (and optionally a second array into the tangent plane of dst)
__global__ void k_scale(size_t m, const float* __restrict__ src, float s, float* dst) {
  const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < m) dst[t] = s * src[t];
}

// bfloat16 copies of the channel-mixing matrices: W [K][N] and W^T [N][K]
__global__ void k_cast_weights(const float* __restrict__ P, uint16_t* wbf, const int* __restrict__ offs) {
  const int w = blockIdx.y;
  const MixW m = mix_w(w);
  uint16_t* dW = wbf + offs[2 * w];
  uint16_t* dWt = wbf + offs[2 * w + 1];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.K * m.N; t += gridDim.x * blockDim.x) {
    const int k = t / m.N, nn = t % m.N;
    const uint32_t u = __float_as_uint(P[m.off + t]);
    const uint16_t b = uint16_t((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    dW[t] = b;
    dWt[nn * m.K + k] = b;
  }
}

__global__ void k_adam(int np, float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  P[t] -= lr * (mt * c1) / (sqrtf(vt * c2) + eps);
}

}  // namespace
}  // namespace gbnet

// =========================================================================================
// host side
// =========================================================================================
using gbpme::Dual;
using gbnet::NetFrame;

struct gbnet_s {
  int max_ions = 0, max_frames = 0, n = 0, nframes = 0, dev = 0;
  std::string err;
  long long launches = 0;
  int adam_step = 0;
  // parameters, optimiser state, gradients
  float *P = nullptr, *am = nullptr, *av = nullptr, *grad = nullptr, *gscratch = nullptr;
  uint16_t* wbf = nullptr;
  int* wbf_offs_d = nullptr;
  int wbf_offs[2 * gbnet::kNumMix] = {};
  int* flags = nullptr;
  // frames and neighbours
  NetFrame* frames_d = nullptr;
  std::vector<int> offsets_h;
  int* frame_of = nullptr;
  int* species = nullptr;
  int *nbr_cnt = nullptr, *nbr_j = nullptr;
  float4* nbr_sh = nullptr;
  // activations (two planes each)
  float *hs[3] = {}, *hv[3] = {}, *A[2] = {}, *B[2] = {}, *ms[2] = {}, *mv[2] = {}, *U[2] = {}, *Y[2] = {};
  float *H = nullptr, *qt = nullptr, *ei = nullptr, *q = nullptr, *mu = nullptr;
  // backward scratch
  float *ghs = nullptr, *ghv = nullptr, *gA = nullptr, *gB = nullptr, *gms = nullptr, *gmv = nullptr,
        *gU = nullptr, *gY = nullptr, *gH = nullptr, *gpos = nullptr, *gq = nullptr, *gmu = nullptr,
        *gq_mean = nullptr, *gesr = nullptr, *part = nullptr;
  size_t part_cap = 0;
  // loss scratch
  double *e_sr = nullptr, *e_pme = nullptr, *cvec = nullptr, *lpart = nullptr;
  float *q_plain = nullptr, *mu_plain = nullptr, *f_pme = nullptr, *field = nullptr, *dpos = nullptr,
        *wneg = nullptr, *mut_neg = nullptr, *gp_scratch = nullptr, *pos_saved = nullptr;
  std::vector<void*> owned;
};

namespace gbnet {
namespace {

int fail(gbnet_t net, int st, const std::string& msg) {
  if (net) net->err = msg;
  return st;
}

int cuda_ok(gbnet_t net, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PME_OK;
  return fail(net, PME_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NET_LAUNCHED(net)                                                          \
  do {                                                                             \
    gbpme::count_launch();                                                         \
    ++(net)->launches;                                                             \
    const cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) return cuda_ok((net), e_, "kernel launch");             \
  } while (0)

inline unsigned blocks_for(size_t m, int t) { return unsigned((m + t - 1) / t); }

int mix(gbnet_t net, cudaStream_t s, int M, int K, int N, const float* X, int w, bool transposed_weights,
        float* Y, bool acc) {
  const uint16_t* W = net->wbf + net->wbf_offs[2 * w + (transposed_weights ? 1 : 0)];
  const int st = launch_mix(s, M, K, N, X, W, Y, acc, net->flags);
  ++net->launches;
  return st ? fail(net, st, "channel mixing") : PME_OK;
}

template <typename T>
MsgArgs msg_args(gbnet_t net, int layer, const float* pos, const float* dpos) {
  MsgArgs a;
  a.frames = net->frames_d;
  a.frame_of = net->frame_of;
  a.nb = Nbr{net->nbr_cnt, net->nbr_j, net->nbr_sh};
  a.pos = pos;
  a.dpos = dpos;
  a.WR = net->P + oLayer0 + layer * kLayerSize + oWR;
  a.n = net->n;
  a.plS = size_t(net->n) * (S + V);
  a.plV = size_t(net->n) * 3 * 2 * V;
  return a;
}

// forward pass; dpos is the position tangent (Dual passes only)
template <typename T>
int forward_pass(gbnet_t net, cudaStream_t s, const float* pos, const float* dpos) {
  constexpr int planes = sizeof(T) / sizeof(float);
  const int n = net->n;
  const size_t plS = size_t(n) * S, plV = size_t(n) * 3 * V, pl48 = size_t(n) * (S + V),
               pl96 = size_t(n) * 3 * 2 * V, pl64 = size_t(n) * 2 * S;
  int st;
  if (n == 0) return PME_OK;
  k_embed<<<blocks_for(size_t(n) * 3 * V, 256), 256, 0, s>>>(net->P, net->species, n, net->hs[0], net->hv[0], plS,
                                                             plV, planes);
  NET_LAUNCHED(net);
  for (int t = 0; t < 2; ++t) {
    if ((st = mix(net, s, planes * n, S, S + V, net->hs[t], 4 * t + 0, true, net->A[t], false))) return st;
    if ((st = mix(net, s, planes * 3 * n, V, 2 * V, net->hv[t], 4 * t + 1, true, net->B[t], false))) return st;
    const MsgArgs a = msg_args<T>(net, t, pos, dpos);
    k_msg_fwd<T><<<blocks_for(n, kWarps), 32 * kWarps, 0, s>>>(a, net->A[t], net->B[t], net->ms[t], net->mv[t]);
    NET_LAUNCHED(net);
    if ((st = mix(net, s, planes * n, S + V, S + V, net->ms[t], 4 * t + 2, true, net->U[t], false))) return st;
    if ((st = mix(net, s, planes * 3 * n, 2 * V, V, net->mv[t], 4 * t + 3, true, net->Y[t], false))) return st;
    k_update_fwd<T><<<blocks_for(size_t(n) * S, 256), 256, 0, s>>>(n, net->U[t], net->Y[t], net->hs[t], net->hv[t],
                                                                  net->hs[t + 1], net->hv[t + 1], pl48, plV, plS, plV);
    NET_LAUNCHED(net);
  }
  if ((st = mix(net, s, planes * n, S, 2 * S, net->hs[2], 8, true, net->H, false))) return st;
  k_readout_fwd<T><<<blocks_for(n, kWarps), 32 * kWarps, 0, s>>>(n, net->P, net->H, net->hv[2], net->qt, net->ei,
                                                                net->mu, pl64, plV, size_t(n));
  NET_LAUNCHED(net);
  k_frame_fwd<T><<<net->nframes, 256, 0, s>>>(net->frames_d, net->qt, net->ei, net->q, net->e_sr, size_t(n));
  NET_LAUNCHED(net);
  (void)pl96;
  return PME_OK;
}

template <typename T, int K, int N>
int wgrad(gbnet_t net, cudaStream_t s, int rows, const float* X, const float* Gy, int poff, float* gv, float* gt,
          bool acc) {
  constexpr int planes = sizeof(T) / sizeof(float);
  if (rows == 0) return PME_OK;
  const int nblk = (rows + kWgRows - 1) / kWgRows;
  k_wgrad<T, K, N><<<nblk, 256, 0, s>>>(rows, X, Gy, size_t(rows) * K, size_t(rows) * N, net->part);
  NET_LAUNCHED(net);
  k_reduce_parts<<<blocks_for(size_t(planes) * K * N, 256), 256, 0, s>>>(
      net->part, nblk, planes, K * N, gv ? gv + poff : nullptr, gt ? gt + poff : nullptr, acc ? 1 : 0);
  NET_LAUNCHED(net);
  return PME_OK;
}

// Backward pass of the last forward_pass<T>. Seeds: gq [planes][n], gmu [planes][n][3] (each
// may be null), gesr_f [F][2] float (value, tangent). Outputs: gpos [planes][n][3] (net->gpos,
// written), parameter gradients: value plane -> gv, tangent plane -> gt (either null to skip;
// both null skips every weight-gradient launch).
template <typename T>
int backward_pass(gbnet_t net, cudaStream_t s, const float* pos, const float* dpos, const float* gq,
                  const float* gmu, const float* gesr_f, float* gv, float* gt, bool acc) {
  constexpr int planes = sizeof(T) / sizeof(float);
  const int n = net->n;
  const size_t plS = size_t(n) * S, plV = size_t(n) * 3 * V, pl48 = size_t(n) * (S + V),
               pl96 = size_t(n) * 3 * 2 * V, pl64 = size_t(n) * 2 * S;
  const bool params = gv || gt;
  int st;
  if ((st = cuda_ok(net, cudaMemsetAsync(net->gpos, 0, sizeof(float) * planes * 3 * size_t(n), s), "memset")))
    return st;
  if (n == 0) return PME_OK;
  if (gq) {
    k_frame_mean<T><<<net->nframes, 256, 0, s>>>(net->frames_d, gq, net->gq_mean, size_t(n));
    NET_LAUNCHED(net);
  }
  ReadoutBwdArgs ra;
  ra.P = net->P;
  ra.frame_of = net->frame_of;
  ra.H = net->H;
  ra.hv = net->hv[2];
  ra.gq = gq;
  ra.gq_mean = net->gq_mean;
  ra.gmu = gmu;
  ra.gesr = gesr_f;
  ra.gH = net->gH;
  ra.ghv = net->ghv;
  ra.part = net->part;
  ra.n = n;
  ra.pln = size_t(n);
  ra.plH = pl64;
  ra.plV = plV;
  const int nb_ion = int(blocks_for(n, kWarps));
  k_readout_bwd<T><<<nb_ion, 32 * kWarps, 0, s>>>(ra);
  NET_LAUNCHED(net);
  if (params) {
    k_reduce_readout<<<blocks_for(size_t(planes) * kReadoutW, 256), 256, 0, s>>>(net->part, nb_ion, planes, gv, gt,
                                                                                 acc ? 1 : 0);
    NET_LAUNCHED(net);
  }
  if ((st = mix(net, s, planes * n, 2 * S, S, net->gH, 8, false, net->ghs, false))) return st;
  if (params && (st = wgrad<T, S, 2 * S>(net, s, n, net->hs[2], net->gH, oWh, gv, gt, acc))) return st;
  for (int t = 1; t >= 0; --t) {
    const int base = oLayer0 + t * kLayerSize;
    k_update_bwd<T><<<blocks_for(size_t(n) * S, 256), 256, 0, s>>>(n, net->U[t], net->Y[t], net->ghs, net->ghv, net->gU,
                                                                   net->gY, pl48, plV, plS, plV);
    NET_LAUNCHED(net);
    if ((st = mix(net, s, planes * n, S + V, S + V, net->gU, 4 * t + 2, false, net->gms, false))) return st;
    if ((st = mix(net, s, planes * 3 * n, V, 2 * V, net->gY, 4 * t + 3, false, net->gmv, false))) return st;
    if (params && (st = wgrad<T, S + V, S + V>(net, s, n, net->ms[t], net->gU, base + oWU, gv, gt, acc))) return st;
    if (params && (st = wgrad<T, 2 * V, V>(net, s, 3 * n, net->mv[t], net->gY, base + oWY, gv, gt, acc))) return st;
    const MsgArgs a = msg_args<T>(net, t, pos, dpos);
    k_msg_bwd<T><<<nb_ion, 32 * kWarps, 0, s>>>(a, net->A[t], net->B[t], net->gms, net->gmv, net->gA, net->gB,
                                               net->gpos, net->part);
    NET_LAUNCHED(net);
    if (params) {
      k_reduce_parts<<<blocks_for(size_t(planes) * NR * NCOL, 256), 256, 0, s>>>(
          net->part, nb_ion, planes, NR * NCOL, gv ? gv + base + oWR : nullptr, gt ? gt + base + oWR : nullptr,
          acc ? 1 : 0);
      NET_LAUNCHED(net);
    }
    if ((st = mix(net, s, planes * n, S + V, S, net->gA, 4 * t + 0, false, net->ghs, true))) return st;
    if ((st = mix(net, s, planes * 3 * n, 2 * V, V, net->gB, 4 * t + 1, false, net->ghv, true))) return st;
    if (params && (st = wgrad<T, S, S + V>(net, s, n, net->hs[t], net->gA, base + oWA, gv, gt, acc))) return st;
    if (params && (st = wgrad<T, V, 2 * V>(net, s, 3 * n, net->hv[t], net->gB, base + oWB, gv, gt, acc))) return st;
  }
  if (params) {
    const int nb = (n + 511) / 512;
    k_emb_bwd<T><<<nb, 256, 0, s>>>(n, net->species, net->ghs, plS, net->part);
    NET_LAUNCHED(net);
    k_reduce_parts<<<blocks_for(size_t(planes) * 2 * S, 256), 256, 0, s>>>(net->part, nb, planes, 2 * S,
                                                                           gv ? gv + oEmb : nullptr,
                                                                           gt ? gt + oEmb : nullptr, acc ? 1 : 0);
    NET_LAUNCHED(net);
  }
  (void)pl96;
  return PME_OK;
}

int build_neighbours(gbnet_t net, cudaStream_t s, const float* pos) {
  if (net->n == 0) return PME_OK;
  k_nbr<<<blocks_for(net->n, kWarps), 32 * kWarps, 0, s>>>(net->frames_d, net->frame_of, pos, net->n, net->nbr_cnt,
                                                          net->nbr_j, net->nbr_sh, net->flags);
  NET_LAUNCHED(net);
  return PME_OK;
}

__global__ void k_gesr_from(int nframes, const double* __restrict__ g, float* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nframes) return;
  out[2 * f] = g ? float(g[f]) : 0.f;
  out[2 * f + 1] = 0.f;
}

__global__ void k_frame_of(const int* __restrict__ offs, int nframes, int* frame_of) {
  const int f = blockIdx.x;
  for (int i = offs[f] + threadIdx.x; i < offs[f + 1]; i += blockDim.x) frame_of[i] = f;
}

bool invert3(const double* a, double* inv) {
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  if (!std::isfinite(det) || std::fabs(det) < 1e-300) return false;
  const double id = 1.0 / det;
  inv[0] = (a[4] * a[8] - a[5] * a[7]) * id;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  inv[3] = (a[5] * a[6] - a[3] * a[8]) * id;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  inv[6] = (a[3] * a[7] - a[4] * a[6]) * id;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return true;
}

}  // namespace
}  // namespace gbnet

using namespace gbnet;

extern "C" {

int gbnet_create(gbnet_t* out, int max_ions, int max_frames) {
  if (!out || max_ions < 0 || max_frames < 1 || max_ions > (1 << 24)) return PME_ERR_ARG;
  *out = nullptr;
  gbnet_t net = new (std::nothrow) gbnet_s;
  if (!net) return PME_ERR_NOMEM;
  net->max_ions = max_ions;
  net->max_frames = max_frames;
  cudaGetDevice(&net->dev);
  const size_t N = size_t(std::max(max_ions, 1));
  bool ok = true;
  auto A = [&](auto** p, size_t bytes) {
    void* q = nullptr;
    if (ok && cudaMalloc(&q, std::max<size_t>(bytes, 16)) == cudaSuccess) {
      net->owned.push_back(q);
      *p = static_cast<std::remove_pointer_t<decltype(p)>>(q);
    } else {
      ok = false;
    }
  };
  const size_t f = sizeof(float);
  A(&net->P, f * kParams);
  A(&net->am, f * kParams);
  A(&net->av, f * kParams);
  A(&net->grad, f * kParams);
  A(&net->gscratch, f * kParams);
  int woff = 0;
  for (int w = 0; w < kNumMix; ++w) {
    const MixW m = mix_w(w);
    net->wbf_offs[2 * w] = woff;
    woff += m.K * m.N;
    net->wbf_offs[2 * w + 1] = woff;
    woff += m.K * m.N;
  }
  A(&net->wbf, sizeof(uint16_t) * woff);
  A(&net->wbf_offs_d, sizeof(int) * 2 * kNumMix);
  A(&net->flags, sizeof(int));
  A(&net->frames_d, sizeof(NetFrame) * max_frames);
  A(&net->frame_of, sizeof(int) * N);
  A(&net->species, sizeof(int) * N);
  A(&net->nbr_cnt, sizeof(int) * N);
  A(&net->nbr_j, sizeof(int) * N * kMaxNbr);
  A(&net->nbr_sh, sizeof(float4) * N * kMaxNbr);
  for (int t = 0; t < 3; ++t) {
    A(&net->hs[t], 2 * f * N * S);
    A(&net->hv[t], 2 * f * N * 3 * V);
  }
  for (int t = 0; t < 2; ++t) {
    A(&net->A[t], 2 * f * N * (S + V));
    A(&net->B[t], 2 * f * N * 3 * 2 * V);
    A(&net->ms[t], 2 * f * N * (S + V));
    A(&net->mv[t], 2 * f * N * 3 * 2 * V);
    A(&net->U[t], 2 * f * N * (S + V));
    A(&net->Y[t], 2 * f * N * 3 * V);
  }
  A(&net->H, 2 * f * N * 2 * S);
  A(&net->qt, 2 * f * N);
  A(&net->ei, 2 * f * N);
  A(&net->q, 2 * f * N);
  A(&net->mu, 2 * f * N * 3);
  A(&net->ghs, 2 * f * N * S);
  A(&net->ghv, 2 * f * N * 3 * V);
  A(&net->gA, 2 * f * N * (S + V));
  A(&net->gB, 2 * f * N * 3 * 2 * V);
  A(&net->gms, 2 * f * N * (S + V));
  A(&net->gmv, 2 * f * N * 3 * 2 * V);
  A(&net->gU, 2 * f * N * (S + V));
  A(&net->gY, 2 * f * N * 3 * V);
  A(&net->gH, 2 * f * N * 2 * S);
  A(&net->gpos, 2 * f * N * 3);
  A(&net->gq, 2 * f * N);
  A(&net->gmu, 2 * f * N * 3);
  A(&net->gq_mean, 2 * f * max_frames);
  A(&net->gesr, 2 * f * max_frames);
  // partial sums: the largest of the weight-gradient, message and readout reductions
  const size_t wg = size_t((3 * N + kWgRows - 1) / kWgRows) * 2 * (S + V) * (S + V);
  const size_t ms = size_t((N + kWarps - 1) / kWarps) * 2 * NR * NCOL;
  const size_t ro = size_t((N + kWarps - 1) / kWarps) * 2 * kReadoutW;
  net->part_cap = std::max(wg, std::max(ms, ro));
  A(&net->part, f * net->part_cap);
  A(&net->e_sr, sizeof(double) * max_frames);
  A(&net->e_pme, sizeof(double) * max_frames);
  A(&net->cvec, sizeof(double) * max_frames);
  A(&net->lpart, sizeof(double) * 2 * max_frames);
  A(&net->q_plain, f * N);
  A(&net->mu_plain, f * N * 3);
  A(&net->f_pme, f * N * 3);
  A(&net->field, f * N * 3);
  A(&net->dpos, f * N * 3);
  A(&net->wneg, f * N * 3);
  A(&net->mut_neg, f * N * 3);
  A(&net->gp_scratch, f * N * 3);
  A(&net->pos_saved, f * N * 3);
  if (!ok) {
    gbnet_destroy(net);
    return PME_ERR_NOMEM;
  }
  if (cudaMemcpy(net->wbf_offs_d, net->wbf_offs, sizeof(int) * 2 * kNumMix, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(net->P, 0, f * kParams) != cudaSuccess || cudaMemset(net->flags, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(net->wbf, 0, sizeof(uint16_t) * woff) != cudaSuccess) {
    gbnet_destroy(net);
    return PME_ERR_CUDA;
  }
  *out = net;
  return PME_OK;
}

int gbnet_destroy(gbnet_t net) {
  if (!net) return PME_ERR_ARG;
  for (void* p : net->owned) cudaFree(p);
  delete net;
  return PME_OK;
}

const char* gbnet_last_error(gbnet_t net) { return net ? net->err.c_str() : "null handle"; }

int gbnet_set_frames(gbnet_t net, void* stream, int nframes, const int* offsets, const double* boxes,
                     const int* species) {
  if (!net || !offsets || !boxes || nframes < 1 || nframes > net->max_frames) return PME_ERR_ARG;
  if (offsets[0] != 0) return fail(net, PME_ERR_ARG, "offsets[0] must be 0");
  for (int f = 0; f < nframes; ++f)
    if (offsets[f + 1] < offsets[f]) return fail(net, PME_ERR_ARG, "offsets must not decrease");
  const int n = offsets[nframes];
  if (n > net->max_ions) return fail(net, PME_ERR_ARG, "more ions than max_ions");
  if (n > 0 && !species) return fail(net, PME_ERR_ARG, "species is NULL");
  std::vector<NetFrame> fr(nframes);
  for (int f = 0; f < nframes; ++f) {
    const double* C = boxes + 9 * f;
    double Ci[9];
    if (!invert3(C, Ci)) return fail(net, PME_ERR_ARG, "singular box");
    const double vol = std::fabs(C[0] * (C[4] * C[8] - C[5] * C[7]) - C[1] * (C[3] * C[8] - C[5] * C[6]) +
                                 C[2] * (C[3] * C[7] - C[4] * C[6]));
    for (int a = 0; a < 3; ++a) {
      const double* u = C + 3 * ((a + 1) % 3);
      const double* v = C + 3 * ((a + 2) % 3);
      const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      const double width = vol / std::sqrt(cx * cx + cy * cy + cz * cz);
      if (width < 2.0 * GBNET_CUTOFF) return fail(net, PME_ERR_ARG, "box narrower than twice the cutoff");
    }
    fr[f].off = offsets[f];
    fr[f].n = offsets[f + 1] - offsets[f];
    for (int k = 0; k < 9; ++k) {
      fr[f].C[k] = float(C[k]);
      fr[f].Ci[k] = float(Ci[k]);
    }
    fr[f].ortho = (C[1] == 0 && C[2] == 0 && C[3] == 0 && C[5] == 0 && C[6] == 0 && C[7] == 0) ? 1 : 0;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  net->offsets_h.assign(offsets, offsets + nframes + 1);
  net->n = n;
  net->nframes = nframes;
  int st;
  if ((st = cuda_ok(net, cudaMemcpyAsync(net->frames_d, fr.data(), sizeof(NetFrame) * nframes,
                                         cudaMemcpyHostToDevice, s), "copy frames")))
    return st;
  // frame_of from the offsets (staged through the tail of the loss scratch)
  int* offs_d = reinterpret_cast<int*>(net->lpart);
  if (size_t(nframes + 1) * sizeof(int) > sizeof(double) * 2 * size_t(net->max_frames))
    return fail(net, PME_ERR_ARG, "too many frames");
  if ((st = cuda_ok(net, cudaMemcpyAsync(offs_d, offsets, sizeof(int) * (nframes + 1), cudaMemcpyHostToDevice, s),
                    "copy offsets")))
    return st;
  k_frame_of<<<nframes, 256, 0, s>>>(offs_d, nframes, net->frame_of);
  NET_LAUNCHED(net);
  if (n > 0 &&
      (st = cuda_ok(net, cudaMemcpyAsync(net->species, species, sizeof(int) * n, cudaMemcpyDeviceToDevice, s),
                    "copy species")))
    return st;
  // the offsets copy above must finish before the host array can go away
  return cuda_ok(net, cudaStreamSynchronize(s), "set frames");
}

int gbnet_set_params(gbnet_t net, void* stream, const float* params) {
  if (!net || !params) return PME_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st;
  if ((st = cuda_ok(net, cudaMemcpyAsync(net->P, params, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, s),
                    "copy params")))
    return st;
  if ((st = cuda_ok(net, cudaMemsetAsync(net->am, 0, sizeof(float) * kParams, s), "memset")) ||
      (st = cuda_ok(net, cudaMemsetAsync(net->av, 0, sizeof(float) * kParams, s), "memset")))
    return st;
  net->adam_step = 0;
  k_cast_weights<<<dim3(8, kNumMix), 256, 0, s>>>(net->P, net->wbf, net->wbf_offs_d);
  NET_LAUNCHED(net);
  return PME_OK;
}

int gbnet_get_params(gbnet_t net, void* stream, float* params) {
  if (!net || !params) return PME_ERR_ARG;
  return cuda_ok(net, cudaMemcpyAsync(params, net->P, sizeof(float) * kParams, cudaMemcpyDeviceToDevice,
                                      static_cast<cudaStream_t>(stream)),
                 "copy params");
}

int gbnet_forward(gbnet_t net, void* stream, const float* pos, float* q, float* mu, double* e_sr) {
  if (!net || (net->n > 0 && !pos)) return PME_ERR_ARG;
  if (net->nframes == 0) return fail(net, PME_ERR_ARG, "no frames set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = size_t(net->n);
  int st;
  // the positions are kept for gbnet_backward (the edge geometry is recomputed there)
  if (n && (st = cuda_ok(net, cudaMemcpyAsync(net->pos_saved, pos, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, s),
                         "copy positions")))
    return st;
  if ((st = build_neighbours(net, s, net->pos_saved))) return st;
  if ((st = forward_pass<float>(net, s, net->pos_saved, nullptr))) return st;
  if (q && n && (st = cuda_ok(net, cudaMemcpyAsync(q, net->q, sizeof(float) * n, cudaMemcpyDeviceToDevice, s), "copy")))
    return st;
  if (mu && n &&
      (st = cuda_ok(net, cudaMemcpyAsync(mu, net->mu, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, s), "copy")))
    return st;
  if (e_sr &&
      (st = cuda_ok(net, cudaMemcpyAsync(e_sr, net->e_sr, sizeof(double) * net->nframes, cudaMemcpyDeviceToDevice, s),
                    "copy")))
    return st;
  return PME_OK;
}

int gbnet_backward(gbnet_t net, void* stream, const float* g_q, const float* g_mu, const double* g_esr,
                   float* g_pos, float* g_params) {
  if (!net) return PME_ERR_ARG;
  if (net->nframes == 0) return fail(net, PME_ERR_ARG, "no frames set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_gesr_from<<<blocks_for(net->nframes, 128), 128, 0, s>>>(net->nframes, g_esr, net->gesr);
  NET_LAUNCHED(net);
  int st;
  if ((st = backward_pass<float>(net, s, net->pos_saved, nullptr, g_q, g_mu, net->gesr, g_params, nullptr, false)))
    return st;
  if (g_pos && net->n &&
      (st = cuda_ok(net, cudaMemcpyAsync(g_pos, net->gpos, sizeof(float) * 3 * size_t(net->n),
                                         cudaMemcpyDeviceToDevice, s), "copy")))
    return st;
  return PME_OK;
}

static int loss_grad(gbnet_t net, pme_plan_t pme, cudaStream_t s, const float* pos, const double* e_ref,
                     const float* f_ref, double lambda_e, double lambda_f, double* loss, float* force, float* grad,
                     bool acc) {
  const int n = net->n, F = net->nframes;
  const size_t nn = size_t(n);
  int st;
  if (pme_batch_frames(pme) != F) return fail(net, PME_ERR_ARG, "the PME plan's frames differ from the network's");
  net->launches = 0;
  if (n && (st = cuda_ok(net, cudaMemcpyAsync(net->pos_saved, pos, sizeof(float) * 3 * nn, cudaMemcpyDeviceToDevice, s),
                         "copy positions")))
    return st;
  // 1. plain forward of the network and of the PME on its charges and dipoles
  if ((st = build_neighbours(net, s, net->pos_saved))) return st;
  if ((st = forward_pass<float>(net, s, net->pos_saved, nullptr))) return st;
  if (n && ((st = cuda_ok(net, cudaMemcpyAsync(net->q_plain, net->q, sizeof(float) * nn, cudaMemcpyDeviceToDevice, s),
                          "copy")) ||
            (st = cuda_ok(net, cudaMemcpyAsync(net->mu_plain, net->mu, sizeof(float) * 3 * nn,
                                               cudaMemcpyDeviceToDevice, s), "copy"))))
    return st;
  // phi goes straight into the value plane of the charge cotangent
  if ((st = pme_batch_forward(pme, s, net->pos_saved, net->q_plain, net->mu_plain, net->e_pme, net->f_pme, net->gq,
                              net->field, nullptr)))
    return fail(net, st, std::string("pme_batch_forward: ") + pme_last_error(pme));
  // 2. plain backward of the network with seeds (phi, dE/dmu = -field, 1): the net's part of dE/dr
  if (n) {
    k_scale<<<blocks_for(3 * nn, 256), 256, 0, s>>>(3 * nn, net->field, -1.f, net->gmu);
    NET_LAUNCHED(net);
  }
  k_seed_esr<<<blocks_for(F, 128), 128, 0, s>>>(F, net->cvec, net->gesr, 0);
  NET_LAUNCHED(net);
  if ((st = backward_pass<float>(net, s, net->pos_saved, nullptr, net->gq, net->gmu, net->gesr, nullptr, nullptr,
                                 false)))
    return st;
  // 3. loss, energy cotangents c_b, position tangent r' = -w
  k_loss<<<F, 256, 0, s>>>(net->frames_d, F, n, net->e_pme, net->e_sr, e_ref, net->f_pme, net->gpos, f_ref, lambda_e,
                           lambda_f, net->cvec, force, net->dpos, net->wneg, net->lpart);
  NET_LAUNCHED(net);
  k_loss_total<<<1, 256, 0, s>>>(net->lpart, F, loss);
  NET_LAUNCHED(net);
  // 4. forward of the network carrying the tangent r'
  if ((st = forward_pass<Dual>(net, s, net->pos_saved, net->dpos))) return st;
  // 5. PME Hessian-vector product along (r', q', mu') plus c_b times the gradient: the tangents
  //    of (dE/dq, dE/dmu) land in the tangent planes of the cotangents
  if (n) {
    k_scale<<<blocks_for(3 * nn, 256), 256, 0, s>>>(3 * nn, net->mu + 3 * nn, -1.f, net->mut_neg);
    NET_LAUNCHED(net);
  }
  if ((st = pme_batch_backward(pme, s, net->pos_saved, net->q_plain, net->mu_plain, net->cvec, net->wneg, net->q + nn,
                               net->mut_neg, net->gp_scratch, net->gq + nn, net->gmu + 3 * nn)))
    return fail(net, st, std::string("pme_batch_backward: ") + pme_last_error(pme));
  // 6. Dual backward of the network with energy seeds 1 + e c_b: its tangent plane is dL/dtheta
  k_seed_esr<<<blocks_for(F, 128), 128, 0, s>>>(F, net->cvec, net->gesr, 1);
  NET_LAUNCHED(net);
  if ((st = backward_pass<Dual>(net, s, net->pos_saved, net->dpos, net->gq, net->gmu, net->gesr, nullptr, grad, acc)))
    return st;
  return PME_OK;
}

int gbnet_loss_grad(gbnet_t net, pme_plan_t pme, void* stream, const float* pos, const double* e_ref,
                    const float* f_ref, double lambda_e, double lambda_f, double* loss, float* force, float* grad,
                    int accumulate) {
  if (!net || !pme || !e_ref || !loss || !grad || (net->n > 0 && (!pos || !f_ref))) return PME_ERR_ARG;
  if (net->nframes == 0) return fail(net, PME_ERR_ARG, "no frames set");
  return loss_grad(net, pme, static_cast<cudaStream_t>(stream), pos, e_ref, f_ref, lambda_e, lambda_f, loss, force,
                   grad, accumulate != 0);
}

int gbnet_adam(gbnet_t net, void* stream, const float* grad, double lr, double beta1, double beta2, double eps) {
  if (!net || !grad) return PME_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ++net->adam_step;
  const double c1 = 1.0 / (1.0 - std::pow(beta1, net->adam_step));
  const double c2 = 1.0 / (1.0 - std::pow(beta2, net->adam_step));
  k_adam<<<blocks_for(kParams, 256), 256, 0, s>>>(kParams, net->P, net->am, net->av, grad, float(lr), float(beta1),
                                                  float(beta2), float(eps), float(c1), float(c2));
  NET_LAUNCHED(net);
  k_cast_weights<<<dim3(8, kNumMix), 256, 0, s>>>(net->P, net->wbf, net->wbf_offs_d);
  NET_LAUNCHED(net);
  return PME_OK;
}

int gbnet_train_step(gbnet_t net, pme_plan_t pme, void* stream, const float* pos, const double* e_ref,
                     const float* f_ref, double lambda_e, double lambda_f, double lr, double* loss) {
  if (!net || !pme || !e_ref || !loss || (net->n > 0 && (!pos || !f_ref))) return PME_ERR_ARG;
  if (net->nframes == 0) return fail(net, PME_ERR_ARG, "no frames set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = loss_grad(net, pme, s, pos, e_ref, f_ref, lambda_e, lambda_f, loss, nullptr, net->grad, false);
  if (st) return st;
  const long long l = net->launches;
  st = gbnet_adam(net, stream, net->grad, lr, 0.9, 0.999, 1e-8);
  net->launches += l;
  return st;
}

int gbnet_mix(void* stream, int M, int k, int nout, const float* X, const unsigned short* wt, float* Y,
              int accumulate, int* err) {
  if (M < 0 || (M > 0 && (!X || !wt || !Y))) return PME_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) return PME_ERR_ARG;
  static int* dummy = nullptr;
  if (!err) {
    if (!dummy && cudaMalloc(&dummy, sizeof(int)) != cudaSuccess) return PME_ERR_NOMEM;
    err = dummy;
  }
  return launch_mix(static_cast<cudaStream_t>(stream), M, k, nout, X, wt, Y, accumulate != 0, err);
}

int gbnet_sync_status(gbnet_t net, void* stream) {
  if (!net) return PME_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int flags = 0;
  int st;
  if ((st = cuda_ok(net, cudaStreamSynchronize(s), "synchronise"))) return st;
  if ((st = cuda_ok(net, cudaMemcpy(&flags, net->flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags"))) return st;
  if ((st = cuda_ok(net, cudaMemset(net->flags, 0, sizeof(int)), "clear flags"))) return st;
  if (flags & kNetFlagTimeout) return fail(net, PME_ERR_TIMEOUT, "a tensor-core wait gave up");
  if (flags & kNetFlagNbrFull) return fail(net, PME_ERR_ARG, "an ion had more than GBNET_MAX_NEIGHBOURS neighbours");
  if (flags & kNetFlagNonFinite) return fail(net, PME_ERR_NONFINITE, "non-finite position");
  return PME_OK;
}

long long gbnet_last_launches(gbnet_t net) { return net ? net->launches : -1; }

}  // extern "C"
