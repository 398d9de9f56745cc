// Real-space pair term with point quadrupoles: the rank-2 channel of the multipole operator
// L_i = q_i + mu_i . grad + Theta_i : grad grad (an extension; the paper names quadrupolar
// channels as future work).
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
// Work split: one thread per ion in pair-cell order. It visits every offset o in
// [-kimg, kimg]^3 of the cell grid (each offset is one periodic image of the cell it wraps to,
// so every image inside rcut is seen once, also for boxes with few cells) and every ion of
// that cell, forming r = (f_i - f_j - o) H from the in-cell offsets. Sums run in a fixed
// order, so the result is reproducible. Output in caller order: out[10] = phi, grad phi,
// grad^2 phi (xx yy zz xy xz yz); qout[4..6] = A : grad^3 phi.
#include <cmath>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kQuadThreads = 128;

struct QuadPairArgs {
  Geometry g;
  PairRecords pr;
  const int* start_c;
  const float* theta;   // [caller index][6]
  float* out;           // [caller index][10]
  float* qout;          // [caller index][8], this kernel writes 4..6
  int n;
  int cell_off;         // first global cell key of the frame
  float alpha;
  float c[6];           // (2 alpha^2)^l / (alpha sqrt(pi)), l = 1..5 at c[l]
};

struct Sym {
  float xx, yy, zz, xy, xz, yz;
};

__device__ __forceinline__ Sym load_sym(const float* t) { return Sym{t[0], t[1], t[2], t[3], t[4], t[5]}; }

__device__ __forceinline__ void mul(const Sym& A, float x, float y, float z, float& ox, float& oy, float& oz) {
  ox = A.xx * x + A.xy * y + A.xz * z;
  oy = A.xy * x + A.yy * y + A.yz * z;
  oz = A.xz * x + A.yz * y + A.zz * z;
}

__global__ void __launch_bounds__(kQuadThreads) k_pair_quad(QuadPairArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const Geometry& g = a.g;
  const int4 ci = a.pr.idx[i];
  const float4 fi = a.pr.fq[i];
  const Sym A = load_sym(a.theta + size_t(ci.w) * 6);
  const float trA = A.xx + A.yy + A.zz;
  const float rc2 = g.rcut2;
  const float al = a.alpha;
  float phi = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  float hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
  float tx = 0.f, ty = 0.f, tz = 0.f;
  const int kx = g.kimg[0], ky = g.kimg[1], kz = g.kimg[2];
  const int ncx = g.ncell[0], ncy = g.ncell[1], ncz = g.ncell[2];
  for (int ox = -kx; ox <= kx; ++ox) {
    int cx = (ci.x + ox) % ncx;
    if (cx < 0) cx += ncx;
    for (int oy = -ky; oy <= ky; ++oy) {
      int cy = (ci.y + oy) % ncy;
      if (cy < 0) cy += ncy;
      for (int oz = -kz; oz <= kz; ++oz) {
        int cz = (ci.z + oz) % ncz;
        if (cz < 0) cz += ncz;
        const int key = a.cell_off + (cx * ncy + cy) * ncz + cz;
        const int lo = a.start_c[key], hi = a.start_c[key + 1];
        const bool self_cell = ox == 0 && oy == 0 && oz == 0;
        for (int j = lo; j < hi; ++j) {
          if (self_cell && j == i) continue;
          const float4 fj = a.pr.fq[j];
          const float ux = fi.x - fj.x - float(ox), uy = fi.y - fj.y - float(oy), uz = fi.z - fj.z - float(oz);
          const float rx = ux * g.H[0] + uy * g.H[3] + uz * g.H[6];
          const float ry = ux * g.H[1] + uy * g.H[4] + uz * g.H[7];
          const float rz = ux * g.H[2] + uy * g.H[5] + uz * g.H[8];
          const float r2 = rx * rx + ry * ry + rz * rz;
          if (!(r2 < rc2)) continue;
          const float rinv = rsqrtf(r2);
          const float rinv2 = rinv * rinv;
          const float ex = expf(-al * al * r2);
          const float B0 = erfcf(al * r2 * rinv) * rinv;
          const float B1 = (B0 + a.c[1] * ex) * rinv2;
          const float B2 = (3.f * B1 + a.c[2] * ex) * rinv2;
          const float B3 = (5.f * B2 + a.c[3] * ex) * rinv2;
          const float B4 = (7.f * B3 + a.c[4] * ex) * rinv2;
          const float B5 = (9.f * B4 + a.c[5] * ex) * rinv2;
          const float4 mj = a.pr.mu[j];
          const float c = mj.w, dx = mj.x, dy = mj.y, dz = mj.z;
          const Sym Bm = load_sym(a.theta + size_t(a.pr.idx[j].w) * 6);
          const float trB = Bm.xx + Bm.yy + Bm.zz;
          float Brx, Bry, Brz, Arx, Ary, Arz;
          mul(Bm, rx, ry, rz, Brx, Bry, Brz);
          mul(A, rx, ry, rz, Arx, Ary, Arz);
          const float dr = dx * rx + dy * ry + dz * rz;
          const float rBr = Brx * rx + Bry * ry + Brz * rz;
          const float rAr = Arx * rx + Ary * ry + Arz * rz;
          // potential, gradient, Hessian
          const float sI = -c * B1 - dr * B2 + trB * B2 - rBr * B3;
          const float srr = c * B2 + dr * B3 - trB * B3 + rBr * B4;
          phi += c * B0 + dr * B1 - trB * B1 + rBr * B2;
          gx += sI * rx + B1 * dx + 2.f * B2 * Brx;
          gy += sI * ry + B1 * dy + 2.f * B2 * Bry;
          gz += sI * rz + B1 * dz + 2.f * B2 * Brz;
          hxx += sI + srr * rx * rx - 2.f * B2 * dx * rx - 4.f * B3 * Brx * rx + 2.f * B2 * Bm.xx;
          hyy += sI + srr * ry * ry - 2.f * B2 * dy * ry - 4.f * B3 * Bry * ry + 2.f * B2 * Bm.yy;
          hzz += sI + srr * rz * rz - 2.f * B2 * dz * rz - 4.f * B3 * Brz * rz + 2.f * B2 * Bm.zz;
          hxy += srr * rx * ry - B2 * (dx * ry + rx * dy) - 2.f * B3 * (Brx * ry + rx * Bry) + 2.f * B2 * Bm.xy;
          hxz += srr * rx * rz - B2 * (dx * rz + rx * dz) - 2.f * B3 * (Brx * rz + rx * Brz) + 2.f * B2 * Bm.xz;
          hyz += srr * ry * rz - B2 * (dy * rz + ry * dz) - 2.f * B3 * (Bry * rz + ry * Brz) + 2.f * B2 * Bm.yz;
          // A : grad^3 phi
          const float AB = A.xx * Bm.xx + A.yy * Bm.yy + A.zz * Bm.zz +
                           2.f * (A.xy * Bm.xy + A.xz * Bm.xz + A.yz * Bm.yz);
          const float Ard = Arx * dx + Ary * dy + Arz * dz;
          const float ArBr = Arx * Brx + Ary * Bry + Arz * Brz;
          float Adx, Ady, Adz, BArx, BAry, BArz, ABrx, ABry, ABrz;
          mul(A, dx, dy, dz, Adx, Ady, Adz);
          mul(Bm, Arx, Ary, Arz, BArx, BAry, BArz);
          mul(A, Brx, Bry, Brz, ABrx, ABry, ABrz);
          const float s_r = c * trA * B2 - c * rAr * B3 + trA * dr * B3 + 2.f * Ard * B3 - rAr * dr * B4 -
                            (trA * trB + 2.f * AB) * B3 + (trA * rBr + trB * rAr + 4.f * ArBr) * B4 -
                            rAr * rBr * B5;
          const float s_Ar = 2.f * c * B2 + 2.f * dr * B3 - 2.f * trB * B3 + 2.f * rBr * B4;
          const float s_Br = -2.f * trA * B3 + 2.f * rAr * B4;
          const float s_d = -trA * B2 + rAr * B3;
          tx += s_r * rx + s_Ar * Arx + s_Br * Brx + s_d * dx - 2.f * B2 * Adx - 4.f * B3 * (BArx + ABrx);
          ty += s_r * ry + s_Ar * Ary + s_Br * Bry + s_d * dy - 2.f * B2 * Ady - 4.f * B3 * (BAry + ABry);
          tz += s_r * rz + s_Ar * Arz + s_Br * Brz + s_d * dz - 2.f * B2 * Adz - 4.f * B3 * (BArz + ABrz);
        }
      }
    }
  }
  float* o = a.out + size_t(ci.w) * 10;
  o[0] = phi;
  o[1] = gx;
  o[2] = gy;
  o[3] = gz;
  o[4] = hxx;
  o[5] = hyy;
  o[6] = hzz;
  o[7] = hxy;
  o[8] = hxz;
  o[9] = hyz;
  float* qo = a.qout + size_t(ci.w) * 8;
  qo[4] = tx;
  qo[5] = ty;
  qo[6] = tz;
}

}  // namespace

int launch_pair_quad(pme_plan_t p, cudaStream_t s, int n, const float* theta, float* out, float* qout) {
  if (p->batch) return set_error(p, PME_ERR_UNSUPPORTED, "quadrupoles need a single-frame plan");
  if (n <= 0) return PME_OK;
  QuadPairArgs a;
  a.g = p->g;
  a.pr = p->pr;
  a.start_c = p->sb.start_c;
  a.theta = theta;
  a.out = out;
  a.qout = qout;
  a.n = n;
  a.cell_off = p->frames_h[0].cell_off;
  a.alpha = float(p->alpha);
  const double al = p->alpha;
  for (int l = 0; l < 6; ++l) a.c[l] = float(std::pow(2.0 * al * al, l) / (al * std::sqrt(kPi)));
  const int grid = (n + kQuadThreads - 1) / kQuadThreads;
  k_pair_quad<<<grid, kQuadThreads, 0, s>>>(a);
  count_launch();
  return check_launch(p, "k_pair_quad");
}

}  // namespace gbpme
