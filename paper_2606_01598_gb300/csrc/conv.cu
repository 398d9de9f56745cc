// Mesh convolution by hand-written transforms (Sections 2.3.3-2.3.4, Eqs. potential_k,
// energy_recip): the R2C transform of every rho (and d rho), the influence multiply with the
// reciprocal energy, and the C2R transform back to Phi (and d Phi), in three passes.
//
//   pass A (k_conv_r2c), one CTA per x-plane of a mesh (several consecutive planes when they
//     are small, transformed together as more lines): the plane's real rows are packed two
//     to a complex row (row 2p as real part, row 2p+1 as imaginary part), transformed along
//     z, separated into the two half spectra (X_k = (Z_k + conj Z_{N-k}) / 2 and
//     Y_k = (Z_k - conj Z_{N-k}) / 2i), transformed along y and stored as plane x of the
//     [Nx][Ny][Nz/2+1] spectrum.
//   pass B (k_conv_x), one CTA per run of C consecutive (n_y, n_z) columns of a frame (for a
//     fixed x they are contiguous in the spectrum; C grows for short x axes so that a tile
//     holds at least 1024 points): transform along x, the influence multiply G C / V of every
//     point with the energy (and virial) sums of the stand-alone influence pass, inverse
//     transform along x. The backward's tangent spectrum rides in the same CTA as extra
//     columns.
//   pass C (k_conv_c2r), one CTA per x-plane (or several): inverse along y, Hermitian extension of each
//     pair of half rows into one complex row, inverse along z, real and imaginary parts
//     stored as two rows of Phi.
//
// The 1D transforms are Stockham autosort FFTs (self-sorting, no bit reversal) of mixed radix
// 8, 4, 2, 3 and 5 in shared memory, in the formulation of Govindaraju et al. (SC 2008): a
// stage of radix R reads its R inputs at stride L/R, applies the twiddles w^(r (j mod Ns)),
// takes an R-point DFT and writes the outputs at stride Ns. All lines of a plane or tile go
// through a stage together, consecutive threads on consecutive lines (row lines are stored
// with an odd stride, so a warp's accesses fall in distinct banks). Twiddles come from
// host-built tables of e^(-2 pi i k / L) (float64 on the host, stored as float32). Global
// loads are issued kLoadBatch at a time per thread before their shared-memory stores, so a
// thread waits for one round trip per batch. Layout and normalisation are those of the usual
// unnormalised R2C / C2R pair, so the spectrum, the energy partials and Phi are laid out as
// with a library transform. Every axis must be 2,3,5-smooth and at most kConvMaxLen long and
// a plane must fit in shared memory; other meshes go through cuFFT.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kConvMinCols = 16;         // narrowest pass-B tile (columns)
constexpr int kConvMaxCols = 64;         // widest pass-B tile
constexpr int kConvBThreads = 256;
constexpr int kConvPlaneThreads = 1024;  // upper bound of the pass A / C block size
constexpr int kLoadBatch = 8;            // global loads a thread keeps in flight
constexpr size_t kConvPlaneTarget = 4096;  // small planes are grouped up to this many entries

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// times -i (forward transform) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// R-point DFTs in place, X_k = sum_n v_n e^(-+2 pi i n k / R) (minus: forward).
template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = rot<INV>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // radix-2 split: even and odd 4-point DFTs, odd outputs times w8^k
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    const float h = 0.70710678118654752f;   // cos(pi / 4)
    o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y)) : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
    o2 = rot<INV>(o2);
    o3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  } else if constexpr (R == 3) {
    const float c = -0.5f, s = 0.86602540378443865f;   // cos, sin of 2 pi / 3
    const float2 a = v[0], sm = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 m = make_float2(a.x + c * sm.x, a.y + c * sm.y);
    const float2 isd = make_float2(-s * d.y, s * d.x);   // i s d
    v[0] = cadd(a, sm);
    v[1] = INV ? cadd(m, isd) : csub(m, isd);
    v[2] = INV ? csub(m, isd) : cadd(m, isd);
  } else {   // R == 5
    const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos 2pi/5, cos 4pi/5
    const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin 2pi/5, sin 4pi/5
    const float2 a = v[0];
    const float2 s14 = cadd(v[1], v[4]), d14 = csub(v[1], v[4]);
    const float2 s23 = cadd(v[2], v[3]), d23 = csub(v[2], v[3]);
    const float2 m1 = make_float2(a.x + c1 * s14.x + c2 * s23.x, a.y + c1 * s14.y + c2 * s23.y);
    const float2 m2 = make_float2(a.x + c2 * s14.x + c1 * s23.x, a.y + c2 * s14.y + c1 * s23.y);
    const float2 n1 = make_float2(s1 * d14.x + s2 * d23.x, s1 * d14.y + s2 * d23.y);
    const float2 n2 = make_float2(s2 * d14.x - s1 * d23.x, s2 * d14.y - s1 * d23.y);
    const float2 in1 = make_float2(-n1.y, n1.x), in2 = make_float2(-n2.y, n2.x);   // i n
    v[0] = cadd(a, cadd(s14, s23));
    v[1] = INV ? cadd(m1, in1) : csub(m1, in1);
    v[4] = INV ? csub(m1, in1) : cadd(m1, in1);
    v[2] = INV ? cadd(m2, in2) : csub(m2, in2);
    v[3] = INV ? csub(m2, in2) : cadd(m2, in2);
  }
}

// Radix of the next stage for a remaining length m (2,3,5-smooth): 8 while it divides m,
// except that 16 goes as 4 x 4 (no radix-2 stage unless the power of two is 2).
__host__ __device__ __forceinline__ int next_radix(int m) {
  if (m % 8 == 0 && m % 32 != 16) return 8;
  if (m % 4 == 0) return 4;
  if (m % 2 == 0) return 2;
  if (m % 3 == 0) return 3;
  return 5;
}

// One Stockham stage of radix R over nl lines of length L: element k of line l sits at
// in[l * ls + k * es] (the output uses the same layout). Ns = product of the radices of the
// stages before. Thread t takes line t mod nl of butterfly t / nl.
template <int R, bool INV>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ in, float2* __restrict__ out, int L,
                                          int Ns, int nl, int ls, int es, const float2* __restrict__ tw) {
  const int nb = L / R;
  const int total = nl * nb;
  const int tstep = L / (Ns * R);
  const float rNs = 1.f / float(Ns);   // j / Ns = floor((j + 0.5) / Ns), exact for j, Ns < 2^12
  const int NT = blockDim.x;
  int l = threadIdx.x % nl, j = threadIdx.x / nl;
  const int dl = NT % nl, dj = NT / nl;
  for (int t = threadIdx.x; t < total; t += NT) {
    const int q = int((float(j) + 0.5f) * rNs);
    const int jm = j - q * Ns;
    const float2* src = in + l * ls + j * es;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[r * nb * es];
    const int tb = jm * tstep;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[r * tb];
      if (INV) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
    dft<R, INV>(v);
    float2* dst = out + l * ls + (q * Ns * R + jm) * es;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns * es] = v[r];
    l += dl;
    j += dj;
    if (l >= nl) {
      l -= nl;
      ++j;
    }
  }
}

// Full 1D transform of nl lines, ping-ponging between a and b; returns the buffer holding
// the result (the other one is free). Ends with a barrier.
template <bool INV>
__device__ float2* fft_lines(float2* a, float2* b, int L, int nl, int ls, int es, const float2* tw) {
  for (int Ns = 1; Ns < L;) {
    const int R = next_radix(L / Ns);
    switch (R) {
      case 8: fft_stage<8, INV>(a, b, L, Ns, nl, ls, es, tw); break;
      case 4: fft_stage<4, INV>(a, b, L, Ns, nl, ls, es, tw); break;
      case 2: fft_stage<2, INV>(a, b, L, Ns, nl, ls, es, tw); break;
      case 3: fft_stage<3, INV>(a, b, L, Ns, nl, ls, es, tw); break;
      default: fft_stage<5, INV>(a, b, L, Ns, nl, ls, es, tw); break;
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

__device__ __forceinline__ void comp_add(float& s, float& c, float v) {
  const float t = s + v;
  c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
  s = t;
}

// Block sum of per-thread compensated pairs: float within a warp, float64 across warps;
// thread 0 gets the total.
__device__ double block_comp_sum(float v, float c, double* wsum) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    c += c2;
    comp_add(v, c, v2);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = double(v) + double(c);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += wsum[w];
  return t;
}

// element t of a tile with c columns: row t / c, column t mod c. The float quotient is off
// by at most one for t < 2^20, which the correction absorbs.
__device__ __forceinline__ void split_rc(int t, int c, float rc, int& row, int& col) {
  row = int((float(t) + 0.5f) * rc);
  col = t - row * c;
  if (col < 0) {
    --row;
    col += c;
  } else if (col >= c) {
    ++row;
    col -= c;
  }
}

struct ConvArgs {
  FrameDesc one;
  FrameMaps maps;
  const int2* planes;   // batched pass A / C: block -> (frame, plane index of the frame)
  const float2* tw;     // twiddle tables
  float* mesh;          // pass A: rho base (input); pass C: Phi base (output)
  float2* spec;
  int tangent;
  int cap;              // complex entries of each plane buffer (pass A / C)
  const float* dconv;
  float inv4a2;
  double* partials;
  double* vparts;
  const float* gtab;
  const int* keep;      // tangent passes: *keep == 0 skips rho / Phi (the forward's stay)
};

// Plane buffers of pass A / C: twiddles of z and y, then two buffers of cap entries.
__device__ __forceinline__ void plane_setup(const ConvArgs& a, const FrameDesc& F, float2* sm, float2*& twz,
                                            float2*& twy, float2*& b0, float2*& b1) {
  const int Ny = F.g.N[1], Nz = F.g.N[2];
  twz = sm;
  twy = sm + Nz;
  b0 = sm + ((Nz + Ny + 1) & ~1);
  b1 = b0 + a.cap;
  for (int k = threadIdx.x; k < Nz; k += blockDim.x) twz[k] = a.tw[F.tw_off[2] + k];
  for (int k = threadIdx.x; k < Ny; k += blockDim.x) twy[k] = a.tw[F.tw_off[1] + k];
}

// Pass A / C block: frame, mesh copy (0: rho / Phi, 1: the tangent one), first plane x0 and
// plane count pc (F.conv_pp consecutive x-planes per block, fewer in the last one).
template <bool BATCH>
__device__ __forceinline__ const FrameDesc& plane_block(const ConvArgs& a, int& copy, int& x0, int& pc) {
  int f = 0, local = blockIdx.x;
  if (BATCH) {
    const int2 m = a.planes[blockIdx.x];
    f = m.x;
    local = m.y;
  }
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, f);
  const int Nx = F.g.N[0], P = F.conv_pp;
  const int per_copy = (Nx + P - 1) / P;
  copy = local >= per_copy ? 1 : 0;
  x0 = (local - copy * per_copy) * P;
  pc = min(P, Nx - x0);
  return F;
}

// Shared-memory layouts of a block's pc planes (np = ceil(Ny / 2) row pairs, Zs = Nz | 1):
//   Z: complex row pp of plane p at (p np + pp) Zs (rows 2pp, 2pp+1 as real, imaginary parts)
//   S: half spectrum entry (y, k) of plane p at y Sw + p Nzh + k, Sw = pc Nzh (the columns of
//      all planes side by side, so one transform along y covers them)
template <bool BATCH>
__global__ void __launch_bounds__(kConvPlaneThreads) k_conv_r2c(ConvArgs a) {
  pdl_begin();
  extern __shared__ __align__(16) float2 csm[];
  int copy, x0, pc;
  const FrameDesc& F = plane_block<BATCH>(a, copy, x0, pc);
  if (copy == 0 && a.keep && *a.keep == 0) return;   // rho's spectrum is not needed again
  const int Ny = F.g.N[1], Nz = F.g.N[2], Nzh = Nz / 2 + 1;
  float2 *twz, *twy, *b0, *b1;
  plane_setup(a, F, csm, twz, twy, b0, b1);
  const int np = (Ny + 1) >> 1, Zs = Nz | 1, Sw = pc * Nzh;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float rnz = 1.f / float(Nz), rny = 1.f / float(Ny), rnzh = 1.f / float(Nzh), rnp = 1.f / float(np);
  const float* src = a.mesh + (copy ? F.tmesh_off : F.mesh_off) + size_t(x0) * Ny * Nz;
  float* zf = reinterpret_cast<float*>(b0);
  {
    // the pc planes are contiguous in the mesh; kLoadBatch loads in flight per thread
    const int total = pc * Ny * Nz;
    for (int t0 = threadIdx.x; t0 < total; t0 += kLoadBatch * blockDim.x) {
      float v[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int t = t0 + u * blockDim.x;
        v[u] = t < total ? src[t] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < total) {
          int row, z, pl = 0, y;
          split_rc(t, Nz, rnz, row, z);
          if (pc > 1) split_rc(row, Ny, rny, pl, y);
          else y = row;
          zf[2 * ((pl * np + (y >> 1)) * Zs + z) + (y & 1)] = v[u];
        }
      }
    }
    if (Ny & 1)   // each plane's unpaired last row has a zero partner
      for (int t = threadIdx.x; t < pc * Nz; t += blockDim.x) {
        int pl, z;
        split_rc(t, Nz, rnz, pl, z);
        zf[2 * ((pl * np + (Ny >> 1)) * Zs + z) + 1] = 0.f;
      }
  }
  __syncthreads();
  float2* r = fft_lines<false>(b0, b1, Nz, pc * np, Zs, 1, twz);
  float2* o = r == b0 ? b1 : b0;
  // separate the two real rows' half spectra into S
  for (int line = wid; line < pc * np; line += nw) {
    int pl, pp;
    split_rc(line, np, rnp, pl, pp);
    const float2* zr = r + line * Zs;
    float2* s0 = o + 2 * pp * Sw + pl * Nzh;
    const bool has_b = 2 * pp + 1 < Ny;
    for (int k = lane; k < Nzh; k += 32) {
      const float2 zk = zr[k];
      const float2 zm = zr[k == 0 ? 0 : Nz - k];
      s0[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      if (has_b) s0[Sw + k] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
  }
  __syncthreads();
  const float2* sres = fft_lines<false>(o, r, Ny, Sw, 1, Sw, twy);
  // plane p's [ky][kz] block is contiguous in the spectrum, the pc planes one after another
  float2* dst = a.spec + (copy ? F.tspec_off : F.spec_off) + size_t(x0) * Ny * Nzh;
  if (pc == 1) {   // one plane: S is the plane's [ky][kz] block itself
    for (int t = threadIdx.x; t < Ny * Nzh; t += blockDim.x) dst[t] = sres[t];
  } else {
    for (int t = threadIdx.x; t < pc * Ny * Nzh; t += blockDim.x) {
      int row, k, pl, y;
      split_rc(t, Nzh, rnzh, row, k);
      split_rc(row, Ny, rny, pl, y);
      dst[t] = sres[y * Sw + pl * Nzh + k];
    }
  }
}

template <bool BATCH>
__global__ void __launch_bounds__(kConvPlaneThreads) k_conv_c2r(ConvArgs a) {
  pdl_begin();
  extern __shared__ __align__(16) float2 csm[];
  int copy, x0, pc;
  const FrameDesc& F = plane_block<BATCH>(a, copy, x0, pc);
  if (copy == 0 && a.keep && *a.keep == 0) return;   // the forward's Phi stays in place
  const int Ny = F.g.N[1], Nz = F.g.N[2], Nzh = Nz / 2 + 1;
  float2 *twz, *twy, *b0, *b1;
  plane_setup(a, F, csm, twz, twy, b0, b1);
  const int np = (Ny + 1) >> 1, Zs = Nz | 1, Sw = pc * Nzh;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float rny = 1.f / float(Ny), rnzh = 1.f / float(Nzh), rnp = 1.f / float(np);
  const float2* src = a.spec + (copy ? F.tspec_off : F.spec_off) + size_t(x0) * Ny * Nzh;
  const int total = pc * Ny * Nzh;
  for (int t0 = threadIdx.x; t0 < total; t0 += kLoadBatch * blockDim.x) {
    float2 v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t < total) v[u] = src[t];
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t < total) {
        if (pc == 1) {   // one plane: S is the plane's [ky][kz] block itself
          b0[t] = v[u];
        } else {
          int row, k, pl, y;
          split_rc(t, Nzh, rnzh, row, k);
          split_rc(row, Ny, rny, pl, y);
          b0[y * Sw + pl * Nzh + k] = v[u];
        }
      }
    }
  }
  __syncthreads();
  float2* s = fft_lines<true>(b0, b1, Ny, Sw, 1, Sw, twy);
  float2* o = s == b0 ? b1 : b0;
  // complex row (p, pp) = (half row 2pp) + i (half row 2pp+1), extended by Hermitian symmetry;
  // the n_z = 0 and Nyquist entries of a real row's spectrum are real
  for (int line = wid; line < pc * np; line += nw) {
    int pl, pp;
    split_rc(line, np, rnp, pl, pp);
    const float2* ra = s + 2 * pp * Sw + pl * Nzh;
    const float2* rb = ra + Sw;
    const bool has_b = 2 * pp + 1 < Ny;
    float2* zr = o + line * Zs;
    for (int k = lane; k < Nz; k += 32) {
      float2 A, B = make_float2(0.f, 0.f);
      if (k < Nzh) {
        A = ra[k];
        if (has_b) B = rb[k];
        if (k == 0 || 2 * k == Nz) {
          A.y = 0.f;
          B.y = 0.f;
        }
      } else {
        A = ra[Nz - k];
        A.y = -A.y;
        if (has_b) {
          B = rb[Nz - k];
          B.y = -B.y;
        }
      }
      zr[k] = make_float2(A.x - B.y, A.y + B.x);
    }
  }
  __syncthreads();
  const float2* z = fft_lines<true>(o, s, Nz, pc * np, Zs, 1, twz);
  const float* zf = reinterpret_cast<const float*>(z);
  float* dst = a.mesh + (copy ? F.tmesh_off : F.mesh_off) + size_t(x0) * Ny * Nz;
  for (int row = wid; row < pc * Ny; row += nw) {
    int pl = 0, y = row;
    if (pc > 1) split_rc(row, Ny, rny, pl, y);
    const float* zr = zf + 2 * (pl * np + (y >> 1)) * Zs + (y & 1);
    float* dr = dst + size_t(row) * Nz;
    for (int k = lane; k < Nz; k += 32) dr[k] = zr[2 * k];
  }
}

template <bool BATCH, bool VIR>
__global__ void __launch_bounds__(kConvBThreads) k_conv_x(ConvArgs a) {
  pdl_begin();
  extern __shared__ __align__(16) float2 csm[];
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, BATCH ? a.maps.blk_frame[blockIdx.x] : 0);
  const Geometry& g = F.g;
  const int N0 = g.N[0], N1 = g.N[1], N2 = g.N[2], Nzh = N2 / 2 + 1;
  const int ncols = N1 * Nzh;   // (n_y, n_z) columns of a plane, contiguous for a fixed x
  const int c0 = (blockIdx.x - F.infl_blk_off) * F.conv_cols;
  const int kw = min(F.conv_cols, ncols - c0);
  // tangent pass on the forward's inputs: rho's columns are not needed again
  const bool rho_cols = !(a.tangent && a.keep && *a.keep == 0);
  const int nrho = rho_cols ? kw : 0;
  const int nc = a.tangent ? nrho + kw : kw;
  const float rnc = 1.f / float(nc), rkw = 1.f / float(kw), rzh = 1.f / float(Nzh);
  float2* tw = csm;
  float2* b0 = csm + ((N0 + 1) & ~1);
  float2* b1 = b0 + N0 * nc;
  for (int k = threadIdx.x; k < N0; k += blockDim.x) tw[k] = a.tw[F.tw_off[0] + k];
  float2* sp = a.spec + F.spec_off + c0;
  float2* tp = a.spec + F.tspec_off + c0;
  // tile [x][c]: columns [0, kw) of the spectrum, then (tangent) [kw, 2 kw) of the tangent one
  for (int t0 = threadIdx.x; t0 < N0 * nc; t0 += kLoadBatch * blockDim.x) {
    float2 v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t < N0 * nc) {
        int x, c;
        split_rc(t, nc, rnc, x, c);
        v[u] = c < nrho ? sp[size_t(x) * ncols + c] : tp[size_t(x) * ncols + c - nrho];
      }
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int t = t0 + u * blockDim.x;
      if (t < N0 * nc) b0[t] = v[u];
    }
  }
  __syncthreads();
  float2* r = fft_lines<false>(b0, b1, N0, nc, 1, nc, tw);
  const float* cx = a.dconv + F.dconv_off;
  const float* cy = cx + N0;
  const float* cz = cy + N1;
  const float four_pi = 12.566370614359172f;
  float e = 0.f, ec = 0.f;
  float sv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, sc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int t = threadIdx.x; t < N0 * kw; t += blockDim.x) {
    int ix, c, iy, iz;
    split_rc(t, kw, rkw, ix, c);
    split_rc(c0 + c, Nzh, rzh, iy, iz);
    const float nx = float(ix <= N0 / 2 ? ix : ix - N0);
    const float ny = float(iy <= N1 / 2 ? iy : iy - N1);
    const float nz = float(iz);
    const float kx = nx * g.bk[0] + ny * g.bk[3] + nz * g.bk[6];
    const float kyv = nx * g.bk[1] + ny * g.bk[4] + nz * g.bk[7];
    const float kz = nx * g.bk[2] + ny * g.bk[5] + nz * g.bk[8];
    const float k2 = kx * kx + kyv * kyv + kz * kz;
    float gc = 0.f;
    if (a.gtab) gc = a.gtab[F.gtab_off + size_t(ix) * ncols + c0 + c];
    else if (k2 > 0.f) gc = four_pi * expf(-k2 * a.inv4a2) / k2 * cx[ix] * cy[iy] * cz[iz];
    float2* pv = r + ix * nc + c;
    const float fac = gc * g.inv_volume;
    if (!rho_cols) {   // tangent columns only; no energy
      const float2 u = *pv;
      *pv = make_float2(u.x * fac, u.y * fac);
      continue;
    }
    const float2 v = *pv;
    const float w = (iz == 0 || (2 * iz == N2)) ? 1.f : 2.f;
    const float eg = w * gc * (v.x * v.x + v.y * v.y);
    comp_add(e, ec, eg);
    if (VIR && k2 > 0.f) {
      const float tt = eg * (1.f / k2 + a.inv4a2);
      comp_add(sv[0], sc[0], tt * kx * kx);
      comp_add(sv[1], sc[1], tt * kyv * kyv);
      comp_add(sv[2], sc[2], tt * kz * kz);
      comp_add(sv[3], sc[3], tt * kx * kyv);
      comp_add(sv[4], sc[4], tt * kx * kz);
      comp_add(sv[5], sc[5], tt * kyv * kz);
    }
    *pv = make_float2(v.x * fac, v.y * fac);
    if (a.tangent) {
      const float2 u = pv[kw];
      pv[kw] = make_float2(u.x * fac, u.y * fac);
    }
  }
  __syncthreads();
  float2* o = fft_lines<true>(r, r == b0 ? b1 : b0, N0, nc, 1, nc, tw);
  for (int t = threadIdx.x; t < N0 * nc; t += blockDim.x) {
    int x, c;
    split_rc(t, nc, rnc, x, c);
    if (c < nrho) sp[size_t(x) * ncols + c] = o[t];
    else tp[size_t(x) * ncols + c - nrho] = o[t];
  }
  __shared__ double wsum[kConvBThreads / 32];
  const double et = block_comp_sum(e, ec, wsum);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = et;
  if (VIR) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double vt = block_comp_sum(sv[c], sc[c], wsum);
      if (threadIdx.x == 0) a.vparts[6 * blockIdx.x + c] = vt;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Power-of-two path: meshes whose every axis is 64 or 128 points. The same three passes, the
// same layouts and the same energy (and virial) partials per pass-B block as the kernels
// above, but each 1D transform of length L = 8 B (B = 8 or 16) is the four-step split of
// Bailey (J. Supercomputing 4, 1990) done in registers with one shared-memory exchange:
//   step 1, for each t < B: the 8-point DFT over m of x[t + B m], times w_L^(t k1), written
//           to slot t + B k1;
//   step 2, for each k1 < 8: the B-point DFT over t of slots t + B k1, which is X[k1 + 8 k2].
// The loads from global memory feed step 1 of the first transform of a pass directly, and
// step 2 of its last transform stores to global memory directly; the real-pair separation of
// the R2C (and the Hermitian extension of the C2R) is folded into the loads of the y (z) step
// 1, and the influence multiply into the forward x step 2. A pass is four steps with three
// barriers. Lengths, strides and index arithmetic are compile-time constants; the twiddles
// w_L^j are read from the plan's table (float64-built) through the read-only cache.
// ---------------------------------------------------------------------------------------
constexpr int kP2PlaneThreads = 1024;

// 16-point DFT in registers: 4 x 4 with the twiddles w16^(n1 k1) between the two radix-4
// steps; output in natural order.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  float2 t[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 a0 = v[n1], a1 = v[n1 + 4], a2 = v[n1 + 8], a3 = v[n1 + 12];
    dft4<INV>(a0, a1, a2, a3);
    t[n1][0] = a0;
    t[n1][1] = a1;
    t[n1][2] = a2;
    t[n1][3] = a3;
  }
  // forward twiddles w16^j = (cos, -sin)(2 pi j / 16); the inverse takes their conjugates
  const float sg = INV ? -1.f : 1.f;
  auto tw = [&](float2 a, float wr, float wi) {   // a (wr + i sg wi)
    const float wj = sg * wi;
    return make_float2(a.x * wr - a.y * wj, a.x * wj + a.y * wr);
  };
  t[1][1] = tw(t[1][1], c1, -s1);   // j = 1
  t[1][2] = tw(t[1][2], h, -h);     // j = 2
  t[1][3] = tw(t[1][3], s1, -c1);   // j = 3
  t[2][1] = tw(t[2][1], h, -h);     // j = 2
  t[2][2] = rot<INV>(t[2][2]);      // j = 4
  t[2][3] = tw(t[2][3], -h, -h);    // j = 6
  t[3][1] = tw(t[3][1], s1, -c1);   // j = 3
  t[3][2] = tw(t[3][2], -h, -h);    // j = 6
  t[3][3] = tw(t[3][3], -c1, s1);   // j = 9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 b0 = t[0][k1], b1 = t[1][k1], b2 = t[2][k1], b3 = t[3][k1];
    dft4<INV>(b0, b1, b2, b3);
    v[k1] = b0;
    v[k1 + 4] = b1;
    v[k1 + 8] = b2;
    v[k1 + 12] = b3;
  }
}

template <int B, bool INV>
__device__ __forceinline__ void dft_b(float2 (&u)[B]) {
  if constexpr (B == 16) dft16<INV>(u);
  else dft<B, INV>(u);
}

// step 1 on v[m] = x[t + B m]: the 8-point DFT and the twiddles w_L^(t k1) (tw: forward table)
template <bool INV>
__device__ __forceinline__ void p2_step1(float2 (&v)[8], int t, const float2* __restrict__ tw) {
  dft<8, INV>(v);
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    float2 w = __ldg(tw + t * k);
    if (INV) w.y = -w.y;
    v[k] = cmul(v[k], w);
  }
}

// Shared-memory float2 entries of one pass A / C plane block: the padded row lines Z
// [NY / 2][NZ + 8] (slot p of a line at p + p / BZ) and a second buffer of the same size
// (A: the z spectra in natural order; C: the half spectra after the y transform), with the
// y-step buffer [NY][NZ / 2 + 1] sharing the first one.
template <int NY, int NZ>
constexpr int p2_plane_entries() {
  return 2 * (NY / 2) * (NZ + 8);
}

template <int NY, int NZ>
__device__ __forceinline__ void r2c_plane_p2(const float* __restrict__ src, float2* __restrict__ dst,
                                             const float2* __restrict__ tz, const float2* __restrict__ ty,
                                             float2* sm) {
  constexpr int NP = NY / 2, LS = NZ + 8, NZH = NZ / 2 + 1, BZ = NZ / 8, BY = NY / 8;
  static_assert(NY * NZH <= NP * LS, "the y buffer fits in the row buffer");
  static_assert(NP * BZ <= kP2PlaneThreads && NP * 8 <= kP2PlaneThreads && NZH * 8 <= kP2PlaneThreads,
                "steps 1 (z) and 2 hold one item per thread");
  float2* Z = sm;              // z step 1 output (padded); then the y step 1 output S [NY][NZH]
  float2* Z2 = sm + NP * LS;   // z spectra, natural order, row stride LS
  float2* S = Z;
  const int tid = threadIdx.x;
  // z step 1: complex row p = rows 2p (real) and 2p + 1 (imaginary), read from global memory
  if (tid < NP * BZ) {
    const int pr = tid / BZ, t = tid - pr * BZ;
    const float* r0 = src + (2 * pr) * NZ + t;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = make_float2(r0[BZ * m], r0[NZ + BZ * m]);
    p2_step1<false>(v, t, tz);
#pragma unroll
    for (int k = 0; k < 8; ++k) Z[pr * LS + t + BZ * k + k] = v[k];
  }
  __syncthreads();
  // z step 2
  if (tid < NP * 8) {
    const int pr = tid >> 3, k1 = tid & 7;
    float2 u[BZ];
#pragma unroll
    for (int t = 0; t < BZ; ++t) u[t] = Z[pr * LS + t + (BZ + 1) * k1];
    dft_b<BZ, false>(u);
#pragma unroll
    for (int k2 = 0; k2 < BZ; ++k2) Z2[pr * LS + k1 + 8 * k2] = u[k2];
  }
  __syncthreads();
  // y step 1 on the real rows' half spectra: row 2p is (Z_k + conj Z_{N-k}) / 2, row 2p + 1
  // is (Z_k - conj Z_{N-k}) / 2i, with Z the spectrum of complex row p
  for (int it = tid; it < BY * NZH; it += blockDim.x) {
    const int t = it / NZH, kz = it - t * NZH;
    const int km = (NZ - kz) & (NZ - 1);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int y = t + BY * m;
      const float2 zk = Z2[(y >> 1) * LS + kz], zm = Z2[(y >> 1) * LS + km];
      v[m] = (y & 1) ? make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x))
                     : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    }
    p2_step1<false>(v, t, ty);
#pragma unroll
    for (int k = 0; k < 8; ++k) S[(t + BY * k) * NZH + kz] = v[k];
  }
  __syncthreads();
  // y step 2, straight to the plane's [ky][kz] block of the spectrum
  if (tid < 8 * NZH) {
    const int k1 = tid / NZH, kz = tid - k1 * NZH;
    float2 u[BY];
#pragma unroll
    for (int t = 0; t < BY; ++t) u[t] = S[(t + BY * k1) * NZH + kz];
    dft_b<BY, false>(u);
#pragma unroll
    for (int k2 = 0; k2 < BY; ++k2) dst[(k1 + 8 * k2) * NZH + kz] = u[k2];
  }
}

template <int NY, int NZ>
__device__ __forceinline__ void c2r_plane_p2(const float2* __restrict__ src, float* __restrict__ dst,
                                             const float2* __restrict__ tz, const float2* __restrict__ ty,
                                             float2* sm) {
  constexpr int NP = NY / 2, LS = NZ + 8, NZH = NZ / 2 + 1, BZ = NZ / 8, BY = NY / 8;
  float2* S = sm;              // y step 1 output [NY][NZH]; then the z step 1 output (padded)
  float2* S2 = sm + NP * LS;   // half spectra after the y transform [NY][NZH]
  float2* Z = S;
  const int tid = threadIdx.x;
  // y step 1, read from the plane's [ky][kz] block
  for (int it = tid; it < BY * NZH; it += blockDim.x) {
    const int t = it / NZH, kz = it - t * NZH;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = src[(t + BY * m) * NZH + kz];
    p2_step1<true>(v, t, ty);
#pragma unroll
    for (int k = 0; k < 8; ++k) S[(t + BY * k) * NZH + kz] = v[k];
  }
  __syncthreads();
  // y step 2
  if (tid < 8 * NZH) {
    const int k1 = tid / NZH, kz = tid - k1 * NZH;
    float2 u[BY];
#pragma unroll
    for (int t = 0; t < BY; ++t) u[t] = S[(t + BY * k1) * NZH + kz];
    dft_b<BY, true>(u);
#pragma unroll
    for (int k2 = 0; k2 < BY; ++k2) S2[(k1 + 8 * k2) * NZH + kz] = u[k2];
  }
  __syncthreads();
  // z step 1 on complex row p = (half row 2p) + i (half row 2p + 1), extended by Hermitian
  // symmetry (the n_z = 0 and Nyquist entries of a real row's spectrum are real)
  if (tid < NP * BZ) {
    const int pr = tid / BZ, t = tid - pr * BZ;
    const float2* ra = S2 + (2 * pr) * NZH;
    const float2* rb = ra + NZH;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + BZ * m;
      float2 A, Bv;
      if (k < NZH) {
        A = ra[k];
        Bv = rb[k];
        if (k == 0 || 2 * k == NZ) {
          A.y = 0.f;
          Bv.y = 0.f;
        }
      } else {
        A = ra[NZ - k];
        Bv = rb[NZ - k];
        A.y = -A.y;
        Bv.y = -Bv.y;
      }
      v[m] = make_float2(A.x - Bv.y, A.y + Bv.x);
    }
    p2_step1<true>(v, t, tz);
#pragma unroll
    for (int k = 0; k < 8; ++k) Z[pr * LS + t + BZ * k + k] = v[k];
  }
  __syncthreads();
  // z step 2: real parts to row 2p, imaginary parts to row 2p + 1
  if (tid < NP * 8) {
    const int pr = tid >> 3, k1 = tid & 7;
    float2 u[BZ];
#pragma unroll
    for (int t = 0; t < BZ; ++t) u[t] = Z[pr * LS + t + (BZ + 1) * k1];
    dft_b<BZ, true>(u);
    float* r0 = dst + (2 * pr) * NZ + k1;
#pragma unroll
    for (int k2 = 0; k2 < BZ; ++k2) {
      r0[8 * k2] = u[k2].x;
      r0[NZ + 8 * k2] = u[k2].y;
    }
  }
}

template <bool BATCH>
__global__ void __launch_bounds__(kP2PlaneThreads, 1) k_conv_r2c_p2(ConvArgs a) {
  pdl_begin();
  extern __shared__ __align__(16) float2 csm[];
  int copy, x0, pc;
  const FrameDesc& F = plane_block<BATCH>(a, copy, x0, pc);
  if (copy == 0 && a.keep && *a.keep == 0) return;   // rho's spectrum is not needed again
  const int Ny = F.g.N[1], Nz = F.g.N[2];
  const float* src = a.mesh + (copy ? F.tmesh_off : F.mesh_off) + size_t(x0) * Ny * Nz;
  float2* dst = a.spec + (copy ? F.tspec_off : F.spec_off) + size_t(x0) * Ny * (Nz / 2 + 1);
  const float2* tz = a.tw + F.tw_off[2];
  const float2* ty = a.tw + F.tw_off[1];
  if (Ny == 128 && Nz == 128) r2c_plane_p2<128, 128>(src, dst, tz, ty, csm);
  else if (Ny == 128) r2c_plane_p2<128, 64>(src, dst, tz, ty, csm);
  else if (Nz == 128) r2c_plane_p2<64, 128>(src, dst, tz, ty, csm);
  else r2c_plane_p2<64, 64>(src, dst, tz, ty, csm);
}

template <bool BATCH>
__global__ void __launch_bounds__(kP2PlaneThreads, 1) k_conv_c2r_p2(ConvArgs a) {
  pdl_begin();
  extern __shared__ __align__(16) float2 csm[];
  int copy, x0, pc;
  const FrameDesc& F = plane_block<BATCH>(a, copy, x0, pc);
  if (copy == 0 && a.keep && *a.keep == 0) return;   // the forward's Phi stays in place
  const int Ny = F.g.N[1], Nz = F.g.N[2];
  const float2* src = a.spec + (copy ? F.tspec_off : F.spec_off) + size_t(x0) * Ny * (Nz / 2 + 1);
  float* dst = a.mesh + (copy ? F.tmesh_off : F.mesh_off) + size_t(x0) * Ny * Nz;
  const float2* tz = a.tw + F.tw_off[2];
  const float2* ty = a.tw + F.tw_off[1];
  if (Ny == 128 && Nz == 128) c2r_plane_p2<128, 128>(src, dst, tz, ty, csm);
  else if (Ny == 128) c2r_plane_p2<128, 64>(src, dst, tz, ty, csm);
  else if (Nz == 128) c2r_plane_p2<64, 128>(src, dst, tz, ty, csm);
  else c2r_plane_p2<64, 64>(src, dst, tz, ty, csm);
}

// Pass B tile of NC columns (KW = 16 of the spectrum, then, in a tangent pass that also
// keeps rho's, the same 16 of the tangent spectrum): forward x transform, influence multiply
// with the energy (and virial) sums, inverse x transform. nrho = the leading rho columns.
constexpr int kP2Cols = 16;

template <int NX, int NC, bool VIR>
__device__ __forceinline__ void x_tile_p2(const ConvArgs& a, const FrameDesc& F, int c0, int nrho, float2* sm) {
  constexpr int BX = NX / 8;
  static_assert(NC * 8 <= kConvBThreads, "one step-2 item per thread");
  const Geometry& g = F.g;
  const int N1 = g.N[1], N2 = g.N[2], Nzh = N2 / 2 + 1;
  const int ncols = N1 * Nzh;
  float2* T = sm;             // step 1 outputs [x][c], row stride NC
  float2* T2 = sm + NX * NC;  // step 2 outputs
  const float2* tw = a.tw + F.tw_off[0];
  const int tid = threadIdx.x;
  // column c of the tile: spectrum column c0 + c (rho), or c0 + c - nrho of the tangent one
  auto col_ptr = [&](int c) { return c < nrho ? a.spec + F.spec_off + c0 + c : a.spec + F.tspec_off + c0 + (c - nrho); };
  // forward step 1 from global memory
  for (int it = tid; it < BX * NC; it += blockDim.x) {
    const int t = it / NC, c = it - t * NC;
    const float2* cp = col_ptr(c);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = cp[size_t(t + BX * m) * ncols];
    p2_step1<false>(v, t, tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) T[(t + BX * k) * NC + c] = v[k];
  }
  __syncthreads();
  // forward step 2, natural order into T2
  if (tid < 8 * NC) {
    const int k1 = tid / NC, c = tid - k1 * NC;
    float2 u[BX];
#pragma unroll
    for (int t = 0; t < BX; ++t) u[t] = T[(t + BX * k1) * NC + c];
    dft_b<BX, false>(u);
#pragma unroll
    for (int k2 = 0; k2 < BX; ++k2) T2[(k1 + 8 * k2) * NC + c] = u[k2];
  }
  __syncthreads();
  // inverse step 1, its inputs multiplied by G C / V first (the energy and virial sums over
  // the rho columns)
  float e = 0.f, ec = 0.f;
  float sv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, sc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float* cx = a.dconv + F.dconv_off;
  for (int it = tid; it < BX * NC; it += blockDim.x) {
    const int t = it / NC, c = it - t * NC;
    const bool rho_col = c < nrho;
    const int col = c0 + (rho_col ? c : c - nrho);
    int iy, iz;
    split_rc(col, Nzh, 1.f / float(Nzh), iy, iz);
    const float ny = float(iy <= N1 / 2 ? iy : iy - N1);
    const float nz = float(iz);
    const float wz = (iz == 0 || (2 * iz == N2)) ? 1.f : 2.f;
    float gcv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int ix = t + BX * m;
      gcv[m] = a.gtab ? __ldg(a.gtab + F.gtab_off + size_t(ix) * ncols + col) : 0.f;
    }
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int ix = t + BX * m;
      const float nx = float(ix <= NX / 2 ? ix : ix - NX);
      const float kx = nx * g.bk[0] + ny * g.bk[3] + nz * g.bk[6];
      const float kyv = nx * g.bk[1] + ny * g.bk[4] + nz * g.bk[7];
      const float kz = nx * g.bk[2] + ny * g.bk[5] + nz * g.bk[8];
      const float k2v = kx * kx + kyv * kyv + kz * kz;
      float gc = gcv[m];
      if (!a.gtab && k2v > 0.f)
        gc = 12.566370614359172f * expf(-k2v * a.inv4a2) / k2v * cx[ix] * cx[NX + iy] * cx[NX + N1 + iz];
      const float2 x = T2[ix * NC + c];
      if (rho_col) {
        const float eg = wz * gc * (x.x * x.x + x.y * x.y);
        comp_add(e, ec, eg);
        if (VIR && k2v > 0.f) {
          const float tt = eg * (1.f / k2v + a.inv4a2);
          comp_add(sv[0], sc[0], tt * kx * kx);
          comp_add(sv[1], sc[1], tt * kyv * kyv);
          comp_add(sv[2], sc[2], tt * kz * kz);
          comp_add(sv[3], sc[3], tt * kx * kyv);
          comp_add(sv[4], sc[4], tt * kx * kz);
          comp_add(sv[5], sc[5], tt * kyv * kz);
        }
      }
      const float fac = gc * g.inv_volume;
      v[m] = make_float2(x.x * fac, x.y * fac);
    }
    p2_step1<true>(v, t, tw);
#pragma unroll
    for (int k = 0; k < 8; ++k) T[(t + BX * k) * NC + c] = v[k];
  }
  __syncthreads();
  // inverse step 2, straight to the spectrum
  if (tid < 8 * NC) {
    const int k1 = tid / NC, c = tid - k1 * NC;
    float2 u[BX];
#pragma unroll
    for (int t = 0; t < BX; ++t) u[t] = T[(t + BX * k1) * NC + c];
    dft_b<BX, true>(u);
    float2* cp = col_ptr(c);
#pragma unroll
    for (int k2 = 0; k2 < BX; ++k2) cp[size_t(k1 + 8 * k2) * ncols] = u[k2];
  }
  __shared__ double wsum[kConvBThreads / 32];
  const double et = block_comp_sum(e, ec, wsum);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = et;
  if (VIR) {
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double vt = block_comp_sum(sv[c], sc[c], wsum);
      if (threadIdx.x == 0) a.vparts[6 * blockIdx.x + c] = vt;
    }
  }
}

template <bool BATCH, bool VIR>
__global__ void __launch_bounds__(kConvBThreads) k_conv_x_p2(ConvArgs a) {
  pdl_begin();
  extern __shared__ __align__(16) float2 csm[];
  const FrameDesc& F = frame_at<BATCH>(a.one, a.maps, BATCH ? a.maps.blk_frame[blockIdx.x] : 0);
  const int c0 = (blockIdx.x - F.infl_blk_off) * kP2Cols;
  // tangent pass on the forward's inputs: rho's columns are not needed again
  const bool rho_cols = !(a.tangent && a.keep && *a.keep == 0);
  const int nrho = rho_cols ? kP2Cols : 0;
  const bool two = a.tangent && rho_cols;
  if (F.g.N[0] == 128) {
    if (two) x_tile_p2<128, 2 * kP2Cols, VIR>(a, F, c0, nrho, csm);
    else x_tile_p2<128, kP2Cols, VIR>(a, F, c0, nrho, csm);
  } else {
    if (two) x_tile_p2<64, 2 * kP2Cols, VIR>(a, F, c0, nrho, csm);
    else x_tile_p2<64, kP2Cols, VIR>(a, F, c0, nrho, csm);
  }
}

ConvArgs conv_args(pme_plan_t p) {
  ConvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.one = p->frames_h[0];
  a.maps = p->maps;
  a.tw = p->conv_tw;
  a.cap = p->conv_cap;
  a.dconv = p->dconv_all;
  a.inv4a2 = float(1.0 / (4.0 * p->alpha * p->alpha));
  a.gtab = p->gtab;
  return a;
}

// The first launch of a kernel on a device raises its dynamic shared-memory limit to the
// device's opt-in maximum (one call per kernel and device; the launch's own size decides the
// occupancy). The plan checked its sizes against that maximum when it was made.
template <typename K>
int set_smem(pme_plan_t p, K kernel, unsigned& done_mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 32 && (done_mask & (1u << dev))) return PME_OK;
  int optin = 0;
  int st = check_cuda(p, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                      "cudaDeviceGetAttribute");
  if (st) return st;
  st = check_cuda(p, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024),
                  "cudaFuncSetAttribute");
  if (!st && dev < 32) done_mask |= 1u << dev;
  return st;
}

}  // namespace

bool conv_p2_ok(const int N[3]) {
  for (int a = 0; a < 3; ++a)
    if (N[a] != 64 && N[a] != 128) return false;
  return true;
}

size_t conv_p2_plane_smem(const int N[3]) {
  return size_t(2 * (N[1] / 2) * (N[2] + 8)) * sizeof(float2);
}

size_t conv_p2_x_smem(const int N[3]) { return size_t(2 * N[0] * 2 * kP2Cols) * sizeof(float2); }

bool conv_axis_ok(int L) {
  if (L < 1 || L > kConvMaxLen) return false;
  for (int f : {2, 3, 5})
    while (L % f == 0) L /= f;
  return L == 1;
}

void conv_tiles(const int N[3], int* ntile, int* cols) {
  int c = kConvMinCols;
  while (c < kConvMaxCols && N[0] * c < 1024) c *= 2;
  const int ncols = N[1] * (N[2] / 2 + 1);
  *cols = c;
  *ntile = (ncols + c - 1) / c;
}

// Complex entries of one plane in either layout.
static size_t plane_entries(const int N[3]) {
  const size_t np = size_t(N[1] + 1) / 2, Zs = size_t(N[2] | 1);
  return std::max(np * Zs, size_t(N[1]) * (N[2] / 2 + 1));
}

int conv_planes_per_block(const int N[3]) {
  const size_t e = plane_entries(N);
  const int p = int(std::max<size_t>(1, kConvPlaneTarget / e));
  return std::min(p, N[0]);
}

size_t conv_plane_cap(const int N[3]) { return conv_planes_per_block(N) * plane_entries(N); }

size_t conv_plane_smem(const int N[3], size_t cap) {
  return (size_t((N[1] + N[2] + 1) & ~1) + 2 * cap) * sizeof(float2);
}

size_t conv_x_smem(const int N[3]) {
  int nt, cols;
  conv_tiles(N, &nt, &cols);
  return (size_t((N[0] + 1) & ~1) + 2 * size_t(N[0]) * 2 * cols) * sizeof(float2);
}

void conv_twiddles(int L, std::vector<float2>& out) {
  for (int k = 0; k < L; ++k) {
    const double t = 2.0 * kPi * double(k) / double(L);
    out.push_back(make_float2(float(std::cos(t)), float(-std::sin(t))));
  }
}

int launch_conv_forward(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh, const int* keep) {
  ConvArgs a = conv_args(p);
  a.keep = tangent ? keep : nullptr;
  a.mesh = mesh;
  a.spec = reinterpret_cast<float2*>(p->spec);
  a.tangent = tangent ? 1 : 0;
  const FrameDesc& F0 = p->frames_h[0];
  const int grid = p->batch ? (tangent ? p->conv_nplanes2 : p->conv_nplanes1)
                            : (tangent ? 2 : 1) * ((F0.g.N[0] + F0.conv_pp - 1) / F0.conv_pp);
  a.planes = tangent ? p->conv_planes2 : p->conv_planes1;
  int st;
  if (p->conv_p2) {
    if (p->batch) {
      static unsigned done = 0;
      if ((st = set_smem(p, k_conv_r2c_p2<true>, done))) return st;
      pdl_launch(k_conv_r2c_p2<true>, grid, kP2PlaneThreads, p->conv_smem_plane, s, a);
    } else {
      static unsigned done = 0;
      if ((st = set_smem(p, k_conv_r2c_p2<false>, done))) return st;
      pdl_launch(k_conv_r2c_p2<false>, grid, kP2PlaneThreads, p->conv_smem_plane, s, a);
    }
    count_launch();
    return check_launch(p, "k_conv_r2c_p2");
  }
  if (p->batch) {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_r2c<true>, done))) return st;
    pdl_launch(k_conv_r2c<true>, grid, p->conv_threads, p->conv_smem_plane, s, a);
  } else {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_r2c<false>, done))) return st;
    pdl_launch(k_conv_r2c<false>, grid, p->conv_threads, p->conv_smem_plane, s, a);
  }
  count_launch();
  return check_launch(p, "k_conv_r2c");
}

int launch_conv_inverse(pme_plan_t p, cudaStream_t s, bool tangent, float* mesh, const int* keep) {
  ConvArgs a = conv_args(p);
  a.keep = tangent ? keep : nullptr;
  a.mesh = mesh;
  a.spec = reinterpret_cast<float2*>(p->spec);
  a.tangent = tangent ? 1 : 0;
  const FrameDesc& F0 = p->frames_h[0];
  const int grid = p->batch ? (tangent ? p->conv_nplanes2 : p->conv_nplanes1)
                            : (tangent ? 2 : 1) * ((F0.g.N[0] + F0.conv_pp - 1) / F0.conv_pp);
  a.planes = tangent ? p->conv_planes2 : p->conv_planes1;
  int st;
  if (p->conv_p2) {
    if (p->batch) {
      static unsigned done = 0;
      if ((st = set_smem(p, k_conv_c2r_p2<true>, done))) return st;
      pdl_launch(k_conv_c2r_p2<true>, grid, kP2PlaneThreads, p->conv_smem_plane, s, a);
    } else {
      static unsigned done = 0;
      if ((st = set_smem(p, k_conv_c2r_p2<false>, done))) return st;
      pdl_launch(k_conv_c2r_p2<false>, grid, kP2PlaneThreads, p->conv_smem_plane, s, a);
    }
    count_launch();
    return check_launch(p, "k_conv_c2r_p2");
  }
  if (p->batch) {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_c2r<true>, done))) return st;
    pdl_launch(k_conv_c2r<true>, grid, p->conv_threads, p->conv_smem_plane, s, a);
  } else {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_c2r<false>, done))) return st;
    pdl_launch(k_conv_c2r<false>, grid, p->conv_threads, p->conv_smem_plane, s, a);
  }
  count_launch();
  return check_launch(p, "k_conv_c2r");
}

int launch_conv_influence(pme_plan_t p, cudaStream_t s, bool tangent, double* partials, double* vparts,
                          const int* keep) {
  ConvArgs a = conv_args(p);
  a.keep = tangent ? keep : nullptr;
  a.spec = reinterpret_cast<float2*>(p->spec);
  a.tangent = tangent ? 1 : 0;
  a.partials = partials;
  a.vparts = vparts;
  const int grid = p->batch ? p->total_blocks : p->frames_h[0].infl_nblk;
  const size_t smem = p->conv_smem_x;
  int st;
#define GB_CONV_X(B, V)                                                  \
  do {                                                                   \
    static unsigned done = 0;                                            \
    if ((st = set_smem(p, k_conv_x<B, V>, done))) return st;             \
    pdl_launch(k_conv_x<B, V>, grid, kConvBThreads, smem, s, a);                 \
  } while (0)
#define GB_CONV_X_P2(B, V)                                               \
  do {                                                                   \
    static unsigned done = 0;                                            \
    if ((st = set_smem(p, k_conv_x_p2<B, V>, done))) return st;          \
    pdl_launch(k_conv_x_p2<B, V>, grid, kConvBThreads, smem, s, a);              \
  } while (0)
  if (p->conv_p2) {
    if (p->batch) {
      if (vparts) GB_CONV_X_P2(true, true);
      else GB_CONV_X_P2(true, false);
    } else {
      if (vparts) GB_CONV_X_P2(false, true);
      else GB_CONV_X_P2(false, false);
    }
    count_launch();
    return check_launch(p, "k_conv_x_p2");
  }
  if (p->batch) {
    if (vparts) GB_CONV_X(true, true);
    else GB_CONV_X(true, false);
  } else {
    if (vparts) GB_CONV_X(false, true);
    else GB_CONV_X(false, false);
  }
#undef GB_CONV_X
#undef GB_CONV_X_P2
  count_launch();
  return check_launch(p, "k_conv_x");
}

}  // namespace gbpme
