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
  if (p->batch) {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_r2c<true>, done))) return st;
    k_conv_r2c<true><<<grid, p->conv_threads, p->conv_smem_plane, s>>>(a);
  } else {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_r2c<false>, done))) return st;
    k_conv_r2c<false><<<grid, p->conv_threads, p->conv_smem_plane, s>>>(a);
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
  if (p->batch) {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_c2r<true>, done))) return st;
    k_conv_c2r<true><<<grid, p->conv_threads, p->conv_smem_plane, s>>>(a);
  } else {
    static unsigned done = 0;
    if ((st = set_smem(p, k_conv_c2r<false>, done))) return st;
    k_conv_c2r<false><<<grid, p->conv_threads, p->conv_smem_plane, s>>>(a);
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
    k_conv_x<B, V><<<grid, kConvBThreads, smem, s>>>(a);                 \
  } while (0)
  if (p->batch) {
    if (vparts) GB_CONV_X(true, true);
    else GB_CONV_X(true, false);
  } else {
    if (vparts) GB_CONV_X(false, true);
    else GB_CONV_X(false, false);
  }
#undef GB_CONV_X
  count_launch();
  return check_launch(p, "k_conv_x");
}

}  // namespace gbpme
