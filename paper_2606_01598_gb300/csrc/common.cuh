// Internal declarations of libgbpme: the plan, launch bookkeeping and device helpers that
// several kernels share (B-spline weights, mesh and cell coordinates, reductions).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/gbpme.h"

namespace gbpme {

constexpr int kMaxOrder = 7;
constexpr int kMaxCandPerDim = 4;   // bricks along one axis that can feed one brick's stencils
constexpr double kPi = 3.14159265358979323846;
constexpr int kProfCap = 4096;
// Ions per item of the per-frame sums (charges, energies): a frame of n ions is split into
// max(1, ceil(n / kRedItem)) items, one kRedItem-thread block each (one ion per thread).
constexpr int kRedItem = 128;

// ----------------------------------------------------------------------------------------
// launch bookkeeping
// ----------------------------------------------------------------------------------------
void count_launch();
// Streaming multiprocessors of the current device (queried once per device; grids of the
// grid-stride kernels are sized in multiples of it).
int device_sm_count();

// Programmatic dependent launch (sm_90 and later): a kernel launched with pdl_launch may be
// scheduled while the previous kernel of its stream is finishing; it must call pdl_begin()
// before touching global memory. pdl_begin waits until the preceding grids have completed and
// their memory is visible (griddepcontrol.wait), then lets the next grid be scheduled
// (griddepcontrol.launch_dependents), so consecutive kernels of a pass overlap only in their
// launch and scheduling, never in their memory accesses. Outside such a launch both are no-ops.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ----------------------------------------------------------------------------------------
// geometry shared by all kernels of one plan (passed by value)
// ----------------------------------------------------------------------------------------
struct Geometry {
  double cinv[9];   // C^{-1}, row-major: s_b = sum_a r_a cinv[a*3+b]
  float D[9];       // D[a*3+b] = N_b cinv[a*3+b]: d/dr_a = sum_b D[a][b] d/dx_b
  float H[9];       // pair cells: rows a_b / ncell_b, r = sum_b u_b H[b]
  int N[3];         // mesh
  int brick[3];     // brick edge per axis
  int nb[3];        // bricks per axis
  int ncell[3];     // pair cells per axis (1 = all images brute force along that axis)
  int kimg[3];      // neighbour cell / image range per axis
  int order;
  float alpha;
  float rcut2;
  double volume;
  float bk[9];        // reciprocal basis, rows b_r = 2 pi C^{-T}: bk[r*3+c] = 2 pi cinv[c*3+r]
  float inv_volume;   // 1 / V
  float bg_fac;       // pi / (V alpha^2), the background potential per unit net charge
  // energy coefficients (host float64, so that the last block of an energy sum divides nothing):
  // 1 / (2V) of the mesh sum, 4 pi / V of the explicit Ewald sum, pi / (2 V alpha^2) of the
  // background term -pi Q^2 / (2 V alpha^2)
  double e_mesh_coef, e_ewald_coef, e_bg_coef;
  // K = diag-scaled C^{-1} as float pairs hi + lo (K[a*3+b] = N_b cinv[a*3+b] for the mesh,
  // ncell_b cinv[a*3+b] for the pair cells): mesh and cell coordinates in compensated float32
  float kmh[9], kml[9], kch[9], kcl[9];
};

// Fill the compensated-float32 copies of N_b C^{-1} and ncell_b C^{-1} (after cinv, N, ncell).
inline void geometry_split(Geometry& g) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double km = double(g.N[b]) * g.cinv[a * 3 + b];
      const double kc = double(g.ncell[b]) * g.cinv[a * 3 + b];
      g.kmh[a * 3 + b] = float(km);
      g.kml[a * 3 + b] = float(km - double(float(km)));
      g.kch[a * 3 + b] = float(kc);
      g.kcl[a * 3 + b] = float(kc - double(float(kc)));
    }
}

// Per-ion records in brick (mesh) order.
struct MeshRecords {
  int4* idx;     // m0x, m0y, m0z (wrapped into [0,N)), original index
  float4* fq;    // fractional offsets fx, fy, fz in [0,1), q
  float4* dm;    // N_b (mu . C^{-1}_{:b}) for b = x,y,z ; w unused
  float4* tq;    // tangent: dq, projected d' = N_b((dmu + q dr) . C^{-1}_{:b})
  float4* tt;    // tangent: t = N_b (dr . C^{-1}_{:b}); w unused
};

// Per-ion records in pair-cell order.
struct PairRecords {
  int4* idx;     // cell x, y, z, original index
  float4* fq;    // offsets inside the cell in cell units fx, fy, fz in [0,1); w = cell z index
                 // (int bits), which gives a candidate's z offset inside a z-run
  float4* mu;    // mu (r-space), w = q
  float4* tq;    // tangent: dq, d' = dmu + q dr (r-space)
  float4* dr;    // tangent: dr (r-space); w unused
};

struct SortBuffers {
  int* key_b;     // [max_ions] global brick key per caller-order ion
  int* key_c;     // [max_ions] global pair cell key
  int* slot_b;    // [max_ions] arrival slot inside the brick
  int* slot_c;
  int* count_b;   // [total bricks + 1]
  int* count_c;   // [total cells + 1]
  int* start_b;   // [total bricks + 1] exclusive scan
  int* start_c;   // [total cells + 1]
  int* perm_b;    // [max_ions] unsorted placement (sorted slot -> caller index)
  int* perm_c;
  double* qpart;  // [2 * items] Q and dQ of each reduction item
  int* qcount;    // [frames] items finished (reset by the last one); null: no charge sums wanted
  // per-ion records formed by the binning pass in caller order (null: the rank pass forms
  // them itself), copied to their sorted slots by the rank pass
  int4* t_bidx;
  float4* t_bfq;
  float4* t_bdm;
  int4* t_cidx;
  float4* t_cfq;
  float4* t_cmu;
  double* qsum;   // [2 * frames] Q and dQ of each frame
};

// Division by an invariant divisor d >= 1 with a multiply-high and a shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", PLDI 1994): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, floor(x / d) = (umulhi(m, x) + x) >> l
// for 0 <= x < 2^31 (the sum cannot overflow there).
struct FastDiv {
  unsigned m;
  int l;
  int d;
};

inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((1ll << f.l) < d) ++f.l;
  f.m = unsigned(((1ull << 32) * ((1ull << f.l) - unsigned(d))) / unsigned(d) + 1ull);
  return f;
}

__device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  return int((__umulhi(f.m, unsigned(x)) + unsigned(x)) >> f.l);
}

// A pass (forward or backward) recorded as a CUDA graph: made on the second consecutive call
// with the same arguments, replayed while they stay the same. The key holds every pointer and
// size of the call and the host-side state the pass depends on; post_* is the host-side state
// the pass leaves behind.
struct PassKey {
  unsigned long long v[24];
  int len;
  bool operator==(const PassKey& o) const {
    if (len != o.len) return false;
    for (int k = 0; k < len; ++k)
      if (v[k] != o.v[k]) return false;
    return true;
  }
};

struct PassGraph {
  PassKey key;
  PassKey last;
  bool have_last;
  cudaGraphExec_t exec;
  long long launches;   // kernels per replay (for pme_launch_count)
  int post_fwd_n;
  bool post_fwd_lists;
};

// One frame of a plan: its geometry and where its data lives in the plan's arrays. A single-
// frame plan passes its one descriptor as a kernel argument; a batched plan keeps a table of
// them in device memory and maps ions / bricks / blocks to frames with the FrameMaps arrays.
struct FrameDesc {
  Geometry g;
  int ion_off, n;           // caller-order ion range
  int sorted_off;           // first position of the frame's ions in both sorted orders
  int brick_off, nbricks;   // global brick keys [brick_off, brick_off + nbricks)
  int cell_off, ncells;     // global pair-cell keys
  long long mesh_off;       // first float of rho / Phi
  long long tmesh_off;      // first float of d rho / d Phi (backward)
  long long spec_off;       // first complex of the spectrum
  long long tspec_off;      // first complex of the tangent spectrum
  long long gtab_off;       // first entry of the frame's P3M influence table
  int cand_off, max_nb;     // candidate-brick table [3][max_nb][1 + kMaxCandPerDim]
  int dconv_off;            // deconvolution tables: x at dconv_off, y at +Nx, z at +Nx+Ny
  int infl_blk_off, infl_nblk;  // influence / energy blocks of this frame
  int tw_off[3];            // hand-written transforms: twiddle tables of the x, y, z lengths
  int conv_cols;            // pass-B tile width in (n_y, n_z) columns
  int conv_pp;              // pass A / C: consecutive x-planes per block
  int item_off, nitems;     // items of the per-frame float64 sums
  FastDiv div_zh, div_y;    // division by Nz/2 + 1 and by Ny (half-spectrum index -> n)
};

struct FrameMaps {
  const FrameDesc* desc;    // [frames]
  const int* ion_frame;     // caller ion -> frame
  const int* sorted_frame;  // sorted position -> frame
  const int* brick_frame;   // global brick key -> frame
  const int* blk_frame;     // influence block -> frame
  const int* item_frame;    // reduction item -> frame
};

template <bool BATCH>
__device__ __forceinline__ const FrameDesc& frame_at(const FrameDesc& one, const FrameMaps& m, int f) {
  if constexpr (BATCH) return m.desc[f];
  else return one;
}

// Spread / gather launch range of one spline order: frames of that order own the contiguous
// global brick keys [brick_lo, brick_hi) and sorted ion positions [sorted_lo, sorted_hi).
struct OrderGroup {
  int order;
  int brick_lo, brick_hi;
  int sorted_lo, sorted_hi;
};

// Frames sharing one mesh shape and order, transformed by one batched cuFFT call: rho of the
// group's frames back to back, then their d rho (and likewise for spectra and potentials).
struct FFTGroup {
  int N[3];
  int count;
  long long mesh_off, spec_off;
  cufftHandle r2c, c2r, r2c2, c2r2;
};

}  // namespace gbpme

struct pme_plan_s {
  gbpme::Geometry g;         // geometry of frame 0 (single-frame plans)
  int nframes = 1;
  bool batch = false;
  gbpme::FrameDesc* frames_h = nullptr;   // [nframes] host copy
  gbpme::FrameDesc* frames_d = nullptr;   // [nframes] device table (batched plans)
  gbpme::FrameMaps maps = {};
  int* map_buf = nullptr;                 // device storage of the maps
  gbpme::OrderGroup ogroups[8];
  int nogroups = 0;
  gbpme::FFTGroup* fgroups = nullptr;
  // hand-written transforms (every axis 2,3,5-smooth and short enough): no cuFFT plans
  bool conv = false;
  bool conv_p2 = false;                    // every axis 64 or 128: the power-of-two kernels
  float2* conv_tw = nullptr;               // twiddle tables
  int2* conv_planes1 = nullptr;            // batched plans: pass A / C block -> (frame, plane)
  int2* conv_planes2 = nullptr;            //   the same with the tangent meshes
  int conv_nplanes1 = 0, conv_nplanes2 = 0;
  int conv_cap = 0, conv_threads = 0;
  size_t conv_smem_plane = 0, conv_smem_x = 0;
  int nfgroups = 0;
  void* fft_work = nullptr;
  double* e_ion = nullptr;                // [max_ions] per-ion energy contributions
  int total_bricks = 0, total_cells = 0, total_blocks = 0, total_items = 0;
  long long total_mesh = 0, total_spec = 0;
  int* frame_offsets = nullptr;           // host copy [nframes + 1]
  double box[9];             // box of frame 0
  double alpha, rcut;
  pme_opts opts;
  int M, Mh;                 // mesh / half-spectrum points of frame 0
  int max_ions;              // ions the buffers hold (batched plans: all frames)
  int device;
  // device scratch
  float* rho;                // meshes of every frame: rho at mesh_off, d rho at tmesh_off
  cufftComplex* spec;        // spectra (same layout with spec_off / tspec_off)
  float* phi;                // potential meshes (layout of rho)
  float* dconv_all;          // per-frame, per-axis deconvolution factors 1/sinc^(2 p gamma)
  float* gtab = nullptr;     // influence tables G C (or P3M), [half spectrum] per frame
  int* cand;                 // per-frame candidate-brick tables
  gbpme::SortBuffers sb;
  gbpme::MeshRecords mr;
  gbpme::PairRecords pr;
  float* mesh_out;           // [max_ions][10] per-ion mesh results (caller order)
  float* pair_out;           // [max_ions][10] per-ion pair results
  float* qb_mesh = nullptr;  // [max_ions][26] quadrupole backward: mesh values and tangents
  float* qb_pair = nullptr;  // [max_ions][26] the same for the pair term
  float* quad_out = nullptr; // [max_ions][8] quadrupole forward: Theta : grad^3 phi of the mesh
                             // (0..2) and of the pair term (4..6); single-frame plans
  double* epart;             // reciprocal energy partials, one per influence (or k) block
  double* eitem;             // [items] per-ion energy partials
  // pair lists recorded by the forward for a backward on the same positions
  float4* plist = nullptr;   // [max_ions][plist_cap] (r, j) per hit, pair-cell order
  int* plist_cnt = nullptr;  // [max_ions] hits per ion, -1 when more than plist_cap
  int plist_cap = 0;
  // inputs of the last forward, kept with its sorted order and records for the backward
  float* in_saved = nullptr;   // [7 max_ions]: positions, then q at 3 max_ions, mu at 4 max_ions
  int* in_flags = nullptr;     // [2]: in_diff, cache_bad (see launch_input_check)
  int* in_diff = nullptr;
  int* cache_bad = nullptr;
  bool counts_clean = false;   // the sort's count arrays are zero (each scan re-zeroes them)
  int fwd_n = -1;              // ions of that forward (-1: nothing saved / no longer valid)
  // virial partial sums
  double* vpart = nullptr;     // [6 * influence blocks] k-space sums S_ab
  float* pvir = nullptr;       // [max_ions][9] per-ion pair virial
  double* vitem = nullptr;     // [9 * items] per-item sums
  bool fwd_lists = false;      // that forward recorded the pair lists
  int* ecount;               // [frames] energy items finished (reset by the last one)
  int* flags;                // device error flags
  // host-pointer staging
  float* stage_f;            // device staging for host arrays, 40 floats per ion
  double* stage_d;           // [2 frames + 2]
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  std::string last_error;
  // explicit Ewald k-sum (recip_method = 1)
  double opts_kmax = 0.0;
  int ew_K = 0;
  int4* ew_kn = nullptr;      // [K] n vector, A(k) in .w
  float4* ew_kv = nullptr;    // [K] k vector
  float2* ew_S = nullptr;     // [K] structure factor
  uint4* ew_fx = nullptr;     // [max_ions] fixed-point fractional coordinates
  float4* ew_qm = nullptr;    // [max_ions] q, mu
  // CUDA graphs of repeated passes (0 forward, 1 backward)
  gbpme::PassGraph* graphs = nullptr;
  cudaStream_t cap_stream = nullptr;   // capture-only stream (nothing runs on it)
  // stage timers
  bool prof = false;
  cudaEvent_t* prof_ev = nullptr;   // [2 * kProfCap]
  int* prof_stage = nullptr;        // [kProfCap]
  int prof_used = 0;
};

namespace gbpme {

int set_error(pme_plan_t plan, int status, const std::string& what);
// Stage timer bracket: returns a slot (or -1 when timers are off or full).
int prof_begin(pme_plan_t plan, int stage, cudaStream_t s);
void prof_end(pme_plan_t plan, int slot, cudaStream_t s);
int check_cuda(pme_plan_t plan, cudaError_t e, const char* what);
int check_launch(pme_plan_t plan, const char* what);

// ----------------------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------------------

// Uniform cardinal B-spline weights. For the offset f in [0,1) of a mesh coordinate from its
// first stencil point m0 (x = m0 + P/2 - 1 + f), w[d][j] is the d-th derivative (d <= DMAX)
// of the centred spline W^(P) at t_j = x - (m0 + j). Built from the recursion
// N_k(y) = (y N_{k-1}(y) + (k - y) N_{k-1}(y - 1)) / (k - 1) on y = f + i, and
// d^d/dy^d N_P(y) = sum_s (-1)^s binom(d, s) N_{P-d}(y - s).
template <int P, int DMAX>
__device__ __forceinline__ void spline_weights(float f, float (&w)[DMAX + 1][P]) {
  float lv[DMAX + 1][P];   // lv[d][i] = N_{P-d}(f + i), zero when P - d < 1
  float b[P];              // running N_k(f + i)
#pragma unroll
  for (int d = 0; d <= DMAX; ++d)
#pragma unroll
    for (int i = 0; i < P; ++i) lv[d][i] = 0.f;
#pragma unroll
  for (int i = 0; i < P; ++i) b[i] = (i == 0) ? 1.f : 0.f;   // N_1(f + i), f in [0,1)
#pragma unroll
  for (int d = 0; d <= DMAX; ++d)
    if (P - d == 1) {
#pragma unroll
      for (int i = 0; i < P; ++i) lv[d][i] = b[i];
    }
#pragma unroll
  for (int k = 2; k <= P; ++k) {
    const float inv = 1.f / float(k - 1);
#pragma unroll
    for (int i = P - 1; i >= 0; --i) {
      if (i <= k - 1) {
        const float left = (i <= k - 2) ? b[i] : 0.f;
        const float right = (i >= 1) ? b[i - 1] : 0.f;
        b[i] = ((f + float(i)) * left + (float(k) - f - float(i)) * right) * inv;
      }
    }
#pragma unroll
    for (int d = 0; d <= DMAX; ++d)
      if (k == P - d) {
#pragma unroll
        for (int i = 0; i < P; ++i) lv[d][i] = b[i];
      }
  }
#pragma unroll
  for (int j = 0; j < P; ++j) {
    const int i = P - 1 - j;
    w[0][j] = lv[0][i];
    if constexpr (DMAX >= 1)
      w[1][j] = lv[1][i] - ((i >= 1) ? lv[1][i - 1] : 0.f);
    if constexpr (DMAX >= 2)
      w[2][j] = lv[2][i] - 2.f * ((i >= 1) ? lv[2][i - 1] : 0.f) + ((i >= 2) ? lv[2][i - 2] : 0.f);
    if constexpr (DMAX >= 3)
      w[3][j] = lv[3][i] - 3.f * ((i >= 1) ? lv[3][i - 1] : 0.f) +
                3.f * ((i >= 2) ? lv[3][i - 2] : 0.f) - ((i >= 3) ? lv[3][i - 3] : 0.f);
    if constexpr (DMAX >= 4)
      w[4][j] = lv[4][i] - 4.f * ((i >= 1) ? lv[4][i - 1] : 0.f) + 6.f * ((i >= 2) ? lv[4][i - 2] : 0.f) -
                4.f * ((i >= 3) ? lv[4][i - 3] : 0.f) + ((i >= 4) ? lv[4][i - 4] : 0.f);
  }
  static_assert(DMAX <= 4, "derivatives up to order 4");
}

// Fractional coordinate s = r C^{-1} wrapped into [0,1), in float64.
__device__ __forceinline__ void frac_coords(const Geometry& g, double rx, double ry, double rz,
                                            double s[3]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    double v = rx * g.cinv[0 * 3 + b] + ry * g.cinv[1 * 3 + b] + rz * g.cinv[2 * 3 + b];
    v -= floor(v);
    if (v >= 1.0) v -= 1.0;
    if (!(v >= 0.0)) v = 0.0;   // NaN guard; the caller flags non-finite inputs
    s[b] = v;
  }
}

// First stencil point m0 (wrapped) and offset f of mesh coordinate x = N s (Eq. w3d):
// m0 = floor(x - P/2) + 1, f = x - P/2 + 1 - floor(x - P/2 + 1).
__device__ __forceinline__ void stencil_origin(double s, int N, int order, int& m0, float& f) {
  const double y = s * double(N) - 0.5 * double(order) + 1.0;
  const double fl = floor(y);
  int m = int(fl);
  float fr = float(y - fl);
  if (fr >= 1.f) { fr = 0.f; m += 1; }   // keep the float offset inside [0,1)
  if (m < 0) m += N;
  if (m >= N) m -= N;
  m0 = m;
  f = fr;
}

// Scaled coordinate x_b = sum_a r_a K[a][b] (K = kh + kl) as hi + lo in float32: exact
// products by fused multiply-add error terms, the sum by the two-sum of Knuth (TAOCP vol. 2,
// 4.2.2), so x is carried to about 2^-45 of |x| -- the float64 result rounded to float32 within
// one unit in the last place -- without the float64 pipe.
__device__ __forceinline__ void scaled_coord(const float* kh, const float* kl, float rx, float ry, float rz,
                                             int b, float& hi, float& lo) {
  const float r[3] = {rx, ry, rz};
  float s = 0.f, e = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float k = kh[a * 3 + b];
    const float p = r[a] * k;
    const float pe = fmaf(r[a], k, -p);
    const float t = s + p;
    const float bb = t - s;
    const float te = (s - (t - bb)) + (p - bb);
    s = t;
    e += te + fmaf(r[a], kl[a * 3 + b], pe);
  }
  hi = s;
  lo = e;
}

// Integer part m and fraction f in [0,1) of hi + lo + c (c a multiple of 1/2); false when the
// value is not finite or too large for the float path (|hi| >= 2^22).
__device__ __forceinline__ bool split_coord(float hi, float lo, float c, int& m, float& f) {
  if (!(fabsf(hi) < 4194304.f) || !(fabsf(lo) < 1.f)) return false;
  const float yh = hi + c;
  const float bb = yh - hi;
  const float yl = lo + ((hi - (yh - bb)) + (c - bb));
  const float fl = floorf(yh);
  float fr = (yh - fl) + yl;
  int k = int(fl);
  if (fr < 0.f) {
    fr += 1.f;
    k -= 1;
  } else if (fr >= 1.f) {
    fr -= 1.f;
    k += 1;
  }
  if (fr >= 1.f) {
    fr = 0.f;
    k += 1;
  }
  m = k;
  f = fr;
  return true;
}

// First stencil point m0 (wrapped) and offset f along axis b from the position, in float32
// (stencil_origin of frac_coords' s to float32 rounding); false: use the float64 path.
__device__ __forceinline__ bool stencil_origin_f(const Geometry& g, float rx, float ry, float rz, int b, int& m0,
                                                 float& f) {
  float hi, lo;
  scaled_coord(g.kmh, g.kml, rx, ry, rz, b, hi, lo);
  int m;
  if (!split_coord(hi, lo, 1.f - 0.5f * float(g.order), m, f)) return false;
  const int N = g.N[b];
  m %= N;
  if (m < 0) m += N;
  m0 = m;
  return true;
}

// Pair cell and in-cell offset along axis b from the position, in float32; false: use the
// float64 path.
__device__ __forceinline__ bool cell_origin_f(const Geometry& g, float rx, float ry, float rz, int b, int& c,
                                              float& f) {
  float hi, lo;
  scaled_coord(g.kch, g.kcl, rx, ry, rz, b, hi, lo);
  int m;
  if (!split_coord(hi, lo, 0.f, m, f)) return false;
  const int nc = g.ncell[b];
  m %= nc;
  if (m < 0) m += nc;
  c = m;
  return true;
}

// Pair cell and in-cell offset of fractional coordinate s along one axis.
__device__ __forceinline__ void cell_origin(double s, int nc, int& c, float& f) {
  const double u = s * double(nc);
  double fl = floor(u);
  if (fl > double(nc - 1)) fl = double(nc - 1);
  if (fl < 0.0) fl = 0.0;
  c = int(fl);
  f = float(u - fl);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Largest butterfly offset of the second level of a block sum over nw warp partials held in
// lanes 0 .. nw-1 (zeros above): the levels at and above the smallest power of two >= nw only
// add zeros to those lanes, so the tree may start below it and still add the same terms in the
// same order as the full five-level tree.
__device__ __forceinline__ int partial_tree_top(int nw) {
  int o = 1;
  while (o < nw) o <<= 1;
  return o >> 1;
}

// Block-wide float64 sum (blockDim.x a multiple of 32, <= 1024). Result valid in thread 0.
__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = int(blockDim.x >> 5);
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) part[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < nw) ? part[lane] : 0.0;
    for (int o = partial_tree_top(nw); o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;
}

// Two block-wide float64 sums at once, each exactly as block_sum_d forms it; their shuffle
// trees are interleaved and share one pair of barriers (GB300's float64 latency makes two
// trees in sequence cost twice one). Results valid in thread 0.
__device__ __forceinline__ void block_sum2_d(double& a, double& b) {
  __shared__ double part2[2][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = int(blockDim.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if (lane == 0) {
    part2[0][wid] = a;
    part2[1][wid] = b;
  }
  __syncthreads();
  double ra = 0.0, rb = 0.0;
  if (wid == 0) {
    ra = (lane < nw) ? part2[0][lane] : 0.0;
    rb = (lane < nw) ? part2[1][lane] : 0.0;
    for (int o = partial_tree_top(nw); o > 0; o >>= 1) {
      ra += __shfl_xor_sync(0xffffffffu, ra, o);
      rb += __shfl_xor_sync(0xffffffffu, rb, o);
    }
  }
  a = ra;
  b = rb;
}

// Two-level deterministic sum, second level: after thread 0 has stored its block's partial,
// every thread calls this; it returns true in the block that finished last among the nitems
// blocks counting on *count (an atomic ticket). That block alone then adds all partials in
// item order (reading them with __ldcg) and resets *count, so the result does not depend on
// which block came last.
__device__ __forceinline__ bool last_item_done(int* count, int nitems) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(count, 1) == nitems - 1;
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// Sum of one float per thread over the block: Neumaier-compensated within each warp, float64
// across the warps; fixed order; valid in thread 0. (blockDim.x a multiple of 32, <= 1024)
__device__ __forceinline__ double block_sum_f(float v) {
  __shared__ double wpart[32];
  float c = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    const float t = v + v2;
    c += c2 + (fabsf(v) >= fabsf(v2) ? (v - t) + v2 : (v2 - t) + v);
    v = t;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = double(v) + double(c);
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < int(blockDim.x >> 5); ++w) r += wpart[w];
  return r;
}

// Two such sums at once, each exactly as block_sum_f forms it (interleaved trees, one pair of
// barriers). Results valid in thread 0.
__device__ __forceinline__ void block_sum2_f(float va, float vb, double& ra, double& rb) {
  __shared__ double wpart2[2][32];
  float ca = 0.f, cb = 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float a2 = __shfl_xor_sync(0xffffffffu, va, o), b2 = __shfl_xor_sync(0xffffffffu, vb, o);
    const float ca2 = __shfl_xor_sync(0xffffffffu, ca, o), cb2 = __shfl_xor_sync(0xffffffffu, cb, o);
    const float ta = va + a2, tb = vb + b2;
    ca += ca2 + (fabsf(va) >= fabsf(a2) ? (va - ta) + a2 : (a2 - ta) + va);
    cb += cb2 + (fabsf(vb) >= fabsf(b2) ? (vb - tb) + b2 : (b2 - tb) + vb);
    va = ta;
    vb = tb;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    wpart2[0][threadIdx.x >> 5] = double(va) + double(ca);
    wpart2[1][threadIdx.x >> 5] = double(vb) + double(cb);
  }
  __syncthreads();
  ra = 0.0;
  rb = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      ra += wpart2[0][w];
      rb += wpart2[1][w];
    }
}

// Sum of src[k * stride] over k = threadIdx.x, threadIdx.x + T, ... < n (T = blockDim.x): eight
// loads in flight at a time (the plain loop waits for each load before the next one), each
// round of eight added as a balanced tree (three dependent float64 adds, not eight) before it
// joins the running sum; a fixed order for a given n and block size. __ldcg reads partials
// other blocks wrote in the same launch.
__device__ __forceinline__ double strided_round(const double* src, int n, int stride, int k0, int T) {
  double v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) v[u] = (k0 + u * T < n) ? __ldcg(src + size_t(k0 + u * T) * stride) : 0.0;
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
}

__device__ __forceinline__ double strided_sum_d(const double* src, int n, int stride = 1) {
  double acc = 0.0;
  const int T = blockDim.x;
  for (int k0 = threadIdx.x; k0 < n; k0 += 8 * T) acc += strided_round(src, n, stride, k0, T);
  return acc;
}

// Two such sums at once (the loads of both in flight together); each equals what
// strided_sum_d returns for it.
__device__ __forceinline__ void strided_sum2_d(const double* a_src, int na, int sa, const double* b_src, int nb,
                                               int sb, double& a, double& b) {
  a = 0.0;
  b = 0.0;
  const int T = blockDim.x, n = max(na, nb);
  for (int k0 = threadIdx.x; k0 < n; k0 += 8 * T) {
    const double ra = strided_round(a_src, na, sa, k0, T);
    const double rb = strided_round(b_src, nb, sb, k0, T);
    if (k0 < na) a += ra;
    if (k0 < nb) b += rb;
  }
}

// Ion range [lo, hi) of reduction item `item` of frame F.
__device__ __forceinline__ void item_range(const FrameDesc& F, int item, int& lo, int& hi) {
  lo = F.ion_off + (item - F.item_off) * kRedItem;
  hi = min(F.ion_off + F.n, lo + kRedItem);
}

// Device error flag bits.
constexpr int kFlagNonFinite = 1;
constexpr int kFlagTimeout = 2;
constexpr int kFlagVirialLost = 4;   // a virial pass fell back to the fused pair kernel
constexpr int kFlagQuadLost = 16;    // a quadrupole backward found an overflowed pair-hit list

// ----------------------------------------------------------------------------------------
// index-checking build (compiled with -DGBPME_BOUNDS): index_ok(i, n) tests 0 <= i < n before
// a kernel touches element i of an array of n; a failed test records a bit in a device word of
// the translation unit and the access is skipped (no trap, no fault). Each translation unit
// provides a reader (GBPME_BOUNDS_READER) that returns and clears its word; in a normal build
// index_ok is always true and the readers return 0.
// ----------------------------------------------------------------------------------------
#ifdef GBPME_BOUNDS
namespace {
__device__ int g_bounds_hit;
}
__device__ __forceinline__ bool index_ok(long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicOr(&g_bounds_hit, 1);
  return false;
}
#define GBPME_BOUNDS_READER(fn)                                                   \
  int fn() {                                                                      \
    int v = 0;                                                                    \
    if (cudaMemcpyFromSymbol(&v, g_bounds_hit, sizeof(int)) != cudaSuccess) {    \
      cudaGetLastError();                                                         \
      return 0;                                                                   \
    }                                                                             \
    if (v) {                                                                      \
      const int z = 0;                                                            \
      cudaMemcpyToSymbol(g_bounds_hit, &z, sizeof(int));                          \
    }                                                                             \
    return v;                                                                     \
  }
#else
__device__ __forceinline__ bool index_ok(long long, long long) { return true; }
#define GBPME_BOUNDS_READER(fn) \
  int fn() { return 0; }
#endif
// readers of the translation units with checks (0 in normal builds)
int bounds_hit_spread();
int bounds_hit_spread_8x8x32();
int bounds_hit_spread_16x8x16();
int bounds_hit_spread_16x16x16();
int bounds_hit_spread_4x8x16();
int bounds_hit_gather();
int bounds_hit_pair();
int bounds_hit_combine();
int bounds_hit_sort();

}  // namespace gbpme
