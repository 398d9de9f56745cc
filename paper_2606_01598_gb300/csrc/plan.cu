// Plan construction (Section 2.3.1: cell, reciprocal basis, mesh; Section 2.3.3: the
// deconvolution tables), host-pointer staging, and the stream orchestration of the forward
// and backward passes behind the C ABI declared in include/gbpme.h.
//
// A plan holds one or more frames. A single-frame plan (pme_plan_create) passes its frame
// descriptor to every kernel as an argument; a batched plan (pme_batch_create) keeps a table
// of descriptors on the device plus maps from ions, bricks and influence blocks to frames,
// so each pipeline stage is one launch for the whole batch (spread and gather: one launch
// per spline order; FFT: one batched cuFFT call per distinct mesh shape).
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <initializer_list>
#include <new>
#include <numeric>
#include <vector>

#include "kernels.h"

namespace gbpme {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int set_error(pme_plan_t plan, int status, const std::string& what) {
  if (plan) plan->last_error = what;
  return status;
}

int check_cuda(pme_plan_t plan, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PME_OK;
  return set_error(plan, e == cudaErrorMemoryAllocation ? PME_ERR_NOMEM : PME_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

int check_launch(pme_plan_t plan, const char* what) {
  return check_cuda(plan, cudaGetLastError(), what);
}

// Stage names for the NVTX ranges that bracket each stage while the timers are on (visible
// in a timeline profiler; without one attached a range costs a few nanoseconds).
static const char* const kStageRange[PME_NUM_STAGES] = {
    "fwd.sort", "fwd.spread", "fwd.fft_r2c", "fwd.influence", "fwd.fft_c2r", "fwd.gather", "fwd.pair",
    "fwd.combine", "fwd.pair_eval", "bwd.sort", "bwd.spread", "bwd.fft_r2c", "bwd.influence",
    "bwd.fft_c2r", "bwd.gather", "bwd.pair", "bwd.combine", "bwd.pair_eval"};

int prof_begin(pme_plan_t p, int stage, cudaStream_t s) {
  if (!p->prof || p->prof_used >= kProfCap) return -1;
  const int slot = p->prof_used++;
  p->prof_stage[slot] = stage;
  nvtxRangePushA(kStageRange[stage]);
  cudaEventRecord(p->prof_ev[2 * slot], s);
  return slot;
}

void prof_end(pme_plan_t p, int slot, cudaStream_t s) {
  if (slot < 0) return;
  cudaEventRecord(p->prof_ev[2 * slot + 1], s);
  nvtxRangePop();
}

static int check_fft(pme_plan_t plan, cufftResult r, const char* what) {
  if (r == CUFFT_SUCCESS) return PME_OK;
  return set_error(plan, PME_ERR_CUFFT, std::string(what) + ": cuFFT error " + std::to_string(int(r)));
}

// ---- geometry helpers (host, float64) ----------------------------------------------------

static bool invert3(const double* a, double* inv, double* det_out) {
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  double scale = 1.0;
  for (int r = 0; r < 3; ++r)
    scale *= std::sqrt(a[3 * r] * a[3 * r] + a[3 * r + 1] * a[3 * r + 1] + a[3 * r + 2] * a[3 * r + 2]);
  if (!(std::fabs(det) > 1e-10 * scale) || !std::isfinite(det)) return false;
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
  *det_out = det;
  return true;
}

// Perpendicular width of the cell along axis a: V / |a_b x a_c|.
static double perp_width(const double* box, int ax, double V) {
  const double* u = box + 3 * ((ax + 1) % 3);
  const double* v = box + 3 * ((ax + 2) % 3);
  const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2],
               cz = u[0] * v[1] - u[1] * v[0];
  return V / std::sqrt(cx * cx + cy * cy + cz * cz);
}

// Bricks along one axis whose ions' stencils can reach each brick: an ion with first stencil
// point m0 covers m0 .. m0 + P - 1 (mod N), so brick [b0, b0 + ext) is fed by m0 in
// [b0 - P + 1, b0 + ext - 1] (mod N).
static bool build_candidates(int N, int B, int P, int nb, int max_nb, int* tab, int axis) {
  for (int b = 0; b < nb; ++b) {
    const int b0 = b * B, ext = std::min(B, N - b0);
    std::vector<int> list;
    if (ext + P - 1 >= N) {
      for (int k = 0; k < nb; ++k) list.push_back(k);
    } else {
      for (int m = b0 - P + 1; m <= b0 + ext - 1; ++m) {
        const int mm = ((m % N) + N) % N;
        const int bi = mm / B;
        if (std::find(list.begin(), list.end(), bi) == list.end()) list.push_back(bi);
      }
    }
    if (int(list.size()) > kMaxCandPerDim) return false;
    int* row = tab + (axis * max_nb + b) * (1 + kMaxCandPerDim);
    row[0] = int(list.size());
    for (size_t k = 0; k < list.size(); ++k) row[1 + k] = list[k];
  }
  return true;
}

static double sinc(double x) {
  if (x == 0.0) return 1.0;
  return std::sin(kPi * x) / (kPi * x);
}

// Box-dependent geometry of one frame (cell matrices, pair cells). g.N, g.order, g.alpha,
// g.rcut2 and the brick shape are set by the caller. Returns false for a singular box.
static bool frame_geometry(Geometry& g, const double* box, double rcut, bool pair, int* ncells,
                           std::string& why) {
  double inv[9], det;
  if (!invert3(box, inv, &det)) {
    why = "singular or non-finite box";
    return false;
  }
  for (int k = 0; k < 9; ++k) g.cinv[k] = inv[k];
  g.volume = std::fabs(det);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g.D[a * 3 + b] = float(double(g.N[b]) * inv[a * 3 + b]);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) g.bk[r * 3 + c] = float(2.0 * kPi * inv[c * 3 + r]);
  g.inv_volume = float(1.0 / g.volume);
  g.bg_fac = float(kPi / (g.volume * double(g.alpha) * double(g.alpha)));
  g.e_mesh_coef = 0.5 / g.volume;
  g.e_ewald_coef = 4.0 * kPi / g.volume;
  g.e_bg_coef = kPi / (2.0 * g.volume * double(g.alpha) * double(g.alpha));
  // pair cells at least rcut/2 wide (at least one per axis); a candidate cell lies at most
  // kimg = ceil(rcut / cell width) cells away along each axis. When an axis has fewer than
  // 2 kimg + 1 cells the offsets wrap onto the same cells again: each offset then stands for
  // a different periodic image, so every image inside rcut is visited exactly once.
  int nc_tot = 1;
  for (int a = 0; a < 3; ++a) {
    const double w = perp_width(box, a, g.volume);
    int nc = pair ? int(std::floor(w / (0.5 * rcut))) : 1;
    nc = std::max(1, std::min(nc, 512));
    g.ncell[a] = nc;
    g.kimg[a] = pair ? std::max(1, int(std::ceil(rcut * nc / w - 1e-9))) : 0;
    nc_tot *= nc;
  }
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) g.H[b * 3 + c] = float(box[b * 3 + c] / g.ncell[b]);
  geometry_split(g);
  *ncells = nc_tot;
  return true;
}

// ---- host-pointer staging ------------------------------------------------------------------

static bool is_device_pointer(const void* ptr) {
  if (!ptr) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Where a caller pointer lives: 0 device (or managed) memory, 1 pinned host memory the device
// can address (*dev: that address), 2 other host memory.
static int pointer_kind(const void* ptr, const void** dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return 2;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return 0;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *dev = at.devicePointer;
    return 1;
  }
  return 2;
}

enum StageSlot {
  kPos = 0, kQ = 3, kMu = 4, kGF = 7, kGPhi = 10, kGField = 11, kOF = 14, kOPhi = 17,
  kOField = 18, kOFG = 21, kOGPos = 27, kOGQ = 30, kOGMu = 31, kTheta = 34, kOGTheta = 40, kStageFloats = 46
};

// The arrays of one staging direction moved by a single kernel (pinned host memory is
// addressable by the device): lengths in floats (float64 arrays count two per value).
constexpr int kMaxStageCopies = 12;
struct StageCopies {
  const float* src[kMaxStageCopies];
  float* dst[kMaxStageCopies];
  long long len[kMaxStageCopies];
  int count;
};

__global__ void __launch_bounds__(256) k_stage_copy(StageCopies c) {
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int k = 0; k < c.count; ++k) {   // uniform
    const float* src = c.src[k];
    float* dst = c.dst[k];
    const long long len = c.len[k];
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
      const long long n4 = len / 4;
      for (long long i = t0; i < n4; i += stride)
        reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(src)[i];
      for (long long i = 4 * n4 + t0; i < len; i += stride) dst[i] = src[i];
    } else {
      for (long long i = t0; i < len; i += stride) dst[i] = src[i];
    }
  }
}

struct Staging {
  pme_plan_t p;
  cudaStream_t s;
  int n;
  int status = PME_OK;
  struct Pending {
    void* host;
    const void* dev;
    size_t bytes;
  };
  std::vector<Pending> outs;   // pageable host outputs (copied with cudaMemcpyAsync)
  StageCopies in_k{}, out_k{};   // pinned host arrays (moved by k_stage_copy)
  bool staged = false;   // some argument is a host pointer

  Staging(pme_plan_t p_, cudaStream_t s_, int n_) : p(p_), s(s_), n(n_) {}

  // one host input of `bytes` into device staging d: by the copy kernel when pinned (and
  // there is room in its table), else by cudaMemcpyAsync
  void stage_in(const void* ptr, void* d, size_t bytes) {
    const void* dp = nullptr;
    if (bytes % 4 == 0 && in_k.count < kMaxStageCopies && pointer_kind(ptr, &dp) == 1) {
      in_k.src[in_k.count] = static_cast<const float*>(dp);
      in_k.dst[in_k.count] = static_cast<float*>(d);
      in_k.len[in_k.count] = (long long)(bytes / 4);
      ++in_k.count;
      return;
    }
    if (bytes && status == PME_OK)
      status = check_cuda(p, cudaMemcpyAsync(d, ptr, bytes, cudaMemcpyHostToDevice, s), "stage input");
  }
  void stage_out(void* ptr, const void* d, size_t bytes) {
    const void* dp = nullptr;
    if (bytes % 4 == 0 && out_k.count < kMaxStageCopies && pointer_kind(ptr, &dp) == 1) {
      out_k.src[out_k.count] = static_cast<const float*>(d);
      out_k.dst[out_k.count] = const_cast<float*>(static_cast<const float*>(dp));
      out_k.len[out_k.count] = (long long)(bytes / 4);
      ++out_k.count;
      return;
    }
    outs.push_back({ptr, d, bytes});
  }
  int launch_copies(const StageCopies& c) {
    long long total = 0;
    for (int k = 0; k < c.count; ++k) total += c.len[k];
    if (total == 0 || status != PME_OK) return status;
    const long long want = (total / 4 + 255) / 256;
    const int grid = int(std::max(1LL, std::min<long long>(want, 4LL * device_sm_count())));
    k_stage_copy<<<grid, 256, 0, s>>>(c);
    count_launch();
    return status = check_launch(p, "k_stage_copy");
  }

  const float* in(const float* ptr, int width, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    staged = true;
    float* d = p->stage_f + size_t(slot) * p->max_ions;
    stage_in(ptr, d, sizeof(float) * size_t(width) * n);
    return d;
  }
  // count doubles (per-frame energies / cotangents / virials); slot 0 = outputs, 1 = inputs,
  // 2 = virials (9 per frame)
  const double* in_d(const double* ptr, int count, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    staged = true;
    double* d = p->stage_d + size_t(slot) * p->nframes;
    stage_in(ptr, d, sizeof(double) * count);
    return d;
  }
  float* out(float* ptr, int width, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    staged = true;
    float* d = p->stage_f + size_t(slot) * p->max_ions;
    stage_out(ptr, d, sizeof(float) * size_t(width) * n);
    return d;
  }
  double* out_d(double* ptr, int count, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    staged = true;
    double* d = p->stage_d + size_t(slot) * p->nframes;
    stage_out(ptr, d, sizeof(double) * count);
    return d;
  }
  // after every in() / out(): the pinned inputs' copy kernel, and the status so far
  int ready() {
    if (status == PME_OK && in_k.count) launch_copies(in_k);
    in_k.count = 0;
    return status;
  }
  int finish() {
    if (status == PME_OK && out_k.count) launch_copies(out_k);
    out_k.count = 0;
    for (auto& o : outs) {
      if (status != PME_OK) break;
      if (o.bytes)
        status = check_cuda(p, cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, s),
                            "stage output");
    }
    return status;
  }
};

static int set_device(pme_plan_t p) {
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return check_cuda(p, cudaSetDevice(p->device), "cudaSetDevice");
  return PME_OK;
}

static int check_common(pme_plan_t p, int n, const float* pos, const float* q) {
  if (!p) return PME_ERR_ARG;
  if (p->batch) return set_error(p, PME_ERR_ARG, "batched plan: use the pme_batch_* calls");
  if (n < 0 || n > p->max_ions)
    return set_error(p, PME_ERR_ARG, "n = " + std::to_string(n) + " outside [0, max_ions = " +
                                         std::to_string(p->max_ions) + "]");
  if (n > 0 && !pos) return set_error(p, PME_ERR_ARG, "pos is NULL");
  if (n > 0 && !q) return set_error(p, PME_ERR_ARG, "q is NULL");
  return set_device(p);
}

static int fork_side(pme_plan_t p, cudaStream_t s) {
  int st = check_cuda(p, cudaEventRecord(p->ev_fork, s), "event record");
  if (st) return st;
  return check_cuda(p, cudaStreamWaitEvent(p->side, p->ev_fork, 0), "stream wait");
}

static int join_side(pme_plan_t p, cudaStream_t s) {
  int st = check_cuda(p, cudaEventRecord(p->ev_join, p->side), "event record");
  if (st) return st;
  return check_cuda(p, cudaStreamWaitEvent(s, p->ev_join, 0), "stream wait");
}

static void drop_graphs(pme_plan_t p);

static void free_plan(pme_plan_t p) {
  if (!p) return;
  void* bufs[] = {p->rho, p->spec, p->phi, p->dconv_all, p->cand, p->sb.key_b, p->sb.key_c,
                  p->sb.slot_b, p->sb.slot_c, p->sb.count_b, p->sb.count_c, p->sb.start_b,
                  p->sb.start_c, p->sb.perm_b, p->sb.perm_c, p->sb.qsum, p->mr.idx, p->mr.fq,
                  p->mr.dm, p->mr.tq, p->mr.tt, p->pr.idx, p->pr.fq, p->pr.mu, p->pr.tq, p->pr.dr,
                  p->mesh_out, p->pair_out, p->e_ion, p->epart, p->flags, p->stage_f,
                  p->stage_d, p->ew_kn, p->ew_kv, p->ew_S, p->ew_fx, p->ew_qm, p->frames_d,
                  p->map_buf, p->fft_work, p->sb.qpart, p->sb.qcount, p->eitem, p->ecount,
                  p->plist, p->plist_cnt, p->in_saved, p->in_flags, p->vpart,
                  p->pvir, p->vitem, p->gtab, p->sb.t_bidx, p->sb.t_bfq,
                  p->sb.t_bdm, p->sb.t_cidx, p->sb.t_cfq, p->sb.t_cmu, p->conv_tw,
                  p->conv_planes1, p->quad_out};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int g = 0; g < p->nfgroups; ++g) {
    FFTGroup& G = p->fgroups[g];
    if (G.r2c) cufftDestroy(G.r2c);
    if (G.c2r) cufftDestroy(G.c2r);
    if (G.r2c2) cufftDestroy(G.r2c2);
    if (G.c2r2) cufftDestroy(G.c2r2);
  }
  delete[] p->fgroups;
  delete[] p->frames_h;
  delete[] p->frame_offsets;
  if (p->prof_ev) {
    for (int k = 0; k < 2 * kProfCap; ++k) cudaEventDestroy(p->prof_ev[k]);
    delete[] p->prof_ev;
    delete[] p->prof_stage;
  }
  drop_graphs(p);
  delete[] p->graphs;
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  delete p;
}

// A failed allocation is reported as PME_ERR_NOMEM and its error is cleared from the runtime,
// so that later launch checks (of this or another plan) do not mistake it for their own.
template <typename T>
static int dalloc(pme_plan_t p, T** ptr, size_t count) {
  *ptr = nullptr;
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
  }
  return check_cuda(p, e, "cudaMalloc");
}

// Count / start arrays of the sort: n + 1 entries padded to a multiple of 4 (the scan moves
// them 16 bytes at a time).
static size_t scan_entries(int n) { return (size_t(n) + 1 + 3) & ~size_t(3); }

// The cell counts start zero (each scan re-zeroes them).
static int alloc_cells(pme_plan_t p) {
  int st;
  if ((st = dalloc(p, &p->sb.count_c, scan_entries(p->total_cells)))) return st;
  if ((st = dalloc(p, &p->sb.start_c, scan_entries(p->total_cells)))) return st;
  return check_cuda(p, cudaMemset(p->sb.count_c, 0, sizeof(int) * scan_entries(p->total_cells)), "cudaMemset");
}

// (Re)build the explicit-Ewald k-vector tables for the current box (single-frame plans).
static int setup_kvectors(pme_plan_t p) {
  std::vector<int4> kn;
  std::vector<float4> kv;
  ewald_build_kvectors(p, kn, kv);
  cudaFree(p->ew_kn);
  cudaFree(p->ew_kv);
  cudaFree(p->ew_S);
  p->ew_kn = nullptr;
  p->ew_kv = nullptr;
  p->ew_S = nullptr;
  p->ew_K = int(kn.size());
  int st;
  if ((st = dalloc(p, &p->ew_kn, kn.size()))) return st;
  if ((st = dalloc(p, &p->ew_kv, kv.size()))) return st;
  if ((st = dalloc(p, &p->ew_S, kn.size()))) return st;
  if (!kn.empty()) {
    if ((st = check_cuda(p, cudaMemcpy(p->ew_kn, kn.data(), sizeof(int4) * kn.size(), cudaMemcpyHostToDevice),
                         "copy k-vectors")))
      return st;
    if ((st = check_cuda(p, cudaMemcpy(p->ew_kv, kv.data(), sizeof(float4) * kv.size(), cudaMemcpyHostToDevice),
                         "copy k-vectors")))
      return st;
  }
  // the energy partials hold one slot per k block; frame 0's "influence blocks" are those
  const int kb = ewald_partial_blocks(p);
  p->frames_h[0].infl_blk_off = 0;
  p->frames_h[0].infl_nblk = kb;
  cudaFree(p->epart);
  p->epart = nullptr;
  return dalloc(p, &p->epart, size_t(std::max(kb, p->total_blocks)) + 1);
}

// ---- plan construction ----------------------------------------------------------------------

struct FrameInput {
  const double* box;
  int mesh[3];
  int order;
  int ion_off, n;
};

// Whether the options ask for the hand-written transforms: fft 2 always; fft 0 (automatic)
// for batched plans of small meshes (no axis above kConvAutoMaxAxis), whose frames then share
// one launch per pass instead of a cuFFT plan per mesh shape. On GB300 these passes beat
// cuFFT on batches of 16-48 point meshes and lose to it at 128^3, where the spectrum stays in
// L2 and cuFFT's per-point cost is lower. The axis lengths and shared-memory sizes are
// checked by the caller.
// Meshes whose every axis is 64 or 128 points take the power-of-two kernels (compile-time
// four-step transforms), which beat cuFFT on GB300 for single frames too (a 128^3 R2C pass in
// a fraction of cuFFT's three kernels), so the automatic choice takes them whenever every
// frame qualifies.
constexpr int kConvAutoMaxAxis = 64;

static bool conv_wanted(const pme_plan_s* p, bool single, const std::vector<FrameInput>& fin) {
  if (p->opts.fft == 2 || p->opts.fft == 3) return true;
  if (p->opts.fft != 0) return false;
  bool p2 = true;
  for (const FrameInput& f : fin) p2 = p2 && conv_p2_ok(f.mesh);
  if (p2) return true;
  if (single) return false;
  for (const FrameInput& f : fin)
    for (int a = 0; a < 3; ++a)
      if (f.mesh[a] > kConvAutoMaxAxis) return false;
  return true;
}

// Build a plan over the given frames. single: one frame whose ion count is chosen per call.
static int build_plan(pme_plan_s* p, const std::vector<FrameInput>& fin, double alpha, double rcut,
                      bool single) {
  const int F = int(fin.size());
  p->nframes = F;
  p->batch = !single;
  p->alpha = alpha;
  p->rcut = rcut;
  p->frames_h = new (std::nothrow) FrameDesc[F];
  p->frame_offsets = new (std::nothrow) int[F + 1];
  if (!p->frames_h || !p->frame_offsets) return set_error(p, PME_ERR_NOMEM, "host tables");
  std::memset(p->frames_h, 0, sizeof(FrameDesc) * F);
  const bool pair = p->opts.include_pair != 0;
  if (p->max_ions > (1 << 27)) return set_error(p, PME_ERR_UNSUPPORTED, "more than 2^27 ions in one plan");
  int brick[3];
  spread_brick_shape(brick);
  if (p->opts.brick[0] > 0 || p->opts.brick[1] > 0 || p->opts.brick[2] > 0) {
    if (!spread_shape_supported(p->opts.brick))
      return set_error(p, PME_ERR_UNSUPPORTED, "brick shape not among the built ones");
    for (int a = 0; a < 3; ++a) brick[a] = p->opts.brick[a];
  }
  // the mesh convolution runs on the hand-written transforms when the options ask for them,
  // every axis of every frame is 2,3,5-smooth and short enough, and a plane (pass A / C) and
  // a pass-B tile fit in shared memory
  {
    bool conv = conv_wanted(p, single, fin);
    size_t cap = 0, smem_plane = 0, smem_x = 0, biggest = 0;
    for (int f = 0; f < F && conv; ++f) {
      for (int a = 0; a < 3; ++a) conv = conv && conv_axis_ok(fin[f].mesh[a]);
      if (!conv) break;
      cap = std::max(cap, conv_plane_cap(fin[f].mesh));
      smem_x = std::max(smem_x, conv_x_smem(fin[f].mesh));
      biggest = std::max(biggest, conv_plane_cap(fin[f].mesh));
    }
    // the power-of-two kernels when every frame qualifies (fft = 3 keeps the general ones)
    bool p2 = conv && p->opts.fft != 3;
    for (int f = 0; f < F && p2; ++f) p2 = conv_p2_ok(fin[f].mesh);
    if (p2) {
      smem_x = 0;
      for (int f = 0; f < F; ++f) {
        smem_plane = std::max(smem_plane, conv_p2_plane_smem(fin[f].mesh));
        smem_x = std::max(smem_x, conv_p2_x_smem(fin[f].mesh));
      }
    }
    if (conv && !p2) {
      for (int f = 0; f < F; ++f) smem_plane = std::max(smem_plane, conv_plane_smem(fin[f].mesh, cap));
    }
    if (conv) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        optin = 0;
      }
      conv = smem_plane + 1024 <= size_t(optin) && smem_x + 1024 <= size_t(optin);
    }
    if (!conv && (p->opts.fft == 2 || p->opts.fft == 3))
      return set_error(p, PME_ERR_UNSUPPORTED, "fft = 2 / 3: a mesh the library's transforms do not take");
    p->conv = conv;
    p->conv_p2 = conv && p2;
    p->conv_cap = int(cap);
    p->conv_smem_plane = smem_plane;
    p->conv_smem_x = smem_x;
    p->conv_threads = biggest >= 8192 ? 1024 : (biggest >= 2048 ? 512 : 256);
  }
  std::vector<int> ncells(F);
  for (int f = 0; f < F; ++f) {
    FrameDesc& D = p->frames_h[f];
    Geometry& g = D.g;
    const FrameInput& in = fin[f];
    if (in.order < 1 || in.order > kMaxOrder) return set_error(p, PME_ERR_ARG, "order outside 1..7");
    for (int a = 0; a < 3; ++a)
      if (in.mesh[a] < in.order || in.mesh[a] > 4096)
        return set_error(p, PME_ERR_ARG, "mesh dimension < order (or > 4096)");
    for (int a = 0; a < 3; ++a) {
      g.N[a] = in.mesh[a];
      g.brick[a] = brick[a];
      g.nb[a] = (g.N[a] + brick[a] - 1) / brick[a];
    }
    g.order = in.order;
    g.alpha = float(alpha);
    g.rcut2 = float(rcut * rcut);
    std::string why;
    if (!frame_geometry(g, in.box, rcut, pair, &ncells[f], why)) return set_error(p, PME_ERR_ARG, why);
    D.ion_off = in.ion_off;
    D.n = in.n;
    D.nbricks = g.nb[0] * g.nb[1] * g.nb[2];
    D.ncells = ncells[f];
    D.max_nb = std::max(g.nb[0], std::max(g.nb[1], g.nb[2]));
    if ((long long)g.N[0] * g.N[1] * (g.N[2] / 2 + 1) >= (1LL << 30))
      return set_error(p, PME_ERR_UNSUPPORTED, "half spectrum of a frame above 2^30 points");
    if (p->conv) {
      conv_tiles(g.N, &D.infl_nblk, &D.conv_cols);
      D.conv_pp = conv_planes_per_block(g.N);
    } else {
      D.infl_nblk = influence_blocks(g);
    }
    D.div_zh = make_fastdiv(g.N[2] / 2 + 1);
    D.div_y = make_fastdiv(g.N[1]);
    D.nitems = single ? std::max(1, (p->max_ions + kRedItem - 1) / kRedItem)
                      : std::max(1, (in.n + kRedItem - 1) / kRedItem);
    p->frame_offsets[f] = in.ion_off;
  }
  p->frame_offsets[F] = single ? p->max_ions : fin[F - 1].ion_off + fin[F - 1].n;
  p->g = p->frames_h[0].g;
  std::memcpy(p->box, fin[0].box, sizeof(double) * 9);

  // internal order of the frames: by spline order, then mesh shape (stable)
  std::vector<int> ord(F);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    const Geometry& ga = p->frames_h[a].g;
    const Geometry& gb = p->frames_h[b].g;
    if (ga.order != gb.order) return ga.order < gb.order;
    for (int k = 0; k < 3; ++k)
      if (ga.N[k] != gb.N[k]) return ga.N[k] < gb.N[k];
    return false;
  });
  long long brick_off = 0, cell_off = 0, sorted_off = 0, cand_off = 0, dconv_off = 0, blk_off = 0,
            item_off = 0;
  for (int f : ord) {
    FrameDesc& D = p->frames_h[f];
    D.brick_off = int(brick_off);
    D.cell_off = int(cell_off);
    D.sorted_off = int(sorted_off);
    D.cand_off = int(cand_off);
    D.dconv_off = int(dconv_off);
    D.infl_blk_off = int(blk_off);
    D.item_off = int(item_off);
    item_off += D.nitems;
    brick_off += D.nbricks;
    cell_off += D.ncells;
    sorted_off += single ? 0 : D.n;
    cand_off += 3LL * D.max_nb * (1 + kMaxCandPerDim);
    dconv_off += D.g.N[0] + D.g.N[1] + D.g.N[2];
    blk_off += D.infl_nblk;
  }
  if (brick_off > (1LL << 30) || cell_off > (1LL << 30)) return set_error(p, PME_ERR_UNSUPPORTED, "too many bricks");
  p->total_bricks = int(brick_off);
  p->total_cells = int(cell_off);
  p->total_blocks = int(blk_off);
  p->total_items = int(item_off);
  // spread / gather launch groups (one per spline order)
  p->nogroups = 0;
  for (int f : ord) {
    const FrameDesc& D = p->frames_h[f];
    if (p->nogroups == 0 || p->ogroups[p->nogroups - 1].order != D.g.order) {
      OrderGroup& G = p->ogroups[p->nogroups++];
      G.order = D.g.order;
      G.brick_lo = D.brick_off;
      G.sorted_lo = D.sorted_off;
    }
    OrderGroup& G = p->ogroups[p->nogroups - 1];
    G.brick_hi = D.brick_off + D.nbricks;
    G.sorted_hi = D.sorted_off + (single ? 0 : D.n);
  }
  // FFT groups (same order and mesh shape): rho of the members, then their d rho
  std::vector<std::vector<int>> groups;
  for (int f : ord) {
    const Geometry& g = p->frames_h[f].g;
    if (groups.empty()) {
      groups.push_back({f});
      continue;
    }
    const Geometry& h = p->frames_h[groups.back()[0]].g;
    if (h.order == g.order && h.N[0] == g.N[0] && h.N[1] == g.N[1] && h.N[2] == g.N[2])
      groups.back().push_back(f);
    else
      groups.push_back({f});
  }
  p->nfgroups = int(groups.size());
  p->fgroups = new (std::nothrow) FFTGroup[p->nfgroups];
  if (!p->fgroups) return set_error(p, PME_ERR_NOMEM, "host tables");
  std::memset(p->fgroups, 0, sizeof(FFTGroup) * p->nfgroups);
  long long mesh_off = 0, spec_off = 0;
  for (int gi = 0; gi < p->nfgroups; ++gi) {
    FFTGroup& G = p->fgroups[gi];
    const Geometry& g = p->frames_h[groups[gi][0]].g;
    const long long M = (long long)g.N[0] * g.N[1] * g.N[2];
    const long long Mh = (long long)g.N[0] * g.N[1] * (g.N[2] / 2 + 1);
    for (int k = 0; k < 3; ++k) G.N[k] = g.N[k];
    G.count = int(groups[gi].size());
    G.mesh_off = mesh_off;
    G.spec_off = spec_off;
    for (int k = 0; k < G.count; ++k) {
      FrameDesc& D = p->frames_h[groups[gi][k]];
      D.mesh_off = mesh_off + k * M;
      D.tmesh_off = mesh_off + (G.count + k) * M;
      D.spec_off = spec_off + k * Mh;
      D.tspec_off = spec_off + (G.count + k) * Mh;
    }
    mesh_off += 2LL * G.count * M;
    spec_off += 2LL * G.count * Mh;
  }
  p->total_mesh = mesh_off;
  long long gtab_total = 0;   // influence tables, one half spectrum per frame
  for (int f = 0; f < F; ++f) {
    FrameDesc& D = p->frames_h[f];
    D.gtab_off = gtab_total;
    gtab_total += (long long)D.g.N[0] * D.g.N[1] * (D.g.N[2] / 2 + 1);
  }
  p->total_spec = spec_off;
  {
    const Geometry& g0 = p->frames_h[0].g;
    p->M = g0.N[0] * g0.N[1] * g0.N[2];
    p->Mh = g0.N[0] * g0.N[1] * (g0.N[2] / 2 + 1);
  }

  // ---- device buffers ----------------------------------------------------------------------
  cudaGetDevice(&p->device);
  int st = PME_OK;
  auto A = [&](auto** ptr, size_t count) {
    if (st == PME_OK) st = dalloc(p, ptr, count);
  };
  const size_t ni = size_t(p->max_ions);
  A(&p->rho, size_t(p->total_mesh));
  A(&p->spec, size_t(p->total_spec));
  A(&p->phi, size_t(p->total_mesh));
  A(&p->dconv_all, size_t(dconv_off));
  A(&p->cand, size_t(cand_off));
  A(&p->sb.key_b, ni);
  A(&p->sb.key_c, ni);
  A(&p->sb.slot_b, ni);
  A(&p->sb.slot_c, ni);
  A(&p->sb.perm_b, ni);
  A(&p->sb.perm_c, ni);
  A(&p->sb.count_b, scan_entries(p->total_bricks));
  A(&p->sb.start_b, scan_entries(p->total_bricks));
  A(&p->sb.qsum, size_t(2) * F);
  A(&p->sb.t_bidx, ni);
  A(&p->sb.t_bfq, ni);
  A(&p->sb.t_bdm, ni);
  A(&p->sb.t_cidx, ni);
  A(&p->sb.t_cfq, ni);
  A(&p->sb.t_cmu, ni);
  A(&p->sb.qpart, size_t(2) * p->total_items);
  A(&p->sb.qcount, size_t(F));
  A(&p->eitem, size_t(p->total_items));
  A(&p->ecount, size_t(F));
  A(&p->mr.idx, ni);
  A(&p->mr.fq, ni);
  A(&p->mr.dm, ni);
  A(&p->mr.tq, ni);
  A(&p->mr.tt, ni);
  A(&p->pr.idx, ni);
  A(&p->pr.fq, ni);
  A(&p->pr.mu, ni);
  A(&p->pr.tq, ni);
  A(&p->pr.dr, ni);
  A(&p->mesh_out, ni * 10);
  A(&p->pair_out, ni * 10);
  A(&p->quad_out, ni * 8);
  A(&p->qb_mesh, ni * 26);
  A(&p->qb_pair, ni * 26);
  A(&p->e_ion, ni);
  A(&p->epart, size_t(p->total_blocks) + 1);
  A(&p->flags, 1);
  A(&p->stage_f, ni * kStageFloats);
  A(&p->stage_d, size_t(11) * F + 2);   // energies, cotangents, virials (9 per frame)
  A(&p->vpart, size_t(6) * p->total_blocks + 6);
  A(&p->pvir, 9 * ni);
  A(&p->vitem, size_t(9) * p->total_items);
  if (st == PME_OK) st = alloc_cells(p);
  if (st == PME_OK)
    st = check_cuda(p, cudaMemset(p->sb.count_b, 0, sizeof(int) * scan_entries(p->total_bricks)), "cudaMemset");
  p->counts_clean = st == PME_OK;
  // pair lists for backward passes on the forward's positions: room for 1.5x the mean number
  // of partners inside rcut (density from the plan's largest n / V) + 64, when that fits in
  // 1 GiB; an ion with more partners marks the lists invalid and the backward recomputes
  if (st == PME_OK && pair) {
    double dens = 0.0;
    for (int f = 0; f < F; ++f) {
      const FrameDesc& D = p->frames_h[f];
      const double nf = single ? double(p->max_ions) : double(D.n);
      dens = std::max(dens, nf / D.g.volume);
    }
    const double mean = 4.0 / 3.0 * kPi * rcut * rcut * rcut * dens;
    int cap = int(std::ceil((1.5 * mean + 64.0) / 32.0)) * 32;
    cap = std::max(64, std::min(cap, 2048));
    if (double(p->max_ions) * cap * sizeof(float4) <= double(1ull << 30)) {
      p->plist_cap = cap;
      A(&p->plist, ni * size_t(cap));
      A(&p->plist_cnt, ni);
    }
  }
  if (p->opts.recip_method == 0) A(&p->gtab, size_t(gtab_total));
  A(&p->in_saved, 7 * ni);
  A(&p->in_flags, 2);
  if (st == PME_OK) {
    p->in_diff = p->in_flags;
    p->cache_bad = p->in_flags + 1;
  }
  if (st) return st;
  if ((st = check_cuda(p, cudaMemset(p->flags, 0, sizeof(int)), "memset"))) return st;
  if ((st = check_cuda(p, cudaMemset(p->sb.qcount, 0, sizeof(int) * F), "memset"))) return st;
  if ((st = check_cuda(p, cudaMemset(p->ecount, 0, sizeof(int) * F), "memset"))) return st;
  // candidate tables and deconvolution tables, frame by frame
  {
    std::vector<int> cand(size_t(cand_off), 0);
    std::vector<float> dc(size_t(dconv_off), 1.f);
    for (int f = 0; f < F; ++f) {
      const FrameDesc& D = p->frames_h[f];
      const Geometry& g = D.g;
      for (int a = 0; a < 3; ++a)
        if (!build_candidates(g.N[a], g.brick[a], g.order, g.nb[a], D.max_nb, cand.data() + D.cand_off, a))
          return set_error(p, PME_ERR_UNSUPPORTED, "mesh / brick / order combination not supported");
      // C(n) = 1 / sinc^(2 p gamma)(n / N) per axis (Eqs. Bk, influence)
      int o = D.dconv_off;
      for (int a = 0; a < 3; ++a)
        for (int i = 0; i < g.N[a]; ++i) {
          const int nsig = (i <= g.N[a] / 2) ? i : i - g.N[a];
          const double b = std::pow(sinc(double(nsig) / g.N[a]), double(g.order));
          dc[o++] = p->opts.deconvolution ? float(std::pow(b * b, -p->opts.influence_power)) : 1.f;
        }
    }
    if ((st = check_cuda(p, cudaMemcpy(p->cand, cand.data(), sizeof(int) * cand.size(), cudaMemcpyHostToDevice),
                         "copy candidates")))
      return st;
    if ((st = check_cuda(p, cudaMemcpy(p->dconv_all, dc.data(), sizeof(float) * dc.size(), cudaMemcpyHostToDevice),
                         "copy deconvolution")))
      return st;
  }
  if (p->conv) {
    // twiddle tables, one per distinct axis length
    std::vector<float2> tw;
    std::vector<int> tw_at(kConvMaxLen + 1, -1);
    for (int f = 0; f < F; ++f)
      for (int a = 0; a < 3; ++a) {
        const int L = p->frames_h[f].g.N[a];
        if (tw_at[L] < 0) {
          tw_at[L] = int(tw.size());
          conv_twiddles(L, tw);
        }
        p->frames_h[f].tw_off[a] = tw_at[L];
      }
    if ((st = dalloc(p, &p->conv_tw, tw.size()))) return st;
    if ((st = check_cuda(p, cudaMemcpy(p->conv_tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice),
                         "copy twiddles")))
      return st;
    if (!single) {
      // pass A / C blocks: (frame, plane) without and with the tangent meshes
      std::vector<int2> planes;
      auto per_copy = [&](int f) {
        const FrameDesc& D = p->frames_h[f];
        return (D.g.N[0] + D.conv_pp - 1) / D.conv_pp;
      };
      for (int f : ord)
        for (int b = 0; b < per_copy(f); ++b) planes.push_back(make_int2(f, b));
      p->conv_nplanes1 = int(planes.size());
      for (int f : ord)
        for (int b = 0; b < 2 * per_copy(f); ++b) planes.push_back(make_int2(f, b));
      p->conv_nplanes2 = int(planes.size()) - p->conv_nplanes1;
      if ((st = dalloc(p, &p->conv_planes1, planes.size()))) return st;
      if ((st = check_cuda(p, cudaMemcpy(p->conv_planes1, planes.data(), sizeof(int2) * planes.size(),
                                         cudaMemcpyHostToDevice),
                           "copy plane maps")))
        return st;
      p->conv_planes2 = p->conv_planes1 + p->conv_nplanes1;
    }
  }
  // batched plans: descriptor table and frame maps on the device
  if (!single) {
    const long long Ntot = p->frame_offsets[F];
    std::vector<int> maps(size_t(2 * Ntot + p->total_bricks + p->total_blocks + p->total_items));
    int* ion_frame = maps.data();
    int* sorted_frame = ion_frame + Ntot;
    int* brick_frame = sorted_frame + Ntot;
    int* blk_frame = brick_frame + p->total_bricks;
    int* item_frame = blk_frame + p->total_blocks;
    for (int f = 0; f < F; ++f) {
      const FrameDesc& D = p->frames_h[f];
      for (int k = 0; k < D.n; ++k) {
        ion_frame[D.ion_off + k] = f;
        sorted_frame[D.sorted_off + k] = f;
      }
      for (int k = 0; k < D.nbricks; ++k) brick_frame[D.brick_off + k] = f;
      for (int k = 0; k < D.infl_nblk; ++k) blk_frame[D.infl_blk_off + k] = f;
      for (int k = 0; k < D.nitems; ++k) item_frame[D.item_off + k] = f;
    }
    if ((st = dalloc(p, &p->map_buf, maps.size()))) return st;
    if ((st = dalloc(p, &p->frames_d, size_t(F)))) return st;
    if ((st = check_cuda(p, cudaMemcpy(p->map_buf, maps.data(), sizeof(int) * maps.size(), cudaMemcpyHostToDevice),
                         "copy maps")))
      return st;
    if ((st = check_cuda(p, cudaMemcpy(p->frames_d, p->frames_h, sizeof(FrameDesc) * F, cudaMemcpyHostToDevice),
                         "copy frames")))
      return st;
    p->maps.desc = p->frames_d;
    p->maps.ion_frame = p->map_buf;
    p->maps.sorted_frame = p->map_buf + Ntot;
    p->maps.brick_frame = p->map_buf + 2 * Ntot;
    p->maps.blk_frame = p->map_buf + 2 * Ntot + p->total_bricks;
    p->maps.item_frame = p->map_buf + 2 * Ntot + p->total_bricks + p->total_blocks;
  }
  // cuFFT: four plans per group sharing one work area
  size_t work = 0;
  for (int gi = 0; gi < p->nfgroups && !p->conv; ++gi) {
    FFTGroup& G = p->fgroups[gi];
    int dims[3] = {G.N[0], G.N[1], G.N[2]};
    cufftHandle* hs[4] = {&G.r2c, &G.c2r, &G.r2c2, &G.c2r2};
    const cufftType ty[4] = {CUFFT_R2C, CUFFT_C2R, CUFFT_R2C, CUFFT_C2R};
    const int batch[4] = {G.count, G.count, 2 * G.count, 2 * G.count};
    for (int k = 0; k < 4; ++k) {
      size_t ws = 0;
      if ((st = check_fft(p, cufftCreate(hs[k]), "cufftCreate"))) return st;
      if ((st = check_fft(p, cufftSetAutoAllocation(*hs[k], 0), "cufftSetAutoAllocation"))) return st;
      if ((st = check_fft(p, cufftMakePlanMany(*hs[k], 3, dims, nullptr, 1, 0, nullptr, 1, 0, ty[k], batch[k], &ws),
                          "cufftMakePlanMany")))
        return st;
      work = std::max(work, ws);
    }
  }
  if (!p->conv && (st = check_cuda(p, cudaMalloc(&p->fft_work, std::max<size_t>(work, 16)), "cudaMalloc")))
    return st;
  for (int gi = 0; gi < p->nfgroups && !p->conv; ++gi) {
    FFTGroup& G = p->fgroups[gi];
    for (cufftHandle h : {G.r2c, G.c2r, G.r2c2, G.c2r2})
      if ((st = check_fft(p, cufftSetWorkArea(h, p->fft_work), "cufftSetWorkArea"))) return st;
  }
  if (p->gtab && ((st = launch_influence_tables(p, 0)) || (st = check_cuda(p, cudaDeviceSynchronize(), "synchronize"))))
    return st;
  p->graphs = new (std::nothrow) PassGraph[2];
  if (!p->graphs) return set_error(p, PME_ERR_NOMEM, "host tables");
  std::memset(p->graphs, 0, sizeof(PassGraph) * 2);
  if ((st = check_cuda(p, cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking), "stream"))) return st;
  if ((st = check_cuda(p, cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking), "stream")) ||
      (st = check_cuda(p, cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming), "event")) ||
      (st = check_cuda(p, cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming), "event")))
    return st;
  return PME_OK;
}

// ---- the passes ----------------------------------------------------------------------------

// keep (own transforms, backward, nullable): *keep == 0 means rho and Phi are the plan's
// forward's, so only the tangent mesh is transformed (Phi stays in place)
static int fft_forward(pme_plan_t p, cudaStream_t s, bool tangent, const int* keep = nullptr) {
  if (p->conv) return launch_conv_forward(p, s, tangent, p->rho, keep);
  int st;
  for (int gi = 0; gi < p->nfgroups; ++gi) {
    FFTGroup& G = p->fgroups[gi];
    cufftHandle h = tangent ? G.r2c2 : G.r2c;
    if ((st = check_fft(p, cufftSetStream(h, s), "set stream"))) return st;
    if ((st = check_fft(p, cufftExecR2C(h, p->rho + G.mesh_off, p->spec + G.spec_off), "exec r2c"))) return st;
  }
  return PME_OK;
}

static int fft_inverse(pme_plan_t p, cudaStream_t s, bool tangent, const int* keep = nullptr) {
  if (p->conv) return launch_conv_inverse(p, s, tangent, p->phi, keep);
  int st;
  for (int gi = 0; gi < p->nfgroups; ++gi) {
    FFTGroup& G = p->fgroups[gi];
    cufftHandle h = tangent ? G.c2r2 : G.c2r;
    if ((st = check_fft(p, cufftSetStream(h, s), "set stream"))) return st;
    if ((st = check_fft(p, cufftExecC2R(h, p->spec + G.spec_off, p->phi + G.mesh_off), "exec c2r"))) return st;
  }
  return PME_OK;
}

// The influence stage: with the hand-written transforms, the x transforms and the multiply
// in one pass (the spectra are then transformed along z and y only); otherwise in place on
// cuFFT's full spectra.
static int multiply_influence(pme_plan_t p, cudaStream_t s, bool tangent, double* vparts,
                              const int* keep = nullptr) {
  if (p->conv) return launch_conv_influence(p, s, tangent, p->epart, vparts, keep);
  return launch_influence(p, s, p->spec, tangent, p->epart, vparts);
}

// Forward with the explicit k-sum in place of the mesh stages (single-frame plans).
static int forward_ewald(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool pair, double* e_out,
                         float* f_out, float* p_out, float* fl_out, float* fg_out) {
  const int n = in.n;
  int st, t;
  t = prof_begin(p, 0, s);
  if ((st = launch_sort(p, s, in, false, false, pair, nullptr))) return st;
  prof_end(p, t, s);
  const bool fork = pair && n > 0;
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (fork) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, 6, ps);
    if ((st = launch_pair(p, ps, n, false, in, nullptr, p->pair_out, nullptr))) return st;
    prof_end(p, t, ps);
  }
  t = prof_begin(p, 3, s);
  if ((st = launch_ewald_recip(p, s, in, p->epart, p->mesh_out))) return st;
  prof_end(p, t, s);
  if (fork && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, 7, s);
  if ((st = launch_combine_forward(p, s, in, true, fork, f_out, p_out, fl_out, fg_out, e_out, 2))) return st;
  prof_end(p, t, s);
  return PME_OK;
}

// Forward pass over every frame of the plan (in.n ions in total).
// ---- CUDA graphs of repeated passes ------------------------------------------------------

static PassKey make_key(std::initializer_list<unsigned long long> vals) {
  PassKey k{};
  for (unsigned long long v : vals) k.v[k.len++] = v;
  return k;
}

static unsigned long long ptr_bits(const void* ptr) { return (unsigned long long)(uintptr_t)ptr; }

static void drop_graphs(pme_plan_t p) {
  if (!p->graphs) return;
  for (int k = 0; k < 2; ++k) {
    if (p->graphs[k].exec) cudaGraphExecDestroy(p->graphs[k].exec);
    p->graphs[k].exec = nullptr;
    p->graphs[k].have_last = false;
  }
}

// Run a pass, through a CUDA graph when the same call (key) comes again: the second identical
// call records the pass on the plan's capture stream and launches the graph; later identical
// calls only launch it. The pass sees device pointers only (host arguments are copied to and
// from the plan's staging buffers on the stream before and after it), so staged calls replay
// too. eligible = false, or stage timers on, runs directly.
template <class Run>
static int run_pass(pme_plan_t p, int which, cudaStream_t s, const PassKey& key, bool eligible, Run&& run) {
  PassGraph& G = p->graphs[which];
  if (!eligible || p->prof) {
    G.have_last = false;
    return run(s);
  }
  if (G.exec && G.key == key) {
    int st = check_cuda(p, cudaGraphLaunch(G.exec, s), "graph launch");
    if (st) return st;
    for (long long k = 0; k < G.launches; ++k) count_launch();
    p->fwd_n = G.post_fwd_n;
    p->fwd_lists = G.post_fwd_lists;
    return PME_OK;
  }
  if (!(G.have_last && G.last == key)) {
    G.last = key;
    G.have_last = true;
    return run(s);
  }
  // second identical call: record the pass (nothing executes while capturing)
  const long long before = pme_launch_count();
  const int save_n = p->fwd_n;
  const bool save_lists = p->fwd_lists;
  cudaGraph_t graph = nullptr;
  int st = check_cuda(p, cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (!st) {
    const int rs = run(p->cap_stream);
    const cudaError_t ce = cudaStreamEndCapture(p->cap_stream, &graph);
    if (rs || ce != cudaSuccess || !graph) st = rs ? rs : check_cuda(p, ce, "end capture");
  }
  const long long captured = pme_launch_count() - before;
  g_launches.fetch_sub(captured, std::memory_order_relaxed);   // recorded, not launched
  cudaGraphExec_t exec = nullptr;
  if (!st) st = check_cuda(p, cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
  if (graph) cudaGraphDestroy(graph);
  if (st) {
    // fall back to a direct run with the host state as it was
    cudaGetLastError();
    p->last_error.clear();
    p->fwd_n = save_n;
    p->fwd_lists = save_lists;
    G.have_last = false;
    return run(s);
  }
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = exec;
  G.key = key;
  G.launches = captured;
  G.post_fwd_n = p->fwd_n;
  G.post_fwd_lists = p->fwd_lists;
  st = check_cuda(p, cudaGraphLaunch(G.exec, s), "graph launch");
  if (st) return st;
  for (long long k = 0; k < G.launches; ++k) count_launch();
  return PME_OK;
}

// v_out (nullable): also the frame virials, [9] per frame (needs e_out).
static int run_forward(pme_plan_t p, cudaStream_t s, const IonInputs& in, double* e_out, float* f_out,
                       float* p_out, float* fl_out, float* fg_out, double* v_out = nullptr) {
  const int n = in.n;
  const bool pair = p->opts.include_pair != 0;
  if (p->opts.recip_method == 1) return forward_ewald(p, s, in, pair, e_out, f_out, p_out, fl_out, fg_out);
  int st, t;
  t = prof_begin(p, 0, s);
  // the binning pass also saves the inputs for a backward on the same ones
  if ((st = launch_sort(p, s, in, false, true, pair, nullptr, n > 0 ? p->in_saved : nullptr))) return st;
  prof_end(p, t, s);
  // the pair term runs on the plan's side stream, concurrently with the mesh stages: a list
  // pass writes each ion's hits (kept for a backward on the same positions), then the
  // list-driven evaluation; if a list overflowed, the fused pass does the work instead
  const bool fork = pair && n > 0;
  const bool record = fork && p->plist;
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (fork) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, 6, ps);
    if (record) {
      if ((st = launch_pair_build(p, ps, n, p->cache_bad))) return st;
      if ((st = launch_pair(p, ps, n, false, in, nullptr, p->pair_out, p->cache_bad, v_out != nullptr)))
        return st;
      const int te = prof_begin(p, 8, ps);
      if ((st = launch_pair_listed(p, ps, n, false, nullptr, p->pair_out, p->cache_bad, v_out != nullptr)))
        return st;
      prof_end(p, te, ps);
    } else if ((st = launch_pair(p, ps, n, false, in, nullptr, p->pair_out, nullptr))) {
      return st;
    }
    prof_end(p, t, ps);
  }
  t = prof_begin(p, 1, s);
  if ((st = launch_spread(p, s, false, p->rho))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 2, s);
  if ((st = fft_forward(p, s, false))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 3, s);
  if ((st = multiply_influence(p, s, false, v_out ? p->vpart : nullptr))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 4, s);
  if ((st = fft_inverse(p, s, false))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 5, s);
  if ((st = launch_gather(p, s, n, p->phi, false, nullptr, p->mesh_out))) return st;
  prof_end(p, t, s);
  if (fork && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, 7, s);
  if ((st = launch_combine_forward(p, s, in, true, fork, f_out, p_out, fl_out, fg_out, e_out, 1, v_out)))
    return st;
  prof_end(p, t, s);
  p->fwd_n = n > 0 ? n : -1;
  p->fwd_lists = record;
  return PME_OK;
}

// Backward pass (gradient plus Hessian-vector product) over every frame of the plan.
static int run_backward(pme_plan_t p, cudaStream_t s, const IonInputs& in, const double* gE,
                        float* o_pos, float* o_q, float* o_mu) {
  const int n = in.n;
  if (n == 0) return PME_OK;
  const bool pair = p->opts.include_pair != 0;
  constexpr int B = PME_STAGES_PER_PASS;
  int st, t;
  // inputs bit for bit those of the plan's last forward (checked on the device): that
  // forward's sorted order, records and pair lists are reused; otherwise everything is redone
  const bool reuse = p->fwd_n == n;
  const bool cached = reuse && pair && p->fwd_lists;
  p->fwd_n = -1;   // a backward leaves nothing for a later one
  t = prof_begin(p, B + 0, s);
  if (reuse && (st = launch_input_check(p, s, in, cached))) return st;
  if ((st = launch_sort(p, s, in, true, true, pair, reuse ? p->in_diff : nullptr))) return st;
  prof_end(p, t, s);
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (pair) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, B + 6, ps);
    if ((st = launch_pair(p, ps, n, true, in, gE, p->pair_out, cached ? p->cache_bad : nullptr)))
      return st;
    if (cached) {
      const int te = prof_begin(p, B + 8, ps);
      if ((st = launch_pair_listed(p, ps, n, true, gE, p->pair_out, p->cache_bad))) return st;
      prof_end(p, te, ps);
    }
    prof_end(p, t, ps);
  }
  t = prof_begin(p, B + 1, s);
  if ((st = launch_spread(p, s, true, p->rho, reuse ? p->in_diff : nullptr))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 2, s);
  const int* keep = reuse ? p->in_diff : nullptr;
  if ((st = fft_forward(p, s, true, keep))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 3, s);
  if ((st = multiply_influence(p, s, true, nullptr, keep))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 4, s);
  if ((st = fft_inverse(p, s, true, keep))) return st;
  prof_end(p, t, s);
  // the pair term (side stream) has long finished by now: join first, so that the tangent
  // gather also does the final per-ion assembly (no separate combine launch)
  if (pair && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, B + 5, s);
  const BackwardFinish fin = backward_finish_args(p, in, o_pos, o_q, o_mu);
  if ((st = launch_gather_finish(p, s, n, p->phi, gE, fin))) return st;
  prof_end(p, t, s);
  return PME_OK;
}

static int validate_opts(pme_plan_s* p, double alpha, double rcut) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return set_error(p, PME_ERR_ARG, "alpha must be > 0");
  if (p->opts.include_pair && !(rcut > 0.0)) return set_error(p, PME_ERR_ARG, "rcut must be > 0");
  if (p->opts.max_ions <= 0) return set_error(p, PME_ERR_ARG, "max_ions must be > 0");
  if (!(p->opts.influence_power >= 0.0)) return set_error(p, PME_ERR_ARG, "influence_power < 0");
  if (p->opts.recip_method < 0 || p->opts.recip_method > 1) return set_error(p, PME_ERR_ARG, "recip_method");
  if (p->opts.influence_kind < 0 || p->opts.influence_kind > 1) return set_error(p, PME_ERR_ARG, "influence_kind");
  if (p->opts.fft < 0 || p->opts.fft > 3) return set_error(p, PME_ERR_ARG, "fft");
  p->opts_kmax = p->opts.ewald_kmax > 0.0 ? p->opts.ewald_kmax : 2.0 * alpha * std::sqrt(std::log(1e8));
  return PME_OK;
}

}  // namespace gbpme

using namespace gbpme;

extern "C" {

void pme_opts_default(pme_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->influence_power = 1.0;
  o->deconvolution = 1;
  o->coulomb_k = 1.0;
  o->include_pair = 1;
  o->include_self = 1;
  o->include_background = 1;
  o->max_ions = 1 << 18;
  o->overlap_pair = 1;
  o->recip_method = 0;
  o->ewald_kmax = 0.0;
  o->autotune = 1;
}

const char* pme_status_string(int s) {
  switch (s) {
    case PME_OK: return "ok";
    case PME_ERR_ARG: return "invalid argument";
    case PME_ERR_CUDA: return "CUDA error";
    case PME_ERR_CUFFT: return "cuFFT error";
    case PME_ERR_NONFINITE: return "non-finite input";
    case PME_ERR_UNSUPPORTED: return "unsupported option";
    case PME_ERR_TIMEOUT: return "device wait timed out";
    case PME_ERR_NOMEM: return "out of device memory";
    case PME_ERR_BOUNDS: return "index check failed";
    default: return "unknown status";
  }
}

const char* pme_last_error(pme_plan_t p) { return p ? p->last_error.c_str() : "null plan"; }

long long pme_launch_count(void) { return g_launches.load(); }

static int next_smooth(int n) {
  for (int m = std::max(1, n);; ++m) {
    int r = m;
    for (int f : {2, 3, 5})
      while (r % f == 0) r /= f;
    if (r == 1) return m;
  }
}

static int next_pow2(int n) {
  int m = 1;
  while (m < n) m <<= 1;
  return m;
}

int pme_mesh_dims(const double box[9], double spacing, int rule, int strategy, int clamp_lo,
                  int clamp_hi, int mesh[3]) {
  if (!box || !mesh || !(spacing > 0.0) || rule < 0 || rule > 1 || strategy < 0 || strategy > 2)
    return PME_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    const double L = std::sqrt(box[3 * a] * box[3 * a] + box[3 * a + 1] * box[3 * a + 1] +
                               box[3 * a + 2] * box[3 * a + 2]);
    const double t = rule == 0 ? std::ceil(2.0 * L / spacing + 1.0) : std::ceil(L / spacing);
    if (!(t >= 1.0 && t < 1e6)) return PME_ERR_ARG;
    int n = int(t);
    if (strategy == 0) n = next_pow2(n);
    else if (strategy == 1) n = next_smooth(n);
    if (clamp_lo > 0) n = std::max(n, clamp_lo);
    if (clamp_hi > 0) n = std::min(n, clamp_hi);
    mesh[a] = n;
  }
  return PME_OK;
}

int pme_plan_create(pme_plan_t* out, const double box[9], const int mesh[3], int order,
                    double alpha, double rcut, const pme_opts* opts) {
  if (!out) return PME_ERR_ARG;
  *out = nullptr;
  if (!box || !mesh) return PME_ERR_ARG;
  pme_plan_s* p = new (std::nothrow) pme_plan_s();
  if (!p) return PME_ERR_NOMEM;
  if (opts) p->opts = *opts;
  else pme_opts_default(&p->opts);
  int st = validate_opts(p, alpha, rcut);
  // automatic brick: the autotuner's (cached) choice for this mesh, order and capacity
  if (st == PME_OK && p->opts.autotune && p->opts.recip_method == 0 && p->opts.brick[0] == 0 &&
      p->opts.brick[1] == 0 && p->opts.brick[2] == 0 && order >= 1 && order <= kMaxOrder) {
    int b[3];
    if (autotune_brick(box, mesh, order, alpha, rcut, p->opts.max_ions, p->opts, b, nullptr, true) == PME_OK)
      for (int a = 0; a < 3; ++a) p->opts.brick[a] = b[a];
  }
  if (st == PME_OK) {
    p->max_ions = p->opts.max_ions;
    FrameInput fi{box, {mesh[0], mesh[1], mesh[2]}, order, 0, p->max_ions};
    st = build_plan(p, {fi}, alpha, rcut, true);
  }
  if (st == PME_OK && p->opts.recip_method == 1) {
    const size_t ni = size_t(p->max_ions);
    if ((st = dalloc(p, &p->ew_fx, ni)) == PME_OK && (st = dalloc(p, &p->ew_qm, ni)) == PME_OK)
      st = setup_kvectors(p);
  }
  if (st) {
    free_plan(p);   // the plan (and its error text) is released; only the status survives
    return st;
  }
  *out = p;
  return PME_OK;
}

int pme_batch_create(pme_plan_t* out, int nframes, const int* offsets, const double* boxes,
                     const int* meshes, const int* orders, double alpha, double rcut,
                     const pme_opts* opts) {
  if (!out) return PME_ERR_ARG;
  *out = nullptr;
  if (nframes <= 0 || !offsets || !boxes || !meshes || !orders) return PME_ERR_ARG;
  if (offsets[0] != 0) return PME_ERR_ARG;
  for (int f = 0; f < nframes; ++f)
    if (offsets[f + 1] < offsets[f]) return PME_ERR_ARG;
  pme_plan_s* p = new (std::nothrow) pme_plan_s();
  if (!p) return PME_ERR_NOMEM;
  if (opts) p->opts = *opts;
  else pme_opts_default(&p->opts);
  int st = validate_opts(p, alpha, rcut);
  if (st == PME_OK && p->opts.recip_method != 0) st = PME_ERR_UNSUPPORTED;
  if (st == PME_OK) {
    p->max_ions = std::max(1, offsets[nframes]);
    std::vector<FrameInput> fin(nframes);
    for (int f = 0; f < nframes; ++f)
      fin[f] = FrameInput{boxes + 9 * f, {meshes[3 * f], meshes[3 * f + 1], meshes[3 * f + 2]}, orders[f],
                          offsets[f], offsets[f + 1] - offsets[f]};
    st = build_plan(p, fin, alpha, rcut, false);
  }
  if (st) {
    free_plan(p);
    return st;
  }
  *out = p;
  return PME_OK;
}

int pme_batch_frames(pme_plan_t p) { return p ? p->nframes : 0; }

int pme_plan_brick(pme_plan_t p, int brick[3]) {
  if (!p || !brick) return PME_ERR_ARG;
  for (int a = 0; a < 3; ++a) brick[a] = p->frames_h[0].g.brick[a];
  return PME_OK;
}

int pme_plan_set_box(pme_plan_t p, const double box[9]) {
  if (!p || !box) return PME_ERR_ARG;
  if (p->batch) return set_error(p, PME_ERR_UNSUPPORTED, "pme_plan_set_box takes a single-frame plan");
  FrameDesc& D = p->frames_h[0];
  Geometry g = D.g;
  int nc = 0;
  std::string why;
  if (!frame_geometry(g, box, p->rcut, p->opts.include_pair != 0, &nc, why)) return set_error(p, PME_ERR_ARG, why);
  int st = check_cuda(p, cudaDeviceSynchronize(), "synchronize");
  if (st) return st;
  D.g = g;
  D.ncells = nc;
  p->g = g;
  p->fwd_n = -1;   // the saved forward belongs to the old box
  drop_graphs(p);  // recorded passes carry the old geometry
  std::memcpy(p->box, box, sizeof(double) * 9);
  if (p->gtab && ((st = launch_influence_tables(p, 0)) || (st = check_cuda(p, cudaDeviceSynchronize(), "synchronize"))))
    return st;
  if (nc > p->total_cells) {
    cudaFree(p->sb.count_c);
    cudaFree(p->sb.start_c);
    p->sb.count_c = p->sb.start_c = nullptr;
    p->total_cells = nc;
    if ((st = alloc_cells(p))) return st;
  }
  p->total_cells = std::max(p->total_cells, nc);
  if (p->opts.recip_method == 1) return setup_kvectors(p);
  return PME_OK;
}

int pme_plan_destroy(pme_plan_t p) {
  if (!p) return PME_ERR_ARG;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  free_plan(p);
  return PME_OK;
}

int pme_plan_fft_kind(pme_plan_t p, int* kind) {
  if (!p || !kind) return PME_ERR_ARG;
  *kind = p->conv ? (p->conv_p2 ? 2 : 0) : 1;
  return PME_OK;
}

int pme_sync_status(pme_plan_t p, void* stream) {
  if (!p) return PME_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = check_cuda(p, cudaStreamSynchronize(s), "stream synchronize");
  if (st) return st;
  int flags = 0;
  if ((st = check_cuda(p, cudaMemcpy(&flags, p->flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags")))
    return st;
  if (flags) cudaMemset(p->flags, 0, sizeof(int));
  if (flags & kFlagNonFinite) return set_error(p, PME_ERR_NONFINITE, "non-finite value in pos, q, mu or theta");
  if (flags & kFlagTimeout) return set_error(p, PME_ERR_TIMEOUT, "device wait timed out");
  if (flags & kFlagVirialLost)
    return set_error(p, PME_ERR_UNSUPPORTED,
                     "virial: a pair-hit list overflowed, so the pair part of the virial is missing");
  if (flags & kFlagQuadLost)
    return set_error(p, PME_ERR_UNSUPPORTED,
                     "quadrupole backward: a pair-hit list overflowed, so the pair part is missing");
  if (pme_bounds_flags()) return set_error(p, PME_ERR_BOUNDS, "an index check failed (index-checking build)");
  return PME_OK;
}

int pme_bounds_flags(void) {
  int v = 0;
  v |= bounds_hit_spread() ? 1 : 0;
  v |= (bounds_hit_spread_8x8x32() | bounds_hit_spread_16x8x16() | bounds_hit_spread_16x16x16() |
        bounds_hit_spread_4x8x16()) ? 1 : 0;
  v |= bounds_hit_gather() ? 2 : 0;
  v |= bounds_hit_pair() ? 4 : 0;
  v |= bounds_hit_combine() ? 8 : 0;
  v |= bounds_hit_sort() ? 16 : 0;
  return v;
}

int pme_bounds_checking(void) {
#ifdef GBPME_BOUNDS
  return 1;
#else
  return 0;
#endif
}

int pme_forward(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
                const float* mu, double* energy, float* force, float* phi, float* field,
                float* field_grad) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.n = n;
  double* e_out = sg.out_d(energy, 1, 0);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if ((st = sg.ready())) return st;
  const PassKey key = make_key({0ull, (unsigned long long)n, ptr_bits(in.pos), ptr_bits(in.q), ptr_bits(in.mu),
                                ptr_bits(e_out), ptr_bits(f_out), ptr_bits(p_out), ptr_bits(fl_out),
                                ptr_bits(fg_out)});
  st = run_pass(p, 0, s, key, true,
                [&](cudaStream_t cs) { return run_forward(p, cs, in, e_out, f_out, p_out, fl_out, fg_out); });
  if (st) return st;
  return sg.finish();
}

int pme_forward_virial(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
                       const float* mu, double* energy, float* force, float* phi, float* field,
                       float* field_grad, double* virial) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  if (!energy || !virial) return set_error(p, PME_ERR_ARG, "pme_forward_virial needs energy and virial");
  if (p->opts.recip_method != 0 || p->opts.influence_kind != 0)
    return set_error(p, PME_ERR_UNSUPPORTED,
                     "the virial needs the particle-mesh method with the sinc-deconvolution influence");
  if (p->opts.include_pair && !p->plist)
    return set_error(p, PME_ERR_UNSUPPORTED, "the virial needs the plan's pair-hit lists (too large for this plan)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.n = n;
  double* e_out = sg.out_d(energy, 1, 0);
  double* v_out = sg.out_d(virial, 9, 2);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if ((st = sg.ready())) return st;
  if ((st = run_forward(p, s, in, e_out, f_out, p_out, fl_out, fg_out, v_out))) return st;
  return sg.finish();
}

// Forward with point quadrupoles (the rank-2 channel) over every frame of the plan: sort,
// quadrupole spread, the mesh convolution, quadrupole gather, the quadrupole pair kernel,
// combine. Runs directly (no graph) and leaves nothing for a backward to reuse.
static int run_forward_quad(pme_plan_t p, cudaStream_t s, const IonInputs& in, double* e_out,
                            float* f_out, float* p_out, float* fl_out, float* fg_out) {
  const int n = in.n;
  const bool pair = p->opts.include_pair != 0;
  int st;
  int t;
  p->fwd_n = -1;
  p->fwd_lists = false;
  t = prof_begin(p, 0, s);
  if ((st = launch_sort(p, s, in, false, true, pair, nullptr))) return st;
  prof_end(p, t, s);
  const bool fork = pair && n > 0;
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (fork) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, 6, ps);
    if (p->plist) {
      // hit lists from the list pass, evaluated per ion; the cell walk only if one overflowed
      if ((st = launch_pair_build(p, ps, n, p->cache_bad))) return st;
      if ((st = launch_pair_quad(p, ps, n, in.theta, p->pair_out, p->quad_out, p->cache_bad))) return st;
      const int te = prof_begin(p, 8, ps);
      if ((st = launch_pair_quad_listed(p, ps, n, in.theta, p->pair_out, p->quad_out, p->cache_bad)))
        return st;
      prof_end(p, te, ps);
    } else if ((st = launch_pair_quad(p, ps, n, in.theta, p->pair_out, p->quad_out))) {
      return st;
    }
    prof_end(p, t, ps);
  }
  t = prof_begin(p, 1, s);
  if ((st = launch_spread_quad(p, s, in.theta, p->rho))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 2, s);
  if ((st = fft_forward(p, s, false))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 3, s);
  if ((st = multiply_influence(p, s, false, nullptr))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 4, s);
  if ((st = fft_inverse(p, s, false))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 5, s);
  if ((st = launch_gather_quad(p, s, n, p->phi, in.theta, p->mesh_out, p->quad_out))) return st;
  prof_end(p, t, s);
  if (fork && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, 7, s);
  st = launch_combine_forward(p, s, in, true, fork, f_out, p_out, fl_out, fg_out, e_out, 1, nullptr,
                              p->quad_out);
  prof_end(p, t, s);
  return st;
}

// The quadrupole density Theta : grad grad W is continuous in r only when the second
// derivative of W is, i.e. for spline order p >= 4 (for p <= 3 it jumps at mesh points and
// the third derivative vanishes between them): below that the mesh energy is not a smooth
// function of the positions and Theta : grad^3 phi is not its gradient, so those orders are
// refused.
static int check_quad_orders(pme_plan_t p) {
  for (int f = 0; f < p->nframes; ++f)
    if (p->frames_h[f].g.order < 4)
      return set_error(p, PME_ERR_UNSUPPORTED, "quadrupoles need spline order >= 4 in every frame");
  return PME_OK;
}

int pme_forward_quad(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
                     const float* mu, const float* theta, double* energy, float* force, float* phi,
                     float* field, float* field_grad) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  if (n > 0 && !theta) return set_error(p, PME_ERR_ARG, "theta is NULL");
  if (p->opts.recip_method != 0)
    return set_error(p, PME_ERR_UNSUPPORTED, "quadrupoles need the particle-mesh method (recip_method 0)");
  if ((st = check_quad_orders(p))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.theta = sg.in(theta, 6, kTheta);
  in.n = n;
  double* e_out = sg.out_d(energy, 1, 0);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if ((st = sg.ready())) return st;
  if ((st = run_forward_quad(p, s, in, e_out, f_out, p_out, fl_out, fg_out))) return st;
  return sg.finish();
}

static int check_batch(pme_plan_t p, const float* pos, const float* q);

int pme_batch_forward_quad(pme_plan_t p, void* stream, const float* pos, const float* q,
                           const float* mu, const float* theta, double* energy, float* force,
                           float* phi, float* field, float* field_grad) {
  int st = check_batch(p, pos, q);
  if (st) return st;
  const int n = p->frame_offsets[p->nframes];
  if (n > 0 && !theta) return set_error(p, PME_ERR_ARG, "theta is NULL");
  if ((st = check_quad_orders(p))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.theta = sg.in(theta, 6, kTheta);
  in.n = n;
  double* e_out = sg.out_d(energy, p->nframes, 0);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if ((st = sg.ready())) return st;
  if ((st = run_forward_quad(p, s, in, e_out, f_out, p_out, fl_out, fg_out))) return st;
  return sg.finish();
}

// Backward with point quadrupoles: the Hessian-vector product along v = (dr, dq, dmu) plus
// g_E times the gradient, in (r, q, mu, Theta). The mesh part spreads rho (with Theta) and the
// tangent density d rho (third spline derivatives), transforms both, and gathers the 13
// quadrupole-forward values with their tangents (moments of Phi to order 4, of d Phi to 3);
// the pair part evaluates the same 13 sums in dual numbers over the hit lists; the combine
// assembles the gradients and their tangents with the self and background terms.
static int run_backward_quad(pme_plan_t p, cudaStream_t s, const IonInputs& in, const double* gE,
                             float* o_pos, float* o_q, float* o_mu, float* o_theta) {
  const int n = in.n;
  if (n == 0) return PME_OK;
  const bool pair = p->opts.include_pair != 0;
  constexpr int B = PME_STAGES_PER_PASS;
  int st, t;
  p->fwd_n = -1;   // nothing of this pass is reused by a later call
  p->fwd_lists = false;
  t = prof_begin(p, B + 0, s);
  if ((st = launch_sort(p, s, in, true, true, pair, nullptr))) return st;
  prof_end(p, t, s);
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (pair) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, B + 6, ps);
    if ((st = launch_pair_build(p, ps, n, p->cache_bad))) return st;
    if ((st = launch_pair_quad_dual(p, ps, n, in.theta, p->qb_pair, p->cache_bad))) return st;
    prof_end(p, t, ps);
  }
  t = prof_begin(p, B + 1, s);
  if ((st = launch_spread_quad(p, s, in.theta, p->rho))) return st;
  if ((st = launch_spread_quad_tangent(p, s, in.theta, p->rho))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 2, s);
  if ((st = fft_forward(p, s, true))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 3, s);
  if ((st = multiply_influence(p, s, true, nullptr))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 4, s);
  if ((st = fft_inverse(p, s, true))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 5, s);
  if ((st = launch_gather_qdual(p, s, n, p->phi, in.theta, p->qb_mesh))) return st;
  prof_end(p, t, s);
  if (pair && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, B + 7, s);
  st = launch_combine_backward_quad(p, s, in, gE, p->qb_mesh, p->qb_pair, o_pos, o_q, o_mu, o_theta);
  prof_end(p, t, s);
  return st;
}

static int backward_quad_common(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
                                const float* mu, const float* theta, const double* g_energy,
                                const float* g_force, const float* g_phi, const float* g_field,
                                float* grad_pos, float* grad_q, float* grad_mu, float* grad_theta, int nE) {
  int st;
  if (n > 0 && !theta) return set_error(p, PME_ERR_ARG, "theta is NULL");
  if ((st = check_quad_orders(p))) return st;
  if (p->opts.include_pair && !p->plist)
    return set_error(p, PME_ERR_UNSUPPORTED, "the quadrupole backward needs the plan's pair-hit lists");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.theta = sg.in(theta, 6, kTheta);
  in.gforce = sg.in(g_force, 3, kGF);
  in.gphi = sg.in(g_phi, 1, kGPhi);
  in.gfield = sg.in(g_field, 3, kGField);
  in.n = n;
  const double* gE = sg.in_d(g_energy, nE, 1);
  float* o_pos = sg.out(grad_pos, 3, kOGPos);
  float* o_q = sg.out(grad_q, 1, kOGQ);
  float* o_mu = sg.out(grad_mu, 3, kOGMu);
  float* o_th = sg.out(grad_theta, 6, kOGTheta);
  if ((st = sg.ready())) return st;
  if ((st = run_backward_quad(p, s, in, gE, o_pos, o_q, o_mu, o_th))) return st;
  return sg.finish();
}

int pme_backward_quad(pme_plan_t p, void* stream, int n, const float* pos, const float* q, const float* mu,
                      const float* theta, const double* g_energy, const float* g_force, const float* g_phi,
                      const float* g_field, float* grad_pos, float* grad_q, float* grad_mu, float* grad_theta) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  if (p->opts.recip_method != 0)
    return set_error(p, PME_ERR_UNSUPPORTED, "quadrupoles need the particle-mesh method (recip_method 0)");
  return backward_quad_common(p, stream, n, pos, q, mu, theta, g_energy, g_force, g_phi, g_field, grad_pos,
                              grad_q, grad_mu, grad_theta, 1);
}

int pme_batch_backward_quad(pme_plan_t p, void* stream, const float* pos, const float* q, const float* mu,
                            const float* theta, const double* g_energy, const float* g_force,
                            const float* g_phi, const float* g_field, float* grad_pos, float* grad_q,
                            float* grad_mu, float* grad_theta) {
  int st = check_batch(p, pos, q);
  if (st) return st;
  const int n = p->frame_offsets[p->nframes];
  return backward_quad_common(p, stream, n, pos, q, mu, theta, g_energy, g_force, g_phi, g_field, grad_pos,
                              grad_q, grad_mu, grad_theta, p->nframes);
}

int pme_backward(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
                 const float* mu, const double* g_energy, const float* g_force,
                 const float* g_phi, const float* g_field, float* grad_pos, float* grad_q,
                 float* grad_mu) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  if (p->opts.recip_method != 0)
    return set_error(p, PME_ERR_UNSUPPORTED, "pme_backward needs the particle-mesh reciprocal method");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.gforce = sg.in(g_force, 3, kGF);
  in.gphi = sg.in(g_phi, 1, kGPhi);
  in.gfield = sg.in(g_field, 3, kGField);
  in.n = n;
  const double* gE = sg.in_d(g_energy, 1, 1);
  float* o_pos = sg.out(grad_pos, 3, kOGPos);
  float* o_q = sg.out(grad_q, 1, kOGQ);
  float* o_mu = sg.out(grad_mu, 3, kOGMu);
  if ((st = sg.ready())) return st;
  const PassKey key = make_key({1ull, (unsigned long long)n, ptr_bits(in.pos), ptr_bits(in.q), ptr_bits(in.mu),
                                ptr_bits(gE), ptr_bits(in.gforce), ptr_bits(in.gphi), ptr_bits(in.gfield),
                                ptr_bits(o_pos), ptr_bits(o_q), ptr_bits(o_mu),
                                (unsigned long long)(long long)p->fwd_n, (unsigned long long)p->fwd_lists});
  st = run_pass(p, 1, s, key, true,
                [&](cudaStream_t cs) { return run_backward(p, cs, in, gE, o_pos, o_q, o_mu); });
  if (st) return st;
  return sg.finish();
}

static int check_batch(pme_plan_t p, const float* pos, const float* q) {
  if (!p) return PME_ERR_ARG;
  if (!p->batch) return set_error(p, PME_ERR_ARG, "single-frame plan: use pme_forward / pme_backward");
  if (p->frame_offsets[p->nframes] > 0 && (!pos || !q)) return set_error(p, PME_ERR_ARG, "pos or q is NULL");
  return set_device(p);
}

int pme_batch_forward(pme_plan_t p, void* stream, const float* pos, const float* q, const float* mu,
                      double* energy, float* force, float* phi, float* field, float* field_grad) {
  int st = check_batch(p, pos, q);
  if (st) return st;
  const int n = p->frame_offsets[p->nframes];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.n = n;
  double* e_out = sg.out_d(energy, p->nframes, 0);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if ((st = sg.ready())) return st;
  const PassKey key = make_key({0ull, (unsigned long long)n, ptr_bits(in.pos), ptr_bits(in.q), ptr_bits(in.mu),
                                ptr_bits(e_out), ptr_bits(f_out), ptr_bits(p_out), ptr_bits(fl_out),
                                ptr_bits(fg_out)});
  st = run_pass(p, 0, s, key, true,
                [&](cudaStream_t cs) { return run_forward(p, cs, in, e_out, f_out, p_out, fl_out, fg_out); });
  if (st) return st;
  return sg.finish();
}

int pme_batch_forward_virial(pme_plan_t p, void* stream, const float* pos, const float* q,
                             const float* mu, double* energy, float* force, float* phi,
                             float* field, float* field_grad, double* virial) {
  int st = check_batch(p, pos, q);
  if (st) return st;
  if (!energy || !virial) return set_error(p, PME_ERR_ARG, "pme_batch_forward_virial needs energy and virial");
  if (p->opts.influence_kind != 0)
    return set_error(p, PME_ERR_UNSUPPORTED, "the virial needs the sinc-deconvolution influence");
  if (p->opts.include_pair && !p->plist)
    return set_error(p, PME_ERR_UNSUPPORTED, "the virial needs the plan's pair-hit lists (too large for this plan)");
  const int n = p->frame_offsets[p->nframes];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.n = n;
  double* e_out = sg.out_d(energy, p->nframes, 0);
  double* v_out = sg.out_d(virial, 9 * p->nframes, 2);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if ((st = sg.ready())) return st;
  if ((st = run_forward(p, s, in, e_out, f_out, p_out, fl_out, fg_out, v_out))) return st;
  return sg.finish();
}

int pme_batch_backward(pme_plan_t p, void* stream, const float* pos, const float* q, const float* mu,
                       const double* g_energy, const float* g_force, const float* g_phi,
                       const float* g_field, float* grad_pos, float* grad_q, float* grad_mu) {
  int st = check_batch(p, pos, q);
  if (st) return st;
  const int n = p->frame_offsets[p->nframes];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Staging sg(p, s, n);
  IonInputs in{};
  in.pos = sg.in(pos, 3, kPos);
  in.q = sg.in(q, 1, kQ);
  in.mu = sg.in(mu, 3, kMu);
  in.gforce = sg.in(g_force, 3, kGF);
  in.gphi = sg.in(g_phi, 1, kGPhi);
  in.gfield = sg.in(g_field, 3, kGField);
  in.n = n;
  const double* gE = sg.in_d(g_energy, p->nframes, 1);
  float* o_pos = sg.out(grad_pos, 3, kOGPos);
  float* o_q = sg.out(grad_q, 1, kOGQ);
  float* o_mu = sg.out(grad_mu, 3, kOGMu);
  if ((st = sg.ready())) return st;
  const PassKey key = make_key({1ull, (unsigned long long)n, ptr_bits(in.pos), ptr_bits(in.q), ptr_bits(in.mu),
                                ptr_bits(gE), ptr_bits(in.gforce), ptr_bits(in.gphi), ptr_bits(in.gfield),
                                ptr_bits(o_pos), ptr_bits(o_q), ptr_bits(o_mu),
                                (unsigned long long)(long long)p->fwd_n, (unsigned long long)p->fwd_lists});
  st = run_pass(p, 1, s, key, true,
                [&](cudaStream_t cs) { return run_backward(p, cs, in, gE, o_pos, o_q, o_mu); });
  if (st) return st;
  return sg.finish();
}

int pme_spread(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
               const float* mu, float* rho) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  if (!rho || !is_device_pointer(rho) || !is_device_pointer(pos) || !is_device_pointer(q) ||
      !is_device_pointer(mu))
    return set_error(p, PME_ERR_ARG, "pme_spread takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IonInputs in{};
  in.pos = pos;
  in.q = q;
  in.mu = mu;
  in.n = n;
  if ((st = launch_sort(p, s, in, false, true, false, nullptr))) return st;
  return launch_spread(p, s, false, rho);   // frame 0's rho sits at offset 0
}

int pme_solve(pme_plan_t p, void* stream, const float* rho, float* phi_mesh, double* e_recip) {
  if (!p) return PME_ERR_ARG;
  int st = check_common(p, 0, nullptr, nullptr);
  if (st) return st;
  if (!rho || !phi_mesh || !is_device_pointer(rho) || !is_device_pointer(phi_mesh) ||
      !is_device_pointer(e_recip))
    return set_error(p, PME_ERR_ARG, "pme_solve takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const FFTGroup& G = p->fgroups[0];
  p->fwd_n = -1;   // the plan's rho is about to be replaced: nothing saved for a backward
  if ((st = check_cuda(p, cudaMemcpyAsync(p->rho, rho, sizeof(float) * p->M, cudaMemcpyDeviceToDevice, s),
                       "copy rho")))
    return st;
  if (p->conv) {
    if ((st = launch_conv_forward(p, s, false, p->rho)) || (st = multiply_influence(p, s, false, nullptr)) ||
        (st = launch_conv_inverse(p, s, false, phi_mesh)))
      return st;
  } else {
    if ((st = check_fft(p, cufftSetStream(G.r2c, s), "set stream"))) return st;
    if ((st = check_fft(p, cufftExecR2C(G.r2c, p->rho, p->spec), "exec r2c"))) return st;
    if ((st = launch_influence(p, s, p->spec, false, p->epart))) return st;
    if ((st = check_fft(p, cufftSetStream(G.c2r, s), "set stream"))) return st;
    if ((st = check_fft(p, cufftExecC2R(G.c2r, p->spec, phi_mesh), "exec c2r"))) return st;
  }
  if (e_recip) return launch_energy_final(p, s, p->epart, 1, false, false, 1.0, 0, e_recip);
  return PME_OK;
}

int pme_gather(pme_plan_t p, void* stream, int n, const float* pos, const float* phi_mesh,
               float* out) {
  int st = check_common(p, n, pos, pos);   // no charges needed: the sort only reads pos
  if (st) return st;
  if (!phi_mesh || !out || !is_device_pointer(pos) || !is_device_pointer(phi_mesh) ||
      !is_device_pointer(out))
    return set_error(p, PME_ERR_ARG, "pme_gather takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IonInputs in{};
  in.pos = pos;
  in.q = nullptr;
  in.n = n;
  if ((st = launch_sort(p, s, in, false, true, false, nullptr))) return st;
  return launch_gather(p, s, n, phi_mesh, false, nullptr, out);
}

int pme_pair(pme_plan_t p, void* stream, int n, const float* pos, const float* q,
             const float* mu, float* out, double* e_pair) {
  int st = check_common(p, n, pos, q);
  if (st) return st;
  if (!p->opts.include_pair) return set_error(p, PME_ERR_UNSUPPORTED, "plan has include_pair = 0");
  if (!out || !is_device_pointer(pos) || !is_device_pointer(q) || !is_device_pointer(mu) ||
      !is_device_pointer(out) || !is_device_pointer(e_pair))
    return set_error(p, PME_ERR_ARG, "pme_pair takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IonInputs in{};
  in.pos = pos;
  in.q = q;
  in.mu = mu;
  in.n = n;
  if ((st = launch_sort(p, s, in, false, false, true, nullptr))) return st;
  if ((st = launch_pair(p, s, n, false, in, nullptr, out, nullptr))) return st;
  if (e_pair) {
    if ((st = launch_pair_energy(p, s, n, in, out))) return st;
    return launch_energy_final(p, s, p->epart, 0, true, false, 1.0, n, e_pair);
  }
  return PME_OK;
}

int pme_profile_enable(pme_plan_t p, int enable) {
  if (!p) return PME_ERR_ARG;
  if (enable && !p->prof_ev) {
    p->prof_ev = new (std::nothrow) cudaEvent_t[2 * kProfCap];
    p->prof_stage = new (std::nothrow) int[kProfCap];
    if (!p->prof_ev || !p->prof_stage) return set_error(p, PME_ERR_NOMEM, "timer pool");
    for (int k = 0; k < 2 * kProfCap; ++k) {
      int st = check_cuda(p, cudaEventCreate(&p->prof_ev[k]), "cudaEventCreate");
      if (st) return st;
    }
  }
  p->prof = enable != 0;
  p->prof_used = 0;
  return PME_OK;
}

int pme_profile_read(pme_plan_t p, double* ms, long long* calls) {
  if (!p) return PME_ERR_ARG;
  double acc[PME_NUM_STAGES] = {0};
  long long cnt[PME_NUM_STAGES] = {0};
  if (p->prof_used > 0) {
    int st = check_cuda(p, cudaDeviceSynchronize(), "synchronize");
    if (st) return st;
    for (int k = 0; k < p->prof_used; ++k) {
      float t = 0.f;
      st = check_cuda(p, cudaEventElapsedTime(&t, p->prof_ev[2 * k], p->prof_ev[2 * k + 1]),
                      "cudaEventElapsedTime");
      if (st) return st;
      acc[p->prof_stage[k]] += t;
      cnt[p->prof_stage[k]] += 1;
    }
  }
  p->prof_used = 0;
  for (int k = 0; k < PME_NUM_STAGES; ++k) {
    if (ms) ms[k] = acc[k];
    if (calls) calls[k] = cnt[k];
  }
  return PME_OK;
}

}  // extern "C"
