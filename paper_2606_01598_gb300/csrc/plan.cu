// Plan construction (Section 2.3.1: cell, reciprocal basis, mesh; Section 2.3.3: the
// deconvolution tables), host-pointer staging, and the stream orchestration of the forward
// and backward passes behind the C ABI declared in include/gbpme.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"

namespace gbpme {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

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

int prof_begin(pme_plan_t p, int stage, cudaStream_t s) {
  if (!p->prof || p->prof_used >= kProfCap) return -1;
  const int slot = p->prof_used++;
  p->prof_stage[slot] = stage;
  cudaEventRecord(p->prof_ev[2 * slot], s);
  return slot;
}

void prof_end(pme_plan_t p, int slot, cudaStream_t s) {
  if (slot >= 0) cudaEventRecord(p->prof_ev[2 * slot + 1], s);
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
static bool build_candidates(int N, int B, int P, int nb, int max_nb, std::vector<int>& tab,
                             int axis) {
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
    int* row = tab.data() + (axis * max_nb + b) * (1 + kMaxCandPerDim);
    row[0] = int(list.size());
    for (size_t k = 0; k < list.size(); ++k) row[1 + k] = list[k];
  }
  return true;
}

static double sinc(double x) {
  if (x == 0.0) return 1.0;
  return std::sin(kPi * x) / (kPi * x);
}

// Geometry that depends on the box (cell matrices, pair cells). Returns false when the box is
// singular.
static bool set_geometry(pme_plan_t p, const double* box, std::string& why) {
  double inv[9], det;
  if (!invert3(box, inv, &det)) {
    why = "singular or non-finite box";
    return false;
  }
  std::memcpy(p->box, box, sizeof(double) * 9);
  Geometry& g = p->g;
  for (int k = 0; k < 9; ++k) g.cinv[k] = inv[k];
  g.volume = std::fabs(det);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g.D[a * 3 + b] = float(double(g.N[b]) * inv[a * 3 + b]);
  // pair cells at least rcut/2 wide; axes too short for 5 cells loop over images instead
  int ncell = 1;
  for (int a = 0; a < 3; ++a) {
    const double w = perp_width(box, a, g.volume);
    int nc = p->opts.include_pair ? int(std::floor(w / (0.5 * p->rcut))) : 1;
    nc = std::min(nc, 512);
    if (nc >= 5) {
      g.ncell[a] = nc;
      g.kimg[a] = 2;
    } else {
      g.ncell[a] = 1;
      g.kimg[a] = p->opts.include_pair ? int(std::ceil(p->rcut / w)) + 1 : 0;
    }
    ncell *= g.ncell[a];
  }
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) g.H[b * 3 + c] = float(box[b * 3 + c] / g.ncell[b]);
  p->ncells = ncell;
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

enum StageSlot {
  kPos = 0, kQ = 3, kMu = 4, kGF = 7, kGPhi = 10, kGField = 11, kOF = 14, kOPhi = 17,
  kOField = 18, kOFG = 21, kOGPos = 27, kOGQ = 30, kOGMu = 31, kStageFloats = 34
};

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
  std::vector<Pending> outs;

  Staging(pme_plan_t p_, cudaStream_t s_, int n_) : p(p_), s(s_), n(n_) {}

  const float* in(const float* ptr, int width, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    float* d = p->stage_f + size_t(slot) * p->max_ions;
    const size_t bytes = sizeof(float) * size_t(width) * n;
    if (bytes && status == PME_OK)
      status = check_cuda(p, cudaMemcpyAsync(d, ptr, bytes, cudaMemcpyHostToDevice, s),
                          "stage input");
    return d;
  }
  const double* in_d(const double* ptr, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    double* d = p->stage_d + slot;
    if (status == PME_OK)
      status = check_cuda(p, cudaMemcpyAsync(d, ptr, sizeof(double), cudaMemcpyHostToDevice, s),
                          "stage input");
    return d;
  }
  float* out(float* ptr, int width, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    float* d = p->stage_f + size_t(slot) * p->max_ions;
    outs.push_back({ptr, d, sizeof(float) * size_t(width) * n});
    return d;
  }
  double* out_d(double* ptr, int slot) {
    if (!ptr || is_device_pointer(ptr)) return ptr;
    double* d = p->stage_d + slot;
    outs.push_back({ptr, d, sizeof(double)});
    return d;
  }
  int finish() {
    for (auto& o : outs) {
      if (status != PME_OK) break;
      if (o.bytes)
        status = check_cuda(p, cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, s),
                            "stage output");
    }
    return status;
  }
};

static int check_common(pme_plan_t p, int n, const float* pos, const float* q) {
  if (!p) return PME_ERR_ARG;
  if (n < 0 || n > p->max_ions)
    return set_error(p, PME_ERR_ARG, "n = " + std::to_string(n) + " outside [0, max_ions = " +
                                         std::to_string(p->max_ions) + "]");
  if (n > 0 && !pos) return set_error(p, PME_ERR_ARG, "pos is NULL");
  if (n > 0 && !q) return set_error(p, PME_ERR_ARG, "q is NULL");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) {
    int st = check_cuda(p, cudaSetDevice(p->device), "cudaSetDevice");
    if (st) return st;
  }
  return PME_OK;
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

static void free_plan(pme_plan_t p) {
  if (!p) return;
  void* bufs[] = {p->rho, p->spec, p->phi, p->dconv[0], p->dconv[1], p->dconv[2], p->cand,
                  p->sb.key_b, p->sb.key_c, p->sb.slot_b, p->sb.slot_c, p->sb.count_b,
                  p->sb.count_c, p->sb.start_b, p->sb.start_c, p->sb.perm_b, p->sb.perm_c,
                  p->sb.qpart, p->sb.qsum, p->mr.idx, p->mr.fq, p->mr.dm, p->mr.tq, p->mr.tt,
                  p->pr.idx, p->pr.fq, p->pr.mu, p->pr.tq, p->pr.dr, p->pr.cz, p->mesh_out, p->pair_out,
                  p->epart, p->flags, p->stage_f, p->stage_d, p->ew_kn, p->ew_kv, p->ew_S,
                  p->ew_fx, p->ew_qm};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p->r2c1) cufftDestroy(p->r2c1);
  if (p->c2r1) cufftDestroy(p->c2r1);
  if (p->r2c2) cufftDestroy(p->r2c2);
  if (p->c2r2) cufftDestroy(p->c2r2);
  if (p->prof_ev) {
    for (int k = 0; k < 2 * kProfCap; ++k) cudaEventDestroy(p->prof_ev[k]);
    delete[] p->prof_ev;
    delete[] p->prof_stage;
  }
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  delete p;
}

template <typename T>
static int dalloc(pme_plan_t p, T** ptr, size_t count) {
  *ptr = nullptr;
  return check_cuda(p, cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * std::max<size_t>(count, 1)),
                    "cudaMalloc");
}

static int alloc_cells(pme_plan_t p) {
  int st;
  if ((st = dalloc(p, &p->sb.count_c, size_t(p->ncells) + 1))) return st;
  if ((st = dalloc(p, &p->sb.start_c, size_t(p->ncells) + 1))) return st;
  return PME_OK;
}

// (Re)build the explicit-Ewald k-vector tables for the current box.
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
  // the energy partials array must hold one slot per k block
  cudaFree(p->epart);
  p->epart = nullptr;
  const int na = std::max(p->nspec_blocks, ewald_partial_blocks(p));
  return dalloc(p, &p->epart, size_t(na) + p->max_blocks);
}

// Forward with the explicit k-sum in place of the mesh stages.
static int forward_ewald(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool pair, double* e_out,
                         float* f_out, float* p_out, float* fl_out, float* fg_out, Staging& sg) {
  const int n = in.n;
  int st, t;
  t = prof_begin(p, 0, s);
  if ((st = launch_sort(p, s, in, false, false, pair))) return st;
  prof_end(p, t, s);
  const bool fork = pair && n > 0;
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (fork) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, 6, ps);
    if ((st = launch_pair(p, ps, n, false, in, nullptr, p->pair_out))) return st;
    prof_end(p, t, ps);
  }
  t = prof_begin(p, 3, s);
  if ((st = launch_ewald_recip(p, s, in, p->epart, p->mesh_out))) return st;
  prof_end(p, t, s);
  if (fork && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  const int na = ewald_partial_blocks(p);
  t = prof_begin(p, 7, s);
  if ((st = launch_combine_forward(p, s, in, true, fork, p->epart + na, f_out, p_out, fl_out, fg_out)))
    return st;
  prof_end(p, t, s);
  if (e_out) {
    const double bgfac =
        p->opts.include_background ? -kPi / (2.0 * p->g.volume * p->alpha * p->alpha) : 0.0;
    if ((st = launch_energy_final(p, s, p->epart, na, combine_blocks(n), 4.0 * kPi / p->g.volume,
                                  p->opts.coulomb_k, bgfac, p->sb.qsum, e_out)))
      return st;
  }
  return sg.finish();
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
  auto fail = [&](int st, const std::string& why) {
    (void)why;   // the plan (and its error text) is released; only the status survives
    free_plan(p);
    return st;
  };
  if (order < 1 || order > kMaxOrder) return fail(PME_ERR_ARG, "order outside 1..7");
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(PME_ERR_ARG, "alpha must be > 0");
  if (p->opts.include_pair && !(rcut > 0.0)) return fail(PME_ERR_ARG, "rcut must be > 0");
  if (p->opts.max_ions <= 0) return fail(PME_ERR_ARG, "max_ions must be > 0");
  for (int a = 0; a < 3; ++a)
    if (mesh[a] < order || mesh[a] > 4096) return fail(PME_ERR_ARG, "mesh dimension < order");
  if (!(p->opts.influence_power >= 0.0)) return fail(PME_ERR_ARG, "influence_power < 0");
  if (p->opts.recip_method < 0 || p->opts.recip_method > 1) return fail(PME_ERR_ARG, "recip_method");
  p->opts_kmax = p->opts.ewald_kmax > 0.0 ? p->opts.ewald_kmax : 2.0 * alpha * std::sqrt(std::log(1e8));
  Geometry& g = p->g;
  for (int a = 0; a < 3; ++a) g.N[a] = mesh[a];
  g.order = order;
  g.alpha = float(alpha);
  g.rcut2 = float(rcut * rcut);
  p->alpha = alpha;
  p->rcut = rcut;
  p->max_ions = p->opts.max_ions;
  p->max_blocks = (p->max_ions + 255) / 256;
  std::string why;
  if (!set_geometry(p, box, why)) return fail(PME_ERR_ARG, why);
  spread_brick_shape(g.brick);
  for (int a = 0; a < 3; ++a) g.nb[a] = (g.N[a] + g.brick[a] - 1) / g.brick[a];
  p->nbricks = g.nb[0] * g.nb[1] * g.nb[2];
  p->max_nb = std::max(g.nb[0], std::max(g.nb[1], g.nb[2]));
  std::vector<int> cand(size_t(3) * p->max_nb * (1 + kMaxCandPerDim), 0);
  for (int a = 0; a < 3; ++a)
    if (!build_candidates(g.N[a], g.brick[a], order, g.nb[a], p->max_nb, cand, a))
      return fail(PME_ERR_UNSUPPORTED, "mesh / brick / order combination not supported");
  p->M = g.N[0] * g.N[1] * g.N[2];
  p->Mh = g.N[0] * g.N[1] * (g.N[2] / 2 + 1);
  cudaGetDevice(&p->device);

  int st = PME_OK;
  auto A = [&](auto** ptr, size_t count) {
    if (st == PME_OK) st = dalloc(p, ptr, count);
  };
  A(&p->rho, size_t(2) * p->M);
  A(&p->spec, size_t(2) * p->Mh);
  A(&p->phi, size_t(2) * p->M);
  for (int a = 0; a < 3; ++a) A(&p->dconv[a], size_t(g.N[a]));
  A(&p->cand, cand.size());
  const size_t ni = size_t(p->max_ions);
  A(&p->sb.key_b, ni);
  A(&p->sb.key_c, ni);
  A(&p->sb.slot_b, ni);
  A(&p->sb.slot_c, ni);
  A(&p->sb.perm_b, ni);
  A(&p->sb.perm_c, ni);
  A(&p->sb.count_b, size_t(p->nbricks) + 1);
  A(&p->sb.start_b, size_t(p->nbricks) + 1);
  A(&p->sb.qpart, size_t(2) * p->max_blocks);
  A(&p->sb.qsum, 2);
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
  A(&p->pr.cz, ni);
  A(&p->mesh_out, ni * 10);
  A(&p->pair_out, ni * 10);
  p->nspec_blocks = influence_grid(p);
  A(&p->epart, size_t(p->nspec_blocks) + p->max_blocks);
  A(&p->flags, 1);
  A(&p->stage_f, ni * kStageFloats);
  A(&p->stage_d, 4);
  if (st == PME_OK) st = alloc_cells(p);
  if (p->opts.recip_method == 1) {
    A(&p->ew_fx, ni);
    A(&p->ew_qm, ni);
    if (st == PME_OK) st = setup_kvectors(p);
  }
  if (st) return fail(st, p->last_error);
  if ((st = check_cuda(p, cudaMemset(p->flags, 0, sizeof(int)), "memset"))) return fail(st, p->last_error);
  if ((st = check_cuda(p, cudaMemcpy(p->cand, cand.data(), sizeof(int) * cand.size(),
                                     cudaMemcpyHostToDevice), "copy candidates")))
    return fail(st, p->last_error);
  // deconvolution C(n) = 1 / sinc^(2 p gamma)(n / N) per axis (Eqs. Bk, influence)
  for (int a = 0; a < 3; ++a) {
    std::vector<float> t(g.N[a]);
    for (int i = 0; i < g.N[a]; ++i) {
      const int nsig = (i <= g.N[a] / 2) ? i : i - g.N[a];
      const double b = std::pow(sinc(double(nsig) / g.N[a]), double(order));
      t[i] = p->opts.deconvolution ? float(std::pow(b * b, -p->opts.influence_power)) : 1.f;
    }
    if ((st = check_cuda(p, cudaMemcpy(p->dconv[a], t.data(), sizeof(float) * t.size(),
                                       cudaMemcpyHostToDevice), "copy deconvolution")))
      return fail(st, p->last_error);
  }
  int dims[3] = {g.N[0], g.N[1], g.N[2]};
  if ((st = check_fft(p, cufftPlanMany(&p->r2c1, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 1), "plan r2c")) ||
      (st = check_fft(p, cufftPlanMany(&p->c2r1, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 1), "plan c2r")) ||
      (st = check_fft(p, cufftPlanMany(&p->r2c2, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_R2C, 2), "plan r2c x2")) ||
      (st = check_fft(p, cufftPlanMany(&p->c2r2, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 2), "plan c2r x2")))
    return fail(st, p->last_error);
  if ((st = check_cuda(p, cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking), "stream")) ||
      (st = check_cuda(p, cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming), "event")) ||
      (st = check_cuda(p, cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming), "event")))
    return fail(st, p->last_error);
  *out = p;
  return PME_OK;
}

int pme_plan_set_box(pme_plan_t p, const double box[9]) {
  if (!p || !box) return PME_ERR_ARG;
  const int old_cells = p->ncells;
  Geometry saved = p->g;
  double saved_box[9];
  std::memcpy(saved_box, p->box, sizeof(saved_box));
  std::string why;
  if (!set_geometry(p, box, why)) {
    p->g = saved;
    std::memcpy(p->box, saved_box, sizeof(saved_box));
    p->ncells = old_cells;
    return set_error(p, PME_ERR_ARG, why);
  }
  if (p->ncells > old_cells) {
    int st = check_cuda(p, cudaDeviceSynchronize(), "synchronize");
    if (st) return st;
    cudaFree(p->sb.count_c);
    cudaFree(p->sb.start_c);
    p->sb.count_c = p->sb.start_c = nullptr;
    if ((st = alloc_cells(p))) return st;
  }
  if (p->opts.recip_method == 1) {
    int st = check_cuda(p, cudaDeviceSynchronize(), "synchronize");
    if (st) return st;
    return setup_kvectors(p);
  }
  return PME_OK;
}

int pme_plan_destroy(pme_plan_t p) {
  if (!p) return PME_ERR_ARG;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  free_plan(p);
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
  if (flags & kFlagNonFinite) return set_error(p, PME_ERR_NONFINITE, "non-finite value in pos, q or mu");
  if (flags & kFlagTimeout) return set_error(p, PME_ERR_TIMEOUT, "device wait timed out");
  return PME_OK;
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
  double* e_out = sg.out_d(energy, 0);
  float* f_out = sg.out(force, 3, kOF);
  float* p_out = sg.out(phi, 1, kOPhi);
  float* fl_out = sg.out(field, 3, kOField);
  float* fg_out = sg.out(field_grad, 6, kOFG);
  if (sg.status) return sg.status;
  const bool pair = p->opts.include_pair != 0;
  int t;
  if (p->opts.recip_method == 1) return forward_ewald(p, s, in, pair, e_out, f_out, p_out, fl_out, fg_out, sg);
  t = prof_begin(p, 0, s);
  if ((st = launch_sort(p, s, in, false, true, pair))) return st;
  prof_end(p, t, s);
  // the pair term runs on the plan's side stream, concurrently with the mesh stages
  const bool fork = pair && n > 0;
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (fork) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, 6, ps);
    if ((st = launch_pair(p, ps, n, false, in, nullptr, p->pair_out))) return st;
    prof_end(p, t, ps);
  }
  t = prof_begin(p, 1, s);
  if ((st = launch_spread(p, s, n, false, p->rho, nullptr))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 2, s);
  if ((st = check_fft(p, cufftSetStream(p->r2c1, s), "set stream"))) return st;
  if ((st = check_fft(p, cufftExecR2C(p->r2c1, p->rho, p->spec), "exec r2c"))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 3, s);
  if ((st = launch_influence(p, s, p->spec, 1, p->epart))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 4, s);
  if ((st = check_fft(p, cufftSetStream(p->c2r1, s), "set stream"))) return st;
  if ((st = check_fft(p, cufftExecC2R(p->c2r1, p->spec, p->phi), "exec c2r"))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, 5, s);
  if ((st = launch_gather(p, s, n, p->phi, nullptr, false, in, nullptr, p->mesh_out))) return st;
  prof_end(p, t, s);
  if (fork && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, 7, s);
  if ((st = launch_combine_forward(p, s, in, true, pair && n > 0, p->epart + p->nspec_blocks,
                                   f_out, p_out, fl_out, fg_out)))
    return st;
  prof_end(p, t, s);
  if (e_out) {
    const double bgfac =
        p->opts.include_background ? -kPi / (2.0 * p->g.volume * p->alpha * p->alpha) : 0.0;
    t = prof_begin(p, 8, s);
    if ((st = launch_energy_final(p, s, p->epart, p->nspec_blocks, combine_blocks(n),
                                  0.5 / p->g.volume, p->opts.coulomb_k, bgfac, p->sb.qsum, e_out)))
      return st;
    prof_end(p, t, s);
  }
  return sg.finish();
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
  const double* gE = sg.in_d(g_energy, 1);
  float* o_pos = sg.out(grad_pos, 3, kOGPos);
  float* o_q = sg.out(grad_q, 1, kOGQ);
  float* o_mu = sg.out(grad_mu, 3, kOGMu);
  if (sg.status) return sg.status;
  if (n == 0) return sg.finish();
  const bool pair = p->opts.include_pair != 0;
  constexpr int B = PME_STAGES_PER_PASS;
  int t;
  t = prof_begin(p, B + 0, s);
  if ((st = launch_sort(p, s, in, true, true, pair))) return st;
  prof_end(p, t, s);
  cudaStream_t ps = p->opts.overlap_pair ? p->side : s;
  if (pair) {
    if (p->opts.overlap_pair && (st = fork_side(p, s))) return st;
    t = prof_begin(p, B + 6, ps);
    if ((st = launch_pair(p, ps, n, true, in, gE, p->pair_out))) return st;
    prof_end(p, t, ps);
  }
  t = prof_begin(p, B + 1, s);
  if ((st = launch_spread(p, s, n, true, p->rho, p->rho + p->M))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 2, s);
  if ((st = check_fft(p, cufftSetStream(p->r2c2, s), "set stream"))) return st;
  if ((st = check_fft(p, cufftExecR2C(p->r2c2, p->rho, p->spec), "exec r2c x2"))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 3, s);
  if ((st = launch_influence(p, s, p->spec, 2, p->epart))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 4, s);
  if ((st = check_fft(p, cufftSetStream(p->c2r2, s), "set stream"))) return st;
  if ((st = check_fft(p, cufftExecC2R(p->c2r2, p->spec, p->phi), "exec c2r x2"))) return st;
  prof_end(p, t, s);
  t = prof_begin(p, B + 5, s);
  if ((st = launch_gather(p, s, n, p->phi, p->phi + p->M, true, in, gE, p->mesh_out))) return st;
  prof_end(p, t, s);
  if (pair && p->opts.overlap_pair && (st = join_side(p, s))) return st;
  t = prof_begin(p, B + 7, s);
  if ((st = launch_combine_backward(p, s, in, gE, o_pos, o_q, o_mu))) return st;
  prof_end(p, t, s);
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
  if ((st = launch_sort(p, s, in, false, true, false))) return st;
  return launch_spread(p, s, n, false, rho, nullptr);
}

int pme_solve(pme_plan_t p, void* stream, const float* rho, float* phi_mesh, double* e_recip) {
  if (!p) return PME_ERR_ARG;
  int st = check_common(p, 0, nullptr, nullptr);
  if (st) return st;
  if (!rho || !phi_mesh || !is_device_pointer(rho) || !is_device_pointer(phi_mesh) ||
      !is_device_pointer(e_recip))
    return set_error(p, PME_ERR_ARG, "pme_solve takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = check_cuda(p, cudaMemcpyAsync(p->rho, rho, sizeof(float) * p->M, cudaMemcpyDeviceToDevice, s), "copy rho")))
    return st;
  if ((st = check_fft(p, cufftSetStream(p->r2c1, s), "set stream"))) return st;
  if ((st = check_fft(p, cufftExecR2C(p->r2c1, p->rho, p->spec), "exec r2c"))) return st;
  if ((st = launch_influence(p, s, p->spec, 1, p->epart))) return st;
  if ((st = check_fft(p, cufftSetStream(p->c2r1, s), "set stream"))) return st;
  if ((st = check_fft(p, cufftExecC2R(p->c2r1, p->spec, phi_mesh), "exec c2r"))) return st;
  if (e_recip)
    return launch_energy_final(p, s, p->epart, p->nspec_blocks, 0, 0.5 / p->g.volume, 1.0, 0.0,
                               nullptr, e_recip);
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
  if ((st = launch_sort(p, s, in, false, true, false))) return st;
  return launch_gather(p, s, n, phi_mesh, nullptr, false, in, nullptr, out);
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
  if ((st = launch_sort(p, s, in, false, false, true))) return st;
  if ((st = launch_pair(p, s, n, false, in, nullptr, out))) return st;
  if (e_pair) {
    if ((st = launch_pair_energy(p, s, n, in, out, p->epart))) return st;
    return launch_energy_final(p, s, p->epart, 0, combine_blocks(n), 1.0, 1.0, 0.0, nullptr, e_pair);
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
