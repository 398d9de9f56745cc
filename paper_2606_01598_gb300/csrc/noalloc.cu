// Allocation-free spread: pme_spread_noalloc (declared in include/gbpme.h).
//
// Some callers cannot allocate device memory when they need the mesh density: a host
// framework that has already reserved the whole device for its own memory pool (so cudaMalloc
// would fail), or an integration loop that must not call cudaMalloc / cudaFree because they
// can synchronise the device. For them this entry point runs the same sort and spread kernels
// as pme_spread, with every piece of scratch (sort keys, counters, permutation, per-ion
// records, candidate-brick table) carved out of one static device array of fixed size,
// instead of plan-owned buffers. It creates no plan and allocates nothing.
//
// The array lives in this translation unit. Host code cannot use its name as a device
// address, so the first call on each device asks the runtime for the address with
// cudaGetSymbolAddress (with that device current) and caches it; later calls reuse it.
// Everything a call writes into the array is formed on the device, on the call's stream (the
// candidate-brick table by a small kernel, the counters by the sort's own clearing), so no
// call copies from host memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kNaMaxIons = PME_NOALLOC_MAX_IONS;
constexpr int kNaMaxMesh = PME_NOALLOC_MAX_MESH;
constexpr int kNaMaxBlocks = (kNaMaxIons + 255) / 256;
constexpr int kNaMaxNb = (kNaMaxMesh + 7) / 8;          // bricks per axis (smallest brick edge 8)
constexpr int kNaMaxBricks = kNaMaxNb * kNaMaxNb * kNaMaxNb;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// scratch layout (byte offsets, each 256-byte aligned)
constexpr size_t kOffKeyB = 0;
constexpr size_t kOffKeyC = kOffKeyB + up(4ull * kNaMaxIons);
constexpr size_t kOffSlotB = kOffKeyC + up(4ull * kNaMaxIons);
constexpr size_t kOffSlotC = kOffSlotB + up(4ull * kNaMaxIons);
constexpr size_t kOffPermB = kOffSlotC + up(4ull * kNaMaxIons);
constexpr size_t kOffPermC = kOffPermB + up(4ull * kNaMaxIons);
constexpr size_t kOffCountB = kOffPermC + up(4ull * kNaMaxIons);
constexpr size_t kOffStartB = kOffCountB + up(4ull * (kNaMaxBricks + 1));
constexpr size_t kOffCountC = kOffStartB + up(4ull * (kNaMaxBricks + 1));
constexpr size_t kOffStartC = kOffCountC + up(4ull * 2);
constexpr size_t kOffQpart = kOffStartC + up(4ull * 2);
constexpr size_t kOffQsum = kOffQpart + up(8ull * 2 * kNaMaxBlocks);
constexpr size_t kOffIdx = kOffQsum + up(8ull * 2);
constexpr size_t kOffFq = kOffIdx + up(16ull * kNaMaxIons);
constexpr size_t kOffDm = kOffFq + up(16ull * kNaMaxIons);
constexpr size_t kOffCand = kOffDm + up(16ull * kNaMaxIons);
constexpr size_t kOffFlags = kOffCand + up(4ull * 3 * kNaMaxNb * (1 + kMaxCandPerDim));
constexpr size_t kScratchBytes = kOffFlags + up(4);
static_assert(kScratchBytes == PME_NOALLOC_SCRATCH_BYTES,
              "PME_NOALLOC_SCRATCH_BYTES in include/gbpme.h must match the layout");

// The scratch array: every device that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return cudaSuccess;
}

bool na_invert(const double* a, double* inv, double* det_out) {
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
  *det_out = det;
  return true;
}

// Source bricks along one axis whose ions' stencils reach brick b (the plan's rule): every
// brick when the brick and its stencil reach cover the axis, else the bricks holding the
// stencil origins m0 in [b0 - P + 1, b0 + ext - 1], wrapped. Returns the count, or -1 when
// more than kMaxCandPerDim bricks would be needed. Host and device share this one routine.
__host__ __device__ inline int na_candidate_row(int N, int B, int P, int nb, int b, int* list) {
  const int b0 = b * B, ext = (N - b0 < B) ? N - b0 : B;
  int cnt = 0;
  if (ext + P - 1 >= N) {
    if (nb > kMaxCandPerDim) return -1;
    for (int k = 0; k < nb; ++k) list[cnt++] = k;
    return cnt;
  }
  for (int m = b0 - P + 1; m <= b0 + ext - 1; ++m) {
    const int bi = (((m % N) + N) % N) / B;
    bool seen = false;
    for (int k = 0; k < cnt; ++k) seen = seen || list[k] == bi;
    if (!seen) {
      if (cnt == kMaxCandPerDim) return -1;
      list[cnt++] = bi;
    }
  }
  return cnt;
}

struct NaAxes {
  int N[3], B[3], nb[3];
};

// One thread per (axis, brick row) of the table [3][max_nb][1 + kMaxCandPerDim]; rows past an
// axis's brick count are zeroed. The host has checked that no row overflows.
__global__ void k_na_candidates(NaAxes ax, int P, int max_nb, int* tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * max_nb) return;
  const int a = t / max_nb, b = t - a * max_nb;
  int* row = tab + t * (1 + kMaxCandPerDim);
  int list[kMaxCandPerDim];
  int cnt = 0;
  if (b < ax.nb[a]) cnt = na_candidate_row(ax.N[a], ax.B[a], P, ax.nb[a], b, list);
  if (cnt < 0) cnt = 0;
  row[0] = cnt;
  for (int k = 0; k < kMaxCandPerDim; ++k) row[1 + k] = k < cnt ? list[k] : 0;
}

// *out = PME_ERR_NONFINITE when the sort flagged a NaN or Inf input, PME_OK otherwise.
__global__ void k_na_status(const int* flags, int* out) {
  if (threadIdx.x == 0) *out = (*flags & kFlagNonFinite) ? PME_ERR_NONFINITE : PME_OK;
}

}  // namespace

}  // namespace gbpme

using namespace gbpme;

extern "C" int pme_spread_noalloc(void* stream, const double box[9], const int mesh[3], int order,
                                  int n, const float* pos, const float* q, const float* mu,
                                  float* rho, int* status) {
  if (!box || !mesh || !rho || order < 1 || order > kMaxOrder) return PME_ERR_ARG;
  if (n < 0 || n > kNaMaxIons) return PME_ERR_ARG;     // beyond the fixed scratch
  if (n > 0 && (!pos || !q)) return PME_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (mesh[a] < order || mesh[a] > kNaMaxMesh) return PME_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PME_ERR_CUDA;
  unsigned char* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return PME_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // a plan-shaped view of the scratch (host structs only; no device memory is allocated)
  pme_plan_s v{};
  FrameDesc fd{};
  Geometry& g = fd.g;
  double inv[9], det;
  if (!na_invert(box, inv, &det)) return PME_ERR_ARG;
  for (int k = 0; k < 9; ++k) g.cinv[k] = inv[k];
  g.volume = std::fabs(det);
  for (int a = 0; a < 3; ++a) g.N[a] = mesh[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g.D[a * 3 + b] = float(double(mesh[b]) * inv[a * 3 + b]);
  for (int k = 0; k < 9; ++k) g.H[k] = float(box[k]);
  for (int a = 0; a < 3; ++a) {
    g.ncell[a] = 1;
    g.kimg[a] = 0;
  }
  geometry_split(g);
  g.order = order;
  g.alpha = 1.f;
  g.rcut2 = 0.f;
  spread_brick_shape(g.brick);
  for (int a = 0; a < 3; ++a) g.nb[a] = (mesh[a] + g.brick[a] - 1) / g.brick[a];
  fd.n = n;
  fd.nbricks = g.nb[0] * g.nb[1] * g.nb[2];
  fd.ncells = 1;
  fd.max_nb = std::max(g.nb[0], std::max(g.nb[1], g.nb[2]));
  if (fd.max_nb > kNaMaxNb) return PME_ERR_ARG;
  v.g = g;
  v.frames_h = &fd;
  v.nframes = 1;
  v.batch = false;
  v.total_bricks = fd.nbricks;
  v.total_cells = 1;
  v.max_ions = kNaMaxIons;
  v.nogroups = 1;
  v.ogroups[0] = OrderGroup{order, 0, fd.nbricks, 0, n};
  NaAxes ax{};
  for (int a = 0; a < 3; ++a) {
    ax.N[a] = mesh[a];
    ax.B[a] = g.brick[a];
    ax.nb[a] = g.nb[a];
    int list[kMaxCandPerDim];
    for (int b = 0; b < g.nb[a]; ++b)   // host check only; the table is formed on the device
      if (na_candidate_row(mesh[a], g.brick[a], order, g.nb[a], b, list) < 0) return PME_ERR_UNSUPPORTED;
  }
  v.sb.key_b = reinterpret_cast<int*>(base + kOffKeyB);
  v.sb.key_c = reinterpret_cast<int*>(base + kOffKeyC);
  v.sb.slot_b = reinterpret_cast<int*>(base + kOffSlotB);
  v.sb.slot_c = reinterpret_cast<int*>(base + kOffSlotC);
  v.sb.perm_b = reinterpret_cast<int*>(base + kOffPermB);
  v.sb.perm_c = reinterpret_cast<int*>(base + kOffPermC);
  v.sb.count_b = reinterpret_cast<int*>(base + kOffCountB);
  v.sb.start_b = reinterpret_cast<int*>(base + kOffStartB);
  v.sb.count_c = reinterpret_cast<int*>(base + kOffCountC);
  v.sb.start_c = reinterpret_cast<int*>(base + kOffStartC);
  v.sb.qpart = reinterpret_cast<double*>(base + kOffQpart);
  v.sb.qcount = nullptr;   // the spread needs no charge sums: the sort skips them
  v.sb.t_bidx = nullptr;   // no room for caller-order records: the rank pass forms them
  v.sb.qsum = reinterpret_cast<double*>(base + kOffQsum);
  v.mr.idx = reinterpret_cast<int4*>(base + kOffIdx);
  v.mr.fq = reinterpret_cast<float4*>(base + kOffFq);
  v.mr.dm = reinterpret_cast<float4*>(base + kOffDm);
  v.mr.tq = nullptr;
  v.mr.tt = nullptr;
  v.cand = reinterpret_cast<int*>(base + kOffCand);
  v.flags = reinterpret_cast<int*>(base + kOffFlags);
  // the candidate table and the error flag are per call: form / clear them on the stream
  k_na_candidates<<<1, 3 * kNaMaxNb, 0, s>>>(ax, order, fd.max_nb, v.cand);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return PME_ERR_CUDA;
  if (cudaMemsetAsync(v.flags, 0, sizeof(int), s) != cudaSuccess) return PME_ERR_CUDA;
  IonInputs in{};
  in.pos = pos;
  in.q = q;
  in.mu = mu;
  in.n = n;
  // launch_sort clears the brick and cell counters on the stream before counting
  int st = launch_sort(&v, s, in, false, true, false, nullptr);
  if (st) return st;
  const int rc = launch_spread(&v, s, false, rho);   // the frame's rho sits at offset 0
  v.frames_h = nullptr;                               // host views only: nothing to release
  if (rc) return rc;
  if (status) {
    k_na_status<<<1, 32, 0, s>>>(v.flags, status);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return PME_ERR_CUDA;
  }
  return PME_OK;
}
