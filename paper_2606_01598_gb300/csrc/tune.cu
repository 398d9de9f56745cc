// Brick autotuner: pme_autotune_brick and the automatic brick choice of pme_plan_create.
//
// The spread kernels are built for a few brick shapes (kSpreadShapes). Which one is fastest
// depends on the mesh, the spline order and the number of ions per brick, so the tuner times
// them: for each shape it builds a temporary plan (pair term off: the pair kernels do not
// depend on the brick), runs the forward and the backward of the mesh part on synthetic ions
// drawn uniformly in the box (the workloads' density is uniform), two calls to warm up
// (and to record the plan's pass graphs, which every later identical call replays, as a
// caller's would), then five timed calls with CUDA events, and keeps the median. The shape
// with the smallest median wins; the default shape is kept unless another is more than 2 %
// faster, so timing noise does not flip the choice between runs. Choices are cached per
// (device, mesh, order, ion count rounded up to a power of two) for the process, and read from
// / appended to the file named by GBPME_TUNE_CACHE when that variable is set.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "kernels.h"

namespace gbpme {

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune_cache;
bool g_file_loaded = false;

std::string tune_key(const int mesh[3], int order, int n) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  long long nb = 64;
  while (nb < n) nb <<= 1;
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s|%dx%dx%d|p%d|n%lld", name.c_str(), mesh[0], mesh[1], mesh[2], order, nb);
  return buf;
}

void load_file_locked() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char* path = std::getenv("GBPME_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[256];
  int bx, by, bz;
  while (std::fscanf(f, "%255s %d %d %d", key, &bx, &by, &bz) == 4) g_tune_cache[key] = {bx, by, bz};
  std::fclose(f);
}

void store_locked(const std::string& key, const int b[3]) {
  g_tune_cache[key] = {b[0], b[1], b[2]};
  const char* path = std::getenv("GBPME_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d\n", key.c_str(), b[0], b[1], b[2]);
  std::fclose(f);
}

// Median milliseconds of forward + backward (mesh part) of a plan with brick `shape`, or a
// negative value when the shape does not apply.
double time_shape(const double box[9], const int mesh[3], int order, double alpha, double rcut, int n,
                  const pme_opts& base, const int shape[3], const float* pos, const float* q, const float* mu,
                  const float* gf, const float* gp, const float* gm, double* e, const double* ge, float* out3,
                  float* out1, float* out3b, cudaStream_t s) {
  pme_opts o = base;
  for (int a = 0; a < 3; ++a) o.brick[a] = shape[a];
  o.autotune = 0;
  o.include_pair = 0;
  o.max_ions = std::max(n, 1);
  pme_plan_t p = nullptr;
  if (pme_plan_create(&p, box, mesh, order, alpha, rcut, &o) != PME_OK) return -1.0;
  auto step = [&]() {
    int st = pme_forward(p, s, n, pos, q, mu, e, out3, out1, out3b, nullptr);
    if (!st) st = pme_backward(p, s, n, pos, q, mu, ge, gf, gp, gm, out3, out1, out3b);
    return st;
  };
  double ms = -1.0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
    bool ok = step() == PME_OK && step() == PME_OK;
    std::vector<double> t;
    for (int k = 0; k < 5 && ok; ++k) {
      cudaEventRecord(a, s);
      ok = step() == PME_OK;
      cudaEventRecord(b, s);
      float el = 0.f;
      ok = ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&el, a, b) == cudaSuccess;
      t.push_back(el);
    }
    if (ok && pme_sync_status(p, s) == PME_OK) {
      std::sort(t.begin(), t.end());
      ms = t[t.size() / 2];
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  pme_plan_destroy(p);
  cudaGetLastError();
  return ms;
}

}  // namespace

int autotune_brick(const double box[9], const int mesh[3], int order, double alpha, double rcut, int n,
                   const pme_opts& base, int out[3], double* ms_out, bool use_cache) {
  spread_brick_shape(out);
  if (n <= 0) n = 1;
  const std::string key = tune_key(mesh, order, n);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  load_file_locked();
  if (use_cache && !ms_out) {
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int a = 0; a < 3; ++a) out[a] = it->second[a];
      return PME_OK;
    }
  }
  // synthetic ions: uniform fractional coordinates, alternating charges +-1 (neutral), small
  // Gaussian dipoles and cotangents
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  std::normal_distribution<double> G(0.0, 0.05);
  std::vector<float> h(size_t(n) * 14);
  float* hp = h.data();
  float* hq = hp + 3 * size_t(n);
  float* hm = hq + n;
  float* hg = hm + 3 * size_t(n);   // g_force [n][3], g_phi [n], g_field [n][3]
  for (int i = 0; i < n; ++i) {
    const double s0 = U(rng), s1 = U(rng), s2 = U(rng);
    for (int c = 0; c < 3; ++c) hp[3 * i + c] = float(s0 * box[c] + s1 * box[3 + c] + s2 * box[6 + c]);
    hq[i] = (i & 1) ? -1.f : 1.f;
    for (int c = 0; c < 3; ++c) hm[3 * i + c] = float(G(rng));
    for (int c = 0; c < 7; ++c) hg[7 * i + c] = float(G(rng) * 20.0);
  }
  const size_t fb = (sizeof(float) * 21 * size_t(n) + 255) / 256 * 256;
  unsigned char* d = nullptr;
  if (cudaMalloc(&d, fb + 64) != cudaSuccess) {
    cudaGetLastError();
    return PME_ERR_NOMEM;
  }
  float* dp = reinterpret_cast<float*>(d);
  float* dq = dp + 3 * size_t(n);
  float* dm = dq + n;
  float* dgf = dm + 3 * size_t(n);
  float* dgp = dgf + 3 * size_t(n);
  float* dgm = dgp + n;
  float* o3 = dgm + 3 * size_t(n);
  float* o1 = o3 + 3 * size_t(n);
  float* o3b = o1 + n;
  double* de = reinterpret_cast<double*>(d + fb);
  double* dge = de + 1;
  // the host layout interleaves the cotangents per ion; copy them apart
  std::vector<float> gf(3 * size_t(n)), gp(n), gm(3 * size_t(n));
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < 3; ++c) gf[3 * i + c] = hg[7 * i + c];
    gp[i] = hg[7 * i + 3];
    for (int c = 0; c < 3; ++c) gm[3 * i + c] = hg[7 * i + 4 + c];
  }
  const double ge1 = 0.5;
  bool ok = cudaMemcpy(dp, hp, sizeof(float) * (7 * size_t(n)), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dgf, gf.data(), sizeof(float) * gf.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dgp, gp.data(), sizeof(float) * gp.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dgm, gm.data(), sizeof(float) * gm.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dge, &ge1, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  cudaStream_t s = nullptr;
  ok = ok && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
  double best = -1.0, def_ms = -1.0;
  int def[3];
  spread_brick_shape(def);
  for (int k = 0; k < kNumSpreadShapes && ok; ++k) {
    const double ms = time_shape(box, mesh, order, alpha, rcut, n, base, kSpreadShapes[k], dp, dq, dm, dgf, dgp, dgm,
                                 de, dge, o3, o1, o3b, s);
    if (ms_out) ms_out[k] = ms;
    if (ms < 0) continue;
    const bool is_def = kSpreadShapes[k][0] == def[0] && kSpreadShapes[k][1] == def[1] && kSpreadShapes[k][2] == def[2];
    if (is_def) def_ms = ms;
    if (best < 0 || ms < best) {
      best = ms;
      for (int a = 0; a < 3; ++a) out[a] = kSpreadShapes[k][a];
    }
  }
  if (def_ms > 0 && def_ms <= 1.02 * best) spread_brick_shape(out);
  if (s) cudaStreamDestroy(s);
  cudaFree(d);
  cudaGetLastError();
  if (!ok) return PME_ERR_CUDA;
  if (best > 0) store_locked(key, out);
  return PME_OK;
}

}  // namespace gbpme

extern "C" int pme_autotune_brick(const double box[9], const int mesh[3], int order, double alpha, double rcut,
                                  int n_ions, const pme_opts* opts, int brick_out[3], double* ms_out) {
  if (!box || !mesh || !brick_out || n_ions < 0 || order < 1 || order > gbpme::kMaxOrder) return PME_ERR_ARG;
  pme_opts o;
  if (opts) o = *opts;
  else pme_opts_default(&o);
  return gbpme::autotune_brick(box, mesh, order, alpha, rcut, n_ions, o, brick_out, ms_out, true);
}
