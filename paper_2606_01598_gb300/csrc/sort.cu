// Sorting ions into mesh bricks and pair cells.
//
// Every ion gets two keys in one pass: the brick holding its first stencil point m0
// (Section 2.3.2, Eq. w3d) and the pair cell holding its position, both offset by its
// frame's first global key, so that one counting sort orders every frame of a batch and the
// ions of a frame stay contiguous. k_bin counts (one integer atomic per ion and key, never
// per stencil point), forms each ion's records and adds up each frame's charges (and tangent
// charges) in a fixed order for the background term; k_scan turns the counts into segment
// starts;
// k_scatter places ions in arrival order, and k_rank_records re-ranks each segment by caller
// index, which makes the order -- and hence every later sum -- deterministic, while writing
// the per-ion records both orders need. (The allocation-free spread, which needs no charge
// sums, skips them.) A backward whose inputs are bit for bit those of the plan's last forward
// (checked on the device first) keeps that forward's order and records and only adds the
// charge sums and the tangent records.
#include <algorithm>

#include "kernels.h"

namespace gbpme {

namespace {

constexpr int kSortThreads = kRedItem;   // binning: one block per reduction item
constexpr int kRankMaxSegment = 2048;   // longer segments keep arrival order

// Exclusive scan of one count array by one block of 1024 threads; start[n] = total. Each
// thread owns a chunk of a multiple of 4 entries and moves it with 16-byte loads and stores,
// so both arrays are allocated padded to a multiple of 4 entries past n + 1 (entries past n
// are read but ignored, and written with scratch values before start[n] is set). The counts
// are dead once scanned: the scan leaves them zero for the next sort.
__device__ void block_exclusive_scan(int* count, int* start, int n) {
  __shared__ int warp_tot[32];
  const int T = blockDim.x;
  const int chunk = ((n + T - 1) / T + 3) & ~3;
  const int lo = min(n, threadIdx.x * chunk), hi = min(n, lo + chunk);
  // chunks of up to 16 entries stay in registers between the two passes
  constexpr int kHold = 4;
  int4 held[kHold];
  const bool hold = hi - lo <= 4 * kHold;
  int local = 0;
  if (hold) {
#pragma unroll
    for (int u = 0; u < kHold; ++u) {
      const int k = lo + 4 * u;
      held[u] = k < hi ? __ldcg(reinterpret_cast<const int4*>(count + k)) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kHold; ++u) {
      const int k = lo + 4 * u;
      if (k < hi) {
        const int4 c = held[u];
        local += c.x + (k + 1 < hi ? c.y : 0) + (k + 2 < hi ? c.z : 0) + (k + 3 < hi ? c.w : 0);
      }
    }
  } else {
#pragma unroll 4
    for (int k = lo; k < hi; k += 4) {
      const int4 c = __ldcg(reinterpret_cast<const int4*>(count + k));
      local += c.x + (k + 1 < hi ? c.y : 0) + (k + 2 < hi ? c.z : 0) + (k + 3 < hi ? c.w : 0);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int v = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < (T >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    warp_tot[lane] = w;   // inclusive prefix over warps
  }
  __syncthreads();
  int run = v - local + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll 4
  for (int k = lo; k < hi; k += 4) {
    const int4 c = hold ? held[(k - lo) >> 2] : __ldcg(reinterpret_cast<const int4*>(count + k));
    int4 o;
    o.x = run;
    o.y = o.x + c.x;
    o.z = o.y + (k + 1 < hi ? c.y : 0);
    o.w = o.z + (k + 2 < hi ? c.z : 0);
    run = o.w + (k + 3 < hi ? c.w : 0);
    *reinterpret_cast<int4*>(start + k) = o;
    *reinterpret_cast<int4*>(count + k) = make_int4(0, 0, 0, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) start[n] = warp_tot[31];
}

// One block per reduction item (kRedItem = kSortThreads ions of one frame, one per thread):
// the ion's brick key and pair-cell key with one counting atomic each, its records in caller
// order, and the item's charge sums (the last item of a frame adds the item partials in
// order).
template <bool BATCH>
__global__ void __launch_bounds__(kSortThreads)
k_bin(FrameDesc one, FrameMaps maps, IonInputs in, SortBuffers sb, int tangent, int* flags,
      int nbricks, int ncells, const int* reuse, float* save, int ld) {
  pdl_begin();
  static_assert(kRedItem == kSortThreads, "one ion per thread");
  const int item = blockIdx.x;
  const int f = BATCH ? maps.item_frame[item] : 0;
  const FrameDesc& F = frame_at<BATCH>(one, maps, f);
  int lo, hi;
  item_range(F, item, lo, hi);
  const int i = lo + int(threadIdx.x);
  // reuse: the inputs are those of the forward whose sort is still in place; only the charge
  // sums are formed
  const bool re = reuse && *reuse == 0;
  float qa = 0.f, qb = 0.f;
  if (re && i < hi) {
    const float qi = in.q ? in.q[i] : 0.f;
    qa = isfinite(qi) ? qi : 0.f;
    qb = (tangent && in.gphi) ? in.gphi[i] : 0.f;
  } else if (i < hi) {
    const Geometry& g = F.g;
    const float rx = in.pos[3 * i], ry = in.pos[3 * i + 1], rz = in.pos[3 * i + 2];
    const float qi = in.q ? in.q[i] : 0.f;
    if (save) {
      // the forward's inputs, bit for bit, for the comparison a later backward makes
      save[3 * i] = rx;
      save[3 * i + 1] = ry;
      save[3 * i + 2] = rz;
      save[3 * ld + i] = qi;
#pragma unroll
      for (int a = 0; a < 3; ++a) save[4 * ld + 3 * i + a] = in.mu ? in.mu[3 * i + a] : 0.f;
    }
    bool ok = isfinite(rx) && isfinite(ry) && isfinite(rz) && isfinite(qi);
    if (in.mu) ok = ok && isfinite(in.mu[3 * i]) && isfinite(in.mu[3 * i + 1]) && isfinite(in.mu[3 * i + 2]);
    if (in.theta) {
#pragma unroll
      for (int a = 0; a < 6; ++a) ok = ok && isfinite(in.theta[6 * i + a]);
    }
    if (!ok) atomicOr(flags, kFlagNonFinite);
    // mesh and cell coordinates in compensated float32 (GB300's float64 rate is a small
    // fraction of its float32 rate); positions beyond the float path's range, or not finite,
    // take the float64 path
    int m0[3], c[3];
    float fb[3], fc[3];
    bool fast = true;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      fast = fast && stencil_origin_f(g, rx, ry, rz, b, m0[b], fb[b]);
      fast = fast && cell_origin_f(g, rx, ry, rz, b, c[b], fc[b]);
    }
    if (!fast) {
      double s[3];
      frac_coords(g, rx, ry, rz, s);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        stencil_origin(s[b], g.N[b], g.order, m0[b], fb[b]);
        cell_origin(s[b], g.ncell[b], c[b], fc[b]);
      }
    }
    const int kb = F.brick_off + ((m0[0] / g.brick[0]) * g.nb[1] + m0[1] / g.brick[1]) * g.nb[2] +
                   m0[2] / g.brick[2];
    const int kc = F.cell_off + (c[0] * g.ncell[1] + c[1]) * g.ncell[2] + c[2];
    sb.key_b[i] = kb;
    sb.key_c[i] = kc;
    sb.slot_b[i] = atomicAdd(&sb.count_b[kb], 1);
    sb.slot_c[i] = atomicAdd(&sb.count_c[kc], 1);
    if (sb.t_bidx) {
      // the primal records of both orders, in caller order (the rank pass moves them)
      const float qs = isfinite(qi) ? qi : 0.f;
      float mu[3] = {0.f, 0.f, 0.f};
      if (in.mu) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          mu[a] = in.mu[3 * i + a];
          if (!isfinite(mu[a])) mu[a] = 0.f;
        }
      }
      float pm[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) pm[b] = mu[0] * g.D[0 * 3 + b] + mu[1] * g.D[1 * 3 + b] + mu[2] * g.D[2 * 3 + b];
      sb.t_bidx[i] = make_int4(m0[0], m0[1], m0[2], i);
      sb.t_bfq[i] = make_float4(fb[0], fb[1], fb[2], qs);
      sb.t_bdm[i] = make_float4(pm[0], pm[1], pm[2], 0.f);
      sb.t_cidx[i] = make_int4(c[0], c[1], c[2], i);
      sb.t_cfq[i] = make_float4(fc[0], fc[1], fc[2], __int_as_float(c[2]));
      sb.t_cmu[i] = make_float4(mu[0], mu[1], mu[2], qs);
    }
    qa = isfinite(qi) ? qi : 0.f;
    qb = (tangent && in.gphi) ? in.gphi[i] : 0.f;
  }
  if (sb.qcount) {
    double A, B;
    block_sum2_f(qa, qb, A, B);
    if (threadIdx.x == 0) {
      sb.qpart[2 * item] = A;
      sb.qpart[2 * item + 1] = B;
    }
    if (last_item_done(sb.qcount + f, F.nitems)) {
      double a, b;
      strided_sum2_d(sb.qpart + 2 * F.item_off, F.nitems, 2, sb.qpart + 2 * F.item_off + 1, F.nitems, 2, a, b);
      block_sum2_d(a, b);
      if (threadIdx.x == 0) {
        sb.qsum[2 * f] = a;
        sb.qsum[2 * f + 1] = b;
        sb.qcount[f] = 0;
      }
    }
  }
  (void)nbricks;
  (void)ncells;
}

// Segment starts from the final counts: block 0 scans the brick counts, block 1 the cell
// counts (1024 threads each). Skipped on reuse.
__global__ void __launch_bounds__(1024) k_scan(SortBuffers sb, int nbricks, int ncells, const int* reuse) {
  pdl_begin();
  if (reuse && *reuse == 0) return;
  if (blockIdx.x == 0) block_exclusive_scan(sb.count_b, sb.start_b, nbricks);
  else block_exclusive_scan(sb.count_c, sb.start_c, ncells);
}

__global__ void __launch_bounds__(kSortThreads)
k_scatter(int n, SortBuffers sb, int need_mesh, int need_pair, const int* reuse) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (reuse && *reuse == 0)) return;
  if (need_mesh) {
    const int d = sb.start_b[sb.key_b[i]] + sb.slot_b[i];
    if (index_ok(d, n)) sb.perm_b[d] = i;
  }
  if (need_pair) {
    const int d = sb.start_c[sb.key_c[i]] + sb.slot_c[i];
    if (index_ok(d, n)) sb.perm_c[d] = i;
  }
}

__device__ __forceinline__ int stable_rank(const int* perm, int seg_lo, int seg_hi, int self,
                                           int fallback) {
  if (seg_hi - seg_lo > kRankMaxSegment) return fallback;
  int r = 0;
#pragma unroll 8
  for (int u = seg_lo; u < seg_hi; ++u) r += (perm[u] < self) ? 1 : 0;   // eight loads in flight
  return seg_lo + r;
}

template <bool BATCH>
__global__ void __launch_bounds__(kSortThreads)
k_rank_records(FrameDesc one, FrameMaps maps, IonInputs in, SortBuffers sb, MeshRecords mr,
               PairRecords pr, int tangent, int need_mesh, int need_pair, const int* reuse) {
  pdl_begin();
  const int n = in.n;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool mesh_side = t < n;
  if (!mesh_side) t -= n;
  if (t >= n) return;
  if (mesh_side && !need_mesh) return;
  if (!mesh_side && !need_pair) return;
  // reuse: the forward's records stay; only the tangent records are written, at the sorted
  // slot the forward gave each ion
  const bool re = reuse && *reuse == 0;
  int i, dest;
  if (re) {
    dest = t;
    i = mesh_side ? mr.idx[t].w : pr.idx[t].w;
  } else if (mesh_side) {
    i = sb.perm_b[t];
    const int k = sb.key_b[i];
    dest = stable_rank(sb.perm_b, sb.start_b[k], sb.start_b[k + 1], i, t);
  } else {
    i = sb.perm_c[t];
    const int k = sb.key_c[i];
    dest = stable_rank(sb.perm_c, sb.start_c[k], sb.start_c[k + 1], i, t);
  }
  if (!index_ok(i, n) || !index_ok(dest, n)) return;
  const int f = BATCH ? maps.ion_frame[i] : 0;
  const FrameDesc& F = frame_at<BATCH>(one, maps, f);
  const Geometry& g = F.g;
  const float rx = in.pos[3 * i], ry = in.pos[3 * i + 1], rz = in.pos[3 * i + 2];
  float qi = in.q ? in.q[i] : 0.f;
  float mu[3] = {0.f, 0.f, 0.f};
  if (in.mu) {
    mu[0] = in.mu[3 * i];
    mu[1] = in.mu[3 * i + 1];
    mu[2] = in.mu[3 * i + 2];
  }
  if (!isfinite(qi)) qi = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (!isfinite(mu[a])) mu[a] = 0.f;
  float dq = 0.f, dr[3] = {0.f, 0.f, 0.f}, dmu[3] = {0.f, 0.f, 0.f};
  if (tangent) {
    if (in.gphi) dq = in.gphi[i];
    if (in.gforce) {
      dr[0] = -in.gforce[3 * i];
      dr[1] = -in.gforce[3 * i + 1];
      dr[2] = -in.gforce[3 * i + 2];
    }
    if (in.gfield) {
      dmu[0] = -in.gfield[3 * i];
      dmu[1] = -in.gfield[3 * i + 1];
      dmu[2] = -in.gfield[3 * i + 2];
    }
  }
  // tangent dipole source d' = dmu + q dr
  const float dp[3] = {dmu[0] + qi * dr[0], dmu[1] + qi * dr[1], dmu[2] + qi * dr[2]};
  if (re) {
    if (mesh_side) {
      float pd[3], pt[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        pd[b] = dp[0] * g.D[0 * 3 + b] + dp[1] * g.D[1 * 3 + b] + dp[2] * g.D[2 * 3 + b];
        pt[b] = dr[0] * g.D[0 * 3 + b] + dr[1] * g.D[1 * 3 + b] + dr[2] * g.D[2 * 3 + b];
      }
      mr.tq[dest] = make_float4(dq, pd[0], pd[1], pd[2]);
      mr.tt[dest] = make_float4(pt[0], pt[1], pt[2], 0.f);
    } else {
      pr.tq[dest] = make_float4(dq, dp[0], dp[1], dp[2]);
      pr.dr[dest] = make_float4(dr[0], dr[1], dr[2], 0.f);
    }
    return;
  }
  if (sb.t_bidx) {
    // primal records from the binning pass; tangent records formed here
    if (mesh_side) {
      mr.idx[dest] = sb.t_bidx[i];
      mr.fq[dest] = sb.t_bfq[i];
      mr.dm[dest] = sb.t_bdm[i];
      if (tangent) {
        float pd[3], pt[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          pd[b] = dp[0] * g.D[0 * 3 + b] + dp[1] * g.D[1 * 3 + b] + dp[2] * g.D[2 * 3 + b];
          pt[b] = dr[0] * g.D[0 * 3 + b] + dr[1] * g.D[1 * 3 + b] + dr[2] * g.D[2 * 3 + b];
        }
        mr.tq[dest] = make_float4(dq, pd[0], pd[1], pd[2]);
        mr.tt[dest] = make_float4(pt[0], pt[1], pt[2], 0.f);
      }
    } else {
      pr.idx[dest] = sb.t_cidx[i];
      pr.fq[dest] = sb.t_cfq[i];
      pr.mu[dest] = sb.t_cmu[i];
      if (tangent) {
        pr.tq[dest] = make_float4(dq, dp[0], dp[1], dp[2]);
        pr.dr[dest] = make_float4(dr[0], dr[1], dr[2], 0.f);
      }
    }
    return;
  }
  // the binning pass's coordinates: compensated float32, float64 where that does not apply
  double s[3];
  bool fast = true;
  int m0[3], cc[3];
  float fm[3], fcl[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (mesh_side) fast = fast && stencil_origin_f(g, rx, ry, rz, b, m0[b], fm[b]);
    else fast = fast && cell_origin_f(g, rx, ry, rz, b, cc[b], fcl[b]);
  }
  if (!fast) frac_coords(g, rx, ry, rz, s);
  if (mesh_side) {
    float fr[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (fast) fr[b] = fm[b];
      else stencil_origin(s[b], g.N[b], g.order, m0[b], fr[b]);
    }
    float pm[3], pd[3], pt[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      pm[b] = mu[0] * g.D[0 * 3 + b] + mu[1] * g.D[1 * 3 + b] + mu[2] * g.D[2 * 3 + b];
      pd[b] = dp[0] * g.D[0 * 3 + b] + dp[1] * g.D[1 * 3 + b] + dp[2] * g.D[2 * 3 + b];
      pt[b] = dr[0] * g.D[0 * 3 + b] + dr[1] * g.D[1 * 3 + b] + dr[2] * g.D[2 * 3 + b];
    }
    mr.idx[dest] = make_int4(m0[0], m0[1], m0[2], i);
    mr.fq[dest] = make_float4(fr[0], fr[1], fr[2], qi);
    mr.dm[dest] = make_float4(pm[0], pm[1], pm[2], 0.f);
    if (tangent) {
      mr.tq[dest] = make_float4(dq, pd[0], pd[1], pd[2]);
      mr.tt[dest] = make_float4(pt[0], pt[1], pt[2], 0.f);
    }
  } else {
    int c[3];
    float fr[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (fast) {
        c[b] = cc[b];
        fr[b] = fcl[b];
      } else {
        cell_origin(s[b], g.ncell[b], c[b], fr[b]);
      }
    }
    pr.idx[dest] = make_int4(c[0], c[1], c[2], i);
    pr.fq[dest] = make_float4(fr[0], fr[1], fr[2], __int_as_float(c[2]));
    pr.mu[dest] = make_float4(mu[0], mu[1], mu[2], qi);
    if (tangent) {
      pr.tq[dest] = make_float4(dq, dp[0], dp[1], dp[2]);
      pr.dr[dest] = make_float4(dr[0], dr[1], dr[2], 0.f);
    }
  }
}

// Bitwise comparison of the backward's inputs with the saved forward inputs.
__global__ void __launch_bounds__(256)
k_input_check(int n, IonInputs in, const float* saved, int ld, const int* list_cnt, int* in_diff,
              int* cache_bad) {
  pdl_begin();
  bool same = true, lists = true;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = t0; k < 3 * n; k += stride) {
    same = same && __float_as_int(in.pos[k]) == __float_as_int(saved[k]);
    const float m = in.mu ? in.mu[k] : 0.f;
    same = same && __float_as_int(m) == __float_as_int(saved[4 * ld + k]);
  }
  for (int k = t0; k < n; k += stride) {
    const float q = in.q ? in.q[k] : 0.f;
    same = same && __float_as_int(q) == __float_as_int(saved[3 * ld + k]);
    if (list_cnt) lists = lists && list_cnt[k] >= 0;
  }
  const bool diff = __any_sync(0xffffffffu, !same);
  const bool bad = __any_sync(0xffffffffu, !lists);
  if ((threadIdx.x & 31) == 0) {
    if (diff) *in_diff = 1;
    if (diff || bad) *cache_bad = 1;
  }
}

template <bool BATCH>
int launch_sort_t(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool tangent, bool need_mesh,
                  bool need_pair, const int* reuse, float* save) {
  const int n = in.n;
  const int nblk = (n + kSortThreads - 1) / kSortThreads;
  FrameDesc one = p->frames_h[0];
  if (!BATCH) {
    one.n = n;
    one.item_off = 0;
    one.nitems = std::max(1, (n + kRedItem - 1) / kRedItem);
  }
  int st = PME_OK;
  if (!p->counts_clean) {
    st = check_cuda(p, cudaMemsetAsync(p->sb.count_b, 0, sizeof(int) * (p->total_bricks + 1), s),
                    "memset brick counts");
    if (st) return st;
    st = check_cuda(p, cudaMemsetAsync(p->sb.count_c, 0, sizeof(int) * (p->total_cells + 1), s),
                    "memset cell counts");
    if (st) return st;
  }
  {
    const int items = BATCH ? p->total_items : one.nitems;
    pdl_launch(k_bin<BATCH>, items, kSortThreads, 0, s, one, p->maps, in, p->sb, tangent ? 1 : 0, p->flags,
                                                p->total_bricks, p->total_cells, reuse, save,
                                                p->max_ions);
    count_launch();
    if ((st = check_launch(p, "k_bin"))) {
      p->counts_clean = false;
      return st;
    }
    pdl_launch(k_scan, 2, 1024, 0, s, p->sb, p->total_bricks, p->total_cells, reuse);
    count_launch();
    if ((st = check_launch(p, "k_scan"))) {
      p->counts_clean = false;
      return st;
    }
  }
  if (nblk > 0) {
    pdl_launch(k_scatter, nblk, kSortThreads, 0, s, n, p->sb, need_mesh ? 1 : 0, need_pair ? 1 : 0, reuse);
    count_launch();
    if ((st = check_launch(p, "k_scatter"))) return st;
    const int nblk2 = (2 * n + kSortThreads - 1) / kSortThreads;
    pdl_launch(k_rank_records<BATCH>, nblk2, kSortThreads, 0, s, one, p->maps, in, p->sb, p->mr, p->pr,
                                                         tangent ? 1 : 0, need_mesh ? 1 : 0,
                                                         need_pair ? 1 : 0, reuse);
    count_launch();
    if ((st = check_launch(p, "k_rank_records"))) return st;
  }
  return PME_OK;
}

}  // namespace

int launch_input_check(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool with_lists) {
  int st = check_cuda(p, cudaMemsetAsync(p->in_flags, 0, 2 * sizeof(int), s), "memset");
  if (st || in.n == 0) return st;
  const int grid = std::min(4 * device_sm_count(), (3 * in.n + 255) / 256);
  pdl_launch(k_input_check, grid, 256, 0, s, in.n, in, p->in_saved, p->max_ions, with_lists ? p->plist_cnt : nullptr,
                                      p->in_diff, p->cache_bad);
  count_launch();
  return check_launch(p, "k_input_check");
}

int launch_sort(pme_plan_t p, cudaStream_t s, const IonInputs& in, bool tangent, bool need_mesh,
                bool need_pair, const int* reuse, float* save) {
  if (!reuse) p->fwd_n = -1;   // the sorted records no longer belong to the saved inputs
  return p->batch ? launch_sort_t<true>(p, s, in, tangent, need_mesh, need_pair, reuse, save)
                  : launch_sort_t<false>(p, s, in, tangent, need_mesh, need_pair, reuse, save);
}

GBPME_BOUNDS_READER(bounds_hit_sort)

}  // namespace gbpme
