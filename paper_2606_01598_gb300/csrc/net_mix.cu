// Channel mixing of the learned charge/dipole network on the fifth-generation tensor cores:
// Y[M][NOUT] (+)= X[M][K] W, with X float32 activations and W a bfloat16 weight matrix.
//
// The network's linear layers (the "self-interaction" products of a Cartesian-tensor message-
// passing layer and the readout's hidden layer, Sections 2.1-2.2) mix channels at every ion:
// M = ions (x 3 Cartesian components for vector features, x 2 when a tangent is carried), K
// and NOUT are 16..64. These are the only dense contractions of the learned model.
//
// Design (sm_103a, tcgen05):
//   * one CTA of 128 threads per 128-row tile; the tile of X is read with coalesced float4
//     loads and split into two bfloat16 parts, X = X_hi + X_lo (X_hi = bf16(X),
//     X_lo = bf16(X - X_hi)), so the products keep about 16 significant bits of the float32
//     activations while the tensor cores only ever see bfloat16 operands (the weights are
//     stored in bfloat16) and accumulate in float32;
//   * both operands are staged in shared memory in the canonical K-major layout without
//     swizzle (8-row x 16-byte core matrices; core matrices adjacent along K are 128 bytes
//     apart, 8-row groups K/8 x 128 bytes apart), described by tcgen05 shared-memory
//     descriptors;
//   * one elected thread issues 2 x K/16 tcgen05.mma.kind::f16 instructions (M = 128,
//     N = NOUT, K = 16 each: first the X_hi products, then the X_lo products accumulated on
//     top) into a float32 accumulator in tensor memory (TMEM), and commits them to an
//     mbarrier;
//   * every warp waits on the mbarrier (bounded: after kSpinLimit polls it records
//     kNetFlagTimeout in the error word and skips the read-back), then reads its 32 rows of
//     the accumulator with tcgen05.ld (row = TMEM lane) and writes (or adds) them to Y;
//   * the TMEM columns are freed by the warp that allocated them before the CTA exits.
#include <cstdint>

#include "net.cuh"

namespace gbnet {

namespace {

constexpr int kTile = 128;
constexpr long kSpinLimit = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// bfloat16 bits of x, round to nearest even (finite inputs).
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float bf16_value(uint32_t b) { return __uint_as_float(b << 16); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte offset
// (between core matrices adjacent along K), stride-dimension byte offset (between 8-row
// groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: float32 accumulator, bfloat16 A and B, both K-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kTile >> 4) << 24);
}

// byte offset of element (row, k) of a K-major no-swizzle tile with K columns
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int K) {
  return uint32_t((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int N>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[N], int c0) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr + uint32_t(c0)));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[c0 + j] = __uint_as_float(r[j]);
}

template <int K, int NOUT>
__global__ void __launch_bounds__(kTile) k_mix(const float* __restrict__ X, const uint16_t* __restrict__ Wt,
                                              float* __restrict__ Y, int M, int accumulate, int* err) {
  static_assert(K % 16 == 0 && K >= 16 && K <= 64, "K: 16..64, multiple of 16");
  static_assert(NOUT % 16 == 0 && NOUT >= 16 && NOUT <= 64, "NOUT: 16..64, multiple of 16");
  constexpr int kCols = NOUT <= 32 ? 32 : 64;            // TMEM columns (power of two >= 32)
  constexpr uint32_t kBytesA = kTile * K * 2;
  constexpr uint32_t kBytesB = NOUT * K * 2;
  __shared__ __align__(1024) unsigned char sA_hi[kBytesA];
  __shared__ __align__(1024) unsigned char sA_lo[kBytesA];
  __shared__ __align__(1024) unsigned char sB[kBytesB];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long row0 = long(blockIdx.x) * kTile;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }

  // X tile -> (X_hi, X_lo) bfloat16 in the K-major layout; the tile is contiguous in memory
  constexpr int kVec = kTile * K / 4;
  const float4* X4 = reinterpret_cast<const float4*>(X + row0 * K);
  const long rows_left = long(M) - row0;
  for (int e = tid; e < kVec; e += kTile) {
    const int row = (e * 4) / K, k = (e * 4) % K;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row < rows_left) x = __ldg(X4 + e);
    const uint32_t h0 = bf16_bits(x.x), h1 = bf16_bits(x.y), h2 = bf16_bits(x.z), h3 = bf16_bits(x.w);
    const uint32_t l0 = bf16_bits(x.x - bf16_value(h0)), l1 = bf16_bits(x.y - bf16_value(h1));
    const uint32_t l2 = bf16_bits(x.z - bf16_value(h2)), l3 = bf16_bits(x.w - bf16_value(h3));
    const uint32_t off = kmajor_off(row, k, K);
    *reinterpret_cast<uint2*>(sA_hi + off) = make_uint2(h0 | (h1 << 16), h2 | (h3 << 16));
    *reinterpret_cast<uint2*>(sA_lo + off) = make_uint2(l0 | (l1 << 16), l2 | (l3 << 16));
  }
  // W^T [NOUT][K] bfloat16 -> K-major layout
  const uint2* W2 = reinterpret_cast<const uint2*>(Wt);
  for (int e = tid; e < NOUT * K / 4; e += kTile) {
    const int n = (e * 4) / K, k = (e * 4) % K;
    *reinterpret_cast<uint2*>(sB + kmajor_off(n, k, K)) = __ldg(W2 + e);
  }
  // make the generic-proxy shared-memory writes visible to the tensor cores (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    constexpr uint32_t idesc = instr_desc(NOUT);
    constexpr uint32_t sbo = (K / 8) * 128;
    const uint32_t a_hi = smem_u32(sA_hi), a_lo = smem_u32(sA_lo), b = smem_u32(sB);
#pragma unroll
    for (int part = 0; part < 2; ++part) {
#pragma unroll
      for (int s = 0; s < K / 16; ++s) {
        const uint64_t ad = smem_desc((part ? a_lo : a_hi) + s * 256, 128, sbo);
        const uint64_t bd = smem_desc(b + s * 256, 128, sbo);
        const uint32_t acc = (part | s) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&mbar)) : "memory");
  }

  // bounded wait for the products (phase 0 of the mbarrier)
  uint32_t done = 0;
  for (long it = 0; it < kSpinLimit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(smem_u32(&mbar)), "r"(0u) : "memory");
  }
  done = __all_sync(0xffffffffu, done);   // tcgen05.ld below is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done) {
    if (lane == 0) atomicOr(err, kNetFlagTimeout);
  } else {
    float v[NOUT];
    const uint32_t taddr = tmem + (uint32_t(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < NOUT; c += 16) tmem_ld16<NOUT>(taddr, v, c);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const long row = row0 + warp * 32 + lane;
    if (row < M) {
      float4* y = reinterpret_cast<float4*>(Y + row * NOUT);
#pragma unroll
      for (int c = 0; c < NOUT / 4; ++c) {
        float4 o = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        if (accumulate) {
          const float4 p = y[c];
          o.x += p.x; o.y += p.y; o.z += p.z; o.w += p.w;
        }
        y[c] = o;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kCols));
  }
}

template <int K, int NOUT>
int launch_mix_kn(cudaStream_t s, int M, const float* X, const uint16_t* Wt, float* Y, bool acc, int* err) {
  if (M <= 0) return 0;
  const int blocks = (M + kTile - 1) / kTile;
  k_mix<K, NOUT><<<blocks, kTile, 0, s>>>(X, Wt, Y, M, acc ? 1 : 0, err);
  gbpme::count_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : PME_ERR_CUDA;
}

}  // namespace

int launch_mix(cudaStream_t s, int M, int K, int NOUT, const float* X, const uint16_t* Wt, float* Y,
               bool accumulate, int* err) {
#define GBNET_MIX_CASE(k, n) \
  if (K == k && NOUT == n) return launch_mix_kn<k, n>(s, M, X, Wt, Y, accumulate, err);
  GBNET_MIX_CASE(32, 48)   // A = h^s WA
  GBNET_MIX_CASE(16, 32)   // B = h^v WB; input gradient of WY
  GBNET_MIX_CASE(48, 48)   // U = m^s WU and its input gradient
  GBNET_MIX_CASE(32, 16)   // Y = m^v WY; input gradient of WB
  GBNET_MIX_CASE(32, 64)   // H = h^s Wh
  GBNET_MIX_CASE(48, 32)   // input gradient of WA
  GBNET_MIX_CASE(64, 32)   // input gradient of Wh
#undef GBNET_MIX_CASE
  return PME_ERR_UNSUPPORTED;
}

}  // namespace gbnet
