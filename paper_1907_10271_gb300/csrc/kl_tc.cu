// KL synthesis on the tensor cores: theta[s][e] = sum_n B[e][n] Xi[s][n] (Eq. inftyKL),
// one tile of 128 elements x 64 samples per MMA chain.
//
// A CTA owns 128 elements (the MMA's M) and walks sample tiles of 64 (its N):
//   warp 16 (one thread): TMA-loads the basis tile once (hi and lo, K blocks of 32
//     terms with 128-byte swizzle), then per sample tile TMA-loads Xi hi/lo and issues
//     3 x (kp / 8) tcgen05.mma kind::tf32 into one of two TMEM accumulators (64
//     columns each), committing to an mbarrier;
//   warps 0-15: wait for the accumulator; warp w reads TMEM lanes 32 (w % 4) .. +31
//     (its elements) and columns 16 (w / 4) .. +15 (its samples) with tcgen05.ld
//     32x32b, releases the buffer, and writes (cos 2t, sin 2t) or t with coalesced
//     stores (lane = element). Sixteen warps keep the sincos epilogue latency-hidden
//     at one CTA per SM.
// So the epilogue of tile k overlaps the loads and MMAs of tile k + 1. Every wait is
// bounded by %globaltimer; on expiry the kernel sets *err and leaves after freeing TMEM.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "kl_tc.h"

namespace mlmc {

namespace {

constexpr int kM = kKlTcElements;
constexpr int kN = kKlTcSamples;
constexpr int kKB = 32;                     // terms per 128-byte swizzle row
static_assert(kKlTcMaxTerms % kKB == 0 && kKlTcMaxTerms / kKB <= 4, "shared memory holds at most 4 K blocks");
constexpr int kABlockBytes = kM * 128;      // one K block of the basis tile
constexpr int kBBlockBytes = kN * 128;      // one K block of the Xi tile
constexpr int kEpiWarps = 16;                // 4 lane quadrants x 4 column slices
constexpr int kEpiCols = kN / (kEpiWarps / 4);
constexpr int kThreads = kEpiWarps * 32 + 32;
static_assert(kEpiCols == 16, "epilogue reads 16 TMEM columns per warp");
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__host__ __device__ inline uint32_t f2u(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
__host__ __device__ inline float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}

// Round to nearest even at TF32 precision (10 stored mantissa bits). Finite inputs.
__host__ __device__ inline float tf32_rn(float x) {
  uint32_t u = f2u(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return u2f(u & 0xFFFFE000u);
}

__host__ __device__ inline void split_one(double x, float& hi, float& lo) {
  hi = tf32_rn((float)x);
  lo = tf32_rn((float)(x - (double)hi));
}

__global__ void k_tf32_split(const double* __restrict__ x, int64_t rows, int n_kl, int kp, float* __restrict__ hi,
                             float* __restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * kp) return;
  const int64_t r = t / kp;
  const int k = (int)(t - r * kp);
  float h = 0.f, l = 0.f;
  if (k < n_kl) split_one(x[r * n_kl + k], h, l);
  hi[t] = h;
  lo[t] = l;
}

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand with 128-byte swizzle: rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), leading byte offset
// unused for this layout; version 1 (bits 46-47), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes (one value per lane and column).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- kernel

__global__ void __launch_bounds__(kThreads, 1)
    k_kl_tc(const __grid_constant__ CUtensorMap a_hi, const __grid_constant__ CUtensorMap a_lo,
            const __grid_constant__ CUtensorMap b_hi, const __grid_constant__ CUtensorMap b_lo, int n_el,
            int64_t nsamp, int kp, float* __restrict__ out, int trig2, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[6];   // a, b, mma[2], free[2]
  __shared__ uint32_t tmem_slot;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kb_count = (kp + kKB - 1) / kKB;
  uint8_t* sa_hi = smem;
  uint8_t* sa_lo = sa_hi + kb_count * kABlockBytes;
  uint8_t* sb_hi = sa_lo + kb_count * kABlockBytes;
  uint8_t* sb_lo = sb_hi + kb_count * kBBlockBytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e0 = blockIdx.x * kM;
  const int64_t ntiles = (nsamp + kN - 1) / kN;
  const int64_t my_tiles = ((int64_t)blockIdx.y < ntiles) ? (ntiles - blockIdx.y + gridDim.y - 1) / gridDim.y : 0;
  const uint32_t bar_a = smem_addr(&bars[0]), bar_b = smem_addr(&bars[1]);
  const uint32_t bar_mma0 = smem_addr(&bars[2]), bar_free0 = smem_addr(&bars[4]);

  if (threadIdx.x == kEpiWarps * 32) {
    mbar_init(bar_a, 1);
    mbar_init(bar_b, 1);
    mbar_init(bar_mma0, 1);
    mbar_init(bar_mma0 + 8, 1);
    mbar_init(bar_free0, kEpiWarps * 32);
    mbar_init(bar_free0 + 8, kEpiWarps * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(2 * kN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == kEpiWarps) {
    if (lane == 0) {
      bool ok = true;
      mbar_expect_tx(bar_a, 2u * kb_count * kABlockBytes);
      for (int kb = 0; kb < kb_count; ++kb) {
        tma_load_2d(smem_addr(sa_hi + kb * kABlockBytes), &a_hi, bar_a, kb * kKB, e0);
        tma_load_2d(smem_addr(sa_lo + kb * kABlockBytes), &a_lo, bar_a, kb * kKB, e0);
      }
      ok = mbar_wait(bar_a, 0);
      const int ksteps = kp / 8;
      for (int64_t k = 0; k < my_tiles && ok; ++k) {
        const int buf = (int)(k & 1);
        const int s0 = (int)((blockIdx.y + k * gridDim.y) * kN);
        // the previous tile's MMAs have read the Xi tile
        if (k >= 1) ok = mbar_wait(bar_mma0 + 8 * ((k - 1) & 1), (uint32_t)(((k - 1) >> 1) & 1));
        if (!ok) break;
        mbar_expect_tx(bar_b, 2u * kb_count * kBBlockBytes);
        for (int kb = 0; kb < kb_count; ++kb) {
          tma_load_2d(smem_addr(sb_hi + kb * kBBlockBytes), &b_hi, bar_b, kb * kKB, s0);
          tma_load_2d(smem_addr(sb_lo + kb * kBBlockBytes), &b_lo, bar_b, kb * kKB, s0);
        }
        ok = mbar_wait(bar_b, (uint32_t)(k & 1));
        // the epilogue has read this accumulator's previous tile
        if (ok && k >= 2) ok = mbar_wait(bar_free0 + 8 * buf, (uint32_t)(((k - 2) >> 1) & 1));
        if (!ok) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kN);
        for (int ks = 0; ks < ksteps; ++ks) {
          const int kb = ks >> 2, off = (ks & 3) * 32;
          const uint64_t ah = sw128_desc(smem_addr(sa_hi + kb * kABlockBytes + off));
          const uint64_t al = sw128_desc(smem_addr(sa_lo + kb * kABlockBytes + off));
          const uint64_t bh = sw128_desc(smem_addr(sb_hi + kb * kBBlockBytes + off));
          const uint64_t bl = sw128_desc(smem_addr(sb_lo + kb * kBBlockBytes + off));
          mma_tf32(d, ah, bh, ks > 0 ? 1u : 0u);
          mma_tf32(d, ah, bl, 1u);
          mma_tf32(d, al, bh, 1u);
        }
        mma_commit(bar_mma0 + 8 * buf);
      }
      if (!ok) atomicExch(err, 1);
    }
  } else {
    const int quad = warp & 3, slice = warp >> 2;
    const int e = e0 + 32 * quad + lane;
    for (int64_t k = 0; k < my_tiles; ++k) {
      const int buf = (int)(k & 1);
      if (!mbar_wait(bar_mma0 + 8 * buf, (uint32_t)((k >> 1) & 1))) {
        atomicExch(err, 1);
        break;
      }
      tc_fence_after();
      float v[kEpiCols];
      tmem_ld16(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(buf * kN + slice * kEpiCols), v);
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(bar_free0 + 8 * buf);
      const int64_t s0 = (blockIdx.y + k * gridDim.y) * (int64_t)kN + slice * kEpiCols;
      if (e < n_el) {
#pragma unroll
        for (int c = 0; c < kEpiCols; ++c) {   // static register indices
          const int64_t s = s0 + c;
          if (s < nsamp) {
            if (trig2) {
              float sn, cs;
              sincosf(2.f * v[c], &sn, &cs);
              reinterpret_cast<float2*>(out)[s * n_el + e] = make_float2(cs, sn);
            } else {
              out[s * n_el + e] = v[c];
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kN) : "memory");
  }
}

size_t kl_tc_smem_bytes(int kp) {
  const int kb = (kp + kKB - 1) / kKB;
  return (size_t)kb * 2 * (kABlockBytes + kBBlockBytes) + 1024;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

void tf32_split_host(const double* x, int64_t rows, int n_kl, int kp, float* hi, float* lo) {
  for (int64_t r = 0; r < rows; ++r)
    for (int k = 0; k < kp; ++k) {
      float h = 0.f, l = 0.f;
      if (k < n_kl) split_one(x[r * n_kl + k], h, l);
      hi[r * kp + k] = h;
      lo[r * kp + k] = l;
    }
}

cudaError_t launch_tf32_split(const double* x, int64_t rows, int n_kl, int kp, float* hi, float* lo,
                              cudaStream_t st) {
  const int64_t n = rows * kp;
  if (n <= 0) return cudaSuccess;
  k_tf32_split<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, rows, n_kl, kp, hi, lo);
  return cudaGetLastError();
}

cudaError_t make_kl_tc_operand(const float* hi, const float* lo, int64_t rows, int kp, int box_rows,
                               KlTcOperand* out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (kp % 8 != 0 || kp > kKlTcMaxTerms || rows <= 0 || (reinterpret_cast<uintptr_t>(hi) & 15) ||
      (reinterpret_cast<uintptr_t>(lo) & 15))
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const float* parts[2] = {hi, lo};
  CUtensorMap* maps[2] = {&out->hi, &out->lo};
  for (int i = 0; i < 2; ++i) {
    CUresult r = enc(maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(parts[i]), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  out->kp = kp;
  return cudaSuccess;
}

cudaError_t launch_kl_synthesis_tc(const KlTcOperand& basis, const KlTcOperand& xi, int n_el, int64_t nsamp,
                                   float* out, bool trig2, int* err, cudaStream_t st) {
  if (nsamp <= 0 || n_el <= 0) return cudaSuccess;
  if (basis.kp != xi.kp || basis.kp % 8 != 0 || basis.kp > kKlTcMaxTerms) return cudaErrorInvalidValue;
  const size_t smem = kl_tc_smem_bytes(basis.kp);
  cudaError_t e = cudaFuncSetAttribute(k_kl_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gx = (n_el + kM - 1) / kM;
  const int64_t ntiles = (nsamp + kN - 1) / kN;
  const int64_t want = std::max<int64_t>(1, (sms + gx - 1) / gx);
  const int gy = (int)std::min<int64_t>(std::min<int64_t>(ntiles, want), 65535);
  k_kl_tc<<<dim3(gx, gy), kThreads, smem, st>>>(basis.hi, basis.lo, xi.hi, xi.lo, n_el, nsamp, basis.kp, out,
                                                 trig2 ? 1 : 0, err);
  return cudaGetLastError();
}

}  // namespace mlmc
