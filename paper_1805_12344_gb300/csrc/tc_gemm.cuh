// tcgen05 (5th-generation tensor core) GEMM for the shared-A batch, sm_103a.
//
//   Cpart[z][M x N] (FP32) = A[M x K_z] * W[K_z x N]
//
// A: TA bfloat16 terms A16[t] (M x K each, tile-major, see a_tiled) with A = sum of the
// terms, each the bfloat16 rounding of what the terms before it leave: TA = 1 when A is
// exact in bfloat16, TA = 3 for any A exact in FP32 (8 + 8 + 8 significant bits).  W: FP32
// row-major (N contiguous), the changes of the batched iterates, each element split the
// same way into three bfloat16 terms.  Every BF16 x BF16 product is exact and the
// accumulation is FP32 in tensor memory; of the term products A_a W_w the kernel issues
// those with a + w <= 2 (3 for TA = 1, 6 for TA = 3): the ones left out are below
// 2^-24 of the product, so the result has FP32 accuracy.
//
// One CTA (128 threads) owns a 128-row tile of C and one K range (split-K over
// gridDim.y).  Both operands are stored tile-major in the no-swizzle K-major core-matrix
// layout the MMA reads (8 rows x 16 bytes per core matrix; core matrices adjacent in K
// 128 bytes apart, adjacent in M/N kKC * 128 bytes): each K step of kTK is, per term,
// one contiguous block in HBM that a single bulk copy (cp.async.bulk, the 1-D form of
// TMA) moves into shared memory, completing on the stage's "full" mbarrier.  One thread
// issues the copies S - 1 steps ahead, waits for a stage, issues 2 x (3 or 6)
// tcgen05.mma (K = 16 each) into the TMEM accumulator and commits them to the stage's
// "empty" mbarrier, which releases the stage for the next copy.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, one lane per row) and
// writes the FP32 partial tile.  Every wait is bounded (kWaitLimitNs).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "async_copy.cuh"

namespace abip {
namespace tc {

constexpr int kTM = 128;          // rows per tile (MMA M)
constexpr int kTK = 32;           // K per staging step
constexpr int kTCThreads = 128;
constexpr int kErrTimeout = 1;
constexpr int kErrShape = 2;



// Shared-memory matrix descriptor: no swizzle, K-major.  lbo: byte distance between core
// matrices adjacent in K; sbo: between core matrices adjacent in M (or N).  Bits 46-48
// hold the fixed descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
  d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor for kind::f16: BF16 A and B (both K-major), FP32 accumulator.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4)                                   // D: F32
         | (1u << 7)                                 // A: BF16
         | (1u << 10)                                // B: BF16
         | (static_cast<uint32_t>(N >> 3) << 17)     // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}



__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Warp-wide: allocate ncols TMEM columns (power of two >= 32), address into *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Warp-wide: 16 consecutive FP32 columns of the warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// K chunks of 8 elements (16 bytes) per tile row, and the byte distance between core
// matrices adjacent in M (or N): a row group of 8 holds kKC core matrices of 128 bytes.
constexpr int kKC = kTK / 8;
constexpr uint32_t kSBO = kKC * 128;

// Byte offset of the 16-byte row chunk (row r, K chunk kc of 8 elements) in a tile of
// core matrices: core (r / 8, kc) at ((r / 8) * kKC + kc) * 128, row r % 8 at 16 (r % 8).
__host__ __device__ __forceinline__ uint32_t core_off(int r, int kc) {
  return static_cast<uint32_t>(((r >> 3) * kKC + kc) * 128 + (r & 7) * 16);
}

// Tile-major bfloat16 layouts (element offsets within one term plane).
// A (R x K, R % kTM == 0, K % kTK == 0): tile (r / kTM, k / kTK) is the contiguous block
// number (r / kTM) * (K / kTK) + k / kTK of kTM * kTK elements, core-matrix ordered.
__host__ __device__ __forceinline__ size_t a_tiled(int r, int k, int K) {
  const size_t tile = (size_t)(r / kTM) * (K / kTK) + k / kTK;
  return tile * (kTM * kTK) + core_off(r % kTM, (k % kTK) >> 3) / 2 + (k & 7);
}
// W (N rows x K, the changes transposed; N % 16 == 0): K step s is the contiguous block s
// of N * kTK elements.
__host__ __device__ __forceinline__ size_t w_tiled(int n, int k, int N) {
  return (size_t)(k / kTK) * N * kTK + core_off(n, (k % kTK) >> 3) / 2 + (k & 7);
}

// ---------------------------------------------------------------------------
// The changes are split beforehand into three bfloat16 arrays Wt[t] (N rows x K, K
// contiguous), so every tile is a plain 16-byte copy.  S shared-memory stages: while the
// MMAs of step j run, cp.async fills the stages of steps j + 1 .. j + S - 1; an mbarrier
// per stage tells when its MMAs have finished reading it.
// ---------------------------------------------------------------------------

// Wt[t] (term t, N * K elements, tile-major as w_tiled) = t-th bfloat16 term of W^T
// (W: K x N FP32 row-major, ldw).
__global__ void split3_kernel(const float* __restrict__ W, int64_t ldw, int K, int N, __nv_bfloat16* __restrict__ Wt) {
  __shared__ float tile[32][33];
  const int k0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, n = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && n < N) ? W[(size_t)k * ldw + n] : 0.f;
  }
  __syncthreads();
  const size_t plane = (size_t)N * K;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int n = n0 + r, k = k0 + threadIdx.x;
    if (n < N && k < K) {
      const float w = tile[threadIdx.x][r];
      const __nv_bfloat16 h = __float2bfloat16_rn(w);
      const float r1 = w - __bfloat162float(h);
      const __nv_bfloat16 md = __float2bfloat16_rn(r1);
      const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(md));
      const size_t e = w_tiled(n, k, N);
      Wt[e] = h;
      Wt[plane + e] = md;
      Wt[2 * plane + e] = lo;
    }
  }
}


__host__ __device__ inline size_t tc2_stage_bytes(int N, int TA) {
  return static_cast<size_t>(TA) * kTM * kTK * 2 + 3 * static_cast<size_t>(N) * kTK * 2;
}
// shared-memory stages: as many as fit in the 227 KB a CTA may use (less 2 KB for the
// 1024-byte alignment of the tiles and the static variables), at most 6
constexpr size_t kTcSmemCap = 227 * 1024 - 2048;
__host__ __device__ inline int tc2_stages(int N, int TA) {
  const int s = static_cast<int>(kTcSmemCap / tc2_stage_bytes(N, TA));
  return s < 6 ? s : 6;
}
__host__ __device__ inline size_t tc2_smem_bytes(int N, int TA) {
  return 1024 + tc2_stages(N, TA) * tc2_stage_bytes(N, TA);
}

// Requirements (refused on the device with kErrShape): M % 128 == 0, K % kTK == 0,
// kchunk % kTK == 0, N % 16 == 0 and 16 <= N <= 256, aplane % 8 == 0, A16 and Wt 16-byte
// aligned, tc2_stages(N, TA) == S >= 2.  A16: TA planes of M x K, aplane elements apart,
// tile-major (a_tiled); Wt: 3 planes of N x K, tile-major (w_tiled).
// Dynamic shared memory: tc2_smem_bytes(N, TA).
template <int S, int TA>
__global__ void __launch_bounds__(kTCThreads, 1)
    tc_gemm2_kernel(const __nv_bfloat16* __restrict__ A16, int64_t aplane, int M, int N, int K,
                    const __nv_bfloat16* __restrict__ Wt, float* __restrict__ Cp, int kchunk, int* err) {
  // shapes the tiles and the bulk copies need; anything else is refused here
  if (M % kTM != 0 || K % kTK != 0 || kchunk <= 0 || kchunk % kTK != 0 || N % 16 != 0 || N < 16 || N > 256 ||
      aplane % 8 != 0 || (reinterpret_cast<uintptr_t>(A16) & 15) != 0 || (reinterpret_cast<uintptr_t>(Wt) & 15) != 0 ||
      tc2_stages(N, TA) != S || S < 2) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) atomicExch(err, kErrShape);
    return;
  }
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ uint64_t full[S], empty[S];
  __shared__ uint32_t tslot;
  __shared__ int failed;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t stage = static_cast<uint32_t>(tc2_stage_bytes(N, TA));
  const uint32_t atile = kTM * kTK * 2, abytes = TA * atile, wbytes = static_cast<uint32_t>(N) * kTK * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTM;
  const int kz0 = blockIdx.y * kchunk, kz1 = min(K, kz0 + kchunk);
  const int steps = kz1 > kz0 ? (kz1 - kz0) / kTK : 0;
  uint32_t ncols = 32;
  while (ncols < static_cast<uint32_t>(N)) ncols <<= 1;
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < S; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    failed = 0;
  }
  if (warp == 0) tmem_alloc(&tslot, ncols);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t idesc = instr_desc(kTM, N);
  const uint32_t s0 = smem_u32(base);
  if (tid == 0) {
    // step j of this CTA: A block (row tile blockIdx.x, K tile kz0 / kTK + j) of each term,
    // W block (K tile kz0 / kTK + j) of each term
    const char* a0p = reinterpret_cast<const char*>(A16) +
                      ((size_t)blockIdx.x * (K / kTK) + kz0 / kTK) * (size_t)atile;
    const char* w0p = reinterpret_cast<const char*>(Wt) + (size_t)(kz0 / kTK) * wbytes;
    const size_t ap = (size_t)aplane * 2, wp = (size_t)N * K * 2;
    auto issue = [&](int j) {
      const int b = j % S;
      const uint32_t sa = s0 + b * stage;
      mbar_arrive_expect_tx(&full[b], abytes + 3 * wbytes);
#pragma unroll
      for (int t = 0; t < TA; ++t) bulk_g2s(sa + t * atile, a0p + t * ap + (size_t)j * atile, atile, &full[b]);
#pragma unroll
      for (int t = 0; t < 3; ++t) bulk_g2s(sa + abytes + t * wbytes, w0p + t * wp + (size_t)j * wbytes, wbytes, &full[b]);
    };
    int issued = 0, committed = 0;
    for (; issued < S && issued < steps; ++issued) issue(issued);
    int j = 0;
    for (; j < steps; ++j) {
      const int b = j % S;
      if (!mbar_wait(&full[b], (j / S) & 1u)) { failed = 1; break; }
      tc_fence_after();
      const uint32_t a0 = s0 + b * stage, w0 = a0 + abytes;
#pragma unroll
      for (int s = 0; s < kTK / 16; ++s) {
#pragma unroll
        for (int ta = 0; ta < TA; ++ta) {
          const uint64_t ad = smem_desc(a0 + ta * atile + s * 256, 128, kSBO);
#pragma unroll
          for (int t = 0; t + ta < 3; ++t) {
            const uint64_t bd = smem_desc(w0 + t * wbytes + s * 256, 128, kSBO);
            mma_bf16(tmem, ad, bd, idesc, (j > 0 || s > 0 || ta > 0 || t > 0) ? 1u : 0u);
          }
        }
      }
      mma_commit(&empty[b]);
      committed = j + 1;
      // the stage of step j - 1 is free once its MMAs are done: refill it with step j - 1 + S
      if (j >= 1 && issued < steps) {
        const int pb = (j - 1) % S;
        if (!mbar_wait(&empty[pb], ((j - 1) / S) & 1u)) { failed = 1; ++j; break; }
        issue(issued++);
      }
    }
    if (!failed && steps > 0) {
      // the last commit covers every earlier MMA of this thread
      const int lb = (steps - 1) % S;
      if (!mbar_wait(&empty[lb], ((steps - 1) / S) & 1u)) failed = 1;
    }
    if (failed) {
      atomicExch(err, kErrTimeout);
      // no copy may still be writing shared memory, and no MMA still running, when the CTA
      // leaves and frees its tensor memory (bounded waits)
      for (int q = j; q < issued; ++q) mbar_wait(&full[q % S], (q / S) & 1u);
      if (committed > 0) mbar_wait(&empty[(committed - 1) % S], ((committed - 1) / S) & 1u);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  float* C = Cp + (size_t)blockIdx.y * M * N;
  const int row = m0 + warp * 32 + lane;
  if (!failed) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      if (steps > 0) {
        tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c0), v);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < 16; q += 4)
        *reinterpret_cast<float4*>(C + (size_t)row * N + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace tc
}  // namespace abip
