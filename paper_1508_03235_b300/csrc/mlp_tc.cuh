// mlp_tc.cuh -- the surrogate's dense layers on the 5th-generation tensor
// cores (sm_100 family): tcgen05.mma with the FP32 accumulator in tensor
// memory (TMEM), issued by one thread, operands in 128-byte-swizzled shared
// memory, completion signalled through an mbarrier, and the bias + GELU
// epilogue reading the accumulator back with tcgen05.ld.
//
// One CTA of 128 threads computes a 128 x NT tile of C = A * B^T (+ bias):
// A is [M][K] and B is [N][K], both K-major (row-major with unit stride in K),
// K >= 16 with K % 16 == 0, M % 128 == 0, and the CTA grid is (M / 128) x
// (N / NT) with NT in {16, 32, 64, 128, 256} dividing N.  K is taken in chunks
// of at most MAXK: each chunk of both operand tiles is staged in shared memory
// (at most 192 KB), its K / 16 MMA steps accumulate into the same TMEM tile
// under one commit, and the next chunk is staged once that commit's mbarrier
// phase completes.  A chunk is stored in 128-byte rows of 64 elements; a last
// partial row block holds only the 16-byte pieces the MMA steps read.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mlpk {
namespace tc {

constexpr int TM = 128;       // rows per CTA = MMA M
constexpr int KATOM = 64;     // bf16 elements in one 128-byte swizzled row
constexpr int THREADS = 128;  // one warpgroup: warp w reads TMEM lanes 32w..32w+31
constexpr int MAXK = 256, MAXN = 256;

__host__ __device__ constexpr int kblocks_of(int K) { return (K + KATOM - 1) / KATOM; }
__host__ __device__ constexpr size_t smem_bytes(int NT, int K) {
  // 1024-byte alignment slack, A and B tiles (whole 128-byte rows), then an
  // 8-byte mbarrier and the 4-byte TMEM address slot
  return 1024 + (size_t)TM * kblocks_of(K) * 128 + (size_t)NT * kblocks_of(K) * 128 + 64;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the leading-dimension offset is unused for this layout)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);        // start address >> 4, bits 0-13
  d |= (uint64_t)(16u >> 4) << 16;                // leading byte offset >> 4, bits 16-29
  d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset >> 4, bits 32-45
  d |= (uint64_t)1 << 46;                         // descriptor version 1, bits 46-47
  d |= (uint64_t)2 << 61;                         // swizzle: 128 bytes, bits 61-63
  return d;
}

// instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4)                      // accumulator format FP32
         | (1u << 7)                    // A format BF16
         | (1u << 10)                   // B format BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// 16-byte asynchronous global -> shared copy (all of a thread's copies are in
// flight together; cp_async_wait_all waits for them)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 consecutive FP32 columns: thread l of the warp gets row
// (lane base + l), columns col .. col + 31
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// the first non-zero status of a call (1: an MMA completion wait ran out)
__device__ unsigned int g_tc_status;

template <typename Epi>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_kernel(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B, int M,
                int NT, int K, Epi epi) {
  extern __shared__ unsigned char raw[];
  // operand tiles start on a 1024-byte boundary (the swizzle pattern's period)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int KC = K < MAXK ? K : MAXK;                         // K of one chunk
  const int kblocks_max = kblocks_of(KC);
  unsigned char* As = base;                                   // [kblocks][128 rows][128 B]
  unsigned char* Bs = base + (size_t)TM * kblocks_max * 128;  // [kblocks][NT rows][128 B]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)NT * kblocks_max * 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * NT;
  const uint32_t ncols = NT < 32 ? 32u : (uint32_t)NT;   // a power of two >= 32

  if (warp == 0) tmem_alloc(tslot, ncols);
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  bool done = true;
  uint32_t tmem = 0;
  for (int k0 = 0, chunk = 0; k0 < K && done; k0 += KC, ++chunk) {
    const int kc = K - k0 < KC ? K - k0 : KC;
    const int kblocks = kblocks_of(kc);
    // operands into shared memory in the canonical 128-byte-swizzled K-major
    // layout: 16-byte piece c of row r goes to piece c ^ (r & 7); pieces past
    // the chunk are neither loaded nor read
    for (int e = tid; e < TM * kblocks * 8; e += THREADS) {
      const int c = e & 7, r = (e >> 3) % TM, kb = (e >> 3) / TM;
      if (kb * KATOM + c * 8 >= kc) continue;
      cp_async16(As + (size_t)kb * TM * 128 + r * 128 + ((c ^ (r & 7)) << 4),
                 A + (size_t)(m0 + r) * K + k0 + kb * KATOM + c * 8);
    }
    for (int e = tid; e < NT * kblocks * 8; e += THREADS) {
      const int c = e & 7, n = (e >> 3) % NT, kb = (e >> 3) / NT;
      if (kb * KATOM + c * 8 >= kc) continue;
      cp_async16(Bs + (size_t)kb * NT * 128 + n * 128 + ((c ^ (n & 7)) << 4),
                 B + (size_t)(n0 + n) * K + k0 + kb * KATOM + c * 8);
    }
    cp_async_wait_all();
    // the copies must be visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    tmem = *tslot;

    if (tid == 0) {
      const uint32_t idesc = instr_desc(TM, NT);
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      for (int kb = 0; kb < kblocks; ++kb)
        for (int ks = 0; ks < KATOM / 16 && kb * KATOM + ks * 16 < kc; ++ks)
          mma(tmem, smem_desc(a0 + kb * TM * 128 + ks * 32), smem_desc(b0 + kb * NT * 128 + ks * 32),
              idesc, (k0 | kb | ks) != 0);
      commit(bar);
    }
    // wait for this chunk's MMAs (bounded: about a second of polling at
    // most); the mbarrier's phase parity alternates chunk by chunk
    bool ok = false;
    for (uint32_t it = 0; it < (1u << 22) && !ok; ++it) {
      ok = mbar_try_wait(bar, (uint32_t)(chunk & 1));
      if (!ok && it > 64) __nanosleep(200);
    }
    done = __syncthreads_and(ok);           // every thread saw the phase complete
    if (!done && tid == 0) atomicCAS(&g_tc_status, 0u, 1u);
    fence_after_sync();
  }

  // epilogue: warp w holds rows 32w .. 32w + 31 of the tile, one per lane
  if (done) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    if (NT == 16) {
      float v[16];
      tmem_ld16(tmem + lanes, v);
      epi(row, n0, v);
    } else {
      for (int col = 0; col < NT; col += 32) {
        float v[32];
        tmem_ld32(tmem + lanes + (uint32_t)col, v);
        epi(row, n0 + col, v);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace tc
}  // namespace mlpk
