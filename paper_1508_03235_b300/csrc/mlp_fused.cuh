// mlp_fused.cuh -- the whole surrogate network's inference in one kernel on
// the 5th-generation tensor cores.  One CTA of 128 threads carries 128 rows of
// the batch through every layer: the activations stay in shared memory in the
// canonical 128-byte-swizzled K-major operand layout, each layer's FP32
// accumulator lives in tensor memory, and only the last layer's output is
// written to HBM.  The weights are packed once (mlp_pack) into the same
// shared-memory image, layer after layer, so that each layer arrives with
// bulk copies (cp.async.bulk, completing on an mbarrier) while the tensor
// cores idle at most for the first one: the next layer's copy is issued as
// soon as the current layer's MMAs have read the weight buffer, and overlaps
// the epilogue.  Arithmetic and summation order are those of the layered
// tcgen05 path (mlp_tc.cuh), so the outputs are the same.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mlp_tc.cuh"

namespace mlpk {
namespace fused {

constexpr int MAXD = 256;                 // widest layer (MMA N and staged K)
constexpr int KB_MAX = MAXD / tc::KATOM;  // 128-byte row blocks of the widest K
// 16 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile) and
// the (w / 4)-th quarter of a layer's columns, so that the bias + GELU
// epilogue, not the tensor cores, sets the pace at four times the width
constexpr int FT = 512;

// byte offsets of one layer's packed weight image and bias inside the image
struct Layer {
  uint32_t w_off, w_bytes;  // [kblocks][N rows][128 B], swizzled
  uint32_t b_off;           // N BF16 biases
  int K, N;
};
struct Plan {
  int n_layers;
  Layer l[8];
  uint32_t bytes;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// the shapes the fused kernel takes: every width a multiple of 16 in 16..256
__host__ inline bool plan_of(int n_layers, const int* dims, Plan& p) {
  if (n_layers < 1 || n_layers > 8) return false;
  p.n_layers = n_layers;
  uint32_t o = 0;
  for (int l = 0; l < n_layers; ++l) {
    const int K = dims[l], N = dims[l + 1];
    if (K < 16 || K > MAXD || K % 16 || N < 16 || N > MAXD || N % 16) return false;
    p.l[l].K = K;
    p.l[l].N = N;
    p.l[l].w_off = o;
    p.l[l].w_bytes = (uint32_t)tc::kblocks_of(K) * N * 128u;
    o += p.l[l].w_bytes;
    p.l[l].b_off = o;
    o = align16(o + 2u * N);
  }
  p.bytes = o;
  return true;
}

// dynamic shared memory: 1024-byte alignment slack, the activation operand
// (128 rows), the weight operand (up to 256 rows), two mbarriers, TMEM slot
constexpr size_t smem_bytes() {
  return 1024 + (size_t)tc::TM * KB_MAX * 128 + (size_t)MAXD * KB_MAX * 128 + 64;
}

// pack: one thread per 16-byte piece of a layer's image (zero where K ends
// inside a row block), biases copied after each layer's weights
__global__ void pack_kernel(const __nv_bfloat16* __restrict__ params, size_t wpos0, Layer L,
                            unsigned char* __restrict__ image) {
  const int kb_n = tc::kblocks_of(L.K);
  const size_t pieces = (size_t)kb_n * L.N * 8;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < pieces + L.N;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e >= pieces) {  // bias element
      const int n = (int)(e - pieces);
      reinterpret_cast<__nv_bfloat16*>(image + L.b_off)[n] = params[wpos0 + (size_t)L.N * L.K + n];
      continue;
    }
    const int c = (int)(e & 7), n = (int)((e >> 3) % L.N), kb = (int)((e >> 3) / L.N);
    uint4 v = make_uint4(0, 0, 0, 0);
    const int k = kb * tc::KATOM + c * 8;
    if (k < L.K) v = *reinterpret_cast<const uint4*>(params + wpos0 + (size_t)n * L.K + k);
    *reinterpret_cast<uint4*>(image + L.w_off + (size_t)kb * L.N * 128 + n * 128 + ((c ^ (n & 7)) << 4)) = v;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_copy(void* smem, const void* gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(smem)),
      "l"(gmem), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}
// a layer's weights into the weight buffer: one expect_tx, then copies of at
// most 32 KB
__device__ __forceinline__ void load_weights(unsigned char* Ws, const unsigned char* image, const Layer& L,
                                             uint64_t* bar) {
  mbar_expect_tx(bar, L.w_bytes);
  for (uint32_t o = 0; o < L.w_bytes; o += 32768u) {
    const uint32_t n = L.w_bytes - o < 32768u ? L.w_bytes - o : 32768u;
    bulk_copy(Ws + o, image + L.w_off + o, n, bar);
  }
}
// bounded wait for phase `parity` of `bar` by every thread of the CTA; false
// (and the status word set) if it ran out
__device__ __forceinline__ bool wait_all(uint64_t* bar, uint32_t parity) {
  bool ok = false;
  for (uint32_t it = 0; it < (1u << 22) && !ok; ++it) {
    ok = tc::mbar_try_wait(bar, parity);
    if (!ok && it > 64) __nanosleep(200);
  }
  const bool all = __syncthreads_and(ok);
  if (!all && threadIdx.x == 0) atomicCAS(&tc::g_tc_status, 0u, 1u);
  return all;
}

// y[B][N_last] (FP32) for x[B][K_0] (BF16); grid B / 128 CTAs of FT threads
__global__ void __launch_bounds__(FT, 1)
    infer_kernel(const __grid_constant__ Plan plan, const unsigned char* __restrict__ image,
                 const __nv_bfloat16* __restrict__ x, float* __restrict__ y) {
  extern __shared__ unsigned char raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* As = base;                                   // [kb][128 rows][128 B]
  unsigned char* Ws = base + (size_t)tc::TM * KB_MAX * 128;   // [kb][N rows][128 B]
  uint64_t* wbar = reinterpret_cast<uint64_t*>(Ws + (size_t)MAXD * KB_MAX * 128);
  uint64_t* mbar = wbar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * tc::TM;
  const int L = plan.n_layers;

  if (warp == 0) tc::tmem_alloc(tslot, MAXD);
  if (tid == 0) {
    tc::mbar_init(wbar, 1);
    tc::mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) load_weights(Ws, image, plan.l[0], wbar);
  // this CTA's 128 input rows into the activation operand
  {
    const int K0 = plan.l[0].K, kbs = tc::kblocks_of(K0);
    for (int e = tid; e < tc::TM * kbs * 8; e += FT) {
      const int c = e & 7, r = (e >> 3) % tc::TM, kb = (e >> 3) / tc::TM;
      if (kb * tc::KATOM + c * 8 >= K0) continue;
      tc::cp_async16(As + (size_t)kb * tc::TM * 128 + r * 128 + ((c ^ (r & 7)) << 4),
                     x + (size_t)(m0 + r) * K0 + kb * tc::KATOM + c * 8);
    }
    tc::cp_async_wait_all();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const int r = (warp & 3) * 32 + lane;    // this thread's row of the tile
  const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
  const int quarter = warp >> 2;
  bool ok = true;
  int pending = 0;                         // layer whose weight copy is in flight (-1: none)

  for (int l = 0; l < L && ok; ++l) {
    const Layer& Ly = plan.l[l];
    ok = wait_all(wbar, (uint32_t)(l & 1));        // this layer's weights are in
    if (!ok) break;
    pending = -1;
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t idesc = tc::instr_desc(tc::TM, Ly.N);
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Ws);
      const int kbs = tc::kblocks_of(Ly.K);
      for (int kb = 0; kb < kbs; ++kb)
        for (int ks = 0; ks < tc::KATOM / 16 && kb * tc::KATOM + ks * 16 < Ly.K; ++ks)
          tc::mma(tmem, tc::smem_desc(a0 + kb * tc::TM * 128 + ks * 32),
                  tc::smem_desc(b0 + kb * Ly.N * 128 + ks * 32), idesc, (kb | ks) != 0);
      tc::commit(mbar);
    }
    ok = wait_all(mbar, (uint32_t)(l & 1));        // the accumulator is complete
    if (!ok) break;
    tc::fence_after_sync();
    // the weight buffer is free: the next layer's copy overlaps this epilogue
    if (l + 1 < L) {
      if (tid == 0) load_weights(Ws, image, plan.l[l + 1], wbar);
      pending = l + 1;
    }
    const __nv_bfloat16* bias = reinterpret_cast<const __nv_bfloat16*>(image + Ly.b_off);
    const bool last = l + 1 == L;
    // this warp's quarter of the columns, in 16-column multiples
    const int cq = ((Ly.N + 63) / 64) * 16, c_lo = quarter * cq;
    const int c_hi = c_lo + cq < Ly.N ? c_lo + cq : Ly.N;
    for (int col = c_lo; col < c_hi; col += 32) {
      float v[32];
      int w = 32;
      if (c_hi - col >= 32) {
        tc::tmem_ld32(tmem + lanes + (uint32_t)col, v);
      } else {
        float h[16];
        tc::tmem_ld16(tmem + lanes + (uint32_t)col, h);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = h[j];
        w = 16;
      }
      // the biases of these columns in 16-byte pieces (the packed image puts
      // each layer's biases on a 16-byte boundary and col is a multiple of 16)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (8 * q >= w) continue;
        const uint4 b8 = *reinterpret_cast<const uint4*>(bias + col + 8 * q);
        const uint32_t bw[4] = {b8.x, b8.y, b8.z, b8.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          v[8 * q + 2 * j] += __uint_as_float(bw[j] << 16);
          v[8 * q + 2 * j + 1] += __uint_as_float(bw[j] & 0xFFFF0000u);
        }
      }
      if (last) {
        float4* p = reinterpret_cast<float4*>(y + (size_t)(m0 + r) * Ly.N + col);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (4 * q < w) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        // GELU, BF16, into the operand layout of the next layer (K = this N)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (8 * q >= w) continue;
          uint32_t pk[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu(v[8 * q + 2 * j]), gelu(v[8 * q + 2 * j + 1]));
            pk[j] = *reinterpret_cast<const uint32_t*>(&h2);
          }
          const int k = col + 8 * q, kb = k / tc::KATOM, c = (k % tc::KATOM) / 8;
          *reinterpret_cast<uint4*>(As + (size_t)kb * tc::TM * 128 + r * 128 + ((c ^ (r & 7)) << 4)) =
              make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
    }
    // the new activations must be visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();
  }
  // after a wait that ran out, give a weight copy still in flight its own
  // bounded wait before the shared memory is released
  if (!ok && pending >= 0) wait_all(wbar, (uint32_t)(pending & 1));
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, MAXD);
}

}  // namespace fused
}  // namespace mlpk
