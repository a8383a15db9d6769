// mlp.cu -- the surrogate network's kernels (include/mlp.h): tensor-core GEMMs
// in BF16 with FP32 accumulation -- tcgen05 (mlp_tc.cuh) for the forward and
// backward GEMMs whose shapes it takes, mma.sync m16n8k16 for the rest -- with
// the bias, GELU and pre-activation store fused into the GEMM epilogue, plus
// the transpose, GELU backward, bias-gradient, MSE and AdamW kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "mlp.h"
#include "mlp_tc.cuh"

namespace mlpk {

constexpr int BM = 64, BN = 64, BK = 32, PAD = 8, THREADS = 128;

struct Gemm {
  int M, N, K;
  const __nv_bfloat16* A;  // A[m][k] = A[m * sAm + k * sAk]
  long long sAm, sAk;
  const __nv_bfloat16* B;  // B[k][n] = B[n * sBn + k * sBk]
  long long sBn, sBk;
  const __nv_bfloat16* bias;  // [N] (BF16 parameter copy) or null
  float* Cf;               // FP32 result (bias added, before GELU) or null
  __nv_bfloat16* Cb;       // BF16 result (after GELU if gelu) or null
  long long ldc;
  int gelu;
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// C[M][N] = A[M][K] * B[K][N] (+ bias); a 64x64 tile per CTA, four warps of
// 32x32, K in steps of 32 staged through shared memory.
__global__ void __launch_bounds__(THREADS) gemm_kernel(const Gemm g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += THREADS) {
      const int r = e / BK, c = e % BK, k = k0 + c;
      const int m = m0 + r, n = n0 + r;
      As[r][c] = (m < g.M && k < g.K) ? g.A[m * g.sAm + k * g.sAk] : zero;
      Bs[r][c] = (n < g.N && k < g.K) ? g.B[n * g.sBn + k * g.sBk] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm + mi * 16 + gid;
        a[mi][0] = ld_pair(&As[r][kk + tig * 2]);
        a[mi][1] = ld_pair(&As[r + 8][kk + tig * 2]);
        a[mi][2] = ld_pair(&As[r][kk + tig * 2 + 8]);
        a[mi][3] = ld_pair(&As[r + 8][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int n = wn + ni * 8 + gid;
        b[ni][0] = ld_pair(&Bs[n][kk + tig * 2]);
        b[ni][1] = ld_pair(&Bs[n][kk + tig * 2 + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int row = m0 + wm + mi * 16 + gid + h * 8;
          const int col = n0 + wn + ni * 8 + tig * 2 + j;
          if (row >= g.M || col >= g.N) continue;
          float v = acc[mi][ni][h * 2 + j] + (g.bias ? __bfloat162float(g.bias[col]) : 0.0f);
          const long long o = row * g.ldc + col;
          if (g.Cf) g.Cf[o] = v;
          if (g.Cb) g.Cb[o] = __float2bfloat16_rn(g.gelu ? gelu(v) : v);
        }
}

// epilogue of the tcgen05 GEMM: W (16 or 32) consecutive columns of one row
// per thread
struct TcEpi {
  const __nv_bfloat16* bias;
  float* Cf;
  __nv_bfloat16* Cb;
  long long ldc;
  int gelu;
  template <int W>
  __device__ void operator()(int row, int col, const float (&v)[W]) const {
    float o[W];
#pragma unroll
    for (int j = 0; j < W; ++j) o[j] = v[j] + (bias ? __bfloat162float(bias[col + j]) : 0.0f);
    if (Cf) {
      float4* p = reinterpret_cast<float4*>(Cf + row * ldc + col);
#pragma unroll
      for (int q = 0; q < W / 4; ++q) p[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
    if (Cb) {
      uint32_t w[W / 2];
#pragma unroll
      for (int j = 0; j < W / 2; ++j) {
        const float a = gelu ? mlpk::gelu(o[2 * j]) : o[2 * j];
        const float b = gelu ? mlpk::gelu(o[2 * j + 1]) : o[2 * j + 1];
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        w[j] = *reinterpret_cast<const uint32_t*>(&h);
      }
      uint4* p = reinterpret_cast<uint4*>(Cb + row * ldc + col);
#pragma unroll
      for (int q = 0; q < W / 8; ++q) p[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
  }
};

}  // namespace mlpk
#include "mlp_fused.cuh"
namespace mlpk {

int g_path = 0;  // 0: tcgen05 where it applies, 1: mma.sync for every GEMM

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// the GEMM shapes the tcgen05 kernel takes (both operands K-major)
bool tc_shape(int M, int N, int K) {
  return g_path == 0 && K >= 16 && K % 16 == 0 && M % tc::TM == 0 && N % 16 == 0 && N <= tc::MAXN;
}

bool tc_applies(const Gemm& g) {
  return g_path == 0 && g.sAk == 1 && g.sAm == g.K && g.sBk == 1 && g.sBn == g.K && tc_shape(g.M, g.N, g.K) &&
         aligned16(g.A) && aligned16(g.B) && (!g.Cf || (aligned16(g.Cf) && g.ldc % 4 == 0)) &&
         (!g.Cb || (aligned16(g.Cb) && g.ldc % 8 == 0));
}

cudaError_t gemm(const Gemm& g, cudaStream_t s) {
  if (tc_applies(g)) {
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(tc::gemm_kernel<TcEpi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)tc::smem_bytes(tc::MAXN, tc::MAXK));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    const TcEpi epi{g.bias, g.Cf, g.Cb, g.ldc, g.gelu};
    // column tiles of 64 (or the whole width if narrower) so that a layer
    // spreads over (M / 128) x (N / 64) CTAs
    const int nt = g.N % 64 == 0 ? 64 : (g.N % 32 == 0 ? 32 : 16);
    const dim3 grid(g.M / tc::TM, g.N / nt);
    const int kc = g.K < tc::MAXK ? g.K : tc::MAXK;
    tc::gemm_kernel<TcEpi><<<grid, tc::THREADS, tc::smem_bytes(nt, kc), s>>>(g.A, g.B, g.M, nt, g.K, epi);
    return cudaGetLastError();
  }
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  gemm_kernel<<<grid, THREADS, 0, s>>>(g);
  return cudaGetLastError();
}

// dst[c][r] = src[r][c] for a rows x cols BF16 matrix (32 x 32 tiles through
// shared memory, so that both the reads and the writes are coalesced)
__global__ void transpose_kernel(const __nv_bfloat16* src, int rows, int cols, __nv_bfloat16* dst) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j, c = c0 + tx;
    if (r < rows && c < cols) t[j][tx] = src[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int c = c0 + j, r = r0 + tx;
    if (r < rows && c < cols) dst[(size_t)c * rows + r] = t[tx][j];
  }
}

cudaError_t transpose(const __nv_bfloat16* src, int rows, int cols, __nv_bfloat16* dst, cudaStream_t s) {
  transpose_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, s>>>(src, rows, cols, dst);
  return cudaGetLastError();
}

// dZ = dA * gelu'(Z) in FP32 and BF16
__global__ void gelu_back_kernel(const float* dA, const float* Z, float* dZf, __nv_bfloat16* dZb,
                                 size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float v = dA[i] * gelu_grad(Z[i]);
    dZf[i] = v;
    dZb[i] = __float2bfloat16_rn(v);
  }
}

// db[n] = sum over rows of dZ[m][n]; 32 columns per CTA, 8 row lanes
__global__ void colsum_kernel(const float* dZ, int M, int N, float* db) {
  __shared__ float part[8][33];
  const int c = threadIdx.x & 31, r = threadIdx.x >> 5, col = blockIdx.x * 32 + c;
  float s = 0.0f;
  if (col < N)
    for (int m = r; m < M; m += 8) s += dZ[(size_t)m * N + col];
  part[r][c] = s;
  __syncthreads();
  if (r == 0 && col < N) {
    float t = 0.0f;
    for (int k = 0; k < 8; ++k) t += part[k][c];
    db[col] = t;
  }
}

__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void mse_kernel(const float* y, const float* t, int B, int D, int used, float* loss,
                           float* dy) {
  __shared__ float part[256];
  const float scale = 1.0f / ((float)B * (float)used);
  float s = 0.0f;
  for (int i = threadIdx.x; i < B * D; i += blockDim.x) {
    const int c = i % D;
    float d = c < used ? y[i] - t[i] : 0.0f;
    s += d * d;
    dy[i] = 2.0f * d * scale;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = part[0] * scale;
}

__global__ void adamw_kernel(size_t n, float* p, __nv_bfloat16* pb, const float* g, float* m,
                             float* v, float lr, float b1, float b2, float eps, float wd, float c1,
                             float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / c1, vh = vi / c2;
    float pi = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

int grid_1d(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)(g > 4096 ? 4096 : (g ? g : 1));
}

bool shape_ok(const mlp_shape* s) {
  if (!s || s->n_layers < 1 || s->n_layers > MLP_MAX_LAYERS) return false;
  for (int l = 0; l <= s->n_layers; ++l)
    if (s->dims[l] < 8 || s->dims[l] % 8 || s->dims[l] > 65536) return false;
  return true;
}

// parameter offsets (floats): W_l then b_l, layer by layer
size_t w_off(const mlp_shape* s, int l) {
  size_t o = 0;
  for (int k = 0; k < l; ++k) o += (size_t)s->dims[k + 1] * s->dims[k] + s->dims[k + 1];
  return o;
}

struct Workspace {
  float* Z[MLP_MAX_LAYERS];           // pre-activations [B][dims[l+1]]
  __nv_bfloat16* A[MLP_MAX_LAYERS];   // activations of hidden layers [B][dims[l+1]]
  float *dAf, *dZf;
  __nv_bfloat16* dZb;
  // K-major copies for the tcgen05 backward GEMMs: dZ^T [N][B], the layer
  // input transposed [K][B], W^T [K][N]
  __nv_bfloat16 *dZt, *inT, *Wt;
  size_t bytes;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

Workspace carve(const mlp_shape* s, int B, void* base) {
  Workspace w;
  unsigned char* p = static_cast<unsigned char*>(base);
  size_t o = 0;
  int maxd = 0;
  for (int l = 0; l <= s->n_layers; ++l) maxd = maxd > s->dims[l] ? maxd : s->dims[l];
  for (int l = 0; l < s->n_layers; ++l) {
    w.Z[l] = reinterpret_cast<float*>(p + o);
    o = a256(o + (size_t)B * s->dims[l + 1] * 4);
    w.A[l] = reinterpret_cast<__nv_bfloat16*>(p + o);
    o = a256(o + (size_t)B * s->dims[l + 1] * 2);
  }
  w.dAf = reinterpret_cast<float*>(p + o);
  o = a256(o + (size_t)B * maxd * 4);
  w.dZf = reinterpret_cast<float*>(p + o);
  o = a256(o + (size_t)B * maxd * 4);
  w.dZb = reinterpret_cast<__nv_bfloat16*>(p + o);
  o = a256(o + (size_t)B * maxd * 2);
  w.dZt = reinterpret_cast<__nv_bfloat16*>(p + o);
  o = a256(o + (size_t)B * maxd * 2);
  w.inT = reinterpret_cast<__nv_bfloat16*>(p + o);
  o = a256(o + (size_t)B * maxd * 2);
  w.Wt = reinterpret_cast<__nv_bfloat16*>(p + o);
  o = a256(o + (size_t)maxd * maxd * 2);
  w.bytes = o;
  return w;
}

}  // namespace mlpk

using namespace mlpk;

extern "C" {

size_t mlp_param_count(const mlp_shape* s) {
  if (!shape_ok(s)) return 0;
  return w_off(s, s->n_layers);
}

size_t mlp_workspace_bytes(const mlp_shape* s, int batch) {
  if (!shape_ok(s) || batch < 1) return 0;
  return carve(s, batch, nullptr).bytes;
}

int mlp_forward(const mlp_shape* s, const uint16_t* params_bf16, const uint16_t* x, int B, float* y,
                void* workspace, void* stream) {
  if (!shape_ok(s) || !params_bf16 || !x || !y || !workspace || B < 1) return MLP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = carve(s, B, workspace);
  const __nv_bfloat16* P = reinterpret_cast<const __nv_bfloat16*>(params_bf16);
  const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(x);
  for (int l = 0; l < s->n_layers; ++l) {
    const int K = s->dims[l], N = s->dims[l + 1];
    const bool last = l == s->n_layers - 1;
    Gemm g;
    g.M = B;
    g.N = N;
    g.K = K;
    g.A = in;                      // activations [B][K]
    g.sAm = K;
    g.sAk = 1;
    g.B = P + w_off(s, l);         // W_l [N][K]: B[k][n] = W[n][k]
    g.sBn = K;
    g.sBk = 1;
    g.bias = P + w_off(s, l) + (size_t)N * K;
    g.Cf = last ? y : w.Z[l];
    g.Cb = last ? nullptr : w.A[l];
    g.ldc = N;
    g.gelu = !last;
    if (gemm(g, st) != cudaSuccess) return MLP_ERR_CUDA;
    in = w.A[l];
  }
  return MLP_OK;
}

int mlp_backward(const mlp_shape* s, const uint16_t* params_bf16, const uint16_t* x, int B,
                 const float* dy, float* grads, void* workspace, void* stream) {
  if (!shape_ok(s) || !params_bf16 || !x || !dy || !grads || !workspace || B < 1) return MLP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = carve(s, B, workspace);
  const __nv_bfloat16* P = reinterpret_cast<const __nv_bfloat16*>(params_bf16);
  const int L = s->n_layers;
  // output layer: dZ = dy
  const size_t nout = (size_t)B * s->dims[L];
  to_bf16_kernel<<<grid_1d(nout), 256, 0, st>>>(dy, w.dZb, nout);
  const float* dZf = dy;
  for (int l = L - 1; l >= 0; --l) {
    const int K = s->dims[l], N = s->dims[l + 1];
    float* gW = grads + w_off(s, l);
    float* gb = gW + (size_t)N * K;
    colsum_kernel<<<(N + 31) / 32, 256, 0, st>>>(dZf, B, N, gb);
    const __nv_bfloat16* prev = l == 0 ? reinterpret_cast<const __nv_bfloat16*>(x) : w.A[l - 1];
    // dW_l[n][k] = sum_m dZ[m][n] * prev[m][k]: a contraction over the batch;
    // on the tensor-core path both operands are first transposed to K-major
    Gemm g;
    g.M = N;
    g.N = K;
    g.K = B;
    if (tc_shape(N, K, B)) {
      if (transpose(w.dZb, B, N, w.dZt, st) != cudaSuccess) return MLP_ERR_CUDA;
      if (transpose(prev, B, K, w.inT, st) != cudaSuccess) return MLP_ERR_CUDA;
      g.A = w.dZt;                 // A[n][m] = dZ^T[n][m]
      g.sAm = B;
      g.sAk = 1;
      g.B = w.inT;                 // B[m][k] = prev^T[k][m]
      g.sBn = B;
      g.sBk = 1;
    } else {
      g.A = w.dZb;                 // A[n][m] = dZ[m][n]
      g.sAm = 1;
      g.sAk = N;
      g.B = prev;                  // B[m][k] = prev[m][k]
      g.sBn = 1;
      g.sBk = K;
    }
    g.bias = nullptr;
    g.Cf = gW;
    g.Cb = nullptr;
    g.ldc = K;
    g.gelu = 0;
    if (gemm(g, st) != cudaSuccess) return MLP_ERR_CUDA;
    if (l == 0) break;
    // dA_{l-1}[m][k] = sum_n dZ[m][n] * W_l[n][k]
    Gemm h;
    h.M = B;
    h.N = K;
    h.K = N;
    h.A = w.dZb;
    h.sAm = N;
    h.sAk = 1;
    if (tc_shape(B, K, N)) {
      if (transpose(P + w_off(s, l), N, K, w.Wt, st) != cudaSuccess) return MLP_ERR_CUDA;
      h.B = w.Wt;                  // B[n][k] = W^T[k][n]
      h.sBn = N;
      h.sBk = 1;
    } else {
      h.B = P + w_off(s, l);       // B[n][k] = W[n][k]
      h.sBn = 1;
      h.sBk = K;
    }
    h.bias = nullptr;
    h.Cf = w.dAf;
    h.Cb = nullptr;
    h.ldc = K;
    h.gelu = 0;
    if (gemm(h, st) != cudaSuccess) return MLP_ERR_CUDA;
    const size_t n = (size_t)B * K;
    gelu_back_kernel<<<grid_1d(n), 256, 0, st>>>(w.dAf, w.Z[l - 1], w.dZf, w.dZb, n);
    dZf = w.dZf;
  }
  return cudaGetLastError() == cudaSuccess ? MLP_OK : MLP_ERR_CUDA;
}

int mlp_mse(const float* y, const float* t, int B, int D, int used, float* loss, float* dy,
            void* stream) {
  if (!y || !t || !loss || !dy || B < 1 || D < 1 || used < 1 || used > D) return MLP_ERR_ARG;
  mse_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(y, t, B, D, used, loss, dy);
  return cudaGetLastError() == cudaSuccess ? MLP_OK : MLP_ERR_CUDA;
}

int mlp_adamw(size_t n, float* params, uint16_t* params_bf16, const float* grads, float* m, float* v,
              float lr, float beta1, float beta2, float eps, float weight_decay, int step,
              void* stream) {
  if (!params || !params_bf16 || !grads || !m || !v || step < 1) return MLP_ERR_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  adamw_kernel<<<grid_1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, params, reinterpret_cast<__nv_bfloat16*>(params_bf16), grads, m, v, lr, beta1, beta2, eps,
      weight_decay, c1, c2);
  return cudaGetLastError() == cudaSuccess ? MLP_OK : MLP_ERR_CUDA;
}

int mlp_to_bf16(const float* src, uint16_t* dst, size_t n, void* stream) {
  if (!src || !dst) return MLP_ERR_ARG;
  to_bf16_kernel<<<grid_1d(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      src, reinterpret_cast<__nv_bfloat16*>(dst), n);
  return cudaGetLastError() == cudaSuccess ? MLP_OK : MLP_ERR_CUDA;
}

size_t mlp_packed_bytes(const mlp_shape* s) {
  mlpk::fused::Plan p;
  if (!shape_ok(s) || !mlpk::fused::plan_of(s->n_layers, s->dims, p)) return 0;
  return p.bytes;
}

int mlp_pack(const mlp_shape* s, const uint16_t* params_bf16, void* packed, void* stream) {
  mlpk::fused::Plan p;
  if (!shape_ok(s) || !params_bf16 || !packed || !mlpk::fused::plan_of(s->n_layers, s->dims, p) ||
      (reinterpret_cast<uintptr_t>(packed) & 15))
    return MLP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int l = 0; l < p.n_layers; ++l) {
    const size_t work = (size_t)mlpk::tc::kblocks_of(p.l[l].K) * p.l[l].N * 8 + p.l[l].N;
    mlpk::fused::pack_kernel<<<grid_1d(work), 256, 0, st>>>(
        reinterpret_cast<const __nv_bfloat16*>(params_bf16), w_off(s, l), p.l[l],
        static_cast<unsigned char*>(packed));
  }
  return cudaGetLastError() == cudaSuccess ? MLP_OK : MLP_ERR_CUDA;
}

int mlp_infer(const mlp_shape* s, const void* packed, const uint16_t* x, int B, float* y, void* stream) {
  mlpk::fused::Plan p;
  if (!shape_ok(s) || !packed || !x || !y || B < mlpk::tc::TM || B % mlpk::tc::TM ||
      !mlpk::fused::plan_of(s->n_layers, s->dims, p) || (reinterpret_cast<uintptr_t>(packed) & 15) ||
      (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(y) & 15))
    return MLP_ERR_ARG;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlpk::fused::infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mlpk::fused::smem_bytes()) != cudaSuccess)
      return MLP_ERR_CUDA;
    attr = true;
  }
  mlpk::fused::infer_kernel<<<B / mlpk::tc::TM, mlpk::fused::FT, mlpk::fused::smem_bytes(),
                              static_cast<cudaStream_t>(stream)>>>(
      p, static_cast<const unsigned char*>(packed), reinterpret_cast<const __nv_bfloat16*>(x), y);
  return cudaGetLastError() == cudaSuccess ? MLP_OK : MLP_ERR_CUDA;
}

int mlp_set_gemm_path(int path) {
  if (path != 0 && path != 1) return -1;
  const int old = mlpk::g_path;
  mlpk::g_path = path;
  return old;
}

int mlp_gemm_status(void) {
  if (cudaDeviceSynchronize() != cudaSuccess) return MLP_ERR_CUDA;
  unsigned int v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, mlpk::tc::g_tc_status, sizeof v) != cudaSuccess) return MLP_ERR_CUDA;
  if (v && cudaMemcpyToSymbol(mlpk::tc::g_tc_status, &zero, sizeof zero) != cudaSuccess)
    return MLP_ERR_CUDA;
  return v ? MLP_ERR_TIMEOUT : MLP_OK;
}

}  // extern "C"
