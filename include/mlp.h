/*
 * mlp.h -- C ABI of the surrogate's kernels in libnoc.so: a small multilayer
 * perceptron (BF16 weights and activations, FP32 accumulation on the tensor
 * cores) trained with AdamW on design point -> simulator outputs pairs.
 *
 * The paper has no surrogate; this serves the design-space screening of the
 * simulator: the network predicts (log mean L2 access latency, deflections per
 * flit, accepted flits per node per cycle) for a design point (Sec. 3 cache
 * policies and load, Sec. 6.2.3 traffic mix), and the exact simulator checks it.
 *
 * Layout: layer l (0-based) maps dims[l] -> dims[l+1] features; weights W_l are
 * row-major [dims[l+1]][dims[l]] followed by the bias b_l [dims[l+1]], layer
 * after layer, in one flat FP32 parameter buffer (mlp_param_count floats) with
 * a BF16 copy of the same layout used by the GEMMs.  Hidden layers apply GELU
 * (the exact erf form); the last layer is linear.  Every pointer argument is
 * DEVICE memory owned by the caller; every call enqueues on `stream` (NULL =
 * default) and returns MLP_OK or MLP_ERR_* without synchronising.  Feature
 * dimensions must be multiples of 8 (pad inputs and outputs with zeros).
 */
#ifndef MLP_H
#define MLP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLP_OK 0
#define MLP_ERR_ARG 1
#define MLP_ERR_TIMEOUT 4
#define MLP_ERR_CUDA 5
#define MLP_MAX_LAYERS 8

typedef struct {
  int32_t n_layers;                 /* 1..MLP_MAX_LAYERS */
  int32_t dims[MLP_MAX_LAYERS + 1]; /* dims[0] inputs ... dims[n_layers] outputs */
} mlp_shape;

/* FP32 parameters (weights and biases) of the shape. */
size_t mlp_param_count(const mlp_shape* shape);
/* Device bytes of the activation workspace for `batch` rows (forward stores
 * what the backward pass reads: pre-activations and activations per layer). */
size_t mlp_workspace_bytes(const mlp_shape* shape, int batch);

/* y[batch][dims[L]] (FP32) = network(x), x BF16 [batch][dims[0]]. */
int mlp_forward(const mlp_shape* shape, const uint16_t* params_bf16, const uint16_t* x, int batch,
                float* y, void* workspace, void* stream);
/* Gradients (FP32, parameter layout) of sum(dy * y) w.r.t. the parameters,
 * for the x of the preceding mlp_forward with the same workspace. */
int mlp_backward(const mlp_shape* shape, const uint16_t* params_bf16, const uint16_t* x, int batch,
                 const float* dy, float* grads, void* workspace, void* stream);
/* Mean squared error over the first `used` of `dim` output columns:
 * *loss = mean (y - t)^2, dy = d loss / d y (0 in padding columns). */
int mlp_mse(const float* y, const float* t, int batch, int dim, int used, float* loss, float* dy,
            void* stream);
/* One AdamW step (decoupled weight decay) on n FP32 parameters; refreshes the
 * BF16 copy.  step counts from 1. */
int mlp_adamw(size_t n, float* params, uint16_t* params_bf16, const float* grads, float* m, float* v,
              float lr, float beta1, float beta2, float eps, float weight_decay, int step,
              void* stream);
/* FP32 -> BF16 (round to nearest even). */
int mlp_to_bf16(const float* src, uint16_t* dst, size_t n, void* stream);

/* Whole-network inference in one kernel (the network's weights packed once
 * into the tensor cores' shared-memory operand layout; activations never leave
 * the SM).  For shapes whose every width is a multiple of 16 in 16..256.
 * mlp_packed_bytes: device bytes of the packed image (0: shape not taken).
 * mlp_pack: write the image from the BF16 parameters (again after every
 * parameter update).  mlp_infer: y[batch][dims[L]] (FP32) = network(x), x
 * BF16 [batch][dims[0]], batch a positive multiple of 128; packed, x and y
 * 16-byte aligned; results equal mlp_forward's on the tensor-core path.
 * MLP_ERR_ARG for a shape, batch or alignment it does not take. */
size_t mlp_packed_bytes(const mlp_shape* shape);
int mlp_pack(const mlp_shape* shape, const uint16_t* params_bf16, void* packed, void* stream);
int mlp_infer(const mlp_shape* shape, const void* packed, const uint16_t* x, int batch, float* y,
              void* stream);

/* GEMM engine of the layers.  path 0 (default): the 5th-generation tensor
 * cores (tcgen05.mma, FP32 accumulator in tensor memory) for every GEMM whose
 * rows are a multiple of 128, output width up to 256 and inner dimension at
 * least 16, both multiples of 16 -- every forward layer at batches that are
 * multiples of 128, and in the backward pass the input gradients (batches
 * that are multiples of 128) and the weight gradients of layers whose output
 * width is a multiple of 128 (batches that are multiples of 16), on K-major
 * transposes the library makes; warp-level mma.sync for the others; path 1:
 * mma.sync for all.
 * mlp_infer is not affected.
 * Returns the previous path, or -1 for an invalid one. */
int mlp_set_gemm_path(int path);
/* Waits for the device; MLP_ERR_TIMEOUT if a tcgen05 GEMM since the last call
 * gave up waiting for its MMAs (its output is then incomplete), else MLP_OK. */
int mlp_gemm_status(void);

#ifdef __cplusplus
}
#endif
#endif
