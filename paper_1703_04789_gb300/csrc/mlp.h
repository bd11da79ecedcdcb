// Learned Davidson correction: device kernels for features, training and inference.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace spmps {
namespace mlp {

constexpr int N_FEATURES = 4;
constexpr int HIDDEN = 256;
// flat FP32 parameter vector: W1 (4 x 256, row-major [feature][unit]), b1 (256),
// W2 (256 x 256, row-major [in][out]), b2 (256), w3 (256), b3 (1)
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + N_FEATURES * HIDDEN;
constexpr int kOffW2 = kOffB1 + HIDDEN;
constexpr int kOffB2 = kOffW2 + HIDDEN * HIDDEN;
constexpr int kOffW3 = kOffB2 + HIDDEN;
constexpr int kOffB3 = kOffW3 + HIDDEN;
constexpr int kParams = kOffB3 + 1;

// Work buffers of one training step for batch B (each B x HIDDEN floats unless noted).
struct TrainBuffers {
    float *Z1, *H1, *Z2, *H2, *dZ2, *dZ1;
    float* dy;          // B
    double* loss_part;  // ceil(B / 256)
};

cudaError_t features(const double* r, const double* d, const double* dh, const double* dn, const double* theta,
                     const double* rr, const double* dd, int64_t n, const int64_t* idx, int64_t count, float* X,
                     cudaStream_t st);
// d = -r / clamp(dh - theta dn) (the diagonal correction).
cudaError_t diag_correction(const double* r, const double* dh, const double* dn, const double* theta, int64_t n,
                            double* d, cudaStream_t st);
// T[j*count + s] = sqrt(n) e_j[idx[s]] / |e_j|, e_j = x* - alpha_j x_j (xs holds n_iter vectors x_j;
// xdot[j] = x_j . x*, xnorm[j] = x_j . x_j, *xx = x* . x*).
cudaError_t targets(const double* xs, const double* xstar, const double* xdot, const double* xnorm, const double* xx,
                    const int64_t* idx, int count, int n_iter, int64_t n, float* T, cudaStream_t st);
cudaError_t prepare_w2(const float* params, __nv_bfloat16* w2core, cudaStream_t st);
// out[i] = network(features of element i) with the 256 x 256 layer on tcgen05 (BF16 operands,
// FP32 accumulation); err[0] is set when the bounded wait for the MMAs gave up after wait_polls
// polls (<= 0: the default of about a second); the kernel then waits once more with the default
// limit for its MMAs in flight, frees its tensor memory and returns.
cudaError_t infer_tc(const double* r, const double* d, const double* dh, const double* dn, const double* theta,
                     const double* rr, const double* dd, int64_t n, const __nv_bfloat16* w2core, const float* params,
                     double* out, int* err, cudaStream_t st, int wait_polls = 0);
cudaError_t infer_f32(const float* X, int64_t n, const float* params, double* out, cudaStream_t st);
// Forward + backward of the mean squared error on (X, T); writes grads (kParams) and *loss.
cudaError_t train_step(TrainBuffers& b, const float* X, const float* T, int B, float* params, float* grads,
                       double* loss, cudaStream_t st);
cudaError_t adam(float* params, const float* grads, float* m, float* v, int step, float lr, cudaStream_t st);
cudaError_t gather_batch(const float* Xall, const float* Tall, int64_t total, int B, uint64_t seed, uint64_t step,
                         float* X, float* T, cudaStream_t st);

}  // namespace mlp
}  // namespace spmps
