// Launch wrappers of the SP-MPS CUDA kernels (sm_103a).  All take device task arrays built
// by the host planner and a table of slot base pointers, and launch on the given stream.
#pragma once

#include <cuda_runtime.h>

#include "core.h"

namespace spmps {

// Grouped FP64 GEMM: one warp per 16x16 output tile of the task list.
cudaError_t launch_gemm_f64(const Slots& slots, const GemmTask* tasks, const GemmSeg* segs,
                            const GemmTile* tiles, const int* cmaps, int n_tiles, cudaStream_t st);

// out[i] = sum_{g < G} partial[g * n + i] (fixed order).
cudaError_t launch_sum_partials(const double* partial, int G, int64_t n, double* out, cudaStream_t st);

// Same task lists on the tensor cores (m16n8k8 TF32, FP32 accumulation, FP64 in and out);
// split3 != 0 uses the 3xTF32 split (hi*hi + hi*lo + lo*hi).
cudaError_t launch_gemm_tf32(const Slots& slots, const GemmTask* tasks, const GemmSeg* segs, const GemmTile* tiles,
                             const int* cmaps, int n_tiles, int split3, cudaStream_t st);

// Operand buffers in pre-split TF32 form (float2 = (hi, lo) per element), indexed by the same slot
// handles as the FP64 buffers.
struct SlotsF {
    float2* p[kMaxSlots];
};
// out[i] = (tf32(float(x[i])), tf32(float(x[i]) - hi)).
cudaError_t launch_split_tf32(const double* x, int64_t n, float2* out, cudaStream_t st);
// The TF32 / 3xTF32 task lists with every A and B operand read from the pre-split buffers of the
// same slots (no conversion in the GEMM); C written in FP64 as launch_gemm_tf32.
cudaError_t launch_gemm_tf32s(const Slots& slots, const SlotsF& split, const GemmTask* tasks, const GemmSeg* segs,
                              const GemmTile* tiles, const int* cmaps, int n_tiles, int split3, cudaStream_t st);

// Linear combination of equally shaped blocks (the MPO-leg contraction).
cudaError_t launch_comb_f64(const Slots& slots, const CombOut* outs, const CombTerm* terms, int n_outs,
                            cudaStream_t st);

// Diagonal of the projected H and N operators on the two-site row-block layout.
cudaError_t launch_diag_f64(const Slots& slots, const DiagBlock* blocks, const DiagTerm* terms, int n_blocks,
                            double* dh, double* dn, cudaStream_t st);

// ---- dense vector kernels for the Davidson solver (length n, column-major bases) ----------

// out[j] = sum_i V[j*ldv + i] * x[i] for j < m (plus a scale); multi-dot with block reduction.
// `partial` is a per-caller scratch of kPartialDoubles doubles.
constexpr int kPartialDoubles = 64 * 32;
cudaError_t launch_multidot(const double* V, int64_t ldv, int m, const double* x, int64_t n, double* out,
                            double* partial, cudaStream_t st);
// y[i] = sum_j V[j*ldv + i] * c[j]  (c on the device), optionally y -= (when sub != 0).
cudaError_t launch_gemv(const double* V, int64_t ldv, int m, const double* c, int64_t n, double* y, int sub,
                        cudaStream_t st);
// dst[:, j] = sum_i src[:, i] * Q[i + j*ldq]  for j < k (dst and src must differ).
cudaError_t launch_basis_rotate(const double* src, int64_t ld, int m, const double* Q, int ldq, int k,
                                int64_t n, double* dst, cudaStream_t st);

// Incremental Ritz step of the Davidson solver (one CTA of 128 threads) on the stored subspace
// matrices h, n (m x m, leading dim ldm, upper triangles column by column): lowest Ritz pair in the
// range of n kept above eps_metric * max diag(n).  The state is kept across the iterations of one
// solve; reset != 0 rebuilds it from the m stored columns.  Writes coef[0..m) and scal[0] = theta,
// scal[1] = number of kept metric directions (0 = singular).
struct RitzState {
    static constexpr int kR = 32;
    double X[kR * kR];   // n-orthonormal coefficient basis, X[i + j*kR]
    double hp[kR * kR];  // X^T h X
    double C[kR * kR];   // eigenvectors of hp (columns)
    int k, m, kc, pad;
};
cudaError_t launch_ritz_inc(const double* h, const double* nmat, int ldm, int m, int reset, double eps_metric,
                            RitzState* state, double* coef, double* scal, cudaStream_t st);

// r = hx - theta * nx, t = preconditioned correction, scal[2] = ||r||^2.
cudaError_t launch_residual_diag(const double* hx, const double* nx, const double* dh, const double* dn,
                                 const double* scal, double clamp, int64_t n, double* r, double* t,
                                 double* red, double* partial, cudaStream_t st);
// sum of squares into *out (two-pass deterministic reduction).
cudaError_t launch_norm2(const double* x, int64_t n, double* out, double* partial, cudaStream_t st);
// x *= 1/sqrt(*nrm2) (device scalar)
cudaError_t launch_scale_inv_sqrt(double* x, int64_t n, const double* nrm2, cudaStream_t st);
// x += alpha * y, alpha = sign * num / den from device scalars (for CG)
// out = v / (diag H - theta diag N) (denominator clamped to |.| >= clamp; theta = scal[0])
cudaError_t launch_precond_apply(const double* v, const double* dh, const double* dn, const double* scal,
                                 double clamp, int64_t n, double* out, cudaStream_t st);
cudaError_t launch_axpy_ratio(double* x, const double* y, int64_t n, const double* num, const double* den,
                              double sign, cudaStream_t st);
// p = r + (num/den) p
cudaError_t launch_xpby_ratio(double* p, const double* r, int64_t n, const double* num, const double* den,
                              cudaStream_t st);
// Two-vector orthonormal restart coefficients in the current basis: Qout (m x 2) from the
// Ritz coefficients c_new and c_old (m each); returns the count in scal_out[0].
cudaError_t launch_restart_coef(const double* c_new, const double* c_old, int m, double* Qout, double* scal_out,
                                cudaStream_t st);

// ---- decimation -------------------------------------------------------------------------------

// Symmetric eigen-decomposition of many small matrices by cyclic Jacobi, one CTA each.
// mats: concatenated row-major n_i x n_i matrices (overwritten by the eigenvector matrices,
// columns = vectors, sorted by descending eigenvalue), evals: concatenated eigenvalues.
// vscratch: same size as mats (used for matrices above the shared-memory limit of 112).
// Matrices up to min(smem_limit, 112) run in shared memory.  With cluster != 0, matrices of
// dimension 65..256 run on a thread-block cluster of 8 CTAs each (rows distributed over the
// CTAs' shared memory), the others on one CTA.
cudaError_t launch_jacobi_batched(double* mats, double* vscratch, double* evals, const int64_t* mat_off,
                                  const int64_t* val_off, const int* dims, int n_mats, int max_dim, int smem_limit,
                                  int cluster, int* status, cudaStream_t st);

// Ordered truncation of singular values sqrt(max(evals, 0)) (one CTA): values within
// tie_rtol * max of their sorted predecessor form a cluster ordered by (n, 2m, index);
// values below drop_abs are dropped; the first D kept.  keep_count[label] receives the
// number kept per label (labels in bond order), keep_total[0] the total and discarded[0] the
// discarded weight.
cudaError_t launch_truncate(const double* evals, const int64_t* val_off, const int* dims, const int* label_n,
                            const int* label_tm, int n_labels, int total, int D, double tie_rtol, double drop_abs,
                            int* keep_count, int* keep_total, double* discarded, int* scratch_idx,
                            double* scratch_val, cudaStream_t st);

// Gather/scatter of sub-blocks: dst[(r)*ld_dst + c] = src[(r)*ld_src + c] * scale for a list.
struct CopyBlock {
    uint64_t src, dst;
    int rows, cols, ld_src, ld_dst;
    int transpose;  // 1: dst(r, c) = src(c, r)
    int pad;
};
cudaError_t launch_copy_blocks(const Slots& slots, const CopyBlock* blocks, int n, cudaStream_t st);

// FP64 FMA throughput of the current device (TFLOP/s), from a kernel of independent chains.
cudaError_t measure_fp64_peak(double* tflops);

}  // namespace spmps
