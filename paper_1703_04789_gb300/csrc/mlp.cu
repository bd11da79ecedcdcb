// Learned correction for the generalised Davidson solver (the paper has no counterpart).
//
// A 3-layer perceptron 4 -> 256 -> 256 -> 1 (ReLU) maps per-element features of the residual
// (normalised residual, normalised diagonal correction, diag N_eff, tanh of the shifted diagonal)
// to a correction.  Pairs (features, error direction) are harvested from plain Davidson solves;
// training runs on the device in FP32 (tiled SIMT GEMMs, backward pass, Adam); inference runs
// the 256 x 256 layer on the 5th-generation tensor cores: BF16 operands in shared memory in the
// no-swizzle K-major core-matrix layout, tcgen05.mma with M = 128, N = 256, K = 16 (16
// instructions), FP32 accumulators in tensor memory, and an epilogue (tcgen05.ld) that fuses the
// bias, the ReLU and the final 256 -> 1 dot product.
#include <cuda_bf16.h>

#include <cmath>

#include "mlp.h"

namespace spmps {
namespace mlp {

namespace {

int grid1(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return static_cast<int>(g);
}

// ---- features ---------------------------------------------------------------------------------
// X[s*4 + f] for element i = idx ? idx[s] : s.  nrm[0] = |r|^2, nrm[1] = |d|^2 (device).
__global__ void k_features(const double* __restrict__ r, const double* __restrict__ d, const double* __restrict__ dh,
                           const double* __restrict__ dn, const double* __restrict__ theta_p,
                           const double* __restrict__ rr, const double* __restrict__ dd, int64_t n,
                           const int64_t* __restrict__ idx, int64_t count, float* __restrict__ X) {
    const double theta = *theta_p;
    const double s = sqrt(static_cast<double>(n));
    const double rn = sqrt(*rr), dnm = sqrt(*dd);
    const double fr = rn > 0.0 ? s / rn : 0.0, fd = dnm > 0.0 ? s / dnm : 0.0;
    const double sc = 1.0 / (1.0 + fabs(theta));
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < count;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = idx ? idx[q] : q;
        X[q * 4 + 0] = static_cast<float>(fr * r[i]);
        X[q * 4 + 1] = static_cast<float>(fd * d[i]);
        X[q * 4 + 2] = static_cast<float>(dn[i]);
        X[q * 4 + 3] = static_cast<float>(tanh((dh[i] - theta * dn[i]) * sc));
    }
}

// d = -r / (dh - theta dn), the denominator clamped to |.| >= 1e-4 (the diagonal correction)
__global__ void k_diag_correction(const double* __restrict__ r, const double* __restrict__ dh,
                                  const double* __restrict__ dn, const double* __restrict__ theta_p, int64_t n,
                                  double* __restrict__ d) {
    const double theta = *theta_p;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double den = dh[i] - theta * dn[i];
        if (fabs(den) < 1e-4) den = den < 0.0 ? -1e-4 : 1e-4;
        d[i] = -r[i] / den;
    }
}

// ---- FP32 SIMT GEMM: C = op(A) op(B) (+ bias[col]) ---------------------------------------------
// A(i, k) = TA ? A[k*lda + i] : A[i*lda + k];  B(k, j) = TB ? B[j*ldb + k] : B[k*ldb + j].
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                               const float* __restrict__ bias) {
    __shared__ float As[16][64 + 1], Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, ii = e % 64;
            const int gi = m0 + ii, gk = k0 + kk, gj = n0 + ii;
            As[kk][ii] = (gi < M && gk < K) ? (TA ? A[static_cast<int64_t>(gk) * lda + gi] : A[static_cast<int64_t>(gi) * lda + gk]) : 0.0f;
            Bs[kk][ii] = (gj < N && gk < K) ? (TB ? B[static_cast<int64_t>(gj) * ldb + gk] : B[static_cast<int64_t>(gk) * ldb + gj]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[kk][ty + 16 * q];
                b[q] = Bs[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = m0 + ty + 16 * p, j = n0 + tx + 16 * q;
            if (i < M && j < N) C[static_cast<int64_t>(i) * ldc + j] = acc[p][q] + (bias ? bias[j] : 0.0f);
        }
}

template <bool TA, bool TB>
void sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, const float* bias,
           cudaStream_t st) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_sgemm<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias);
}

__global__ void k_relu(const float* __restrict__ z, float* __restrict__ h, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        h[i] = fmaxf(z[i], 0.0f);
}

// y[b] = H2[b, :] . w3 + b3;  dy = 2 (y - t) / B;  loss partial sums (one per block)
__global__ void __launch_bounds__(256) k_head(const float* __restrict__ H2, const float* __restrict__ w3,
                                              const float* __restrict__ b3, const float* __restrict__ t, int B,
                                              float* __restrict__ dy, double* __restrict__ loss_part) {
    __shared__ double sh[256];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        float y = b3[0];
        for (int j = 0; j < HIDDEN; ++j) y = fmaf(H2[static_cast<int64_t>(b) * HIDDEN + j], w3[j], y);
        const float diff = y - t[b];
        dy[b] = 2.0f * diff / static_cast<float>(B);
        l = static_cast<double>(diff) * diff;
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0];
}

// dZ2[b, j] = dy[b] * w3[j] * (Z2[b, j] > 0)
__global__ void k_back_head(const float* __restrict__ dy, const float* __restrict__ w3, const float* __restrict__ Z2,
                            float* __restrict__ dZ2, int B) {
    const int64_t n = static_cast<int64_t>(B) * HIDDEN;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = e / HIDDEN;
        const int j = static_cast<int>(e % HIDDEN);
        dZ2[e] = Z2[e] > 0.0f ? dy[b] * w3[j] : 0.0f;
    }
}

__global__ void k_mask(float* __restrict__ d, const float* __restrict__ z, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        if (!(z[i] > 0.0f)) d[i] = 0.0f;
}

// out[j] = sum_b M[b, j]  (column sums, fixed order), out[j] for j < cols
__global__ void k_colsum(const float* __restrict__ Mx, int rows, int cols, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double acc = 0.0;
    for (int b = 0; b < rows; ++b) acc += Mx[static_cast<int64_t>(b) * cols + j];
    out[j] = static_cast<float>(acc);
}

__global__ void k_sum_loss(const double* __restrict__ part, int nb, int B, const float* __restrict__ dy,
                           double* __restrict__ loss, float* __restrict__ gb3) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = 0.0, g = 0.0;
    for (int i = 0; i < nb; ++i) acc += part[i];
    for (int b = 0; b < B; ++b) g += dy[b];
    *loss = acc / B;
    *gb3 = static_cast<float>(g);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float mi = b1 * m[i] + (1.0f - b1) * g[i];
        const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Minibatch gather: rows (hash of step, position) of the harvested set.
__global__ void k_gather_batch(const float* __restrict__ Xall, const float* __restrict__ Tall, int64_t total, int B,
                               uint64_t seed, uint64_t step, float* __restrict__ X, float* __restrict__ T) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    // SplitMix64 of (seed, step, b): a fixed, published mixing function
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (step * 1048576ull + static_cast<uint64_t>(b) + 1ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int64_t i = static_cast<int64_t>(z % static_cast<uint64_t>(total));
    for (int f = 0; f < N_FEATURES; ++f) X[b * N_FEATURES + f] = Xall[i * N_FEATURES + f];
    T[b] = Tall[i];
}

// ---- harvesting: targets from the converged vector -------------------------------------------
// For stored iteration j: e = x* - alpha_j x_j with alpha_j = (x_j . x*) / (x_j . x_j);
// target at sample s = sqrt(n) e[i_s] / |e|, |e|^2 = x*.x* - 2 alpha (x_j . x*) + alpha^2 x_j.x_j.
__global__ void k_targets(const double* __restrict__ xs, const double* __restrict__ xstar,
                          const double* __restrict__ xdot, const double* __restrict__ xnorm,
                          const double* __restrict__ xx_p, const int64_t* __restrict__ idx, int count, int n_iter,
                          int64_t n, float* __restrict__ T) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count * n_iter) return;
    const int j = q / count, s = q - j * count;
    const double xs_xs = xnorm[j], xj_x = xdot[j], xx = *xx_p;
    const double alpha = xs_xs > 0.0 ? xj_x / xs_xs : 0.0;
    const double e2 = fmax(xx - 2.0 * alpha * xj_x + alpha * alpha * xs_xs, 0.0);
    const int64_t i = idx[s];
    const double e = xstar[i] - alpha * xs[static_cast<int64_t>(j) * n + i];
    T[q] = e2 > 0.0 ? static_cast<float>(sqrt(static_cast<double>(n)) * e / sqrt(e2)) : 0.0f;
}

// ---- BF16 tensor-core inference (tcgen05) -----------------------------------------------------
constexpr int kTileM = 128;
constexpr uint32_t kTmemCols = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// No-swizzle K-major matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets of the 8 x 16-byte core matrices, descriptor version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFF) >> 4);
    d |= static_cast<uint64_t>((lbo & 0x3FFFF) >> 4) << 16;
    d |= static_cast<uint64_t>((sbo & 0x3FFFF) >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;  // version
    return d;                             // base offset 0, lbo mode 0, layout SWIZZLE_NONE (0)
}

// Byte offset of element (row, k) of a rows x 256 K-major BF16 operand in the core layout:
// core (row/8, k/8) at ((row/8) * 32 + k/8) * 128, rows 16 bytes apart, k elements 2 bytes apart.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return (static_cast<uint32_t>((row >> 3) * 32 + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__global__ void k_w2_core(const float* __restrict__ W2, __nv_bfloat16* __restrict__ out) {
    // out holds B(k, n) = W2[k][n] K-major: element (n, k) at core_off(n, k)
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= HIDDEN * HIDDEN) return;
    const int k = e / HIDDEN, n = e % HIDDEN;
    reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(out) + core_off(n, k))[0] =
        __float2bfloat16_rn(W2[e]);
}

constexpr int kWaitPolls = 1 << 24;  // default limit of the bounded mbarrier waits (about a second)
constexpr size_t kInferSmem = static_cast<size_t>(kTileM) * HIDDEN * 2 + static_cast<size_t>(HIDDEN) * HIDDEN * 2 +
                              (N_FEATURES * HIDDEN + 3 * HIDDEN + 4) * sizeof(float) + 64;

__global__ void __launch_bounds__(128, 1) k_infer_tc(const double* __restrict__ r, const double* __restrict__ d,
                                                     const double* __restrict__ dh, const double* __restrict__ dn,
                                                     const double* __restrict__ theta_p, const double* __restrict__ rr,
                                                     const double* __restrict__ dd, int64_t n,
                                                     const __nv_bfloat16* __restrict__ w2core,
                                                     const float* __restrict__ params, double* __restrict__ out,
                                                     int* __restrict__ err, int wait_polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* As = smem;                                     // 128 x 256 bf16, 64 KB
    unsigned char* Bs = smem + kTileM * HIDDEN * 2;               // 256 x 256 bf16, 128 KB
    float* W1s = reinterpret_cast<float*>(Bs + HIDDEN * HIDDEN * 2);
    float* b1s = W1s + N_FEATURES * HIDDEN;
    float* b2s = b1s + HIDDEN;
    float* w3s = b2s + HIDDEN;
    float* b3s = w3s + HIDDEN;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b3s + 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    volatile uint32_t* wait_ok = tslot + 1;  // outcome of thread 0's bounded wait, read by every thread
    const int tid = threadIdx.x, warp = tid >> 5;
    // weights into shared memory
    {
        const uint4* src = reinterpret_cast<const uint4*>(w2core);
        uint4* dst = reinterpret_cast<uint4*>(Bs);
        for (int e = tid; e < HIDDEN * HIDDEN * 2 / 16; e += blockDim.x) dst[e] = src[e];
        for (int e = tid; e < N_FEATURES * HIDDEN; e += blockDim.x) W1s[e] = params[kOffW1 + e];
        for (int e = tid; e < HIDDEN; e += blockDim.x) {
            b1s[e] = params[kOffB1 + e];
            b2s[e] = params[kOffB2 + e];
            w3s[e] = params[kOffW3 + e];
        }
        if (tid == 0) b3s[0] = params[kOffB3];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const double theta = *theta_p;
    const double sq = sqrt(static_cast<double>(n));
    const double rn = sqrt(*rr), dnm = sqrt(*dd);
    const double fr = rn > 0.0 ? sq / rn : 0.0, fd = dnm > 0.0 ? sq / dnm : 0.0;
    const double sc = 1.0 / (1.0 + fabs(theta));
    // instruction descriptor: F32 accumulate, BF16 A and B, both K-major, N = 256, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((HIDDEN >> 3) << 17) | ((kTileM >> 4) << 24);
    uint32_t phase = 0;
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile * kTileM < n && !failed; tile += gridDim.x) {
        const int64_t row = tile * kTileM + tid;
        const bool valid = row < n;
        float f[N_FEATURES] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (valid) {
            f[0] = static_cast<float>(fr * r[row]);
            f[1] = static_cast<float>(fd * d[row]);
            f[2] = static_cast<float>(dn[row]);
            f[3] = static_cast<float>(tanh((dh[row] - theta * dn[row]) * sc));
        }
        // layer 1 on the CUDA cores into the A tile (row = tid), 8 bf16 (16 bytes) at a time
        for (int jb = 0; jb < HIDDEN / 8; ++jb) {
            __align__(16) __nv_bfloat16 hv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = jb * 8 + q;
                float z = b1s[j];
#pragma unroll
                for (int c = 0; c < N_FEATURES; ++c) z = fmaf(f[c], W1s[c * HIDDEN + j], z);
                hv[q] = __float2bfloat16_rn(fmaxf(z, 0.0f));
            }
            *reinterpret_cast<uint4*>(As + core_off(tid, jb * 8)) = *reinterpret_cast<const uint4*>(hv);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int kk = 0; kk < HIDDEN / 16; ++kk) {
                const uint64_t da = make_desc(a0 + kk * 256, 128, 32 * 128);
                const uint64_t db = make_desc(b0 + kk * 256, 128, 32 * 128);
                const uint32_t acc = kk > 0 ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar)));
        }
        // bounded wait for the MMAs by thread 0; the outcome goes to every thread through shared
        // memory, so the whole CTA takes the same path (the epilogue's loads are warp-collective)
        if (tid == 0) {
            uint32_t done = 0;
            for (int it = 0; it < wait_polls && !done; ++it) {
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(smem_u32(mbar)), "r"(phase));
            }
            *wait_ok = done;
        }
        __syncthreads();
        if (!*wait_ok) {
            failed = true;
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: thread tid owns TMEM lane tid (warp w: lanes 32w..32w+31)
        float y = b3s[0];
        for (int c = 0; c < HIDDEN / 32; ++c) {
            uint32_t v[32];
            const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int j = c * 32 + q;
                const float z = __uint_as_float(v[q]) + b2s[j];
                y = fmaf(fmaxf(z, 0.0f), w3s[j], y);
            }
        }
        if (valid) out[row] = static_cast<double>(y);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (failed && tid == 0) {
        // give the in-flight MMAs a further bounded wait (the default limit) before the tensor
        // memory is released
        uint32_t done = 0;
        for (int it = 0; it < kWaitPolls && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(mbar)), "r"(phase));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// FP32 SIMT inference (same network, float weights): reference path for tests and small n.
__global__ void __launch_bounds__(256) k_infer_f32(const float* __restrict__ X, int64_t n, const float* __restrict__ p,
                                                  double* __restrict__ out) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float h1[HIDDEN];
        for (int j = 0; j < HIDDEN; ++j) {
            float z = p[kOffB1 + j];
            for (int c = 0; c < N_FEATURES; ++c) z = fmaf(X[i * N_FEATURES + c], p[kOffW1 + c * HIDDEN + j], z);
            h1[j] = fmaxf(z, 0.0f);
        }
        float y = p[kOffB3];
        for (int j = 0; j < HIDDEN; ++j) {
            float z = p[kOffB2 + j];
            for (int l = 0; l < HIDDEN; ++l) z = fmaf(h1[l], p[kOffW2 + l * HIDDEN + j], z);
            y = fmaf(fmaxf(z, 0.0f), p[kOffW3 + j], y);
        }
        out[i] = y;
    }
}

}  // namespace

// ---- host API -------------------------------------------------------------------------------------

cudaError_t features(const double* r, const double* d, const double* dh, const double* dn, const double* theta,
                     const double* rr, const double* dd, int64_t n, const int64_t* idx, int64_t count, float* X,
                     cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_features<<<grid1(count, 256, 4096), 256, 0, st>>>(r, d, dh, dn, theta, rr, dd, n, idx, count, X);
    return cudaGetLastError();
}

cudaError_t diag_correction(const double* r, const double* dh, const double* dn, const double* theta, int64_t n,
                            double* d, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_diag_correction<<<grid1(n, 256, 4096), 256, 0, st>>>(r, dh, dn, theta, n, d);
    return cudaGetLastError();
}

cudaError_t targets(const double* xs, const double* xstar, const double* xdot, const double* xnorm, const double* xx,
                    const int64_t* idx, int count, int n_iter, int64_t n, float* T, cudaStream_t st) {
    const int tot = count * n_iter;
    if (tot <= 0) return cudaSuccess;
    k_targets<<<(tot + 255) / 256, 256, 0, st>>>(xs, xstar, xdot, xnorm, xx, idx, count, n_iter, n, T);
    return cudaGetLastError();
}

cudaError_t prepare_w2(const float* params, __nv_bfloat16* w2core, cudaStream_t st) {
    k_w2_core<<<(HIDDEN * HIDDEN + 255) / 256, 256, 0, st>>>(params + kOffW2, w2core);
    return cudaGetLastError();
}

cudaError_t infer_tc(const double* r, const double* d, const double* dh, const double* dn, const double* theta,
                     const double* rr, const double* dd, int64_t n, const __nv_bfloat16* w2core, const float* params,
                     double* out, int* err, cudaStream_t st, int wait_polls) {
    if (n <= 0) return cudaSuccess;
    if (wait_polls <= 0) wait_polls = kWaitPolls;
    static int attr_device = -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (attr_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kInferSmem));
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + kTileM - 1) / kTileM;
    const int grid = static_cast<int>(tiles < sms ? tiles : sms);
    k_infer_tc<<<grid, 128, kInferSmem, st>>>(r, d, dh, dn, theta, rr, dd, n, w2core, params, out, err, wait_polls);
    return cudaGetLastError();
}

cudaError_t infer_f32(const float* X, int64_t n, const float* params, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_infer_f32<<<grid1(n, 256, 2048), 256, 0, st>>>(X, n, params, out);
    return cudaGetLastError();
}

cudaError_t train_step(TrainBuffers& b, const float* X, const float* T, int B, float* params, float* grads,
                       double* loss, cudaStream_t st) {
    const int H = HIDDEN;
    // forward
    sgemm<false, false>(B, H, N_FEATURES, X, N_FEATURES, params + kOffW1, H, b.Z1, H, params + kOffB1, st);
    k_relu<<<grid1(static_cast<int64_t>(B) * H, 256, 4096), 256, 0, st>>>(b.Z1, b.H1, static_cast<int64_t>(B) * H);
    sgemm<false, false>(B, H, H, b.H1, H, params + kOffW2, H, b.Z2, H, params + kOffB2, st);
    k_relu<<<grid1(static_cast<int64_t>(B) * H, 256, 4096), 256, 0, st>>>(b.Z2, b.H2, static_cast<int64_t>(B) * H);
    const int nb = (B + 255) / 256;
    k_head<<<nb, 256, 0, st>>>(b.H2, params + kOffW3, params + kOffB3, T, B, b.dy, b.loss_part);
    k_sum_loss<<<1, 32, 0, st>>>(b.loss_part, nb, B, b.dy, loss, grads + kOffB3);
    // backward
    sgemm<true, false>(H, 1, B, b.H2, H, b.dy, 1, grads + kOffW3, 1, nullptr, st);  // gw3 = H2^T dy
    k_back_head<<<grid1(static_cast<int64_t>(B) * H, 256, 4096), 256, 0, st>>>(b.dy, params + kOffW3, b.Z2, b.dZ2, B);
    sgemm<true, false>(H, H, B, b.H1, H, b.dZ2, H, grads + kOffW2, H, nullptr, st);      // gW2 = H1^T dZ2
    k_colsum<<<(H + 255) / 256, 256, 0, st>>>(b.dZ2, B, H, grads + kOffB2);
    sgemm<false, true>(B, H, H, b.dZ2, H, params + kOffW2, H, b.dZ1, H, nullptr, st);     // dH1 = dZ2 W2^T
    k_mask<<<grid1(static_cast<int64_t>(B) * H, 256, 4096), 256, 0, st>>>(b.dZ1, b.Z1, static_cast<int64_t>(B) * H);
    sgemm<true, false>(N_FEATURES, H, B, X, N_FEATURES, b.dZ1, H, grads + kOffW1, H, nullptr, st);  // gW1 = X^T dZ1
    k_colsum<<<(H + 255) / 256, 256, 0, st>>>(b.dZ1, B, H, grads + kOffB1);
    return cudaGetLastError();
}

cudaError_t adam(float* params, const float* grads, float* m, float* v, int step, float lr, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, static_cast<float>(step)), c2 = 1.0f - powf(b2, static_cast<float>(step));
    k_adam<<<grid1(kParams, 256, 1024), 256, 0, st>>>(params, grads, m, v, kParams, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t gather_batch(const float* Xall, const float* Tall, int64_t total, int B, uint64_t seed, uint64_t step,
                         float* X, float* T, cudaStream_t st) {
    k_gather_batch<<<(B + 255) / 256, 256, 0, st>>>(Xall, Tall, total, B, seed, step, X, T);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace spmps
