// CUDA kernels of the SP-MPS library (sm_103a, FP64).
//
// The contractions of the projected action and of the environment updates are lists of small
// dense block products produced by the host planner (Abelian (N, M) blocks on the bra side,
// N-only blocks on the rotated ket side).  They run as grouped launches: one warp per output
// tile of any task, every task of every beta point in the same launch.
#include <cfloat>
#include <cmath>
#include <cooperative_groups.h>

#include "kernels.h"

namespace spmps {

namespace {

__device__ __forceinline__ double* resolve(const Slots& S, uint64_t h) {
    return S.p[h >> 56] + static_cast<int64_t>(h & 0x00FFFFFFFFFFFFFFull);
}

// ---- grouped FP64 GEMM ----------------------------------------------------------------------
// Tile shapes (rows x cols per warp; each lane owns RM x CN outputs on a LR x LC lane grid):
//   0: 16 x 16  (LR 8, LC 4, RM 2, CN 4)      1: 4 x 64  (LR 4, LC 8, RM 1, CN 8)
//   2: 64 x 4   (LR 8, LC 4, RM 8, CN 1)      3: 32 x 8  (LR 8, LC 4, RM 4, CN 2)
//   4: 8 x 32   (LR 4, LC 8, RM 2, CN 4)
template <int LR, int LC, int RM, int CN>
__device__ __forceinline__ void gemm_tile(const Slots& S, const GemmTask& T, const GemmSeg* __restrict__ segs,
                                          const int* __restrict__ cmaps, int m0, int n0, int lane) {
    const int lr = lane / LC, lc = lane % LC;
    int rows[RM], cols[CN];
    bool rv[RM], cv[CN];
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        rows[i] = m0 + lr + i * LR;
        rv[i] = rows[i] < T.M;
    }
#pragma unroll
    for (int j = 0; j < CN; ++j) {
        cols[j] = n0 + lc + j * LC;
        cv[j] = cols[j] < T.N;
    }
    double acc[RM][CN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < CN; ++j) acc[i][j] = 0.0;

    for (int sgi = 0; sgi < T.nseg; ++sgi) {
        const GemmSeg sg = segs[T.seg0 + sgi];
        const double* __restrict__ A = resolve(S, sg.a);
        const double* __restrict__ B = resolve(S, sg.b);
        for (int k = 0; k < sg.K; ++k) {
            double a[RM], b[CN];
#pragma unroll
            for (int i = 0; i < RM; ++i)
                a[i] = rv[i] ? __ldg(A + static_cast<int64_t>(rows[i]) * sg.a_rs + static_cast<int64_t>(k) * sg.a_cs)
                             : 0.0;
#pragma unroll
            for (int j = 0; j < CN; ++j)
                b[j] = cv[j] ? __ldg(B + static_cast<int64_t>(k) * sg.b_rs + static_cast<int64_t>(cols[j]) * sg.b_cs)
                             : 0.0;
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < CN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    double* C = resolve(S, T.c);
    const int* cm = T.cmap >= 0 ? cmaps + T.cmap : nullptr;
#pragma unroll
    for (int j = 0; j < CN; ++j) {
        if (!cv[j]) continue;
        const int64_t cc = cm ? cm[cols[j]] : cols[j];
#pragma unroll
        for (int i = 0; i < RM; ++i)
            if (rv[i]) C[static_cast<int64_t>(rows[i]) * T.ldc + cc] = acc[i][j];
    }
}

// Warp-block tile (shape 5): one warp computes a whole tm x tn output block (tm, tn <= 32,
// tm * tn <= 256) of a task with a long reduction.  K is staged in chunks of 16 through the
// warp's shared-memory slice with coalesced loads (two rows of 16 k per warp load), then every lane accumulates
// its flattened outputs o = lane + 32 q (q < NQ) from shared memory, so the operand rows are read
// once per block and no FMA is spent on padding beyond the last partial row of 32 outputs.
constexpr int kWbK = 16;                    // K chunk
constexpr int kWbStride = kWbK + 1;         // padded row stride of the staged chunks
constexpr int kWbWarpSmem = 2 * 32 * kWbStride;  // doubles per warp (A rows and B rows)

template <int NQ>
__device__ __forceinline__ void gemm_tile_wb(const Slots& S, const GemmTask& T, const GemmSeg* __restrict__ segs,
                                             const int* __restrict__ cmaps, int m0, int n0, int tm, int tn, int lane,
                                             double* __restrict__ sm) {
    double* As = sm;
    double* Bs = sm + 32 * kWbStride;
    const int nout = tm * tn;
    double v[NQ];
    int oa[NQ], ob[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        v[q] = 0.0;
        const int o = lane + 32 * q;
        const int oo = o < nout ? o : 0;
        oa[q] = (oo / tn) * kWbStride;
        ob[q] = (oo % tn) * kWbStride;
    }
    for (int sgi = 0; sgi < T.nseg; ++sgi) {
        const GemmSeg sg = segs[T.seg0 + sgi];
        const double* __restrict__ A = resolve(S, sg.a) + static_cast<int64_t>(m0) * sg.a_rs;
        const double* __restrict__ B = resolve(S, sg.b) + static_cast<int64_t>(n0) * sg.b_cs;
        const int kl = lane & 15, rl = lane >> 4;
        for (int k0 = 0; k0 < sg.K; k0 += kWbK) {
            const int kc = min(kWbK, sg.K - k0);
            const bool kv = kl < kc;
            const int64_t ka = static_cast<int64_t>(k0 + kl) * sg.a_cs;
            const int64_t kb = static_cast<int64_t>(k0 + kl) * sg.b_rs;
            for (int i = rl; i < tm; i += 2)
                As[i * kWbStride + kl] = kv ? __ldg(A + static_cast<int64_t>(i) * sg.a_rs + ka) : 0.0;
            for (int j = rl; j < tn; j += 2)
                Bs[j * kWbStride + kl] = kv ? __ldg(B + kb + static_cast<int64_t>(j) * sg.b_cs) : 0.0;
            __syncwarp();
            for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) v[q] = fma(As[oa[q] + kk], Bs[ob[q] + kk], v[q]);
            }
            __syncwarp();
        }
    }
    double* C = resolve(S, T.c);
    const int* cm = T.cmap >= 0 ? cmaps + T.cmap : nullptr;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int o = lane + 32 * q;
        if (o < nout) {
            const int i = o / tn, j = o % tn;
            const int64_t cc = cm ? cm[n0 + j] : n0 + j;
            C[static_cast<int64_t>(m0 + i) * T.ldc + cc] = v[q];
        }
    }
}

__global__ void __launch_bounds__(128) k_gemm_f64(Slots S, const GemmTask* __restrict__ tasks,
                                                  const GemmSeg* __restrict__ segs, const GemmTile* __restrict__ tiles,
                                                  const int* __restrict__ cmaps, int n_tiles) {
    __shared__ double wb_smem[4 * kWbWarpSmem];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_tiles) return;
    const GemmTile tl = tiles[warp];
    const GemmTask T = tasks[tl.task];
    if (tl.shape == 5) {
        double* sm = wb_smem + (threadIdx.x >> 5) * kWbWarpSmem;
        const int nq = (tl.tm * tl.tn + 31) / 32;
        switch (nq) {
            case 1: gemm_tile_wb<1>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            case 2: gemm_tile_wb<2>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            case 3: gemm_tile_wb<3>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            case 4: gemm_tile_wb<4>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            case 5: gemm_tile_wb<5>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            case 6: gemm_tile_wb<6>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            case 7: gemm_tile_wb<7>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
            default: gemm_tile_wb<8>(S, T, segs, cmaps, tl.m0, tl.n0, tl.tm, tl.tn, lane, sm); break;
        }
        return;
    }
    switch (tl.shape) {
        case 1: gemm_tile<4, 8, 1, 8>(S, T, segs, cmaps, tl.m0, tl.n0, lane); break;
        case 2: gemm_tile<8, 4, 8, 1>(S, T, segs, cmaps, tl.m0, tl.n0, lane); break;
        case 3: gemm_tile<8, 4, 4, 2>(S, T, segs, cmaps, tl.m0, tl.n0, lane); break;
        case 4: gemm_tile<4, 8, 2, 4>(S, T, segs, cmaps, tl.m0, tl.n0, lane); break;
        default: gemm_tile<8, 4, 2, 4>(S, T, segs, cmaps, tl.m0, tl.n0, lane); break;
    }
}

// ---- beta reduction of the output partials ------------------------------------------------------
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ partial, int G, int64_t n,
                                                      double* __restrict__ out) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int g = 0; g < G; ++g) acc += partial[g * n + i];
        out[i] = acc;
    }
}

// ---- block linear combination (MPO legs) ------------------------------------------------------
__global__ void __launch_bounds__(256) k_comb_f64(Slots S, const CombOut* __restrict__ outs,
                                                  const CombTerm* __restrict__ terms, int n_outs) {
    const int ob = blockIdx.x;
    if (ob >= n_outs) return;
    const CombOut o = outs[ob];
    double* dst = resolve(S, o.dst);
    const int n = o.rows * o.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int r = e / o.cols, c = e - r * o.cols;
        double acc = 0.0;
        for (int t = 0; t < o.nterm; ++t) {
            const CombTerm tm = terms[o.term0 + t];
            acc = fma(tm.coef, __ldg(resolve(S, tm.src) + static_cast<int64_t>(r) * tm.ld + c), acc);
        }
        dst[static_cast<int64_t>(r) * o.ld + c] = acc;
    }
}

// ---- diagonal of the projected operators ------------------------------------------------------
__global__ void __launch_bounds__(256) k_diag_f64(Slots S, const DiagBlock* __restrict__ blocks,
                                                  const DiagTerm* __restrict__ terms, int n_blocks, double* dh,
                                                  double* dn) {
    const int bi = blockIdx.x;
    if (bi >= n_blocks) return;
    const DiagBlock b = blocks[bi];
    double* out = b.out == 0 ? dh : dn;
    const int n = b.rows * b.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / b.cols, j = e - i * b.cols;
        double acc = 0.0;
        for (int t = 0; t < b.nterm; ++t) {
            const DiagTerm tm = terms[b.term0 + t];
            acc = fma(tm.coef * resolve(S, tm.l)[static_cast<int64_t>(i) * tm.l_step],
                      resolve(S, tm.r)[static_cast<int64_t>(j) * tm.r_step], acc);
        }
        out[b.off + static_cast<int64_t>(i) * b.ld + j] = acc;
    }
}

// ---- reductions and vector kernels ------------------------------------------------------------
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;  // valid in thread 0
}

constexpr int kRedBlocks = 64;

// partial[j * kRedBlocks + b] = sum over chunk b of V[:, j] . x
__global__ void __launch_bounds__(256) k_multidot_partial(const double* __restrict__ V, int64_t ldv,
                                                          const double* __restrict__ x, int64_t n,
                                                          double* __restrict__ partial) {
    __shared__ double sh[32];
    const int j = blockIdx.y;
    const double* v = V + j * ldv;
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        acc = fma(v[i], x[i], acc);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[j * kRedBlocks + blockIdx.x] = acc;
}
__global__ void k_multidot_final(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    // one warp per output, fixed summation order
    const int j = blockIdx.x;
    const int lane = threadIdx.x;
    double acc = 0.0;
    for (int b = lane; b < nb; b += 32) acc += partial[j * kRedBlocks + b];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[j] = acc;
}

__global__ void __launch_bounds__(256) k_gemv(const double* __restrict__ V, int64_t ldv, int m,
                                              const double* __restrict__ c, int64_t n, double* __restrict__ y,
                                              int sub) {
    __shared__ double cs[64];
    if (threadIdx.x < m) cs[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < m; ++j) acc = fma(V[j * ldv + i], cs[j], acc);
        y[i] = sub ? y[i] - acc : acc;
    }
}

__global__ void __launch_bounds__(256) k_basis_rotate(const double* __restrict__ src, int64_t ld, int m,
                                                      const double* __restrict__ Q, int ldq, int k, int64_t n,
                                                      double* __restrict__ dst) {
    __shared__ double qs[64 * 4];
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int i = e % m, j = e / m;
        qs[j * 64 + i] = Q[i + j * ldq];
    }
    __syncthreads();
    for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        for (int j = 0; j < k; ++j) {
            double acc = 0.0;
            for (int i = 0; i < m; ++i) acc = fma(src[i * ld + r], qs[j * 64 + i], acc);
            dst[j * ld + r] = acc;
        }
    }
}

__global__ void __launch_bounds__(256) k_norm2_partial(const double* __restrict__ x, int64_t n,
                                                       double* __restrict__ partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        acc = fma(x[i], x[i], acc);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) k_scale_inv_sqrt(double* __restrict__ x, int64_t n,
                                                        const double* __restrict__ nrm2) {
    const double v = *nrm2;
    const double s = v > 1e-300 ? 1.0 / sqrt(v) : 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[i] *= s;
}

__global__ void __launch_bounds__(256) k_residual_diag(const double* __restrict__ hx, const double* __restrict__ nx,
                                                       const double* __restrict__ dh, const double* __restrict__ dn,
                                                       const double* __restrict__ scal, double clamp, int64_t n,
                                                       double* __restrict__ r, double* __restrict__ t) {
    const double theta = scal[0];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double ri = hx[i] - theta * nx[i];
        r[i] = ri;
        double den = dh[i] - theta * dn[i];
        if (fabs(den) < clamp) den = den < 0.0 ? -clamp : clamp;
        t[i] = -ri / den;
    }
}

// out = v / (diag H - theta diag N), the denominator clamped as in k_residual_diag
__global__ void __launch_bounds__(256) k_precond_apply(const double* __restrict__ v, const double* __restrict__ dh,
                                                       const double* __restrict__ dn,
                                                       const double* __restrict__ scal, double clamp, int64_t n,
                                                       double* __restrict__ out) {
    const double theta = scal[0];
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double den = dh[i] - theta * dn[i];
        if (fabs(den) < clamp) den = den < 0.0 ? -clamp : clamp;
        out[i] = v[i] / den;
    }
}

__global__ void __launch_bounds__(256) k_axpy_ratio(double* __restrict__ x, const double* __restrict__ y, int64_t n,
                                                    const double* __restrict__ num, const double* __restrict__ den,
                                                    double sign) {
    const double d = *den;
    const double a = d != 0.0 ? sign * (*num) / d : 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        x[i] = fma(a, y[i], x[i]);
}

__global__ void __launch_bounds__(256) k_xpby_ratio(double* __restrict__ p, const double* __restrict__ r, int64_t n,
                                                    const double* __restrict__ num, const double* __restrict__ den) {
    const double d = *den;
    const double b = d != 0.0 ? (*num) / d : 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = fma(b, p[i], r[i]);
}

// ---- one-CTA cyclic Jacobi (parallel round-robin ordering) ------------------------------------
// A (n x n, row stride lda) symmetric, V (row stride ldv) receives the eigenvectors as columns.
// Returns the number of sweeps used (max_sweeps + 1 if not converged).
__device__ int jacobi_cta(double* A, int lda, double* V, int ldv, int n, int max_sweeps, double* cs_sh,
                          int* pq_sh, double* red_sh) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e - i * n;
        V[i * ldv + j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    if (n <= 1) return 0;
    const int np = (n + 1) & ~1;  // players, even
    const int half = np / 2;
    int sweep = 0;
    double off_prev = INFINITY;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += nt) {
            const int i = e / n, j = e - i * n;
            const double v = A[i * lda + j];
            tot += v * v;
            if (i != j) off += v * v;
        }
        off = block_sum(off, red_sh);
        if (tid == 0) red_sh[33] = off;
        tot = block_sum(tot, red_sh);
        if (tid == 0) red_sh[34] = tot;
        __syncthreads();
        off = red_sh[33];
        tot = red_sh[34];
        // converged, or near convergence and at the rounding-noise floor (a sweep no longer reduces
        // the off-diagonal norm: Jacobi converges quadratically until rounding noise dominates)
        if (off <= 1e-28 * tot || off == 0.0 || (off <= 1e-20 * tot && off > 0.25 * off_prev)) break;
        off_prev = off;
        const double tiny = 1e-18 * sqrt(tot);
        for (int round = 0; round < np - 1; ++round) {
            for (int i = tid; i < half; i += nt) {
                auto player = [&](int k) { return k == 0 ? 0 : 1 + ((k - 1 + round) % (np - 1)); };
                int p = player(i), q = player(np - 1 - i);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[p * lda + q];
                    if (fabs(apq) > tiny) {
                        const double app = A[p * lda + p], aqq = A[q * lda + q];
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    } else {
                        q = -1;  // negligible coupling: no rotation, no update
                    }
                } else {
                    q = -1;
                }
                pq_sh[2 * i] = p;
                pq_sh[2 * i + 1] = q;
                cs_sh[2 * i] = c;
                cs_sh[2 * i + 1] = s;
            }
            __syncthreads();
            // rows p, q
            for (int e = tid; e < half * n; e += nt) {
                const int i = e / n, j = e - i * n;
                const int p = pq_sh[2 * i], q = pq_sh[2 * i + 1];
                if (q < 0) continue;
                const double c = cs_sh[2 * i], s = cs_sh[2 * i + 1];
                const double ap = A[p * lda + j], aq = A[q * lda + j];
                A[p * lda + j] = c * ap - s * aq;
                A[q * lda + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns p, q of A and V
            for (int e = tid; e < half * n; e += nt) {
                const int i = e / n, j = e - i * n;
                const int p = pq_sh[2 * i], q = pq_sh[2 * i + 1];
                if (q < 0) continue;
                const double c = cs_sh[2 * i], s = cs_sh[2 * i + 1];
                const double ap = A[j * lda + p], aq = A[j * lda + q];
                A[j * lda + p] = c * ap - s * aq;
                A[j * lda + q] = s * ap + c * aq;
                const double vp = V[j * ldv + p], vq = V[j * ldv + q];
                V[j * ldv + p] = c * vp - s * vq;
                V[j * ldv + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    return sweep;
}

// ---- one-warp cyclic Jacobi in FP32 --------------------------------------------------------------
// The same round-robin pairs, rotation formula and ordering (rows, then columns) as jacobi_cta, on
// one warp with warp-level synchronisation; A (n x n, row stride ld) symmetric, V receives the
// rotations (eigenvectors as columns).  Used for the eigenbasis of the Ritz problem, whose lowest
// pair is then refined in FP64.
__device__ __forceinline__ float warp_sumf(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ void jacobi_warp_f32(float* A, float* V, int ld, int n, float* cs, int* pq) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e - i * n;
        V[i * ld + j] = i == j ? 1.0f : 0.0f;
    }
    __syncwarp();
    if (n <= 1) return;
    const int np = (n + 1) & ~1;
    const int half = np / 2;
    float off_prev = INFINITY;
    for (int sweep = 0; sweep < 30; ++sweep) {
        float off = 0.0f, tot = 0.0f;
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e - i * n;
            const float v = A[i * ld + j];
            tot += v * v;
            if (i != j) off += v * v;
        }
        off = warp_sumf(off);
        tot = warp_sumf(tot);
        // off-diagonal below 3e-5 of the matrix (the FP64 refinement of the lowest pair reduces
        // its error by about that factor per correction), or no longer decreasing
        if (off <= 1e-9f * tot || off == 0.0f || (off <= 1e-6f * tot && off > 0.25f * off_prev)) break;
        off_prev = off;
        const float tiny = 1e-10f * sqrtf(tot);
        for (int round = 0; round < np - 1; ++round) {
            if (lane < half) {
                auto player = [&](int k) { return k == 0 ? 0 : 1 + ((k - 1 + round) % (np - 1)); };
                int p = player(lane), q = player(np - 1 - lane);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                float c = 1.0f, s = 0.0f;
                if (q < n && fabsf(A[p * ld + q]) > tiny) {
                    const float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
                    const float theta = (aqq - app) / (2.0f * apq);
                    const float t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
                    c = 1.0f / sqrtf(t * t + 1.0f);
                    s = t * c;
                } else {
                    q = -1;
                }
                pq[2 * lane] = p;
                pq[2 * lane + 1] = q;
                cs[2 * lane] = c;
                cs[2 * lane + 1] = s;
            }
            __syncwarp();
            for (int e = lane; e < half * n; e += 32) {  // rows p, q
                const int i = e / n, j = e - i * n;
                const int p = pq[2 * i], q = pq[2 * i + 1];
                if (q < 0) continue;
                const float c = cs[2 * i], s = cs[2 * i + 1];
                const float ap = A[p * ld + j], aq = A[q * ld + j];
                A[p * ld + j] = c * ap - s * aq;
                A[q * ld + j] = s * ap + c * aq;
            }
            __syncwarp();
            for (int e = lane; e < half * n; e += 32) {  // columns p, q of A and V
                const int i = e / n, j = e - i * n;
                const int p = pq[2 * i], q = pq[2 * i + 1];
                if (q < 0) continue;
                const float c = cs[2 * i], s = cs[2 * i + 1];
                const float ap = A[j * ld + p], aq = A[j * ld + q];
                A[j * ld + p] = c * ap - s * aq;
                A[j * ld + q] = s * ap + c * aq;
                const float vp = V[j * ld + p], vq = V[j * ld + q];
                V[j * ld + p] = c * vp - s * vq;
                V[j * ld + q] = s * vp + c * vq;
            }
            __syncwarp();
        }
    }
}

constexpr int kRitzMax = 32;

// ---- incremental Ritz step --------------------------------------------------------------------
// Keeps, across the iterations of one Davidson solve, an n-orthonormal coefficient basis X
// (Y = V X has Y^T N Y = I), the projected matrix hp = X^T h X and the eigenvectors C of hp.
// Adding basis vector v_m: classical Gram-Schmidt of e_m against X in the n inner product,
// twice; the direction is kept when its n-norm^2 exceeds eps * max(diag n) (numerically null
// directions of the metric are dropped, as in canonical orthogonalisation).  hp grows by one row
// and column; its eigenbasis is re-solved by one-warp FP32 Jacobi started from the previous
// eigenvectors (so only the new coupling has to be rotated away), and the lowest pair is refined in
// FP64 against hp (below).
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Incremental Ritz step (one CTA of 128 threads: one warp per SM sub-partition for the
// Gram-Schmidt and the products; the Jacobi sweeps and the FP64 refinement run on warp 0).
constexpr double kMetricFloor = 1e-14;

__global__ void __launch_bounds__(128) k_ritz_inc(const double* __restrict__ h, const double* __restrict__ nm, int ldm,
                                                  int m, int reset, double eps, RitzState* __restrict__ st,
                                                  double* __restrict__ coef, double* __restrict__ scal) {
    constexpr int R = RitzState::kR;
    extern __shared__ double rs_smem[];
    double* X = rs_smem;           // n-orthonormal coefficient basis, X[i + j*R]
    double* HP = X + R * R;        // X^T h X
    double* CC = HP + R * R;       // previous eigenvectors of HP (columns)
    double* A = CC + R * R;
    double* T = A + R * R;
    double* NS = T + R * R;        // n, full symmetric, NS[i*R + j]
    double* HS = NS + R * R;       // h, full symmetric
    __shared__ double cs_sh[R + 2], red_sh[40];
    __shared__ int pq_sh[R + 2];
    __shared__ int k_sh;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    int k = 0, m0 = 0, kc = 0;
    if (!reset) {
        k = st->k;
        m0 = st->m;
        kc = st->kc;
        for (int e = tid; e < R * R; e += nt) {
            X[e] = st->X[e];
            HP[e] = st->hp[e];
            CC[e] = st->C[e];
        }
    }
    for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e - i * m;
        const int hi = i > j ? i : j, lo = i > j ? j : i;
        NS[i * R + j] = nm[hi * ldm + lo];
        HS[i * R + j] = h[hi * ldm + lo];
    }
    __syncthreads();
    // new columns of the n-orthonormal basis (32-long vectors: warp 0)
    if (tid < 32) {
        double dmax = 0.0;
        for (int i = 0; i < m; ++i) dmax = fmax(dmax, NS[i * R + i]);
        for (int col = m0; col < m; ++col) {
            // y = e_col - X (X^T n y), twice, in the n inner product (lane i holds y_i, i <= col)
            double y = lane == col ? 1.0 : 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                double ny = 0.0;
                for (int l = 0; l <= col; ++l) {
                    const double yl = __shfl_sync(0xffffffffu, y, l);
                    if (lane <= col) ny = fma(NS[lane * R + l], yl, ny);
                }
                double corr = 0.0;
                for (int j = 0; j < k; ++j) {
                    const double cj = warp_sum(lane <= col ? X[lane + j * R] * ny : 0.0);
                    if (lane <= col) corr = fma(X[lane + j * R], cj, corr);
                }
                y -= corr;
            }
            double ny = 0.0;
            for (int l = 0; l <= col; ++l) {
                const double yl = __shfl_sync(0xffffffffu, y, l);
                if (lane <= col) ny = fma(NS[lane * R + l], yl, ny);
            }
            const double nu2 = warp_sum(lane <= col ? y * ny : 0.0);
            // the basis vectors have unit norm and |N_eff| <= 1: below kMetricFloor the metric is
            // numerically zero (no state of the target spin is reachable), whatever eps says
            if (nu2 > eps * dmax && nu2 > kMetricFloor) {
                const double inv = 1.0 / sqrt(nu2);
                X[lane + k * R] = lane <= col ? y * inv : 0.0;
                __syncwarp();
                double hx = 0.0;
                for (int l = 0; l <= col; ++l)
                    if (lane <= col) hx = fma(HS[lane * R + l], X[l + k * R], hx);
                for (int j = 0; j <= k; ++j) {
                    const double v = warp_sum(lane <= col ? X[lane + j * R] * hx : 0.0);
                    if (lane == 0) { HP[j * R + k] = v; HP[k * R + j] = v; }
                }
                ++k;
            }
            __syncwarp();
        }
        if (lane == 0) k_sh = k;
    }
    __syncthreads();
    k = k_sh;
    // The Ritz pair.  FP32 Jacobi on W0^T HP W0, W0 = previous eigenvectors padded with the
    // identity (so only the new row and column have to be rotated away), gives the eigenbasis W of
    // HP to FP32 accuracy; the lowest pair is then refined in FP64 against HP itself: Rayleigh
    // quotient y^T HP y / y^T y, residual r = HP y - theta y, and the correction
    // sum_{j != min} w_j (w_j^T r) / (theta - lambda_j) through W's spectrum, three times, so theta
    // and the coefficients are FP64-accurate while the O(k^3) work runs in FP32.
    constexpr int LF = R + 1;
    float* Af = reinterpret_cast<float*>(A);   // W0^T HP W0, then its Jacobi-diagonalised form
    float* Vf = reinterpret_cast<float*>(T);   // HP W0, then the Jacobi rotations
    float* W0 = reinterpret_cast<float*>(NS);  // start basis
    float* Wf = reinterpret_cast<float*>(HS);  // eigenbasis W = W0 V
    __shared__ float cs32[2 * R];
    __shared__ int pq32[2 * R];
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e - i * k;
        W0[i * LF + j] = (i < kc && j < kc) ? static_cast<float>(CC[i * R + j]) : (i == j ? 1.0f : 0.0f);
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {  // HP W0
        const int i = e / k, j = e - i * k;
        float acc = 0.0f;
        for (int l = 0; l < k; ++l) acc = fmaf(static_cast<float>(HP[i * R + l]), W0[l * LF + j], acc);
        Vf[i * LF + j] = acc;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {  // W0^T (HP W0)
        const int i = e / k, j = e - i * k;
        float acc = 0.0f;
        for (int l = 0; l < k; ++l) acc = fmaf(W0[l * LF + i], Vf[l * LF + j], acc);
        Af[i * LF + j] = acc;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {  // symmetrise
        const int i = e / k, j = e - i * k;
        if (i < j) {
            const float v = 0.5f * (Af[i * LF + j] + Af[j * LF + i]);
            Af[i * LF + j] = v;
            Af[j * LF + i] = v;
        }
    }
    __syncthreads();
    if (tid < 32) jacobi_warp_f32(Af, Vf, LF, k, cs32, pq32);
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {  // W = W0 V
        const int i = e / k, j = e - i * k;
        float acc = 0.0f;
        for (int l = 0; l < k; ++l) acc = fmaf(W0[i * LF + l], Vf[l * LF + j], acc);
        Wf[i * LF + j] = acc;
    }
    __syncthreads();
    if (tid < 32) {
        // lowest diagonal entry of the rotated matrix
        float lam = lane < k ? Af[lane * LF + lane] : INFINITY;
        float best = lam;
        int jmin = lane < k ? lane : R;
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, jmin, o);
            if (ob < best || (ob == best && oj < jmin)) {
                best = ob;
                jmin = oj;
            }
        }
        double y = (lane < k && jmin < R) ? static_cast<double>(Wf[lane * LF + jmin]) : 0.0;
        double theta = 0.0;
        for (int it = 0; it <= 3; ++it) {
            double hy = 0.0;
            for (int l = 0; l < k; ++l) {
                const double yl = __shfl_sync(0xffffffffu, y, l);
                if (lane < k) hy = fma(HP[lane * R + l], yl, hy);
            }
            const double yy = warp_sum(y * y), yhy = warp_sum(y * hy);
            theta = yy > 0.0 ? yhy / yy : 0.0;
            if (it == 3) {
                y = yy > 0.0 ? y / sqrt(yy) : 0.0;
                break;
            }
            const double r = lane < k ? hy - theta * y : 0.0;
            double c = 0.0;  // lane j: w_j^T r
            for (int i = 0; i < k; ++i) {
                const double ri = __shfl_sync(0xffffffffu, r, i);
                if (lane < k) c = fma(static_cast<double>(Wf[i * LF + lane]), ri, c);
            }
            const double den = theta - static_cast<double>(lam);
            // components (nearly) degenerate with the lowest one are left as they are
            const bool use = lane < k && lane != jmin && fabs(den) > 1e-7 * (fabs(theta) + fabs(static_cast<double>(lam)) + 1e-300);
            c = use ? c / den : 0.0;
            double d = 0.0;
            for (int j = 0; j < k; ++j) {
                const double cj = __shfl_sync(0xffffffffu, c, j);
                if (lane < k) d = fma(static_cast<double>(Wf[lane * LF + j]), cj, d);
            }
            y += d;
        }
        if (lane == 0) {
            scal[0] = k > 0 ? theta : 0.0;
            scal[1] = static_cast<double>(k);
        }
        // coefficients of the Ritz vector in the basis V: X y
        double acc = 0.0;
        for (int j = 0; j < k; ++j) {
            const double yj = __shfl_sync(0xffffffffu, y, j);
            if (lane < m) acc = fma(X[lane + j * R], yj, acc);
        }
        if (lane < m) coef[lane] = k > 0 ? acc : 0.0;
    }
    for (int e = tid; e < R * R; e += nt) {
        const int i = e / R, j = e - i * R;
        st->C[e] = (i < k && j < k) ? static_cast<double>(Wf[i * LF + j]) : 0.0;
        st->X[e] = X[e];
        st->hp[e] = HP[e];
    }
    if (tid == 0) {
        st->k = k;
        st->m = m;
        st->kc = k;
    }
}

// Orthonormal restart coefficients from [c_new, c_old] (Gram-Schmidt, twice).
__global__ void k_restart_coef(const double* __restrict__ cn, const double* __restrict__ co, int m,
                               double* __restrict__ Q, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double a[kRitzMax], b[kRitzMax];
    double na = 0.0;
    for (int i = 0; i < m; ++i) { a[i] = cn[i]; na += a[i] * a[i]; }
    na = sqrt(na);
    for (int i = 0; i < m; ++i) a[i] /= na;
    for (int i = 0; i < m; ++i) b[i] = co[i];
    for (int pass = 0; pass < 2; ++pass) {
        double d = 0.0;
        for (int i = 0; i < m; ++i) d += a[i] * b[i];
        for (int i = 0; i < m; ++i) b[i] -= d * a[i];
    }
    double nb = 0.0;
    for (int i = 0; i < m; ++i) nb += b[i] * b[i];
    nb = sqrt(nb);
    int k = 1;
    for (int i = 0; i < m; ++i) Q[i] = a[i];
    if (nb > 1e-10) {
        k = 2;
        for (int i = 0; i < m; ++i) Q[m + i] = b[i] / nb;
    } else {
        for (int i = 0; i < m; ++i) Q[m + i] = 0.0;  // a zero second column (dropped downstream)
    }
    out[0] = k;
    // coefficients of the current Ritz vector in the rotated basis: Q^T c_new
    double d0 = 0.0, d1 = 0.0;
    for (int i = 0; i < m; ++i) { d0 += Q[i] * cn[i]; if (k == 2) d1 += Q[m + i] * cn[i]; }
    out[1] = d0;
    out[2] = d1;
}

// ---- batched Jacobi for the decimation --------------------------------------------------------
constexpr int kJacobiSmemMax = 112;
// cluster Jacobi: kJcC CTAs per matrix for dimensions in (kJcMin, kJcMax]
constexpr int kJcC = 8;
constexpr int kJcMin = 64;
constexpr int kJcMax = 256;

__global__ void __launch_bounds__(512) k_jacobi_batched(double* __restrict__ mats, double* __restrict__ vscratch,
                                                        double* __restrict__ evals,
                                                        const int64_t* __restrict__ mat_off,
                                                        const int64_t* __restrict__ val_off,
                                                        const int* __restrict__ dims, int smem_dim,
                                                        int skip_cluster, int* __restrict__ status) {
    extern __shared__ double smem[];
    __shared__ double cs_sh[2 * 256 + 4], red_sh[40], dg[512];
    __shared__ int pq_sh[2 * 256 + 4];
    const int b = blockIdx.x;
    const int n = dims[b];
    if (n <= 0) return;
    if (skip_cluster && n > kJcMin && n <= kJcMax) return;  // handled by k_jacobi_cluster
    double* M = mats + mat_off[b];
    double *A, *V;
    if (n <= smem_dim) {  // the launch sized the dynamic shared memory for smem_dim
        A = smem;
        V = smem + n * n;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = M[e];
    } else {
        A = M;  // in place; eigenvectors in the caller's scratch
        V = vscratch + mat_off[b];
    }
    __syncthreads();
    const int sweeps = jacobi_cta(A, n, V, n, n, 60, cs_sh, pq_sh, red_sh);
    if (threadIdx.x == 0 && sweeps >= 60) atomicExch(status, 1);  // cap reached (not at the noise floor)
    for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = A[i * n + i];
    __syncthreads();
    // eigenpairs sorted by descending eigenvalue (rank sort, ties by index)
    double* ev = evals + val_off[b];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double vi = dg[i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const double vj = dg[j];
            if (vj > vi || (vj == vi && j < i)) ++rank;
        }
        ev[rank] = vi;
        for (int r = 0; r < n; ++r) M[r * n + rank] = V[r * n + i];
    }
}

// ---- cluster Jacobi for the larger decimation blocks ------------------------------------------
// One thread-block cluster of kJcC CTAs per density matrix of dimension in (kJcMin, kJcMax]: row r
// of A and row r of V^T live in the shared memory of CTA r % kJcC.  The sweeps use the same
// round-robin pairs, rotation formula, skip rule and stopping rule as jacobi_cta, so every element
// receives the same rotations in the same order; each round is
//   params of the CTA's pairs (from rows p and q, possibly remote) -> cluster barrier ->
//   column update of the CTA's own rows (all pairs, local) -> cluster barrier ->
//   row update of rows p, q of A and V^T for the CTA's pairs (distributed shared memory) ->
//   cluster barrier.
// The barriers are hardware cluster barriers that every CTA of the cluster executes the same
// number of times (the stopping decision is made from the same partial sums on every CTA).
namespace cgx = cooperative_groups;

__global__ void __cluster_dims__(kJcC, 1, 1) __launch_bounds__(256)
    k_jacobi_cluster(double* __restrict__ mats, double* __restrict__ evals, const int64_t* __restrict__ mat_off,
                     const int64_t* __restrict__ val_off, const int* __restrict__ dims, int* __restrict__ status) {
    extern __shared__ double jc_smem[];
    __shared__ double cs_loc[2 * (kJcMax / 2) + 2];
    __shared__ int pq_loc[2 * (kJcMax / 2) + 2];
    __shared__ double part[2], red_sh[40];
    cgx::cluster_group cl = cgx::this_cluster();
    const int rank = static_cast<int>(cl.block_rank());
    const int b = blockIdx.x / kJcC;
    const int n = dims[b];
    if (n <= kJcMin || n > kJcMax) return;  // uniform over the cluster
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rows = (n - rank + kJcC - 1) / kJcC;  // rows r = rank + kJcC * i
    const int rmax = (n + kJcC - 1) / kJcC;
    double* Ar = jc_smem;                 // [rmax][n]
    double* Vt = jc_smem + rmax * n;      // [rmax][n]
    double* cs_own = Vt + rmax * n;       // params of this CTA's pairs, read by the others
    int* pq_own = reinterpret_cast<int*>(cs_own + 2 * (kJcMax / 2) + 2);
    double* M = mats + mat_off[b];
    for (int e = tid; e < rows * n; e += nt) {
        const int i = e / n, j = e - i * n;
        const int r = rank + kJcC * i;
        Ar[i * n + j] = M[static_cast<int64_t>(r) * n + j];
        Vt[i * n + j] = r == j ? 1.0 : 0.0;
    }
    cl.sync();
    auto row_ptr = [&](double* base, int r) -> double* {
        double* local = base + (r / kJcC) * n;
        return cl.map_shared_rank(local, r % kJcC);
    };
    const int np = (n + 1) & ~1, half = np / 2;
    double off_prev = INFINITY;
    int sweep = 0;
    for (; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < rows * n; e += nt) {
            const int i = e / n, j = e - i * n;
            const int r = rank + kJcC * i;
            const double v = Ar[i * n + j];
            tot += v * v;
            if (r != j) off += v * v;
        }
        off = block_sum(off, red_sh);
        if (tid == 0) part[0] = off;
        tot = block_sum(tot, red_sh);
        if (tid == 0) part[1] = tot;
        cl.sync();
        off = 0.0;
        tot = 0.0;
        for (int c = 0; c < kJcC; ++c) {  // same order on every CTA
            const double* pr = cl.map_shared_rank(part, c);
            off += pr[0];
            tot += pr[1];
        }
        cl.sync();  // the partials are read before they are overwritten
        if (off <= 1e-28 * tot || off == 0.0 || (off <= 1e-20 * tot && off > 0.25 * off_prev)) break;
        off_prev = off;
        const double tiny = 1e-18 * sqrt(tot);
        for (int round = 0; round < np - 1; ++round) {
            // rotation parameters of the pairs i = rank, rank + kJcC, ...
            for (int i = rank + kJcC * tid; i < half; i += kJcC * nt) {
                auto player = [&](int k) { return k == 0 ? 0 : 1 + ((k - 1 + round) % (np - 1)); };
                int p = player(i), q = player(np - 1 - i);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, sn = 0.0;
                if (q < n) {
                    const double apq = row_ptr(Ar, p)[q];
                    if (fabs(apq) > tiny) {
                        const double app = row_ptr(Ar, p)[p], aqq = row_ptr(Ar, q)[q];
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sn = t * c;
                    } else {
                        q = -1;
                    }
                } else {
                    q = -1;
                }
                pq_own[2 * i] = p;
                pq_own[2 * i + 1] = q;
                cs_own[2 * i] = c;
                cs_own[2 * i + 1] = sn;
            }
            cl.sync();
            for (int i = tid; i < half; i += nt) {
                const int src = i % kJcC;
                const int* pqr = cl.map_shared_rank(pq_own, src);
                const double* csr = cl.map_shared_rank(cs_own, src);
                pq_loc[2 * i] = pqr[2 * i];
                pq_loc[2 * i + 1] = pqr[2 * i + 1];
                cs_loc[2 * i] = csr[2 * i];
                cs_loc[2 * i + 1] = csr[2 * i + 1];
            }
            __syncthreads();
            // columns p, q of the own rows
            for (int e = tid; e < rows * half; e += nt) {
                const int i = e / half, pi = e - i * half;
                const int p = pq_loc[2 * pi], q = pq_loc[2 * pi + 1];
                if (q < 0) continue;
                const double c = cs_loc[2 * pi], sn = cs_loc[2 * pi + 1];
                const double ap = Ar[i * n + p], aq = Ar[i * n + q];
                Ar[i * n + p] = c * ap - sn * aq;
                Ar[i * n + q] = sn * ap + c * aq;
            }
            cl.sync();
            // rows p, q of A and of V^T for this CTA's pairs
            for (int i = rank; i < half; i += kJcC) {
                const int p = pq_loc[2 * i], q = pq_loc[2 * i + 1];
                if (q < 0) continue;
                const double c = cs_loc[2 * i], sn = cs_loc[2 * i + 1];
                double* ap = row_ptr(Ar, p);
                double* aq = row_ptr(Ar, q);
                double* vp = row_ptr(Vt, p);
                double* vq = row_ptr(Vt, q);
                for (int j = tid; j < n; j += nt) {
                    const double x = ap[j], y = aq[j];
                    ap[j] = c * x - sn * y;
                    aq[j] = sn * x + c * y;
                    const double u = vp[j], w = vq[j];
                    vp[j] = c * u - sn * w;
                    vq[j] = sn * u + c * w;
                }
            }
            cl.sync();
        }
    }
    if (tid == 0 && rank == 0 && sweep >= 60) atomicExch(status, 1);
    // eigenpairs sorted by descending eigenvalue (rank sort, ties by index): the CTA writes the
    // eigenvalues and eigenvector columns of its own rows
    double* ev = evals + val_off[b];
    for (int i = tid; i < rows; i += nt) {
        const int r = rank + kJcC * i;
        const double vi = Ar[i * n + r];
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const double vj = row_ptr(Ar, j)[j];
            if (vj > vi || (vj == vi && j < r)) ++rk;
        }
        ev[rk] = vi;
        for (int q = 0; q < n; ++q) M[static_cast<int64_t>(q) * n + rk] = Vt[i * n + q];
    }
    cl.sync();  // no CTA leaves while others still read its shared memory
}

// ---- ordered truncation (one CTA) ---------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_truncate(const double* __restrict__ evals, const int64_t* __restrict__ val_off,
                                                   const int* __restrict__ dims, const int* __restrict__ label_n,
                                                   const int* __restrict__ label_tm, int n_labels, int total, int D,
                                                   double tie_rtol, double drop_abs, int* __restrict__ keep_count,
                                                   int* __restrict__ keep_total, double* __restrict__ discarded,
                                                   int* __restrict__ idx_buf, double* __restrict__ val_buf) {
    // idx_buf: 3*total ints (label, index-in-label, sorted position), val_buf: 2*total doubles
    int* lab = idx_buf;
    int* pos = idx_buf + total;
    int* order = idx_buf + 2 * total;
    double* sig = val_buf;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int l = tid; l < n_labels; l += nt) {
        const int64_t o = val_off[l];
        int base = 0;
        for (int q = 0; q < l; ++q) base += dims[q];
        for (int i = 0; i < dims[l]; ++i) {
            const double v = evals[o + i];
            sig[base + i] = v > 0.0 ? sqrt(v) : 0.0;
            lab[base + i] = l;
            pos[base + i] = i;
        }
        keep_count[l] = 0;
    }
    __syncthreads();
    // rank sort by descending value, ties by flat index
    for (int i = tid; i < total; i += nt) {
        const double vi = sig[i];
        int rank = 0;
        for (int j = 0; j < total; ++j) {
            const double vj = sig[j];
            if (vj > vi || (vj == vi && j < i)) ++rank;
        }
        order[rank] = i;
    }
    __syncthreads();
    if (tid != 0) return;
    const double vmax = total > 0 ? sig[order[0]] : 0.0;
    // clusters, ordered inside by (n, 2m, index)
    int start = 0;
    while (start < total) {
        int end = start + 1;
        while (end < total && sig[order[end - 1]] - sig[order[end]] <= tie_rtol * vmax) ++end;
        for (int a = start + 1; a < end; ++a) {  // insertion sort of the cluster
            const int key = order[a];
            int b2 = a - 1;
            while (b2 >= start) {
                const int o2 = order[b2];
                const int ln = label_n[lab[o2]], kn = label_n[lab[key]];
                const int lt = label_tm[lab[o2]], kt = label_tm[lab[key]];
                const bool greater = ln > kn || (ln == kn && (lt > kt || (lt == kt && pos[o2] > pos[key])));
                if (!greater) break;
                order[b2 + 1] = o2;
                --b2;
            }
            order[b2 + 1] = key;
        }
        start = end;
    }
    int kept = 0;
    double disc = 0.0;
    for (int r = 0; r < total; ++r) {
        const int i = order[r];
        if (kept < D && sig[i] >= drop_abs) {
            keep_count[lab[i]] += 1;
            ++kept;
        } else {
            disc += sig[i] * sig[i];
        }
    }
    keep_total[0] = kept;
    discarded[0] = disc;
}

// ---- block copies ------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_copy_blocks(Slots S, const CopyBlock* __restrict__ blocks, int n) {
    const int bi = blockIdx.x;
    if (bi >= n) return;
    const CopyBlock b = blocks[bi];
    const double* src = resolve(S, b.src);
    double* dst = resolve(S, b.dst);
    const int tot = b.rows * b.cols;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const int r = e / b.cols, c = e - r * b.cols;
        const double v = b.transpose ? src[static_cast<int64_t>(c) * b.ld_src + r] : src[static_cast<int64_t>(r) * b.ld_src + c];
        dst[static_cast<int64_t>(r) * b.ld_dst + c] = v;
    }
}

// FP64 throughput probe: 8 independent FMA chains per thread.
__global__ void __launch_bounds__(256) k_fp64_peak(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-7, x1 = x0 + 1e-8, x2 = x0 + 2e-8, x3 = x0 + 3e-8;
    double x4 = x0 + 4e-8, x5 = x0 + 5e-8, x6 = x0 + 6e-8, x7 = x0 + 7e-8;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const double r = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (r == 12345.678) out[0] = r;  // keeps the chains live
}

int grid_for(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return static_cast<int>(g);
}

}  // namespace

// ---- launch wrappers ----------------------------------------------------------------------------

cudaError_t launch_gemm_f64(const Slots& slots, const GemmTask* tasks, const GemmSeg* segs, const GemmTile* tiles,
                            const int* cmaps, int n_tiles, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const int warps_per_cta = 4;
    const int grid = (n_tiles + warps_per_cta - 1) / warps_per_cta;
    k_gemm_f64<<<grid, 32 * warps_per_cta, 0, st>>>(slots, tasks, segs, tiles, cmaps, n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partial, int G, int64_t n, double* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_sum_partials<<<grid_for(n, 256, 4096), 256, 0, st>>>(partial, G, n, out);
    return cudaGetLastError();
}

cudaError_t launch_comb_f64(const Slots& slots, const CombOut* outs, const CombTerm* terms, int n_outs,
                            cudaStream_t st) {
    if (n_outs <= 0) return cudaSuccess;
    k_comb_f64<<<n_outs, 256, 0, st>>>(slots, outs, terms, n_outs);
    return cudaGetLastError();
}

cudaError_t launch_diag_f64(const Slots& slots, const DiagBlock* blocks, const DiagTerm* terms, int n_blocks,
                            double* dh, double* dn, cudaStream_t st) {
    if (n_blocks <= 0) return cudaSuccess;
    k_diag_f64<<<n_blocks, 256, 0, st>>>(slots, blocks, terms, n_blocks, dh, dn);
    return cudaGetLastError();
}

cudaError_t launch_multidot(const double* V, int64_t ldv, int m, const double* x, int64_t n, double* out,
                            double* partial, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    if (m > kRitzMax) return cudaErrorInvalidValue;
    const int nb = grid_for(n, 256, kRedBlocks);
    k_multidot_partial<<<dim3(nb, m), 256, 0, st>>>(V, ldv, x, n, partial);
    k_multidot_final<<<m, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_gemv(const double* V, int64_t ldv, int m, const double* c, int64_t n, double* y, int sub,
                        cudaStream_t st) {
    if (m > 64) return cudaErrorInvalidValue;
    k_gemv<<<grid_for(n, 256, 2048), 256, 0, st>>>(V, ldv, m, c, n, y, sub);
    return cudaGetLastError();
}

cudaError_t launch_basis_rotate(const double* src, int64_t ld, int m, const double* Q, int ldq, int k, int64_t n,
                                double* dst, cudaStream_t st) {
    if (m > 64 || k > 4) return cudaErrorInvalidValue;
    k_basis_rotate<<<grid_for(n, 256, 2048), 256, 0, st>>>(src, ld, m, Q, ldq, k, n, dst);
    return cudaGetLastError();
}


cudaError_t launch_ritz_inc(const double* h, const double* nmat, int ldm, int m, int reset, double eps_metric,
                            RitzState* state, double* coef, double* scal, cudaStream_t st) {
    if (m > RitzState::kR) return cudaErrorInvalidValue;
    constexpr int smem = 7 * RitzState::kR * RitzState::kR * static_cast<int>(sizeof(double));
    static int attr_device = -1;  // the attribute is per device; set it once per device in use
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_ritz_inc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    k_ritz_inc<<<1, 128, smem, st>>>(h, nmat, ldm, m, reset, eps_metric, state, coef, scal);
    return cudaGetLastError();
}

cudaError_t launch_residual_diag(const double* hx, const double* nx, const double* dh, const double* dn,
                                 const double* scal, double clamp, int64_t n, double* r, double* t, double* red,
                                 double* partial, cudaStream_t st) {
    k_residual_diag<<<grid_for(n, 256, 2048), 256, 0, st>>>(hx, nx, dh, dn, scal, clamp, n, r, t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_norm2(r, n, red, partial, st);
}

cudaError_t launch_precond_apply(const double* v, const double* dh, const double* dn, const double* scal,
                                 double clamp, int64_t n, double* out, cudaStream_t st) {
    k_precond_apply<<<grid_for(n, 256, 2048), 256, 0, st>>>(v, dh, dn, scal, clamp, n, out);
    return cudaGetLastError();
}

cudaError_t launch_norm2(const double* x, int64_t n, double* out, double* partial, cudaStream_t st) {
    const int nb = grid_for(n, 256, kRedBlocks);
    k_norm2_partial<<<nb, 256, 0, st>>>(x, n, partial);
    k_multidot_final<<<1, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_inv_sqrt(double* x, int64_t n, const double* nrm2, cudaStream_t st) {
    k_scale_inv_sqrt<<<grid_for(n, 256, 2048), 256, 0, st>>>(x, n, nrm2);
    return cudaGetLastError();
}

cudaError_t launch_axpy_ratio(double* x, const double* y, int64_t n, const double* num, const double* den,
                              double sign, cudaStream_t st) {
    k_axpy_ratio<<<grid_for(n, 256, 2048), 256, 0, st>>>(x, y, n, num, den, sign);
    return cudaGetLastError();
}

cudaError_t launch_xpby_ratio(double* p, const double* r, int64_t n, const double* num, const double* den,
                              cudaStream_t st) {
    k_xpby_ratio<<<grid_for(n, 256, 2048), 256, 0, st>>>(p, r, n, num, den);
    return cudaGetLastError();
}

cudaError_t launch_restart_coef(const double* c_new, const double* c_old, int m, double* Qout, double* scal_out,
                                cudaStream_t st) {
    if (m > kRitzMax) return cudaErrorInvalidValue;
    k_restart_coef<<<1, 32, 0, st>>>(c_new, c_old, m, Qout, scal_out);
    return cudaGetLastError();
}

cudaError_t launch_jacobi_batched(double* mats, double* vscratch, double* evals, const int64_t* mat_off,
                                  const int64_t* val_off, const int* dims, int n_mats, int max_dim, int smem_limit,
                                  int cluster, int* status, cudaStream_t st) {
    if (n_mats <= 0) return cudaSuccess;
    if (max_dim > 512) return cudaErrorInvalidValue;  // pair tables hold at most 256 pairs
    // matrices up to sm_dim run in shared memory (A and V), larger ones in global memory
    const int lim = smem_limit < kJacobiSmemMax ? smem_limit : kJacobiSmemMax;
    const int sm_dim = max_dim < lim ? max_dim : lim;
    const size_t smem = static_cast<size_t>(2) * sm_dim * sm_dim * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_jacobi_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * kJacobiSmemMax * kJacobiSmemMax * static_cast<int>(sizeof(double)));
    if (e != cudaSuccess) return e;
    const bool use_cluster = cluster && max_dim > kJcMin;
    if (use_cluster) {
        // rows of A and V^T per CTA, plus the pair table of the CTA
        const int dmax = max_dim < kJcMax ? max_dim : kJcMax;
        const int rmax = (dmax + kJcC - 1) / kJcC;
        const size_t csm = (static_cast<size_t>(2) * rmax * dmax + 2 * (kJcMax / 2) + 2) * sizeof(double) +
                           (2 * (kJcMax / 2) + 2) * sizeof(int);
        e = cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(csm));
        if (e != cudaSuccess) return e;
        k_jacobi_cluster<<<n_mats * kJcC, 256, csm, st>>>(mats, evals, mat_off, val_off, dims, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_jacobi_batched<<<n_mats, 512, smem, st>>>(mats, vscratch, evals, mat_off, val_off, dims, sm_dim,
                                                use_cluster ? 1 : 0, status);
    return cudaGetLastError();
}

cudaError_t launch_truncate(const double* evals, const int64_t* val_off, const int* dims, const int* label_n,
                            const int* label_tm, int n_labels, int total, int D, double tie_rtol, double drop_abs,
                            int* keep_count, int* keep_total, double* discarded, int* scratch_idx,
                            double* scratch_val, cudaStream_t st) {
    k_truncate<<<1, 1024, 0, st>>>(evals, val_off, dims, label_n, label_tm, n_labels, total, D, tie_rtol, drop_abs,
                                   keep_count, keep_total, discarded, scratch_idx, scratch_val);
    return cudaGetLastError();
}

cudaError_t measure_fp64_peak(double* tflops) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double));
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256, iters = 1 << 14;
    k_fp64_peak<<<blocks, threads>>>(out, 256, 0.999999, 1e-9);  // warm-up
    cudaEventRecord(e0);
    k_fp64_peak<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 8.0 * iters * static_cast<double>(blocks) * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaGetLastError();
}

cudaError_t launch_copy_blocks(const Slots& slots, const CopyBlock* blocks, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_copy_blocks<<<n, 256, 0, st>>>(slots, blocks, n);
    return cudaGetLastError();
}

}  // namespace spmps
