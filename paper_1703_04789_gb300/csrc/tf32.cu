// TF32 / 3xTF32 tensor-core variant of the grouped block GEMM (the bulk H_eff x products).
//
// The blocks of the projected action are small (rows = a label or an N-group of a bond, a few
// to a few tens; K = a label dimension, or the reduction over channels), below the 64/128-row
// tiles of tcgen05, so this variant uses the warp-level m16n8k8 TF32 tensor-core instruction on
// the same task and tile lists as k_gemm_f64: each warp covers its tile's output region in
// 32 x 32 sub-tiles (2 x 4 instructions per k-step of 8), converting the FP64 operands to TF32
// on load.  The 3xTF32 form splits every operand into hi = tf32(x) and lo = tf32(x - hi) and
// accumulates hi*hi + hi*lo + lo*hi in FP32 (about FP32 accuracy); plain TF32 uses hi*hi only.
// Results are written back as FP64.
#include <cuda_runtime.h>

#include "kernels.h"

namespace spmps {

namespace {

__device__ __forceinline__ double* resolve_t(const Slots& S, uint64_t h) {
    return S.p[h >> 56] + static_cast<int64_t>(h & 0x00FFFFFFFFFFFFFFull);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split(double v, uint32_t& hi, uint32_t& lo) {
    const float f = static_cast<float>(v);
    hi = to_tf32(f);
    lo = to_tf32(f - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Output region of a tile: register-tiled shapes of k_gemm_f64, or the explicit extent (shape 5).
__device__ __forceinline__ void region(const GemmTile& t, int& h, int& w) {
    switch (t.shape) {
        case 1: h = 4; w = 64; break;
        case 2: h = 64; w = 4; break;
        case 3: h = 32; w = 8; break;
        case 4: h = 8; w = 32; break;
        case 5:
        case 6: h = t.tm; w = t.tn; break;
        default: h = 16; w = 16; break;
    }
}

template <bool SPLIT3>
__global__ void __launch_bounds__(128) k_gemm_tf32(Slots S, const GemmTask* __restrict__ tasks,
                                                   const GemmSeg* __restrict__ segs, const GemmTile* __restrict__ tiles,
                                                   const int* __restrict__ cmaps, int n_tiles) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_tiles) return;
    const GemmTile tl = tiles[warp];
    const GemmTask T = tasks[tl.task];
    int rh, rw;
    region(tl, rh, rw);
    const int rmax = min(T.M, tl.m0 + rh), cmax = min(T.N, tl.n0 + rw);
    const int g = lane >> 2, q = lane & 3;
    double* C = resolve_t(S, T.c);
    const int* cm = T.cmap >= 0 ? cmaps + T.cmap : nullptr;
    for (int sm0 = tl.m0; sm0 < rmax; sm0 += 32)
        for (int sn0 = tl.n0; sn0 < cmax; sn0 += 32) {
            float acc[2][4][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
            const int mt = (min(32, rmax - sm0) + 15) / 16;  // 1 or 2 row tiles
            const int nt = (min(32, cmax - sn0) + 7) / 8;    // 1..4 column tiles
            for (int sgi = 0; sgi < T.nseg; ++sgi) {
                const GemmSeg sg = segs[T.seg0 + sgi];
                const double* __restrict__ A = resolve_t(S, sg.a);
                const double* __restrict__ B = resolve_t(S, sg.b);
                for (int k0 = 0; k0 < sg.K; k0 += 8) {
                    uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int r = sm0 + 16 * i + g + ((e & 1) ? 8 : 0);
                            const int k = k0 + q + ((e & 2) ? 4 : 0);
                            const double v = (i < mt && r < rmax && k < sg.K)
                                                 ? __ldg(A + static_cast<int64_t>(r) * sg.a_rs + static_cast<int64_t>(k) * sg.a_cs)
                                                 : 0.0;
                            split(v, ah[i][e], al[i][e]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int k = k0 + q + (e ? 4 : 0);
                            const int c = sn0 + 8 * j + g;
                            const double v = (j < nt && c < cmax && k < sg.K)
                                                 ? __ldg(B + static_cast<int64_t>(k) * sg.b_rs + static_cast<int64_t>(c) * sg.b_cs)
                                                 : 0.0;
                            split(v, bh[j][e], bl[j][e]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        if (i >= mt) continue;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (j >= nt) continue;
                            mma_tf32(acc[i][j], ah[i], bh[j]);
                            if (SPLIT3) {
                                mma_tf32(acc[i][j], ah[i], bl[j]);
                                mma_tf32(acc[i][j], al[i], bh[j]);
                            }
                        }
                    }
                }
            }
            // D fragment: (row g, cols 2q, 2q+1) and (row g+8, same cols) of each 16 x 8 tile
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i >= mt) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j >= nt) continue;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = sm0 + 16 * i + g + ((e & 2) ? 8 : 0);
                        const int c = sn0 + 8 * j + 2 * q + (e & 1);
                        if (r < rmax && c < cmax) {
                            const int64_t cc = cm ? cm[c] : c;
                            C[static_cast<int64_t>(r) * T.ldc + cc] = static_cast<double>(acc[i][j][e]);
                        }
                    }
                }
            }
        }
}

// ---- pre-split operands -----------------------------------------------------------------------
// The conversion FP64 -> FP32 -> (hi, lo) runs once per operand buffer (environment after its
// update, x and the phase-B output once per action) instead of once per fragment load: on this
// part the FP64 conversions run at the FP64 rate, so converting inside the GEMM made it as slow
// as the FP64 kernel.  hi = tf32(float(v)), lo = tf32(float(v) - hi), stored as one float2.
__global__ void __launch_bounds__(256) k_split_tf32(const double* __restrict__ x, int64_t n, float2* __restrict__ out) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint32_t hi, lo;
        split(x[i], hi, lo);
        out[i] = make_float2(__uint_as_float(hi), __uint_as_float(lo));
    }
}

__device__ __forceinline__ const float2* resolve_s(const SlotsF& F, uint64_t h) {
    return F.p[h >> 56] + static_cast<int64_t>(h & 0x00FFFFFFFFFFFFFFull);
}

template <bool SPLIT3>
__global__ void __launch_bounds__(128, 4) k_gemm_tf32s(Slots S, SlotsF F, const GemmTask* __restrict__ tasks,
                                                    const GemmSeg* __restrict__ segs, const GemmTile* __restrict__ tiles,
                                                    const int* __restrict__ cmaps, int n_tiles) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_tiles) return;
    const GemmTile tl = tiles[warp];
    const GemmTask T = tasks[tl.task];
    int rh, rw;
    region(tl, rh, rw);
    const int rmax = min(T.M, tl.m0 + rh), cmax = min(T.N, tl.n0 + rw);
    const int g = lane >> 2, q = lane & 3;
    double* C = resolve_t(S, T.c);
    const int* cm = T.cmap >= 0 ? cmaps + T.cmap : nullptr;
    const float2 zero = make_float2(0.0f, 0.0f);
    for (int sm0 = tl.m0; sm0 < rmax; sm0 += 32)
        for (int sn0 = tl.n0; sn0 < cmax; sn0 += 32) {
            float acc[2][4][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
            const int mt = (min(32, rmax - sm0) + 15) / 16;
            const int nt = (min(32, cmax - sn0) + 7) / 8;
            for (int sgi = 0; sgi < T.nseg; ++sgi) {
                const GemmSeg sg = segs[T.seg0 + sgi];
                const float2* __restrict__ A = resolve_s(F, sg.a);
                const float2* __restrict__ B = resolve_s(F, sg.b);
                for (int k0 = 0; k0 < sg.K; k0 += 8) {
                    uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int r = sm0 + 16 * i + g + ((e & 1) ? 8 : 0);
                            const int k = k0 + q + ((e & 2) ? 4 : 0);
                            const float2 v = (i < mt && r < rmax && k < sg.K)
                                                 ? A[static_cast<int64_t>(r) * sg.a_rs + static_cast<int64_t>(k) * sg.a_cs]
                                                 : zero;
                            ah[i][e] = __float_as_uint(v.x);
                            al[i][e] = __float_as_uint(v.y);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int k = k0 + q + (e ? 4 : 0);
                            const int c = sn0 + 8 * j + g;
                            const float2 v = (j < nt && c < cmax && k < sg.K)
                                                 ? B[static_cast<int64_t>(k) * sg.b_rs + static_cast<int64_t>(c) * sg.b_cs]
                                                 : zero;
                            bh[j][e] = __float_as_uint(v.x);
                            bl[j][e] = __float_as_uint(v.y);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        if (i >= mt) continue;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (j >= nt) continue;
                            mma_tf32(acc[i][j], ah[i], bh[j]);
                            if (SPLIT3) {
                                mma_tf32(acc[i][j], ah[i], bl[j]);
                                mma_tf32(acc[i][j], al[i], bh[j]);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (i >= mt) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j >= nt) continue;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = sm0 + 16 * i + g + ((e & 2) ? 8 : 0);
                        const int c = sn0 + 8 * j + 2 * q + (e & 1);
                        if (r < rmax && c < cmax) {
                            const int64_t cc = cm ? cm[c] : c;
                            C[static_cast<int64_t>(r) * T.ldc + cc] = static_cast<double>(acc[i][j][e]);
                        }
                    }
                }
            }
        }
}

}  // namespace

cudaError_t launch_gemm_tf32(const Slots& slots, const GemmTask* tasks, const GemmSeg* segs, const GemmTile* tiles,
                             const int* cmaps, int n_tiles, int split3, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const int grid = (n_tiles + 3) / 4;
    if (split3)
        k_gemm_tf32<true><<<grid, 128, 0, st>>>(slots, tasks, segs, tiles, cmaps, n_tiles);
    else
        k_gemm_tf32<false><<<grid, 128, 0, st>>>(slots, tasks, segs, tiles, cmaps, n_tiles);
    return cudaGetLastError();
}


cudaError_t launch_split_tf32(const double* x, int64_t n, float2* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_split_tf32<<<static_cast<int>(blocks), 256, 0, st>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tf32s(const Slots& slots, const SlotsF& split, const GemmTask* tasks, const GemmSeg* segs,
                              const GemmTile* tiles, const int* cmaps, int n_tiles, int split3, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const int grid = (n_tiles + 3) / 4;
    if (split3)
        k_gemm_tf32s<true><<<grid, 128, 0, st>>>(slots, split, tasks, segs, tiles, cmaps, n_tiles);
    else
        k_gemm_tf32s<false><<<grid, 128, 0, st>>>(slots, split, tasks, segs, tiles, cmaps, n_tiles);
    return cudaGetLastError();
}

}  // namespace spmps
