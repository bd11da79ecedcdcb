// Throughput microbenchmarks of the TF32 tensor-core paths of this device, the roofline
// denominators of the reduced-precision action: the warp-level mma.sync.m16n8k8 TF32 instruction
// (used by the block GEMMs) and tcgen05.mma kind::tf32 (M = 128, N = 256, K = 8, accumulator in
// tensor memory), each on a chosen number of SMs, one CTA per SM.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/spmps.h"

namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Independent accumulator chains per warp: 8 m16n8k8 MMAs in flight per loop step.
__global__ void __launch_bounds__(1024) k_mma_sync_tf32_peak(int iters, float* out) {
    uint32_t a[4], b[2];
    for (int q = 0; q < 4; ++q) a[q] = __float_as_uint(1e-3f * (threadIdx.x + q));
    for (int q = 0; q < 2; ++q) b[q] = __float_as_uint(1e-3f * (threadIdx.x - q));
    float acc[8][4];
    for (int c = 0; c < 8; ++c)
        for (int q = 0; q < 4; ++q) acc[c][q] = 0.0f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0.0f;
    for (int c = 0; c < 8; ++c)
        for (int q = 0; q < 4; ++q) s += acc[c][q];
    if (s == 1234.5f) out[0] = s;  // keeps the chains alive
}

// INT8 (s8 x s8 -> s32) warp-level MMAs, 8 independent chains per warp: the integer rate that an
// Ozaki-style FP64 emulation (exact integer products of split mantissas) would run at.
__global__ void __launch_bounds__(1024) k_mma_sync_s8_peak(int iters, int* out) {
    uint32_t a[4], b[2];
    for (int q = 0; q < 4; ++q) a[q] = 0x01020304u * (threadIdx.x + q + 1);
    for (int q = 0; q < 2; ++q) b[q] = 0x01010101u * (threadIdx.x + q + 1);
    int acc[8][4];
    for (int c = 0; c < 8; ++c)
        for (int q = 0; q < 4; ++q) acc[c][q] = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
    for (int c = 0; c < 8; ++c)
        for (int q = 0; q < 4; ++q) s += acc[c][q];
    if (s == 12345) out[0] = s;
}

constexpr int kPeakM = 128, kPeakN = 256, kPeakK = 32;  // smem tiles: A 128 x 32, B 256 x 32 (tf32)
constexpr int kPeakSmem = (kPeakM + kPeakN) * kPeakK * 4 + 64;

// No-swizzle K-major shared-memory descriptor: core matrices of 8 rows x 16 bytes, `lbo` bytes
// apart along K and `sbo` bytes apart between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFF) >> 4);
    d |= static_cast<uint64_t>((lbo & 0x3FFFF) >> 4) << 16;
    d |= static_cast<uint64_t>((sbo & 0x3FFFF) >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

// One thread issues iters x 4 MMAs (K = 32 per round) into a 128 x 256 FP32 accumulator in tensor
// memory; a bounded wait for their completion sets *status on giving up.
__global__ void __launch_bounds__(128, 1) k_tcgen05_tf32_peak(int iters, float* out, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float* tiles = reinterpret_cast<float*>(smem);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + (kPeakM + kPeakN) * kPeakK * 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    volatile uint32_t* ok = tslot + 1;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int e = tid; e < (kPeakM + kPeakN) * kPeakK; e += blockDim.x) tiles[e] = 1e-3f * static_cast<float>(e & 63);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(kPeakN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    // F32 accumulate, TF32 A and B (format 2), both K-major, N = 256, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((kPeakN >> 3) << 17) | ((kPeakM >> 4) << 24);
    if (tid == 0) {
        const uint32_t a0 = smem_addr(tiles), b0 = smem_addr(tiles + kPeakM * kPeakK);
        const uint32_t sbo = (kPeakK / 4) * 128;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int kk = 0; kk < kPeakK / 8; ++kk) {
                const uint64_t da = smem_desc(a0 + kk * 256, 128, sbo);
                const uint64_t db = smem_desc(b0 + kk * 256, 128, sbo);
                const uint32_t acc = (it | kk) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(mbar)));
        uint32_t done = 0;
        for (int it = 0; it < (1 << 24) && !done; ++it)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_addr(mbar)), "r"(0));
        *ok = done;
        if (!done) atomicExch(status, 1);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (*ok && warp == 0) {
        uint32_t v;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(tmem));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (__uint_as_float(v) == 1234.5f) out[0] = 1.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPeakN));
    }
}

}  // namespace

extern "C" spmps_status spmps_device_tf32_peak(int device, int kind, int sms, double* tflops) {
    if (!tflops || kind < 0 || kind > 2 || sms < 0) return SPMPS_ERR_BAD_INPUT;
    if (cudaSetDevice(device) != cudaSuccess) return SPMPS_ERR_CUDA;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SPMPS_ERR_CUDA;
    const int blocks = sms == 0 || sms > nsm ? nsm : sms;
    float* out = nullptr;
    int* status = nullptr;
    if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) return SPMPS_ERR_OOM;
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) {
        cudaFree(out);
        return SPMPS_ERR_OOM;
    }
    cudaMemset(status, 0, sizeof(int));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double flops = 0.0;
    float ms = 0.0f;
    cudaError_t e = cudaSuccess;
    if (kind == 0) {
        const int threads = 1024, iters = 1 << 13;  // one CTA of 32 warps per SM
        k_mma_sync_tf32_peak<<<blocks, threads>>>(64, out);
        cudaEventRecord(e0);
        k_mma_sync_tf32_peak<<<blocks, threads>>>(iters, out);
        cudaEventRecord(e1);
        flops = 2.0 * 16 * 8 * 8 * 8.0 * iters * (threads / 32) * static_cast<double>(blocks);
    } else if (kind == 2) {
        const int threads = 1024, iters = 1 << 13;
        k_mma_sync_s8_peak<<<blocks, threads>>>(64, reinterpret_cast<int*>(out));
        cudaEventRecord(e0);
        k_mma_sync_s8_peak<<<blocks, threads>>>(iters, reinterpret_cast<int*>(out));
        cudaEventRecord(e1);
        flops = 2.0 * 16 * 8 * 32 * 8.0 * iters * (threads / 32) * static_cast<double>(blocks);
    } else {
        const int iters = 1 << 12;
        e = cudaFuncSetAttribute(k_tcgen05_tf32_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem);
        if (e == cudaSuccess) {
            k_tcgen05_tf32_peak<<<blocks, 128, kPeakSmem>>>(16, out, status);
            cudaEventRecord(e0);
            k_tcgen05_tf32_peak<<<blocks, 128, kPeakSmem>>>(iters, out, status);
            cudaEventRecord(e1);
            flops = 2.0 * kPeakM * kPeakN * kPeakK * static_cast<double>(iters) * blocks;
        }
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(status);
    if (e != cudaSuccess) return SPMPS_ERR_CUDA;
    if (bad) return SPMPS_ERR_TIMEOUT;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return SPMPS_OK;
}
