// Stacked block GEMMs on tcgen05 (see tc_gemm.h): host stacking of the task lists and the kernel.
#include <map>

#include "tc_gemm.h"

namespace spmps {

bool build_tc_plan(const GemmPlan& G, const std::vector<int>& task_rng, int n_ranges, int nt, TcPlan& P) {
    P.clear();
    P.nt = nt;
    P.unit_rng.assign(n_ranges + 1, 0);
    for (int r = 0; r < n_ranges; ++r) {
        P.unit_rng[r] = static_cast<int>(P.units.size());
        std::map<int, std::vector<int>> by_key;
        for (int t = task_rng[r]; t < task_rng[r + 1]; ++t) by_key[G.tasks[t].key].push_back(t);
        for (const auto& kv : by_key) {
            const std::vector<int>& ts = kv.second;
            const GemmTask& T0 = G.tasks[ts[0]];
            TcStack S{};
            S.N = T0.N;
            S.cmap = T0.cmap;
            S.row0 = static_cast<int>(P.rows.size());
            S.seg0 = static_cast<int>(P.segs.size());
            // the union of the tasks' K segments, identified by their B operand
            std::map<uint64_t, int> seg_of;
            for (int t : ts) {
                const GemmTask& T = G.tasks[t];
                if (T.N != S.N || T.cmap != S.cmap) return false;
                for (int q = 0; q < T.nseg; ++q) {
                    const GemmSeg& sg = G.segs[T.seg0 + q];
                    if (sg.a_cs != 1 || sg.K <= 0) return false;
                    auto it = seg_of.find(sg.b);
                    if (it == seg_of.end()) {
                        seg_of.emplace(sg.b, static_cast<int>(P.segs.size()) - S.seg0);
                        TcSeg ts2{};
                        ts2.b = sg.b;
                        ts2.K = sg.K;
                        ts2.b_ks = sg.b_rs;
                        ts2.b_ns = sg.b_cs;
                        P.segs.push_back(ts2);
                    } else if (P.segs[S.seg0 + it->second].K != sg.K) {
                        return false;
                    }
                }
            }
            S.nseg = static_cast<int>(P.segs.size()) - S.seg0;
            S.atab0 = static_cast<int64_t>(P.atab.size());
            for (int t : ts) {
                const GemmTask& T = G.tasks[t];
                std::vector<uint64_t> aseg(S.nseg, kNoOperand);
                std::vector<int> ars(S.nseg, 0);
                for (int q = 0; q < T.nseg; ++q) {
                    const GemmSeg& sg = G.segs[T.seg0 + q];
                    const int s = seg_of[sg.b];
                    aseg[s] = sg.a;
                    ars[s] = sg.a_rs;
                }
                for (int i = 0; i < T.M; ++i) {
                    TcRow row{};
                    row.c = T.c + static_cast<uint64_t>(static_cast<int64_t>(i) * T.ldc);
                    P.rows.push_back(row);
                    for (int s = 0; s < S.nseg; ++s)
                        P.atab.push_back(aseg[s] == kNoOperand ? kNoOperand
                                                               : aseg[s] + static_cast<uint64_t>(static_cast<int64_t>(i) * ars[s]));
                }
            }
            S.nrows = static_cast<int>(P.rows.size()) - S.row0;
            const int si = static_cast<int>(P.stacks.size());
            P.stacks.push_back(S);
            for (int m0 = 0; m0 < S.nrows; m0 += 128)
                for (int n0 = 0; n0 < S.N; n0 += nt) P.units.push_back(make_int4(si, m0, n0, 0));
        }
    }
    P.unit_rng[n_ranges] = static_cast<int>(P.units.size());
    P.ok = true;
    return true;
}

namespace {

constexpr int kTileM = 128;
constexpr int kTileK = 32;                        // K per shared-memory stage (4 MMAs of K = 8)
constexpr int kTileBytesA = kTileM * kTileK * 4;  // one TF32 plane of A
constexpr int kMaxNt = 128;
constexpr int kDefaultWaitPolls = 1 << 24;
constexpr int kCtrlBytes = 1024;  // mbarrier, tensor-memory address and flags, padded to the tile alignment
constexpr int kTileBytes = 2 * kTileBytesA + 2 * kMaxNt * kTileK * 4;
constexpr int kStageBytes = kTileM * (kMaxNt + 1) * 4;  // FP32 output stage (padded rows)
constexpr size_t kSmemBytes = kCtrlBytes + (kTileBytes > kStageBytes ? kTileBytes : kStageBytes);

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// K-major no-swizzle layout of a 32-wide K stage: core matrices of 8 rows x 16 bytes (4 TF32),
// the 8 K-cores of an 8-row group contiguous (128 bytes apart), row groups 1024 bytes apart.
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
    return static_cast<uint32_t>(((row >> 3) * 8 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t kdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr & 0x3FFFF) >> 4);
    d |= static_cast<uint64_t>(128 >> 4) << 16;   // leading byte offset: next core along K
    d |= static_cast<uint64_t>(1024 >> 4) << 32;  // stride byte offset: next 8-row group
    d |= static_cast<uint64_t>(1) << 46;          // descriptor version
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint32_t poll(uint32_t mbar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity));
    return done;
}

template <bool SPLIT3>
__global__ void __launch_bounds__(128, 3) k_gemm_tc(Slots S, SlotsF F, const TcStack* __restrict__ stacks,
                                                   const TcRow* __restrict__ rows, const TcSeg* __restrict__ segs,
                                                   const uint64_t* __restrict__ atab, const int* __restrict__ cmaps,
                                                   const int4* __restrict__ units, int u0, int nt,
                                                   int* __restrict__ err, int wait_polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // control words first, then the operand tiles (1024-aligned); after the K loop the tiles'
    // space holds the FP32 output stage of the epilogue
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    unsigned char* Ahi = smem + kCtrlBytes;
    unsigned char* Alo = Ahi + kTileBytesA;
    unsigned char* Bhi = Alo + kTileBytesA;
    unsigned char* Blo = Bhi + kMaxNt * kTileK * 4;
    volatile uint32_t* flag = tslot + 1;    // outcome of thread 0's bounded wait
    volatile uint32_t* issued = tslot + 2;  // whether any MMA wrote the accumulator
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 U = units[u0 + blockIdx.x];
    const TcStack st = stacks[U.x];
    const int m0 = U.y, n0 = U.z;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)), "r"(nt));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *issued = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    // F32 accumulator, TF32 A and B (format 2), both K-major, N = nt, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(nt >> 3) << 17) |
                           (static_cast<uint32_t>(kTileM >> 4) << 24);
    const int row = m0 + tid;
    const bool rvalid = row < st.nrows;
    const float2 zero = make_float2(0.0f, 0.0f);
    const int nb = nt * kTileK / 128;  // B elements per thread per stage (8, 16 or 32)
    // K stages run over the segments in order; the operands of stage c + 1 are loaded into
    // registers while the MMAs of stage c run
    float2 ra[kTileK], rb[kMaxNt * kTileK / 128];
    int seg = 0, k0 = 0;       // stage being loaded
    auto load_stage = [&](int s, int kb) {
        const TcSeg sg = segs[st.seg0 + s];
        const int kc = min(kTileK, sg.K - kb);
        const uint64_t ah = rvalid ? atab[st.atab0 + static_cast<int64_t>(row) * st.nseg + s] : kNoOperand;
        const float2* __restrict__ A =
            ah == kNoOperand ? nullptr : F.p[ah >> 56] + static_cast<int64_t>(ah & 0x00FFFFFFFFFFFFFFull);
        const float2* __restrict__ B = F.p[sg.b >> 56] + static_cast<int64_t>(sg.b & 0x00FFFFFFFFFFFFFFull);
#pragma unroll
        for (int k = 0; k < kTileK; ++k) ra[k] = (A && k < kc) ? A[kb + k] : zero;
        if (sg.b_ks == 1) {  // unit stride along K: lanes along K
#pragma unroll
            for (int q = 0; q < kMaxNt * kTileK / 128; ++q) {
                const int e = q * 128 + tid, n = e / kTileK, k = e % kTileK, col = n0 + n;
                rb[q] = (q < nb && col < st.N && k < kc)
                            ? B[static_cast<int64_t>(kb + k) + static_cast<int64_t>(col) * sg.b_ns]
                            : zero;
            }
        } else {  // lanes along N
#pragma unroll
            for (int q = 0; q < kMaxNt * kTileK / 128; ++q) {
                const int e = q * 128 + tid, n = e % nt, k = e / nt, col = n0 + n;
                rb[q] = (q < nb && col < st.N && k < kc)
                            ? B[static_cast<int64_t>(kb + k) * sg.b_ks + static_cast<int64_t>(col) * sg.b_ns]
                            : zero;
            }
        }
    };
    auto store_stage = [&](int b_ks) {
#pragma unroll
        for (int k = 0; k < kTileK; ++k) {
            const uint32_t o = kmajor_off(tid, k);
            *reinterpret_cast<float*>(Ahi + o) = ra[k].x;
            *reinterpret_cast<float*>(Alo + o) = ra[k].y;
        }
#pragma unroll
        for (int q = 0; q < kMaxNt * kTileK / 128; ++q) {
            if (q >= nb) break;
            const int e = q * 128 + tid;
            const int n = b_ks == 1 ? e / kTileK : e % nt, k = b_ks == 1 ? e % kTileK : e / nt;
            const uint32_t o = kmajor_off(n, k);
            *reinterpret_cast<float*>(Bhi + o) = rb[q].x;
            *reinterpret_cast<float*>(Blo + o) = rb[q].y;
        }
    };
    uint32_t phase = 0;
    bool failed = false, first = true;
    if (st.nseg > 0) load_stage(0, 0);
    while (seg < st.nseg && !failed) {
        const TcSeg sg = segs[st.seg0 + seg];
        const int kc = min(kTileK, sg.K - k0);
        store_stage(sg.b_ks);
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah0 = saddr(Ahi), al0 = saddr(Alo), bh0 = saddr(Bhi), bl0 = saddr(Blo);
            const int nk = (kc + 7) / 8;
            for (int kk = 0; kk < nk; ++kk) {
                const uint32_t ko = static_cast<uint32_t>(kk) * 256;
                mma_tf32(tmem, kdesc(ah0 + ko), kdesc(bh0 + ko), idesc, first ? 0u : 1u);
                first = false;
                if (SPLIT3) {
                    mma_tf32(tmem, kdesc(ah0 + ko), kdesc(bl0 + ko), idesc, 1u);
                    mma_tf32(tmem, kdesc(al0 + ko), kdesc(bh0 + ko), idesc, 1u);
                }
            }
            *issued = 1;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                saddr(mbar)));
        }
        // next stage: advance and load its operands while the MMAs run
        k0 += kTileK;
        if (k0 >= sg.K) {
            ++seg;
            k0 = 0;
        }
        if (seg < st.nseg) load_stage(seg, k0);
        if (tid == 0) {
            // the stage buffers are reused by the next K stage: wait for these MMAs
            *flag = poll(saddr(mbar), phase, wait_polls);
            if (!*flag) atomicExch(err, 1);
        }
        __syncthreads();
        if (!*flag) failed = true;
        phase ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!failed) {
        // epilogue: warp w reads TMEM lanes 32w .. 32w + 31 (tile rows) into a shared-memory stage
        // (the operand buffers are free now), then every warp writes whole rows with its lanes
        // along the columns, so the stores of a row are contiguous
        float* stage = reinterpret_cast<float*>(smem + kCtrlBytes);
        const int ld = nt + 1;
        const bool any = *issued != 0;
        for (int cb = 0; cb < nt; cb += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(cb);
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
            for (int q = 0; q < 32; ++q) stage[(warp * 32 + lane) * ld + cb + q] = any ? __uint_as_float(v[q]) : 0.0f;
        }
        __syncthreads();
        const int* cm = st.cmap >= 0 ? cmaps + st.cmap : nullptr;
        const int ncols = min(nt, st.N - n0);
        for (int rr = warp; rr < kTileM; rr += 4) {
            const int r = m0 + rr;
            if (r >= st.nrows) break;
            const uint64_t c = rows[st.row0 + r].c;
            double* C = S.p[c >> 56] + static_cast<int64_t>(c & 0x00FFFFFFFFFFFFFFull);
            for (int q = lane; q < ncols; q += 32) {
                const int n = n0 + q;
                C[cm ? cm[n] : n] = static_cast<double>(stage[rr * ld + q]);
            }
        }
    } else if (tid == 0) {
        // give the MMAs in flight a further bounded wait (default limit) before releasing the memory
        poll(saddr(mbar), phase ^ 1u, kDefaultWaitPolls);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nt));
    }
}

}  // namespace

cudaError_t launch_gemm_tc(const Slots& slots, const SlotsF& split, const TcStack* stacks, const TcRow* rows,
                           const TcSeg* segs, const uint64_t* atab, const int* cmaps, const int4* units, int u0,
                           int u1, int nt, int split3, int* err, int wait_polls, cudaStream_t st) {
    if (u1 <= u0) return cudaSuccess;
    if (nt != 32 && nt != 64 && nt != 128) return cudaErrorInvalidValue;
    if (wait_polls <= 0) wait_polls = kDefaultWaitPolls;
    const size_t smem = kSmemBytes;
    static int attr_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    const int grid = u1 - u0;
    if (split3)
        k_gemm_tc<true><<<grid, 128, smem, st>>>(slots, split, stacks, rows, segs, atab, cmaps, units, u0, nt, err,
                                                 wait_polls);
    else
        k_gemm_tc<false><<<grid, 128, smem, st>>>(slots, split, stacks, rows, segs, atab, cmaps, units, u0, nt, err,
                                                  wait_polls);
    return cudaGetLastError();
}

}  // namespace spmps
