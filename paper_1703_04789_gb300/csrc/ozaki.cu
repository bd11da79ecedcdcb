// FP64-accurate stacked block GEMMs on the tensor cores (see tc_gemm.h, launch_gemm_oz).
//
// The FP64 products are split into exact products of 8-bit integer digits (the error-free
// splitting of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012; with an FP32 tensor-core
// accumulator kept exact by bounding the partial sums below 2^24, as in Mukunoki, Ozaki, Ogita and
// Imamura, ISC 2020).  Per K stage of 32:
//
//   1. row i of A gets the exponent field E_i of its largest entry in the stage, column j of B
//      likewise E_j; every entry becomes F = floor(|a| 2^(56 - e)) < 2^56 (e = E - 1022, the
//      frexp exponent of the line maximum; zero and subnormal entries give 0), cut into seven
//      base-256 digits with the entry's sign, each an exact FP16 value;
//   2. for every level l = p + q = 2 .. 9, the digit products a_(p) b_(q) with p + q = l are summed
//      by tcgen05.mma kind::f16 into one FP32 accumulator in tensor memory: at most 7 pairs of
//      products below 2^16 over 32 terms, |v_l| < 32 * 7 * 255^2 < 2^24, so every partial sum is an
//      exactly representable integer;
//   3. each thread reads its row's 8 level sums for its 16 of the tile's 32 columns and forms the integer
//      T = sum_{l <= 7} v_l 2^(56 - 8l) + floor(v_8 2^-8) + floor(v_9 2^-16) (|T| < 2^62), and adds
//      T 2^(e_i + e_j - 56) to its FP64 accumulators.
//
// Levels above 9 are dropped (below 5 * 32 * 2^-64 of 2^(e_i + e_j)); with the digit truncation
// (2^-56 of the line maximum per entry) the error of a stage is of the order of 32 * 2^-55
// max|a_i.| max|b_.j|, the size of FP64 rounding in the same stage.
#include "tc_gemm.h"

#include <cuda_fp16.h>

#include <type_traits>

namespace spmps {

namespace {

constexpr int kOzM = 128;      // rows per CTA tile (one per thread)
constexpr int kOzN = 32;       // columns per CTA tile
constexpr int kOzK = 32;       // K per stage (two MMAs of K = 16)
constexpr int kSlices = 7;     // digits per entry
constexpr int kLevels = 8;     // levels l = 2 .. 9
constexpr uint32_t kTmemCols = kLevels * kOzN;  // 256: one 32-column accumulator per level
constexpr int kDefaultWaitPolls = 1 << 24;
constexpr int kPlaneA = kOzM * kOzK * 2;  // one FP16 digit plane of A (8 KB)
constexpr int kPlaneB = kOzN * kOzK * 2;  // one FP16 digit plane of B (2 KB)
constexpr int kOzThreads = 256;  // two threads per tile row
// control block: mbarrier, tensor-memory address and flag at 0, column exponent fields at 128, the
// row exponent fields of the two K halves at 256
constexpr int kOffColE = 128;
constexpr int kOffRowE = 256;
constexpr int kOffPlanesA = 1024;
constexpr int kOffPlanesB = kOffPlanesA + kSlices * kPlaneA;
constexpr int kOffRawA = kOffPlanesB + kSlices * kPlaneB;  // FP64 A stage, 128 x 32, swizzled
constexpr int kOffRawB = kOffRawA + kOzM * kOzK * 8;        // FP64 B stage, 32 x 32, swizzled
constexpr size_t kOzSmem = kOffRawB + kOzN * kOzK * 8;
static_assert(kOffRowE + 2 * kOzM * 2 <= kOffPlanesA, "exponent fields overlap the digit planes");

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// K-major no-swizzle layout of a 16-bit operand with a 32-wide K stage: core matrices of 8 rows x
// 16 bytes (8 elements), the 4 K-cores of an 8-row group contiguous (128 bytes apart), row groups
// 512 bytes apart.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
    return static_cast<uint32_t>(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t desc(uint32_t addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr & 0x3FFFF) >> 4);
    d |= static_cast<uint64_t>(128 >> 4) << 16;  // leading byte offset: next core along K
    d |= static_cast<uint64_t>(512 >> 4) << 32;  // stride byte offset: next 8-row group
    d |= static_cast<uint64_t>(1) << 46;         // descriptor version
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
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

__device__ __forceinline__ void cp_async8(uint32_t dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src));
}

__device__ __forceinline__ int expo(double v) { return static_cast<int>((__double_as_longlong(v) >> 52) & 0x7FF); }

// Fixed-point magnitude F = floor(|v| 2^(56 - e)) against the line's exponent field E (e = E - 1022).
__device__ __forceinline__ uint64_t fixed56(double v, int E) {
    const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(v));
    const int ev = static_cast<int>((bits >> 52) & 0x7FF);
    if (ev == 0) return 0;  // zero or subnormal
    const uint64_t mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ev - E + 3;  // <= 3 because ev <= E
    return sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
}

// Signed digit p (0 = most significant, byte 6 - p of F) of NV (8 or 4) entries as FP16, packed
// along K into 2 NV bytes: the two bytes of a pair are moved into the low bytes of two halves (byte permute), the
// halves become 1024 + d (FP16 has unit spacing on [1024, 2048)), and s (1024 + d) - 1024 s = s d
// in one exact FP16 fma, s = +-1 the entries' signs.
template <int NV>
__device__ __forceinline__ typename std::conditional<NV == 8, uint4, uint2>::type digit_plane(
    const uint32_t Flo[NV], const uint32_t Fhi[NV], const __half2 sg[NV / 2], const __half2 off[NV / 2], int p) {
    const int b = 6 - p;  // byte of F
    uint32_t w[NV / 2];
#pragma unroll
    for (int c = 0; c < NV; c += 2) {
        const uint32_t x = b >= 4 ? Fhi[c] : Flo[c], y = b >= 4 ? Fhi[c + 1] : Flo[c + 1];
        const uint32_t pr = __byte_perm(x, y, static_cast<uint32_t>((b & 3) | ((4 + (b & 3)) << 4)));
        const uint32_t v = (pr & 0x000000FFu) | ((pr & 0x0000FF00u) << 8) | 0x64006400u;
        const __half2 h = __hfma2(*reinterpret_cast<const __half2*>(&v), sg[c >> 1], off[c >> 1]);
        w[c >> 1] = *reinterpret_cast<const uint32_t*>(&h);
    }
    if constexpr (NV == 8)
        return make_uint4(w[0], w[1], w[2], w[3]);
    else
        return make_uint2(w[0], w[1]);
}

// Signs of NV entries as FP16 pairs (s, and -1024 s for the digit fma).
template <int NV>
__device__ __forceinline__ void pair_signs(const double v[NV], __half2 sg[NV / 2], __half2 off[NV / 2]) {
#pragma unroll
    for (int c = 0; c < NV; c += 2) {
        const uint32_t s0 = static_cast<uint32_t>(static_cast<unsigned long long>(__double_as_longlong(v[c])) >> 63);
        const uint32_t s1 = static_cast<uint32_t>(static_cast<unsigned long long>(__double_as_longlong(v[c + 1])) >> 63);
        const uint32_t one = 0x3C003C00u | (s0 << 15) | (s1 << 31);        // (+-1, +-1)
        const uint32_t k1024 = 0xE400E400u ^ ((s0 << 15) | (s1 << 31));    // (-+1024, -+1024)
        sg[c >> 1] = *reinterpret_cast<const __half2*>(&one);
        off[c >> 1] = *reinterpret_cast<const __half2*>(&k1024);
    }
}

// One CTA of 256 threads per 128 x 32 tile: warp w serves tensor-memory lanes 32 (w mod 4) .. + 31
// (tile rows) and the column half (K half while splitting) w / 4, so every row has two threads.
// Two CTAs per SM (shared memory and tensor memory each allow two): one CTA's copies and digit
// splitting overlap the other's MMAs and combination.
__global__ void __launch_bounds__(kOzThreads, 2) k_gemm_oz(Slots S, const TcStack* __restrict__ stacks,
                                                          const TcRow* __restrict__ rows, const TcSeg* __restrict__ segs,
                                                          const uint64_t* __restrict__ atab, const int* __restrict__ cmaps,
                                                          const int4* __restrict__ units, int u0, int* __restrict__ err,
                                                          int wait_polls) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    volatile uint32_t* flag = tslot + 1;
    int* colE = reinterpret_cast<int*>(smem + kOffColE);
    short* rowE2 = reinterpret_cast<short*>(smem + kOffRowE);  // [K half][row]
    unsigned char* planesA = smem + kOffPlanesA;
    unsigned char* planesB = smem + kOffPlanesB;
    double* rawA = reinterpret_cast<double*>(smem + kOffRawA);
    double* rawB = reinterpret_cast<double*>(smem + kOffRawB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, h = warp >> 2;
    const int r = q * 32 + lane;  // tile row of this thread
    const int4 U = units[u0 + blockIdx.x];
    const TcStack st = stacks[U.x];
    const int m0 = U.y, n0 = U.z;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tslot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    // F32 accumulator, F16 A and B (format 0), both K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | (static_cast<uint32_t>(kOzN >> 3) << 17) | (static_cast<uint32_t>(kOzM >> 4) << 24);
    const int row = m0 + r;
    const bool rvalid = row < st.nrows;
    // raw FP64 operands of a stage into shared memory with asynchronous copies (zeros outside)
    auto issue_loads = [&](int s, int kb) {
        const TcSeg sg = segs[st.seg0 + s];
        const int kc = min(kOzK, sg.K - kb);
        const uint64_t ah = rvalid ? atab[st.atab0 + static_cast<int64_t>(row) * st.nseg + s] : kNoOperand;
        const double* arow = ah == kNoOperand ? nullptr : S.p[ah >> 56] + static_cast<int64_t>(ah & 0x00FFFFFFFFFFFFFFull);
        // A: warp w copies rows 32 q + 16 h .. + 15 (their pointers sit in its own lanes 16 h ..),
        // one row per step with the lanes along K (coalesced)
        for (int j = 0; j < 16; ++j) {
            const double* p = reinterpret_cast<const double*>(__shfl_sync(
                0xffffffffu, static_cast<unsigned long long>(reinterpret_cast<uintptr_t>(arow)), 16 * h + j));
            const int rr = q * 32 + 16 * h + j;
            double* dst = rawA + rr * kOzK + (lane ^ (rr & 31));
            if (p && lane < kc)
                cp_async8(saddr(dst), p + kb + lane);
            else
                *dst = 0.0;
        }
        const double* B = S.p[sg.b >> 56] + static_cast<int64_t>(sg.b & 0x00FFFFFFFFFFFFFFull);
        if (sg.b_ks == 1) {  // columns contiguous along K: lanes along K, warp w takes 4 columns
            for (int c = 0; c < 4; ++c) {
                const int n = warp * 4 + c;
                double* dst = rawB + n * kOzK + (lane ^ n);
                if (n0 + n < st.N && lane < kc)
                    cp_async8(saddr(dst), B + static_cast<int64_t>(kb + lane) + static_cast<int64_t>(n0 + n) * sg.b_ns);
                else
                    *dst = 0.0;
            }
        } else {  // lanes along N, warp w takes 4 values of K
            for (int c = 0; c < 4; ++c) {
                const int k = warp * 4 + c;
                double* dst = rawB + lane * kOzK + (k ^ lane);
                if (n0 + lane < st.N && k < kc)
                    cp_async8(saddr(dst), B + static_cast<int64_t>(kb + k) * sg.b_ks + static_cast<int64_t>(n0 + lane) * sg.b_ns);
                else
                    *dst = 0.0;
            }
        }
        asm volatile("cp.async.commit_group;");
    };
    double acc[kOzN / 2];
#pragma unroll
    for (int n = 0; n < kOzN / 2; ++n) acc[n] = 0.0;
    uint32_t phase = 0;
    bool failed = false;
    int seg = 0, k0 = 0;
    const int ncols_t = min(kOzN, st.N - n0);
    if (st.nseg > 0) issue_loads(0, 0);
    while (seg < st.nseg && !failed) {
        asm volatile("cp.async.wait_group 0;");
        __syncthreads();
        // 1. exponents (row maxima over both K halves through shared memory) and digit planes
        const double* arow = rawA + r * kOzK;
        const int sw = r & 31;
        {
            int Eh = 0;
#pragma unroll
            for (int k = 0; k < kOzK / 2; ++k) Eh = max(Eh, expo(arow[(16 * h + k) ^ sw]));
            rowE2[h * kOzM + r] = static_cast<short>(Eh);
        }
        {
            const int n = tid >> 3, kq = (tid & 7) * 4;
            double b[4];
            int Ec = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                b[c] = rawB[n * kOzK + ((kq + c) ^ n)];
                Ec = max(Ec, expo(b[c]));
            }
            Ec = max(Ec, __shfl_xor_sync(0xffffffffu, Ec, 1));
            Ec = max(Ec, __shfl_xor_sync(0xffffffffu, Ec, 2));
            Ec = max(Ec, __shfl_xor_sync(0xffffffffu, Ec, 4));
            if ((tid & 7) == 0) colE[n] = Ec;
            uint32_t Flo[4], Fhi[4];
            __half2 sg[2], off[2];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint64_t F = fixed56(b[c], Ec);
                Flo[c] = static_cast<uint32_t>(F);
                Fhi[c] = static_cast<uint32_t>(F >> 32);
            }
            pair_signs<4>(b, sg, off);
            const uint32_t o = core_off(n, kq);
#pragma unroll
            for (int p = 0; p < kSlices; ++p)
                *reinterpret_cast<uint2*>(planesB + p * kPlaneB + o) = digit_plane<4>(Flo, Fhi, sg, off, p);
        }
        __syncthreads();
        const int Er = max(static_cast<int>(rowE2[r]), static_cast<int>(rowE2[kOzM + r]));
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int kq = 16 * h + 8 * g;
            double a[8];
            uint32_t Flo[8], Fhi[8];
            __half2 sg[4], off[4];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                a[c] = arow[(kq + c) ^ sw];
                const uint64_t F = fixed56(a[c], Er);
                Flo[c] = static_cast<uint32_t>(F);
                Fhi[c] = static_cast<uint32_t>(F >> 32);
            }
            pair_signs<8>(a, sg, off);
            const uint32_t o = core_off(r, kq);
#pragma unroll
            for (int p = 0; p < kSlices; ++p)
                *reinterpret_cast<uint4*>(planesA + p * kPlaneA + o) = digit_plane<8>(Flo, Fhi, sg, off, p);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        // 2. the next stage's copies fly while the MMAs and the combination of this one run
        int nk = 0;  // MMAs of K = 16 that hold data in this stage
        {
            const TcSeg sg = segs[st.seg0 + seg];
            nk = (min(kOzK, sg.K - k0) + 15) / 16;
            k0 += kOzK;
            if (k0 >= sg.K) {
                ++seg;
                k0 = 0;
            }
        }
        if (seg < st.nseg) issue_loads(seg, k0);
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = saddr(planesA), b0 = saddr(planesB);
#pragma unroll
            for (int l = 2; l <= kSlices + 2; ++l) {
                bool first = true;
                for (int p = max(1, l - kSlices); p <= min(kSlices, l - 1); ++p) {
                    const int qq = l - p;
#pragma unroll
                    for (int kk = 0; kk < kOzK / 16; ++kk) {
                        if (kk >= nk) break;
                        mma_f16(tmem + static_cast<uint32_t>((l - 2) * kOzN),
                                desc(a0 + static_cast<uint32_t>((p - 1) * kPlaneA + kk * 256)),
                                desc(b0 + static_cast<uint32_t>((qq - 1) * kPlaneB + kk * 256)), idesc, first ? 0u : 1u);
                        first = false;
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                saddr(mbar)));
            *flag = poll(saddr(mbar), phase, wait_polls);
            if (!*flag) atomicExch(err, 1);
        }
        __syncthreads();
        phase ^= 1u;
        if (!*flag) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // 3. exact level sums -> FP64: warp (q, h) reads lanes 32 q .. and columns 16 h .. 16 h + 15
#pragma unroll
        for (int cb = 0; cb < kOzN / 2; cb += 4) {
            if (16 * h + cb >= ncols_t) break;  // uniform over the warp
            uint32_t v[kLevels][4];
#pragma unroll
            for (int L = 0; L < kLevels; ++L) {
                const uint32_t taddr = tmem + (static_cast<uint32_t>(q * 32) << 16) +
                                       static_cast<uint32_t>(L * kOzN + 16 * h + cb);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v[L][0]), "=r"(v[L][1]), "=r"(v[L][2]), "=r"(v[L][3])
                             : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int iv[kLevels];
#pragma unroll
                for (int L = 0; L < kLevels; ++L) iv[L] = __float2int_rz(__uint_as_float(v[L][j]));
                // T = sum_l v_l 2^(56 - 8l): levels 2-3 and 4-5 paired in 32 bits (below 2^30 and
                // 2^31), the rest in one 64-bit multiply-add
                const int a = iv[0] * 256 + iv[1];
                const int bb = iv[2] * 256 + iv[3];
                const long long c = static_cast<long long>(iv[4]) * 256 + (iv[5] + (iv[6] >> 8) + (iv[7] >> 16));
                const long long T = static_cast<long long>(bb) * 65536 + c + static_cast<long long>(a) * 4294967296ll;
                const int fe = Er + colE[16 * h + cb + j] - 1077;  // biased exponent of the unit 2^(e_i + e_j - 56)
                const double unit = fe > 0 && fe < 2047 ? __longlong_as_double(static_cast<long long>(fe) << 52) : 0.0;
                acc[cb + j] = fma(static_cast<double>(T), unit, acc[cb + j]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    asm volatile("cp.async.wait_all;");
    if (failed && tid == 0) poll(saddr(mbar), phase ^ 1u, kDefaultWaitPolls);  // MMAs still in flight
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (!failed) {
        // output rows through shared memory (the raw A stage is free), stored with lanes along N
        double* stage = rawA;
#pragma unroll
        for (int n = 0; n < kOzN / 2; ++n) stage[r * kOzN + ((16 * h + n) ^ (r & 31))] = acc[n];
        __syncthreads();
        const int* cm = st.cmap >= 0 ? cmaps + st.cmap : nullptr;
        for (int rr = warp; rr < kOzM; rr += kOzThreads / 32) {
            const int gr = m0 + rr;
            if (gr >= st.nrows) break;
            if (lane < ncols_t) {
                const uint64_t c = rows[st.row0 + gr].c;
                double* C = S.p[c >> 56] + static_cast<int64_t>(c & 0x00FFFFFFFFFFFFFFull);
                const int n = n0 + lane;
                C[cm ? cm[n] : n] = stage[rr * kOzN + (lane ^ (rr & 31))];
            }
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace

cudaError_t launch_gemm_oz(const Slots& slots, const TcStack* stacks, const TcRow* rows, const TcSeg* segs,
                           const uint64_t* atab, const int* cmaps, const int4* units, int u0, int u1, int* err,
                           int wait_polls, cudaStream_t st) {
    if (u1 <= u0) return cudaSuccess;
    if (wait_polls <= 0) wait_polls = kDefaultWaitPolls;
    static int attr_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_device != dev) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kOzSmem));
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    k_gemm_oz<<<u1 - u0, kOzThreads, kOzSmem, st>>>(slots, stacks, rows, segs, atab, cmaps, units, u0, err, wait_polls);
    return cudaGetLastError();
}

int gemm_oz_columns() { return kOzN; }

}  // namespace spmps
