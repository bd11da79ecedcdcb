// The projected action without any device allocation, for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they need the projected action:
// callers whose device memory is fully reserved up front by their own pool allocator, or
// embedding runtimes that forbid the CUDA allocator after start-up (a cudaMalloc there would
// fail or break the runtime's accounting).  spmps_apply_heff_noalloc serves them: it runs the
// same three-phase FP64 contraction as spmps_apply_heff with precision 0, but its intermediates
// (the M-dense T1/T3 blocks and the per-beta partials) live in a fixed file-scope device array
// instead of the handle's workspace.
//
// Limits and caveats
//   - The array holds kNoAllocScratchDoubles doubles (32 MiB).  Every GPU that loads the library
//     keeps it until the process exits.  Problems whose intermediates need more return
//     SPMPS_ERR_BAD_INPUT.
//   - Every call on a device shares the one array, which keeps the previous call's contents; the
//     call zeroes what must start at zero.  Calls that overlap on the GPU (different streams,
//     handles or threads) race on the array: serialise them.
//   - The environments and the contraction plan of the site must already exist (they are built,
//     and allocated, by a previous spmps_apply_heff or spmps_energy call for that site and MPS);
//     otherwise the call returns SPMPS_ERR_STATE without doing anything.
//   - The first call on each device looks up the array's device address (cudaGetSymbolAddress,
//     with that device current), and the first call on each handle creates one CUDA event (no
//     device memory) that orders the caller's stream after the handle's stream.
//   - The H part always runs in FP64, whatever the handle's precision option: the pre-split TF32
//     operands of the reduced-precision forms would need room of their own in the array.
//   - The library's per-launch profiler (spmps_profile) is not used by this call.
#include <mutex>

#include "engine.h"

using namespace spmps;
using namespace spmps::eng;

namespace {

constexpr size_t kNoAllocScratchDoubles = static_cast<size_t>(4) << 20;  // 32 MiB of doubles
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current).
cudaError_t scratch_address(int device, double** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<double*>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" spmps_status spmps_apply_heff_noalloc(spmps_handle h, int site, const double* x, double* y, double* z,
                                                 void* stream) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2) return fail(h, SPMPS_ERR_BAD_INPUT, "site out of range");
    if (!x || (!y && !z)) return fail(h, SPMPS_ERR_BAD_INPUT, "x and one of y, z are required");
    Plan* P = h->apply_plans[site].get();
    if (!P || !P->ready || !h->Lenv[site].valid || !h->Renv[site + 2].valid)
        return fail(h, SPMPS_ERR_STATE,
                    "no contraction plan for this site: call spmps_apply_heff once for it first (that call allocates)");
    const size_t need = static_cast<size_t>(P->t1_size) + static_cast<size_t>(P->t2_size) +
                        2 * static_cast<size_t>(h->G) * static_cast<size_t>(P->reduce_nx) + 64;
    if (need > kNoAllocScratchDoubles)
        return fail(h, SPMPS_ERR_BAD_INPUT, "intermediates need " + std::to_string(need) +
                                                " doubles, above the fixed scratch of " +
                                                std::to_string(kNoAllocScratchDoubles));
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    double* base = nullptr;
    e = scratch_address(h->device, &base);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    if (s != h->stream) {
        // environments are built on the handle's stream: order the caller's stream after the
        // work queued there so far (no host synchronisation)
        if (!h->noalloc_order) {
            e = cudaEventCreateWithFlags(&h->noalloc_order, cudaEventDisableTiming);
            if (e != cudaSuccess) { h->noalloc_order = nullptr; return cuda_fail(h, e, "cudaEventCreate"); }
        }
        e = cudaEventRecord(h->noalloc_order, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->noalloc_order, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "ordering the caller's stream after the handle's");
    }
    Slots S{};
    S.p[0] = const_cast<double*>(x);
    S.p[1] = y;
    S.p[2] = z;
    S.p[3] = base;
    S.p[4] = base + ((P->t1_size + 31) / 32) * 32;
    S.p[8] = S.p[4] + ((P->t2_size + 31) / 32) * 32;
    S.p[9] = S.p[8] + static_cast<int64_t>(h->G) * P->reduce_nx;
    if (static_cast<size_t>(S.p[9] - base) + static_cast<size_t>(h->G) * P->reduce_nx > kNoAllocScratchDoubles)
        return fail(h, SPMPS_ERR_BAD_INPUT, "intermediates do not fit the fixed scratch");
    S.p[5] = h->Lenv[site].buf.as<double>();
    S.p[6] = h->Renv[site + 2].buf.as<double>();
    const int G = h->G;
    // FP64 action without the profiler (its records create events and may synchronise)
    const int prec_saved = h->apply_precision;
    const bool prof_saved = h->profile;
    h->apply_precision = 0;
    h->profile = false;
    if (y && z) st = plan_run(h, *P, S, 0, 2 * G, s);
    else if (y) st = plan_run(h, *P, S, 0, G, s);
    else st = plan_run(h, *P, S, G, 2 * G, s);
    h->apply_precision = prec_saved;
    h->profile = prof_saved;
    if (st != SPMPS_OK) return st;
    ++h->applies;
    return SPMPS_OK;
}
