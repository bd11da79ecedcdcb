// The SP-MPS handle: device state, environment cache and the contraction planner.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "../../include/spmps.h"
#include "core.h"
#include "kernels.h"
#include "mlp.h"
#include "tc_gemm.h"

namespace spmps {

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem&) = delete;
    DevMem& operator=(const DevMem&) = delete;
    DevMem(DevMem&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevMem& operator=(DevMem&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevMem() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t nb) {
        if (nb <= bytes && p) return cudaSuccess;
        release();
        size_t want = nb < 256 ? 256 : nb;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) { p = nullptr; return e; }
        bytes = want;
        return cudaSuccess;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Per-op layout of one environment tensor on one bond: block (w, G) of gdim(G) x gdim(G')
// with G' the group of n(G) - cn[w]; -1 where absent.
struct EnvLayout {
    int n_groups = 0;
    std::vector<int64_t> off;  // [w * n_groups + G]
    std::vector<int> ld;       // [w * n_groups + G] = gdim(G')
    int64_t size = 0;
};
EnvLayout make_env_layout(const Bond& b, const std::vector<int>& cn);

// A set of operators sharing the environment machinery: H and the projector norm (identity)
// for the energy; S^2 for its expectation value.
struct OpSet {
    std::vector<MPO> mpo;                  // per op, unrotated
    std::vector<std::vector<MPO>> rot;     // [op][g], rotation on the ket leg
    int n_ops() const { return static_cast<int>(mpo.size()); }
};

struct EnvStore {
    DevMem buf;
    std::vector<EnvLayout> lay;    // per op
    std::vector<int64_t> base;     // [op * G + g]
    int64_t total = 0;
    bool valid = false;
    uint64_t version = 0;          // changes whenever buf is rewritten
    DevMem split;                  // pre-split TF32 copy (float2 per element) for the tensor-core action
    uint64_t split_version = 0;    // version of buf that split was made from (0: none)
};

// Frobenius norms of the (bra label, ket label) sub-blocks of one bond's environments, per
// operator, beta point and channel (the approximate M-sector screening).
struct EnvNorms {
    int ngroups = 0;
    std::vector<int> dw, wbase;   // per op: channels, first (g, w) slot
    std::vector<double> wmax;     // per (op, g, w) slot: largest sub-block norm of the channel
    std::vector<int64_t> start;   // per (slot, bra group): first norm, -1 if the block is absent
    std::vector<int> ncols;       // per (slot, bra group): labels of the ket group
    std::vector<double> norms;
    int slot(int op, int g, int w) const { return wbase[op] + g * dw[op] + w; }
    // below tau * (largest norm of the channel): the block product is dropped
    bool dropped(int op, int g, int w, int ga, int la_local, int lp_local, double tau) const {
        const int sl = slot(op, g, w);
        const int64_t st = start[static_cast<int64_t>(sl) * ngroups + ga];
        if (st < 0) return true;
        return norms[st + static_cast<int64_t>(la_local) * ncols[static_cast<int64_t>(sl) * ngroups + ga] + lp_local] <
               tau * wmax[sl];
    }
};

// A three-phase contraction plan (GEMM, MPO-leg combination, GEMM), uploaded to the device.
struct Plan {
    GemmPlan A, C;
    CombPlan B;
    TilePolicy polA, polC;  // tile policies of phases A and C (autotuned per site, or the default)
    std::vector<int> tileA_rng, tileC_rng, combB_rng;  // [op * G + g] .. [op * G + g + 1]
    // the builders write task ranges into tileA_rng / tileC_rng; the first upload keeps them here
    // and every upload turns them into tile ranges for the tiles of its policy
    std::vector<int> taskA_rng, taskC_rng;
    bool task_rng_kept = false;
    std::vector<double> flopsA_rng, flopsB_rng, flopsC_rng;  // algorithmic flops per range
    int64_t t1_size = 0, t2_size = 0;
    int64_t reduce_nx = 0;  // > 0: phase C writes per-beta partials of this length (slots 8, 9)
    double flops = 0.0;
    double flops_op[4] = {0, 0, 0, 0};
    double bytesA_op[4] = {0, 0, 0, 0}, bytesB_op[4] = {0, 0, 0, 0}, bytesC_op[4] = {0, 0, 0, 0};
    double flopsA_op[4] = {0, 0, 0, 0}, flopsB_op[4] = {0, 0, 0, 0}, flopsC_op[4] = {0, 0, 0, 0};
    DevMem d_tasksA, d_segsA, d_tilesA, d_cmapsA, d_outsB, d_termsB, d_tasksC, d_segsC, d_tilesC, d_cmapsC;
    DevMem d_tcA, d_tcC;                     // tensor-core tile lists
    std::vector<int> tcA_rng, tcC_rng;       // their ranges per (op, g)
    TcPlan stA, stC;                         // tcgen05 stacks of the H part, phases A and C
    DevMem d_stA[5], d_stC[5];               // their stacks, rows, segments, A table, units
    TcPlan ozA, ozC;                         // stacks of all (op, g) ranges for the FP64-accurate
    DevMem d_ozA[5], d_ozC[5];               // split-product GEMM (fp64_tensor_cores)
    // diagonal (apply plans only)
    std::vector<DiagBlock> diag_blocks;
    std::vector<DiagTerm> diag_terms;
    DevMem d_diag_blocks, d_diag_terms;
    bool ready = false;
    // environment versions the plan was built for (screened plans depend on their values)
    uint64_t envL_version = 0, envR_version = 0;
};

}  // namespace spmps

// A lower state of a state-specific excited-state optimisation (Sec. 2.3.2): its MPS (fixed) and
// the per-beta environments of <running state| exp(+i b_g S_y) |lower state> (bra = the state
// being optimised, ket = the lower state, the identity MPO rotated by -beta_g, one channel), from
// which the B vector of Eq. orthoB follows at every two-site step.
struct LowerState {
    std::vector<spmps::Bond> bonds;
    std::vector<spmps::RowBlockLayout> alay;
    std::vector<std::unique_ptr<spmps::DevMem>> A;
    std::vector<spmps::MPO> rot;  // per beta point
    std::vector<spmps::EnvStore> L, R;
};

// State of the learned Davidson correction.
struct MlpState {
    spmps::DevMem params, grads, m, v, w2core, err;
    spmps::DevMem X, T, Z1, H1, Z2, H2, dZ2, dZ1, dy, loss_part, loss;  // training step buffers
    spmps::DevMem data_x, data_t;  // harvested set (features, targets)
    int64_t count = 0, capacity = 0;
    int batch = 0, step = 0;
    bool ready = false;  // parameters present on the device
    // harvesting
    bool harvest = false;
    int samples = 512, max_iters = 32;
    spmps::DevMem h_idx, h_feat, h_x, h_norm, h_dots;  // per solve
};

struct spmps_t {
    int K = 0, N = 0, twoM = 0, twoS = 0, G = 0, D = 0;
    spmps_options opt{};
    std::string err;
    int device = 0;
    cudaStream_t stream = nullptr;
    // second stream of the mixed-precision action: the FP64 N_eff products run on it while the
    // tensor-core H products run on the action's stream (created on first use)
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
    // orders a caller's stream after the handle's stream in spmps_apply_heff_noalloc
    cudaEvent_t noalloc_order = nullptr;
    spmps::DevMem tc_err;  // set by the stacked tensor-core GEMM when a bounded wait gave up
    std::vector<LowerState> lower;  // lower states of an excited-state optimisation (Eq. orthoB)
    std::vector<double> beta, cg;

    bool has_ham = false, has_mps = false;
    // the integrals of the Hamiltonian (kept for the fragment energies); empty after spmps_set_mpo
    std::vector<double> ints_h1, ints_h2;
    double ints_ecore = 0.0;
    // autotuner: chosen tile candidate per site for phases A and C (-1 = not tuned yet)
    std::vector<int> tune_a, tune_c;
    spmps::DevMem tunebuf;
    uint64_t env_counter = 0;      // source of EnvStore versions
    spmps::DevMem xsplit, t3split; // pre-split TF32 copies of x and of the phase-B output
    spmps::OpSet ops;        // H, N
    std::vector<spmps::Bond> bonds;           // K+1
    std::vector<spmps::RowBlockLayout> alay;  // per site, ns = 4
    std::vector<std::unique_ptr<spmps::DevMem>> A;  // per site
    int center = 0;
    std::vector<spmps::EnvStore> Lenv, Renv;  // per bond
    std::vector<std::unique_ptr<spmps::Plan>> apply_plans;  // per site
    spmps::DevMem work1, work2, work3, partial;
    spmps::DevMem xbuf, ybuf, zbuf;  // host-API staging
    MlpState mlp;
    int apply_precision = 0;  // precision of the H part of projected actions issued now (0 = FP64)
    int64_t launches = 0, applies = 0, dav_iters = 0, refine_iters = 0;
    double last_apply_flops = 0.0, last_discarded = 0.0, apply_flops_total = 0.0;
    // per-launch event profiler
    struct TimerRec {
        cudaEvent_t a, b;
        int kind;
        double flops;
    };
    bool profile = false;
    std::vector<TimerRec> timers_live, timers_free;
    static constexpr int kProfKinds = 10;
    int64_t prof_launches[kProfKinds] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double prof_ms[kProfKinds] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, prof_flops[kProfKinds] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
};

namespace spmps {
namespace eng {

spmps_status fail(spmps_t* h, spmps_status st, const std::string& msg);
spmps_status cuda_fail(spmps_t* h, cudaError_t e, const char* where);

template <class T>
cudaError_t upload(DevMem& m, const std::vector<T>& v, cudaStream_t st) {
    cudaError_t e = m.ensure(std::max<size_t>(1, v.size()) * sizeof(T));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(m.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

bool validate_plan(const Plan& P, const int64_t* sizes, std::string* why);
bool validate_gemm(const GemmPlan& G, const int64_t* sizes, std::string* why);
spmps_status plan_upload(spmps_t* h, Plan& P);
spmps_status plan_run(spmps_t* h, Plan& P, Slots S, int r0, int r1, cudaStream_t st, cudaEvent_t* ev = nullptr,
                      const SlotsF* split = nullptr);
spmps_status update_left(spmps_t* h, int i);
spmps_status env_subblock_norms(spmps_t* h, const EnvStore& E, const Bond& b, int bond, EnvNorms& out);
// Excited states: the B vectors of every lower state at sites (k, k+1), orthonormalised (QR by
// Gram-Schmidt twice) into V (n_x x count, device); *count = number of independent columns.
spmps_status excited_constraints(spmps_t* h, int k, DevMem& V, int* count);
// The cross environments follow the running MPS: after a decimation at k (move_right: left
// environment of bond k+1; else right environment of bond k+1).
spmps_status excited_after_step(spmps_t* h, int k, bool move_right);
void excited_invalidate(spmps_t* h);
spmps_status update_right(spmps_t* h, int i);
spmps_status ensure_envs(spmps_t* h, int k);
void invalidate_all(spmps_t* h);
spmps_status get_apply_plan(spmps_t* h, int k, Plan** out);
spmps_status do_apply(spmps_t* h, int k, const double* x, double* y, double* z, cudaStream_t st,
                      cudaEvent_t* ev = nullptr);
spmps_status check_ready(spmps_t* h);
spmps_status set_ops(spmps_t* h, MPO H);
spmps_status build_opset(spmps_t* h, const MPO& H, OpSet* out);
// profiler: a started record's events are recorded on stream st around one launch
int prof_begin(spmps_t* h, cudaStream_t st, int kind, double flops);
void prof_end(spmps_t* h, cudaStream_t st, int rec);
spmps_status prof_collect(spmps_t* h);

}  // namespace eng
}  // namespace spmps

#define CK(expr)                                                                  \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) return ::spmps::eng::cuda_fail(h, _e, #expr);      \
    } while (0)
