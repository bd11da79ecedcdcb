// Stacked block GEMMs of the projected action on the 5th-generation tensor cores (tcgen05.mma
// kind::tf32, accumulator in tensor memory, operands staged in shared memory).
//
// The block products of phases A and C are small (a label or an N-group of rows, reductions of 5
// to a few hundred), far below the 128-row tiles of tcgen05.  Tasks that share their B operand are
// stacked along M: in phase A every (channel, bra group) product of one ket label l reads the same
// rows of x; in phase C every output block (la, s, lb) with the same right label lb reads the same
// rows of the right environments, channel by channel.  A stack is then one GEMM of
// (sum of the tasks' rows) x N with K split into segments (phase C: one per channel u), every
// stacked row carrying its own output address and its own A address per segment (or none, when the
// task has no such segment).  One CTA computes a 128-row by NT-column tile of a stack.
#pragma once

#include <cstdint>
#include <vector>

#include "core.h"
#include "kernels.h"

namespace spmps {

struct TcStack {
    int row0, nrows;  // stacked rows rows[row0 .. row0 + nrows)
    int seg0, nseg;   // K segments segs[seg0 ..)
    int N;            // columns
    int cmap;         // column map offset into the plan's cmaps, -1 for identity
    int64_t atab0;    // A handles atab[atab0 + r * nseg + s] for stacked row r and segment s
};
struct TcRow {
    uint64_t c;  // handle of the row's first output element: C(r, n) = C[c + map(n)]
};
struct TcSeg {
    uint64_t b;       // B(n, k) = B[b + k * b_ks + n * b_ns]
    int K, b_ks, b_ns, pad;
};
constexpr uint64_t kNoOperand = ~static_cast<uint64_t>(0);

struct TcPlan {
    std::vector<TcStack> stacks;
    std::vector<TcRow> rows;
    std::vector<TcSeg> segs;
    std::vector<uint64_t> atab;   // A(r, s, k) = A[atab + k], contiguous along K
    std::vector<int4> units;      // (stack, m0, n0, 0): one CTA each
    std::vector<int> unit_rng;    // per beta range: units [unit_rng[g], unit_rng[g + 1])
    int nt = 64;                  // columns per CTA tile (32, 64 or 128)
    bool ok = false;              // every task of the range could be stacked
    void clear() {
        stacks.clear(); rows.clear(); segs.clear(); atab.clear(); units.clear(); unit_rng.clear();
        ok = false;
    }
};

// Stack the tasks of G (task ranges task_rng[g] .. task_rng[g + 1] for g < n_ranges) by their key;
// nt = columns per CTA.  Returns false (and leaves P.ok false) when a task does not fit the stacked
// form (A not contiguous along K).
bool build_tc_plan(const GemmPlan& G, const std::vector<int>& task_rng, int n_ranges, int nt, TcPlan& P);

// One launch over units [u0, u1): C = sum over segments of A B^T for every unit tile, with A and B
// read from the pre-split (hi, lo) TF32 buffers; split3 != 0 accumulates hi*hi + hi*lo + lo*hi,
// else hi*hi.  err[0] is set when a bounded wait for the MMAs gave up (the kernel then still
// waits, with the default limit, for its MMAs in flight and frees its tensor memory).
cudaError_t launch_gemm_tc(const Slots& slots, const SlotsF& split, const TcStack* stacks, const TcRow* rows,
                           const TcSeg* segs, const uint64_t* atab, const int* cmaps, const int4* units, int u0,
                           int u1, int nt, int split3, int* err, int wait_polls, cudaStream_t st);

// FP64-accurate variant over the same stacks (tiles of 128 rows x gemm_oz_columns() columns, so the
// plan must be built with nt = gemm_oz_columns()): A and B read in FP64, every K stage of 32 split
// into seven signed 8-bit digits per entry against per-row and per-column exponents, the digit
// products summed exactly by tcgen05.mma kind::f16 (FP16 digits, FP32 accumulators in tensor
// memory, one per level p + q = 2 .. 9, every partial sum an integer below 2^24) and combined in
// FP64 (the splitting scheme of Ozaki, Ogita, Oishi and Rump).  Error per stage of the order of
// 32 * 2^-55 max|a_i.| max|b_.j|.  err[0] and wait_polls as for launch_gemm_tc.
cudaError_t launch_gemm_oz(const Slots& slots, const TcStack* stacks, const TcRow* rows, const TcSeg* segs,
                           const uint64_t* atab, const int* cmaps, const int4* units, int u0, int u1, int* err,
                           int wait_polls, cudaStream_t st);
int gemm_oz_columns();

}  // namespace spmps
