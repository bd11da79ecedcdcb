// Inverse of the projected metric's symmetry blocks: the Davidson correction t = (N_eff + s I)^-1 r
// and the minimal-norm representative (N_eff + s I)^-1 N_eff x taken before decimation.
//
// N_eff (Fig. spmpsOpt (c)) is the network of the identity MPO rotated by beta_g, summed with the
// weights c_g of Eq. pmpo: sum_g c_g LN_g (x) r_g (x) r_g (x) RN_g.  Each factor conserves the
// particle number of its own part (left block, site k, site k+1, right block), so N_eff is
// exactly block-diagonal in (N-group of the left index, n(s1), n(s2)).  The blocks are dense
// (the rotations mix M), assembled from the N environments, shifted by s and factorised by a
// batched FP64 Cholesky once per two-site step; every Davidson iteration then solves with them.
#pragma once

#include <cstdint>
#include <vector>

#include "engine.h"

namespace spmps {

// One diagonal block of N_eff: `dim` entries of the two-site vector (elements elem_off ..),
// its factor in dim x dim row-major doubles at mat_off (lower triangle used), and the offsets of
// its left / right N-environment group blocks (added to the per-beta bases of op 1).
struct MetricBlock {
    int64_t elem_off, mat_off, loff, roff;
    int dim, lda, ldb, pad;
};
// Element of a block: offset in the row-block layout, index in the left N-group, and
// b * 16 + s (index in the right N-group, two-site local state s = 4 s1 + s2).
struct MetricElem {
    int64_t xo;
    int a, bs;
};
// Per beta point: c_g, the site rotation r(beta_g) (bra x ket) and the bases of op 1's left and
// right environments.
struct MetricBeta {
    double c, r[16];
    int64_t lbase, rbase;
};

struct MetricState {
    int site = -1;
    bool ok = false;  // factors present for `site` and the current environments
    int64_t n_x = 0, n_elems = 0, mat_total = 0;
    int n_blocks = 0, max_dim = 0;
    std::vector<MetricBlock> blocks;  // sorted by dim, largest first
    std::vector<MetricElem> elems;
    std::vector<int> steps_trsm, steps_syrk;   // per panel step: offset into prefix arrays
    std::vector<int> alive;                    // per panel step: blocks with dim > p0
    DevMem d_blocks, d_elems, d_betas, d_tiles, d_prefix, mats, ybuf, status;
};

// Shift s of the metric blocks (|N_eff| <= 1 with the weights of Eq. PSMM): directions of N-norm
// well above s are inverted exactly, near-null ones damped.
constexpr double kMetricShift = 1e-7;
// Largest total factor storage (doubles) the solver allocates; above it the diagonal correction
// is used for that step.
constexpr int64_t kMetricMaxDoubles = int64_t(1) << 30;
// Blocks above this dimension (default of spmps_options.metric_max_dim) are not factorised: their
// entries keep the diagonal correction (the factorisation costs dim^3 / 3 FP64 flops per block).
constexpr int kMetricDefaultMaxDim = 3072;

namespace eng {
// Build, assemble and factorise the blocks of site k (environments must be current).  Sets M.ok
// (false when the factor storage would exceed kMetricMaxDoubles or a pivot was not positive; the
// caller then keeps the diagonal correction).
spmps_status metric_prepare(spmps_t* h, int k, MetricState& M);
// out = (N_eff + s I)^-1 in on the entries of the factorised blocks of the prepared site; the
// other entries of out are left as they are.
spmps_status metric_solve(spmps_t* h, MetricState& M, const double* in, double* out, cudaStream_t st);
}  // namespace eng

}  // namespace spmps
