// Inverse of the symmetry blocks of the projected metric N_eff (see metric.h): host planner,
// block assembly from the N environments, batched blocked Cholesky and the per-iteration solve.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "metric.h"

namespace spmps {

namespace {

constexpr int kMaxBeta = 64;
constexpr int kPanel = 32;      // Cholesky panel width
constexpr int kTrsmRows = 128;  // rows per CTA of the panel solve
constexpr int kSyrkTile = 64;   // trailing-update tile (rows and columns)

// ---- assembly -----------------------------------------------------------------------------------
// One CTA per 32 x 32 lower tile of a block: entry (i, j), j <= i, of
// sum_g c_g LN_g[a_i, a_j] r_g[s1_i, s1_j] r_g[s2_i, s2_j] RN_g[b_i, b_j] (+ shift on the diagonal).
__global__ void __launch_bounds__(256) k_metric_assemble(const MetricBlock* __restrict__ blocks,
                                                         const MetricElem* __restrict__ elems,
                                                         const MetricBeta* __restrict__ betas, int G,
                                                         const double* __restrict__ Lenv,
                                                         const double* __restrict__ Renv,
                                                         const int4* __restrict__ tiles, double shift,
                                                         double* __restrict__ mats) {
    __shared__ MetricBeta sb[kMaxBeta];
    for (int q = threadIdx.x; q < G; q += blockDim.x) sb[q] = betas[q];
    __syncthreads();
    const int4 tl = tiles[blockIdx.x];
    const MetricBlock B = blocks[tl.x];
    const int i0 = tl.y * 32, j0 = tl.z * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int j = j0 + tx;
    if (j >= B.dim) return;
    const MetricElem ej = elems[B.elem_off + j];
    const int bj = ej.bs >> 4, s1j = (ej.bs >> 2) & 3, s2j = ej.bs & 3;
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q;
        if (i >= B.dim || j > i) continue;
        const MetricElem ei = elems[B.elem_off + i];
        const int bi = ei.bs >> 4, s1i = (ei.bs >> 2) & 3, s2i = ei.bs & 3;
        const int64_t la = B.loff + static_cast<int64_t>(ei.a) * B.lda + ej.a;
        const int64_t ra = B.roff + static_cast<int64_t>(bi) * B.ldb + bj;
        double acc = 0.0;
        for (int g = 0; g < G; ++g) {
            const double rr = sb[g].r[s1i * 4 + s1j] * sb[g].r[s2i * 4 + s2j];
            if (rr == 0.0) continue;
            acc += sb[g].c * rr * Lenv[sb[g].lbase + la] * Renv[sb[g].rbase + ra];
        }
        if (i == j) acc += shift;
        mats[B.mat_off + static_cast<int64_t>(i) * B.dim + j] = acc;
    }
}

// ---- batched blocked Cholesky (lower), one panel step per launch triple --------------------------

// The diagonal kPanel x kPanel tile of panel p0 of each live block (one warp per block).
__global__ void __launch_bounds__(32) k_chol_diag(const MetricBlock* __restrict__ blocks, double* __restrict__ mats,
                                                  int p0, int* __restrict__ status) {
    __shared__ double A[kPanel][kPanel + 1];
    const MetricBlock B = blocks[blockIdx.x];
    const int w = min(kPanel, B.dim - p0);
    const int lane = threadIdx.x;
    double* base = mats + B.mat_off + static_cast<int64_t>(p0) * B.dim + p0;
    for (int r = 0; r < w; ++r) A[r][lane] = lane <= r ? base[static_cast<int64_t>(r) * B.dim + lane] : 0.0;
    __syncwarp();
    for (int j = 0; j < w; ++j) {
        if (lane == j) {
            double d = A[j][j];
            if (!(d > 0.0)) {
                atomicOr(status, 1);
                d = 1.0;
            }
            A[j][j] = sqrt(d);
        }
        __syncwarp();
        if (lane > j && lane < w) A[lane][j] /= A[j][j];
        __syncwarp();
        if (lane > j && lane < w)
            for (int c = j + 1; c <= lane; ++c) A[lane][c] -= A[lane][j] * A[c][j];
        __syncwarp();
    }
    for (int r = 0; r < w; ++r)
        if (lane <= r) base[static_cast<int64_t>(r) * B.dim + lane] = A[r][lane];
}

// Index of the block owning unit u given the prefix sums pre[0..n] (pre[0] = 0).
__device__ __forceinline__ int owner(const int* __restrict__ pre, int n, int u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Rows below the diagonal tile: A[i, p0:p0+32] <- A[i, p0:p0+32] L_pp^-T (one thread per row).
__global__ void __launch_bounds__(kTrsmRows) k_chol_trsm(const MetricBlock* __restrict__ blocks,
                                                         double* __restrict__ mats, int p0,
                                                         const int* __restrict__ pre, int n_alive) {
    __shared__ double Lp[kPanel][kPanel + 1];
    const int b = owner(pre, n_alive, blockIdx.x);
    const MetricBlock B = blocks[b];
    const int chunk = blockIdx.x - pre[b];
    const double* diag = mats + B.mat_off + static_cast<int64_t>(p0) * B.dim + p0;
    for (int q = threadIdx.x; q < kPanel * kPanel; q += blockDim.x) {
        const int r = q / kPanel, c = q % kPanel;
        Lp[r][c] = c <= r ? diag[static_cast<int64_t>(r) * B.dim + c] : 0.0;
    }
    __syncthreads();
    const int i = p0 + kPanel + chunk * kTrsmRows + threadIdx.x;
    if (i >= B.dim) return;
    double* row = mats + B.mat_off + static_cast<int64_t>(i) * B.dim + p0;
    double x[kPanel];
#pragma unroll
    for (int c = 0; c < kPanel; ++c) x[c] = row[c];
#pragma unroll
    for (int j = 0; j < kPanel; ++j) {
        double v = x[j];
#pragma unroll
        for (int c = 0; c < j; ++c) v -= x[c] * Lp[j][c];
        x[j] = v / Lp[j][j];
    }
#pragma unroll
    for (int c = 0; c < kPanel; ++c) row[c] = x[c];
}

// Trailing update A[i, j] -= sum_c A[i, p0 + c] A[j, p0 + c] for p0 + 32 <= j <= i, on 64 x 64
// lower tiles (256 threads, 4 x 4 outputs each).
__global__ void __launch_bounds__(256) k_chol_syrk(const MetricBlock* __restrict__ blocks, double* __restrict__ mats,
                                                   int p0, const int* __restrict__ pre, int n_alive) {
    __shared__ double Ai[kSyrkTile][kPanel + 1];
    __shared__ double Aj[kSyrkTile][kPanel + 1];
    const int b = owner(pre, n_alive, blockIdx.x);
    const MetricBlock B = blocks[b];
    const int t = blockIdx.x - pre[b];
    // lower-triangular tile index t -> (ti, tj), tj <= ti
    int ti = static_cast<int>((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int m0 = p0 + kPanel;
    const int ib = m0 + ti * kSyrkTile, jb = m0 + tj * kSyrkTile;
    double* M = mats + B.mat_off;
    for (int q = threadIdx.x; q < kSyrkTile * kPanel; q += blockDim.x) {
        const int r = q / kPanel, c = q % kPanel;
        Ai[r][c] = ib + r < B.dim ? M[static_cast<int64_t>(ib + r) * B.dim + p0 + c] : 0.0;
        Aj[r][c] = jb + r < B.dim ? M[static_cast<int64_t>(jb + r) * B.dim + p0 + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
#pragma unroll 8
    for (int k = 0; k < kPanel; ++k) {
        double ai[4], aj[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            ai[a] = Ai[ty * 4 + a][k];
            aj[a] = Aj[tx * 4 + a][k];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] += ai[a] * aj[c];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = ib + ty * 4 + a;
        if (i >= B.dim) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = jb + tx * 4 + c;
            if (j < B.dim && j <= i) M[static_cast<int64_t>(i) * B.dim + j] -= acc[a][c];
        }
    }
}

// ---- solve ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out = (L L^T)^-1 in on every block (one CTA per block): gather, forward substitution by panels
// of 32 (warp 0 solves the diagonal tile, all warps update the rows below), backward substitution
// with L^T (column sums of the rows below reduced over the warps), scatter.
__global__ void __launch_bounds__(512) k_metric_solve(const MetricBlock* __restrict__ blocks,
                                                      const MetricElem* __restrict__ elems,
                                                      const double* __restrict__ mats, const double* __restrict__ in,
                                                      double* __restrict__ out, double* __restrict__ ybuf) {
    __shared__ double red[16][33];
    const MetricBlock B = blocks[blockIdx.x];
    const int dim = B.dim;
    const double* L = mats + B.mat_off;
    const MetricElem* E = elems + B.elem_off;
    double* y = ybuf + B.elem_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = threadIdx.x; e < dim; e += blockDim.x) y[e] = in[E[e].xo];
    __syncthreads();
    for (int p0 = 0; p0 < dim; p0 += 32) {
        const int w = min(32, dim - p0);
        if (warp == 0) {
            double v = lane < w ? y[p0 + lane] : 0.0;
            for (int j = 0; j < w; ++j) {
                if (lane == j) v /= L[static_cast<int64_t>(p0 + j) * dim + p0 + j];
                const double yj = __shfl_sync(0xffffffffu, v, j);
                if (lane > j && lane < w) v -= L[static_cast<int64_t>(p0 + lane) * dim + p0 + j] * yj;
            }
            if (lane < w) y[p0 + lane] = v;
        }
        __syncthreads();
        const double yl = lane < w ? y[p0 + lane] : 0.0;
        for (int i = p0 + w + warp; i < dim; i += nw) {
            double part = lane < w ? L[static_cast<int64_t>(i) * dim + p0 + lane] * yl : 0.0;
            part = warp_sum(part);
            if (lane == 0) y[i] -= part;
        }
        __syncthreads();
    }
    for (int p0 = ((dim - 1) / 32) * 32; p0 >= 0; p0 -= 32) {
        const int w = min(32, dim - p0);
        double acc = 0.0;
        for (int i = p0 + w + warp; i < dim; i += nw)
            if (lane < w) acc += L[static_cast<int64_t>(i) * dim + p0 + lane] * y[i];
        red[warp][lane] = acc;
        __syncthreads();
        if (warp == 0) {
            double s = 0.0;
            for (int q = 0; q < nw; ++q) s += red[q][lane];
            double v = lane < w ? y[p0 + lane] - s : 0.0;
            for (int j = w - 1; j >= 0; --j) {
                if (lane == j) v /= L[static_cast<int64_t>(p0 + j) * dim + p0 + j];
                const double yj = __shfl_sync(0xffffffffu, v, j);
                if (lane < j) v -= L[static_cast<int64_t>(p0 + j) * dim + p0 + lane] * yj;
            }
            if (lane < w) y[p0 + lane] = v;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < dim; e += blockDim.x) out[E[e].xo] = y[e];
}

}  // namespace

namespace eng {

spmps_status metric_prepare(spmps_t* h, int k, MetricState& M) {
    M.ok = false;
    M.site = k;
    const int G = h->G;
    const int max_dim = h->opt.metric_max_dim > 0 ? h->opt.metric_max_dim : kMetricDefaultMaxDim;
    if (G > kMaxBeta || h->ops.n_ops() < 2) return SPMPS_OK;
    const Bond& bl = h->bonds[k];
    const Bond& br = h->bonds[k + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    const EnvStore& Le = h->Lenv[k];
    const EnvStore& Re = h->Renv[k + 2];
    if (!Le.valid || !Re.valid) return fail(h, SPMPS_ERR_STATE, "metric blocks need current environments");
    const int ngl = static_cast<int>(bl.groups.size()), ngr = static_cast<int>(br.groups.size());
    // blocks in (left group, n(s1), n(s2)) order with their elements
    struct Tmp {
        MetricBlock b;
        std::vector<MetricElem> e;
    };
    std::vector<Tmp> tmp;
    for (int ga = 0; ga < ngl; ++ga) {
        const Group& Ga = bl.groups[ga];
        for (int n1 = 0; n1 < 3; ++n1)
            for (int n2 = 0; n2 < 3; ++n2) {
                Tmp T{};
                int gb = -1;
                for (int la = Ga.first; la < Ga.first + Ga.count; ++la) {
                    const Label& La = bl.labels[la];
                    for (int i = 0; i < La.dim; ++i)
                        for (int s1 = 0; s1 < 4; ++s1) {
                            if (kLocalN[s1] != n1) continue;
                            for (int s2 = 0; s2 < 4; ++s2) {
                                if (kLocalN[s2] != n2) continue;
                                const int s = s1 * 4 + s2;
                                const int lb = xl.seg_label[la * 16 + s];
                                if (lb < 0) continue;
                                const Label& Lb = br.labels[lb];
                                gb = Lb.group;
                                const int boff = Lb.off - br.groups[Lb.group].off;
                                for (int j = 0; j < Lb.dim; ++j) {
                                    MetricElem el{};
                                    el.xo = xl.row_off[la] + static_cast<int64_t>(i) * xl.width[la] + xl.seg_col[la * 16 + s] + j;
                                    el.a = La.off - Ga.off + i;
                                    el.bs = (boff + j) * 16 + s;
                                    T.e.push_back(el);
                                }
                            }
                        }
                }
                if (T.e.empty()) continue;
                if (static_cast<int>(T.e.size()) > max_dim) continue;  // left to the diagonal correction
                const int64_t loff = Le.lay[1].off[ga];
                const int64_t roff = Re.lay[1].off[gb];
                if (loff < 0 || roff < 0) return SPMPS_OK;  // no N environment block: keep the diagonal correction
                T.b.dim = static_cast<int>(T.e.size());
                T.b.lda = Ga.dim;
                T.b.ldb = br.groups[gb].dim;
                T.b.loff = loff;
                T.b.roff = roff;
                tmp.push_back(std::move(T));
            }
    }
    (void)ngr;
    std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp& a, const Tmp& b) { return a.b.dim > b.b.dim; });
    M.blocks.clear();
    M.elems.clear();
    int64_t mat = 0;
    for (Tmp& T : tmp) {
        T.b.elem_off = static_cast<int64_t>(M.elems.size());
        T.b.mat_off = mat;
        mat += (static_cast<int64_t>(T.b.dim) * T.b.dim + 31) / 32 * 32;
        M.elems.insert(M.elems.end(), T.e.begin(), T.e.end());
        M.blocks.push_back(T.b);
    }
    M.n_blocks = static_cast<int>(M.blocks.size());
    M.n_x = xl.size;
    M.mat_total = mat;
    M.max_dim = M.n_blocks ? M.blocks[0].dim : 0;
    M.n_elems = static_cast<int64_t>(M.elems.size());
    if (M.n_blocks == 0 || mat > kMetricMaxDoubles) return SPMPS_OK;
    // per-beta constants
    std::vector<MetricBeta> betas(G);
    for (int g = 0; g < G; ++g) {
        betas[g].c = h->cg[g];
        site_rotation(h->beta[g], betas[g].r);
        betas[g].lbase = Le.base[1 * G + g];
        betas[g].rbase = Re.base[1 * G + g];
    }
    // assembly tiles (lower 32 x 32 tiles) and the panel steps of the factorisation
    std::vector<int4> tiles;
    for (int b = 0; b < M.n_blocks; ++b) {
        const int T = (M.blocks[b].dim + 31) / 32;
        for (int ti = 0; ti < T; ++ti)
            for (int tj = 0; tj <= ti; ++tj) tiles.push_back(make_int4(b, ti, tj, 0));
    }
    std::vector<int> prefix;
    M.alive.clear();
    M.steps_trsm.clear();
    M.steps_syrk.clear();
    for (int p0 = 0; p0 < M.max_dim; p0 += kPanel) {
        int alive = 0;
        while (alive < M.n_blocks && M.blocks[alive].dim > p0) ++alive;
        M.alive.push_back(alive);
        M.steps_trsm.push_back(static_cast<int>(prefix.size()));
        int acc = 0;
        for (int b = 0; b < alive; ++b) {
            prefix.push_back(acc);
            const int below = std::max(0, M.blocks[b].dim - p0 - kPanel);
            acc += (below + kTrsmRows - 1) / kTrsmRows;
        }
        prefix.push_back(acc);
        M.steps_syrk.push_back(static_cast<int>(prefix.size()));
        acc = 0;
        for (int b = 0; b < alive; ++b) {
            prefix.push_back(acc);
            const int below = std::max(0, M.blocks[b].dim - p0 - kPanel);
            const int T = (below + kSyrkTile - 1) / kSyrkTile;
            acc += T * (T + 1) / 2;
        }
        prefix.push_back(acc);
    }
    cudaStream_t st = h->stream;
    CK(upload(M.d_blocks, M.blocks, st));
    CK(upload(M.d_elems, M.elems, st));
    CK(upload(M.d_betas, betas, st));
    CK(upload(M.d_tiles, tiles, st));
    CK(upload(M.d_prefix, prefix, st));
    CK(M.mats.ensure(std::max<int64_t>(1, M.mat_total) * sizeof(double)));
    CK(M.ybuf.ensure(std::max<int64_t>(1, M.n_elems) * sizeof(double)));
    CK(M.status.ensure(sizeof(int)));
    CK(cudaMemsetAsync(M.status.p, 0, sizeof(int), st));
    const MetricBlock* db = M.d_blocks.as<MetricBlock>();
    double* mats = M.mats.as<double>();
    k_metric_assemble<<<static_cast<unsigned>(tiles.size()), 256, 0, st>>>(
        db, M.d_elems.as<MetricElem>(), M.d_betas.as<MetricBeta>(), G, Le.buf.as<double>(), Re.buf.as<double>(),
        M.d_tiles.as<int4>(), kMetricShift, mats);
    CK(cudaGetLastError());
    ++h->launches;
    const int* pre = M.d_prefix.as<int>();
    for (size_t step = 0; step < M.alive.size(); ++step) {
        const int p0 = static_cast<int>(step) * kPanel;
        const int alive = M.alive[step];
        k_chol_diag<<<alive, 32, 0, st>>>(db, mats, p0, M.status.as<int>());
        CK(cudaGetLastError());
        ++h->launches;
        const int nt = prefix[M.steps_trsm[step] + alive];
        if (nt > 0) {
            k_chol_trsm<<<nt, kTrsmRows, 0, st>>>(db, mats, p0, pre + M.steps_trsm[step], alive);
            CK(cudaGetLastError());
            ++h->launches;
        }
        const int ns = prefix[M.steps_syrk[step] + alive];
        if (ns > 0) {
            k_chol_syrk<<<ns, 256, 0, st>>>(db, mats, p0, pre + M.steps_syrk[step], alive);
            CK(cudaGetLastError());
            ++h->launches;
        }
    }
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, M.status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    M.ok = bad == 0;
    return SPMPS_OK;
}

spmps_status metric_solve(spmps_t* h, MetricState& M, const double* in, double* out, cudaStream_t st) {
    if (!M.ok) return fail(h, SPMPS_ERR_STATE, "metric blocks not prepared");
    k_metric_solve<<<M.n_blocks, 512, 0, st>>>(M.d_blocks.as<MetricBlock>(), M.d_elems.as<MetricElem>(),
                                                M.mats.as<double>(), in, out, M.ybuf.as<double>());
    CK(cudaGetLastError());
    ++h->launches;
    return SPMPS_OK;
}

}  // namespace eng
}  // namespace spmps
