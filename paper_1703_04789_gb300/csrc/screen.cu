// Approximate M-sector screening (Sec. 2.3.1, closing paragraph): Frobenius norms of the
// (bra label, ket label) sub-blocks of an environment, per operator, beta point and channel, on
// the device; the planner drops the block products whose environment sub-block is below a
// threshold relative to the largest sub-block of its channel.
#include <algorithm>
#include <cmath>

#include "engine.h"

namespace spmps {

namespace {

struct SubBlock {
    int64_t off;
    int rows, cols, ld, pad;
};

// One warp per sub-block: its Frobenius norm.
__global__ void __launch_bounds__(256) k_subblock_norms(const double* __restrict__ E, const SubBlock* __restrict__ sb,
                                                        int n, double* __restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n) return;
    const SubBlock b = sb[w];
    double acc = 0.0;
    for (int e = lane; e < b.rows * b.cols; e += 32) {
        const double v = E[b.off + static_cast<int64_t>(e / b.cols) * b.ld + e % b.cols];
        acc = fma(v, v, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[w] = sqrt(acc);
}

}  // namespace

namespace eng {

spmps_status env_subblock_norms(spmps_t* h, const EnvStore& E, const Bond& b, int bond, EnvNorms& out) {
    const int G = h->G, nops = h->ops.n_ops();
    const int ng = static_cast<int>(b.groups.size());
    out.start.clear();
    out.ncols.clear();
    out.wmax.clear();
    out.wbase.assign(nops + 1, 0);
    out.dw.assign(nops, 0);
    out.ngroups = ng;
    std::vector<SubBlock> list;
    std::vector<int> owner;  // (op, g, w) slot of each sub-block
    for (int op = 0; op < nops; ++op) {
        const std::vector<int>& cn = h->ops.mpo[op].cn[bond];
        const int dw = static_cast<int>(cn.size());
        out.dw[op] = dw;
        out.wbase[op] = static_cast<int>(out.wmax.size());
        for (int g = 0; g < G; ++g)
            for (int w = 0; w < dw; ++w) {
                const int slot = static_cast<int>(out.wmax.size());
                out.wmax.push_back(0.0);
                for (int ga = 0; ga < ng; ++ga) {
                    const int64_t loff = E.lay[op].off[w * ng + ga];
                    const int gp = b.group_of(b.groups[ga].n - cn[w]);
                    if (loff < 0 || gp < 0) {
                        out.start.push_back(-1);
                        out.ncols.push_back(0);
                        continue;
                    }
                    const Group& Ga = b.groups[ga];
                    const Group& Gp = b.groups[gp];
                    out.start.push_back(static_cast<int64_t>(list.size()));
                    out.ncols.push_back(Gp.count);
                    for (int la = Ga.first; la < Ga.first + Ga.count; ++la)
                        for (int lp = Gp.first; lp < Gp.first + Gp.count; ++lp) {
                            SubBlock s{};
                            s.off = E.base[op * G + g] + loff + static_cast<int64_t>(b.labels[la].off - Ga.off) * Gp.dim +
                                    (b.labels[lp].off - Gp.off);
                            s.rows = b.labels[la].dim;
                            s.cols = b.labels[lp].dim;
                            s.ld = Gp.dim;
                            list.push_back(s);
                            owner.push_back(slot);
                        }
                }
            }
    }
    out.wbase[nops] = static_cast<int>(out.wmax.size());
    out.norms.assign(list.size(), 0.0);
    if (list.empty()) return SPMPS_OK;
    DevMem d_list, d_out;
    CK(upload(d_list, list, h->stream));
    CK(d_out.ensure(list.size() * sizeof(double)));
    const int n = static_cast<int>(list.size());
    k_subblock_norms<<<(n + 7) / 8, 256, 0, h->stream>>>(E.buf.as<double>(), d_list.as<SubBlock>(), n, d_out.as<double>());
    CK(cudaGetLastError());
    ++h->launches;
    CK(cudaMemcpyAsync(out.norms.data(), d_out.p, list.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < owner.size(); ++i) out.wmax[owner[i]] = std::max(out.wmax[owner[i]], out.norms[i]);
    return SPMPS_OK;
}

}  // namespace eng
}  // namespace spmps
