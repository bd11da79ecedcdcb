// Host-side model of the SP-MPS problem: bond labels and block layouts, the MPOs, and the
// quadrature of the spin projector.
//
// Quadrature: Eq. PSMM reduces the projector to an integral over beta with weight
// sin(beta) d^S_MM(beta); Eq. pmpo evaluates it with Gauss-Legendre points in x = cos(beta).
// The rotation of one site is the 4x4 matrix of Eq. expSy.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "core.h"

namespace spmps {

// ---- bonds ----------------------------------------------------------------------------------

int Bond::find(int n, int tm) const {
    int lo = 0, hi = static_cast<int>(labels.size());
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        const Label& l = labels[mid];
        if (l.n < n || (l.n == n && l.tm < tm)) lo = mid + 1; else hi = mid;
    }
    if (lo < static_cast<int>(labels.size()) && labels[lo].n == n && labels[lo].tm == tm) return lo;
    return -1;
}

int Bond::group_of(int n) const {
    for (size_t g = 0; g < groups.size(); ++g)
        if (groups[g].n == n) return static_cast<int>(g);
    return -1;
}

void Bond::finalize() {
    std::sort(labels.begin(), labels.end(), [](const Label& a, const Label& b) {
        return a.n < b.n || (a.n == b.n && a.tm < b.tm);
    });
    groups.clear();
    int off = 0;
    for (size_t i = 0; i < labels.size(); ++i) {
        Label& l = labels[i];
        l.off = off;
        if (groups.empty() || groups.back().n != l.n)
            groups.push_back(Group{l.n, off, 0, static_cast<int>(i), 0});
        groups.back().dim += l.dim;
        groups.back().count += 1;
        l.group = static_cast<int>(groups.size()) - 1;
        off += l.dim;
    }
    D = off;
}

RowBlockLayout make_row_block_layout(const Bond& left, const Bond& right, int ns) {
    RowBlockLayout L;
    L.ns = ns;
    const int nl = static_cast<int>(left.labels.size());
    L.row_off.resize(nl);
    L.width.resize(nl);
    L.seg_col.assign(static_cast<size_t>(nl) * ns, -1);
    L.seg_label.assign(static_cast<size_t>(nl) * ns, -1);
    int64_t off = 0;
    for (int i = 0; i < nl; ++i) {
        const Label& a = left.labels[i];
        int w = 0;
        for (int s = 0; s < ns; ++s) {
            int r = right.find(a.n + qn_n(ns, s), a.tm + qn_m(ns, s));
            if (r < 0) continue;
            L.seg_col[i * ns + s] = w;
            L.seg_label[i * ns + s] = r;
            w += right.labels[r].dim;
        }
        L.row_off[i] = off;
        L.width[i] = w;
        off += static_cast<int64_t>(a.dim) * w;
    }
    L.size = off;
    return L;
}

ColLayout make_col_layout(const Bond& right, int n0, int ns, int sign) {
    ColLayout C;
    C.col.assign(ns, -1);
    C.group.assign(ns, -1);
    int w = 0;
    for (int s = 0; s < ns; ++s) {
        int g = right.group_of(n0 + sign * qn_n(ns, s));
        if (g < 0) continue;
        C.col[s] = w;
        C.group[s] = g;
        w += right.groups[g].dim;
    }
    C.width = w;
    return C;
}

TilePolicy tile_candidate(int i) {
    TilePolicy p;
    switch (i) {
        case 1: p.wb_kmin = 32; break;
        case 2: p.wb_kmin = 128; break;
        case 3: p.wb_kmin = 1 << 30; break;  // register tiles only
        case 4: p.wb_mn_max = 1024; break;
        case 5: p.wb_elems = 128; break;
        default: break;
    }
    return p;
}

void GemmPlan::add_tiles(const TilePolicy& pol) {
    // register-tiled shapes 0..4 (rows x cols per warp); shape 5 = warp block for long reductions
    static const int shp[5][2] = {{16, 16}, {4, 64}, {64, 4}, {32, 8}, {8, 32}};
    tiles.clear();
    for (size_t t = 0; t < tasks.size(); ++t) {
        const GemmTask& T = tasks[t];
        int64_t ktot = 0;
        for (int q = 0; q < T.nseg; ++q) ktot += segs[T.seg0 + q].K;
        if (ktot >= pol.wb_kmin && static_cast<int64_t>(T.M) * T.N <= pol.wb_mn_max) {
            const int tm = T.M < 32 ? T.M : 32;
            int tn = (pol.wb_elems < 256 ? pol.wb_elems : 256) / tm;  // the kernel holds <= 256 outputs
            if (tn < 1) tn = 1;
            if (tn > 32) tn = 32;
            if (tn > T.N) tn = T.N;
            for (int m0 = 0; m0 < T.M; m0 += tm)
                for (int n0 = 0; n0 < T.N; n0 += tn) {
                    GemmTile g{};
                    g.task = static_cast<int>(t);
                    g.m0 = static_cast<int16_t>(m0);
                    g.n0 = static_cast<int16_t>(n0);
                    g.tm = static_cast<int16_t>(T.M - m0 < tm ? T.M - m0 : tm);
                    g.tn = static_cast<int16_t>(T.N - n0 < tn ? T.N - n0 : tn);
                    g.shape = 5;
                    tiles.push_back(g);
                }
            continue;
        }
        int best = 0;
        int64_t best_cost = -1;
        for (int s = 0; s < 5; ++s) {
            const int64_t tm = shp[s][0], tn = shp[s][1];
            const int64_t cost = ((T.M + tm - 1) / tm) * tm * ((T.N + tn - 1) / tn) * tn;
            if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = s; }
        }
        for (int m0 = 0; m0 < T.M; m0 += shp[best][0])
            for (int n0 = 0; n0 < T.N; n0 += shp[best][1]) {
                GemmTile g{};
                g.task = static_cast<int>(t);
                g.m0 = static_cast<int16_t>(m0);
                g.n0 = static_cast<int16_t>(n0);
                g.shape = best;
                tiles.push_back(g);
            }
    }
}

void GemmPlan::add_tc_tiles() {
    tc_tiles.clear();
    for (size_t t = 0; t < tasks.size(); ++t) {
        const GemmTask& T = tasks[t];
        for (int m0 = 0; m0 < T.M; m0 += 32)
            for (int n0 = 0; n0 < T.N; n0 += 32) {
                GemmTile g{};
                g.task = static_cast<int>(t);
                g.m0 = static_cast<int16_t>(m0);
                g.n0 = static_cast<int16_t>(n0);
                g.tm = static_cast<int16_t>(T.M - m0 < 32 ? T.M - m0 : 32);
                g.tn = static_cast<int16_t>(T.N - n0 < 32 ? T.N - n0 : 32);
                g.shape = 6;
                tc_tiles.push_back(g);
            }
    }
}

// ---- MPOs -----------------------------------------------------------------------------------

namespace {
// One spin-orbital (Eq. JWtrans): a+ = [[0,0],[1,0]], sigma_z = diag(1,-1).  A spatial site is
// alpha (x) beta with alpha first: a+_alpha = a+ (x) 1, a+_beta = sigma_z (x) a+.
void kron2(const double a[4], const double b[4], double out[16]) {
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) out[(2 * i + k) * 4 + (2 * j + l)] = a[i * 2 + j] * b[k * 2 + l];
}
void matmul4(const double a[16], const double b[16], double out[16]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += a[i * 4 + k] * b[k * 4 + j];
            out[i * 4 + j] = s;
        }
}
void transpose4(const double a[16], double out[16]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) out[j * 4 + i] = a[i * 4 + j];
}
struct LocalOps {
    double I[16], P[16], cdag_a[16], cdag_b[16], c_a[16], c_b[16], n_a[16], n_b[16];
    LocalOps() {
        const double id[4] = {1, 0, 0, 1}, sz[4] = {1, 0, 0, -1}, cd[4] = {0, 0, 1, 0};
        kron2(id, id, I);
        kron2(sz, sz, P);
        kron2(cd, id, cdag_a);
        kron2(sz, cd, cdag_b);
        transpose4(cdag_a, c_a);
        transpose4(cdag_b, c_b);
        matmul4(cdag_a, c_a, n_a);
        matmul4(cdag_b, c_b, n_b);
    }
};

MPO make_mpo(int K, int dw_bulk) {
    std::vector<int> dims(K + 1, dw_bulk);
    dims[0] = dims[K] = 1;
    MPO m;
    m.init(K, dims);
    return m;
}

// Place the bulk operator matrix `op` at (wl, wr) of every site, restricted to the boundary row
// `first` on site 0 and the boundary column `last` on site K-1.
void place(MPO& m, int wl, int wr, const double op[16], double scale, int first, int last) {
    for (int k = 0; k < m.K; ++k) {
        int l = wl, r = wr;
        if (k == 0) { if (wl != first) continue; l = 0; }
        if (k == m.K - 1) { if (wr != last) continue; r = 0; }
        m.add(k, l, r, op, scale);
    }
}
}  // namespace

void MPO::init(int K_, const std::vector<int>& dims) {
    K = K_;
    dw = dims;
    cn.clear();
    E.assign(K, {});
    wr_ptr.assign(K, {});
    by_wl.assign(K, {});
    wl_ptr.assign(K, {});
    pending_.assign(K, {});
}

void MPO::add(int k, int wl, int wr, const double* op, double scale) {
    if (pending_.size() != static_cast<size_t>(K)) pending_.assign(K, {});
    MpoEntry e;
    e.wl = wl;
    e.wr = wr;
    for (int i = 0; i < 16; ++i) e.op[i] = scale * op[i];
    pending_[k].push_back({(static_cast<uint64_t>(wr) << 32) | static_cast<uint32_t>(wl), static_cast<int>(E[k].size())});
    E[k].push_back(e);
}

void MPO::finalize() {
    if (pending_.size() != static_cast<size_t>(K)) pending_.assign(K, {});
    for (int k = 0; k < K; ++k) {
        auto& pend = pending_[k];
        // stable order by (wr, wl), then merge duplicates
        std::stable_sort(pend.begin(), pend.end(),
                         [](const std::pair<uint64_t, int>& a, const std::pair<uint64_t, int>& b) { return a.first < b.first; });
        std::vector<MpoEntry> out;
        out.reserve(E[k].size());
        if (pend.empty()) {
            // already finalized once (or built without add): re-sort the stored entries
            std::vector<MpoEntry> cur = E[k];
            std::stable_sort(cur.begin(), cur.end(), [](const MpoEntry& a, const MpoEntry& b) {
                return a.wr != b.wr ? a.wr < b.wr : a.wl < b.wl;
            });
            for (const auto& e : cur) {
                if (!out.empty() && out.back().wl == e.wl && out.back().wr == e.wr) {
                    for (int i = 0; i < 16; ++i) out.back().op[i] += e.op[i];
                } else {
                    out.push_back(e);
                }
            }
        } else {
            for (size_t i = 0; i < pend.size(); ++i) {
                const MpoEntry& e = E[k][pend[i].second];
                if (!out.empty() && out.back().wl == e.wl && out.back().wr == e.wr) {
                    for (int q = 0; q < 16; ++q) out.back().op[q] += e.op[q];
                } else {
                    out.push_back(e);
                }
            }
        }
        // drop all-zero entries
        std::vector<MpoEntry> nz;
        nz.reserve(out.size());
        for (const auto& e : out) {
            bool any = false;
            for (double v : e.op) any = any || v != 0.0;
            if (any) nz.push_back(e);
        }
        E[k].swap(nz);
        pend.clear();
        pend.shrink_to_fit();
        // indices
        const int dr = dw[k + 1], dl = dw[k];
        wr_ptr[k].assign(dr + 1, 0);
        for (const auto& e : E[k]) ++wr_ptr[k][e.wr + 1];
        for (int u = 0; u < dr; ++u) wr_ptr[k][u + 1] += wr_ptr[k][u];
        by_wl[k].resize(E[k].size());
        for (size_t i = 0; i < E[k].size(); ++i) by_wl[k][i] = static_cast<int>(i);
        std::stable_sort(by_wl[k].begin(), by_wl[k].end(), [&](int a, int b) {
            const MpoEntry& x = E[k][a];
            const MpoEntry& y = E[k][b];
            return x.wl != y.wl ? x.wl < y.wl : x.wr < y.wr;
        });
        wl_ptr[k].assign(dl + 1, 0);
        for (const auto& e : E[k]) ++wl_ptr[k][e.wl + 1];
        for (int w = 0; w < dl; ++w) wl_ptr[k][w + 1] += wl_ptr[k][w];
    }
}

double MPO::get(int k, int wl, int wr, int s, int t) const {
    const auto& v = E[k];
    int lo = wr_ptr[k][wr], hi = wr_ptr[k][wr + 1];
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (v[mid].wl < wl) lo = mid + 1;
        else hi = mid;
    }
    if (lo < wr_ptr[k][wr + 1] && v[lo].wl == wl) return v[lo].op[s * 4 + t];
    return 0.0;
}

size_t MPO::entries() const {
    size_t n = 0;
    for (const auto& v : E) n += v.size();
    return n;
}

bool MPO::finalize_charges(std::string* err) {
    cn.assign(K + 1, {});
    for (int b = 0; b <= K; ++b) cn[b].assign(dw[b], 0);
    std::vector<std::vector<char>> seen(K + 1);
    for (int b = 0; b <= K; ++b) seen[b].assign(dw[b], 0);
    seen[0][0] = 1;
    bool pruned = false;
    for (int k = 0; k < K; ++k) {
        // entries leaving a channel that no nonzero path from the left boundary reaches cannot
        // contribute (their left environment vanishes): drop them
        std::vector<MpoEntry> live;
        live.reserve(E[k].size());
        for (const auto& e : E[k])
            if (seen[k][e.wl]) live.push_back(e);
        if (live.size() != E[k].size()) {
            E[k].swap(live);
            pruned = true;
        }
        for (const auto& e : E[k])
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    if (e.op[s * 4 + t] == 0.0) continue;
                    const int c = cn[k][e.wl] + kLocalN[s] - kLocalN[t];
                    if (!seen[k + 1][e.wr]) {
                        seen[k + 1][e.wr] = 1;
                        cn[k + 1][e.wr] = c;
                    } else if (cn[k + 1][e.wr] != c) {
                        if (err) *err = "MPO does not conserve particle number";
                        return false;
                    }
                }
    }
    if (cn[K][0] != 0) {
        if (err) *err = "MPO changes the particle number";
        return false;
    }
    if (pruned) finalize();  // rebuild the per-wr / per-wl indices
    return true;
}

MPO mpo_nearest_neighbour(int K, const std::vector<double>& eps, const std::vector<double>& hop,
                          const std::vector<double>& U, double ecore) {
    // H = sum_k eps_k (n_ka + n_kb) + sum_k hop_k sum_s (a+_{k s} a_{k+1 s} + h.c.)
    //     + sum_k U_k n_ka n_kb + ecore.
    // Channels: 0 = nothing placed, 1..4 = a+_a P, a+_b P, P a_a, P a_b placed on the left
    // (P the site parity, the Jordan-Wigner string of the site), 5 = complete.
    static const LocalOps o;
    MPO m = make_mpo(K, 6);
    double tmp[16], local[16];
    place(m, 0, 0, o.I, 1.0, 0, 5);
    place(m, 5, 5, o.I, 1.0, 0, 5);
    for (int k = 0; k < K; ++k) {
        // on-site part of site k only: write it on that site's (0, 5) entry
        matmul4(o.n_a, o.n_b, tmp);
        for (int i = 0; i < 16; ++i) local[i] = U[k] * tmp[i] + eps[k] * (o.n_a[i] + o.n_b[i]);
        if (k == 0) for (int i = 0; i < 16; ++i) local[i] += ecore * o.I[i];
        const int l = 0, r = k == K - 1 ? 0 : 5;
        m.add(k, l, r, local);
    }
    for (int k = 0; k + 1 < K; ++k) {
        // opening legs on site k, closing legs (times hop_k) on site k+1
        const int l = 0, r_open[4] = {1, 2, 3, 4};
        const double* opens[4];
        double oa[16], ob[16], oc[16], od[16];
        matmul4(o.cdag_a, o.P, oa);
        matmul4(o.cdag_b, o.P, ob);
        matmul4(o.P, o.c_a, oc);
        matmul4(o.P, o.c_b, od);
        opens[0] = oa; opens[1] = ob; opens[2] = oc; opens[3] = od;
        const double* closes[4] = {o.c_a, o.c_b, o.cdag_a, o.cdag_b};
        for (int c = 0; c < 4; ++c) {
            m.add(k, l, r_open[c], opens[c]);
            const int rr = k + 1 == K - 1 ? 0 : 5;
            m.add(k + 1, r_open[c], rr, closes[c], hop[k]);
        }
    }
    m.finalize();
    return m;
}

MPO mpo_hubbard(int K, double t, double U) {
    return mpo_nearest_neighbour(K, std::vector<double>(K, 0.0), std::vector<double>(K > 1 ? K - 1 : 0, -t),
                                 std::vector<double>(K, U), 0.0);
}

MPO mpo_s2(int K) {
    // Eq. Sfac: rows/columns (S^2, S+, S-, Sz, I) of the recursion over the right part.
    static const LocalOps o;
    double sp[16] = {0}, sm[16] = {0}, szz[16] = {0}, s2[16] = {0};
    sp[2 * 4 + 1] = 1.0;
    sm[1 * 4 + 2] = 1.0;
    szz[1 * 4 + 1] = -0.5;
    szz[2 * 4 + 2] = 0.5;
    s2[1 * 4 + 1] = 0.75;
    s2[2 * 4 + 2] = 0.75;
    MPO m = make_mpo(K, 5);
    place(m, 0, 0, o.I, 1.0, 0, 4);
    place(m, 0, 1, sm, 1.0, 0, 4);
    place(m, 0, 2, sp, 1.0, 0, 4);
    place(m, 0, 3, szz, 2.0, 0, 4);
    place(m, 0, 4, s2, 1.0, 0, 4);
    place(m, 1, 1, o.I, 1.0, 0, 4);
    place(m, 1, 4, sp, 1.0, 0, 4);
    place(m, 2, 2, o.I, 1.0, 0, 4);
    place(m, 2, 4, sm, 1.0, 0, 4);
    place(m, 3, 3, o.I, 1.0, 0, 4);
    place(m, 3, 4, szz, 1.0, 0, 4);
    place(m, 4, 4, o.I, 1.0, 0, 4);
    m.finalize();
    return m;
}

MPO mpo_identity(int K) {
    static const LocalOps o;
    MPO m = make_mpo(K, 1);
    place(m, 0, 0, o.I, 1.0, 0, 0);
    m.finalize();
    return m;
}

void site_rotation(double beta, double r[16]) {
    // Eq. expSy in the basis {0, b, a, ab}
    const double c = std::cos(0.5 * beta), s = std::sin(0.5 * beta);
    for (int i = 0; i < 16; ++i) r[i] = 0.0;
    r[0] = 1.0;
    r[1 * 4 + 1] = c;
    r[1 * 4 + 2] = s;
    r[2 * 4 + 1] = -s;
    r[2 * 4 + 2] = c;
    r[15] = 1.0;
}

MPO mpo_rotated(const MPO& m, double beta) {
    double r[16];
    site_rotation(beta, r);
    MPO out = m;
    for (int k = 0; k < m.K; ++k)
        for (auto& e : out.E[k]) {
            double tmp[16];
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    double acc = 0.0;
                    for (int u = 0; u < 4; ++u) acc += e.op[s * 4 + u] * r[u * 4 + t];
                    tmp[s * 4 + t] = acc;
                }
            for (int i = 0; i < 16; ++i) e.op[i] = tmp[i];
        }
    return out;
}

// ---- quadrature -----------------------------------------------------------------------------

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    // Newton iteration on the Legendre polynomial P_n from the standard first guesses
    // cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2).
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            if (n == 0) p1 = 1.0;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    // ascending order
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
    std::vector<double> xs(n), ws(n);
    for (int i = 0; i < n; ++i) { xs[i] = x[idx[i]]; ws[i] = w[idx[i]]; }
    x.swap(xs);
    w.swap(ws);
}

double wigner_small_d(int two_j, int two_mp, int two_m, double beta) {
    // Wigner's explicit sum for d^j_{m'm}(beta), evaluated with log-factorials.
    auto lf = [](int k) { return std::lgamma(static_cast<double>(k) + 1.0); };
    const int jpmp = (two_j + two_mp) / 2, jmmp = (two_j - two_mp) / 2;
    const int jpm = (two_j + two_m) / 2, jmm = (two_j - two_m) / 2;
    const int mpmm = (two_mp - two_m) / 2;
    const double c = std::cos(0.5 * beta), s = std::sin(0.5 * beta);
    const double half = 0.5 * (lf(jpmp) + lf(jmmp) + lf(jpm) + lf(jmm));
    long double sum = 0.0L;
    for (int k = 0; k <= two_j; ++k) {
        const int a1 = jpm - k, a2 = mpmm + k, a3 = jmmp - k;
        if (a1 < 0 || a2 < 0 || a3 < 0) continue;
        const double mag = std::exp(half - lf(a1) - lf(k) - lf(a2) - lf(a3));
        const int pc = a1 + a3, ps = a2 + k;
        double term = mag * std::pow(c, pc) * std::pow(s, ps);
        if ((a2 & 1) != 0) term = -term;
        sum += term;
    }
    return static_cast<double>(sum);
}

}  // namespace spmps
