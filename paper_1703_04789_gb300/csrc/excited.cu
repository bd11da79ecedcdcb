// State-specific excited states (Sec. 2.3.2, Eq. orthoB, Fig. spmpsex): the running state is
// optimised subject to <Psi_j|P|Psi> = 0 for every lower state Psi_j.  At sites (k, k+1) the
// overlap is linear in the two-site tensor x, <Psi_j|P|Psi> = B_j . x, and the local problem
// (Eq. geproblem) is solved in the range of Q = 1 - V V^T, V the QR of the B_j.
//
// B_j = sum_g c_g (L_g^T) x0_j (r_g^T (x) r_g^T) (R_g^T)-network: with the cross environments built
// with bra = the running state and ket = Psi_j, and every site rotation taken at -beta_g
// (r(-b) = r(b)^T), B_j is the projected metric action of this network on the lower state's
// two-site tensor x0_j: the three contraction phases of the projected action with the identity
// MPO (one channel), bra and ket on different bond structures.
#include <algorithm>
#include <cmath>

#include "engine.h"

namespace spmps {
namespace eng {

namespace {

// Layout of a cross environment on one bond: per bra N-group, a block gdim_bra(G) x gdim_ket(G')
// with G' the ket group of the same particle number (the rotated identity conserves it).
EnvLayout make_cross_layout(const Bond& bra, const Bond& ket) {
    EnvLayout L;
    L.n_groups = static_cast<int>(bra.groups.size());
    L.off.assign(L.n_groups, -1);
    L.ld.assign(L.n_groups, 0);
    int64_t off = 0;
    for (int g = 0; g < L.n_groups; ++g) {
        const int gk = ket.group_of(bra.groups[g].n);
        if (gk < 0) continue;
        L.off[g] = off;
        L.ld[g] = ket.groups[gk].dim;
        off += static_cast<int64_t>(bra.groups[g].dim) * ket.groups[gk].dim;
    }
    L.size = off;
    return L;
}

spmps_status cross_prepare(spmps_t* h, EnvStore& E, const Bond& bra, const Bond& ket) {
    E.lay.assign(1, make_cross_layout(bra, ket));
    E.base.assign(h->G, 0);
    for (int g = 0; g < h->G; ++g) E.base[g] = static_cast<int64_t>(g) * E.lay[0].size;
    E.total = static_cast<int64_t>(h->G) * E.lay[0].size;
    CK(E.buf.ensure(std::max<int64_t>(1, E.total) * sizeof(double)));
    return SPMPS_OK;
}

// boundary bonds 0 and K: a single 1 x 1 block of value 1 per beta point
spmps_status cross_boundary(spmps_t* h, EnvStore& E, const Bond& bra, const Bond& ket) {
    spmps_status st = cross_prepare(h, E, bra, ket);
    if (st != SPMPS_OK) return st;
    std::vector<double> ones(static_cast<size_t>(std::max<int64_t>(E.total, 1)), 0.0);
    for (int g = 0; g < h->G; ++g)
        for (size_t i = 0; i < E.lay[0].off.size(); ++i)
            if (E.lay[0].off[i] >= 0) ones[E.base[g] + E.lay[0].off[i]] = 1.0;
    CK(cudaMemcpyAsync(E.buf.p, ones.data(), E.total * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    E.valid = true;
    return SPMPS_OK;
}

void set_ranges(Plan& P, int G) {
    P.A.clear(); P.B.clear(); P.C.clear();
    P.task_rng_kept = false;
    P.tileA_rng.assign(G + 1, 0);
    P.tileC_rng.assign(G + 1, 0);
    P.combB_rng.assign(G + 1, 0);
}

void close_ranges(Plan& P, int G, int64_t t1, int64_t t2) {
    P.tileA_rng[G] = static_cast<int>(P.A.tasks.size());
    P.combB_rng[G] = static_cast<int>(P.B.outs.size());
    P.tileC_rng[G] = static_cast<int>(P.C.tasks.size());
    P.t1_size = t1;
    P.t2_size = t2;
    P.flops = P.A.flops + P.B.flops + P.C.flops;
}

// Left update at site i: L'(bond i+1) from L(bond i), bra A = running A[i] (slot 1), ket A = the
// lower state's A[i] (slot 0).  Slots: 3 = T1, 4 = T2, 5 = L, 7 = L'.
void build_cross_left(spmps_t* h, const LowerState& Ls, int i, const EnvStore& Lo, const EnvStore& Ln, Plan& P) {
    const Bond& bl = h->bonds[i];
    const Bond& br = h->bonds[i + 1];
    const RowBlockLayout& ab = h->alay[i];
    const Bond& kl = Ls.bonds[i];
    const Bond& kr = Ls.bonds[i + 1];
    const RowBlockLayout& ak = Ls.alay[i];
    const int G = h->G, ngl = static_cast<int>(bl.groups.size()), ngr = static_cast<int>(br.groups.size());
    set_ranges(P, G);
    std::vector<int> cmap_off(kl.labels.size(), -1);
    for (size_t l = 0; l < kl.labels.size(); ++l) {
        if (ak.width[l] == 0) continue;
        const ColLayout CL = make_col_layout(kr, kl.labels[l].n, 4, +1);
        cmap_off[l] = static_cast<int>(P.A.cmaps.size());
        for (int s = 0; s < 4; ++s) {
            const int lb = ak.seg_label[l * 4 + s];
            if (lb < 0) continue;
            const Label& Lb = kr.labels[lb];
            const int base = CL.col[s] + (Lb.off - kr.groups[Lb.group].off);
            for (int j = 0; j < Lb.dim; ++j) P.A.cmaps.push_back(base + j);
        }
    }
    int64_t t1 = 0, t2 = 0;
    for (int g = 0; g < G; ++g) {
        const MpoEntry& e = Ls.rot[g].E[i][0];
        P.tileA_rng[g] = static_cast<int>(P.A.tasks.size());
        P.combB_rng[g] = static_cast<int>(P.B.outs.size());
        P.tileC_rng[g] = static_cast<int>(P.C.tasks.size());
        std::vector<int64_t> o1(ngl, -1), o2(ngl, -1);
        std::vector<ColLayout> c1(ngl);
        for (int ga = 0; ga < ngl; ++ga) {
            const int n0 = bl.groups[ga].n;
            const int gk = kl.group_of(n0);
            const int64_t loff = Lo.lay[0].off[ga];
            if (gk < 0 || loff < 0) continue;
            ColLayout CL = make_col_layout(kr, n0, 4, +1);
            if (CL.width == 0) continue;
            const int M = bl.groups[ga].dim;
            o1[ga] = t1;
            for (int l = kl.groups[gk].first; l < kl.groups[gk].first + kl.groups[gk].count; ++l) {
                if (ak.width[l] == 0) continue;
                const Label& Ll = kl.labels[l];
                GemmTask T{};
                T.c = handle(3, t1);
                T.cmap = cmap_off[l];
                T.M = M;
                T.N = ak.width[l];
                T.ldc = CL.width;
                T.seg0 = static_cast<int>(P.A.segs.size());
                T.nseg = 1;
                GemmSeg sg{};
                sg.a = handle(5, Lo.base[g] + loff + (Ll.off - kl.groups[gk].off));
                sg.a_rs = kl.groups[gk].dim;
                sg.a_cs = 1;
                sg.K = Ll.dim;
                sg.b = handle(0, ak.row_off[l]);
                sg.b_rs = ak.width[l];
                sg.b_cs = 1;
                P.A.segs.push_back(sg);
                P.A.tasks.push_back(T);
                P.A.flops += 2.0 * T.M * T.N * sg.K;
            }
            t1 += static_cast<int64_t>(M) * CL.width;
            c1[ga] = CL;
        }
        // T2[Ga][:, s, :] = sum_t r(-b)[s, t] T1[Ga][:, t, :]  (the ket's columns for both)
        for (int ga = 0; ga < ngl; ++ga) {
            if (o1[ga] < 0) continue;
            const ColLayout& CL = c1[ga];
            const int M = bl.groups[ga].dim;
            o2[ga] = t2;
            for (int s = 0; s < 4; ++s) {
                if (CL.col[s] < 0) continue;
                CombOut O{};
                O.dst = handle(4, t2 + CL.col[s]);
                O.rows = M;
                O.cols = kr.groups[CL.group[s]].dim;
                O.ld = CL.width;
                O.term0 = static_cast<int>(P.B.terms.size());
                for (int t = 0; t < 4; ++t) {
                    const double cf = e.op[s * 4 + t];
                    if (cf == 0.0 || CL.col[t] < 0) continue;
                    CombTerm tm{};
                    tm.src = handle(3, o1[ga] + CL.col[t]);
                    tm.ld = CL.width;
                    tm.coef = cf;
                    P.B.terms.push_back(tm);
                }
                O.nterm = static_cast<int>(P.B.terms.size()) - O.term0;
                P.B.flops += 2.0 * O.rows * O.cols * O.nterm;
                P.B.outs.push_back(O);
            }
            t2 += static_cast<int64_t>(M) * CL.width;
        }
        // L'[Gb][lb rows, :] = sum_{la, s: la + q(s) = lb} A_bra[la, s, lb]^T T2[Ga(la)][la rows, s cols]
        for (int gb = 0; gb < ngr; ++gb) {
            const int64_t noff = Ln.lay[0].off[gb];
            if (noff < 0) continue;
            const int ldn = Ln.lay[0].ld[gb];
            for (int lb = br.groups[gb].first; lb < br.groups[gb].first + br.groups[gb].count; ++lb) {
                const Label& Lb = br.labels[lb];
                GemmTask T{};
                T.c = handle(7, Ln.base[g] + noff + static_cast<int64_t>(Lb.off - br.groups[gb].off) * ldn);
                T.cmap = -1;
                T.M = Lb.dim;
                T.N = ldn;
                T.ldc = ldn;
                T.seg0 = static_cast<int>(P.C.segs.size());
                for (size_t la = 0; la < bl.labels.size(); ++la)
                    for (int s = 0; s < 4; ++s) {
                        if (ab.seg_label[la * 4 + s] != lb) continue;
                        const Label& La = bl.labels[la];
                        const int ga = La.group;
                        if (o2[ga] < 0 || c1[ga].col[s] < 0) continue;
                        GemmSeg sg{};
                        sg.a = handle(1, ab.row_off[la] + ab.seg_col[la * 4 + s]);
                        sg.a_rs = 1;
                        sg.a_cs = ab.width[la];
                        sg.K = La.dim;
                        sg.b = handle(4, o2[ga] + static_cast<int64_t>(La.off - bl.groups[ga].off) * c1[ga].width +
                                             c1[ga].col[s]);
                        sg.b_rs = c1[ga].width;
                        sg.b_cs = 1;
                        P.C.segs.push_back(sg);
                        P.C.flops += 2.0 * T.M * T.N * sg.K;
                    }
                T.nseg = static_cast<int>(P.C.segs.size()) - T.seg0;
                P.C.tasks.push_back(T);
            }
        }
    }
    close_ranges(P, G, t1, t2);
}

// Right update at site i: R'(bond i) from R(bond i+1); slots as the left update (6 = R, 7 = R').
void build_cross_right(spmps_t* h, const LowerState& Ls, int i, const EnvStore& Ro, const EnvStore& Rn, Plan& P) {
    const Bond& bl = h->bonds[i];
    const Bond& br = h->bonds[i + 1];
    const RowBlockLayout& ab = h->alay[i];
    const Bond& kl = Ls.bonds[i];
    const Bond& kr = Ls.bonds[i + 1];
    const RowBlockLayout& ak = Ls.alay[i];
    const int G = h->G, ngl = static_cast<int>(bl.groups.size()), ngr = static_cast<int>(br.groups.size());
    set_ranges(P, G);
    int64_t t1 = 0, t2 = 0;
    for (int g = 0; g < G; ++g) {
        const MpoEntry& e = Ls.rot[g].E[i][0];
        P.tileA_rng[g] = static_cast<int>(P.A.tasks.size());
        P.combB_rng[g] = static_cast<int>(P.B.outs.size());
        P.tileC_rng[g] = static_cast<int>(P.C.tasks.size());
        std::vector<int64_t> o1(ngr, -1), o2(ngr, -1);
        std::vector<ColLayout> c1(ngr);
        // T1[Gb][b rows, (t, a') cols] = sum_b' R[Gb][b, b'] A_ket[a', t, b']
        for (int gb = 0; gb < ngr; ++gb) {
            const int n0 = br.groups[gb].n;
            const int gkp = kr.group_of(n0);
            const int64_t roff = Ro.lay[0].off[gb];
            if (gkp < 0 || roff < 0) continue;
            ColLayout CL = make_col_layout(kl, n0, 4, -1);
            if (CL.width == 0) continue;
            const int M = br.groups[gb].dim;
            o1[gb] = t1;
            for (int lbp = kr.groups[gkp].first; lbp < kr.groups[gkp].first + kr.groups[gkp].count; ++lbp) {
                const Label& Lbp = kr.labels[lbp];
                for (int t = 0; t < 4; ++t) {
                    const int lap = kl.find(Lbp.n - kLocalN[t], Lbp.tm - kLocal2M[t]);
                    if (lap < 0 || ak.seg_label[lap * 4 + t] != lbp) continue;
                    const Label& Lap = kl.labels[lap];
                    GemmTask T{};
                    T.c = handle(3, t1 + CL.col[t] + (Lap.off - kl.groups[Lap.group].off));
                    T.cmap = -1;
                    T.M = M;
                    T.N = Lap.dim;
                    T.ldc = CL.width;
                    T.seg0 = static_cast<int>(P.A.segs.size());
                    T.nseg = 1;
                    GemmSeg sg{};
                    sg.a = handle(6, Ro.base[g] + roff + (Lbp.off - kr.groups[gkp].off));
                    sg.a_rs = kr.groups[gkp].dim;
                    sg.a_cs = 1;
                    sg.K = Lbp.dim;
                    sg.b = handle(0, ak.row_off[lap] + ak.seg_col[lap * 4 + t]);
                    sg.b_rs = 1;
                    sg.b_cs = ak.width[lap];
                    P.A.segs.push_back(sg);
                    P.A.tasks.push_back(T);
                    P.A.flops += 2.0 * T.M * T.N * sg.K;
                }
            }
            t1 += static_cast<int64_t>(M) * CL.width;
            c1[gb] = CL;
        }
        for (int gb = 0; gb < ngr; ++gb) {
            if (o1[gb] < 0) continue;
            const ColLayout& CL = c1[gb];
            const int M = br.groups[gb].dim;
            o2[gb] = t2;
            for (int s = 0; s < 4; ++s) {
                if (CL.col[s] < 0) continue;
                CombOut O{};
                O.dst = handle(4, t2 + CL.col[s]);
                O.rows = M;
                O.cols = kl.groups[CL.group[s]].dim;
                O.ld = CL.width;
                O.term0 = static_cast<int>(P.B.terms.size());
                for (int t = 0; t < 4; ++t) {
                    const double cf = e.op[s * 4 + t];
                    if (cf == 0.0 || CL.col[t] < 0) continue;
                    CombTerm tm{};
                    tm.src = handle(3, o1[gb] + CL.col[t]);
                    tm.ld = CL.width;
                    tm.coef = cf;
                    P.B.terms.push_back(tm);
                }
                O.nterm = static_cast<int>(P.B.terms.size()) - O.term0;
                P.B.flops += 2.0 * O.rows * O.cols * O.nterm;
                P.B.outs.push_back(O);
            }
            t2 += static_cast<int64_t>(M) * CL.width;
        }
        // R'[Ga][la rows, :] = sum_s A_bra[la, s, lb] T2[Gb(lb)][lb rows, s cols]
        for (int ga = 0; ga < ngl; ++ga) {
            const int64_t noff = Rn.lay[0].off[ga];
            if (noff < 0) continue;
            const int ldn = Rn.lay[0].ld[ga];
            for (int la = bl.groups[ga].first; la < bl.groups[ga].first + bl.groups[ga].count; ++la) {
                const Label& La = bl.labels[la];
                GemmTask T{};
                T.c = handle(7, Rn.base[g] + noff + static_cast<int64_t>(La.off - bl.groups[ga].off) * ldn);
                T.cmap = -1;
                T.M = La.dim;
                T.N = ldn;
                T.ldc = ldn;
                T.seg0 = static_cast<int>(P.C.segs.size());
                for (int s = 0; s < 4; ++s) {
                    const int lb = ab.seg_label[la * 4 + s];
                    if (lb < 0) continue;
                    const Label& Lb = br.labels[lb];
                    const int gb = Lb.group;
                    if (o2[gb] < 0 || c1[gb].col[s] < 0) continue;
                    GemmSeg sg{};
                    sg.a = handle(1, ab.row_off[la] + ab.seg_col[la * 4 + s]);
                    sg.a_rs = ab.width[la];
                    sg.a_cs = 1;
                    sg.K = Lb.dim;
                    sg.b = handle(4, o2[gb] + static_cast<int64_t>(Lb.off - br.groups[gb].off) * c1[gb].width +
                                         c1[gb].col[s]);
                    sg.b_rs = c1[gb].width;
                    sg.b_cs = 1;
                    P.C.segs.push_back(sg);
                    P.C.flops += 2.0 * T.M * T.N * sg.K;
                }
                T.nseg = static_cast<int>(P.C.segs.size()) - T.seg0;
                P.C.tasks.push_back(T);
            }
        }
    }
    close_ranges(P, G, t1, t2);
}

// B at sites (k, k+1): per beta, phase A (L x0 on the lower state's layout), phase B (the two-site
// rotation at -beta with weight c_g), phase C (R, output on the running state's layout) into
// per-beta partials (slot 8) summed into slot 1.  Slots: 0 = x0, 3 = T1, 4 = T3, 5 = L, 6 = R.
void build_cross_B(spmps_t* h, const LowerState& Ls, int k, const EnvStore& Le, const EnvStore& Re, Plan& P) {
    const Bond& bl = h->bonds[k];
    const Bond& br = h->bonds[k + 2];
    const Bond& kl = Ls.bonds[k];
    const Bond& kr = Ls.bonds[k + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    const RowBlockLayout x0l = make_row_block_layout(kl, kr, 16);
    const int G = h->G, ngl = static_cast<int>(bl.groups.size());
    set_ranges(P, G);
    std::vector<int> cmap_off(kl.labels.size(), -1);
    for (size_t l = 0; l < kl.labels.size(); ++l) {
        if (x0l.width[l] == 0) continue;
        const ColLayout CL = make_col_layout(kr, kl.labels[l].n, 16, +1);
        cmap_off[l] = static_cast<int>(P.A.cmaps.size());
        for (int s = 0; s < 16; ++s) {
            const int lb = x0l.seg_label[l * 16 + s];
            if (lb < 0) continue;
            const Label& Lb = kr.labels[lb];
            const int base = CL.col[s] + (Lb.off - kr.groups[Lb.group].off);
            for (int j = 0; j < Lb.dim; ++j) P.A.cmaps.push_back(base + j);
        }
    }
    int64_t t1 = 0, t3 = 0;
    const int64_t nx = xl.size;
    for (int g = 0; g < G; ++g) {
        const double* r1 = Ls.rot[g].E[k][0].op;
        const double* r2 = Ls.rot[g].E[k + 1][0].op;
        const double cg = h->cg[g];
        P.tileA_rng[g] = static_cast<int>(P.A.tasks.size());
        P.combB_rng[g] = static_cast<int>(P.B.outs.size());
        std::vector<int64_t> o1(ngl, -1), o3(ngl, -1);
        std::vector<ColLayout> c1(ngl);
        for (int ga = 0; ga < ngl; ++ga) {
            const int n0 = bl.groups[ga].n;
            const int gk = kl.group_of(n0);
            const int64_t loff = Le.lay[0].off[ga];
            if (gk < 0 || loff < 0) continue;
            ColLayout CL = make_col_layout(kr, n0, 16, +1);
            if (CL.width == 0) continue;
            const int M = bl.groups[ga].dim;
            o1[ga] = t1;
            for (int l = kl.groups[gk].first; l < kl.groups[gk].first + kl.groups[gk].count; ++l) {
                if (x0l.width[l] == 0) continue;
                const Label& Ll = kl.labels[l];
                GemmTask T{};
                T.c = handle(3, t1);
                T.cmap = cmap_off[l];
                T.M = M;
                T.N = x0l.width[l];
                T.ldc = CL.width;
                T.seg0 = static_cast<int>(P.A.segs.size());
                T.nseg = 1;
                GemmSeg sg{};
                sg.a = handle(5, Le.base[g] + loff + (Ll.off - kl.groups[gk].off));
                sg.a_rs = kl.groups[gk].dim;
                sg.a_cs = 1;
                sg.K = Ll.dim;
                sg.b = handle(0, x0l.row_off[l]);
                sg.b_rs = x0l.width[l];
                sg.b_cs = 1;
                P.A.segs.push_back(sg);
                P.A.tasks.push_back(T);
                P.A.flops += 2.0 * T.M * T.N * sg.K;
            }
            t1 += static_cast<int64_t>(M) * CL.width;
            c1[ga] = CL;
        }
        // T3[Ga][:, s, :] = c_g sum_t r(-b)(s1, t1) r(-b)(s2, t2) T1[Ga][:, t, :]
        for (int ga = 0; ga < ngl; ++ga) {
            if (o1[ga] < 0) continue;
            const ColLayout& CL = c1[ga];
            const int M = bl.groups[ga].dim;
            o3[ga] = t3;
            for (int s = 0; s < 16; ++s) {
                if (CL.col[s] < 0) continue;
                CombOut O{};
                O.dst = handle(4, t3 + CL.col[s]);
                O.rows = M;
                O.cols = kr.groups[CL.group[s]].dim;
                O.ld = CL.width;
                O.term0 = static_cast<int>(P.B.terms.size());
                for (int t = 0; t < 16; ++t) {
                    const double cf = cg * r1[(s >> 2) * 4 + (t >> 2)] * r2[(s & 3) * 4 + (t & 3)];
                    if (cf == 0.0 || CL.col[t] < 0) continue;
                    CombTerm tm{};
                    tm.src = handle(3, o1[ga] + CL.col[t]);
                    tm.ld = CL.width;
                    tm.coef = cf;
                    P.B.terms.push_back(tm);
                }
                O.nterm = static_cast<int>(P.B.terms.size()) - O.term0;
                P.B.flops += 2.0 * O.rows * O.cols * O.nterm;
                P.B.outs.push_back(O);
            }
            t3 += static_cast<int64_t>(M) * CL.width;
            // (c1 keeps the column layout: T3 uses the same one)
        }
        P.tileC_rng[g] = static_cast<int>(P.C.tasks.size());
        for (size_t la = 0; la < bl.labels.size(); ++la) {
            const Label& La = bl.labels[la];
            const int ga = La.group;
            for (int s = 0; s < 16; ++s) {
                const int lb = xl.seg_label[la * 16 + s];
                if (lb < 0) continue;
                const Label& Lb = br.labels[lb];
                const int gb = Lb.group;
                GemmTask T{};
                T.c = handle(8, static_cast<int64_t>(g) * nx + xl.row_off[la] + xl.seg_col[la * 16 + s]);
                T.cmap = -1;
                T.M = La.dim;
                T.N = Lb.dim;
                T.ldc = xl.width[la];
                T.seg0 = static_cast<int>(P.C.segs.size());
                const int64_t roff = Re.lay[0].off[gb];
                if (o3[ga] >= 0 && c1[ga].col[s] >= 0 && roff >= 0) {
                    const ColLayout& C3 = c1[ga];
                    const int K = kr.groups[C3.group[s]].dim;
                    GemmSeg sg{};
                    sg.a = handle(4, o3[ga] + static_cast<int64_t>(La.off - bl.groups[ga].off) * C3.width + C3.col[s]);
                    sg.a_rs = C3.width;
                    sg.a_cs = 1;
                    sg.K = K;
                    sg.b = handle(6, Re.base[g] + roff + static_cast<int64_t>(Lb.off - br.groups[gb].off) * K);
                    sg.b_rs = 1;
                    sg.b_cs = K;
                    P.C.segs.push_back(sg);
                    P.C.flops += 2.0 * T.M * T.N * K;
                }
                T.nseg = static_cast<int>(P.C.segs.size()) - T.seg0;
                P.C.tasks.push_back(T);
            }
        }
    }
    P.reduce_nx = nx;
    close_ranges(P, G, t1, t3);
}

spmps_status run_checked(spmps_t* h, Plan& P, const int64_t* sz, const char* what, Slots S) {
    std::string why;
    if (!validate_plan(P, sz, &why)) return fail(h, SPMPS_ERR_CUDA, std::string("internal plan check (") + what + "): " + why);
    spmps_status st = plan_upload(h, P);
    if (st != SPMPS_OK) return st;
    S.p[3] = h->work1.as<double>();
    S.p[4] = h->work2.as<double>();
    const int saved = h->apply_precision;
    h->apply_precision = 0;  // the constraint side is FP64
    st = plan_run(h, P, S, 0, h->G, h->stream);
    h->apply_precision = saved;
    if (st != SPMPS_OK) return st;
    CK(cudaStreamSynchronize(h->stream));  // plan buffers are freed on return
    return SPMPS_OK;
}

spmps_status cross_update_left(spmps_t* h, LowerState& Ls, int i) {
    EnvStore& Lo = Ls.L[i];
    EnvStore& Ln = Ls.L[i + 1];
    spmps_status st = cross_prepare(h, Ln, h->bonds[i + 1], Ls.bonds[i + 1]);
    if (st != SPMPS_OK) return st;
    Plan P;
    build_cross_left(h, Ls, i, Lo, Ln, P);
    int64_t sz[kMaxSlots];
    for (auto& v : sz) v = -1;
    sz[0] = Ls.alay[i].size;
    sz[1] = h->alay[i].size;
    sz[3] = P.t1_size;
    sz[4] = P.t2_size;
    sz[5] = Lo.total;
    sz[7] = Ln.total;
    Slots S{};
    S.p[0] = Ls.A[i]->as<double>();
    S.p[1] = h->A[i]->as<double>();
    S.p[5] = Lo.buf.as<double>();
    S.p[7] = Ln.buf.as<double>();
    st = run_checked(h, P, sz, "cross left", S);
    if (st != SPMPS_OK) return st;
    Ln.valid = true;
    return SPMPS_OK;
}

spmps_status cross_update_right(spmps_t* h, LowerState& Ls, int i) {
    EnvStore& Ro = Ls.R[i + 1];
    EnvStore& Rn = Ls.R[i];
    spmps_status st = cross_prepare(h, Rn, h->bonds[i], Ls.bonds[i]);
    if (st != SPMPS_OK) return st;
    Plan P;
    build_cross_right(h, Ls, i, Ro, Rn, P);
    int64_t sz[kMaxSlots];
    for (auto& v : sz) v = -1;
    sz[0] = Ls.alay[i].size;
    sz[1] = h->alay[i].size;
    sz[3] = P.t1_size;
    sz[4] = P.t2_size;
    sz[6] = Ro.total;
    sz[7] = Rn.total;
    Slots S{};
    S.p[0] = Ls.A[i]->as<double>();
    S.p[1] = h->A[i]->as<double>();
    S.p[6] = Ro.buf.as<double>();
    S.p[7] = Rn.buf.as<double>();
    st = run_checked(h, P, sz, "cross right", S);
    if (st != SPMPS_OK) return st;
    Rn.valid = true;
    return SPMPS_OK;
}

spmps_status ensure_cross(spmps_t* h, LowerState& Ls, int k) {
    const int K = h->K;
    if (Ls.L.size() != static_cast<size_t>(K + 1)) {
        Ls.L.clear();
        Ls.R.clear();
        Ls.L.resize(K + 1);
        Ls.R.resize(K + 1);
    }
    if (!Ls.L[0].valid) {
        spmps_status st = cross_boundary(h, Ls.L[0], h->bonds[0], Ls.bonds[0]);
        if (st != SPMPS_OK) return st;
    }
    if (!Ls.R[K].valid) {
        spmps_status st = cross_boundary(h, Ls.R[K], h->bonds[K], Ls.bonds[K]);
        if (st != SPMPS_OK) return st;
    }
    int b = k;
    while (!Ls.L[b].valid) --b;
    for (int i = b; i < k; ++i) {
        spmps_status st = cross_update_left(h, Ls, i);
        if (st != SPMPS_OK) return st;
    }
    int r = k + 2;
    while (!Ls.R[r].valid) ++r;
    for (int i = r - 1; i >= k + 2; --i) {
        spmps_status st = cross_update_right(h, Ls, i);
        if (st != SPMPS_OK) return st;
    }
    return SPMPS_OK;
}

// The lower state's two-site tensor at sites (k, k+1) into x0 (its own row-block layout).
spmps_status lower_two_site(spmps_t* h, const LowerState& Ls, int k, DevMem& x0, int64_t* n0) {
    const Bond& bl = Ls.bonds[k];
    const Bond& bm = Ls.bonds[k + 1];
    const Bond& br = Ls.bonds[k + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    const RowBlockLayout& a0 = Ls.alay[k];
    const RowBlockLayout& a1 = Ls.alay[k + 1];
    Plan P;
    P.tileA_rng.assign(2, 0);
    for (size_t la = 0; la < bl.labels.size(); ++la)
        for (int s = 0; s < 16; ++s) {
            const int lb = xl.seg_label[la * 16 + s];
            if (lb < 0) continue;
            GemmTask T{};
            T.c = handle(2, xl.row_off[la] + xl.seg_col[la * 16 + s]);
            T.cmap = -1;
            T.M = bl.labels[la].dim;
            T.N = br.labels[lb].dim;
            T.ldc = xl.width[la];
            T.seg0 = static_cast<int>(P.A.segs.size());
            const int lc = a0.seg_label[la * 4 + (s >> 2)];
            if (lc >= 0 && a1.seg_label[lc * 4 + (s & 3)] == lb) {
                GemmSeg sg{};
                sg.a = handle(0, a0.row_off[la] + a0.seg_col[la * 4 + (s >> 2)]);
                sg.a_rs = a0.width[la];
                sg.a_cs = 1;
                sg.K = bm.labels[lc].dim;
                sg.b = handle(1, a1.row_off[lc] + a1.seg_col[lc * 4 + (s & 3)]);
                sg.b_rs = a1.width[lc];
                sg.b_cs = 1;
                P.A.segs.push_back(sg);
            }
            T.nseg = static_cast<int>(P.A.segs.size()) - T.seg0;
            P.A.tasks.push_back(T);
        }
    P.A.add_tiles();
    int64_t sz[kMaxSlots];
    for (auto& v : sz) v = -1;
    sz[0] = a0.size;
    sz[1] = a1.size;
    sz[2] = xl.size;
    std::string why;
    if (!validate_plan(P, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (lower two-site): " + why);
    CK(x0.ensure(std::max<int64_t>(1, xl.size) * sizeof(double)));
    CK(upload(P.d_tasksA, P.A.tasks, h->stream));
    CK(upload(P.d_segsA, P.A.segs, h->stream));
    CK(upload(P.d_tilesA, P.A.tiles, h->stream));
    CK(upload(P.d_cmapsA, P.A.cmaps, h->stream));
    Slots S{};
    S.p[0] = Ls.A[k]->as<double>();
    S.p[1] = Ls.A[k + 1]->as<double>();
    S.p[2] = x0.as<double>();
    CK(launch_gemm_f64(S, P.d_tasksA.as<GemmTask>(), P.d_segsA.as<GemmSeg>(), P.d_tilesA.as<GemmTile>(),
                       P.d_cmapsA.as<int>(), static_cast<int>(P.A.tiles.size()), h->stream));
    ++h->launches;
    CK(cudaStreamSynchronize(h->stream));
    *n0 = xl.size;
    return SPMPS_OK;
}

// B of lower state j at sites (k, k+1) into out (n_x of the running state's layout).
spmps_status lower_B(spmps_t* h, int j, int k, double* out) {
    LowerState& Ls = h->lower[j];
    spmps_status st = ensure_cross(h, Ls, k);
    if (st != SPMPS_OK) return st;
    DevMem x0, part;
    int64_t n0 = 0;
    st = lower_two_site(h, Ls, k, x0, &n0);
    if (st != SPMPS_OK) return st;
    Plan P;
    build_cross_B(h, Ls, k, Ls.L[k], Ls.R[k + 2], P);
    const int64_t nx = P.reduce_nx;
    CK(part.ensure(std::max<int64_t>(1, static_cast<int64_t>(h->G) * nx) * sizeof(double)));
    int64_t sz[kMaxSlots];
    for (auto& v : sz) v = -1;
    sz[0] = n0;
    sz[1] = nx;
    sz[3] = P.t1_size;
    sz[4] = P.t2_size;
    sz[5] = Ls.L[k].total;
    sz[6] = Ls.R[k + 2].total;
    sz[8] = static_cast<int64_t>(h->G) * nx;
    Slots S{};
    S.p[0] = x0.as<double>();
    S.p[1] = out;
    S.p[5] = Ls.L[k].buf.as<double>();
    S.p[6] = Ls.R[k + 2].buf.as<double>();
    S.p[8] = part.as<double>();
    return run_checked(h, P, sz, "excited-state B", S);
}

}  // namespace

void excited_invalidate(spmps_t* h) {
    for (LowerState& Ls : h->lower) {
        for (EnvStore& e : Ls.L) e.valid = false;
        for (EnvStore& e : Ls.R) e.valid = false;
    }
}

spmps_status excited_after_step(spmps_t* h, int k, bool move_right) {
    for (LowerState& Ls : h->lower) {
        if (Ls.L.size() != static_cast<size_t>(h->K + 1)) continue;
        if (move_right) {
            for (int b = k + 1; b <= h->K; ++b) Ls.L[b].valid = false;
            for (int b = 0; b <= k + 1; ++b) Ls.R[b].valid = false;
            if (Ls.L[k].valid) {
                spmps_status st = cross_update_left(h, Ls, k);
                if (st != SPMPS_OK) return st;
            }
        } else {
            for (int b = k + 1; b <= h->K; ++b) Ls.L[b].valid = false;
            for (int b = 0; b <= k + 1; ++b) Ls.R[b].valid = false;
            if (Ls.R[k + 2].valid) {
                spmps_status st = cross_update_right(h, Ls, k + 1);
                if (st != SPMPS_OK) return st;
            }
        }
    }
    return SPMPS_OK;
}

spmps_status excited_constraints(spmps_t* h, int k, DevMem& V, int* count) {
    *count = 0;
    const int nl = static_cast<int>(h->lower.size());
    if (nl == 0) return SPMPS_OK;
    const int64_t n = make_row_block_layout(h->bonds[k], h->bonds[k + 2], 16).size;
    CK(V.ensure(std::max<int64_t>(1, n) * nl * sizeof(double)));
    DevMem dots, nrm;
    CK(dots.ensure(64 * sizeof(double)));
    CK(nrm.ensure(2 * sizeof(double)));
    CK(h->partial.ensure(kPartialDoubles * sizeof(double)));
    double* Vp = V.as<double>();
    int m = 0;
    for (int j = 0; j < nl; ++j) {
        double* col = Vp + static_cast<int64_t>(m) * n;
        spmps_status st = lower_B(h, j, k, col);
        if (st != SPMPS_OK) return st;
        // Gram-Schmidt twice against the kept columns (QR of the B vectors)
        for (int pass = 0; pass < 2 && m > 0; ++pass) {
            CK(launch_multidot(Vp, n, m, col, n, dots.as<double>(), h->partial.as<double>(), h->stream));
            CK(launch_gemv(Vp, n, m, dots.as<double>(), n, col, 1, h->stream));
            h->launches += 3;
        }
        CK(launch_norm2(col, n, nrm.as<double>(), h->partial.as<double>(), h->stream));
        double nn = 0.0;
        CK(cudaMemcpyAsync(&nn, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (!(nn > 1e-28)) continue;  // B vanishes here (or depends on the others): no constraint
        CK(launch_scale_inv_sqrt(col, n, nrm.as<double>(), h->stream));
        h->launches += 3;
        ++m;
    }
    *count = m;
    return SPMPS_OK;
}

}  // namespace eng
}  // namespace spmps

using namespace spmps;
using namespace spmps::eng;

extern "C" {

spmps_status spmps_add_lower_state(spmps_handle h, const int* bond_dims, const int* labels, const double* const* sites) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (!bond_dims || !labels || !sites) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    if (h->lower.size() >= 16) return fail(h, SPMPS_ERR_BAD_INPUT, "at most 16 lower states");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    // validate and lay out the lower state with the handle's own loader, then move it aside
    std::vector<Bond> bonds_saved = h->bonds;
    std::vector<RowBlockLayout> alay_saved = h->alay;
    std::vector<std::unique_ptr<DevMem>> A_saved;
    for (auto& a : h->A) A_saved.push_back(std::move(a));
    const int center_saved = h->center;
    const bool had_mps = h->has_mps;
    st = spmps_set_mps(h, bond_dims, labels, sites, 0);
    LowerState Ls;
    if (st == SPMPS_OK) {
        Ls.bonds = h->bonds;
        Ls.alay = h->alay;
        for (auto& a : h->A) Ls.A.push_back(std::move(a));
    }
    h->bonds = bonds_saved;
    h->alay = alay_saved;
    h->A.clear();
    for (auto& a : A_saved) h->A.push_back(std::move(a));
    h->center = center_saved;
    h->has_mps = had_mps;
    invalidate_all(h);
    if (st != SPMPS_OK) return st;
    for (int g = 0; g < h->G; ++g) Ls.rot.push_back(mpo_rotated(mpo_identity(h->K), -h->beta[g]));
    h->lower.push_back(std::move(Ls));
    excited_invalidate(h);
    return SPMPS_OK;
}

spmps_status spmps_clear_lower_states(spmps_handle h) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    h->lower.clear();
    return SPMPS_OK;
}

spmps_status spmps_lower_overlap(spmps_handle h, int j, double* value) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (!value || j < 0 || j >= static_cast<int>(h->lower.size())) return fail(h, SPMPS_ERR_BAD_INPUT, "bad lower state");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    const int k = std::min(h->center, h->K - 2);
    const int64_t n = make_row_block_layout(h->bonds[k], h->bonds[k + 2], 16).size;
    DevMem B, x, d;
    CK(B.ensure(std::max<int64_t>(1, n) * sizeof(double)));
    CK(x.ensure(std::max<int64_t>(1, n) * sizeof(double)));
    CK(d.ensure(sizeof(double)));
    st = lower_B(h, j, k, B.as<double>());
    if (st != SPMPS_OK) return st;
    st = spmps_two_site(h, k, x.as<double>());
    if (st != SPMPS_OK) return st;
    CK(h->partial.ensure(kPartialDoubles * sizeof(double)));
    CK(launch_multidot(B.as<double>(), 0, 1, x.as<double>(), n, d.as<double>(), h->partial.as<double>(), h->stream));
    CK(cudaMemcpyAsync(value, d.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->launches += 2;
    return SPMPS_OK;
}

}  // extern "C"
