// Spin-free properties of the projected state (Eq. PropSpinFree): <O> = <Psi|O P|Psi> / <Psi|P|Psi>
// for an operator O that commutes with the projector, evaluated with the same environments and
// projected action as the energy, O in place of H.  The operators are the ones the paper names:
// fragment energies (the terms of Eq. sumH grouped by spatial orbital), the spin-free 1RDM
// (E_pq), spin-spin correlations S_X . S_Y and the seniority number operator.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "engine.h"

using namespace spmps;
using namespace spmps::eng;

namespace {

// <O P> / <P> with O as operator 0 of a temporary operator set; the handle's Hamiltonian,
// environments and plans are restored afterwards.
spmps_status expect_with(spmps_t* h, const MPO& O, double* value) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    OpSet saved = std::move(h->ops);
    std::vector<EnvStore> sl = std::move(h->Lenv), sr = std::move(h->Renv);
    h->Lenv.clear();
    h->Renv.clear();
    h->Lenv.resize(h->K + 1);
    h->Renv.resize(h->K + 1);
    for (auto& p : h->apply_plans) p.reset();
    st = build_opset(h, O, &h->ops);
    double nP = 0.0;
    if (st == SPMPS_OK) st = spmps_energy(h, value, &nP);
    h->ops = std::move(saved);
    h->Lenv = std::move(sl);
    h->Renv = std::move(sr);
    for (auto& p : h->apply_plans) p.reset();
    return st;
}

// local operators in the basis {0, b, a, ab}: S+ = a+_alpha a_beta, S-, Sz, S.S on one site
void spin_ops(double sp[16], double sm[16], double sz[16], double ss[16]) {
    for (int i = 0; i < 16; ++i) sp[i] = sm[i] = sz[i] = ss[i] = 0.0;
    sp[2 * 4 + 1] = 1.0;
    sm[1 * 4 + 2] = 1.0;
    sz[1 * 4 + 1] = -0.5;
    sz[2 * 4 + 2] = 0.5;
    ss[1 * 4 + 1] = 0.75;
    ss[2 * 4 + 2] = 0.75;
}

// S_X . S_Y = 1/2 (S+_X S-_Y + S-_X S+_Y) + Sz_X Sz_Y (spin operators are even: no string).
// Channels: 0 start; 1-3 an X operator placed (S+, S-, Sz), waiting for its Y partner; 4-6 a Y
// operator placed (S+, S-, Sz), waiting for its X partner; 7 done.
MPO mpo_spin_dot(int K, const std::vector<char>& inX, const std::vector<char>& inY) {
    double I[16] = {0}, sp[16], sm[16], sz[16], ss[16];
    for (int i = 0; i < 4; ++i) I[i * 4 + i] = 1.0;
    spin_ops(sp, sm, sz, ss);
    const double* op3[3] = {sp, sm, sz};
    // partner of a placed operator and its coefficient: S+ <-> S- (1/2), Sz <-> Sz (1)
    const double* partner[3] = {sm, sp, sz};
    const double pc[3] = {0.5, 0.5, 1.0};
    std::vector<int> dims(K + 1, 8);
    dims[0] = dims[K] = 1;
    MPO m;
    m.init(K, dims);
    for (int k = 0; k < K; ++k) {
        auto L = [&](int w) { return k == 0 ? (w == 0 ? 0 : -1) : w; };
        auto R = [&](int w) { return k == K - 1 ? (w == 7 ? 0 : -1) : w; };
        auto add = [&](int wl, int wr, const double* op, double c) {
            const int l = L(wl), r = R(wr);
            if (l >= 0 && r >= 0) m.add(k, l, r, op, c);
        };
        add(0, 0, I, 1.0);
        add(7, 7, I, 1.0);
        for (int c = 0; c < 3; ++c) {
            add(1 + c, 1 + c, I, 1.0);
            add(4 + c, 4 + c, I, 1.0);
        }
        if (inX[k] && inY[k]) add(0, 7, ss, 1.0);
        for (int c = 0; c < 3; ++c) {
            if (inX[k]) {
                add(0, 1 + c, op3[c], 1.0);           // X operator placed
                add(4 + c, 7, partner[c], pc[c]);     // Y operator waiting: close with X
            }
            if (inY[k]) {
                add(0, 4 + c, op3[c], 1.0);           // Y operator placed
                add(1 + c, 7, partner[c], pc[c]);     // X operator waiting: close with Y
            }
        }
    }
    m.finalize();
    return m;
}

// Omega = sum_k Omega_k, Omega_k = diag(0, 1, 1, 0): bond dimension 2
MPO mpo_seniority(int K) {
    double I[16] = {0}, om[16] = {0};
    for (int i = 0; i < 4; ++i) I[i * 4 + i] = 1.0;
    om[1 * 4 + 1] = om[2 * 4 + 2] = 1.0;
    std::vector<int> dims(K + 1, 2);
    dims[0] = dims[K] = 1;
    MPO m;
    m.init(K, dims);
    for (int k = 0; k < K; ++k) {
        const int l0 = 0, l1 = k == 0 ? -1 : 1;
        const int r0 = k == K - 1 ? -1 : 0, r1 = k == K - 1 ? 0 : 1;
        if (r0 >= 0) m.add(k, l0, r0, I);
        m.add(k, l0, r1, om);
        if (l1 >= 0) m.add(k, l1, r1, I);
    }
    m.finalize();
    return m;
}

spmps_status finalize_or_fail(spmps_t* h, MPO& m) {
    std::string why;
    if (!m.finalize_charges(&why)) return fail(h, SPMPS_ERR_BAD_INPUT, why);
    return SPMPS_OK;
}

}  // namespace

extern "C" {

spmps_status spmps_expect_mpo(spmps_handle h, const int* bond_dims, const double* const* sites, double* value) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!bond_dims || !sites || !value) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    const int K = h->K;
    if (bond_dims[0] != 1 || bond_dims[K] != 1) return fail(h, SPMPS_ERR_BAD_INPUT, "boundary MPO bonds must have dimension 1");
    std::vector<int> dims(bond_dims, bond_dims + K + 1);
    MPO m;
    m.init(K, dims);
    for (int k = 0; k < K; ++k) {
        if (dims[k] < 1 || dims[k + 1] < 1 || !sites[k]) return fail(h, SPMPS_ERR_BAD_INPUT, "bad MPO site tensor");
        for (int wl = 0; wl < dims[k]; ++wl)
            for (int wr = 0; wr < dims[k + 1]; ++wr) {
                const double* op = sites[k] + (static_cast<size_t>(wl) * dims[k + 1] + wr) * 16;
                bool any = false;
                for (int i = 0; i < 16; ++i) {
                    if (!std::isfinite(op[i])) return fail(h, SPMPS_ERR_BAD_INPUT, "MPO entry not finite");
                    any = any || op[i] != 0.0;
                }
                if (any) m.add(k, wl, wr, op);
            }
    }
    m.finalize();
    spmps_status st = finalize_or_fail(h, m);
    if (st != SPMPS_OK) return st;
    return expect_with(h, m, value);
}

spmps_status spmps_fragment_energies(spmps_handle h, double* e) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!e) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL output");
    if (h->ints_h1.empty()) return fail(h, SPMPS_ERR_STATE, "fragment energies need the integrals (spmps_set_hamiltonian or spmps_set_hubbard)");
    const int K = h->K;
    const size_t Kz = static_cast<size_t>(K), K3 = Kz * Kz * Kz;
    std::vector<double> h1(Kz * Kz), h2;
    for (int p = 0; p < K; ++p) {
        std::fill(h1.begin(), h1.end(), 0.0);
        for (int q = 0; q < K; ++q) h1[p * K + q] = h->ints_h1[p * K + q];
        const double* h2p = nullptr;
        if (!h->ints_h2.empty()) {
            h2.assign(Kz * K3, 0.0);
            std::copy(h->ints_h2.begin() + p * K3, h->ints_h2.begin() + (p + 1) * K3, h2.begin() + p * K3);
            h2p = h2.data();
        }
        MPO m;
        std::string why;
        if (!mpo_ab_initio(K, h1.data(), h2p, 0.0, 1 << 20, &m, &why)) {
            e[p] = 0.0;  // no terms start on orbital p
            continue;
        }
        spmps_status st = expect_with(h, m, e + p);
        if (st != SPMPS_OK) return st;
    }
    return SPMPS_OK;
}

spmps_status spmps_rdm1(spmps_handle h, double* gamma) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!gamma) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL output");
    const int K = h->K;
    std::vector<double> e(static_cast<size_t>(K) * K, 0.0);
    for (int p = 0; p < K; ++p)
        for (int q = p; q < K; ++q) {
            std::fill(e.begin(), e.end(), 0.0);
            e[p * K + q] = 1.0;
            MPO m;
            std::string why;
            if (!mpo_ab_initio(K, e.data(), nullptr, 0.0, 1 << 20, &m, &why)) return fail(h, SPMPS_ERR_BAD_INPUT, why);
            double v = 0.0;
            spmps_status st = expect_with(h, m, &v);
            if (st != SPMPS_OK) return st;
            gamma[p * K + q] = gamma[q * K + p] = v;  // real wavefunction: gamma symmetric
        }
    return SPMPS_OK;
}

spmps_status spmps_spin_correlation(spmps_handle h, const int* X, int nx, const int* Y, int ny, double* value) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!X || !Y || !value || nx < 1 || ny < 1) return fail(h, SPMPS_ERR_BAD_INPUT, "empty orbital set or NULL argument");
    const int K = h->K;
    std::vector<char> inX(K, 0), inY(K, 0);
    for (int i = 0; i < nx; ++i) {
        if (X[i] < 0 || X[i] >= K) return fail(h, SPMPS_ERR_BAD_INPUT, "orbital index out of range");
        inX[X[i]] = 1;
    }
    for (int i = 0; i < ny; ++i) {
        if (Y[i] < 0 || Y[i] >= K) return fail(h, SPMPS_ERR_BAD_INPUT, "orbital index out of range");
        inY[Y[i]] = 1;
    }
    MPO m = mpo_spin_dot(K, inX, inY);
    spmps_status st = finalize_or_fail(h, m);
    if (st != SPMPS_OK) return st;
    return expect_with(h, m, value);
}

spmps_status spmps_seniority(spmps_handle h, double* value) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!value) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL output");
    MPO m = mpo_seniority(h->K);
    spmps_status st = finalize_or_fail(h, m);
    if (st != SPMPS_OK) return st;
    return expect_with(h, m, value);
}

}  // extern "C"
