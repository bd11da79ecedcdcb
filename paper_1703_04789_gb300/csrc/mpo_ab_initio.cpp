// Ab initio MPO of Eq. sqH on spatial-orbital sites.
//
// Every term (h_pq a+_p a_q, and (1/2)(pq|rs) a+_p a+_r a_s a_q over spin-orbitals) is written
// as a product of one-spin-orbital operators in site order (Jordan-Wigner: the operator on
// spin-orbital j is its own sigma's times sigma_z to the power of the number of the term's
// operators on later spin-orbitals; the permutation that sorts the operators by site gives the
// sign).  At each cut c between spin-orbitals c-1 and c a term sits in one channel, named by the
// part of it that is a single product of operators:
//   START            nothing placed yet (left part = identity)
//   L1(o)            one operator o on the left; the right part holds the sum of the rest
//   PAIR_L(o1, o2)   two operators on the left        (cuts with n_left <= n_right)
//   PAIR_R(o3, o4)   two operators on the right       (cuts with n_left >  n_right)
//   R1(o)            one operator o on the right; the left part holds the sum of the rest
//   DONE             all placed (right part = identity)
// so the bond dimension at a cut is 2 + 2 n_left + 2 n_right + (pairs of the smaller side),
// O(K^2) as stated after Eq. sumH.  START, L1 and PAIR_L name their left part, PAIR_R, R1 and
// DONE their right part; a term passes from the first kind to the second exactly once, and its
// coefficient is written on that site-tensor entry; every other entry it uses is the bare
// operator (the same for all terms through that entry).  The spin-orbital MPO is then merged in
// pairs (alpha, beta) into spatial sites with local index 2 n_alpha + n_beta (Sec. 2.1).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "core.h"

namespace spmps {

namespace {

enum Kind : int { START = 0, L1 = 1, PAIR_L = 2, PAIR_R = 3, R1 = 4, DONE = 5 };
using Op2 = std::array<double, 4>;  // 2 x 2, row-major (bra, ket)

constexpr Op2 kI = {1, 0, 0, 1};
constexpr Op2 kZ = {1, 0, 0, -1};
constexpr Op2 kCdag = {0, 0, 1, 0};  // a+ |0> = |1>
constexpr Op2 kC = {0, 1, 0, 0};

Op2 mul(const Op2& a, const Op2& b) {
    return {a[0] * b[0] + a[1] * b[2], a[0] * b[1] + a[1] * b[3], a[2] * b[0] + a[3] * b[2], a[2] * b[1] + a[3] * b[3]};
}

// one elementary operator: spin-orbital site and creation flag, encoded as 2*site + create
struct Term {
    int m = 0;       // number of operators (2 or 4)
    int e[4];        // encoded operators in site order
    double coef = 0;
};

inline int site_of(int e) { return e >> 1; }
inline uint32_t key_of(int kind, int a = 0, int b = 0) {
    return static_cast<uint32_t>(kind) | (static_cast<uint32_t>(a) << 4) | (static_cast<uint32_t>(b) << 14);
}

struct Chan {
    uint32_t key;
    int lo, hi;  // cuts on which the channel exists
    int kind;
};

struct Builder {
    int n;  // spin-orbitals
    std::vector<Chan> chans;
    std::unordered_map<uint32_t, int> id;
    // entries of spin-orbital site j, keyed by (channel id at cut j, channel id at cut j+1)
    std::vector<std::unordered_map<uint64_t, Op2>> ents;
    bool consistent = true;

    bool left_indexed_pairs(int c) const { return 2 * c <= n; }

    int chan(uint32_t key, int kind, int c) {
        auto it = id.find(key);
        if (it == id.end()) {
            id.emplace(key, static_cast<int>(chans.size()));
            chans.push_back(Chan{key, c, c, kind});
            return static_cast<int>(chans.size()) - 1;
        }
        Chan& ch = chans[it->second];
        ch.lo = std::min(ch.lo, c);
        ch.hi = std::max(ch.hi, c);
        return it->second;
    }

    // channel of a term at cut c, given nl = number of its operators on sites < c
    int channel_at(const Term& t, int nl, int c) {
        if (nl == 0) return chan(key_of(START), START, c);
        if (nl == t.m) return chan(key_of(DONE), DONE, c);
        if (nl == 1) return chan(key_of(L1, t.e[0]), L1, c);
        if (nl == 3) return chan(key_of(R1, t.e[3]), R1, c);
        // nl == 2 of a four-operator term
        if (left_indexed_pairs(c)) return chan(key_of(PAIR_L, t.e[0], t.e[1]), PAIR_L, c);
        return chan(key_of(PAIR_R, t.e[2], t.e[3]), PAIR_R, c);
    }

    static bool is_left(int kind) { return kind <= PAIR_L; }

    // bare entries must agree between terms; coefficient-carrying ones add up
    void put(int j, int a, int b, const Op2& op, bool inject) {
        const uint64_t key = (static_cast<uint64_t>(a) << 32) | static_cast<uint32_t>(b);
        auto it = ents[j].find(key);
        if (it == ents[j].end()) {
            ents[j].emplace(key, op);
            return;
        }
        if (inject) {
            for (int i = 0; i < 4; ++i) it->second[i] += op[i];
            return;
        }
        for (int i = 0; i < 4; ++i)
            if (it->second[i] != op[i]) consistent = false;
    }

    void add_term(const Term& t) {
        // the channel is constant on runs of cuts [prev, next operator site]; a pair run may
        // cross the switch cut, where the term passes from PAIR_L to PAIR_R
        int prev = 0, nl = 0, k = 0;
        while (true) {
            const int last = k < t.m ? site_of(t.e[k]) : n;
            const int a = channel_at(t, nl, prev);
            const int b = channel_at(t, nl, last);
            if (a != b) {
                const int csw = n / 2;  // last cut with left-indexed pairs
                const int a2 = channel_at(t, nl, csw);
                const int b2 = channel_at(t, nl, csw + 1);
                put(csw, a2, b2, Op2{t.coef, 0.0, 0.0, t.coef}, true);
            }
            if (k == t.m) break;
            // the operators on spin-orbital j (one or two), times sigma_z^(operators further right)
            const int j = site_of(t.e[k]);
            int k2 = k;
            Op2 op = kI;
            while (k2 < t.m && site_of(t.e[k2]) == j) {
                op = mul(op, (t.e[k2] & 1) ? kCdag : kC);
                ++k2;
            }
            if ((t.m - k2) & 1) op = mul(op, kZ);
            const int ca = channel_at(t, k, j);
            const int cb = channel_at(t, k2, j + 1);
            const bool inject = is_left(chans[ca].kind) && !is_left(chans[cb].kind);
            if (inject)
                for (double& v : op) v *= t.coef;
            put(j, ca, cb, op, inject);
            nl = k2;
            prev = j + 1;
            k = k2;
        }
    }
};

// sort the operators of a term by spin-orbital (stable) and fold the permutation sign into coef
bool normalise(Term& t) {
    int sign = 1;
    for (int i = 1; i < t.m; ++i)
        for (int j = i; j > 0 && site_of(t.e[j - 1]) > site_of(t.e[j]); --j) {
            std::swap(t.e[j - 1], t.e[j]);
            sign = -sign;
        }
    // two operators on one spin-orbital must be a+ a (= n); a+ a+ or a a vanish
    for (int i = 1; i < t.m; ++i)
        if (site_of(t.e[i - 1]) == site_of(t.e[i]) && (!(t.e[i - 1] & 1) || (t.e[i] & 1))) return false;
    t.coef *= sign;
    return true;
}

}  // namespace

bool mpo_ab_initio(int K, const double* h1, const double* h2, double ecore, int max_dw, MPO* out, std::string* err) {
    Builder B;
    B.n = 2 * K;
    const int n = B.n;
    B.ents.resize(n);
    auto enc = [](int so, bool create) { return 2 * so + (create ? 1 : 0); };
    // one-body terms
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            const double v = h1[i * K + j];
            if (v == 0.0) continue;
            for (int s = 0; s < 2; ++s) {
                Term t;
                t.m = 2;
                t.e[0] = enc(2 * i + s, true);
                t.e[1] = enc(2 * j + s, false);
                t.coef = v;
                if (normalise(t)) B.add_term(t);
            }
        }
    // two-body terms (1/2)(ij|kl) a+_{i s} a+_{k u} a_{l u} a_{j s}
    if (h2) {
        const size_t Kz = static_cast<size_t>(K);
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j)
                for (int k = 0; k < K; ++k)
                    for (int l = 0; l < K; ++l) {
                        const double v = h2[((i * Kz + j) * Kz + k) * Kz + l];
                        if (v == 0.0) continue;
                        for (int s = 0; s < 2; ++s)
                            for (int u = 0; u < 2; ++u) {
                                const int p = 2 * i + s, q = 2 * j + s, r = 2 * k + u, w = 2 * l + u;
                                if (p == r || q == w) continue;
                                Term t;
                                t.m = 4;
                                t.e[0] = enc(p, true);
                                t.e[1] = enc(r, true);
                                t.e[2] = enc(w, false);
                                t.e[3] = enc(q, false);
                                t.coef = 0.5 * v;
                                if (normalise(t)) B.add_term(t);
                            }
                    }
    }
    // the constant: START -> DONE on spin-orbital 0
    if (ecore != 0.0) {
        const int a = B.chan(key_of(START), START, 0);
        const int b = B.chan(key_of(DONE), DONE, 1);
        B.put(0, a, b, Op2{ecore, 0.0, 0.0, ecore}, true);
    }
    if (B.chans.empty()) {
        if (err) *err = "the Hamiltonian has no terms";
        return false;
    }
    // START and DONE run over every cut they can reach: START from 0, DONE to n
    {
        const int a = B.chan(key_of(START), START, 0);
        const int b = B.chan(key_of(DONE), DONE, n);
        (void)a;
        (void)b;
    }
    // channel indices per cut: START first, DONE last, the rest by (kind, key)
    const int nch = static_cast<int>(B.chans.size());
    std::vector<int> order(nch);
    for (int i = 0; i < nch; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        const Chan& a = B.chans[x];
        const Chan& b = B.chans[y];
        if (a.kind != b.kind) return a.kind < b.kind;
        return a.key < b.key;
    });
    std::vector<std::unordered_map<int, int>> idx(n + 1);
    std::vector<int> dso(n + 1, 0);
    for (int o : order) {
        const Chan& ch = B.chans[o];
        for (int c = ch.lo; c <= ch.hi; ++c) idx[c][o] = dso[c]++;
    }
    if (dso[0] != 1 || dso[n] != 1) {
        if (err) *err = "internal: boundary bonds of the ab initio MPO are not one-dimensional";
        return false;
    }
    // pass-through entries: sigma_z^(operators still to the right) while the channel persists
    for (int o = 0; o < nch; ++o) {
        const Chan& ch = B.chans[o];
        const bool odd = ch.kind == L1 || ch.kind == R1;
        for (int j = ch.lo; j < ch.hi; ++j) B.put(j, o, o, odd ? kZ : kI, false);
    }
    if (!B.consistent) {
        if (err) *err = "internal: inconsistent ab initio MPO entry";
        return false;
    }
    // spin-orbital site tensors with per-cut channel indices
    std::vector<std::unordered_map<uint64_t, Op2>> so(n);
    for (int j = 0; j < n; ++j)
        for (const auto& kv : B.ents[j]) {
            const int a = static_cast<int>(kv.first >> 32), b = static_cast<int>(kv.first & 0xffffffffu);
            const auto ia = idx[j].find(a);
            const auto ib = idx[j + 1].find(b);
            if (ia == idx[j].end() || ib == idx[j + 1].end()) {
                if (err) *err = "internal: ab initio MPO entry outside its channel range";
                return false;
            }
            so[j].emplace((static_cast<uint64_t>(ia->second) << 32) | static_cast<uint32_t>(ib->second), kv.second);
        }
    // merge spin-orbitals (2k, 2k+1) into spatial site k
    MPO m;
    m.K = K;
    m.dw.assign(K + 1, 1);
    for (int b = 0; b <= K; ++b) m.dw[b] = dso[2 * b];
    for (int b = 0; b <= K; ++b)
        if (m.dw[b] > max_dw) {
            if (err) *err = "ab initio MPO bond dimension " + std::to_string(m.dw[b]) + " above the limit " +
                            std::to_string(max_dw);
            return false;
        }
    std::vector<int> dims(m.dw);
    m.init(K, dims);
    for (int k = 0; k < K; ++k) {
        // entries of spin-orbital 2k+1 grouped by their left index
        std::unordered_map<int, std::vector<std::pair<int, Op2>>> right;
        for (const auto& kv : so[2 * k + 1])
            right[static_cast<int>(kv.first >> 32)].push_back({static_cast<int>(kv.first & 0xffffffffu), kv.second});
        for (const auto& kv : so[2 * k]) {
            const int wl = static_cast<int>(kv.first >> 32), mid = static_cast<int>(kv.first & 0xffffffffu);
            const Op2& oa = kv.second;
            auto it = right.find(mid);
            if (it == right.end()) continue;
            for (const auto& rb : it->second) {
                const Op2& ob = rb.second;
                double op[16];
                for (int sa = 0; sa < 2; ++sa)
                    for (int ta = 0; ta < 2; ++ta)
                        for (int sb = 0; sb < 2; ++sb)
                            for (int tb = 0; tb < 2; ++tb)
                                op[(2 * sa + sb) * 4 + (2 * ta + tb)] = oa[sa * 2 + ta] * ob[sb * 2 + tb];
                m.add(k, wl, rb.first, op);
            }
        }
    }
    m.finalize();
    std::string why;
    if (!m.finalize_charges(&why)) {
        if (err) *err = "internal: " + why;
        return false;
    }
    *out = std::move(m);
    return true;
}

}  // namespace spmps
