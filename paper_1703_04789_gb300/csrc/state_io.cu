// MPS initialisation and checkpoint files: spmps_init_random, spmps_init_determinant,
// spmps_save, spmps_load.  Host code on top of spmps_set_mps / spmps_get_mps.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "engine.h"

using namespace spmps;
using namespace spmps::eng;

namespace {

double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return std::floor(r + 0.5);
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based stream, Box-Muller normals
uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
double normal_at(uint64_t seed, uint64_t i) {
    const uint64_t a = splitmix64(seed * 0x100000001B3ull + 2 * i);
    const uint64_t b = splitmix64(seed * 0x100000001B3ull + 2 * i + 1);
    const double u1 = (static_cast<double>(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = static_cast<double>(b >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

struct Sector {
    int n, tm;
    double left, right;
};

// labels (n, 2m) of bond i reachable from the left and completable on the right
std::vector<Sector> sectors(int K, int Na, int Nb, int i) {
    std::vector<Sector> out;
    for (int na = 0; na <= i; ++na)
        for (int nb = 0; nb <= i; ++nb) {
            const int ra = Na - na, rb = Nb - nb;
            if (ra < 0 || rb < 0 || ra > K - i || rb > K - i) continue;
            out.push_back(Sector{na + nb, na - nb, binom(i, na) * binom(i, nb), binom(K - i, ra) * binom(K - i, rb)});
        }
    std::sort(out.begin(), out.end(), [](const Sector& a, const Sector& b) { return a.n != b.n ? a.n < b.n : a.tm < b.tm; });
    return out;
}

std::vector<int> largest_remainder(const std::vector<double>& w, int total) {
    double s = 0.0;
    for (double v : w) s += v;
    std::vector<int> out(w.size(), 0);
    if (s <= total) {
        for (size_t j = 0; j < w.size(); ++j) out[j] = static_cast<int>(w[j]);
        return out;
    }
    std::vector<double> frac(w.size());
    int used = 0;
    for (size_t j = 0; j < w.size(); ++j) {
        const double share = total * w[j] / s;
        out[j] = static_cast<int>(std::floor(share));
        frac[j] = share - out[j];
        used += out[j];
    }
    std::vector<int> order(w.size());
    for (size_t j = 0; j < w.size(); ++j) order[j] = static_cast<int>(j);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return frac[a] > frac[b]; });
    for (int q = 0; q < total - used && q < static_cast<int>(order.size()); ++q) ++out[order[q]];
    return out;
}

// dense host MPS in the spmps_set_mps format
struct HostMps {
    std::vector<int> dims;
    std::vector<int> labels;                 // 2 per index, all bonds
    std::vector<std::vector<double>> sites;  // (D_k, 4, D_k+1)
};

spmps_status put_mps(spmps_t* h, HostMps& M, int center) {
    std::vector<const double*> ptrs(M.sites.size());
    for (size_t k = 0; k < M.sites.size(); ++k) ptrs[k] = M.sites[k].data();
    return spmps_set_mps(h, M.dims.data(), M.labels.data(), ptrs.data(), center);
}

constexpr char kMagic[8] = {'S', 'P', 'M', 'P', 'S', 'C', 'K', '1'};

}  // namespace

extern "C" {

spmps_status spmps_init_determinant(spmps_handle h, const int8_t* occ) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!occ) return fail(h, SPMPS_ERR_BAD_INPUT, "occ is NULL");
    const int K = h->K;
    HostMps M;
    M.dims.assign(K + 1, 1);
    int n = 0, tm = 0;
    M.labels = {0, 0};
    for (int k = 0; k < K; ++k) {
        const int s = occ[k];
        if (s < 0 || s > 3) return fail(h, SPMPS_ERR_BAD_INPUT, "occupation codes are 0, 1 (beta), 2 (alpha), 3 (both)");
        n += kLocalN[s];
        tm += kLocal2M[s];
        M.labels.push_back(n);
        M.labels.push_back(tm);
        std::vector<double> t(4, 0.0);
        t[s] = 1.0;
        M.sites.push_back(t);
    }
    if (n != h->N || tm != h->twoM) return fail(h, SPMPS_ERR_BAD_INPUT, "determinant has the wrong (N, 2M)");
    return put_mps(h, M, 0);
}

spmps_status spmps_init_random(spmps_handle h, uint64_t seed) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    const int K = h->K, D = h->D;
    const int Na = (h->N + h->twoM) / 2, Nb = (h->N - h->twoM) / 2;
    if (Na < 0 || Nb < 0 || Na > K || Nb > K) return fail(h, SPMPS_ERR_BAD_INPUT, "(N, 2M) not representable");
    std::vector<std::map<std::pair<int, int>, int>> bonds(K + 1);
    for (int i = 0; i <= K; ++i) {
        const std::vector<Sector> sec = sectors(K, Na, Nb, i);
        std::vector<double> w;
        for (const Sector& s : sec) w.push_back(std::min(s.left, s.right));
        const std::vector<int> d = largest_remainder(w, D);
        for (size_t j = 0; j < sec.size(); ++j)
            if (d[j] > 0) bonds[i][{sec[j].n, sec[j].tm}] = d[j];
    }
    // drop labels without a live neighbour label on either side, until stable
    for (bool changed = true; changed;) {
        changed = false;
        for (int i = 1; i <= K; ++i)
            for (auto it = bonds[i].begin(); it != bonds[i].end();) {
                bool ok = false;
                for (int s = 0; s < 4 && !ok; ++s) ok = bonds[i - 1].count({it->first.first - kLocalN[s], it->first.second - kLocal2M[s]}) > 0;
                if (!ok) { it = bonds[i].erase(it); changed = true; } else { ++it; }
            }
        for (int i = K - 1; i >= 0; --i)
            for (auto it = bonds[i].begin(); it != bonds[i].end();) {
                bool ok = false;
                for (int s = 0; s < 4 && !ok; ++s) ok = bonds[i + 1].count({it->first.first + kLocalN[s], it->first.second + kLocal2M[s]}) > 0;
                if (!ok) { it = bonds[i].erase(it); changed = true; } else { ++it; }
            }
    }
    HostMps M;
    std::vector<std::vector<std::pair<int, int>>> q(K + 1);
    for (int i = 0; i <= K; ++i) {
        if (bonds[i].empty()) return fail(h, SPMPS_ERR_BAD_INPUT, "empty bond in the random MPS structure");
        int dim = 0;
        for (const auto& kv : bonds[i])
            for (int j = 0; j < kv.second; ++j) {
                q[i].push_back(kv.first);
                M.labels.push_back(kv.first.first);
                M.labels.push_back(kv.first.second);
                ++dim;
            }
        M.dims.push_back(dim);
    }
    uint64_t counter = 0;
    for (int k = 0; k < K; ++k) {
        const int Dl = M.dims[k], Dr = M.dims[k + 1];
        std::vector<double> t(static_cast<size_t>(Dl) * 4 * Dr, 0.0);
        for (int a = 0; a < Dl; ++a)
            for (int s = 0; s < 4; ++s)
                for (int b = 0; b < Dr; ++b) {
                    const double v = normal_at(seed, counter++);
                    if (q[k][a].first + kLocalN[s] == q[k + 1][b].first && q[k][a].second + kLocal2M[s] == q[k + 1][b].second)
                        t[(static_cast<size_t>(a) * 4 + s) * Dr + b] = v;
                }
        M.sites.push_back(std::move(t));
    }
    spmps_status st = put_mps(h, M, 0);
    if (st != SPMPS_OK) return st;
    return spmps_canonicalize(h);
}

spmps_status spmps_save(spmps_handle h, const char* path) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!path) return fail(h, SPMPS_ERR_BAD_INPUT, "path is NULL");
    const int K = h->K;
    std::vector<int> dims(K + 1);
    int center = 0;
    spmps_status st = spmps_get_mps(h, dims.data(), nullptr, nullptr, &center);
    if (st != SPMPS_OK) return st;
    int64_t tot = 0;
    for (int v : dims) tot += v;
    std::vector<int> labels(2 * tot);
    std::vector<std::vector<double>> sites(K);
    std::vector<double*> ptrs(K);
    for (int k = 0; k < K; ++k) {
        sites[k].assign(static_cast<size_t>(dims[k]) * 4 * dims[k + 1], 0.0);
        ptrs[k] = sites[k].data();
    }
    st = spmps_get_mps(h, dims.data(), labels.data(), ptrs.data(), &center);
    if (st != SPMPS_OK) return st;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, SPMPS_ERR_BAD_INPUT, std::string("cannot open ") + path + " for writing");
    const int32_t hdr[6] = {h->K, h->N, h->twoM, h->twoS, center, 0};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 6, f) == 6 &&
              std::fwrite(dims.data(), sizeof(int), dims.size(), f) == dims.size() &&
              std::fwrite(labels.data(), sizeof(int), labels.size(), f) == labels.size();
    for (int k = 0; k < K && ok; ++k) ok = std::fwrite(sites[k].data(), sizeof(double), sites[k].size(), f) == sites[k].size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(h, SPMPS_ERR_BAD_INPUT, std::string("write to ") + path + " failed");
    return SPMPS_OK;
}

spmps_status spmps_load(spmps_handle h, const char* path) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!path) return fail(h, SPMPS_ERR_BAD_INPUT, "path is NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, SPMPS_ERR_BAD_INPUT, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[6];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(int32_t), 6, f) == 6;
    if (!ok || hdr[0] != h->K || hdr[1] != h->N || hdr[2] != h->twoM) {
        std::fclose(f);
        return fail(h, SPMPS_ERR_BAD_INPUT, "not a checkpoint of this problem (K, N, 2M)");
    }
    const int K = h->K;
    HostMps M;
    M.dims.resize(K + 1);
    ok = std::fread(M.dims.data(), sizeof(int), K + 1, f) == static_cast<size_t>(K + 1);
    int64_t tot = 0;
    for (int v : M.dims) {
        if (v < 1 || v > (1 << 20)) ok = false;
        tot += v;
    }
    if (ok) {
        M.labels.resize(2 * tot);
        ok = std::fread(M.labels.data(), sizeof(int), M.labels.size(), f) == M.labels.size();
    }
    for (int k = 0; k < K && ok; ++k) {
        M.sites.emplace_back(static_cast<size_t>(M.dims[k]) * 4 * M.dims[k + 1]);
        ok = std::fread(M.sites.back().data(), sizeof(double), M.sites.back().size(), f) == M.sites.back().size();
    }
    std::fclose(f);
    if (!ok) return fail(h, SPMPS_ERR_BAD_INPUT, std::string("truncated or corrupt checkpoint ") + path);
    return put_mps(h, M, hdr[4]);
}

}  // extern "C"
