// Internal structures of the SP-MPS library: bond labels, block layouts, MPOs, contraction
// plans and the device-side task records consumed by the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace spmps {

// Local basis {|0>, |b>, |a>, |ab>} (index 2*n_alpha + n_beta): particle number and 2*Sz.
constexpr int kLocalN[4] = {0, 1, 1, 2};
constexpr int kLocal2M[4] = {0, -1, 1, 0};

inline int qn_n(int ns, int s) { return ns == 4 ? kLocalN[s] : kLocalN[s >> 2] + kLocalN[s & 3]; }
inline int qn_m(int ns, int s) { return ns == 4 ? kLocal2M[s] : kLocal2M[s >> 2] + kLocal2M[s & 3]; }

// ---------------------------------------------------------------------------------------------
// Bonds: labels (n, 2m) sorted, contiguous; N-groups = runs of labels with equal n.
struct Label {
    int n, tm, dim;
    int off;    // first index of the label on the bond
    int group;  // index of its N-group
};
struct Group {
    int n, off, dim;   // first index and total dimension of the run
    int first, count;  // labels [first, first+count)
};
struct Bond {
    std::vector<Label> labels;
    std::vector<Group> groups;
    int D = 0;
    int find(int n, int tm) const;
    int group_of(int n) const;
    void finalize();  // fills off, group, groups, D from (n, tm, dim)
};

// Row-block layout of a tensor with rows on the labels of a left bond and columns over
// (local index s in [0, ns), indices of the right label lambda + q(s)).
struct RowBlockLayout {
    int ns = 0;
    std::vector<int64_t> row_off;  // per left label
    std::vector<int> width;        // per left label
    std::vector<int> seg_col;      // [l*ns + s]: column offset of segment s, -1 if absent
    std::vector<int> seg_label;    // [l*ns + s]: right label index, -1 if absent
    int64_t size = 0;
};
RowBlockLayout make_row_block_layout(const Bond& left, const Bond& right, int ns);

// Column layout of the M-dense intermediates: for base particle number n0 and local index s,
// the columns of the right N-group with n = n0 + sign * n(s).
struct ColLayout {
    std::vector<int> col;    // [s] column offset, -1 if the group is absent
    std::vector<int> group;  // [s] group index on the right bond, -1 if absent
    int width = 0;
};
ColLayout make_col_layout(const Bond& right, int n0, int ns, int sign);

// ---------------------------------------------------------------------------------------------
// MPO site tensors, stored sparsely: per site k the entries (wl, wr, op) with op[s*4 + t] =
// <s| W[k][wl][wr] |t> (s = output/bra index, t = input/ket index).  Built by add() (entries with
// the same (wl, wr) accumulate), then finalize(): entries sorted by (wr, wl), all-zero ones
// dropped, and the per-wr / per-wl indices filled.
struct MpoEntry {
    int wl, wr;
    double op[16];
};
struct MPO {
    int K = 0;
    std::vector<int> dw;                  // K+1 bond dimensions, dw[0] = dw[K] = 1
    std::vector<std::vector<int>> cn;     // per bond, per channel: particle-number charge
    std::vector<std::vector<MpoEntry>> E; // per site
    std::vector<std::vector<int>> wr_ptr; // per site: entries with wr = u are E[k][wr_ptr[u] .. wr_ptr[u+1])
    std::vector<std::vector<int>> by_wl;  // per site: entry indices ordered by (wl, wr)
    std::vector<std::vector<int>> wl_ptr; // per site: by_wl[k][wl_ptr[w] .. wl_ptr[w+1]) have wl = w

    void init(int K_, const std::vector<int>& dims);
    void add(int k, int wl, int wr, const double* op, double scale = 1.0);
    void finalize();
    double get(int k, int wl, int wr, int s, int t) const;  // lookup by binary search
    size_t entries() const;
    bool finalize_charges(std::string* err);  // derive cn from the nonzero pattern

  private:
    std::vector<std::vector<std::pair<uint64_t, int>>> pending_;  // unsorted (key, entry) while building
};
MPO mpo_hubbard(int K, double t, double U);
// General nearest-neighbour one-band Hamiltonian: on-site energies eps (K), hoppings hop (K-1)
// between sites k and k+1, on-site repulsions U (K) and a constant.
MPO mpo_nearest_neighbour(int K, const std::vector<double>& eps, const std::vector<double>& hop,
                          const std::vector<double>& U, double ecore);
MPO mpo_s2(int K);
// General second-quantised Hamiltonian of Eq. sqH from spatial integrals h1 (K x K) and chemist
// (pq|rs) (K^4, may be NULL), built term by term with complementary-operator channels; false and
// a message when the result would not fit (bond dimension above max_dw).
bool mpo_ab_initio(int K, const double* h1, const double* h2, double ecore, int max_dw, MPO* out, std::string* err);
MPO mpo_identity(int K);
MPO mpo_rotated(const MPO& m, double beta);  // W . r(beta) on the ket leg (Eq. expSy)

// Quadrature (Eq. pmpo): Gauss-Legendre nodes/weights on [-1, 1] and Wigner small d.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
double wigner_small_d(int two_j, int two_mp, int two_m, double beta);
void site_rotation(double beta, double r[16]);

// ---------------------------------------------------------------------------------------------
// Device task records.  Pointers are "slot handles": slot in the top 8 bits, element offset in
// the low 56 bits; the kernels resolve them against a table of base pointers.
constexpr int kMaxSlots = 16;
inline uint64_t handle(int slot, int64_t off) {
    return (static_cast<uint64_t>(slot) << 56) | static_cast<uint64_t>(off);
}
struct Slots {
    double* p[kMaxSlots];
};

// C (M x N) = sum over segments of A(M x K) B(K x N); C(i, j) is stored at
// C[i*ldc + cmap[j]] (cmap = -1: j).  A(i, k) = A[i*a_rs + k*a_cs], B(k, j) = B[k*b_rs + j*b_cs].
struct GemmTask {
    uint64_t c;
    int cmap;  // offset into the plan's column-map array, -1 for identity
    int M, N, ldc;
    int seg0, nseg;
    int key;   // tasks of one beta range with equal key share their B operand (tensor-core stacks)
};
struct GemmSeg {
    uint64_t a, b;
    int K, a_rs, a_cs, b_rs, b_cs;
    int pad;
};
struct GemmTile {
    int task;
    int16_t m0, n0;  // first output row / column of the tile
    int16_t tm, tn;  // tile extent (warp-block shape only)
    int shape;       // 0 16x16, 1 4x64, 2 64x4, 3 32x8, 4 8x32 register tiles; 5 warp block
};

// dst (rows x cols, ld) = sum over terms of coef * src (rows x cols, ld_src).
struct CombOut {
    uint64_t dst;
    int rows, cols, ld;
    int term0, nterm;
    int pad;
};
struct CombTerm {
    uint64_t src;
    int ld;
    int pad;
    double coef;
};

// Diagonal of the projected operators: for output block b, element (i, j) of the block
// (rows x cols at x offset off, row stride ld) gets sum over terms of
// coef * Ld[i*(gl+1) + i0] * Rd[j*(gr+1) + j0] with the term's own L/R diagonal starts.
struct DiagBlock {
    int64_t off;
    int rows, cols, ld;
    int term0, nterm;
    int out;  // 0 = H (y), 1 = N (z)
};
struct DiagTerm {
    uint64_t l, r;  // handle of the first diagonal element used
    int l_step, r_step;
    double coef;
};

// A host-side plan of grouped GEMMs.
// Tile policy of a grouped GEMM: tasks with a total reduction length >= wb_kmin and at most
// wb_mn_max outputs get warp-block tiles (shape 5) of about wb_elems outputs per warp; the rest
// the register-tiled shape with the least padding.
struct TilePolicy {
    int wb_kmin = 64;
    int wb_mn_max = 4096;
    int wb_elems = 256;
};
constexpr int kTileCandidates = 6;
TilePolicy tile_candidate(int i);  // i = 0 is the default policy

struct GemmPlan {
    std::vector<GemmTask> tasks;
    std::vector<GemmSeg> segs;
    std::vector<GemmTile> tiles;
    std::vector<int> cmaps;
    double flops = 0.0;
    void add_tiles(const TilePolicy& pol = TilePolicy());
    // tiles for the tensor-core kernel: regions of at most 32 x 32 outputs (one MMA sub-tile per
    // warp), shape 6
    std::vector<GemmTile> tc_tiles;
    void add_tc_tiles();
    void clear() { tasks.clear(); segs.clear(); tiles.clear(); tc_tiles.clear(); cmaps.clear(); flops = 0.0; }
};
struct CombPlan {
    std::vector<CombOut> outs;
    std::vector<CombTerm> terms;
    double flops = 0.0;
    void clear() { outs.clear(); terms.clear(); flops = 0.0; }
};

}  // namespace spmps
