// SP-MPS engine: the C-ABI entry points, the environment cache and the block planner.
//
// The projected action at sites (k, k+1) (Eq. geproblem, Fig. spmpsOpt) is
//   y = sum_g c_g Pi_(N,M) sum_{w,v,u} L_g[w] (W^g_k[w,v] (x) W^g_k+1[v,u]) R_g[u] x,
// where W^g = W exp(-i beta_g S_y) on the ket leg (Eq. pmpo, Eq. expSy).  The rotation keeps
// the particle number but mixes M, so environments are blocked by N only on the ket side
// (Sec. 2.3.1, last paragraph), while x and the outputs keep (N, M) blocks.  The plan is
//   phase A: T1[w] = L_g[w] x            (one GEMM per ket label of x, all w, g in one launch)
//   phase B: T3[u] = sum c_g WW^g T1      (MPO legs; WW^g = W^g_k W^g_k+1 over v)
//   phase C: y    = sum_{g,u} T3[u] R_g[u]^T on the (N, M)-allowed output blocks only.
// Environment updates use the same three phases with one site.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <unordered_map>

#include "engine.h"

using namespace spmps;
using namespace spmps::eng;

namespace spmps {
namespace eng {

thread_local std::string g_static_err;

spmps_status fail(spmps_t* h, spmps_status st, const std::string& msg) {
    if (h) h->err = msg; else g_static_err = msg;
    return st;
}

spmps_status cuda_fail(spmps_t* h, cudaError_t e, const char* where) {
    std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? SPMPS_ERR_OOM : SPMPS_ERR_CUDA, m);
}


}  // namespace eng

EnvLayout make_env_layout(const Bond& b, const std::vector<int>& cn) {
    EnvLayout L;
    L.n_groups = static_cast<int>(b.groups.size());
    const int nw = static_cast<int>(cn.size());
    L.off.assign(static_cast<size_t>(nw) * L.n_groups, -1);
    L.ld.assign(static_cast<size_t>(nw) * L.n_groups, 0);
    int64_t off = 0;
    for (int w = 0; w < nw; ++w)
        for (int g = 0; g < L.n_groups; ++g) {
            const int gp = b.group_of(b.groups[g].n - cn[w]);
            if (gp < 0) continue;
            L.off[w * L.n_groups + g] = off;
            L.ld[w * L.n_groups + g] = b.groups[gp].dim;
            off += static_cast<int64_t>(b.groups[g].dim) * b.groups[gp].dim;
        }
    L.size = off;
    return L;
}

namespace eng {

// ---- environment storage -----------------------------------------------------------------------

spmps_status env_prepare(spmps_t* h, EnvStore& E, const Bond& b, int bond) {
    const int nops = h->ops.n_ops();
    E.lay.resize(nops);
    E.base.assign(static_cast<size_t>(nops) * h->G, 0);
    int64_t off = 0;
    for (int op = 0; op < nops; ++op) {
        E.lay[op] = make_env_layout(b, h->ops.mpo[op].cn[bond]);
        for (int g = 0; g < h->G; ++g) {
            E.base[op * h->G + g] = off;
            off += E.lay[op].size;
        }
    }
    E.total = off;
    CK(E.buf.ensure(std::max<int64_t>(1, off) * sizeof(double)));
    return SPMPS_OK;
}

// Boundary environments: a single 1 x 1 block per (op, g).
spmps_status env_boundary(spmps_t* h, EnvStore& E, int bond) {
    spmps_status st = env_prepare(h, E, h->bonds[bond], bond);
    if (st != SPMPS_OK) return st;
    std::vector<double> ones(static_cast<size_t>(std::max<int64_t>(E.total, 1)), 0.0);
    for (int op = 0; op < h->ops.n_ops(); ++op)
        for (int g = 0; g < h->G; ++g) {
            const EnvLayout& L = E.lay[op];
            for (size_t i = 0; i < L.off.size(); ++i)
                if (L.off[i] >= 0) ones[E.base[op * h->G + g] + L.off[i]] = 1.0;
        }
    CK(cudaMemcpyAsync(E.buf.p, ones.data(), E.total * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    E.valid = true;
    E.version = ++h->env_counter;
    return SPMPS_OK;
}

// ---- plan validation ------------------------------------------------------------------------
// Every element a plan touches must lie inside the buffer bound to its slot; checked on the
// host before the plan's first launch so that a planner error cannot turn into a device fault.
bool in_range(uint64_t hd, int64_t last, const int64_t* sizes, std::string* why, const char* what) {
    const int slot = static_cast<int>(hd >> 56);
    const int64_t off = static_cast<int64_t>(hd & 0x00FFFFFFFFFFFFFFull);
    if (slot < 0 || slot >= kMaxSlots || sizes[slot] < 0 || off < 0 || off + last >= sizes[slot] || last < 0) {
        char buf[200];
        std::snprintf(buf, sizeof buf, "%s out of range: slot %d offset %lld last %lld size %lld", what, slot,
                      static_cast<long long>(off), static_cast<long long>(last),
                      static_cast<long long>(slot >= 0 && slot < kMaxSlots ? sizes[slot] : -1));
        *why = buf;
        return false;
    }
    return true;
}

bool validate_tiles(const GemmPlan& G, std::string* why);

bool validate_gemm(const GemmPlan& G, const int64_t* sizes, std::string* why) {
    for (const GemmTask& T : G.tasks) {
        if (T.M <= 0 || T.N <= 0) { *why = "empty GEMM task"; return false; }
        int64_t maxc = T.N - 1;
        if (T.cmap >= 0) {
            if (T.cmap + T.N > static_cast<int>(G.cmaps.size())) { *why = "column map out of range"; return false; }
            maxc = 0;
            for (int j = 0; j < T.N; ++j) {
                if (G.cmaps[T.cmap + j] < 0) { *why = "negative column map"; return false; }
                maxc = std::max<int64_t>(maxc, G.cmaps[T.cmap + j]);
            }
        }
        if (maxc >= T.ldc && T.M > 1) { *why = "column beyond leading dimension"; return false; }
        if (!in_range(T.c, static_cast<int64_t>(T.M - 1) * T.ldc + maxc, sizes, why, "GEMM C")) return false;
        for (int q = 0; q < T.nseg; ++q) {
            const GemmSeg& sg = G.segs[T.seg0 + q];
            if (sg.K <= 0 || sg.a_rs < 0 || sg.a_cs < 0 || sg.b_rs < 0 || sg.b_cs < 0) { *why = "bad segment"; return false; }
            if (!in_range(sg.a, static_cast<int64_t>(T.M - 1) * sg.a_rs + static_cast<int64_t>(sg.K - 1) * sg.a_cs, sizes,
                          why, "GEMM A"))
                return false;
            if (!in_range(sg.b, static_cast<int64_t>(sg.K - 1) * sg.b_rs + static_cast<int64_t>(T.N - 1) * sg.b_cs, sizes,
                          why, "GEMM B"))
                return false;
        }
    }
    return validate_tiles(G, why);
}

bool validate_tile_list(const GemmPlan& G, const std::vector<GemmTile>& tiles, std::string* why);

bool validate_tiles(const GemmPlan& G, std::string* why) {
    return validate_tile_list(G, G.tiles, why) && validate_tile_list(G, G.tc_tiles, why);
}

bool validate_tile_list(const GemmPlan& G, const std::vector<GemmTile>& tiles, std::string* why) {
    for (const GemmTile& t : tiles) {
        if (t.task < 0 || t.task >= static_cast<int>(G.tasks.size()) || t.shape < 0 || t.shape > 6) {
            *why = "bad tile";
            return false;
        }
        const GemmTask& T = G.tasks[t.task];
        if (t.m0 < 0 || t.n0 < 0 || t.m0 >= T.M || t.n0 >= T.N) { *why = "tile outside its task"; return false; }
        if (t.shape == 5 && (t.tm < 1 || t.tn < 1 || t.tm > 32 || t.tn > 32 || t.tm * t.tn > 256 ||
                             t.m0 + t.tm > T.M || t.n0 + t.tn > T.N)) {
            *why = "bad warp-block tile";
            return false;
        }
        if (t.shape == 6 && (t.tm < 1 || t.tn < 1 || t.tm > 32 || t.tn > 32 || t.m0 + t.tm > T.M || t.n0 + t.tn > T.N)) {
            *why = "bad tensor-core tile";
            return false;
        }
    }
    return true;
}

bool validate_plan(const Plan& P, const int64_t* sizes, std::string* why) {
    if (!validate_gemm(P.A, sizes, why) || !validate_gemm(P.C, sizes, why)) return false;
    for (const CombOut& o : P.B.outs) {
        if (o.rows <= 0 || o.cols <= 0 || o.cols > o.ld) { *why = "bad combination block"; return false; }
        if (!in_range(o.dst, static_cast<int64_t>(o.rows - 1) * o.ld + o.cols - 1, sizes, why, "comb dst")) return false;
        for (int q = 0; q < o.nterm; ++q) {
            const CombTerm& t = P.B.terms[o.term0 + q];
            if (!in_range(t.src, static_cast<int64_t>(o.rows - 1) * t.ld + o.cols - 1, sizes, why, "comb src")) return false;
        }
    }
    for (const DiagBlock& b : P.diag_blocks) {
        for (int q = 0; q < b.nterm; ++q) {
            const DiagTerm& t = P.diag_terms[b.term0 + q];
            if (!in_range(t.l, static_cast<int64_t>(b.rows - 1) * t.l_step, sizes, why, "diag L")) return false;
            if (!in_range(t.r, static_cast<int64_t>(b.cols - 1) * t.r_step, sizes, why, "diag R")) return false;
        }
    }
    return true;
}

// ---- plan upload and launch -------------------------------------------------------------------

spmps_status plan_upload(spmps_t* h, Plan& P) {
    const auto t0 = std::chrono::steady_clock::now();
    struct Done {
        spmps_t* h;
        std::chrono::steady_clock::time_point t0;
        ~Done() {
            if (!h->profile) return;
            h->prof_launches[5] += 1;
            h->prof_ms[5] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    } done{h, t0};
    P.A.add_tiles(P.polA);
    P.C.add_tiles(P.polC);
    P.A.add_tc_tiles();
    P.C.add_tc_tiles();
    {
        std::string why;
        if (!validate_tiles(P.A, &why) || !validate_tiles(P.C, &why)) return fail(h, SPMPS_ERR_CUDA, "internal tile check: " + why);
    }
    CK(upload(P.d_tasksA, P.A.tasks, h->stream));
    CK(upload(P.d_segsA, P.A.segs, h->stream));
    CK(upload(P.d_tilesA, P.A.tiles, h->stream));
    CK(upload(P.d_cmapsA, P.A.cmaps, h->stream));
    CK(upload(P.d_outsB, P.B.outs, h->stream));
    CK(upload(P.d_termsB, P.B.terms, h->stream));
    CK(upload(P.d_tasksC, P.C.tasks, h->stream));
    CK(upload(P.d_segsC, P.C.segs, h->stream));
    CK(upload(P.d_tilesC, P.C.tiles, h->stream));
    CK(upload(P.d_cmapsC, P.C.cmaps, h->stream));
    CK(upload(P.d_tcA, P.A.tc_tiles, h->stream));
    CK(upload(P.d_tcC, P.C.tc_tiles, h->stream));
    CK(upload(P.d_diag_blocks, P.diag_blocks, h->stream));
    CK(upload(P.d_diag_terms, P.diag_terms, h->stream));
    // tile and output ranges per (op, g): tasks were appended in (op, g) order
    auto ranges = [&](const std::vector<GemmTile>& tiles, const std::vector<int>& task_rng, std::vector<int>& out) {
        out.assign(task_rng.size(), 0);
        size_t t = 0;
        for (size_t r = 0; r < task_rng.size(); ++r) {
            while (t < tiles.size() && tiles[t].task < task_rng[r]) ++t;
            out[r] = static_cast<int>(t);
        }
    };
    if (!P.task_rng_kept) {
        P.taskA_rng = P.tileA_rng;
        P.taskC_rng = P.tileC_rng;
        P.task_rng_kept = true;
    }
    const std::vector<int>& a_task_rng = P.taskA_rng;
    const std::vector<int>& c_task_rng = P.taskC_rng;
    auto task_flops = [](const GemmPlan& gp, const std::vector<int>& rng, std::vector<double>& out) {
        out.assign(rng.size(), 0.0);
        for (size_t r = 0; r + 1 < rng.size(); ++r)
            for (int t = rng[r]; t < rng[r + 1]; ++t) {
                const GemmTask& T = gp.tasks[t];
                for (int q = 0; q < T.nseg; ++q) out[r] += 2.0 * T.M * T.N * gp.segs[T.seg0 + q].K;
            }
    };
    task_flops(P.A, a_task_rng, P.flopsA_rng);
    task_flops(P.C, c_task_rng, P.flopsC_rng);
    P.flopsB_rng.assign(P.combB_rng.size(), 0.0);
    for (size_t r = 0; r + 1 < P.combB_rng.size(); ++r)
        for (int o = P.combB_rng[r]; o < P.combB_rng[r + 1]; ++o)
            P.flopsB_rng[r] += 2.0 * P.B.outs[o].rows * P.B.outs[o].cols * P.B.outs[o].nterm;
    ranges(P.A.tiles, a_task_rng, P.tileA_rng);
    ranges(P.C.tiles, c_task_rng, P.tileC_rng);
    ranges(P.A.tc_tiles, a_task_rng, P.tcA_rng);
    ranges(P.C.tc_tiles, c_task_rng, P.tcC_rng);
    // tcgen05 stacks of the H part (op 0) of an apply plan: phase A by ket label (x rows shared),
    // phase C by right label (environment rows shared)
    P.stA.clear();
    P.stC.clear();
    if (P.reduce_nx > 0 && static_cast<int>(a_task_rng.size()) > h->G && static_cast<int>(c_task_rng.size()) > h->G) {
        const bool okA = build_tc_plan(P.A, a_task_rng, h->G, 128, P.stA);
        const bool okC = build_tc_plan(P.C, c_task_rng, h->G, 64, P.stC);
        if (okA && okC) {
            for (TcPlan* T : {&P.stA, &P.stC}) {
                DevMem* d = T == &P.stA ? P.d_stA : P.d_stC;
                CK(upload(d[0], T->stacks, h->stream));
                CK(upload(d[1], T->rows, h->stream));
                CK(upload(d[2], T->segs, h->stream));
                CK(upload(d[3], T->atab, h->stream));
                CK(upload(d[4], T->units, h->stream));
            }
        } else {
            P.stA.ok = P.stC.ok = false;
        }
    }
    // stacks of every (op, g) range for the FP64-accurate split-product GEMM; its status word is
    // allocated here so that running the plan allocates nothing
    P.ozA.clear();
    P.ozC.clear();
    if (P.reduce_nx > 0 && h->opt.fp64_tensor_cores && a_task_rng.size() > 1 && c_task_rng.size() > 1) {
        const bool okA = build_tc_plan(P.A, a_task_rng, static_cast<int>(a_task_rng.size()) - 1, gemm_oz_columns(), P.ozA);
        const bool okC = build_tc_plan(P.C, c_task_rng, static_cast<int>(c_task_rng.size()) - 1, gemm_oz_columns(), P.ozC);
        if (okA && okC) {
            for (TcPlan* T : {&P.ozA, &P.ozC}) {
                DevMem* d = T == &P.ozA ? P.d_ozA : P.d_ozC;
                CK(upload(d[0], T->stacks, h->stream));
                CK(upload(d[1], T->rows, h->stream));
                CK(upload(d[2], T->segs, h->stream));
                CK(upload(d[3], T->atab, h->stream));
                CK(upload(d[4], T->units, h->stream));
            }
            if (!h->tc_err.p) {
                CK(h->tc_err.ensure(sizeof(int)));
                CK(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream));
            }
        } else {
            P.ozA.ok = P.ozC.ok = false;
        }
    }
    CK(h->work1.ensure(std::max<int64_t>(1, P.t1_size) * sizeof(double)));
    CK(h->work2.ensure(std::max<int64_t>(1, P.t2_size) * sizeof(double)));
    CK(cudaStreamSynchronize(h->stream));
    P.ready = true;
    return SPMPS_OK;
}

// Run the three phases for the (op, g) ranges [r0, r1) (all of them when batched).  When ev
// is given, events ev[0..4] are recorded around the zero fill and the phases.
spmps_status plan_run(spmps_t* h, Plan& P, Slots S, int r0, int r1, cudaStream_t st, cudaEvent_t* ev,
                      const SlotsF* split) {
    const bool batched = h->opt.batched != 0;
    if (ev) CK(cudaEventRecord(ev[0], st));
    CK(cudaMemsetAsync(S.p[3], 0, std::max<int64_t>(1, P.t1_size) * sizeof(double), st));
    if (ev) CK(cudaEventRecord(ev[1], st));
    ++h->launches;
    // flops of a range of (op, g) entries, for the profiler
    auto range_flops = [&](const std::vector<double>& f, int a, int b) {
        double acc = 0.0;
        for (int r = a; r < b && r < static_cast<int>(f.size()); ++r) acc += f[r];
        return acc;
    };
    // the H part (op 0) of a projected action may run on the tensor cores (precision 1 or 2)
    const int prec = P.reduce_nx > 0 ? h->apply_precision : 0;
    const int G = h->G;
    auto gemm = [&](const DevMem& tasks, const DevMem& segs, const DevMem& tiles, const DevMem& cmaps,
                    const std::vector<int>& rng, const std::vector<double>& fl, const DevMem& tc,
                    const std::vector<int>& tc_rng, int a, int b) -> cudaError_t {
        auto one = [&](int lo, int hi, int tf) -> cudaError_t {
            if (hi <= lo) return cudaSuccess;
            const TcPlan& OZ = &tasks == &P.d_tasksA ? P.ozA : P.ozC;
            if (!tf && OZ.ok && h->opt.fp64_tensor_cores && h->tc_err.p) {
                // FP64-accurate split products on the tensor cores over the units of [lo, hi)
                const DevMem* d = &tasks == &P.d_tasksA ? P.d_ozA : P.d_ozC;
                ++h->launches;
                const int rec = h->profile ? prof_begin(h, st, 9, range_flops(fl, lo, hi)) : -1;
                const cudaError_t e2 = launch_gemm_oz(S, d[0].as<TcStack>(), d[1].as<TcRow>(), d[2].as<TcSeg>(),
                                                      d[3].as<uint64_t>(), cmaps.as<int>(), d[4].as<int4>(),
                                                      OZ.unit_rng[lo], OZ.unit_rng[hi], h->tc_err.as<int>(),
                                                      h->opt.tc_wait_polls, st);
                if (rec >= 0) prof_end(h, st, rec);
                return e2;
            }
            const TcPlan& TP = &tasks == &P.d_tasksA ? P.stA : P.stC;
            if (tf && split && TP.ok && h->opt.tensor_core_kernel == 0 && hi <= G) {
                // stacked tcgen05 GEMM over the units of the H-part ranges [lo, hi)
                const DevMem* d = &tasks == &P.d_tasksA ? P.d_stA : P.d_stC;
                ++h->launches;
                const int rec = h->profile ? prof_begin(h, st, 8, range_flops(fl, lo, hi)) : -1;
                cudaError_t e2 = cudaSuccess;
                if (!h->tc_err.p) {
                    e2 = h->tc_err.ensure(sizeof(int));
                    if (e2 == cudaSuccess) e2 = cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), st);
                }
                if (e2 == cudaSuccess)
                    e2 = launch_gemm_tc(S, *split, d[0].as<TcStack>(), d[1].as<TcRow>(), d[2].as<TcSeg>(),
                                        d[3].as<uint64_t>(), cmaps.as<int>(), d[4].as<int4>(), TP.unit_rng[lo],
                                        TP.unit_rng[hi], TP.nt, tf == 2, h->tc_err.as<int>(), h->opt.tc_wait_polls, st);
                if (rec >= 0) prof_end(h, st, rec);
                return e2;
            }
            const bool use_tc = tf && split;
            const int t0 = use_tc ? tc_rng[lo] : rng[lo], t1 = use_tc ? tc_rng[hi] : rng[hi];
            ++h->launches;
            const int rec = h->profile ? prof_begin(h, st, tf ? 8 : 0, range_flops(fl, lo, hi)) : -1;
            cudaError_t e;
            if (use_tc)
                e = launch_gemm_tf32s(S, *split, tasks.as<GemmTask>(), segs.as<GemmSeg>(), tc.as<GemmTile>() + t0,
                                      cmaps.as<int>(), t1 - t0, tf == 2, st);
            else if (tf)
                e = launch_gemm_tf32(S, tasks.as<GemmTask>(), segs.as<GemmSeg>(), tiles.as<GemmTile>() + t0,
                                     cmaps.as<int>(), t1 - t0, tf == 2, st);
            else
                e = launch_gemm_f64(S, tasks.as<GemmTask>(), segs.as<GemmSeg>(), tiles.as<GemmTile>() + t0,
                                    cmaps.as<int>(), t1 - t0, st);
            if (rec >= 0) prof_end(h, st, rec);
            return e;
        };
        if (prec == 0) return one(a, b, 0);
        if (!split || b <= G || a >= G) {
            cudaError_t e = one(a, std::min(b, G), prec);
            if (e != cudaSuccess) return e;
            return one(std::max(a, G), b, 0);
        }
        // H part on the tensor cores on this stream, N part (FP64 pipe) concurrently on the second
        // stream; the outputs are disjoint
        if (!h->aux_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->aux_fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->aux_join, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaEventRecord(h->aux_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux_stream, h->aux_fork, 0);
        if (e != cudaSuccess) return e;
        {
            const cudaStream_t main_st = st;
            st = h->aux_stream;  // `one` launches on st
            e = one(std::max(a, G), b, 0);
            st = main_st;
            if (e != cudaSuccess) return e;
        }
        e = cudaEventRecord(h->aux_join, h->aux_stream);
        if (e != cudaSuccess) return e;
        e = one(a, std::min(b, G), prec);
        if (e != cudaSuccess) return e;
        return cudaStreamWaitEvent(st, h->aux_join, 0);
    };
    auto runA = [&](int a, int b) -> cudaError_t {
        return gemm(P.d_tasksA, P.d_segsA, P.d_tilesA, P.d_cmapsA, P.tileA_rng, P.flopsA_rng, P.d_tcA, P.tcA_rng, a, b);
    };
    auto runB = [&](int a, int b) -> cudaError_t {
        const int o0 = P.combB_rng[a], o1 = P.combB_rng[b];
        ++h->launches;
        const int rec = h->profile ? prof_begin(h, st, 1, range_flops(P.flopsB_rng, a, b)) : -1;
        cudaError_t e = launch_comb_f64(S, P.d_outsB.as<CombOut>() + o0, P.d_termsB.as<CombTerm>(), o1 - o0, st);
        if (rec >= 0) prof_end(h, st, rec);
        return e;
    };
    auto runC = [&](int a, int b) -> cudaError_t {
        return gemm(P.d_tasksC, P.d_segsC, P.d_tilesC, P.d_cmapsC, P.tileC_rng, P.flopsC_rng, P.d_tcC, P.tcC_rng, a, b);
    };
    // tensor-core phases read pre-split operands: x before phase A, the phase-B output before C
    const bool pre_split = prec > 0 && split && r0 < G;
    if (pre_split) {
        CK(launch_split_tf32(S.p[0], P.reduce_nx, split->p[0], st));
        ++h->launches;
    }
    auto split_t3 = [&]() -> cudaError_t {
        if (!pre_split) return cudaSuccess;
        ++h->launches;
        return launch_split_tf32(S.p[4], P.t2_size, split->p[4], st);
    };
    if (batched) {
        CK(runA(r0, r1));
        if (ev) CK(cudaEventRecord(ev[2], st));
        CK(runB(r0, r1));
        CK(split_t3());
        if (ev) CK(cudaEventRecord(ev[3], st));
        CK(runC(r0, r1));
    } else {
        for (int r = r0; r < r1; ++r) CK(runA(r, r + 1));
        if (ev) CK(cudaEventRecord(ev[2], st));
        for (int r = r0; r < r1; ++r) CK(runB(r, r + 1));
        CK(split_t3());
        if (ev) CK(cudaEventRecord(ev[3], st));
        for (int r = r0; r < r1; ++r) CK(runC(r, r + 1));
    }
    if (P.reduce_nx > 0) {
        // outputs of op: y (slot 1) from the partials in slot 8, z (slot 2) from slot 9
        for (int op = r0 / G; op < (r1 + G - 1) / G && op < 2; ++op) {
            CK(launch_sum_partials(S.p[8 + op], G, P.reduce_nx, S.p[1 + op], st));
            ++h->launches;
        }
    }
    if (ev) CK(cudaEventRecord(ev[4], st));
    return SPMPS_OK;
}

// ---- environment update plans ------------------------------------------------------------------

// Left update at site i: L(bond i+1) from L(bond i) and A[i].
// Slots: 0 = A[i], 3 = T1, 4 = T2, 5 = L(bond i), 7 = L(bond i+1).
void build_left_plan(spmps_t* h, int i, const EnvStore& Lo, const EnvStore& Ln, Plan& P) {
    const Bond& bl = h->bonds[i];
    const Bond& br = h->bonds[i + 1];
    const RowBlockLayout& al = h->alay[i];
    const int G = h->G, nops = h->ops.n_ops();
    const int ngl = static_cast<int>(bl.groups.size()), ngr = static_cast<int>(br.groups.size());
    P.A.clear(); P.B.clear(); P.C.clear();
    P.task_rng_kept = false;
    P.tileA_rng.assign(nops * G + 1, 0);
    P.tileC_rng.assign(nops * G + 1, 0);
    P.combB_rng.assign(nops * G + 1, 0);
    // column maps of the site's row blocks into the N-dense T1 columns (depend on the label only)
    std::vector<int> cmap_off(bl.labels.size(), -1);
    for (size_t l = 0; l < bl.labels.size(); ++l) {
        if (al.width[l] == 0) continue;
        const ColLayout CL = make_col_layout(br, bl.labels[l].n, 4, +1);
        cmap_off[l] = static_cast<int>(P.A.cmaps.size());
        for (int s = 0; s < 4; ++s) {
            const int lb = al.seg_label[l * 4 + s];
            if (lb < 0) continue;
            const Label& Lb = br.labels[lb];
            const int base = CL.col[s] + (Lb.off - br.groups[Lb.group].off);
            for (int j = 0; j < Lb.dim; ++j) P.A.cmaps.push_back(base + j);
        }
    }
    int64_t t1 = 0, t2 = 0;
    std::vector<int64_t> t1_off, t2_off;  // [((op*G+g)*nw + w)*ngl + Ga]
    std::vector<ColLayout> cl1, cl2;
    for (int op = 0; op < nops; ++op) {
        const MPO& m = h->ops.mpo[op];
        const int dwl = m.dw[i], dwr = m.dw[i + 1];
        const std::vector<int>& cnl = m.cn[i];
        const std::vector<int>& cnr = m.cn[i + 1];
        for (int g = 0; g < G; ++g) {
            const MPO& W = h->ops.rot[op][g];
            const int og = op * G + g;
            P.tileA_rng[og] = static_cast<int>(P.A.tasks.size());
            P.combB_rng[og] = static_cast<int>(P.B.outs.size());
            P.tileC_rng[og] = static_cast<int>(P.C.tasks.size());
            // phase A
            std::vector<int64_t> o1(static_cast<size_t>(dwl) * ngl, -1);
            std::vector<ColLayout> c1(static_cast<size_t>(dwl) * ngl);
            for (int w = 0; w < dwl; ++w)
                for (int ga = 0; ga < ngl; ++ga) {
                    const int n0 = bl.groups[ga].n - cnl[w];
                    const int gap = bl.group_of(n0);
                    const int64_t loff = Lo.lay[op].off[w * ngl + ga];
                    if (gap < 0 || loff < 0) continue;
                    ColLayout CL = make_col_layout(br, n0, 4, +1);
                    if (CL.width == 0) continue;
                    const int M = bl.groups[ga].dim;
                    o1[w * ngl + ga] = t1;
                    for (int l = bl.groups[gap].first; l < bl.groups[gap].first + bl.groups[gap].count; ++l) {
                        if (al.width[l] == 0) continue;
                        const Label& Ll = bl.labels[l];
                        GemmTask T{};
                        T.c = handle(3, t1);
                        T.cmap = cmap_off[l];
                        T.M = M;
                        T.N = al.width[l];
                        T.ldc = CL.width;
                        T.seg0 = static_cast<int>(P.A.segs.size());
                        T.nseg = 1;
                        GemmSeg sg{};
                        sg.a = handle(5, Lo.base[og] + loff + (Ll.off - bl.groups[gap].off));
                        sg.a_rs = bl.groups[gap].dim;
                        sg.a_cs = 1;
                        sg.K = Ll.dim;
                        sg.b = handle(0, al.row_off[l]);
                        sg.b_rs = al.width[l];
                        sg.b_cs = 1;
                                                P.A.segs.push_back(sg);
                        P.A.tasks.push_back(T);
                        P.A.flops += 2.0 * T.M * T.N * sg.K;
                    }
                    t1 += static_cast<int64_t>(M) * CL.width;
                    c1[w * ngl + ga] = CL;
                }
            // phase B: T2[u][Ga][:, s, :] = sum_{w,t} W[w,u,s,t] T1[w][Ga][:, t, :]
            std::vector<int64_t> o2(static_cast<size_t>(dwr) * ngl, -1);
            std::vector<ColLayout> c2(static_cast<size_t>(dwr) * ngl);
            for (int u = 0; u < dwr; ++u)
                for (int ga = 0; ga < ngl; ++ga) {
                    const int n0 = bl.groups[ga].n - cnr[u];
                    ColLayout CL = make_col_layout(br, n0, 4, +1);
                    if (CL.width == 0) continue;
                    const int M = bl.groups[ga].dim;
                    o2[u * ngl + ga] = t2;
                    for (int s = 0; s < 4; ++s) {
                        if (CL.col[s] < 0) continue;
                        CombOut O{};
                        O.dst = handle(4, t2 + CL.col[s]);
                        O.rows = M;
                        O.cols = br.groups[CL.group[s]].dim;
                        O.ld = CL.width;
                        O.term0 = static_cast<int>(P.B.terms.size());
                        for (int ei = W.wr_ptr[i][u]; ei < W.wr_ptr[i][u + 1]; ++ei) {
                            const MpoEntry& e = W.E[i][ei];
                            const int w = e.wl;
                            const int64_t s1 = o1[w * ngl + ga];
                            if (s1 < 0) continue;
                            const ColLayout& C1 = c1[w * ngl + ga];
                            for (int t = 0; t < 4; ++t) {
                                const double cf = e.op[s * 4 + t];
                                if (cf == 0.0 || C1.col[t] < 0) continue;
                                CombTerm tm{};
                                tm.src = handle(3, s1 + C1.col[t]);
                                tm.ld = C1.width;
                                tm.coef = cf;
                                P.B.terms.push_back(tm);
                            }
                        }
                        O.nterm = static_cast<int>(P.B.terms.size()) - O.term0;
                        P.B.flops += 2.0 * O.rows * O.cols * O.nterm;
                        P.B.outs.push_back(O);
                    }
                    t2 += static_cast<int64_t>(M) * CL.width;
                    c2[u * ngl + ga] = CL;
                }
            // phase C: Lnew[u][Gb][lb rows, :] = sum_{la, s: la+q(s)=lb} A[la,s,lb]^T T2[u][Ga(la)][la rows, s cols]
            for (int u = 0; u < dwr; ++u)
                for (int gb = 0; gb < ngr; ++gb) {
                    const int64_t noff = Ln.lay[op].off[u * ngr + gb];
                    if (noff < 0) continue;
                    const int ldn = Ln.lay[op].ld[u * ngr + gb];
                    for (int lb = br.groups[gb].first; lb < br.groups[gb].first + br.groups[gb].count; ++lb) {
                        const Label& Lb = br.labels[lb];
                        GemmTask T{};
                        T.c = handle(7, Ln.base[og] + noff + static_cast<int64_t>(Lb.off - br.groups[gb].off) * ldn);
                        T.cmap = -1;
                        T.M = Lb.dim;
                        T.N = ldn;
                        T.ldc = ldn;
                        T.seg0 = static_cast<int>(P.C.segs.size());
                        for (size_t la = 0; la < bl.labels.size(); ++la)
                            for (int s = 0; s < 4; ++s) {
                                if (al.seg_label[la * 4 + s] != lb) continue;
                                const Label& La = bl.labels[la];
                                const int ga = La.group;
                                const int64_t s2 = o2[u * ngl + ga];
                                if (s2 < 0) continue;
                                const ColLayout& C2 = c2[u * ngl + ga];
                                if (C2.col[s] < 0) continue;
                                GemmSeg sg{};
                                sg.a = handle(0, al.row_off[la] + al.seg_col[la * 4 + s]);
                                sg.a_rs = 1;
                                sg.a_cs = al.width[la];
                                sg.K = La.dim;
                                sg.b = handle(4, s2 + static_cast<int64_t>(La.off - bl.groups[ga].off) * C2.width + C2.col[s]);
                                sg.b_rs = C2.width;
                                sg.b_cs = 1;
                                                                P.C.segs.push_back(sg);
                                P.C.flops += 2.0 * T.M * T.N * sg.K;
                            }
                        T.nseg = static_cast<int>(P.C.segs.size()) - T.seg0;
                        P.C.tasks.push_back(T);
                    }
                }
        }
    }
    P.tileA_rng[nops * G] = static_cast<int>(P.A.tasks.size());
    P.combB_rng[nops * G] = static_cast<int>(P.B.outs.size());
    P.tileC_rng[nops * G] = static_cast<int>(P.C.tasks.size());
    P.t1_size = t1;
    P.t2_size = t2;
    P.flops = P.A.flops + P.B.flops + P.C.flops;
}

// Right update at site i: R(bond i) from R(bond i+1) and A[i].
// Slots: 0 = A[i], 3 = T1, 4 = T2, 6 = R(bond i+1), 7 = R(bond i).
void build_right_plan(spmps_t* h, int i, const EnvStore& Ro, const EnvStore& Rn, Plan& P) {
    const Bond& bl = h->bonds[i];
    const Bond& br = h->bonds[i + 1];
    const RowBlockLayout& al = h->alay[i];
    const int G = h->G, nops = h->ops.n_ops();
    const int ngl = static_cast<int>(bl.groups.size()), ngr = static_cast<int>(br.groups.size());
    P.A.clear(); P.B.clear(); P.C.clear();
    P.task_rng_kept = false;
    P.tileA_rng.assign(nops * G + 1, 0);
    P.tileC_rng.assign(nops * G + 1, 0);
    P.combB_rng.assign(nops * G + 1, 0);
    int64_t t1 = 0, t2 = 0;
    for (int op = 0; op < nops; ++op) {
        const MPO& m = h->ops.mpo[op];
        const int dwl = m.dw[i], dwr = m.dw[i + 1];
        const std::vector<int>& cnl = m.cn[i];
        const std::vector<int>& cnr = m.cn[i + 1];
        for (int g = 0; g < G; ++g) {
            const MPO& W = h->ops.rot[op][g];
            const int og = op * G + g;
            P.tileA_rng[og] = static_cast<int>(P.A.tasks.size());
            P.combB_rng[og] = static_cast<int>(P.B.outs.size());
            P.tileC_rng[og] = static_cast<int>(P.C.tasks.size());
            // phase A: T1[u][Gb][b, (t, a')] = sum_b' R[u][b, b'] A[a', t, b']
            std::vector<int64_t> o1(static_cast<size_t>(dwr) * ngr, -1);
            std::vector<ColLayout> c1(static_cast<size_t>(dwr) * ngr);
            for (int u = 0; u < dwr; ++u)
                for (int gb = 0; gb < ngr; ++gb) {
                    const int n0 = br.groups[gb].n - cnr[u];
                    const int gbp = br.group_of(n0);
                    const int64_t roff = Ro.lay[op].off[u * ngr + gb];
                    if (gbp < 0 || roff < 0) continue;
                    ColLayout CL = make_col_layout(bl, n0, 4, -1);
                    if (CL.width == 0) continue;
                    const int M = br.groups[gb].dim;
                    o1[u * ngr + gb] = t1;
                    for (int lbp = br.groups[gbp].first; lbp < br.groups[gbp].first + br.groups[gbp].count; ++lbp) {
                        const Label& Lbp = br.labels[lbp];
                        for (int t = 0; t < 4; ++t) {
                            const int lap = bl.find(Lbp.n - kLocalN[t], Lbp.tm - kLocal2M[t]);
                            if (lap < 0 || al.seg_label[lap * 4 + t] != lbp) continue;
                            const Label& Lap = bl.labels[lap];
                            GemmTask T{};
                            T.c = handle(3, t1 + CL.col[t] + (Lap.off - bl.groups[Lap.group].off));
                            T.cmap = -1;
                            T.M = M;
                            T.N = Lap.dim;
                            T.ldc = CL.width;
                            T.seg0 = static_cast<int>(P.A.segs.size());
                            T.nseg = 1;
                            GemmSeg sg{};
                            sg.a = handle(6, Ro.base[og] + roff + (Lbp.off - br.groups[gbp].off));
                            sg.a_rs = br.groups[gbp].dim;
                            sg.a_cs = 1;
                            sg.K = Lbp.dim;
                            sg.b = handle(0, al.row_off[lap] + al.seg_col[lap * 4 + t]);
                            sg.b_rs = 1;
                            sg.b_cs = al.width[lap];
                                                        P.A.segs.push_back(sg);
                            P.A.tasks.push_back(T);
                            P.A.flops += 2.0 * T.M * T.N * sg.K;
                        }
                    }
                    t1 += static_cast<int64_t>(M) * CL.width;
                    c1[u * ngr + gb] = CL;
                }
            // phase B: T2[w][Gb][:, s, :] = sum_{u,t} W[w,u,s,t] T1[u][Gb][:, t, :]
            std::vector<int64_t> o2(static_cast<size_t>(dwl) * ngr, -1);
            std::vector<ColLayout> c2(static_cast<size_t>(dwl) * ngr);
            for (int w = 0; w < dwl; ++w)
                for (int gb = 0; gb < ngr; ++gb) {
                    const int n0 = br.groups[gb].n - cnl[w];
                    ColLayout CL = make_col_layout(bl, n0, 4, -1);
                    if (CL.width == 0) continue;
                    const int M = br.groups[gb].dim;
                    o2[w * ngr + gb] = t2;
                    for (int s = 0; s < 4; ++s) {
                        if (CL.col[s] < 0) continue;
                        CombOut O{};
                        O.dst = handle(4, t2 + CL.col[s]);
                        O.rows = M;
                        O.cols = bl.groups[CL.group[s]].dim;
                        O.ld = CL.width;
                        O.term0 = static_cast<int>(P.B.terms.size());
                        for (int q = W.wl_ptr[i][w]; q < W.wl_ptr[i][w + 1]; ++q) {
                            const MpoEntry& e = W.E[i][W.by_wl[i][q]];
                            const int u = e.wr;
                            const int64_t s1 = o1[u * ngr + gb];
                            if (s1 < 0) continue;
                            const ColLayout& C1 = c1[u * ngr + gb];
                            for (int t = 0; t < 4; ++t) {
                                const double cf = e.op[s * 4 + t];
                                if (cf == 0.0 || C1.col[t] < 0) continue;
                                CombTerm tm{};
                                tm.src = handle(3, s1 + C1.col[t]);
                                tm.ld = C1.width;
                                tm.coef = cf;
                                P.B.terms.push_back(tm);
                            }
                        }
                        O.nterm = static_cast<int>(P.B.terms.size()) - O.term0;
                        P.B.flops += 2.0 * O.rows * O.cols * O.nterm;
                        P.B.outs.push_back(O);
                    }
                    t2 += static_cast<int64_t>(M) * CL.width;
                    c2[w * ngr + gb] = CL;
                }
            // phase C: Rnew[w][Ga][la rows, :] = sum_s A[la, s, lb] T2[w][Gb(lb)][lb rows, s cols]
            for (int w = 0; w < dwl; ++w)
                for (int ga = 0; ga < ngl; ++ga) {
                    const int64_t noff = Rn.lay[op].off[w * ngl + ga];
                    if (noff < 0) continue;
                    const int ldn = Rn.lay[op].ld[w * ngl + ga];
                    for (int la = bl.groups[ga].first; la < bl.groups[ga].first + bl.groups[ga].count; ++la) {
                        const Label& La = bl.labels[la];
                        GemmTask T{};
                        T.c = handle(7, Rn.base[og] + noff + static_cast<int64_t>(La.off - bl.groups[ga].off) * ldn);
                        T.cmap = -1;
                        T.M = La.dim;
                        T.N = ldn;
                        T.ldc = ldn;
                        T.seg0 = static_cast<int>(P.C.segs.size());
                        for (int s = 0; s < 4; ++s) {
                            const int lb = al.seg_label[la * 4 + s];
                            if (lb < 0) continue;
                            const Label& Lb = br.labels[lb];
                            const int gb = Lb.group;
                            const int64_t s2 = o2[w * ngr + gb];
                            if (s2 < 0) continue;
                            const ColLayout& C2 = c2[w * ngr + gb];
                            if (C2.col[s] < 0) continue;
                            GemmSeg sg{};
                            sg.a = handle(0, al.row_off[la] + al.seg_col[la * 4 + s]);
                            sg.a_rs = al.width[la];
                            sg.a_cs = 1;
                            sg.K = Lb.dim;
                            sg.b = handle(4, s2 + static_cast<int64_t>(Lb.off - br.groups[gb].off) * C2.width + C2.col[s]);
                            sg.b_rs = C2.width;
                            sg.b_cs = 1;
                                                        P.C.segs.push_back(sg);
                            P.C.flops += 2.0 * T.M * T.N * sg.K;
                        }
                        T.nseg = static_cast<int>(P.C.segs.size()) - T.seg0;
                        P.C.tasks.push_back(T);
                    }
                }
        }
    }
    P.tileA_rng[nops * G] = static_cast<int>(P.A.tasks.size());
    P.combB_rng[nops * G] = static_cast<int>(P.B.outs.size());
    P.tileC_rng[nops * G] = static_cast<int>(P.C.tasks.size());
    P.t1_size = t1;
    P.t2_size = t2;
    P.flops = P.A.flops + P.B.flops + P.C.flops;
}

// diagonal WW coefficients of one channel pair (w, u), per two-site local state
struct DiagPair {
    int w, u;
    double c[16];
};

// ---- the projected action plan ---------------------------------------------------------------
// Slots: 0 = x, 1 = y, 2 = z, 3 = T1, 4 = T3, 5 = L(bond k), 6 = R(bond k+2).
void build_apply_plan(spmps_t* h, int k, const EnvStore& Le, const EnvStore& Re, Plan& P, const EnvNorms* nL,
                      const EnvNorms* nR, double tau) {
    const bool screen = tau > 0.0 && nL && nR;
    const Bond& bl = h->bonds[k];
    const Bond& br = h->bonds[k + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    const int G = h->G, nops = h->ops.n_ops();
    const int ngl = static_cast<int>(bl.groups.size()), ngr = static_cast<int>(br.groups.size());
    P.A.clear(); P.B.clear(); P.C.clear();
    P.task_rng_kept = false;
    P.diag_blocks.clear();
    P.diag_terms.clear();
    P.tileA_rng.assign(nops * G + 1, 0);
    P.tileC_rng.assign(nops * G + 1, 0);
    P.combB_rng.assign(nops * G + 1, 0);
    for (double& f : P.flops_op) f = 0.0;
    std::vector<int> cmap_off(bl.labels.size(), -1);
    for (size_t l = 0; l < bl.labels.size(); ++l) {
        if (xl.width[l] == 0) continue;
        const ColLayout CL = make_col_layout(br, bl.labels[l].n, 16, +1);
        cmap_off[l] = static_cast<int>(P.A.cmaps.size());
        for (int s = 0; s < 16; ++s) {
            const int lb = xl.seg_label[l * 16 + s];
            if (lb < 0) continue;
            const Label& Lb = br.labels[lb];
            const int base = CL.col[s] + (Lb.off - br.groups[Lb.group].off);
            for (int j = 0; j < Lb.dim; ++j) P.A.cmaps.push_back(base + j);
        }
    }
    int64_t t1 = 0, t3 = 0, t1_op0 = 0, t3_op0 = 0;
    std::vector<int64_t> t3_op_end(nops, 0), t3_op_begin(nops, 0);
    // per (op, g): offsets of T3 blocks for the output phase, kept for all g
    std::vector<std::vector<int64_t>> o3_all(static_cast<size_t>(nops) * G);
    std::vector<std::vector<DiagPair>> diag_all(static_cast<size_t>(nops) * G);
    std::vector<std::vector<ColLayout>> c3_all(static_cast<size_t>(nops) * G);
    for (int op = 0; op < nops; ++op) {
        const MPO& m = h->ops.mpo[op];
        const int dwl = m.dw[k], dwr = m.dw[k + 2];
        const std::vector<int>& cnl = m.cn[k];
        const std::vector<int>& cnr = m.cn[k + 2];
        t3_op_begin[op] = t3;
        for (int g = 0; g < G; ++g) {
            const MPO& W = h->ops.rot[op][g];
            const int og = op * G + g;
            const double cgw = h->cg[g];
            P.tileA_rng[og] = static_cast<int>(P.A.tasks.size());
            P.combB_rng[og] = static_cast<int>(P.B.outs.size());
            const double fa0 = P.A.flops, fb0 = P.B.flops;
            // WW[w][u][(s1 s2)][(t1 t2)] = c_g sum_v W_k[w,v,s1,t1] W_k+1[v,u,s2,t2], kept for the
            // (w, u) pairs joined by some v; ww_u[u] lists (w, pair) ordered by w
            std::unordered_map<uint64_t, int> ww_id;
            std::vector<std::array<double, 256>> ww;
            std::vector<std::vector<std::pair<int, int>>> ww_u(dwr);
            for (const MpoEntry& a : W.E[k]) {
                const int v = a.wr;
                for (int q = W.wl_ptr[k + 1][v]; q < W.wl_ptr[k + 1][v + 1]; ++q) {
                    const MpoEntry& b = W.E[k + 1][W.by_wl[k + 1][q]];
                    const uint64_t key = (static_cast<uint64_t>(a.wl) << 32) | static_cast<uint32_t>(b.wr);
                    auto it = ww_id.find(key);
                    int id;
                    if (it == ww_id.end()) {
                        id = static_cast<int>(ww.size());
                        ww_id.emplace(key, id);
                        ww.emplace_back();
                        ww.back().fill(0.0);
                        ww_u[b.wr].push_back({a.wl, id});
                    } else {
                        id = it->second;
                    }
                    std::array<double, 256>& dst = ww[id];
                    for (int s1 = 0; s1 < 4; ++s1)
                        for (int t1i = 0; t1i < 4; ++t1i) {
                            const double av = a.op[s1 * 4 + t1i];
                            if (av == 0.0) continue;
                            for (int s2 = 0; s2 < 4; ++s2)
                                for (int t2i = 0; t2i < 4; ++t2i) {
                                    const double bv = b.op[s2 * 4 + t2i];
                                    if (bv == 0.0) continue;
                                    dst[(s1 * 4 + s2) * 16 + (t1i * 4 + t2i)] += cgw * av * bv;
                                }
                        }
                }
            }
            for (auto& lst : ww_u) std::sort(lst.begin(), lst.end());
            // diagonal coefficients of the pairs between charge-0 channels, for the preconditioner
            {
                std::vector<DiagPair>& dp = diag_all[og];
                dp.clear();
                for (int u = 0; u < dwr; ++u) {
                    if (cnr[u] != 0) continue;
                    for (const auto& wp : ww_u[u]) {
                        if (cnl[wp.first] != 0) continue;
                        DiagPair d{};
                        d.w = wp.first;
                        d.u = u;
                        bool any = false;
                        for (int q = 0; q < 16; ++q) {
                            d.c[q] = ww[wp.second][q * 16 + q];
                            any = any || d.c[q] != 0.0;
                        }
                        if (any) dp.push_back(d);
                    }
                }
                std::sort(dp.begin(), dp.end(), [](const DiagPair& a, const DiagPair& b) {
                    return a.w != b.w ? a.w < b.w : a.u < b.u;
                });
            }
            // phase A
            std::vector<int64_t> o1(static_cast<size_t>(dwl) * ngl, -1);
            std::vector<ColLayout> c1(static_cast<size_t>(dwl) * ngl);
            for (int w = 0; w < dwl; ++w)
                for (int ga = 0; ga < ngl; ++ga) {
                    const int n0 = bl.groups[ga].n - cnl[w];
                    const int gap = bl.group_of(n0);
                    const int64_t loff = Le.lay[op].off[w * ngl + ga];
                    if (gap < 0 || loff < 0) continue;
                    ColLayout CL = make_col_layout(br, n0, 16, +1);
                    if (CL.width == 0) continue;
                    const int M = bl.groups[ga].dim;
                    o1[w * ngl + ga] = t1;
                    const Group& Ga = bl.groups[ga];
                    for (int l = bl.groups[gap].first; l < bl.groups[gap].first + bl.groups[gap].count; ++l) {
                        if (xl.width[l] == 0) continue;
                        const Label& Ll = bl.labels[l];
                        // unscreened: one task over all bra rows of the group; screened: one task per
                        // bra label, dropped when its environment sub-block is below the threshold
                        const int nsub = screen ? Ga.count : 1;
                        for (int q = 0; q < nsub; ++q) {
                            const int row0 = screen ? bl.labels[Ga.first + q].off - Ga.off : 0;
                            const int rows = screen ? bl.labels[Ga.first + q].dim : M;
                            if (screen && nL->dropped(op, g, w, ga, q, l - bl.groups[gap].first, tau)) continue;
                            GemmTask T{};
                            T.c = handle(3, t1 + static_cast<int64_t>(row0) * CL.width);
                            T.cmap = cmap_off[l];
                            T.M = rows;
                            T.N = xl.width[l];
                            T.key = static_cast<int>(l);  // all products of one ket label read x[l]
                            T.ldc = CL.width;
                            T.seg0 = static_cast<int>(P.A.segs.size());
                            T.nseg = 1;
                            GemmSeg sg{};
                            sg.a = handle(5, Le.base[og] + loff + static_cast<int64_t>(row0) * bl.groups[gap].dim +
                                                 (Ll.off - bl.groups[gap].off));
                            sg.a_rs = bl.groups[gap].dim;
                            sg.a_cs = 1;
                            sg.K = Ll.dim;
                            sg.b = handle(0, xl.row_off[l]);
                            sg.b_rs = xl.width[l];
                            sg.b_cs = 1;
                            P.A.segs.push_back(sg);
                            P.A.tasks.push_back(T);
                            P.A.flops += 2.0 * T.M * T.N * sg.K;
                        }
                    }
                    t1 += static_cast<int64_t>(M) * CL.width;
                    c1[w * ngl + ga] = CL;
                }
            // phase B: T3[u][Ga][:, s, :] = sum_{w,t} WW[w,u,s,t] T1[w][Ga][:, t, :]
            std::vector<int64_t>& o3 = o3_all[og];
            std::vector<ColLayout>& c3 = c3_all[og];
            o3.assign(static_cast<size_t>(dwr) * ngl, -1);
            c3.assign(static_cast<size_t>(dwr) * ngl, ColLayout{});
            for (int u = 0; u < dwr; ++u)
                for (int ga = 0; ga < ngl; ++ga) {
                    const int n0 = bl.groups[ga].n - cnr[u];
                    ColLayout CL = make_col_layout(br, n0, 16, +1);
                    if (CL.width == 0) continue;
                    const int M = bl.groups[ga].dim;
                    o3[u * ngl + ga] = t3;
                    for (int s = 0; s < 16; ++s) {
                        if (CL.col[s] < 0) continue;
                        CombOut O{};
                        O.dst = handle(4, t3 + CL.col[s]);
                        O.rows = M;
                        O.cols = br.groups[CL.group[s]].dim;
                        O.ld = CL.width;
                        O.term0 = static_cast<int>(P.B.terms.size());
                        for (const auto& wp : ww_u[u]) {
                            const int w = wp.first;
                            const int64_t s1 = o1[w * ngl + ga];
                            if (s1 < 0) continue;
                            const ColLayout& C1 = c1[w * ngl + ga];
                            const std::array<double, 256>& cw = ww[wp.second];
                            for (int t = 0; t < 16; ++t) {
                                const double cf = cw[s * 16 + t];
                                if (cf == 0.0 || C1.col[t] < 0) continue;
                                CombTerm tm{};
                                tm.src = handle(3, s1 + C1.col[t]);
                                tm.ld = C1.width;
                                tm.coef = cf;
                                P.B.terms.push_back(tm);
                            }
                        }
                        O.nterm = static_cast<int>(P.B.terms.size()) - O.term0;
                        P.B.flops += 2.0 * O.rows * O.cols * O.nterm;
                        P.B.outs.push_back(O);
                    }
                    t3 += static_cast<int64_t>(M) * CL.width;
                    c3[u * ngl + ga] = CL;
                }
            P.flops_op[op] += (P.A.flops - fa0) + (P.B.flops - fb0);
            P.flopsA_op[op] += P.A.flops - fa0;
            P.flopsB_op[op] += P.B.flops - fb0;
        }
        // algorithmic bytes of phase A for this op: its environment, x and T1, each once per g
        P.bytesA_op[op] = 8.0 * (static_cast<double>(G) * (Le.lay[op].size + xl.size)) + 8.0 * static_cast<double>(t1 - t1_op0);
        P.bytesB_op[op] = 8.0 * static_cast<double>((t1 - t1_op0) + (t3 - t3_op0));
        t1_op0 = t1;
        t3_op0 = t3;
    }
    // phase C: one task per (N, M)-allowed output block and beta point, writing the partial sum
    // over the channels u into the per-g slice of the partial buffer (slot 8 for y, 9 for z); a
    // deterministic reduction over g (launch_sum_partials) produces y and z
    const int64_t nx = xl.size;
    for (int op = 0; op < nops; ++op) {
        const MPO& m = h->ops.mpo[op];
        const int dwr = m.dw[k + 2];
        const double fc0 = P.C.flops;
        for (int g = 0; g < G; ++g) {
            const int og = op * G + g;
            P.tileC_rng[og] = static_cast<int>(P.C.tasks.size());
            for (size_t la = 0; la < bl.labels.size(); ++la) {
                const Label& La = bl.labels[la];
                const int ga = La.group;
                for (int s = 0; s < 16; ++s) {
                    const int lb = xl.seg_label[la * 16 + s];
                    if (lb < 0) continue;
                    const Label& Lb = br.labels[lb];
                    const int gb = Lb.group;
                    GemmTask T{};
                    T.c = handle(8 + op, static_cast<int64_t>(g) * nx + xl.row_off[la] + xl.seg_col[la * 16 + s]);
                    T.cmap = -1;
                    T.M = La.dim;
                    T.N = Lb.dim;
                    T.key = lb;  // all output blocks of one right label read its environment rows
                    T.ldc = xl.width[la];
                    T.seg0 = static_cast<int>(P.C.segs.size());
                    for (int u = 0; u < dwr; ++u) {
                        const int64_t s3 = o3_all[og][u * ngl + ga];
                        if (s3 < 0) continue;
                        const ColLayout& C3 = c3_all[og][u * ngl + ga];
                        if (C3.col[s] < 0) continue;
                        const int64_t roff = Re.lay[op].off[u * ngr + gb];
                        if (roff < 0) continue;
                        const Group& Gk = br.groups[C3.group[s]];
                        const int K = Gk.dim;
                        // unscreened: one segment over the ket group; screened: one per ket label,
                        // dropped when its environment sub-block is below the threshold
                        const int nsub = screen ? Gk.count : 1;
                        for (int q = 0; q < nsub; ++q) {
                            const int k0 = screen ? br.labels[Gk.first + q].off - Gk.off : 0;
                            const int kl = screen ? br.labels[Gk.first + q].dim : K;
                            if (screen && nR->dropped(op, g, u, gb, lb - br.groups[gb].first, q, tau))
                                continue;
                            GemmSeg sg{};
                            sg.a = handle(4, s3 + static_cast<int64_t>(La.off - bl.groups[ga].off) * C3.width + C3.col[s] +
                                                 k0);
                            sg.a_rs = C3.width;
                            sg.a_cs = 1;
                            sg.K = kl;
                            sg.b = handle(6, Re.base[og] + roff + static_cast<int64_t>(Lb.off - br.groups[gb].off) * K + k0);
                            sg.b_rs = 1;
                            sg.b_cs = K;
                            P.C.segs.push_back(sg);
                            P.C.flops += 2.0 * T.M * T.N * kl;
                        }
                    }
                    T.nseg = static_cast<int>(P.C.segs.size()) - T.seg0;
                    P.C.tasks.push_back(T);
                }
            }
        }
        P.flops_op[op] += P.C.flops - fc0;
        P.flopsC_op[op] += P.C.flops - fc0;
        // phase C reads this op's T3 and right environment and writes G partial outputs
        const int64_t t3_op = (op + 1 < nops ? t3_op_begin[op + 1] : t3) - t3_op_begin[op];
        P.bytesC_op[op] = 8.0 * (static_cast<double>(t3_op) + static_cast<double>(G) * (Re.lay[op].size + nx));
    }
    P.reduce_nx = nx;
    P.tileA_rng[nops * G] = static_cast<int>(P.A.tasks.size());
    P.combB_rng[nops * G] = static_cast<int>(P.B.outs.size());
    P.tileC_rng[nops * G] = static_cast<int>(P.C.tasks.size());
    P.t1_size = t1;
    P.t2_size = t3;
    P.flops = P.A.flops + P.B.flops + P.C.flops;

    // diagonal of the projected operators on the x layout: for each output block and beta point,
    // the pairs (w, u) of charge-0 channels with a nonzero diagonal WW coefficient
    for (int op = 0; op < nops; ++op) {
        for (size_t la = 0; la < bl.labels.size(); ++la) {
            const Label& La = bl.labels[la];
            const int ga = La.group;
            for (int s = 0; s < 16; ++s) {
                const int lb = xl.seg_label[la * 16 + s];
                if (lb < 0) continue;
                const Label& Lb = br.labels[lb];
                const int gb = Lb.group;
                DiagBlock B{};
                B.off = xl.row_off[la] + xl.seg_col[la * 16 + s];
                B.rows = La.dim;
                B.cols = Lb.dim;
                B.ld = xl.width[la];
                B.out = op;
                B.term0 = static_cast<int>(P.diag_terms.size());
                for (int g = 0; g < G; ++g) {
                    const int og = op * G + g;
                    for (const DiagPair& d : diag_all[og]) {
                        const double cf = d.c[s];
                        if (cf == 0.0) continue;
                        const int64_t loff = Le.lay[op].off[d.w * ngl + ga];
                        if (loff < 0) continue;
                        const int64_t roff = Re.lay[op].off[d.u * ngr + gb];
                        if (roff < 0) continue;
                        const int gdl = bl.groups[ga].dim, gdr = br.groups[gb].dim;
                        DiagTerm t{};
                        t.l = handle(5, Le.base[og] + loff + static_cast<int64_t>(La.off - bl.groups[ga].off) * (gdl + 1));
                        t.l_step = gdl + 1;
                        t.r = handle(6, Re.base[og] + roff + static_cast<int64_t>(Lb.off - br.groups[gb].off) * (gdr + 1));
                        t.r_step = gdr + 1;
                        t.coef = cf;
                        P.diag_terms.push_back(t);
                    }
                }
                B.nterm = static_cast<int>(P.diag_terms.size()) - B.term0;
                P.diag_blocks.push_back(B);
            }
        }
    }
}

// ---- environment maintenance -------------------------------------------------------------------

spmps_status update_left(spmps_t* h, int i) {
    EnvStore& Lo = h->Lenv[i];
    EnvStore& Ln = h->Lenv[i + 1];
    spmps_status st = env_prepare(h, Ln, h->bonds[i + 1], i + 1);
    if (st != SPMPS_OK) return st;
    Plan P;
    build_left_plan(h, i, Lo, Ln, P);
    {
        int64_t sz[kMaxSlots];
        for (auto& v : sz) v = -1;
        sz[0] = h->alay[i].size;
        sz[3] = P.t1_size;
        sz[4] = P.t2_size;
        sz[5] = Lo.total;
        sz[7] = Ln.total;
        std::string why;
        if (!validate_plan(P, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (left update): " + why);
    }
    st = plan_upload(h, P);
    if (st != SPMPS_OK) return st;
    Slots S{};
    S.p[0] = h->A[i]->as<double>();
    S.p[3] = h->work1.as<double>();
    S.p[4] = h->work2.as<double>();
    S.p[5] = Lo.buf.as<double>();
    S.p[7] = Ln.buf.as<double>();
    st = plan_run(h, P, S, 0, h->ops.n_ops() * h->G, h->stream);
    if (st != SPMPS_OK) return st;
    CK(cudaStreamSynchronize(h->stream));  // plan buffers are freed on return
    Ln.valid = true;
    Ln.version = ++h->env_counter;
    return SPMPS_OK;
}

spmps_status update_right(spmps_t* h, int i) {
    EnvStore& Ro = h->Renv[i + 1];
    EnvStore& Rn = h->Renv[i];
    spmps_status st = env_prepare(h, Rn, h->bonds[i], i);
    if (st != SPMPS_OK) return st;
    Plan P;
    build_right_plan(h, i, Ro, Rn, P);
    {
        int64_t sz[kMaxSlots];
        for (auto& v : sz) v = -1;
        sz[0] = h->alay[i].size;
        sz[3] = P.t1_size;
        sz[4] = P.t2_size;
        sz[6] = Ro.total;
        sz[7] = Rn.total;
        std::string why;
        if (!validate_plan(P, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (right update): " + why);
    }
    st = plan_upload(h, P);
    if (st != SPMPS_OK) return st;
    Slots S{};
    S.p[0] = h->A[i]->as<double>();
    S.p[3] = h->work1.as<double>();
    S.p[4] = h->work2.as<double>();
    S.p[6] = Ro.buf.as<double>();
    S.p[7] = Rn.buf.as<double>();
    st = plan_run(h, P, S, 0, h->ops.n_ops() * h->G, h->stream);
    if (st != SPMPS_OK) return st;
    CK(cudaStreamSynchronize(h->stream));
    Rn.valid = true;
    Rn.version = ++h->env_counter;
    return SPMPS_OK;
}

spmps_status ensure_envs(spmps_t* h, int k) {
    // L(bond k) and R(bond k+2)
    if (!h->Lenv[0].valid) {
        spmps_status st = env_boundary(h, h->Lenv[0], 0);
        if (st != SPMPS_OK) return st;
    }
    if (!h->Renv[h->K].valid) {
        spmps_status st = env_boundary(h, h->Renv[h->K], h->K);
        if (st != SPMPS_OK) return st;
    }
    int b = k;
    while (!h->Lenv[b].valid) --b;
    for (int i = b; i < k; ++i) {
        spmps_status st = update_left(h, i);
        if (st != SPMPS_OK) return st;
    }
    int r = k + 2;
    while (!h->Renv[r].valid) ++r;
    for (int i = r - 1; i >= k + 2; --i) {
        spmps_status st = update_right(h, i);
        if (st != SPMPS_OK) return st;
    }
    return SPMPS_OK;
}

void invalidate_all(spmps_t* h) {
    for (auto& e : h->Lenv) e.valid = false;
    for (auto& e : h->Renv) e.valid = false;
    for (auto& p : h->apply_plans) p.reset();
    excited_invalidate(h);
}

// Autotuner: time every tile candidate for phases A and C of the site's action plan (one warm-up
// and two timed actions each on zero scratch vectors, CUDA events around the phases) and keep
// the fastest per phase; the choice is cached per site for the life of the handle.
spmps_status tune_apply_plan(spmps_t* h, int k, Plan& P) {
    if (h->tune_a.size() != static_cast<size_t>(h->K)) {
        h->tune_a.assign(h->K, -1);
        h->tune_c.assign(h->K, -1);
    }
    if (h->tune_a[k] < 0) {
        struct Prec {  // tune with the FP64 kernels whatever the solver stage
            spmps_t* h;
            int saved;
            ~Prec() { h->apply_precision = saved; }
        } prec{h, h->apply_precision};
        h->apply_precision = 0;
        const int64_t nx = std::max<int64_t>(1, P.reduce_nx);
        CK(h->tunebuf.ensure(3 * nx * sizeof(double)));
        CK(cudaMemsetAsync(h->tunebuf.p, 0, 3 * nx * sizeof(double), h->stream));
        CK(h->work3.ensure(std::max<int64_t>(1, 2 * static_cast<int64_t>(h->G) * P.reduce_nx) * sizeof(double)));
        cudaEvent_t ev[5];
        for (auto& e : ev) CK(cudaEventCreate(&e));
        float best_a = INFINITY, best_c = INFINITY;
        int ia = 0, ic = 0;
        spmps_status st = SPMPS_OK;
        for (int c = 0; c < kTileCandidates && st == SPMPS_OK; ++c) {
            P.polA = P.polC = tile_candidate(c);
            st = plan_upload(h, P);
            if (st != SPMPS_OK) break;
            Slots S{};
            S.p[0] = h->tunebuf.as<double>();
            S.p[1] = S.p[0] + nx;
            S.p[2] = S.p[0] + 2 * nx;
            S.p[3] = h->work1.as<double>();
            S.p[4] = h->work2.as<double>();
            S.p[5] = h->Lenv[k].buf.as<double>();
            S.p[6] = h->Renv[k + 2].buf.as<double>();
            S.p[8] = h->work3.as<double>();
            S.p[9] = h->work3.as<double>() + static_cast<int64_t>(h->G) * P.reduce_nx;
            float ta = 0.0f, tc = 0.0f;
            for (int rep = 0; rep < 3 && st == SPMPS_OK; ++rep) {
                st = plan_run(h, P, S, 0, 2 * h->G, h->stream, ev);
                if (st != SPMPS_OK) break;
                if (cudaEventSynchronize(ev[4]) != cudaSuccess) { st = fail(h, SPMPS_ERR_CUDA, "autotune timing"); break; }
                if (rep == 0) continue;
                float a = 0.0f, cc = 0.0f;
                cudaEventElapsedTime(&a, ev[1], ev[2]);
                cudaEventElapsedTime(&cc, ev[3], ev[4]);
                ta += a;
                tc += cc;
            }
            if (ta < best_a) { best_a = ta; ia = c; }
            if (tc < best_c) { best_c = tc; ic = c; }
        }
        for (auto& e : ev) cudaEventDestroy(e);
        if (st != SPMPS_OK) return st;
        h->tune_a[k] = ia;
        h->tune_c[k] = ic;
    }
    P.polA = tile_candidate(h->tune_a[k]);
    P.polC = tile_candidate(h->tune_c[k]);
    return SPMPS_OK;
}

spmps_status get_apply_plan(spmps_t* h, int k, Plan** out) {
    spmps_status st = ensure_envs(h, k);
    if (st != SPMPS_OK) return st;
    const double tau = h->opt.m_screen;
    if (tau > 0.0 && h->apply_plans[k] &&
        (h->apply_plans[k]->envL_version != h->Lenv[k].version || h->apply_plans[k]->envR_version != h->Renv[k + 2].version))
        h->apply_plans[k].reset();  // screened plans follow the environment values
    if (!h->apply_plans[k]) {
        auto P = std::make_unique<Plan>();
        EnvNorms nL, nR;
        if (tau > 0.0) {
            st = env_subblock_norms(h, h->Lenv[k], h->bonds[k], k, nL);
            if (st != SPMPS_OK) return st;
            st = env_subblock_norms(h, h->Renv[k + 2], h->bonds[k + 2], k + 2, nR);
            if (st != SPMPS_OK) return st;
        }
        build_apply_plan(h, k, h->Lenv[k], h->Renv[k + 2], *P, &nL, &nR, tau);
        P->envL_version = h->Lenv[k].version;
        P->envR_version = h->Renv[k + 2].version;
        {
            int64_t sz[kMaxSlots];
            for (auto& v : sz) v = -1;
            const int64_t nx = make_row_block_layout(h->bonds[k], h->bonds[k + 2], 16).size;
            sz[0] = sz[1] = sz[2] = nx;
            sz[3] = P->t1_size;
            sz[4] = P->t2_size;
            sz[5] = h->Lenv[k].total;
            sz[6] = h->Renv[k + 2].total;
            sz[8] = sz[9] = static_cast<int64_t>(h->G) * nx;
            std::string why;
            if (!validate_plan(*P, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (apply): " + why);
        }
        if (h->opt.autotune) {
            st = tune_apply_plan(h, k, *P);
            if (st != SPMPS_OK) return st;
        }
        st = plan_upload(h, *P);
        if (st != SPMPS_OK) return st;
        CK(h->work3.ensure(std::max<int64_t>(1, 2 * static_cast<int64_t>(h->G) * P->reduce_nx) * sizeof(double)));
        h->apply_plans[k] = std::move(P);
    }
    *out = h->apply_plans[k].get();
    return SPMPS_OK;
}

spmps_status do_apply(spmps_t* h, int k, const double* x, double* y, double* z, cudaStream_t st,
                      cudaEvent_t* ev) {
    Plan* P = nullptr;
    spmps_status s = get_apply_plan(h, k, &P);
    if (s != SPMPS_OK) return s;
    Slots S{};
    S.p[0] = const_cast<double*>(x);
    S.p[1] = y;
    S.p[2] = z;
    S.p[3] = h->work1.as<double>();
    S.p[4] = h->work2.as<double>();
    S.p[5] = h->Lenv[k].buf.as<double>();
    S.p[6] = h->Renv[k + 2].buf.as<double>();
    S.p[8] = h->work3.as<double>();
    S.p[9] = h->work3.as<double>() + static_cast<int64_t>(h->G) * P->reduce_nx;
    const int G = h->G;
    SlotsF SF{};
    const SlotsF* split = nullptr;
    if (h->apply_precision > 0 && y) {
        // pre-split TF32 operands: environments once per update, x and T3 per action (plan_run)
        for (EnvStore* E : {&h->Lenv[k], &h->Renv[k + 2]}) {
            if (E->split_version != E->version) {
                CK(E->split.ensure(std::max<int64_t>(1, E->total) * sizeof(float2)));
                CK(launch_split_tf32(E->buf.as<double>(), E->total, static_cast<float2*>(E->split.p), st));
                ++h->launches;
                E->split_version = E->version;
            }
        }
        CK(h->xsplit.ensure(std::max<int64_t>(1, P->reduce_nx) * sizeof(float2)));
        CK(h->t3split.ensure(std::max<int64_t>(1, P->t2_size) * sizeof(float2)));
        SF.p[0] = static_cast<float2*>(h->xsplit.p);
        SF.p[4] = static_cast<float2*>(h->t3split.p);
        SF.p[5] = static_cast<float2*>(h->Lenv[k].split.p);
        SF.p[6] = static_cast<float2*>(h->Renv[k + 2].split.p);
        split = &SF;
    }
    if (y && z) s = plan_run(h, *P, S, 0, 2 * G, st, ev, split);
    else if (y) s = plan_run(h, *P, S, 0, G, st, ev, split);
    else if (z) s = plan_run(h, *P, S, G, 2 * G, st, ev, split);
    if (s != SPMPS_OK) return s;
    ++h->applies;
    h->last_apply_flops = P->flops;
    h->apply_flops_total += (y ? P->flops_op[0] : 0.0) + (z ? P->flops_op[1] : 0.0);
    return SPMPS_OK;
}

// ---- profiler ---------------------------------------------------------------------------------

int prof_begin(spmps_t* h, cudaStream_t st, int kind, double flops) {
    spmps_t::TimerRec r{};
    if (!h->timers_free.empty()) {
        r = h->timers_free.back();
        h->timers_free.pop_back();
    } else {
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
    }
    r.kind = kind;
    r.flops = flops;
    if (cudaEventRecord(r.a, st) != cudaSuccess) {
        h->timers_free.push_back(r);
        return -1;
    }
    h->timers_live.push_back(r);
    return static_cast<int>(h->timers_live.size()) - 1;
}

void prof_end(spmps_t* h, cudaStream_t st, int rec) {
    cudaEventRecord(h->timers_live[rec].b, st);
    if (h->timers_live.size() >= 4096) prof_collect(h);
}

spmps_status prof_collect(spmps_t* h) {
    for (auto& r : h->timers_live) {
        CK(cudaEventSynchronize(r.b));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        h->prof_launches[r.kind] += 1;
        h->prof_ms[r.kind] += ms;
        h->prof_flops[r.kind] += r.flops;
        h->timers_free.push_back(r);
    }
    h->timers_live.clear();
    return SPMPS_OK;
}

spmps_status check_ready(spmps_t* h) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!h->has_ham) return fail(h, SPMPS_ERR_STATE, "no Hamiltonian set");
    if (!h->has_mps) return fail(h, SPMPS_ERR_STATE, "no MPS set");
    return SPMPS_OK;
}

spmps_status build_opset(spmps_t* h, const MPO& Hin, OpSet* out) {
    std::string e;
    MPO H = Hin;
    if (!H.finalize_charges(&e)) return fail(h, SPMPS_ERR_BAD_INPUT, e);
    MPO I = mpo_identity(h->K);
    I.finalize_charges(&e);
    out->mpo.clear();
    out->mpo.push_back(H);
    out->mpo.push_back(I);
    out->rot.assign(2, {});
    for (int op = 0; op < 2; ++op)
        for (int g = 0; g < h->G; ++g) {
            MPO r = mpo_rotated(out->mpo[op], h->beta[g]);
            r.cn = out->mpo[op].cn;
            out->rot[op].push_back(r);
        }
    return SPMPS_OK;
}

spmps_status set_ops(spmps_t* h, MPO H) {
    spmps_status st = build_opset(h, H, &h->ops);
    if (st != SPMPS_OK) return st;
    h->has_ham = true;
    invalidate_all(h);
    return SPMPS_OK;
}

}  // namespace eng
}  // namespace spmps

// =============================================================================================
// C ABI
// =============================================================================================

extern "C" {

void spmps_default_options(spmps_options* o) {
    if (!o) return;
    o->batched = 1;
    o->precond = 0;
    o->cg_steps = 5;
    o->dav_tol_r = 1e-6;
    o->dav_tol_theta = 1e-10;
    o->dav_max_sub = 20;
    o->dav_max_iter = 200;
    o->device = 0;
    o->jacobi_smem_max = 0;
    o->precision = 0;
    o->autotune = 0;
    o->metric_max_dim = 0;
    o->tc_wait_polls = 0;
    o->tensor_core_kernel = 0;
    o->m_screen = 0.0;
    o->fp64_tensor_cores = 0;
}

const char* spmps_last_error(spmps_handle h) { return h ? h->err.c_str() : g_static_err.c_str(); }

spmps_status spmps_create(int K, int N, int twoM, int twoS, int n_beta, int D, const spmps_options* opt,
                          spmps_handle* out) {
    if (!out) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "out is NULL");
    *out = nullptr;
    if (K < 2 || D < 1 || n_beta < 1) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "need K >= 2, D >= 1, n_beta >= 1");
    if (N < 0 || N > 2 * K) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "N out of range");
    if (((N + twoM) & 1) != 0) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "N + 2M must be even");
    if (twoS < (twoM < 0 ? -twoM : twoM)) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "need 2S >= |2M|");
    if (((twoS + N) & 1) != 0) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "2S + N must be even");
    const int na = (N + twoM) / 2, nb = (N - twoM) / 2;
    if (na < 0 || na > K || nb < 0 || nb > K) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "electron counts out of range");
    spmps_options o;
    spmps_default_options(&o);
    if (opt) o = *opt;
    if (o.dav_max_sub < 4 || o.dav_max_sub > 32) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "dav_max_sub must be in [4, 32]");
    if (o.dav_max_iter < 1) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "dav_max_iter must be >= 1");
    if (!(o.m_screen >= 0.0 && o.m_screen < 1.0)) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "m_screen must be in [0, 1)");
    if (o.tensor_core_kernel < 0 || o.tensor_core_kernel > 1)
        return fail(nullptr, SPMPS_ERR_BAD_INPUT, "tensor_core_kernel must be 0 or 1");
    if (o.fp64_tensor_cores < 0 || o.fp64_tensor_cores > 1)
        return fail(nullptr, SPMPS_ERR_BAD_INPUT, "fp64_tensor_cores must be 0 or 1");
    if (o.metric_max_dim < 0 || o.tc_wait_polls < 0)
        return fail(nullptr, SPMPS_ERR_BAD_INPUT, "metric_max_dim and tc_wait_polls must be >= 0");
    if (o.jacobi_smem_max < 0 || o.jacobi_smem_max > 112)
        return fail(nullptr, SPMPS_ERR_BAD_INPUT, "jacobi_smem_max must be in [0, 112]");
    if (o.jacobi_smem_max == 0) o.jacobi_smem_max = 112;
    if (o.precond < 0 || o.precond > 4) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "precond must be 0, 1, 2, 3 or 4");
    if (o.precision < 0 || o.precision > 2) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "precision must be 0, 1 or 2");
    if (o.autotune != 0 && o.autotune != 1) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "autotune must be 0 or 1");
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev <= o.device)
        return fail(nullptr, SPMPS_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(ce));
    auto* h = new spmps_t();
    h->K = K; h->N = N; h->twoM = twoM; h->twoS = twoS; h->G = n_beta; h->D = D;
    h->opt = o;
    h->device = o.device;
    if (cudaSetDevice(h->device) != cudaSuccess || cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return fail(nullptr, SPMPS_ERR_CUDA, "cannot create a stream on the device");
    }
    // quadrature of Eq. pmpo with the (2S+1)/2 prefactor of Eq. PSMM folded into the weights
    std::vector<double> x, w;
    gauss_legendre(n_beta, x, w);
    h->beta.resize(n_beta);
    h->cg.resize(n_beta);
    for (int g = 0; g < n_beta; ++g) {
        h->beta[g] = std::acos(x[g]);
        h->cg[g] = 0.5 * (twoS + 1) * w[g] * wigner_small_d(twoS, twoM, twoM, h->beta[g]);
    }
    h->Lenv.resize(K + 1);
    h->Renv.resize(K + 1);
    h->apply_plans.resize(K);
    if (h->partial.ensure(kPartialDoubles * sizeof(double)) != cudaSuccess) {
        delete h;
        return fail(nullptr, SPMPS_ERR_OOM, "workspace");
    }
    *out = h;
    return SPMPS_OK;
}

spmps_status spmps_destroy(spmps_handle h) {
    if (!h) return SPMPS_OK;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& r : h->timers_live) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto& r : h->timers_free) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    h->apply_plans.clear();
    h->Lenv.clear();
    h->Renv.clear();
    h->A.clear();
    if (h->aux_stream) {
        cudaStreamSynchronize(h->aux_stream);
        cudaStreamDestroy(h->aux_stream);
    }
    if (h->aux_fork) cudaEventDestroy(h->aux_fork);
    if (h->aux_join) cudaEventDestroy(h->aux_join);
    if (h->noalloc_order) cudaEventDestroy(h->noalloc_order);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return SPMPS_OK;
}

spmps_status spmps_set_hubbard(spmps_handle h, double t, double U) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!std::isfinite(t) || !std::isfinite(U)) return fail(h, SPMPS_ERR_BAD_INPUT, "t and U must be finite");
    const int K = h->K;
    const size_t Kz = static_cast<size_t>(K);
    std::vector<double> h1(Kz * Kz, 0.0), h2(Kz * Kz * Kz * Kz, 0.0);
    for (int p = 0; p + 1 < K; ++p) h1[p * K + p + 1] = h1[(p + 1) * K + p] = -t;
    for (size_t p = 0; p < Kz; ++p) h2[((p * Kz + p) * Kz + p) * Kz + p] = U;
    spmps_status st = set_ops(h, mpo_hubbard(K, t, U));
    if (st != SPMPS_OK) return st;
    h->ints_h1.swap(h1);
    h->ints_h2.swap(h2);
    h->ints_ecore = 0.0;
    return SPMPS_OK;
}

namespace {
// Integrals that only couple nearest neighbours (h1) and repeat one orbital ((pp|pp)) take the
// bond-dimension-6 Hubbard-like MPO; anything else the general builder.
bool nearest_neighbour_only(int K, const double* h1, const double* h2) {
    for (int p = 0; p < K; ++p)
        for (int q = 0; q < K; ++q)
            if (std::abs(p - q) > 1 && h1[p * K + q] != 0.0) return false;
    if (!h2) return true;
    const size_t Kz = static_cast<size_t>(K);
    for (size_t p = 0; p < Kz; ++p)
        for (size_t q = 0; q < Kz; ++q)
            for (size_t r = 0; r < Kz; ++r)
                for (size_t s = 0; s < Kz; ++s)
                    if (h2[((p * Kz + q) * Kz + r) * Kz + s] != 0.0 && !(p == q && q == r && r == s)) return false;
    return true;
}

spmps_status check_integrals(spmps_t* h, int K, const double* h1, const double* h2, double ecore) {
    if (!h1) return fail(h, SPMPS_ERR_BAD_INPUT, "h1 is NULL");
    if (!std::isfinite(ecore)) return fail(h, SPMPS_ERR_BAD_INPUT, "ecore not finite");
    for (int p = 0; p < K * K; ++p)
        if (!std::isfinite(h1[p])) return fail(h, SPMPS_ERR_BAD_INPUT, "h1 not finite");
    if (h2) {
        const size_t n4 = static_cast<size_t>(K) * K * K * K;
        for (size_t i = 0; i < n4; ++i)
            if (!std::isfinite(h2[i])) return fail(h, SPMPS_ERR_BAD_INPUT, "h2 not finite");
    }
    return SPMPS_OK;
}

// the library's MPO site tensors (one copy per beta point) are held on the host: keep them within this size
constexpr double kMaxMpoHostBytes = 4.0e9;

bool mpo_fits(const MPO& m, int copies, std::string* why) {
    const double bytes = static_cast<double>(m.entries()) * sizeof(MpoEntry);
    if (bytes * copies > kMaxMpoHostBytes) {
        if (why) *why = "MPO site tensors need " + std::to_string(bytes * copies / 1e9) + " GB of host memory";
        return false;
    }
    return true;
}
}  // namespace

spmps_status spmps_set_hamiltonian(spmps_handle h, const double* h1, const double* h2, double ecore) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    const int K = h->K;
    spmps_status st = check_integrals(h, K, h1, h2, ecore);
    if (st != SPMPS_OK) return st;
    // Davidson needs a Hermitian H: h_pq = h_qp and (pq|rs) = (qp|sr) for real orbitals
    for (int p = 0; p < K; ++p)
        for (int q = 0; q < p; ++q)
            if (std::fabs(h1[p * K + q] - h1[q * K + p]) > 1e-12 * (1.0 + std::fabs(h1[p * K + q])))
                return fail(h, SPMPS_ERR_BAD_INPUT, "h1 is not symmetric");
    if (h2) {
        const size_t Kz = static_cast<size_t>(K);
        for (size_t p = 0; p < Kz; ++p)
            for (size_t q = 0; q < Kz; ++q)
                for (size_t r = 0; r < Kz; ++r)
                    for (size_t s2 = 0; s2 < Kz; ++s2) {
                        const double a = h2[((p * Kz + q) * Kz + r) * Kz + s2], b = h2[((q * Kz + p) * Kz + s2) * Kz + r];
                        if (std::fabs(a - b) > 1e-12 * (1.0 + std::fabs(a)))
                            return fail(h, SPMPS_ERR_BAD_INPUT, "h2 is not Hermitian: (pq|rs) != (qp|sr)");
                    }
    }
    if (nearest_neighbour_only(K, h1, h2)) {
        std::vector<double> eps(K), hop(K > 1 ? K - 1 : 0), U(K, 0.0);
        for (int p = 0; p < K; ++p) eps[p] = h1[p * K + p];
        for (int p = 0; p + 1 < K; ++p) hop[p] = h1[p * K + p + 1];
        if (h2) {
            const size_t Kz = static_cast<size_t>(K);
            for (size_t p = 0; p < Kz; ++p) U[p] = h2[((p * Kz + p) * Kz + p) * Kz + p];
        }
        st = set_ops(h, mpo_nearest_neighbour(K, eps, hop, U, ecore));
    } else {
        MPO m;
        std::string why;
        if (!mpo_ab_initio(K, h1, h2, ecore, 1 << 20, &m, &why)) return fail(h, SPMPS_ERR_BAD_INPUT, why);
        if (!mpo_fits(m, h->G + 1, &why)) return fail(h, SPMPS_ERR_UNSUPPORTED, why);
        st = set_ops(h, std::move(m));
    }
    if (st != SPMPS_OK) return st;
    const size_t Kz = static_cast<size_t>(K);
    h->ints_h1.assign(h1, h1 + Kz * Kz);
    if (h2) h->ints_h2.assign(h2, h2 + Kz * Kz * Kz * Kz);
    else h->ints_h2.clear();
    h->ints_ecore = ecore;
    return SPMPS_OK;
}

spmps_status spmps_set_mpo(spmps_handle h, const int* bond_dims, const double* const* sites) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!bond_dims || !sites) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    const int K = h->K;
    if (bond_dims[0] != 1 || bond_dims[K] != 1) return fail(h, SPMPS_ERR_BAD_INPUT, "boundary MPO bonds must have dimension 1");
    std::vector<int> dims(bond_dims, bond_dims + K + 1);
    for (int b = 0; b <= K; ++b)
        if (dims[b] < 1) return fail(h, SPMPS_ERR_BAD_INPUT, "MPO bond dimension < 1");
    MPO m;
    m.init(K, dims);
    for (int k = 0; k < K; ++k) {
        if (!sites[k]) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL MPO site tensor");
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
    std::string why;
    if (!mpo_fits(m, h->G + 1, &why)) return fail(h, SPMPS_ERR_UNSUPPORTED, why);
    if (!m.finalize_charges(&why)) return fail(h, SPMPS_ERR_BAD_INPUT, why);
    h->ints_h1.clear();
    h->ints_h2.clear();
    h->ints_ecore = 0.0;
    return set_ops(h, std::move(m));
}

spmps_status spmps_mpo_from_integrals(int K, const double* h1, const double* h2, double ecore, int* bond_dims,
                                      double* const* sites) {
    if (K < 2) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "need K >= 2");
    if (!bond_dims) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "bond_dims is NULL");
    spmps_status st = check_integrals(nullptr, K, h1, h2, ecore);
    if (st != SPMPS_OK) return st;
    MPO m;
    std::string why;
    if (!mpo_ab_initio(K, h1, h2, ecore, 1 << 20, &m, &why)) return fail(nullptr, SPMPS_ERR_BAD_INPUT, why);
    for (int b = 0; b <= K; ++b) bond_dims[b] = m.dw[b];
    if (!sites) return SPMPS_OK;
    for (int k = 0; k < K; ++k) {
        if (!sites[k]) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "NULL site pointer");
        const size_t n = static_cast<size_t>(m.dw[k]) * m.dw[k + 1] * 16;
        std::fill(sites[k], sites[k] + n, 0.0);
        for (const auto& e : m.E[k])
            std::copy(e.op, e.op + 16, sites[k] + (static_cast<size_t>(e.wl) * m.dw[k + 1] + e.wr) * 16);
    }
    return SPMPS_OK;
}

spmps_status spmps_set_mps(spmps_handle h, const int* bond_dims, const int* labels, const double* const* sites,
                           int center) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!bond_dims || !labels || !sites) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    const int K = h->K;
    if (bond_dims[0] != 1 || bond_dims[K] != 1) return fail(h, SPMPS_ERR_BAD_INPUT, "boundary bonds must have dimension 1");
    if (center < 0 || center >= K) return fail(h, SPMPS_ERR_BAD_INPUT, "center out of range");
    std::vector<Bond> bonds(K + 1);
    const int* lp = labels;
    for (int b = 0; b <= K; ++b) {
        const int Db = bond_dims[b];
        if (Db < 1) return fail(h, SPMPS_ERR_BAD_INPUT, "bond dimension < 1");
        for (int i = 0; i < Db; ++i) {
            const int n = lp[2 * i], tm = lp[2 * i + 1];
            if (i > 0) {
                const int pn = lp[2 * i - 2], ptm = lp[2 * i - 1];
                if (pn > n || (pn == n && ptm > tm)) return fail(h, SPMPS_ERR_BAD_INPUT, "bond labels not sorted");
                if (pn == n && ptm == tm) { bonds[b].labels.back().dim += 1; continue; }
            }
            bonds[b].labels.push_back(Label{n, tm, 1, 0, 0});
        }
        lp += 2 * Db;
        bonds[b].finalize();
    }
    if (bonds[0].labels[0].n != 0 || bonds[0].labels[0].tm != 0)
        return fail(h, SPMPS_ERR_BAD_INPUT, "bond 0 must carry (0, 0)");
    if (bonds[K].labels[0].n != h->N || bonds[K].labels[0].tm != h->twoM)
        return fail(h, SPMPS_ERR_BAD_INPUT, "bond K must carry (N, 2M)");
    h->bonds = bonds;
    h->alay.resize(K);
    h->A.clear();
    for (int k = 0; k < K; ++k) {
        const Bond& bl = h->bonds[k];
        const Bond& br = h->bonds[k + 1];
        h->alay[k] = make_row_block_layout(bl, br, 4);
        const RowBlockLayout& L = h->alay[k];
        std::vector<double> host(static_cast<size_t>(std::max<int64_t>(L.size, 1)), 0.0);
        const double* src = sites[k];
        if (!src) return fail(h, SPMPS_ERR_BAD_INPUT, "site pointer is NULL");
        for (size_t la = 0; la < bl.labels.size(); ++la) {
            const Label& La = bl.labels[la];
            for (int s = 0; s < 4; ++s) {
                const int lb = L.seg_label[la * 4 + s];
                if (lb < 0) continue;
                const Label& Lb = br.labels[lb];
                for (int i = 0; i < La.dim; ++i)
                    for (int j = 0; j < Lb.dim; ++j) {
                        const double v = src[(static_cast<size_t>(La.off + i) * 4 + s) * br.D + Lb.off + j];
                        if (!std::isfinite(v)) return fail(h, SPMPS_ERR_BAD_INPUT, "MPS entry not finite");
                        host[L.row_off[la] + static_cast<int64_t>(i) * L.width[la] + L.seg_col[la * 4 + s] + j] = v;
                    }
            }
        }
        auto m = std::make_unique<DevMem>();
        CK(m->ensure(host.size() * sizeof(double)));
        CK(cudaMemcpyAsync(m->p, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        h->A.push_back(std::move(m));
    }
    CK(cudaStreamSynchronize(h->stream));
    h->center = center;
    h->has_mps = true;
    invalidate_all(h);
    return SPMPS_OK;
}

spmps_status spmps_x_layout(spmps_handle h, int site, int64_t* n_x, int* n_blocks, int* blocks,
                            int64_t* row_block_offsets, int* row_block_widths, int* n_left_labels) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (!h->has_mps) return fail(h, SPMPS_ERR_STATE, "no MPS set");
    if (site < 0 || site > h->K - 2) return fail(h, SPMPS_ERR_BAD_INPUT, "site out of range");
    const Bond& bl = h->bonds[site];
    const Bond& br = h->bonds[site + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    if (n_x) *n_x = xl.size;
    if (n_left_labels) *n_left_labels = static_cast<int>(bl.labels.size());
    int nb = 0;
    for (size_t la = 0; la < bl.labels.size(); ++la) {
        if (row_block_offsets) row_block_offsets[la] = xl.row_off[la];
        if (row_block_widths) row_block_widths[la] = xl.width[la];
        for (int s = 0; s < 16; ++s) {
            const int lb = xl.seg_label[la * 16 + s];
            if (lb < 0) continue;
            if (blocks) {
                blocks[5 * nb + 0] = static_cast<int>(la);
                blocks[5 * nb + 1] = s;
                blocks[5 * nb + 2] = xl.seg_col[la * 16 + s];
                blocks[5 * nb + 3] = bl.labels[la].dim;
                blocks[5 * nb + 4] = br.labels[lb].dim;
            }
            ++nb;
        }
    }
    if (n_blocks) *n_blocks = nb;
    return SPMPS_OK;
}

spmps_status spmps_apply_heff(spmps_handle h, int site, const double* x, double* y, double* z, void* stream) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2) return fail(h, SPMPS_ERR_BAD_INPUT, "site out of range");
    if (!x || (!y && !z)) return fail(h, SPMPS_ERR_BAD_INPUT, "x and one of y, z are required");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    if (s != h->stream) {
        // environments are built on the handle's stream; order the caller's stream after it
        Plan* P = nullptr;
        st = get_apply_plan(h, site, &P);
        if (st != SPMPS_OK) return st;
        CK(cudaStreamSynchronize(h->stream));
    }
    h->apply_precision = h->opt.precision;
    st = do_apply(h, site, x, y, z, s);
    h->apply_precision = 0;
    return st;
}

spmps_status spmps_apply_heff_timed(spmps_handle h, int site, const double* x, double* y, double* z, void* stream,
                                    double* phase_ms) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2) return fail(h, SPMPS_ERR_BAD_INPUT, "site out of range");
    if (!x || (!y && !z) || !phase_ms) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    Plan* P = nullptr;
    st = get_apply_plan(h, site, &P);
    if (st != SPMPS_OK) return st;
    CK(cudaStreamSynchronize(h->stream));
    cudaEvent_t ev[5];
    for (auto& e : ev) CK(cudaEventCreate(&e));
    h->apply_precision = h->opt.precision;
    st = do_apply(h, site, x, y, z, s, ev);
    h->apply_precision = 0;
    if (st == SPMPS_OK) {
        CK(cudaEventSynchronize(ev[4]));
        for (int i = 0; i < 4; ++i) {
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            phase_ms[i] = ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return st;
}

spmps_status spmps_apply_costs(spmps_handle h, int site, double* flops6, double* bytes6) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2 || (!bytes6 && !flops6)) return fail(h, SPMPS_ERR_BAD_INPUT, "bad site or NULL");
    Plan* P = nullptr;
    st = get_apply_plan(h, site, &P);
    if (st != SPMPS_OK) return st;
    for (int op = 0; op < 2; ++op) {
        if (flops6) {
            flops6[3 * op + 0] = P->flopsA_op[op];
            flops6[3 * op + 1] = P->flopsB_op[op];
            flops6[3 * op + 2] = P->flopsC_op[op];
        }
        if (bytes6) {
            bytes6[3 * op + 0] = P->bytesA_op[op];
            bytes6[3 * op + 1] = P->bytesB_op[op];
            bytes6[3 * op + 2] = P->bytesC_op[op];
        }
    }
    return SPMPS_OK;
}

spmps_status spmps_apply_flops(spmps_handle h, int site, double* flops3) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2 || !flops3) return fail(h, SPMPS_ERR_BAD_INPUT, "bad site or NULL");
    Plan* P = nullptr;
    st = get_apply_plan(h, site, &P);
    if (st != SPMPS_OK) return st;
    flops3[0] = P->A.flops;
    flops3[1] = P->B.flops;
    flops3[2] = P->C.flops;
    return SPMPS_OK;
}

spmps_status spmps_device_fp64_peak(int device, double* tflops) {
    if (!tflops) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "NULL argument");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(nullptr, SPMPS_ERR_CUDA, cudaGetErrorString(e));
    e = measure_fp64_peak(tflops);
    if (e != cudaSuccess) return fail(nullptr, SPMPS_ERR_CUDA, cudaGetErrorString(e));
    return SPMPS_OK;
}

spmps_status spmps_apply_heff_host(spmps_handle h, int site, const double* x, double* y, double* z) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    int64_t n = 0;
    st = spmps_x_layout(h, site, &n, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != SPMPS_OK) return st;
    if (!x || (!y && !z)) return fail(h, SPMPS_ERR_BAD_INPUT, "x and one of y, z are required");
    const size_t nb = std::max<int64_t>(n, 1) * sizeof(double);
    CK(h->xbuf.ensure(nb));
    CK(h->ybuf.ensure(nb));
    CK(h->zbuf.ensure(nb));
    CK(cudaMemcpyAsync(h->xbuf.p, x, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->apply_precision = h->opt.precision;
    st = do_apply(h, site, h->xbuf.as<double>(), y ? h->ybuf.as<double>() : nullptr, z ? h->zbuf.as<double>() : nullptr,
                  h->stream);
    h->apply_precision = 0;
    if (st != SPMPS_OK) return st;
    if (y) CK(cudaMemcpyAsync(y, h->ybuf.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (z) CK(cudaMemcpyAsync(z, h->zbuf.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SPMPS_OK;
}

spmps_status spmps_two_site(spmps_handle h, int site, double* x) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2 || !x) return fail(h, SPMPS_ERR_BAD_INPUT, "bad site or NULL x");
    const Bond& bl = h->bonds[site];
    const Bond& bm = h->bonds[site + 1];
    const Bond& br = h->bonds[site + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    const RowBlockLayout& a0 = h->alay[site];
    const RowBlockLayout& a1 = h->alay[site + 1];
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
            const int s1 = s >> 2, s2 = s & 3;
            const int lc = a0.seg_label[la * 4 + s1];
            if (lc >= 0 && a1.seg_label[lc * 4 + s2] == lb) {
                GemmSeg sg{};
                sg.a = handle(0, a0.row_off[la] + a0.seg_col[la * 4 + s1]);
                sg.a_rs = a0.width[la];
                sg.a_cs = 1;
                sg.K = bm.labels[lc].dim;
                sg.b = handle(1, a1.row_off[lc] + a1.seg_col[lc * 4 + s2]);
                sg.b_rs = a1.width[lc];
                sg.b_cs = 1;
                                P.A.segs.push_back(sg);
            }
            T.nseg = static_cast<int>(P.A.segs.size()) - T.seg0;
            P.A.tasks.push_back(T);
        }
    P.A.add_tiles();
    {
        int64_t sz[kMaxSlots];
        for (auto& v : sz) v = -1;
        sz[0] = a0.size;
        sz[1] = a1.size;
        sz[2] = xl.size;
        std::string why;
        if (!validate_plan(P, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (two-site): " + why);
    }
    CK(upload(P.d_tasksA, P.A.tasks, h->stream));
    CK(upload(P.d_segsA, P.A.segs, h->stream));
    CK(upload(P.d_tilesA, P.A.tiles, h->stream));
    CK(upload(P.d_cmapsA, P.A.cmaps, h->stream));
    Slots S{};
    S.p[0] = h->A[site]->as<double>();
    S.p[1] = h->A[site + 1]->as<double>();
    S.p[2] = x;
    CK(launch_gemm_f64(S, P.d_tasksA.as<GemmTask>(), P.d_segsA.as<GemmSeg>(), P.d_tilesA.as<GemmTile>(),
                       P.d_cmapsA.as<int>(), static_cast<int>(P.A.tiles.size()), h->stream));
    ++h->launches;
    CK(cudaStreamSynchronize(h->stream));
    return SPMPS_OK;
}

spmps_status spmps_energy(spmps_handle h, double* E, double* norm_P) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    const int k = h->center < h->K - 1 ? h->center : h->K - 2;
    int64_t n = 0;
    st = spmps_x_layout(h, k, &n, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != SPMPS_OK) return st;
    const size_t nb = std::max<int64_t>(n, 1) * sizeof(double);
    CK(h->xbuf.ensure(nb));
    CK(h->ybuf.ensure(nb));
    CK(h->zbuf.ensure(nb));
    st = spmps_two_site(h, k, h->xbuf.as<double>());
    if (st != SPMPS_OK) return st;
    st = do_apply(h, k, h->xbuf.as<double>(), h->ybuf.as<double>(), h->zbuf.as<double>(), h->stream);
    if (st != SPMPS_OK) return st;
    DevMem dots;
    CK(dots.ensure(4 * sizeof(double)));
    double* d = dots.as<double>();
    CK(launch_multidot(h->xbuf.as<double>(), 0, 1, h->ybuf.as<double>(), n, d, h->partial.as<double>(), h->stream));
    CK(launch_multidot(h->xbuf.as<double>(), 0, 1, h->zbuf.as<double>(), n, d + 1, h->partial.as<double>(), h->stream));
    CK(launch_multidot(h->xbuf.as<double>(), 0, 1, h->xbuf.as<double>(), n, d + 2, h->partial.as<double>(), h->stream));
    h->launches += 6;
    double hd[3];
    CK(cudaMemcpyAsync(hd, d, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!std::isfinite(hd[0]) || !std::isfinite(hd[1])) return fail(h, SPMPS_ERR_NAN, "non-finite energy");
    if (hd[1] <= 0.0) return fail(h, SPMPS_ERR_SINGULAR_METRIC, "<Psi|P|Psi> is not positive");
    if (E) *E = hd[0] / hd[1];
    if (norm_P) *norm_P = hd[1] / hd[2];
    return SPMPS_OK;
}

spmps_status spmps_stats(spmps_handle h, int64_t* counts, double* values) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (counts) {
        counts[0] = h->dav_iters;
        counts[1] = h->applies;
        counts[2] = h->launches;
    }
    if (values) {
        values[0] = h->last_apply_flops;
        values[1] = h->last_discarded;
        values[2] = h->apply_flops_total;
    }
    return SPMPS_OK;
}

spmps_status spmps_davidson_stats(spmps_handle h, int64_t* iterations, int64_t* refine_iterations) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (iterations) *iterations = h->dav_iters;
    if (refine_iterations) *refine_iterations = h->refine_iters;
    return SPMPS_OK;
}

spmps_status spmps_get_mps(spmps_handle h, int* bond_dims, int* labels, double* const* sites, int* center) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (!bond_dims) return fail(h, SPMPS_ERR_BAD_INPUT, "bond_dims is NULL");
    const int K = h->K;
    for (int b = 0; b <= K; ++b) bond_dims[b] = h->bonds[b].D;
    if (center) *center = h->center;
    if (labels) {
        int* lp = labels;
        for (int b = 0; b <= K; ++b)
            for (const Label& l : h->bonds[b].labels)
                for (int i = 0; i < l.dim; ++i) { *lp++ = l.n; *lp++ = l.tm; }
    }
    if (!sites) return SPMPS_OK;
    for (int k = 0; k < K; ++k) {
        const Bond& bl = h->bonds[k];
        const Bond& br = h->bonds[k + 1];
        const RowBlockLayout& L = h->alay[k];
        std::vector<double> rb(static_cast<size_t>(std::max<int64_t>(L.size, 1)));
        CK(cudaMemcpyAsync(rb.data(), h->A[k]->p, L.size * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        double* dst = sites[k];
        if (!dst) continue;
        std::fill(dst, dst + static_cast<size_t>(bl.D) * 4 * br.D, 0.0);
        for (size_t la = 0; la < bl.labels.size(); ++la) {
            const Label& La = bl.labels[la];
            for (int s = 0; s < 4; ++s) {
                const int lb = L.seg_label[la * 4 + s];
                if (lb < 0) continue;
                const Label& Lb = br.labels[lb];
                for (int i = 0; i < La.dim; ++i)
                    for (int j = 0; j < Lb.dim; ++j)
                        dst[(static_cast<size_t>(La.off + i) * 4 + s) * br.D + Lb.off + j] =
                            rb[L.row_off[la] + static_cast<int64_t>(i) * L.width[la] + L.seg_col[la * 4 + s] + j];
            }
        }
    }
    return SPMPS_OK;
}

spmps_status spmps_stream(spmps_handle h, void** stream) {
    if (!h || !stream) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    *stream = h->stream;
    return SPMPS_OK;
}

spmps_status spmps_profile(spmps_handle h, int enable) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    spmps_status st = prof_collect(h);
    if (st != SPMPS_OK) return st;
    h->profile = enable != 0;
    if (enable) {
        for (int k = 0; k < spmps_t::kProfKinds; ++k) {
            h->prof_launches[k] = 0;
            h->prof_ms[k] = 0.0;
            h->prof_flops[k] = 0.0;
        }
    }
    return SPMPS_OK;
}

spmps_status spmps_kernel_stats(spmps_handle h, int kind, int64_t* launches, double* ms, double* flops) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (kind < 0 || kind >= spmps_t::kProfKinds) return fail(h, SPMPS_ERR_BAD_INPUT, "kind out of range");
    spmps_status st = prof_collect(h);
    if (st != SPMPS_OK) return st;
    if (launches) *launches = h->prof_launches[kind];
    if (ms) *ms = h->prof_ms[kind];
    if (flops) *flops = h->prof_flops[kind];
    return SPMPS_OK;
}

spmps_status spmps_quadrature(spmps_handle h, double* beta, double* c) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    for (int g = 0; g < h->G; ++g) {
        if (beta) beta[g] = h->beta[g];
        if (c) c[g] = h->cg[g];
    }
    return SPMPS_OK;
}

}  // extern "C"
