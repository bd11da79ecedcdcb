// Sweep-level entry points: generalised Davidson for H_eff x = theta N_eff x (Eq. geproblem),
// decimation of the two-site tensor in the canonical gauge (Sec. 2.3.1), two-site sweeps,
// canonicalisation and <S^2> (Eq. Sfac).
//
// The Davidson iteration keeps a Euclidean-orthonormal basis V (classical Gram-Schmidt
// applied twice) with its images HV = H_eff V and NV = N_eff V; the Ritz problem h c = theta n c
// (h = V^T HV, n = V^T NV) is solved on the device by canonical orthogonalisation of n
// (directions with eigenvalue below 1e-12 of the largest are dropped: N_eff is singular, its
// kernel lies in the kernel of H_eff when the quadrature is exact), the lowest Ritz value is
// taken, and the correction is t = -r / (diag H - theta diag N) (clamped) or a few conjugate-
// gradient steps on N_eff t = r.  The host only reads scalars (theta, |r|) to steer the loop.
//
// The decimation forms the reduced density matrix of each middle label (n, 2m), X X^T for a
// left-to-right step or X^T X for a right-to-left step, diagonalises all of them with one
// batched Jacobi launch, keeps the D largest singular values with a deterministic order of
// ties, and writes the new site tensors with grouped GEMMs: U and U^T X, or X V and V^T.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <vector>

#include "engine.h"
#include "metric.h"

using namespace spmps;
using namespace spmps::eng;

namespace {

constexpr double kTieRtol = 1e-10;   // relative gap below which singular values are tied
// Singular values below this are dropped (|x| = 1, so the dropped weight per value is < 1e-14).
// It sits above the noise floor of density-matrix eigenvalues in FP64 (~1e-16 absolute, i.e.
// ~1e-8 in singular values), so numerically null directions are never kept.
constexpr double kDropAbs = 1e-7;
constexpr double kEpsMetric = 1e-12;
constexpr double kClamp = 1e-4;

struct DavidsonOut {
    double theta = 0.0, resid = 0.0;
    int iters = 0;
    bool converged = false;
};

int64_t x_size(spmps_t* h, int k) { return make_row_block_layout(h->bonds[k], h->bonds[k + 2], 16).size; }

// Device work buffers of the Davidson solver.
struct DavBuffers {
    DevMem V, HV, NV, hm, nm, coef, coef_prev, scal, x, hx, nx, r, t, dh, dn, Q, tmp, cg_p, cg_ap, cg_res, dot, ritz;
    MetricState metric;  // factors of the metric blocks (precond == 4)
    DevMem Vc;           // orthonormal constraint vectors (excited states, Eq. orthoB)
    int ncon = 0;
};

// t <- (1 - Vc Vc^T) t, twice (excited states: the solve stays in the range of Q)
spmps_status project_constraints(spmps_t* h, DavBuffers& B, int64_t n, double* t) {
    for (int pass = 0; pass < 2 && B.ncon > 0; ++pass) {
        CK(launch_multidot(B.Vc.as<double>(), n, B.ncon, t, n, B.dot.as<double>() + 32, h->partial.as<double>(),
                           h->stream));
        CK(launch_gemv(B.Vc.as<double>(), n, B.ncon, B.dot.as<double>() + 32, n, t, 1, h->stream));
        h->launches += 3;
    }
    return SPMPS_OK;
}

spmps_status ensure_dav(spmps_t* h, DavBuffers& B, int64_t n, int ms) {
    const size_t v = static_cast<size_t>(std::max<int64_t>(n, 1)) * sizeof(double);
    CK(B.V.ensure(v * ms));
    CK(B.HV.ensure(v * ms));
    CK(B.NV.ensure(v * ms));
    CK(B.tmp.ensure(v * 2));
    for (DevMem* m : {&B.x, &B.hx, &B.nx, &B.r, &B.t, &B.dh, &B.dn, &B.cg_p, &B.cg_ap, &B.cg_res}) CK(m->ensure(v));
    CK(B.hm.ensure(sizeof(double) * ms * ms));
    CK(B.nm.ensure(sizeof(double) * ms * ms));
    CK(B.coef.ensure(sizeof(double) * 64));
    CK(B.coef_prev.ensure(sizeof(double) * 64));
    CK(B.Q.ensure(sizeof(double) * 64 * 2));
    CK(B.scal.ensure(sizeof(double) * 16));
    CK(B.dot.ensure(sizeof(double) * 64));
    CK(B.ritz.ensure(sizeof(RitzState)));
    return SPMPS_OK;
}

// Subspace matrix columns for basis column j: h[j*ms + i] = V_i . HV_j (i <= j), same for n.
spmps_status subspace_column(spmps_t* h, DavBuffers& B, int64_t n, int ms, int j) {
    double* V = B.V.as<double>();
    CK(launch_multidot(V, n, j + 1, B.HV.as<double>() + j * n, n, B.hm.as<double>() + j * ms, h->partial.as<double>(),
                       h->stream));
    CK(launch_multidot(V, n, j + 1, B.NV.as<double>() + j * n, n, B.nm.as<double>() + j * ms, h->partial.as<double>(),
                       h->stream));
    h->launches += 4;
    return SPMPS_OK;
}

spmps_status apply_column(spmps_t* h, int k, DavBuffers& B, int64_t n, int j) {
    return do_apply(h, k, B.V.as<double>() + j * n, B.HV.as<double>() + j * n, B.NV.as<double>() + j * n, h->stream);
}

// t <- t - V (V^T t), twice; returns |t|^2 (host)
spmps_status orthogonalise(spmps_t* h, DavBuffers& B, int64_t n, int m, double* t, double* nrm2) {
    for (int pass = 0; pass < 2; ++pass) {
        CK(launch_multidot(B.V.as<double>(), n, m, t, n, B.dot.as<double>(), h->partial.as<double>(), h->stream));
        CK(launch_gemv(B.V.as<double>(), n, m, B.dot.as<double>(), n, t, 1, h->stream));
        h->launches += 3;
    }
    CK(launch_norm2(t, n, B.scal.as<double>() + 3, h->partial.as<double>(), h->stream));
    h->launches += 2;
    CK(cudaMemcpyAsync(nrm2, B.scal.as<double>() + 3, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SPMPS_OK;
}

// t = approximately N_eff^+ r by cg_steps conjugate-gradient steps from t = 0.
spmps_status metric_cg(spmps_t* h, int k, DavBuffers& B, int64_t n, const double* r, double* t) {
    double* p = B.cg_p.as<double>();
    double* ap = B.cg_ap.as<double>();
    double* res = B.cg_res.as<double>();
    double* sc = B.scal.as<double>();  // sc[8] = rr, sc[9] = pAp, sc[10] = rr_new
    CK(cudaMemsetAsync(t, 0, n * sizeof(double), h->stream));
    CK(cudaMemcpyAsync(res, r, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(p, r, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(launch_norm2(res, n, sc + 8, h->partial.as<double>(), h->stream));
    for (int it = 0; it < h->opt.cg_steps; ++it) {
        spmps_status st = do_apply(h, k, p, nullptr, ap, h->stream);
        if (st != SPMPS_OK) return st;
        CK(launch_multidot(p, 0, 1, ap, n, sc + 9, h->partial.as<double>(), h->stream));
        CK(launch_axpy_ratio(t, p, n, sc + 8, sc + 9, 1.0, h->stream));
        CK(launch_axpy_ratio(res, ap, n, sc + 8, sc + 9, -1.0, h->stream));
        CK(launch_norm2(res, n, sc + 10, h->partial.as<double>(), h->stream));
        CK(launch_xpby_ratio(p, res, n, sc + 10, sc + 8, h->stream));
        CK(cudaMemcpyAsync(sc + 8, sc + 10, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->launches += 8;
    }
    return SPMPS_OK;
}

// Lowest generalised eigenpair at sites (k, k+1), starting from the device vector x0 (n).
// On return B.x holds x with x^T N x = 1.  tol_r / tol_theta / cap are this stage's criteria.
spmps_status davidson_stage(spmps_t* h, int k, const double* x0, DavBuffers& B, DavidsonOut* out, double tol_r,
                            double tol_theta, int cap, double switch_tol);

spmps_status davidson(spmps_t* h, int k, const double* x0, DavBuffers& B, DavidsonOut* out) {
    B.metric.ok = false;
    B.ncon = 0;
    if (!h->lower.empty()) {
        // excited state: the B vectors of the lower states at this step, orthonormalised (Eq. orthoB)
        spmps_status st = excited_constraints(h, k, B.Vc, &B.ncon);
        if (st != SPMPS_OK) return st;
    }
    if (h->opt.precond == 4) {
        // factors of the metric blocks for the correction (environments built first)
        Plan* P = nullptr;
        spmps_status st = get_apply_plan(h, k, &P);
        if (st != SPMPS_OK) return st;
        const int rec = h->profile ? prof_begin(h, h->stream, 6, 0.0) : -1;
        st = metric_prepare(h, k, B.metric);
        if (rec >= 0) prof_end(h, h->stream, rec);
        if (st != SPMPS_OK) return st;
    }
    spmps_status st;
    if (h->opt.precision == 0) {
        h->apply_precision = 0;
        st = davidson_stage(h, k, x0, B, out, h->opt.dav_tol_r, h->opt.dav_tol_theta, h->opt.dav_max_iter, 0.0);
    } else {
        // reduced-precision H_eff x (tensor cores) until |r| < switch_tol, then the basis products
        // are recomputed in FP64 and the same solve continues in FP64 to the final criteria
        const double switch_tol = std::max(h->opt.precision == 1 ? 1e-3 : 1e-5, h->opt.dav_tol_r);
        h->apply_precision = h->opt.precision;
        st = davidson_stage(h, k, x0, B, out, h->opt.dav_tol_r, h->opt.dav_tol_theta, h->opt.dav_max_iter,
                            switch_tol);
        h->apply_precision = 0;
    }
    if (st != SPMPS_OK || !B.metric.ok) return st;
    // x is defined modulo ker N_eff: decimate the representative (N + s)^-1 N x (on the entries of
    // the factorised blocks), which keeps the projected state and drops the (near-)null components
    // that would otherwise dominate the singular values of x
    return metric_solve(h, B.metric, B.nx.as<double>(), B.x.as<double>(), h->stream);
}

spmps_status davidson_stage(spmps_t* h, int k, const double* x0, DavBuffers& B, DavidsonOut* out, double tol_r,
                            double tol_theta, int cap, double switch_tol) {
    const int64_t n = x_size(h, k);
    const int ms = h->opt.dav_max_sub;
    spmps_status st = ensure_dav(h, B, n, ms);
    if (st != SPMPS_OK) return st;
    Plan* P = nullptr;
    st = get_apply_plan(h, k, &P);
    if (st != SPMPS_OK) return st;
    // diagonal of H_eff and N_eff for the preconditioner
    {
        Slots S{};
        S.p[5] = h->Lenv[k].buf.as<double>();
        S.p[6] = h->Renv[k + 2].buf.as<double>();
        CK(launch_diag_f64(S, P->d_diag_blocks.as<DiagBlock>(), P->d_diag_terms.as<DiagTerm>(),
                           static_cast<int>(P->diag_blocks.size()), B.dh.as<double>(), B.dn.as<double>(), h->stream));
        ++h->launches;
    }
    double* V = B.V.as<double>();
    double* sc = B.scal.as<double>();
    CK(cudaMemcpyAsync(V, x0, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    st = project_constraints(h, B, n, V);
    if (st != SPMPS_OK) return st;
    CK(launch_norm2(V, n, sc + 3, h->partial.as<double>(), h->stream));
    CK(launch_scale_inv_sqrt(V, n, sc + 3, h->stream));
    h->launches += 3;
    st = apply_column(h, k, B, n, 0);
    if (st != SPMPS_OK) return st;
    st = subspace_column(h, B, n, ms, 0);
    if (st != SPMPS_OK) return st;
    int m = 1;
    int reset = 1;  // rebuild the incremental Ritz state from the stored columns
    double theta_prev = INFINITY;
    bool switched = !(switch_tol > 0.0);  // FP64 action from here on
    int switch_it = 0;
    // the reduced-precision action has a noise floor: switch also when |r| has not improved on its
    // best value by 10 % for kStagnation iterations
    constexpr int kStagnation = 12;
    double best_rn = INFINITY;
    int best_it = 0;
    // recompute H V and N V of the stored basis in FP64 and rebuild the subspace matrices
    auto switch_to_fp64 = [&](int it_now) -> spmps_status {
        h->apply_precision = 0;
        for (int j2 = 0; j2 < m; ++j2) {
            spmps_status s2 = apply_column(h, k, B, n, j2);
            if (s2 != SPMPS_OK) return s2;
            s2 = subspace_column(h, B, n, ms, j2);
            if (s2 != SPMPS_OK) return s2;
        }
        switched = true;
        switch_it = it_now;
        reset = 1;
        theta_prev = INFINITY;
        return SPMPS_OK;
    };
    // harvesting of (features, error direction) pairs for the learned correction
    MlpState& ML = h->mlp;
    const bool harvest = ML.harvest && ML.count < ML.capacity;
    const int hs = harvest ? static_cast<int>(std::min<int64_t>(ML.samples, n)) : 0;
    int stored = 0;
    if (harvest) {
        std::vector<int64_t> idx(hs);
        for (int q = 0; q < hs; ++q) idx[q] = (static_cast<int64_t>(q) * n) / hs;
        CK(upload(ML.h_idx, idx, h->stream));
        CK(ML.h_feat.ensure(static_cast<size_t>(ML.max_iters) * hs * mlp::N_FEATURES * sizeof(float)));
        CK(ML.h_x.ensure(static_cast<size_t>(ML.max_iters) * n * sizeof(double)));
        CK(ML.h_norm.ensure(64 * sizeof(double)));
        CK(ML.h_dots.ensure(64 * sizeof(double)));
    }
    const bool learned = h->opt.precond == 2 && ML.ready;
    if (learned) CK(ML.err.ensure(sizeof(int)));
    // the learned correction is used until |r| stops improving by 10 % for kStagnation iterations;
    // the solve then continues with the diagonal correction
    bool learned_on = learned;
    auto finish_harvest = [&]() -> spmps_status {
        if (!harvest || stored == 0) return SPMPS_OK;
        const int64_t room = ML.capacity - ML.count;
        const int use = static_cast<int>(std::min<int64_t>(stored, room / std::max(hs, 1)));
        if (use <= 0) return SPMPS_OK;
        CK(launch_multidot(ML.h_x.as<double>(), n, use, B.x.as<double>(), n, ML.h_dots.as<double>(),
                           h->partial.as<double>(), h->stream));
        CK(launch_norm2(B.x.as<double>(), n, ML.h_dots.as<double>() + 32, h->partial.as<double>(), h->stream));
        CK(mlp::targets(ML.h_x.as<double>(), B.x.as<double>(), ML.h_dots.as<double>(), ML.h_norm.as<double>(),
                        ML.h_dots.as<double>() + 32, ML.h_idx.as<int64_t>(), hs, use, n,
                        ML.data_t.as<float>() + ML.count, h->stream));
        CK(cudaMemcpyAsync(ML.data_x.as<float>() + ML.count * mlp::N_FEATURES, ML.h_feat.p,
                           static_cast<size_t>(use) * hs * mlp::N_FEATURES * sizeof(float), cudaMemcpyDeviceToDevice,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->launches += 5;
        ML.count += static_cast<int64_t>(use) * hs;
        return SPMPS_OK;
    };
    double host[4];
    out->converged = false;
    for (int it = 1; it <= cap; ++it) {
        int rec = h->profile ? prof_begin(h, h->stream, 2, 0.0) : -1;
        // with a reduced-precision H the relation ker N_eff in ker H_eff holds only to that precision:
        // directions of small N-norm would carry spurious Ritz values of order eps |H| / nu, so the
        // metric range kept before the switch to FP64 is cut well above that error
        const double eps_metric = switched ? kEpsMetric : (h->apply_precision == 1 ? 1e-2 : 1e-6);
        CK(launch_ritz_inc(B.hm.as<double>(), B.nm.as<double>(), ms, m, reset, eps_metric, B.ritz.as<RitzState>(),
                           B.coef.as<double>(), sc, h->stream));
        if (rec >= 0) prof_end(h, h->stream, rec);
        reset = 0;
        rec = h->profile ? prof_begin(h, h->stream, 3, 0.0) : -1;
        CK(launch_gemv(V, n, m, B.coef.as<double>(), n, B.x.as<double>(), 0, h->stream));
        CK(launch_gemv(B.HV.as<double>(), n, m, B.coef.as<double>(), n, B.hx.as<double>(), 0, h->stream));
        CK(launch_gemv(B.NV.as<double>(), n, m, B.coef.as<double>(), n, B.nx.as<double>(), 0, h->stream));
        CK(launch_residual_diag(B.hx.as<double>(), B.nx.as<double>(), B.dh.as<double>(), B.dn.as<double>(), sc, kClamp,
                                n, B.r.as<double>(), B.t.as<double>(), sc + 2, h->partial.as<double>(), h->stream));
        h->launches += 7;
        if (B.ncon > 0) {
            // the residual within the range of Q, its norm and the diagonal correction of it
            st = project_constraints(h, B, n, B.r.as<double>());
            if (st != SPMPS_OK) return st;
            CK(launch_norm2(B.r.as<double>(), n, sc + 2, h->partial.as<double>(), h->stream));
            CK(launch_precond_apply(B.r.as<double>(), B.dh.as<double>(), B.dn.as<double>(), sc, kClamp, n,
                                    B.t.as<double>(), h->stream));
            h->launches += 3;
        }
        if (rec >= 0) prof_end(h, h->stream, rec);
        if (h->opt.precond == 1) {
            st = metric_cg(h, k, B, n, B.r.as<double>(), B.t.as<double>());
            if (st != SPMPS_OK) return st;
        } else if (B.metric.ok) {
            // t = (N_eff + s I)^-1 r through the factors of the metric blocks
            const int mrec = h->profile ? prof_begin(h, h->stream, 7, 0.0) : -1;
            st = metric_solve(h, B.metric, B.r.as<double>(), B.t.as<double>(), h->stream);
            if (mrec >= 0) prof_end(h, h->stream, mrec);
            if (st != SPMPS_OK) return st;
        } else if (h->opt.precond == 3) {
            // Olsen: t = M^-1 (-r + eps N x), eps such that x^T N t = 0, M = diag H - theta diag N:
            // t = t_diag + eps u, u = M^-1 N x, eps = -(Nx . t_diag) / (Nx . u)
            CK(launch_precond_apply(B.nx.as<double>(), B.dh.as<double>(), B.dn.as<double>(), sc, kClamp, n,
                                    B.cg_ap.as<double>(), h->stream));
            CK(launch_multidot(B.nx.as<double>(), 0, 1, B.t.as<double>(), n, sc + 11, h->partial.as<double>(), h->stream));
            CK(launch_multidot(B.nx.as<double>(), 0, 1, B.cg_ap.as<double>(), n, sc + 12, h->partial.as<double>(),
                               h->stream));
            CK(launch_axpy_ratio(B.t.as<double>(), B.cg_ap.as<double>(), n, sc + 11, sc + 12, -1.0, h->stream));
            h->launches += 6;
        }
        if (harvest || learned_on) {
            // |d|^2 of the diagonal correction (sc[7]) for the features
            CK(launch_norm2(B.t.as<double>(), n, sc + 7, h->partial.as<double>(), h->stream));
            h->launches += 2;
        }
        if (harvest && stored < ML.max_iters) {
            CK(mlp::features(B.r.as<double>(), B.t.as<double>(), B.dh.as<double>(), B.dn.as<double>(), sc, sc + 2,
                             sc + 7, n, ML.h_idx.as<int64_t>(), hs,
                             ML.h_feat.as<float>() + static_cast<size_t>(stored) * hs * mlp::N_FEATURES, h->stream));
            CK(cudaMemcpyAsync(ML.h_x.as<double>() + static_cast<int64_t>(stored) * n, B.x.p, n * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->stream));
            CK(launch_norm2(B.x.as<double>(), n, ML.h_norm.as<double>() + stored, h->partial.as<double>(), h->stream));
            h->launches += 3;
            ++stored;
        }
        const double* tsrc = B.t.as<double>();  // the correction to append: diagonal, CG, or learned
        if (learned_on) {
            CK(cudaMemsetAsync(ML.err.p, 0, sizeof(int), h->stream));
            CK(mlp::infer_tc(B.r.as<double>(), B.t.as<double>(), B.dh.as<double>(), B.dn.as<double>(), sc, sc + 2,
                             sc + 7, n, ML.w2core.as<__nv_bfloat16>(), ML.params.as<float>(), B.cg_p.as<double>(),
                             ML.err.as<int>(), h->stream, h->opt.tc_wait_polls));
            ++h->launches;
            tsrc = B.cg_p.as<double>();
        }
        rec = h->profile ? prof_begin(h, h->stream, 3, 0.0) : -1;
        if (m == ms) {
            // thick restart on [x, previous x]; a second column that is (nearly) parallel to the
            // first comes back as zero and is dropped by the n-orthonormalisation
            CK(launch_restart_coef(B.coef.as<double>(), B.coef_prev.as<double>(), m, B.Q.as<double>(), sc + 4, h->stream));
            for (DevMem* buf : {&B.V, &B.HV, &B.NV}) {
                CK(launch_basis_rotate(buf->as<double>(), n, m, B.Q.as<double>(), m, 2, n, B.tmp.as<double>(), h->stream));
                CK(cudaMemcpyAsync(buf->as<double>(), B.tmp.as<double>(), 2 * n * sizeof(double), cudaMemcpyDeviceToDevice,
                                   h->stream));
                h->launches += 1;
            }
            m = 2;
            for (int j2 = 0; j2 < m; ++j2) {
                st = subspace_column(h, B, n, ms, j2);
                if (st != SPMPS_OK) return st;
            }
            reset = 1;
            // coefficients of the current Ritz vector in the rotated basis: (scal[5], scal[6], 0, ...)
            CK(cudaMemsetAsync(B.coef_prev.p, 0, 64 * sizeof(double), h->stream));
            CK(cudaMemcpyAsync(B.coef_prev.p, sc + 5, 2 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        } else {
            CK(cudaMemsetAsync(B.coef_prev.p, 0, 64 * sizeof(double), h->stream));
            CK(cudaMemcpyAsync(B.coef_prev.p, B.coef.p, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        }
        // new direction into column m: t orthogonalised twice against V, normalised
        double* tcol = V + static_cast<int64_t>(m) * n;
        CK(cudaMemcpyAsync(tcol, tsrc, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        st = project_constraints(h, B, n, tcol);
        if (st != SPMPS_OK) return st;
        for (int pass = 0; pass < 2; ++pass) {
            CK(launch_multidot(V, n, m, tcol, n, B.dot.as<double>(), h->partial.as<double>(), h->stream));
            CK(launch_gemv(V, n, m, B.dot.as<double>(), n, tcol, 1, h->stream));
            h->launches += 3;
        }
        CK(launch_norm2(tcol, n, sc + 3, h->partial.as<double>(), h->stream));
        CK(launch_scale_inv_sqrt(tcol, n, sc + 3, h->stream));
        h->launches += 3;
        if (rec >= 0) prof_end(h, h->stream, rec);
        // one host read per iteration: theta, kept metric directions, |r|^2, |t|^2
        CK(cudaMemcpyAsync(host, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        int infer_err = 0, tc_err = 0;
        const bool inferred = learned_on;  // whether this iteration's correction came from the network
        if (inferred) CK(cudaMemcpyAsync(&infer_err, ML.err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        if (h->tc_err.p) CK(cudaMemcpyAsync(&tc_err, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        ++h->dav_iters;
        if (infer_err) return fail(h, SPMPS_ERR_TIMEOUT, "learned correction: a bounded tensor-core wait gave up");
        if (tc_err) {
            // clear the status word so that the handle stays usable after reporting
            cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), h->stream);
            cudaStreamSynchronize(h->stream);
            return fail(h, SPMPS_ERR_TIMEOUT, "tensor-core block GEMM: a bounded wait gave up");
        }
        if (host[1] < 0.5) return fail(h, SPMPS_ERR_SINGULAR_METRIC, "projected metric has no usable direction");
        if (!std::isfinite(host[0]) || !std::isfinite(host[2])) return fail(h, SPMPS_ERR_NAN, "non-finite Ritz value");
        const double theta = host[0], rn = std::sqrt(std::max(host[2], 0.0));
        out->theta = theta;
        out->resid = rn;
        out->iters = it;
        if (switched && rn < tol_r && std::fabs(theta - theta_prev) < tol_theta) {
            out->converged = true;
            h->refine_iters += switch_it > 0 ? it - switch_it : 0;
            return finish_harvest();
        }
        theta_prev = theta;
        if (rn < 0.9 * best_rn) {
            best_rn = rn;
            best_it = it;
        }
        // plain TF32 (precision 1) has a noise floor near its switch tolerance: switch on stagnation
        // too; 3xTF32 reaches its tolerance well above its floor
        const bool stagnated = h->apply_precision == 1 && it - best_it >= kStagnation;
        if (learned_on && it - best_it >= kStagnation) learned_on = false;
        // and every solve finishes in FP64: switch at half the iteration cap at the latest
        // the error of the reduced-precision products grows with the scale of H: the switch level
        // is relative to |theta| (about 1e-6 for 3xTF32 and 1e-3 for TF32) where that is above
        // the absolute one
        const double switch_at = std::max(switch_tol, (h->apply_precision == 1 ? 1e-3 : 1e-6) * std::fabs(theta));
        if (!switched && (rn < switch_at || stagnated || it >= cap / 2)) {
            // the new direction (column m) is applied in FP64 below
            st = switch_to_fp64(it);
            if (st != SPMPS_OK) return st;
        }
        if (!(host[3] > 1e-28)) {
            // the correction lies in the basis: fall back to the diagonal correction (after a
            // learned one), then to the residual itself
            double nrm2 = 0.0;
            if (inferred) {
                CK(cudaMemcpyAsync(tcol, B.t.as<double>(), n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
                st = orthogonalise(h, B, n, m, tcol, &nrm2);
                if (st != SPMPS_OK) return st;
            }
            if (!(nrm2 > 1e-28)) {
                CK(cudaMemcpyAsync(tcol, B.r.as<double>(), n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
                st = orthogonalise(h, B, n, m, tcol, &nrm2);
                if (st != SPMPS_OK) return st;
            }
            if (!(nrm2 > 1e-28)) {
                // the basis spans the reachable space: finish in FP64
                if (!switched) {
                    st = switch_to_fp64(it);
                    if (st != SPMPS_OK) return st;
                    continue;
                }
                h->refine_iters += switch_it > 0 ? it - switch_it : 0;
                return finish_harvest();
            }
            CK(launch_scale_inv_sqrt(tcol, n, sc + 3, h->stream));
            ++h->launches;
        }
        st = apply_column(h, k, B, n, m);
        if (st != SPMPS_OK) return st;
        st = subspace_column(h, B, n, ms, m);
        if (st != SPMPS_OK) return st;
        ++m;
    }
    h->refine_iters += switch_it > 0 ? cap - switch_it : 0;
    return finish_harvest();
}

// ---- decimation ------------------------------------------------------------------------------

struct MidLabel {
    int n, tm;
    std::vector<std::pair<int, int>> rows;  // (left label, s1) contributing rows, in order
    std::vector<std::pair<int, int>> cols;  // (s2, right label) contributing columns, in order
    std::vector<int> row_start, col_start;
    int nr = 0, nc = 0;
    int64_t mat_off = 0, val_off = 0;
    int dim = 0;  // matrix dimension (nr for left-to-right, nc for right-to-left)
};

struct DecBuffers {
    DevMem mats, vscr, evals, mat_off, val_off, dims, ln, ltm, keep, keep_total, disc, status, sidx, sval;
    DevMem tasks, segs, tiles, cmaps, copies, newA0, newA1;
};

// Decimate the two-site tensor x (row-block layout at sites (k, k+1), device) into new site
// tensors k and k+1 with at most Dmax states on the middle bond; move_right selects the
// canonical side (left-canonical A[k] when true, right-canonical A[k+1] otherwise).
spmps_status decimate(spmps_t* h, int k, double* x, int Dmax, bool move_right, DecBuffers& B, double* discarded) {
    const Bond& bl = h->bonds[k];
    const Bond& br = h->bonds[k + 2];
    const RowBlockLayout xl = make_row_block_layout(bl, br, 16);
    const int64_t n = xl.size;
    // unit norm
    CK(h->partial.ensure(kPartialDoubles * sizeof(double)));
    DevMem nrm;
    CK(nrm.ensure(2 * sizeof(double)));
    CK(launch_norm2(x, n, nrm.as<double>(), h->partial.as<double>(), h->stream));
    CK(launch_scale_inv_sqrt(x, n, nrm.as<double>(), h->stream));
    h->launches += 3;
    // middle labels: (n, 2m) of a + s1 for which some right label completes
    std::map<std::pair<int, int>, MidLabel> mids;
    for (size_t la = 0; la < bl.labels.size(); ++la)
        for (int s1 = 0; s1 < 4; ++s1) {
            const int mn = bl.labels[la].n + kLocalN[s1], mt = bl.labels[la].tm + kLocal2M[s1];
            bool any = false;
            for (int s2 = 0; s2 < 4 && !any; ++s2) any = xl.seg_label[la * 16 + s1 * 4 + s2] >= 0;
            if (!any) continue;
            MidLabel& M = mids[{mn, mt}];
            M.n = mn;
            M.tm = mt;
            M.rows.push_back({static_cast<int>(la), s1});
        }
    for (auto& kv : mids) {
        MidLabel& M = kv.second;
        for (int s2 = 0; s2 < 4; ++s2) {
            const int lb = br.find(M.n + kLocalN[s2], M.tm + kLocal2M[s2]);
            if (lb >= 0) M.cols.push_back({s2, lb});
        }
        int acc = 0;
        for (auto& rw : M.rows) { M.row_start.push_back(acc); acc += bl.labels[rw.first].dim; }
        M.nr = acc;
        acc = 0;
        for (auto& cl : M.cols) { M.col_start.push_back(acc); acc += br.labels[cl.second].dim; }
        M.nc = acc;
        M.dim = move_right ? M.nr : M.nc;
    }
    std::vector<MidLabel*> list;
    for (auto& kv : mids)
        if (kv.second.nr > 0 && kv.second.nc > 0) list.push_back(&kv.second);
    int64_t moff = 0, voff = 0;
    int maxdim = 0, total = 0;
    for (MidLabel* M : list) {
        M->mat_off = moff;
        M->val_off = voff;
        moff += static_cast<int64_t>(M->dim) * M->dim;
        voff += M->dim;
        maxdim = std::max(maxdim, M->dim);
        total += M->dim;
    }
    if (maxdim > 512) return fail(h, SPMPS_ERR_UNSUPPORTED, "decimation block larger than 512");
    // density matrices by grouped GEMMs: slot 0 = x, slot 1 = mats
    GemmPlan G;
    auto xblock = [&](int la, int s) { return xl.row_off[la] + xl.seg_col[la * 16 + s]; };
    for (MidLabel* M : list) {
        if (move_right) {
            for (size_t i = 0; i < M->rows.size(); ++i)
                for (size_t j = 0; j < M->rows.size(); ++j) {
                    const int la = M->rows[i].first, s1 = M->rows[i].second;
                    const int la2 = M->rows[j].first, s1b = M->rows[j].second;
                    GemmTask T{};
                    T.c = handle(1, M->mat_off + static_cast<int64_t>(M->row_start[i]) * M->dim + M->row_start[j]);
                    T.cmap = -1;
                    T.M = bl.labels[la].dim;
                    T.N = bl.labels[la2].dim;
                    T.ldc = M->dim;
                    T.seg0 = static_cast<int>(G.segs.size());
                    for (size_t c = 0; c < M->cols.size(); ++c) {
                        const int s2 = M->cols[c].first;
                        const int sa = s1 * 4 + s2, sb = s1b * 4 + s2;
                        if (xl.seg_label[la * 16 + sa] < 0 || xl.seg_label[la2 * 16 + sb] < 0) continue;
                        GemmSeg sg{};
                        sg.a = handle(0, xblock(la, sa));
                        sg.a_rs = xl.width[la];
                        sg.a_cs = 1;
                        sg.K = br.labels[M->cols[c].second].dim;
                        sg.b = handle(0, xblock(la2, sb));
                        sg.b_rs = 1;
                        sg.b_cs = xl.width[la2];
                                                G.segs.push_back(sg);
                    }
                    T.nseg = static_cast<int>(G.segs.size()) - T.seg0;
                    G.tasks.push_back(T);
                }
        } else {
            for (size_t i = 0; i < M->cols.size(); ++i)
                for (size_t j = 0; j < M->cols.size(); ++j) {
                    const int s2 = M->cols[i].first, lb = M->cols[i].second;
                    const int s2b = M->cols[j].first, lb2 = M->cols[j].second;
                    GemmTask T{};
                    T.c = handle(1, M->mat_off + static_cast<int64_t>(M->col_start[i]) * M->dim + M->col_start[j]);
                    T.cmap = -1;
                    T.M = br.labels[lb].dim;
                    T.N = br.labels[lb2].dim;
                    T.ldc = M->dim;
                    T.seg0 = static_cast<int>(G.segs.size());
                    for (size_t r = 0; r < M->rows.size(); ++r) {
                        const int la = M->rows[r].first, s1 = M->rows[r].second;
                        const int sa = s1 * 4 + s2, sb = s1 * 4 + s2b;
                        if (xl.seg_label[la * 16 + sa] < 0 || xl.seg_label[la * 16 + sb] < 0) continue;
                        GemmSeg sg{};
                        sg.a = handle(0, xblock(la, sa));
                        sg.a_rs = 1;
                        sg.a_cs = xl.width[la];
                        sg.K = bl.labels[la].dim;
                        sg.b = handle(0, xblock(la, sb));
                        sg.b_rs = xl.width[la];
                        sg.b_cs = 1;
                                                G.segs.push_back(sg);
                    }
                    T.nseg = static_cast<int>(G.segs.size()) - T.seg0;
                    G.tasks.push_back(T);
                }
        }
    }
    G.add_tiles();
    {
        int64_t sz[kMaxSlots];
        for (auto& v : sz) v = -1;
        sz[0] = n;
        sz[1] = moff;
        std::string why;
        if (!validate_gemm(G, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (density matrix): " + why);
    }
    CK(B.mats.ensure(std::max<int64_t>(moff, 1) * sizeof(double)));
    CK(B.vscr.ensure(std::max<int64_t>(moff, 1) * sizeof(double)));
    CK(B.evals.ensure(std::max<int64_t>(voff, 1) * sizeof(double)));
    CK(upload(B.tasks, G.tasks, h->stream));
    CK(upload(B.segs, G.segs, h->stream));
    CK(upload(B.tiles, G.tiles, h->stream));
    CK(upload(B.cmaps, G.cmaps, h->stream));
    Slots S{};
    S.p[0] = x;
    S.p[1] = B.mats.as<double>();
    {
        double fl = 0.0;
        for (const GemmTask& T : G.tasks)
            for (int q = 0; q < T.nseg; ++q) fl += 2.0 * T.M * T.N * G.segs[T.seg0 + q].K;
        const int rec = h->profile ? prof_begin(h, h->stream, 0, fl) : -1;
        CK(launch_gemm_f64(S, B.tasks.as<GemmTask>(), B.segs.as<GemmSeg>(), B.tiles.as<GemmTile>(), B.cmaps.as<int>(),
                           static_cast<int>(G.tiles.size()), h->stream));
        if (rec >= 0) prof_end(h, h->stream, rec);
    }
    ++h->launches;
    // batched Jacobi and ordered truncation
    std::vector<int64_t> mo, vo;
    std::vector<int> dims, lns, ltms;
    for (MidLabel* M : list) {
        mo.push_back(M->mat_off);
        vo.push_back(M->val_off);
        dims.push_back(M->dim);
        lns.push_back(M->n);
        ltms.push_back(M->tm);
    }
    const int nm = static_cast<int>(list.size());
    CK(upload(B.mat_off, mo, h->stream));
    CK(upload(B.val_off, vo, h->stream));
    CK(upload(B.dims, dims, h->stream));
    CK(upload(B.ln, lns, h->stream));
    CK(upload(B.ltm, ltms, h->stream));
    CK(B.keep.ensure(std::max(nm, 1) * sizeof(int)));
    CK(B.keep_total.ensure(sizeof(int)));
    CK(B.disc.ensure(sizeof(double)));
    CK(B.status.ensure(sizeof(int)));
    CK(B.sidx.ensure(std::max(3 * total, 1) * sizeof(int)));
    CK(B.sval.ensure(std::max(2 * total, 1) * sizeof(double)));
    CK(cudaMemsetAsync(B.status.p, 0, sizeof(int), h->stream));
    const int rec_eig = h->profile ? prof_begin(h, h->stream, 4, 0.0) : -1;
    CK(launch_jacobi_batched(B.mats.as<double>(), B.vscr.as<double>(), B.evals.as<double>(), B.mat_off.as<int64_t>(),
                             B.val_off.as<int64_t>(), B.dims.as<int>(), nm, maxdim, h->opt.jacobi_smem_max, 1,
                             B.status.as<int>(), h->stream));
    CK(launch_truncate(B.evals.as<double>(), B.val_off.as<int64_t>(), B.dims.as<int>(), B.ln.as<int>(), B.ltm.as<int>(),
                       nm, total, Dmax, kTieRtol, kDropAbs, B.keep.as<int>(), B.keep_total.as<int>(), B.disc.as<double>(),
                       B.sidx.as<int>(), B.sval.as<double>(), h->stream));
    if (rec_eig >= 0) prof_end(h, h->stream, rec_eig);
    h->launches += 2;
    std::vector<int> keep(std::max(nm, 1));
    int jac_status = 0;
    double disc = 0.0;
    CK(cudaMemcpyAsync(keep.data(), B.keep.p, std::max(nm, 1) * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&jac_status, B.status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&disc, B.disc.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (discarded) *discarded = disc;
    // new middle bond
    Bond nb;
    for (int i = 0; i < nm; ++i)
        if (keep[i] > 0) nb.labels.push_back(Label{list[i]->n, list[i]->tm, keep[i], 0, 0});
    if (nb.labels.empty()) return fail(h, SPMPS_ERR_NAN, "decimation kept no state");
    nb.finalize();
    const RowBlockLayout a0 = make_row_block_layout(bl, nb, 4);
    const RowBlockLayout a1 = make_row_block_layout(nb, br, 4);
    // new tensors: slot 0 = x, 1 = mats (vectors), 2 = new A[k], 3 = new A[k+1]
    GemmPlan W;
    std::vector<CopyBlock> copies;
    for (int i = 0; i < nm; ++i) {
        const MidLabel& M = *list[i];
        const int kc = keep[i];
        if (kc == 0) continue;
        const int lc = nb.find(M.n, M.tm);
        if (move_right) {
            // A[k][la][:, seg(s1)] = U[rows(la, s1), :kc]
            for (size_t r = 0; r < M.rows.size(); ++r) {
                const int la = M.rows[r].first, s1 = M.rows[r].second;
                if (a0.seg_label[la * 4 + s1] != lc) continue;
                CopyBlock cb{};
                cb.src = handle(1, M.mat_off + static_cast<int64_t>(M.row_start[r]) * M.dim);
                cb.ld_src = M.dim;
                cb.dst = handle(2, a0.row_off[la] + a0.seg_col[la * 4 + s1]);
                cb.ld_dst = a0.width[la];
                cb.rows = bl.labels[la].dim;
                cb.cols = kc;
                cb.transpose = 0;
                copies.push_back(cb);
            }
            // A[k+1][lc][:, seg(s2)] = sum_(la,s1) U[rows(la,s1), :kc]^T X[la, (s1, s2)]
            for (size_t c = 0; c < M.cols.size(); ++c) {
                const int s2 = M.cols[c].first, lb = M.cols[c].second;
                if (a1.seg_label[lc * 4 + s2] != lb) continue;
                GemmTask T{};
                T.c = handle(3, a1.row_off[lc] + a1.seg_col[lc * 4 + s2]);
                T.cmap = -1;
                T.M = kc;
                T.N = br.labels[lb].dim;
                T.ldc = a1.width[lc];
                T.seg0 = static_cast<int>(W.segs.size());
                for (size_t r = 0; r < M.rows.size(); ++r) {
                    const int la = M.rows[r].first, s1 = M.rows[r].second;
                    const int s = s1 * 4 + s2;
                    if (xl.seg_label[la * 16 + s] != lb) continue;
                    GemmSeg sg{};
                    sg.a = handle(1, M.mat_off + static_cast<int64_t>(M.row_start[r]) * M.dim);
                    sg.a_rs = 1;
                    sg.a_cs = M.dim;
                    sg.K = bl.labels[la].dim;
                    sg.b = handle(0, xblock(la, s));
                    sg.b_rs = xl.width[la];
                    sg.b_cs = 1;
                                        W.segs.push_back(sg);
                }
                T.nseg = static_cast<int>(W.segs.size()) - T.seg0;
                W.tasks.push_back(T);
            }
        } else {
            // A[k+1][lc][:, seg(s2)] = V[rows(s2, lb), :kc]^T
            for (size_t c = 0; c < M.cols.size(); ++c) {
                const int s2 = M.cols[c].first, lb = M.cols[c].second;
                if (a1.seg_label[lc * 4 + s2] != lb) continue;
                CopyBlock cb{};
                cb.src = handle(1, M.mat_off + static_cast<int64_t>(M.col_start[c]) * M.dim);
                cb.ld_src = M.dim;
                cb.dst = handle(3, a1.row_off[lc] + a1.seg_col[lc * 4 + s2]);
                cb.ld_dst = a1.width[lc];
                cb.rows = kc;
                cb.cols = br.labels[lb].dim;
                cb.transpose = 1;
                copies.push_back(cb);
            }
            // A[k][la][:, seg(s1)] = sum_s2 X[la, (s1, s2)] V[rows(s2, lb), :kc]
            for (size_t r = 0; r < M.rows.size(); ++r) {
                const int la = M.rows[r].first, s1 = M.rows[r].second;
                if (a0.seg_label[la * 4 + s1] != lc) continue;
                GemmTask T{};
                T.c = handle(2, a0.row_off[la] + a0.seg_col[la * 4 + s1]);
                T.cmap = -1;
                T.M = bl.labels[la].dim;
                T.N = kc;
                T.ldc = a0.width[la];
                T.seg0 = static_cast<int>(W.segs.size());
                for (size_t c = 0; c < M.cols.size(); ++c) {
                    const int s2 = M.cols[c].first, lb = M.cols[c].second;
                    const int s = s1 * 4 + s2;
                    if (xl.seg_label[la * 16 + s] != lb) continue;
                    GemmSeg sg{};
                    sg.a = handle(0, xblock(la, s));
                    sg.a_rs = xl.width[la];
                    sg.a_cs = 1;
                    sg.K = br.labels[lb].dim;
                    sg.b = handle(1, M.mat_off + static_cast<int64_t>(M.col_start[c]) * M.dim);
                    sg.b_rs = M.dim;
                    sg.b_cs = 1;
                                        W.segs.push_back(sg);
                }
                T.nseg = static_cast<int>(W.segs.size()) - T.seg0;
                W.tasks.push_back(T);
            }
        }
    }
    W.add_tiles();
    {
        int64_t sz[kMaxSlots];
        for (auto& v : sz) v = -1;
        sz[0] = n;
        sz[1] = moff;
        sz[2] = a0.size;
        sz[3] = a1.size;
        std::string why;
        if (!validate_gemm(W, sz, &why)) return fail(h, SPMPS_ERR_CUDA, "internal plan check (new tensors): " + why);
        for (const CopyBlock& cb : copies) {
            const int64_t last_src = cb.transpose ? static_cast<int64_t>(cb.cols - 1) * cb.ld_src + cb.rows - 1
                                                  : static_cast<int64_t>(cb.rows - 1) * cb.ld_src + cb.cols - 1;
            const int64_t last_dst = static_cast<int64_t>(cb.rows - 1) * cb.ld_dst + cb.cols - 1;
            const int ss = static_cast<int>(cb.src >> 56), ds = static_cast<int>(cb.dst >> 56);
            const int64_t so = static_cast<int64_t>(cb.src & 0x00FFFFFFFFFFFFFFull);
            const int64_t dof = static_cast<int64_t>(cb.dst & 0x00FFFFFFFFFFFFFFull);
            if (so + last_src >= sz[ss] || dof + last_dst >= sz[ds])
                return fail(h, SPMPS_ERR_CUDA, "internal plan check (copies)");
        }
    }
    auto A0 = std::make_unique<DevMem>();
    auto A1 = std::make_unique<DevMem>();
    CK(A0->ensure(std::max<int64_t>(a0.size, 1) * sizeof(double)));
    CK(A1->ensure(std::max<int64_t>(a1.size, 1) * sizeof(double)));
    CK(cudaMemsetAsync(A0->p, 0, std::max<int64_t>(a0.size, 1) * sizeof(double), h->stream));
    CK(cudaMemsetAsync(A1->p, 0, std::max<int64_t>(a1.size, 1) * sizeof(double), h->stream));
    DevMem d_tasks, d_segs, d_tiles, d_cmaps, d_copies;
    CK(upload(d_tasks, W.tasks, h->stream));
    CK(upload(d_segs, W.segs, h->stream));
    CK(upload(d_tiles, W.tiles, h->stream));
    CK(upload(d_cmaps, W.cmaps, h->stream));
    CK(upload(d_copies, copies, h->stream));
    Slots S2{};
    S2.p[0] = x;
    S2.p[1] = B.mats.as<double>();
    S2.p[2] = A0->as<double>();
    S2.p[3] = A1->as<double>();
    {
        double fl = 0.0;
        for (const GemmTask& T : W.tasks)
            for (int q = 0; q < T.nseg; ++q) fl += 2.0 * T.M * T.N * W.segs[T.seg0 + q].K;
        const int rec = h->profile ? prof_begin(h, h->stream, 0, fl) : -1;
        CK(launch_gemm_f64(S2, d_tasks.as<GemmTask>(), d_segs.as<GemmSeg>(), d_tiles.as<GemmTile>(), d_cmaps.as<int>(),
                           static_cast<int>(W.tiles.size()), h->stream));
        if (rec >= 0) prof_end(h, h->stream, rec);
    }
    CK(launch_copy_blocks(S2, d_copies.as<CopyBlock>(), static_cast<int>(copies.size()), h->stream));
    h->launches += 4;
    CK(cudaStreamSynchronize(h->stream));
    (void)jac_status;
    // install
    h->bonds[k + 1] = nb;
    h->alay[k] = a0;
    h->alay[k + 1] = a1;
    h->A[k] = std::move(A0);
    h->A[k + 1] = std::move(A1);
    for (int b = k + 1; b <= h->K; ++b) h->Lenv[b].valid = false;
    for (int b = 0; b <= k + 1; ++b) h->Renv[b].valid = false;
    for (int j = std::max(0, k - 1); j <= std::min(h->K - 2, k + 1); ++j) h->apply_plans[j].reset();
    return SPMPS_OK;
}

}  // namespace

// =============================================================================================

extern "C" {

spmps_status spmps_canonicalize(spmps_handle h) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    DecBuffers B;
    DevMem xb;
    for (int k = h->K - 2; k >= 0; --k) {
        const int64_t n = x_size(h, k);
        CK(xb.ensure(std::max<int64_t>(n, 1) * sizeof(double)));
        st = spmps_two_site(h, k, xb.as<double>());
        if (st != SPMPS_OK) return st;
        st = decimate(h, k, xb.as<double>(), h->D, false, B, nullptr);
        if (st != SPMPS_OK) return st;
    }
    invalidate_all(h);
    h->center = 0;
    return SPMPS_OK;
}

spmps_status spmps_optimize_step(spmps_handle h, int site, int move_right, double* theta, int* iterations) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (site < 0 || site > h->K - 2) return fail(h, SPMPS_ERR_BAD_INPUT, "site out of range");
    if (h->center != site && h->center != site + 1) return fail(h, SPMPS_ERR_STATE, "the centre must be in the pair");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    DavBuffers DB;
    DecBuffers EB;
    DevMem x0;
    const int64_t n = x_size(h, site);
    CK(x0.ensure(std::max<int64_t>(n, 1) * sizeof(double)));
    st = spmps_two_site(h, site, x0.as<double>());
    if (st != SPMPS_OK) return st;
    DavidsonOut out;
    st = davidson(h, site, x0.as<double>(), DB, &out);
    if (st != SPMPS_OK) return st;
    double disc = 0.0;
    st = decimate(h, site, DB.x.as<double>(), h->D, move_right != 0, EB, &disc);
    if (st != SPMPS_OK) return st;
    h->last_discarded = disc;
    if (move_right) {
        st = update_left(h, site);
        h->center = site + 1;
    } else {
        st = update_right(h, site + 1);
        h->center = site;
    }
    if (st != SPMPS_OK) return st;
    st = excited_after_step(h, site, move_right != 0);
    if (st != SPMPS_OK) return st;
    if (theta) *theta = out.theta;
    if (iterations) *iterations = out.iters;
    if (!out.converged) return fail(h, SPMPS_ERR_NOT_CONVERGED, "Davidson reached its iteration cap");
    return SPMPS_OK;
}

spmps_status spmps_sweep(spmps_handle h, int n_sweeps, double* energies) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (n_sweeps < 0) return fail(h, SPMPS_ERR_BAD_INPUT, "n_sweeps < 0");
    if (h->center != 0) return fail(h, SPMPS_ERR_STATE, "sweeps start with the centre on site 0");
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, SPMPS_ERR_CUDA, "cudaSetDevice");
    const int K = h->K;
    std::vector<std::pair<int, bool>> sched;
    for (int k = 0; k + 2 < K; ++k) sched.push_back({k, true});
    for (int k = K - 2; k >= 0; --k) sched.push_back({k, false});
    DavBuffers DB;
    DecBuffers EB;
    DevMem x0;
    bool all_converged = true;
    h->dav_iters = 0;
    h->refine_iters = 0;
    double disc_total = 0.0;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        double theta = 0.0;
        for (auto& step : sched) {
            const int k = step.first;
            const bool mr = step.second;
            st = ensure_envs(h, k);
            if (st != SPMPS_OK) return st;
            const int64_t n = x_size(h, k);
            CK(x0.ensure(std::max<int64_t>(n, 1) * sizeof(double)));
            st = spmps_two_site(h, k, x0.as<double>());
            if (st != SPMPS_OK) return st;
            DavidsonOut out;
            st = davidson(h, k, x0.as<double>(), DB, &out);
            if (st != SPMPS_OK) return st;
            all_converged = all_converged && out.converged;
            theta = out.theta;
            double disc = 0.0;
            st = decimate(h, k, DB.x.as<double>(), h->D, mr, EB, &disc);
            if (st != SPMPS_OK) return st;
            disc_total += disc;
            if (mr) {
                st = update_left(h, k);
                h->center = k + 1;
            } else {
                st = update_right(h, k + 1);
                h->center = k;
            }
            if (st != SPMPS_OK) return st;
            st = excited_after_step(h, k, mr);
            if (st != SPMPS_OK) return st;
        }
        if (energies) energies[sw] = theta;
    }
    h->last_discarded = disc_total;
    if (!all_converged) return fail(h, SPMPS_ERR_NOT_CONVERGED, "a Davidson solve reached its iteration cap");
    return SPMPS_OK;
}

spmps_status spmps_expect_s2(spmps_handle h, double* s2) {
    spmps_status st = check_ready(h);
    if (st != SPMPS_OK) return st;
    if (!s2) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL output");
    OpSet saved = std::move(h->ops);
    std::vector<EnvStore> sl = std::move(h->Lenv), sr = std::move(h->Renv);
    h->Lenv.clear();
    h->Renv.clear();
    h->Lenv.resize(h->K + 1);
    h->Renv.resize(h->K + 1);
    for (auto& p : h->apply_plans) p.reset();
    st = build_opset(h, mpo_s2(h->K), &h->ops);
    double nP = 0.0;
    if (st == SPMPS_OK) st = spmps_energy(h, s2, &nP);
    h->ops = std::move(saved);
    h->Lenv = std::move(sl);
    h->Renv = std::move(sr);
    for (auto& p : h->apply_plans) p.reset();
    return st;
}

}  // extern "C"
