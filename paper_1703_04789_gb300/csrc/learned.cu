// C ABI of the learned Davidson correction: harvesting, training, parameters, inference.
#include <cmath>
#include <vector>

#include "engine.h"

using namespace spmps;
using namespace spmps::eng;

namespace {

spmps_status ensure_params(spmps_t* h) {
    MlpState& M = h->mlp;
    CK(M.params.ensure(mlp::kParams * sizeof(float)));
    CK(M.grads.ensure(mlp::kParams * sizeof(float)));
    CK(M.m.ensure(mlp::kParams * sizeof(float)));
    CK(M.v.ensure(mlp::kParams * sizeof(float)));
    CK(M.w2core.ensure(mlp::HIDDEN * mlp::HIDDEN * sizeof(__nv_bfloat16)));
    CK(M.err.ensure(sizeof(int)));
    CK(M.loss.ensure(sizeof(double)));
    return SPMPS_OK;
}

spmps_status ensure_batch(spmps_t* h, int B) {
    MlpState& M = h->mlp;
    if (M.batch >= B) return SPMPS_OK;
    const size_t a = static_cast<size_t>(B) * mlp::HIDDEN * sizeof(float);
    CK(M.X.ensure(static_cast<size_t>(B) * mlp::N_FEATURES * sizeof(float)));
    CK(M.T.ensure(static_cast<size_t>(B) * sizeof(float)));
    for (DevMem* d : {&M.Z1, &M.H1, &M.Z2, &M.H2, &M.dZ2, &M.dZ1}) CK(d->ensure(a));
    CK(M.dy.ensure(static_cast<size_t>(B) * sizeof(float)));
    CK(M.loss_part.ensure(static_cast<size_t>((B + 255) / 256) * sizeof(double)));
    M.batch = B;
    return SPMPS_OK;
}

mlp::TrainBuffers buffers(MlpState& M) {
    mlp::TrainBuffers b{};
    b.Z1 = M.Z1.as<float>();
    b.H1 = M.H1.as<float>();
    b.Z2 = M.Z2.as<float>();
    b.H2 = M.H2.as<float>();
    b.dZ2 = M.dZ2.as<float>();
    b.dZ1 = M.dZ1.as<float>();
    b.dy = M.dy.as<float>();
    b.loss_part = M.loss_part.as<double>();
    return b;
}

// He-normal initial weights from a counter-based generator (SplitMix64 + Box-Muller).
void init_host(std::vector<float>& p, uint64_t seed) {
    p.assign(mlp::kParams, 0.0f);
    uint64_t ctr = 0;
    auto u01 = [&]() {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (++ctr);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (static_cast<double>(z >> 11) + 0.5) / 9007199254740992.0;
    };
    auto normal = [&]() { return std::sqrt(-2.0 * std::log(u01())) * std::cos(6.283185307179586 * u01()); };
    for (int i = 0; i < mlp::N_FEATURES * mlp::HIDDEN; ++i)
        p[mlp::kOffW1 + i] = static_cast<float>(normal() * std::sqrt(2.0 / mlp::N_FEATURES));
    for (int i = 0; i < mlp::HIDDEN * mlp::HIDDEN; ++i)
        p[mlp::kOffW2 + i] = static_cast<float>(normal() * std::sqrt(2.0 / mlp::HIDDEN));
    for (int i = 0; i < mlp::HIDDEN; ++i) p[mlp::kOffW3 + i] = static_cast<float>(normal() * std::sqrt(1.0 / mlp::HIDDEN));
}

}  // namespace

extern "C" {

spmps_status spmps_mlp_harvest(spmps_handle h, int enable, int samples_per_iteration, int64_t capacity) {
    if (!h) return fail(nullptr, SPMPS_ERR_BAD_INPUT, "null handle");
    if (samples_per_iteration < 1 || samples_per_iteration > 65536 || capacity < 0)
        return fail(h, SPMPS_ERR_BAD_INPUT, "samples_per_iteration in [1, 65536], capacity >= 0");
    MlpState& M = h->mlp;
    M.harvest = enable != 0;
    M.samples = samples_per_iteration;
    if (enable && capacity > M.capacity) {
        CK(M.data_x.ensure(static_cast<size_t>(capacity) * mlp::N_FEATURES * sizeof(float)));
        CK(M.data_t.ensure(static_cast<size_t>(capacity) * sizeof(float)));
        if (M.count > 0) M.count = 0;  // the buffers were reallocated
        M.capacity = capacity;
    }
    return SPMPS_OK;
}

spmps_status spmps_mlp_data(spmps_handle h, int64_t* count, float* features, float* targets) {
    if (!h || !count) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    *count = h->mlp.count;
    if (features && h->mlp.count > 0)
        CK(cudaMemcpy(features, h->mlp.data_x.p, h->mlp.count * mlp::N_FEATURES * sizeof(float), cudaMemcpyDeviceToHost));
    if (targets && h->mlp.count > 0)
        CK(cudaMemcpy(targets, h->mlp.data_t.p, h->mlp.count * sizeof(float), cudaMemcpyDeviceToHost));
    return SPMPS_OK;
}

spmps_status spmps_mlp_params(spmps_handle h, float* params, int set) {
    if (!h || !params) return fail(h, SPMPS_ERR_BAD_INPUT, "NULL argument");
    spmps_status st = ensure_params(h);
    if (st != SPMPS_OK) return st;
    MlpState& M = h->mlp;
    if (set) {
        for (int i = 0; i < mlp::kParams; ++i)
            if (!std::isfinite(params[i])) return fail(h, SPMPS_ERR_BAD_INPUT, "parameters not finite");
        CK(cudaMemcpyAsync(M.params.p, params, mlp::kParams * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(mlp::prepare_w2(M.params.as<float>(), M.w2core.as<__nv_bfloat16>(), h->stream));
        CK(cudaStreamSynchronize(h->stream));
        M.ready = true;
    } else {
        if (!M.ready) return fail(h, SPMPS_ERR_STATE, "no parameters");
        CK(cudaMemcpyAsync(params, M.params.p, mlp::kParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return SPMPS_OK;
}

spmps_status spmps_mlp_loss_grad(spmps_handle h, const float* X, const float* T, int B, double* loss, float* grads) {
    if (!h || !X || !T || B < 1) return fail(h, SPMPS_ERR_BAD_INPUT, "bad argument");
    MlpState& M = h->mlp;
    if (!M.ready) return fail(h, SPMPS_ERR_STATE, "no parameters");
    spmps_status st = ensure_batch(h, B);
    if (st != SPMPS_OK) return st;
    CK(cudaMemcpyAsync(M.X.p, X, static_cast<size_t>(B) * mlp::N_FEATURES * sizeof(float), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(M.T.p, T, static_cast<size_t>(B) * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    mlp::TrainBuffers b = buffers(M);
    CK(mlp::train_step(b, M.X.as<float>(), M.T.as<float>(), B, M.params.as<float>(), M.grads.as<float>(),
                       M.loss.as<double>(), h->stream));
    h->launches += 14;
    if (loss) CK(cudaMemcpyAsync(loss, M.loss.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (grads) CK(cudaMemcpyAsync(grads, M.grads.p, mlp::kParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SPMPS_OK;
}

spmps_status spmps_mlp_train(spmps_handle h, int steps, int batch, double lr, uint64_t seed, int reinit,
                             double* loss_first, double* loss_last) {
    if (!h || steps < 0 || batch < 1 || !(lr > 0.0)) return fail(h, SPMPS_ERR_BAD_INPUT, "bad argument");
    MlpState& M = h->mlp;
    if (M.count < 1) return fail(h, SPMPS_ERR_STATE, "no harvested data");
    spmps_status st = ensure_params(h);
    if (st != SPMPS_OK) return st;
    if (reinit || !M.ready) {
        std::vector<float> p;
        init_host(p, seed);
        CK(cudaMemcpyAsync(M.params.p, p.data(), mlp::kParams * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemsetAsync(M.m.p, 0, mlp::kParams * sizeof(float), h->stream));
        CK(cudaMemsetAsync(M.v.p, 0, mlp::kParams * sizeof(float), h->stream));
        M.step = 0;
        M.ready = true;
    }
    st = ensure_batch(h, batch);
    if (st != SPMPS_OK) return st;
    mlp::TrainBuffers b = buffers(M);
    for (int s = 0; s < steps; ++s) {
        CK(mlp::gather_batch(M.data_x.as<float>(), M.data_t.as<float>(), M.count, batch, seed,
                             static_cast<uint64_t>(M.step), M.X.as<float>(), M.T.as<float>(), h->stream));
        CK(mlp::train_step(b, M.X.as<float>(), M.T.as<float>(), batch, M.params.as<float>(), M.grads.as<float>(),
                           M.loss.as<double>(), h->stream));
        ++M.step;
        CK(mlp::adam(M.params.as<float>(), M.grads.as<float>(), M.m.as<float>(), M.v.as<float>(), M.step,
                     static_cast<float>(lr), h->stream));
        h->launches += 16;
        if (s == 0 && loss_first) {
            CK(cudaMemcpyAsync(loss_first, M.loss.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
        }
    }
    CK(mlp::prepare_w2(M.params.as<float>(), M.w2core.as<__nv_bfloat16>(), h->stream));
    if (loss_last) CK(cudaMemcpyAsync(loss_last, M.loss.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SPMPS_OK;
}

spmps_status spmps_mlp_infer(spmps_handle h, const double* r, const double* dh, const double* dn, double theta,
                             int64_t n, double* t, int tensor_cores) {
    if (!h || !r || !dh || !dn || !t || n < 1) return fail(h, SPMPS_ERR_BAD_INPUT, "bad argument");
    MlpState& M = h->mlp;
    if (!M.ready) return fail(h, SPMPS_ERR_STATE, "no parameters");
    DevMem dr, ddh, ddn, dd, dout, dsc, dX;
    const size_t nb = static_cast<size_t>(n) * sizeof(double);
    CK(dr.ensure(nb));
    CK(ddh.ensure(nb));
    CK(ddn.ensure(nb));
    CK(dd.ensure(nb));
    CK(dout.ensure(nb));
    CK(dsc.ensure(16 * sizeof(double)));
    CK(cudaMemcpyAsync(dr.p, r, nb, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(ddh.p, dh, nb, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(ddn.p, dn, nb, cudaMemcpyHostToDevice, h->stream));
    double* sc = dsc.as<double>();
    CK(cudaMemcpyAsync(sc, &theta, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(mlp::diag_correction(dr.as<double>(), ddh.as<double>(), ddn.as<double>(), sc, n, dd.as<double>(), h->stream));
    CK(launch_norm2(dr.as<double>(), n, sc + 2, h->partial.as<double>(), h->stream));
    CK(launch_norm2(dd.as<double>(), n, sc + 7, h->partial.as<double>(), h->stream));
    CK(cudaMemsetAsync(M.err.p, 0, sizeof(int), h->stream));
    if (tensor_cores) {
        CK(mlp::infer_tc(dr.as<double>(), dd.as<double>(), ddh.as<double>(), ddn.as<double>(), sc, sc + 2, sc + 7, n,
                         M.w2core.as<__nv_bfloat16>(), M.params.as<float>(), dout.as<double>(), M.err.as<int>(),
                         h->stream, h->opt.tc_wait_polls));
    } else {
        CK(dX.ensure(static_cast<size_t>(n) * mlp::N_FEATURES * sizeof(float)));
        CK(mlp::features(dr.as<double>(), dd.as<double>(), ddh.as<double>(), ddn.as<double>(), sc, sc + 2, sc + 7, n,
                         nullptr, n, dX.as<float>(), h->stream));
        CK(mlp::infer_f32(dX.as<float>(), n, M.params.as<float>(), dout.as<double>(), h->stream));
    }
    int err = 0;
    CK(cudaMemcpyAsync(t, dout.p, nb, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&err, M.err.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->launches += 5;
    if (err) return fail(h, SPMPS_ERR_TIMEOUT, "tensor-core inference: a bounded wait gave up");
    return SPMPS_OK;
}

}  // extern "C"
