// C-ABI of the boundary-MPS approximate contraction (bmps.cu): the norm, one
// expectation value, or the norm and every <X_k> and nearest-neighbour
// <Z_i Z_j> of a lattice, each network contracted by one block in a single
// launch (one contraction per observable, as Sec. 5 counts them, each
// approximated with boundary bond chi).
#include <cmath>
#include <vector>

#include "runtime.h"

namespace tn {
tn_status result_from_array(const double* r, int L, int W, tn_precision prec, const Plan& p, tn_result* out);
namespace {

// Contract the given networks; out receives (mantissa, exponent) per network.
tn_status bmps_run(tn_lattice* lat, int chi, tn_precision prec, std::vector<BmpsTask>& tasks,
                   std::vector<double>* out) {
    tn_ctx* ctx = lat->ctx;
    const int L = lat->L, W = lat->W, D = lat->D;
    if (lat->cplx) { set_error("the boundary MPS takes real site tensors"); return TN_ERR_INVALID; }
    if (prec != TN_FP64 && prec != TN_FP32) { set_error("the boundary MPS runs in FP64 or FP32"); return TN_ERR_INVALID; }
    if (chi < 1 || bmps_bond_max(D, chi) > 512) {
        set_error("chi out of range: max(chi, D^2) * D^2 must not exceed 512");
        return TN_ERR_INVALID;
    }
    if (!ctx || ctx->device < 0) { set_error("context has no device"); return TN_ERR_NO_DEVICE; }
    cudaSetDevice(ctx->device);
    const size_t nel = lat->host.size();
    const long long ws = bmps_workspace(W, D, chi);
    const size_t n = tasks.size();
    const size_t off_tasks = (nel * 8 + 255) / 256 * 256;
    const size_t off_out = off_tasks + (n * sizeof(BmpsTask) + 255) / 256 * 256;
    const size_t off_ws = off_out + (n * 2 * 8 + 255) / 256 * 256;
    const size_t total = off_ws + n * (size_t)ws * 8;
    if (ctx->used + total > ctx->budget) { set_error("boundary-MPS workspace exceeds the budget"); return TN_ERR_OVER_BUDGET; }
    char* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, total);
    if (e != cudaSuccess) return cuda_status(e, "boundary-MPS workspace");
    ctx->used += total;
    const double* dA = reinterpret_cast<const double*>(buf);
    for (size_t k = 0; k < n; ++k) {
        tasks[k].A = dA;
        tasks[k].ws = reinterpret_cast<double*>(buf + off_ws) + k * (size_t)ws;
        tasks[k].out = reinterpret_cast<double*>(buf + off_out) + 2 * k;
        tasks[k].L = L; tasks[k].W = W; tasks[k].D = D; tasks[k].chi = chi;
    }
    cudaStream_t st = ctx->stream;
    out->assign(2 * n, 0.0);
    e = cudaMemcpyAsync(buf, lat->host.data(), nel * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf + off_tasks, tasks.data(), n * sizeof(BmpsTask), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_bmps(prec == TN_FP64 ? 0 : 1, reinterpret_cast<const BmpsTask*>(buf + off_tasks), (int)n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->data(), buf + off_out, 2 * n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    ctx->used -= total;
    return cuda_status(e, "boundary-MPS contraction");
}

BmpsTask plain_task() {
    BmpsTask t{};
    t.op_site[0] = t.op_site[1] = -1;
    return t;
}

double ratio(const std::vector<double>& o, size_t k) {
    return o[2 * k] / o[0] * std::ldexp(1.0, (int)(o[2 * k + 1] - o[1]));
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_bmps_norm(tn_lattice* lat, int chi, tn_precision prec, tn_scalar* out) {
    try {
        if (!lat || !out) return TN_ERR_INVALID;
        std::vector<BmpsTask> tasks{plain_task()};
        std::vector<double> o;
        const tn_status s = bmps_run(lat, chi, prec, tasks, &o);
        if (s != TN_OK) return s;
        out->mant = o[0];
        out->exp2 = (int64_t)o[1];
        if (!std::isfinite(o[0]) || o[0] == 0.0) { set_error("zero or non-finite norm"); return TN_ERR_NUMERIC; }
        return TN_OK;
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

tn_status tn_bmps_expectation(tn_lattice* lat, int chi, tn_precision prec, int op_i, int i, int op_j, int j,
                               double* out) {
    try {
        if (!lat || !out) return TN_ERR_INVALID;
        const int N = lat->L * lat->W;
        auto op_ok = [](int op) { return op == TN_OP_X || op == TN_OP_Z; };
        if (!op_ok(op_i) || i < 0 || i >= N || (op_j != 0 && (!op_ok(op_j) || j < 0 || j >= N || j == i))) {
            set_error("operators must be TN_OP_X or TN_OP_Z on distinct sites (op_j = 0: one operator)");
            return TN_ERR_INVALID;
        }
        std::vector<BmpsTask> tasks{plain_task(), plain_task()};
        tasks[1].op_site[0] = i;
        tasks[1].op_code[0] = op_i == TN_OP_X ? 1 : 2;
        if (op_j != 0) {
            tasks[1].op_site[1] = j;
            tasks[1].op_code[1] = op_j == TN_OP_X ? 1 : 2;
        }
        std::vector<double> o;
        const tn_status s = bmps_run(lat, chi, prec, tasks, &o);
        if (s != TN_OK) return s;
        *out = ratio(o, 1);
        return std::isfinite(*out) ? TN_OK : TN_ERR_NUMERIC;
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

tn_status tn_bmps_energy(tn_lattice* lat, int chi, tn_precision prec, double J, double h, tn_result* out) {
    try {
        if (!lat || !out) return TN_ERR_INVALID;
        const int L = lat->L, W = lat->W, N = L * W;
        std::vector<BmpsTask> tasks{plain_task()};
        for (int k = 0; k < N; ++k) {
            BmpsTask t = plain_task();
            t.op_site[0] = k;
            t.op_code[0] = 1;
            tasks.push_back(t);
        }
        std::vector<std::pair<int, int>> bonds;
        for (int r = 0; r < L; ++r)
            for (int c = 0; c + 1 < W; ++c) bonds.push_back({r * W + c, r * W + c + 1});
        for (int r = 0; r + 1 < L; ++r)
            for (int c = 0; c < W; ++c) bonds.push_back({r * W + c, (r + 1) * W + c});
        for (auto& b : bonds) {
            BmpsTask t = plain_task();
            t.op_site[0] = b.first; t.op_code[0] = 2;
            t.op_site[1] = b.second; t.op_code[1] = 2;
            tasks.push_back(t);
        }
        std::vector<double> o;
        const tn_status s = bmps_run(lat, chi, prec, tasks, &o);
        if (s != TN_OK) return s;
        double sx = 0.0, szz = 0.0;
        for (int k = 0; k < N; ++k) {
            const double v = ratio(o, 1 + k);
            sx += v;
            if (out->sx) out->sx[k] = v;
        }
        for (size_t b = 0; b < bonds.size(); ++b) {
            const double v = ratio(o, 1 + N + b);
            szz += v;
            if (out->szsz) out->szsz[b] = v;
        }
        out->energy = -J * szz - h * sx;
        out->energy_per_site = out->energy / N;
        out->norm.mant = o[0];
        out->norm.exp2 = (int64_t)o[1];
        out->precision = prec;
        out->err_bound_est = 0.0;
        out->schedule_o = out->schedule_i = out->schedule_j = -1;
        if (!std::isfinite(out->energy)) { set_error("non-finite energy"); return TN_ERR_NUMERIC; }
        return TN_OK;
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

}  // extern "C"
