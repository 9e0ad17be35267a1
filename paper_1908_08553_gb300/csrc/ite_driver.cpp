// Imaginary time evolution driver (Sec. 5): the state is evolved on the device
// by second-order Trotter steps U^Gamma(dtau/2) U^J(dtau) U^Gamma(dtau/2),
// normalised after every set of operators by its norm from the exact FP64
// contraction (the library's own norm program), and its energy is evaluated
// by the exact contraction every `energy_every` steps.
//
// The site tensors live in the input area of the norm program's batch, so a
// normalisation is one batch run plus one scaling kernel with no copies and no
// host round trip; energies are copied device to device into a small array
// read once at the end.  Bonds are updated in four classes of disjoint bonds
// (horizontal with even left column, odd, vertical with even upper row, odd),
// one launch per class, one block per bond.
#include <cmath>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace tn {
namespace {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    tn_ctx* ctx = nullptr;
    ~DevBuf() {
        if (p) {
            cudaFree(p);
            ctx->used -= bytes;
        }
    }
    tn_status alloc(tn_ctx* c, size_t n) {
        ctx = c;
        if (ctx->used + n > ctx->budget) { set_error("ITE workspace exceeds the budget"); return TN_ERR_OVER_BUDGET; }
        const cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) { p = nullptr; return cuda_status(e, "ITE workspace"); }
        bytes = n;
        ctx->used += n;
        return TN_OK;
    }
};

void site_dims_of(int L, int W, int D, int r, int c, int* d) {   // {2, u, l, dn, rt}
    d[0] = 2;
    d[1] = r == 0 ? 1 : D;
    d[2] = c == 0 ? 1 : D;
    d[3] = r == L - 1 ? 1 : D;
    d[4] = c == W - 1 ? 1 : D;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_ite_init_product(tn_lattice* lat) {
    if (!lat) return TN_ERR_INVALID;
    const int L = lat->L, W = lat->W, D = lat->D;
    if (lat->cplx) {   // back to real site tensors
        for (auto& kv : lat->cache) batch_destroy(kv.second);
        lat->cache.clear();
        lat->cplx = false;
        lat->host.assign(lat->host.size() / 2, 0.0);
    }
    std::fill(lat->host.begin(), lat->host.end(), 0.0);
    size_t off = 0;
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            int d[5];
            site_dims_of(L, W, D, r, c, d);
            const size_t half = (size_t)d[1] * d[2] * d[3] * d[4];
            lat->host[off] = 1.0 / std::sqrt(2.0);          // A[0][0][0][0][0]
            lat->host[off + half] = 1.0 / std::sqrt(2.0);   // A[1][0][0][0][0]
            off += 2 * half;
        }
    return TN_OK;
}

tn_status tn_ite_run(tn_lattice* lat, const tn_ite_params* prm, double* energies, int* bond_dims,
                     double* max_discarded) {
    try {
        if (!lat || !prm) return TN_ERR_INVALID;
        if (lat->cplx) { set_error("imaginary time evolution takes real site tensors"); return TN_ERR_INVALID; }
        if (!lat->ctx || lat->ctx->device < 0) { set_error("context has no device"); return TN_ERR_NO_DEVICE; }
        const int L = lat->L, W = lat->W, D = lat->D;
        if (prm->chi_max != D || prm->steps < 0 || !(prm->dtau >= 0.0) || !std::isfinite(prm->dtau) ||
            !(prm->eps >= 0.0 && prm->eps < 1.0) || prm->energy_every < 0 || !std::isfinite(prm->J) ||
            !std::isfinite(prm->gamma) || prm->precision < TN_FP64 || prm->precision > TN_BF16X6) {
            set_error("bad ITE parameters (chi_max must equal the lattice's bond dimension)");
            return TN_ERR_INVALID;
        }
        tn_ctx* ctx = lat->ctx;
        cudaSetDevice(ctx->device);
        const int nsites = L * W;
        // site offsets in FP64 entries (the input layout)
        std::vector<long long> soff(nsites + 1, 0);
        std::vector<int> dims(5 * nsites);
        for (int r = 0; r < L; ++r)
            for (int c = 0; c < W; ++c) {
                const int s = r * W + c;
                site_dims_of(L, W, D, r, c, &dims[5 * s]);
                const int* d = &dims[5 * s];
                soff[s + 1] = soff[s] + 2LL * d[1] * d[2] * d[3] * d[4];
            }
        const long long nel = soff[nsites];
        // bond classes, each bond with its index in the output order (horizontal
        // row-major, then vertical row-major)
        std::vector<std::vector<std::pair<IteBondTask, int>>> classes(4);
        for (int par = 0; par < 2; ++par)
            for (int r = 0; r < L; ++r)
                for (int c = par; c + 1 < W; c += 2) {
                    IteBondTask t{};
                    const int i = r * W + c, j = i + 1;
                    t.off_i = soff[i]; t.off_j = soff[j];
                    std::memcpy(t.dims_i, &dims[5 * i], sizeof(t.dims_i));
                    std::memcpy(t.dims_j, &dims[5 * j], sizeof(t.dims_j));
                    t.horizontal = 1;
                    t.m = 2 * t.dims_i[1] * t.dims_i[2] * t.dims_i[3];
                    t.n = 2 * t.dims_j[1] * t.dims_j[3] * t.dims_j[4];
                    classes[par].push_back({t, r * (W - 1) + c});
                }
        for (int par = 0; par < 2; ++par)
            for (int r = par; r + 1 < L; r += 2)
                for (int c = 0; c < W; ++c) {
                    IteBondTask t{};
                    const int i = r * W + c, j = i + W;
                    t.off_i = soff[i]; t.off_j = soff[j];
                    std::memcpy(t.dims_i, &dims[5 * i], sizeof(t.dims_i));
                    std::memcpy(t.dims_j, &dims[5 * j], sizeof(t.dims_j));
                    t.horizontal = 0;
                    t.m = 2 * t.dims_i[1] * t.dims_i[2] * t.dims_i[4];
                    t.n = 2 * t.dims_j[2] * t.dims_j[3] * t.dims_j[4];
                    classes[2 + par].push_back({t, L * (W - 1) + r * W + c});
                }
        long long ws_need = 0;
        size_t ntask_all = 0;
        for (auto& cl : classes) {
            long long off = 0;
            for (auto& tb : cl) {
                const long long n2 = tb.first.n + (tb.first.n & 1);
                tb.first.ws_off = off;
                off += (long long)tb.first.m * n2 + n2 * n2;
            }
            ws_need = std::max(ws_need, off);
            ntask_all += cl.size();
        }
        const int nb = L * (W - 1) + W * (L - 1);
        const int n_e = prm->energy_every > 0 ? prm->steps / prm->energy_every : 0;

        // the norm program's batch holds the state; the energy program's reads a copy
        tn_batch* bN = nullptr;
        tn_batch* bE = nullptr;
        tn_status st = batch_create(ctx, 1, &L, &W, &D, TN_FP64, TN_SCHED_AUTO, TN_WORK_NORM, true, &bN, nullptr);
        if (st != TN_OK) return st;
        struct Guard {
            tn_batch* a;
            tn_batch* b;
            ~Guard() { batch_destroy(a); batch_destroy(b); }
        } guard{bN, nullptr};
        if (n_e > 0) {
            st = batch_create(ctx, 1, &L, &W, &D, (tn_precision)prm->precision, TN_SCHED_AUTO, TN_WORK_ENERGY, true,
                              &bE, nullptr);
            if (st != TN_OK) return st;
            guard.b = bE;
            bE->h_final[0].J = prm->J;
            bE->h_final[0].h = prm->gamma;
        }
        cudaStream_t s = bN->stream;
        double* dA = reinterpret_cast<double*>(bN->buf + bN->lay.in_off);
        const double* d_log2n = reinterpret_cast<const double*>(bN->buf + bN->lay.res_off) + 1;
        // device tables and workspace in one buffer
        const size_t b_off = (size_t)(nsites + 1) * sizeof(long long);
        const size_t b_tasks = b_off;
        const size_t b_kept = b_tasks + ntask_all * sizeof(IteBondTask);
        const size_t b_disc = (b_kept + (size_t)ntask_all * sizeof(int) + 15) / 16 * 16;
        const size_t b_en = b_disc + 16;
        const size_t b_ws = (b_en + (size_t)std::max(n_e, 1) * sizeof(double) + 255) / 256 * 256;
        const size_t total = b_ws + (size_t)ws_need * sizeof(double);
        DevBuf buf;
        st = buf.alloc(ctx, total);
        if (st != TN_OK) return st;
        char* base = static_cast<char*>(buf.p);
        std::vector<IteBondTask> htasks;
        std::vector<size_t> cls_first;
        for (auto& cl : classes) {
            cls_first.push_back(htasks.size());
            for (auto& tb : cl) htasks.push_back(tb.first);
        }
        cudaError_t e = cudaMemcpyAsync(base, soff.data(), b_off, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !htasks.empty())
            e = cudaMemcpyAsync(base + b_tasks, htasks.data(), htasks.size() * sizeof(IteBondTask),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(base + b_disc, 0, 16, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dA, lat->host.data(), (size_t)nel * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_status(e, "ITE upload");
        const long long* d_soff = reinterpret_cast<const long long*>(base);
        const IteBondTask* d_tasks = reinterpret_cast<const IteBondTask*>(base + b_tasks);
        int* d_kept = reinterpret_cast<int*>(base + b_kept);
        auto* d_disc = reinterpret_cast<unsigned long long*>(base + b_disc);
        double* d_en = reinterpret_cast<double*>(base + b_en);
        double* d_ws = reinterpret_cast<double*>(base + b_ws);

        const double a = prm->gamma * prm->dtau / 2.0;
        const double g1[4] = {std::cosh(a), std::sinh(a), std::sinh(a), std::cosh(a)};
        const double bj = prm->J * prm->dtau;   // exp(J dtau z_p z_q), z = (-1, +1)
        const double g2[4] = {std::exp(bj), std::exp(-bj), std::exp(-bj), std::exp(bj)};
        auto normalise = [&]() -> tn_status {
            tn_status r = batch_run(bN, s);
            if (r != TN_OK) return r;
            return cuda_status(launch_ite_scale(dA, nel, d_log2n, nsites, s), "ITE scale");
        };
        int ek = 0;
        for (int step = 1; step <= prm->steps; ++step) {
            if ((st = cuda_status(launch_ite_one_body(dA, d_soff, nsites, g1, s), "ITE one-body")) != TN_OK) return st;
            if ((st = normalise()) != TN_OK) return st;
            for (int c = 0; c < 4; ++c) {
                const int nt = (int)classes[c].size();
                st = cuda_status(launch_ite_bonds(dA, d_tasks + cls_first[c], nt, d_ws, g2, prm->chi_max, prm->eps,
                                                  d_kept + cls_first[c], d_disc, s),
                                 "ITE bonds");
                if (st != TN_OK) return st;
            }
            if ((st = normalise()) != TN_OK) return st;
            if ((st = cuda_status(launch_ite_one_body(dA, d_soff, nsites, g1, s), "ITE one-body")) != TN_OK) return st;
            if ((st = normalise()) != TN_OK) return st;
            if (n_e > 0 && step % prm->energy_every == 0 && ek < n_e) {
                e = cudaMemcpyAsync(bE->buf + bE->lay.in_off, dA, (size_t)nel * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return cuda_status(e, "ITE energy input");
                if ((st = batch_run(bE, s)) != TN_OK) return st;
                e = cudaMemcpyAsync(d_en + ek, bE->buf + bE->lay.res_off, sizeof(double), cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return cuda_status(e, "ITE energy copy");
                ++ek;
            }
        }
        std::vector<int> hkept(std::max<size_t>(ntask_all, 1));
        unsigned long long hdisc = 0;
        std::vector<double> hen(std::max(n_e, 1));
        e = cudaMemcpyAsync(lat->host.data(), dA, (size_t)nel * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && ntask_all)
            e = cudaMemcpyAsync(hkept.data(), d_kept, ntask_all * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hdisc, d_disc, sizeof(hdisc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && n_e > 0)
            e = cudaMemcpyAsync(hen.data(), d_en, (size_t)n_e * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_status(e, "ITE read-back");
        if (energies)
            for (int k = 0; k < ek; ++k) energies[k] = hen[k];
        if (bond_dims) {
            for (int k = 0; k < nb; ++k) bond_dims[k] = prm->steps > 0 ? 0 : 1;
            if (prm->steps > 0)
                for (int c = 0; c < 4; ++c)
                    for (size_t q = 0; q < classes[c].size(); ++q)
                        bond_dims[classes[c][q].second] = hkept[cls_first[c] + q];
        }
        if (max_discarded) {
            double d;
            std::memcpy(&d, &hdisc, sizeof(d));
            *max_discarded = d;
        }
        for (int k = 0; k < ek; ++k)
            if (!std::isfinite(hen[k])) { set_error("non-finite ITE energy"); return TN_ERR_NUMERIC; }
        return TN_OK;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return TN_ERR_OOM;
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

}  // extern "C"
