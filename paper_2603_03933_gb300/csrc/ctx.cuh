// The lb_ctx object behind the C ABI and its host-side drivers.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/lbtr.h"
#include "plan.cuh"

namespace lbtr {
extern template class Plan<float>;
extern template class Plan<double>;
}

struct lb_ctx {
    lb_problem prob{};
    lb_precision prec = LB_FP64;
    std::string err;
    lbtr::Plan<double>* p64 = nullptr;   // FP64 operators (both precisions: the outer loop is FP64)
    lbtr::Plan<float>* p32 = nullptr;    // float operators (LB_MIXED)
    void* scratch = nullptr;             // field-sized temporaries
    size_t scratch_bytes = 0;
    double* d_scal = nullptr;            // small device scalars
    static constexpr int NW = 8, NF = 8;
    void* tmp_w[NW] = {};                // working-type fields
    double* f64[NF] = {};                // FP64 fields of the outer loop
    void* lz_base = nullptr;             // Lanczos basis and its scratch (allocated on first use)
    size_t lz_bytes = 0;
    lbtr::Prof prof;                     // per-kernel-class event timing (profiling aid)
    // staging of lb_hessvec_host (allocated on first use): phi and HS_SLOTS (v, Hv) slots on
    // the device, one copy stream per direction, the events that order the slots
    static constexpr int HS_SLOTS = 3;
    void* hs_base = nullptr;
    cudaStream_t hs_in = nullptr, hs_out = nullptr;
    cudaEvent_t hs_phi = nullptr, hs_ev[3][HS_SLOTS] = {};   // [0] copied in, [1] computed, [2] copied out

    ~lb_ctx() {
        delete p64;
        delete p32;
        if (scratch) cudaFree(scratch);
        if (lz_base) cudaFree(lz_base);
        if (hs_base) cudaFree(hs_base);
        if (hs_in) cudaStreamDestroy(hs_in);
        if (hs_out) cudaStreamDestroy(hs_out);
        if (hs_phi) cudaEventDestroy(hs_phi);
        for (auto& row : hs_ev)
            for (auto& e : row)
                if (e) cudaEventDestroy(e);
    }

    long long n() const { return p64->n(); }

    int init() {
        p64 = new lbtr::Plan<double>();
        int st = p64->init(prob.dim, prob.n, prob.box, prob.xi, prob.tau, prob.gamma, err);
        if (st) return st;
        if (prec == LB_MIXED) {
            p32 = new lbtr::Plan<float>();
            st = p32->init(prob.dim, prob.n, prob.box, prob.xi, prob.tau, prob.gamma, err);
            if (st) return st;
        }
        const size_t nn = (size_t)p64->n();
        const size_t wsz = prec == LB_FP64 ? sizeof(double) : sizeof(float);
        auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
        scratch_bytes = up(64 * sizeof(double)) + NW * up(nn * wsz) + NF * up(nn * sizeof(double));
        if (cudaMalloc(&scratch, scratch_bytes) != cudaSuccess) {
            scratch = nullptr;
            err = "cudaMalloc of the context scratch failed";
            return LB_ERR_OOM;
        }
        cudaMemset(scratch, 0, scratch_bytes);
        char* b = static_cast<char*>(scratch);
        d_scal = reinterpret_cast<double*>(b);
        b += up(64 * sizeof(double));
        for (int i = 0; i < NW; ++i) { tmp_w[i] = b; b += up(nn * wsz); }
        for (int i = 0; i < NF; ++i) { f64[i] = reinterpret_cast<double*>(b); b += up(nn * sizeof(double)); }
        return 0;
    }

    size_t workspace_bytes() const {
        return (p64 ? p64->bytes() : 0) + (p32 ? p32->bytes() : 0) + scratch_bytes;
    }

    lb_status sync_read(double* host, const double* dev, int count, cudaStream_t s, const char* where);

    lb_status launch_status(const char* where) {
        cudaError_t e = cudaGetLastError();
        cudaError_t c = p64 ? p64->take_launch_error() : cudaSuccess;
        if (c == cudaSuccess && p32) c = p32->take_launch_error();
        if (e == cudaSuccess) e = c;
        if (e != cudaSuccess) { err = std::string(where) + ": " + cudaGetErrorString(e); return LB_ERR_CUDA; }
        return LB_OK;
    }

    // E, g, max|g| with the zero-mean and finiteness checks of the ABI.
    template <typename T>
    lb_status energy_grad(lbtr::Plan<T>& p, const T* phi, double* energy, T* grad, double* gmax, cudaStream_t s) {
        p.energy_grad(phi, grad, s);
        lb_status st = launch_status("lb_energy_grad");
        if (st) return st;
        double ef[4], eg[1], gm[1] = {0.0};
        if ((st = sync_read(ef, p.slot(lbtr::S_EF), 4, s, "lb_energy_grad"))) return st;
        if ((st = sync_read(eg, p.slot(lbtr::S_EG), 1, s, "lb_energy_grad"))) return st;
        if (grad && (st = sync_read(gm, p.slot(lbtr::S_GMAX), 1, s, "lb_energy_grad"))) return st;
        const double nn = (double)p.n();
        const double mean = ef[2] / nn, rms = std::sqrt(std::fmax(ef[3] / nn, 0.0));
        if (!std::isfinite(ef[0]) || !std::isfinite(ef[1]) || !std::isfinite(eg[0]) || !std::isfinite(ef[3]) ||
            !std::isfinite(gm[0])) {
            err = "lb_energy_grad: non-finite value in the input or a reduction";
            return LB_ERR_NONFINITE;
        }
        const double tol = sizeof(T) == 8 ? 1e-10 : 1e-5;
        if (std::fabs(mean) > tol * std::fmax(1.0, rms)) {
            err = "lb_energy_grad: phi does not have zero mean (mean " + std::to_string(mean) + ")";
            return LB_ERR_NOT_ZERO_MEAN;
        }
        *energy = eg[0] + ef[0] / nn;
        if (gmax) *gmax = gm[0];
        return LB_OK;
    }

    // E and its derivatives with respect to tau, gamma and the box lengths (grid values of phi
    // held fixed); the gradient into grad when non-null.
    template <typename T>
    lb_status energy_derivs(lbtr::Plan<T>& p, const T* phi, double* out, T* grad, cudaStream_t s) {
        double e = 0.0;
        lb_status st = energy_grad(p, phi, &e, grad, nullptr, s);
        if (st) return st;
        p.phys_reduce(lbtr::R_POW23, phi, nullptr, lbtr::S_RED1, s);
        double pw[2], bx[3];
        if ((st = sync_read(pw, p.slot(lbtr::S_RED1), 2, s, "lb_energy_derivs"))) return st;
        p.box_derivs(phi, s);
        if ((st = launch_status("lb_energy_derivs"))) return st;
        if ((st = sync_read(bx, p.slot(lbtr::S_DBOX), 3, s, "lb_energy_derivs"))) return st;
        const double nn = (double)p.n();
        out[0] = e;
        out[1] = 0.5 * pw[0] / nn;            // dE/dtau = <phi^2 / 2>_N
        out[2] = -pw[1] / (6.0 * nn);         // dE/dgamma = -<phi^3 / 6>_N
        for (int a = 0; a < 3; ++a) out[3 + a] = a < prob.dim ? bx[a] / prob.box[a] : 0.0;
        for (int a = 0; a < 6; ++a)
            if (!std::isfinite(out[a])) { err = "lb_energy_derivs: non-finite result"; return LB_ERR_NONFINITE; }
        return LB_OK;
    }

    // Algorithm 3 driver.
    template <typename T>
    lb_status subproblem(lbtr::Plan<T>& p, const T* phi, const T* g, double r, const T* d0, const lb_sub_opts& o,
                         T* d, lb_sub_info* info, cudaStream_t s) {
        p.eta = o.eta;
        lb_status st;
        // ||g|| (and max |g| for the finiteness check)
        p.phys_reduce(lbtr::R_SUMSQ_MAX, g, nullptr, lbtr::S_RED1, s);
        double gs[2];
        if ((st = sync_read(gs, p.slot(lbtr::S_RED1), 2, s, "lb_tr_subproblem"))) return st;
        if (!std::isfinite(gs[0])) { err = "lb_tr_subproblem: non-finite gradient"; return LB_ERR_NONFINITE; }
        const double gnorm = std::sqrt(gs[0] / (double)p.n());
        if (!d0 && !(gnorm > 0.0)) {
            err = "lb_tr_subproblem: g = 0 and no initial point given";
            return LB_ERR_INVALID_ARG;
        }
        double dscale = d0 ? 0.0 : -r / gnorm;
        cudaMemcpyAsync(d_scal, &dscale, sizeof(double), cudaMemcpyHostToDevice, s);
        p.reset_barrier(s);
        lbtr::ImexState hs;
        if (p.imex_persistent_available()) {
            // the whole inner loop and the returned iterate in one launch
            p.imex_persistent(phi, g, d0, d_scal, d, r, o.eps_sub, o.rel_tol * gnorm, o.max_iter, s);
            if ((st = launch_status("lb_tr_subproblem/persistent"))) return st;
            cudaMemcpyAsync(&hs, p.imex_state(), sizeof(hs), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { err = std::string("lb_tr_subproblem: ") + cudaGetErrorString(e); return LB_ERR_CUDA; }
            if (p.read_error(s)) { err = "lb_tr_subproblem: a grid barrier timed out"; return LB_ERR_TIMEOUT; }
            if (!hs.done) { err = "lb_tr_subproblem: the persistent solve ended without a result"; return LB_ERR_CUDA; }
        } else {
        p.imex_init(phi, g, d0, d_scal, r, o.eps_sub, o.rel_tol * gnorm, o.max_iter, s);
        if ((st = launch_status("lb_tr_subproblem/init"))) return st;
        int j = 1;
        int chunk = 2;     // chunks grow 2, 4, 8, ... up to check_every: little work is wasted
                           // on no-op launches after an early convergence
        while (true) {
            int cnt = std::min(chunk, std::max(2, o.check_every));
            if (cnt % 2) ++cnt;
            chunk = std::min(2 * chunk, std::max(2, o.check_every));
            p.imex_iterate(phi, g, j, cnt, s);
            j += cnt;
            if ((st = launch_status("lb_tr_subproblem/iterate"))) return st;
            cudaMemcpyAsync(&hs, p.imex_state(), sizeof(hs), cudaMemcpyDeviceToHost, s);
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { err = std::string("lb_tr_subproblem: ") + cudaGetErrorString(e); return LB_ERR_CUDA; }
            int be = p.read_error(s);
            if (be) { err = "lb_tr_subproblem: a grid barrier timed out"; return LB_ERR_TIMEOUT; }
            if (hs.done) break;
            if (j > o.max_iter + 2 * o.check_every + 4) { err = "lb_tr_subproblem: driver overran"; return LB_ERR_CUDA; }
        }
        p.imex_final(d, s);
        if ((st = launch_status("lb_tr_subproblem/final"))) return st;
        }
        // ||d|| and f(d) = <g,d> + <d,Hd>/2
        T* hd = static_cast<T*>(tmp_w[7]);
        p.hessvec(phi, d, hd, s);
        p.phys_reduce(lbtr::R_DOT, g, d, lbtr::S_RED0, s);
        double gd[1], dhd[1], dd[2];
        if ((st = sync_read(gd, p.slot(lbtr::S_RED0), 1, s, "lb_tr_subproblem"))) return st;
        p.phys_reduce(lbtr::R_DOT, d, hd, lbtr::S_RED0, s);
        if ((st = sync_read(dhd, p.slot(lbtr::S_RED0), 1, s, "lb_tr_subproblem"))) return st;
        p.phys_reduce(lbtr::R_SUMSQ_MAX, d, nullptr, lbtr::S_RED1, s);
        if ((st = sync_read(dd, p.slot(lbtr::S_RED1), 2, s, "lb_tr_subproblem"))) return st;
        const double nn = (double)p.n();
        info->iterations = hs.it;
        info->converged = hs.done == 1;
        info->stalled = hs.done == 4;
        info->residual = hs.residual;
        info->rel_residual = gnorm > 0.0 ? hs.residual / gnorm : hs.residual;
        info->lambda = hs.final_lam;
        info->dnorm = std::sqrt(dd[0] / nn);
        info->model_value = gd[0] / nn + 0.5 * dhd[0] / nn;
        info->newton_steps = hs.newton;
        if (hs.done == 3) { err = "lb_tr_subproblem: non-finite residual"; return LB_ERR_NONFINITE; }
        if (hs.done == 2) { err = "lb_tr_subproblem: iteration cap reached"; return LB_ERR_NOCONV; }
        if (hs.done == 4) {
            err = "lb_tr_subproblem: stalled (no progress in " + std::to_string(p.stall_k()) +
                  " checked iterations) at residual " + std::to_string(hs.residual);
            return LB_ERR_NOCONV;
        }
        return LB_OK;
    }

    template <typename T>
    lb_status lambda_min(lbtr::Plan<T>& p, const T* phi, const lb_eig_opts& o, T* vec, lb_eig_info* info,
                         cudaStream_t s);

    // ||x||^2 (sum over points / N) and related helpers on physical fields
    template <typename T> lb_status dot(lbtr::Plan<T>& p, const T* x, const T* y, double* out, cudaStream_t s) {
        p.phys_reduce(lbtr::R_DOT, x, y, lbtr::S_RED0, s);
        double v;
        lb_status st = sync_read(&v, p.slot(lbtr::S_RED0), 1, s, "dot");
        *out = v / (double)p.n();
        return st;
    }

    // (H + shift I) x = -g by preconditioned CG; returns ||x|| in *xnorm
    template <typename T>
    lb_status pcg(lbtr::Plan<T>& p, const T* phi, const T* g, double shift, double rtol, int max_iter, T* x,
                  double* xnorm, int* iters, cudaStream_t s);

    template <typename T> lb_status random_ball(lbtr::Plan<T>& p, T* out, double r, unsigned long long seed,
                                                unsigned stream, cudaStream_t s);

    lb_status tr_solve(double* phi, const lb_tr_opts& o, lb_tr_info* info, cudaStream_t s);
    lb_status sis_solve(double* phi, const lb_sis_opts& o, lb_sis_info* info, cudaStream_t s);
};
