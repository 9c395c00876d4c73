// C ABI of the LB IMEX-TR library: contexts and the per-call drivers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <string>

#include "../../include/lbtr.h"
#include "ctx.cuh"

using namespace lbtr;

// ---------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------
static lb_status fail(lb_ctx* c, lb_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

static lb_status cuda_check(lb_ctx* c, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return LB_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

lb_status lb_ctx::sync_read(double* host, const double* dev, int count, cudaStream_t s, const char* where) {
    cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(this, LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return LB_OK;
}

extern "C" {

void lb_default_sub_opts(lb_sub_opts* o) {
    if (!o) return;
    o->eta = 0.1;
    o->eps_sub = 1e-13;
    o->rel_tol = 0.0;
    o->max_iter = 20000;
    o->check_every = 64;
}

void lb_default_eig_opts(lb_eig_opts* o) {
    if (!o) return;
    o->max_steps = 300;
    o->tol = 1e-8;
    o->sigma = 0.0;
    o->check_every = 10;
    o->seed = 12345;
}

void lb_default_tr_opts(lb_tr_opts* o) {
    if (!o) return;
    o->gamma_c = 0.5; o->gamma_e = 2.0; o->gamma_lam = 1.5; o->theta = 1e-4;
    o->mu_lo = 1.0; o->mu_hi = 1e5; o->mu0 = 1.0; o->r0 = 1.0; o->nu0 = 5.0;
    o->eps = 1e-10;
    o->max_outer = 500;
    o->second_order = 1;
    o->tol2 = 1e-8;
    lb_default_sub_opts(&o->sub);
    lb_default_eig_opts(&o->eig);
    o->pcg_max_iter = 2000;
    o->pcg_rtol = 1e-10;
    o->hard_tol = 0.0;
    o->checkpoint_path = nullptr;
    o->checkpoint_every = 0;
    o->resume = 0;
}

lb_status lb_create(const lb_problem* prob, lb_precision prec, lb_ctx** out) {
    if (!prob || !out) return LB_ERR_INVALID_ARG;
    *out = nullptr;
    if (prob->dim != 2 && prob->dim != 3) return LB_ERR_UNSUPPORTED;
    if (!is_pow2(prob->n) || prob->n < 8 || prob->n > (prob->dim == 2 ? 512 : 256)) return LB_ERR_UNSUPPORTED;
    for (int a = 0; a < prob->dim; ++a)
        if (!(prob->box[a] > 0.0) || !std::isfinite(prob->box[a])) return LB_ERR_INVALID_ARG;
    if (!std::isfinite(prob->xi) || !std::isfinite(prob->tau) || !std::isfinite(prob->gamma))
        return LB_ERR_INVALID_ARG;
    if (prec != LB_FP64 && prec != LB_MIXED) return LB_ERR_INVALID_ARG;
    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return LB_ERR_OOM;
    c->prob = *prob;
    if (c->prob.dim == 2) c->prob.box[2] = 1.0;
    c->prec = prec;
    int st = c->init();
    if (st != 0) {
        lb_status s = (lb_status)st;
        delete c;
        return s;
    }
    *out = c;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx* ctx) {
    delete ctx;
    return LB_OK;
}

const char* lb_last_error(const lb_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

size_t lb_workspace_bytes(const lb_ctx* ctx) { return ctx ? ctx->workspace_bytes() : 0; }

lb_status lb_set_params(lb_ctx* ctx, double xi, double tau, double gamma) {
    if (!ctx) return LB_ERR_INVALID_ARG;
    if (!std::isfinite(xi) || !std::isfinite(tau) || !std::isfinite(gamma)) return LB_ERR_INVALID_ARG;
    ctx->prob.xi = xi; ctx->prob.tau = tau; ctx->prob.gamma = gamma;
    if (ctx->p64) ctx->p64->set_params(xi, tau, gamma);
    if (ctx->p32) ctx->p32->set_params(xi, tau, gamma);
    return LB_OK;
}

lb_status lb_profile_enable(lb_ctx* ctx, int enable) {
    if (!ctx) return LB_ERR_INVALID_ARG;
    ctx->prof.reset();
    lbtr::Prof* p = enable ? &ctx->prof : nullptr;
    if (ctx->p64) ctx->p64->set_prof(p);
    if (ctx->p32) ctx->p32->set_prof(p);
    return LB_OK;
}

lb_status lb_profile_read(lb_ctx* ctx, int kclass, double* total_ms, long long* launches, double* alg_bytes) {
    if (!ctx || kclass < 0 || kclass >= LB_K_COUNT) return LB_ERR_INVALID_ARG;
    ctx->prof.flush();
    if (total_ms) *total_ms = ctx->prof.ms(kclass);
    if (launches) *launches = ctx->prof.launches(kclass);
    if (alg_bytes) *alg_bytes = ctx->prof.bytes(kclass);
    return LB_OK;
}

// FP64 FMA throughput probe: every thread runs 8 independent chains of dependent fused
// multiply-adds (enough in flight per warp to hide the FP64 pipe latency); the result is
// written only under a condition that never holds, so the loop cannot be removed.
__global__ void k_fp64_fma_loop(double* sink, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-9 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += x[k];
    if (t == -1.0) sink[0] = t;
}

lb_status lb_measure_fp64_rate(double* tflops, lb_stream stream) {
    if (!tflops) return LB_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LB_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LB_ERR_CUDA;
    const int blocks = 8 * nsm, threads = 256, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LB_ERR_CUDA;
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {      // the first run is a warm-up
        cudaEventRecord(e0, s);
        k_fp64_fma_loop<<<blocks, threads, 0, s>>>(nullptr, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return LB_ERR_CUDA; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
        if (rep > 0 && ms > 0.0f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return LB_ERR_CUDA;
    *tflops = best;
    return LB_OK;
}

lb_status lb_set_barrier_budget(lb_ctx* ctx, long long cycles) {
    if (!ctx) return LB_ERR_INVALID_ARG;
    if (ctx->p64) ctx->p64->set_barrier_budget(cycles);
    if (ctx->p32) ctx->p32->set_barrier_budget(cycles);
    return LB_OK;
}

lb_status lb_set_persistent_subproblem(lb_ctx* ctx, int enable) {
    if (!ctx) return LB_ERR_INVALID_ARG;
    if (ctx->p32) ctx->p32->set_imex_persistent(enable != 0);
    if (ctx->p64) ctx->p64->set_imex_persistent(enable != 0);
    return LB_OK;
}

lb_status lb_persistent_subproblem_available(lb_ctx* ctx, int* available) {
    if (!ctx || !available) return LB_ERR_INVALID_ARG;
    *available = (ctx->p32 && ctx->p32->imex_persistent_available()) ||
                 (ctx->p64 && ctx->p64->imex_persistent_available());
    return LB_OK;
}

lb_status lb_energy_grad(lb_ctx* ctx, const void* phi, double* energy, void* grad, double* gmax,
                         lb_stream stream) {
    if (!ctx || !phi || !energy) return fail(ctx, LB_ERR_INVALID_ARG, "lb_energy_grad: null argument");
    if (!aligned16(phi) || (grad && !aligned16(grad)))
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_energy_grad: fields must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->prec == LB_FP64) return ctx->energy_grad<double>(*ctx->p64, (const double*)phi, energy, (double*)grad, gmax, s);
    return ctx->energy_grad<float>(*ctx->p32, (const float*)phi, energy, (float*)grad, gmax, s);
}

lb_status lb_energy_derivs(lb_ctx* ctx, const void* phi, double* out, void* grad, lb_stream stream) {
    if (!ctx || !phi || !out) return fail(ctx, LB_ERR_INVALID_ARG, "lb_energy_derivs: null argument");
    if (!aligned16(phi) || (grad && !aligned16(grad)))
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_energy_derivs: fields must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->prec == LB_FP64) return ctx->energy_derivs<double>(*ctx->p64, (const double*)phi, out, (double*)grad, s);
    return ctx->energy_derivs<float>(*ctx->p32, (const float*)phi, out, (float*)grad, s);
}

lb_status lb_hessvec(lb_ctx* ctx, const void* phi, const void* v, void* hv, lb_stream stream) {
    if (!ctx || !phi || !v || !hv) return fail(ctx, LB_ERR_INVALID_ARG, "lb_hessvec: null argument");
    if (!aligned16(phi) || !aligned16(v) || !aligned16(hv))
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_hessvec: fields must be 16-byte aligned");
    if (hv == phi || hv == v) return fail(ctx, LB_ERR_INVALID_ARG, "lb_hessvec: output aliases an input");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->prec == LB_FP64) ctx->p64->hessvec((const double*)phi, (const double*)v, (double*)hv, s);
    else ctx->p32->hessvec((const float*)phi, (const float*)v, (float*)hv, s);
    return cuda_check(ctx, "lb_hessvec");
}

lb_status lb_hessvec_host(lb_ctx* ctx, const void* phi, int count, const void* const* v, void* const* hv,
                          lb_stream stream) {
    if (!ctx || !phi || count < 0 || (count > 0 && (!v || !hv)))
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_hessvec_host: null argument or negative count");
    for (int i = 0; i < count; ++i) {
        if (!v[i] || !hv[i]) return fail(ctx, LB_ERR_INVALID_ARG, "lb_hessvec_host: null field pointer");
        if (hv[i] == phi || hv[i] == v[i]) return fail(ctx, LB_ERR_INVALID_ARG, "lb_hessvec_host: output aliases an input");
    }
    if (count == 0) return LB_OK;
    constexpr int K = lb_ctx::HS_SLOTS;
    const size_t wsz = ctx->prec == LB_FP64 ? sizeof(double) : sizeof(float);
    const size_t fb = (size_t)ctx->n() * wsz;
    const size_t fa = (fb + 255) & ~size_t(255);
    if (!ctx->hs_base) {
        if (cudaMalloc(&ctx->hs_base, (1 + 2 * K) * fa) != cudaSuccess) {
            ctx->hs_base = nullptr;
            cudaGetLastError();
            return fail(ctx, LB_ERR_CUDA, "lb_hessvec_host: cudaMalloc of the staging failed");
        }
        bool ok = cudaStreamCreateWithFlags(&ctx->hs_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&ctx->hs_out, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ctx->hs_phi, cudaEventDisableTiming) == cudaSuccess;
        for (auto& row : ctx->hs_ev)
            for (auto& e : row) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return fail(ctx, LB_ERR_CUDA, "lb_hessvec_host: stream or event creation failed");
    }
    char* base = static_cast<char*>(ctx->hs_base);
    void* phi_d = base;
    auto v_d = [&](int k) { return (void*)(base + (1 + k) * fa); };
    auto hv_d = [&](int k) { return (void*)(base + (1 + K + k) * fa); };
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t in = ctx->hs_in, out = ctx->hs_out;
    cudaEvent_t (&ev)[3][K] = ctx->hs_ev;
    // the copy-in stream starts after everything already on `stream` (the staging's last users)
    cudaEventRecord(ctx->hs_phi, s);
    cudaStreamWaitEvent(in, ctx->hs_phi, 0);
    cudaMemcpyAsync(phi_d, phi, fb, cudaMemcpyHostToDevice, in);
    for (int i = 0; i < count; ++i) {
        const int k = i % K;
        if (i >= K) cudaStreamWaitEvent(in, ev[1][k], 0);        // slot k's v consumed by product i - K
        cudaMemcpyAsync(v_d(k), v[i], fb, cudaMemcpyHostToDevice, in);
        cudaEventRecord(ev[0][k], in);
        cudaStreamWaitEvent(s, ev[0][k], 0);                      // phi (copied first) and v_i in place
        if (i >= K) cudaStreamWaitEvent(s, ev[2][k], 0);          // slot k's Hv copied out
        if (ctx->prec == LB_FP64) ctx->p64->hessvec((const double*)phi_d, (const double*)v_d(k), (double*)hv_d(k), s);
        else ctx->p32->hessvec((const float*)phi_d, (const float*)v_d(k), (float*)hv_d(k), s);
        cudaEventRecord(ev[1][k], s);
        cudaStreamWaitEvent(out, ev[1][k], 0);
        cudaMemcpyAsync(hv[i], hv_d(k), fb, cudaMemcpyDeviceToHost, out);
        cudaEventRecord(ev[2][k], out);
    }
    for (int k = 0; k < K && k < count; ++k) cudaStreamWaitEvent(s, ev[2][k], 0);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, LB_ERR_CUDA, std::string("lb_hessvec_host: ") + cudaGetErrorString(e));
    return cuda_check(ctx, "lb_hessvec_host");
}

lb_status lb_tr_subproblem(lb_ctx* ctx, const void* phi, const void* g, double r, const void* d0,
                           const lb_sub_opts* opts, void* d, lb_sub_info* info, lb_stream stream) {
    if (!ctx || !phi || !g || !d) return fail(ctx, LB_ERR_INVALID_ARG, "lb_tr_subproblem: null argument");
    if (!(r > 0.0) || !std::isfinite(r)) return fail(ctx, LB_ERR_INVALID_ARG, "lb_tr_subproblem: r must be > 0");
    if (!aligned16(phi) || !aligned16(g) || !aligned16(d) || (d0 && !aligned16(d0)))
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_tr_subproblem: fields must be 16-byte aligned");
    lb_sub_opts o;
    lb_default_sub_opts(&o);
    if (opts) o = *opts;
    if (!(o.eta > 0.0) || o.max_iter < 1) return fail(ctx, LB_ERR_INVALID_ARG, "lb_tr_subproblem: bad options");
    if (o.check_every < 1) o.check_every = 64;
    cudaStream_t s = (cudaStream_t)stream;
    lb_sub_info inf;
    std::memset(&inf, 0, sizeof(inf));
    lb_status st;
    if (ctx->prec == LB_FP64)
        st = ctx->subproblem<double>(*ctx->p64, (const double*)phi, (const double*)g, r, (const double*)d0, o,
                                     (double*)d, &inf, s);
    else
        st = ctx->subproblem<float>(*ctx->p32, (const float*)phi, (const float*)g, r, (const float*)d0, o,
                                    (float*)d, &inf, s);
    if (info) *info = inf;
    return st;
}

lb_status lb_lambda_min(lb_ctx* ctx, const void* phi, const lb_eig_opts* opts, void* vec, lb_eig_info* info,
                        lb_stream stream) {
    if (!ctx || !phi) return fail(ctx, LB_ERR_INVALID_ARG, "lb_lambda_min: null argument");
    if (!aligned16(phi) || (vec && !aligned16(vec)))
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_lambda_min: fields must be 16-byte aligned");
    lb_eig_opts o;
    lb_default_eig_opts(&o);
    if (opts) o = *opts;
    if (o.max_steps < 2 || o.max_steps > 600)
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_lambda_min: max_steps must be in [2, 600]");
    if (o.check_every < 1) o.check_every = 10;
    lb_eig_info inf;
    std::memset(&inf, 0, sizeof(inf));
    cudaStream_t s = (cudaStream_t)stream;
    lb_status st;
    if (ctx->prec == LB_FP64)
        st = ctx->lambda_min<double>(*ctx->p64, (const double*)phi, o, (double*)vec, &inf, s);
    else
        st = ctx->lambda_min<float>(*ctx->p32, (const float*)phi, o, (float*)vec, &inf, s);
    if (info) *info = inf;
    return st;
}

lb_status lb_imex_tr_solve(lb_ctx* ctx, double* phi_inout, const lb_tr_opts* opts, lb_tr_info* info,
                           lb_stream stream) {
    if (!ctx || !phi_inout) return fail(ctx, LB_ERR_INVALID_ARG, "lb_imex_tr_solve: null argument");
    if (!aligned16(phi_inout)) return fail(ctx, LB_ERR_INVALID_ARG, "lb_imex_tr_solve: field must be 16-byte aligned");
    lb_tr_opts o;
    lb_default_tr_opts(&o);
    if (opts) o = *opts;
    lb_tr_info inf;
    std::memset(&inf, 0, sizeof(inf));
    inf.lambda_min = std::numeric_limits<double>::quiet_NaN();
    inf.g1_min = std::numeric_limits<double>::quiet_NaN();
    lb_status st = ctx->tr_solve(phi_inout, o, &inf, (cudaStream_t)stream);
    inf.status = (int)st;
    if (info) *info = inf;
    return st;
}

void lb_default_sis_opts(lb_sis_opts* o) {
    if (!o) return;
    o->dt = 1.0;
    o->eps = 1e-8;
    o->max_steps = 10000;
    o->check_every = 10;
}

lb_status lb_sis_solve(lb_ctx* ctx, double* phi_inout, const lb_sis_opts* opts, lb_sis_info* info,
                       lb_stream stream) {
    if (!ctx || !phi_inout) return fail(ctx, LB_ERR_INVALID_ARG, "lb_sis_solve: null argument");
    if (!aligned16(phi_inout)) return fail(ctx, LB_ERR_INVALID_ARG, "lb_sis_solve: field must be 16-byte aligned");
    lb_sis_opts o;
    lb_default_sis_opts(&o);
    if (opts) o = *opts;
    if (!(o.dt > 0.0) || !std::isfinite(o.dt) || o.max_steps < 0)
        return fail(ctx, LB_ERR_INVALID_ARG, "lb_sis_solve: dt must be positive and max_steps >= 0");
    lb_sis_info inf;
    std::memset(&inf, 0, sizeof(inf));
    lb_status st = ctx->sis_solve(phi_inout, o, &inf, (cudaStream_t)stream);
    inf.status = (int)st;
    if (info) *info = inf;
    return st;
}

}  // extern "C"
