// Outer IMEX-TR loop (Algorithms 1 and 2 of the paper) and the Lanczos lambda_min driver.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <vector>

#include "checkpoint.h"
#include "ctx.cuh"
#include "dense_eig.cuh"

using namespace lbtr;

template <typename T> static T* wbuf(lb_ctx* c, int i) {
    if (sizeof(T) == 8) return reinterpret_cast<T*>(c->f64[i]);
    return reinterpret_cast<T*>(c->tmp_w[i]);
}

// ---------------------------------------------------------------------------------
// Lanczos on K = M^{-1/2} H M^{-1/2} (M = Lambda + sigma) with Rayleigh-Ritz for H on
// V = M^{-1/2} Q.  Vectors are paper-normalised half spectra; dot products are
// accumulated in double; the tridiagonal T_k, the Gram matrix G_k = Q^T M^{-1} Q and
// the pencil solve are FP64 on the host.
// ---------------------------------------------------------------------------------
template <typename T>
lb_status lb_ctx::lambda_min(Plan<T>& p, const T* phi, const lb_eig_opts& o, T* vec, lb_eig_info* info,
                             cudaStream_t s) {
    using C = cplx<T>;
    const long long len = p.spec_len();
    const int kmax = o.max_steps;
    const int nvec = kmax + 1;
    const int blk = 256, E = SPEC_MD_E;
    const int nblk = (int)((len + (long long)blk * E - 1) / ((long long)blk * E));
    // workspace: basis, one work vector, partials, coefficients
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = up(sizeof(C) * len * (size_t)nvec) + up(sizeof(C) * len) + up(sizeof(C) * len) +
                        up(sizeof(double) * (size_t)nvec * nblk) + up(sizeof(double) * 2 * (size_t)nvec);
    if (need > lz_bytes) {
        if (lz_base) cudaFree(lz_base);
        lz_base = nullptr;
        lz_bytes = 0;
        if (cudaMalloc(&lz_base, need) != cudaSuccess) {
            err = "lb_lambda_min: cannot allocate the Lanczos basis";
            return LB_ERR_OOM;
        }
        lz_bytes = need;
    }
    char* b = static_cast<char*>(lz_base);
    C* Q = reinterpret_cast<C*>(b); b += up(sizeof(C) * len * (size_t)nvec);
    C* w = reinterpret_cast<C*>(b); b += up(sizeof(C) * len);
    C* ritz = reinterpret_cast<C*>(b); b += up(sizeof(C) * len);
    double* part = reinterpret_cast<double*>(b); b += up(sizeof(double) * (size_t)nvec * nblk);
    double* coef = reinterpret_cast<double*>(b);

    SpecGeom g{len, p.dim(), p.m(), p.rows(), p.qtab()};
    const T xi2 = p.xi2();
    lb_status st;

    // sigma of the congruence: max(1e-2, max_x |F''(phi)|), F'' = tau - gamma phi + phi^2/2
    double sigma = o.sigma;
    if (!(sigma > 0.0)) {
        p.phys_reduce(R_SUMSQ_MAX, phi, nullptr, S_RED1, s);
        double red[2];
        if ((st = sync_read(red, p.slot(S_RED1), 2, s, "lb_lambda_min"))) return st;
        const double pm = red[1];
        const double tau = prob.tau, gam = prob.gamma;
        // |F''| on [-pm, pm] is bounded by its values at -pm, pm and at the vertex phi = gamma
        double f2max = std::max(std::fabs(tau + gam * pm + 0.5 * pm * pm), std::fabs(tau - gam * pm + 0.5 * pm * pm));
        if (std::fabs(gam) <= pm) f2max = std::max(f2max, std::fabs(tau - 0.5 * gam * gam));
        f2max = std::max(f2max, std::fabs(tau));
        sigma = std::max(1e-2, f2max);
    }

    auto multidot = [&](const C* Qs, int nv, const C* x, int minv, double* host_out) -> lb_status {
        size_t sm = sizeof(double) * (size_t)nv * (blk / 32);
        k_spec_multidot<T><<<nblk, blk, sm, s>>>(Qs, len, nv, x, g, minv, xi2, (T)sigma, part);
        k_partials_sum<<<(nv + 7) / 8, 256, 0, s>>>(part, nblk, nv, coef);
        cudaMemcpyAsync(host_out, coef, sizeof(double) * nv, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { err = std::string("lb_lambda_min: ") + cudaGetErrorString(e); return LB_ERR_CUDA; }
        return LB_OK;
    };
    auto multiaxpy = [&](const C* Qs, int nv, const std::vector<double>& c, C* y) {
        cudaMemcpyAsync(coef + nvec, c.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, s);
        int grid = (int)std::min<long long>(4096, (len + 255) / 256);
        k_spec_multiaxpy<T><<<grid, 256, sizeof(double) * nv, s>>>(Qs, len, nv, coef + nvec, y, len);
    };
    auto scale = [&](C* y, const C* x, double a) {
        int grid = (int)std::min<long long>(4096, (len + 255) / 256);
        k_spec_axpby<T><<<grid, 256, 0, s>>>(y, x, a, 0.0, nullptr, 0, len);
    };

    // start vector: Philox normal samples in physical space, to the spectrum, k = 0 removed
    T* tmp = wbuf<T>(this, 3);
    T* tmp2 = wbuf<T>(this, 4);
    p.random_normal(tmp, o.seed, 7u, s);
    p.to_spectrum(tmp, Q, s);
    cudaMemsetAsync(Q, 0, sizeof(C), s);
    std::vector<double> hv(nvec);
    if ((st = multidot(Q, 1, Q, 0, hv.data()))) return st;
    scale(Q, Q, 1.0 / std::sqrt(hv[0]));

    std::vector<double> alpha, beta;
    std::vector<double> G;                     // Gram matrix Q^T M^{-1} Q, (kmax+1)^2 row-major
    G.assign((size_t)nvec * nvec, 0.0);
    if ((st = multidot(Q, 1, Q, 1, hv.data()))) return st;
    G[0] = hv[0];
    double theta = 0.0, kappa = 0.0, resid = INFINITY;
    int steps = 0;
    bool converged = false;
    std::vector<double> ybest;
    std::vector<double> c1(nvec), c2(nvec);
    for (int j = 0; j < kmax; ++j) {
        C* qj = Q + (size_t)j * len;
        p.kop(phi, qj, w, sigma, s);
        if ((st = launch_status("lb_lambda_min/kop"))) return st;
        // classical Gram-Schmidt twice against the whole basis
        if ((st = multidot(Q, j + 1, w, 0, c1.data()))) return st;
        multiaxpy(Q, j + 1, c1, w);
        if ((st = multidot(Q, j + 1, w, 0, c2.data()))) return st;
        multiaxpy(Q, j + 1, c2, w);
        alpha.push_back(c1[j] + c2[j]);
        cudaMemsetAsync(w, 0, sizeof(C), s);    // K maps the constant field to 0: keep it out
        if ((st = multidot(w, 1, w, 0, hv.data()))) return st;
        const double bnorm = std::sqrt(std::max(hv[0], 0.0));
        steps = j + 1;
        const bool last = (j + 1 == kmax) || !(bnorm > 1e-14 * std::fabs(alpha.back()) + 1e-300);
        if (!last) {
            beta.push_back(bnorm);
            C* qn = Q + (size_t)(j + 1) * len;
            scale(qn, w, 1.0 / bnorm);
            if ((st = multidot(Q, j + 2, qn, 1, hv.data()))) return st;
            for (int i = 0; i <= j + 1; ++i) G[(size_t)i * nvec + (j + 1)] = G[(size_t)(j + 1) * nvec + i] = hv[i];
        }
        const int k = j + 1;
        if ((k % o.check_every == 0) || last) {
            std::vector<double> Tm((size_t)k * k, 0.0), Gk((size_t)k * k);
            for (int i = 0; i < k; ++i) {
                Tm[(size_t)i * k + i] = alpha[i];
                if (i + 1 < k) Tm[(size_t)i * k + i + 1] = Tm[(size_t)(i + 1) * k + i] = beta[i];
                for (int l = 0; l < k; ++l) Gk[(size_t)i * k + l] = G[(size_t)i * nvec + l];
            }
            std::vector<double> y;
            double th;
            if (!dense::smallest_generalized(k, Tm, Gk, th, y)) {
                err = "lb_lambda_min: Gram matrix lost positive definiteness";
                return LB_ERR_NONFINITE;
            }
            std::vector<double> I((size_t)k * k, 0.0), yk;
            for (int i = 0; i < k; ++i) I[(size_t)i * k + i] = 1.0;
            double kap;
            dense::smallest_generalized(k, Tm, I, kap, yk);
            // Ritz vector u = M^{-1/2} Q y (physical), normalised; residual ||H u - theta u||
            std::vector<double> ny(k);
            for (int i = 0; i < k; ++i) ny[i] = -y[i];
            cudaMemsetAsync(ritz, 0, sizeof(C) * len, s);
            multiaxpy(Q, k, ny, ritz);
            p.from_spectrum(ritz, tmp, true, sigma, s);
            double uu;
            if ((st = dot(p, tmp, tmp, &uu, s))) return st;
            p.axpby(tmp, tmp, 1.0 / std::sqrt(uu), 0.0, s);
            p.hessvec(phi, tmp, tmp2, s);
            p.axpby(tmp2, tmp, -th, 1.0, s);
            double rr;
            if ((st = dot(p, tmp2, tmp2, &rr, s))) return st;
            theta = th;
            kappa = kap;
            resid = std::sqrt(std::max(rr, 0.0));
            if (vec) p.axpby(vec, tmp, 1.0, 0.0, s);
            if (resid <= o.tol) { converged = true; break; }
        }
        if (last) break;
    }
    info->lambda_min = theta;
    info->kappa_min = kappa;
    info->residual = resid;
    info->steps = steps;
    info->converged = converged;
    if ((st = launch_status("lb_lambda_min"))) return st;
    if (!converged) { err = "lb_lambda_min: step cap reached before the residual tolerance"; return LB_ERR_NOCONV; }
    return LB_OK;
}
template lb_status lb_ctx::lambda_min<float>(Plan<float>&, const float*, const lb_eig_opts&, float*,
                                             lb_eig_info*, cudaStream_t);
template lb_status lb_ctx::lambda_min<double>(Plan<double>&, const double*, const lb_eig_opts&, double*,
                                              lb_eig_info*, cudaStream_t);

// ---------------------------------------------------------------------------------
// PCG for the CONTRACT systems (H + shift I) x = -g, preconditioner (Lambda + shift + c)^{-1},
// c = max(0, mean F''(phi)) = max(0, tau + mean(phi^2)/2) for zero-mean phi.
// ---------------------------------------------------------------------------------
template <typename T>
lb_status lb_ctx::pcg(Plan<T>& p, const T* phi, const T* gvec, double shift, double rtol, int max_iter, T* x,
                      double* xnorm, int* iters, cudaStream_t s) {
    T* r = wbuf<T>(this, 3);
    T* z = wbuf<T>(this, 4);
    T* d = wbuf<T>(this, 5);
    T* ad = wbuf<T>(this, 6);
    lb_status st;
    double pp, gg;
    if ((st = dot(p, phi, phi, &pp, s))) return st;
    const double c = std::max(0.0, prob.tau + 0.5 * pp);
    if ((st = dot(p, gvec, gvec, &gg, s))) return st;
    const double bn = std::sqrt(gg);
    p.axpby(x, gvec, 0.0, 0.0, s);
    p.axpby(r, gvec, -1.0, 0.0, s);
    if (!(bn > 0.0)) { *xnorm = 0.0; *iters = 0; return LB_OK; }
    p.precond(r, z, shift + c, s);
    p.axpby(d, z, 1.0, 0.0, s);
    double rz;
    if ((st = dot(p, r, z, &rz, s))) return st;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        p.hessvec(phi, d, ad, s);
        p.axpby(ad, d, shift, 1.0, s);
        double dad;
        if ((st = dot(p, d, ad, &dad, s))) return st;
        if (!(dad > 0.0)) break;
        const double al = rz / dad;
        p.axpby(x, d, al, 1.0, s);
        p.axpby(r, ad, -al, 1.0, s);
        double rr;
        if ((st = dot(p, r, r, &rr, s))) return st;
        if (std::sqrt(std::max(rr, 0.0)) <= rtol * bn) break;
        p.precond(r, z, shift + c, s);
        double rzn;
        if ((st = dot(p, r, z, &rzn, s))) return st;
        p.axpby(d, z, 1.0, rzn / rz, s);
        rz = rzn;
    }
    double xx;
    if ((st = dot(p, x, x, &xx, s))) return st;
    *xnorm = std::sqrt(std::max(xx, 0.0));
    *iters = it;
    return launch_status("pcg");
}

// A zero-mean field from a continuous distribution supported on the ball ||s|| <= r
// (the randomised start of the hard-case remark): a Gaussian direction, projected and
// normalised, times r U^{1/(N-1)} with U uniform from the same generator.
template <typename T>
lb_status lb_ctx::random_ball(Plan<T>& p, T* out, double r, unsigned long long seed, unsigned stream,
                              cudaStream_t s) {
    lb_status st;
    p.random_normal(out, seed, stream, s);
    p.phys_reduce(R_SUM_SUMSQ, out, nullptr, S_RED1, s);
    double red[2];
    if ((st = sync_read(red, p.slot(S_RED1), 2, s, "random_ball"))) return st;
    const double n = (double)p.n();
    const double mean = red[0] / n;
    p.sub_scalar(out, p.slot(S_RED1), 1.0 / n, s);          // remove the mean (the k = 0 mode)
    const double nrm = std::sqrt(std::max(red[1] / n - mean * mean, 1e-300));
    u32x4 ru = philox4x32_10(u32x4{0xFFFFFFFFu, 0u, stream, 1u}, (unsigned)seed, (unsigned)(seed >> 32));
    const double U = ((double)ru.x + 0.5) / 4294967296.0;
    const double rad = r * std::pow(U, 1.0 / std::max(n - 1.0, 1.0));
    p.axpby(out, out, rad / nrm, 0.0, s);
    return launch_status("random_ball");
}

// ---------------------------------------------------------------------------------
// Algorithm 1 (IMEX-TR, the TRACE outer loop) with CONTRACT (Algorithm 2).
// ---------------------------------------------------------------------------------
namespace {
struct TrState {
    double r, nu, mu, rho_prev;
    bool have_rho;
};
}  // namespace

lb_status lb_ctx::tr_solve(double* v, const lb_tr_opts& o, lb_tr_info* info, cudaStream_t s) {
    Plan<double>& P = *p64;
    double* g = f64[0];
    double* sd = f64[1];
    double* tmp = f64[2];
    const double n = (double)P.n();
    lb_status st;
    TrState S{o.r0, o.nu0, o.mu0, 0.0, false};
    bool random_next = false;
    unsigned rstream = 1;
    P.eta = o.sub.eta;
    if (p32) p32->eta = o.sub.eta;
    info->lambda_min = std::numeric_limits<double>::quiet_NaN();
    const char* tr_env = std::getenv("LBTR_TRACE");
    const bool trace = tr_env && tr_env[0] == '1';   // one JSON line per outer iteration on stderr
    lb_status result = LB_ERR_NOCONV;
    int j = 0, j0 = 0;
    double E = 0.0, gmax = 0.0;
    // the problem and settings a checkpoint of this solve belongs to
    auto ckpt_identity = [&]() {
        TrCheckpoint c;
        c.dim = prob.dim; c.n = prob.n;
        for (int a = 0; a < 3; ++a) c.box[a] = a < prob.dim ? prob.box[a] : 0.0;
        c.xi = prob.xi; c.tau = prob.tau; c.gamma = prob.gamma;
        c.eta = o.sub.eta; c.precision = (int)prec;
        return c;
    };
    if (o.resume && o.checkpoint_path) {
        TrCheckpoint c;
        std::vector<double> field;
        std::string e;
        if (!read_checkpoint(o.checkpoint_path, c, field, e)) { err = "lb_imex_tr_solve: " + e; return LB_ERR_INVALID_ARG; }
        if (!checkpoint_matches(c, ckpt_identity(), e) || (long long)field.size() != P.n()) {
            err = "lb_imex_tr_solve: " + (e.empty() ? std::string("the checkpoint holds another grid") : e);
            return LB_ERR_INVALID_ARG;
        }
        cudaMemcpyAsync(v, field.data(), field.size() * sizeof(double), cudaMemcpyHostToDevice, s);
        cudaError_t ce = cudaStreamSynchronize(s);      // the host copy goes out of scope below
        if (ce != cudaSuccess) { err = std::string("lb_imex_tr_solve: ") + cudaGetErrorString(ce); return LB_ERR_CUDA; }
        S = TrState{c.r, c.nu, c.mu, c.rho_prev, c.have_rho != 0};
        random_next = c.random_next != 0;
        rstream = c.rstream;
        j0 = c.j;
        info->accepted = c.accepted;
        info->contracted = c.contracted;
        info->shrunk = c.shrunk;
        info->randomized = c.randomized;
        info->inner = c.inner;
        info->g1_min = c.g1_min;
        info->sub_stalled = c.sub_stalled;
        info->sub_capped = c.sub_capped;
        info->sub_worst_rel_res = c.sub_worst_rel_res;
    }
    // the state carried into outer iteration `next`, written to the checkpoint files
    auto checkpoint = [&](int next) -> lb_status {
        std::vector<double> field((size_t)P.n());
        cudaMemcpyAsync(field.data(), v, field.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaError_t ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { err = std::string("lb_imex_tr_solve: ") + cudaGetErrorString(ce); return LB_ERR_CUDA; }
        TrCheckpoint c = ckpt_identity();
        c.j = next;
        c.r = S.r; c.nu = S.nu; c.mu = S.mu; c.rho_prev = S.rho_prev; c.have_rho = S.have_rho ? 1 : 0;
        c.random_next = random_next ? 1 : 0; c.rstream = rstream;
        c.accepted = info->accepted; c.contracted = info->contracted; c.shrunk = info->shrunk;
        c.randomized = info->randomized; c.inner = info->inner; c.g1_min = info->g1_min;
        c.sub_stalled = info->sub_stalled; c.sub_capped = info->sub_capped;
        c.sub_worst_rel_res = info->sub_worst_rel_res;
        std::string e;
        if (!write_checkpoint(o.checkpoint_path, c, field.data(), (long long)field.size(), e)) {
            err = "lb_imex_tr_solve: " + e;
            return LB_ERR_INVALID_ARG;
        }
        return LB_OK;
    };
    for (j = j0; j < o.max_outer; ++j) {
        if ((st = energy_grad<double>(P, v, &E, g, &gmax, s))) return st;
        info->energy = E;
        info->gmax = gmax;
        info->outer = j;
        if (gmax < o.eps && !random_next) {
            if (!o.second_order) { result = LB_OK; break; }
            lb_eig_info ei;
            std::memset(&ei, 0, sizeof(ei));
            lb_status es = lambda_min<double>(P, v, o.eig, nullptr, &ei, s);
            if (es != LB_OK && es != LB_ERR_NOCONV) return es;
            info->lambda_min = ei.lambda_min;
            if (ei.lambda_min >= -o.tol2) { result = LB_OK; break; }
            random_next = true;   // a saddle: leave it from a random point of the ball
        }
        if (o.hard_tol > 0.0 && !random_next) {
            // the nearly hard case: g (almost) orthogonal to the eigenvector of a negative
            // lambda_min, which the deterministic start -r g / ||g|| can then never reach
            double* u = f64[7];
            lb_eig_info ei;
            std::memset(&ei, 0, sizeof(ei));
            lb_status es = lambda_min<double>(P, v, o.eig, u, &ei, s);
            if (es != LB_OK && es != LB_ERR_NOCONV) return es;
            double gu = 0.0, uu = 0.0;
            if ((st = dot<double>(P, g, u, &gu, s))) return st;
            if ((st = dot<double>(P, u, u, &uu, s))) return st;
            const double g1 = std::fabs(gu) / std::sqrt(std::max(uu, 1e-300));
            info->lambda_min = ei.lambda_min;
            if (!(g1 >= info->g1_min)) info->g1_min = g1;
            if (ei.lambda_min < 0.0 && g1 <= o.hard_tol) random_next = true;
        }
        // ---- subproblem (Algorithm 3) in the working precision ----
        lb_sub_info si;
        std::memset(&si, 0, sizeof(si));
        lb_status ss;
        if (prec == LB_FP64) {
            double* d0 = nullptr;
            if (random_next) {
                d0 = wbuf<double>(this, 6);
                if ((st = random_ball<double>(P, d0, S.r, o.eig.seed, rstream++, s))) return st;
            }
            ss = subproblem<double>(P, v, g, S.r, d0, o.sub, sd, &si, s);
        } else {
            Plan<float>& Q = *p32;
            float* v32 = reinterpret_cast<float*>(tmp_w[0]);
            float* g32 = reinterpret_cast<float*>(tmp_w[1]);
            float* d32 = reinterpret_cast<float*>(tmp_w[2]);
            const int grid = (int)std::min<long long>(4096, (P.n() + 255) / 256);
            k_convert<float, double><<<grid, 256, 0, s>>>(v32, v, P.n());
            k_convert<float, double><<<grid, 256, 0, s>>>(g32, g, P.n());
            float* d0 = nullptr;
            if (random_next) {
                d0 = wbuf<float>(this, 6);
                if ((st = random_ball<float>(Q, d0, S.r, o.eig.seed, rstream++, s))) return st;
            }
            lb_sub_opts so = o.sub;
            if (!(so.rel_tol > 0.0)) so.rel_tol = 1e-6;
            ss = subproblem<float>(Q, v32, g32, S.r, d0, so, d32, &si, s);
            k_convert<double, float><<<grid, 256, 0, s>>>(sd, d32, P.n());
        }
        if (random_next) ++info->randomized;
        random_next = false;
        if (ss != LB_OK && ss != LB_ERR_NOCONV) return ss;
        info->inner += si.iterations;
        if (!si.converged) {
            if (si.stalled) ++info->sub_stalled;
            else ++info->sub_capped;
            info->sub_worst_rel_res = std::max(info->sub_worst_rel_res, si.rel_residual);
        }
        // project the step onto zero mean in FP64 (P of §3): a float step carries a rounding
        // mean that would otherwise accumulate in the iterate
        P.phys_reduce(R_SUM_SUMSQ, sd, nullptr, S_RED1, s);
        double ss2[2];
        if ((st = sync_read(ss2, P.slot(S_RED1), 2, s, "step"))) return st;
        P.sub_scalar(sd, P.slot(S_RED1), 1.0 / n, s);
        const double smean = ss2[0] / n;
        const double sn2 = ss2[1] / n - smean * smean;
        const double sn = std::sqrt(std::max(sn2, 0.0));
        const double lam = si.lambda;
        if (!(sn > 0.0)) { err = "lb_imex_tr_solve: zero step"; return LB_ERR_NONFINITE; }
        if (j > 0 && S.have_rho && S.rho_prev < o.theta) S.mu = std::max(S.mu, lam / sn);
        // rho_j with the exact expansion E(v+s) - E(v) = <g,s> + G(s) + mean R(v, s)
        double gs;
        if ((st = dot(P, g, sd, &gs, s))) return st;
        P.quad_energy(sd, s);
        double Gs;
        if ((st = sync_read(&Gs, P.slot(S_QUAD), 1, s, "ratio"))) return st;
        P.taylor_rem(v, sd, S_RED1, s);
        double R;
        if ((st = sync_read(&R, P.slot(S_RED1), 1, s, "ratio"))) return st;
        const double drop = -(gs + Gs + R / n);
        const double rho = drop / (sn * sn * sn);
        // lambda <= mu ||s|| in the form of the mu update above (lambda / ||s|| <= mu), so that
        // after that update the test holds exactly as Algorithm 1 intends; the product form
        // can miss by one ulp and the shrink branch would then repeat the same subproblem
        if (rho >= o.theta && (lam / sn <= S.mu || std::fabs(sn - S.nu) <= 1e-12 * S.nu)) {
            P.axpby(v, sd, 1.0, 1.0, s);
            const double nu_new = std::max(S.nu, o.gamma_e * sn);
            S.r = std::min(nu_new, std::max(S.r, o.gamma_e * sn));
            S.mu = std::max(S.mu, lam / sn);
            S.nu = nu_new;
            info->accepted++;
        } else if (rho < o.theta) {
            // CONTRACT (Algorithm 2)
            double gn2;
            if ((st = dot(P, g, g, &gn2, s))) return st;
            const double gn = std::sqrt(gn2);
            auto solve_norm = [&](double shift, double* xn) -> lb_status {
                int it;
                if (prec == LB_FP64)
                    return pcg<double>(P, v, g, shift, o.pcg_rtol, o.pcg_max_iter, tmp, xn, &it, s);
                Plan<float>& Q = *p32;
                return pcg<float>(Q, reinterpret_cast<float*>(tmp_w[0]), reinterpret_cast<float*>(tmp_w[1]), shift,
                                  std::max(o.pcg_rtol, 1e-6), o.pcg_max_iter, reinterpret_cast<float*>(tmp_w[2]),
                                  xn, &it, s);
            };
            double rnew;
            if (lam < o.mu_lo * sn) {
                const double lhat = lam + std::sqrt(o.mu_lo * gn);
                double xn;
                if ((st = solve_norm(lhat, &xn))) return st;
                if (lhat / xn <= o.mu_hi) {
                    rnew = xn;
                } else {
                    double lo = lam, hi = lhat, xm = xn;
                    for (int b = 0; b < 60; ++b) {
                        const double mid = 0.5 * (lo + hi);
                        if ((st = solve_norm(mid, &xm))) return st;
                        const double ratio = mid / xm;
                        if (ratio < o.mu_lo) lo = mid;
                        else if (ratio > o.mu_hi) hi = mid;
                        else break;
                    }
                    rnew = xm;
                }
            } else {
                double xn;
                if ((st = solve_norm(o.gamma_lam * lam, &xn))) return st;
                rnew = xn >= o.gamma_c * sn ? xn : o.gamma_c * sn;
            }
            S.r = rnew;
            info->contracted++;
        } else {
            S.r = std::min(S.nu, lam / S.mu);
            info->shrunk++;
        }
        S.rho_prev = rho;
        S.have_rho = true;
        if (trace)
            std::fprintf(stderr,
                         "{\"j\": %d, \"E\": %.15g, \"gmax\": %.3e, \"r\": %.6g, \"nu\": %.6g, \"mu\": %.6g, "
                         "\"lambda\": %.6g, \"snorm\": %.6g, \"rho\": %.6g, \"inner\": %d, \"sub_status\": %d, "
                         "\"sub_stalled\": %d, \"sub_rel_res\": %.3e, "
                         "\"acc\": %d, \"con\": %d, \"shr\": %d}\n",
                         j, E, gmax, S.r, S.nu, S.mu, lam, sn, rho, si.iterations, (int)ss, si.stalled, si.rel_residual,
                         info->accepted,
                         info->contracted, info->shrunk);
        if (o.checkpoint_path && o.checkpoint_every > 0 && (j + 1) % o.checkpoint_every == 0)
            if ((st = checkpoint(j + 1))) return st;
    }
    info->outer = j;
    if (result != LB_OK) {
        // final energy at the last iterate
        if ((st = energy_grad<double>(P, v, &E, g, &gmax, s))) return st;
        info->energy = E;
        info->gmax = gmax;
        err = "lb_imex_tr_solve: outer iteration cap reached";
    }
    return result;
}

// ---------------------------------------------------------------------------------
// Semi-implicit gradient flow: phi <- phi - dt (I + dt Lambda)^{-1} g(phi), i.e. the
// preconditioner of the CONTRACT solves at shift 1/dt applied to g and subtracted
// (dt (I + dt Lambda)^{-1} = (Lambda + 1/dt)^{-1}); FP64.
// ---------------------------------------------------------------------------------
lb_status lb_ctx::sis_solve(double* phi, const lb_sis_opts& o, lb_sis_info* info, cudaStream_t s) {
    Plan<double>& p = *p64;
    double* g = f64[0];
    double* z = f64[1];
    lb_status st;
    double e = 0.0, gm = 0.0;
    info->steps = 0;
    if ((st = energy_grad(p, (const double*)phi, &e, g, &gm, s))) return st;
    const int ce = std::max(1, o.check_every);
    int steps = 0;
    while (!(gm < o.eps) && steps < o.max_steps) {
        p.precond(g, z, 1.0 / o.dt, s);
        p.axpby(phi, z, -1.0, 1.0, s);
        ++steps;
        if (steps % ce == 0 || steps == o.max_steps) {
            if ((st = energy_grad(p, (const double*)phi, &e, g, &gm, s))) break;
        } else {
            p.energy_grad(phi, g, s);
            if ((st = launch_status("lb_sis_solve"))) break;
        }
    }
    info->steps = steps;
    info->energy = e;
    info->gmax = gm;
    if (st) return st;
    if (!(gm < o.eps)) { err = "lb_sis_solve: step cap reached"; return LB_ERR_NOCONV; }
    return LB_OK;
}
