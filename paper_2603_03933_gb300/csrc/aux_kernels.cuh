// Secular-equation solve, physical-space reductions and elementwise kernels.
#pragma once
#include "common.cuh"
#include "reduce.cuh"

namespace lbtr {

// Device-side state of one subproblem solve (Algorithm 3).
struct ImexState {
    double lam;          // multiplier of the next iterate d_{j+1} = B[j&1] / (1 + eta (Lambda + lam))
    double final_lam;    // multiplier of the returned iterate
    double residual;     // ||g + (H + lam I) d|| of the last checked iterate
    double bnorm2;       // ||b_j||^2 of the last iterate
    long long newton;    // Newton steps summed
    int it;              // iterations completed
    int done;            // 0 running, 1 converged, 2 iteration cap, 3 non-finite, 4 stalled
    int final_src;       // which B buffer holds b_{j-1} of the returned iterate
    int pad;
    double best2;        // smallest (eta residual)^2 seen by the stall test, and its iteration
    int best_it;         //   (0: none yet)
    int pad2;
};

// Stall test of the float inner iteration: the residual counts as improved when it falls
// below 0.98 of the best squared value so far; no improvement in `k` checked iterations
// (k > 0) ends the iteration.  Returns the stall flag and updates (best2, best_it).
__device__ __forceinline__ bool stall_update(int k, int j, double res2, double& best2, int& best_it) {
    if (k <= 0) return false;
    const bool stall = best_it > 0 && j - best_it > k;
    if (best_it == 0 || res2 < 0.98 * best2) { best2 = res2; best_it = j; }
    return stall;
}

template <typename T> struct SecArgs {
    const cplx<T>* bmain;     // b_j (unnormalised DFT), zero k = 0
    const cplx<T>* bnyq;
    const T* qtab;            // [3][M] (2 pi / L_a)^2 wavenum^2
    const double* res;        // reduction results of the IMEX_OUT pass: [0] sum w|db|^2/N^2, [1] sum w|b|^2/N^2
    ImexState* st;
    double* partials;         // [2][3][gridDim]
    GridBar bar;
    int dim, m, rows;
    double inv_n2;            // 1/N^2
    double eta, r, rtol, steptol;
    double eps_abs, eps_rel_abs;  // stop when residual < max(eps_abs, eps_rel_abs)
    int stall;                // or after this many checked iterations without progress (0: off)
    int check;                // 0 on the initial call (no iterate to check)
    int max_iter;
    T xi2;
};

// phi(lam) = sum_i c_i / (a_i + eta lam)^2 and its derivative (the function before
// eq. lambda_update_rule), with c_i = w |B_i|^2 / N^2, a_i = 1 + eta Lambda_i, over
// this block's share of the spectrum.  With zero0 it also returns phi(0).
template <typename T, bool ZERO0>
__device__ void secular_terms(const SecArgs<T>& a, const T* qt, double lam, double out[3]) {
    const int H = a.m >> 1;
    const long long nmain = (long long)a.rows * H;
    const long long ntot = nmain + a.rows;
    const T el = (T)(a.eta * lam), eta = (T)a.eta;
    const T n2 = (T)a.inv_n2;
    Acc<T> s0, s1, s2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ntot;
         i += (long long)gridDim.x * blockDim.x) {
        int kx, row;
        cplx<T> b;
        T w;
        if (i < nmain) { kx = (int)(i % H); row = (int)(i / H); b = a.bmain[i]; w = kx ? (T)2 : (T)1; }
        else { kx = H; row = (int)(i - nmain); b = a.bnyq[row]; w = (T)1; }
        T bk2;
        if (a.dim == 3) bk2 = qt[kx] + qt[a.m + (row % a.m)] + qt[2 * a.m + row / a.m];
        else bk2 = qt[kx] + qt[a.m + row];
        T t = (T)1 - bk2;
        T aa = (T)1 + eta * a.xi2 * t * t;
        T c = w * (b.x * b.x + b.y * b.y) * n2;
        T den = aa + el;
        T q = c / (den * den);
        s1.add(q);
        s2.add((T)-2 * eta * q / den);
        if (ZERO0) s0.add(c / (aa * aa));
    }
    __shared__ double scr[3 * 32];
    Acc<T> acc3[3] = {s0, s1, s2};
    block_sum<T, 3>(acc3, scr, out);
}

// Sum the per-block partials of quantity set `buf` (identical order in every block).
__device__ __forceinline__ void sum_partials(const double* p, int nq, double* out) {
    __shared__ double tot[3];
    if (threadIdx.x < 32) {
        for (int q = 0; q < nq; ++q) {
            double s = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += ((volatile const double*)p)[q * gridDim.x + b];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (threadIdx.x == 0) tot[q] = s;
        }
    }
    __syncthreads();
    for (int q = 0; q < nq; ++q) out[q] = tot[q];
    __syncthreads();
}

// One Newton step towards the root of phi(lambda) = r^2 (eq. lambda_update_rule), taken on
// the equivalent equation psi(lambda) = phi(lambda)^(-1/2) - 1/r = 0, which has the same
// root.  For phi = sum_i c_i / (a_i + eta lambda)^2 with a_i > 0, psi is increasing and
// concave (the secular-equation argument of More and Sorensen, 1983) and exactly linear
// when one term dominates, so from the left the step never overshoots and from a warm
// start near the root one or two steps reach the tolerance.  With psi' = -phi' phi^(-3/2) / 2
// the step is lambda + 2 phi (1 - sqrt(phi) / r) / phi'; it is clamped at 0.
__device__ __forceinline__ double secular_newton_step(double lam, double phi, double dphi, double r) {
    double ln = lam + 2.0 * phi * (1.0 - sqrt(phi) / r) / dphi;
    if (!isfinite(ln)) ln = lam - (phi - r * r) / dphi;
    return ln > 0.0 ? ln : 0.0;
}

// Convergence check of the iterate d_j (residual identity g + (H + lam_j) d_j =
// (b_{j-1} - b_j)/eta, which follows from eq. imex-scheme), then the lambda rule of
// eq. lambda_update_rule for the next iterate: lam = 0 if phi(0) <= r^2, else Newton
// (secular_newton_step) from the previous multiplier instead of 0; the root is the same,
// phi being decreasing.
template <typename T>
__global__ void k_secular(SecArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* qt = reinterpret_cast<T*>(smem_raw);
    for (int i = threadIdx.x; i < 3 * a.m; i += blockDim.x) qt[i] = a.qtab[i];
    __syncthreads();
    ImexState* st = a.st;
    if (*(volatile int*)&st->done) return;
    const double lam_prev = st->lam;
    const int j = st->it + 1;          // iteration that produced b_j (device-side count)
    double best2 = st->best2;
    int best_it = st->best_it;
    if (a.check) {
        double res = sqrt(fmax(a.res[0], 0.0)) / a.eta;
        bool bad = !isfinite(res) || !isfinite(a.res[1]);
        const bool stall = stall_update(a.stall, j, a.res[0], best2, best_it);
        const bool conv = res < a.eps_abs || res < a.eps_rel_abs;
        if (bad || conv || stall || j >= a.max_iter) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->residual = res;
                st->bnorm2 = a.res[1];
                st->final_lam = lam_prev;
                st->final_src = (j - 1) & 1;
                st->it = j;
                st->done = bad ? 3 : conv ? 1 : stall ? 4 : 2;
            }
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) { st->residual = res; st->bnorm2 = a.res[1]; }
    }
    const double r2 = a.r * a.r;
    double part[3];
    int stepi = 0;
    secular_terms<T, true>(a, qt, lam_prev, part);
    double* P = a.partials;
    const int G = gridDim.x;
    if (threadIdx.x == 0) for (int q = 0; q < 3; ++q) P[(stepi & 1) * 3 * G + q * G + blockIdx.x] = part[q];
    if (!grid_sync(a.bar)) return;
    double tot[3];
    sum_partials(P + (stepi & 1) * 3 * G, 3, tot);
    ++stepi;
    double lam = 0.0;
    long long newton = 0;
    if (!(tot[0] <= r2)) {
        lam = lam_prev;
        double phi = tot[1], dphi = tot[2];
        if (lam_prev == 0.0) { phi = tot[0]; dphi = tot[2]; }
        for (int it = 0; it < 60; ++it) {
            if (fabs(phi - r2) <= a.rtol * r2) break;
            const double ln = secular_newton_step(lam, phi, dphi, a.r);
            ++newton;
            bool small = fabs(ln - lam) <= a.steptol * (1.0 + ln);
            lam = ln;
            if (small) break;
            secular_terms<T, false>(a, qt, lam, part);
            if (threadIdx.x == 0) for (int q = 0; q < 3; ++q) P[(stepi & 1) * 3 * G + q * G + blockIdx.x] = part[q];
            if (!grid_sync(a.bar)) return;
            sum_partials(P + (stepi & 1) * 3 * G, 3, tot);
            ++stepi;
            phi = tot[1];
            dphi = tot[2];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {       // after the grid barriers: every block has read st
        st->lam = lam;
        st->newton += newton;
        if (a.check) { st->it = j; st->best2 = best2; st->best_it = best_it; }
    }
}

// ---- physical-space reductions --------------------------------------------------
enum RedOp { R_DOT = 0, R_SUMSQ_MAX = 1, R_SUM_SUMSQ = 2, R_POW23 = 3 };

template <typename T> struct PhysRedArgs {
    const T* x;
    const T* y;
    long long n;
    RedSlot red;
};

// R_DOT: [0] sum x y.  R_SUMSQ_MAX: [0] sum x^2, [1] max |x|.  R_SUM_SUMSQ: [0] sum x, [1] sum x^2.
// R_POW23: [0] sum x^2, [1] sum x^3.
template <typename T, int OP>
__global__ void k_physred(PhysRedArgs<T> a) {
    __shared__ double scr[64];
    Acc<T> acc[2];
    double mx = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
         i += (long long)gridDim.x * blockDim.x) {
        T x = a.x[i];
        if (OP == R_DOT) acc[0].add(x * a.y[i]);
        else if (OP == R_SUMSQ_MAX) { acc[0].add(x * x); mx = fmax(mx, fabs((double)x)); }
        else if (OP == R_POW23) { acc[0].add(x * x); acc[1].add(x * x * x); }
        else { acc[0].add(x); acc[1].add(x * x); }
    }
    double tot[2];
    if (OP == R_SUMSQ_MAX) {
        block_sum<T, 1>(*reinterpret_cast<Acc<T>(*)[1]>(&acc[0]), scr, tot);
        double m = block_max(mx, scr);
        if (threadIdx.x == 0) tot[1] = m;
    } else if (OP == R_DOT) {
        block_sum<T, 1>(*reinterpret_cast<Acc<T>(*)[1]>(&acc[0]), scr, tot);
    } else {
        block_sum<T, 2>(acc, scr, tot);
    }
    finalize_partials(a.red, tot);
}

// y = alpha x + beta y  (alpha, beta from device scalars when non-null pointers given)
template <typename T>
__global__ void k_axpby(T* y, const T* x, double alpha, double beta, const double* alpha_dev,
                        double alpha_dev_scale, long long n) {
    double al = alpha_dev ? (*alpha_dev) * alpha_dev_scale : alpha;
    T a = (T)al, b = (T)beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + (beta == 0.0 ? (T)0 : b * y[i]);
}

// y -= (*c) * scale  (a device scalar, e.g. a mean from a reduction slot)
template <typename T>
__global__ void k_sub_scalar(T* y, const double* c, double scale, long long n) {
    const T v = (T)(*c * scale);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] -= v;
}

// Precision conversion and shift: dst = (TD)src + add (add may be null)
template <typename TD, typename TS>
__global__ void k_convert(TD* dst, const TS* src, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (TD)src[i];
}

// Spectrum-space weighted multi-dot for Lanczos re-orthogonalisation:
// out[j] = sum_k w_k Re(conj(Q_j,k) x_k) (* sc), optionally with weight 1/(Lambda+sigma).
template <typename T> struct SpecDotArgs {
    const cplx<T>* q;       // [nvec][len] vectors (main followed by nyq, len = rows*(H+1))
    const cplx<T>* x;
    long long len;          // rows * (H + 1)
    int nvec;
    int dim, m, rows;
    const T* qtab;
    T xi2, sigma;
    int minv;               // 1: weight by 1/(Lambda + sigma)
    double* partials;       // [nvec][gridDim]
    double* out;            // [nvec]
    unsigned* ticket;
};

}  // namespace lbtr
