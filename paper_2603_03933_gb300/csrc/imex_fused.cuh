// One IMEX iteration's reciprocal-space work in a single cooperative kernel.
//
// The CTAs of a cooperative grid own fixed tiles of columns of the innermost axis
// (z in 3D, y in 2D) and keep them in shared memory across grid barriers:
//   1. forward transform of b_j's columns, k = 0 removed; b_j stored for the next
//      residual; ||b_{j-1} - b_j||^2 / eta^2 (the Algorithm 3 residual of d_j, by the
//      identity g + (H + lambda_j I) d_j = (b_{j-1} - b_j) / eta) and the secular sums
//      at lambda = 0 and at the previous multiplier are reduced over the grid;
//   2. the convergence test of Algorithm 3; then the multiplier rule of
//      eq. lambda_update_rule (Newton on phi(lambda) = r^2), each Newton step a sum over
//      the register-resident terms c_i = w_i |b_i|^2 / N^2 and a_i = 1 + eta Lambda_i;
//   3. d_{j+1} = b_j / (1 + eta (Lambda + lambda_{j+1})) (eq. imex-scheme) in place and the
//      inverse transform of the columns, written for the next x/y pass.
// Each spectrum element is read from and written to HBM once per iteration here,
// instead of three separate passes plus a re-read per Newton step.
#pragma once
#include "aux_kernels.cuh"
#include "passes.cuh"
#include "lines.cuh"

namespace lbtr {

template <typename T> struct ZfArgs {
    cplx<T>* work;            // in: b_j after the outer transforms; out: d_{j+1} after the inner inverse
    const cplx<T>* bold;      // b_{j-1} (fully transformed)
    cplx<T>* bnew;            // b_j (fully transformed) is written here
    const cplx<T>* tw;
    const T* qtab;
    ColSeg seg[2];
    int nb_main;              // main-segment tiles
    int ntiles;               // all tiles
    int dim, m;
    ImexState* st;
    double* partials;         // [2][NQ][gridDim]
    GridBar bar;
    T xi2, eta;
    double inv_n, inv_n2;
    double r, rtol, steptol, eps_abs, eps_rel_abs;
    int stall;                // also stop after this many checked iterations without progress (0: off)
    int check, max_iter;
    long long spec_half;      // rows * H: offset of nyq within a spectrum
    // the tests of each step in the working precision (k_imex_lines)
    T t_thr_abs2, t_thr_rel2; // (eps_abs eta)^2, (eps_rel_abs eta)^2: residual^2 eta^2 below either = converged
    T t_r2, t_rtol_r2;        // r^2 and rtol r^2 of the multiplier rule
    T t_inv_n2;
};

__host__ __device__ constexpr int zf_nt(int m, int tpc) { return 2 * m * tpc > 1024 ? 1024 : 2 * m * tpc; }
template <typename T> __host__ __device__ constexpr size_t zf_smem(int m, int tpc) {
    return sizeof(cplx<T>) * ((size_t)m + (size_t)m * (16 * tpc + 1)) + 3 * (size_t)m * sizeof(T) + 256 * sizeof(double);
}

template <typename T, int M, int TPC>
__global__ void __launch_bounds__(zf_nt(M, TPC)) k_imex_zfused(ZfArgs<T> a) {
    constexpr int NL = 16 * TPC, NT = zf_nt(M, TPC), LD = NL + 1, H = M / 2;
    constexpr int ESTEP = NT / NL, IT = M / ESTEP;
    constexpr int HSH = (H >= 256) ? 8 : (H >= 128) ? 7 : (H >= 64) ? 6 : (H >= 32) ? 5 : (H >= 16) ? 4 : (H >= 8) ? 3 : 2;
    static_assert(NT % NL == 0 && M % ESTEP == 0, "tile mapping");
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + M;
    T* qt = reinterpret_cast<T*>(buf + M * LD);
    double* red = reinterpret_cast<double*>(qt + 3 * M);
    ImexState* st = a.st;
    if (*(volatile int*)&st->done) return;
    const C zero = mk<T>((T)0, (T)0);

    // this thread's line: tile q of the CTA, line l within the tile
    const int Lloc = threadIdx.x % NL;
    const int e0 = threadIdx.x / NL;
    const int q = Lloc / 16, l = Lloc % 16;
    const int gt = blockIdx.x * TPC + q;
    const int segi = gt < a.nb_main ? 0 : 1;
    const ColSeg s = a.seg[segi];
    const int l0 = (segi == 0 ? gt : gt - a.nb_main) * 16;
    const bool ok = gt < a.ntiles && (l0 + l) < s.nlines;
    const long long lmask = (1LL << s.lg_shift) - 1;
    const int Lg = l0 + l;
    const long long base = ok ? (long long)(Lg >> s.lg_shift) * s.lhi + (long long)(Lg & lmask) * s.llo : 0;
    const long long soff = segi == 0 ? 0 : a.spec_half;

    // 1. loads: b_j columns (work) and b_{j-1} (bold), all issued up front
    C v[IT], old[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int e = e0 + t * ESTEP;
        const long long ad = soff + base + (long long)e * s.es;
        v[t] = ok ? a.work[ad] : zero;
        old[t] = (ok && a.check) ? a.bold[ad] : zero;
    }
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
    for (int i = threadIdx.x; i < 3 * M; i += NT) qt[i] = a.qtab[i];
#pragma unroll
    for (int t = 0; t < IT; ++t) buf[(e0 + t * ESTEP) * LD + Lloc] = v[t];
    __syncthreads();
    fft_lines<T, -1, M, NL, NT>(buf, tw, M);

    // 2. residual, secular terms, store b_j
    const T eta = a.eta, n2 = (T)a.inv_n2;
    const double lam_prev = st->lam;
    const int j = st->it + 1;
    double best2 = st->best2;          // read before the first barrier; block 0 writes after it
    int best_it = st->best_it;
    T cc[IT], aa[IT];
    Acc<T> acc[5];
    const T elp = (T)(a.eta * lam_prev);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int e = e0 + t * ESTEP;
        C x = buf[e * LD + Lloc];
        const int kx = s.kx_const >= 0 ? s.kx_const : (Lg & (H - 1));
        T by, bz;
        bool zo;
        if (a.dim == 3) {
            const int y = s.kx_const >= 0 ? Lg : (Lg >> HSH);
            by = qt[M + y];
            bz = qt[2 * M + e];
            zo = (y == 0);
        } else {
            by = qt[M + e];
            bz = (T)0;
            zo = true;
        }
        const T wgt = (s.kx_const < 0 && kx > 0) ? (T)2 : (T)1;
        const bool is0 = (s.kx_const < 0) && kx == 0 && zo && e == 0;
        if (is0 || !ok) x = zero;
        buf[e * LD + Lloc] = x;
        const T tt = (T)1 - (qt[kx] + by + bz);
        const T ai = (T)1 + eta * a.xi2 * tt * tt;
        const T ci = ok ? wgt * (x.x * x.x + x.y * x.y) * n2 : (T)0;
        cc[t] = ci;
        aa[t] = ai;
        if (ok) {
            const T dx = old[t].x - x.x, dy = old[t].y - x.y;
            acc[0].add(wgt * (dx * dx + dy * dy));
            acc[1].add(wgt * (x.x * x.x + x.y * x.y));
            const T den = ai + elp;
            const T qv = ci / (den * den);
            acc[2].add(ci / (ai * ai));
            acc[3].add(qv);
            acc[4].add((T)-2 * eta * qv / den);
            a.bnew[soff + base + (long long)e * s.es] = x;
        }
    }
    double tot[5];
    block_sum<T, 5>(acc, red, tot);
    double* P = a.partials;
    const int G = gridDim.x;
    int stepi = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) P[(stepi & 1) * 5 * G + k * G + blockIdx.x] = tot[k];
    if (!grid_sync(a.bar)) return;
    double sums[5];
    {
        __shared__ double sh[5];
        if (threadIdx.x < 32) {
            for (int k = 0; k < 5; ++k) {
                double x = 0.0;
                for (int b = threadIdx.x; b < G; b += 32) x += ((volatile double*)P)[(stepi & 1) * 5 * G + k * G + b];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
                if (threadIdx.x == 0) sh[k] = x;
            }
        }
        __syncthreads();
        for (int k = 0; k < 5; ++k) sums[k] = sh[k] * (k < 2 ? a.inv_n2 : 1.0);
        __syncthreads();
    }
    ++stepi;

    // convergence of d_j (skipped on the initial call, which only sets up lambda_1)
    if (a.check) {
        const double res = sqrt(fmax(sums[0], 0.0)) / a.eta;
        const bool bad = !isfinite(res) || !isfinite(sums[1]);
        const bool stall = stall_update(a.stall, j, sums[0], best2, best_it);
        if (blockIdx.x == 0 && threadIdx.x == 0) { st->best2 = best2; st->best_it = best_it; }
        const bool conv = res < a.eps_abs || res < a.eps_rel_abs;
        if (bad || conv || stall || j >= a.max_iter) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->residual = res;
                st->bnorm2 = sums[1];
                st->final_lam = lam_prev;
                st->final_src = (j - 1) & 1;
                st->it = j;
                st->done = bad ? 3 : conv ? 1 : stall ? 4 : 2;
            }
            return;
        }
    }

    // the multiplier rule: 0 if phi(0) <= r^2, else Newton from the previous multiplier
    const double r2 = a.r * a.r;
    double lam = 0.0;
    long long newton = 0;
    if (!(sums[2] <= r2)) {
        lam = lam_prev;
        double phi = lam_prev == 0.0 ? sums[2] : sums[3], dphi = sums[4];
        for (int it = 0; it < 60; ++it) {
            if (fabs(phi - r2) <= a.rtol * r2) break;
            const double ln = secular_newton_step(lam, phi, dphi, a.r);
            ++newton;
            const bool small = fabs(ln - lam) <= a.steptol * (1.0 + ln);
            lam = ln;
            if (small) break;
            const T el = (T)(a.eta * lam);
            Acc<T> ac2[2];
#pragma unroll
            for (int t = 0; t < IT; ++t) {
                const T den = aa[t] + el;
                const T qv = cc[t] / (den * den);
                ac2[0].add(qv);
                ac2[1].add((T)-2 * eta * qv / den);
            }
            double t2[2];
            block_sum<T, 2>(ac2, red, t2);
            if (threadIdx.x == 0) {
                P[(stepi & 1) * 5 * G + 0 * G + blockIdx.x] = t2[0];
                P[(stepi & 1) * 5 * G + 1 * G + blockIdx.x] = t2[1];
            }
            if (!grid_sync(a.bar)) return;
            __shared__ double sh2[2];
            if (threadIdx.x < 32) {
                for (int k = 0; k < 2; ++k) {
                    double x = 0.0;
                    for (int b = threadIdx.x; b < G; b += 32) x += ((volatile double*)P)[(stepi & 1) * 5 * G + k * G + b];
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
                    if (threadIdx.x == 0) sh2[k] = x;
                }
            }
            __syncthreads();
            phi = sh2[0];
            dphi = sh2[1];
            __syncthreads();
            ++stepi;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->lam = lam;
        st->newton += newton;
        if (a.check) {
            st->it = j;
            st->residual = sqrt(fmax(sums[0], 0.0)) / a.eta;
            st->bnorm2 = sums[1];
        }
    }

    // 3. the implicit diagonal solve and the inverse transform of the columns
    const T el = (T)(a.eta * lam);
    const T ks = (T)a.inv_n;
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int e = e0 + t * ESTEP;
        C x = buf[e * LD + Lloc];
        const T f = ks / (aa[t] + el);
        buf[e * LD + Lloc] = mk<T>(x.x * f, x.y * f);
    }
    __syncthreads();
    fft_lines<T, +1, M, NL, NT>(buf, tw, M);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int e = e0 + t * ESTEP;
        if (ok) a.work[soff + base + (long long)e * s.es] = buf[e * LD + Lloc];
    }
}


// ---------------------------------------------------------------------------------
// The same iteration with the columns held in registers as four-step line transforms
// (the layout of k_lines): one cooperative grid of TPC tiles of LN_NL lines per CTA, every
// tile of the spectrum resident at once.  Thread (l, i) of a tile keeps the L1 elements of
// line l that the forward transform leaves with it, with their a = 1 + eta Lambda, across
// the grid barriers of the multiplier rule (c = w |b|^2 / N^2 is recomputed from them).
// The scalar part of each barrier step (the Algorithm 3 test, the Newton update of the
// multiplier) runs in one thread per CTA and reaches the others through shared memory;
// every CTA reads the same partial sums in the same order, so all take the same decision.
// ---------------------------------------------------------------------------------
__host__ __device__ constexpr int zl_nt(int m, int tpc) { return LN_NL * fs_l2(m) * tpc; }
template <typename T> __host__ __device__ constexpr size_t zl_smem(int m, int tpc) {
    return 2 * (size_t)tpc * LN_NL * (m + 1) * sizeof(cplx<T>) + 32 * 5 * sizeof(double);
}

// Newton update of the multiplier (secular_newton_step) with the stopping tests of the
// rule; true if phi and phi' at the new lambda are needed for another step
struct NewtonState {
    double lam, r, r2, rtol, steptol;
    long long newton;
    int steps;
};
__device__ __forceinline__ bool newton_update(NewtonState& ns, double phi, double dphi) {
    if (ns.steps >= 60) return false;
    if (fabs(phi - ns.r2) <= ns.rtol * ns.r2) return false;
    const double ln = secular_newton_step(ns.lam, phi, dphi, ns.r);
    ++ns.newton;
    ++ns.steps;
    const bool small = fabs(ln - ns.lam) <= ns.steptol * (1.0 + ln);
    ns.lam = ln;
    return !small;
}

// correctly rounded reciprocal in the working precision
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

template <typename T, int M, int TPC>
__global__ void __launch_bounds__(zl_nt(M, TPC), TPC == 1 ? 4 : 1) k_imex_lines(ZfArgs<T> a) {
    constexpr int NL = LN_NL, L1 = fs_l1(M), L2 = fs_l2(M), RR = L1 / L2, TS = M + 1, H = M / 2;
    constexpr int NTT = NL * L2;            // threads per tile
    constexpr int HSH = (H >= 256) ? 8 : (H >= 128) ? 7 : (H >= 64) ? 6 : (H >= 32) ? 5 : (H >= 16) ? 4 : (H >= 8) ? 3 : 2;
    static_assert((1 << HSH) == H, "H must be a power of two");
    enum { ACT_RETURN = 0, ACT_EVAL = 1, ACT_SOLVE = 2 };
    using C = cplx<T>;
    ImexState* st = a.st;
    if (*(volatile int*)&st->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int q = threadIdx.x / NTT, lt = threadIdx.x % NTT;
    C* TA = reinterpret_cast<C*>(smem_raw) + (size_t)q * 2 * NL * TS;
    C* TB = TA + NL * TS;
    double* red = reinterpret_cast<double*>(reinterpret_cast<C*>(smem_raw) + (size_t)TPC * 2 * NL * TS);
    __shared__ double s_lam, s_lamp;
    __shared__ T s_el, s_elp;
    __shared__ int s_act;
    __shared__ Part<T> sh[5];
    __shared__ NewtonState ns;
    __shared__ double s_best2;
    __shared__ int s_best_it;
    if (threadIdx.x == 0) {            // state of iteration j, read before block 0 updates it
        s_lamp = st->lam;
        s_elp = (T)(a.eta * s_lamp);
        s_best2 = st->best2;
        s_best_it = st->best_it;
    }
    const int l = lt % NL, i = lt / NL;
    const C zero = mk<T>((T)0, (T)0);
    const T* __restrict__ qt = a.qtab;

    // this thread's line
    const int tile = blockIdx.x * TPC + q;
    const int segi = tile < a.nb_main ? 0 : 1;
    const ColSeg& s = a.seg[segi];
    const int L = (tile - (segi ? a.nb_main : 0)) * NL + l;
    const bool ok = tile < a.ntiles && L < s.nlines;
    const long long lmask = (1LL << s.lg_shift) - 1;
    const long long base = (ok ? (long long)(L >> s.lg_shift) * s.lhi + (long long)(L & lmask) * s.llo : 0) +
                           (segi ? a.spec_half : 0);
    const long long es = s.es;
    auto fo = [&](int m) { return i + L2 * (m / L2) + L1 * (m % L2); };   // element in slot m after the forward

    // 1. b_j in the forward-input layout
    C v[L1];
#pragma unroll
    for (int m = 0; m < L1; ++m) v[m] = ok ? a.work[base + (long long)(i + L2 * m) * es] : zero;

    // 2. forward transform of the columns
    dft_r<-1, L1, T>(v);
#pragma unroll
    for (int m = 1; m < L1; ++m) v[m] = cmul(v[m], __ldg(&a.tw[i * m]));
#pragma unroll
    for (int m = 0; m < L1; ++m) TA[l * TS + m * L2 + i] = v[m];
    __syncthreads();
    // b_{j-1} in the forward-output layout (in flight during the second half of the transform)
    C old[L1];
#pragma unroll
    for (int m = 0; m < L1; ++m) old[m] = (ok && a.check) ? a.bold[base + (long long)fo(m) * es] : zero;
#pragma unroll
    for (int sb = 0; sb < RR; ++sb) {
        const int aq = i + L2 * sb;
#pragma unroll
        for (int jj = 0; jj < L2; ++jj) v[sb * L2 + jj] = TA[l * TS + aq * L2 + jj];
        dft_r<-1, L2, T>(&v[sb * L2]);
    }

    // 3. zero k = 0, store b_j, residual and secular sums
    const int kx = s.kx_const >= 0 ? s.kx_const : (L & (H - 1));
    T byz;
    bool zo;
    if (a.dim == 3) {
        const int y = s.kx_const >= 0 ? L : (L >> HSH);
        byz = qt[kx] + qt[M + y];
        zo = (y == 0);
    } else {
        byz = qt[kx];
        zo = true;
    }
    const T wgt = (s.kx_const < 0 && kx > 0) ? (T)2 : (T)1;
    const bool k0line = (s.kx_const < 0) && kx == 0 && zo;
    const T* qe = qt + (a.dim == 3 ? 2 * M : M);
    const T eta = a.eta;
    const int j = st->it + 1;
    const T elp = s_elp;
    T aa[L1];
    const T cw = wgt * a.t_inv_n2;
    // per-thread sums in two interleaved halves (pairwise), then float-float over the grid
    T sm0[2][5] = {};
#pragma unroll
    for (int m = 0; m < L1; ++m) {
        const int e = fo(m);
        C x = v[m];
        if (!ok || (k0line && e == 0)) x = zero;
        v[m] = x;
        const T tt = (T)1 - (byz + qe[e]);
        const T ai = (T)1 + eta * a.xi2 * tt * tt;
        const T x2 = x.x * x.x + x.y * x.y;
        const T ci = cw * x2;
        aa[m] = ai;
        if (ok) {
            const T dx = old[m].x - x.x, dy = old[m].y - x.y;
            const T rd = rcp_t(ai + elp), ra = rcp_t(ai);
            const T qv = ci * rd * rd;
            sm0[m & 1][0] += wgt * (dx * dx + dy * dy);
            sm0[m & 1][1] += wgt * x2;
            sm0[m & 1][2] += ci * ra * ra;
            sm0[m & 1][3] += qv;
            sm0[m & 1][4] += (T)-2 * eta * qv * rd;
        }
    }
    Part<T>* P = reinterpret_cast<Part<T>*>(a.partials);
    const int G = gridDim.x;
    {
        Acc<T> acc[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) { acc[k].add(sm0[0][k]); acc[k].add(sm0[1][k]); }
        Part<T> tot[5];
        block_part<T, 5>(acc, red, tot);
        if (!grid_reduce_sync<T, 5>(a.bar, tot, P, P + 5 * G, P + 5 * G + 5 * 64, sh)) return;
    }
    if (threadIdx.x == 0) {
        // the tests of every iteration in the working precision; double only for Newton steps
        const T res2 = part_to_T(sh[0], T()) * a.t_inv_n2;        // (eta * residual)^2
        const T bn2 = part_to_T(sh[1], T()) * a.t_inv_n2;
        int act = ACT_SOLVE;
        // convergence of d_j (not on the initial call, which only sets up lambda_1)
        if (a.check) {
            const bool bad = !isfinite(res2) || !isfinite(bn2);
            double best2 = s_best2;
            int best_it = s_best_it;
            const bool stall = stall_update(a.stall, j, (double)res2, best2, best_it);
            if (blockIdx.x == 0) { st->best2 = best2; st->best_it = best_it; }
            const bool conv = res2 < a.t_thr_abs2 || res2 < a.t_thr_rel2;
            if (bad || conv || stall || j >= a.max_iter) {
                if (blockIdx.x == 0) {
                    st->residual = (double)(sqrt(res2 > (T)0 ? res2 : (T)0) / eta);
                    st->bnorm2 = (double)bn2;
                    st->final_lam = s_lamp;
                    st->final_src = (j - 1) & 1;
                    st->it = j;
                    st->done = bad ? 3 : conv ? 1 : stall ? 4 : 2;
                }
                act = ACT_RETURN;
            }
        }
        if (act != ACT_RETURN) {
            // the multiplier rule: 0 if phi(0) <= r^2, else the root of phi = r^2 by Newton
            // from the previous multiplier (no step when that one already meets the tolerance)
            ns.newton = 0;
            ns.steps = 0;
            s_el = elp;
            s_lam = s_lamp;
            if (part_to_T(sh[2], T()) <= a.t_r2) {
                s_lam = 0.0;
                s_el = (T)0;
            } else {
                const Part<T> phip = elp == (T)0 ? sh[2] : sh[3];
                const T dev = part_to_T(phip, T()) - a.t_r2;
                if (!(fabs(dev) <= a.t_rtol_r2)) {
                    ns.r = a.r;
                    ns.r2 = a.r * a.r;
                    ns.rtol = a.rtol;
                    ns.steptol = a.steptol;
                    ns.lam = s_lamp;
                    if (newton_update(ns, part_to_double(phip), part_to_double(sh[4]))) act = ACT_EVAL;
                    s_lam = ns.lam;
                    s_el = (T)(a.eta * ns.lam);
                }
            }
            if (a.check && blockIdx.x == 0) {
                st->it = j;
                st->residual = (double)(sqrt(res2 > (T)0 ? res2 : (T)0) / eta);
                st->bnorm2 = (double)bn2;
            }
        }
        s_act = act;
    }
    __syncthreads();
    if (s_act == ACT_RETURN) return;
    while (s_act == ACT_EVAL) {
        const T el = s_el;
        T sm1[2][2] = {};
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const T rd = rcp_t(aa[m] + el);
            const T qv = cw * (v[m].x * v[m].x + v[m].y * v[m].y) * rd * rd;
            sm1[m & 1][0] += qv;
            sm1[m & 1][1] += (T)-2 * eta * qv * rd;
        }
        Acc<T> ac2[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) { ac2[k].add(sm1[0][k]); ac2[k].add(sm1[1][k]); }
        Part<T> t2[2];
        block_part<T, 2>(ac2, red, t2);
        if (!grid_reduce_sync<T, 2>(a.bar, t2, P, P + 5 * G, P + 5 * G + 5 * 64, sh)) return;
        if (threadIdx.x == 0) {
            const bool more = newton_update(ns, part_to_double(sh[0]), part_to_double(sh[1]));
            s_lam = ns.lam;
            s_el = (T)(a.eta * ns.lam);
            s_act = more ? ACT_EVAL : ACT_SOLVE;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->lam = s_lam;
        st->newton += ns.newton;
    }

    // b_j for the next iteration's residual, stored only now: a grid barrier's fence waits
    // for a block's outstanding stores, and nothing in this launch reads b_j back
    if (ok) {
#pragma unroll
        for (int m = 0; m < L1; ++m) a.bnew[base + (long long)fo(m) * es] = v[m];
    }

    // 4. the implicit diagonal solve and the inverse transform of the columns
    const T el = s_el;
    const T ks = (T)a.inv_n;
#pragma unroll
    for (int m = 0; m < L1; ++m) {
        const T f = ks * rcp_t(aa[m] + el);
        v[m] = mk<T>(v[m].x * f, v[m].y * f);
    }
#pragma unroll
    for (int sb = 0; sb < RR; ++sb) {
        const int aq = i + L2 * sb;
        dft_r<+1, L2, T>(&v[sb * L2]);
#pragma unroll
        for (int c = 1; c < L2; ++c) v[sb * L2 + c] = cmul(v[sb * L2 + c], cconj(__ldg(&a.tw[c * aq])));
#pragma unroll
        for (int c = 0; c < L2; ++c) TB[l * TS + aq * L2 + c] = v[sb * L2 + c];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < L1; ++m) v[m] = TB[l * TS + m * L2 + i];
    dft_r<+1, L1, T>(v);
    if (ok) {
#pragma unroll
        for (int m = 0; m < L1; ++m) a.work[base + (long long)(i + L2 * m) * es] = v[m];
    }
}

}  // namespace lbtr
