// Hessian-vector product of 3D 128^3 float grids as one cooperative kernel with warp-local
// exchanges.
//
//   Hv = P[F^{-1}(Lambda F v) + F''(phi) v]      (paper §2 Hessian formulas; §3.2, H = D + T)
//
// The product's own spectrum is internal to the kernel, so it is laid out for it:
// S[z][kx][ky] (kx = 0..M/2, ky fastest).  One CTA of 1024 threads per SM:
//
//   phase 1 (planes)   per z-plane: the x transform of the plane's rows (eight threads per
//                      row, 64 complex pairs z[n] = v[2n] + i v[2n+1], an 8 x 8 four-step with
//                      its transpose in the warp's own shared memory), the real-spectrum fold
//                      (mirror pairs X[k], X[H - k] exchanged between two lanes of the row by
//                      shuffles), ONE block-wide hand-off through shared memory, and the y
//                      transform of the 64 packed columns (sixteen threads per column: an
//                      8-point DFT in registers, an exchange through the warp's shared memory,
//                      another 8-point DFT and a 2-point DFT between neighbouring lanes).  The
//                      real columns kx = 0 and kx = M/2 travel as one complex column and are
//                      separated after the y transform.  Also sums F''(phi) v per plane.
//   grid barrier
//   phase 2 (z lines)  every warp of the grid takes groups of four (kx, ky) lines: the z
//                      transform (16 x 8 four-step, transpose in the warp's shared memory),
//                      Lambda / N with k = 0 removed, the inverse z transform.
//   grid barrier
//   phase 3 (planes)   the mirror image of phase 1, then Hv = x + F''(phi) v - mean(F''(phi) v)
//                      written row by row.
//
// Every exchange except the x <-> y hand-off is inside one warp (__syncwarp or shuffles), so a
// plane costs one block-wide barrier per direction, and the product is one launch.
#pragma once
#include "passes.cuh"

namespace lbtr {

template <typename T> struct Hvp3Args {
    const T* v;
    const T* phi;
    T* hv;
    cplx<T>* spec;          // [M][M/2 + 1][M] complex scratch
    const cplx<T>* tw;      // W_M^j = exp(-2 pi i j / M), j < M
    const T* qtab;          // [3][M]: (2 pi / L_a)^2 * wavenumber(i)^2 for axis a = x, y, z
    Model<T> model;
    double* partials;       // [M]: sum of F''(phi) v over each z-plane
    GridBar bar;            // grid barrier of the fused kernel
    double inv_n;
    T xi2;
    T kscale;               // 1 / N
};

// geometry of the 128^3 kernels
struct H3 {
    static constexpr int M = 128, H = 64, NT = 1024;
    static constexpr int NKX = H + 1;                // spectrum columns kx = 0..64
    static constexpr int PS = 132;                   // hand-off column stride (complex)
    static constexpr int XRS = 76;                   // x transpose: row stride within a warp
    static constexpr int QS = 9;                     // y exchange: stride of a thread's 8 values
    static constexpr int WS = 4 * XRS > 2 * 16 * QS + 16 ? 4 * XRS : 2 * 16 * QS + 16;   // per-warp scratch
    static constexpr size_t SMEM = (size_t)(H * PS + 32 * WS) * 8 + 64 * sizeof(double);
    // z lines: four per warp
    static constexpr int ZTS = 148;                  // transpose: line stride (complex), 2 ZTS = 8 mod 32 banks
    static constexpr size_t ZWARP = (size_t)4 * ZTS * 8;    // z-line scratch of one warp (bytes)
    static constexpr int NLINES = NKX * M;           // 8320 z-lines
    static constexpr int NTASKS = NLINES / 4;        // four lines per warp
    // the fused kernel: one CTA of 1024 threads per SM holds either phase's shared memory
    // (keeping the plane's F''(phi) v in shared memory from phase 1 to phase 3 was measured
    // slower: the larger carve-out leaves less L1 for the loads of phase 1)
    static constexpr size_t FSMEM = (32 * ZWARP > SMEM ? 32 * ZWARP : SMEM);
};

// W_16^k = exp(-2 pi i k / 16), k = 0..7, as constants (k is a compile-time index in the
// unrolled loops that call this)
template <typename T> __device__ __forceinline__ cplx<T> h3_w16(int k) {
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
    switch (k & 7) {
        case 0: return mk<T>((T)1, (T)0);
        case 1: return mk<T>(c1, -s1);
        case 2: return mk<T>(h, -h);
        case 3: return mk<T>(s1, -c1);
        case 4: return mk<T>((T)0, (T)-1);
        case 5: return mk<T>(-s1, -c1);
        case 6: return mk<T>(-h, -h);
        default: return mk<T>(-c1, -s1);
    }
}

// w[q] = b^q for q = 1..7 (w[0] = 1) by repeated products: one table load per thread
// instead of seven; the powers carry a few roundings, far below the float transform's own
template <typename T> __device__ __forceinline__ void h3_pow7(cplx<T> b, cplx<T> (&w)[8]) {
    w[0] = mk<T>((T)1, (T)0);
    w[1] = b;
    w[2] = cmul(b, b);
    w[3] = cmul(w[2], b);
    w[4] = cmul(w[2], w[2]);
    w[5] = cmul(w[4], b);
    w[6] = cmul(w[3], w[3]);
    w[7] = cmul(w[6], b);
}

// f''(u) = tau - gamma u + u^2 / 2 (as f2v of passes.cuh)
template <typename T> __device__ __forceinline__ T h3_f2(const Model<T>& m, T u) {
    return m.tau + u * ((T)0.5 * u - m.gamma);
}

// ---------------------------------------------------------------------------------
// x and y forward transforms of one plane.  Thread (y = tid / 8, j = tid % 8) holds
// u[m] = z[j + 8 m], the complex pairs z[n] = x[2n] + i x[2n+1] of row y; the plane's
// spectrum goes to spec[z][kx][ky].  `handoff` runs once, right after the block-wide
// hand-off barrier (the shared scratch after the hand-off buffer is then readable).
// ---------------------------------------------------------------------------------
template <typename T, typename F>
__device__ __forceinline__ void h3_fwd_xy(const cplx<T>* __restrict__ tw, cplx<T>* spec, int z,
                                          unsigned char* smem_raw, cplx<T> (&u)[8], F&& handoff) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, H = G::H;
    C* P = reinterpret_cast<C*>(smem_raw);                   // [64][PS]
    C* ws = P + H * G::PS + (threadIdx.x >> 5) * G::WS;      // this warp's scratch
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y = tid >> 3, j = tid & 7;                     // x: row y, thread j holds z[j + 8 m]
    const int c = tid >> 4, t = tid & 15;                    // y: column c, thread t holds Y[t + 16 m]
    const C tw2j = __ldg(&tw[2 * j]), twj = __ldg(&tw[j]), twt = __ldg(&tw[t]);
    dft_r<-1, 8, T>(u);                                      // over m
    {
        C w[8];
        h3_pow7<T>(tw2j, w);                                 // W_64^{jq}
#pragma unroll
        for (int q = 1; q < 8; ++q) u[q] = cmul(u[q], w[q]);
    }
    {
        C* xs = ws + (y & 3) * G::XRS;
#pragma unroll
        for (int q = 0; q < 8; ++q) xs[q * 9 + j] = u[q];
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) u[jj] = xs[j * 9 + jj];
    }
    dft_r<-1, 8, T>(u);                                      // over jj: u[k2] = Z[j + 8 k2]
    // real-spectrum fold: X[k] = E + W_M^k O, E, O from Z[k] and Z[H - k]
    {
        const int partner = (lane & ~7) | ((8 - j) & 7);
        const T hf = (T)0.5;
        C out[8];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            const C s = mk<T>(__shfl_sync(0xffffffffu, u[7 - k2].x, partner),
                              __shfl_sync(0xffffffffu, u[7 - k2].y, partner));
            const C zm = (j == 0) ? u[(8 - k2) & 7] : s;
            const C zk = u[k2];
            if (j == 0 && k2 == 0) {
                out[0] = mk<T>(zk.x + zk.y, zk.x - zk.y);    // X(0) + i X(H), both real
            } else {
                const C e = mk<T>(hf * (zk.x + zm.x), hf * (zk.y - zm.y));
                const C o = mk<T>(hf * (zk.y + zm.y), -hf * (zk.x - zm.x));
                out[k2] = cadd(e, cmul(cmul(twj, h3_w16<T>(k2)), o));     // W_M^{j + 8 k2}
            }
        }
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) P[(j + 8 * k2) * G::PS + y] = out[k2];
    }
    __syncthreads();
    handoff();

    // ---- y ----
    C x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = P[c * G::PS + t + 16 * m];
    dft_r<-1, 8, T>(x);                                      // over m
    {
        C w[8];
        h3_pow7<T>(twt, w);                                  // W_M^{tq}
#pragma unroll
        for (int q = 1; q < 8; ++q) x[q] = cmul(x[q], w[q]);
    }
    const int qb = (lane >> 4) * 16 * G::QS;
#pragma unroll
    for (int q = 0; q < 8; ++q) ws[qb + t * G::QS + q] = x[q];
    __syncwarp();
    const int aa = t >> 1, t1 = t & 1;
#pragma unroll
    for (int t2 = 0; t2 < 8; ++t2) x[t2] = ws[qb + (t1 + 2 * t2) * G::QS + aa];
    dft_r<-1, 8, T>(x);                                      // over t2
    if (t1) {
#pragma unroll
        for (int k = 1; k < 8; ++k) x[k] = cmul(x[k], h3_w16<T>(k));                     // W_16^k
    }
    {
        // t1 = 0: own + partner's; t1 = 1: partner's - own
        const T sg = t1 ? (T)-1 : (T)1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const T ox = __shfl_xor_sync(0xffffffffu, x[k].x, 1), oy = __shfl_xor_sync(0xffffffffu, x[k].y, 1);
            x[k] = mk<T>(fma(sg, x[k].x, ox), fma(sg, x[k].y, oy));
        }
    }
    // thread (aa, t1) of column c now holds Y[ky] for ky = aa + 8 k + 64 t1 at x[k]
    C* S = spec + (size_t)z * G::NKX * M;
    if (c != 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) S[(size_t)c * M + aa + 8 * k + 64 * t1] = x[k];
    }
    if (warp == 0) {
        // the packed column: Y = F[X(0)] + i F[X(H)] with both sequences real in y
        __syncwarp();
        if (lane < 16) {
#pragma unroll
            for (int k = 0; k < 8; ++k) ws[aa + 8 * k + 64 * t1] = x[k];
        }
        __syncwarp();
        if (lane < 16) {
            const T hf = (T)0.5;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int ky = aa + 8 * k + 64 * t1;
                const C zk = x[k], zm = ws[(M - ky) & (M - 1)];
                S[ky] = mk<T>(hf * (zk.x + zm.x), hf * (zk.y - zm.y));
                S[(size_t)H * M + ky] = mk<T>(hf * (zk.y + zm.y), -hf * (zk.x - zm.x));
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// phase 1: v (real plane z) -> S[z][kx][ky]; the plane's sum of F''(phi) v -> partials[z]
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void h3_fwd_plane(const Hvp3Args<T>& a, int z, unsigned char* smem_raw) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, H = G::H;
    double* red = reinterpret_cast<double*>(reinterpret_cast<C*>(smem_raw) + H * G::PS + 32 * G::WS);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y = tid >> 3, j = tid & 7;
    const size_t row = (size_t)z * M + y;
    C u[8], p[8];
    {
        const C* vr = reinterpret_cast<const C*>(a.v) + row * H;
        const C* pr = reinterpret_cast<const C*>(a.phi) + row * H;
#pragma unroll
        for (int m = 0; m < 8; ++m) { u[m] = vr[j + 8 * m]; p[m] = pr[j + 8 * m]; }
    }
    {
        // the thread's 16 terms of the projection sum of F''(phi) v in the working precision,
        // then the warp's total in double-word form; warp totals are added after the hand-off
        T sum = (T)0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            sum = fma(h3_f2(a.model, p[m].x), u[m].x, sum);
            sum = fma(h3_f2(a.model, p[m].y), u[m].y, sum);
        }
        Acc<T> acc;
        acc.add(sum);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc.add_shfl(off);
        if (lane == 0) red[warp] = acc.get();
    }
    h3_fwd_xy<T>(a.tw, a.spec, z, smem_raw, u, [&]() {
        if (warp == 1) {
            // the plane's projection sum: the 32 warp totals in a fixed order
            double q = red[lane];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
            if (lane == 0) a.partials[z] = q;
        }
    });
}

// ---------------------------------------------------------------------------------
// z lines of task q (lines 4q..4q+3 of kx * M + ky): four lines per warp, thread i of line l
// (lane = 4 i + l).  h3_zfwd loads and transforms them (v[s * 8 + b] = X[kz], kz = i + 8 s +
// 16 b); h3_zinv transforms back and stores in place.  ts: the warp's scratch.
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void h3_zfwd(const cplx<T>* __restrict__ tw, const cplx<T>* spec, int task, cplx<T>* ts,
                                        cplx<T> (&v)[16]) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, NL = G::NLINES;
    const int lane = threadIdx.x & 31;
    const int l = lane & 3, i = lane >> 2;
    const C* base = spec + task * 4 + l;
    const C twi = __ldg(&tw[i]);
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = base[(size_t)(i + 8 * m) * NL];
    // forward: DFT16 over m, twiddle W_M^{i q}, transpose, DFT8 over i
    dft_r<-1, 16, T>(v);
    {
        // W_M^{iq}: two running products of depth 7 (q = 1..7 and q = 8..15), few registers
        C wa = twi, wb = __ldg(&tw[(8 * i) & (M - 1)]);
        v[8] = cmul(v[8], wb);
#pragma unroll
        for (int q = 1; q < 8; ++q) {
            v[q] = cmul(v[q], wa);
            wb = cmul(wb, twi);
            v[q + 8] = cmul(v[q + 8], wb);
            wa = cmul(wa, twi);
        }
    }
    C* tl = ts + l * G::ZTS;                                 // element (q, i) at tl[9 q + i]
#pragma unroll
    for (int q = 0; q < 16; ++q) tl[q * 9 + i] = v[q];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int q = i + 8 * s;
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) v[s * 8 + ii] = tl[q * 9 + ii];
        dft_r<-1, 8, T>(&v[s * 8]);
    }
}

template <typename T>
__device__ __forceinline__ void h3_zinv(const cplx<T>* __restrict__ tw, cplx<T>* spec, int task, cplx<T>* ts,
                                        cplx<T> (&v)[16]) {
    using G = H3;
    using C = cplx<T>;
    constexpr int NL = G::NLINES;
    const int lane = threadIdx.x & 31;
    const int l = lane & 3, i = lane >> 2;
    const C twi = __ldg(&tw[i]);
    C* tl = ts + l * G::ZTS;
    // inverse: DFT8 over b, twiddle W_M^{-c q} (q = i + 8 s), transpose back, DFT16
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        dft_r<+1, 8, T>(&v[s * 8]);
        // running product of W_M^{-q}, q = i + 8 s
        const C wq1 = s ? cconj(cmul(twi, __ldg(&tw[8]))) : cconj(twi);
        C wc = wq1;
#pragma unroll
        for (int c = 1; c < 8; ++c) {
            v[s * 8 + c] = cmul(v[s * 8 + c], wc);
            wc = cmul(wc, wq1);
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int q = i + 8 * s;
#pragma unroll
        for (int c = 0; c < 8; ++c) tl[q * 9 + c] = v[s * 8 + c];
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = tl[q * 9 + i];
    dft_r<+1, 16, T>(v);
    C* base = spec + task * 4 + l;
#pragma unroll
    for (int m = 0; m < 16; ++m) base[(size_t)(i + 8 * m) * NL] = v[m];
    __syncwarp();                                            // the scratch is free for the next task
}

// phase 2 of the product: forward, Lambda / N with k = 0 removed, inverse
template <typename T>
__device__ __forceinline__ void h3_zline_task(const Hvp3Args<T>& a, int task, cplx<T>* ts) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M;
    const int lane = threadIdx.x & 31;
    const int l = lane & 3, i = lane >> 2;
    const int line = task * 4 + l;                           // kx * M + ky
    const int kx = line >> 7, ky = line & (M - 1);
    const T* __restrict__ qt = a.qtab;
    const T bxy = __ldg(&qt[kx]) + __ldg(&qt[M + ky]);
    const T qzc = __ldg(&qt[2 * M + 1]);                     // (2 pi / L_z)^2: |Bk|^2 of kz is qzc * k^2
    C v[16];
    h3_zfwd<T>(a.tw, a.spec, task, ts, v);
    {
        const bool k0 = (kx == 0 && ky == 0);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int kz = i + 8 * s + 16 * b;
                const T kk = (T)(kz < M / 2 ? kz : kz - M);
                const T tt = (T)1 - (bxy + qzc * (kk * kk));
                T f = a.xi2 * tt * tt * a.kscale;
                if (k0 && kz == 0) f = (T)0;
                v[s * 8 + b] = mk<T>(v[s * 8 + b].x * f, v[s * 8 + b].y * f);
            }
    }
    h3_zinv<T>(a.tw, a.spec, task, ts, v);
}

// ---------------------------------------------------------------------------------
// y and x inverse transforms of one plane: spec[z][kx][ky] -> u[m] = z[j + 8 m] of row
// y = tid / 8 (unscaled).  `early` runs once between the column loads and the first
// exchange (the shared scratch after the hand-off buffer is free then).
// ---------------------------------------------------------------------------------
template <typename T, typename F>
__device__ __forceinline__ void h3_inv_xy(const cplx<T>* __restrict__ tw, const cplx<T>* spec, int z,
                                          unsigned char* smem_raw, cplx<T> (&u)[8], F&& early) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, H = G::H;
    C* P = reinterpret_cast<C*>(smem_raw);
    C* ws = P + H * G::PS + (threadIdx.x >> 5) * G::WS;
    const int tid = threadIdx.x, lane = tid & 31;
    const C* S = spec + (size_t)z * G::NKX * M;
    const int c = tid >> 4, t = tid & 15, aa = t >> 1, t1 = t & 1;
    const int y = tid >> 3, j = tid & 7;
    const C tw2j = __ldg(&tw[2 * j]), twj = __ldg(&tw[j]), twt = __ldg(&tw[t]);
    // ---- y inverse: column c, thread (aa, t1) loads Y[ky], ky = aa + 8 k + 64 t1 ----
    C x[8];
    if (c != 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = S[(size_t)c * M + aa + 8 * k + 64 * t1];
    } else {
        // pack the Hermitian parts of the real columns kx = 0 and kx = H
        const T hf = (T)0.5;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int ky = aa + 8 * k + 64 * t1, km = (M - ky) & (M - 1);
            const C x0 = S[ky], x0m = S[km], xh = S[(size_t)H * M + ky], xhm = S[(size_t)H * M + km];
            const C e = mk<T>(hf * (x0.x + x0m.x), hf * (x0.y - x0m.y));
            const C f = mk<T>(hf * (xh.x + xhm.x), hf * (xh.y - xhm.y));
            x[k] = mk<T>(e.x - f.y, e.y + f.x);
        }
    }
    early();
    // 2-point step between the lanes t1 = 0, 1, then W_16^{-k} on the odd half
    {
        const T sg = t1 ? (T)-1 : (T)1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const T ox = __shfl_xor_sync(0xffffffffu, x[k].x, 1), oy = __shfl_xor_sync(0xffffffffu, x[k].y, 1);
            x[k] = mk<T>(fma(sg, x[k].x, ox), fma(sg, x[k].y, oy));
        }
    }
    if (t1) {
#pragma unroll
        for (int k = 1; k < 8; ++k) x[k] = cmul(x[k], cconj(h3_w16<T>(k)));
    }
    dft_r<+1, 8, T>(x);                                      // over k: x[t2] = D_aa[t1 + 2 t2]
    const int qb = (lane >> 4) * 16 * G::QS;
#pragma unroll
    for (int t2 = 0; t2 < 8; ++t2) ws[qb + (t1 + 2 * t2) * G::QS + aa] = x[t2];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = ws[qb + t * G::QS + q];
    {
        C w[8];
        h3_pow7<T>(twt, w);                                  // W_M^{-tq} = conj W_M^{tq}
#pragma unroll
        for (int q = 1; q < 8; ++q) x[q] = cmul(x[q], cconj(w[q]));
    }
    dft_r<+1, 8, T>(x);                                      // over q: x[m] = column value at y = t + 16 m
#pragma unroll
    for (int m = 0; m < 8; ++m) P[c * G::PS + t + 16 * m] = x[m];
    __syncthreads();

    // ---- x inverse: row y, thread j ----
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) u[k2] = P[(j + 8 * k2) * G::PS + y];
    // complex-to-real pre-step: Z[k] = (X[k] + conj X[H-k]) + i (X[k] - conj X[H-k]) conj(W_M^k)
    {
        const int partner = (lane & ~7) | ((8 - j) & 7);
        C zz[8];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            const C s = mk<T>(__shfl_sync(0xffffffffu, u[7 - k2].x, partner),
                              __shfl_sync(0xffffffffu, u[7 - k2].y, partner));
            const C xm = (j == 0) ? u[(8 - k2) & 7] : s;
            const C xk = u[k2];
            if (j == 0 && k2 == 0) {
                zz[0] = mk<T>(xk.x + xk.y, xk.x - xk.y);     // X(0) = x0, X(H) = xh (packed)
            } else {
                const C e = mk<T>(xk.x + xm.x, xk.y - xm.y);
                const C d = mk<T>(xk.x - xm.x, xk.y + xm.y);
                const C o = cmul(d, cconj(cmul(twj, h3_w16<T>(k2))));
                zz[k2] = mk<T>(e.x - o.y, e.y + o.x);
            }
        }
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) u[k2] = zz[k2];
    }
    // inverse 64-point transform: thread j holds Z[j + 8 k]; DFT8 over k, W_64^{-jj j}, transpose, DFT8
    dft_r<+1, 8, T>(u);                                      // u[jj] = V_j[jj]
    {
        C w[8];
        h3_pow7<T>(tw2j, w);                                 // W_64^{-j jj} = conj W_64^{j jj}
#pragma unroll
        for (int jj = 1; jj < 8; ++jj) u[jj] = cmul(u[jj], cconj(w[jj]));
    }
    {
        C* xs = ws + (y & 3) * G::XRS;
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) xs[jj * 9 + j] = u[jj];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] = xs[j * 9 + q];
    }
    dft_r<+1, 8, T>(u);                                      // u[m] = z[j + 8 m] (unscaled)
}

// ---------------------------------------------------------------------------------
// phase 3: S[z][kx][ky] -> Hv (real plane z) with F''(phi) v - mean
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void h3_inv_plane(const Hvp3Args<T>& a, int z, unsigned char* smem_raw) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, H = G::H;
    T* s_mean = reinterpret_cast<T*>(reinterpret_cast<C*>(smem_raw) + H * G::PS + 32 * G::WS);
    const int tid = threadIdx.x, lane = tid & 31;
    const int y = tid >> 3, j = tid & 7;
    C u[8];
    h3_inv_xy<T>(a.tw, a.spec, z, smem_raw, u, [&]() {
        if (tid >= 32 && tid < 64) {
            // mean of F''(phi) v: warp 1 adds the planes' partial sums in a fixed order
            double q = 0.0;
#pragma unroll
            for (int k = 0; k < M / 32; ++k) q += __ldcg(&a.partials[lane + 32 * k]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
            if (lane == 0) *s_mean = (T)(q * a.inv_n);
        }
    });
    const T mean = *s_mean;                                  // written before the hand-off barrier
    const size_t row = (size_t)z * M + y;
    const C* vr = reinterpret_cast<const C*>(a.v) + row * H;
    const C* pr = reinterpret_cast<const C*>(a.phi) + row * H;
    C* hr = reinterpret_cast<C*>(a.hv) + row * H;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const C pp = pr[j + 8 * m], vv = vr[j + 8 * m];
        C o;
        o.x = u[m].x + h3_f2(a.model, pp.x) * vv.x - mean;
        o.y = u[m].y + h3_f2(a.model, pp.y) * vv.y - mean;
        hr[j + 8 * m] = o;
    }
}

// ---------------------------------------------------------------------------------
// The product as ONE cooperative launch: one CTA of 1024 threads per SM walks the planes
// (phase 1), a bounded grid barrier, every warp of the grid takes z-line tasks (phase 2),
// a second barrier, and the planes again (phase 3).  A barrier that gives up (its budget
// exhausted: a fault, not a state cooperative residency can reach) sets the context's error
// flag and the CTAs leave; Hv is then left unwritten and the next synchronising call on the
// context reports LB_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024, 1) k_hvp_fused(Hvp3Args<T> a) {
    using G = H3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = gridDim.x, z = blockIdx.x;
    for (int zz = z; zz < G::M; zz += nb) {
        h3_fwd_plane<T>(a, zz, smem_raw);
        __syncthreads();                                     // shared memory reused by the next plane
    }
    if (!grid_sync_acqrel(a.bar)) return;
    {
        // z-line tasks on the first warps of every CTA, interleaved over CTAs
        const int warp = threadIdx.x >> 5, nw = (G::NTASKS + nb - 1) / nb;
        const int nwork = nw < 32 ? nw : 32;
        cplx<T>* ts = reinterpret_cast<cplx<T>*>(smem_raw + warp * G::ZWARP);
        if (warp < nwork) {
#pragma unroll 1
            for (int q = warp * nb + z; q < G::NTASKS; q += nwork * nb) h3_zline_task<T>(a, q, ts);
        }
    }
    if (!grid_sync_acqrel(a.bar)) return;
    for (int zz = z; zz < G::M; zz += nb) {
        h3_inv_plane<T>(a, zz, smem_raw);
        __syncthreads();
    }
}

}  // namespace lbtr
