// Shared-memory FFT building blocks for the LB kernels (sm_103a, CUDA cores).
//
// The discrete transform of the paper's §2 factorises over axes; each axis is a
// batch of 1-D DFTs of length L (a power of two, 2..512).  A CTA holds NL lines in
// shared memory, element-major: element e of line l lives at buf[e * LD + l] with
// LD = NL + 1 (the pad keeps both line-parallel and element-parallel accesses free
// of bank conflicts).  Lines are transformed by a mixed-radix Stockham autosort
// factorisation (radix 8, then 4 or 2 for the remainder): pass (R, p) reads
// x[i + r L/R], multiplies by W_{pR}^{r (i mod p)}, applies a radix-R DFT and writes
// y[(i - i mod p) R + i mod p + r p].  Passes are separated by __syncthreads().
// Twiddles W_M^j = exp(-2 pi i j / M) come from a host-computed table copied to
// shared memory; the inverse direction uses conjugates.
//
// Real transforms along x use the half-length method: a real line of M samples is
// viewed as M/2 complex samples z[n] = x[2n] + i x[2n+1]; its spectrum X[0..M/2]
// follows from Z = DFT(z) by X[k] = E + W^k O, X[M/2-k] = conj(E - W^k O) with
// E = (Z[k] + conj Z[M/2-k]) / 2, O = -i (Z[k] - conj Z[M/2-k]) / 2, and the inverse
// reverses these steps.  Forward transforms carry no 1/N factor; callers fold it in.
#pragma once
#include "common.cuh"

namespace lbtr {

// ---- radix-R DFT in registers, X_k = sum_j u_j exp(SIGN 2 pi i j k / R) -------------
template <int SIGN, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a; a = cadd(t, b); b = csub(t, b);
}

template <int SIGN, typename C> __device__ __forceinline__ void dft4(C* u) {
    C a0 = cadd(u[0], u[2]), a1 = csub(u[0], u[2]);
    C b0 = cadd(u[1], u[3]), b1 = cmul_i<SIGN>(csub(u[1], u[3]));
    u[0] = cadd(a0, b0);
    u[2] = csub(a0, b0);
    u[1] = cadd(a1, b1);
    u[3] = csub(a1, b1);
}

template <int SIGN, typename T> __device__ __forceinline__ void dft8(cplx<T>* u) {
    using C = cplx<T>;
    const T s = (T)0.70710678118654752440084436210484903928;
    C a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) { a[j] = cadd(u[j], u[j + 4]); b[j] = csub(u[j], u[j + 4]); }
    // b_j *= exp(SIGN 2 pi i j / 8)
    {
        C t = b[1];   // (1 + SIGN i)/sqrt2
        b[1] = mk<T>(s * (t.x - (T)SIGN * t.y), s * (t.y + (T)SIGN * t.x));
        b[2] = cmul_i<SIGN>(b[2]);
        t = b[3];     // (-1 + SIGN i)/sqrt2
        b[3] = mk<T>(s * (-t.x - (T)SIGN * t.y), s * (-t.y + (T)SIGN * t.x));
    }
    dft4<SIGN>(a);
    dft4<SIGN>(b);
#pragma unroll
    for (int m = 0; m < 4; ++m) { u[2 * m] = a[m]; u[2 * m + 1] = b[m]; }
}

// x * (c + i s)
template <typename T> __device__ __forceinline__ cplx<T> crot(cplx<T> x, T c, T s) {
    return mk<T>(x.x * c - x.y * s, x.x * s + x.y * c);
}

// 16 points as 4 x 4: n = n1 + 4 n2, k = k2 + 4 k1; length-4 DFTs over n2, the twiddle
// exp(SIGN 2 pi i n1 k2 / 16), length-4 DFTs over n1.  Output in natural order.
template <int SIGN, typename T> __device__ __forceinline__ void dft16(cplx<T>* u) {
    using C = cplx<T>;
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;   // cos, sin of pi/8
    const T h = (T)0.70710678118654752440, sg = (T)SIGN;
    C v[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        C t[4] = {u[n1], u[n1 + 4], u[n1 + 8], u[n1 + 12]};
        dft4<SIGN>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[n1][k2] = t[k2];
    }
    v[1][1] = crot(v[1][1], c1, sg * s1);     // angle 1 * 2 pi / 16
    v[1][2] = crot(v[1][2], h, sg * h);       // 2
    v[1][3] = crot(v[1][3], s1, sg * c1);     // 3
    v[2][1] = crot(v[2][1], h, sg * h);       // 2
    v[2][2] = cmul_i<SIGN>(v[2][2]);          // 4
    v[2][3] = crot(v[2][3], -h, sg * h);      // 6
    v[3][1] = crot(v[3][1], s1, sg * c1);     // 3
    v[3][2] = crot(v[3][2], -h, sg * h);      // 6
    v[3][3] = crot(v[3][3], -c1, -sg * s1);   // 9
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        C t[4] = {v[0][k2], v[1][k2], v[2][k2], v[3][k2]};
        dft4<SIGN>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) u[k2 + 4 * k1] = t[k1];
    }
}

template <int SIGN, int R, typename T> __device__ __forceinline__ void dft_r(cplx<T>* u) {
    if (R == 2) dft2<SIGN>(u[0], u[1]);
    else if (R == 4) dft4<SIGN>(u);
    else if (R == 8) dft8<SIGN, T>(u);
    else dft16<SIGN, T>(u);
}

// ---- radix plan: 8s first, then 4/2; 16 is done as 4*4 ---------------------------
__host__ __device__ constexpr int plan_npass(int L) {
    return L <= 2 ? 1 : L == 4 ? 1 : L == 8 ? 1 : L == 16 ? 2 : L == 32 ? 2 : L == 64 ? 2
         : L == 128 ? 3 : L == 256 ? 3 : 3;
}
__host__ __device__ constexpr int plan_radix(int L, int pass) {
    return L == 2 ? 2 : L == 4 ? 4 : L == 8 ? 8 : L == 16 ? 4 : L == 32 ? (pass == 0 ? 8 : 4)
         : L == 64 ? 8 : L == 128 ? (pass == 0 ? 8 : 4) : L == 256 ? (pass < 2 ? 8 : 4) : 8;
}
__host__ __device__ constexpr int plan_p(int L, int pass) {
    return pass == 0 ? 1 : plan_p(L, pass - 1) * plan_radix(L, pass - 1);
}

// One Stockham pass of radix R with stride product P on NL lines of length L.
// Element e of line l sits at buf[e * ES + l * LS].  Thread tid of NT handles work
// items w = tid + t NT (line = w % NL, butterfly = w / NL).
template <typename T, int SIGN, int L, int R, int P, int NL, int NT, int ES, int LS>
__device__ __forceinline__ void stockham_pass_s(cplx<T>* buf, const cplx<T>* tw, int mtab) {
    constexpr int NB = L / R;             // butterflies per line
    constexpr int TOT = NB * NL;
    constexpr int IT = (TOT + NT - 1) / NT;
    using C = cplx<T>;
    C u[IT][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        int w = tid + t * NT;
        if (TOT % NT == 0 || w < TOT) {
            int l = w % NL, i = w / NL;
            int k = i % P;
#pragma unroll
            for (int r = 0; r < R; ++r) u[t][r] = buf[(i + r * NB) * ES + l * LS];
            if (P > 1) {
                int step = mtab / (P * R);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C wv = tw[(r * k * step)];
                    if (SIGN > 0) wv.y = -wv.y;
                    u[t][r] = cmul(u[t][r], wv);
                }
            }
            dft_r<SIGN, R, T>(u[t]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        int w = tid + t * NT;
        if (TOT % NT == 0 || w < TOT) {
            int l = w % NL, i = w / NL;
            int k = i % P;
            int j = (i - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(j + r * P) * ES + l * LS] = u[t][r];
        }
    }
    __syncthreads();
}

template <typename T, int SIGN, int L, int R, int P, int NL, int NT>
__device__ __forceinline__ void stockham_pass(cplx<T>* buf, const cplx<T>* tw, int mtab) {
    stockham_pass_s<T, SIGN, L, R, P, NL, NT, NL + 1, 1>(buf, tw, mtab);
}

// Full in-place DFT of NL lines of length L in shared memory (sign SIGN, unscaled),
// element e of line l at buf[e * ES + l * LS].  Requires a __syncthreads() between
// the producer of buf and this call.
template <typename T, int SIGN, int L, int NL, int NT, int ES, int LS>
__device__ __forceinline__ void fft_lines_s(cplx<T>* buf, const cplx<T>* tw, int mtab) {
    constexpr int NP = plan_npass(L);
    stockham_pass_s<T, SIGN, L, plan_radix(L, 0), plan_p(L, 0), NL, NT, ES, LS>(buf, tw, mtab);
    if (NP > 1) stockham_pass_s<T, SIGN, L, plan_radix(L, NP > 1 ? 1 : 0), plan_p(L, NP > 1 ? 1 : 0), NL, NT, ES, LS>(buf, tw, mtab);
    if (NP > 2) stockham_pass_s<T, SIGN, L, plan_radix(L, NP > 2 ? 2 : 0), plan_p(L, NP > 2 ? 2 : 0), NL, NT, ES, LS>(buf, tw, mtab);
}

template <typename T, int SIGN, int L, int NL, int NT>
__device__ __forceinline__ void fft_lines(cplx<T>* buf, const cplx<T>* tw, int mtab) {
    fft_lines_s<T, SIGN, L, NL, NT, NL + 1, 1>(buf, tw, mtab);
}

// After a forward length-H DFT of z[n] = x[2n] + i x[2n+1] on NL lines, turn Z into the
// real spectrum X[0..H-1] in place and X[H] into the slot at element index H of each
// line (element stride ES, line stride LS; table W_M of size 2H).
template <typename T, int H, int NL, int NT, int ES, int LS>
__device__ __forceinline__ void r2c_post_s(cplx<T>* buf, const cplx<T>* tw, int mtab) {
    constexpr int NPAIR = H / 2 + 1;        // k = 0..H/2
    using C = cplx<T>;
    const int step = mtab / (2 * H);
    for (int w = threadIdx.x; w < NPAIR * NL; w += NT) {
        int l = w % NL, k = w / NL;
        if (k == 0) {
            C z = buf[l * LS];
            buf[l * LS] = mk<T>(z.x + z.y, (T)0);
            buf[H * ES + l * LS] = mk<T>(z.x - z.y, (T)0);
        } else {
            C zk = buf[k * ES + l * LS];
            C zm = buf[(H - k) * ES + l * LS];
            C e = mk<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
            C o = mk<T>((T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x));
            C wo = cmul(tw[k * step], o);
            buf[k * ES + l * LS] = cadd(e, wo);
            if (2 * k != H) buf[(H - k) * ES + l * LS] = cconj(csub(e, wo));
        }
    }
    __syncthreads();
}

// Inverse of r2c_post_s: from X[0..H] (X[H] at element index H) build
// Z[k] = (X[k] + conj X[H-k]) + i (X[k] - conj X[H-k]) conj(W^k) for k < H.
template <typename T, int H, int NL, int NT, int ES, int LS>
__device__ __forceinline__ void c2r_pre_s(cplx<T>* buf, const cplx<T>* tw, int mtab) {
    constexpr int NPAIR = H / 2 + 1;
    using C = cplx<T>;
    const int step = mtab / (2 * H);
    for (int w = threadIdx.x; w < NPAIR * NL; w += NT) {
        int l = w % NL, k = w / NL;
        if (k == 0) {
            T x0 = buf[l * LS].x, xh = buf[H * ES + l * LS].x;
            buf[l * LS] = mk<T>(x0 + xh, x0 - xh);
        } else {
            C xk = buf[k * ES + l * LS];
            C xm = buf[(H - k) * ES + l * LS];
            C e = mk<T>(xk.x + xm.x, xk.y - xm.y);
            C d = mk<T>(xk.x - xm.x, xk.y + xm.y);
            C wc = tw[k * step]; wc.y = -wc.y;
            C o = cmul(d, wc);
            buf[k * ES + l * LS] = mk<T>(e.x - o.y, e.y + o.x);
            if (2 * k != H) buf[(H - k) * ES + l * LS] = mk<T>(e.x + o.y, -e.y + o.x);
        }
    }
    __syncthreads();
}

// After a forward length-H DFT of z[n] = x[2n] + i x[2n+1], turn Z into the real
// spectrum X[0..H-1] in place and X[H] into nyq[l] (H = M/2, table W_M of size 2H).
template <typename T, int H, int NL, int NT>
__device__ __forceinline__ void r2c_post(cplx<T>* buf, cplx<T>* nyq, const cplx<T>* tw, int mtab) {
    constexpr int LD = NL + 1;
    constexpr int NPAIR = H / 2 + 1;        // k = 0..H/2
    using C = cplx<T>;
    const int step = mtab / (2 * H);
    for (int w = threadIdx.x; w < NPAIR * NL; w += NT) {
        int l = w % NL, k = w / NL;
        if (k == 0) {
            C z = buf[l];
            buf[l] = mk<T>(z.x + z.y, (T)0);
            nyq[l] = mk<T>(z.x - z.y, (T)0);
        } else {
            C zk = buf[k * LD + l];
            C zm = buf[(H - k) * LD + l];
            C e = mk<T>((T)0.5 * (zk.x + zm.x), (T)0.5 * (zk.y - zm.y));
            // o = -i (zk - conj zm) / 2
            C o = mk<T>((T)0.5 * (zk.y + zm.y), (T)-0.5 * (zk.x - zm.x));
            C wo = cmul(tw[k * step], o);
            buf[k * LD + l] = cadd(e, wo);
            if (2 * k != H) buf[(H - k) * LD + l] = cconj(csub(e, wo));
        }
    }
    __syncthreads();
}

// Inverse of r2c_post: from X[0..H-1] in buf and X[H] in nyq[l] build
// Z[k] = (X[k] + conj X[H-k]) + i (X[k] - conj X[H-k]) conj(W^k); an inverse length-H
// DFT of Z then yields z[n] = x[2n] + i x[2n+1] (unscaled).
template <typename T, int H, int NL, int NT>
__device__ __forceinline__ void c2r_pre(cplx<T>* buf, const cplx<T>* nyq, const cplx<T>* tw, int mtab) {
    constexpr int LD = NL + 1;
    constexpr int NPAIR = H / 2 + 1;
    using C = cplx<T>;
    const int step = mtab / (2 * H);
    for (int w = threadIdx.x; w < NPAIR * NL; w += NT) {
        int l = w % NL, k = w / NL;
        if (k == 0) {
            T x0 = buf[l].x, xh = nyq[l].x;
            buf[l] = mk<T>(x0 + xh, x0 - xh);
        } else {
            C xk = buf[k * LD + l];
            C xm = buf[(H - k) * LD + l];
            C e = mk<T>(xk.x + xm.x, xk.y - xm.y);          // X[k] + conj X[H-k]
            C d = mk<T>(xk.x - xm.x, xk.y + xm.y);          // X[k] - conj X[H-k]
            C wc = tw[k * step]; wc.y = -wc.y;
            C o = cmul(d, wc);
            // Z[k] = e + i o ; Z[H-k] = conj(e) + i conj(o)
            buf[k * LD + l] = mk<T>(e.x - o.y, e.y + o.x);
            if (2 * k != H) buf[(H - k) * LD + l] = mk<T>(e.x + o.y, -e.y + o.x);
        }
    }
    __syncthreads();
}

}  // namespace lbtr
