// Pass kernels of the FFT-based LB operators (sm_103a).
//
// Storage of a spectrum (internal): the half spectrum of the real-to-complex
// transform along x is split into
//   main[rows][H]  complex, kx = 0..H-1 (H = M/2), rows = [z][y] (3D) or [y] (2D)
//   nyq[rows]      complex, kx = M/2 (the Nyquist plane of the x transform)
// so that every contiguous run is a power of two.  Entries are unnormalised DFTs;
// the paper's 1/N is folded into the spectral operations.
//
// A d-dimensional transform is a sequence of passes, one per axis:
//   X pass  (rows of M reals <-> H+1 complex; kernels k_xfwd / k_xinv / k_xmid)
//   Y pass  (columns along y)  and  Z pass (columns along z): k_cols.
// The innermost pass (Y in 2D, Z in 3D) sees complete 1-D spectra and applies the
// reciprocal-space diagonal there (Lambda multiply, the IMEX solve, Parseval sums).
// The X passes apply the physical-space diagonal and its reductions.
#pragma once
#include "common.cuh"
#include "fft_core.cuh"
#include "reduce.cuh"

namespace lbtr {

// ------------------------------------------------------------------------------
// Pointwise model functions F', F'' (paper §2: Gamma, Gamma'), F and F'''.
// ------------------------------------------------------------------------------
template <typename T> struct Model { T tau, gamma, eta; };

template <typename T> __device__ __forceinline__ T f0v(const Model<T>& m, T u) {
    T u2 = u * u;
    return u2 * (m.tau * (T)0.5 - m.gamma * u * (T)(1.0 / 6.0) + u2 * (T)(1.0 / 24.0));
}
template <typename T> __device__ __forceinline__ T f1v(const Model<T>& m, T u) {
    return u * (m.tau - m.gamma * (T)0.5 * u + u * u * (T)(1.0 / 6.0));
}
template <typename T> __device__ __forceinline__ T f2v(const Model<T>& m, T u) {
    return m.tau - m.gamma * u + (T)0.5 * u * u;
}

// ------------------------------------------------------------------------------
// Launch geometry helpers shared by host and device.
// ------------------------------------------------------------------------------
__host__ __device__ constexpr int x_nl(int m) { return (m / 2) >= 64 ? 16 : 1024 / (m / 2); }
__host__ __device__ constexpr int x_nt(int m) { return (m / 2) * x_nl(m) / 8; }
constexpr int COL_NL = 16;
__host__ __device__ constexpr int col_nt(int m) { return m * COL_NL / 8 < 32 ? 32 : m * COL_NL / 8; }

template <typename T> __host__ __device__ constexpr size_t x_smem(int m) {
    return sizeof(cplx<T>) * ((size_t)m + (size_t)(m / 2) * (x_nl(m) + 1) + x_nl(m)) + 128 * sizeof(double);
}
template <typename T> __host__ __device__ constexpr size_t col_smem(int m) {
    return sizeof(cplx<T>) * ((size_t)m + (size_t)m * (COL_NL + 1)) + 3 * (size_t)m * sizeof(T) + 64 * sizeof(double);
}

// ------------------------------------------------------------------------------
// X pass, forward: real rows -> spectrum rows (main + nyq), with optional
// pointwise preprocessing and reductions.
// ------------------------------------------------------------------------------
enum XfMode {
    XF_PLAIN = 0,    // transform in[]
    XF_HVPMEAN = 1,  // transform in[] = v, reduce sum F''(phi) v
    XF_ENERGY = 2,   // transform in[] = phi, reduce sum F(phi), sum F'(phi), sum phi, sum phi^2
    XF_IMEX0 = 3,    // transform b = d - eta (g + F''(phi) d), d = d0[] or dscale * g
};

template <typename T> struct XfArgs {
    const T* in;            // field transformed (XF_PLAIN/HVPMEAN/ENERGY)
    const T* phi;
    const T* g;
    const T* d0;            // XF_IMEX0: initial point (may be null)
    const double* dscale;   // XF_IMEX0 with d0 == null: d = (*dscale) * g
    cplx<T>* main;
    cplx<T>* nyq;
    const cplx<T>* tw;      // W_M table
    int rows;
    Model<T> model;
    RedSlot red;
    const int* done;        // if non-null and *done != 0: return at once
};

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(x_nt(M)) k_xfwd(XfArgs<T> a) {
    constexpr int H = M / 2, NL = x_nl(M), NT = x_nt(M), LD = NL + 1;
    constexpr int IT = H * NL / NT;          // complex pairs per thread (8)
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + M;
    C* nyqs = buf + H * LD;
    double* red = reinterpret_cast<double*>(nyqs + NL);
    const int row0 = blockIdx.x * NL;
    const C zero = mk<T>((T)0, (T)0);

    // issue every global load of this thread before using any of them
    C z[IT], p[IT], gg[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int n = w % H, row = row0 + w / H;
        const bool ok = row < a.rows;
        const size_t idx = (size_t)row * H + n;
        if (MODE == XF_IMEX0) {
            p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
            gg[t] = ok ? reinterpret_cast<const C*>(a.g)[idx] : zero;
            z[t] = (ok && a.d0) ? reinterpret_cast<const C*>(a.d0)[idx] : zero;
        } else {
            z[t] = ok ? reinterpret_cast<const C*>(a.in)[idx] : zero;
            if (MODE == XF_HVPMEAN) p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        }
    }
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];

    constexpr int NQ = (MODE == XF_ENERGY) ? 4 : 1;
    Acc<T> acc[NQ];
    T ds = (T)0;
    if (MODE == XF_IMEX0 && a.d0 == nullptr) ds = (T)(*a.dscale);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int n = w % H, l = w / H;
        C v = z[t];
        if (MODE == XF_IMEX0) {
            C d = a.d0 ? v : mk<T>(ds * gg[t].x, ds * gg[t].y);
            v.x = d.x - a.model.eta * (gg[t].x + f2v(a.model, p[t].x) * d.x);
            v.y = d.y - a.model.eta * (gg[t].y + f2v(a.model, p[t].y) * d.y);
            if (row0 + l >= a.rows) v = zero;
        } else if (MODE == XF_HVPMEAN) {
            acc[0].add(f2v(a.model, p[t].x) * v.x);
            acc[0].add(f2v(a.model, p[t].y) * v.y);
        } else if (MODE == XF_ENERGY) {
            if (row0 + l < a.rows) {
                acc[0].add(f0v(a.model, v.x));
                acc[0].add(f0v(a.model, v.y));
                acc[NQ > 1 ? 1 : 0].add(f1v(a.model, v.x));
                acc[NQ > 1 ? 1 : 0].add(f1v(a.model, v.y));
                acc[NQ > 2 ? 2 : 0].add(v.x + v.y);
                acc[NQ > 3 ? 3 : 0].add(v.x * v.x + v.y * v.y);
            }
        }
        buf[n * LD + l] = v;
    }
    __syncthreads();
    fft_lines<T, -1, H, NL, NT>(buf, tw, M);
    r2c_post<T, H, NL, NT>(buf, nyqs, tw, M);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int k = w % H, l = w / H;
        const int row = row0 + l;
        if (row < a.rows) a.main[(size_t)row * H + k] = buf[k * LD + l];
    }
    for (int l = threadIdx.x; l < NL; l += NT)
        if (row0 + l < a.rows) a.nyq[row0 + l] = nyqs[l];
    if (MODE == XF_HVPMEAN || MODE == XF_ENERGY) {
        double tot[NQ];
        block_sum<T, NQ>(acc, red, tot);
        finalize_partials(a.red, tot);
    }
}

// ------------------------------------------------------------------------------
// X pass, inverse: spectrum rows -> real rows, with pointwise postprocessing.
// ------------------------------------------------------------------------------
enum XiMode {
    XI_PLAIN = 0,  // out = x * oscale
    XI_HVP = 1,    // out = x + F''(phi) v - mean(F'' v)   (mean from msum / N)
    XI_GRAD = 2,   // out = x + F'(phi) - mean(F'(phi)); reduce max |out|
};

template <typename T> struct XiArgs {
    const cplx<T>* main;
    const cplx<T>* nyq;
    T* out;
    const T* phi;
    const T* v;
    const double* msum;     // XI_HVP / XI_GRAD: sum whose /N is subtracted
    double inv_n;
    T oscale;
    const cplx<T>* tw;
    int rows;
    Model<T> model;
    RedSlot red;            // XI_GRAD: max |out|
    const int* done;
};

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(x_nt(M)) k_xinv(XiArgs<T> a) {
    constexpr int H = M / 2, NL = x_nl(M), NT = x_nt(M), LD = NL + 1;
    constexpr int IT = H * NL / NT;
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + M;
    C* nyqs = buf + H * LD;
    double* red = reinterpret_cast<double*>(nyqs + NL);
    const int row0 = blockIdx.x * NL;
    const C zero = mk<T>((T)0, (T)0);
    // spectrum rows, and the physical fields of the epilogue, all requested up front
    C sp[IT], p[IT], vv[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int k = w % H, row = row0 + w / H;
        const bool ok = row < a.rows;
        const size_t idx = (size_t)row * H + k;
        sp[t] = ok ? a.main[idx] : zero;
        if (MODE != XI_PLAIN) p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        if (MODE == XI_HVP) vv[t] = ok ? reinterpret_cast<const C*>(a.v)[idx] : zero;
    }
    for (int l = threadIdx.x; l < NL; l += NT)
        nyqs[l] = (row0 + l < a.rows) ? a.nyq[row0 + l] : zero;
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
    T mean = (T)0;
    if (MODE != XI_PLAIN) mean = (T)(*a.msum * a.inv_n);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        buf[(w % H) * LD + w / H] = sp[t];
    }
    __syncthreads();
    c2r_pre<T, H, NL, NT>(buf, nyqs, tw, M);
    fft_lines<T, +1, H, NL, NT>(buf, tw, M);
    double mx = 0.0;
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int n = w % H, l = w / H;
        const int row = row0 + l;
        C zz = buf[n * LD + l];
        C o;
        if (MODE == XI_PLAIN) {
            o = mk<T>(zz.x * a.oscale, zz.y * a.oscale);
        } else if (MODE == XI_HVP) {
            o.x = zz.x + f2v(a.model, p[t].x) * vv[t].x - mean;
            o.y = zz.y + f2v(a.model, p[t].y) * vv[t].y - mean;
        } else {
            o.x = zz.x + f1v(a.model, p[t].x) - mean;
            o.y = zz.y + f1v(a.model, p[t].y) - mean;
            if (row < a.rows) mx = fmax(mx, fmax(fabs((double)o.x), fabs((double)o.y)));
        }
        if (row < a.rows) reinterpret_cast<C*>(a.out)[(size_t)row * H + n] = o;
    }
    if (MODE == XI_GRAD) {
        double m = block_max(mx, red);
        finalize_partials(a.red, &m);
    }
}

// ------------------------------------------------------------------------------
// X pass, fused inverse -> pointwise -> forward (spectrum rows in and out).
// ------------------------------------------------------------------------------
enum XmMode {
    XM_IMEX = 0,   // d = x; b = d - eta (g + F''(phi) d)     (Algorithm 3, b_k)
    XM_TOP = 1,    // y = x; out = F''(phi) y                   (T applied in physical space)
};

template <typename T> struct XmArgs {
    cplx<T>* main;          // in and out
    cplx<T>* nyq;
    const T* phi;
    const T* g;
    const cplx<T>* tw;
    int rows;
    T scale;                // applied to x after the inverse transform
    Model<T> model;
    const int* done;
};

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(x_nt(M)) k_xmid(XmArgs<T> a) {
    constexpr int H = M / 2, NL = x_nl(M), NT = x_nt(M), LD = NL + 1;
    constexpr int IT = H * NL / NT;
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + M;
    C* nyqs = buf + H * LD;
    const int row0 = blockIdx.x * NL;
    const C zero = mk<T>((T)0, (T)0);
    C sp[IT], p[IT], gg[IT];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int k = w % H, row = row0 + w / H;
        const bool ok = row < a.rows;
        const size_t idx = (size_t)row * H + k;
        sp[t] = ok ? a.main[idx] : zero;
        p[t] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
        if (MODE == XM_IMEX) gg[t] = ok ? reinterpret_cast<const C*>(a.g)[idx] : zero;
    }
    for (int l = threadIdx.x; l < NL; l += NT)
        nyqs[l] = (row0 + l < a.rows) ? a.nyq[row0 + l] : zero;
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        buf[(w % H) * LD + w / H] = sp[t];
    }
    __syncthreads();
    c2r_pre<T, H, NL, NT>(buf, nyqs, tw, M);
    fft_lines<T, +1, H, NL, NT>(buf, tw, M);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int n = w % H, l = w / H;
        C zz = buf[n * LD + l];
        C o = zero;
        if (row0 + l < a.rows) {
            T dx = zz.x * a.scale, dy = zz.y * a.scale;
            if (MODE == XM_IMEX) {
                o.x = dx - a.model.eta * (gg[t].x + f2v(a.model, p[t].x) * dx);
                o.y = dy - a.model.eta * (gg[t].y + f2v(a.model, p[t].y) * dy);
            } else {
                o.x = f2v(a.model, p[t].x) * dx;
                o.y = f2v(a.model, p[t].y) * dy;
            }
        }
        buf[n * LD + l] = o;
    }
    __syncthreads();
    fft_lines<T, -1, H, NL, NT>(buf, tw, M);
    r2c_post<T, H, NL, NT>(buf, nyqs, tw, M);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT;
        const int k = w % H, l = w / H;
        const int row = row0 + l;
        if (row < a.rows) a.main[(size_t)row * H + k] = buf[k * LD + l];
    }
    for (int l = threadIdx.x; l < NL; l += NT)
        if (row0 + l < a.rows) a.nyq[row0 + l] = nyqs[l];
}

// ------------------------------------------------------------------------------
// Column passes (Y, Z) with the reciprocal-space operations of the innermost axis.
// ------------------------------------------------------------------------------
enum ColMode {
    C_FWD = 0,       // forward DFT along the column
    C_INV = 1,       // inverse DFT
    C_LAM = 2,       // fwd, * Lambda * kscale, zero k = 0, inv         (D of H = D + T)
    C_LAM_E = 3,     // as C_LAM, also reduce 1/2 sum_k w Lambda |X|^2 * escale  (energy G)
    C_QUAD_E = 4,    // fwd only, reduce 1/2 sum_k w Lambda |X|^2 * escale (no store)
    C_IMEX_IN = 5,   // load bsrc, * kscale / (1 + eta (Lambda + lam)), zero k0, inv, store dst
    C_IMEX_OUT = 6,  // fwd, zero k0, store dst; reduce sum w |bold - X|^2 and sum w |X|^2 (* escale)
    C_TOP_OUT = 7,   // fwd of T-part, combine out = msc * (Lambda * msc * q + X * kscale), zero k0
    C_MSCALE_IN = 8, // load q, * msc * kscale, zero k0, inv, store dst
    C_SOLVE = 9,     // fwd, * kscale / (Lambda + sigma), zero k0, inv   (PCG preconditioner)
    C_DBOX = 10,     // fwd only, reduce sum_k w/2 |X|^2 4 xi^2 (1 - |Bk|^2) (Bk)_a^2 * escale, a = x, y, z
};

struct ColSeg {
    int nlines;        // lines in this segment
    int lg_shift;      // line l -> base (l >> lg_shift) * lhi + (l & ((1 << lg_shift) - 1)) * llo
    long long lhi, llo;
    long long es;      // element stride
    int elem_contig;   // 1 if es == 1 (load along elements)
    int kx_const;      // -1: kx = l % H (main); else fixed kx index (nyq: H)
};

template <typename T> struct ColArgs {
    cplx<T>* main;           // spectrum the pass transforms (input)
    cplx<T>* nyq;
    cplx<T>* dst_main;       // output (C_IMEX_IN / C_IMEX_OUT / C_TOP_OUT / C_MSCALE_IN); else in place
    cplx<T>* dst_nyq;
    const cplx<T>* src_main; // C_IMEX_IN: b source; C_IMEX_OUT: b old; C_TOP_OUT/C_MSCALE_IN: q
    const cplx<T>* src_nyq;
    const cplx<T>* tw;
    const T* qtab;           // [3][M] (2 pi / L_a)^2 * wavenum(i)^2 for a = x, y, z
    ColSeg seg[2];           // main, nyq
    int nb_main;             // number of blocks of the main segment
    int dim;
    T xi2;
    T kscale;                // multiplier folded into the spectral op (1/N for C_LAM)
    double escale;           // multiplier of reductions (1/N^2)
    T eta;
    T sigma;                 // C_TOP_OUT / C_MSCALE_IN: shift of M = Lambda + sigma
    const double* lam;       // C_IMEX_IN: device multiplier lambda
    RedSlot red;
    const int* done;
};

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(col_nt(M)) k_cols(ColArgs<T> a) {
    constexpr int NL = COL_NL, NT = col_nt(M), LD = NL + 1, H = M / 2;
    constexpr int IT = (M * NL + NT - 1) / NT;
    constexpr int HSH = (H >= 256) ? 8 : (H >= 128) ? 7 : (H >= 64) ? 6 : (H >= 32) ? 5 : (H >= 16) ? 4 : (H >= 8) ? 3 : 2;
    static_assert((1 << HSH) == H, "H must be a power of two");
    static_assert(NT % NL == 0, "each thread keeps one line in the line-major mapping");
    using C = cplx<T>;
    constexpr bool PRE = (MODE == C_IMEX_IN || MODE == C_MSCALE_IN);
    constexpr bool POST = (MODE == C_LAM || MODE == C_LAM_E || MODE == C_QUAD_E || MODE == C_IMEX_OUT ||
                           MODE == C_TOP_OUT || MODE == C_SOLVE || MODE == C_DBOX);
    constexpr bool AUX = (MODE == C_IMEX_OUT || MODE == C_TOP_OUT);
    constexpr bool NEED_Q = PRE || (POST && MODE != C_IMEX_OUT);
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + M;
    T* qt = reinterpret_cast<T*>(buf + M * LD);
    double* red = reinterpret_cast<double*>(qt + 3 * M);
    const C zero = mk<T>((T)0, (T)0);

    const int segi = blockIdx.x < a.nb_main ? 0 : 1;
    const ColSeg s = a.seg[segi];
    const int l0 = (segi == 0 ? blockIdx.x : blockIdx.x - a.nb_main) * NL;
    const C* src = PRE ? (segi == 0 ? a.src_main : a.src_nyq) : (segi == 0 ? a.main : a.nyq);
    C* dst = (PRE || AUX) ? (segi == 0 ? a.dst_main : a.dst_nyq) : (segi == 0 ? a.main : a.nyq);
    const C* aux = segi == 0 ? a.src_main : a.src_nyq;
    const int nval = s.nlines - l0 < NL ? s.nlines - l0 : NL;
    const long long lmask = (1LL << s.lg_shift) - 1;
    auto base = [&](int l) -> long long {
        return (long long)(l >> s.lg_shift) * s.lhi + (long long)(l & lmask) * s.llo;
    };
    // wavenumber data of element (global line L, element e) of the innermost axis
    auto kinfo = [&](int L, int e, T& bk2, T& wgt, bool& is0) {
        const int kx = s.kx_const >= 0 ? s.kx_const : (L & (H - 1));
        T by, bz;
        bool zero_other;
        if (a.dim == 3) {
            const int y = s.kx_const >= 0 ? L : (L >> HSH);
            by = qt[M + y];
            bz = qt[2 * M + e];
            zero_other = (y == 0);
        } else {
            by = qt[M + e];
            bz = (T)0;
            zero_other = true;
        }
        bk2 = qt[kx] + by + bz;
        wgt = (s.kx_const < 0 && kx > 0) ? (T)2 : (T)1;
        is0 = (s.kx_const < 0) && kx == 0 && zero_other && e == 0;
    };

    // line-major mapping: each thread keeps line l = tid % NL and walks elements
    const int lm_l = threadIdx.x % NL;
    const int lm_e0 = threadIdx.x / NL;
    constexpr int LM_ESTEP = NT / NL;
    const bool lm_ok = lm_l < nval;
    const long long lm_base = lm_ok ? base(l0 + lm_l) : 0;

    // 1. issue all loads of the tile (and of the auxiliary spectrum)
    C v[IT], x[AUX ? IT : 1];
    if (s.elem_contig) {
#pragma unroll
        for (int t = 0; t < IT; ++t) {
            const int w = threadIdx.x + t * NT;
            const int e = w % M, l = w / M;
            v[t] = (w < M * NL && l < nval) ? src[base(l0 + l) + e] : zero;
        }
    } else {
#pragma unroll
        for (int t = 0; t < IT; ++t) {
            const int e = lm_e0 + t * LM_ESTEP;
            v[t] = (e < M && lm_ok) ? src[lm_base + (long long)e * s.es] : zero;
        }
    }
    if (AUX) {
#pragma unroll
        for (int t = 0; t < IT; ++t) {
            const int e = lm_e0 + t * LM_ESTEP;
            x[AUX ? t : 0] = (e < M && lm_ok) ? aux[lm_base + (long long)e * s.es] : zero;
        }
    }
    for (int i = threadIdx.x; i < M; i += NT) tw[i] = a.tw[i];
    if (NEED_Q)
        for (int i = threadIdx.x; i < 3 * M; i += NT) qt[i] = a.qtab[i];
    T lamv = (T)0;
    if (MODE == C_IMEX_IN) lamv = (T)(*a.lam);
    if (PRE) __syncthreads();     // qt ready for the scaling below

    // 2. (optional pre-scaling) and stage the tile in shared memory
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        int e, l;
        if (s.elem_contig) { const int w = threadIdx.x + t * NT; e = w % M; l = w / M; if (w >= M * NL) continue; }
        else { e = lm_e0 + t * LM_ESTEP; l = lm_l; if (e >= M) continue; }
        C val = v[t];
        if (PRE && l < nval) {
            T bk2, wgt; bool is0;
            kinfo(l0 + l, e, bk2, wgt, is0);
            const T tt = (T)1 - bk2;
            const T lamk = a.xi2 * tt * tt;
            T f;
            if (MODE == C_IMEX_IN) f = a.kscale / ((T)1 + a.eta * (lamk + lamv));
            else f = a.kscale / sqrt(lamk + a.sigma);
            val = is0 ? zero : mk<T>(val.x * f, val.y * f);
        }
        buf[e * LD + l] = val;
    }
    __syncthreads();

    constexpr int NQ = (MODE == C_IMEX_OUT) ? 2 : (MODE == C_DBOX) ? 3 : 1;
    Acc<T> acc[NQ];
    // 3. transform, with the reciprocal-space operation of the innermost axis
    if (PRE || MODE == C_INV) {
        fft_lines<T, +1, M, NL, NT>(buf, tw, M);
    } else {
        fft_lines<T, -1, M, NL, NT>(buf, tw, M);
        if (POST) {
#pragma unroll
            for (int t = 0; t < IT; ++t) {
                const int e = lm_e0 + t * LM_ESTEP;
                if (e >= M || !lm_ok) continue;
                C val = buf[e * LD + lm_l];
                T bk2, wgt; bool is0;
                if (MODE != C_IMEX_OUT) {
                    kinfo(l0 + lm_l, e, bk2, wgt, is0);
                } else {
                    const int L = l0 + lm_l;
                    const int kx = s.kx_const >= 0 ? s.kx_const : (L & (H - 1));
                    const bool zo = (a.dim == 3) ? ((s.kx_const >= 0 ? L : (L >> HSH)) == 0) : true;
                    wgt = (s.kx_const < 0 && kx > 0) ? (T)2 : (T)1;
                    is0 = (s.kx_const < 0) && kx == 0 && zo && e == 0;
                    bk2 = (T)0;
                }
                if (is0) val = zero;
                if (MODE == C_IMEX_OUT) {
                    const C old = x[AUX ? t : 0];
                    const T dx = old.x - val.x, dy = old.y - val.y;
                    acc[0].add(wgt * (dx * dx + dy * dy));
                    acc[NQ - 1].add(wgt * (val.x * val.x + val.y * val.y));
                    buf[e * LD + lm_l] = val;
                    continue;
                }
                const T tt = (T)1 - bk2;
                const T lamk = a.xi2 * tt * tt;
                if (MODE == C_DBOX) {
                    // dLambda/dL_a = 4 xi^2 (1 - |Bk|^2) (Bk)_a^2 / L_a; the 1/L_a is applied by the host
                    const int L = l0 + lm_l;
                    const int kx = s.kx_const >= 0 ? s.kx_const : (L & (H - 1));
                    T qy, qz;
                    if (a.dim == 3) {
                        qy = qt[M + (s.kx_const >= 0 ? L : (L >> HSH))];
                        qz = qt[2 * M + e];
                    } else {
                        qy = qt[M + e];
                        qz = (T)0;
                    }
                    const T c = (T)2 * wgt * a.xi2 * tt * (val.x * val.x + val.y * val.y);
                    acc[0].add(c * qt[kx]);
                    acc[NQ > 1 ? 1 : 0].add(c * qy);
                    acc[NQ > 2 ? 2 : 0].add(c * qz);
                    continue;
                }
                if (MODE == C_LAM_E || MODE == C_QUAD_E) acc[0].add((T)0.5 * wgt * lamk * (val.x * val.x + val.y * val.y));
                if (MODE == C_TOP_OUT) {
                    const C q = x[AUX ? t : 0];
                    const T ms = (T)1 / sqrt(lamk + a.sigma);
                    const T c1 = lamk * ms * ms, c2 = ms * a.kscale;
                    val = is0 ? zero : mk<T>(c1 * q.x + c2 * val.x, c1 * q.y + c2 * val.y);
                } else if (MODE == C_SOLVE) {
                    const T f = a.kscale / (lamk + a.sigma);
                    val = is0 ? zero : mk<T>(val.x * f, val.y * f);
                } else {
                    const T f = lamk * a.kscale;
                    val = mk<T>(val.x * f, val.y * f);
                }
                buf[e * LD + lm_l] = val;
            }
            __syncthreads();
            if (MODE == C_LAM || MODE == C_LAM_E || MODE == C_SOLVE) fft_lines<T, +1, M, NL, NT>(buf, tw, M);
        }
    }

    // 4. store
    if (MODE != C_QUAD_E && MODE != C_DBOX) {
        if (s.elem_contig) {
#pragma unroll
            for (int t = 0; t < IT; ++t) {
                const int w = threadIdx.x + t * NT;
                const int e = w % M, l = w / M;
                if (w < M * NL && l < nval) dst[base(l0 + l) + e] = buf[e * LD + l];
            }
        } else {
#pragma unroll
            for (int t = 0; t < IT; ++t) {
                const int e = lm_e0 + t * LM_ESTEP;
                if (e < M && lm_ok) dst[lm_base + (long long)e * s.es] = buf[e * LD + lm_l];
            }
        }
    }
    if (MODE == C_LAM_E || MODE == C_QUAD_E || MODE == C_IMEX_OUT || MODE == C_DBOX) {
        double tot[NQ];
        block_sum<T, NQ>(acc, red, tot);
        if (threadIdx.x == 0)
            for (int q = 0; q < NQ; ++q) tot[q] *= a.escale;
        finalize_partials(a.red, tot);
    }
}

// sum_x s^2 (F''(v)/2 + F'''(v) s/6 + s^2/24) = sum_x [F(v+s) - F(v) - F'(v) s]: the
// exact Taylor remainder of the quartic bulk density, free of cancellation.
template <typename T>
__global__ void k_taylor_rem(const T* v, const T* sd, long long n, Model<T> m, RedSlot red) {
    __shared__ double scr[64];
    Acc<T> acc[1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T u = v[i], s = sd[i];
        acc[0].add(s * s * (f2v(m, u) * (T)0.5 + (u - m.gamma) * s * (T)(1.0 / 6.0) + s * s * (T)(1.0 / 24.0)));
    }
    double tot[1];
    block_sum<T, 1>(acc, scr, tot);
    finalize_partials(red, tot);
}

}  // namespace lbtr
