// Column passes (y or z lines of the spectrum) as register-resident four-step transforms
// with a software pipeline over tiles.
//
// A tile is NL consecutive lines of one segment (the main spectrum or the Nyquist
// column), addressed as in ColSeg.  Thread (l, i) of the CTA (l < NL, i < L2) holds the
// L1 elements e = i + L2 m of line l; the forward transform is DFT_L1 over m in registers,
// the twiddle W_M^{i a}, one transpose through shared memory and DFT_L2 in registers, after
// which thread (l, i) holds X[a + L1 b] for a = i + L2 s (s < L1 / L2), b < L2.  The
// reciprocal-space operation of the mode is applied there and the inverse runs the mirror
// image back to the first layout.  The grid is persistent: each CTA walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and issues the loads of its next tile before it
// transforms the current one, so that memory and arithmetic overlap within the CTA.
#pragma once
#include "passes.cuh"
#include "planes.cuh"

namespace lbtr {

constexpr int LN_NL = 16;   // lines per tile
__host__ __device__ constexpr int ln_nt(int m) { return LN_NL * fs_l2(m); }
template <typename T> __host__ __device__ constexpr size_t ln_smem(int m) {
    return 2 * (size_t)LN_NL * (m + 1) * sizeof(cplx<T>) + 64 * sizeof(double);
}

// Modes handled here: C_FWD, C_INV, C_LAM, C_LAM_E, C_SOLVE (others stay on k_cols).
__host__ __device__ constexpr bool ln_mode_ok(int mode) {
    return mode == C_FWD || mode == C_INV || mode == C_LAM || mode == C_LAM_E || mode == C_SOLVE;
}

template <typename T, int M, int MODE>
__device__ __forceinline__ void lines_body(const ColArgs<T>& a, int ntiles) {
    constexpr int NL = LN_NL, L1 = fs_l1(M), L2 = fs_l2(M), RR = L1 / L2, TS = M + 1, H = M / 2;
    constexpr int HSH = (H >= 256) ? 8 : (H >= 128) ? 7 : (H >= 64) ? 6 : (H >= 32) ? 5 : (H >= 16) ? 4 : (H >= 8) ? 3 : 2;
    static_assert((1 << HSH) == H, "H must be a power of two");
    constexpr bool FWD = MODE != C_INV;
    constexpr bool INV = MODE != C_FWD;
    constexpr bool OP = FWD && INV;
    using C = cplx<T>;
    if (a.done && *(volatile const int*)a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* TA = reinterpret_cast<C*>(smem_raw);
    C* TB = TA + NL * TS;
    double* red = reinterpret_cast<double*>(TB + NL * TS);
    const int l = threadIdx.x % NL, i = threadIdx.x / NL;
    const C zero = mk<T>((T)0, (T)0);
    const T* __restrict__ qt = a.qtab;

    // element positions of this thread in the input and output layouts
    auto in_elem = [&](int m) -> int {          // element held in slot m on entry
        if (FWD) return i + L2 * m;
        const int s = m / L2, b = m % L2;
        return i + L2 * s + L1 * b;
    };
    auto out_elem = [&](int m) -> int {
        if (INV) return i + L2 * m;
        const int s = m / L2, b = m % L2;
        return i + L2 * s + L1 * b;
    };
    struct TileRef { long long base; int L, segi; bool ok; };
    auto tile_ref = [&](int t) -> TileRef {
        TileRef r;
        r.segi = t < a.nb_main ? 0 : 1;
        const ColSeg& s = a.seg[r.segi];
        r.L = (t - (r.segi ? a.nb_main : 0)) * NL + l;
        r.ok = t < ntiles && r.L < s.nlines;
        const long long lmask = (1LL << s.lg_shift) - 1;
        r.base = r.ok ? (long long)(r.L >> s.lg_shift) * s.lhi + (long long)(r.L & lmask) * s.llo : 0;
        return r;
    };
    auto load = [&](const TileRef& r, C (&v)[L1]) {
        const C* src = r.segi == 0 ? a.main : a.nyq;
        const long long es = a.seg[r.segi].es;
#pragma unroll
        for (int m = 0; m < L1; ++m) v[m] = r.ok ? src[r.base + (long long)in_elem(m) * es] : zero;
    };

    Acc<T> acc[1];
    int t = blockIdx.x;
    TileRef cr = tile_ref(t);
    C cur[L1];
    load(cr, cur);
    for (; t < ntiles; t += gridDim.x) {
        // prefetch of the next tile (registers; consumed one iteration later)
        const TileRef nr = tile_ref(t + gridDim.x);
        C nxt[L1];
        load(nr, nxt);
        const ColSeg& s = a.seg[cr.segi];
        if (FWD) {
            dft_r<-1, L1, T>(cur);
#pragma unroll
            for (int q = 1; q < L1; ++q) cur[q] = cmul(cur[q], __ldg(&a.tw[i * q]));     // W_M^{iq}
#pragma unroll
            for (int q = 0; q < L1; ++q) TA[l * TS + q * L2 + i] = cur[q];
            __syncthreads();
#pragma unroll
            for (int sb = 0; sb < RR; ++sb) {
                const int q = i + L2 * sb;
#pragma unroll
                for (int jj = 0; jj < L2; ++jj) cur[sb * L2 + jj] = TA[l * TS + q * L2 + jj];
                dft_r<-1, L2, T>(&cur[sb * L2]);
            }
        }
        if (OP && cr.ok) {
            const int kx = s.kx_const >= 0 ? s.kx_const : (cr.L & (H - 1));
            T byz;     // the part of |Bk|^2 from the other axis
            bool zo;
            if (a.dim == 3) {
                const int y = s.kx_const >= 0 ? cr.L : (cr.L >> HSH);
                byz = qt[kx] + qt[M + y];
                zo = (y == 0);
            } else {
                byz = qt[kx];
                zo = true;
            }
            const T wgt = (s.kx_const < 0 && kx > 0) ? (T)2 : (T)1;
            const bool k0line = (s.kx_const < 0) && kx == 0 && zo;
            const T* qe = qt + (a.dim == 3 ? 2 * M : M);
#pragma unroll
            for (int m = 0; m < L1; ++m) {
                const int e = i + L2 * (m / L2) + L1 * (m % L2);
                const T tt = (T)1 - (byz + qe[e]);
                const T lamk = a.xi2 * tt * tt;
                C v = cur[m];
                if (k0line && e == 0) v = zero;
                if (MODE == C_LAM_E) acc[0].add((T)0.5 * wgt * lamk * (v.x * v.x + v.y * v.y));
                const T f = (MODE == C_SOLVE) ? a.kscale / (lamk + a.sigma) : lamk * a.kscale;
                cur[m] = mk<T>(v.x * f, v.y * f);
            }
        }
        if (INV) {
#pragma unroll
            for (int sb = 0; sb < RR; ++sb) {
                const int q = i + L2 * sb;
                dft_r<+1, L2, T>(&cur[sb * L2]);
#pragma unroll
                for (int c = 1; c < L2; ++c) cur[sb * L2 + c] = cmul(cur[sb * L2 + c], cconj(__ldg(&a.tw[c * q])));
#pragma unroll
                for (int c = 0; c < L2; ++c) TB[l * TS + q * L2 + c] = cur[sb * L2 + c];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < L1; ++q) cur[q] = TB[l * TS + q * L2 + i];
            dft_r<+1, L1, T>(cur);
        }
        if (cr.ok) {
            C* dst = cr.segi == 0 ? a.main : a.nyq;
#pragma unroll
            for (int m = 0; m < L1; ++m) dst[cr.base + (long long)out_elem(m) * s.es] = cur[m];
        }
        if (!OP) __syncthreads();    // one transpose buffer per tile: its reads end before the next writes
#pragma unroll
        for (int m = 0; m < L1; ++m) cur[m] = nxt[m];
        cr = nr;
    }
    if (MODE == C_LAM_E) {
        double tot[1];
        block_sum<T, 1>(acc, red, tot);
        if (threadIdx.x == 0) tot[0] *= a.escale;
        finalize_partials(a.red, tot);
    }
}

template <typename T, int M, int MODE>
__global__ void __launch_bounds__(ln_nt(M)) k_lines(ColArgs<T> a, int ntiles) { lines_body<T, M, MODE>(a, ntiles); }

// The three line passes of a 3D product on the x-row path -- y forward, z with Lambda / N,
// y inverse -- as one cooperative launch with two bounded grid barriers: the spectrum is
// read back right after it was written, while it is still in L2, and two launch boundaries
// (the drain of one pass's stores and the next launch) become barriers.  The launch also
// adds up the product's sum of F''(phi) v from the row kernel's per-block partials (rpart,
// nrpart of them): each CTA a share in the first phase (into l2[blockIdx.x]), CTA 0 the
// shares in the last, into *msum for the inverse row kernel -- in place of a ticket
// reduction at the end of the row kernel, whose last block would add thousands of partials
// on the critical path.  The order of the additions depends only on indices.
template <typename T, int M>
__global__ void __launch_bounds__(ln_nt(M)) k_lines3(ColArgs<T> yf, ColArgs<T> zl, ColArgs<T> yi, int ty, int tz,
                                                     GridBar bar, const double* rpart, int nrpart, double* l2,
                                                     double* msum) {
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = blockIdx.x + gridDim.x * threadIdx.x; i < nrpart; i += 32 * gridDim.x) s += __ldcg(&rpart[i]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) l2[blockIdx.x] = s;
    }
    lines_body<T, M, C_FWD>(yf, ty);
    if (!grid_sync_acqrel(bar)) return;
    lines_body<T, M, C_LAM>(zl, tz);
    if (!grid_sync_acqrel(bar)) return;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        // all loads in flight at once (grids of at most 512 CTAs), then a fixed order
        constexpr int K = 16;
        double x[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = threadIdx.x + 32 * k;
            x[k] = i < (int)gridDim.x ? __ldcg(&l2[i]) : 0.0;
        }
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) s += x[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) *msum = s;
    }
    lines_body<T, M, C_INV>(yi, ty);
}
// many problems of the same size per launch: blockIdx.y selects the problem's arguments
template <typename T, int M, int MODE>
__global__ void __launch_bounds__(ln_nt(M)) k_lines_b(const ColArgs<T>* __restrict__ args, int ntiles) {
    lines_body<T, M, MODE>(args[blockIdx.y], ntiles);
}

}  // namespace lbtr
