// The Hessian-vector products of a whole batch of 2D problems (a phase-diagram sweep over
// (tau, gamma, M)) as ONE persistent launch that takes its work from device-side queues.
//
// Every 2D product is three passes: the x rows forward (with the sum of F''(phi) v), the y
// lines with Lambda / N, the x rows inverse (with F''(phi) v - mean).  The kernel runs the
// three passes of ALL problems as three phases separated by bounded grid barriers; within a
// phase each CTA repeatedly takes the next task from the phase's queue (a device array of
// (problem, task) pairs, largest grids first, popped with one atomic increment of the queue
// head), looks up the problem's arguments and runs the task for that problem's grid size.
// Problems of different sizes therefore share one launch and balance dynamically.  A row
// task covers `group` consecutive row blocks (the tuned granularity), a line task one tile
// of 128 / L2 lines of the four-step transform.  The per-problem sum of F''(phi) v is
// written as one partial per row task (no atomics); the inverse tasks add a problem's
// partials in a fixed order.
#pragma once
#include "passes.cuh"
#include "rows.cuh"

namespace lbtr {

// one problem of the sweep as the kernel sees it
template <typename T> struct SweepProb {
    XfArgs<T> xf;           // rows forward (in = v, phi, main/nyq = the problem's spectrum)
    ColArgs<T> ca;          // the y lines (Lambda / N)
    XiArgs<T> xi;           // rows inverse (out = Hv)
    double* part;           // [row blocks] partial sums of F''(phi) v
    int m;                  // points per axis
    int row_blocks;         // ceil(rows / NR)
    int line_tiles;         // tiles of the y pass (main + Nyquist)
};

struct SweepTask { int prob, task; };

template <typename T> struct SweepArgs {
    const SweepProb<T>* probs;
    const SweepTask* tasks[3];   // rows forward, lines, rows inverse
    int ntasks[3];
    int group;                   // row blocks per row task
    unsigned* heads;             // three queue heads, 32 words apart, zero at launch
    GridBar bar;
};

// lines per tile of the y pass with 128 threads: L2 threads per line
__host__ __device__ constexpr int sw_nl(int m) { return 128 / fs_l2(m); }
template <typename T> __host__ __device__ constexpr size_t sw_lines_smem(int m) {
    return 2 * (size_t)sw_nl(m) * (m + 1) * sizeof(cplx<T>);
}
template <typename T> __host__ __device__ constexpr size_t sw_smem_m(int m) {
    return (m == 16 ? rows_smem<T, 16>() : m == 32 ? rows_smem<T, 32>() : m == 64 ? rows_smem<T, 64>()
            : m == 128 ? rows_smem<T, 128>() : m == 256 ? rows_smem<T, 256>() : rows_smem<T, 512>()) >
                   sw_lines_smem<T>(m)
               ? (m == 16 ? rows_smem<T, 16>() : m == 32 ? rows_smem<T, 32>() : m == 64 ? rows_smem<T, 64>()
                  : m == 128 ? rows_smem<T, 128>() : m == 256 ? rows_smem<T, 256>() : rows_smem<T, 512>())
               : sw_lines_smem<T>(m);
}
template <typename T> __host__ __device__ constexpr size_t sw_smem() {
    size_t s = 0;
    for (int m = 16; m <= 512; m *= 2) s = sw_smem_m<T>(m) > s ? sw_smem_m<T>(m) : s;
    return s;
}

// ---- rows forward of row block `blk`: x transform, fold, store; returns the block's sum of
//      F''(phi) v to thread 0 ----
template <typename T, int M>
__device__ __forceinline__ double sw_rows_fwd(const XfArgs<T>& a, int blk, unsigned char* smem_raw) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int L1 = G::L1;
    const RowSmem<T, M> sm(smem_raw);
    const long long row0 = (long long)blk * G::NR;
    const bool ok = row0 + threadIdx.x / G::L2 < a.rows;
    const C zero = mk<T>((T)0, (T)0);
    C u[L1], p[L1];
#pragma unroll
    for (int m = 0; m < L1; ++m) {
        const long long idx = rows_idx<M>(row0, m);
        u[m] = ok ? reinterpret_cast<const C*>(a.in)[idx] : zero;
        p[m] = ok ? reinterpret_cast<const C*>(a.phi)[idx] : zero;
    }
    Acc<T> acc[1];
    {
        T sum = (T)0;
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            sum = fma(f2v(a.model, p[m].x), u[m].x, sum);
            sum = fma(f2v(a.model, p[m].y), u[m].y, sum);
        }
        acc[0].add(sum);
    }
    rows_fwd<T, M>(u, sm, a.tw);
    rows_fold_store<T, M>(sm, a.main, a.nyq, row0, a.rows, a.tw);
    double tot[1] = {0.0};
    block_sum<T, 1>(acc, sm.red, tot);
    return tot[0];
}

// ---- rows inverse of row block `blk` with Hv = x + F''(phi) v - mean ----
template <typename T, int M>
__device__ __forceinline__ void sw_rows_inv(const XiArgs<T>& a, int blk, T mean, unsigned char* smem_raw) {
    using G = RowGeo<M>;
    using C = cplx<T>;
    constexpr int L1 = G::L1;
    const RowSmem<T, M> sm(smem_raw);
    const long long row0 = (long long)blk * G::NR;
    const bool ok = row0 + threadIdx.x / G::L2 < a.rows;
    rows_load_spec<T, M>(sm, a.main, a.nyq, row0, a.rows);
    C u[L1];
    rows_inv<T, M>(u, sm, a.tw);
    if (ok) {
        // the pointwise operands after the transform: fewer live registers, which sets the
        // occupancy of the whole persistent kernel
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const long long idx = rows_idx<M>(row0, m);
            const C pp = reinterpret_cast<const C*>(a.phi)[idx], vv = reinterpret_cast<const C*>(a.v)[idx];
            C o;
            o.x = u[m].x + f2v(a.model, pp.x) * vv.x - mean;
            o.y = u[m].y + f2v(a.model, pp.y) * vv.y - mean;
            reinterpret_cast<C*>(a.out)[idx] = o;
        }
    }
}

// ---- y lines tile `tile` of a 2D problem: forward transform, Lambda / N (k = 0 removed),
//      inverse transform, in place.  sw_nl(M) lines per tile, L2 threads per line (thread
//      (l, i) holds elements e = i + L2 m of line l, the layout of lines.cuh); tiles past
//      the main segment hold the Nyquist column kx = M/2. ----
template <typename T, int M>
__device__ __forceinline__ void sw_lines2d(const ColArgs<T>& a, int tile, unsigned char* smem_raw) {
    constexpr int L1 = fs_l1(M), L2 = fs_l2(M), RR = L1 / L2, TS = M + 1, H = M / 2, NL = sw_nl(M);
    static_assert(NL * L2 == 128 && RR >= 1, "128 threads per tile, L1 >= L2");
    using C = cplx<T>;
    C* TA = reinterpret_cast<C*>(smem_raw);
    C* TB = TA + NL * TS;
    const int l = threadIdx.x % NL, i = threadIdx.x / NL;
    const int nmt = (H + NL - 1) / NL;
    const bool ny = tile >= nmt;
    const int L = ny ? l : tile * NL + l;
    const bool ok = ny ? (l == 0) : (L < H);
    C* buf = ny ? a.nyq : a.main;
    const long long es = ny ? 1 : H;
    const long long base = ny ? 0 : L;
    const C zero = mk<T>((T)0, (T)0);
    const C* __restrict__ tw = a.tw;
    C cur[L1];
#pragma unroll
    for (int m = 0; m < L1; ++m) cur[m] = ok ? buf[base + (long long)(i + L2 * m) * es] : zero;
    dft_r<-1, L1, T>(cur);
#pragma unroll
    for (int q = 1; q < L1; ++q) cur[q] = cmul(cur[q], __ldg(&tw[i * q]));          // W_M^{iq}
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
    {
        const T* __restrict__ qt = a.qtab;
        const int kx = ny ? H : L;
        const T bx = qt[kx];
        const bool k0line = !ny && kx == 0;
#pragma unroll
        for (int m = 0; m < L1; ++m) {
            const int e = i + L2 * (m / L2) + L1 * (m % L2);
            const T tt = (T)1 - (bx + qt[M + e]);
            T f = a.xi2 * tt * tt * a.kscale;
            if (k0line && e == 0) f = (T)0;
            cur[m] = mk<T>(cur[m].x * f, cur[m].y * f);
        }
    }
#pragma unroll
    for (int sb = 0; sb < RR; ++sb) {
        const int q = i + L2 * sb;
        dft_r<+1, L2, T>(&cur[sb * L2]);
#pragma unroll
        for (int c = 1; c < L2; ++c) cur[sb * L2 + c] = cmul(cur[sb * L2 + c], cconj(__ldg(&tw[c * q])));
#pragma unroll
        for (int c = 0; c < L2; ++c) TB[l * TS + q * L2 + c] = cur[sb * L2 + c];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < L1; ++q) cur[q] = TB[l * TS + q * L2 + i];
    dft_r<+1, L1, T>(cur);
    if (ok) {
#pragma unroll
        for (int m = 0; m < L1; ++m) buf[base + (long long)(i + L2 * m) * es] = cur[m];
    }
}

// ---- the same y-lines tile for M = 512, where the register four-step would need more
//      than 16 values per thread: sw_nl(512) = 4 lines staged in shared memory (element e
//      of line l at buf[e (NL + 1) + l]) and transformed by radix-8 Stockham passes ----
template <typename T, int M>
__device__ __forceinline__ void sw_lines2d_smem(const ColArgs<T>& a, int tile, unsigned char* smem_raw) {
    constexpr int NL = sw_nl(M), NT = 128, LD = NL + 1, H = M / 2, IT = M * NL / NT;
    static_assert((M * NL) % NT == 0, "whole elements per thread");
    using C = cplx<T>;
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int nmt = (H + NL - 1) / NL;
    const bool ny = tile >= nmt;
    C* src = ny ? a.nyq : a.main;
    const long long es = ny ? 1 : H;
    const C zero = mk<T>((T)0, (T)0);
    auto line_ok = [&](int l) { return ny ? (l == 0) : (tile * NL + l < H); };
    auto line_base = [&](int l) -> long long { return ny ? 0 : (long long)(tile * NL + l); };
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT, l = w % NL, e = w / NL;
        buf[e * LD + l] = line_ok(l) ? src[line_base(l) + (long long)e * es] : zero;
    }
    __syncthreads();
    fft_lines<T, -1, M, NL, NT>(buf, a.tw, M);
    {
        const T* __restrict__ qt = a.qtab;
#pragma unroll
        for (int t = 0; t < IT; ++t) {
            const int w = threadIdx.x + t * NT, l = w % NL, e = w / NL;
            const int kx = ny ? H : tile * NL + l;
            const T tt = (T)1 - (qt[kx < H ? kx : H] + qt[M + e]);
            T f = a.xi2 * tt * tt * a.kscale;
            if (!ny && kx == 0 && e == 0) f = (T)0;
            const C x = buf[e * LD + l];
            buf[e * LD + l] = mk<T>(x.x * f, x.y * f);
        }
    }
    __syncthreads();
    fft_lines<T, +1, M, NL, NT>(buf, a.tw, M);
#pragma unroll
    for (int t = 0; t < IT; ++t) {
        const int w = threadIdx.x + t * NT, l = w % NL, e = w / NL;
        if (line_ok(l)) src[line_base(l) + (long long)e * es] = buf[e * LD + l];
    }
}

// dispatch a task body over the supported 2D grid sizes
#define SW_SWITCH_M(mval, ...)                                      \
    switch (mval) {                                                 \
        case 16: { constexpr int M = 16; __VA_ARGS__; } break;      \
        case 32: { constexpr int M = 32; __VA_ARGS__; } break;      \
        case 64: { constexpr int M = 64; __VA_ARGS__; } break;      \
        case 128: { constexpr int M = 128; __VA_ARGS__; } break;    \
        case 256: { constexpr int M = 256; __VA_ARGS__; } break;    \
        case 512: { constexpr int M = 512; __VA_ARGS__; } break;    \
        default: break;                                             \
    }

// next task of queue q for this CTA (-1 when the queue is empty); thread 0 pops, all see it
__device__ __forceinline__ int sw_pop(unsigned* head, int ntasks) {
    __shared__ int s_task;
    __syncthreads();                                             // the previous task's shared memory is free
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(head, 1u);
        s_task = t < (unsigned)ntasks ? (int)t : -1;
    }
    __syncthreads();
    return s_task;
}

// MINB: the resident CTAs per SM the register allocation is sized for (a tuned choice:
// more CTAs per SM hide more latency, fewer registers per thread spill more)
template <typename T, int MINB>
__global__ void __launch_bounds__(128, MINB) k_sweep_hvp(SweepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // phase 0: rows forward, `group` row blocks per task, one partial per row block
    for (int t = sw_pop(&a.heads[0], a.ntasks[0]); t >= 0; t = sw_pop(&a.heads[0], a.ntasks[0])) {
        const SweepTask k = a.tasks[0][t];
        const SweepProb<T>& p = a.probs[k.prob];
        for (int b = k.task * a.group; b < (k.task + 1) * a.group && b < p.row_blocks; ++b) {
            double s = 0.0;
            SW_SWITCH_M(p.m, s = sw_rows_fwd<T, M>(p.xf, b, smem_raw));
            if (threadIdx.x == 0) p.part[b] = s;
            __syncthreads();
        }
    }
    if (!grid_sync_acqrel(a.bar)) return;
    // phase 1: y lines with Lambda / N
    for (int t = sw_pop(&a.heads[32], a.ntasks[1]); t >= 0; t = sw_pop(&a.heads[32], a.ntasks[1])) {
        const SweepTask k = a.tasks[1][t];
        const SweepProb<T>& p = a.probs[k.prob];
        if (p.m == 512) sw_lines2d_smem<T, 512>(p.ca, k.task, smem_raw);
        else SW_SWITCH_M(p.m, if constexpr (M < 512) sw_lines2d<T, M>(p.ca, k.task, smem_raw));
    }
    if (!grid_sync_acqrel(a.bar)) return;
    // phase 2: rows inverse; the problem's mean of F''(phi) v from its partials, fixed order
    for (int t = sw_pop(&a.heads[64], a.ntasks[2]); t >= 0; t = sw_pop(&a.heads[64], a.ntasks[2])) {
        const SweepTask k = a.tasks[2][t];
        const SweepProb<T>& p = a.probs[k.prob];
        __shared__ T s_mean;
        if (threadIdx.x < 32) {
            double q = 0.0;
            for (int b = threadIdx.x; b < p.row_blocks; b += 32) q += __ldcg(&p.part[b]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
            if (threadIdx.x == 0) s_mean = (T)(q * p.xi.inv_n);
        }
        __syncthreads();
        const T mean = s_mean;
        for (int b = k.task * a.group; b < (k.task + 1) * a.group && b < p.row_blocks; ++b) {
            SW_SWITCH_M(p.m, sw_rows_inv<T, M>(p.xi, b, mean, smem_raw));
            __syncthreads();
        }
    }
}

}  // namespace lbtr
