// Reductions for the LB kernels.
//
// Dot products, norms and energies are always accumulated to double accuracy.  On
// GB300 double-precision arithmetic runs at a small fraction of the float rate, so
// the float path accumulates in "double-float" form (an unevaluated sum hi + lo of
// two floats, each addition done with Knuth's error-free TwoSum), reduces warps and
// blocks in that form, and converts to double once per block.  The double path
// accumulates in double.  Block results go to a per-launch partials array; the last
// block to finish (atomic ticket) sums them in index order, so results are
// deterministic run to run.
#pragma once
#include "common.cuh"

namespace lbtr {

struct ff { float hi, lo; };

// TwoSum: s + e == a + b exactly.
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ ff ff_add(ff a, float b) {
    ff s = two_sum(a.hi, b);
    s.lo += a.lo;
    return two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return two_sum(s.hi, s.lo);
}

template <typename T> struct Acc;
template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ Acc() : v(0.0) {}
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void add_shfl(int off) { v += __shfl_down_sync(0xffffffffu, v, off); }
    __device__ __forceinline__ double get() const { return v; }
    __device__ __forceinline__ void merge(const Acc& o) { v += o.v; }
};
template <> struct Acc<float> {
    ff v;
    __device__ __forceinline__ Acc() { v.hi = 0.f; v.lo = 0.f; }
    __device__ __forceinline__ void add(float x) { v = ff_add(v, x); }
    __device__ __forceinline__ void add_shfl(int off) {
        ff o;
        o.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
        o.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
        v = ff_add(v, o);
    }
    __device__ __forceinline__ double get() const { return (double)v.hi + (double)v.lo; }
    __device__ __forceinline__ void merge(const Acc& o) { v = ff_add(v, o.v); }
};

// Block and grid partial sums in the accumulator's own form: a float-float pair for the
// float path (all arithmetic on the FP32 pipe), a double for the double path.
template <typename T> struct PartOf;
template <> struct PartOf<float> { using type = ff; };
template <> struct PartOf<double> { using type = double; };
template <typename T> using Part = typename PartOf<T>::type;

__device__ __forceinline__ ff part_of(const Acc<float>& a) { return a.v; }
__device__ __forceinline__ double part_of(const Acc<double>& a) { return a.v; }
__device__ __forceinline__ void part_zero(ff& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void part_zero(double& a) { a = 0.0; }
__device__ __forceinline__ ff part_add(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ double part_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff part_shfl_down(ff a, int off) {
    ff o;
    o.hi = __shfl_down_sync(0xffffffffu, a.hi, off);
    o.lo = __shfl_down_sync(0xffffffffu, a.lo, off);
    return o;
}
__device__ __forceinline__ double part_shfl_down(double a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }
__device__ __forceinline__ double part_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double part_to_double(double a) { return a; }
__device__ __forceinline__ float part_to_T(ff a, float) { return a.hi + a.lo; }
__device__ __forceinline__ double part_to_T(double a, double) { return a; }
// L2 load of a partial written by another block before a grid barrier
__device__ __forceinline__ ff part_ldcg(const ff* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    ff r;
    r.hi = v.x;
    r.lo = v.y;
    return r;
}
__device__ __forceinline__ double part_ldcg(const double* p) { return __ldcg(p); }

// Reduce NQ accumulators over the block; thread 0 receives the totals in out[] in the
// accumulator's form.  scratch: at least 32 * NQ doubles of shared memory.
template <typename T, int NQ>
__device__ __forceinline__ void block_part(Acc<T> (&a)[NQ], double* scratch, Part<T>* out) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a[q].add_shfl(off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    Part<T>* sp = reinterpret_cast<Part<T>*>(scratch);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) sp[q * 32 + warp] = part_of(a[q]);
    __syncthreads();
    // the warp totals are summed by warp 0 as a fixed shuffle tree (deterministic)
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            Part<T> t;
            if (lane < nw) t = sp[q * 32 + lane];
            else part_zero(t);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t = part_add(t, part_shfl_down(t, off));
            if (lane == 0) out[q] = t;
        }
    }
    __syncthreads();
}

// As block_part, with the totals converted to double (one conversion per quantity).
template <typename T, int NQ>
__device__ __forceinline__ void block_sum(Acc<T> (&a)[NQ], double* scratch, double* out) {
    Part<T> t[NQ];
    block_part<T, NQ>(a, scratch, t);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] = part_to_double(t[q]);
}

// Max-reduction of a non-negative value over the block; thread 0 receives it.
__device__ __forceinline__ double block_max(double v, double* scratch) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double m = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w) m = fmax(m, scratch[w]);
    __syncthreads();
    return m;
}

// GPU-scope atomics and loads with acquire / release semantics (PTX memory model)
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Partial-sum bookkeeping of one reduction launch.
struct RedSlot {
    double* partials;    // [nq][gridDim.x]
    double* result;      // [nq] finalised totals (max for quantities flagged in max_mask)
    unsigned* ticket;    // zero between launches; null: write the partials only
    int nq;
    unsigned max_mask;   // bit q set: quantity q is a max, not a sum
};

// Called by every block after thread 0 holds its block totals in vals[0..nq).
// The last block to arrive combines all partials in index order and resets the ticket.
__device__ __forceinline__ void finalize_partials(const RedSlot& rs, const double* vals) {
    __shared__ int am_last;
    const unsigned G = gridDim.x;
    if (!rs.ticket) {
        // partials only: a later kernel combines them
        if (threadIdx.x == 0)
            for (int q = 0; q < rs.nq; ++q) rs.partials[q * G + blockIdx.x] = vals[q];
        return;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < rs.nq; ++q) rs.partials[q * G + blockIdx.x] = vals[q];
        // release: this block's partials before its ticket; acquire: all partials for the last
        am_last = (atom_add_acq_rel_gpu(rs.ticket, 1u) == G - 1u);
    }
    __syncthreads();
    if (am_last) {
        for (int q = threadIdx.x >> 5; q < rs.nq; q += (blockDim.x >> 5) > 0 ? (blockDim.x >> 5) : 1) {
            // one warp per quantity; lane l sums blocks l, l + 32, ... in that order (deterministic);
            // the loads of a batch of 8 are independent, so they are in flight together
            const int lane = threadIdx.x & 31;
            const bool is_max = (rs.max_mask >> q) & 1u;
            double s = 0.0;
            for (unsigned b0 = lane; b0 < G; b0 += 256) {
                double x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = (b0 + 32 * j < G) ? __ldcg(&rs.partials[q * G + b0 + 32 * j]) : 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (b0 + 32 * j < G) s = is_max ? fmax(s, x[j]) : s + x[j];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                double o = __shfl_down_sync(0xffffffffu, s, off);
                s = is_max ? fmax(s, o) : s + o;
            }
            if (lane == 0) rs.result[q] = s;
        }
        if (threadIdx.x == 0) *rs.ticket = 0u;
    }
}

// Grid-wide barrier for cooperative launches with a bounded spin.
// Returns false (and sets *err = 5, the timeout status) if the wait exceeded
// `budget` SM clock cycles; callers then leave the kernel.
struct GridBar {
    unsigned* count;
    volatile unsigned* gen;
    int* err;
    long long budget;
    unsigned* tree;          // grid_reduce_sync: [0] groups done, [32 (1 + g)] arrivals of group g
                             // (every counter on its own 128-byte line, apart from gen)
};

__device__ __forceinline__ bool grid_sync(const GridBar& gb) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned my_gen = *gb.gen;
        __threadfence();
        unsigned arrived = atomicAdd(gb.count, 1u);
        if (arrived == gridDim.x - 1) {
            *gb.count = 0u;
            __threadfence();
            atomicAdd((unsigned*)gb.gen, 1u);
        } else {
            long long t0 = clock64();
            while (*gb.gen == my_gen) {
                if (*(volatile int*)gb.err != 0 || clock64() - t0 > gb.budget) {
                    atomicCAS(gb.err, 0, 5);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Grid barrier of the persistent kernels (the fused 128^3 product, the batched sweep): thread 0 of each CTA arrives with an acquire-release
// atomic (its CTA's earlier stores published by the release), the last arrival resets the
// count and releases the generation word, the others poll it with acquire loads.  The spin
// is bounded by gb.budget clock cycles; on expiry the error flag is set and false returned.
__device__ __forceinline__ bool grid_sync_acqrel(const GridBar& gb) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        unsigned* gen = (unsigned*)gb.gen;
        const unsigned my_gen = ld_acquire_gpu(gen);
        if (atom_add_acq_rel_gpu(gb.count, 1u) == gridDim.x - 1u) {
            *gb.count = 0u;
            red_add_release_gpu(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_gpu(gen) == my_gen) {
                if (clock64() - t0 > gb.budget || *(volatile int*)gb.err != 0) {
                    atomicCAS(gb.err, 0, 5);
                    ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

// Grid barrier that also sums NQ per-block values over a two-level tree.  Thread 0 of every
// block passes its block's values in `mine`.  Blocks form groups of 32 consecutive blocks;
// the last block of a group to arrive sums the group's values with one warp (one coalesced
// load per quantity, a fixed shuffle tree), and the last group to finish sums the group
// totals the same way, writes the totals to `tot` and releases the others.  Summation
// order depends only on block indices, so results do not depend on arrival order.  Every
// block leaves with the totals in `sh` (shared, NQ entries).  Storage: P [NQ][gridDim],
// Q [NQ][64] group totals (grids of at most 2048 blocks), tot [NQ]; gb.tree holds the
// group-completion counter and one arrival counter per group (each on its own 128-byte
// line, away from gen, which every waiting block polls), all zero between barriers.
// The spin of the waiting blocks is bounded as in grid_sync.
template <typename T, int NQ>
__device__ __forceinline__ bool grid_reduce_sync(const GridBar& gb, const Part<T>* mine, Part<T>* P, Part<T>* Q,
                                                 Part<T>* tot, Part<T>* sh) {
    __shared__ int s_role, s_ok;               // 0: wait, 1: sums its group, 2: sums the groups
    const int G = gridDim.x, blk = blockIdx.x, grp = blk >> 5;
    const int gsize = (G - (grp << 5)) < 32 ? (G - (grp << 5)) : 32, ng = (G + 31) >> 5;
    const int lane = threadIdx.x & 31;
    unsigned* gen = (unsigned*)gb.gen;
    unsigned my_gen = 0;
    if (threadIdx.x == 0) {
        s_ok = 1;
        s_role = 0;
        my_gen = ld_acquire_gpu(gen);            // read before arriving
#pragma unroll
        for (int q = 0; q < NQ; ++q) P[q * G + blk] = mine[q];
        // release: this block's values before its arrival; acquire: the group's values for its last
        if (atom_add_acq_rel_gpu(&gb.tree[32 * (1 + grp)], 1u) == (unsigned)gsize - 1u) s_role = 1;
    }
    __syncthreads();
    if (s_role >= 1 && threadIdx.x < 32) {
        Part<T> x[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (lane < gsize) x[q] = part_ldcg(&P[q * G + (grp << 5) + lane]);
            else part_zero(x[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x[q] = part_add(x[q], part_shfl_down(x[q], off));
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) Q[q * 64 + grp] = x[q];
            gb.tree[32 * (1 + grp)] = 0u;
            if (atom_add_acq_rel_gpu(&gb.tree[0], 1u) == (unsigned)ng - 1u) s_role = 2;
        }
        __syncwarp();
        if (__shfl_sync(0xffffffffu, s_role, 0) == 2) {
            // groups 0..31: one independent load per lane and quantity, all in flight together
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (lane < ng) x[q] = part_ldcg(&Q[q * 64 + lane]);
                else part_zero(x[q]);
            }
            if (ng > 32) {
                Part<T> y[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    if (lane + 32 < ng) y[q] = part_ldcg(&Q[q * 64 + 32 + lane]);
                    else part_zero(y[q]);
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q) x[q] = part_add(x[q], y[q]);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) x[q] = part_add(x[q], part_shfl_down(x[q], off));
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) { tot[q] = x[q]; sh[q] = x[q]; }
                gb.tree[0] = 0u;
                red_add_release_gpu(gen, 1u);        // totals and counter resets before the release
            }
        }
    }
    __syncthreads();
    if (s_role != 2 && threadIdx.x == 0) {
        const long long t0 = clock64();
        unsigned ns = 32;
        while (ld_acquire_gpu(gen) == my_gen) {
            if (*(volatile int*)gb.err != 0 || clock64() - t0 > gb.budget) {
                atomicCAS(gb.err, 0, 5);
                s_ok = 0;
                break;
            }
            __nanosleep(ns);               // back off: fewer polls of gen while the tree works
            if (ns < 256) ns *= 2;
        }
        if (s_ok)
#pragma unroll
            for (int q = 0; q < NQ; ++q) sh[q] = part_ldcg(&tot[q]);
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace lbtr
