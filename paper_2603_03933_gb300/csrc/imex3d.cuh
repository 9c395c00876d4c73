// A whole subproblem solve (Algorithm 3, §3.2) of a 3D 128^3 float grid as ONE cooperative
// launch: the inner loop runs on the device from b_0 to the returned iterate d.
//
// Iteration j (d_j's spectrum after the z inverse sits in `spec`, laid out S[z][kx][ky] as
// in hvp3d.cuh):
//   phase A (planes)  y and x inverse transforms -> d_j in registers;
//                     b_j = d_j - eta (g + F''(phi) d_j) (eq. imex-scheme, right-hand side);
//                     x and y forward transforms back into `spec` (j = 0: d_0 is read from
//                     d0, or is dscale * g, and only the forward half runs)
//   grid barrier
//   phase B (z lines) forward z transform of four lines per warp, k = 0 removed; the sums of
//                     the stop test and the multiplier rule over the grid (one barrier): the
//                     residual ||b_{j-1} - b_j|| / eta of d_j (the identity g + (H + lambda_j
//                     I) d_j = (b_{j-1} - b_j) / eta), ||b_j||, the secular function at 0 and
//                     at lambda_j and its derivative; every CTA then takes the same decisions
//                     from the same totals (the Alg. 3 test, the lambda rule of eq.
//                     lambda_update_rule, a further grid sum per Newton step); b_j stored for
//                     the next residual, d_{j+1} = b_j / (1 + eta (Lambda + lambda_{j+1})) and
//                     the inverse z transform into `spec`.  The lines are parked in shared
//                     memory across the sums (every warp owns at most one task), and the solve
//                     and inverse with the current multiplier run while the grid sum's barrier
//                     waits; they are redone only when the rule moves the multiplier.
//   grid barrier
// When the test ends the loop at iteration j, the returned iterate d_j = F^{-1}[b_{j-1} /
// (1 + eta (Lambda + lambda_j))] is formed by one more z step and the planes' inverse and
// written to d.  The decisions are those of k_imex_lines (the same tests in the working
// precision, FP64 for the Newton steps, the same stall rule), and the state record that the
// host reads afterwards is the same ImexState.
//
// With phi, g, the spectrum and the two b buffers (42 MB) resident in the 129 MB L2, an
// iteration after the first moves almost nothing through HBM; its cost is three grid
// barriers, one L2 round of partial sums and the transforms.  Every barrier is bounded
// (GridBar budget): on expiry the error flag is set and the CTAs leave.
#pragma once
#include "hvp3d.cuh"
#include "imex_fused.cuh"

namespace lbtr {

template <typename T> struct Imex3Args {
    const T* phi;
    const T* g;
    const T* d0;              // initial point, or null: d_0 = (*dscale) g
    const double* dscale;
    T* d;                     // out: the returned iterate
    cplx<T>* spec;            // [M][M/2 + 1][M] complex work spectrum
    cplx<T>* b0;              // b_j for even j (same layout)
    cplx<T>* b1;              // b_j for odd j
    const cplx<T>* tw;
    const T* qtab;
    Model<T> model;           // tau, gamma and eta
    ImexState* st;            // zero before the launch
    Part<T>* partials;        // [2][5][gridDim]: per-CTA sums of two alternating rounds
    GridBar bar;
    T xi2, eta, kscale;       // kscale = 1 / N
    double r, rtol, steptol;
    int stall, max_iter;
    T t_thr_abs2, t_thr_rel2; // (eps_abs eta)^2, (eps_rel_abs eta)^2: residual^2 eta^2 below either = converged
    T t_r2, t_rtol_r2;        // r^2 and rtol r^2 of the multiplier rule
    T t_inv_n2;               // 1 / N^2
};

// dynamic shared memory: the fused product's plus the block-sum scratch (32 x 5 partials)
constexpr size_t I3_SMEM = H3::FSMEM + 32 * 5 * sizeof(double);
// largest grid the grid sums read in one round (the host launches at most this many CTAs)
constexpr int I3_MAXG = 256;
// z-line task warps per CTA; task warp w parks its lines in the scratch of warp w + that
// count, which has no task (so a grid needs at most 16 task warps per CTA)
__host__ __device__ constexpr int i3_task_warps(int grid) { return (H3::NTASKS + grid - 1) / grid; }

// phase A on plane z: b = d - eta (g + F''(phi) d), forward x and y transforms into spec
template <typename T>
__device__ __forceinline__ void i3_plane_b(const Imex3Args<T>& a, int z, bool first, unsigned char* smem_raw) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, H = G::H;
    const int tid = threadIdx.x, y = tid >> 3, j = tid & 7;
    const size_t row = (size_t)z * M + y;
    const C* pr = reinterpret_cast<const C*>(a.phi) + row * H;
    const C* gr = reinterpret_cast<const C*>(a.g) + row * H;
    C u[8];
    if (first) {
        if (a.d0) {
            const C* dr = reinterpret_cast<const C*>(a.d0) + row * H;
#pragma unroll
            for (int m = 0; m < 8; ++m) u[m] = dr[j + 8 * m];
        } else {
            const T ds = (T)(*a.dscale);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const C gg = gr[j + 8 * m];
                u[m] = mk<T>(ds * gg.x, ds * gg.y);
            }
        }
    } else {
        h3_inv_xy<T>(a.tw, a.spec, z, smem_raw, u, []() {});
    }
    const T eta = a.eta;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const C p = pr[j + 8 * m], gg = gr[j + 8 * m];
        u[m].x = u[m].x - eta * (gg.x + h3_f2(a.model, p.x) * u[m].x);
        u[m].y = u[m].y - eta * (gg.y + h3_f2(a.model, p.y) * u[m].y);
    }
    if (!first) __syncthreads();     // the inverse's reads of the hand-off buffer precede the forward's writes
    h3_fwd_xy<T>(a.tw, a.spec, z, smem_raw, u, []() {});
}

// Sum NQ per-CTA values over the grid.  Thread 0 of each CTA passes its CTA's totals in
// mine[]; after the barrier, warp q of every CTA adds all CTAs' values of quantity q in the
// same order (lane l: CTAs l, l + 32, ..., then a fixed shuffle tree), so every CTA leaves
// with the same totals in out[] (shared).  P: this round's [NQ][gridDim] buffer; consecutive rounds must
// alternate between two buffers (a CTA writes round k + 1 only after every CTA has arrived
// at round k + 1's barrier, i.e. has finished reading round k - 1).
template <typename T, int NQ>
__device__ __forceinline__ bool i3_grid_sum(const GridBar& bar, Part<T>* P, const Part<T>* mine, Part<T>* out) {
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) P[q * G + blockIdx.x] = mine[q];
    }
    if (!grid_sync_acqrel(bar)) return false;
    if ((int)(threadIdx.x >> 5) < NQ) {
        // warp q sums quantity q: every load issued before the first addition (one L2 round
        // trip), then the fixed order of the sums (the same in every CTA)
        const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
        Part<T> x[I3_MAXG / 32];
#pragma unroll
        for (int k = 0; k < I3_MAXG / 32; ++k) {
            if (lane + 32 * k < G) x[k] = part_ldcg(&P[q * G + lane + 32 * k]);
            else part_zero(x[k]);
        }
        Part<T> s = x[0];
#pragma unroll
        for (int k = 1; k < I3_MAXG / 32; ++k) s = part_add(s, x[k]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s = part_add(s, part_shfl_down(s, off));
        if (lane == 0) out[q] = s;
    }
    __syncthreads();
    return true;
}

// The first half of i3_grid_sum for NQ = 5, split so that work can run between the arrival
// and the wait: thread 0 publishes the CTA's totals, reads the barrier generation and
// arrives; the last arrival releases the others.  *gen_out / *last_out: shared results.
template <typename T>
__device__ __forceinline__ void i3_publish_arrive(const GridBar& bar, Part<T>* P, const Part<T>* mine,
                                                  unsigned* gen_out, int* last_out) {
    if (threadIdx.x == 0) {
        const int G = gridDim.x;
#pragma unroll
        for (int q = 0; q < 5; ++q) P[q * G + blockIdx.x] = mine[q];
        unsigned* gen = (unsigned*)bar.gen;
        *gen_out = ld_acquire_gpu(gen);
        const bool last = atom_add_acq_rel_gpu(bar.count, 1u) == (unsigned)G - 1u;
        if (last) {
            *bar.count = 0u;
            red_add_release_gpu(gen, 1u);
        }
        *last_out = last ? 1 : 0;
    }
    __syncthreads();
}

// The second half: thread `waiter` waits (bounded) for the generation to move on, then warp q
// sums quantity q of all CTAs in a fixed order into out[q] (as i3_grid_sum).  False when the
// wait gave up (the error flag is set).
template <typename T>
__device__ __forceinline__ bool i3_wait_sum(const GridBar& bar, const Part<T>* P, unsigned gen0, int last, int waiter,
                                            Part<T>* out) {
    __shared__ int s_ok;
    if ((int)threadIdx.x == waiter) {
        s_ok = 1;
        if (!last) {
            const unsigned* gen = (const unsigned*)bar.gen;
            const long long t0 = clock64();
            while (ld_acquire_gpu(gen) == gen0) {
                if (clock64() - t0 > bar.budget || *(volatile int*)bar.err != 0) {
                    atomicCAS(bar.err, 0, 5);
                    s_ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    if (!s_ok) return false;
    const int G = gridDim.x;
    if ((int)(threadIdx.x >> 5) < 5) {
        const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
        Part<T> x[I3_MAXG / 32];
#pragma unroll
        for (int k = 0; k < I3_MAXG / 32; ++k) {
            if (lane + 32 * k < G) x[k] = part_ldcg(&P[q * G + lane + 32 * k]);
            else part_zero(x[k]);
        }
        Part<T> s = x[0];
#pragma unroll
        for (int k = 1; k < I3_MAXG / 32; ++k) s = part_add(s, x[k]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s = part_add(s, part_shfl_down(s, off));
        if (lane == 0) out[q] = s;
    }
    __syncthreads();
    return true;
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_imex3(Imex3Args<T> a) {
    using G = H3;
    using C = cplx<T>;
    constexpr int M = G::M, NL = G::NLINES;
    enum { ACT_RETURN = 0, ACT_EVAL = 1, ACT_SOLVE = 2 };
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw + G::FSMEM);
    __shared__ Part<T> sh[5];
    __shared__ NewtonState ns;
    __shared__ double s_lam, s_lamp, s_best2;
    __shared__ T s_el, s_elp;
    __shared__ int s_act, s_best_it;
    ImexState* st = a.st;
    const int nb = gridDim.x, z = blockIdx.x;
    // The z-line geometry of this thread (its warp's task, the line, the weights) is
    // recomputed where it is used rather than carried through the plane phases, which need
    // every register.  One task per warp: the host launches at least NTASKS / 16 CTAs.
    struct Geo {
        int task, line, i;
        bool has, k0line;
        T bxy, qzc, wgt;
    };
    auto geo = [&]() {
        Geo q;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int nw = (G::NTASKS + nb - 1) / nb;
        q.task = warp * nb + z;
        q.has = warp < nw && q.task < G::NTASKS;
        q.i = lane >> 2;
        q.line = q.task * 4 + (lane & 3);
        const int kx = q.line >> 7, ky = q.line & (M - 1);
        q.bxy = q.has ? __ldg(&a.qtab[kx]) + __ldg(&a.qtab[M + ky]) : (T)0;
        q.qzc = __ldg(&a.qtab[2 * M + 1]);
        q.wgt = (kx == 0 || kx == G::H) ? (T)1 : (T)2;      // half-spectrum weight
        q.k0line = q.has && kx == 0 && ky == 0;
        return q;
    };
    // a_e = 1 + eta Lambda of element e = s * 8 + b of this thread (kz = i + 8 s + 16 b)
    auto kz_of = [](const Geo& q, int e) { return q.i + 8 * (e >> 3) + 16 * (e & 7); };
    auto a_of = [&](const Geo& q, int e) {
        const int kz = kz_of(q, e);
        const T kk = (T)(kz < M / 2 ? kz : kz - M);
        const T tt = (T)1 - (q.bxy + q.qzc * (kk * kk));
        return (T)1 + a.eta * a.xi2 * tt * tt;
    };
    auto scratch = [&]() { return reinterpret_cast<C*>(smem_raw + (threadIdx.x >> 5) * G::ZWARP); };
    // the lines of b_j parked across the grid sums (lane-private slots), in the z scratch of a
    // warp without a task: shared memory the plane phase reuses, but not before barrier B
    auto keepbuf = [&]() {
        return reinterpret_cast<C*>(smem_raw + (size_t)((threadIdx.x >> 5) + i3_task_warps(nb)) * G::ZWARP);
    };
    __shared__ unsigned s_gen;
    __shared__ int s_last;
    // the thread that waits at the sums' barrier: the first of the first warp without a z-line
    // task (the host launches grids with at most 16 task warps per CTA), so that the task
    // warps' speculative solve runs during the wait
    const int waiter = 32 * i3_task_warps(nb);
    if (threadIdx.x == 0) {
        s_lamp = 0.0;
        s_elp = (T)0;
        s_best2 = 0.0;
        s_best_it = 0;
    }
    Part<T>* P = a.partials;
    int round = 0;
    int j = 0;
    for (;; ++j) {
        const bool check = j > 0;
        // ---- phase A ----
        for (int zz = z; zz < M; zz += nb) {
            i3_plane_b<T>(a, zz, j == 0, smem_raw);
            __syncthreads();
        }
        if (!grid_sync_acqrel(a.bar)) return;
        // ---- phase B: forward z, the sums ----
        const Geo q = geo();
        const T elp = s_elp, eta = a.eta, cw = q.wgt * a.t_inv_n2;
        const C* bold = (j & 1) ? a.b0 : a.b1;               // b_{j-1}
        C* bnew = (j & 1) ? a.b1 : a.b0;                     // b_j
        const int lane = threadIdx.x & 31;
        C v[16];
        {
            T sm[2][5] = {};
            if (q.has) {
                h3_zfwd<T>(a.tw, a.spec, q.task, scratch(), v);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int kz = kz_of(q, e);
                    if (q.k0line && kz == 0) v[e] = mk<T>((T)0, (T)0);
                    const T ai = a_of(q, e);
                    const T x2 = v[e].x * v[e].x + v[e].y * v[e].y;
                    const T ci = cw * x2;
                    const T rd = rcp_t(ai + elp), ra = rcp_t(ai);
                    const T qv = ci * rd * rd;
                    sm[e & 1][1] += q.wgt * x2;
                    sm[e & 1][2] += ci * ra * ra;
                    sm[e & 1][3] += qv;
                    sm[e & 1][4] += (T)-2 * eta * qv * rd;
                }
                // the lines are parked in the warp's keep slots (lane-private) across the grid sums
                C* keep = keepbuf();
#pragma unroll
                for (int e = 0; e < 16; ++e) keep[e * 32 + lane] = v[e];
                if (check) {
                    // the residual ||b_{j-1} - b_j||^2: the loads of b_{j-1} in two batches of eight
                    // in flight at once (the lines' registers are free again), then the differences
                    // (measured: staging them in shared memory by asynchronous copies issued before
                    // the transform was slower, the copies competing with the transform's loads)
#pragma unroll
                    for (int h = 0; h < 16; h += 8) {
                        C o[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) o[e] = bold[(size_t)kz_of(q, h + e) * NL + q.line];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const C x = keep[(h + e) * 32 + lane];
                            const T dx = o[e].x - x.x, dy = o[e].y - x.y;
                            sm[e & 1][0] += q.wgt * (dx * dx + dy * dy);
                        }
                    }
                }
            }
            Acc<T> acc[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) { acc[k].add(sm[0][k]); acc[k].add(sm[1][k]); }
            Part<T> tot[5];
            block_part<T, 5>(acc, red, tot);
            i3_publish_arrive<T>(a.bar, P + (round & 1) * 5 * nb, tot, &s_gen, &s_last);
            // while the other CTAs arrive: b_j kept for the next residual, and d_{j+1} solved
            // with the current multiplier, the most common outcome of the lambda rule (redone
            // below when the rule moves lambda)
            if (q.has) {
                const T ks = a.kscale;
                const C* keep = keepbuf();
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    v[e] = keep[e * 32 + lane];
                    bnew[(size_t)kz_of(q, e) * NL + q.line] = v[e];
                    const T f = ks * rcp_t(a_of(q, e) + elp);
                    v[e] = mk<T>(v[e].x * f, v[e].y * f);
                }
                h3_zinv<T>(a.tw, a.spec, q.task, scratch(), v);
            }
            if (!i3_wait_sum<T>(a.bar, P + (round & 1) * 5 * nb, s_gen, s_last, waiter, sh)) return;
            ++round;
        }
        if (threadIdx.x == 0) {
            const T res2 = part_to_T(sh[0], T()) * a.t_inv_n2;        // (eta * residual)^2
            const T bn2 = part_to_T(sh[1], T()) * a.t_inv_n2;
            int act = ACT_SOLVE;
            if (check) {
                const bool bad = !isfinite(res2) || !isfinite(bn2);
                double best2 = s_best2;
                int best_it = s_best_it;
                const bool stall = stall_update(a.stall, j, (double)res2, best2, best_it);
                s_best2 = best2;
                s_best_it = best_it;
                const bool conv = res2 < a.t_thr_abs2 || res2 < a.t_thr_rel2;
                if (z == 0) { st->best2 = best2; st->best_it = best_it; }
                if (bad || conv || stall || j >= a.max_iter) {
                    if (z == 0) {
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
                if (check && z == 0) {
                    st->it = j;
                    st->residual = (double)(sqrt(res2 > (T)0 ? res2 : (T)0) / eta);
                    st->bnorm2 = (double)bn2;
                }
            }
            s_act = act;
        }
        __syncthreads();
        if (s_act == ACT_RETURN) break;
        while (s_act == ACT_EVAL) {
            const T el = s_el;
            T sm1[2][2] = {};
            if (q.has) {
                const C* keep = keepbuf();
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const C x = keep[e * 32 + (threadIdx.x & 31)];
                    const T rd = rcp_t(a_of(q, e) + el);
                    const T qv = cw * (x.x * x.x + x.y * x.y) * rd * rd;
                    sm1[e & 1][0] += qv;
                    sm1[e & 1][1] += (T)-2 * eta * qv * rd;
                }
            }
            Acc<T> ac2[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) { ac2[k].add(sm1[0][k]); ac2[k].add(sm1[1][k]); }
            Part<T> t2[2];
            block_part<T, 2>(ac2, red, t2);
            if (!i3_grid_sum<T, 2>(a.bar, P + (round & 1) * 5 * nb, t2, sh)) return;
            ++round;
            if (threadIdx.x == 0) {
                const bool more = newton_update(ns, part_to_double(sh[0]), part_to_double(sh[1]));
                s_lam = ns.lam;
                s_el = (T)(a.eta * ns.lam);
                s_act = more ? ACT_EVAL : ACT_SOLVE;
            }
            __syncthreads();
        }
        if (z == 0 && threadIdx.x == 0) {
            st->lam = s_lam;
            st->newton += ns.newton;
        }
        // ---- the diagonal solve and inverse z again, when the rule moved the multiplier ----
        // (s_el is bitwise elp whenever lambda_{j+1} = lambda_j: the rule then copies it)
        if (q.has && s_el != elp) {
            const T el = s_el, ks = a.kscale;
            const C* keep = keepbuf();
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                v[e] = keep[e * 32 + lane];
                const T f = ks * rcp_t(a_of(q, e) + el);
                v[e] = mk<T>(v[e].x * f, v[e].y * f);
            }
            h3_zinv<T>(a.tw, a.spec, q.task, scratch(), v);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_lamp = s_lam;
            s_elp = s_el;
        }
        if (!grid_sync_acqrel(a.bar)) return;
    }
    // ---- the returned iterate d_j from b_{j-1} and lambda_j ----
    {
        const Geo q = geo();
        if (q.has) {
            const C* bf = ((j - 1) & 1) ? a.b1 : a.b0;
            const T el = s_elp, ks = a.kscale;
            C v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const C o = bf[(size_t)kz_of(q, e) * NL + q.line];
                const T f = ks * rcp_t(a_of(q, e) + el);
                v[e] = mk<T>(o.x * f, o.y * f);
            }
            h3_zinv<T>(a.tw, a.spec, q.task, scratch(), v);
        }
    }
    if (!grid_sync_acqrel(a.bar)) return;
    for (int zz = z; zz < M; zz += nb) {
        C u[8];
        h3_inv_xy<T>(a.tw, a.spec, zz, smem_raw, u, []() {});
        const int y = threadIdx.x >> 3, jj = threadIdx.x & 7;
        C* dr = reinterpret_cast<C*>(a.d) + ((size_t)zz * M + y) * G::H;
#pragma unroll
        for (int m = 0; m < 8; ++m) dr[jj + 8 * m] = u[m];
        __syncthreads();
    }
}

}  // namespace lbtr
