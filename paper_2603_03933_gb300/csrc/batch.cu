// Batches of independent problems (the phase-diagram sweep): one context per problem and
// the Hessian-vector products of all of them recorded as one CUDA graph.
//
// Problems on the x-row path (2D grids, 3D grids above 128^3) are grouped by grid size and
// precision; each group runs as three launches (rows forward, innermost lines, rows
// inverse) whose blockIdx.y selects a problem's argument struct from a device array, so a
// sweep of hundreds of small problems is a dozen launches instead of three per problem.
// Other problems (3D plane path) are separate branches.  Branches fork from a private
// capture stream into up to 16 side streams, largest first onto the least-loaded stream
// (a longest-first list schedule); they share no data and no scratch (one context each),
// so the GPU runs them side by side.  The graph is recorded on the first call with a given
// set of field pointers and replayed by later calls with the same pointers.
//
// Whole solves of a batch (lb_batch_tr_solve) run on a pool of host threads, one side
// stream each, that take problems from a shared queue, largest first; each thread drives
// Algorithm 1 for its problem as lb_imex_tr_solve does, so the GPU works on several
// problems at once while each driver waits on its own scalars.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ctx.cuh"
#include "sweep.cuh"

struct BatchGroup {                         // problems of one size on the x-row path
    int m = 0, rows = 0, col_grid = 0, col_tiles = 0;
    std::vector<int> members;
    void* args = nullptr;                     // device: [count] XfArgs, [count] ColArgs, [count] XiArgs
};

// The 2D problems of a batch whose products run as one persistent launch (sweep.cuh).
struct SweepState {
    std::vector<int> members;                // problems in the launch, largest first
    void* dev = nullptr;                     // device: probs, tasks (3 phases), partials, heads, barrier
    void* probs = nullptr;
    void* tasks[3] = {nullptr, nullptr, nullptr};
    int ntasks[3] = {0, 0, 0};
    unsigned* heads = nullptr;
    unsigned* bar = nullptr;
    int* err = nullptr;
    int grid = 0;                            // CTAs of the launch
    int occ = 0;                             // resident CTAs per SM the kernel allows
    int nsm = 0;
    int ctas_per_sm = 0;                     // chosen (0: occ)
    int group = 1;                           // row blocks per row task
    int min_blocks = 4;                      // register allocation of the kernel (float: 4 or 5)
    bool enabled = false;                    // the 2D problems take the persistent launch
    size_t smem = 0;
    void release() {
        if (dev) cudaFree(dev);
        dev = nullptr;
        members.clear();
    }
};

struct lb_batch {
    std::vector<lb_ctx*> ctx;
    SweepState sweep;
    lb_batch_tuning tuning{};               // the last tuning table (count 0: never tuned)
    std::vector<BatchGroup> groups;
    std::vector<int> order;                 // problems, largest first
    std::vector<int> lane;                  // side stream of each problem
    int nstreams = 0;
    cudaStream_t cap = nullptr;             // capture stream (never the caller's)
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;           // the pointers the graph was recorded with
    std::string err;

    void free_groups() {
        for (BatchGroup& g : groups) if (g.args) cudaFree(g.args);
        groups.clear();
    }
    ~lb_batch() {
        free_groups();
        sweep.release();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t s : side) if (s) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
        for (lb_ctx* c : ctx) lb_destroy(c);
    }
};

#define LB_SWEEP_M(mval, ...)                                       \
    switch (mval) {                                                 \
        case 16: { constexpr int M = 16; __VA_ARGS__; } break;      \
        case 32: { constexpr int M = 32; __VA_ARGS__; } break;      \
        case 64: { constexpr int M = 64; __VA_ARGS__; } break;      \
        case 128: { constexpr int M = 128; __VA_ARGS__; } break;    \
        case 256: { constexpr int M = 256; __VA_ARGS__; } break;    \
        case 512: { constexpr int M = 512; __VA_ARGS__; } break;    \
        default: break;                                             \
    }

namespace {
lb_status batch_fail(lb_batch* b, lb_status st, const std::string& msg) {
    if (b) b->err = msg;
    return st;
}
lb_status batch_cuda(lb_batch* b, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LB_OK;
    return batch_fail(b, LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
}  // namespace

// row blocks and line tiles of a 2D problem of M points per axis in the sweep kernel
static int sweep_row_blocks(int m) {
    int nr = 0;
    LB_SWEEP_M(m, nr = lbtr::RowGeo<M>::NR);
    return nr > 0 ? (m + nr - 1) / nr : 0;
}
static int sweep_line_tiles(int m) {
    const int nl = lbtr::sw_nl(m);
    return (m / 2 + nl - 1) / nl + 1;
}

// the instantiation of the persistent kernel for a register allocation of min_blocks CTAs
// per SM (float: 4 or 5; double: 1)
template <typename T> static const void* sweep_kernel(int min_blocks) {
    if constexpr (sizeof(T) == 8) return (const void*)lbtr::k_sweep_hvp<double, 1>;
    else return min_blocks >= 5 ? (const void*)lbtr::k_sweep_hvp<float, 5> : (const void*)lbtr::k_sweep_hvp<float, 4>;
}

// Collect the batch's 2D problems of working type T (16 <= M <= 512), build their argument
// structs for the given field pointers and the three task queues (largest grids first) and
// upload them; `group` row blocks form one row task.
template <typename T>
static lb_status build_sweep(lb_batch* b, const void* const* phi, const void* const* v, void* const* hv, int group) {
    SweepState& sw = b->sweep;
    sw.release();
    const bool want64 = sizeof(T) == 8;
    std::vector<lbtr::SweepProb<T>> probs;
    std::vector<long long> part_off;
    long long npart = 0;
    for (int i : b->order) {
        lb_ctx* c = b->ctx[i];
        if (c->prob.dim != 2 || c->prob.n < 16 || c->prob.n > 512 || (c->prec == LB_FP64) != want64) continue;
        lbtr::Plan<T>* pl = want64 ? reinterpret_cast<lbtr::Plan<T>*>(c->p64) : reinterpret_cast<lbtr::Plan<T>*>(c->p32);
        lbtr::SweepProb<T> sp{};
        int cg = 0, ct = 0;
        if (!pl->hvp_args((const T*)phi[i], (const T*)v[i], (T*)hv[i], sp.xf, sp.ca, cg, ct, sp.xi, true)) continue;
        sp.m = c->prob.n;
        sp.row_blocks = sweep_row_blocks(sp.m);
        sp.line_tiles = sweep_line_tiles(sp.m);
        part_off.push_back(npart);
        npart += sp.row_blocks;
        probs.push_back(sp);
        sw.members.push_back(i);
    }
    if (probs.empty()) return LB_OK;
    std::vector<lbtr::SweepTask> tk[3];
    for (int q = 0; q < (int)probs.size(); ++q) {
        const int rt = (probs[q].row_blocks + group - 1) / group;
        for (int t = 0; t < rt; ++t) { tk[0].push_back({q, t}); tk[2].push_back({q, t}); }
        for (int t = 0; t < probs[q].line_tiles; ++t) tk[1].push_back({q, t});
    }
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    const size_t o_probs = off; off += up(probs.size() * sizeof(lbtr::SweepProb<T>));
    size_t o_tk[3];
    for (int ph = 0; ph < 3; ++ph) { o_tk[ph] = off; off += up(tk[ph].size() * sizeof(lbtr::SweepTask)); }
    const size_t o_part = off; off += up((size_t)npart * sizeof(double));
    const size_t o_heads = off; off += up(3 * 32 * sizeof(unsigned));
    const size_t o_bar = off; off += up((64 + 32 * 65) * sizeof(unsigned));
    const size_t o_err = off; off += up(sizeof(int));
    lb_status st = batch_cuda(b, cudaMalloc(&sw.dev, off), "lb_batch_hessvec/sweep");
    if (st) { sw.dev = nullptr; return st; }
    char* base = static_cast<char*>(sw.dev);
    double* part = reinterpret_cast<double*>(base + o_part);
    for (size_t q = 0; q < probs.size(); ++q) probs[q].part = part + part_off[q];
    sw.probs = base + o_probs;
    for (int ph = 0; ph < 3; ++ph) { sw.tasks[ph] = base + o_tk[ph]; sw.ntasks[ph] = (int)tk[ph].size(); }
    sw.heads = reinterpret_cast<unsigned*>(base + o_heads);
    sw.bar = reinterpret_cast<unsigned*>(base + o_bar);
    sw.err = reinterpret_cast<int*>(base + o_err);
    sw.group = group;
    st = batch_cuda(b, cudaMemset(sw.dev, 0, off), "lb_batch_hessvec/sweep");
    if (!st) st = batch_cuda(b, cudaMemcpy(sw.probs, probs.data(), probs.size() * sizeof(lbtr::SweepProb<T>),
                                           cudaMemcpyHostToDevice), "lb_batch_hessvec/sweep");
    for (int ph = 0; ph < 3 && !st; ++ph)
        st = batch_cuda(b, cudaMemcpy(sw.tasks[ph], tk[ph].data(), tk[ph].size() * sizeof(lbtr::SweepTask),
                                      cudaMemcpyHostToDevice), "lb_batch_hessvec/sweep");
    if (st) return st;
    // residency: the launch is cooperative, at most occ CTAs per SM
    const size_t smem = lbtr::sw_smem<T>();
    const void* kern = sweep_kernel<T>(sw.min_blocks);
    st = batch_cuda(b, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                    "lb_batch_hessvec/sweep");
    int dev = 0;
    if (!st) st = batch_cuda(b, cudaGetDevice(&dev), "lb_batch_hessvec/sweep");
    if (!st) st = batch_cuda(b, cudaDeviceGetAttribute(&sw.nsm, cudaDevAttrMultiProcessorCount, dev), "lb_batch_hessvec/sweep");
    if (!st) st = batch_cuda(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sw.occ, kern, 128, smem),
                             "lb_batch_hessvec/sweep");
    if (st) return st;
    if (sw.occ < 1) { sw.release(); return LB_OK; }       // cannot be resident: the grouped launches serve
    sw.smem = smem;
    const int cps = sw.ctas_per_sm > 0 ? std::min(sw.ctas_per_sm, sw.occ) : sw.occ;
    sw.grid = sw.nsm * cps;
    return LB_OK;
}

// enqueue the persistent launch (the queue heads reset first) on stream s
template <typename T> static cudaError_t launch_sweep(lb_batch* b, cudaStream_t s) {
    SweepState& sw = b->sweep;
    cudaError_t e = cudaMemsetAsync(sw.heads, 0, 3 * 32 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    lbtr::SweepArgs<T> a{};
    a.probs = static_cast<const lbtr::SweepProb<T>*>(sw.probs);
    for (int ph = 0; ph < 3; ++ph) { a.tasks[ph] = static_cast<const lbtr::SweepTask*>(sw.tasks[ph]); a.ntasks[ph] = sw.ntasks[ph]; }
    a.group = sw.group;
    a.heads = sw.heads;
    a.bar.count = sw.bar; a.bar.gen = sw.bar + 32; a.bar.err = sw.err; a.bar.tree = sw.bar + 64;
    a.bar.budget = 4000000000LL;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(sweep_kernel<T>(sw.min_blocks), dim3(sw.grid), dim3(128), args, sw.smem, s);
}

// Group the problems on the x-row path by (precision, dimension, size) and upload each
// group's argument structs (they hold the field pointers of this call).
template <typename T>
static lb_status upload_group(lb_batch* b, BatchGroup& g, const void* const* phi, const void* const* v,
                              void* const* hv) {
    const int cnt = (int)g.members.size();
    std::vector<lbtr::XfArgs<T>> xf(cnt);
    std::vector<lbtr::ColArgs<T>> ca(cnt);
    std::vector<lbtr::XiArgs<T>> xi(cnt);
    for (int q = 0; q < cnt; ++q) {
        const int i = g.members[q];
        lbtr::Plan<T>* p = sizeof(T) == 8 ? reinterpret_cast<lbtr::Plan<T>*>(b->ctx[i]->p64)
                                          : reinterpret_cast<lbtr::Plan<T>*>(b->ctx[i]->p32);
        int cg = 0, ct = 0;
        p->hvp_args((const T*)phi[i], (const T*)v[i], (T*)hv[i], xf[q], ca[q], cg, ct, xi[q]);
    }
    const size_t bytes = cnt * (sizeof(lbtr::XfArgs<T>) + sizeof(lbtr::ColArgs<T>) + sizeof(lbtr::XiArgs<T>));
    lb_status st = batch_cuda(b, cudaMalloc(&g.args, bytes), "lb_batch_hessvec/arguments");
    if (st) { g.args = nullptr; return st; }
    char* d = static_cast<char*>(g.args);
    cudaMemcpy(d, xf.data(), cnt * sizeof(lbtr::XfArgs<T>), cudaMemcpyHostToDevice);
    d += cnt * sizeof(lbtr::XfArgs<T>);
    cudaMemcpy(d, ca.data(), cnt * sizeof(lbtr::ColArgs<T>), cudaMemcpyHostToDevice);
    d += cnt * sizeof(lbtr::ColArgs<T>);
    return batch_cuda(b, cudaMemcpy(d, xi.data(), cnt * sizeof(lbtr::XiArgs<T>), cudaMemcpyHostToDevice),
                      "lb_batch_hessvec/arguments");
}

static lb_status record_groups(lb_batch* b, const void* const* phi, const void* const* v, void* const* hv) {
    b->free_groups();
    const int n = (int)b->ctx.size();
    // the 2D problems run as one persistent launch when that strategy is chosen; the others
    // (and all problems otherwise) as grouped launches / branches
    b->sweep.release();
    if (b->sweep.enabled) {
        const int group = b->sweep.group > 0 ? b->sweep.group : 1;
        lb_status st = b->ctx[0]->prec == LB_FP64 ? build_sweep<double>(b, phi, v, hv, group)
                                                  : build_sweep<float>(b, phi, v, hv, group);
        if (st) return st;
    }
    std::vector<char> in_sweep(n, 0);
    for (int i : b->sweep.members) in_sweep[i] = 1;
    for (int i : b->order) {
        if (in_sweep[i]) continue;
        lb_ctx* c = b->ctx[i];
        int m = c->prob.n, rows = 0, cg = 0, ct = 0;
        bool ok;
        // 2D problems of 512 points per axis have no persistent line kernel: they stay branches
        // (measured: one grouped launch of 512-point Stockham line tiles, 307 us per replay of
        // the C4 sweep, was slower than the branches on forked streams, 262 us)
        const bool any_lines = false;
        if (c->prec == LB_FP64) {
            lbtr::XfArgs<double> xf; lbtr::ColArgs<double> ca; lbtr::XiArgs<double> xi;
            ok = c->p64->hvp_args((const double*)phi[i], (const double*)v[i], (double*)hv[i], xf, ca, cg, ct, xi,
                                  any_lines);
            rows = xf.rows;
        } else {
            lbtr::XfArgs<float> xf; lbtr::ColArgs<float> ca; lbtr::XiArgs<float> xi;
            ok = c->p32->hvp_args((const float*)phi[i], (const float*)v[i], (float*)hv[i], xf, ca, cg, ct, xi,
                                  any_lines);
            rows = xf.rows;
        }
        if (!ok) continue;
        BatchGroup* g = nullptr;
        for (BatchGroup& x : b->groups) {
            lb_ctx* c0 = b->ctx[x.members[0]];
            if (x.m == m && x.rows == rows && c0->prec == c->prec && c0->prob.dim == c->prob.dim &&
                x.col_grid == cg && x.col_tiles == ct) { g = &x; break; }
        }
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->m = m; g->rows = rows; g->col_grid = cg; g->col_tiles = ct;
        }
        g->members.push_back(i);
    }
    (void)n;
    for (BatchGroup& g : b->groups) {
        lb_status st = b->ctx[g.members[0]]->prec == LB_FP64 ? upload_group<double>(b, g, phi, v, hv)
                                                             : upload_group<float>(b, g, phi, v, hv);
        if (st) return st;
    }
    return LB_OK;
}

extern "C" {

lb_status lb_batch_create(const lb_problem* probs, int count, lb_precision prec, lb_batch** out) {
    if (!out) return LB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!probs || count <= 0) return LB_ERR_INVALID_ARG;
    lb_batch* b = new lb_batch();
    b->ctx.assign(count, nullptr);
    for (int i = 0; i < count; ++i) {
        lb_status st = lb_create(&probs[i], prec, &b->ctx[i]);
        if (st != LB_OK) {
            delete b;
            return st;
        }
    }
    // largest first, each onto the least-loaded side stream
    b->nstreams = std::min(count, 16);
    b->order.resize(count);
    for (int i = 0; i < count; ++i) b->order[i] = i;
    auto npts = [&](int i) { return b->ctx[i]->n(); };
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return npts(x) > npts(y); });
    std::vector<long long> load(b->nstreams, 0);
    b->lane.assign(count, 0);
    for (int i : b->order) {
        int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->lane[i] = k;
        load[k] += npts(i);
    }
    lb_status st = batch_cuda(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "lb_batch_create");
    b->side.assign(b->nstreams, nullptr);
    b->join.assign(b->nstreams, nullptr);
    for (int k = 0; k < b->nstreams && !st; ++k) {
        st = batch_cuda(b, cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking), "lb_batch_create");
        if (!st) st = batch_cuda(b, cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming), "lb_batch_create");
    }
    if (!st) st = batch_cuda(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "lb_batch_create");
    if (st) {
        delete b;
        return st;
    }
    *out = b;
    return LB_OK;
}

void lb_batch_destroy(lb_batch* b) { delete b; }

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err.c_str() : "null batch"; }

int lb_batch_size(const lb_batch* b) { return b ? (int)b->ctx.size() : 0; }

lb_status lb_batch_hessvec(lb_batch* b, const void* const* phi, const void* const* v, void* const* hv,
                           lb_stream stream) {
    if (!b || !phi || !v || !hv) return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_hessvec: null argument");
    const int n = (int)b->ctx.size();
    std::vector<const void*> key(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!phi[i] || !v[i] || !hv[i])
            return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_hessvec: null field pointer");
        if (((uintptr_t)phi[i] | (uintptr_t)v[i] | (uintptr_t)hv[i]) & 15u)
            return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_hessvec: fields must be 16-byte aligned");
        if (hv[i] == phi[i] || hv[i] == v[i])
            return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_hessvec: an output aliases an input");
        key[3 * i] = phi[i];
        key[3 * i + 1] = v[i];
        key[3 * i + 2] = hv[i];
    }
    lb_status st = LB_OK;
    if (!b->exec || key != b->key) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        b->key.clear();
        if ((st = record_groups(b, phi, v, hv))) return st;
        if ((st = batch_cuda(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal),
                             "lb_batch_hessvec/capture")))
            return st;
        cudaEventRecord(b->fork, b->cap);
        for (int k = 0; k < b->nstreams; ++k) cudaStreamWaitEvent(b->side[k], b->fork, 0);
        std::vector<long long> load(b->nstreams, 0);
        auto least = [&]() { return (int)(std::min_element(load.begin(), load.end()) - load.begin()); };
        std::vector<char> grouped(n, 0);
        cudaError_t le = cudaSuccess;
        if (!b->sweep.members.empty()) {
            const int k = least();
            long long pts = 0;
            for (int i : b->sweep.members) { grouped[i] = 1; pts += b->ctx[i]->n(); }
            load[k] += pts;
            cudaError_t e = b->ctx[0]->prec == LB_FP64 ? launch_sweep<double>(b, b->side[k])
                                                       : launch_sweep<float>(b, b->side[k]);
            if (e != cudaSuccess) le = e;
        }
        for (BatchGroup& g : b->groups) {
            const int k = least();
            const int cnt = (int)g.members.size();
            long long pts = 0;
            for (int i : g.members) { grouped[i] = 1; pts += b->ctx[i]->n(); }
            load[k] += pts;
            const lb_precision pr = b->ctx[g.members[0]]->prec;
            cudaError_t e;
            if (pr == LB_FP64) {
                auto* xf = static_cast<lbtr::XfArgs<double>*>(g.args);
                auto* ca = reinterpret_cast<lbtr::ColArgs<double>*>(xf + cnt);
                auto* xi = reinterpret_cast<lbtr::XiArgs<double>*>(ca + cnt);
                e = lbtr::launch_hvp_batch<double>(g.m, g.rows, cnt, xf, ca, g.col_grid, g.col_tiles, xi, b->side[k]);
            } else {
                auto* xf = static_cast<lbtr::XfArgs<float>*>(g.args);
                auto* ca = reinterpret_cast<lbtr::ColArgs<float>*>(xf + cnt);
                auto* xi = reinterpret_cast<lbtr::XiArgs<float>*>(ca + cnt);
                e = lbtr::launch_hvp_batch<float>(g.m, g.rows, cnt, xf, ca, g.col_grid, g.col_tiles, xi, b->side[k]);
            }
            if (e != cudaSuccess && le == cudaSuccess) le = e;
        }
        for (int i : b->order) {
            if (grouped[i]) continue;
            lb_ctx* c = b->ctx[i];
            const int k = least();
            load[k] += c->n();
            cudaStream_t s = b->side[k];
            if (c->prec == LB_FP64) c->p64->hessvec((const double*)phi[i], (const double*)v[i], (double*)hv[i], s);
            else c->p32->hessvec((const float*)phi[i], (const float*)v[i], (float*)hv[i], s);
        }
        for (int k = 0; k < b->nstreams; ++k) {
            cudaEventRecord(b->join[k], b->side[k]);
            cudaStreamWaitEvent(b->cap, b->join[k], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        cudaError_t le2 = cudaGetLastError();
        if (e == cudaSuccess) e = le != cudaSuccess ? le : le2;
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return batch_cuda(b, e, "lb_batch_hessvec/record");
        }
        b->graph = g;
        if ((st = batch_cuda(b, cudaGraphInstantiate(&b->exec, b->graph, 0), "lb_batch_hessvec/instantiate"))) {
            b->exec = nullptr;
            return st;
        }
        b->key = key;
    }
    return batch_cuda(b, cudaGraphLaunch(b->exec, (cudaStream_t)stream), "lb_batch_hessvec/launch");
}

// drop the recorded graph: the next product call records it with the current configuration
static void batch_invalidate(lb_batch* b) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->key.clear();
}

lb_status lb_batch_set_launch(lb_batch* b, int strategy, int min_blocks, int ctas_per_sm, int group) {
    if (!b || (strategy != 0 && strategy != 1) || ctas_per_sm < 0 || group < 1)
        return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_set_launch: bad argument");
    b->sweep.enabled = strategy == 1;
    b->sweep.min_blocks = min_blocks >= 5 ? 5 : 4;
    b->sweep.ctas_per_sm = ctas_per_sm;
    b->sweep.group = group;
    batch_invalidate(b);
    return LB_OK;
}

lb_status lb_batch_tune(lb_batch* b, const void* const* phi, const void* const* v, void* const* hv, int replays,
                        lb_batch_tuning* out, lb_stream stream) {
    if (!b || !phi || !v || !hv || replays < 1) return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_tune: bad argument");
    const bool f64 = b->ctx[0]->prec == LB_FP64;
    cudaStream_t s = (cudaStream_t)stream;
    SweepState& sw = b->sweep;
    // candidates: the grouped launches, then the persistent launch over register allocations,
    // resident CTAs per SM and row blocks per task
    struct Cand { int strategy, minb, cps, group; };
    std::vector<Cand> cand;
    cand.push_back({0, 0, 0, 1});
    for (int minb : (f64 ? std::vector<int>{4} : std::vector<int>{4, 5})) {
        int occ = 0;
        const void* kern = f64 ? sweep_kernel<double>(minb) : sweep_kernel<float>(minb);
        const size_t smem = f64 ? lbtr::sw_smem<double>() : lbtr::sw_smem<float>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 128, smem) != cudaSuccess || occ < 1)
            continue;
        std::vector<int> cps{occ};
        if ((occ + 1) / 2 < occ) cps.insert(cps.begin(), (occ + 1) / 2);
        for (int c : cps)
            for (int g : {1, 4})
                if ((int)cand.size() < 12) cand.push_back({1, minb, c, g});
    }
    const int keep_strategy = sw.enabled ? 1 : 0;
    const Cand keep{keep_strategy, sw.min_blocks, sw.ctas_per_sm, sw.group};
    lb_batch_tuning t{};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lb_status st = batch_cuda(b, cudaEventCreate(&e0), "lb_batch_tune");
    if (!st) st = batch_cuda(b, cudaEventCreate(&e1), "lb_batch_tune");
    for (const Cand& c : cand) {
        if (st) break;
        lb_batch_set_launch(b, c.strategy, c.minb, c.cps, c.group);
        // each candidate is timed as what a product call runs: its recorded graph, replayed
        for (int r = 0; r < 2 && !st; ++r) st = lb_batch_hessvec(b, phi, v, hv, stream);
        if (!st) st = batch_cuda(b, cudaEventRecord(e0, s), "lb_batch_tune");
        for (int r = 0; r < replays && !st; ++r) st = lb_batch_hessvec(b, phi, v, hv, stream);
        if (!st) st = batch_cuda(b, cudaEventRecord(e1, s), "lb_batch_tune");
        if (!st) st = batch_cuda(b, cudaEventSynchronize(e1), "lb_batch_tune");
        float ms = 0.f;
        if (!st) st = batch_cuda(b, cudaEventElapsedTime(&ms, e0, e1), "lb_batch_tune");
        if (!st && c.strategy == 1 && sw.err) {
            int herr = 0;
            cudaMemcpy(&herr, sw.err, sizeof(int), cudaMemcpyDeviceToHost);
            if (herr) st = batch_fail(b, LB_ERR_TIMEOUT, "lb_batch_tune: a grid barrier timed out");
        }
        if (st) break;
        t.strategy[t.count] = c.strategy;
        t.min_blocks[t.count] = c.minb;
        t.ctas_per_sm[t.count] = c.strategy ? std::min(c.cps, sw.occ) : 0;
        t.group[t.count] = c.group;
        t.us[t.count] = 1e3 * ms / replays;
        ++t.count;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) {
        lb_batch_set_launch(b, keep.strategy, keep.minb, keep.cps, keep.group);
        return st;
    }
    int best = 0;
    for (int k = 1; k < t.count; ++k)
        if (t.us[k] < t.us[best]) best = k;
    t.chosen = best;
    lb_batch_set_launch(b, t.strategy[best], t.min_blocks[best], t.ctas_per_sm[best], t.group[best]);
    b->tuning = t;
    if (out) *out = t;
    return LB_OK;
}

lb_status lb_batch_tr_solve(lb_batch* b, double* const* phi, const lb_tr_opts* opts, lb_tr_info* info,
                            int nthreads, lb_stream stream) {
    if (!b || !phi) return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_tr_solve: null argument");
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; ++i) {
        if (!phi[i]) return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_tr_solve: null field pointer");
        if ((uintptr_t)phi[i] & 15u)
            return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_tr_solve: fields must be 16-byte aligned");
        for (int j = 0; j < i; ++j)
            if (phi[j] == phi[i]) return batch_fail(b, LB_ERR_INVALID_ARG, "lb_batch_tr_solve: aliased fields");
    }
    const int nw = std::max(1, std::min({nthreads > 0 ? nthreads : 8, n, b->nstreams}));
    int dev = 0;
    lb_status st = batch_cuda(b, cudaGetDevice(&dev), "lb_batch_tr_solve");
    // the solves start after the caller's stream has produced the fields
    if (!st) st = batch_cuda(b, cudaEventRecord(b->fork, (cudaStream_t)stream), "lb_batch_tr_solve");
    for (int k = 0; k < nw && !st; ++k)
        st = batch_cuda(b, cudaStreamWaitEvent(b->side[k], b->fork, 0), "lb_batch_tr_solve");
    if (st) return st;
    std::vector<lb_tr_info> inf(n);
    std::vector<int> status(n, (int)LB_ERR_CUDA);     // until a worker has solved the problem
    std::atomic<int> next(0);
    auto worker = [&](int k) {
        if (cudaSetDevice(dev) != cudaSuccess) return;     // the other workers take its share
        for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
            const int i = b->order[q];
            lb_tr_opts oi;
            lb_default_tr_opts(&oi);
            if (opts) oi = *opts;
            std::string cp;     // each problem checkpoints to its own files
            if (oi.checkpoint_path) {
                cp = std::string(oi.checkpoint_path) + "." + std::to_string(i);
                oi.checkpoint_path = cp.c_str();
            }
            status[i] = (int)lb_imex_tr_solve(b->ctx[i], phi[i], &oi, &inf[i], (lb_stream)b->side[k]);
        }
    };
    std::vector<std::thread> pool;
    for (int k = 1; k < nw; ++k) {
        try {
            pool.emplace_back(worker, k);
        } catch (...) {     // no exception crosses the C ABI: run with the threads already started
            break;
        }
    }
    worker(0);
    for (std::thread& t : pool) t.join();
    // later work on the caller's stream sees the solved fields
    for (int k = 0; k < nw && !st; ++k) {
        st = batch_cuda(b, cudaEventRecord(b->join[k], b->side[k]), "lb_batch_tr_solve");
        if (!st) st = batch_cuda(b, cudaStreamWaitEvent((cudaStream_t)stream, b->join[k], 0), "lb_batch_tr_solve");
    }
    if (info) for (int i = 0; i < n; ++i) info[i] = inf[i];
    for (int i = 0; i < n && !st; ++i)
        if (status[i] != LB_OK) {
            st = (lb_status)status[i];
            b->err = "lb_batch_tr_solve: problem " + std::to_string(i) + ": " +
                     (next.load() > n ? lb_last_error(b->ctx[i]) : "no worker could select the device");
        }
    return st;
}

}  // extern "C"
