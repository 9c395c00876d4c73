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

struct BatchGroup {                         // problems of one size on the x-row path
    int m = 0, rows = 0, col_grid = 0, col_tiles = 0;
    std::vector<int> members;
    void* args = nullptr;                     // device: [count] XfArgs, [count] ColArgs, [count] XiArgs
};

struct lb_batch {
    std::vector<lb_ctx*> ctx;
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
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        for (cudaStream_t s : side) if (s) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
        for (lb_ctx* c : ctx) lb_destroy(c);
    }
};

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
    for (int i : b->order) {
        lb_ctx* c = b->ctx[i];
        int m = c->prob.n, rows = 0, cg = 0, ct = 0;
        bool ok;
        if (c->prec == LB_FP64) {
            lbtr::XfArgs<double> xf; lbtr::ColArgs<double> ca; lbtr::XiArgs<double> xi;
            ok = c->p64->hvp_args((const double*)phi[i], (const double*)v[i], (double*)hv[i], xf, ca, cg, ct, xi);
            rows = xf.rows;
        } else {
            lbtr::XfArgs<float> xf; lbtr::ColArgs<float> ca; lbtr::XiArgs<float> xi;
            ok = c->p32->hvp_args((const float*)phi[i], (const float*)v[i], (float*)hv[i], xf, ca, cg, ct, xi);
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
