// Batches of independent problems (the phase-diagram sweep): one context per problem and
// the Hessian-vector products of all of them recorded as one CUDA graph.
//
// The graph forks from a private capture stream into up to 16 side streams; problems are
// placed largest first on the side stream with the least work so far (a longest-first
// list schedule, the static work queue of the batch), each as the three launches of its
// own hessvec.  Branches on different side streams share no data and no scratch, so the
// GPU runs them concurrently; the small grids of small problems fill the SMs together.
// The graph is recorded on the first call with a given set of field pointers and
// replayed by later calls with the same pointers.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"

struct lb_batch {
    std::vector<lb_ctx*> ctx;
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

    ~lb_batch() {
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
        if ((st = batch_cuda(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal),
                             "lb_batch_hessvec/capture")))
            return st;
        cudaEventRecord(b->fork, b->cap);
        for (int k = 0; k < b->nstreams; ++k) cudaStreamWaitEvent(b->side[k], b->fork, 0);
        for (int i : b->order) {
            lb_ctx* c = b->ctx[i];
            cudaStream_t s = b->side[b->lane[i]];
            if (c->prec == LB_FP64) c->p64->hessvec((const double*)phi[i], (const double*)v[i], (double*)hv[i], s);
            else c->p32->hessvec((const float*)phi[i], (const float*)v[i], (float*)hv[i], s);
        }
        for (int k = 0; k < b->nstreams; ++k) {
            cudaEventRecord(b->join[k], b->side[k]);
            cudaStreamWaitEvent(b->cap, b->join[k], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        cudaError_t le = cudaGetLastError();
        if (e == cudaSuccess) e = le;
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

}  // extern "C"
