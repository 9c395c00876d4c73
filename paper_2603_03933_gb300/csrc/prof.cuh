// Event-based per-kernel-class timing of a context's launches (profiling aid).
#pragma once
#include <cuda_runtime.h>
#include <vector>

namespace lbtr {

enum KClass { K_XFWD = 0, K_XINV = 1, K_XMID = 2, K_COLY = 3, K_COLI = 4, K_SECULAR = 5, K_REDUCE = 6, K_COUNT = 7 };

class Prof {
public:
    ~Prof() {
        for (auto e : pool_) cudaEventDestroy(e);
    }
    void reset() {
        flush();
        for (int i = 0; i < K_COUNT; ++i) { ms_[i] = 0.0; bytes_[i] = 0.0; launches_[i] = 0; }
    }
    cudaEvent_t begin(cudaStream_t s) {
        cudaEvent_t e = take();
        cudaEventRecord(e, s);
        return e;
    }
    void end(int cls, cudaEvent_t e0, cudaStream_t s, double bytes) {
        cudaEvent_t e1 = take();
        cudaEventRecord(e1, s);
        pending_.push_back(Rec{cls, e0, e1, bytes});
        if (pending_.size() >= 1024) flush();
    }
    // wait for every recorded pair and fold it into the totals
    void flush() {
        for (auto& r : pending_) {
            cudaEventSynchronize(r.b);
            float t = 0.f;
            cudaEventElapsedTime(&t, r.a, r.b);
            ms_[r.cls] += t;
            bytes_[r.cls] += r.bytes;
            launches_[r.cls] += 1;
        }
        pending_.clear();
        next_ = 0;
    }
    double ms(int c) const { return ms_[c]; }
    double bytes(int c) const { return bytes_[c]; }
    long long launches(int c) const { return launches_[c]; }

private:
    struct Rec { int cls; cudaEvent_t a, b; double bytes; };
    cudaEvent_t take() {
        if (next_ == pool_.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool_.push_back(e);
        }
        return pool_[next_++];
    }
    std::vector<cudaEvent_t> pool_;
    size_t next_ = 0;
    std::vector<Rec> pending_;
    double ms_[K_COUNT] = {0}, bytes_[K_COUNT] = {0};
    long long launches_[K_COUNT] = {0};
};

}  // namespace lbtr
