// Event-pair timing of individual kernel launches (pdc_set_profiling).
#pragma once
#include <cstring>
#include <string>
#include <vector>

#include "pdc_internal.cuh"

namespace pdc {

// Event-pair timing of individual launches, or of a run of back-to-back
// launches of one kernel between a single pair of events (pdc_set_profiling).
struct Profiler {
    bool on = false;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
        double bytes;
        int launches;  // kernel launches between the two events
    };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<Rec> pending;
    std::vector<std::string> names;
    std::vector<pdc_kernel_time> acc;
    ~Profiler() {
        for (auto e : pool) cudaEventDestroy(e);
    }
    cudaEvent_t ev() {
        if (used == pool.size()) {
            cudaEvent_t e;
            PDC_CK(cudaEventCreate(&e));
            pool.push_back(e);
        }
        return pool[used++];
    }
    int kind(const char *name) {
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == name) return (int)i;
        names.push_back(name);
        pdc_kernel_time t;
        std::memset(&t, 0, sizeof(t));
        std::strncpy(t.name, name, sizeof(t.name) - 1);
        acc.push_back(t);
        return (int)names.size() - 1;
    }
    std::vector<size_t> open;  // nested begin/end pairs
    void begin(cudaStream_t s, const char *name, double bytes, int launches = 1) {
        Rec r;
        r.kind = kind(name);
        r.a = ev();
        r.b = ev();
        r.bytes = bytes;
        r.launches = launches;
        PDC_CK(cudaEventRecord(r.a, s));
        open.push_back(pending.size());
        pending.push_back(r);
    }
    void end(cudaStream_t s) {
        PDC_CK(cudaEventRecord(pending[open.back()].b, s));
        open.pop_back();
    }
    void flush() {
        for (auto &r : pending) {
            PDC_CK(cudaEventSynchronize(r.b));
            float ms = 0.f;
            PDC_CK(cudaEventElapsedTime(&ms, r.a, r.b));
            acc[r.kind].launches += r.launches;
            acc[r.kind].total_ms += ms;
            acc[r.kind].algo_bytes += r.bytes;
        }
        pending.clear();
        open.clear();
        used = 0;
    }
    void reset() {
        open.clear();
        pending.clear();
        used = 0;
        names.clear();
        acc.clear();
    }
};


}  // namespace pdc
