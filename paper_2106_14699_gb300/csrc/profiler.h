// Optional per-launch CUDA-event timing of a plan's kernels (instrumentation).
#pragma once
#include <cuda_runtime.h>
#include <vector>

namespace cmif {

struct Profiler {
    bool enabled = false;
    std::vector<cudaEvent_t> ev;  // pairs (start, stop)
    std::vector<const char*> names;
    size_t used = 0;              // pairs recorded in the current call
    int open = -1;

    void reset() { used = 0; open = -1; }
    void begin(const char* name, cudaStream_t s) {
        if (!enabled) return;
        if (2 * (used + 1) > ev.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            ev.push_back(a);
            ev.push_back(b);
        }
        if (names.size() < used + 1) names.resize(used + 1);
        names[used] = name;
        cudaEventRecord(ev[2 * used], s);
        open = (int)used;
    }
    void end(cudaStream_t s) {
        if (!enabled || open < 0) return;
        cudaEventRecord(ev[2 * open + 1], s);
        used = open + 1;
        open = -1;
    }
    void destroy() {
        for (auto e : ev) cudaEventDestroy(e);
        ev.clear();
    }
};

}  // namespace cmif
