// Per-kernel timing of libmrcm launches: CUDA events recorded on the
// launching stream around each kernel, and a launch counter that is always on.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

namespace mrcm {

struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;             // start/end pairs, reused after each report
    size_t used = 0;
    std::vector<int> kid;                      // kernel name id of each recorded pair
    std::vector<std::string> names;
    std::map<std::string, int> ids;
    long long launches = 0;                    // kernel launches since the last reset

    int id_of(const char* name) {
        auto it = ids.find(name);
        if (it != ids.end()) return it->second;
        int id = (int)names.size();
        names.emplace_back(name);
        ids.emplace(name, id);
        return id;
    }
    void begin(const char* name, cudaStream_t st) {
        ++launches;
        if (!on) return;
        while (pool.size() < used + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
            pool.push_back(e);
        }
        kid.push_back(id_of(name));
        cudaEventRecord(pool[used], st);
    }
    void end(cudaStream_t st) {
        if (!on) return;
        cudaEventRecord(pool[used + 1], st);
        used += 2;
    }
    void reset() { used = 0; kid.clear(); launches = 0; }
    void release() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
        pool.clear();
        reset();
    }
};

}  // namespace mrcm

// Launch a kernel with profiling brackets: MRCM_LAUNCH(prof, "name", stream, kernel<<<...>>>(...));
#define MRCM_LAUNCH(P, NAME, ST, ...) \
    do {                              \
        (P).begin(NAME, ST);          \
        __VA_ARGS__;                  \
        (P).end(ST);                  \
    } while (0)
