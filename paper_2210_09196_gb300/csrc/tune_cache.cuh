// Launch-shape tuning shared by pusch_autotune (single-cell handle) and pusch_batch_autotune (ragged batch): a
// text cache of "<key> | <value>" lines and CUDA-event timing of candidates.
#pragma once

#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace pusch {
namespace tune {

// Cache file: one "<key> | <value>" line per tuned item; later lines override earlier ones.
inline std::map<std::string, std::string> read_cache(const char *path) {
    std::map<std::string, std::string> m;
    if (!path) return m;
    FILE *f = fopen(path, "r");
    if (!f) return m;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        std::string l(line);
        while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
        const size_t bar = l.find(" | ");
        if (l.empty() || l[0] == '#' || bar == std::string::npos) continue;
        m[l.substr(0, bar)] = l.substr(bar + 3);
    }
    fclose(f);
    return m;
}

inline int value_of(const std::string &v, const char *name, int dflt) {
    const std::string pat = std::string(name) + "=";
    const size_t p = v.find(pat);
    if (p == std::string::npos) return dflt;
    return atoi(v.c_str() + p + pat.size());
}

// Mean milliseconds of `reps` runs of f on stream s (after one warm-up run).
template <typename F>
float time_ms(cudaStream_t s, int reps, F &&f, cudaError_t *err) {
    cudaEvent_t e0, e1;
    *err = cudaEventCreate(&e0);
    if (*err != cudaSuccess) return 0.f;
    if ((*err = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 0.f;
    }
    f();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) f();
    cudaEventRecord(e1, s);
    *err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (*err == cudaSuccess) *err = cudaEventElapsedTime(&ms, e0, e1);
    if (*err == cudaSuccess) *err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

// Appends lines to the cache file; false if it cannot be opened.
inline bool append_cache(const char *path, const std::vector<std::string> &lines) {
    if (!path || lines.empty()) return true;
    FILE *f = fopen(path, "a");
    if (!f) return false;
    for (const auto &l : lines) fprintf(f, "%s\n", l.c_str());
    fclose(f);
    return true;
}

}  // namespace tune
}  // namespace pusch
