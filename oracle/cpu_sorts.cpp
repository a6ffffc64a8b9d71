// cpu_sorts.cpp -- the conventional CPU sorts the paper compares NN-sort against (Sec.
// "Experimental Study": std::sort and other library sorts), timed on the host cores as a baseline.
//
// TEST AND BASELINE INFRASTRUCTURE ONLY, beside the oracle: the benchmark's CPU-baseline leg is the
// only caller. The CUDA library never links, loads or calls this file.
//
//   algo 0: std::stable_sort, one thread
//   algo 1: std::sort, one thread
//   algo 2: parallel sort over `threads` host threads: std::sort of equal chunks, one per thread,
//           then rounds of pairwise std::merge (each round's merges run in parallel)
// Keys are float32, float64 or uint64, compared with operator< (NaN-free inputs). The sorted keys
// go to `out`; the return value is the wall time in seconds of the sort alone.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

template <typename T>
double run(const T *in, uint64_t n, T *out, int algo, int threads) {
    std::memcpy(out, in, n * sizeof(T));
    const auto t0 = std::chrono::steady_clock::now();
    if (algo == 0) {
        std::stable_sort(out, out + n);
    } else if (algo == 1) {
        std::sort(out, out + n);
    } else {
        const int T_ = std::max(1, threads);
        std::vector<uint64_t> cut(T_ + 1);
        for (int t = 0; t <= T_; ++t) cut[t] = n * (uint64_t)t / (uint64_t)T_;
        std::vector<std::thread> th;
        for (int t = 0; t < T_; ++t) th.emplace_back([&, t] { std::sort(out + cut[t], out + cut[t + 1]); });
        for (auto &x : th) x.join();
        std::vector<T> tmp(n);
        T *src = out, *dst = tmp.data();
        for (int width = 1; width < T_; width *= 2) {
            th.clear();
            for (int t = 0; t < T_; t += 2 * width) {
                const uint64_t a = cut[t], b = cut[std::min(t + width, T_)], c = cut[std::min(t + 2 * width, T_)];
                th.emplace_back([=] { std::merge(src + a, src + b, src + b, src + c, dst + a); });
            }
            for (auto &x : th) x.join();
            std::swap(src, dst);
        }
        if (src != out) std::memcpy(out, src, n * sizeof(T));
    }
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" double cpu_sort(const void *keys, int dtype, uint64_t n, void *out, int algo, int threads) {
    switch (dtype) {
    case 0: return run(static_cast<const float *>(keys), n, static_cast<float *>(out), algo, threads);
    case 1: return run(static_cast<const double *>(keys), n, static_cast<double *>(out), algo, threads);
    case 3: return run(static_cast<const uint64_t *>(keys), n, static_cast<uint64_t *>(out), algo, threads);
    default: return -1.0;
    }
}
