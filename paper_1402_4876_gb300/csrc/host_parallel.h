// Host threads over independent chunks of work (SAM records, FASTQ
// records).  No CUDA.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

namespace mica {

constexpr unsigned MAX_HOST_THREADS = 256;

// The hardware's thread count, at least 1 and at most MAX_HOST_THREADS.
inline unsigned host_threads()
{
    return std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), MAX_HOST_THREADS));
}

// Runs f(c) for c = 0..n-1 on up to `threads` host threads (the caller's
// among them).  f must not throw.
template <typename F> void parallel_chunks(uint64_t n, unsigned threads, F f)
{
    std::atomic<uint64_t> next{0};
    auto worker = [&]() {
        for (uint64_t c; (c = next.fetch_add(1, std::memory_order_relaxed)) < n;) f(c);
    };
    const unsigned t = (unsigned)std::min<uint64_t>(threads, n);
    std::vector<std::thread> pool;
    try {
        pool.reserve(t);
        for (unsigned i = 1; i < t; i++) pool.emplace_back(worker);
    } catch (...) {   // fewer threads than asked: the started ones and this one finish the work
    }
    worker();
    for (auto &th : pool) th.join();
}

}  // namespace mica
