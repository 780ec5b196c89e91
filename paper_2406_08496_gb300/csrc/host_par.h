// Host-side work spread over the host's threads (load-time preprocessing of
// the runtime, the assignment helpers).
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

namespace lpsim {

// f(first, last, piece) over fixed-size pieces of [0, n), spread over the
// host's threads; piece boundaries do not depend on the thread count, so
// anything reduced per piece and then added in piece order is reproducible.
constexpr uint64_t kPiece = 16384;

template <class F>
void parallel_pieces(uint64_t n, F &&f) {
    const uint64_t np = (n + kPiece - 1) / kPiece;
    const uint64_t hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nt = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(np, hw));
    if (nt <= 1) {
        for (uint64_t p = 0; p < np; p++) f(p * kPiece, std::min(n, (p + 1) * kPiece), p);
        return;
    }
    std::atomic<uint64_t> next{0};
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++)
        th.emplace_back([&] {
            for (uint64_t p; (p = next.fetch_add(1)) < np;) f(p * kPiece, std::min(n, (p + 1) * kPiece), p);
        });
    for (auto &x : th) x.join();
}

}  // namespace lpsim
