// partition.cu -- splitting a batch of covers among GPUs by byte volume.
//
// Covers and video frames are independent (the paper repeats its per-row
// routine for every row and frame, Section VI, last paragraph), so a batch
// shards across GPUs with no exchange step: each GPU embeds or extracts its
// own covers and only the per-cover results are gathered afterwards.  The
// split here balances the bytes each GPU streams: covers in decreasing size
// (ties by index), each to the GPU with the fewest bytes so far (ties to the
// lowest rank).  Every GPU then ends within one cover's bytes of every
// other: when the last cover a GPU received was placed, that GPU had the
// fewest bytes, and no later cover is larger.
//
// Host code only; no CUDA call.
#include <algorithm>
#include <functional>
#include <numeric>
#include <queue>
#include <utility>
#include <vector>

#include "internal.cuh"

// More ranks than any machine runs processes for is a caller's mistake.
constexpr uint32_t kMaxWorld = 1u << 16;

extern "C" int stego_partition(const uint64_t *bytes, uint32_t n, uint32_t world,
                               uint32_t *rank_of, uint64_t *rank_bytes)
{
    if (world == 0 || world > kMaxWorld || (n > 0 && (!bytes || !rank_of)))
        return STEGO_E_INVAL;
    std::vector<uint64_t> load(world, 0);
    std::vector<uint32_t> order(n);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return bytes[a] > bytes[b]; });
    // the least-loaded rank (the lowest of equals) on top of a heap
    using Entry = std::pair<uint64_t, uint32_t>;
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
    for (uint32_t r = 0; r < world; ++r)
        heap.push(Entry(0, r));
    for (uint32_t i : order) {
        const Entry e = heap.top();
        heap.pop();
        rank_of[i] = e.second;
        load[e.second] = e.first + bytes[i];
        heap.push(Entry(load[e.second], e.second));
    }
    if (rank_bytes)
        std::copy(load.begin(), load.end(), rank_bytes);
    return STEGO_OK;
}
