// host_common.h -- host-side helpers shared by the library's translation
// units: launch bookkeeping (look-back launch indices, optional per-launch
// CUDA-event timing) and the sort launcher's declaration.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dev_common.cuh"

namespace domagg {

// Kernel kinds for timing (see domagg_timing_kind_name).
enum Kind {
    KIND_ENCODE = 0,
    KIND_HIST_POINTS,
    KIND_SORT_POINTS,
    KIND_RANK,
    KIND_COUNT_SCAN,
    KIND_EXPAND,
    KIND_HIST_RECORDS,
    KIND_SORT_RECORDS,
    KIND_SEGSCAN,
    KIND_REDUCE,
    KIND_SMALL,  // begin, tile maps, digit offsets
    KIND_H2D,
    KIND_D2H,
    KIND_WAVELET,  // the level-wise passes
    KIND_SORT_GROUPS,  // m = 2: the points by their group of ranks
    KIND_GROUP,        // m = 2: the deep levels in shared memory (k_group)
    KIND_TOP,          // m = 2: the top levels per tile (k_top)
    KIND_COUNT_
};

struct TimedLaunch {
    int kind;
    double bytes;
    cudaEvent_t a, b;
};

struct Launcher {
    cudaStream_t stream = nullptr;
    Ctl* ctl = nullptr;
    int next_lookback = 0;
    bool timing = false;
    std::vector<TimedLaunch>* log = nullptr;
    std::vector<cudaEvent_t>* pool = nullptr;
    size_t* pool_used = nullptr;
    int pending_kind = -1;
    double pending_bytes = 0;
    cudaEvent_t pending_a = nullptr;
    int launches = 0;  // kernels launched (all kinds)
    bool frozen = false;  // a planned run: no allocation, no attribute changes (may be under stream capture)
    int ranges_per_cta = 4;   // sort: ranges per resident CTA (tunable)
    int blocks_per_sm = 16;   // flat map and reduction: grid-stride blocks per SM (tunable)

    // Index of the next look-back launch (its tile counter and epoch).  A run
    // restarts the count at every k_begin; the clamp keeps a miscount from
    // indexing past the counters.
    int lookback_index() {
        const int i = next_lookback++;
        return i < MAX_LAUNCHES ? i : MAX_LAUNCHES - 1;
    }

    cudaEvent_t take_event() {
        if (*pool_used == pool->size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool->push_back(e);
        }
        return (*pool)[(*pool_used)++];
    }
    void start(int kind, double bytes) {
        ++launches;
        if (!timing) return;
        pending_kind = kind;
        pending_bytes = bytes;
        pending_a = take_event();
        cudaEventRecord(pending_a, stream);
    }
    void stop() {
        if (!timing) return;
        cudaEvent_t b = take_event();
        cudaEventRecord(b, stream);
        log->push_back({pending_kind, pending_bytes, pending_a, b});
    }
};

// Workspace for one segmented sort.
struct SortSpace {
    const u32* seg_off;         // [nseg+1] device
    int nseg;
    const std::vector<u64>* seg_sizes;  // host copy of the segment sizes, or null (planned run: see bound_items)
    u32* tile_off;              // [nseg+1] device scratch (the sort's tile map)
    u32* hist;                  // [nseg*npass*RADIX]
    u32* digit_off;             // [nseg*npass*RADIX]
    u64* status;                // [tiles*RADIX], tiles of at least SORT_MIN_TILE items
    double n_items;             // items sorted (for the algorithmic byte model)
    u32* range_scratch = nullptr;  // [range_scratch_ranges*RADIX]: first-pass bases per range
    u64 range_scratch_ranges = 0;
    const std::vector<u32>* seg_bits_host = nullptr;  // host copy of seg_bits (byte model)
    u64 bound_items = 0;  // without seg_sizes: an upper bound on the items (the segment sizes are on the device only)
};



// Smallest tile any sort instantiation uses (status words are sized by it).
constexpr u32 SORT_MIN_TILE = 2048;
inline u64 tiles_of(const std::vector<u64>& sizes, u64 tile) {
    u64 t = 0;
    for (u64 n : sizes) t += (n + tile - 1) / tile;
    return t;
}

// Ranges the onesweep uses at most for these segment sizes (upper bound).
inline u64 sort_range_bound(const std::vector<u64>& sizes) {
    u64 t = 0;
    for (u64 n : sizes) t += (n + SORT_MIN_TILE - 1) / SORT_MIN_TILE;
    const u64 cap = 4096 + sizes.size();  // about four ranges per resident CTA, at least one per segment
    return t < cap ? t : cap;
}

// The same bound from the item count alone (segment sizes unknown on the host).
inline u64 sort_range_bound_n(u64 items, u64 nseg) {
    const u64 t = items / SORT_MIN_TILE + nseg;
    const u64 cap = 4096 + nseg;
    return t < cap ? t : cap;
}

// Point-phase scans (ranks, count scan) tile the points in 4096s.
constexpr u32 POINT_TILE = 4096;

// Checked build: the site of the first out-of-range index the kernels of
// sort.cu met (0 if none), cleared when `clear`.  Always 0 in the product
// build.
u32 bounds_site_sort(bool clear);

// Stable LSD sort of (key, value) pairs by bits [0, total_bits) of
// (key & keymask), segment by segment.  keys[0]/vals[0] hold the input;
// returns the index (0 or 1) of the buffers that hold the result.  With
// iota, the input values are the items' global indices (vals[0] unused).
// With seg_bits (device, one entry per segment), segment s is sorted by its
// first seg_bits[s] bits only and its result is in buffer
// ceil(seg_bits[s] / 8) % 2; the return value is then meaningless.
// stable = false allows any order among equal digits (for sorts whose result
// is only the sorted key sequence).  uniform: the keys' digits are spread
// evenly (m <= 2 node keys), which lets the histogram skip its skew guard.
template <typename K, typename V>
int sort_pairs(Launcher& L, const SortSpace& sp, K* keys[2], V* vals[2], bool iota, int total_bits, K keymask,
               int kind_hist, int kind_pass, const u32* seg_bits = nullptr, bool stable = true,
               bool uniform = false);

}  // namespace domagg
