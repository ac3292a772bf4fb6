// sort.cu -- host launcher of the segmented onesweep radix sort.
#include "host_common.h"
#include "k_points.cuh"
#include "k_radix.cuh"

#include <algorithm>
#include <atomic>

namespace domagg {

// Persistent grid: as many CTAs as fit on the GPU at once (from the
// occupancy calculator).
// Cached per device, so that a planned run (possibly under stream capture)
// makes no occupancy query.
template <typename K, typename V>
static u64 resident_ctas(size_t smem) {
    static std::atomic<int> cache[64];
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64) per_sm = cache[dev].load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<K, V, false, true>, ONESWEEP_THREADS, smem);
        per_sm = std::max(per_sm, 1);
        if (dev >= 0 && dev < 64) cache[dev].store(per_sm, std::memory_order_relaxed);
    }
    return (u64)std::max(sms, 1) * (u64)per_sm;
}

template <typename K, typename V, bool IOTA, bool STABLE>
static void launch_pass(Launcher& L, unsigned grid, size_t smem, K* kin, V* vin, K* kout, V* vout,
                        const SortSpace& sp, u32 range_items, const u32* seg_bits, const u32* range_base, int npass,
                        int p, K keymask, int li, bool uniform) {
    k_onesweep<K, V, IOTA, STABLE><<<grid, ONESWEEP_THREADS, smem, L.stream>>>(
        kin, vin, kout, vout, sp.seg_off, sp.tile_off, sp.nseg, range_items, seg_bits, range_base, sp.digit_off,
        npass, p, p * RADIX_BITS, keymask, sp.status, L.ctl, li, uniform ? 1 : 0);
}

template <typename K, typename V>
int sort_pairs(Launcher& L, const SortSpace& sp, K* keys[2], V* vals[2], bool iota, int total_bits, K keymask,
               int kind_hist, int kind_pass, const u32* seg_bits, bool stable, bool uniform) {
    constexpr u32 TILE = ONESWEEP_THREADS * onesweep_items<K, V>();
    static_assert(TILE >= SORT_MIN_TILE, "status words are sized for SORT_MIN_TILE");
    const int npass = (total_bits + RADIX_BITS - 1) / RADIX_BITS;
    // without host segment sizes, bounds: sum ceil(n_s / t) <= items / t + nseg
    const u64 ntiles = sp.seg_sizes ? tiles_of(*sp.seg_sizes, TILE) : sp.bound_items / TILE + sp.nseg;
    if (npass == 0 || ntiles == 0) return 0;
    constexpr size_t smem = onesweep_smem<K, V>();
    // the histogram's limit is set for the most passes a key type can need, so
    // that no later call lowers it under a captured launch that needs more
    constexpr int hist_smem_max = 8 * (int)(sizeof(K) * 8 / RADIX_BITS) * RADIX * (int)sizeof(u32);
    if (!L.frozen) {  // a planned run was preceded by an unfrozen one that set these
        cudaFuncSetAttribute(k_onesweep<K, V, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_onesweep<K, V, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_onesweep<K, V, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_onesweep<K, V, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_radix_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, hist_smem_max);
    }
    // ranges: about L.ranges_per_cta (4) per resident CTA, whole tiles, never
    // across segments.
    // With seg_bits, every pass ranges only the segments it moves (a segment
    // whose keys have no digit left stays in place), so later passes, which
    // move fewer segments, still spread over every CTA.
    const u64 G = resident_ctas<K, V>(smem);
    auto tiles_moved = [&](int p, u64 tile) -> u64 {
        if (!sp.seg_sizes) return sp.bound_items / tile + sp.nseg;  // bound: sum ceil(n_s / t) <= items / t + nseg
        if (!seg_bits || !sp.seg_bits_host) return tiles_of(*sp.seg_sizes, tile);
        u64 t = 0;
        for (size_t i = 0; i < sp.seg_sizes->size(); ++i)
            if ((u32)p * RADIX_BITS < (*sp.seg_bits_host)[i]) t += ((*sp.seg_sizes)[i] + tile - 1) / tile;
        return t;
    };
    auto plan_ranges = [&](int p, u32& range_items, u64& nranges) {
        const u64 nt = tiles_moved(p, TILE);
        const u64 R = (u64)std::max(1, L.ranges_per_cta) * G;
        const u64 rt = std::max<u64>(1, (nt + R - 1) / R);
        range_items = (u32)std::min<u64>(rt * TILE, 1ull << 30);
        nranges = nt == 0 ? 0 : tiles_moved(p, range_items);
    };
    u32 range_items = 0;
    u64 nranges = 0;
    plan_ranges(0, range_items, nranges);
    if (nranges == 0) return 0;
    // the first pass takes its range bases from the histogram (no count, no look-back)
    u32* range_base = (sp.range_scratch && nranges <= sp.range_scratch_ranges) ? sp.range_scratch : nullptr;
    L.start(KIND_SMALL, 0.0);
    k_make_tiles<<<1, 1024, 0, L.stream>>>(sp.seg_off, sp.nseg, range_items, sp.tile_off, seg_bits, 0u);
    L.stop();
    const int hist_smem = 8 * npass * RADIX * (int)sizeof(u32);  // per-warp histograms of every pass
    const size_t hist_bytes = (size_t)sp.nseg * npass * RADIX * sizeof(u32);
    cudaMemsetAsync(sp.hist, 0, hist_bytes, L.stream);
    L.start(kind_hist, sp.n_items * sizeof(K));
    k_radix_hist<K><<<(unsigned)nranges, 256, hist_smem, L.stream>>>(
        keys[0], sp.seg_off, sp.tile_off, sp.nseg, range_items, npass, 0, keymask, sp.hist, range_base, seg_bits,
        uniform ? 1 : 0);
    L.stop();
    L.start(KIND_SMALL, 0.0);
    k_radix_offsets<<<sp.nseg * npass, RADIX, 0, L.stream>>>(sp.hist, sp.seg_off, npass, sp.digit_off);
    L.stop();
    if (range_base) {
        L.start(KIND_SMALL, 0.0);
        k_range_bases<<<dim3(sp.nseg, RADIX / 32), RB_WARPS * 32, 0, L.stream>>>(sp.tile_off, sp.digit_off, npass,
                                                                                  range_base);
        L.stop();
    }
    int cur = 0;
    for (int p = 0; p < npass; ++p) {
        if (p > 0 && seg_bits) {  // this pass's own ranges
            plan_ranges(p, range_items, nranges);
            if (nranges == 0) break;  // no segment has digits left (nor will in later passes)
            L.start(KIND_SMALL, 0.0);
            k_make_tiles<<<1, 1024, 0, L.stream>>>(sp.seg_off, sp.nseg, range_items, sp.tile_off, seg_bits,
                                                   (u32)p * RADIX_BITS);
            L.stop();
        }
        const unsigned grid = (unsigned)std::min<u64>(G, nranges);
        const int li = L.lookback_index();
        // each pass reads and writes every (key, value) pair it moves once;
        // segments whose keys have fewer digits are not moved
        double moved = sp.n_items;
        if (seg_bits && sp.seg_bits_host && sp.seg_sizes) {
            moved = 0;
            for (size_t sgi = 0; sgi < sp.seg_sizes->size(); ++sgi)
                if ((u32)p * RADIX_BITS < (*sp.seg_bits_host)[sgi]) moved += (double)(*sp.seg_sizes)[sgi];
        }
        const double vbytes = (iota && p == 0) ? sizeof(V) : 2.0 * sizeof(V);
        L.start(kind_pass, moved * (2.0 * sizeof(K) + vbytes));
        const u32* rb = p == 0 ? range_base : nullptr;
        K *ki = keys[cur], *ko = keys[cur ^ 1];
        V *vi = vals[cur], *vo = vals[cur ^ 1];
        if (iota && p == 0) {
            if (stable) launch_pass<K, V, true, true>(L, grid, smem, ki, vi, ko, vo, sp, range_items, seg_bits, rb, npass, p, keymask, li, uniform);
            else launch_pass<K, V, true, false>(L, grid, smem, ki, vi, ko, vo, sp, range_items, seg_bits, rb, npass, p, keymask, li, uniform);
        } else {
            if (stable) launch_pass<K, V, false, true>(L, grid, smem, ki, vi, ko, vo, sp, range_items, seg_bits, rb, npass, p, keymask, li, uniform);
            else launch_pass<K, V, false, false>(L, grid, smem, ki, vi, ko, vo, sp, range_items, seg_bits, rb, npass, p, keymask, li, uniform);
        }
        L.stop();
        cur ^= 1;
    }
    return cur;
}

u32 bounds_site_sort(bool clear) {
#ifdef DOMAGG_CHECKED
    u32 hit = 0, site = 0;
    cudaMemcpyFromSymbol(&hit, g_bounds_hit, sizeof(u32));
    cudaMemcpyFromSymbol(&site, g_bounds_site, sizeof(u32));
    if (clear && hit) {
        const u32 z = 0;
        cudaMemcpyToSymbol(g_bounds_hit, &z, sizeof(u32));
    }
    cudaGetLastError();
    return hit ? (site ? site : 1u) : 0u;
#else
    (void)clear;
    return 0u;
#endif
}

template int sort_pairs<u32, u32>(Launcher&, const SortSpace&, u32**, u32**, bool, int, u32, int, int,
                                     const u32*, bool, bool);
template int sort_pairs<u64, u32>(Launcher&, const SortSpace&, u64**, u32**, bool, int, u64, int, int,
                                     const u32*, bool, bool);
template int sort_pairs<u32, u64>(Launcher&, const SortSpace&, u32**, u64**, bool, int, u32, int, int,
                                     const u32*, bool, bool);

}  // namespace domagg
