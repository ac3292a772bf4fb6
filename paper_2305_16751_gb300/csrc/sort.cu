// sort.cu -- host launcher of the segmented onesweep radix sort.
#include "host_common.h"
#include "k_points.cuh"
#include "k_radix.cuh"

#include <algorithm>

namespace domagg {

// Persistent grid: as many CTAs as fit on the GPU at once (from the
// occupancy calculator).
template <typename K, typename V, bool IOTA>
static u64 resident_ctas(size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<K, V, IOTA>, ONESWEEP_THREADS, smem);
    return (u64)std::max(sms, 1) * (u64)std::max(per_sm, 1);
}

template <typename K, typename V>
int sort_pairs(Launcher& L, const SortSpace& sp, K* keys[2], V* vals[2], bool iota, int total_bits, K keymask,
               int kind_hist, int kind_pass, const u32* seg_bits) {
    constexpr u32 TILE = ONESWEEP_THREADS * onesweep_items<K, V>();
    static_assert(TILE >= SORT_MIN_TILE, "status words are sized for SORT_MIN_TILE");
    const int npass = (total_bits + RADIX_BITS - 1) / RADIX_BITS;
    const u64 ntiles = tiles_of(*sp.seg_sizes, TILE);
    if (npass == 0 || ntiles == 0) return 0;
    constexpr size_t smem = onesweep_smem<K, V>();
    cudaFuncSetAttribute(k_onesweep<K, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_onesweep<K, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // ranges: about four per resident CTA, whole tiles, never across segments
    const u64 G = resident_ctas<K, V, false>(smem);
    const u64 rt = std::max<u64>(1, (ntiles + 4 * G - 1) / (4 * G));
    const u32 range_items = (u32)std::min<u64>(rt * TILE, 1ull << 30);
    const u64 nranges = tiles_of(*sp.seg_sizes, range_items);
    const unsigned grid = (unsigned)std::min<u64>(G, nranges);
    L.start(KIND_SMALL, 0.0);
    k_make_tiles<<<1, 1024, 0, L.stream>>>(sp.seg_off, sp.nseg, range_items, sp.tile_off);
    L.stop();
    const int hist_smem = 8 * npass * RADIX * (int)sizeof(u32);  // per-warp histograms of every pass
    cudaFuncSetAttribute(k_radix_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, hist_smem);
    const size_t hist_bytes = (size_t)sp.nseg * npass * RADIX * sizeof(u32);
    cudaMemsetAsync(sp.hist, 0, hist_bytes, L.stream);
    L.start(kind_hist, sp.n_items * sizeof(K));
    k_radix_hist<K><<<(unsigned)nranges, 256, hist_smem, L.stream>>>(
        keys[0], sp.seg_off, sp.tile_off, sp.nseg, range_items, npass, 0, keymask, sp.hist);
    L.stop();
    L.start(KIND_SMALL, 0.0);
    k_radix_offsets<<<sp.nseg * npass, RADIX, 0, L.stream>>>(sp.hist, sp.seg_off, npass, sp.digit_off);
    L.stop();
    int cur = 0;
    for (int p = 0; p < npass; ++p) {
        const int li = L.lookback_index();
        // each pass reads and writes every (key, value) pair once
        const double vbytes = (iota && p == 0) ? sizeof(V) : 2.0 * sizeof(V);
        L.start(kind_pass, sp.n_items * (2.0 * sizeof(K) + vbytes));
        if (iota && p == 0)
            k_onesweep<K, V, true><<<grid, ONESWEEP_THREADS, smem, L.stream>>>(
                keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], sp.seg_off, sp.tile_off, sp.nseg, range_items,
                seg_bits, sp.digit_off, npass, p, p * RADIX_BITS, keymask, sp.status, L.ctl, li);
        else
            k_onesweep<K, V, false><<<grid, ONESWEEP_THREADS, smem, L.stream>>>(
                keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], sp.seg_off, sp.tile_off, sp.nseg, range_items,
                seg_bits, sp.digit_off, npass, p, p * RADIX_BITS, keymask, sp.status, L.ctl, li);
        L.stop();
        cur ^= 1;
    }
    return cur;
}

template int sort_pairs<u32, u32>(Launcher&, const SortSpace&, u32**, u32**, bool, int, u32, int, int,
                                     const u32*);
template int sort_pairs<u64, u32>(Launcher&, const SortSpace&, u64**, u32**, bool, int, u64, int, int,
                                     const u32*);
template int sort_pairs<u32, u64>(Launcher&, const SortSpace&, u32**, u64**, bool, int, u32, int, int,
                                     const u32*);
template int sort_pairs<u64, u64>(Launcher&, const SortSpace&, u64**, u64**, bool, int, u64, int, int,
                                     const u32*);

}  // namespace domagg
