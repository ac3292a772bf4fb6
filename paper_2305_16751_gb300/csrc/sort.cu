// sort.cu -- host launcher of the segmented onesweep radix sort.
#include "host_common.h"
#include "k_radix.cuh"

namespace domagg {

template <typename K, typename V>
int sort_pairs(Launcher& L, const SortSpace& sp, K* keys[2], V* vals[2], bool iota, int total_bits, K keymask,
               int kind_hist, int kind_pass) {
    const int npass = (total_bits + RADIX_BITS - 1) / RADIX_BITS;
    if (npass == 0 || sp.ntiles == 0) return 0;
    const size_t hist_bytes = (size_t)sp.nseg * npass * RADIX * sizeof(u32);
    cudaMemsetAsync(sp.hist, 0, hist_bytes, L.stream);
    L.start(kind_hist, sp.n_items * sizeof(K));
    k_radix_hist<K, SORT_THREADS, SORT_ITEMS>
        <<<sp.ntiles, SORT_THREADS, npass * RADIX * sizeof(u32), L.stream>>>(keys[0], sp.seg_off, sp.tile_off,
                                                                             sp.nseg, npass, 0, keymask, sp.hist);
    L.stop();
    L.start(KIND_SMALL, 0.0);
    k_radix_offsets<<<sp.nseg * npass, RADIX, 0, L.stream>>>(sp.hist, sp.seg_off, npass, sp.digit_off);
    L.stop();
    constexpr size_t smem = onesweep_smem<K, V, SORT_THREADS, SORT_ITEMS>();
    cudaFuncSetAttribute(k_onesweep<K, V, SORT_THREADS, SORT_ITEMS, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_onesweep<K, V, SORT_THREADS, SORT_ITEMS, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int cur = 0;
    for (int p = 0; p < npass; ++p) {
        const int li = L.lookback_index();
        // each pass reads and writes every (key, value) pair once
        const double vbytes = (iota && p == 0) ? sizeof(V) : 2.0 * sizeof(V);
        L.start(kind_pass, sp.n_items * (2.0 * sizeof(K) + vbytes));
        if (iota && p == 0)
            k_onesweep<K, V, SORT_THREADS, SORT_ITEMS, true><<<sp.ntiles, SORT_THREADS, smem, L.stream>>>(
                keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], sp.seg_off, sp.tile_off, sp.nseg, sp.digit_off,
                npass, p, p * RADIX_BITS, keymask, sp.status, L.ctl, li);
        else
            k_onesweep<K, V, SORT_THREADS, SORT_ITEMS, false><<<sp.ntiles, SORT_THREADS, smem, L.stream>>>(
                keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], sp.seg_off, sp.tile_off, sp.nseg, sp.digit_off,
                npass, p, p * RADIX_BITS, keymask, sp.status, L.ctl, li);
        L.stop();
        cur ^= 1;
    }
    return cur;
}

template int sort_pairs<u32, u32>(Launcher&, const SortSpace&, u32**, u32**, bool, int, u32, int, int);
template int sort_pairs<u64, u32>(Launcher&, const SortSpace&, u64**, u32**, bool, int, u64, int, int);
template int sort_pairs<u32, u64>(Launcher&, const SortSpace&, u32**, u64**, bool, int, u32, int, int);
template int sort_pairs<u64, u64>(Launcher&, const SortSpace&, u64**, u64**, bool, int, u64, int, int);

}  // namespace domagg
