// k_radix.cuh -- segmented, stable LSD radix sort of (key, value) pairs.
//
// This is the sort primitive of the paper (Definition "Sort", Sec. 2.2) as a
// GPU "onesweep" sort: one histogram pass computes the digit counts of every
// pass per segment, then every pass is one kernel whose tiles rank their keys
// locally and find their global output position with a decoupled look-back
// over the tiles before them.  Segments (problem instances of a batch) are
// sorted independently: tiles never straddle a segment and the look-back
// chains stop at the segment's first tile.  Stability (items with equal
// digits keep their order) is what lets the pipeline pre-order points by the
// last coordinate and then sort records by node key only (Sec. 5).
#pragma once
#include "dev_common.cuh"

namespace domagg {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;

template <typename K>
__device__ __forceinline__ u32 digit_of(K k, K keymask, int shift) {
    return (u32)((k & keymask) >> shift) & (u32)(RADIX - 1);
}

// Locates tile t: its segment and the half-open item range [start, end).
struct TileLoc {
    int seg;
    u32 seg_begin, seg_end, start, end;
    bool first;
};
template <int TILE>
__device__ __forceinline__ TileLoc locate_tile(u32 t, const u32* seg_off, const u32* tile_off, int nseg) {
    TileLoc L;
    L.seg = upper_index(tile_off, nseg + 1, t);
    L.seg_begin = __ldg(seg_off + L.seg);
    L.seg_end = __ldg(seg_off + L.seg + 1);
    u32 first_tile = __ldg(tile_off + L.seg);
    L.start = L.seg_begin + (t - first_tile) * (u32)TILE;
    L.end = min(L.start + (u32)TILE, L.seg_end);
    L.first = (t == first_tile);
    return L;
}

// Digit histograms of all passes, per segment: hist[(seg*npass + p)*RADIX + d].
template <typename K, int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS) void k_radix_hist(const K* __restrict__ keys, const u32* __restrict__ seg_off,
                                                        const u32* __restrict__ tile_off, int nseg, int npass,
                                                        int shift0, K keymask, u32* __restrict__ hist) {
    constexpr int TILE = THREADS * ITEMS;
    extern __shared__ u32 sh_hist[];  // [npass][RADIX]
    const u32 t = blockIdx.x;
    if (t >= __ldg(tile_off + nseg)) return;
    for (int x = threadIdx.x; x < npass * RADIX; x += THREADS) sh_hist[x] = 0;
    __syncthreads();
    TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    const u32 lt = lanemask_lt();
    for (u32 base = L.start; base < L.end; base += THREADS) {
        const u32 i = base + threadIdx.x;
        const bool valid = i < L.end;
        K k = valid ? keys[i] : K(0);
        for (int p = 0; p < npass; ++p) {
            u32 d = valid ? digit_of(k, keymask, shift0 + p * RADIX_BITS) : 0xffffu;
            u32 peers = __match_any_sync(0xffffffffu, d);
            if (valid && (peers & lt) == 0) atomicAdd(&sh_hist[p * RADIX + d], (u32)__popc(peers));
        }
    }
    __syncthreads();
    u32* gh = hist + (u64)L.seg * npass * RADIX;
    for (int x = threadIdx.x; x < npass * RADIX; x += THREADS)
        if (sh_hist[x]) atomicAdd(gh + x, sh_hist[x]);
}

// Exclusive scan of every (segment, pass) histogram plus the segment start:
// digit_off[(seg*npass + p)*RADIX + d] = global position of digit d's first item.
static __global__ __launch_bounds__(RADIX) void k_radix_offsets(const u32* __restrict__ hist, const u32* __restrict__ seg_off,
                                                         int npass, u32* __restrict__ digit_off) {
    __shared__ u32 warp_sum[RADIX / 32];
    const int sp = blockIdx.x, seg = sp / npass;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 v = hist[(u64)sp * RADIX + threadIdx.x];
    u32 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    u32 add = 0;
    for (int w = 0; w < warp; ++w) add += warp_sum[w];
    digit_off[(u64)sp * RADIX + threadIdx.x] = __ldg(seg_off + seg) + add + inc - v;
}

// Shared-memory footprint of one onesweep tile.
template <typename K, typename V, int THREADS, int ITEMS>
constexpr size_t onesweep_smem() {
    return (size_t)THREADS * ITEMS * (sizeof(K) + sizeof(V)) + (size_t)(THREADS / 32) * (RADIX + 1) * 4 +
           2 * RADIX * 4;
}

// One LSD pass: stable scatter of every segment by digit `pass`.
// IOTA: the values are the items' own global indices (first pass of a sort
// that returns a permutation); `vin` is not read.
template <typename K, typename V, int THREADS, int ITEMS, bool IOTA>
__global__ __launch_bounds__(THREADS) void k_onesweep(const K* __restrict__ kin, const V* __restrict__ vin,
                                                      K* __restrict__ kout, V* __restrict__ vout,
                                                      const u32* __restrict__ seg_off,
                                                      const u32* __restrict__ tile_off, int nseg,
                                                      const u32* __restrict__ digit_off, int npass, int pass,
                                                      int shift, K keymask, u64* status, Ctl* ctl,
                                                      int launch_idx) {
    constexpr int WARPS = THREADS / 32, TILE = THREADS * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    K* s_keys = reinterpret_cast<K*>(smem);
    V* s_vals = reinterpret_cast<V*>(s_keys + TILE);
    u32* s_whist = reinterpret_cast<u32*>(s_vals + TILE);  // [WARPS][RADIX+1]
    u32* s_dstart = s_whist + WARPS * (RADIX + 1);         // tile-local digit starts
    u32* s_gbase = s_dstart + RADIX;                       // counts, then global bases
    __shared__ u32 s_info[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_info[0] = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        s_info[1] = ctl->epoch_base + (u32)launch_idx;
    }
    for (int x = tid; x < WARPS * (RADIX + 1); x += THREADS) s_whist[x] = 0;
    __syncthreads();
    const u32 t = s_info[0], epoch = s_info[1];
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);

    // load: warp w owns items [start + w*32*ITEMS, ...), item i of lane l at
    // offset i*32 + l (coalesced), which is also the order of ranking.
    K key[ITEMS];
    V val[ITEMS];
    u32 dig[ITEMS], rnk[ITEMS];
    const u32 wbase = L.start + (u32)warp * 32u * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 idx = wbase + (u32)i * 32u + (u32)lane;
        if (idx < L.end) {
            key[i] = kin[idx];
            val[i] = IOTA ? (V)idx : vin[idx];
            dig[i] = digit_of(key[i], keymask, shift);
        } else {
            key[i] = K(0);
            val[i] = V(0);
            dig[i] = RADIX;  // padding: counted apart, never written
        }
    }
    // warp-level stable ranking
    u32* wh = s_whist + warp * (RADIX + 1);
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 d = dig[i];
        const u32 peers = __match_any_sync(0xffffffffu, d);
        const u32 before = wh[d];
        __syncwarp();
        rnk[i] = before + __popc(peers & lt);
        if ((peers & lt) == 0) wh[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive offsets of the warps, and the tile's count
    for (int d = tid; d < RADIX; d += THREADS) {
        u32 sum = 0;
        for (int w = 0; w < WARPS; ++w) {
            const u32 c = s_whist[w * (RADIX + 1) + d];
            s_whist[w * (RADIX + 1) + d] = sum;
            sum += c;
        }
        s_gbase[d] = sum;
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the tile counts over the digits
        constexpr int PER = RADIX / 32;
        u32 v[PER], s = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            v[j] = s_gbase[lane * PER + j];
            s += v[j];
        }
        u32 inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        u32 ex = inc - s;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            s_dstart[lane * PER + j] = ex;
            ex += v[j];
        }
    }
    __syncthreads();
    // publish, look back, and turn counts into global bases
    const u32 first_tile = t - (L.start - L.seg_begin) / (u32)TILE;
    for (int d = tid; d < RADIX; d += THREADS) {
        const u32 cnt = s_gbase[d];
        u64* st = status + (u64)t * RADIX + d;
        u32 excl = 0;
        if (L.first) {
            st_store(st, st_pack(epoch, ST_PREFIX, cnt));
        } else {
            st_store(st, st_pack(epoch, ST_AGG, cnt));
            excl = lookback_u32(status, RADIX, d, t, first_tile, epoch, ctl, 1u);
            st_store(st, st_pack(epoch, ST_PREFIX, excl + cnt));
        }
        s_gbase[d] = __ldg(digit_off + ((u64)L.seg * npass + pass) * RADIX + d) + excl - s_dstart[d];
    }
    __syncthreads();
    // local scatter: items grouped by digit, stable
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (dig[i] < RADIX) {
            const u32 pos = s_dstart[dig[i]] + s_whist[warp * (RADIX + 1) + dig[i]] + rnk[i];
            s_keys[pos] = key[i];
            s_vals[pos] = val[i];
        }
    }
    __syncthreads();
    // global scatter: consecutive threads write consecutive positions of a digit
    const u32 n = L.end - L.start;
    for (u32 x = tid; x < n; x += THREADS) {
        const K k = s_keys[x];
        const u32 dst = s_gbase[digit_of(k, keymask, shift)] + x;
        if (dst >= L.seg_begin && dst < L.seg_end) {  // only fails after a timed-out wait
            kout[dst] = k;
            vout[dst] = s_vals[x];
        }
    }
}

}  // namespace domagg
