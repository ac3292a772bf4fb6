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

// Locates range r of `range_items` items: its segment and [start, end).
__device__ __forceinline__ TileLoc locate_range(u32 r, const u32* seg_off, const u32* range_off, int nseg,
                                                u32 range_items) {
    TileLoc L;
    L.seg = upper_index(range_off, nseg + 1, r);
    L.seg_begin = __ldg(seg_off + L.seg);
    L.seg_end = __ldg(seg_off + L.seg + 1);
    const u32 first = __ldg(range_off + L.seg);
    L.start = L.seg_begin + (r - first) * range_items;
    L.end = min(L.start + range_items, L.seg_end);
    L.first = (r == first);
    return L;
}

// Digit histograms of all passes, per segment: hist[(seg*npass + p)*RADIX + d].
// One block per range of `range_items` items (ranges never straddle a
// segment); counts are aggregated per warp with match_any before the
// shared-memory atomics, so skewed digits do not serialise.  With seg_bits,
// a segment only counts the passes its keys have digits for (the others
// skip it).  With `uniform` (keys whose digits are spread evenly, as the
// m <= 2 node keys: a prefix of a dense rank), digits with at least 5
// significant bits are counted with plain shared atomics.
template <typename K>
__global__ __launch_bounds__(256) void k_radix_hist(const K* __restrict__ keys, const u32* __restrict__ seg_off,
                                                    const u32* __restrict__ range_off, int nseg, u32 range_items,
                                                    int npass, int shift0, K keymask, u32* __restrict__ hist,
                                                    u32* __restrict__ range_cnt0, const u32* __restrict__ seg_bits,
                                                    int uniform) {
    extern __shared__ u32 sh_hist[];  // [8 warps][npass][RADIX]
    const u32 r = blockIdx.x;
    if (r >= __ldg(range_off + nseg)) return;
    const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int x = threadIdx.x; x < 8 * npass * RADIX; x += 256) sh_hist[x] = 0;
    __syncthreads();
    const TileLoc L = locate_range(r, seg_off, range_off, nseg, range_items);
    const int sbits = seg_bits ? (int)__ldg(seg_bits + L.seg) : 0;
    const int np = seg_bits ? min(npass, (sbits + RADIX_BITS - 1) / RADIX_BITS) : npass;
    // passes [0, spread) have digits with at least 5 significant bits
    const int spread = (seg_bits && uniform && sbits >= 5) ? min(np, (sbits - 5) / RADIX_BITS + 1) : 0;
    u32* wh = sh_hist + warp * npass * RADIX;
    for (u32 base = L.start; base < L.end; base += 256u * 8u) {
        K kk[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const u32 x = base + (u32)j * 256u + threadIdx.x;
            kk[j] = x < L.end ? keys[x] : K(0);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool valid = base + (u32)j * 256u + threadIdx.x < L.end;
            for (int p = 0; p < np; ++p) {
                const u32 d = digit_of(kk[j], keymask, shift0 + p * RADIX_BITS);
                // a digit with at least 5 significant bits of a node key is spread
                // out: plain shared atomics; otherwise (and for point keys, whose
                // spread is unknown) lanes sharing lane 0's digit add together
                if (p < spread) {
                    if (valid) atomicAdd(wh + p * RADIX + d, 1u);
                } else {
                    warp_hist_add(wh + p * RADIX, d, valid, lane);
                }
            }
        }
    }
    __syncthreads();
    u32* gh = hist + (u64)L.seg * npass * RADIX;
    for (int x = threadIdx.x; x < npass * RADIX; x += 256) {
        u32 c = 0;
        for (int w = 0; w < 8; ++w) c += sh_hist[w * npass * RADIX + x];
        if (c) atomicAdd(gh + x, c);
        if (range_cnt0 && x < RADIX) range_cnt0[(u64)r * RADIX + x] = c;  // this range's first-pass counts
    }
}

// First-pass global position of every (range, digit): the digit's start in
// the segment plus the counts of the segment's earlier ranges.  In place over
// the per-range counts.  Grid (segment, group of 32 digits); the 32 warps of
// a block split the segment's ranges into 32 slices (lane = digit): slice
// sums, an exclusive scan of them in shared memory, then the running bases.
constexpr int RB_WARPS = 32;
static __global__ __launch_bounds__(RB_WARPS * 32) void k_range_bases(const u32* __restrict__ range_off,
                                                                     const u32* __restrict__ digit_off, int npass,
                                                                     u32* __restrict__ range_cnt0) {
    __shared__ u32 s_sum[RB_WARPS][33];
    const int seg = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = blockIdx.y * 32 + lane;
    const u32 r0 = __ldg(range_off + seg), r1 = __ldg(range_off + seg + 1);
    const u32 n = r1 - r0, per = (n + RB_WARPS - 1) / RB_WARPS;
    const u32 a = r0 + min(n, (u32)warp * per), b = r0 + min(n, (u32)(warp + 1) * per);
    u32 sum = 0;
    for (u32 r = a; r < b; r += 16) {  // 16 loads in flight
        u32 c[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) c[i] = r + i < b ? range_cnt0[(u64)(r + i) * RADIX + d] : 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) sum += c[i];
    }
    s_sum[warp][lane] = sum;
    __syncthreads();
    u32 run = __ldg(digit_off + (u64)seg * npass * RADIX + d);  // pass 0
    for (int w = 0; w < warp; ++w) run += s_sum[w][lane];
    for (u32 r = a; r < b; r += 16) {
        u32 c[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) c[i] = r + i < b ? range_cnt0[(u64)(r + i) * RADIX + d] : 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (r + i < b) range_cnt0[(u64)(r + i) * RADIX + d] = run;
            run += c[i];
        }
    }
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

// Items per thread of a onesweep tile: ONESWEEP_TILE_BYTES of (key, value)
// pairs per tile.
#ifndef ONESWEEP_TILE_BYTES
#define ONESWEEP_TILE_BYTES 32768
#endif
template <typename K, typename V>
__host__ __device__ constexpr int onesweep_items() {
    return ONESWEEP_TILE_BYTES / 256 / (int)(sizeof(K) + sizeof(V));
}
constexpr int ONESWEEP_THREADS = 256;
#ifndef ONESWEEP_MIN_CTAS
#define ONESWEEP_MIN_CTAS 3
#endif

// Shared-memory layout of the persistent onesweep kernel: two tile buffers
// (keys, then values, each with 16 bytes of alignment slack at both ends),
// the warp histograms and the per-digit bases.
template <typename K, typename V, int TILE>
struct OnesweepSmem {
    static constexpr int WARPS = ONESWEEP_THREADS / 32;
    static constexpr size_t KBYTES = ((size_t)(TILE + 2 * 16 / sizeof(K)) * sizeof(K) + 15) & ~(size_t)15;
    static constexpr size_t VBYTES = ((size_t)(TILE + 2 * 16 / sizeof(V)) * sizeof(V) + 15) & ~(size_t)15;
    static constexpr size_t BUF = KBYTES + VBYTES;
    static constexpr size_t WHIST = (size_t)WARPS * (RADIX + 1) * 4;
    static constexpr size_t TOTAL = 2 * BUF + WHIST + 2 * RADIX * 4 + 64;
};

template <typename K, typename V>
__host__ __device__ constexpr size_t onesweep_smem() {
    return OnesweepSmem<K, V, ONESWEEP_THREADS * onesweep_items<K, V>()>::TOTAL;
}

// One LSD pass: stable scatter of every segment by digit `pass`.
//
// Persistent CTAs claim ranges of consecutive tiles from a global counter,
// in increasing order.  For a range the CTA
//   1. counts its digits (one read of the keys),
//   2. publishes the count and runs one decoupled look-back over the earlier
//      ranges of the segment (bounded waits), which gives the global position
//      of the range's first item of every digit,
//   3. streams the range tile by tile: the next tile's keys and values are
//      fetched into the other shared-memory buffer by TMA bulk copies
//      (cp.async.bulk, completion on an mbarrier) while the current tile is
//      ranked (warp-level stable match_any ranking), sorted locally in shared
//      memory and written out with coalesced stores at running per-digit
//      positions.
// There is no inter-CTA wait inside a range; the look-back runs once per
// range (hundreds of thousands of items), not once per tile.
//
// IOTA: the values are the items' own global indices (first pass of a sort
// that returns a permutation); `vin` is not read.
// STABLE = false (the dense-rank sorts, where only the sorted key sequence
// matters) ranks with one shared-memory atomic per item instead of the digit
// match.  range_base (first pass only, may be null) holds every range's
// global position per digit, which replaces the range's count and look-back.
template <typename K, typename V, bool IOTA, bool STABLE>
__global__ __launch_bounds__(ONESWEEP_THREADS, ONESWEEP_MIN_CTAS) void k_onesweep(
    const K* __restrict__ kin, const V* __restrict__ vin, K* __restrict__ kout, V* __restrict__ vout,
    const u32* __restrict__ seg_off, const u32* __restrict__ range_off, int nseg, u32 range_items,
    const u32* __restrict__ seg_bits, const u32* __restrict__ range_base, const u32* __restrict__ digit_off,
    int npass, int pass, int shift, K keymask, u64* status, Ctl* ctl, int launch_idx, int uniform) {
    constexpr int THREADS = ONESWEEP_THREADS, ITEMS = onesweep_items<K, V>();
    constexpr int TILE = THREADS * ITEMS, WARPS = THREADS / 32;
    typedef OnesweepSmem<K, V, TILE> SM;
    constexpr u32 KAL = 16 / sizeof(K), VAL = 16 / sizeof(V);  // items per 16 bytes
    extern __shared__ __align__(128) unsigned char smem[];
    u32* s_whist = reinterpret_cast<u32*>(smem + 2 * SM::BUF);  // [WARPS][RADIX+1]
    u32* s_dstart = s_whist + WARPS * (RADIX + 1);              // tile-local digit starts
    u32* s_run = s_dstart + RADIX;                              // next global position per digit
    u64* s_bar = reinterpret_cast<u64*>(s_run + RADIX);         // [2]
    u32* s_info = reinterpret_cast<u32*>(s_bar + 2);            // range, koff[2], voff[2], epoch, abort

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 nranges = __ldg(range_off + nseg);
    const u32 lt = lanemask_lt();
    // TMA loads of items [a, e) into buffer b (one thread)
    auto issue = [&](int b, u32 a, u32 e) {
        const u32 ka = a / KAL * KAL, kb = (e + KAL - 1) / KAL * KAL;
        const u32 kbytes = (kb - ka) * (u32)sizeof(K);
        u32 vbytes = 0, va = 0;
        if (!IOTA) {
            va = a / VAL * VAL;
            const u32 vb = (e + VAL - 1) / VAL * VAL;
            vbytes = (vb - va) * (u32)sizeof(V);
        }
        s_info[1 + b] = a - ka;
        s_info[3 + b] = a - va;
        unsigned char* buf = smem + b * SM::BUF;
        mbar_arrive_expect_tx(&s_bar[b], kbytes + vbytes);
        bulk_g2s(buf, kin + ka, kbytes, &s_bar[b]);
        if (!IOTA) bulk_g2s(buf + SM::KBYTES, vin + va, vbytes, &s_bar[b]);
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        s_info[5] = ctl->epoch_base + (u32)launch_idx;
        s_info[6] = 0;
    }
    __syncthreads();
    const u32 epoch = s_info[5];
    u32 phase[2] = {0u, 0u};
    bool pending[2] = {false, false};  // thread 0's view of copies in flight
    int b = 0;
    for (;;) {
        if (tid == 0) s_info[0] = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        for (int x = tid; x < WARPS * (RADIX + 1); x += THREADS) s_whist[x] = 0;
        __syncthreads();
        const u32 r = s_info[0];
        if (r >= nranges) break;
        const TileLoc L = locate_range(r, seg_off, range_off, nseg, range_items);
        // a segment whose keys have fewer digits is already in place (the
        // barrier keeps thread 0's next claim from overwriting s_info[0]
        // before every thread has read it)
        if (seg_bits && (u32)pass * RADIX_BITS >= __ldg(seg_bits + L.seg)) {
            __syncthreads();
            continue;
        }
        const u32 ntile = (L.end - L.start + TILE - 1) / TILE;
        if (tid == 0) {  // the first tile's load overlaps the range histogram
            fence_proxy_async_smem();
            issue(b, L.start, min(L.start + (u32)TILE, L.end));
            pending[b] = true;
        }
        // 1. digit counts of the range (per-warp histograms, then summed)
        if (range_base) {
            for (int d = tid; d < RADIX; d += THREADS) s_run[d] = __ldg(range_base + (u64)r * RADIX + d);
        } else {
            u32* wh = s_whist + warp * (RADIX + 1);
            // evenly spread digits (see k_radix_hist): plain shared atomics
            const bool plain = uniform && seg_bits && (int)__ldg(seg_bits + L.seg) - shift >= 5;
            for (u32 base = L.start; base < L.end; base += (u32)THREADS * 8u) {
                K kk[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const u32 x = base + (u32)j * THREADS + (u32)tid;
                    kk[j] = x < L.end ? kin[x] : K(0);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const u32 d = digit_of(kk[j], keymask, shift);
                    const bool valid = base + (u32)j * THREADS + (u32)tid < L.end;
                    if (plain) {
                        if (valid) atomicAdd(&wh[d], 1u);
                    } else {
                        warp_hist_add(wh, d, valid, (u32)lane);
                    }
                }
            }
            __syncthreads();
            for (int d = tid; d < RADIX; d += THREADS) {
                u32 c = 0;
                for (int w = 0; w < WARPS; ++w) c += s_whist[w * (RADIX + 1) + d];
                s_dstart[d] = c;
            }
            __syncthreads();
        // 2. publish the range's counts and look back over the earlier ranges
        {
            const u32 first_range = r - (L.start - L.seg_begin) / range_items;
            for (int d = tid; d < RADIX; d += THREADS) {
                const u32 cnt = s_dstart[d];
                u64* st = status + (u64)r * RADIX + d;
                u32 excl = 0;
                if (L.first) {
                    st_store(st, st_pack(epoch, ST_PREFIX, cnt));
                } else {
                    st_store(st, st_pack(epoch, ST_AGG, cnt));
                    excl = lookback_u32(status, RADIX, d, r, first_range, epoch, ctl, 1u);
                    st_store(st, st_pack(epoch, ST_PREFIX, excl + cnt));
                }
                s_run[d] = __ldg(digit_off + ((u64)L.seg * npass + pass) * RADIX + d) + excl;
            }
        }
        }
        // 3. the tiles of the range, in order
        for (u32 j = 0; j < ntile; ++j) {
            const u32 a = L.start + j * (u32)TILE;
            const u32 n = min(a + (u32)TILE, L.end) - a;
            for (int x = tid; x < WARPS * (RADIX + 1); x += THREADS) s_whist[x] = 0;
            fence_proxy_async_smem();
            __syncthreads();  // counters cleared; the other buffer is free
            if (tid == 0 && j + 1 < ntile) {
                const u32 a2 = a + (u32)TILE;
                issue(b ^ 1, a2, min(a2 + (u32)TILE, L.end));
                pending[b ^ 1] = true;
            }
            // every thread observes the completion of the copy it reads
            if (mbar_wait_bounded(&s_bar[b], phase[b], ctl, 5u)) {
                phase[b] ^= 1u;
                if (tid == 0) pending[b] = false;
            } else {
                s_info[6] = 1u;
            }
            __syncthreads();
            if (s_info[6]) break;
            const K* bk = reinterpret_cast<const K*>(smem + b * SM::BUF) + s_info[1 + b];
            const V* bv = reinterpret_cast<const V*>(smem + b * SM::BUF + SM::KBYTES) + s_info[3 + b];
            // warp w ranks items [w*32*ITEMS, ...); item i of lane l at i*32 + l
            K key[ITEMS];
            u32 pos[ITEMS];
            const u32 wbase = (u32)warp * 32u * ITEMS;
            u32* wh = s_whist + warp * (RADIX + 1);
            if (!STABLE) {
                // any order inside a digit will do: one atomic per item
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const u32 x = wbase + (u32)i * 32u + (u32)lane;
                    key[i] = x < n ? bk[x] : K(0);
                    pos[i] = x < n ? atomicAdd(&wh[digit_of(key[i], keymask, shift)], 1u) : 0u;
                }
            } else {
            // digit matches of all items first (independent ballots pipeline) ...
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const u32 x = wbase + (u32)i * 32u + (u32)lane;
                const bool valid = x < n;
                key[i] = valid ? bk[x] : K(0);
                pos[i] = match_digit8(digit_of(key[i], keymask, shift), __ballot_sync(0xffffffffu, valid));
            }
            // ... then, item by item, the group's leader advances the warp's
            // count of the digit (shared-memory atomics of one warp are
            // performed in program order) and shares the old count
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const u32 x = wbase + (u32)i * 32u + (u32)lane;
                const u32 peers = pos[i];
                const bool valid = x < n;
                const int leader = valid ? __ffs(peers) - 1 : lane;
                u32 old = 0;
                if (valid && lane == leader) old = atomicAdd(&wh[digit_of(key[i], keymask, shift)], (u32)__popc(peers));
                pos[i] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
            }
            }
            __syncthreads();
            for (int d = tid; d < RADIX; d += THREADS) {  // exclusive over warps; tile count
                u32 sum = 0;
                for (int w = 0; w < WARPS; ++w) {
                    const u32 c = s_whist[w * (RADIX + 1) + d];
                    s_whist[w * (RADIX + 1) + d] = sum;
                    sum += c;
                }
                s_dstart[d] = sum;
            }
            __syncthreads();
            if (warp == 0) {  // exclusive scan of the tile counts over the digits (in place)
                constexpr int PER = RADIX / 32;
                u32 v[PER], sacc = 0;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    v[q] = s_dstart[lane * PER + q];
                    sacc += v[q];
                }
                u32 inc = sacc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 nn = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += nn;
                }
                u32 ex = inc - sacc;
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    s_dstart[lane * PER + q] = ex;
                    ex += v[q];
                }
            }
            __syncthreads();
            // per (warp, digit): the warp's first local position; per digit:
            // the global position of local index 0
            // (then s_dstart is reused for the latter and the running
            // positions advance by the tile's counts)
            static_assert(THREADS == RADIX, "one thread per digit");
            {
                const int d = tid;
                const u32 ds = s_dstart[d];
                const u32 dn = d + 1 < RADIX ? s_dstart[d + 1] : n;
                for (int w = 0; w < WARPS; ++w) s_whist[w * (RADIX + 1) + d] += ds;
                const u32 gdst = s_run[d] - ds;
                s_run[d] += dn - ds;
                __syncthreads();
                s_dstart[d] = gdst;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const u32 x = wbase + (u32)i * 32u + (u32)lane;
                if (x < n) pos[i] += wh[digit_of(key[i], keymask, shift)];
            }
            K* sk = reinterpret_cast<K*>(smem + b * SM::BUF);
            V* sv = reinterpret_cast<V*>(smem + b * SM::BUF + SM::KBYTES);
            __syncthreads();  // all keys are in registers: stage over the key buffer
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const u32 x = wbase + (u32)i * 32u + (u32)lane;
                if (x < n && DOMAGG_GUARD(pos[i] < n, SITE_SORT_LOCAL)) sk[pos[i]] = key[i];
            }
            V val[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const u32 x = wbase + (u32)i * 32u + (u32)lane;
                val[i] = IOTA ? (V)(a + x) : (x < n ? bv[x] : V(0));
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const u32 x = wbase + (u32)i * 32u + (u32)lane;
                if (x < n && DOMAGG_GUARD(pos[i] < n, SITE_SORT_LOCAL)) sv[pos[i]] = val[i];
            }
            __syncthreads();
            const u32 seg_len = L.seg_end - L.seg_begin;
            for (u32 x = tid; x < n; x += THREADS) {
                const K k = sk[x];
                const u32 dst = s_dstart[digit_of(k, keymask, shift)] + x;  // (global position of index 0)
                if (domagg_check(dst - L.seg_begin < seg_len, SITE_SORT_SCATTER)) {  // only fails after a timed-out wait
                    kout[dst] = k;
                    vout[dst] = sv[x];
                }
            }
            b ^= 1;
        }
        __syncthreads();
        if (s_info[6]) break;
    }
    // a copy may still be in flight if a wait ran out: wait for it (bounded)
    if (tid == 0) {
        for (int bb = 0; bb < 2; ++bb)
            if (pending[bb]) mbar_wait_bounded(&s_bar[bb], phase[bb], ctl, 6u);
    }
}

}  // namespace domagg
