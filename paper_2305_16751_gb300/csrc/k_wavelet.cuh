// k_wavelet.cuh -- the level-wise formulation of the m <= 2 dominance
// aggregation: the P0/P1 decomposition of the first coordinate's rank
// (Sec. 5) evaluated level by level on the points themselves, without
// materialising the n log n flat-map records.
//
// Write r for a point's dense rank in the first coordinate (b bits) and
// order the points by the last coordinate, queries first on ties (Sec. 5).
// d < q in the first coordinate exactly when, at the highest bit where the
// ranks differ, d has a 0 and q a 1 (Lemma 1); the records of level l of the
// flat map group the points by the prefix r >> (l + 1).  Processing the
// levels from the top, keep the points ordered by (r >> (l + 1), last
// coordinate): then every prefix group is a contiguous run in the order of
// the last coordinate, and level l is one segmented scan over the array
// (data with bit l = 0 contribute, queries with bit l = 1 read the running
// value), after which a stable partition of the whole array by bit l yields
// the order of level l - 1 (groups stay contiguous: the array becomes
// ordered by bit l, then by the previous order).
//
// One pass handles D = 1 or 2 levels: the digit c = (r >> s) & (2^D - 1)
// below the group prefix r >> (s + D).  Within a group, a query with digit
// c receives F over the preceding data with digit < c, split as in a binary
// trie over the digit: the 2^D - 1 trie nodes are scan channels; a data
// point feeds the nodes where its path turns left, a query reads those where
// its path turns right.  The pass is a onesweep radix pass on the digit (the
// global stable partition: digit bucket bases from a histogram of all
// passes, counts of earlier tiles by decoupled look-back) fused with the
// segmented scan of the channels (carried across tiles by the same
// look-back).  The last pass writes each query's value to its output.
#pragma once
#include "dev_common.cuh"
#include "k_records.cuh"

namespace domagg {

constexpr int WV_THREADS = 256;
#ifndef DOMAGG_WV_ITEMS
#define DOMAGG_WV_ITEMS 8  // points per thread of a tile (the tile is staged in static shared memory: <= 10)
#endif
constexpr int WV_ITEMS = DOMAGG_WV_ITEMS;
constexpr u32 WV_TILE = WV_THREADS * WV_ITEMS;
constexpr int WV_MAX_PASSES = 32;
constexpr u32 WV_QUERY = 0x80000000u;  // in WElem::key: the point is a query
#ifndef DOMAGG_WV_MIN_BLOCKS
#define DOMAGG_WV_MIN_BLOCKS 3  // resident blocks per SM the register budget is cut for
#endif
constexpr int WV_MIN_BLOCKS = DOMAGG_WV_MIN_BLOCKS;

// One point of the level-wise arrays (16 bytes, moved whole by every pass).
struct alignas(16) WElem {
    u32 key;  // dense rank in the first coordinate, WV_QUERY for a query
    u32 aux;  // a query's index within the instance
    u64 val;  // data: its weight as Op::Acc; query: F over what it has received
};

// Pass geometry: pass p handles the bits [shift[p], shift[p] + width[p]) of
// the rank, from the top bit down.
struct WvPasses {
    int n;
    u32 shift[WV_MAX_PASSES];
    u32 width[WV_MAX_PASSES];
};

template <typename Acc>
__device__ __forceinline__ u64 wv_bits(Acc a) {
    u64 b = 0;
    memcpy(&b, &a, sizeof(Acc));
    return b;
}
template <typename Acc>
__device__ __forceinline__ Acc wv_acc(u64 b) {
    Acc a;
    memcpy(&a, &b, sizeof(Acc));
    return a;
}

// A data point's weight as the scan's accumulator type.
template <class Op>
__device__ __forceinline__ typename Op::Acc wv_weight(const void* dw, u32 i) {
    if constexpr (std::is_same<Op, OpCount>::value) {
        return Op::from_pay(0u);
    } else if constexpr (Op::GATHER) {
        return Op::from_w((typename Op::W) reinterpret_cast<const long long*>(dw)[i]);
    } else {
        return Op::from_pay(reinterpret_cast<const u32*>(dw)[i]);
    }
}

// a[c] of a small register array without dynamic indexing
template <int N>
__device__ __forceinline__ u32 wv_sel(const u32 (&a)[N], u32 c) {
    u32 v = a[0];
#pragma unroll
    for (int k = 1; k < N; ++k)
        if (c == (u32)k) v = a[k];
    return v;
}

// Look-back record of one tile: the tile's digit counts and, per channel,
// F over the data after the tile's last group start (ST_AGG); or the
// inclusive counts and the channels' carry at the tile's end (ST_PREFIX).
template <typename Acc>
struct alignas(16) WvStatus {
    u32 flag;      // (epoch << 2) | ST_AGG / ST_PREFIX
    u32 has_head;  // a group starts inside the tile (with ST_AGG)
    u32 cnt_agg[4];
    u32 cnt_incl[4];
    u32 pad[2];
    Acc sum_agg[3];
    Acc sum_incl[3];
};

__device__ __forceinline__ u32 wv_pidx(u32 x) { return x + (x >> 3); }  // 16-byte slots, padded per 8

// Digit histogram of every pass (order-independent): hist[p * 4 + c] counts
// the points whose rank has digit c at pass p.  For m = 1 the rank is the
// role bit (data 0, query 1): every datum precedes every query in it.  A
// thread counts its 16 points in 8-bit fields (one 32-bit word per pass,
// the pass geometry held in registers), then warp sums go to shared memory.
constexpr int WV_HIST_PASSES = 16;  // passes of width 2 cover ranks of up to 32 bits
template <int M>
__global__ __launch_bounds__(256) void k_wavelet_hist(const u32* __restrict__ r0, const Inst* __restrict__ inst,
                                                     u32 n, WvPasses ps, u32* __restrict__ hist) {
    constexpr int ITEMS = 16;
    __shared__ u32 s_h[WV_HIST_PASSES * 4];
    for (int i = threadIdx.x; i < WV_HIST_PASSES * 4; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const int np = ps.n < WV_HIST_PASSES ? ps.n : WV_HIST_PASSES;
    u32 sh[WV_HIST_PASSES], mk[WV_HIST_PASSES], c[WV_HIST_PASSES];
#pragma unroll
    for (int p = 0; p < WV_HIST_PASSES; ++p) {
        sh[p] = p < np ? ps.shift[p] : 0u;
        mk[p] = p < np ? (1u << ps.width[p]) - 1u : 0u;
        c[p] = 0;
    }
    const u32 nQ = inst[0].nQ;
    const u32 j0 = blockIdx.x * (256u * ITEMS);
#pragma unroll 4
    for (int i = 0; i < ITEMS; ++i) {
        const u32 j = j0 + (u32)i * 256u + threadIdx.x;
        if (j < n) {
            const u32 r = M == 1 ? (j < nQ ? 1u : 0u) : r0[j];
#pragma unroll
            for (int p = 0; p < WV_HIST_PASSES; ++p) c[p] += 1u << (8u * ((r >> sh[p]) & mk[p]));
        }
    }
#pragma unroll
    for (int p = 0; p < WV_HIST_PASSES; ++p) {
        if (p < np) {
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const u32 v = __reduce_add_sync(0xffffffffu, (c[p] >> (8 * d)) & 0xffu);
                if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_h[p * 4 + d], v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np * 4; i += blockDim.x)
        if (s_h[i]) atomicAdd(hist + i, s_h[i]);
}

// Branch-free trie updates (D <= 2 levels per pass; the channels of trie
// level t are [2^(D-1-t) - 1, 2^(D-t) - 1), selected by the digit's bits
// above t).  feed: F the value v into the channel of every level where the
// digit's bit is 0 (pass v = e for a query: F(x, e) = x exactly).  read: F
// into acc the channel of every level where the digit's bit is 1.
template <class Op, int D>
__device__ __forceinline__ void wv_feed(typename Op::Acc (&s)[(1 << D) - 1], u32 c, typename Op::Acc v) {
#pragma unroll
    for (int t = D - 1; t >= 0; --t) {
        const int lo = (1 << (D - 1 - t)) - 1, cnt = 1 << (D - 1 - t);
        const u32 sel = c >> (t + 1);  // which channel of the level
        typename Op::Acc cur = s[lo];
#pragma unroll
        for (int k = 1; k < cnt; ++k)
            if (sel == (u32)k) cur = s[lo + k];
        const typename Op::Acc nv = Op::F(cur, ((c >> t) & 1u) ? Op::e() : v);
#pragma unroll
        for (int k = 0; k < cnt; ++k)
            if (sel == (u32)k) s[lo + k] = nv;
    }
}
template <class Op, int D>
__device__ __forceinline__ typename Op::Acc wv_read(const typename Op::Acc (&s)[(1 << D) - 1], u32 c,
                                                    typename Op::Acc acc) {
#pragma unroll
    for (int t = D - 1; t >= 0; --t) {
        const int lo = (1 << (D - 1 - t)) - 1, cnt = 1 << (D - 1 - t);
        const u32 sel = c >> (t + 1);
        typename Op::Acc cur = s[lo];
#pragma unroll
        for (int k = 1; k < cnt; ++k)
            if (sel == (u32)k) cur = s[lo + k];
        acc = Op::F(acc, ((c >> t) & 1u) ? cur : Op::e());
    }
    return acc;
}

// One pass over D levels.  first: the elements are built from the order of
// the last coordinate (perm), the ranks and the weights; otherwise read from
// `in`.  last: queries write their outputs; otherwise the tile is written,
// partitioned by digit, to `out_el`.
//
// Within the tile every value is first computed without the carry from
// earlier tiles (the channels of the group that continues into the tile):
// warp 0 publishes the tile's aggregate and looks back while the other
// warps compute, so a tile's inclusive prefix follows its aggregate by one
// look-back only (short chains for the tiles after it); the carry is added
// to the queries of that first group when the tile is written out.
template <class Op, int D, int M>
__global__ __launch_bounds__(WV_THREADS, WV_MIN_BLOCKS) void k_wavelet_pass(
    const WElem* __restrict__ in, WElem* __restrict__ out_el, const u32* __restrict__ perm,
    const u32* __restrict__ r0, const Inst* __restrict__ inst, u32 n, u32 shift, int first, int last,
    const u32* __restrict__ hist, WvStatus<typename Op::Acc>* status, Ctl* ctl, int launch_idx) {
    typedef typename Op::Acc Acc;
    constexpr int WARPS = WV_THREADS / 32, NDIG = 1 << D, NCH = NDIG - 1;
    constexpr u32 DMASK = (u32)NDIG - 1u;
    __shared__ uint4 s_el[WV_TILE + WV_TILE / 8];
    __shared__ Acc s_wsum[WARPS][NCH];
    __shared__ u32 s_whead[WARPS];
    __shared__ unsigned long long s_wcnt[WARPS];
    __shared__ Acc s_carry[NCH];
    __shared__ u32 s_prev[NDIG], s_dbase[NDIG];
    __shared__ u32 s_info[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_info[0] = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        s_info[1] = ctl->epoch_base + (u32)launch_idx;
        u32 a = 0;
        for (int c = 0; c < NDIG; ++c) {
            s_dbase[c] = a;
            a += hist[c];
        }
    }
    __syncthreads();
    const u32 t = s_info[0], epoch = s_info[1];
    const u32 base = t * WV_TILE;
    if (base >= n) return;
    const u32 cnt = min(WV_TILE, n - base);
    const u32 gshift = shift + (u32)D;  // the group is the rank above the digit

    // ---- load the tile (coalesced) into shared memory
    if (first) {
        const Inst& I = inst[0];
        const u32 nQ = I.nQ;
        const bool rev = (I.flags >> (M - 1)) & 1u;  // non-strict last coordinate: its order read backwards
        for (int i = 0; i < WV_ITEMS; ++i) {
            const u32 x = (u32)i * WV_THREADS + threadIdx.x;
            if (x < cnt) {
                const u32 pos = base + x;
                u32 j = perm[rev ? n - 1u - pos : pos];
                if (j >= n) j = 0;  // never taken for a valid permutation
                const bool q = j < nQ;
                WElem e;
                e.key = (M == 1 ? (q ? 1u : 0u) : r0[j]) | (q ? WV_QUERY : 0u);
                e.aux = q ? j : 0u;
                e.val = wv_bits<Acc>(q ? Op::e() : wv_weight<Op>(I.dw, j - nQ));
                s_el[wv_pidx(x)] = *reinterpret_cast<uint4*>(&e);
            }
        }
    } else {
        const uint4* src = reinterpret_cast<const uint4*>(in) + base;
        for (int i = 0; i < WV_ITEMS; ++i) {
            const u32 x = (u32)i * WV_THREADS + threadIdx.x;
            if (x < cnt) s_el[wv_pidx(x)] = __ldcs(src + x);
        }
    }
    __syncthreads();

    // ---- my items (blocked), and the group of the element before them
    const u32 lx0 = threadIdx.x * WV_ITEMS;
    uint4 it[WV_ITEMS];
#pragma unroll
    for (int i = 0; i < WV_ITEMS; ++i) it[i] = lx0 + i < cnt ? s_el[wv_pidx(lx0 + i)] : make_uint4(0, 0, 0, 0);
    bool has_prev = base + lx0 > 0;
    u32 prevg = 0;
    if (has_prev && lx0 < cnt && !first)
        prevg = ((lx0 == 0 ? in[base - 1].key : s_el[wv_pidx(lx0 - 1)].x) & ~WV_QUERY) >> gshift;
    // (first pass: every rank is below 2^(shift + D), a single group)
    if (threadIdx.x == 0) {
        // the tile's first group continues from the previous tile unless it starts here
        const u32 g0 = (it[0].x & ~WV_QUERY) >> gshift;
        s_info[2] = (has_prev && g0 == prevg) ? (g0 | 0x80000000u) : 0u;  // bit 31: carry applies
    }

    // thread aggregate: (group start seen, channels after the last start), digit counts
    bool head_any = false;
    u32 headmask = 0;
    Acc tsum[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) tsum[ch] = Op::e();
    unsigned long long tcnt = 0;  // 16-bit count per digit
#pragma unroll
    for (int i = 0; i < WV_ITEMS; ++i) {
        if (lx0 + i < cnt) {
            const u32 kn = it[i].x & ~WV_QUERY;
            const u32 g = kn >> gshift, c = (kn >> shift) & DMASK;
            const bool head = !has_prev || g != prevg;
            has_prev = true;
            prevg = g;
            if (head) {
                head_any = true;
                headmask |= 1u << i;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) tsum[ch] = Op::e();
            }
            tcnt += 1ull << (16 * c);
            const bool q = (it[i].x & WV_QUERY) != 0u;
            wv_feed<Op, D>(tsum, c, q ? Op::e() : wv_acc<Acc>(((u64)it[i].w << 32) | it[i].z));
        }
    }

    // ---- block-wide exclusive scan of the thread aggregates
    bool ihead = head_any;
    Acc isum[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) isum[ch] = tsum[ch];
    unsigned long long icnt = tcnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int nh = __shfl_up_sync(0xffffffffu, (int)ihead, o);
        const unsigned long long nc = __shfl_up_sync(0xffffffffu, icnt, o);
        Acc ns[NCH];
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) ns[ch] = wv_acc<Acc>(__shfl_up_sync(0xffffffffu, wv_bits(isum[ch]), o));
        if (lane >= o) {
            if (!ihead) {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) isum[ch] = Op::F(ns[ch], isum[ch]);
            }
            ihead = ihead || nh;
            icnt += nc;
        }
    }
    if (lane == 31) {
        s_whead[warp] = ihead ? 1u : 0u;
        s_wcnt[warp] = icnt;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) s_wsum[warp][ch] = isum[ch];
    }
    // exclusive within the warp: the inclusive value of lane - 1
    bool lhead = __shfl_up_sync(0xffffffffu, (int)ihead, 1) != 0;
    unsigned long long lcnt = __shfl_up_sync(0xffffffffu, icnt, 1);
    Acc lsum[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) lsum[ch] = wv_acc<Acc>(__shfl_up_sync(0xffffffffu, wv_bits(isum[ch]), 1));
    if (lane == 0) {
        lhead = false;
        lcnt = 0;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) lsum[ch] = Op::e();
    }
    __syncthreads();
    // earlier warps, and the tile's digit counts
    unsigned long long wcnt = 0, tc = 0;
    Acc run[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) run[ch] = Op::e();
    for (int w = 0; w < WARPS; ++w) {
        const unsigned long long cw = s_wcnt[w];
        tc += cw;
        if (w < warp) {
            wcnt += cw;
            if (s_whead[w]) {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) run[ch] = s_wsum[w][ch];
            } else {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) run[ch] = Op::F(run[ch], s_wsum[w][ch]);
            }
        }
    }
    // the running channels at my first item, without the carry of earlier tiles
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) run[ch] = lhead ? lsum[ch] : Op::F(run[ch], lsum[ch]);
    unsigned long long xcnt = wcnt + lcnt;
    u32 tstart[NDIG];
    {
        u32 a = 0;
#pragma unroll
        for (int c = 0; c < NDIG; ++c) {
            tstart[c] = a;
            a += (u32)(tc >> (16 * c)) & 0xffffu;
        }
    }

    // ---- tile aggregate, published before anything waits (warp 0, lane 0)
    WvStatus<Acc>* my = status + t;
    bool thead = false;
    Acc ts[NCH];
    if (warp == 0) {
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) ts[ch] = Op::e();
        for (int w = 0; w < WARPS; ++w) {
            if (s_whead[w]) {
                thead = true;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) ts[ch] = s_wsum[w][ch];
            } else {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) ts[ch] = Op::F(ts[ch], s_wsum[w][ch]);
            }
        }
        if (lane == 0 && t > 0) {
#pragma unroll
            for (int c = 0; c < NDIG; ++c) my->cnt_agg[c] = (u32)(tc >> (16 * c)) & 0xffffu;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) my->sum_agg[ch] = ts[ch];
            my->has_head = thead ? 1u : 0u;
            __threadfence();
            st_store_release(&my->flag, ((epoch & EPOCH_MASK) << 2) | ST_AGG);
        }
    }

    // ---- look-back (warp 0): counts of earlier tiles, carry of the first group
    if (warp == 0) {
        u32 ecnt[NDIG];
        Acc esum[NCH];
#pragma unroll
        for (int c = 0; c < NDIG; ++c) ecnt[c] = 0;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) esum[ch] = Op::e();
        if (t > 0) {
            bool sums_open = true;
            u32 u = t;  // tiles [u, t) are combined
            u32 spins = 0;
            while (u > 0) {
                const bool exists = (u32)lane < u;
                bool ready = false, term = false, hd = false;
                u32 c4[NDIG];
                Acc s3[NCH];
#pragma unroll
                for (int c = 0; c < NDIG; ++c) c4[c] = 0;
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) s3[ch] = Op::e();
                if (exists) {
                    const WvStatus<Acc>* ps = status + (u - 1u - (u32)lane);
                    const u32 f = st_load_acquire(&ps->flag);
                    ready = (f >> 2) == (epoch & EPOCH_MASK) && (f & 3u);
                    if (ready) {
                        if ((f & 3u) == ST_PREFIX) {
                            term = hd = true;
#pragma unroll
                            for (int c = 0; c < NDIG; ++c)
                                c4[c] = *reinterpret_cast<const volatile u32*>(&ps->cnt_incl[c]);
#pragma unroll
                            for (int ch = 0; ch < NCH; ++ch) s3[ch] = volatile_read(&ps->sum_incl[ch]);
                        } else {
                            hd = *reinterpret_cast<const volatile u32*>(&ps->has_head) != 0u;
#pragma unroll
                            for (int c = 0; c < NDIG; ++c)
                                c4[c] = *reinterpret_cast<const volatile u32*>(&ps->cnt_agg[c]);
#pragma unroll
                            for (int ch = 0; ch < NCH; ++ch) s3[ch] = volatile_read(&ps->sum_agg[ch]);
                        }
                    }
                }
                const u32 nr = __ballot_sync(0xffffffffu, !ready);
                const u32 tm = __ballot_sync(0xffffffffu, term);
                const int k_nr = nr ? __ffs(nr) - 1 : 32;
                const int k_tm = tm ? __ffs(tm) - 1 : 32;
                const bool finish = k_tm < k_nr;
                const int take = finish ? k_tm + 1 : k_nr;  // lanes [0, take) are combined
                if (take > 0) {
#pragma unroll
                    for (int c = 0; c < NDIG; ++c) ecnt[c] += __reduce_add_sync(0xffffffffu, lane < take ? c4[c] : 0u);
                    if (sums_open) {
                        // the channels stop at the nearest tile holding a group start
                        const u32 hm = __ballot_sync(0xffffffffu, hd && lane < take);
                        const int k_hd = hm ? __ffs(hm) - 1 : 32;
                        const int take_s = k_hd < take ? k_hd + 1 : take;
#pragma unroll
                        for (int ch = 0; ch < NCH; ++ch) {
                            Acc r = lane < take_s ? s3[ch] : Op::e();
#pragma unroll
                            for (int o = 16; o >= 1; o >>= 1) r = Op::F(r, shfl_xor_acc(r, o));
                            esum[ch] = Op::F(r, esum[ch]);
                        }
                        if (k_hd < take) sums_open = false;
                    }
                    u -= (u32)take;
                }
                if (finish) break;
                if (take == 0) {
                    if (++spins > SPIN_LIMIT || ((spins & 255u) == 0 && timed_out(ctl))) {
                        if (lane == 0) {
                            atomicOr(&ctl->error, ERR_TIMEOUT);
                            ctl->timeout_where = 9u;
                        }
                        break;
                    }
                    if (spins > 64) __nanosleep(256);
                }
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < NDIG; ++c) my->cnt_incl[c] = ecnt[c] + ((u32)(tc >> (16 * c)) & 0xffffu);
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) my->sum_incl[ch] = thead ? ts[ch] : Op::F(esum[ch], ts[ch]);
            __threadfence();
            st_store_release(&my->flag, ((epoch & EPOCH_MASK) << 2) | ST_PREFIX);
#pragma unroll
            for (int c = 0; c < NDIG; ++c) s_prev[c] = ecnt[c];
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) s_carry[ch] = esum[ch];
        }
    }
    // ---- second walk: queries receive, data feed; staged by digit
#pragma unroll
    for (int i = 0; i < WV_ITEMS; ++i) {
        if (lx0 + i < cnt) {
            const u32 kn = it[i].x & ~WV_QUERY;
            const u32 c = (kn >> shift) & DMASK;
            if (headmask & (1u << i)) {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) run[ch] = Op::e();
            }
            const bool q = (it[i].x & WV_QUERY) != 0u;
            const Acc v = wv_acc<Acc>(((u64)it[i].w << 32) | it[i].z);
            if (q) {
                const u64 b = wv_bits(wv_read<Op, D>(run, c, v));
                it[i].z = (u32)b;
                it[i].w = (u32)(b >> 32);
            }
            wv_feed<Op, D>(run, c, q ? Op::e() : v);
            const u32 slot = wv_sel<NDIG>(tstart, c) + ((u32)(xcnt >> (16 * c)) & 0xffffu);
            xcnt += 1ull << (16 * c);
            s_el[wv_pidx(slot)] = it[i];
        }
    }

    __syncthreads();

    // ---- write the tile out, partitioned by digit (runs of one digit are
    // contiguous); the queries of the continuing first group receive the carry
    const u32 cont = s_info[2];
    Acc carry[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) carry[ch] = s_carry[ch];
    uint4* dst = reinterpret_cast<uint4*>(out_el);
    typename Op::Out* outp = reinterpret_cast<typename Op::Out*>(inst[0].out);
    for (int i = 0; i < WV_ITEMS; ++i) {
        const u32 x = (u32)i * WV_THREADS + threadIdx.x;
        if (x < cnt) {
            uint4 e = s_el[wv_pidx(x)];
            const u32 kn = e.x & ~WV_QUERY;
            const u32 c = (kn >> shift) & DMASK;
            const bool q = (e.x & WV_QUERY) != 0u;
            if (q && (cont >> 31) && (kn >> gshift) == (cont & 0x7fffffffu)) {
                const u64 b = wv_bits(wv_read<Op, D>(carry, c, wv_acc<Acc>(((u64)e.w << 32) | e.z)));
                e.z = (u32)b;
                e.w = (u32)(b >> 32);
            }
            if (last) {
                if (q && DOMAGG_GUARD(e.y < inst[0].nQ, SITE_WAVELET_OUT))
                    outp[e.y] = Op::to_out(wv_acc<Acc>(((u64)e.w << 32) | e.z));
            } else {
                const u32 at = s_dbase[c] + s_prev[c] + (x - wv_sel<NDIG>(tstart, c));
                if (DOMAGG_GUARD(at < n, SITE_WAVELET_EL)) __stcs(dst + at, e);
            }
        }
    }
}

}  // namespace domagg
