// k_group3.cuh -- the deep first-rank levels of m = 3 in shared memory.
//
// For m = 3 a record of first-rank level lv is keyed by the node r0 >> (lv+1)
// of the first rank refined by a node r1 >> (j+1) of the second rank, one
// record per second-rank level j at which the point emits too (Sec. 5 with
// two bitstring coordinates).  As for m = 2 (k_group.cuh), the points, in
// the order of the last coordinate, are sorted stably by their group
// g = r0 >> gS, and one CTA takes a group of at most G3_CAP points: every
// record of a level lv < gS lies in one group, and the CTA forms, sorts and
// scans them in shared memory.
//
// Inside a node of level lv (a "block": the points sharing r0 >> (lv+1)),
// the records are the points level lv emits (data with rank bit lv = 0, the
// P0 set; queries with bit lv = 1, the P1 set) crossed with their
// second-rank nodes, and a query's partial results are exactly those of the
// m = 2 problem on the block's emitting points with the second rank as its
// ranked coordinate (every datum of P0 precedes every query of P1 in the
// first coordinate, Lemma 1).  So per level lv, from gS-1 down to 0:
//   1. the group's points are in the order of level lv, (r0 >> (lv+1), last
//      coordinate) -- the outer order; the group starts in the order of the
//      last coordinate, and a stable split by bit lv inside every node gives
//      the order of level lv-1 (as k_group does);
//   2. the emitting points are compacted in the outer order into the inner
//      array (blocks stay contiguous and keep the order of the last
//      coordinate), and a bitmap marks where each block starts;
//   3. the second rank's levels are walked over the inner array as k_group
//      walks the first rank's: per level j a segmented scan of F over the
//      nodes (block, r1 >> (j+1)) -- a node starts where the prefix changes
//      or a block starts -- then a stable split by bit j.
// Only comparisons of second ranks inside the group matter, so the walk
// uses each point's dense rank among the group's second ranks (below 2^14:
// fewer levels than the global rank, and 32-bit handles).  From the first
// level whose blocks all hold at most G3_PAIR_MAX points down, step 3 is
// replaced by its definition (g3_pairwise): each emitting query takes F over
// the block's earlier emitting data of smaller local second rank.  A query
// keeps F over all its partial results of these levels and writes it, as
// one partial, at its position in the order of the last coordinate; the
// levels lv >= gS go through the records in HBM, and the per-query
// reduction joins the parts.  A group with more points than G3_CAP (heavy
// ties) is not taken here: its queries' part is the unit and its points'
// levels below gS go through HBM too (k_group_plan flags it).
#pragma once
#include "k_group.cuh"

namespace domagg {

constexpr int G3_THREADS = 1024;
constexpr int G3_ITEMS = 10;                    // points per thread, at most
constexpr u32 G3_CAP = G3_THREADS * G3_ITEMS;   // points per group in shared memory
constexpr u32 G3_LBITS = 14;                    // bits of a local index or local second rank
constexpr u32 G3_LMASK = (1u << G3_LBITS) - 1u;
constexpr u32 G3_BMAP_WORDS = G3_CAP / 32 + 2;  // block heads by position (and one word beyond)
static_assert(G3_CAP <= (1u << G3_LBITS), "local indices and ranks fit 14 bits");

// Shared-memory layout: values by local index, outer and inner handles
// (padded), local second ranks by index, zero counts by node-head position,
// the block-head bitmap.
template <typename Acc>
struct G3Smem {
    static constexpr size_t VAL = 0;
    static constexpr size_t OXH = VAL + (size_t)G3_CAP * sizeof(Acc);
    static constexpr size_t IXH = OXH + (size_t)Padded<G3_CAP>::value * 4;
    static constexpr size_t R1L = IXH + (size_t)Padded<G3_CAP>::value * 4;
    static constexpr size_t HZ = R1L + (size_t)G3_CAP * 2;
    static constexpr size_t BMAP = HZ + (size_t)G3_CAP * 2;
    static constexpr size_t TOTAL = BMAP + (size_t)G3_BMAP_WORDS * 4;
};

// Exclusive block sum of one u32 per thread; *total gets the sum of all.
// Two barriers; s_tmp holds 33 words.
__device__ __forceinline__ u32 g3_exscan_u32(u32 v, u32* s_tmp, u32* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const u32 w = lane < (int)(blockDim.x >> 5) ? s_tmp[lane] : 0u;
        u32 wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 x = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += x;
        }
        s_tmp[lane] = wi - w;
        if (lane == 31) s_tmp[32] = wi;
    }
    __syncthreads();
    *total = s_tmp[32];
    return s_tmp[warp] + inc - v;
}

template <typename Acc>
__device__ __forceinline__ Acc g3_shfl_up_acc(Acc a, int o) {
    if constexpr (sizeof(Acc) == 8) {
        unsigned long long bits = *reinterpret_cast<const unsigned long long*>(&a);
        bits = __shfl_up_sync(0xffffffffu, bits, o);
        return *reinterpret_cast<Acc*>(&bits);
    } else {
        u32 bits = *reinterpret_cast<const u32*>(&a);
        bits = __shfl_up_sync(0xffffffffu, bits, o);
        return *reinterpret_cast<Acc*>(&bits);
    }
}

// One level of a walk over n points (a multiple of IT, padded with inert
// points) in xh, IT per thread, contiguous.  A handle holds the rank bits
// (rmask), the query bit at qsh and the local index above it; the level's
// nodes are the runs of equal r >> (lv+1) and, with BMAP, also start at
// the positions marked in bmap.  With SCAN, the segmented scan of F: a
// datum with bit lv = 0 feeds its node, a query with bit lv = 1 takes F over
// the node's feeding data before it (into val by its index, combined with
// what it holds).  Then, with split, the stable split of every node by bit
// lv (zero counts kept per node at its head position in hz).  The scan
// element is packed: bit 31 a head seen, bits 16..30 the last head's
// position, bits 0..15 the zero count since it.
template <class Op, int IT, bool SCAN, bool BMAP>
__device__ __noinline__ void g3_walk(u32 n, u32 lv, u32 rmask, u32 qsh, bool split, typename Op::Acc* val, u32* xh,
                                        unsigned short* hz, const u32* bmap, u32* s_pk, typename Op::Acc* s_acc) {
    typedef typename Op::Acc Acc;
    constexpr u32 NONE = 0xffffffffu, HD = 0x80000000u;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 p0 = (u32)tid * IT;
    const bool active = p0 < n;
    const u32 sh = lv + 1u;
    __syncthreads();  // the level's order is in xh
    u32 h[IT];
    u32 zin[(IT + 1) / 2];
    u32 bm = 0;  // (BMAP) bit j: position p0 + j starts a block; bit IT: the next thread's first
    u32 loc = 0, prevnode = NONE, z_first = 0, hp = 0;
    Acc lacc = Op::e();
    int first_head = IT;
    bool first_ends = false;
    if (active) {
        prevnode = p0 > 0 ? (xh[pidx(p0 - 1u)] & rmask) >> sh : NONE;
        const u32 nextnode = p0 + IT < n ? (xh[pidx(p0 + IT)] & rmask) >> sh : NONE;
#pragma unroll
        for (int j = 0; j < IT; ++j) h[j] = xh[pidx(p0 + j)];
        if (BMAP) {
            const u32 w0 = p0 >> 5, o = p0 & 31u;
            const unsigned long long two = (unsigned long long)bmap[w0] | ((unsigned long long)bmap[w0 + 1] << 32);
            bm = (u32)(two >> o) & ((2u << IT) - 1u);
        }
#pragma unroll
        for (int j = 0; j < (IT + 1) / 2; ++j) zin[j] = 0u;
        Acc acc = Op::e();
        u32 zc = 0, pn = prevnode;
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const u32 p = p0 + j, r = h[j] & rmask, nd = r >> sh;
            const bool head = nd != pn || (BMAP && ((bm >> j) & 1u));
            if (head) {
                if (first_head == IT) {
                    first_head = j;
                    z_first = zc;
                    first_ends = j > 0;
                } else {
                    hz[hp] = (unsigned short)zc;  // the node before ended at j-1
                }
                acc = Op::e();
                zc = 0u;
                hp = p;
            }
            pn = nd;
            const u32 bit = (r >> lv) & 1u;
            if (SCAN) {
                const u32 q = (h[j] >> qsh) & 1u, i = h[j] >> (qsh + 1u);
                if (DOMAGG_GUARD(i < G3_CAP, SITE_GROUP_VAL)) {
                    // F(acc, v) serves both roles (a datum's sum, a query's value)
                    const Acc v = val[i], sum = Op::Fc(acc, v);
                    if (q && bit) val[i] = sum;
                    acc = (!q && !bit) ? sum : acc;
                }
            }
            zin[j >> 1] |= zc << (16 * (j & 1));
            zc += bit ^ 1u;
        }
        // the thread's last node ends here unless the next point continues it
        if (nextnode != pn || (BMAP && ((bm >> IT) & 1u))) {
            if (first_head < IT) {
                hz[hp] = (unsigned short)zc;
            } else {
                z_first = zc;
                first_ends = true;
            }
        }
        loc = (first_head < IT ? HD : 0u) | (hp << 16) | zc;
        lacc = acc;
    }
    // exclusive segmented scan of the threads' tails
    u32 inc = loc;
    Acc iacc = lacc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 np = __shfl_up_sync(0xffffffffu, inc, o);
        Acc na = Op::e();
        if (SCAN) na = g3_shfl_up_acc(iacc, o);
        if (lane >= o) {
            if (SCAN && !(inc & HD)) iacc = Op::Fc(na, iacc);
            if (!(inc & HD)) inc = np + (inc & 0xffffu);
        }
    }
    u32 lex = __shfl_up_sync(0xffffffffu, inc, 1);
    Acc lexa = Op::e();
    if (SCAN) lexa = g3_shfl_up_acc(iacc, 1);
    if (lane == 0) {
        lex = 0u;
        lexa = Op::e();
    }
    if (lane == 31) {
        s_pk[warp] = inc;
        if (SCAN) s_acc[warp] = iacc;
    }
    __syncthreads();
    if (warp == 0) {  // one warp scans the 32 warp totals (exclusive, in place)
        u32 wi = s_pk[lane];
        Acc wa = Op::e();
        if (SCAN) wa = s_acc[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 np = __shfl_up_sync(0xffffffffu, wi, o);
            Acc na = Op::e();
            if (SCAN) na = g3_shfl_up_acc(wa, o);
            if (lane >= o) {
                if (SCAN && !(wi & HD)) wa = Op::Fc(na, wa);
                if (!(wi & HD)) wi = np + (wi & 0xffffu);
            }
        }
        u32 wx = __shfl_up_sync(0xffffffffu, wi, 1);
        Acc wxa = Op::e();
        if (SCAN) wxa = g3_shfl_up_acc(wa, 1);
        if (lane == 0) {
            wx = 0u;
            wxa = Op::e();
        }
        s_pk[lane] = wx;
        if (SCAN) s_acc[lane] = wxa;
    }
    __syncthreads();
    // ex = (the warps before) then (the lanes before)
    const u32 wpk = s_pk[warp];
    const u32 ex = (lex & HD) ? lex : wpk + (lex & 0xffffu);
    Acc exa = Op::e();
    if (SCAN) exa = (lex & HD) ? lexa : Op::Fc(s_acc[warp], lexa);
    const u32 ex_zc = ex & 0xffffu, ex_hp = (ex >> 16) & 0x7fffu;
    // the points before the thread's first head continue a node from the left
    if (active && first_head > 0) {
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            if (j >= first_head) break;
            if (SCAN) {
                const u32 r = h[j] & rmask, bit = (r >> lv) & 1u, q = (h[j] >> qsh) & 1u;
                if (q && bit) {
                    const u32 i = h[j] >> (qsh + 1u);
                    val[i] = Op::Fc(val[i], exa);
                }
            }
            zin[j >> 1] += ex_zc << (16 * (j & 1));
        }
        if (first_ends) hz[ex_hp] = (unsigned short)(ex_zc + z_first);
    }
    __syncthreads();  // zero counts known; xh read
    if (!split || !active) return;
    u32 pn = prevnode, cur = ex_hp;  // the head of the node the thread starts in
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const u32 p = p0 + j, r = h[j] & rmask, nd = r >> sh, bit = (r >> lv) & 1u;
        if (nd != pn || (BMAP && ((bm >> j) & 1u))) cur = p;
        pn = nd;
        const u32 z = (zin[j >> 1] >> (16 * (j & 1))) & 0xffffu;
        const u32 np = bit ? cur + (u32)hz[cur] + (p - cur - z) : cur + z;
        if (DOMAGG_GUARD(np < n, SITE_GROUP_SPLIT)) xh[pidx(np)] = h[j];
    }
}

// Points per thread of a walk over n points: G3_IT_SMALL up to
// G3_IT_SMALL x 1024 points (fewer warps then hold them), else G3_ITEMS.
#ifndef DOMAGG_G3_IT_SMALL
#define DOMAGG_G3_IT_SMALL 5
#endif
constexpr u32 G3_IT_SMALL = DOMAGG_G3_IT_SMALL;
__device__ __forceinline__ u32 g3_items(u32 n) { return n <= G3_IT_SMALL * G3_THREADS ? G3_IT_SMALL : (u32)G3_ITEMS; }

template <class Op, bool SCAN, bool BMAP>
__device__ __forceinline__ void g3_walk_any(u32 n, u32 lv, u32 rmask, u32 qsh, bool split, typename Op::Acc* val,
                                            u32* xh, unsigned short* hz, const u32* bmap, u32* s_pk,
                                            typename Op::Acc* s_acc) {
    if (n <= G3_IT_SMALL * G3_THREADS)
        g3_walk<Op, G3_IT_SMALL, SCAN, BMAP>(n, lv, rmask, qsh, split, val, xh, hz, bmap, s_pk, s_acc);
    else
        g3_walk<Op, G3_ITEMS, SCAN, BMAP>(n, lv, rmask, qsh, split, val, xh, hz, bmap, s_pk, s_acc);
}

// The points level lv emits (data with rank bit lv = 0, queries with 1), in
// the outer order (n points, padded to a multiple of IT): their inner
// handles (local second rank | query bit << 14 | local index << 15) and, in
// bmap (cleared here), the first position of every block.  Returns their
// number.
template <int IT>
__device__ __noinline__ u32 g3_compact(u32 n, u32 lv, u32 gS, const u32* oxh, u32* ixh,
                                          const unsigned short* r1l, u32* bmap, u32* s_tmp) {
    constexpr u32 NONE = 0xffffffffu;
    const int tid = threadIdx.x;
    const u32 lrmask = (1u << gS) - 1u, sh = lv + 1u;
    const u32 p0 = (u32)tid * IT;
    const bool active = p0 < n;
    __syncthreads();  // the outer order is in oxh; the previous level is done with ixh and bmap
    for (u32 w = (u32)tid; w < G3_BMAP_WORDS; w += blockDim.x) bmap[w] = 0u;
    u32 h[IT];
    u32 emask = 0, cnt = 0;
    if (active) {
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            h[j] = oxh[pidx(p0 + j)];
            const u32 r = h[j] & lrmask, q = (h[j] >> gS) & 1u, bit = (r >> lv) & 1u;
            const u32 e = q == bit ? 1u : 0u;
            emask |= e << j;
            cnt += e;
        }
    }
    u32 m = 0;
    u32 c = g3_exscan_u32(cnt, s_tmp, &m);  // (its barriers also order the bitmap's clearing)
    if (active) {
        u32 prevblk = p0 > 0 ? (oxh[pidx(p0 - 1u)] & lrmask) >> sh : NONE;
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const u32 r = h[j] & lrmask, blk = r >> sh;
            if (blk != prevblk && c < m) atomicOr(&bmap[c >> 5], 1u << (c & 31u));
            prevblk = blk;
            if ((emask >> j) & 1u) {
                const u32 q = (h[j] >> gS) & 1u, i = h[j] >> (gS + 1u);
                if (DOMAGG_GUARD(c < G3_CAP && i < G3_CAP, SITE_GROUP_SPLIT))
                    ixh[pidx(c)] = (u32)r1l[i] | (q << G3_LBITS) | (i << (G3_LBITS + 1u));
                ++c;
            }
        }
    }
    return m;
}

// Level lv by pairs, for levels whose blocks are small (at most
// G3_PAIR_MAX points): every query that level lv emits (bit lv = 1) walks
// back over its block in the outer order (the block's points before it in
// the order of the last coordinate) and takes F over the data the level
// emits (bit lv = 0) whose local second rank is below its own -- the
// block's m = 2 problem by its definition, cheaper than the second rank's
// 13-14 level walks when blocks hold a few dozen points (measured at 2^21
// per side: group kernel 2.77 ms without, 2.31 with blocks up to 64
// points, 2.40 up to 128, 2.80 up to 256).
#ifndef DOMAGG_G3_PAIR_MAX
#define DOMAGG_G3_PAIR_MAX 64
#endif
constexpr u32 G3_PAIR_MAX = DOMAGG_G3_PAIR_MAX;
template <class Op, int IT>
__device__ __noinline__ void g3_pairwise(u32 n, u32 lv, u32 gS, const u32* oxh, const unsigned short* r1l,
                                         typename Op::Acc* val) {
    typedef typename Op::Acc Acc;
    const u32 lrmask = (1u << gS) - 1u, sh = lv + 1u;
    const u32 p0 = (u32)threadIdx.x * IT;
    __syncthreads();  // the outer order is in oxh
    if (p0 >= n) return;
#pragma unroll 1
    for (int j = 0; j < IT; ++j) {
        const u32 p = p0 + (u32)j, h = oxh[pidx(p)], r = h & lrmask;
        if (!((h >> gS) & 1u) || !((r >> lv) & 1u)) continue;  // a query that level lv emits
        const u32 blk = r >> sh, i = h >> (gS + 1u), rq = r1l[i];
        Acc acc = Op::e();
        for (u32 k = p; k-- > 0u;) {
            const u32 hk = oxh[pidx(k)], rk = hk & lrmask;
            if ((rk >> sh) != blk) break;
            if (!((hk >> gS) & 1u) && !((rk >> lv) & 1u)) {
                const u32 ik = hk >> (gS + 1u);
                if (DOMAGG_GUARD(ik < G3_CAP, SITE_GROUP_VAL) && r1l[ik] < rq) acc = Op::Fc(acc, val[ik]);
            }
        }
        if (DOMAGG_GUARD(i < G3_CAP, SITE_GROUP_VAL)) val[i] = Op::Fc(val[i], acc);
    }
}

// The largest block of level lv in group g: the points of 2^(lv+1) ranks
// (2^lv undoubled ones for a non-strict first coordinate), from the
// rank-sorted start positions rs of ranks [lo, hi).  Two barriers.
__device__ __forceinline__ u32 g3_max_block(const u32* __restrict__ rs, u32 lo, u32 hi, u32 ub, u32* s_tmp) {
    u32 mx = 0;
    for (u32 b = lo + ((u32)threadIdx.x << ub); b < hi; b += blockDim.x << ub)
        mx = max(mx, __ldg(rs + min(b + (1u << ub), hi)) - __ldg(rs + b));
    for (int o = 16; o >= 1; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = mx;
    __syncthreads();
    u32 m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_tmp[w]);
    return m;
}

// Dense ranks of the group's second ranks: the keys (in ixh, padded; pads
// all ones) and local indices (in hz) are sorted by one stable split per key
// bit, then ranked.  Writes r1l[i] for i < n; returns the largest rank.
template <int IT>
__device__ __noinline__ u32 g3_rerank(u32 n, u32 npad, u32 kbits, u32* key, unsigned short* idx,
                                         unsigned short* r1l, u32* s_tmp) {
    const int tid = threadIdx.x;
    const u32 p0 = (u32)tid * IT;
    const bool active = p0 < npad;
    for (u32 t = 0; t < kbits; ++t) {
        __syncthreads();
        u32 kk[IT];
        unsigned short ii[IT];
        u32 z = 0;
        if (active) {
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                kk[j] = key[pidx(p0 + j)];
                ii[j] = idx[p0 + j];
                z += ((kk[j] >> t) & 1u) ^ 1u;
            }
        }
        u32 Z = 0;
        const u32 zb = g3_exscan_u32(z, s_tmp, &Z);
        if (active) {
            u32 zs = zb;
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const u32 p = p0 + j, bit = (kk[j] >> t) & 1u;
                const u32 np = bit ? Z + (p - zs) : zs;
                zs += bit ^ 1u;
                if (DOMAGG_GUARD(np < npad, SITE_GROUP_SPLIT)) {
                    key[pidx(np)] = kk[j];
                    idx[np] = ii[j];
                }
            }
        }
    }
    __syncthreads();
    // rank = the number of key changes up to the position
    u32 kk[IT], f = 0;
    u32 prev = 0;
    if (active) {
        prev = p0 > 0 ? key[pidx(p0 - 1u)] : key[pidx(0)];
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            kk[j] = key[pidx(p0 + j)];
            f += kk[j] != (j ? kk[j - 1] : prev) ? 1u : 0u;
        }
    }
    u32 F = 0;
    u32 rk = g3_exscan_u32(f, s_tmp, &F);
    if (active) {
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            rk += kk[j] != (j ? kk[j - 1] : prev) ? 1u : 0u;
            const u32 i = idx[p0 + j];
            if (i < n) r1l[i] = (unsigned short)rk;
            if (p0 + j == n - 1u) s_tmp[34] = rk;  // the real points sort before the pads
        }
    }
    __syncthreads();
    return s_tmp[34];
}

// The deep levels of every m = 3 group (see the file comment).  Persistent
// CTAs (one per SM) take groups from a counter.  Inputs: the group-sorted
// points gv (per instance in buffer gv0 or gv1, by the parity of the group
// sort's passes): (rank | QUERY_BIT) << 32 | the point's position x in the
// order of the last coordinate; pr1 (second ranks) and pw (weights) by x.
// Writes gacc[x] = F over the query's partial results of the levels below
// gS, as a partial (read in that order by the per-query reduction).
template <class Op, int WT>
__global__ __launch_bounds__(G3_THREADS, 1) void k_group3(const Inst* __restrict__ inst, int k,
                                                          const u32* __restrict__ gslot_off,
                                                          const u32* __restrict__ rstart, const u64* __restrict__ gv0,
                                                          const u64* __restrict__ gv1, const u32* __restrict__ pr1,
                                                          const typename Op::W* __restrict__ pw,
                                                          typename Op::Part* __restrict__ gacc, Ctl* ctl,
                                                          int launch_idx) {
    typedef typename Op::Acc Acc;
    typedef G3Smem<Acc> SM;
    constexpr int T = G3_THREADS;
    extern __shared__ __align__(128) unsigned char smem[];
    Acc* val = reinterpret_cast<Acc*>(smem + SM::VAL);
    u32* oxh = reinterpret_cast<u32*>(smem + SM::OXH);
    u32* ixh = reinterpret_cast<u32*>(smem + SM::IXH);
    unsigned short* r1l = reinterpret_cast<unsigned short*>(smem + SM::R1L);
    unsigned short* hz = reinterpret_cast<unsigned short*>(smem + SM::HZ);
    u32* bmap = reinterpret_cast<u32*>(smem + SM::BMAP);
    __shared__ u32 s_tmp[36];
    __shared__ Acc s_acc[32];
    __shared__ u32 s_slot;
    const int tid = threadIdx.x;
    const u32 total = __ldg(gslot_off + k);
    for (;;) {
        if (tid == 0) s_slot = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        __syncthreads();
        const u32 slot = s_slot;
        if (slot >= total) break;
        const int s = upper_index(gslot_off, k + 1, slot);
        const Inst& I = inst[s];
        const u32 g = I.shard + (slot - __ldg(gslot_off + s)) * max(I.nshards, 1u);
        const u32 gS = I.gS, ns = I.flags & 1u;
        const u32 us = gS - ns, Uu = ns ? I.U[0] / 2u : I.U[0];
        const u32* rs = rstart + I.pt_off + (u32)s;
        const u32 a = __ldg(rs + (g << us)), e = __ldg(rs + min((g + 1u) << us, Uu));
        const bool odd = ((I.b[0] - gS + RADIX_BITS - 1) / RADIX_BITS) & 1u;
        const u64* __restrict__ gv = (odd ? gv1 : gv0) + I.pt_off + a;
        if (e - a > G3_CAP) {  // too large for shared memory: its levels go through HBM
            group_unit_parts<Op>(gv, e - a, I, gacc);
            __syncthreads();
            continue;
        }
        const u32 n = e - a;
        const u32 lrmask = (1u << gS) - 1u, b1 = I.b[1];
        const u32 npad = (n + g3_items(n) - 1u) / g3_items(n) * g3_items(n);
        // the group's points in the order of the last coordinate: outer
        // handles (rank bits below gS | query bit | local index), values,
        // and the second ranks to be ranked locally
        for (u32 i = tid; i < npad; i += T) {
            if (i < n) {
                const u64 v = gv[i];
                const u32 pr = (u32)(v >> 32), x = (u32)v;
                const bool q = (pr & QUERY_BIT) != 0u;
                const bool ok = domagg_check(x - I.pt_off < I.nD + I.nQ, SITE_GROUP_OUT);
                oxh[pidx(i)] = (pr & lrmask) | ((q ? 1u : 0u) << gS) | (i << (gS + 1u));
                if (q || !ok) val[i] = Op::e();
                else if constexpr (WT == 3) val[i] = Op::from_pay(0u);
                else if constexpr (Op::GATHER) val[i] = Op::from_w(__ldg(pw + x));
                else val[i] = Op::from_pay((u32)__ldg(pw + x));
                ixh[pidx(i)] = ok ? __ldg(pr1 + x) & low_mask(b1) : 0u;
            } else {
                // inert points: data whose rank bits are all ones (they never
                // feed, never receive, and stay behind every real point)
                oxh[pidx(i)] = lrmask;
                ixh[pidx(i)] = 0xffffffffu;
            }
            hz[i] = (unsigned short)i;
        }
        if (n == 0) {  // (uniform; every thread has read s_slot before the next claim)
            __syncthreads();
            continue;
        }
        const u32 rmax = n <= G3_IT_SMALL * T ? g3_rerank<G3_IT_SMALL>(n, npad, b1, ixh, hz, r1l, s_tmp)
                                              : g3_rerank<G3_ITEMS>(n, npad, b1, ixh, hz, r1l, s_tmp);
        const u32 nb1 = rmax ? 32u - (u32)__clz(rmax) : 0u;  // levels of the local second rank
        bool pairs = false;  // blocks shrink with the level: once small, small below too
        for (int lv = (int)gS - 1; lv >= 0; --lv) {
            if (!pairs && nb1 > 0)
                pairs = g3_max_block(rs, g << us, min((g + 1u) << us, Uu), (u32)lv + 1u - ns, s_tmp) <= G3_PAIR_MAX;
            if (pairs) {
                if (nb1 > 0) {
                    if (n <= G3_IT_SMALL * T) g3_pairwise<Op, G3_IT_SMALL>(npad, (u32)lv, gS, oxh, r1l, val);
                    else g3_pairwise<Op, G3_ITEMS>(npad, (u32)lv, gS, oxh, r1l, val);
                }
                if (lv > 0)
                    g3_walk_any<Op, false, false>(npad, (u32)lv, lrmask, gS, true, val, oxh, hz, bmap, s_tmp, s_acc);
                continue;
            }
            const u32 m = n <= G3_IT_SMALL * T ? g3_compact<G3_IT_SMALL>(npad, (u32)lv, gS, oxh, ixh, r1l, bmap, s_tmp)
                                               : g3_compact<G3_ITEMS>(npad, (u32)lv, gS, oxh, ixh, r1l, bmap, s_tmp);
            if (m > 0 && nb1 > 0) {
                const u32 mpad = (m + g3_items(m) - 1u) / g3_items(m) * g3_items(m);
                for (u32 x = m + (u32)tid; x < mpad; x += T) ixh[pidx(x)] = G3_LMASK;  // inert
                for (int j = (int)nb1 - 1; j >= 0; --j)
                    g3_walk_any<Op, true, true>(mpad, (u32)j, G3_LMASK, G3_LBITS, j > 0, val, ixh, hz, bmap, s_tmp,
                                                s_acc);
            }
            if (lv > 0)  // the order of level lv-1: split every node by bit lv
                g3_walk_any<Op, false, false>(npad, (u32)lv, lrmask, gS, true, val, oxh, hz, bmap, s_tmp, s_acc);
        }
        __syncthreads();
        // every query of the group: F over its partial results of the levels
        // below gS (the unit e if it has none), at its position
        for (u32 i = tid; i < n; i += T) {
            const u64 v = gv[i];
            if ((u32)(v >> 32) & QUERY_BIT) {
                const u32 x = (u32)v;
                if (domagg_check(x - I.pt_off < I.nD + I.nQ, SITE_GROUP_OUT)) gacc[x] = Op::to_part(val[i]);
            }
        }
        __syncthreads();  // shared memory is free for the next group
    }
}

}  // namespace domagg
