// k_group.cuh -- the deep rank levels of m = 2 in shared memory.
//
// For m = 2 a record of level lv is keyed by the prefix r0 >> (lv+1) of the
// first coordinate's rank (Sec. 5; the node of Sec. 3's P0/P1 sets).  All
// records of a point share the top bits of their keys with the point's rank,
// so the records sort (instruction 6m+2) can take its most significant
// digits on the points, before the flat map: the points, in the order of
// the last coordinate, are sorted stably by their group g = r0 >> gS (the
// top bits of every key of the levels lv < gS).  A group then holds every
// record of those levels whose node lies in it: the node of level lv covers
// 2^(lv+1) ranks and gS >= lv+1.  One CTA takes a group of at most
// GROUP_CAP points into shared memory and, level by level from lv = gS-1
// down to 0, forms the level's records there, finishes their sort on the
// remaining node-key bit and runs the segmented scan of F over them
// (instruction 6m+3); each query keeps F over its partial results of these
// levels (what instructions 6m+4, 6m+5 collect) and writes it, as one
// partial, at its position in the order of the last coordinate.  The levels
// lv >= gS go to k_top (per tile of points, k_top.cuh) or through the
// records in HBM, and the per-query reduction joins the parts.
//
// Shared-memory sort, level by level.  The group's points start in the
// order of the last coordinate, which is the order of the level gS-1
// records (one node: the whole group).  The order of level lv-1 is the
// order of level lv split stably by bit lv of the rank inside every node of
// level lv -- an MSD radix sort of the node keys, one bit per level, done
// on the points because a level's records are exactly its emitting points
// (data with bit lv = 0: P0; queries with bit lv = 1: P1).  Within a node the
// points keep the order of the last coordinate (queries before data on a
// tie), which is what the segmented scan needs (Sec. 5).
#pragma once
#include <type_traits>

#include "dev_common.cuh"
#include "k_points.cuh"

namespace domagg {

constexpr int GROUP_MAX_BITS = 13;       // gS <= 13: nodes of up to 2^13 ranks
constexpr int GROUP_THREADS = 1024;
constexpr int GROUP_ITEMS = 12;          // points per thread, at most
constexpr u32 GROUP_CAP = GROUP_THREADS * GROUP_ITEMS;  // points per group in shared memory
constexpr u32 GROUP_NODES = 1u << (GROUP_MAX_BITS - 1);  // nodes of one level in a group, at most

template <typename Acc>
__host__ __device__ constexpr size_t group_smem_bytes() {
    return (size_t)GROUP_CAP * sizeof(Acc) + (size_t)Padded<GROUP_CAP>::value * sizeof(u32) +
           2 * GROUP_NODES * sizeof(unsigned short);
}

// Per instance (one block each): the largest gS <= min(GROUP_MAX_BITS, b0)
// whose groups of 2^gS ranks that hold more than `cap` points each (too
// many for shared memory: heavy ties) hold at most a quarter of the points,
// and the number of groups G (m = 2: k_group; m = 3: k_group3); gS = 0 (no
// level in groups) if no width qualifies, or if the instance takes another
// path.  govf[pt_off + g] = 1 marks this shard's groups that overflow: their
// points' levels below gS go through the records in HBM.  With top_bits > 0, the
// levels from tS = max(gS, b0 - top_bits) up go to k_top, and the levels
// [gS, tS) through the records in HBM (lvmask); both masks hold this
// shard's levels only.
// rstart (per instance, at pt_off + s) holds the rank-sorted position of the
// first point of every (undoubled) rank, and n at index U.  A non-strict
// first coordinate doubles the ranks (2r for data, 2r+1 for queries), so a
// group of 2^gS ranks is 2^(gS-1) undoubled ranks.  Also writes gbits[s],
// the bits of the group id (b0 - gS) the group sort sorts.
template <int M>
__global__ __launch_bounds__(1024) void k_group_plan(Inst* inst, const u32* __restrict__ rstart,
                                                    u32* __restrict__ gbits, unsigned char* __restrict__ govf,
                                                    u32 cap, int max_bits, int top_bits) {
    __shared__ u32 s_ovf[32];
    __shared__ u32 s_done;
    const int s = blockIdx.x;
    Inst& I = inst[s];
    const u32 n = I.nD + I.nQ;
    const u32 ns = I.flags & 1u;
    const u32 U = I.U[0], b0 = I.b[0];
    const u32 Uu = ns ? U / 2u : U;
    const u32* rs = rstart + I.pt_off + (u32)s;
    u32 chosen = 0, G = 0;
    const bool eligible = (M == 2 || M == 3) && rstart && n > 0 && b0 > 0 &&
                          !(I.flags & (FLAG_WAVELET | FLAG_VIRTUAL_LAST));
    for (int S = eligible ? min(min(max_bits, GROUP_MAX_BITS), (int)b0) : 0; S >= 1; --S) {
        const u32 us = (u32)S - ns;  // undoubled ranks per group: 2^us
        const u32 g_n = (Uu + (1u << us) - 1u) >> us;
        u32 ov = 0;  // points in groups too large for shared memory
        for (u32 g = threadIdx.x; g < g_n; g += blockDim.x) {
            const u32 lo = g << us, hi = min((g + 1u) << us, Uu);
            const u32 c = __ldg(rs + hi) - __ldg(rs + lo);
            if (c > cap) ov += c;
        }
        for (int o = 16; o >= 1; o >>= 1) ov += __shfl_xor_sync(0xffffffffu, ov, o);
        if ((threadIdx.x & 31) == 0) s_ovf[threadIdx.x >> 5] = ov;
        __syncthreads();
        if (threadIdx.x == 0) {
            u32 t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_ovf[w];
            s_done = t <= n / 4u ? 1u : 0u;
        }
        __syncthreads();
        const bool ok = s_done != 0u;
        __syncthreads();
        if (ok) {
            chosen = (u32)S;
            G = g_n;
            break;
        }
    }
    if (chosen && govf) {  // this shard's groups that overflow
        const u32 us = chosen - ns, nsh = max(I.nshards, 1u);
        for (u32 g = threadIdx.x; g < G; g += blockDim.x) {
            const u32 lo = g << us, hi = min((g + 1u) << us, Uu);
            govf[I.pt_off + g] = (__ldg(rs + hi) - __ldg(rs + lo) > cap && g % nsh == I.shard) ? 1u : 0u;
        }
    }
    if (threadIdx.x == 0) {
        I.gS = chosen;
        I.G = chosen ? G : 0u;
        if (gbits) gbits[s] = chosen ? b0 - chosen : 0u;
        // the levels >= gS of this shard: from tS up per tile (k_top), below
        // tS through the records in HBM
        const u32 nlev = M == 1 ? 1u : b0;
        const u32 ns = max(I.nshards, 1u);
        const bool top = M == 2 && top_bits > 0 && n > 0 && b0 > 0 && !(I.flags & (FLAG_WAVELET | FLAG_VIRTUAL_LAST));
        const u32 tS = top ? max(chosen, b0 > (u32)top_bits ? b0 - (u32)top_bits : 0u) : nlev;
        u32 mask = 0, tmask = 0;
        for (u32 lv = chosen; lv < nlev && lv < 32u; ++lv)
            if ((lv - chosen) % ns == I.shard) {
                if (lv >= tS) tmask |= 1u << lv;
                else mask |= 1u << lv;
            }
        I.tS = tS;
        I.topmask = n > 0 ? tmask : 0u;
        I.lvmask = n > 0 ? mask : 0u;
    }
}

// Work list of k_group: slot offsets of the instances' groups (exclusive
// scan of G over the instances that use groups).  One block.
static __global__ __launch_bounds__(1024) void k_group_slots(const Inst* __restrict__ inst, int k,
                                                            u32* __restrict__ gslot_off) {
    __shared__ u32 carry;
    __shared__ u32 warp_sum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < k; base += blockDim.x) {
        const int s = base + threadIdx.x;
        u32 v = 0;
        if (s < k && inst[s].gS) {  // groups g with g % nshards == shard
            const u32 ns = max(inst[s].nshards, 1u), sh = inst[s].shard, G = inst[s].G;
            v = sh < G ? (G - sh + ns - 1) / ns : 0u;
        }
        u32 inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        if (lane == 31) warp_sum[warp] = inc;
        __syncthreads();
        u32 add = carry;
        for (int w = 0; w < warp; ++w) add += warp_sum[w];
        if (s < k) gslot_off[s] = add + inc - v;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) carry += warp_sum[w];
        __syncthreads();
    }
    if (threadIdx.x == 0) gslot_off[k] = carry;
}

// Segmented-scan element of a level: a node head seen, F over the emitting
// data since the last head, and the points with rank bit lv = 0 since it.
template <typename Acc>
struct GScan {
    u32 hd;
    Acc acc;
    u32 zc;
};
// a precedes b; float-float sums combine without renormalisation (the
// block scan's tree is ten levels deep, so the low parts stay tiny)
template <class Op>
__device__ __forceinline__ GScan<typename Op::Acc> gscan_combine(const GScan<typename Op::Acc>& a,
                                                                const GScan<typename Op::Acc>& b) {
    GScan<typename Op::Acc> r;
    r.hd = a.hd | b.hd;
    r.acc = b.hd ? b.acc : Op::Fc(a.acc, b.acc);
    r.zc = b.hd ? b.zc : a.zc + b.zc;
    return r;
}
template <typename Acc>
__device__ __forceinline__ GScan<Acc> gscan_shfl_up(const GScan<Acc>& v, int o) {
    GScan<Acc> r;
    r.hd = __shfl_up_sync(0xffffffffu, v.hd, o);
    r.zc = __shfl_up_sync(0xffffffffu, v.zc, o);
    if constexpr (sizeof(Acc) == 8) {
        unsigned long long bits = *reinterpret_cast<const unsigned long long*>(&v.acc);
        bits = __shfl_up_sync(0xffffffffu, bits, o);
        r.acc = *reinterpret_cast<Acc*>(&bits);
    } else {
        u32 bits = *reinterpret_cast<const u32*>(&v.acc);
        bits = __shfl_up_sync(0xffffffffu, bits, o);
        r.acc = *reinterpret_cast<Acc*>(&bits);
    }
    return r;
}

// The nb rank levels d = nb-1 .. 0 of one block of points (handles in xh,
// padded layout: the nb rank bits of the levels, the query bit above them,
// the point's index above that; values in val by that index), in the order
// of the last coordinate.  A group (k_group) is nb = gS levels of nodes that
// lie wholly inside it; with TOP (k_top) the block is a tile of a range of
// points in the order of the last coordinate, the nodes continue across the
// range's tiles, and frun (heap order: level d's nodes from (1 << (nb-1-d))
// - 1) holds F over each node's data in the range's earlier tiles; only the
// levels in scan_mask are scanned (the others are only split).
// IT points per thread, contiguous: thread t holds positions
// [t*IT, t*IT + IT).  Per level, one walk over a thread's points applies the
// thread-local part of the segmented scan (queries add F over the node's
// data before them within the thread; the exclusive count of rank bit d = 0
// inside the node is kept per point), a block scan of the threads' tails
// gives each thread the part from before it, a second walk adds that part
// to the points before the thread's first node head only, and the split
// scatters every point to its place in the next level's order.  With TOP,
// a node's scan starts at its head from frun (so every query of the node
// receives the earlier tiles' part with the rest), and F at the node's end
// (ntot, preset to frun for nodes the tile does not hold; two halves of
// 2^(nb-1) entries taken by alternate levels, so that a level's preset
// never meets the previous level's readers) becomes the new frun.
// One walk combines every point's value with the running F (the sum of a
// datum is kept, a query's own value takes it): the same operation for
// both roles, so a warp does not run the two one after the other.
template <class Op, int IT, bool TOP>
__device__ __forceinline__ void group_levels(u32 n, u32 nb, u32 scan_mask, typename Op::Acc* val, u32* xh,
                                             unsigned short* nstart, unsigned short* nzero,
                                             GScan<typename Op::Acc>* s_w, typename Op::Acc* frun,
                                             typename Op::Acc* ntot) {
    typedef typename Op::Acc Acc;
    typedef GScan<Acc> E;
    constexpr u32 NONE = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const E ident{0u, Op::e(), 0u};
    const u32 p0 = (u32)tid * IT;
    const bool active = p0 < n;
    const u32 lrmask = (1u << nb) - 1u;
    const u32 gS = nb;  // the query bit sits above the rank bits
    for (int lv = (int)nb - 1; lv >= 0; --lv) {
        const bool scan = !TOP || ((scan_mask >> lv) & 1u);
        const u32 nnodes = 1u << (nb - 1u - (u32)lv), hoff = nnodes - 1u;  // (TOP) the level's nodes in frun
        Acc* lnt = TOP ? ntot + ((u32)(lv & 1) << (nb - 1u)) : nullptr;
        if (TOP && scan)
            for (u32 x = (u32)tid; x < nnodes; x += blockDim.x) lnt[x] = frun[hoff + x];
        __syncthreads();  // the handles of this level's order are in xh
        const u32 sh = (u32)lv + 1u;
        u32 h[IT];
        u32 zin[IT / 2];
        E loc = ident;
        int first_head = IT;   // first point of the thread that starts a node
        u32 z_first = 0;       // the first (continuing) node's zero count in this thread
        Acc a_first = Op::e();  // (TOP) and its F over the thread's data
        bool first_ends = false;
        u32 first_node = NONE;
        if (active) {
            const u32 prevnode = p0 > 0 ? (xh[pidx(p0 - 1)] & lrmask) >> sh : NONE;
            const u32 nextnode = p0 + IT < n ? (xh[pidx(p0 + IT)] & lrmask) >> sh : NONE;
#pragma unroll
            for (int j = 0; j < IT; ++j) h[j] = xh[pidx(p0 + j)];
#pragma unroll
            for (int j = 0; j < IT / 2; ++j) zin[j] = 0u;
            Acc acc = Op::e();
            u32 zc = 0, pn = prevnode;
            first_node = (h[0] & lrmask) >> sh;
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const u32 p = p0 + j;
                {
                    const u32 lr = h[j] & lrmask, nd = lr >> sh;
                    if (nd != pn) {
                        if (first_head == IT) {
                            first_head = j;
                            z_first = zc;
                            if (TOP) a_first = acc;
                            first_ends = j > 0;
                        } else {
                            nzero[pn] = (unsigned short)zc;  // the node before ended at j-1 and began here
                            if (TOP && scan) lnt[pn] = acc;
                        }
                        acc = (TOP && scan) ? frun[hoff + nd] : Op::e();
                        zc = 0u;
                        nstart[nd] = (unsigned short)p;
                    }
                    pn = nd;
                    const u32 bit = (lr >> lv) & 1u, q = (h[j] >> gS) & 1u, i = h[j] >> (gS + 1u);
                    if (scan && DOMAGG_GUARD(i < GROUP_CAP && nd < GROUP_NODES, SITE_GROUP_VAL)) {
                        // F(acc, v) serves both roles (a datum's sum, a query's value)
                        const Acc v = val[i], sum = Op::Fc(acc, v);
                        if (q && bit) val[i] = sum;
                        acc = (!q && !bit) ? sum : acc;
                    }
                    zin[j >> 1] |= zc << (16 * (j & 1));
                    zc += bit ^ 1u;
                }
            }
            // the thread's last node ends here unless the next point continues it
            if (nextnode != pn) {
                if (first_head < IT) {
                    nzero[pn] = (unsigned short)zc;
                    if (TOP && scan) lnt[pn] = acc;
                } else {
                    z_first = zc;
                    if (TOP) a_first = acc;
                    first_ends = true;
                }
            }
            loc.hd = first_head < IT ? 1u : 0u;
            loc.acc = acc;
            loc.zc = zc;
        }
        // exclusive segmented scan of the threads' tails: the part of each
        // thread's first node that lies before the thread
        E inc = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const E nb = gscan_shfl_up(inc, o);
            if (lane >= o) inc = gscan_combine<Op>(nb, inc);
        }
        E lex = gscan_shfl_up(inc, 1);
        if (lane == 0) lex = ident;
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {  // one warp scans the 32 warp totals (exclusive, in place)
            E wi = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const E nb = gscan_shfl_up(wi, o);
                if (lane >= o) wi = gscan_combine<Op>(nb, wi);
            }
            E wx = gscan_shfl_up(wi, 1);
            if (lane == 0) wx = ident;
            s_w[lane] = wx;
        }
        __syncthreads();
        const E ex = gscan_combine<Op>(s_w[warp], lex);
        // the points before the thread's first head continue a node from the left
        if (active && first_head > 0) {
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                if (j >= first_head) break;
                {
                    const u32 lr = h[j] & lrmask, bit = (lr >> lv) & 1u, q = (h[j] >> gS) & 1u;
                    if (scan && q && bit) {
                        const u32 i = h[j] >> (gS + 1u);
                        val[i] = Op::Fc(val[i], ex.acc);
                    }
                    zin[j >> 1] += ex.zc << (16 * (j & 1));
                }
            }
            if (first_ends) {
                nzero[first_node] = (unsigned short)(ex.zc + z_first);
                if (TOP && scan) lnt[first_node] = Op::Fc(ex.acc, a_first);
            }
        }
        __syncthreads();  // node starts and zero counts known; xh read
        if (TOP && scan)  // the range's running F per node, renormalised
            for (u32 x = (u32)tid; x < nnodes; x += blockDim.x) frun[hoff + x] = Op::F(Op::e(), lnt[x]);
        if (lv == 0) break;
        // stable split of every node by bit lv: the order of level lv-1
        if (active) {
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const u32 p = p0 + j;
                {
                    const u32 lr = h[j] & lrmask, nd = lr >> sh, bit = (lr >> lv) & 1u;
                    const u32 st = nstart[nd], z = (zin[j >> 1] >> (16 * (j & 1))) & 0xffffu;
                    const u32 np = bit ? st + nzero[nd] + (p - st - z) : st + z;
                    if (DOMAGG_GUARD(np < n && nd < GROUP_NODES, SITE_GROUP_SPLIT)) xh[pidx(np)] = h[j];
                }
            }
        }
    }
}

// A group too large for shared memory: its queries' group part is the unit
// (their levels below gS go through the records in HBM).
template <class Op>
__device__ __forceinline__ void group_unit_parts(const u64* __restrict__ gv, u32 n, const Inst& I,
                                                 typename Op::Part* __restrict__ gacc) {
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
        const u64 v = gv[i];
        if ((u32)(v >> 32) & QUERY_BIT) {
            const u32 x = (u32)v;
            if (domagg_check(x - I.pt_off < I.nD + I.nQ, SITE_GROUP_OUT)) gacc[x] = Op::to_part(Op::e());
        }
    }
}

// The deep levels of every group (see the file comment).  Persistent CTAs
// (one per SM) take groups from a counter.  Inputs: the group-sorted points
// gv (per instance in buffer gv0 or gv1, by the parity of the group sort's
// passes): (rank | QUERY_BIT) << 32 | payload, the payload being a query's
// position x in the order of the last coordinate, a datum's weight bits, or
// (8-byte weights) the datum's position in pw.  Writes gacc[x] = F over the
// query's partial results of the levels below gS, as a partial (rounded once,
// like a level's partial; read in that order by k_top and the per-query
// reduction).
template <class Op>
__global__ __launch_bounds__(GROUP_THREADS, 1) void k_group(const Inst* __restrict__ inst, int k,
                                                            const u32* __restrict__ gslot_off,
                                                            const u32* __restrict__ rstart, const u64* __restrict__ gv0,
                                                            const u64* __restrict__ gv1,
                                                            const typename Op::W* __restrict__ pw,
                                                            typename Op::Part* __restrict__ gacc, Ctl* ctl,
                                                            int launch_idx) {
    typedef typename Op::Acc Acc;
    typedef GScan<Acc> E;
    constexpr int T = GROUP_THREADS;
    extern __shared__ __align__(128) unsigned char smem[];
    Acc* val = reinterpret_cast<Acc*>(smem);                              // by original index
    u32* xh = reinterpret_cast<u32*>(smem + (size_t)GROUP_CAP * sizeof(Acc));  // handles, padded
    unsigned short* nstart = reinterpret_cast<unsigned short*>(xh + Padded<GROUP_CAP>::value);
    unsigned short* nzero = nstart + GROUP_NODES;
    __shared__ E s_w[T / 32];
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
        if (e - a > GROUP_CAP) {  // too large for shared memory: its levels go through HBM
            group_unit_parts<Op>(gv, e - a, I, gacc);
            __syncthreads();
            continue;
        }
        const u32 n = e - a;
        const u32 lrmask = (1u << gS) - 1u;
        // the group's points in the order of the last coordinate: handles
        // (rank bits below gS | query bit | original index) and values
        for (u32 i = tid; i < n; i += T) {
            const u64 v = gv[i];
            const u32 pr = (u32)(v >> 32), pv = (u32)v;
            const bool q = (pr & QUERY_BIT) != 0u;
            xh[pidx(i)] = (pr & lrmask) | ((q ? 1u : 0u) << gS) | (i << (gS + 1u));
            if (q) val[i] = Op::e();
            else if constexpr (Op::GATHER) val[i] = Op::from_w(__ldg(pw + pv));
            else val[i] = Op::from_pay(pv);
        }
        static_assert(GROUP_ITEMS == 12, "items per thread dispatched below");
        {
            const u32 itp = n <= 8u * T ? 8u : 12u;
            const u32 npad = (n + itp - 1) / itp * itp;
            // the last thread's tail is padded with inert points (data whose rank
            // bits are all ones: they never contribute, never receive, and stay
            // behind every real point of their node), so no walk checks bounds
            for (u32 i = n + tid; i < npad; i += T) xh[pidx(i)] = lrmask;
            __syncthreads();
            if (n <= 8u * T) group_levels<Op, 8, false>(npad, gS, ~0u, val, xh, nstart, nzero, s_w, nullptr, nullptr);
            else group_levels<Op, 12, false>(npad, gS, ~0u, val, xh, nstart, nzero, s_w, nullptr, nullptr);
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
