// k_top.cuh -- m = 2: the top rank levels per tile of points in the order of
// the last coordinate.
//
// A record of level lv is keyed by the node r0 >> (lv+1) (Sec. 5); the top
// levels lv >= tS (tS >= b0 - TOP_MAX_BITS) have at most 2^(TOP_MAX_BITS-1)
// nodes each.  The points, already in the order of the last coordinate (the
// order of the top level's records: one node), are cut into ranges of whole
// tiles; one CTA takes a range tile by tile, and in each tile forms, sorts
// and scans the records of every top level in shared memory as k_group does
// for a group (the order of level lv-1 is the order of level lv split stably
// by bit lv inside every node; a level's segmented scan of F runs in that
// order, instructions 6m+1 .. 6m+3).  A node's records continue across
// tiles and ranges, so the scan carries, per node, F over the node's data in
// the range's earlier tiles (frun, in shared memory), and every query keeps
// F over its partial results of the range's top levels and of the levels
// below gS (those from k_group, by position: gacc) in topv.  What the
// range's nodes gathered (agg) is then scanned across the ranges of the
// instance in a fixed order (k_top_carry), and the per-query reduction adds
// to each query, for every top level where it has a record, the carry of its
// node from the ranges before its own (k_reduce_top).
#pragma once
#include <type_traits>

#include "dev_common.cuh"
#include "k_group.cuh"
#include "k_points.cuh"

namespace domagg {

constexpr int TOP_MAX_BITS = 12;                     // top levels: at most 2^11 nodes each
constexpr u32 TOP_STRIDE = 1u << TOP_MAX_BITS;       // per range: F of every top-level node (heap order)
constexpr u32 TOP_NODES = TOP_STRIDE / 2;            // nodes of one level, at most
constexpr int TOP_RANGES_PER_SM = 4;                  // ranges of tiles per SM over all points
constexpr int TOP_THREADS = GROUP_THREADS;
constexpr u32 TOP_TILE = GROUP_CAP;                  // points per tile
static_assert(TOP_TILE % TOP_THREADS == 0, "whole rounds of the tile load");

// Shared memory of k_top: values (by the point's index in the tile),
// handles (padded), node starts and zero counts, the range's F per node
// (heap order) and the nodes' F over the tile (two halves).
template <typename Acc>
struct TopSmem {
    static constexpr size_t OFF_VAL = 0;
    static constexpr size_t OFF_XH = OFF_VAL + (size_t)TOP_TILE * sizeof(Acc);
    static constexpr size_t OFF_NSTART = OFF_XH + (size_t)Padded<TOP_TILE>::value * sizeof(u32);
    static constexpr size_t OFF_NZERO = OFF_NSTART + (size_t)TOP_NODES * sizeof(unsigned short);
    static constexpr size_t OFF_FRUN = (OFF_NZERO + (size_t)TOP_NODES * sizeof(unsigned short) + 15) & ~(size_t)15;
    static constexpr size_t OFF_NTOT = OFF_FRUN + (size_t)TOP_STRIDE * sizeof(Acc);
    static constexpr size_t TOTAL = OFF_NTOT + (size_t)TOP_STRIDE * sizeof(Acc);
};

// Range r (of all instances: prange_off[s] is instance s's first) of
// range_pts points: its instance and the points [start, end).
struct TopRange {
    int s;
    u32 rr, ps, start, end;
};
__device__ __forceinline__ TopRange top_range(u32 r, const u32* prange_off, int k, const u32* pt_offs,
                                              u32 range_pts) {
    TopRange R;
    R.s = upper_index(prange_off, k + 1, r);
    R.rr = r - __ldg(prange_off + R.s);
    R.ps = __ldg(pt_offs + R.s);
    R.start = R.ps + R.rr * range_pts;
    R.end = min(R.start + range_pts, __ldg(pt_offs + R.s + 1));
    return R;
}

// The top levels of every range (see the file comment).  Persistent CTAs
// (one per SM) take ranges from a counter.  Inputs, in the order of the last
// coordinate: pr0 (rank | QUERY_BIT), pw (a datum's weight bits, or its
// 8-byte weight for WT = 1) and, for an instance with groups, gacc (a
// query's F over the levels below gS).  Writes topv[x] (queries: F over
// their partial results of the range's top levels and the levels below gS,
// the unit if none) and agg[r][h] (F over the range's data of node h, heap
// order; rows r < nrows, the rows the caller reserved: a range outside them
// is skipped).
template <class Op, int WT>
__global__ __launch_bounds__(TOP_THREADS, 1) void k_top(const Inst* __restrict__ inst, int k,
                                                        const u32* __restrict__ prange_off,
                                                        const u32* __restrict__ pt_offs, u32 range_pts,
                                                        const u32* __restrict__ pr0,
                                                        const typename Op::W* __restrict__ pw,
                                                        const typename Op::Part* __restrict__ gacc,
                                                        typename Op::Acc* __restrict__ topv,
                                                        typename Op::Acc* __restrict__ agg, u32 nrows, Ctl* ctl,
                                                        int launch_idx) {
    typedef typename Op::Acc Acc;
    typedef TopSmem<Acc> SM;
    constexpr int T = TOP_THREADS;
    extern __shared__ __align__(128) unsigned char smem[];
    Acc* val = reinterpret_cast<Acc*>(smem + SM::OFF_VAL);
    u32* xh = reinterpret_cast<u32*>(smem + SM::OFF_XH);
    unsigned short* nstart = reinterpret_cast<unsigned short*>(smem + SM::OFF_NSTART);
    unsigned short* nzero = reinterpret_cast<unsigned short*>(smem + SM::OFF_NZERO);
    Acc* frun = reinterpret_cast<Acc*>(smem + SM::OFF_FRUN);
    Acc* ntot = reinterpret_cast<Acc*>(smem + SM::OFF_NTOT);
    __shared__ GScan<Acc> s_w[T / 32];
    __shared__ u32 s_slot;
    __shared__ u32 s_qmask[T];  // per thread: which of its tile points are queries
    const int tid = threadIdx.x;
    const u32 total = __ldg(prange_off + k);
    for (;;) {
        if (tid == 0) s_slot = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        __syncthreads();
        const u32 r = s_slot;
        if (r >= total) break;
        if (!domagg_check(r < nrows, SITE_GROUP_OUT)) {  // never taken for a table of this call
            __syncthreads();
            continue;
        }
        const TopRange R = top_range(r, prange_off, k, pt_offs, range_pts);
        const Inst& I = inst[R.s];
        const u32 tmask = I.topmask, tS = I.tS, b0 = I.b[0];
        const bool grouped = I.gS != 0u;
        // (the instance's levels from tS up: nb <= TOP_MAX_BITS by k_group_plan)
        const u32 nb = tmask ? b0 - tS : 0u;
        if (nb > 0u && DOMAGG_GUARD(nb <= (u32)TOP_MAX_BITS, SITE_GROUP_NODE)) {
            const u32 lrmask = (1u << nb) - 1u, stride = 1u << nb;
            for (u32 h = tid; h < stride; h += T) frun[h] = Op::e();
            for (u32 a0 = R.start; a0 < R.end; a0 += TOP_TILE) {
                const u32 n = min(R.end - a0, TOP_TILE);
                __syncthreads();  // frun reset, or the previous tile's values written out
                // thread t loads points t + k*T, half a tile's rounds at a time
                // (their loads in flight together); s_qmask bit k: that point
                // is a query
                u32 qmask = 0;
                constexpr int K = TOP_TILE / T, KH = K / 2;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    u32 v[KH];
#pragma unroll
                    for (int kk = 0; kk < KH; ++kk) {
                        const u32 i = (u32)tid + (u32)(half * KH + kk) * T;
                        v[kk] = i < n ? pr0[a0 + i] : 0u;
                    }
                    Acc w[KH];
#pragma unroll
                    for (int kk = 0; kk < KH; ++kk) {
                        const u32 i = (u32)tid + (u32)(half * KH + kk) * T;
                        const bool q = (v[kk] & QUERY_BIT) != 0u;
                        w[kk] = Op::e();
                        if (i < n) {
                            if (q) w[kk] = grouped ? Op::from_part(gacc[a0 + i]) : Op::e();
                            else if constexpr (Op::GATHER) w[kk] = Op::from_w(pw[a0 + i]);
                            else if constexpr (WT == 3) w[kk] = Op::from_pay(0u);
                            else w[kk] = Op::from_pay((typename Op::Pay)pw[a0 + i]);
                        }
                    }
#pragma unroll
                    for (int kk = 0; kk < KH; ++kk) {
                        const u32 i = (u32)tid + (u32)(half * KH + kk) * T;
                        if (i < n) {
                            const bool q = (v[kk] & QUERY_BIT) != 0u;
                            xh[pidx(i)] = (((v[kk] & ~QUERY_BIT) >> tS) & lrmask) | ((q ? 1u : 0u) << nb) |
                                          (i << (nb + 1u));
                            val[i] = w[kk];
                            qmask |= (q ? 1u : 0u) << (half * KH + kk);
                        }
                    }
                }
                s_qmask[tid] = qmask;
                const u32 itp = n <= 8u * T ? 8u : 12u;
                const u32 npad = (n + itp - 1) / itp * itp;
                // inert padding: data whose rank bits are all ones (see k_group)
                for (u32 i = n + tid; i < npad; i += T) xh[pidx(i)] = lrmask;
                __syncthreads();
                if (n <= 8u * T) group_levels<Op, 8, true>(npad, nb, tmask >> tS, val, xh, nstart, nzero, s_w, frun, ntot);
                else group_levels<Op, 12, true>(npad, nb, tmask >> tS, val, xh, nstart, nzero, s_w, frun, ntot);
                __syncthreads();
                const u32 qm = s_qmask[tid];
#pragma unroll
                for (int kk = 0; kk < K; ++kk)
                    if ((qm >> kk) & 1u) topv[a0 + (u32)tid + (u32)kk * T] = val[(u32)tid + (u32)kk * T];
            }
            __syncthreads();  // the last tile's node totals are in frun
            for (u32 h = tid; h < stride; h += T) agg[(u64)r * TOP_STRIDE + h] = frun[h];
        }
        __syncthreads();  // shared memory (and s_slot) free for the next range
    }
}

// Exclusive scan, in place, of the ranges' F per node over the ranges of
// one instance: agg[r][h] becomes F over agg[r'][h] of the instance's ranges
// r' < r (the first range's row is left as it is; nothing reads it).  One
// block per (instance with two or more ranges, 32 nodes); its 32 warps split
// the ranges into consecutive slices (lane = node): slice totals, their
// exclusive combination in slice order, then the running prefixes -- a
// fixed order, so float-float sums repeat exactly.
template <class Op>
__global__ __launch_bounds__(1024) void k_top_carry(const u32* __restrict__ multi, const u32* __restrict__ prange_off,
                                                   const Inst* __restrict__ inst, typename Op::Acc* __restrict__ agg,
                                                   u32 nrows) {
    typedef typename Op::Acc Acc;
    __shared__ Acc s_sum[32][33];
    const int s = (int)__ldg(multi + blockIdx.x);
    const Inst& I = inst[s];
    if (I.topmask == 0u) return;
    const u32 stride = 1u << (I.b[0] - I.tS);
    if (blockIdx.y * 32u >= stride) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 h = blockIdx.y * 32u + (u32)lane;
    const bool on = h < stride;
    const u32 r0 = __ldg(prange_off + s), r1 = __ldg(prange_off + s + 1);
    if (!domagg_check(r1 <= nrows && r0 <= r1, SITE_GROUP_OUT)) return;  // never taken for a table of this call
    const u32 n = r1 - r0, per = (n + 31) / 32;
    const u32 a = r0 + min(n, (u32)warp * per), b = r0 + min(n, (u32)(warp + 1) * per);
    Acc sum = Op::e();
    for (u32 r = a; r < b; r += 8) {
        Acc v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (on && r + i < b) ? agg[(u64)(r + i) * TOP_STRIDE + h] : Op::e();
#pragma unroll
        for (int i = 0; i < 8; ++i) sum = Op::F(sum, v[i]);
    }
    s_sum[warp][lane] = sum;
    __syncthreads();
    Acc run = Op::e();
    for (int w = 0; w < warp; ++w) run = Op::F(run, s_sum[w][lane]);
    for (u32 r = a; r < b; r += 8) {
        Acc v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (on && r + i < b) ? agg[(u64)(r + i) * TOP_STRIDE + h] : Op::e();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (on && r + i < b) agg[(u64)(r + i) * TOP_STRIDE + h] = run;
            run = Op::F(run, v[i]);
        }
    }
}

// Per-query reduction of m = 2 with top levels (replaces k_reduce there):
// one block of TOP_RED_THREADS per range of the chunk's instances [k0, k1).
// For each query: F over topv (the range's top levels and the levels below
// gS; gacc alone for an instance without top levels), its partials of the
// levels that went through the records in HBM (slots as in k_reduce) and,
// for every top level where it has a record, the carry of its node from the
// instance's earlier ranges (staged in shared memory).
constexpr int TOP_RED_THREADS = 1024;
template <class Op>
__global__ __launch_bounds__(TOP_RED_THREADS) void k_reduce_top(int k, int k0, const u32* __restrict__ prange_off, u32 range_pts,
                                                    const u32* __restrict__ chunk_off, const u32* __restrict__ pt_offs,
                                                    const u32* __restrict__ pr0, const u32* __restrict__ pj,
                                                    const u32* __restrict__ qchunk_base,
                                                    const u32* __restrict__ pt_tiles, const u32* __restrict__ tile_excl,
                                                    const u32* __restrict__ qseg_base /*[k1-k0][LMAX]*/,
                                                    const Inst* __restrict__ inst,
                                                    const typename Op::Part* __restrict__ partial, u32 n_partial,
                                                    const typename Op::Part* __restrict__ gacc,
                                                    const typename Op::Acc* __restrict__ topv,
                                                    const typename Op::Acc* __restrict__ carry, u32 nrows,
                                                    const unsigned char* __restrict__ govf) {
    typedef typename Op::Acc Acc;
    __shared__ Acc s_carry[TOP_STRIDE];
    constexpr u32 WARPS = TOP_RED_THREADS / 32;
    __shared__ u32 s_mask[WARPS][LMAX];  // per warp: query lanes holding a record of level lv
    __shared__ u32 s_base[WARPS][LMAX];  // per warp: first partial slot of level lv in this chunk
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 lt = lanemask_lt();
    const u32 r = __ldg(prange_off + k0) + blockIdx.x;
    const TopRange R = top_range(r, prange_off, k, pt_offs, range_pts);
    const int s = R.s;
    const Inst& I = inst[s];
    const u32 tmask = I.topmask, b0 = I.b[0];
    const bool carried = tmask != 0u && R.rr > 0u && domagg_check(r < nrows, SITE_REDUCE);
    if (carried) {
        const u32 stride = 1u << (b0 - I.tS);
        for (u32 h = threadIdx.x; h < stride; h += blockDim.x) s_carry[h] = carry[(u64)r * TOP_STRIDE + h];
    }
    __syncthreads();
    const u32 nQ = I.nQ;
    const u32 c0 = __ldg(chunk_off + s);
    const u32 cb = c0 + (R.start - R.ps) / 32u, ce = c0 + (R.end - R.ps + 31u) / 32u;
    for (u32 c = cb + (u32)warp; c < ce; c += WARPS) {
        const u32 p = R.ps + (c - c0) * 32u + (u32)lane;
        const bool valid = p < R.end;
        u32 local = 0, a = 0, bits0 = 0;
        bool q = false;
        if (valid) {
            u32 j = pj[p];
            if (j - R.ps >= __ldg(pt_offs + s + 1) - R.ps) j = R.ps;  // never taken for a valid permutation
            local = j - R.ps;
            q = local < nQ;
            if (q) {
                a = pr0[p] & ~QUERY_BIT;
                bits0 = a & low_mask(b0);  // a query's records: the 1-digits of its rank
            }
        }
        if (__ballot_sync(0xffffffffu, q) == 0u) continue;
        Acc acc = Op::e();
        if (q) acc = tmask ? topv[p] : (I.gS ? Op::from_part(gacc[p]) : Op::e());
        const u32 rec = q ? bits0 & hbm_levels(I, a, govf) : 0u;
        if (__ballot_sync(0xffffffffu, rec != 0u)) {  // levels whose records went through HBM: their partials
            if ((u32)lane < b0)
                s_base[warp][lane] =
                    __ldg(qseg_base + (u64)(s - k0) * LMAX + lane) + __ldg(qchunk_base + (u64)c * LMAX + lane) +
                    __ldg(tile_excl + (u64)(__ldg(pt_tiles + s) + (c - c0) / CS_CHUNKS) * CS_COUNTERS + LMAX + lane);
            s_mask[warp][lane] = warp_transpose32(rec, (u32)lane);  // lanes of level `lane`
            __syncwarp();
            u32 rem = rec;
#pragma unroll 4
            while (rem) {
                const u32 lv = __ffs(rem) - 1;
                rem &= rem - 1;
                const u32 slot = s_base[warp][lv] + (u32)__popc(s_mask[warp][lv] & lt);
                if (domagg_check(slot < n_partial, SITE_REDUCE)) acc = Op::F(acc, Op::from_part(partial[slot]));
            }
        }
        if (q && carried) {  // the carries of its top-level nodes (a short sum: combined without renormalising)
            Acc cs = Op::e();
            for (u32 top = bits0 & tmask; top; top &= top - 1) {
                const u32 lv = __ffs(top) - 1;
                cs = Op::Fc(cs, s_carry[(1u << (b0 - 1u - lv)) - 1u + (a >> (lv + 1u))]);
            }
            acc = Op::F(acc, cs);
        }
        if (q) {
            bool done = false;
            if constexpr (std::is_same<Op, OpSumF32>::value) {
                if (I.out_lo) {  // a shard keeps the float-float pair
                    reinterpret_cast<float*>(I.out)[local] = acc.hi;
                    I.out_lo[local] = acc.lo;
                    done = true;
                }
            }
            if (!done) reinterpret_cast<typename Op::Out*>(I.out)[local] = Op::to_out(acc);
        }
        __syncwarp();
    }
}

}  // namespace domagg
