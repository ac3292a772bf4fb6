// k_records.cuh -- the aggregation over the sorted records: the segmented
// scan of F (instruction 6m+3) and the per-query reduction of the partial
// results (what instructions 6m+4, 6m+5 compute, without the ID sort).
#pragma once
#include <type_traits>

#include "dev_common.cuh"
#include "k_radix.cuh"

namespace domagg {

// Record layout of a planned run, computed on the device from the count
// scan's per-(instance, level) totals (the host-side layout of an unplanned
// call, which needs their values on the host, as one block of 1024 threads).
// slot_map lists the chunk's segment slots, (instance - k0) << 5 | level, with
// every instance reserving as many slots as its rank digits can be at most;
// slots beyond an instance's actual levels are empty.  Writes the segment
// offsets and key bits and the per-(instance, level) record and query-slot
// bases.  If the records exceed a class's reserved capacity (T_cap for class
// 0, T1_cap for class 1) or the query slots Tq_cap, every segment is made
// empty and ERR_CAPACITY is raised: the kernels after it then write nothing
// outside their buffers (the chunk's outputs are undefined).
//
// Slots [0, nslot0) are class 0 (the key type of the pipeline), slots
// [nslot0, nslot) class 1 (32-bit keys, m >= 3): each class has its own
// record arrays, so its offsets (so: class 0's nslot0 + 1, then class 1's)
// and the bases in sbase restart at 0; query slots run on across both.
template <int M>
__global__ __launch_bounds__(1024) void k_layout(const Inst* __restrict__ inst, int k0,
                                                 const u32* __restrict__ lvl_tot, const u32* __restrict__ qlvl_tot,
                                                 const u32* __restrict__ slot_map, int nslot, int nslot0, u64 T_cap,
                                                 u64 T1_cap, u64 Tq_cap, u32* __restrict__ so, u32* __restrict__ sbits,
                                                 u32* __restrict__ sbase, u32* __restrict__ qsbase, Ctl* ctl) {
    __shared__ u64 w_a[32], w_q[32];
    __shared__ u64 carry_a, carry_q;
    __shared__ int s_over;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto sizes = [&](int g, u32& lv, u32& srel, u32& na, u32& nq, u32& bits) {
        const u32 sm = __ldg(slot_map + g);
        srel = sm >> 5;
        lv = sm & 31u;
        const Inst& I = inst[k0 + (int)srel];
        const u32 nlev = M == 1 ? 1u : I.b[0];
        na = nq = bits = 0;
        // the counts hold only the records this call puts through HBM
        // (hbm_levels: this shard's levels outside the groups and the
        // top-level tiles, and an overflowing group's levels below gS)
        if (lv < nlev) {
            na = __ldg(lvl_tot + (u64)(k0 + (int)srel) * LMAX + lv);
            nq = __ldg(qlvl_tot + (u64)(k0 + (int)srel) * LMAX + lv);
            if (M >= 2) bits = I.b[0] - 1u - lv + (M >= 3 ? I.b[1] : 0u) + (M >= 4 ? I.b[2] : 0u);
        }
    };
    // totals first (per class): the capacity decides between the layout and empty segments
    u64 ta0 = 0, ta1 = 0, tq = 0;
    for (int g = tid; g < nslot; g += 1024) {
        u32 lv, srel, na, nq, bits;
        sizes(g, lv, srel, na, nq, bits);
        if (g < nslot0) ta0 += na;
        else ta1 += na;
        tq += nq;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        ta0 += __shfl_xor_sync(0xffffffffu, ta0, o);
        ta1 += __shfl_xor_sync(0xffffffffu, ta1, o);
        tq += __shfl_xor_sync(0xffffffffu, tq, o);
    }
    __shared__ u64 w_b[32];
    if (lane == 0) {
        w_a[warp] = ta0;
        w_b[warp] = ta1;
        w_q[warp] = tq;
    }
    __syncthreads();
    if (tid == 0) {
        u64 A = 0, B = 0, Q = 0;
        for (int w = 0; w < 32; ++w) {
            A += w_a[w];
            B += w_b[w];
            Q += w_q[w];
        }
        s_over = (A > T_cap || B > T1_cap || Q > Tq_cap) ? 1 : 0;
        if (s_over) atomicOr(&ctl->error, ERR_CAPACITY);
        carry_a = carry_q = 0;
    }
    __syncthreads();
    const bool over = s_over != 0;
    for (int cls = 0; cls < 2; ++cls) {
    const int lo = cls == 0 ? 0 : nslot0, hi = cls == 0 ? nslot0 : nslot;
    u32* so_c = cls == 0 ? so : so + nslot0 + 1;
    if (tid == 0) carry_a = 0;  // each class's records restart at 0
    __syncthreads();
    for (int base = lo; base < hi; base += 1024) {
        const int g = base + tid;
        u32 lv = 0, srel = 0, na = 0, nq = 0, bits = 0;
        if (g < hi) sizes(g, lv, srel, na, nq, bits);
        if (over) na = nq = bits = 0;
        u64 ia = na, iq = nq;
        for (int o = 1; o < 32; o <<= 1) {
            const u64 xa = __shfl_up_sync(0xffffffffu, ia, o), xq = __shfl_up_sync(0xffffffffu, iq, o);
            if (lane >= o) {
                ia += xa;
                iq += xq;
            }
        }
        if (lane == 31) {
            w_a[warp] = ia;
            w_q[warp] = iq;
        }
        __syncthreads();
        u64 ea = carry_a, eq = carry_q;
        for (int w = 0; w < warp; ++w) {
            ea += w_a[w];
            eq += w_q[w];
        }
        ea += ia - na;
        eq += iq - nq;
        if (g < hi) {
            so_c[g - lo] = (u32)ea;
            sbits[g] = bits;
            sbase[(u64)srel * LMAX + lv] = (u32)ea;
            qsbase[(u64)srel * LMAX + lv] = (u32)eq;
        }
        __syncthreads();
        if (tid == 1023) {
            carry_a = ea + na;
            carry_q = eq + nq;
        }
        __syncthreads();
    }
    if (tid == 0) so_c[hi - lo] = (u32)carry_a;
    __syncthreads();
    }
}

// Look-back status of the segmented scan.  The aggregate and the inclusive
// prefix live in separate fields, each written once before the flag that
// announces it (release), and read after that flag (acquire): a reader that
// saw ST_AGG never meets a half-written prefix.
template <typename Acc>
struct alignas(32) SegStatus {
    u32 flag;      // (epoch << 2) | ST_AGG / ST_PREFIX
    u32 has_head;  // a segment starts inside the tile (with ST_AGG)
    Acc agg;       // F over the tile's items after its last head (ST_AGG)
    Acc incl;      // inclusive prefix at the tile's end (ST_PREFIX)
};

template <typename Acc>
__device__ __forceinline__ void seg_publish_agg(SegStatus<Acc>* s, u32 epoch, bool head, Acc v) {
    s->has_head = head ? 1u : 0u;
    s->agg = v;
    __threadfence();
    st_store_release(&s->flag, ((epoch & EPOCH_MASK) << 2) | ST_AGG);
}
template <typename Acc>
__device__ __forceinline__ void seg_publish_prefix(SegStatus<Acc>* s, u32 epoch, Acc v) {
    s->incl = v;
    __threadfence();
    st_store_release(&s->flag, ((epoch & EPOCH_MASK) << 2) | ST_PREFIX);
}
template <typename Acc>
__device__ __forceinline__ Acc shfl_xor_acc(Acc v, int o) {
    if constexpr (sizeof(Acc) == 8) {
        unsigned long long bits = *reinterpret_cast<unsigned long long*>(&v);
        bits = __shfl_xor_sync(0xffffffffu, bits, o);
        return *reinterpret_cast<Acc*>(&bits);
    } else {
        u32 bits = *reinterpret_cast<u32*>(&v);
        bits = __shfl_xor_sync(0xffffffffu, bits, o);
        return *reinterpret_cast<Acc*>(&bits);
    }
}
template <typename Acc>
__device__ __forceinline__ Acc shfl_up_acc(Acc v, int o) {
    if constexpr (sizeof(Acc) == 8) {
        unsigned long long bits = *reinterpret_cast<unsigned long long*>(&v);
        bits = __shfl_up_sync(0xffffffffu, bits, o);
        return *reinterpret_cast<Acc*>(&bits);
    } else {
        u32 bits = *reinterpret_cast<u32*>(&v);
        bits = __shfl_up_sync(0xffffffffu, bits, o);
        return *reinterpret_cast<Acc*>(&bits);
    }
}
template <typename Acc>
__device__ __forceinline__ Acc volatile_read(const Acc* p) {
    Acc v;
    if constexpr (sizeof(Acc) == 8) {
        unsigned long long bits = *reinterpret_cast<const volatile unsigned long long*>(p);
        v = *reinterpret_cast<Acc*>(&bits);
    } else {
        u32 bits = *reinterpret_cast<const volatile u32*>(p);
        v = *reinterpret_cast<Acc*>(&bits);
    }
    return v;
}

// Tile summary of the segmented scan: whether a segment starts inside the
// tile, and F over the tile's records after its last start.
template <typename Acc>
struct TileAgg {
    u32 hd;
    Acc agg;
};

// Segmented scan of F over the sorted records of every instance (Definition
// "Segmented scan", Sec. 2.2): a segment is a maximal run of equal node keys
// (the role bit ignored).  Data records contribute their weight, query
// records the unit e (Sec. 2.1).  Because queries precede data on a tie of
// the last coordinate, the running value at a query record is F over exactly
// the data of its node with a smaller last coordinate; it is stored in the
// query record's partial slot.
//
// Reduce, then scan: the kernel runs twice over the same tiles of 4096
// records.  With APPLY = false each tile writes its summary (TileAgg);
// k_seg_carry scans the summaries of all tiles in one block; with APPLY =
// true each tile reads the carry from the tiles before it and writes the
// query records' partials.  No tile waits on another (a decoupled look-back
// made long segments wait on their predecessors' prefixes); the price is a
// second read of the records.
template <class Op, typename K, int THREADS, int ITEMS, bool APPLY>
__global__ __launch_bounds__(THREADS) void k_segscan(const K* __restrict__ keys0, const K* __restrict__ keys1,
                                                     const typename Op::Pay* __restrict__ pays0,
                                                     const typename Op::Pay* __restrict__ pays1,
                                                     const u32* __restrict__ seg_off,
                                                     const u32* __restrict__ tile_off, int nseg,
                                                     const u32* __restrict__ seg_bits,
                                                     const typename Op::W* __restrict__ wgt,
                                                     typename Op::Part* __restrict__ partial, u32 n_partial,
                                                     TileAgg<typename Op::Acc>* __restrict__ tagg,
                                                     const typename Op::Acc* __restrict__ carry) {
    typedef typename Op::Acc Acc;
    typedef typename Op::Pay Pay;
    constexpr int TILE = THREADS * ITEMS, WARPS = THREADS / 32;
    const K role = K(1) << (sizeof(K) * 8 - 1);
    __shared__ K s_keys[Padded<TILE>::value];
    __shared__ Pay s_pays[Padded<TILE>::value];
    __shared__ Acc s_wacc[WARPS];
    __shared__ u32 s_whead[WARPS];
    const u32 t = blockIdx.x;
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    // the sort left this segment in the buffer of its pass count's parity
    const bool odd = ((__ldg(seg_bits + L.seg) + RADIX_BITS - 1) / RADIX_BITS) & 1u;
    const K* __restrict__ keys = odd ? keys1 : keys0;
    const typename Op::Pay* __restrict__ pays = odd ? pays1 : pays0;
    // coalesced loads, all in flight together, then into shared memory
    {
        constexpr int HALF = ITEMS / 2;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            K kv[HALF];
            Pay pv[HALF];
#pragma unroll
            for (int i = 0; i < HALF; ++i) {
                const u32 x = (u32)(h2 * HALF + i) * THREADS + threadIdx.x;
                const bool in = L.start + x < L.end;
                kv[i] = in ? keys[L.start + x] : K(0);
                pv[i] = in ? pays[L.start + x] : Pay(0);
            }
#pragma unroll
            for (int i = 0; i < HALF; ++i) {
                const u32 x = (u32)(h2 * HALF + i) * THREADS + threadIdx.x;
                s_keys[pidx(x)] = kv[i];
                s_pays[pidx(x)] = pv[i];
            }
        }
    }
    __syncthreads();
    const u32 lx0 = threadIdx.x * ITEMS;  // tile-local index of my first item
    const u32 x0 = L.start + lx0;
    K prev = 0;
    bool has_prev = x0 > L.seg_begin;
    if (has_prev && x0 < L.end) prev = lx0 == 0 ? keys[x0 - 1] : s_keys[pidx(lx0 - 1)];
    prev &= ~role;
    // thread aggregate: (head seen, F over items after the last head)
    bool head_any = false;
    Acc agg = Op::e();
    u32 headmask = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (x0 + i < L.end) {
            const K kx = s_keys[pidx(lx0 + i)];
            const K kn = kx & ~role;
            const bool head = !has_prev || kn != prev;
            has_prev = true;
            prev = kn;
            if (head) {
                head_any = true;
                headmask |= 1u << i;
                agg = Op::e();
            }
            if (!(kx & role)) {
                const Pay py = s_pays[pidx(lx0 + i)];
                if constexpr (Op::GATHER) agg = Op::Fc(agg, Op::from_w(__ldg(wgt + py)));
                else agg = Op::Fc(agg, Op::from_pay(py));
            }
        }
    }
    // block-wide scan of (head, agg) with the segmented operator
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool ihead = head_any;
    Acc iacc = agg;  // inclusive within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int nh = __shfl_up_sync(0xffffffffu, (int)ihead, o);
        const Acc na = shfl_up_acc(iacc, o);
        if (lane >= o) {
            if (!ihead) iacc = Op::F(na, iacc);
            ihead = ihead || nh;
        }
    }
    if (lane == 31) {
        s_wacc[warp] = iacc;
        s_whead[warp] = ihead ? 1u : 0u;
    }
    __syncthreads();
    if constexpr (!APPLY) {
        // the tile's summary
        if (threadIdx.x == 0) {
            Acc ta = Op::e();
            bool th = false;
            for (int w = 0; w < WARPS; ++w) {
                if (s_whead[w]) {
                    ta = s_wacc[w];
                    th = true;
                } else {
                    ta = Op::F(ta, s_wacc[w]);
                }
            }
            tagg[t].hd = th ? 1u : 0u;
            tagg[t].agg = ta;
        }
        return;
    } else {
        // exclusive prefix of this thread within the tile
        Acc wex = Op::e();  // prefix from earlier warps
        bool wex_head = false;
        for (int w = 0; w < warp; ++w) {
            if (s_whead[w]) {
                wex = s_wacc[w];
                wex_head = true;
            } else {
                wex = Op::F(wex, s_wacc[w]);
            }
        }
        Acc lex = shfl_up_acc(iacc, 1);
        int lhead = __shfl_up_sync(0xffffffffu, (int)ihead, 1);
        if (lane == 0) {
            lex = Op::e();
            lhead = 0;
        }
        const Acc texcl = lhead ? lex : Op::F(wex, lex);  // within-tile exclusive prefix
        const bool texcl_head = lhead || wex_head;        // a head occurs before me in the tile
        // a thread before the tile's first head continues the segment coming
        // from the tiles before (their carry)
        Acc run = texcl_head ? texcl : Op::F(carry[t], texcl);
        // output walk: the running value at every query record
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (x0 + i < L.end) {
                if ((headmask >> i) & 1u) run = Op::e();
                const K kx = s_keys[pidx(lx0 + i)];
                const Pay py = s_pays[pidx(lx0 + i)];
                if (kx & role) {
                    if (domagg_check((u32)py < n_partial, SITE_SEGSCAN_PARTIAL)) partial[py] = Op::to_part(run);
                } else {
                    if constexpr (Op::GATHER) run = Op::Fc(run, Op::from_w(__ldg(wgt + py)));
                    else run = Op::Fc(run, Op::from_pay(py));
                }
            }
        }
    }
}

// Carries of the segmented scan: for every tile (over all segments, in
// order), F over the records of its segment in the tiles before it, from the
// tiles' summaries.  One block; each thread scans a run of consecutive tiles,
// then a block scan joins the runs.  A segment's first tile holds a head (its
// first record), so carries never cross segments.
template <class Op>
__global__ __launch_bounds__(1024) void k_seg_carry(const u32* __restrict__ tile_off, int nseg,
                                                    const TileAgg<typename Op::Acc>* __restrict__ tagg,
                                                    typename Op::Acc* __restrict__ carry) {
    typedef typename Op::Acc Acc;
    __shared__ Acc s_wacc[32];
    __shared__ u32 s_whead[32];
    const u32 n = __ldg(tile_off + nseg);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const u32 per = (n + blockDim.x - 1) / blockDim.x;
    const u32 a = min(n, (u32)tid * per), b = min(n, a + per);
    bool hd = false;
    Acc acc = Op::e();
    for (u32 t0 = a; t0 < b; t0 += 8) {  // eight summaries in flight
        TileAgg<Acc> g[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = t0 + j < b ? tagg[t0 + j] : TileAgg<Acc>{0u, Op::e()};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (g[j].hd) {
                acc = g[j].agg;
                hd = true;
            } else {
                acc = Op::F(acc, g[j].agg);
            }
        }
    }
    bool ihead = hd;
    Acc iacc = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int nh = __shfl_up_sync(0xffffffffu, (int)ihead, o);
        const Acc na = shfl_up_acc(iacc, o);
        if (lane >= o) {
            if (!ihead) iacc = Op::F(na, iacc);
            ihead = ihead || nh;
        }
    }
    if (lane == 31) {
        s_wacc[warp] = iacc;
        s_whead[warp] = ihead ? 1u : 0u;
    }
    __syncthreads();
    Acc wex = Op::e();
    for (int w = 0; w < warp; ++w) wex = s_whead[w] ? s_wacc[w] : Op::F(wex, s_wacc[w]);
    Acc lex = shfl_up_acc(iacc, 1);
    int lhead = __shfl_up_sync(0xffffffffu, (int)ihead, 1);
    if (lane == 0) {
        lex = Op::e();
        lhead = 0;
    }
    Acc run = lhead ? lex : Op::F(wex, lex);
    for (u32 t0 = a; t0 < b; t0 += 8) {
        TileAgg<Acc> g[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) g[j] = t0 + j < b ? tagg[t0 + j] : TileAgg<Acc>{0u, Op::e()};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (t0 + j < b) carry[t0 + j] = run;
            run = g[j].hd ? g[j].agg : Op::F(run, g[j].agg);
        }
    }
}

// The same segmented scan in one pass, each tile taking its carry by a
// decoupled look-back over the tiles before it (warp-cooperative: lane l
// examines tile u-1-l).  Used where segments are short (m >= 3: node keys of
// two ranks), so look-back chains stop within a few tiles and one read of
// the records suffices; long segments (m <= 2) use k_segscan, whose
// reduce-then-scan does not wait on chains and combines float sums in a
// fixed order.
template <class Op, typename K, int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS) void k_segscan_lb(const K* __restrict__ keys0, const K* __restrict__ keys1,
                                                     const typename Op::Pay* __restrict__ pays0,
                                                     const typename Op::Pay* __restrict__ pays1,
                                                     const u32* __restrict__ seg_off,
                                                     const u32* __restrict__ tile_off, int nseg,
                                                     const u32* __restrict__ seg_bits,
                                                     const typename Op::W* __restrict__ wgt,
                                                     typename Op::Part* __restrict__ partial, u32 n_partial,
                                                     SegStatus<typename Op::Acc>* status, Ctl* ctl, int launch_idx) {
    typedef typename Op::Acc Acc;
    typedef typename Op::Pay Pay;
    constexpr int TILE = THREADS * ITEMS, WARPS = THREADS / 32;
    const K role = K(1) << (sizeof(K) * 8 - 1);
    __shared__ K s_keys[Padded<TILE>::value];
    __shared__ Pay s_pays[Padded<TILE>::value];
    __shared__ Acc s_wacc[WARPS];
    __shared__ u32 s_whead[WARPS];
    __shared__ Acc s_excl;
    __shared__ u32 s_info[2];
    if (threadIdx.x == 0) {
        s_info[0] = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        s_info[1] = ctl->epoch_base + (u32)launch_idx;
    }
    __syncthreads();
    const u32 t = s_info[0], epoch = s_info[1];
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    // the sort left this segment in the buffer of its pass count's parity
    const bool odd = ((__ldg(seg_bits + L.seg) + RADIX_BITS - 1) / RADIX_BITS) & 1u;
    const K* __restrict__ keys = odd ? keys1 : keys0;
    const typename Op::Pay* __restrict__ pays = odd ? pays1 : pays0;
    // coalesced load into shared memory, then blocked reads
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = (u32)i * THREADS + threadIdx.x;
        if (L.start + x < L.end) {
            s_keys[pidx(x)] = keys[L.start + x];
            s_pays[pidx(x)] = pays[L.start + x];
        }
    }
    __syncthreads();
    const u32 lx0 = threadIdx.x * ITEMS;  // tile-local index of my first item
    const u32 x0 = L.start + lx0;
    K prev = 0;
    bool has_prev = x0 > L.seg_begin;
    if (has_prev && x0 < L.end) prev = lx0 == 0 ? keys[x0 - 1] : s_keys[pidx(lx0 - 1)];
    prev &= ~role;
    // thread aggregate: (head seen, F over items after the last head); the
    // running value at every query record is kept for the output pass
    bool head_any = false;
    Acc agg = Op::e();
    u32 headmask = 0, qmask = 0;
    Acc loc[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        loc[i] = Op::e();
        if (x0 + i < L.end) {
            const K kx = s_keys[pidx(lx0 + i)];
            const K kn = kx & ~role;
            const bool head = !has_prev || kn != prev;
            has_prev = true;
            prev = kn;
            if (head) {
                head_any = true;
                headmask |= 1u << i;
                agg = Op::e();
            }
            if (kx & role) {
                qmask |= 1u << i;
                loc[i] = agg;
            } else {
                const Pay py = s_pays[pidx(lx0 + i)];
                if constexpr (Op::GATHER) agg = Op::F(agg, Op::from_w(__ldg(wgt + py)));
                else agg = Op::F(agg, Op::from_pay(py));
            }
        }
    }
    // block-wide exclusive scan of (head, agg) with the segmented operator
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool ihead = head_any;
    Acc iacc = agg;  // inclusive within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int nh = __shfl_up_sync(0xffffffffu, (int)ihead, o);
        Acc na;
        if constexpr (sizeof(Acc) == 8) {
            unsigned long long bits = *reinterpret_cast<unsigned long long*>(&iacc);
            bits = __shfl_up_sync(0xffffffffu, bits, o);
            na = *reinterpret_cast<Acc*>(&bits);
        } else {
            u32 bits = *reinterpret_cast<u32*>(&iacc);
            bits = __shfl_up_sync(0xffffffffu, bits, o);
            na = *reinterpret_cast<Acc*>(&bits);
        }
        if (lane >= o) {
            if (!ihead) iacc = Op::F(na, iacc);
            ihead = ihead || nh;
        }
    }
    if (lane == 31) {
        s_wacc[warp] = iacc;
        s_whead[warp] = ihead ? 1u : 0u;
    }
    __syncthreads();
    // exclusive prefix of this thread within the tile
    Acc wex = Op::e();  // prefix from earlier warps
    bool wex_head = false;
    for (int w = 0; w < warp; ++w) {
        if (s_whead[w]) {
            wex = s_wacc[w];
            wex_head = true;
        } else {
            wex = Op::F(wex, s_wacc[w]);
        }
    }
    // exclusive within warp: inclusive of lane-1
    Acc lex;
    int lhead;
    {
        Acc src = iacc;
        if constexpr (sizeof(Acc) == 8) {
            unsigned long long bits = *reinterpret_cast<unsigned long long*>(&src);
            bits = __shfl_up_sync(0xffffffffu, bits, 1);
            lex = *reinterpret_cast<Acc*>(&bits);
        } else {
            u32 bits = *reinterpret_cast<u32*>(&src);
            bits = __shfl_up_sync(0xffffffffu, bits, 1);
            lex = *reinterpret_cast<Acc*>(&bits);
        }
        lhead = __shfl_up_sync(0xffffffffu, (int)ihead, 1);
        if (lane == 0) {
            lex = Op::e();
            lhead = 0;
        }
    }
    Acc texcl = lhead ? lex : Op::F(wex, lex);  // within-tile exclusive prefix
    const bool texcl_head = lhead || wex_head;  // a head occurs before me in the tile
    // tile aggregate, look-back and publication (warp 0).  The look-back is
    // warp-cooperative: lane l examines tile u-1-l, so one round trip to L2
    // covers 32 predecessors; the aggregates up to the first tile that ends
    // the chain (a published prefix, or a segment head inside the tile) are
    // combined with a masked warp reduction.
    if (warp == 0) {
        Acc tagg = Op::e();
        bool thead = false;
        for (int w = 0; w < WARPS; ++w) {
            if (s_whead[w]) {
                tagg = s_wacc[w];
                thead = true;
            } else {
                tagg = Op::F(tagg, s_wacc[w]);
            }
        }
        SegStatus<Acc>* my = status + t;
        const bool starts_fresh = L.first || (__shfl_sync(0xffffffffu, headmask, 0) & 1u);
        Acc excl = Op::e();
        if (starts_fresh) {
            if (lane == 0) seg_publish_prefix(my, epoch, tagg);
        } else {
            if (lane == 0) seg_publish_agg(my, epoch, thead, tagg);
            const u32 first_tile = t - (L.start - L.seg_begin) / (u32)TILE;
            u32 u = t;  // tiles [u, t) have been combined into excl
            u32 spins = 0;
            while (u > first_tile) {
                const bool exists = u - 1 - (u32)lane >= first_tile && (u32)lane < u - first_tile;
                u32 f = 0, hh = 0;
                Acc v = Op::e();
                bool ready = true, term = false;
                if (exists) {
                    const SegStatus<Acc>* ps = status + (u - 1 - lane);
                    f = st_load_acquire(&ps->flag);
                    ready = (f >> 2) == (epoch & EPOCH_MASK) && (f & 3u);
                    if (ready) {
                        if ((f & 3u) == ST_PREFIX) {
                            v = volatile_read(&ps->incl);
                            term = true;
                        } else {
                            hh = *reinterpret_cast<const volatile u32*>(&ps->has_head);
                            v = volatile_read(&ps->agg);
                            term = hh != 0;
                        }
                    }
                } else {
                    ready = false;  // beyond the chain start: never consumed
                }
                const u32 nr = __ballot_sync(0xffffffffu, !ready);
                const u32 tm = __ballot_sync(0xffffffffu, term);
                const int k_nr = nr ? __ffs(nr) - 1 : 32;
                const int k_tm = tm ? __ffs(tm) - 1 : 32;
                const bool finish = k_tm < k_nr;
                const int take = finish ? k_tm + 1 : k_nr;  // lanes [0, take) are combined
                if (take > 0) {
                    Acc r = lane < take ? v : Op::e();
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) r = Op::F(r, shfl_xor_acc(r, o));
                    excl = Op::F(r, excl);
                    u -= (u32)take;
                }
                if (finish) break;
                if (take == 0) {
                    if (++spins > SPIN_LIMIT || ((spins & 255u) == 0 && timed_out(ctl))) {
                        if (lane == 0) {
                            atomicOr(&ctl->error, ERR_TIMEOUT);
                            ctl->timeout_where = 4u;
                        }
                        break;
                    }
                    if (spins > 64) __nanosleep(256);
                }
            }
            if (lane == 0) seg_publish_prefix(my, epoch, thead ? tagg : Op::F(excl, tagg));
        }
        if (lane == 0) s_excl = excl;
    }
    __syncthreads();
    // output: a query record before the thread's first head continues the
    // segment coming from the left (prefix); after it, its own run suffices
    const Acc prefix = texcl_head ? texcl : Op::F(s_excl, texcl);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (qmask & (1u << i)) {
            const u64 slot = (u64)s_pays[pidx(lx0 + i)];
            const bool own = (headmask & ((2u << i) - 1u)) != 0;
            if (domagg_check(slot < n_partial, SITE_SEGSCAN_PARTIAL)) partial[slot] = Op::to_part(own ? loc[i] : Op::F(prefix, loc[i]));
        }
    }
}

// a[0 .. n) = e: a shard's group parts start at the unit (k_group writes
// only its own groups' queries).
template <class Op>
__global__ void k_fill_e(typename Op::Part* __restrict__ a, u32 n) {
    const u32 g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) a[g] = Op::to_part(Op::e());
}

// out[q] = F over the shards' partial outputs (float32 sums: the shards'
// float-float pairs added in float-float, rounded once).
constexpr int MAX_SHARDS = 64;
struct ShardParts {
    const void* part[MAX_SHARDS];
    const float* lo[MAX_SHARDS];
};
template <class Op>
__global__ void k_combine(int nparts, const ShardParts parts, u32 nQ, void* __restrict__ out) {
    const u32 q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nQ) return;
    typename Op::Acc acc = Op::e();
    for (int s = 0; s < nparts; ++s) {
        typename Op::Acc v = Op::from_out(reinterpret_cast<const typename Op::Out*>(parts.part[s])[q]);
        if constexpr (std::is_same<Op, OpSumF32>::value)
            if (parts.lo[s]) v.lo = parts.lo[s][q];
        acc = Op::F(acc, v);
    }
    reinterpret_cast<typename Op::Out*>(out)[q] = Op::to_out(acc);
}

// Per-query reduction: out[q] = F over the query's partial results.  This
// replaces the sort by ID and the ID-segmented scan of instructions 6m+4,
// 6m+5 (the broadcast of 6m+6 .. 6m+9 is not needed for one output per
// query).  The partials of level lv are a dense range in which queries keep
// the order of the last coordinate, so a warp walking one chunk of 32
// consecutive points reads every level's partials as one contiguous run:
// the chunk's query base of the level plus the query lanes before it.
template <class Op, int M>
__global__ __launch_bounds__(256) void k_reduce(const u32* __restrict__ chunk_off, int k, int k0, int k1,
                                                const u32* __restrict__ pt_offs, const u32* __restrict__ pr0,
                                                const u32* __restrict__ pr1, const u32* __restrict__ pr2,
                                                const u32* __restrict__ pj,
                                                const u32* __restrict__ qchunk_base,
                                                const u32* __restrict__ pt_tiles, const u32* __restrict__ tile_excl,
                                                const u32* __restrict__ qseg_base /*[k1-k0][LMAX]*/,
                                                const Inst* __restrict__ inst,
                                                const typename Op::Part* __restrict__ partial, u32 n_partial,
                                                const typename Op::Part* __restrict__ gacc,
                                                const unsigned char* __restrict__ govf) {
    typedef typename Op::Part Part;
    __shared__ u32 s_mask[8][LMAX];  // per warp: query lanes holding a record of level lv
    __shared__ u32 s_base[8][LMAX];  // per warp: first partial slot of level lv in this chunk
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 lt = lanemask_lt();
    const u32 c_begin = __ldg(chunk_off + k0), c_end = __ldg(chunk_off + k1);
    const u32 warps = (gridDim.x * blockDim.x) >> 5;
    for (u32 c = c_begin + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < c_end; c += warps) {
        const int s = upper_index(chunk_off, k + 1, c);
        const Inst& I = inst[s];
        const u32 ps = __ldg(pt_offs + s), pe = __ldg(pt_offs + s + 1);
        const u32 p = ps + (c - __ldg(chunk_off + s)) * 32u + (u32)lane;
        const bool valid = p < pe;
        const u32 nQ = I.nQ;
        const u32 nlev = levels_of<M>(I);
        u32 local = 0, bits0 = 0, bits1 = 0, c1 = 1;
        bool q = false;
        if (valid) {
            u32 j = pj[p];
            if (j - ps >= pe - ps) j = ps;  // never taken for a valid permutation
            local = j - ps;
            q = local < nQ;
            if (q) {
                if (M >= 2) bits0 = pr0[p] & low_mask(I.b[0]);
                if (M >= 2) bits0 &= hbm_levels(I, pr0[p] & ~QUERY_BIT, govf);  // (the group kernels took the others)
                if (M >= 3) {
                    bits1 = pr1[p] & low_mask(I.b[1]);
                    c1 = (u32)__popc(bits1);
                }
                if (M >= 4) c1 *= (u32)__popc(pr2[p] & low_mask(I.b[2]));
                if (M == 1) bits0 = 1u & I.lvmask;
                if (M >= 3 && c1 == 0) bits0 = 0;
            }
        }
        if (__ballot_sync(0xffffffffu, q) == 0u) continue;
        // per level: which lanes have a record there, and the level's base
        if ((u32)lane < nlev)
            s_base[warp][lane] = __ldg(qseg_base + (u64)(s - k0) * LMAX + lane) +
                                 __ldg(qchunk_base + (u64)c * LMAX + lane) +
                                 __ldg(tile_excl + (u64)(__ldg(pt_tiles + s) + (c - __ldg(chunk_off + s)) / CS_CHUNKS) *
                                                       CS_COUNTERS + LMAX + lane);
        s_mask[warp][lane] = warp_transpose32(bits0, (u32)lane);  // lanes of level `lane`
        __syncwarp();
        typename Op::Acc acc = Op::e();
        // m = 2, 3 with groups: F over the levels below gS, by position
        if ((M == 2 || M == 3) && q && I.gS) acc = Op::from_part(gacc[p]);
        if (M <= 2) {
            // one partial per query and level, at the level's base plus the
            // query lanes of that level before this one; each lane walks only
            // its own levels (unrolled so the loads run ahead of the adds)
            u32 rem = bits0;
#pragma unroll 4
            while (rem) {
                const u32 lv = __ffs(rem) - 1;
                rem &= rem - 1;
                const u32 slot = s_base[warp][lv] + (u32)__popc(s_mask[warp][lv] & lt);
                if (domagg_check(slot < n_partial, SITE_REDUCE)) acc = Op::F(acc, Op::from_part(partial[slot]));
            }
        }
        if (M >= 3) {
            // m >= 3: exclusive sums of the records per point (c1) over the
            // lanes of each level (warp-uniform loop)
            for (u32 lv = 0; lv < nlev; ++lv) {
                const bool has = (bits0 >> lv) & 1u;
                if (s_mask[warp][lv] == 0u) continue;
                const u32 wq = has ? c1 : 0u;
                u32 inc = wq;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 nn = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += nn;
                }
                if (has) {
                    const u32 base = s_base[warp][lv] + inc - wq;
                    for (u32 kk = 0; kk < c1 && base + kk < n_partial; ++kk)
                        acc = Op::F(acc, Op::from_part(partial[base + kk]));
                }
            }
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
