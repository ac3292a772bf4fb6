// k_points.cuh -- kernels of the point phase: coordinate keys, dense ranks,
// the count / offset scan of the flat map and the flat map itself.
#pragma once
#include "dev_common.cuh"
#include "k_radix.cuh"

namespace domagg {

// Pipeline start: advance the look-back epoch and clear the tile counters.
static __global__ void k_begin(Ctl* ctl) {
    if (threadIdx.x == 0) {
        if (ctl->epoch_base > EPOCH_MASK - 4u * MAX_LAUNCHES) atomicOr(&ctl->error, ERR_EPOCH);
        ctl->epoch_base += MAX_LAUNCHES;
        ctl->T_total = 0;
        ctl->Tq_total = 0;
        ctl->max_key_bits = 0;
    }
    for (int i = threadIdx.x; i < MAX_LAUNCHES; i += blockDim.x) ctl->tile_ctr[i] = 0;
}

// Epoch guard of a replayed plan (no host in the loop to reset the epochs):
// once the epoch counter comes within `margin` of its limit, the status words
// are cleared and the counter restarts at 0 (two launches, stream-ordered).
static __global__ void k_epoch_clear(const Ctl* ctl, u64* a, u64 na, u64* b, u64 nb, u32 margin) {
    if (*reinterpret_cast<const volatile u32*>(&ctl->epoch_base) <= EPOCH_MASK - margin) return;
    const u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < na; i += stride) a[i] = 0;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) b[i] = 0;
}
static __global__ void k_epoch_restart(Ctl* ctl, u32 margin) {
    if (threadIdx.x == 0 && ctl->epoch_base > EPOCH_MASK - margin) ctl->epoch_base = 0;
}

// Self-test of the wait limits: one thread waits on something that never
// happens -- which = 0: a look-back on a predecessor status that nothing
// publishes (epoch EPOCH_MASK, which no pipeline run uses); which = 1: an
// mbarrier phase whose expected bytes are never sent (no copy is issued, so
// nothing is in flight when the kernel returns).  Both give up, record
// ERR_TIMEOUT and return.
static __global__ void k_selftest_wait(int which, const u64* status, Ctl* ctl) {
    __shared__ u64 bar;
    if (threadIdx.x != 0) return;
    if (which == 0) {
        (void)lookback_u32(status, 1, 0, 1u, 0u, EPOCH_MASK, ctl, 7u);
    } else {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, 16u);
        (void)mbar_wait_bounded(&bar, 0u, ctl, 8u);
    }
}

// Tiles of size `tile` over segments: tile_off[s] = sum over s' < s of
// ceil(len(s') / tile), tile_off[nseg] = total.  One block.
// With seg_bits, segments whose keys have at most `skip_upto` bits get no
// tiles (a radix pass starting at that bit leaves them where they are).
static __global__ void k_make_tiles(const u32* __restrict__ seg_off, int nseg, u32 tile, u32* __restrict__ tile_off,
                                    const u32* __restrict__ seg_bits = nullptr, u32 skip_upto = 0) {
    __shared__ u32 carry;
    __shared__ u32 warp_sum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < nseg; base += blockDim.x) {
        const int s = base + threadIdx.x;
        u32 v = 0;
        if (s < nseg && !(seg_bits && __ldg(seg_bits + s) <= skip_upto))
            v = (__ldg(seg_off + s + 1) - __ldg(seg_off + s) + tile - 1) / tile;
        u32 inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            u32 n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        if (lane == 31) warp_sum[warp] = inc;
        __syncthreads();
        u32 add = carry;
        for (int w = 0; w < warp; ++w) add += warp_sum[w];
        if (s < nseg) tile_off[s] = add + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) {
            u32 tot = 0;
            for (int w = 0; w < nw; ++w) tot += warp_sum[w];
            carry += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_off[nseg] = carry;
}

// Order-preserving 32-bit keys (Sec. 4, instructions 5i-4: S_i = the i-th
// coordinate of every point).  int32: flip the sign bit.  float32: -0 -> +0,
// then flip all bits of negatives and the sign bit of positives.  With
// `negate` the key is complemented, which reverses the order (the backward
// pass aggregates over dominating points).  NaN sets ERR_NAN.
template <bool F32>
__device__ __forceinline__ u32 coord_key(const void* base, u32 row, int m, int i, bool negate, bool& nan) {
    u32 k;
    if (F32) {
        float f = reinterpret_cast<const float*>(base)[(u64)row * m + i];
        if (f != f) nan = true;
        u32 u = __float_as_uint(f);
        if ((u & 0x7fffffffu) == 0u) u = 0u;
        k = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    } else {
        k = (u32)reinterpret_cast<const int*>(base)[(u64)row * m + i] ^ 0x80000000u;
    }
    return negate ? ~k : k;
}

// Keys of every point of every instance.  Point p of instance s has local
// index p - pt_off; queries come first, then data (see Inst).
template <int M, bool F32>
__global__ void k_encode(const Inst* __restrict__ inst, const u32* __restrict__ pt_offs, int k, u32 N,
                         u32* __restrict__ rk0, u32* __restrict__ rk1, u32* __restrict__ rk2, u32* __restrict__ lk,
                         int negate, Ctl* ctl) {
    const u32 p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int s = upper_index(pt_offs, k + 1, p);
    const u32 local = p - __ldg(pt_offs + s);
    const u32 nQ = inst[s].nQ;
    const void* base = local < nQ ? inst[s].qco : inst[s].dco;
    const u32 row = local < nQ ? local : local - nQ;
    bool nan = false;
    const u32 flags = inst[s].flags;
    const bool virt = (flags & FLAG_VIRTUAL_LAST) != 0u;
    const int stride = virt ? M - 1 : M;  // stored coordinates per point
    if (M >= 2) rk0[p] = coord_key<F32>(base, row, stride, 0, negate, nan);
    if (M >= 3) rk1[p] = coord_key<F32>(base, row, stride, 1, negate, nan);
    if (M >= 4) rk2[p] = coord_key<F32>(base, row, stride, 2, negate, nan);
    u32 key = virt ? 0u : coord_key<F32>(base, row, stride, M - 1, negate, nan);
    // a non-strict last coordinate is sorted descending and read back in
    // reverse, which puts data before queries on ties
    if ((flags >> (M - 1)) & 1u) key = ~key;
    lk[p] = key;
    if (nan) atomicOr(&ctl->error, ERR_NAN);
}

// Loads a tile of u32 [start, end) in blocked order (thread t gets items
// t*ITEMS .. t*ITEMS+ITEMS-1) through shared memory, coalesced.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void load_blocked_u32(const u32* __restrict__ src, u32 start, u32 end, u32* sbuf,
                                                 u32 (&out)[ITEMS], u32 fill) {
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = (u32)i * THREADS + threadIdx.x;
        sbuf[pidx(x)] = (start + x < end) ? src[start + x] : fill;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) out[i] = sbuf[pidx(threadIdx.x * ITEMS + i)];
    __syncthreads();
}

// Block-wide exclusive scan of C counters per thread; returns the tile totals
// in `tot`.  `scratch` holds (THREADS/32)*C u32.
template <int THREADS, int C>
__device__ __forceinline__ void block_exscan(u32 (&v)[C], u32 (&tot)[C], u32* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int WARPS = THREADS / 32;
    u32 inc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        inc[c] = v[c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u32 n = __shfl_up_sync(0xffffffffu, inc[c], o);
            if (lane >= o) inc[c] += n;
        }
        if (lane == 31) scratch[c * WARPS + warp] = inc[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
        u32 add = 0, all = 0;
        for (int w = 0; w < WARPS; ++w) {
            const u32 x = scratch[c * WARPS + w];
            if (w < warp) add += x;
            all += x;
        }
        v[c] = add + inc[c] - v[c];
        tot[c] = all;
    }
    __syncthreads();
}

// Dense ranks (Sec. 4, instructions 5i-2 .. 5i and 5m+i): over the keys
// sorted per instance, flag every key that differs from its predecessor,
// scan the flags, and scatter rank = (flags up to here) - 1 to the point's
// own slot.  U = number of distinct keys; b = ceil(log2 U) digits.  For a
// coordinate compared non-strictly the rank is 2r for data and 2r + 1 for
// queries (U doubles), so that d_i <= q_i  <=>  rank(d) < rank(q).
//
// Computed in three launches without a look-back chain (one instance is a
// single chain of thousands of tiles, whose decoupled look-back walks were
// the cost): (1) per tile, the number of keys that differ from their
// predecessor; (2) per instance, the exclusive scan of those counts over its
// tiles (one warp per instance); (3) k_rank_apply: flags again, a block scan
// plus the tile's prefix, and the scatter by index.  The scatter writes
// 4 bytes at random; it runs in windows of destination indices [win_lo,
// win_hi) small enough for the 129 MB L2 to hold while its sectors fill
// (one launch per window; the first also writes rstart and U, b).
template <int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS) void k_rank_count(const u32* __restrict__ skeys, const u32* __restrict__ seg_off,
                                                        const u32* __restrict__ tile_off, int nseg,
                                                        u32* __restrict__ tile_cnt) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ u32 warp_sum[THREADS / 32];
    const u32 t = blockIdx.x;
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    u32 c = 0;
#pragma unroll 4
    for (int i = 0; i < ITEMS; ++i) {  // striped: coalesced, the predecessor from the same lines
        const u32 x = L.start + (u32)i * THREADS + threadIdx.x;
        if (x < L.end) c += (x == L.seg_begin || __ldg(skeys + x) != __ldg(skeys + x - 1)) ? 1u : 0u;
    }
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 tot = 0;
        for (int w = 0; w < THREADS / 32; ++w) tot += warp_sum[w];
        tile_cnt[t] = tot;
    }
}

// Exclusive scan, in place, of the column c[0], c[stride], ... c[(n-1)*stride]
// by one warp: 8 consecutive entries per lane per round (their loads in
// flight together), 256 per round.  Returns the total (64 bits).
__device__ __forceinline__ u64 warp_exscan_column(u32* __restrict__ c, u64 stride, u32 n, int lane) {
    u64 carry = 0;
    for (u32 base = 0; base < n; base += 256) {
        u32 v[8];
        const u32 x0 = base + (u32)lane * 8u;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = x0 + i < n ? c[(u64)(x0 + i) * stride] : 0u;
        u32 sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) sum += v[i];
        u32 inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const u32 nb = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += nb;
        }
        u64 run = carry + (inc - sum);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (x0 + i < n) c[(u64)(x0 + i) * stride] = (u32)run;
            run += v[i];
        }
        carry += __shfl_sync(0xffffffffu, inc, 31);  // 256 tiles hold < 2^32
    }
    return carry;
}

// Exclusive scan of per-tile counts within every segment (in place), one
// block per segment: its 32 warps scan 32 consecutive slices of the tiles,
// then add the slices before them.
static __global__ __launch_bounds__(1024) void k_tile_exscan(const u32* __restrict__ tile_off, int nseg,
                                                            u32* __restrict__ cnt) {
    __shared__ u64 s_sum[32];
    const int seg = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (seg >= nseg) return;
    const u32 t0 = __ldg(tile_off + seg), n = __ldg(tile_off + seg + 1) - t0, per = (n + 31) / 32;
    const u32 a = min(n, (u32)warp * per), b = min(n, (u32)(warp + 1) * per);
    const u64 tot = warp_exscan_column(cnt + t0 + a, 1, b - a, lane);
    if (lane == 0) s_sum[warp] = tot;
    __syncthreads();
    u64 off = 0;
    for (int w = 0; w < warp; ++w) off += s_sum[w];
    for (u32 t = a + (u32)lane; t < b; t += 32) cnt[t0 + t] += (u32)off;
}

template <int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS, 4) void k_rank_apply(const u32* __restrict__ skeys, const u32* __restrict__ sidx,
                                                        const u32* __restrict__ seg_off,
                                                        const u32* __restrict__ tile_off, int nseg,
                                                        const u32* __restrict__ tile_excl, u32* __restrict__ rank_out,
                                                        Inst* inst, int dim, u32* __restrict__ rstart, u32 win_lo,
                                                        u32 win_hi) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ u32 sbuf[Padded<TILE>::value];
    __shared__ u32 scratch[THREADS / 32];
    const u32 t = blockIdx.x;
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    const bool nonstrict = (inst[L.seg].flags >> dim) & 1u;
    const u32 nQ = inst[L.seg].nQ;
    const bool first_window = win_lo == 0u;
    u32 key[ITEMS];
    load_blocked_u32<THREADS, ITEMS>(skeys, L.start, L.end, sbuf, key, 0u);
    const u32 x0 = L.start + threadIdx.x * ITEMS;
    u32 prev = 0;
    bool has_prev = x0 > L.seg_begin;
    if (has_prev && x0 < L.end) prev = skeys[x0 - 1];
    u32 cnt[1] = {0};
    u32 fmask = 0;  // bit i: item i starts a new key
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = x0 + i;
        const u32 f = (x < L.end && (!has_prev || key[i] != prev)) ? 1u : 0u;
        has_prev = true;
        prev = key[i];
        fmask |= f << i;
        cnt[0] += f;
    }
    u32 tot[1];
    block_exscan<THREADS, 1>(cnt, tot, scratch);
    u32 run = __ldg(tile_excl + t) + cnt[0];
    const u32 lx0 = threadIdx.x * ITEMS;
    // rstart (first coordinate of m = 2): per instance, at seg_begin + seg,
    // the instance-local sorted position of every rank's first point, and
    // the instance's size at index U (the group sizes of k_group_plan)
    u32* rs = (rstart && first_window) ? rstart + L.seg_begin + (u32)L.seg : nullptr;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = x0 + i;
        run += (fmask >> i) & 1u;
        sbuf[pidx(lx0 + i)] = run - 1u;
        if (rs && ((fmask >> i) & 1u)) rs[run - 1u] = x - L.seg_begin;
        if (first_window && x < L.end && x + 1 == L.seg_end) {
            const u32 U = nonstrict ? 2u * run : run;
            inst[L.seg].U[dim] = U;
            inst[L.seg].b[dim] = U <= 1u ? 0u : 32u - __clz(U - 1u);
            if (rs) rs[run] = L.seg_end - L.seg_begin;
        }
    }
    // the scatter's indices, all in flight before the barrier
    u32 dsts[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = L.start + (u32)i * THREADS + threadIdx.x;
        dsts[i] = x < L.end ? sidx[x] : 0xffffffffu;
    }
    __syncthreads();
    const u32 n_total = __ldg(seg_off + nseg);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = (u32)i * THREADS + threadIdx.x;
        const u32 dst = dsts[i];
        if (L.start + x < L.end && dst - win_lo < win_hi - win_lo) {
            u32 r = sbuf[pidx(x)];
            if (nonstrict) r = 2u * r + ((dst - L.seg_begin) < nQ ? 1u : 0u);
            if (domagg_check(dst < n_total, SITE_RANK)) rank_out[dst] = r;
        }
    }
}

// Records of a point (instruction 6m+1 with Sec. 5): the product over the
// first m-1 dimensions of the prefix sets of its ranks -- P0 (0-digits) for a
// data point, P1 (1-digits) for a query; a level of the first rank carries
// prod_{i>0} |P(r_i)| records of the point.

// Levels of the flat map (Sec. 5 records, grouped by the level of their
// first node).  A record of the first rank dimension at bit position j
// (prefix length b0-1-j) belongs to level j.  Records are laid out level
// by level (per instance); inside a level they keep the order of the last
// coordinate, and the sort then only needs the bits of the prefix.  m = 1
// has a single level holding every point.
constexpr int LMAX = 32;

template <int M>
__device__ __forceinline__ u32 levels_of(const Inst& I) {
    return M == 1 ? 1u : I.b[0];
}

// Count and offset scan of the flat map, in the order of the last
// coordinate (points were sorted by it, queries first on ties).  Tiles of
// 4096 points never straddle an instance; every warp walks 16 chunks of 32
// consecutive points.  It counts 2 x LMAX counters: the records of every
// level, and the query records (= partial slots) of every level.  The chunk
// bases it writes are relative to the tile; k_tile_exscan_counters then
// scans the tiles' totals per instance, and the flat map and the reduction
// add the tile's prefix (no look-back chain over the thousands of tiles of
// one instance).  Writes, in this order, the point's
// ranks (the first with the query flag in bit 31), index and weight (data
// points; so the flat map reads them without a dependent gather); per chunk
// of 32 points the exclusive count of both kinds
// at the chunk's first point, for every level; per instance both totals of
// every level.  The partial slots of a level are thereby a dense range in
// which each query's records keep the order of the last coordinate.  The
// counters hold the records this call puts through HBM (hbm_levels: the
// levels of the call's shard that no group or top-level tile takes);
// rec_all[instance] (if given) adds up every record of the flat map.
constexpr int CS_ROUNDS = 16;
constexpr int CS_COUNTERS = 2 * LMAX;             // per tile: records and query records of every level
constexpr u32 CS_CHUNKS = 8 * CS_ROUNDS;          // 32-point chunks per tile
constexpr u32 QUERY_BIT = 0x80000000u;  // in pr0: the point is a query (ranks are below 2^31)
template <int M, typename W, int WT>
__global__ __launch_bounds__(256) void k_count_scan(
    const u32* __restrict__ perm, const u32* __restrict__ seg_off, const u32* __restrict__ tile_off, int nseg,
    const u32* __restrict__ chunk_off, const u32* __restrict__ r0, const u32* __restrict__ r1,
    const u32* __restrict__ r2, Inst* inst, u32* __restrict__ pr0, u32* __restrict__ pr1, u32* __restrict__ pr2,
    u32* __restrict__ pj, W* __restrict__ pw,
    u32* __restrict__ chunk_base, u32* __restrict__ qchunk_base, u32* __restrict__ tile_cnt,
    u32* __restrict__ gkey, u64* __restrict__ gval, const unsigned char* __restrict__ govf,
    unsigned long long* __restrict__ rec_all) {
    constexpr int WARPS = 8, C = 2 * LMAX, TILE = WARPS * CS_ROUNDS * 32;
    static_assert(TILE == 4096, "point tiles");
    __shared__ u32 s_w[WARPS][C];
    __shared__ unsigned long long s_all[WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 t = blockIdx.x;
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    const Inst& I = inst[L.seg];
    const u32 nQ = I.nQ;
    const u32 nlev = levels_of<M>(I);
    const u32 b0 = M >= 2 ? I.b[0] : 0u, b1 = M >= 3 ? I.b[1] : 0u, b2 = M >= 4 ? I.b[2] : 0u;
    const u32 m0 = low_mask(b0), m1 = low_mask(b1), m2 = low_mask(b2);
    const u32 n_total = __ldg(seg_off + nseg);
    const bool rev = (I.flags >> (M - 1)) & 1u;  // non-strict last coordinate: its order read backwards
    const u32 wstart = L.start + (u32)warp * CS_ROUNDS * 32u;
    // per lane (= level): the counts of every chunk of the warp
    u32 rc[CS_ROUNDS], qc[CS_ROUNDS];
    u32 run_all = 0, run_q = 0;
    unsigned long long recs = 0;  // every record of the lane's points
    // eight rounds at a time: their permutation loads, then their gathers of
    // the first rank, all in flight together
    constexpr int BATCH = 8;
    static_assert(CS_ROUNDS % BATCH == 0, "whole batches");
    u32 jb[BATCH], ab[BATCH];
#pragma unroll
    for (int i = 0; i < CS_ROUNDS; ++i) {
        const u32 x = wstart + (u32)i * 32u + (u32)lane;
        const bool valid = x < L.end;
        if (i % BATCH == 0) {
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const u32 xb = wstart + (u32)(i + b) * 32u + (u32)lane;
                u32 jj = xb < L.end ? perm[rev ? L.seg_begin + (L.seg_end - 1u - xb) : xb] : L.seg_begin;
                if (jj >= n_total) jj = L.seg_begin;  // never taken for a valid permutation
                jb[b] = jj;
            }
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const u32 xb = wstart + (u32)(i + b) * 32u + (u32)lane;
                ab[b] = (M >= 2 && xb < L.end) ? r0[jb[b]] : 0u;
            }
        }
        const u32 j = jb[i % BATCH];
        const bool q = valid && (j - L.seg_begin) < nQ;
        u32 a = ab[i % BATCH], c = 0, bits0 = 0, c1 = 1;
        if (M >= 3 && valid) c = r1[j];
        u32 e2 = 0;
        if (M >= 4 && valid) e2 = r2[j];
        if (M >= 2) bits0 = (q ? a : ~a) & m0;
        if (M >= 3) c1 = (u32)__popc((q ? c : ~c) & m1);
        if (M >= 4) c1 *= (u32)__popc((q ? e2 : ~e2) & m2);
        if (M == 1) bits0 = 1u;
        if (!valid) bits0 = 0;
        recs += (unsigned long long)__popc(bits0) * c1;
        // the levels whose records this call puts through HBM
        u32 hb = bits0;
        if (M >= 2 && valid) hb &= hbm_levels(I, a, govf);
        if (M == 1) hb &= I.lvmask;
        if (valid) {
            if (M >= 2) pr0[x] = q ? (a | QUERY_BIT) : a;
            if (M >= 3) pr1[x] = c;
            if (M >= 4) pr2[x] = e2;
            pj[x] = j;
            u32 wbits = 0;
            if (WT != 3 && !q) {
                const u32 local = j - L.seg_begin;
                if (WT == 1) {
                    pw[x] = (W)reinterpret_cast<const long long*>(I.dw)[local - nQ];
                } else {
                    wbits = reinterpret_cast<const u32*>(I.dw)[local - nQ];
                    pw[x] = (W)wbits;
                }
            }
            // m = 2, 3 with groups: the group sort's key (the group: rank >>
            // gS) and value (rank | query bit, then a query's position in
            // this order, a datum's weight bits or, for 8-byte weights and
            // for m = 3, its position x)
            if ((M == 2 || M == 3) && gkey && I.gS) {
                const u32 pv = (q || WT == 1 || M == 3) ? x : wbits;
                gkey[x] = a >> I.gS;
                gval[x] = ((u64)(q ? (a | QUERY_BIT) : a) << 32) | (u64)pv;
            }
        }
        u32 mine = 0, mine_q = 0;
        if (M <= 2) {
            // one record per level: lane lv counts the lanes with bit lv set
            mine = (u32)__popc(warp_transpose32(hb, (u32)lane));
            mine_q = (u32)__popc(warp_transpose32(q ? hb : 0u, (u32)lane));
        } else {
            for (u32 lv = 0; lv < nlev; ++lv) {
                const u32 w = ((hb >> lv) & 1u) ? c1 : 0u;
                const u32 sa = __reduce_add_sync(0xffffffffu, w);
                const u32 sq = __reduce_add_sync(0xffffffffu, q ? w : 0u);
                if ((u32)lane == lv) {
                    mine = sa;
                    mine_q = sq;
                }
            }
        }
        rc[i] = mine;
        qc[i] = mine_q;
        run_all += mine;
        run_q += mine_q;
    }
    s_w[warp][lane] = run_all;
    s_w[warp][LMAX + lane] = run_q;
    for (int o = 16; o >= 1; o >>= 1) recs += __shfl_xor_sync(0xffffffffu, recs, o);
    if (lane == 0) s_all[warp] = recs;
    __syncthreads();
    if (threadIdx.x == 0 && rec_all) {
        unsigned long long t = 0;
        for (int w = 0; w < WARPS; ++w) t += s_all[w];
        if (t) atomicAdd(rec_all + L.seg, t);
    }
    if (threadIdx.x < C) {  // exclusive over the warps; the tile's totals
        const int c = threadIdx.x;
        u32 sum = 0;
        for (int w = 0; w < WARPS; ++w) {
            const u32 v = s_w[w][c];
            s_w[w][c] = sum;
            sum += v;
        }
        tile_cnt[(u64)t * C + c] = sum;
    }
    __syncthreads();
    const u32 base_all = s_w[warp][lane];  // relative to the tile
    const u32 base_q = s_w[warp][LMAX + lane];
    const u32 cbase = __ldg(chunk_off + L.seg) + (wstart - L.seg_begin) / 32u;
    u32 ra = 0, rq = 0;
#pragma unroll
    for (int i = 0; i < CS_ROUNDS; ++i) {
        if (wstart + (u32)i * 32u < L.end && (u32)lane < nlev) {
            chunk_base[(u64)(cbase + i) * LMAX + lane] = base_all + ra;
            qchunk_base[(u64)(cbase + i) * LMAX + lane] = base_q + rq;
        }
        ra += rc[i];
        rq += qc[i];
    }
}

// Per instance and counter, the exclusive scan of the tiles' totals (in
// place), and the instance's totals per level (lvl_tot, qlvl_tot).  Grid
// (instance, CS_COUNTERS / 32): the 32 warps of a block split the instance's
// tiles into 32 consecutive slices, lane = counter (so a warp's loads are a
// tile's 32 consecutive counters): slice sums, their exclusive combination
// in shared memory, then the running prefixes.  A total that does not fit 32
// bits raises ERR_OVERFLOW.
static __global__ __launch_bounds__(1024) void k_tile_exscan_counters(const u32* __restrict__ tile_off, int nseg,
                                                                     u32* __restrict__ cnt, u32* __restrict__ lvl_tot,
                                                                     u32* __restrict__ qlvl_tot, Ctl* ctl) {
    __shared__ u64 s_sum[32][33];
    const int seg = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = (int)blockIdx.y * 32 + lane;
    const u32 t0 = __ldg(tile_off + seg), n = __ldg(tile_off + seg + 1) - t0, per = (n + 31) / 32;
    const u32 a = t0 + min(n, (u32)warp * per), b = t0 + min(n, (u32)(warp + 1) * per);
    u64 sum = 0;
    for (u32 t = a; t < b; t += 16) {
        u32 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = t + i < b ? cnt[(u64)(t + i) * CS_COUNTERS + c] : 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) sum += v[i];
    }
    s_sum[warp][lane] = sum;
    __syncthreads();
    u64 run = 0;
    for (int w = 0; w < warp; ++w) run += s_sum[w][lane];
    for (u32 t = a; t < b; t += 16) {
        u32 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = t + i < b ? cnt[(u64)(t + i) * CS_COUNTERS + c] : 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (t + i < b) cnt[(u64)(t + i) * CS_COUNTERS + c] = (u32)run;
            run += v[i];
        }
    }
    if (warp == 31) {  // the last slice ends at the instance's last tile: run is the total
        if (run >> 32) atomicOr(&ctl->error, ERR_OVERFLOW);
        if (c < LMAX) lvl_tot[(u64)seg * LMAX + c] = (u32)run;
        else qlvl_tot[(u64)seg * LMAX + (c - LMAX)] = (u32)run;
    }
}

// Flat map (instruction 6m+1, Sec. 5), level by level.  Every point writes
// its records (sort key | role bit, payload) into the segment of their
// level; a warp handles one chunk of 32 consecutive points of an instance and
// writes each level's records contiguously (the chunk's base from the count
// scan plus the exclusive count of the lanes before), so stores coalesce.
// Sort key: the prefix of the first rank at that level, v0 = r0 >> (j+1);
// for m = 3 followed by the canonical node of the second rank (node_of),
// v0 << b1 | node1.  The role bit (top bit of the key) marks query records.
// Payload: data -> the weight's bits (Op::Pay), query -> its partial slot,
// a dense per-level position (query slot base of the level + the chunk's
// query count of the level + the lanes before).
template <int M, typename K, typename Pay, typename W, int WT>
__global__ __launch_bounds__(256) void k_expand(
    const u32* __restrict__ chunk_off, int k, int k0, int k1, const u32* __restrict__ pt_offs,
    const u32* __restrict__ pr0, const u32* __restrict__ pr1, const u32* __restrict__ pr2,
    const u32* __restrict__ pj, const W* __restrict__ pw, const u32* __restrict__ chunk_base, const u32* __restrict__ qchunk_base,
    const u32* __restrict__ pt_tiles, const u32* __restrict__ tile_excl,
    const Inst* __restrict__ inst, const u32* __restrict__ seg_base /*[k1-k0][LMAX]*/,
    const u32* __restrict__ qseg_base /*[k1-k0][LMAX]*/, const u32* __restrict__ narrow_mask /*[k1-k0] or null*/,
    u32 n_rec, K* __restrict__ kout, Pay* __restrict__ pout, u32 n_rec1, u32* __restrict__ kout1,
    Pay* __restrict__ pout1, const unsigned char* __restrict__ govf) {
    const int lane = threadIdx.x & 31;
    const u32 lt = lanemask_lt();
    const u32 c_begin = __ldg(chunk_off + k0), c_end = __ldg(chunk_off + k1);
    const u32 warps = (gridDim.x * blockDim.x) >> 5;
    const K role = K(1) << (sizeof(K) * 8 - 1);
    // a warp's chunk: what its lanes read before writing records
    struct Chunk {
        u32 c, ps, p, nlev, b1, b2, nmask, my_all, my_q, a, cc, ee, bits0, bits1, bits2, c1;
        int s;
        bool q;
        Pay w;
    };
    auto load = [&](u32 c) {
        Chunk X;
        X.c = c;
        X.s = upper_index(chunk_off, k + 1, c);
        const Inst& I = inst[X.s];
        X.ps = __ldg(pt_offs + X.s);
        const u32 pe = __ldg(pt_offs + X.s + 1);
        X.p = X.ps + (c - __ldg(chunk_off + X.s)) * 32u + (u32)lane;
        const bool valid = X.p < pe;
        const u32 nQ = I.nQ;
        X.nlev = levels_of<M>(I);
        X.b1 = M >= 3 ? I.b[1] : 0u;
        X.b2 = M >= 4 ? I.b[2] : 0u;
        const u32 tile = __ldg(pt_tiles + X.s) + (c - __ldg(chunk_off + X.s)) / CS_CHUNKS;  // the count scan's tile
        // m >= 3: levels whose node keys fit 31 bits go to the 32-bit-key records (class 1)
        X.nmask = narrow_mask ? __ldg(narrow_mask + (X.s - k0)) : 0u;
        // lane lv holds the bases of level lv (read once, shuffled below)
        X.my_all = (u32)lane < X.nlev ? __ldg(seg_base + (u64)(X.s - k0) * LMAX + lane) +
                                            __ldg(chunk_base + (u64)c * LMAX + lane) +
                                            __ldg(tile_excl + (u64)tile * CS_COUNTERS + lane)
                                      : 0u;
        X.my_q = (u32)lane < X.nlev ? __ldg(qseg_base + (u64)(X.s - k0) * LMAX + lane) +
                                          __ldg(qchunk_base + (u64)c * LMAX + lane) +
                                          __ldg(tile_excl + (u64)tile * CS_COUNTERS + LMAX + lane)
                                    : 0u;
        X.a = X.cc = X.ee = X.bits0 = X.bits1 = X.bits2 = 0;
        X.c1 = 1;
        X.q = false;
        X.w = 0;
        if (valid) {
            // coalesced reads in the order of the last coordinate (count scan)
            if (M >= 2) {
                X.a = pr0[X.p];
                X.q = (X.a & QUERY_BIT) != 0u;
                X.a &= ~QUERY_BIT;
                X.bits0 = (X.q ? X.a : ~X.a) & low_mask(I.b[0]);
                X.bits0 &= hbm_levels(I, X.a, govf);  // the levels this call takes through HBM
            } else {
                X.q = pj[X.p] - X.ps < nQ;
                X.bits0 = 1u & I.lvmask;  // the single level, unless another shard takes it
            }
            if (M >= 3) {
                X.cc = pr1[X.p];
                X.bits1 = (X.q ? X.cc : ~X.cc) & low_mask(X.b1);
                X.c1 = (u32)__popc(X.bits1);
            }
            if (M >= 4) {
                X.ee = pr2[X.p];
                X.bits2 = (X.q ? X.ee : ~X.ee) & low_mask(X.b2);
                X.c1 *= (u32)__popc(X.bits2);
            }
            // 8-byte weights stay in pw: the record carries their position
            if (!X.q && WT != 3) X.w = WT == 1 ? (Pay)X.p : (Pay)pw[X.p];
        }
        return X;
    };
    // the next chunk's reads are issued before this chunk's records are written
    u32 c = c_begin + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    Chunk nxt;
    if (c < c_end) nxt = load(c);
    for (; c < c_end; c += warps) {
        const Chunk X = nxt;
        if (c + warps < c_end) nxt = load(c + warps);
        const u32 nlev = X.nlev, b1 = X.b1, b2 = X.b2, nmask = X.nmask, my_all = X.my_all, my_q = X.my_q;
        const u32 a = X.a, cc = X.cc, ee = X.ee, bits1 = X.bits1, bits2 = X.bits2, c1 = X.c1;
        u32 bits0 = X.bits0;
        const bool q = X.q;
        const Pay w = X.w;
        (void)b2;
        (void)ee;
        (void)bits2;
        if (M >= 3 && c1 == 0) bits0 = 0;  // no records at all
        const u32 live = __ballot_sync(0xffffffffu, bits0 != 0u);
        if (live == 0u) continue;
        for (u32 lv = 0; lv < nlev; ++lv) {
            const bool has = (bits0 >> lv) & 1u;
            const u32 hb = __ballot_sync(0xffffffffu, has);
            if (hb == 0u) continue;
            const u32 qb = __ballot_sync(0xffffffffu, has && q);
            const u32 base_all = __shfl_sync(0xffffffffu, my_all, lv);
            const u32 base_q = __shfl_sync(0xffffffffu, my_q, lv);
            u32 ex, exq;
            if (M <= 2) {
                ex = (u32)__popc(hb & lt);
                exq = (u32)__popc(qb & lt);
            } else {
                const u32 wv = has ? c1 : 0u, wq = (has && q) ? c1 : 0u;
                u32 inc = wv, incq = wq;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 n1 = __shfl_up_sync(0xffffffffu, inc, o);
                    const u32 n2 = __shfl_up_sync(0xffffffffu, incq, o);
                    if (lane >= o) {
                        inc += n1;
                        incq += n2;
                    }
                }
                ex = inc - wv;
                exq = incq - wq;
            }
            const u32 pos = base_all + ex;
            const Pay pay = q ? (Pay)(base_q + exq) : w;
            const K kv = M == 1 ? K(0) : (K)(a >> (lv + 1));
            if (M <= 2) {
                if (has && domagg_check(pos < n_rec, SITE_EXPAND)) {
                    kout[pos] = q ? (kv | role) : kv;
                    pout[pos] = pay;
                }
            } else {
                // the warp writes one point's records at a time, lane j taking
                // the record of the second rank's digit j (its rank among the
                // point's digits is its place): contiguous, coalesced stores
                for (u32 act = hb; act; act &= act - 1) {
                    const int src = __ffs(act) - 1;
                    const u32 sb = __shfl_sync(0xffffffffu, bits1, src);
                    const u32 scc = __shfl_sync(0xffffffffu, cc, src);
                    const K skv = __shfl_sync(0xffffffffu, kv, src);
                    const u32 spos = __shfl_sync(0xffffffffu, pos, src);
                    const Pay spay = __shfl_sync(0xffffffffu, pay, src);
                    const bool sq = (qb >> src) & 1u;
                    const bool narrow = (nmask >> lv) & 1u;
                    // one store of a record into its class's arrays
                    auto put = [&](u32 at, K key, u32 r) {
                        if (narrow) {
                            if (domagg_check(at < n_rec1, SITE_EXPAND)) {
                                kout1[at] = sq ? ((u32)key | 0x80000000u) : (u32)key;
                                pout1[at] = sq ? (Pay)(spay + r) : spay;
                            }
                        } else if (domagg_check(at < n_rec, SITE_EXPAND)) {
                            kout[at] = sq ? (key | role) : key;
                            pout[at] = sq ? (Pay)(spay + r) : spay;
                        }
                    };
                    if (M == 3) {
                        if ((sb >> lane) & 1u) {
                            const u32 r = (u32)__popc(sb & lt);
                            put(spos + r, (skv << b1) | (K)node_of(scc, (u32)lane), r);
                        }
                    } else {
                        // m = 4: the third rank's digits across the lanes, the
                        // second rank's digits one after the other
                        const u32 sb2 = __shfl_sync(0xffffffffu, bits2, src);
                        const u32 see = __shfl_sync(0xffffffffu, ee, src);
                        const u32 c2 = (u32)__popc(sb2);
                        u32 t1 = 0;
                        for (u32 r1 = sb; r1; r1 &= r1 - 1, ++t1) {
                            const u32 j1 = __ffs(r1) - 1;
                            if ((sb2 >> lane) & 1u) {
                                const u32 r = t1 * c2 + (u32)__popc(sb2 & lt);
                                put(spos + r,
                                    ((((skv << b1) | (K)node_of(scc, j1)) << b2)) | (K)node_of(see, (u32)lane), r);
                            }
                        }
                    }
                }
            }
        }
    }
}

}  // namespace domagg
