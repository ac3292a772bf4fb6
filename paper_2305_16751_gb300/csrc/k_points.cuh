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

// Tiles of size `tile` over segments: tile_off[s] = sum over s' < s of
// ceil(len(s') / tile), tile_off[nseg] = total.  One block.
static __global__ void k_make_tiles(const u32* __restrict__ seg_off, int nseg, u32 tile, u32* __restrict__ tile_off) {
    __shared__ u32 carry;
    __shared__ u32 warp_sum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < nseg; base += blockDim.x) {
        const int s = base + threadIdx.x;
        u32 v = 0;
        if (s < nseg) v = (__ldg(seg_off + s + 1) - __ldg(seg_off + s) + tile - 1) / tile;
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
                         u32* __restrict__ rk0, u32* __restrict__ rk1, u32* __restrict__ lk, int negate, Ctl* ctl) {
    const u32 p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int s = upper_index(pt_offs, k + 1, p);
    const u32 local = p - __ldg(pt_offs + s);
    const u32 nQ = inst[s].nQ;
    const void* base = local < nQ ? inst[s].qco : inst[s].dco;
    const u32 row = local < nQ ? local : local - nQ;
    bool nan = false;
    if (M >= 2) rk0[p] = coord_key<F32>(base, row, M, 0, negate, nan);
    if (M >= 3) rk1[p] = coord_key<F32>(base, row, M, 1, negate, nan);
    lk[p] = coord_key<F32>(base, row, M, M - 1, negate, nan);
    if (nan) atomicOr(&ctl->error, ERR_NAN);
}

// Loads a tile of u32 [start, end) in blocked order (thread t gets items
// t*ITEMS .. t*ITEMS+ITEMS-1) through shared memory, coalesced.
template <int THREADS, int ITEMS>
__device__ __forceinline__ void load_blocked_u32(const u32* __restrict__ src, u32 start, u32 end, u32* sbuf,
                                                 u32 (&out)[ITEMS], u32 fill) {
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
// own slot.  U = number of distinct keys; b = ceil(log2 U) digits.
template <int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS) void k_rank(const u32* __restrict__ skeys, const u32* __restrict__ sidx,
                                                  const u32* __restrict__ seg_off, const u32* __restrict__ tile_off,
                                                  int nseg, u32* __restrict__ rank_out, Inst* inst, int dim,
                                                  u64* status, Ctl* ctl, int launch_idx) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ u32 sbuf[Padded<TILE>::value];
    __shared__ u32 scratch[THREADS / 32];
    __shared__ u32 s_info[3];
    if (threadIdx.x == 0) {
        s_info[0] = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        s_info[1] = ctl->epoch_base + (u32)launch_idx;
    }
    __syncthreads();
    const u32 t = s_info[0], epoch = s_info[1];
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    u32 key[ITEMS];
    load_blocked_u32<THREADS, ITEMS>(skeys, L.start, L.end, sbuf, key, 0u);
    // predecessor of each thread's first item
    const u32 x0 = L.start + threadIdx.x * ITEMS;
    u32 prev = 0;
    bool has_prev = x0 > L.seg_begin;
    if (has_prev && x0 < L.end) prev = skeys[x0 - 1];
    u32 cnt[1] = {0};
    u32 f[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = x0 + i;
        f[i] = (x < L.end && (!has_prev || key[i] != prev)) ? 1u : 0u;
        has_prev = true;
        prev = key[i];
        cnt[0] += f[i];
    }
    u32 tot[1];
    block_exscan<THREADS, 1>(cnt, tot, scratch);
    if (threadIdx.x == 0) {
        u64* st = status + t;
        u32 excl = 0;
        const u32 first_tile = t - (L.start - L.seg_begin) / (u32)TILE;
        if (L.first) {
            st_store(st, st_pack(epoch, ST_PREFIX, tot[0]));
        } else {
            st_store(st, st_pack(epoch, ST_AGG, tot[0]));
            excl = lookback_u32(status, 1, 0, t, first_tile, epoch, ctl, 2u);
            st_store(st, st_pack(epoch, ST_PREFIX, excl + tot[0]));
        }
        s_info[2] = excl;
    }
    __syncthreads();
    u32 run = s_info[2] + cnt[0];
    const u32 n_total = __ldg(seg_off + nseg);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = x0 + i;
        if (x < L.end) {
            run += f[i];
            const u32 dst = sidx[x];
            if (dst < n_total) rank_out[dst] = run - 1u;
            if (x + 1 == L.seg_end) {
                const u32 U = run;
                inst[L.seg].U[dim] = U;
                inst[L.seg].b[dim] = U <= 1u ? 0u : 32u - __clz(U - 1u);
            }
        }
    }
}

// Records of a point (instruction 6m+1 with Sec. 5): the product over the
// first m-1 dimensions of the prefix sets of its ranks -- P0 (0-digits) for a
// data point, P1 (1-digits) for a query.  bits_i selects those digits.
template <int M>
__device__ __forceinline__ u32 record_count(u32 bits0, u32 bits1) {
    if (M == 1) return 1u;
    if (M == 2) return (u32)__popc(bits0);
    return (u32)__popc(bits0) * (u32)__popc(bits1);
}

// Count and offset scan of the flat map, in the order of the last
// coordinate (points were sorted by it, queries first on ties).  Per
// instance (segmented chains) it scans three counters: records, query
// records (= partial slots) and query points.  Writes the point's ranks,
// index and offsets in this order, and per query (in this order) its slot
// base and its index in Q.  The instance's last tile stores T and Tq.
template <int M, int THREADS, int ITEMS>
__global__ __launch_bounds__(THREADS) void k_count_scan(
    const u32* __restrict__ perm, const u32* __restrict__ seg_off, const u32* __restrict__ tile_off, int nseg,
    const u32* __restrict__ r0, const u32* __restrict__ r1, Inst* inst, const u32* __restrict__ q_offs,
    u32* __restrict__ pr0, u32* __restrict__ pr1, u32* __restrict__ pj, u32* __restrict__ poff,
    u32* __restrict__ pqoff, u32* __restrict__ qslot, u32* __restrict__ qidx, u64* status, Ctl* ctl,
    int launch_idx) {
    constexpr int TILE = THREADS * ITEMS;
    __shared__ u32 sbuf[Padded<TILE>::value];
    __shared__ u32 scratch[3 * (THREADS / 32)];
    __shared__ u32 s_info[2];
    __shared__ u32 s_excl[3];
    if (threadIdx.x == 0) {
        s_info[0] = atomicAdd(&ctl->tile_ctr[launch_idx], 1u);
        s_info[1] = ctl->epoch_base + (u32)launch_idx;
    }
    __syncthreads();
    const u32 t = s_info[0], epoch = s_info[1];
    if (t >= __ldg(tile_off + nseg)) return;
    const TileLoc L = locate_tile<TILE>(t, seg_off, tile_off, nseg);
    const u32 nQ = inst[L.seg].nQ;
    const u32 b0 = M >= 2 ? inst[L.seg].b[0] : 0u, b1 = M >= 3 ? inst[L.seg].b[1] : 0u;
    const u32 m0 = low_mask(b0), m1 = low_mask(b1);
    u32 j[ITEMS];
    load_blocked_u32<THREADS, ITEMS>(perm, L.start, L.end, sbuf, j, 0u);
    const u32 x0 = L.start + threadIdx.x * ITEMS;
    const u32 n_total = __ldg(seg_off + nseg);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i)  // a permutation entry outside the point space is never followed
        if (j[i] >= n_total) j[i] = L.seg_begin + nQ;
    u32 c[3] = {0, 0, 0};
    u32 rr0[ITEMS], rr1[ITEMS], cnt[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        rr0[i] = rr1[i] = cnt[i] = 0;
        if (x0 + i < L.end) {
            const bool q = (j[i] - L.seg_begin) < nQ;
            if (M >= 2) rr0[i] = r0[j[i]];
            if (M >= 3) rr1[i] = r1[j[i]];
            const u32 bits0 = (q ? rr0[i] : ~rr0[i]) & m0;
            const u32 bits1 = (q ? rr1[i] : ~rr1[i]) & m1;
            cnt[i] = record_count<M>(bits0, bits1);
            c[0] += cnt[i];
            if (q) {
                c[1] += cnt[i];
                c[2] += 1;
            }
        }
    }
    u32 tot[3];
    block_exscan<THREADS, 3>(c, tot, scratch);
    if (threadIdx.x < 3) {
        const int cc = threadIdx.x;
        u64* st = status + (u64)t * 3 + cc;
        u32 excl = 0;
        const u32 first_tile = t - (L.start - L.seg_begin) / (u32)TILE;
        if (L.first) {
            st_store(st, st_pack(epoch, ST_PREFIX, tot[cc]));
        } else {
            st_store(st, st_pack(epoch, ST_AGG, tot[cc]));
            excl = lookback_u32(status, 3, cc, t, first_tile, epoch, ctl, 3u);
            st_store(st, st_pack(epoch, ST_PREFIX, excl + tot[cc]));
        }
        if (excl + tot[cc] < excl) atomicOr(&ctl->error, ERR_OVERFLOW);
        s_excl[cc] = excl;
        if (L.end == L.seg_end) {  // last tile of the instance
            if (cc == 0) inst[L.seg].T = excl + tot[0];
            if (cc == 1) inst[L.seg].Tq = excl + tot[1];
        }
    }
    __syncthreads();
    u32 off = s_excl[0] + c[0], qoff = s_excl[1] + c[1], qr = s_excl[2] + c[2];
    const u32 qbase = __ldg(q_offs + L.seg);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const u32 x = x0 + i;
        if (x < L.end) {
            const u32 local = j[i] - L.seg_begin;
            const bool q = local < nQ;
            if (M >= 2) pr0[x] = rr0[i];
            if (M >= 3) pr1[x] = rr1[i];
            pj[x] = j[i];
            poff[x] = off;
            pqoff[x] = qoff;
            if (q && qr < nQ) {
                qslot[qbase + qr] = qoff;
                qidx[qbase + qr] = local;
                qoff += cnt[i];
                qr += 1;
            }
            off += cnt[i];
        }
    }
}

// Flat map (instruction 6m+1, Sec. 5): every point writes its records,
// (node key | role bit, payload), at its offset in the record array of its
// chunk.  The node key concatenates the canonical node of every one of the
// first m-1 ranks (node_of): for m = 3, node0 << b1 | node1.  The role bit
// (top bit of the key) marks query records; it is not part of the sort key.
// Payload: data -> the weight's bits (Op::Pay), query -> its partial slot.
//
// One warp handles 32 consecutive points.  Each lane enumerates its own
// point's records (lowest set bit first: one find-first-set per record) into
// a per-warp staging buffer in shared memory, EXPAND_STAGE_BYTES at a time;
// the warp then copies the staged run to global memory with coalesced stores.
constexpr int EXPAND_THREADS = 256;
constexpr int EXPAND_STAGE_BYTES = 8192;  // per warp
template <int M, typename K, typename Pay, int WT>
__global__ __launch_bounds__(EXPAND_THREADS) void k_expand(
    u32 p_begin, u32 p_end, const u32* __restrict__ pr0, const u32* __restrict__ pr1,
    const u32* __restrict__ pj, const u32* __restrict__ poff, const u32* __restrict__ pqoff,
    const Inst* __restrict__ inst, const u32* __restrict__ pt_offs, int k, const u32* __restrict__ rec_base,
    const u32* __restrict__ qrec_base, int k0, u32 n_rec, K* __restrict__ kout, Pay* __restrict__ pout) {
    constexpr u32 CH = EXPAND_STAGE_BYTES / (sizeof(K) + sizeof(Pay));  // records staged per warp
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    K* sk = reinterpret_cast<K*>(smem + warp * EXPAND_STAGE_BYTES);
    Pay* sp = reinterpret_cast<Pay*>(sk + CH);
    const u32 warps = (gridDim.x * blockDim.x) >> 5;
    const K role = K(1) << (sizeof(K) * 8 - 1);
    for (u32 wb = p_begin + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; wb < p_end; wb += warps * 32u) {
        const u32 p = wb + lane;
        const bool valid = p < p_end;
        u32 r0 = 0, r1 = 0, bits0 = 0, bits1 = 0, b1 = 0, cnt = 0, gbase = 0;
        bool q = false;
        Pay pay = 0;
        if (valid) {
            const int s = upper_index(pt_offs, k + 1, p);
            u32 j = pj[p];
            const u32 nQ = inst[s].nQ, nD = inst[s].nD;
            if (j - __ldg(pt_offs + s) >= nQ + nD) j = __ldg(pt_offs + s);  // never taken for a valid permutation
            const u32 local = j - __ldg(pt_offs + s);
            q = local < nQ;
            if (M >= 2) {
                r0 = pr0[p];
                bits0 = (q ? r0 : ~r0) & low_mask(inst[s].b[0]);
            }
            if (M >= 3) {
                r1 = pr1[p];
                b1 = inst[s].b[1];
                bits1 = (q ? r1 : ~r1) & low_mask(b1);
            }
            cnt = record_count<M>(bits0, bits1);
            gbase = __ldg(rec_base + (s - k0)) + poff[p];
            if (q) {
                pay = (Pay)(__ldg(qrec_base + (s - k0)) + pqoff[p]);
            } else if (WT == 1) {  // int64 weights
                pay = (Pay)reinterpret_cast<const long long*>(inst[s].dw)[local - nQ];
            } else if (WT == 0 || WT == 2) {  // 32-bit weights
                pay = (Pay)reinterpret_cast<const u32*>(inst[s].dw)[local - nQ];
            }
        }
        // records of this warp: [wstart, wstart + R)
        const u32 wstart = __shfl_sync(0xffffffffu, gbase, 0);
        const u32 off_rel = valid ? gbase - wstart : 0u;
        u32 R = valid ? off_rel + cnt : 0u;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) R = max(R, __shfl_xor_sync(0xffffffffu, R, o));
        // enumeration state: the current node of dimension 0 (lowest pending
        // bit of rem0) and the pending bits of dimension 1
        u32 rem0 = bits0, rem1 = bits1, kk = 0;
        for (u32 c0 = 0; c0 < R; c0 += CH) {
            const u32 c1 = min(c0 + CH, R);
            for (u32 idx = off_rel + kk; kk < cnt && idx < c1; ++kk, ++idx) {
                K key;
                if (M == 1) {
                    key = K(0);
                } else if (M == 2) {
                    const u32 j0 = __ffs(rem0) - 1;
                    rem0 &= rem0 - 1;
                    key = (K)node_of(r0, j0);
                } else {
                    const u32 j0 = __ffs(rem0) - 1, j1 = __ffs(rem1) - 1;
                    key = ((K)node_of(r0, j0) << b1) | (K)node_of(r1, j1);
                    rem1 &= rem1 - 1;
                    if (rem1 == 0) {  // next node of dimension 0
                        rem0 &= rem0 - 1;
                        rem1 = bits1;
                    }
                }
                if (q) key |= role;
                sk[idx - c0] = key;
                sp[idx - c0] = q ? (Pay)(pay + kk) : pay;
            }
            __syncwarp();
            for (u32 x = c0 + lane; x < c1; x += 32u) {
                if (wstart + x < n_rec) {
                    kout[wstart + x] = sk[x - c0];
                    pout[wstart + x] = sp[x - c0];
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace domagg
