// dev_common.cuh -- device-side building blocks shared by the kernels:
// control block, per-instance table, decoupled look-back status words,
// float-float arithmetic and the aggregation operators F with their units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace domagg {

typedef uint32_t u32;
typedef uint64_t u64;

// Error bits recorded on the device (Ctl::error).
enum : u32 {
    ERR_TIMEOUT = 1u,   // a bounded wait on a predecessor tile ran out
    ERR_NAN = 2u,       // a NaN coordinate was met
    ERR_OVERFLOW = 4u,  // the record count does not fit 32 bits
    ERR_EPOCH = 8u,     // the look-back epoch counter is about to wrap
    ERR_CAPACITY = 16u, // a planned run met more records than its plan reserved
};

constexpr int MAX_LAUNCHES = 64;  // look-back launches per pipeline run

// Device control block (one per handle).
struct Ctl {
    u32 epoch_base;        // advanced by MAX_LAUNCHES at every pipeline start
    u32 error;             // ERR_* bits, cleared by the host
    u32 timeout_where;     // kind of the launch whose wait ran out (diagnostics)
    u32 pad0;
    u32 tile_ctr[MAX_LAUNCHES];  // dynamic tile counters, zeroed at pipeline start
    // totals written by the count/offset scan (read by the host)
    u32 T_total;           // records
    u32 Tq_total;          // query records (= partial slots)
    u32 max_key_bits;      // widest node key over the instances
    u32 pad1;
};

// Per-instance table.  The host fills the first block; the kernels fill the
// second.  Point index space of an instance: queries first (local 0..nQ-1),
// then data points (local nQ..nQ+nD-1), so that a stable sort by the last
// coordinate puts queries before data on ties (Sec. 5).
struct Inst {
    const void* dco;   // data coordinates [nD][m]
    const void* qco;   // query coordinates [nQ][m]
    const void* dw;    // data weights [nD]
    void* out;         // outputs [nQ]
    u32 nD, nQ;
    u32 pt_off;        // first point in the concatenated point space
    u32 q_off;         // first query in the concatenated query space
    // device-computed
    u32 U[3];          // distinct values of the first m-1 coordinates
    u32 b[3];          // binary digits of the ranks: ceil(log2 U)
    u32 rec_off, T;    // records of this instance
    u32 qrec_off, Tq;  // query records (partial slots) of this instance
    u32 key_bits;      // bits of the node key
    u32 flags;         // bit i (i < 3): coordinate i compared non-strictly; FLAG_VIRTUAL_LAST
    // m = 2, 3: rank levels below gS are aggregated per group of 2^gS ranks
    // in shared memory (k_group, k_group3); G groups.  gS = 0: every level
    // goes through the records in HBM.  A group with more points than shared
    // memory holds (a heavy tie) sends its points' levels below gS through
    // the records too (its flag in the groups' overflow array).
    u32 gS, G;
    // m = 2: rank levels tS .. b0-1 (at most TOP_MAX_BITS) are taken per tile
    // of points in the order of the last coordinate (k_top); topmask: those
    // of this call's shard (bit lv; device-computed)
    u32 tS, topmask;
    // levels of the first rank whose records this call takes through HBM
    // (bit lv; device-computed), and the call's shard of the flat map: shard
    // `shard` of `nshards` takes the levels >= gS with (lv - gS) % nshards ==
    // shard and the groups g with g % nshards == shard (host-filled; 0 of 1
    // for a whole forward)
    u32 lvmask, shard, nshards;
    float* out_lo;  // float32 sums of a shard: the low halves of the float-float partials (or null)
};
// The last of the M coordinates is not stored but constant (the basic
// variant of Sec. 4 run as the Sec. 5 pipeline with one more coordinate).
constexpr u32 FLAG_VIRTUAL_LAST = 1u << 8;
// Inst::flags: evaluate the levels of the first coordinate one by one on the
// points (the level-wise formulation, m <= 2) instead of expanding records
constexpr u32 FLAG_WAVELET = 1u << 9;

// The first-rank levels whose records a point with (level) rank `rank` puts
// through HBM in this call: the instance's (lvmask) and, if the point's
// group overflowed shared memory (govf[pt_off + group], set by k_group_plan
// for this call's groups), every level below gS as well.
__device__ __forceinline__ u32 hbm_levels(const Inst& I, u32 rank, const unsigned char* __restrict__ govf) {
    u32 m = I.lvmask;
    if (I.gS && govf && govf[I.pt_off + (rank >> I.gS)]) m |= (1u << I.gS) - 1u;
    return m;
}

// ---------------------------------------------------------------------
// decoupled look-back status words: [63:34] epoch, [33:32] flag, [31:0] value
// ---------------------------------------------------------------------
enum : u32 { ST_AGG = 1u, ST_PREFIX = 2u };
constexpr u32 EPOCH_MASK = (1u << 30) - 1u;
constexpr u32 SPIN_LIMIT = 1u << 21;  // ~1-2 s of polling with back-off

__device__ __forceinline__ u64 st_pack(u32 epoch, u32 flag, u32 v) {
    return ((u64)(epoch & EPOCH_MASK) << 34) | ((u64)flag << 32) | (u64)v;
}
__device__ __forceinline__ void st_store(u64* p, u64 v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ u64 st_load(const u64* p) {
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_store_release(u32* p, u32 v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ u32 st_load_acquire(const u32* p) {
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// True once any bounded wait of this pipeline has run out: the other waits
// then give up at once instead of each running out in turn.
__device__ __forceinline__ bool timed_out(const Ctl* ctl) {
    return (*reinterpret_cast<const volatile u32*>(&ctl->error) & ERR_TIMEOUT) != 0u;
}

// Exclusive prefix of counter c for tile t over the chain of tiles
// [chain_first, t).  Tiles publish ST_AGG (own count) before looking back and
// ST_PREFIX (inclusive prefix) after; chain_first publishes ST_PREFIX at once,
// so the walk always ends.  The walk reads LOOKBACK_BATCH predecessors per
// round (independent loads in flight) and consumes them in order, stopping at
// the first that is not yet published; long chains of aggregates therefore
// cost one L2 round trip per batch, not per tile.  Every wait is bounded:
// when it runs out the kernel records ERR_TIMEOUT and goes on with a wrong
// (but finite) value.
constexpr int LOOKBACK_BATCH = 16;
__device__ __forceinline__ bool st_ready(u64 s, u32 epoch) {
    return (u32)(s >> 34) == (epoch & EPOCH_MASK) && ((u32)(s >> 32) & 3u);
}
__device__ __forceinline__ u32 lookback_u32(const u64* status, int C, int c, u32 t, u32 chain_first,
                                            u32 epoch, Ctl* ctl, u32 where) {
    u32 excl = 0;
    u32 u = t;  // tiles [u, t) are consumed
    u32 spins = 0;
    while (u > chain_first) {
        u64 s[LOOKBACK_BATCH];
        const u32 avail = u - chain_first;
#pragma unroll
        for (int j = 0; j < LOOKBACK_BATCH; ++j)
            s[j] = (u32)j < avail ? st_load(status + (u64)(u - 1 - j) * (u64)C + (u64)c) : 0ull;
        u32 used = 0;
        bool done = false;
#pragma unroll
        for (int j = 0; j < LOOKBACK_BATCH; ++j) {
            if (done || (u32)j >= avail || used != (u32)j) continue;
            if (!st_ready(s[j], epoch)) continue;
            excl += (u32)s[j];
            used = j + 1;
            if (((u32)(s[j] >> 32) & 3u) == ST_PREFIX) done = true;
        }
        if (done) break;
        u -= used;
        if (used == 0) {
            if (++spins > SPIN_LIMIT || ((spins & 255u) == 0 && timed_out(ctl))) {
                atomicOr(&ctl->error, ERR_TIMEOUT);
                ctl->timeout_where = where;
                return excl;
            }
            if (spins > 64) __nanosleep(256);
        }
    }
    return excl;
}

// ---------------------------------------------------------------------
// checked build (compiled with DOMAGG_CHECKED): every computed index the
// kernels store through or load from is tested against its buffer; a miss
// records which site it was in a per-translation-unit device flag, the
// access is skipped, and the host reports DOMAGG_ERR_BOUNDS.  Nothing traps.
// domagg_check(ok, site) guards an access that the product build bounds as
// well (it returns ok); DOMAGG_GUARD(ok, site) adds a test that the product
// build leaves out (it is `true` there).
// ---------------------------------------------------------------------
enum : u32 {
    SITE_EXPAND = 1, SITE_SORT_SCATTER = 2, SITE_SORT_LOCAL = 3, SITE_SEGSCAN_PARTIAL = 4, SITE_REDUCE = 5,
    SITE_GROUP_OUT = 6, SITE_GROUP_SPLIT = 7, SITE_GROUP_NODE = 8, SITE_GROUP_VAL = 9, SITE_RANK = 10,
    SITE_WAVELET_OUT = 11, SITE_WAVELET_EL = 12, SITE_SEGSCAN_TILE = 13, SITE_COUNT_CHUNK = 14
};
#ifdef DOMAGG_CHECKED
static __device__ u32 g_bounds_hit;    // one per translation unit
static __device__ u32 g_bounds_site;
__device__ __forceinline__ bool domagg_check(bool ok, u32 site) {
    if (!ok) {
        atomicOr(&g_bounds_hit, 1u);
        g_bounds_site = site;
    }
    return ok;
}
#define DOMAGG_GUARD(ok, site) domagg::domagg_check((ok), (site))
#else
__device__ __forceinline__ bool domagg_check(bool ok, u32) { return ok; }
#define DOMAGG_GUARD(ok, site) true
#endif

// ---------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------
__device__ __forceinline__ u32 lanemask_lt() {
    u32 r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Lanes of the warp whose 8-bit digit equals this lane's, among the lanes in
// `valid` (all lanes call it).  Built from one ballot per digit bit: the
// hardware match instruction has a far lower throughput than ballots.
__device__ __forceinline__ u32 match_digit8(u32 d, u32 valid) {
    u32 m = valid;
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
        const u32 set = (d >> bit) & 1u;
        const u32 bal = __ballot_sync(0xffffffffu, set);
        m &= set ? bal : ~bal;
    }
    return m;
}

// Adds one count for digit d (if valid) to a per-warp histogram h.  Lanes that
// share lane 0's digit are added together (one atomic), which removes the
// contention of skewed digit distributions where one digit dominates; the
// other lanes add one each.
__device__ __forceinline__ void warp_hist_add(u32* h, u32 d, bool valid, u32 lane) {
    const u32 d0 = __shfl_sync(0xffffffffu, d, 0);
    const bool same = valid && d == d0;
    const u32 grp = __ballot_sync(0xffffffffu, same);
    if (valid && !same) atomicAdd(&h[d], 1u);
    else if (same && lane == (u32)(__ffs(grp) - 1)) atomicAdd(&h[d0], (u32)__popc(grp));
}

// Transpose of the warp's 32x32 bit matrix (lane l holds row l): returns the
// lane's column, whose bit k is bit `lane` of lane k's row.  Five rounds that
// swap off-diagonal blocks of 16, 8, 4, 2, 1 bits.
__device__ __forceinline__ u32 warp_transpose32(u32 row, u32 lane) {
    const u32 masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const u32 j = 16u >> s, m = masks[s];
        const u32 x = __shfl_xor_sync(0xffffffffu, row, j);
        row = (lane & j) ? ((row & ~m) | ((x & ~m) >> j)) : ((row & m) | ((x & m) << j));
    }
    return row;
}

// Index of the last entry of the non-decreasing array a[0..n) that is <= x
// (a[0] <= x is assumed).
__device__ __forceinline__ int upper_index(const u32* a, int n, u32 x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(a + mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Padded shared-memory index: one spare element per 32, so that reading a
// tile in blocked order (thread t takes elements t*ITEMS ..) and in striped
// order are both free of bank conflicts.
__device__ __forceinline__ u32 pidx(u32 x) { return x + (x >> 5); }
template <int N>
struct Padded {
    static constexpr int value = N + N / 32 + 1;
};

// Mask of the low b bits (b <= 32).
__device__ __forceinline__ u32 low_mask(u32 b) { return b >= 32 ? 0xffffffffu : ((1u << b) - 1u); }

// Canonical range-tree node of the prefix that ends just above bit j of the
// b-digit rank r (Sec. 3): the prefix v = r >> (j+1) of length b-1-j is
// encoded as (v << (j+1)) | (1 << j), i.e. r with bit j set and the bits below
// it cleared.  The encoding is injective over all (length, prefix) pairs and
// stays below 2^b.  A data point emits it for the 0-digits of its rank (P0),
// a query for the 1-digits (P1).
__device__ __forceinline__ u32 node_of(u32 r, u32 j) { return ((r >> j) | 1u) << j; }

// ---------------------------------------------------------------------
// TMA bulk copies into shared memory, completed on an mbarrier
// ---------------------------------------------------------------------
__device__ __forceinline__ u32 smem_addr(const void* p) { return (u32)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy; both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ u64 globaltimer_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for phase `parity` of an mbarrier: at most MBAR_WAIT_NS of
// wall time (checked every 1024 polls) and MBAR_SPIN_LIMIT polls, and it
// gives up at once when another wait of the pipeline already ran out.
// Returns false (and records ERR_TIMEOUT) if the phase did not complete.
constexpr u32 MBAR_SPIN_LIMIT = 1u << 22;
constexpr u64 MBAR_WAIT_NS = 1000000000ull;
__device__ __forceinline__ bool mbar_wait_bounded(u64* bar, u32 parity, Ctl* ctl, u32 where) {
    u64 t0 = 0;
    for (u32 i = 0; i < MBAR_SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 1023u) {
            const u64 now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > MBAR_WAIT_NS) break;
            if (timed_out(ctl)) break;
        }
    }
    atomicOr(&ctl->error, ERR_TIMEOUT);
    ctl->timeout_where = where;
    return false;
}

// ---------------------------------------------------------------------
// float-float arithmetic (error-free transformations, Knuth's TwoSum)
// ---------------------------------------------------------------------
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
// x + y without the final renormalisation (a cascaded sum): hi carries the
// rounded sum, lo the exact rounding errors plus both low parts.  Used only
// for short runs (a thread's few items, a query's few levels) whose pairs
// then enter ff_add, so lo stays tiny against the sum of the magnitudes.
__device__ __forceinline__ ff ff_add_cascade(ff x, ff y) {
    const ff s = ff_two_sum(x.hi, y.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = ff_two_sum(x.hi, y.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return ff_fast_two_sum(s.hi, lo);
}

// ---------------------------------------------------------------------
// aggregation operators F with unit e (Sec. 1)
// ---------------------------------------------------------------------
// Each operator defines: Acc (scan accumulator), Part (stored partial), Out
// (output element), Pay (32-bit record payload), W (a weight as stored in
// the order of the last coordinate), e(), F(a, b), Fc(a, b) (F for short
// runs: for float-float sums without renormalisation), to_part, from_part,
// to_out, from_out (an output read back as an accumulator: the shared-memory
// levels' result, completed by the records' levels), and either from_pay (the
// payload is the weight's bits) or, with
// GATHER, from_w (the payload is the position of the weight, read from the
// L2-resident weight array: 8-byte weights do not ride through the sort).
struct OpSumF32 {
    typedef ff Acc;
    typedef float Part;
    typedef float Out;
    typedef u32 Pay;
    typedef u32 W;
    static constexpr bool GATHER = false;
    __device__ static Acc e() { return {0.f, 0.f}; }
    __device__ static Acc from_pay(Pay p) { return {__uint_as_float(p), 0.f}; }
    __device__ static Acc F(Acc a, Acc b) { return ff_add(a, b); }
    __device__ static Acc Fc(Acc a, Acc b) { return ff_add_cascade(a, b); }
    __device__ static Part to_part(Acc a) { return __fadd_rn(a.hi, a.lo); }
    __device__ static Acc from_part(Part p) { return {p, 0.f}; }
    __device__ static Out to_out(Acc a) { return __fadd_rn(a.hi, a.lo); }
    __device__ static Acc from_out(Out o) { return {o, 0.f}; }
};
struct OpSumI64 {
    typedef long long Acc;
    typedef long long Part;
    typedef long long Out;
    typedef u32 Pay;  // a data record carries the position of its weight (GATHER)
    typedef u64 W;
    static constexpr bool GATHER = true;
    __device__ static Acc e() { return 0; }
    __device__ static Acc from_w(W w) { return (long long)w; }
    __device__ static Acc F(Acc a, Acc b) { return (long long)((u64)a + (u64)b); }
    __device__ static Acc Fc(Acc a, Acc b) { return F(a, b); }
    __device__ static Part to_part(Acc a) { return a; }
    __device__ static Acc from_part(Part p) { return p; }
    __device__ static Out to_out(Acc a) { return a; }
    __device__ static Acc from_out(Out o) { return o; }
};
struct OpMaxI32 {
    typedef int Acc;
    typedef int Part;
    typedef int Out;
    typedef u32 Pay;
    typedef u32 W;
    static constexpr bool GATHER = false;
    __device__ static Acc e() { return (int)0x80000000; }
    __device__ static Acc from_pay(Pay p) { return (int)p; }
    __device__ static Acc F(Acc a, Acc b) { return a > b ? a : b; }
    __device__ static Acc Fc(Acc a, Acc b) { return F(a, b); }
    __device__ static Part to_part(Acc a) { return a; }
    __device__ static Acc from_part(Part p) { return p; }
    __device__ static Out to_out(Acc a) { return a; }
    __device__ static Acc from_out(Out o) { return o; }
};
struct OpMaxF32 {
    typedef float Acc;
    typedef float Part;
    typedef float Out;
    typedef u32 Pay;
    typedef u32 W;
    static constexpr bool GATHER = false;
    __device__ static Acc e() { return -__int_as_float(0x7f800000); }
    __device__ static Acc from_pay(Pay p) { return __uint_as_float(p); }
    __device__ static Acc F(Acc a, Acc b) { return fmaxf(a, b); }
    __device__ static Acc Fc(Acc a, Acc b) { return F(a, b); }
    __device__ static Part to_part(Acc a) { return a; }
    __device__ static Acc from_part(Part p) { return p; }
    __device__ static Out to_out(Acc a) { return a; }
    __device__ static Acc from_out(Out o) { return o; }
};
struct OpMinI32 {
    typedef int Acc;
    typedef int Part;
    typedef int Out;
    typedef u32 Pay;
    typedef u32 W;
    static constexpr bool GATHER = false;
    __device__ static Acc e() { return 0x7fffffff; }
    __device__ static Acc from_pay(Pay p) { return (int)p; }
    __device__ static Acc F(Acc a, Acc b) { return a < b ? a : b; }
    __device__ static Acc Fc(Acc a, Acc b) { return F(a, b); }
    __device__ static Part to_part(Acc a) { return a; }
    __device__ static Acc from_part(Part p) { return p; }
    __device__ static Out to_out(Acc a) { return a; }
    __device__ static Acc from_out(Out o) { return o; }
};
struct OpMinF32 {
    typedef float Acc;
    typedef float Part;
    typedef float Out;
    typedef u32 Pay;
    typedef u32 W;
    static constexpr bool GATHER = false;
    __device__ static Acc e() { return __int_as_float(0x7f800000); }
    __device__ static Acc from_pay(Pay p) { return __uint_as_float(p); }
    __device__ static Acc F(Acc a, Acc b) { return fminf(a, b); }  // a NaN weight never wins
    __device__ static Acc Fc(Acc a, Acc b) { return F(a, b); }
    __device__ static Part to_part(Acc a) { return a; }
    __device__ static Acc from_part(Part p) { return p; }
    __device__ static Out to_out(Acc a) { return a; }
    __device__ static Acc from_out(Out o) { return o; }
};
struct OpCount {
    typedef u32 Acc;
    typedef u32 Part;
    typedef long long Out;
    typedef u32 Pay;
    typedef u32 W;
    static constexpr bool GATHER = false;
    __device__ static Acc e() { return 0u; }
    __device__ static Acc from_pay(Pay) { return 1u; }
    __device__ static Acc F(Acc a, Acc b) { return a + b; }
    __device__ static Acc Fc(Acc a, Acc b) { return F(a, b); }
    __device__ static Part to_part(Acc a) { return a; }
    __device__ static Acc from_part(Part p) { return p; }
    __device__ static Out to_out(Acc a) { return (long long)a; }
    __device__ static Acc from_out(Out o) { return (u32)o; }
};

}  // namespace domagg
