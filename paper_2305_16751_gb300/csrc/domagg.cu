// domagg.cu -- the C ABI (include/domagg.h) and the host orchestration of the
// pipeline: point phase (keys, ranks, order of the last coordinate, count /
// offset scan), one device->host read of the record counts, then per chunk of
// instances the record phase (flat map, records sort, segmented scan,
// per-query reduction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/domagg.h"
#include "host_common.h"
#include "k_points.cuh"
#include "k_radix.cuh"
#include "k_group.cuh"
#include "k_group3.cuh"
#include "k_records.cuh"
#include "k_top.cuh"
#include "k_wavelet.cuh"

using namespace domagg;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Sub-allocator over one buffer; a first pass with base == nullptr measures.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T>
    T* take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T* r = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T) + 64;  // slack: 16-byte-aligned bulk reads may run past the end
        return r;
    }
};

constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 16;  // rank and count scan
// segmented scan tiles: threads per block, items per thread for 8-byte records
#ifndef DOMAGG_SEG_THREADS
#define DOMAGG_SEG_THREADS 256
#endif
#ifndef DOMAGG_SEG_ITEMS_NARROW
#define DOMAGG_SEG_ITEMS_NARROW 16
#endif
static_assert(SCAN_THREADS * SCAN_ITEMS == (int)POINT_TILE, "point scan tiles");

}  // namespace

struct domagg_ctx {
    int device = 0;
    size_t max_ws = 0;
    Ctl* ctl = nullptr;
    DevBuf pts, recs, st_multi, st_seg, stage;
    DevBuf st_wv;  // look-back records of the level-wise passes (their own layout)
    void* h_pin = nullptr;
    size_t h_pin_cap = 0;
    std::string err;
    domagg_stats stats{};
    bool timing = false;
    std::vector<TimedLaunch> log;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    u64 epoch_mirror = 0;  // host copy of Ctl::epoch_base
    bool frozen = false;   // owned by a plan: its workspace must not grow any more
    bool no_alloc = false; // buffers are fixed slices of a static array: never free or allocate
    int sms = 152;         // multiprocessors of the device
    // the point phase's independent sorts run on two more streams (fork /
    // join by events); off for the allocation-free entry point
    bool overlap = false;
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
    // domagg_forward_host: the weights' copy runs on its own stream beside
    // the point phase (nothing reads them before the count scan); the
    // pipeline's stream waits for ev_w there while w_pending
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_w = nullptr;
    bool w_pending = false;
    // the last unplanned run's records through HBM per (instance, level)
    std::vector<u32> meas_lvl;
    int ranges_per_cta = 4, blocks_per_sm = 16;  // launch shapes (domagg_plan_autotune)
    // m = 2: the rank levels below gS <= group_bits are aggregated per group
    // in shared memory (k_group); 0 = every level through the records in HBM
    int group_bits = GROUP_MAX_BITS;
    // m = 2: the top top_bits rank levels (at most 2^(top_bits-1) nodes
    // each) per tile in shared memory (k_top); 0 = every level from gS up
    // through the records in HBM
    int top_bits = TOP_MAX_BITS;
    // windows of the rank scatter (0: about 48 MB of ranks each)
    int rank_windows = 0;

    size_t held() const { return pts.cap + recs.cap + st_multi.cap + st_seg.cap + stage.cap + st_wv.cap; }
};

namespace {

domagg_status fail(domagg_ctx* h, domagg_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

domagg_status cuda_fail(domagg_ctx* h, cudaError_t e, const char* where) {
    return fail(h, DOMAGG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Grows a device buffer to at least `bytes` (contents are not kept).  Status
// buffers are zeroed when (re)allocated: fresh memory may hold old data of
// this process, and a stale word must never look like a status of the
// current epoch.
domagg_status grow(domagg_ctx* h, DevBuf& b, size_t bytes, bool zero = false) {
    if (b.cap >= bytes) return DOMAGG_OK;
    if (h->no_alloc) return fail(h, DOMAGG_ERR_OOM, "the fixed scratch is too small for this input");
    if (h->frozen) return fail(h, DOMAGG_ERR_OOM, "a planned run needs more workspace than its plan reserved");
    size_t want = std::max(bytes, b.cap + b.cap / 4);
    if (h->max_ws && h->held() - b.cap + want > h->max_ws) {
        want = bytes;
        if (h->held() - b.cap + want > h->max_ws)
            return fail(h, DOMAGG_ERR_OOM, "workspace would exceed max_workspace_bytes");
    }
    if (b.p) {
        cudaFree(b.p);  // waits for the device
        b.p = nullptr;
        b.cap = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(h, DOMAGG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
        want = bytes;
    }
    b.cap = want;
    if (zero) {
        e = cudaMemset(b.p, 0, want);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();  // ordered before any stream's next kernel
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemset of status words");
    }
    return DOMAGG_OK;
}

domagg_status grow_pinned(domagg_ctx* h, size_t bytes) {
    if (h->h_pin_cap >= bytes) return DOMAGG_OK;
    if (h->no_alloc) return fail(h, DOMAGG_ERR_OOM, "the fixed host staging area is too small for this input");
    if (h->frozen) return fail(h, DOMAGG_ERR_OOM, "a planned run needs more pinned memory than its plan reserved");
    if (h->h_pin) {
        cudaDeviceSynchronize();
        cudaFreeHost(h->h_pin);
        h->h_pin = nullptr;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMallocHost(&h->h_pin, want);
    if (e != cudaSuccess) {
        h->h_pin_cap = 0;
        return cuda_fail(h, e, "cudaMallocHost");
    }
    h->h_pin_cap = want;
    return DOMAGG_OK;
}

// Checked build: the site of the first out-of-range index any kernel met
// (this translation unit's and sort.cu's flags), 0 if none; cleared.
u32 bounds_site(bool clear) {
#ifdef DOMAGG_CHECKED
    u32 hit = 0, site = 0;
    cudaMemcpyFromSymbol(&hit, g_bounds_hit, sizeof(u32));
    cudaMemcpyFromSymbol(&site, g_bounds_site, sizeof(u32));
    if (clear && hit) {
        const u32 z = 0;
        cudaMemcpyToSymbol(g_bounds_hit, &z, sizeof(u32));
    }
    cudaGetLastError();
    const u32 mine = hit ? (site ? site : 1u) : 0u;
    const u32 sorts = bounds_site_sort(clear);
    return mine ? mine : sorts;
#else
    (void)clear;
    return 0u;
#endif
}

domagg_status bounds_error(domagg_ctx* h, u32 site) {
    return fail(h, DOMAGG_ERR_BOUNDS, "checked build: an index out of range was caught (site " + std::to_string(site) + ")");
}

domagg_status device_error(domagg_ctx* h, u32 bits) {
    if (bits & ERR_NAN) return fail(h, DOMAGG_ERR_NAN, "a coordinate is NaN");
    if (bits & ERR_OVERFLOW) return fail(h, DOMAGG_ERR_UNSUPPORTED, "more than 2^32 flat-map records");
    if (bits & ERR_TIMEOUT) return fail(h, DOMAGG_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (bits & ERR_EPOCH) return fail(h, DOMAGG_ERR_TIMEOUT, "look-back epoch counter wrapped");
    if (bits & ERR_CAPACITY) return fail(h, DOMAGG_ERR_OOM, "more records than the plan reserved (outputs undefined)");
    return DOMAGG_OK;
}

template <class Op>
struct OpTraits;
template <>
struct OpTraits<OpSumF32> {
    static constexpr int WT = 2;
};
template <>
struct OpTraits<OpSumI64> {
    static constexpr int WT = 1;
};
template <>
struct OpTraits<OpMaxI32> {
    static constexpr int WT = 0;
};
template <>
struct OpTraits<OpMaxF32> {
    static constexpr int WT = 2;
};
template <>
struct OpTraits<OpMinI32> {
    static constexpr int WT = 0;
};
template <>
struct OpTraits<OpMinF32> {
    static constexpr int WT = 2;
};
template <>
struct OpTraits<OpCount> {
    static constexpr int WT = 3;
};

// Resets the look-back epoch and the status words when the epoch counter
// approaches its 30-bit limit.
void maybe_reset_epochs(domagg_ctx* h, cudaStream_t s) {
    if (h->epoch_mirror + 8 * MAX_LAUNCHES < EPOCH_MASK) return;
    if (h->st_multi.p) cudaMemsetAsync(h->st_multi.p, 0, h->st_multi.cap, s);
    if (h->st_seg.p) cudaMemsetAsync(h->st_seg.p, 0, h->st_seg.cap, s);
    if (h->st_wv.p) cudaMemsetAsync(h->st_wv.p, 0, h->st_wv.cap, s);
    cudaMemsetAsync(&h->ctl->epoch_base, 0, sizeof(u32), s);
    h->epoch_mirror = 0;
}

// A record chunk of a planned batch: whole instances [k0, k1) whose records
// get a fixed capacity, laid out on the device (k_layout) instead of on the
// host, so a planned run never reads a count back.
struct PlannedChunk {
    int k0 = 0, k1 = 0;
    u64 T_cap = 0, Tq_cap = 0;  // reserved records of class 0 and query records (>= 1)
    u64 T1_cap = 0;             // reserved records of class 1 (m >= 3)
    int nslot = 0;              // segment slots: every instance's largest possible level count
    int nslot0 = 0;             // slots of class 0 (listed first); the rest are class 1 (32-bit keys, m >= 3)
    int key_bits = 0, key_bits1 = 0;  // bounds on the node-key bits of the two classes
    u32* d_slot_map = nullptr;  // device [nslot]: (instance - k0) << 5 | level
    u32* d_nmask = nullptr;     // device [k1 - k0]: class-1 levels of every instance (m >= 3)
};

// ---------------------------------------------------------------------------
// the pipeline for instances with the same m
// ---------------------------------------------------------------------------
// With `planned`, the run takes its record chunks and capacities from a plan
// and neither synchronises, allocates, copies from the host nor changes a
// kernel attribute (it may be captured in a CUDA graph); the point tables were
// uploaded by the plan's earlier runs and are still in place.
// The level-wise formulation (m <= 2, one instance), after the point
// phase: the passes of k_wavelet_pass over the first coordinate's rank bits,
// two levels per pass from the top (one in the last pass when the bit count
// is odd).  One synchronisation reads the rank bits.
template <int M, class Op>
domagg_status run_wavelet(domagg_ctx* h, std::vector<Inst>& inst, Inst* d_inst, const u32* perm, const u32* r0,
                          u64 N, Launcher& L, cudaStream_t stream, char* hp, size_t ctl_pos) {
    typedef typename Op::Acc Acc;
    if (inst.size() != 1 || !hp) return fail(h, DOMAGG_ERR_UNSUPPORTED, "the level-wise formulation takes one problem");
    Inst* h_inst = (Inst*)hp;
    Ctl* h_ctl = (Ctl*)(hp + ctl_pos);
    L.start(KIND_D2H, 0.0);
    cudaMemcpyAsync(h_inst, d_inst, sizeof(Inst), cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream);
    L.stop();
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "point phase");
    if (h_ctl->error) {
        const u32 bits = h_ctl->error;
        cudaMemsetAsync(&h->ctl->error, 0, sizeof(u32), stream);
        cudaStreamSynchronize(stream);
        return device_error(h, bits);
    }
    inst[0] = h_inst[0];
    // m = 1: the rank is the role bit (every datum below every query)
    u32 b = M == 1 ? 1u : inst[0].b[0];
    if (b == 0) b = 1;  // a single rank: one pass, every output e
    if (b > 31) return fail(h, DOMAGG_ERR_UNSUPPORTED, "ranks of more than 31 bits");
    WvPasses ps;
    ps.n = 0;
    for (u32 top = b; top > 0;) {
        const u32 w = top >= 2 ? 2u : 1u;
        ps.shift[ps.n] = top - w;
        ps.width[ps.n] = w;
        ++ps.n;
        top -= w;
    }
    if (ps.n > WV_HIST_PASSES) return fail(h, DOMAGG_ERR_UNSUPPORTED, "too many level-wise passes");
    const u64 ntiles = (N + WV_TILE - 1) / WV_TILE;
    auto carve = [&](Carver& c, void** R) {
        R[0] = c.take<WElem>(N);
        R[1] = c.take<WElem>(N);
        R[2] = c.take<u32>(WV_MAX_PASSES * 4);
    };
    void* R[3];
    {
        Carver c(nullptr);
        carve(c, R);
        domagg_status st = grow(h, h->recs, c.off);
        if (st) return st;
        Carver c2(h->recs.p);
        carve(c2, R);
        st = grow(h, h->st_wv, (size_t)ntiles * sizeof(WvStatus<Acc>), true);
        if (st) return st;
    }
    WElem* el[2] = {(WElem*)R[0], (WElem*)R[1]};
    u32* hist = (u32*)R[2];
    maybe_reset_epochs(h, stream);
    L.start(KIND_SMALL, 0.0);
    k_begin<<<1, 64, 0, stream>>>(h->ctl);
    L.stop();
    h->epoch_mirror += MAX_LAUNCHES;
    L.next_lookback = 0;
    cudaMemsetAsync(hist, 0, sizeof(u32) * WV_MAX_PASSES * 4, stream);
    L.start(KIND_SMALL, (double)N * 4);
    k_wavelet_hist<M><<<(unsigned)((N + 4095) / 4096), 256, 0, stream>>>(r0, d_inst, (u32)N, ps, hist);
    L.stop();
    const double wbytes = Op::GATHER ? 8.0 : (std::is_same<Op, OpCount>::value ? 0.0 : 4.0);
    const double obytes = (double)sizeof(typename Op::Out);
    int cur = 0;
    for (int p = 0; p < ps.n; ++p) {
        const bool first = p == 0, last = p == ps.n - 1;
        const double bytes = (first ? (double)N * (M == 1 ? 4.0 : 8.0) + (double)inst[0].nD * wbytes
                                    : (double)N * sizeof(WElem)) +
                             (last ? (double)inst[0].nQ * obytes : (double)N * sizeof(WElem));
        const int li = L.lookback_index();
        L.start(KIND_WAVELET, bytes);
        auto* st = (WvStatus<Acc>*)h->st_wv.p;
        if (ps.width[p] == 2)
            k_wavelet_pass<Op, 2, M><<<(unsigned)ntiles, WV_THREADS, 0, stream>>>(
                el[cur], el[cur ^ 1], perm, r0, d_inst, (u32)N, ps.shift[p], first, last, hist + 4 * p, st, h->ctl, li);
        else
            k_wavelet_pass<Op, 1, M><<<(unsigned)ntiles, WV_THREADS, 0, stream>>>(
                el[cur], el[cur ^ 1], perm, r0, d_inst, (u32)N, ps.shift[p], first, last, hist + 4 * p, st, h->ctl, li);
        L.stop();
        cur ^= 1;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "launch");
    if (L.next_lookback > MAX_LAUNCHES) return fail(h, DOMAGG_ERR_UNSUPPORTED, "too many look-back launches");
    domagg_stats& S = h->stats;
    S.n_points = (int64_t)N;
    S.n_records = 0;
    S.n_records_shared = 0;
    S.n_query_records = 0;
    S.m = M;
    for (int i = 0; i < 3; ++i) {
        S.rank_bits[i] = (i < M - 1) ? (int32_t)inst[0].b[i] : 0;
        S.distinct[i] = (i < M - 1) ? (int64_t)inst[0].U[i] : 0;
    }
    S.record_key_bits = (int)b;
    S.record_passes = ps.n;
    S.workspace_bytes = (int64_t)h->held();
    return DOMAGG_OK;
}

template <int M, class Op, bool F32>
domagg_status run(domagg_ctx* h, std::vector<Inst>& inst, bool negate, cudaStream_t stream,
                  const std::vector<PlannedChunk>* planned = nullptr) {
    typedef typename std::conditional<M >= 3, u64, u32>::type K;
    typedef typename Op::Pay Pay;  // 32 bits: the weight's bits, a weight position (GATHER) or a slot
    typedef typename Op::W W;      // a weight in the order of the last coordinate
    typedef typename Op::Part Part;
    constexpr int WT = OpTraits<Op>::WT;
    constexpr int SEG_ITEMS = (sizeof(K) + sizeof(Pay) == 8) ? DOMAGG_SEG_ITEMS_NARROW : 8;
    constexpr int SEG_THREADS = DOMAGG_SEG_THREADS;
    constexpr u32 SEG_TILE = SEG_THREADS * SEG_ITEMS;
    constexpr int SEG_ITEMS1 = (4 + sizeof(Pay) == 8) ? DOMAGG_SEG_ITEMS_NARROW : 8;  // class 1: 32-bit keys
    constexpr u32 SEG_TILE1 = SEG_THREADS * SEG_ITEMS1;
    const int k = (int)inst.size();

    // ---- host-side layout of the point space
    std::vector<u32> pt_offs(k + 1), q_offs(k + 1), chunk_off(k + 1);
    std::vector<u64> pt_sizes(k);
    u64 N = 0, NQ = 0, ntp = 0, NC = 0;
    for (int s = 0; s < k; ++s) {
        pt_offs[s] = (u32)N;
        q_offs[s] = (u32)NQ;
        chunk_off[s] = (u32)NC;
        inst[s].pt_off = (u32)N;
        inst[s].q_off = (u32)NQ;
        for (int i = 0; i < 3; ++i) inst[s].U[i] = inst[s].b[i] = 0;
        inst[s].T = inst[s].Tq = inst[s].rec_off = inst[s].qrec_off = inst[s].key_bits = 0;
        const u64 n = (u64)inst[s].nD + inst[s].nQ;
        pt_sizes[s] = n;
        N += n;
        NQ += inst[s].nQ;
        NC += (n + 31) / 32;
        ntp += (n + POINT_TILE - 1) / POINT_TILE;
    }
    pt_offs[k] = (u32)N;
    q_offs[k] = (u32)NQ;
    chunk_off[k] = (u32)NC;
    if (N >= (1ull << 31)) return fail(h, DOMAGG_ERR_UNSUPPORTED, "more than 2^31 points in one call");
    if (NQ == 0) return DOMAGG_OK;
    // m = 2, 3, the records path: the deep rank levels go through k_group
    // (m = 2) or k_group3 (m = 3)
    const bool use_groups = (M == 2 || M == 3) && h->group_bits > 0 && !(inst[0].flags & FLAG_WAVELET);
    // m = 2: the top rank levels per range of whole tiles (k_top): about
    // TOP_RANGES_PER_SM ranges per SM over all points (a function of the
    // sizes alone: a planned run reuses the table its measuring run
    // uploaded); prange_off[s] is instance s's first range; `multi` lists the
    // instances of two or more ranges
    const bool use_top = M == 2 && h->top_bits > 0 && !(inst[0].flags & FLAG_WAVELET);
    u32 range_pts = TOP_TILE;
    std::vector<u32> prange_off(k + 1, 0), multi;
    if (use_top) {
        const u64 want = (u64)TOP_RANGES_PER_SM * (u64)std::max(h->sms, 1);
        const u64 tiles = (N + TOP_TILE - 1) / TOP_TILE;
        range_pts = (u32)std::min<u64>(TOP_TILE * std::max<u64>(1, (tiles + want - 1) / want), 1ull << 30);
        u64 nr = 0;
        for (int s = 0; s < k; ++s) {
            prange_off[s] = (u32)nr;
            const u64 r = (pt_sizes[s] + range_pts - 1) / range_pts;
            if (r >= 2) multi.push_back((u32)s);
            nr += r;
        }
        prange_off[k] = (u32)nr;
    }
    const u64 nranges = prange_off[k];

    // ---- point workspace
    auto carve_points = [&](Carver& c, void** P) {
        P[0] = c.take<Inst>(k);
        P[1] = c.take<u32>(k + 1);  // pt_offs
        P[2] = c.take<u32>(k + 1);  // q_offs
        P[3] = c.take<u32>(k + 1);  // point tiles
        P[4] = c.take<u32>(N);      // rk0
        P[5] = c.take<u32>(M >= 3 ? N : 0);  // rk1
        P[6] = c.take<u32>(N);      // lk
        P[7] = c.take<u32>(N);      // key alt
        P[8] = c.take<u32>(N);      // vA
        P[9] = c.take<u32>(N);      // vB
        P[10] = c.take<u32>(M >= 2 ? N : 0);  // r0
        P[11] = c.take<u32>(M >= 3 ? N : 0);  // r1
        P[12] = c.take<u32>(M >= 2 ? N : 0);  // pr0
        P[13] = c.take<u32>(M >= 3 ? N : 0);  // pr1
        P[14] = c.take<u32>(N);     // pj
        P[15] = c.take<u32>(k + 1);  // chunk offsets
        P[16] = c.take<u32>((size_t)NC * LMAX);  // query chunk bases per level
        P[17] = c.take<u32>((size_t)k * LMAX);   // query records per (instance, level)
        P[18] = c.take<W>(WT == 3 ? 0 : N);  // weights in the order of the last coordinate
        P[19] = c.take<u32>((size_t)k * 4 * RADIX);  // hist
        P[20] = c.take<u32>((size_t)k * 4 * RADIX);  // digit offsets
        P[21] = c.take<u32>(k + 1);                  // the sorts' tile map
        P[22] = c.take<u32>((size_t)NC * LMAX);      // chunk bases per level
        P[23] = c.take<u32>((size_t)k * LMAX);       // records per (instance, level)
        P[24] = c.take<u32>((size_t)sort_range_bound(pt_sizes) * RADIX);  // first-pass range bases
        P[25] = c.take<u32>((size_t)ntp * CS_COUNTERS);                   // per point tile: rank / flat-map counts
        P[26] = c.take<u32>(M >= 4 ? N : 0);  // rk2
        P[27] = c.take<u32>(M >= 4 ? N : 0);  // r2
        P[28] = c.take<u32>(M >= 4 ? N : 0);  // pr2
        // scratch of the sorts that run beside the first (chain 1: the last
        // coordinate; chain 2: the second rank coordinate), when overlapping
        for (int ch = 1; ch <= 2; ++ch) {
            const bool used = h->overlap && (ch == 1 || M >= 3);
            const u64 n = used ? N : 0, kk = used ? (u64)k : 0;
            P[29 + (ch - 1) * 8 + 0] = c.take<u32>(n);                                  // key ping-pong
            P[29 + (ch - 1) * 8 + 1] = c.take<u32>(n);                                  // values A
            P[29 + (ch - 1) * 8 + 2] = c.take<u32>(n);                                  // values B
            P[29 + (ch - 1) * 8 + 3] = c.take<u32>(kk + 1);                             // tile map
            P[29 + (ch - 1) * 8 + 4] = c.take<u32>(kk * 4 * RADIX);                     // hist
            P[29 + (ch - 1) * 8 + 5] = c.take<u32>(kk * 4 * RADIX);                     // digit offsets
            P[29 + (ch - 1) * 8 + 6] = c.take<u32>(used ? (size_t)sort_range_bound(pt_sizes) * RADIX : 0);
            P[29 + (ch - 1) * 8 + 7] = c.take<u32>(used ? (size_t)ntp : 0);             // rank tile counts
        }
        // m = 2, 3 groups: rank starts, the group sort's keys and values
        // (ping-pong), per-instance group-id bits and group slots
        const bool grp = use_groups;
        P[45] = c.take<u32>(grp ? N + k : 0);    // rank starts
        P[46] = c.take<u32>(grp ? N : 0);        // group keys
        P[47] = c.take<u32>(grp ? N : 0);
        P[48] = c.take<u64>(grp ? N : 0);        // group values
        P[49] = c.take<u64>(grp ? N : 0);
        P[50] = c.take<u32>(grp ? k : 0);        // group-id bits per instance
        P[51] = c.take<u32>(grp ? k + 1 : 0);    // group slot offsets
        // m = 2 top levels: per query F over its range's top levels, per range
        // F of every top-level node (then the carries), the range table, the
        // instances of several ranges
        P[52] = c.take<typename Op::Acc>(use_top ? N : 0);
        P[53] = c.take<typename Op::Acc>(use_top ? (size_t)nranges * TOP_STRIDE : 0);
        P[54] = c.take<u32>(use_top ? k + 1 : 0);
        P[55] = c.take<u32>(use_top ? std::max<size_t>(multi.size(), 1) : 0);
        // groups: per query (by position in the order of the last
        // coordinate) F over the levels below gS
        P[56] = c.take<typename Op::Part>(grp ? N : 0);
        // groups: this call's groups too large for shared memory (a flag per
        // group, at the instance's point offset); per instance, every
        // record of the flat map (a statistic)
        P[57] = c.take<unsigned char>(grp ? N : 0);
        P[58] = c.take<unsigned long long>(k);
    };
    void* P[59];
    {
        Carver c(nullptr);
        carve_points(c, P);
        domagg_status st = grow(h, h->pts, c.off);
        if (st) return st;
        Carver c2(h->pts.p);
        carve_points(c2, P);
    }
    Inst* d_inst = (Inst*)P[0];
    u32 *d_pt_offs = (u32*)P[1], *d_q_offs = (u32*)P[2], *d_pt_tiles = (u32*)P[3];
    u32 *rk0 = (u32*)P[4], *rk1 = (u32*)P[5], *lk = (u32*)P[6], *kalt = (u32*)P[7];
    u32 *vA = (u32*)P[8], *vB = (u32*)P[9], *r0 = (u32*)P[10], *r1 = (u32*)P[11];
    u32 *pr0 = (u32*)P[12], *pr1 = (u32*)P[13], *pj = (u32*)P[14], *d_chunk_off = (u32*)P[15];
    u32 *rk2 = (u32*)P[26], *r2 = (u32*)P[27], *pr2 = (u32*)P[28];
    u32 *qchunk_base = (u32*)P[16], *qlvl_tot = (u32*)P[17];
    u32 *hist = (u32*)P[19], *digit_off = (u32*)P[20];
    u32* d_sort_tiles = (u32*)P[21];
    u32 *chunk_base = (u32*)P[22], *lvl_tot = (u32*)P[23];
    u32 *rstart = (u32*)P[45], *gkey[2] = {(u32*)P[46], (u32*)P[47]}, *gbits = (u32*)P[50], *gslot = (u32*)P[51];
    u64* gval[2] = {(u64*)P[48], (u64*)P[49]};
    typename Op::Acc* topv = (typename Op::Acc*)P[52];
    typename Op::Part* gacc = (typename Op::Part*)P[56];
    unsigned char* govf = use_groups ? (unsigned char*)P[57] : nullptr;
    unsigned long long* rec_all = (unsigned long long*)P[58];
    typename Op::Acc* top_agg = (typename Op::Acc*)P[53];
    u32 *d_prange = (u32*)P[54], *d_multi = (u32*)P[55];

    // status words: point tiles x 256 digits (the records sort grows it later)
    {
        const u64 nst = std::max<u64>(std::max<u64>(tiles_of(pt_sizes, SORT_MIN_TILE), ntp), 1);
        const int chains = h->overlap ? (M >= 3 ? 3 : 2) : 1;
        domagg_status st = grow(h, h->st_multi, (size_t)nst * RADIX * sizeof(u64) * chains, true);
        if (st) return st;
    }

    // ---- upload the instance table and offsets
    const size_t up_bytes = sizeof(Inst) * k + 3 * sizeof(u32) * (k + 1) + (use_top ? sizeof(u32) * (2 * k + 2) : 0);
    const size_t lvl_pos = (up_bytes + 63) & ~(size_t)63;                          // level totals (read back)
    const size_t rec_pos = (lvl_pos + 2 * sizeof(u32) * k * LMAX + 63) & ~(size_t)63;  // records per instance (read back)
    const size_t ctl_pos = (rec_pos + sizeof(unsigned long long) * k + 63) & ~(size_t)63;  // control block (read back)
    char* hp = nullptr;
    if (!planned) {
        domagg_status st = grow_pinned(h, ctl_pos + sizeof(Ctl) + 64);
        if (st) return st;
        hp = (char*)h->h_pin;
        memcpy(hp, inst.data(), sizeof(Inst) * k);
        memcpy(hp + sizeof(Inst) * k, pt_offs.data(), sizeof(u32) * (k + 1));
        memcpy(hp + sizeof(Inst) * k + sizeof(u32) * (k + 1), q_offs.data(), sizeof(u32) * (k + 1));
        memcpy(hp + sizeof(Inst) * k + 2 * sizeof(u32) * (k + 1), chunk_off.data(), sizeof(u32) * (k + 1));
        cudaMemcpyAsync(d_inst, hp, sizeof(Inst) * k, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(d_pt_offs, hp + sizeof(Inst) * k, sizeof(u32) * (k + 1), cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(d_q_offs, hp + sizeof(Inst) * k + sizeof(u32) * (k + 1), sizeof(u32) * (k + 1),
                        cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(d_chunk_off, hp + sizeof(Inst) * k + 2 * sizeof(u32) * (k + 1), sizeof(u32) * (k + 1),
                        cudaMemcpyHostToDevice, stream);
        if (use_top) {  // (a planned run reuses the tables its measuring run uploaded)
            u32* hr = (u32*)(hp + sizeof(Inst) * k + 3 * sizeof(u32) * (k + 1));
            memcpy(hr, prange_off.data(), sizeof(u32) * (k + 1));
            memcpy(hr + k + 1, multi.data(), sizeof(u32) * multi.size());
            cudaMemcpyAsync(d_prange, hr, sizeof(u32) * (k + 1), cudaMemcpyHostToDevice, stream);
            if (!multi.empty())
                cudaMemcpyAsync(d_multi, hr + k + 1, sizeof(u32) * multi.size(), cudaMemcpyHostToDevice, stream);
        }
        maybe_reset_epochs(h, stream);
    }

    Launcher L;
    L.frozen = h->frozen;  // the first planned run (not yet frozen) sets the kernel attributes
    L.stream = stream;
    L.ctl = h->ctl;
    L.timing = h->timing && !planned;
    L.ranges_per_cta = h->ranges_per_cta;
    L.blocks_per_sm = h->blocks_per_sm;
    L.log = &h->log;
    L.pool = &h->pool;
    L.pool_used = &h->pool_used;

    L.start(KIND_SMALL, 0.0);
    k_begin<<<1, 64, 0, stream>>>(h->ctl);
    L.stop();
    h->epoch_mirror += MAX_LAUNCHES;
    L.start(KIND_SMALL, 0.0);
    k_make_tiles<<<1, 1024, 0, stream>>>(d_pt_offs, k, POINT_TILE, d_pt_tiles);
    L.stop();

    // ---- keys (instruction 0 and 5i-4)
    L.start(KIND_ENCODE, (double)N * M * 4 * 2);
    k_encode<M, F32><<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(d_inst, d_pt_offs, k, (u32)N, rk0, rk1, rk2, lk,
                                                                      negate ? 1 : 0, h->ctl);
    L.stop();

    // ---- the point-phase sorts (5i-3 .. 5i, 5m+i, and the Sec. 5 order of the
    // last coordinate).  They are independent: with overlap, the last
    // coordinate's sort (chain 1) and the second rank coordinate (chain 2)
    // run on their own streams, forked after the keys and joined before the
    // count scan, each with its own scratch and status words.
    const u64 nst_chain = std::max<u64>(std::max<u64>(tiles_of(pt_sizes, SORT_MIN_TILE), ntp), 1) * RADIX;
    struct Chain {
        cudaStream_t stream;
        u32 *kalt, *vA, *vB, *tiles, *hist, *digit, *range, *tile_cnt;
        u64* status;
    };
    auto chain = [&](int ch) -> Chain {
        if (ch == 0 || !h->overlap)
            return Chain{stream, kalt, vA, vB, d_sort_tiles, hist, digit_off, (u32*)P[24], (u32*)P[25],
                         (u64*)h->st_multi.p};
        void** Q = P + 29 + (ch - 1) * 8;
        return Chain{h->aux[ch - 1], (u32*)Q[0], (u32*)Q[1], (u32*)Q[2], (u32*)Q[3], (u32*)Q[4], (u32*)Q[5],
                     (u32*)Q[6], (u32*)Q[7], (u64*)h->st_multi.p + (u64)ch * nst_chain};
    };
    auto rank_dim = [&](int i, const Chain& C) {
        L.stream = C.stream;
        SortSpace sp{d_pt_offs, k, &pt_sizes, C.tiles, C.hist, C.digit, C.status, (double)N, C.range,
                     sort_range_bound(pt_sizes)};
        u32* keys[2] = {i == 0 ? rk0 : (i == 1 ? rk1 : rk2), C.kalt};
        u32* vals[2] = {C.vA, C.vB};
        // only the sorted key sequence matters for dense ranks: any order of equal digits
        const int cur = sort_pairs<u32, u32>(L, sp, keys, vals, true, 32, 0xffffffffu, KIND_HIST_POINTS,
                                             KIND_SORT_POINTS, nullptr, false);
        L.start(KIND_RANK, (double)N * 4);
        k_rank_count<SCAN_THREADS, SCAN_ITEMS><<<(unsigned)ntp, SCAN_THREADS, 0, C.stream>>>(keys[cur], d_pt_offs,
                                                                                          d_pt_tiles, k, C.tile_cnt);
        L.stop();
        L.start(KIND_SMALL, 0.0);
        k_tile_exscan<<<(unsigned)k, 1024, 0, C.stream>>>(d_pt_tiles, k, C.tile_cnt);
        L.stop();
        // the rank scatter in windows of destinations (each about 48 MB of
        // ranks, so the L2 holds a window while its sectors fill)
        const u64 nwin = h->rank_windows > 0 ? (u64)h->rank_windows
                                             : std::max<u64>(1, (N * sizeof(u32) + (48ull << 20) - 1) / (48ull << 20));
        const u64 span = (N + nwin - 1) / nwin;
        for (u64 w = 0; w < nwin; ++w) {
            const u64 lo = w * span, hi = std::min<u64>(N, lo + span);
            if (lo >= hi && w > 0) break;
            L.start(KIND_RANK, (double)N * 8 * (w == 0 ? 1 : 0) + (double)(hi - lo) * 4);
            k_rank_apply<SCAN_THREADS, SCAN_ITEMS><<<(unsigned)ntp, SCAN_THREADS, 0, C.stream>>>(
                keys[cur], vals[cur], d_pt_offs, d_pt_tiles, k, C.tile_cnt, i == 0 ? r0 : (i == 1 ? r1 : r2), d_inst,
                i, (i == 0 && use_groups) ? rstart : nullptr, (u32)lo, (u32)hi);
            L.stop();
        }
    };
    auto last_dim = [&](const Chain& C) -> u32* {  // order of the last coordinate, queries first on ties (Sec. 5)
        L.stream = C.stream;
        SortSpace sp{d_pt_offs, k, &pt_sizes, C.tiles, C.hist, C.digit, C.status, (double)N, C.range,
                     sort_range_bound(pt_sizes)};
        u32* keys[2] = {lk, C.kalt};
        u32* vals[2] = {C.vA, C.vB};
        const int cur = sort_pairs<u32, u32>(L, sp, keys, vals, true, 32, 0xffffffffu, KIND_HIST_POINTS,
                                             KIND_SORT_POINTS);
        return vals[cur];
    };
    u32* perm;
    if (h->overlap) {
        cudaEventRecord(h->ev_fork, stream);
        cudaStreamWaitEvent(h->aux[0], h->ev_fork, 0);
        if (M >= 3) cudaStreamWaitEvent(h->aux[1], h->ev_fork, 0);
        perm = last_dim(chain(1));
        if (M >= 3) rank_dim(1, chain(2));
        if (M >= 2) rank_dim(0, chain(0));
        if (M >= 4) rank_dim(2, chain(0));
        cudaEventRecord(h->ev_join[0], h->aux[0]);
        cudaStreamWaitEvent(stream, h->ev_join[0], 0);
        if (M >= 3) {
            cudaEventRecord(h->ev_join[1], h->aux[1]);
            cudaStreamWaitEvent(stream, h->ev_join[1], 0);
        }
    } else {  // one stream: the rank sorts first, the permutation last (they share buffers)
        for (int i = 0; i < M - 1; ++i) rank_dim(i, chain(0));
        perm = last_dim(chain(0));
    }
    L.stream = stream;
    if (h->w_pending) {  // the weights' host copy (domagg_forward_host), first read below
        cudaStreamWaitEvent(stream, h->ev_w, 0);
        h->w_pending = false;
    }
    if (inst[0].flags & FLAG_WAVELET) {
        if constexpr (M <= 2) return run_wavelet<M, Op>(h, inst, d_inst, perm, r0, N, L, stream, hp, ctl_pos);
        else return fail(h, DOMAGG_ERR_UNSUPPORTED, "the level-wise formulation takes m <= 2");
    }
    // ---- the levels whose records go through HBM (this shard's, and for
    // m = 2 the levels above the groups of ranks that k_group takes)
    L.start(KIND_SMALL, 0.0);
    k_group_plan<M><<<k, 1024, 0, stream>>>(d_inst, use_groups ? rstart : nullptr, use_groups ? gbits : nullptr,
                                            govf, M == 3 ? G3_CAP : GROUP_CAP, use_groups ? h->group_bits : 0,
                                            use_top ? h->top_bits : 0);
    cudaMemsetAsync(rec_all, 0, sizeof(unsigned long long) * k, stream);
    L.stop();
    // ---- count / offset scan of the flat map, per level
    {
        // perm, gathered ranks, ranks / index / weight written in order, weight gathered
        L.start(KIND_COUNT_SCAN, (double)N * (4 + 8.0 * (M - 1) + 4 + (WT == 3 ? 0 : 2.0 * sizeof(W))) +
                                     (double)NC * 8 * LMAX);
        k_count_scan<M, W, WT><<<(unsigned)ntp, 256, 0, stream>>>(
            perm, d_pt_offs, d_pt_tiles, k, d_chunk_off, r0, r1, r2, d_inst, pr0, pr1, pr2, pj, (W*)P[18], chunk_base,
            qchunk_base, (u32*)P[25], use_groups ? gkey[0] : nullptr, use_groups ? gval[0] : nullptr, govf, rec_all);
        L.stop();
        L.start(KIND_SMALL, 0.0);
        k_tile_exscan_counters<<<dim3((unsigned)k, CS_COUNTERS / 32), 1024, 0, stream>>>(
            d_pt_tiles, k, (u32*)P[25], lvl_tot, qlvl_tot, h->ctl);
        L.stop();
    }
    // ---- record chunks: from the counts (one synchronisation) or from the plan
    // Records of m >= 3 come in two key classes: levels whose node keys fit
    // 31 bits (class 1) are sorted and scanned with 32-bit keys, the others
    // (class 0) with 64-bit keys; for m <= 2 every level is class 0 (32-bit
    // keys already).  Each class has its own record arrays and segment table.
    struct Chunk {
        int k0 = 0, k1 = 0;
        u64 T = 0, Tq = 0, nseg = 0;
        u64 T0 = 0, T1 = 0, nseg0 = 0, nseg1 = 0;  // per class (planned: capacities and slots)
        int key_bits = 0, key_bits1 = 0;           // per class
        const u32* slot_map = nullptr;             // planned: the chunk's segment slots (device)
        const u32* nmask = nullptr;                // planned: class-1 levels per instance (device)
    };
    std::vector<Chunk> chunks;
    std::vector<u32> nlev(k), lvl, qlvl;
    u64 T_flat = 0, T_shared = 0;  // flat-map records in all, and those k_group forms in shared memory
    auto level_bits = [&](int s, u32 lv) -> u32 {
        if (M == 1) return 0u;
        const u32 b = inst[s].b[0] - 1u - lv;  // prefix length of level lv
        return b + (M >= 3 ? inst[s].b[1] : 0u) + (M >= 4 ? inst[s].b[2] : 0u);
    };
    auto narrow_level = [&](int s, u32 lv) -> bool { return M >= 3 && level_bits(s, lv) <= 31u; };
    // pinned upload area of every chunk: per instance record and slot bases,
    // per segment offsets and key bits, per (instance, level) segment bases
    auto chunk_upload_words = [&](const Chunk& c) -> size_t {
        const size_t kc = (size_t)(c.k1 - c.k0);
        return 2 * (kc + 1) + (c.nseg0 + 1) + (c.nseg1 + 1) + c.nseg + 2 * kc * LMAX + kc;
    };
    std::vector<size_t> base_pos;
    cudaError_t e = cudaSuccess;
    if (planned) {
        for (const PlannedChunk& pc : *planned) {
            Chunk c;
            c.k0 = pc.k0;
            c.k1 = pc.k1;
            c.T1 = pc.nslot > pc.nslot0 ? pc.T1_cap : 0;
            c.T = pc.T_cap + c.T1;
            c.Tq = pc.Tq_cap;
            c.nseg = (u64)pc.nslot;
            c.nseg0 = (u64)pc.nslot0;
            c.nseg1 = (u64)(pc.nslot - pc.nslot0);
            c.T0 = pc.T_cap;
            c.key_bits = pc.key_bits;
            c.key_bits1 = pc.key_bits1;
            c.slot_map = pc.d_slot_map;
            c.nmask = pc.d_nmask;
            chunks.push_back(c);
        }
    } else {
        // the one synchronisation: record counts and device errors
        Inst* h_inst = (Inst*)hp;
        u32* h_lvl = (u32*)(hp + lvl_pos);
        Ctl* h_ctl = (Ctl*)(hp + ctl_pos);
        L.start(KIND_D2H, 0.0);
        cudaMemcpyAsync(h_inst, d_inst, sizeof(Inst) * k, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(h_lvl, lvl_tot, sizeof(u32) * k * LMAX, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(h_lvl + (size_t)k * LMAX, qlvl_tot, sizeof(u32) * k * LMAX, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(hp + rec_pos, rec_all, sizeof(unsigned long long) * k, cudaMemcpyDeviceToHost, stream);
        cudaMemcpyAsync(h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream);
        L.stop();
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "point phase");
        if (const u32 site = bounds_site(true)) return bounds_error(h, site);
        if (h_ctl->error) {
            const u32 bits = h_ctl->error;
            cudaMemsetAsync(&h->ctl->error, 0, sizeof(u32), stream);
            cudaStreamSynchronize(stream);
            return device_error(h, bits);
        }
        // per instance: its levels, their record counts and sort-key bits
        lvl.assign(h_lvl, h_lvl + (size_t)k * LMAX);
        qlvl.assign(h_lvl + (size_t)k * LMAX, h_lvl + (size_t)2 * k * LMAX);
        const unsigned long long* h_rec = (const unsigned long long*)(hp + rec_pos);
        for (int s = 0; s < k; ++s) {
            inst[s] = h_inst[s];
            nlev[s] = inst[s].nQ + inst[s].nD == 0 ? 0u : (M == 1 ? 1u : inst[s].b[0]);
            // the counts hold the records this call puts through HBM: the
            // levels of this shard that no group (k_group, k_group3: below
            // gS, unless the point's group overflowed) or top-level tile
            // (k_top: from tS up) takes in shared memory
            u64 T = 0, Tq = 0;
            for (u32 lv = 0; lv < nlev[s]; ++lv) {
                T += lvl[(size_t)s * LMAX + lv];
                Tq += qlvl[(size_t)s * LMAX + lv];
            }
            T_flat += h_rec[s];
            T_shared += h_rec[s] - std::min<u64>(h_rec[s], T);
            if (T >= (1ull << 32)) return fail(h, DOMAGG_ERR_UNSUPPORTED, "more than 2^32 flat-map records");
            // the node key (and the role bit above it) must fit 64 bits
            if (M >= 4 && nlev[s] > 0 && inst[s].b[0] - 1u + inst[s].b[1] + inst[s].b[2] > 63u)
                return fail(h, DOMAGG_ERR_UNSUPPORTED, "node keys of more than 63 bits (m = 4, too many distinct values)");
            inst[s].T = (u32)T;
            inst[s].Tq = (u32)Tq;
        }
        h->meas_lvl = lvl;  // (a plan splits its capacities by key class from these)

        // chunks of instances whose records fit one record workspace: below
        // 2^32 records and ~60% of the free memory (plus the record workspace
        // already held)
        u64 chunk_cap = (1ull << 32) - 65536;
        {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
                const double per_rec = 2.0 * sizeof(K) + 2.0 * sizeof(Pay) + sizeof(Part) + 8.0;
                double budget = std::max(0.6 * (double)free_b + (double)h->recs.cap, 2.0e9);
                // a capped handle also caps the records of one chunk
                if (h->max_ws) budget = std::min(budget, 0.5 * (double)(h->max_ws - std::min(h->max_ws, h->held() - h->recs.cap)));
                chunk_cap = std::max<u64>(1, std::min<u64>(chunk_cap, (u64)(budget / per_rec)));
            } else {
                cudaGetLastError();
            }
        }
        {
            Chunk c;
            for (int s = 0; s < k; ++s) {
                const u64 Ts = inst[s].T;
                if (c.k1 > c.k0 && c.T + Ts > chunk_cap) {
                    chunks.push_back(c);
                    c = Chunk();
                    c.k0 = c.k1 = s;
                }
                c.k1 = s + 1;
                c.T += Ts;
                c.Tq += inst[s].Tq;
                c.nseg += nlev[s];
                for (u32 lv = 0; lv < nlev[s]; ++lv) {
                    const int bits = (int)level_bits(s, lv);
                    if (narrow_level(s, lv)) {
                        c.nseg1 += 1;
                        c.T1 += lvl[(size_t)s * LMAX + lv];
                        c.key_bits1 = std::max(c.key_bits1, bits);
                    } else {
                        c.nseg0 += 1;
                        c.T0 += lvl[(size_t)s * LMAX + lv];
                        c.key_bits = std::max(c.key_bits, bits);
                    }
                }
            }
            if (c.k1 > c.k0) chunks.push_back(c);
        }
        base_pos.resize(chunks.size());
        size_t pin_need = ctl_pos + sizeof(Ctl);
        for (size_t ci = 0; ci < chunks.size(); ++ci) {
            base_pos[ci] = (pin_need + 63) & ~(size_t)63;
            pin_need = base_pos[ci] + sizeof(u32) * chunk_upload_words(chunks[ci]);
        }
        if (pin_need > h->h_pin_cap) {
            // grow_pinned keeps nothing; the instance table is already in `inst`
            domagg_status st = grow_pinned(h, pin_need);
            if (st) return st;
            hp = (char*)h->h_pin;
        }
    }

    // ---- a shard's group parts start at the unit (its group kernel writes
    // only its own groups' queries)
    if (use_groups && inst[0].nshards > 1 && N > 0) {
        L.start(KIND_SMALL, 0.0);
        k_fill_e<Op><<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(gacc, (u32)N);
        L.stop();
    }
    // ---- m = 2, 3: the deep rank levels by groups, in shared memory
    // (k_group, k_group3): a stable sort of the points (in the order of the
    // last coordinate) by their group of ranks, then one CTA per group
    if (use_groups) {
        std::vector<u32> gb_host;
        int gbits_max = 0;
        if (!planned) {
            gb_host.resize(k);
            for (int s = 0; s < k; ++s) {
                gb_host[s] = inst[s].gS ? inst[s].b[0] - inst[s].gS : 0u;
                gbits_max = std::max(gbits_max, (int)gb_host[s]);
            }
        } else {  // bound: ranks below 2n (a non-strict first coordinate doubles them)
            for (int s = 0; s < k; ++s) {
                int bb = 0;
                while (bb < 32 && (1ull << bb) < 2 * pt_sizes[s]) ++bb;
                gbits_max = std::max(gbits_max, bb);
            }
        }
        SortSpace gs{d_pt_offs, k, planned ? nullptr : &pt_sizes, d_sort_tiles, hist, digit_off,
                     (u64*)h->st_multi.p, (double)N, (u32*)P[24], sort_range_bound(pt_sizes),
                     planned ? nullptr : &gb_host, N};
        sort_pairs<u32, u64>(L, gs, gkey, gval, false, gbits_max, 0xffffffffu, KIND_HIST_POINTS, KIND_SORT_GROUPS,
                             gbits, true, false);
        L.start(KIND_SMALL, 0.0);
        k_group_slots<<<1, 1024, 0, stream>>>(d_inst, k, gslot);
        L.stop();
        typedef typename Op::Acc Acc;
        const int li = L.lookback_index();
        if constexpr (M == 2) {
            constexpr size_t gsm = group_smem_bytes<Acc>();
            if (!L.frozen) cudaFuncSetAttribute(k_group<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
            L.start(KIND_GROUP, (double)N * 8.0 + (double)NQ * sizeof(Part));
            k_group<Op><<<(unsigned)h->sms, GROUP_THREADS, gsm, stream>>>(d_inst, k, gslot, rstart, gval[0], gval[1],
                                                                          (const W*)P[18], gacc, h->ctl, li);
            L.stop();
        } else {
            // m = 3: the group-sorted rank and position, the second rank and
            // (data) the weight gathered by position, a partial per query
            constexpr size_t gsm = G3Smem<Acc>::TOTAL;
            if (!L.frozen) cudaFuncSetAttribute(k_group3<Op, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
            L.start(KIND_GROUP, (double)N * (8.0 + 4.0) + (double)(N - NQ) * (WT == 3 ? 0.0 : sizeof(W)) +
                                    (double)NQ * sizeof(Part));
            k_group3<Op, WT><<<(unsigned)h->sms, G3_THREADS, gsm, stream>>>(d_inst, k, gslot, rstart, gval[0],
                                                                            gval[1], pr1, (const W*)P[18], gacc,
                                                                            h->ctl, li);
            L.stop();
        }
    }
    // ---- m = 2: the top levels per range of tiles in the order of the last
    // coordinate (k_top), then the nodes' carries across the ranges
    if (use_top && nranges > 0) {
        typedef typename Op::Acc Acc;
        constexpr size_t tsm = TopSmem<Acc>::TOTAL;
        if (!L.frozen) cudaFuncSetAttribute(k_top<Op, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm);
        const int li = L.lookback_index();
        L.start(KIND_TOP, (double)N * (4.0 + (WT == 3 ? 0.0 : sizeof(W))) +
                              (double)NQ * (sizeof(Acc) + (use_groups ? sizeof(Part) : 0.0)) +
                              (double)nranges * TOP_STRIDE * sizeof(Acc));
        k_top<Op, WT><<<(unsigned)h->sms, TOP_THREADS, tsm, stream>>>(d_inst, k, d_prange, d_pt_offs, range_pts, pr0,
                                                                      (const W*)P[18], gacc, topv, top_agg,
                                                                      (u32)nranges, h->ctl, li);
        L.stop();
        if (!multi.empty()) {
            L.start(KIND_SMALL, 0.0);
            k_top_carry<Op><<<dim3((unsigned)multi.size(), TOP_STRIDE / 32), 1024, 0, stream>>>(
                d_multi, d_prange, d_inst, top_agg, (u32)nranges);
            L.stop();
        }
    }

    u64 Tq_all = 0;
    int kb_all = 0, passes_all = 0;
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const Chunk& C = chunks[ci];
        const int kc = C.k1 - C.k0;
        const u64 nseg = C.nseg, nseg0 = C.nseg0, nseg1 = C.nseg1;
        // host tables (unplanned): record and slot bases per instance, the two
        // classes' segment offsets, key bits (class 0 then class 1), bases per
        // (instance, level) within the level's class, slot bases, class-1 masks
        u32 *hb = nullptr, *h_rb = nullptr, *h_qb = nullptr, *h_so = nullptr, *h_so1 = nullptr, *h_sbits = nullptr,
            *h_sbase = nullptr, *h_qsbase = nullptr, *h_nmask = nullptr;
        if (!planned) {
            hb = (u32*)(hp + base_pos[ci]);
            h_rb = hb;
            h_qb = hb + kc + 1;
            h_so = h_qb + kc + 1;
            h_so1 = h_so + nseg0 + 1;
            h_sbits = h_so1 + nseg1 + 1;
            h_sbase = h_sbits + nseg;
            h_qsbase = h_sbase + (size_t)kc * LMAX;
            h_nmask = h_qsbase + (size_t)kc * LMAX;
        }
        std::vector<u64> seg_sizes0(planned ? 0 : nseg0), seg_sizes1(planned ? 0 : nseg1);
        u64 nts0 = 0, nts1 = 0;
        if (planned) {
            nts0 = C.T0 / SEG_TILE + nseg0;  // bounds: sum ceil(n_s / tile) <= T / tile + nseg
            nts1 = nseg1 ? C.T1 / SEG_TILE + nseg1 : 0;
        } else {
            u64 a0 = 0, a1 = 0, b = 0, g0 = 0, g1 = 0;
            for (int s = C.k0; s < C.k1; ++s) {
                h_rb[s - C.k0] = (u32)(a0 + a1);
                h_qb[s - C.k0] = (u32)b;
                h_nmask[s - C.k0] = 0;
                for (u32 lv = 0; lv < LMAX; ++lv) {
                    h_sbase[(size_t)(s - C.k0) * LMAX + lv] = 0;
                    h_qsbase[(size_t)(s - C.k0) * LMAX + lv] = 0;
                }
                for (u32 lv = 0; lv < nlev[s]; ++lv) {
                    const u64 sz = lvl[(size_t)s * LMAX + lv];
                    const bool nar = narrow_level(s, lv);
                    u64& a = nar ? a1 : a0;
                    const u64 g = nar ? nseg0 + g1 : g0;
                    (nar ? h_so1[g1] : h_so[g0]) = (u32)a;
                    h_sbits[g] = level_bits(s, lv);
                    h_sbase[(size_t)(s - C.k0) * LMAX + lv] = (u32)a;
                    h_qsbase[(size_t)(s - C.k0) * LMAX + lv] = (u32)b;
                    if (nar) {
                        h_nmask[s - C.k0] |= 1u << lv;
                        seg_sizes1[g1++] = sz;
                        nts1 += (sz + SEG_TILE - 1) / SEG_TILE;
                    } else {
                        seg_sizes0[g0++] = sz;
                        nts0 += (sz + SEG_TILE - 1) / SEG_TILE;
                    }
                    a += sz;
                    b += qlvl[(size_t)s * LMAX + lv];
                }
            }
            h_rb[kc] = (u32)(a0 + a1);
            h_qb[kc] = (u32)b;
            h_so[nseg0] = (u32)a0;
            h_so1[nseg1] = (u32)a1;
        }
        const int npass0 = (C.key_bits + RADIX_BITS - 1) / RADIX_BITS;
        const int npass1 = (C.key_bits1 + RADIX_BITS - 1) / RADIX_BITS;
        const u64 ntr0 = planned ? C.T0 / SORT_MIN_TILE + nseg0 : tiles_of(seg_sizes0, SORT_MIN_TILE);
        const u64 ntr1 = planned ? (nseg1 ? C.T1 / SORT_MIN_TILE + nseg1 : 0) : tiles_of(seg_sizes1, SORT_MIN_TILE);
        const u64 nrb0 = planned ? sort_range_bound_n(C.T0, nseg0) : sort_range_bound(seg_sizes0);
        const u64 nrb1 = planned ? (nseg1 ? sort_range_bound_n(C.T1, nseg1) : 0) : sort_range_bound(seg_sizes1);
        const u64 nseg_max = std::max(nseg0, nseg1);
        const size_t hist_words = std::max<size_t>((size_t)nseg0 * std::max(npass0, 1),
                                                   (size_t)nseg1 * std::max(npass1, 1)) * RADIX;
        // record workspace
        auto carve_recs = [&](Carver& c, void** R) {
            R[0] = c.take<u32>(chunk_upload_words(C));  // the uploaded bases and segment tables
            R[1] = c.take<u32>(nseg_max + 1);            // sort ranges
            R[2] = c.take<u32>(nseg0 + 1);               // segscan tiles, class 0
            R[3] = c.take<K>(C.T0);
            R[4] = c.take<K>(C.T0);
            R[5] = c.take<Pay>(C.T0);
            R[6] = c.take<Pay>(C.T0);
            R[7] = c.take<Part>(C.Tq);
            R[8] = c.take<u32>(hist_words);
            R[9] = c.take<u32>(hist_words);
            R[10] = c.take<u32>((size_t)std::max(nrb0, nrb1) * RADIX);  // first-pass range bases
            R[11] = c.take<u32>(C.T1);                   // class 1: 32-bit keys
            R[12] = c.take<u32>(C.T1);
            R[13] = c.take<Pay>(C.T1);
            R[14] = c.take<Pay>(C.T1);
            R[15] = c.take<u32>(nseg1 + 1);              // segscan tiles, class 1
        };
        void* R[16];
        {
            Carver c(nullptr);
            carve_recs(c, R);
            domagg_status st = grow(h, h->recs, c.off);
            if (st) return st;
            Carver c2(h->recs.p);
            carve_recs(c2, R);
            const u64 nst = std::max<u64>(std::max(std::max(ntr0, ntr1), ntp), 1);
            st = grow(h, h->st_multi, (size_t)nst * RADIX * sizeof(u64), true);
            if (st) return st;
            // the segmented scan's tile summaries and carries
            st = grow(h, h->st_seg, (size_t)std::max<u64>(std::max(nts0, nts1), 1) *
                                        std::max(sizeof(TileAgg<typename Op::Acc>) + sizeof(typename Op::Acc),
                                                 sizeof(SegStatus<typename Op::Acc>)), true);
            if (st) return st;
        }
        u32* d_up = (u32*)R[0];
        u32* d_qb = d_up + kc + 1;
        u32* d_so = d_qb + kc + 1;
        u32* d_so1 = d_so + nseg0 + 1;
        u32* d_sbits = d_so1 + nseg1 + 1;
        u32* d_sbase = d_sbits + nseg;
        u32* d_qsbase = d_sbase + (size_t)kc * LMAX;
        const u32* d_nmask = planned ? C.nmask : d_qsbase + (size_t)kc * LMAX;
        u32 *d_rtiles = (u32*)R[1], *d_stiles = (u32*)R[2], *d_stiles1 = (u32*)R[15];
        K* keys[2] = {(K*)R[3], (K*)R[4]};
        Pay* pays[2] = {(Pay*)R[5], (Pay*)R[6]};
        u32* keys1[2] = {(u32*)R[11], (u32*)R[12]};
        Pay* pays1[2] = {(Pay*)R[13], (Pay*)R[14]};
        Part* partial = (Part*)R[7];
        if (!planned) {
            cudaMemcpyAsync(d_up, hb, sizeof(u32) * chunk_upload_words(C), cudaMemcpyHostToDevice, stream);
            maybe_reset_epochs(h, stream);
        }
        // fresh epoch and tile counters for the record phase of this chunk
        L.start(KIND_SMALL, 0.0);
        k_begin<<<1, 64, 0, stream>>>(h->ctl);
        L.stop();
        h->epoch_mirror += MAX_LAUNCHES;
        L.next_lookback = 0;
        if (planned) {
            L.start(KIND_SMALL, 0.0);
            k_layout<M><<<1, 1024, 0, stream>>>(d_inst, C.k0, lvl_tot, qlvl_tot, C.slot_map, (int)nseg, (int)nseg0,
                                                C.T0, C.T1, C.Tq, d_so, d_sbits, d_sbase, d_qsbase, h->ctl);
            L.stop();
        }
        L.start(KIND_SMALL, 0.0);
        k_make_tiles<<<1, 1024, 0, stream>>>(d_so, (int)nseg0, SEG_TILE, d_stiles);
        if (nseg1) k_make_tiles<<<1, 1024, 0, stream>>>(d_so1, (int)nseg1, SEG_TILE1, d_stiles1);
        L.stop();

        // flat map (6m+1), level by level
        const u64 nchunk = chunk_off[C.k1] - chunk_off[C.k0];
        if (C.T > 0) {
            const unsigned grid = (unsigned)std::min<u64>((nchunk + 7) / 8, (u64)h->sms * L.blocks_per_sm);
            L.start(KIND_EXPAND, (double)(pt_offs[C.k1] - pt_offs[C.k0]) * (4.0 * (M - 1) + (Op::GATHER ? 0 : sizeof(W))) +
                                     (double)C.T0 * (sizeof(K) + sizeof(Pay)) + (double)C.T1 * (4 + sizeof(Pay)));
            k_expand<M, K, Pay, W, WT><<<grid, 256, 0, stream>>>(
                d_chunk_off, k, C.k0, C.k1, d_pt_offs, pr0, pr1, pr2, pj, (const W*)P[18], chunk_base, qchunk_base,
                d_pt_tiles, (const u32*)P[25], d_inst, d_sbase, d_qsbase, M >= 3 ? d_nmask : nullptr, (u32)C.T0,
                keys[0], pays[0], (u32)C.T1, keys1[0], pays1[0], govf);
            L.stop();
        }
        // records sort (6m+2): stable, each level by the bits of its prefix; one
        // sort per key class
        if (C.T0 > 0 && npass0 > 0 && nseg0 > 0) {
            std::vector<u32> sbits_host;
            if (!planned) sbits_host.assign(h_sbits, h_sbits + nseg0);
            SortSpace rs{d_so, (int)nseg0, planned ? nullptr : &seg_sizes0, d_rtiles, (u32*)R[8], (u32*)R[9],
                         (u64*)h->st_multi.p, (double)C.T0, (u32*)R[10], nrb0, planned ? nullptr : &sbits_host, C.T0};
            const K keymask = ~(K(1) << (sizeof(K) * 8 - 1));  // all but the role bit
            sort_pairs<K, Pay>(L, rs, keys, pays, false, C.key_bits, keymask, KIND_HIST_RECORDS, KIND_SORT_RECORDS,
                               d_sbits, true, M <= 2);
        }
        if (C.T1 > 0 && npass1 > 0 && nseg1 > 0) {
            std::vector<u32> sbits_host;
            if (!planned) sbits_host.assign(h_sbits + nseg0, h_sbits + nseg);
            SortSpace rs{d_so1, (int)nseg1, planned ? nullptr : &seg_sizes1, d_rtiles, (u32*)R[8], (u32*)R[9],
                         (u64*)h->st_multi.p, (double)C.T1, (u32*)R[10], nrb1, planned ? nullptr : &sbits_host, C.T1};
            sort_pairs<u32, Pay>(L, rs, keys1, pays1, false, C.key_bits1, 0x7fffffffu, KIND_HIST_RECORDS,
                                 KIND_SORT_RECORDS, d_sbits + nseg0);
        }
        // segmented scan (6m+3), per key class: tile summaries, their scan, the partials
        typedef typename Op::Acc Acc;
        TileAgg<Acc>* tagg = (TileAgg<Acc>*)h->st_seg.p;
        auto segscan = [&](auto kc, u64 ntiles, u32 nseg_c, const auto* k0p, const auto* k1p, const Pay* p0p,
                           const Pay* p1p, const u32* so, const u32* stiles, const u32* sbits, double rec_bytes) {
            typedef std::remove_cv_t<std::remove_pointer_t<decltype(k0p)>> KC;
            constexpr int ITEMS_C = decltype(kc)::value;
            if constexpr (M >= 3) {
                // short segments (node keys of two ranks): one pass, carries by look-back
                const int li = L.lookback_index();
                L.start(KIND_SEGSCAN, rec_bytes + (double)C.Tq * sizeof(Part) +
                                          (Op::GATHER ? (double)(pt_offs[C.k1] - pt_offs[C.k0]) * sizeof(W) : 0.0));
                k_segscan_lb<Op, KC, SEG_THREADS, ITEMS_C><<<(unsigned)ntiles, SEG_THREADS, 0, stream>>>(
                    k0p, k1p, p0p, p1p, so, stiles, (int)nseg_c, sbits, (const W*)P[18], partial, (u32)C.Tq,
                    (SegStatus<Acc>*)h->st_seg.p, h->ctl, li);
                L.stop();
                return;
            }
            Acc* carry = (Acc*)(tagg + ntiles);
            L.start(KIND_SEGSCAN, rec_bytes);
            k_segscan<Op, KC, SEG_THREADS, ITEMS_C, false><<<(unsigned)ntiles, SEG_THREADS, 0, stream>>>(
                k0p, k1p, p0p, p1p, so, stiles, (int)nseg_c, sbits, (const W*)P[18], partial, (u32)C.Tq, tagg, carry);
            L.stop();
            L.start(KIND_SMALL, 0.0);
            k_seg_carry<Op><<<1, 1024, 0, stream>>>(stiles, (int)nseg_c, tagg, carry);
            L.stop();
            L.start(KIND_SEGSCAN, rec_bytes + (double)C.Tq * sizeof(Part) +
                                      (Op::GATHER ? (double)(pt_offs[C.k1] - pt_offs[C.k0]) * sizeof(W) : 0.0));
            k_segscan<Op, KC, SEG_THREADS, ITEMS_C, true><<<(unsigned)ntiles, SEG_THREADS, 0, stream>>>(
                k0p, k1p, p0p, p1p, so, stiles, (int)nseg_c, sbits, (const W*)P[18], partial, (u32)C.Tq, tagg, carry);
            L.stop();
        };
        if (C.T0 > 0 && nseg0 > 0)
            segscan(std::integral_constant<int, SEG_ITEMS>(), nts0, (u32)nseg0, keys[0], keys[1], pays[0], pays[1], d_so,
                    d_stiles, d_sbits, (double)C.T0 * (sizeof(K) + sizeof(Pay)));
        if (C.T1 > 0 && nseg1 > 0)
            segscan(std::integral_constant<int, SEG_ITEMS1>(), nts1, (u32)nseg1, keys1[0], keys1[1], pays1[0],
                    pays1[1], d_so1, d_stiles1, d_sbits + nseg0, (double)C.T1 * (4 + sizeof(Pay)));
        // per-query reduction (replaces 6m+4 .. 6m+9)
        const u32 qb = q_offs[C.k0], qe = q_offs[C.k1];
        if (qe > qb && use_top) {
            // m = 2 with top levels: one block per range of the chunk's instances
            const unsigned grid = prange_off[C.k1] - prange_off[C.k0];
            // every point's index; a query's rank, top-level value and output
            L.start(KIND_REDUCE, (double)C.Tq * sizeof(Part) + (double)(pt_offs[C.k1] - pt_offs[C.k0]) * 4 +
                                     (double)(qe - qb) * (4 + sizeof(typename Op::Acc) + sizeof(typename Op::Out)));
            if (grid)
                k_reduce_top<Op><<<grid, TOP_RED_THREADS, 0, stream>>>(
                    k, C.k0, d_prange, range_pts, d_chunk_off, d_pt_offs, pr0, pj, qchunk_base, d_pt_tiles,
                    (const u32*)P[25], d_qsbase, d_inst, partial, (u32)C.Tq, gacc, topv, top_agg, (u32)nranges,
                    govf);
            L.stop();
        } else if (qe > qb) {
            const unsigned grid = (unsigned)std::min<u64>((nchunk + 7) / 8, (u64)h->sms * L.blocks_per_sm);
            L.start(KIND_REDUCE, (double)C.Tq * sizeof(Part) + (double)(qe - qb) * (8 + sizeof(typename Op::Out)));
            k_reduce<Op, M><<<grid, 256, 0, stream>>>(d_chunk_off, k, C.k0, C.k1, d_pt_offs, pr0, pr1, pr2, pj,
                                                      qchunk_base, d_pt_tiles, (const u32*)P[25], d_qsbase, d_inst,
                                                      partial, (u32)C.Tq, gacc, govf);
            L.stop();
        }
        Tq_all += C.Tq;
        kb_all = std::max(kb_all, std::max(C.key_bits, C.key_bits1));
        passes_all = std::max(passes_all, std::max(npass0, npass1));
        if (chunks.size() > 1 && !planned) {
            e = cudaStreamSynchronize(stream);  // the next chunk's host tables reuse the pinned area
            if (e != cudaSuccess) return cuda_fail(h, e, "record phase");
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "launch");
    if (L.next_lookback > MAX_LAUNCHES) return fail(h, DOMAGG_ERR_UNSUPPORTED, "too many look-back launches");
    if (planned) return DOMAGG_OK;  // the counts stay on the device

    domagg_stats& S = h->stats;
    S.n_points = (int64_t)N;
    S.n_records = (int64_t)T_flat;  // every record of the flat map, wherever it is formed
    S.n_records_shared = (int64_t)T_shared;
    S.n_query_records = (int64_t)Tq_all;
    S.m = M;
    for (int i = 0; i < 3; ++i) {
        S.rank_bits[i] = (k == 1 && i < M - 1) ? (int32_t)inst[0].b[i] : 0;
        S.distinct[i] = (k == 1 && i < M - 1) ? (int64_t)inst[0].U[i] : 0;
    }
    S.record_key_bits = kb_all;
    S.record_passes = passes_all;
    S.workspace_bytes = (int64_t)h->held();
    return DOMAGG_OK;
}

typedef std::vector<PlannedChunk> Planned;

template <int M, class Op>
domagg_status run_ct(domagg_ctx* h, std::vector<Inst>& inst, domagg_dtype ct, bool negate, cudaStream_t s,
                     const Planned* pl) {
    return ct == DOMAGG_F32 ? run<M, Op, true>(h, inst, negate, s, pl) : run<M, Op, false>(h, inst, negate, s, pl);
}

template <class Op>
domagg_status run_m(domagg_ctx* h, int m, std::vector<Inst>& inst, domagg_dtype ct, bool negate, cudaStream_t s,
                    const Planned* pl) {
    switch (m) {
        case 1: return run_ct<1, Op>(h, inst, ct, negate, s, pl);
        case 2: return run_ct<2, Op>(h, inst, ct, negate, s, pl);
        case 3: return run_ct<3, Op>(h, inst, ct, negate, s, pl);
        default: return run_ct<4, Op>(h, inst, ct, negate, s, pl);
    }
}

domagg_status dispatch(domagg_ctx* h, int m, std::vector<Inst>& inst, domagg_dtype ct, domagg_dtype wt,
                       domagg_op op, bool negate, cudaStream_t s, const Planned* pl = nullptr) {
    if (op == DOMAGG_COUNT) return run_m<OpCount>(h, m, inst, ct, negate, s, pl);
    if (op == DOMAGG_SUM && wt == DOMAGG_F32) return run_m<OpSumF32>(h, m, inst, ct, negate, s, pl);
    if (op == DOMAGG_SUM && wt == DOMAGG_I64) return run_m<OpSumI64>(h, m, inst, ct, negate, s, pl);
    if (op == DOMAGG_MAX && wt == DOMAGG_I32) return run_m<OpMaxI32>(h, m, inst, ct, negate, s, pl);
    if (op == DOMAGG_MAX && wt == DOMAGG_F32) return run_m<OpMaxF32>(h, m, inst, ct, negate, s, pl);
    if (op == DOMAGG_MIN && wt == DOMAGG_I32) return run_m<OpMinI32>(h, m, inst, ct, negate, s, pl);
    if (op == DOMAGG_MIN && wt == DOMAGG_F32) return run_m<OpMinF32>(h, m, inst, ct, negate, s, pl);
    return fail(h, DOMAGG_ERR_INVALID_ARG, "unsupported (op, weight dtype) pair");
}

// Device bytes per record of a chunk: key and payload double-buffered, a
// partial per (query) record and the status words, rounded up.
size_t record_bytes(int m, domagg_dtype wt, domagg_op op) {
    const size_t kb = m == 3 ? 8 : 4;
    const size_t pb = 4;  // every payload is 32 bits (8-byte weights are gathered by position)
    (void)wt;
    const size_t part = (op == DOMAGG_MAX || op == DOMAGG_MIN || (op == DOMAGG_SUM && wt == DOMAGG_F32)) ? 4 : 8;
    // m >= 3 plans reserve both key classes (64- and 32-bit keys) at the full capacity
    const size_t class1 = m >= 3 ? 2 * 4 + 2 * pb : 0;
    return 2 * kb + 2 * pb + class1 + part + 8;
}

domagg_status check_common(domagg_ctx* h, int m, int64_t nD, int64_t nQ, domagg_dtype ct, domagg_dtype wt,
                           domagg_op op) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    h->err.clear();
    if (m < 1) return fail(h, DOMAGG_ERR_INVALID_ARG, "m must be >= 1");
    if (m > 4) return fail(h, DOMAGG_ERR_UNSUPPORTED, "m > 4 is not supported");
    if (nD < 0 || nQ < 0) return fail(h, DOMAGG_ERR_INVALID_ARG, "negative size");
    if (nD + nQ >= (int64_t)1 << 31) return fail(h, DOMAGG_ERR_UNSUPPORTED, "nD + nQ must be below 2^31");
    if (ct != DOMAGG_I32 && ct != DOMAGG_F32) return fail(h, DOMAGG_ERR_INVALID_ARG, "coordinates must be i32 or f32");
    if (op != DOMAGG_SUM && op != DOMAGG_MAX && op != DOMAGG_COUNT && op != DOMAGG_MIN)
        return fail(h, DOMAGG_ERR_INVALID_ARG, "bad op");
    if (op == DOMAGG_SUM && wt != DOMAGG_I64 && wt != DOMAGG_F32)
        return fail(h, DOMAGG_ERR_INVALID_ARG, "SUM takes i64 or f32 weights");
    if ((op == DOMAGG_MAX || op == DOMAGG_MIN) && wt != DOMAGG_I32 && wt != DOMAGG_F32)
        return fail(h, DOMAGG_ERR_INVALID_ARG, "MAX takes i32 or f32 weights");
    return DOMAGG_OK;
}

size_t dtype_size(domagg_dtype t) { return t == DOMAGG_I64 ? 8 : 4; }

size_t out_size(domagg_op op, domagg_dtype wt) {
    if (op == DOMAGG_COUNT) return 8;
    return dtype_size(wt);
}

Inst make_inst(const void* dco, int64_t nD, const void* qco, int64_t nQ, const void* dw, void* out) {
    Inst I;
    memset(&I, 0, sizeof(I));
    I.dco = dco;
    I.qco = qco;
    I.dw = dw;
    I.out = out;
    I.nD = (u32)nD;
    I.nQ = (u32)nQ;
    return I;
}

// Tuning knobs by name (domagg_set_tuning, DOMAGG_TUNE).
bool set_tuning(domagg_ctx* h, const std::string& name, int value) {
    if (name == "group_bits") {
        if (value < 0 || value > GROUP_MAX_BITS) return false;
        h->group_bits = value;
    } else if (name == "top_bits") {
        if (value < 0 || value > TOP_MAX_BITS) return false;
        h->top_bits = value;
    } else if (name == "rank_windows") {
        if (value < 0 || value > 64) return false;
        h->rank_windows = value;
    } else if (name == "ranges_per_cta") {
        if (value < 1 || value > 64) return false;
        h->ranges_per_cta = value;
    } else if (name == "blocks_per_sm") {
        if (value < 1 || value > 64) return false;
        h->blocks_per_sm = value;
    } else {
        return false;
    }
    return true;
}

// DOMAGG_TUNE="name=value,name=value" overrides the defaults of a new handle
// (malformed or unknown entries are ignored).
void apply_tune_env(domagg_ctx* h) {
    const char* env = std::getenv("DOMAGG_TUNE");
    if (!env) return;
    std::string all(env);
    size_t pos = 0;
    while (pos <= all.size()) {
        size_t end = all.find(',', pos);
        if (end == std::string::npos) end = all.size();
        const std::string item = all.substr(pos, end - pos);
        const size_t eq = item.find('=');
        if (eq != std::string::npos) {
            char* stop = nullptr;
            const long v = std::strtol(item.c_str() + eq + 1, &stop, 10);
            if (stop && *stop == '\0' && stop != item.c_str() + eq + 1) set_tuning(h, item.substr(0, eq), (int)v);
        }
        pos = end + 1;
    }
}

}  // namespace

extern "C" {

domagg_status domagg_set_tuning(domagg_handle h, const char* name, int value) {
    if (!h || !name) return DOMAGG_ERR_INVALID_ARG;
    if (!set_tuning(h, name, value)) return fail(h, DOMAGG_ERR_INVALID_ARG, std::string("unknown tuning knob or value: ") + name);
    return DOMAGG_OK;
}

domagg_status domagg_create(domagg_handle* out, int device, size_t max_workspace_bytes) {
    if (!out) return DOMAGG_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DOMAGG_ERR_INVALID_ARG;
    }
    domagg_ctx* h = new (std::nothrow) domagg_ctx();
    if (!h) return DOMAGG_ERR_OOM;
    h->device = device;
    h->max_ws = max_workspace_bytes;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    if (h->sms <= 0) h->sms = 152;
    apply_tune_env(h);
    h->overlap = cudaStreamCreateWithFlags(&h->aux[0], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaStreamCreateWithFlags(&h->aux[1], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_join[0], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_join[1], cudaEventDisableTiming) == cudaSuccess;
    if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_w, cudaEventDisableTiming) != cudaSuccess) {
        h->copy_stream = nullptr;  // the weights then go on the call's stream
        h->ev_w = nullptr;
    }
    cudaGetLastError();
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&h->ctl, sizeof(Ctl)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return DOMAGG_ERR_CUDA;
    }
    cudaMemset(h->ctl, 0, sizeof(Ctl));
    cudaDeviceSynchronize();
    *out = h;
    return DOMAGG_OK;
}

domagg_status domagg_destroy(domagg_handle h) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (DevBuf* b : {&h->pts, &h->recs, &h->st_multi, &h->st_seg, &h->stage, &h->st_wv})
        if (b->p) cudaFree(b->p);
    if (h->ctl) cudaFree(h->ctl);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
    for (cudaStream_t s : h->aux)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : {h->ev_fork, h->ev_join[0], h->ev_join[1], h->ev_w})
        if (e) cudaEventDestroy(e);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
    return DOMAGG_OK;
}

domagg_status domagg_forward(domagg_handle h, int m, const void* d_coords, int64_t nD, const void* q_coords,
                             int64_t nQ, domagg_dtype coord_dtype, const void* d_weights, domagg_dtype weight_dtype,
                             domagg_op op, void* out, void* stream) {
    domagg_status st = check_common(h, m, nD, nQ, coord_dtype, weight_dtype, op);
    if (st) return st;
    if ((nD > 0 && !d_coords) || (nQ > 0 && (!q_coords || !out)) ||
        (op != DOMAGG_COUNT && nD > 0 && !d_weights))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nQ == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    std::vector<Inst> inst{make_inst(d_coords, nD, q_coords, nQ, d_weights, out)};
    return dispatch(h, m, inst, coord_dtype, weight_dtype, op, false, (cudaStream_t)stream);
}

domagg_status domagg_forward_ex(domagg_handle h, int m, const void* d_coords, int64_t nD, const void* q_coords,
                                int64_t nQ, domagg_dtype coord_dtype, const void* d_weights, domagg_dtype weight_dtype,
                                domagg_op op, uint32_t nonstrict_mask, domagg_variant variant, void* out,
                                void* stream) {
    if (variant != DOMAGG_IMPROVED && variant != DOMAGG_BASIC && variant != DOMAGG_WAVELET)
        return fail(h, DOMAGG_ERR_INVALID_ARG, "bad variant");
    if (variant == DOMAGG_WAVELET && h && m > 2)
        return fail(h, DOMAGG_ERR_UNSUPPORTED, "the level-wise formulation takes m <= 2");
    const int M = variant == DOMAGG_BASIC ? m + 1 : m;  // the pipeline's coordinates
    domagg_status st = check_common(h, M, nD, nQ, coord_dtype, weight_dtype, op);
    if (st) return variant == DOMAGG_BASIC && M > 4 ? fail(h, DOMAGG_ERR_UNSUPPORTED, "basic variant: m <= 3") : st;
    if (m < 1 || (nonstrict_mask >> m) != 0u) return fail(h, DOMAGG_ERR_INVALID_ARG, "nonstrict_mask has bits >= m");
    if ((nD > 0 && !d_coords) || (nQ > 0 && (!q_coords || !out)) ||
        (op != DOMAGG_COUNT && nD > 0 && !d_weights))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nQ == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    std::vector<Inst> inst{make_inst(d_coords, nD, q_coords, nQ, d_weights, out)};
    inst[0].flags = nonstrict_mask;
    // basic variant: all m stored coordinates become bitstrings, and a
    // constant last coordinate compared non-strictly puts every data record
    // of a node tuple before its queries
    if (variant == DOMAGG_BASIC) inst[0].flags |= FLAG_VIRTUAL_LAST | (1u << m);
    if (variant == DOMAGG_WAVELET) inst[0].flags |= FLAG_WAVELET;
    return dispatch(h, M, inst, coord_dtype, weight_dtype, op, false, (cudaStream_t)stream);
}

domagg_status domagg_forward_shard(domagg_handle h, int shard, int nshards, int m, const void* d_coords, int64_t nD,
                                   const void* q_coords, int64_t nQ, domagg_dtype coord_dtype, const void* d_weights,
                                   domagg_dtype weight_dtype, domagg_op op, void* out, float* out_lo, void* stream) {
    if (nshards < 1 || nshards > MAX_SHARDS || shard < 0 || shard >= nshards)
        return fail(h, DOMAGG_ERR_INVALID_ARG, "shard must be in [0, nshards), nshards in [1, 64]");
    domagg_status st = check_common(h, m, nD, nQ, coord_dtype, weight_dtype, op);
    if (st) return st;
    const bool ffsum = op == DOMAGG_SUM && weight_dtype == DOMAGG_F32;
    if (ffsum && nQ > 0 && !out_lo) return fail(h, DOMAGG_ERR_INVALID_ARG, "float32 sums need out_lo");
    if ((nD > 0 && !d_coords) || (nQ > 0 && (!q_coords || !out)) || (op != DOMAGG_COUNT && nD > 0 && !d_weights))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nQ == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    std::vector<Inst> inst{make_inst(d_coords, nD, q_coords, nQ, d_weights, out)};
    inst[0].shard = (u32)shard;
    inst[0].nshards = (u32)nshards;
    inst[0].out_lo = ffsum ? out_lo : nullptr;
    return dispatch(h, m, inst, coord_dtype, weight_dtype, op, false, (cudaStream_t)stream);
}

domagg_status domagg_combine(domagg_handle h, domagg_op op, domagg_dtype weight_dtype, int nparts,
                             const void* const* parts, const float* const* parts_lo, int64_t nQ, void* out,
                             void* stream) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    if (nparts < 1 || nparts > MAX_SHARDS || !parts || nQ < 0 || (nQ > 0 && !out) || nQ >= (1ll << 31))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "bad parts, size or output");
    ShardParts P;
    memset(&P, 0, sizeof(P));
    for (int s = 0; s < nparts; ++s) {
        if (nQ > 0 && !parts[s]) return fail(h, DOMAGG_ERR_INVALID_ARG, "null part");
        P.part[s] = parts[s];
        P.lo[s] = parts_lo ? parts_lo[s] : nullptr;
    }
    if (nQ == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    const unsigned grid = (unsigned)((nQ + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    const int code = op * 8 + (op == DOMAGG_COUNT ? 0 : (int)weight_dtype);
    switch (code) {
        case DOMAGG_SUM * 8 + DOMAGG_F32: k_combine<OpSumF32><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        case DOMAGG_SUM * 8 + DOMAGG_I64: k_combine<OpSumI64><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        case DOMAGG_MAX * 8 + DOMAGG_I32: k_combine<OpMaxI32><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        case DOMAGG_MAX * 8 + DOMAGG_F32: k_combine<OpMaxF32><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        case DOMAGG_MIN * 8 + DOMAGG_I32: k_combine<OpMinI32><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        case DOMAGG_MIN * 8 + DOMAGG_F32: k_combine<OpMinF32><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        case DOMAGG_COUNT * 8: k_combine<OpCount><<<grid, 256, 0, s>>>(nparts, P, (u32)nQ, out); break;
        default: return fail(h, DOMAGG_ERR_INVALID_ARG, "unsupported op / weight dtype");
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DOMAGG_OK : cuda_fail(h, e, "combine");
}

// max over z of |cx[z] * inv_x - cy[z] * inv_y|: a block-wide max, then an
// atomic max on the bits of the (non-negative) double, which order as
// integers.
static __global__ __launch_bounds__(256) void k_ecdf_max(const long long* __restrict__ cx,
                                                        const long long* __restrict__ cy, u64 nz, double inv_x,
                                                        double inv_y, unsigned long long* out_bits) {
    __shared__ double s_max[8];
    double m = 0.0;
    for (u64 z = (u64)blockIdx.x * blockDim.x + threadIdx.x; z < nz; z += (u64)gridDim.x * blockDim.x)
        m = fmax(m, fabs(__dsub_rn(__dmul_rn((double)cx[z], inv_x), __dmul_rn((double)cy[z], inv_y))));
    for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_max[w]);
        atomicMax(out_bits, (unsigned long long)__double_as_longlong(m));
    }
}

domagg_status domagg_ecdf_distance(domagg_handle h, const int64_t* count_x, const int64_t* count_y, int64_t nz,
                                   int64_t nx, int64_t ny, double* d_out, void* stream) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    if (!d_out || nz < 0 || nx <= 0 || ny <= 0 || (nz > 0 && (!count_x || !count_y)))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer or non-positive sample size");
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(d_out, 0, sizeof(double), s);
    if (nz > 0) {
        const unsigned grid = (unsigned)std::min<int64_t>((nz + 255) / 256, (int64_t)h->sms * 8);
        k_ecdf_max<<<grid, 256, 0, s>>>(reinterpret_cast<const long long*>(count_x),
                                        reinterpret_cast<const long long*>(count_y), (u64)nz, 1.0 / (double)nx,
                                        1.0 / (double)ny, reinterpret_cast<unsigned long long*>(d_out));
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DOMAGG_OK : cuda_fail(h, e, "ecdf distance");
}

domagg_status domagg_forward_host(domagg_handle h, int m, const void* d_coords, int64_t nD, const void* q_coords,
                                  int64_t nQ, domagg_dtype coord_dtype, const void* d_weights,
                                  domagg_dtype weight_dtype, domagg_op op, void* out, void* stream) {
    domagg_status st = check_common(h, m, nD, nQ, coord_dtype, weight_dtype, op);
    if (st) return st;
    if ((nD > 0 && !d_coords) || (nQ > 0 && (!q_coords || !out)) ||
        (op != DOMAGG_COUNT && nD > 0 && !d_weights))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nQ == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bd = (size_t)nD * m * 4, bq = (size_t)nQ * m * 4;
    const size_t bw = op == DOMAGG_COUNT ? 0 : (size_t)nD * dtype_size(weight_dtype);
    const size_t bo = (size_t)nQ * out_size(op, weight_dtype);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    st = grow(h, h->stage, al(bd) + al(bq) + al(bw) + al(bo));
    if (st) return st;
    char* base = (char*)h->stage.p;
    char *dd = base, *dq = dd + al(bd), *dw = dq + al(bq), *dout = dw + al(bw);
    Launcher L;
    L.stream = s;
    L.timing = h->timing;
    L.log = &h->log;
    L.pool = &h->pool;
    L.pool_used = &h->pool_used;
    L.start(KIND_H2D, (double)(bd + bq + bw));
    if (bd) cudaMemcpyAsync(dd, d_coords, bd, cudaMemcpyHostToDevice, s);
    if (bq) cudaMemcpyAsync(dq, q_coords, bq, cudaMemcpyHostToDevice, s);
    // the weights beside the point phase: the pipeline waits for them before
    // the count scan, their first reader (the staging buffer is idle: the
    // previous call synchronised)
    if (bw && h->copy_stream) {
        cudaMemcpyAsync(dw, d_weights, bw, cudaMemcpyHostToDevice, h->copy_stream);
        cudaEventRecord(h->ev_w, h->copy_stream);
        h->w_pending = true;
    } else if (bw) {
        cudaMemcpyAsync(dw, d_weights, bw, cudaMemcpyHostToDevice, s);
    }
    L.stop();
    std::vector<Inst> inst{make_inst(dd, nD, dq, nQ, bw ? dw : nullptr, dout)};
    st = dispatch(h, m, inst, coord_dtype, weight_dtype, op, false, s);
    if (h->w_pending) {  // a path that read no weights (or failed before): join the copy anyway
        cudaStreamWaitEvent(s, h->ev_w, 0);
        h->w_pending = false;
    }
    if (st) {
        cudaStreamSynchronize(h->copy_stream ? h->copy_stream : s);  // the copy reads the caller's buffer
        return st;
    }
    L.start(KIND_D2H, (double)bo);
    cudaMemcpyAsync(out, dout, bo, cudaMemcpyDeviceToHost, s);
    L.stop();
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "forward_host");
    return DOMAGG_OK;
}

domagg_status domagg_backward(domagg_handle h, int m, const void* d_coords, int64_t nD, const void* q_coords,
                              int64_t nQ, domagg_dtype coord_dtype, const float* grad_out, float* grad_w,
                              void* stream) {
    domagg_status st = check_common(h, m, nD, nQ, coord_dtype, DOMAGG_F32, DOMAGG_SUM);
    if (st) return st;
    if ((nD > 0 && (!d_coords || !grad_w)) || (nQ > 0 && (!q_coords || !grad_out)))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nD == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    // reverse dominance: the queries act as data (weights grad_out), the data
    // points as queries, and every key is negated.
    std::vector<Inst> inst{make_inst(q_coords, nQ, d_coords, nD, grad_out, grad_w)};
    return dispatch(h, m, inst, coord_dtype, DOMAGG_F32, DOMAGG_SUM, true, (cudaStream_t)stream);
}

domagg_status domagg_backward_ex(domagg_handle h, int m, const void* d_coords, int64_t nD, const void* q_coords,
                                 int64_t nQ, domagg_dtype coord_dtype, const float* grad_out, float* grad_w,
                                 uint32_t nonstrict_mask, domagg_variant variant, void* stream) {
    domagg_status st = check_common(h, m, nD, nQ, coord_dtype, DOMAGG_F32, DOMAGG_SUM);
    if (st) return st;
    if ((nonstrict_mask >> m) != 0u) return fail(h, DOMAGG_ERR_INVALID_ARG, "nonstrict_mask has bits >= m");
    if (variant != DOMAGG_IMPROVED && variant != DOMAGG_WAVELET)
        return fail(h, variant == DOMAGG_BASIC ? DOMAGG_ERR_UNSUPPORTED : DOMAGG_ERR_INVALID_ARG,
                    "backward variants: improved, wavelet");
    if (variant == DOMAGG_WAVELET && m > 2)
        return fail(h, DOMAGG_ERR_UNSUPPORTED, "the level-wise formulation takes m <= 2");
    if ((nD > 0 && (!d_coords || !grad_w)) || (nQ > 0 && (!q_coords || !grad_out)))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nD == 0) return DOMAGG_OK;
    cudaSetDevice(h->device);
    // as domagg_backward; a non-strict coordinate stays non-strict under the
    // swap of roles and the negated keys (d_i <= q_i  <=>  -q_i <= -d_i)
    std::vector<Inst> inst{make_inst(q_coords, nQ, d_coords, nD, grad_out, grad_w)};
    inst[0].flags = nonstrict_mask | (variant == DOMAGG_WAVELET ? FLAG_WAVELET : 0u);
    return dispatch(h, m, inst, coord_dtype, DOMAGG_F32, DOMAGG_SUM, true, (cudaStream_t)stream);
}

domagg_status domagg_batch(domagg_handle h, int k, const domagg_instance* inst, domagg_dtype coord_dtype,
                           domagg_dtype weight_dtype, domagg_op op, void* stream) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    if (k < 0 || (k > 0 && !inst)) return fail(h, DOMAGG_ERR_INVALID_ARG, "bad instance array");
    std::vector<Inst> groups[5];
    int64_t total[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < k; ++i) {
        const domagg_instance& I = inst[i];
        domagg_status st = check_common(h, I.m, I.nD, I.nQ, coord_dtype, weight_dtype, op);
        if (st) return st;
        if ((I.nD > 0 && !I.d_coords) || (I.nQ > 0 && (!I.q_coords || !I.out)) ||
            (op != DOMAGG_COUNT && I.nD > 0 && !I.d_weights))
            return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer in instance " + std::to_string(i));
        if (I.nQ == 0) continue;
        total[I.m] += I.nD + I.nQ;
        groups[I.m].push_back(make_inst(I.d_coords, I.nD, I.q_coords, I.nQ, I.d_weights, I.out));
    }
    cudaSetDevice(h->device);
    for (int m = 1; m <= 4; ++m) {
        if (groups[m].empty()) continue;
        // one call per group of at most 2^31 - 1 points
        std::vector<Inst> part;
        int64_t acc = 0;
        for (size_t i = 0; i <= groups[m].size(); ++i) {
            const bool flush = i == groups[m].size() ||
                               (acc + (int64_t)groups[m][i].nD + groups[m][i].nQ >= ((int64_t)1 << 31) - 1);
            if (flush && !part.empty()) {
                domagg_status st = dispatch(h, m, part, coord_dtype, weight_dtype, op, false, (cudaStream_t)stream);
                if (st) return st;
                part.clear();
                acc = 0;
            }
            if (i < groups[m].size()) {
                part.push_back(groups[m][i]);
                acc += (int64_t)groups[m][i].nD + groups[m][i].nQ;
            }
        }
    }
    (void)total;
    return DOMAGG_OK;
}

}  // extern "C"

struct domagg_plan_s {
    struct Group {
        int m = 0;
        domagg_ctx* ctx = nullptr;      // private workspace of this group
        std::vector<Inst> inst;         // as given (sizes and pointers)
        std::vector<PlannedChunk> chunks;
        u32 margin = 0;                 // epoch guard margin
    };
    int device = 0;
    domagg_dtype ct = DOMAGG_I32, wt = DOMAGG_I32;
    domagg_op op = DOMAGG_SUM;
    std::vector<Group> groups;
    std::string err;
};

namespace {

void plan_free(domagg_plan p) {
    if (!p) return;
    cudaSetDevice(p->device);
    for (auto& g : p->groups) {
        for (auto& c : g.chunks) {
            if (c.d_slot_map) cudaFree(c.d_slot_map);
            if (c.d_nmask) cudaFree(c.d_nmask);
        }
        if (g.ctx) domagg_destroy(g.ctx);
    }
    delete p;
}

// The message of the last failed domagg_batch_plan of this thread (the plan
// itself is freed): domagg_plan_last_error(NULL) returns it.
thread_local std::string g_plan_create_error;

domagg_status plan_fail(domagg_plan p, domagg_status st, const std::string& msg) {
    p->err = msg;
    return st;
}

// One planned run of a group: the epoch guard, then the pipeline.
domagg_status plan_group_run(domagg_plan p, domagg_plan_s::Group& g, cudaStream_t s) {
    domagg_ctx* h = g.ctx;
    k_epoch_clear<<<304, 256, 0, s>>>(h->ctl, (u64*)h->st_multi.p, h->st_multi.cap / sizeof(u64), (u64*)h->st_seg.p,
                                       h->st_seg.cap / sizeof(u64), g.margin);
    k_epoch_restart<<<1, 32, 0, s>>>(h->ctl, g.margin);
    std::vector<Inst> I = g.inst;
    domagg_status st = dispatch(h, g.m, I, p->ct, p->wt, p->op, false, s, &g.chunks);
    if (st) return plan_fail(p, st, h->err);
    return DOMAGG_OK;
}

// Largest number of levels (rank digits of the first coordinate) an
// instance of n points can have: b = ceil(log2 U) with U <= n.
u32 level_bound(int m, u64 n) {
    if (m == 1) return 1u;
    u32 b = 0;
    while (b < 31 && (1ull << b) < n) ++b;
    return b;
}

// Plans one group (same m, < 2^31 points): measures the record counts with an
// unplanned run, cuts chunks with capacity (1 + headroom) x the measured
// counts, then makes one planned run that allocates the workspace for good.
domagg_status plan_group(domagg_plan p, int m, const std::vector<Inst>& part, double headroom, cudaStream_t s) {
    domagg_plan_s::Group g;
    g.m = m;
    g.inst = part;
    domagg_status st = domagg_create(&g.ctx, p->device, 0);
    if (st) return plan_fail(p, st, "creating the plan's workspace");
    p->groups.push_back(g);
    domagg_plan_s::Group& G = p->groups.back();
    std::vector<Inst> measured = part;
    st = dispatch(G.ctx, m, measured, p->ct, p->wt, p->op, false, s);
    if (st) return plan_fail(p, st, G.ctx->err);
    if (cudaStreamSynchronize(s) != cudaSuccess) return plan_fail(p, DOMAGG_ERR_CUDA, "measuring run");
    // capacity budget: 2^32 positions and ~60% of the free device memory
    const double per_rec = (double)record_bytes(m, p->wt, p->op);
    u64 cap_limit = (1ull << 32) - (1ull << 20);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
        cap_limit = std::min<u64>(cap_limit, (u64)std::max<double>(0.6 * (double)free_b / per_rec, 1.0e6));
    else
        cudaGetLastError();
    const int k = (int)part.size();
    auto scaled = [&](u32 v) { return (u64)std::ceil((double)v * (1.0 + headroom)); };
    PlannedChunk c;
    // per chunk: slots of class 0, then of class 1 (their bound fits 31 bits,
    // m >= 3), and the class-1 level masks of its instances
    std::vector<std::vector<u32>> maps, masks;
    std::vector<u32> map0, map1, mask;
    auto close = [&]() {
        c.T_cap += 1024;  // never 0: the chunk's launches are the same whatever the data
        c.T1_cap += 1024;
        c.Tq_cap += 1024;
        c.nslot0 = (int)map0.size();
        c.nslot = (int)(map0.size() + map1.size());
        G.chunks.push_back(c);
        map0.insert(map0.end(), map1.begin(), map1.end());
        maps.push_back(map0);
        masks.push_back(mask);
        map0.clear();
        map1.clear();
        mask.clear();
    };
    // the measured records of every instance split by the key class the
    // plan gives their level (from the level-count bound, as the slots below)
    const std::vector<u32>& ml = G.ctx->meas_lvl;
    auto class1_records = [&](int i) -> u64 {
        if (m < 3 || ml.size() < (size_t)k * LMAX) return 0;
        const u32 nb = level_bound(m, (u64)part[i].nD + part[i].nQ);
        u64 t = 0;
        for (u32 lv = 0; lv < nb && lv < (u32)LMAX; ++lv)
            if ((int)(nb - 1 - lv) + (int)nb * (m - 2) <= 31) t += ml[(size_t)i * LMAX + lv];
        return std::min<u64>(t, measured[i].T);
    };
    for (int i = 0; i < k; ++i) {
        const u64 T1m = class1_records(i);
        const u64 Ti0 = scaled((u32)(measured[i].T - T1m)), Ti1 = scaled((u32)T1m), Tqi = scaled(measured[i].Tq);
        const u64 Ti = Ti0 + Ti1;
        if (Ti + 2048 > cap_limit) return plan_fail(p, DOMAGG_ERR_UNSUPPORTED, "one instance exceeds a record chunk");
        if (c.k1 > c.k0 && c.T_cap + c.T1_cap + Ti + 2048 > cap_limit) {
            close();
            c = PlannedChunk();
            c.k0 = c.k1 = i;
        }
        c.k1 = i + 1;
        c.T_cap += Ti0;
        c.T1_cap += Ti1;
        c.Tq_cap += Tqi;
        const u32 nb = level_bound(m, (u64)part[i].nD + part[i].nQ);
        u32 msk = 0;
        for (u32 lv = 0; lv < nb; ++lv) {
            // bound on the key bits of level lv: (b - 1 - lv) + b per further rank
            const int bits = m == 1 ? 0 : (int)(nb - 1 - lv) + (int)nb * (m - 2);
            if (bits > 63) return plan_fail(p, DOMAGG_ERR_UNSUPPORTED, "node keys of more than 63 bits (m = 4, large instance)");
            const u32 slot = ((u32)(i - c.k0) << 5) | lv;
            if (m >= 3 && bits <= 31) {
                map1.push_back(slot);
                msk |= 1u << lv;
                c.key_bits1 = std::max(c.key_bits1, bits);
            } else {
                map0.push_back(slot);
                c.key_bits = std::max(c.key_bits, bits);
            }
        }
        mask.push_back(msk);
    }
    if (c.k1 > c.k0) close();
    for (size_t ci = 0; ci < G.chunks.size(); ++ci) {
        PlannedChunk& pc = G.chunks[ci];
        const size_t bytes = std::max<size_t>(maps[ci].size(), 1) * sizeof(u32);
        const size_t mbytes = std::max<size_t>(masks[ci].size(), 1) * sizeof(u32);
        if (cudaMalloc(&pc.d_slot_map, bytes) != cudaSuccess || cudaMalloc(&pc.d_nmask, mbytes) != cudaSuccess) {
            cudaGetLastError();
            return plan_fail(p, DOMAGG_ERR_OOM, "slot map");
        }
        if (!maps[ci].empty()) cudaMemcpy(pc.d_slot_map, maps[ci].data(), maps[ci].size() * sizeof(u32),
                                          cudaMemcpyHostToDevice);
        if (!masks[ci].empty()) cudaMemcpy(pc.d_nmask, masks[ci].data(), masks[ci].size() * sizeof(u32),
                                           cudaMemcpyHostToDevice);
    }
    G.margin = (u32)(G.chunks.size() + 6) * MAX_LAUNCHES;
    // the warm planned run: allocates the workspace at its final size (and
    // loads every kernel a planned run launches)
    st = plan_group_run(p, G, s);
    if (st) return st;
    st = domagg_sync_status(G.ctx, s);
    if (st) return plan_fail(p, st, G.ctx->err);
    G.ctx->frozen = true;
    return DOMAGG_OK;
}

}  // namespace

extern "C" {

domagg_status domagg_batch_plan(domagg_plan* out, int device, int k, const domagg_instance* inst,
                                domagg_dtype coord_dtype, domagg_dtype weight_dtype, domagg_op op, double headroom,
                                void* stream) {
    if (!out) return DOMAGG_ERR_INVALID_ARG;
    *out = nullptr;
    if (k < 0 || (k > 0 && !inst) || !(headroom >= 0.0) || headroom > 1.0e6) return DOMAGG_ERR_INVALID_ARG;
    domagg_plan p = new (std::nothrow) domagg_plan_s();
    if (!p) return DOMAGG_ERR_OOM;
    p->device = device;
    p->ct = coord_dtype;
    p->wt = weight_dtype;
    p->op = op;
    domagg_ctx probe;  // argument checks only (no device resources)
    std::vector<Inst> groups[5];
    for (int i = 0; i < k; ++i) {
        const domagg_instance& I = inst[i];
        domagg_status st = check_common(&probe, I.m, I.nD, I.nQ, coord_dtype, weight_dtype, op);
        if (st) {
            delete p;
            return st;
        }
        if ((I.nD > 0 && !I.d_coords) || (I.nQ > 0 && (!I.q_coords || !I.out)) ||
            (op != DOMAGG_COUNT && I.nD > 0 && !I.d_weights)) {
            delete p;
            return DOMAGG_ERR_INVALID_ARG;
        }
        if (I.nQ == 0) continue;
        groups[I.m].push_back(make_inst(I.d_coords, I.nD, I.q_coords, I.nQ, I.d_weights, I.out));
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return DOMAGG_ERR_INVALID_ARG;
    }
    for (int m = 1; m <= 4; ++m) {
        std::vector<Inst> part;
        int64_t acc = 0;
        for (size_t i = 0; i <= groups[m].size(); ++i) {
            const bool flush = i == groups[m].size() ||
                               (acc + (int64_t)groups[m][i].nD + groups[m][i].nQ >= ((int64_t)1 << 31) - 1);
            if (flush && !part.empty()) {
                domagg_status st = plan_group(p, m, part, headroom, (cudaStream_t)stream);
                if (st) {
                    g_plan_create_error = "m = " + std::to_string(m) + ": " + p->err;
                    plan_free(p);
                    return st;
                }
                part.clear();
                acc = 0;
            }
            if (i < groups[m].size()) {
                part.push_back(groups[m][i]);
                acc += (int64_t)groups[m][i].nD + groups[m][i].nQ;
            }
        }
    }
    *out = p;
    return DOMAGG_OK;
}

domagg_status domagg_plan_run(domagg_plan p, void* stream) {
    if (!p) return DOMAGG_ERR_INVALID_ARG;
    p->err.clear();
    cudaSetDevice(p->device);
    const cudaStream_t s = (cudaStream_t)stream;
    for (auto& g : p->groups) {
        domagg_status st = plan_group_run(p, g, s);
        if (st) return st;
    }
    return DOMAGG_OK;
}

domagg_status domagg_plan_status(domagg_plan p, void* stream) {
    if (!p) return DOMAGG_ERR_INVALID_ARG;
    domagg_status first = DOMAGG_OK;
    for (auto& g : p->groups) {
        domagg_status st = domagg_sync_status(g.ctx, stream);
        if (st && !first) {
            first = st;
            p->err = g.ctx->err;
        }
    }
    return first;
}

const char* domagg_plan_last_error(domagg_plan p) { return p ? p->err.c_str() : g_plan_create_error.c_str(); }

domagg_status domagg_plan_autotune(domagg_plan p, void* stream, double* best_ms) {
    if (!p) return DOMAGG_ERR_INVALID_ARG;
    p->err.clear();
    cudaSetDevice(p->device);
    const cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return plan_fail(p, DOMAGG_ERR_CUDA, "cudaEventCreate");
    }
    static const int kRanges[3] = {2, 4, 8}, kBlocks[3] = {8, 16, 32};
    double total = 0.0;
    domagg_status st = DOMAGG_OK;
    for (auto& g : p->groups) {
        double best = 1e30;
        int br = g.ctx->ranges_per_cta, bb = g.ctx->blocks_per_sm;
        for (int ri = 0; ri < 3 && !st; ++ri) {
            for (int bi = 0; bi < 3 && !st; ++bi) {
                g.ctx->ranges_per_cta = kRanges[ri];
                g.ctx->blocks_per_sm = kBlocks[bi];
                st = plan_group_run(p, g, s);  // warm-up of this shape
                double ms = 0.0;
                for (int rep = 0; rep < 2 && !st; ++rep) {
                    cudaEventRecord(e0, s);
                    st = plan_group_run(p, g, s);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) st = plan_fail(p, DOMAGG_ERR_CUDA, "autotune");
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms += t / 2.0;
                }
                if (!st && ms < best) {
                    best = ms;
                    br = kRanges[ri];
                    bb = kBlocks[bi];
                }
            }
        }
        g.ctx->ranges_per_cta = br;
        g.ctx->blocks_per_sm = bb;
        if (!st) {
            const domagg_status ss = domagg_sync_status(g.ctx, stream);
            if (ss) st = plan_fail(p, ss, g.ctx->err);
        }
        total += best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = total;
    return st;
}

int64_t domagg_plan_workspace_bytes(domagg_plan p) {
    if (!p) return -1;
    int64_t b = 0;
    for (auto& g : p->groups) b += (int64_t)g.ctx->held();
    return b;
}

domagg_status domagg_plan_destroy(domagg_plan p) {
    if (!p) return DOMAGG_ERR_INVALID_ARG;
    plan_free(p);
    return DOMAGG_OK;
}

domagg_status domagg_selftest_timeout(domagg_handle h, int which, void* stream) {
    if (!h || (which != 0 && which != 1)) return DOMAGG_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    const cudaStream_t s = (cudaStream_t)stream;
    domagg_status st = grow(h, h->st_multi, 4096, true);  // a zeroed status word to wait on
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "selftest");
    cudaMemsetAsync(&h->ctl->error, 0, sizeof(u32), s);
    k_selftest_wait<<<1, 32, 0, s>>>(which, (const u64*)h->st_multi.p, h->ctl);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "selftest launch");
    return domagg_sync_status(h, stream);
}

domagg_status domagg_sync_status(domagg_handle h, void* stream) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    if (const u32 site = bounds_site(true)) return bounds_error(h, site);
    u32 bits = 0;
    e = cudaMemcpy(&bits, &h->ctl->error, sizeof(u32), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    if (bits) {
        cudaMemset(&h->ctl->error, 0, sizeof(u32));
        cudaDeviceSynchronize();
        return device_error(h, bits);
    }
    return DOMAGG_OK;
}

const char* domagg_last_error(domagg_handle h) { return h ? h->err.c_str() : "null handle"; }

domagg_status domagg_get_stats(domagg_handle h, domagg_stats* out) {
    if (!h || !out) return DOMAGG_ERR_INVALID_ARG;
    *out = h->stats;
    out->workspace_bytes = (int64_t)h->held();
    return DOMAGG_OK;
}

domagg_status domagg_timing_enable(domagg_handle h, int enable) {
    if (!h) return DOMAGG_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return DOMAGG_OK;
}

domagg_status domagg_timing_read(domagg_handle h, domagg_timing* out) {
    if (!h || !out) return DOMAGG_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    cudaSetDevice(h->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "timing");
    for (const TimedLaunch& t : h->log) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        if (t.kind < 0 || t.kind >= DOMAGG_TIMING_KINDS) continue;
        out->launches[t.kind] += 1;
        out->ms[t.kind] += ms;
        out->bytes[t.kind] += t.bytes;
    }
    h->log.clear();
    h->pool_used = 0;
    return DOMAGG_OK;
}

const char* domagg_timing_kind_name(int kind) {
    static const char* names[] = {"encode",  "hist_points",  "sort_points", "rank",     "count_scan",
                                  "expand",  "hist_records", "sort_records", "segscan", "reduce",
                                  "small",   "h2d",          "d2h",          "wavelet",  "sort_groups",
                                  "group",   "top"};
    if (kind < 0 || kind >= (int)(sizeof(names) / sizeof(names[0]))) return "";
    return names[kind];
}

#ifdef DOMAGG_CHECKED
const char* domagg_version(void) { return "domagg 0.2 (sm_103a, checked build)"; }
#else
const char* domagg_version(void) { return "domagg 0.2 (sm_103a)"; }
#endif

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward pass without any allocation, for callers that cannot allocate
// device memory: code that runs where cudaMalloc is not allowed or not
// wanted (an allocator-free runtime, a caller that reserves all device
// memory up front, a real-time path that must not block in the allocator).
// The paper has no counterpart; this is a deployment convenience.
//
// All scratch (control block, point and record buffers, look-back status
// words) lives in one file-scope device array of NOALLOC_BYTES.  Every GPU
// that loads this library holds that array until the process exits.  Calls
// share it and it keeps the last call's contents: the control block and the
// status words are zeroed once per device when the entry point first runs,
// and the look-back epochs keep later calls from reading stale statuses.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t NOALLOC_BYTES = (size_t)32 << 20;
constexpr size_t NOALLOC_CTL = 4096;
constexpr size_t NOALLOC_PTS = (size_t)8 << 20;
constexpr size_t NOALLOC_STM = (size_t)4 << 20;
constexpr size_t NOALLOC_STS = (size_t)1 << 20;
constexpr size_t NOALLOC_RECS = NOALLOC_BYTES - NOALLOC_CTL - NOALLOC_PTS - NOALLOC_STM - NOALLOC_STS;
constexpr int64_t NOALLOC_MAX_POINTS = 65536;
constexpr int NOALLOC_MAX_DEVICES = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
struct NoAllocSlot {
    bool ready = false;
    domagg_ctx ctx;
    alignas(64) unsigned char host_stage[16384];  // instance table and counts (pageable)
};
NoAllocSlot g_noalloc[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

// Once per device, with that device current: the device address of the
// scratch array (its name in host code is only a stand-in), zeroed control
// block and status words, and a handle whose buffers are fixed slices of it.
domagg_status noalloc_setup(int dev, domagg_ctx** out) {
    NoAllocSlot& S = g_noalloc[dev];
    if (!S.ready) {
        unsigned char* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) {
            S.ctx.err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            *out = &S.ctx;
            return DOMAGG_ERR_CUDA;
        }
        e = cudaMemset(ptr, 0, NOALLOC_CTL + NOALLOC_PTS);  // control block (and points, harmlessly)
        if (e == cudaSuccess) e = cudaMemset(ptr + NOALLOC_CTL + NOALLOC_PTS + NOALLOC_RECS, 0, NOALLOC_STM + NOALLOC_STS);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            S.ctx.err = std::string("clearing the scratch: ") + cudaGetErrorString(e);
            *out = &S.ctx;
            return DOMAGG_ERR_CUDA;
        }
        domagg_ctx& h = S.ctx;
        h.device = dev;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) h.sms = sms;
        else cudaGetLastError();  // keep the default of 152
        h.ctl = reinterpret_cast<Ctl*>(ptr);
        h.pts = {ptr + NOALLOC_CTL, NOALLOC_PTS};
        h.recs = {ptr + NOALLOC_CTL + NOALLOC_PTS, NOALLOC_RECS};
        h.st_multi = {ptr + NOALLOC_CTL + NOALLOC_PTS + NOALLOC_RECS, NOALLOC_STM};
        h.st_seg = {ptr + NOALLOC_CTL + NOALLOC_PTS + NOALLOC_RECS + NOALLOC_STM, NOALLOC_STS};
        h.stage = {nullptr, 0};
        // every buffer is full-size and the cap equals their sum, so a request
        // that does not fit is refused before anything could be freed
        h.max_ws = h.held();
        h.h_pin = S.host_stage;
        h.h_pin_cap = sizeof(S.host_stage);
        h.timing = false;
        // grow() and grow_pinned() refuse (DOMAGG_ERR_OOM, reported as
        // UNSUPPORTED) instead of freeing these slices or allocating
        h.no_alloc = true;
        S.ready = true;
    }
    *out = &S.ctx;
    return DOMAGG_OK;
}
}  // namespace

extern "C" domagg_status domagg_forward_noalloc(int m, const void* d_coords, int64_t nD, const void* q_coords,
                                                int64_t nQ, domagg_dtype coord_dtype, const void* d_weights,
                                                domagg_dtype weight_dtype, domagg_op op, void* out, void* stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return DOMAGG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    domagg_ctx* h = nullptr;
    domagg_status st = noalloc_setup(dev, &h);
    if (st) return st;
    st = check_common(h, m, nD, nQ, coord_dtype, weight_dtype, op);
    if (st) return st;
    if (nD + nQ > NOALLOC_MAX_POINTS)
        return fail(h, DOMAGG_ERR_UNSUPPORTED, "domagg_forward_noalloc takes at most 65536 points (nD + nQ)");
    if ((nD > 0 && !d_coords) || (nQ > 0 && (!q_coords || !out)) || (op != DOMAGG_COUNT && nD > 0 && !d_weights))
        return fail(h, DOMAGG_ERR_INVALID_ARG, "null pointer");
    if (nQ == 0) return DOMAGG_OK;
    std::vector<Inst> inst{make_inst(d_coords, nD, q_coords, nQ, d_weights, out)};
    st = dispatch(h, m, inst, coord_dtype, weight_dtype, op, false, (cudaStream_t)stream);
    if (st == DOMAGG_ERR_OOM)
        return fail(h, DOMAGG_ERR_UNSUPPORTED,
                    "the flat map of this input does not fit the 32 MiB static scratch of domagg_forward_noalloc");
    return st;
}
