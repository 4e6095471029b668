// APRIL intermediate filter on sm_103a: context, device upload, and the
// filter kernels behind april_filter_pairs.
//
// Every kernel computes, per candidate pair (r, s), Algorithm 2 of the paper
// (Sec. 4.2): IntervalJoin(A(r), A(s)); if it finds no overlap the pair is a
// true negative; else IntervalJoin(A(r), F(s)) or IntervalJoin(F(r), A(s))
// finding an overlap makes it a true hit; else it is inconclusive.
//
// Interval convention: [st, end) with end stored mod 2^32; all comparisons
// use last = end - 1 (uint32), so an interval that reaches cell 2^32-1 works.
//   X_i overlaps Y_j   <=>  X_i.st <= Y_j.last  and  Y_j.st <= X_i.last
//   merge step         :    advance X if X_i.last <= Y_j.last, else Y.
//
// Parallel joins.  "Does any interval of X overlap one of Y" has one answer
// however the merge is split.  The sequential merge visits the states
// (i, j) of the merge path of X and Y ordered by `last` (ties: X first) and
// at each state tests X_i against Y_j; the element emitted at that state is
// the smaller of the two.  So the set of tests the merge performs is
//   { (X_i, Y_rank_Y(X_i)) }  u  { (X_rank_X(Y_j), Y_j) }
// where rank_Y(X_i) = #{ j : Y_j.last < X_i.last } and
//       rank_X(Y_j) = #{ i : X_i.last <= Y_j.last }.
// A group of lanes loads a window of both lists, computes these ranks inside
// the window by binary search over registers (shuffles), runs the tests of
// the first W merge positions at once, and advances by the number of X and Y
// elements those W positions consumed.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "april_internal.h"
#include "geom.h"
#include "join_device.cuh"

using namespace april_dev;

namespace {

// status bits in the context's device status block
constexpr uint32_t ST_BAD_ID = 1u;
constexpr uint32_t ST_TIMEOUT = 2u;
static_assert(kMbarSpinLimit == APRIL_WAIT_LIMIT_DEFAULT, "the documented default wait limit");

constexpr uint32_t kBlock = 256;                 // threads per CTA for K1/K3
constexpr uint32_t kWarpsPerBlock = kBlock / 32;
constexpr uint32_t kWarpWMax = 256;              // largest warp window per list
constexpr uint32_t kCtaWMax = 2048;              // largest CTA window per list
// cta_threshold value meaning "no long pairs": every pair goes to the lane
// groups, whatever its length, and the binning kernel is not launched
constexpr uint32_t kNoLongPairs = 0xffffffffu;
// join_order value meaning: AA, AF, FA when the triage ran (the pairs left are
// mostly true negatives and inconclusive pairs, which AA settles or must
// see), AF, AA, FA otherwise (most true hits end in AF)
constexpr uint32_t kJoinOrderAuto = 2;
static inline uint32_t join_order_of(uint32_t jo, bool triaged) {
    return jo == kJoinOrderAuto ? (triaged ? 1u : 0u) : jo;
}
constexpr uint32_t kWarpFirstWindow = 64;        // first window of a join in APRIL_MODE_WARP
constexpr uint32_t kWarpBuf = kWarpWMax + 2;     // staging buffer per list (odd start + rounding)
constexpr uint32_t kCtaBuf = kCtaWMax + 2;
// Compile-time knobs (defaults are the shipped configuration):
//   APRIL_MIN_BLOCKS  minimum resident CTAs per SM requested for k_persistent
//   APRIL_GROUP_PER   diagonals each lane walks per window in the group engine
//   APRIL_GENERAL_MIN_BLOCKS  minimum resident CTAs per SM requested for k_general
//   APRIL_STAGE2      1: a lane group's two windows are copied by two lanes (mbarrier count 2)
#ifdef APRIL_MIN_BLOCKS
#define APRIL_PERSISTENT_BOUNDS __launch_bounds__(256, APRIL_MIN_BLOCKS)
#else
// the lane-group instances over raw lists run five CTAs per SM (at most 51
// registers a thread: their warps wait on memory, more of them hide more);
// the others leave the register count to the compiler
#define APRIL_PERSISTENT_BOUNDS __launch_bounds__(256, (G < 32 && !SetsT::kPacked) ? 5 : 0)
#endif
#ifndef APRIL_STAGE2
#define APRIL_STAGE2 1
#endif
constexpr bool kStage2 = APRIL_STAGE2 != 0;  // lane groups stage their two windows from two lanes
#ifndef APRIL_GROUP_PER
#define APRIL_GROUP_PER 8
#endif
constexpr uint32_t kGroupPer = APRIL_GROUP_PER;
// intervals of shared staging per warp for kernels with whole-warp joins only
// (K1, K7): two windows of a warp, and a CTA's two windows across its warps
constexpr uint32_t kWarpShare = 2 * (kWarpWMax + 2);
constexpr uint32_t kSharedIv = kWarpsPerBlock * kWarpShare > 2 * kCtaBuf ? kWarpsPerBlock * kWarpShare : 2 * kCtaBuf;
static_assert(kWarpBuf % 2 == 0 && kCtaBuf % 2 == 0, "buffers must stay 16-byte aligned");

// scratch of the batched mode: counters, the list of long pairs, the routed
// entries of partitioned sets, then the queue of joins handed from the lane
// groups to whole warps (one uint4 {pair, step, i0, j0} each, room for a
// quarter of the pairs; when it is full a group finishes its join itself)
constexpr uint32_t C_BIG_COUNT = 0, C_BIG_HEAD = 1, C_CHUNK_HEAD = 2, C_ESC_COUNT = 3, C_ESC_HEAD = 4,
                   C_REST_COUNT = 5;
static inline uint64_t esc_capacity(uint64_t n) { return (n + 3) / 4; }
constexpr uint32_t kMaxEscalateWindows = 64;
constexpr size_t kCounterBytes = 256;

__device__ __forceinline__ uint4 shfl4(const uint4 &v, uint32_t src) {
    return make_uint4(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src), __shfl_sync(kFull, v.z, src),
                      __shfl_sync(kFull, v.w, src));
}

// Entry-level views of a set for the warp and CTA joins.  RawSets reads the
// interval lists; PackedSets reads the compressed lists of Sec. 5.1.
struct RawSets {
    static constexpr bool kPacked = false;
    DevSet s;
    using Desc = uint4;  // {a_off, a_len, f_off, f_len}
    __device__ __forceinline__ uint32_t n() const { return s.n; }
    __device__ __forceinline__ Desc load(uint32_t e) const { return __ldg(s.desc + e); }
    static __device__ __forceinline__ uint32_t a_len(const Desc &d) { return d.y; }
    static __device__ __forceinline__ Desc shfl(const Desc &d, uint32_t src) { return shfl4(d, src); }
    __device__ __forceinline__ RawList list(const Desc &d, bool f) const {
        const uint32_t off = f ? d.z : d.x;
        return RawList{s.iv + off, f ? d.w : d.y, s.posts + off / 16};
    }
};

struct PackedSets {
    static constexpr bool kPacked = true;
    const uint4 *pdesc;    // per entry {a_block, a_len, f_block, f_len}
    const uint2 *blocks;   // block table {anchor, gap_off64 | wide << 31}
    const uint8_t *gaps;
    uint32_t nent;
    using Desc = uint4;
    __device__ __forceinline__ uint32_t n() const { return nent; }
    __device__ __forceinline__ Desc load(uint32_t e) const { return __ldg(pdesc + e); }
    static __device__ __forceinline__ uint32_t a_len(const Desc &d) { return d.y; }
    static __device__ __forceinline__ Desc shfl(const Desc &d, uint32_t src) { return shfl4(d, src); }
    __device__ __forceinline__ PackedList list(const Desc &d, bool f) const {
        return f ? PackedList{blocks + d.z, gaps, d.w} : PackedList{blocks + d.x, gaps, d.y};
    }
};

// ------------------------------------------------------- K0: thread/pair
__global__ void __launch_bounds__(256) k_plain(DevSet R, DevSet S, const uint32_t *__restrict__ pr,
                                               const uint32_t *__restrict__ ps, uint64_t n,
                                               uint8_t *__restrict__ out, uint32_t *status) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = __ldg(pr + k), s = __ldg(ps + k);
        if (r >= R.n || s >= S.n) {
            out[k] = APRIL_VERDICT_ERROR;
            atomicOr(status, ST_BAD_ID);
            continue;
        }
        const uint4 dr = __ldg(R.desc + r), ds = __ldg(S.desc + s);
        uint8_t v;
        if (!seq_join(R.iv + dr.x, dr.y, S.iv + ds.x, ds.y)) v = APRIL_TRUE_NEGATIVE;
        else if (seq_join(R.iv + dr.x, dr.y, S.iv + ds.z, ds.w)) v = APRIL_TRUE_HIT;
        else if (seq_join(R.iv + dr.z, dr.w, S.iv + ds.x, ds.y)) v = APRIL_TRUE_HIT;
        else v = APRIL_INCONCLUSIVE;
        out[k] = v;
    }
}

// Algorithm 2 for one pair by one warp: AA; if no overlap, a true negative;
// else AF, then FA.
// Shared-memory synchronisation state of a warp or CTA join: the mbarrier the
// window copies complete on, its phase bit, and a timeout flag.
struct JoinSync;

// The order of a pair's joins in the batched kernels (april_tune.join_order).
// The verdicts of Sec. 4.2 do not depend on it (F is a subset of A, so an AF
// or FA overlap implies an AA overlap).
//   order 0, AF AA FA: AF first settles most true hits in one join; a pair
//     without an AF overlap takes AA (none: true negative), then FA.
//   order 1, AA AF FA (Algorithm 2's): a true negative takes one join.
// Step s joins X = F(r) when s == 2 (else A(r)) with Y = F(s) when s is the
// AF step (else A(s)).  A join with an empty list has no overlap.
__device__ __forceinline__ bool step_x_f(uint32_t s, uint32_t jo) { return s == 2; }
__device__ __forceinline__ bool step_y_f(uint32_t s, uint32_t jo) { return s == (jo ? 1u : 0u); }
// The verdict after step s found `overlap` (>= 0), or -1 with s advanced.
__device__ __forceinline__ int step_outcome(uint32_t &s, bool overlap, uint32_t jo) {
    if (s == 2) return overlap ? APRIL_TRUE_HIT : APRIL_INCONCLUSIVE;
    const bool aa = (s == 0) == (jo != 0);  // this step is AA
    if (aa && !overlap) return APRIL_TRUE_NEGATIVE;
    if (!aa && overlap) return APRIL_TRUE_HIT;
    ++s;
    return -1;
}

struct JoinSync {
    uint32_t bar;
    uint32_t phase;
    bool timeout;
};

// With resume, the pair's join step st0 continues from merge position
// (ri, rj), where the lane groups left it (see k_long).
template <class SetsT>
__device__ __forceinline__ uint8_t warp_verdict(const SetsT &R, const SetsT &S, const typename SetsT::Desc &dr,
                                                const typename SetsT::Desc &ds, uint2 *xs, uint2 *ys, uint32_t lane,
                                                uint32_t w0, JoinSync &js, uint32_t jo, uint32_t st0 = 0,
                                                bool resume = false, uint32_t ri = 0, uint32_t rj = 0) {
    uint32_t st = st0;
    for (;;) {
        const bool ov = tile_join<WarpScope, 32, kWarpWMax>(R.list(dr, step_x_f(st, jo)), S.list(ds, step_y_f(st, jo)),
                                                            xs, ys, nullptr, lane, w0, js.bar, &js.phase, &js.timeout,
                                                            0, 0, resume, ri, rj);
        if (js.timeout) return APRIL_VERDICT_ERROR;
        resume = false;
        const int v = step_outcome(st, ov, jo);
        if (v >= 0) return (uint8_t)v;
    }
}

// The same for one pair by the whole CTA.
template <class SetsT>
__device__ __forceinline__ uint8_t cta_verdict(const SetsT &R, const SetsT &S, const typename SetsT::Desc &dr,
                                               const typename SetsT::Desc &ds, uint2 *xs, uint2 *ys, uint32_t *slot,
                                               uint32_t tid, uint32_t w0, JoinSync &js, uint32_t jo) {
    uint32_t st = 0;
    for (;;) {
        const bool ov = tile_join<CtaScope, kBlock, kCtaWMax>(R.list(dr, step_x_f(st, jo)), S.list(ds, step_y_f(st, jo)),
                                                              xs, ys, slot, tid, w0, js.bar, &js.phase, &js.timeout);
        if (js.timeout) return APRIL_VERDICT_ERROR;
        const int v = step_outcome(st, ov, jo);
        if (v >= 0) return (uint8_t)v;
    }
}

// One warp filters the 32 pairs starting at `base`: every lane fetches the
// ids and descriptors of its own pair at once (coalesced ids, 32 descriptor
// gathers in flight), then the warp joins the pairs one after another.  Pairs
// whose cost |A(r)| + |A(s)| exceeds cta_threshold are left to the CTA phase
// (pass UINT32_MAX to take every pair).
template <class SetsT>
__device__ __forceinline__ bool warp_chunk(const SetsT &R, const SetsT &S, const uint32_t *__restrict__ pr,
                                           const uint32_t *__restrict__ ps, uint64_t n, uint64_t base,
                                           uint8_t *__restrict__ out, uint32_t *status, uint2 *xs, uint2 *ys,
                                           uint32_t lane, uint32_t w0, uint32_t cta_threshold, bool flag_bad,
                                           JoinSync &js, uint32_t jo) {
    const uint64_t k = base + lane;
    typename SetsT::Desc dr{}, ds{};
    bool take = false;
    if (k < n) {
        const uint32_t r = __ldg(pr + k), s = __ldg(ps + k);
        if (r < R.n() && s < S.n()) {
            dr = R.load(r);
            ds = S.load(s);
            take = cta_threshold == kNoLongPairs ||
                   (uint64_t)SetsT::a_len(dr) + SetsT::a_len(ds) <= (uint64_t)cta_threshold;
        } else if (flag_bad) {
            out[k] = APRIL_VERDICT_ERROR;
            atomicOr(status, ST_BAD_ID);
        }
    }
    uint32_t todo = __ballot_sync(kFull, take);
    uint8_t mine = 0;
    while (todo) {
        const uint32_t t = __ffs(todo) - 1;
        todo &= todo - 1;
        const typename SetsT::Desc a = SetsT::shfl(dr, t), b = SetsT::shfl(ds, t);
        const uint8_t v = warp_verdict(R, S, a, b, xs, ys, lane, w0, js, jo);
        if (lane == t) mine = v;
        if (js.timeout) {  // the pairs of the chunk not decided yet read as errors
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            if (take) out[k] = (lane == t || ((todo >> lane) & 1u)) ? (uint8_t)APRIL_VERDICT_ERROR : mine;
            return false;
        }
    }
    if (take) out[k] = mine;
    return true;
}

// Initialises `count` mbarriers (8 bytes each, 8-byte aligned) at bars;
// every thread of the block must call it.
__device__ __forceinline__ void init_barriers(uint64_t *bars, uint32_t count) {
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) mbar_init(smem_addr(bars + i), 1);
    if (threadIdx.x == 0) mbar_init_fence();
    __syncthreads();
}

// ------------------------------------------------------- K1: warp/pair
__global__ void __launch_bounds__(kBlock) k_warp(DevSet R, DevSet S, const uint32_t *__restrict__ pr,
                                                 const uint32_t *__restrict__ ps, uint64_t n,
                                                 uint8_t *__restrict__ out, uint32_t *status, uint32_t w0,
                                                 uint32_t jo) {
    __shared__ __align__(16) uint2 sm[kWarpsPerBlock][2][kWarpBuf];
    __shared__ uint64_t bars[kWarpsPerBlock];
    init_barriers(bars, kWarpsPerBlock);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    JoinSync js{smem_addr(&bars[warp]), 0u, false};
    const uint64_t stride = (uint64_t)gridDim.x * kWarpsPerBlock * 32;
    for (uint64_t base = ((uint64_t)blockIdx.x * kWarpsPerBlock + warp) * 32; base < n; base += stride)
        if (!warp_chunk(RawSets{R}, RawSets{S}, pr, ps, n, base, out, status, sm[warp][0], sm[warp][1], lane, w0,
                        0xffffffffu, true, js, jo))
            return;
}

// --------------------------------------------- K4: length binning (batched)
// Validates ids (error verdicts), and appends every pair whose cost
// |A(r)| + |A(s)| exceeds the threshold to the long-pair list (warp-
// aggregated atomics).  Not launched when the threshold is kNoLongPairs: the
// lane groups then take every pair and report bad ids themselves.
template <class SetsT>
__global__ void __launch_bounds__(256) k_bin(SetsT R, SetsT S, const uint32_t *__restrict__ pr,
                                             const uint32_t *__restrict__ ps, uint64_t n, uint8_t *__restrict__ out,
                                             uint32_t *status, uint32_t cta_threshold, uint32_t *big_list,
                                             uint32_t *counters) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t kb = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); kb < n; kb += stride) {
        const uint64_t k = kb + lane;
        bool big = false;
        if (k < n) {
            const uint32_t r = __ldg(pr + k), s = __ldg(ps + k);
            if (r < R.n() && s < S.n()) {
                big = (uint64_t)SetsT::a_len(R.load(r)) + SetsT::a_len(S.load(s)) > (uint64_t)cta_threshold;
            } else {
                out[k] = APRIL_VERDICT_ERROR;
                atomicOr(status, ST_BAD_ID);
            }
        }
        const uint32_t mask = __ballot_sync(kFull, big);
        if (mask) {
            const uint32_t leader = __ffs(mask) - 1;
            uint32_t pos = 0;
            if (lane == leader) pos = atomicAdd(&counters[C_BIG_COUNT], __popc(mask));
            pos = __shfl_sync(kFull, pos, leader) + __popc(mask & ((1u << lane) - 1u));
            if (big) big_list[pos] = (uint32_t)k;
        }
    }
}

// --------------------------------------------------- K2: triage (batched)
// A true hit proven by one cell.  The cell c under the centre of
// MBR(r) n MBR(s), on the sets' grid, is looked up in A(r) and F(s), then in
// F(r) and A(s): if one pair of lists holds it, the AF or FA join has an
// overlap and Algorithm 2's verdict is a true hit (Sec. 4.2: an AF or FA
// overlap implies the AA one, so the verdict is the same in any join order).
// The pairs the probe does not settle are listed, with warp-aggregated
// appends, for the lane groups; out-of-range ids get error verdicts.  A
// thread takes two pairs at once (k_triage).  A lookup is a binary search
// over the list's skip index (posts below c), then over the at most 16
// intervals that follow; over compressed lists, over the block table, then
// one block decoded.
struct TriageGrid {
    int64_t ox, oy;
    uint32_t log2_cell, order;
};

// The table of april_geom::hilbert_lut_build, passed by value to the
// triage kernel, which copies it to shared memory.
struct HilbertLut {
    uint8_t e[64];
};

static HilbertLut triage_lut() {
    HilbertLut L{};
    april_geom::hilbert_lut_build(L.e);
    return L;
}

// Lookups of cell c0 in list L0 and of c1 in L1 (for two pairs a thread
// handles at once), each only where `on`: binary searches in lockstep, so that
// their loads overlap.  A list holds cell c when its first interval whose
// last cell reaches c starts at or before c; the search runs over the list's
// skip index (posts below c), then over the at most 16 intervals that follow.
__device__ __forceinline__ void holds2(const RawList &L0, uint32_t c0, bool on0, const RawList &L1, uint32_t c1,
                                       bool on1, bool &h0, bool &h1) {
    on0 = on0 && L0.n;
    on1 = on1 && L1.n;
    uint32_t lo0 = 0, hi0 = on0 ? L0.keys_n() : 0u, lo1 = 0, hi1 = on1 ? L1.keys_n() : 0u;
    while (lo0 < hi0 || lo1 < hi1) {
        const bool a0 = lo0 < hi0, a1 = lo1 < hi1;
        const uint32_t m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
        const uint32_t k0 = a0 ? L0.key(m0) : 0u, k1 = a1 ? L1.key(m1) : 0u;
        if (a0) {
            if (k0 < c0) lo0 = m0 + 1;
            else hi0 = m0;
        }
        if (a1) {
            if (k1 < c1) lo1 = m1 + 1;
            else hi1 = m1;
        }
    }
    uint32_t a = on0 ? L0.start_of(lo0) : 0u, b = on0 ? min(L0.n, a + 16u) : 0u;
    uint32_t p = on1 ? L1.start_of(lo1) : 0u, q = on1 ? min(L1.n, p + 16u) : 0u;
    while (a < b || p < q) {
        const bool a0 = a < b, a1 = p < q;
        const uint32_t m0 = (a + b) >> 1, m1 = (p + q) >> 1;
        const uint32_t l0 = a0 ? __ldg(&L0.p[m0].y) - 1u : 0u, l1 = a1 ? __ldg(&L1.p[m1].y) - 1u : 0u;
        if (a0) {
            if (l0 < c0) a = m0 + 1;
            else b = m0;
        }
        if (a1) {
            if (l1 < c1) p = m1 + 1;
            else q = m1;
        }
    }
    const bool r0 = on0 && a < L0.n, r1 = on1 && p < L1.n;
    const uint32_t s0 = r0 ? __ldg(&L0.p[a].x) : 0u, s1 = r1 ? __ldg(&L1.p[p].x) : 0u;
    h0 = r0 && s0 <= c0;
    h1 = r1 && s1 <= c1;
}

// Whether a block of a compressed list (ne of its 32 endpoints in the list)
// holds cell c: its endpoints (the anchor, then the gaps at gw, read with
// 16-byte loads, 16-bit or 32-bit) taken as [start, end) pairs.  The 32
// endpoints of a block are 16 whole intervals.
template <bool WIDE>
__device__ __forceinline__ bool block_holds(const uint4 *gw, uint32_t anchor, uint32_t ne, uint32_t c) {
    constexpr uint32_t PER = WIDE ? 4u : 8u, WORDS = 32u / PER;
    uint32_t e = anchor, st = 0;
    bool held = false;
#pragma unroll
    for (uint32_t w = 0; w < WORDS; ++w) {
        const uint4 q = __ldg(gw + w);
        const uint32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (uint32_t i = 0; i < PER; ++i) {
            const uint32_t j = w * PER + i;  // slot j gives endpoint j (slot 0: the anchor itself)
            const uint32_t gap = WIDE ? v[i] : (i & 1u ? v[i >> 1] >> 16 : v[i >> 1] & 0xFFFFu);
            if (j > 0) e += gap;
            if (j < ne) {
                if (!(j & 1u)) st = e;
                else held = held || (st <= c && c <= e - 1u);
            }
        }
    }
    return held;
}

// Whether compressed lists L0 and L1 (Sec. 5.1 blocks of 32 endpoints: an
// anchor and 31 gaps) hold cells c0 and c1 (for two pairs a thread handles
// at once), each only where `on`: the last block whose anchor (the start of
// its first interval) is at most c, by binary searches over the block tables
// in lockstep (an earlier block's intervals end before that anchor, a later
// block's start after c), then that block decoded.
__device__ __forceinline__ void holds2_packed(const PackedList &L0, uint32_t c0, bool on0, const PackedList &L1,
                                              uint32_t c1, bool on1, bool &h0, bool &h1) {
    on0 = on0 && L0.n;
    on1 = on1 && L1.n;
    uint32_t lo0 = 0, hi0 = on0 ? (2 * L0.n + 31) / 32 : 0u, lo1 = 0, hi1 = on1 ? (2 * L1.n + 31) / 32 : 0u;
    while (lo0 < hi0 || lo1 < hi1) {
        const bool a0 = lo0 < hi0, a1 = lo1 < hi1;
        const uint32_t m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
        const uint32_t k0 = a0 ? __ldg(&L0.blocks[m0].x) : 0u, k1 = a1 ? __ldg(&L1.blocks[m1].x) : 0u;
        if (a0) {
            if (k0 <= c0) lo0 = m0 + 1;
            else hi0 = m0;
        }
        if (a1) {
            if (k1 <= c1) lo1 = m1 + 1;
            else hi1 = m1;
        }
    }
    on0 = on0 && lo0 > 0;
    on1 = on1 && lo1 > 0;
    const uint2 m0 = on0 ? __ldg(L0.blocks + lo0 - 1) : make_uint2(0, 0);
    const uint2 m1 = on1 ? __ldg(L1.blocks + lo1 - 1) : make_uint2(0, 0);
    h0 = h1 = false;
    if (on0) {
        const uint4 *gw = (const uint4 *)(L0.gaps + 64ull * (m0.y & 0x7FFFFFFFu));
        const uint32_t ne = min(32u, 2 * L0.n - 32 * (lo0 - 1));
        h0 = m0.y >> 31 ? block_holds<true>(gw, m0.x, ne, c0) : block_holds<false>(gw, m0.x, ne, c0);
    }
    if (on1) {
        const uint4 *gw = (const uint4 *)(L1.gaps + 64ull * (m1.y & 0x7FFFFFFFu));
        const uint32_t ne = min(32u, 2 * L1.n - 32 * (lo1 - 1));
        h1 = m1.y >> 31 ? block_holds<true>(gw, m1.x, ne, c1) : block_holds<false>(gw, m1.x, ne, c1);
    }
}

// The lookups of two pairs' cells, in lockstep: raw lists (holds2),
// compressed lists (holds2_packed).
__device__ __forceinline__ void lookup2(const RawList &L0, uint32_t c0, bool on0, const RawList &L1, uint32_t c1,
                                        bool on1, bool &h0, bool &h1) {
    holds2(L0, c0, on0, L1, c1, on1, h0, h1);
}
__device__ __forceinline__ void lookup2(const PackedList &L0, uint32_t c0, bool on0, const PackedList &L1, uint32_t c1,
                                        bool on1, bool &h0, bool &h1) {
    holds2_packed(L0, c0, on0, L1, c1, on1, h0, h1);
}

// The probe cell of pair (r, s): the cell under the centre of
// MBR(r) n MBR(s); false when the MBRs are disjoint or the centre is off the grid.
__device__ __forceinline__ bool triage_cell(const int4 *__restrict__ mbr_r, const int4 *__restrict__ mbr_s,
                                            const TriageGrid &g, const uint8_t *lut, uint32_t r, uint32_t s,
                                            uint32_t &c) {
    const int4 a = __ldg(mbr_r + r), b = __ldg(mbr_s + s);
    const int64_t x0 = max(a.x, b.x), y0 = max(a.y, b.y), x1 = min(a.z, b.z), y1 = min(a.w, b.w);
    if (x0 > x1 || y0 > y1) return false;
    const int64_t cx = ((x0 + x1) / 2 - g.ox) >> g.log2_cell, cy = ((y0 + y1) / 2 - g.oy) >> g.log2_cell;
    const int64_t side = (int64_t)1 << g.order;
    if (cx < 0 || cy < 0 || cx >= side || cy >= side) return false;
    c = (uint32_t)april_geom::hilbert_id_lut(lut, g.order, (uint32_t)cx, (uint32_t)cy);
    return true;
}

// One thread per two pairs (k and k + 32 of its warp's 64): ids, probe cells,
// then F(s) and, where it holds the cell, A(r); then F(r) and A(s) for the
// pairs not settled yet.  Over partitioned sets (PART, Sec. 5.2) the pairs'
// entries come from the routing (er, es), the MBRs from the objects (pr, ps),
// and the grid from the entry's partition.  The rest list holds pair indices
// plus k_base (a launch over one chunk of a longer pair array).  Six CTAs per
// SM (at most 40 registers a thread): the kernel waits on chains of dependent
// loads, and more threads hide more.
#ifndef APRIL_TRIAGE_MIN_BLOCKS
#define APRIL_TRIAGE_MIN_BLOCKS 6
#endif
struct TriageArgs {
    const int4 *mbr_r, *mbr_s;
    TriageGrid g;                // one-grid sets
    const int64_t *part_grid;    // PART: per partition {ox, oy, log2_cell, used}
    const uint32_t *entry_pid;   // PART: R's entries' partitions
    const uint32_t *er, *es;     // PART: the routed entries of the pairs
};

template <bool PART, class SetsT>
__global__ void __launch_bounds__(256, APRIL_TRIAGE_MIN_BLOCKS) k_triage(SetsT R, SetsT S, TriageArgs ta,
                                                                          HilbertLut lut_in,
                                                                          const uint32_t *__restrict__ pr,
                                                                          const uint32_t *__restrict__ ps, uint64_t n,
                                                                          uint8_t *__restrict__ out, uint32_t *status,
                                                                          uint32_t *rest, uint32_t *counters,
                                                                          uint32_t k_base) {
    __shared__ uint8_t lut[64];
    if (threadIdx.x < 64) lut[threadIdx.x] = lut_in.e[threadIdx.x];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t stride = 2ull * gridDim.x * blockDim.x;
    for (uint64_t kb = 2ull * ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)); kb < n; kb += stride) {
        const uint64_t k[2] = {kb + lane, kb + 32 + lane};
        bool valid[2], probe[2] = {false, false}, hit[2] = {false, false};
        uint32_t c[2] = {0, 0};
        uint4 dr[2], ds[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            valid[h] = false;
            dr[h] = ds[h] = make_uint4(0, 0, 0, 0);
            if (k[h] < n) {
                uint32_t r = __ldg(pr + k[h]), s = __ldg(ps + k[h]);  // objects
                const uint32_t ro = r, so = s;
                if constexpr (PART) {  // their entries (out of range when the routing found none)
                    r = __ldg(ta.er + k[h]);
                    s = __ldg(ta.es + k[h]);
                }
                if (r < R.n() && s < S.n()) {
                    valid[h] = true;
                    dr[h] = R.load(r);
                    ds[h] = S.load(s);
                    if constexpr (PART) {
                        const int64_t *pg = ta.part_grid + 4 * (size_t)__ldg(ta.entry_pid + r);
                        const TriageGrid g{__ldg(pg), __ldg(pg + 1), (uint32_t)__ldg(pg + 2), ta.g.order};
                        probe[h] = __ldg(pg + 3) != 0 && triage_cell(ta.mbr_r, ta.mbr_s, g, lut, ro, so, c[h]);
                    } else {
                        probe[h] = triage_cell(ta.mbr_r, ta.mbr_s, ta.g, lut, ro, so, c[h]);
                    }
                } else {
                    out[k[h]] = APRIL_VERDICT_ERROR;
                    atomicOr(status, ST_BAD_ID);
                }
            }
        }
        bool f0, f1;
        lookup2(S.list(ds[0], true), c[0], probe[0], S.list(ds[1], true), c[1], probe[1], f0, f1);  // F(s)
        lookup2(R.list(dr[0], false), c[0], f0, R.list(dr[1], false), c[1], f1, hit[0], hit[1]);    // A(r)
        lookup2(R.list(dr[0], true), c[0], probe[0] && !hit[0], R.list(dr[1], true), c[1], probe[1] && !hit[1], f0,
                f1);                                                                                   // F(r)
        bool g0, g1;
        lookup2(S.list(ds[0], false), c[0], f0, S.list(ds[1], false), c[1], f1, g0, g1);            // A(s)
        hit[0] = hit[0] || g0;
        hit[1] = hit[1] || g1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (valid[h] && hit[h]) out[k[h]] = APRIL_TRUE_HIT;
            const bool keep = valid[h] && !hit[h];
            const uint32_t mask = __ballot_sync(kFull, keep);
            if (mask) {
                const uint32_t leader = __ffs(mask) - 1;
                uint32_t pos = 0;
                if (lane == leader) pos = atomicAdd(&counters[C_REST_COUNT], __popc(mask));
                pos = __shfl_sync(kFull, pos, leader) + __popc(mask & ((1u << lane) - 1u));
                if (keep) rest[pos] = (uint32_t)k[h] + k_base;
            }
        }
    }
}

// K2c: the triage of the different-granularity filter (Sec. 5.3).  For a
// pair whose MBR-intersection centre lies in cell c of the coarser set's
// grid, c in the coarse side's F-list and an interval of the finer side's
// A-list meeting the fine cells of c (ids c << sh to ((c + 1) << sh) - 1 on
// nested grids, the coarsening the plan applies) mean that the plan's F join
// (the finer side's A, coarsened, against the coarse side's F) has an overlap,
// and with it the AA join: a true hit.  The other pairs are listed for the
// variant kernel; out-of-range ids get error verdicts.  One thread per pair.
__device__ __forceinline__ bool list_meets(const RawList &L, uint32_t lo, uint32_t hi) {
    if (!L.n) return false;  // whether an interval has last cell >= lo and start <= hi
    uint32_t a = 0, b = L.keys_n();
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (L.key(m) < lo) a = m + 1;
        else b = m;
    }
    uint32_t i = L.start_of(a), j = min(L.n, i + 16u);
    while (i < j) {
        const uint32_t m = (i + j) >> 1;
        if (__ldg(&L.p[m].y) - 1u < lo) i = m + 1;
        else j = m;
    }
    return i < L.n && __ldg(&L.p[i].x) <= hi;
}

__global__ void __launch_bounds__(256) k_triage_coarse(RawSets R, RawSets S, const int4 *__restrict__ mbr_r,
                                                       const int4 *__restrict__ mbr_s, TriageGrid g,
                                                       HilbertLut lut_in, uint32_t sh, bool r_finer,
                                                       const uint32_t *__restrict__ pr,
                                                       const uint32_t *__restrict__ ps, uint64_t n,
                                                       uint8_t *__restrict__ out, uint32_t *status, uint32_t *rest,
                                                       uint32_t *counters) {
    __shared__ uint8_t lut[64];
    if (threadIdx.x < 64) lut[threadIdx.x] = lut_in.e[threadIdx.x];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t kb = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); kb < n; kb += stride) {
        const uint64_t k = kb + lane;
        bool keep = false;
        if (k < n) {
            const uint32_t r = __ldg(pr + k), s = __ldg(ps + k);
            if (r < R.n() && s < S.n()) {
                uint32_t c = 0;
                bool hit = false;
                if (triage_cell(mbr_r, mbr_s, g, lut, r, s, c)) {
                    const uint4 dr = R.load(r), ds = S.load(s);
                    const uint32_t lo = c << sh, hi = ((c + 1) << sh) - 1u;  // wraps to 2^32 - 1 at the top
                    hit = r_finer ? list_meets(S.list(ds, true), c, c) && list_meets(R.list(dr, false), lo, hi)
                                  : list_meets(R.list(dr, true), c, c) && list_meets(S.list(ds, false), lo, hi);
                }
                keep = !hit;
                if (hit) out[k] = APRIL_TRUE_HIT;
            } else {
                out[k] = APRIL_VERDICT_ERROR;
                atomicOr(status, ST_BAD_ID);
            }
        }
        const uint32_t mask = __ballot_sync(kFull, keep);
        if (mask) {
            const uint32_t leader = __ffs(mask) - 1;
            uint32_t pos = 0;
            if (lane == leader) pos = atomicAdd(&counters[C_REST_COUNT], __popc(mask));
            pos = __shfl_sync(kFull, pos, leader) + __popc(mask & ((1u << lane) - 1u));
            if (keep) rest[pos] = (uint32_t)k;
        }
    }
}

// ------------------------------------------ K3: persistent filter (batched)
// Group engine.  A warp is split into 32/G groups of G lanes; each group
// filters one pair at a time (its joins in the tuned order, see
// step_outcome), with its own window of at most 8*G intervals per list
// staged in shared memory.
// One pass of the loop below advances every group's current join by one
// window, so the fixed cost of a window step (staging, the per-thread merge-
// path search, the vote) is shared by 32/G joins.  When a group finishes its
// pair it takes the next one from the warp's current chunk of 32 pairs, whose
// eligible pairs are listed compacted in shared memory (a group takes the
// entry at the list's cursor plus its rank among the groups asking); the warp
// pops a new chunk from a global counter when the list is used up.  The
// pairs are all n, or, after the triage (K2), the ones it listed.  Pairs
// above a CTA threshold, when one is set, are skipped here (phase 1 did
// them).
template <uint32_t G>
struct GroupCfg {
    static constexpr uint32_t NG = 32 / G;
    static constexpr uint32_t WMAX = kGroupPer * G;
    static constexpr uint32_t BUF = WMAX + 2;
    static constexpr uint32_t LEADS = G == 32 ? 1u : G == 16 ? 0x00010001u : G == 8 ? 0x01010101u : 0x11111111u;
    // intervals of shared staging per warp: the groups' buffers, or two warp
    // windows for the long pairs joined by the warp
    static constexpr uint32_t SHARE = NG * 2 * BUF > 2 * kWarpBuf ? NG * 2 * BUF : 2 * kWarpBuf;
    // mbarriers: [0] the CTA phase, [1 + warp * NG + group] the group engine,
    // [1 + kWarpsPerBlock * NG + warp] long pairs joined by warps
    static constexpr uint32_t BARS = 1 + kWarpsPerBlock * (NG + 1);
    static __device__ __forceinline__ uint32_t group_bar(uint32_t warp, uint32_t g) { return 1 + warp * NG + g; }
    static __device__ __forceinline__ uint32_t warp_bar(uint32_t warp) { return 1 + kWarpsPerBlock * NG + warp; }
};
static_assert(2 * kCtaBuf <= kWarpsPerBlock * GroupCfg<32>::SHARE, "CTA windows must fit in the warps' buffers");
static_assert(GroupCfg<4>::SHARE % 2 == 0 && GroupCfg<8>::SHARE % 2 == 0 && GroupCfg<16>::SHARE % 2 == 0,
              "warp shares keep 16-byte alignment");

// Lists of join step `stage` of a pair (in join order jo, see step_outcome);
// false when one of them is empty (the join then has no overlap).
template <class SetsT, class ListT>
__device__ __forceinline__ bool join_lists(const SetsT &R, const SetsT &S, const uint4 &dr, const uint4 &ds,
                                           uint32_t stage, ListT &X, ListT &Y, uint32_t jo) {
    X = R.list(dr, step_x_f(stage, jo));
    Y = S.list(ds, step_y_f(stage, jo));
    return X.n != 0 && Y.n != 0;
}

// The start searches of every group of a warp at once (warp-collective;
// `need` names a group's lists to search, bit 0 X and bit 1 Y, 0 for none).
// A fresh join searches each list longer than a first window for its first
// interval whose last cell reaches the other list's first start; a galloping
// search (a window advanced one list only) searches that list, from its
// merge position, against the target `gt` (the other list's current start).
// Both lists are searched in the same rounds over their search keys (the skip
// index's posts for raw lists, block anchors for compressed lists; see
// RawList / PackedList).  Each probing round every lane probes P evenly spaced
// keys per list (fan-out G*P) and the group counts the probes below the
// target (a prefix, the keys being sorted), which leaves one gap of the
// spacing.  The probing stops once both ranges fit one vector round of
// 4 G kPostVec keys, and that round ends the search.
#ifndef APRIL_SEARCH_MIN
#define APRIL_SEARCH_MIN 0
#endif
constexpr uint32_t kSearchProbes = 1;
constexpr uint32_t kSearchMin = APRIL_SEARCH_MIN;  // lists up to this long are not searched by fresh joins
template <uint32_t G, class ListT>
__device__ __forceinline__ void dual_search(const ListT &X, const ListT &Y, uint32_t need, bool fresh, uint32_t gt,
                                            uint32_t t, uint32_t gbits, uint32_t &i0, uint32_t &j0) {
    constexpr uint32_t P = kSearchProbes, F = G * P;
    // probing stops once a range fits one vector round (post_count) over the
    // skip index (raw lists) or the block anchors (compressed lists)
    constexpr uint32_t PER = 4 / ListT::kKeyStride;  // keys per 16-byte load
    constexpr uint32_t LIMIT = PER * G * kPostVec - (PER - 1);
    const bool sx = need & 1u, sy = need & 2u;
    uint32_t loX = sx ? X.key_lo(i0) : 0, hiX = sx ? X.keys_n() : 0;
    uint32_t loY = sy ? Y.key_lo(j0) : 0, hiY = sy ? Y.keys_n() : 0;
    // the targets: a fresh join's other list's first start, loaded with the
    // first round's probes, whose positions do not depend on them
    const uint32_t kx = sx ? (fresh ? Y.first_start() : gt) : 0u, ky = sy ? (fresh ? X.first_start() : gt) : 0u;
    while (__any_sync(kFull, hiX - loX > LIMIT || hiY - loY > LIMIT)) {  // lo <= hi throughout
        const bool ax = hiX - loX > LIMIT, ay = hiY - loY > LIMIT;
        const uint32_t sX = ax ? (hiX - loX + F - 1) / F : 1, sY = ay ? (hiY - loY + F - 1) / F : 1;
        uint32_t vX[P], vY[P];
#pragma unroll
        for (uint32_t q = 0; q < P; ++q) {
            const uint32_t px = loX + (t * P + q + 1) * sX - 1, py = loY + (t * P + q + 1) * sY - 1;
            vX[q] = (ax && px < hiX) ? X.key(px) : 0u;
            vY[q] = (ay && py < hiY) ? Y.key(py) : 0u;
        }
        uint32_t cX = 0, cY = 0;
#pragma unroll
        for (uint32_t q = 0; q < P; ++q) {
            const uint32_t px = loX + (t * P + q + 1) * sX - 1, py = loY + (t * P + q + 1) * sY - 1;
            cX += __popc(__ballot_sync(kFull, ax && px < hiX && vX[q] < kx) & gbits);
            cY += __popc(__ballot_sync(kFull, ay && py < hiY && vY[q] < ky) & gbits);
        }
        // c below-probes leave the gap after the c-th probe, if that probe
        // exists (c < probes in [lo, hi)), else the tail after the last one
        if (ax) {
            if (loX + (cX + 1) * sX <= hiX) hiX = loX + (cX + 1) * sX - 1;
            loX += cX * sX;
        }
        if (ay) {
            if (loY + (cY + 1) * sY <= hiY) hiY = loY + (cY + 1) * sY - 1;
            loY += cY * sY;
        }
    }
    if (__any_sync(kFull, hiX > loX || hiY > loY)) {
        // the last round: each lane counts its vectors of keys of both lists;
        // the group sums (X in the low half, Y in the high half)
        constexpr uint32_t KS = ListT::kKeyStride;
        uint32_t v = post_count<KS>(X.keys(), loX, hiX, 0, kx, t, G) | (post_count<KS>(Y.keys(), loY, hiY, 0, ky, t, G) << 16);
#pragma unroll
        for (uint32_t m = 1; m < G; m <<= 1) v += __shfl_xor_sync(kFull, v, m);
        loX += v & 0xFFFFu;
        loY += v >> 16;
    }
    if (sx) i0 = max(i0, X.start_of(loX));
    if (sy) j0 = max(j0, Y.start_of(loY));
}

template <uint32_t G, class SetsT>
__device__ __forceinline__ void group_engine(const SetsT &R, const SetsT &S, const uint32_t *__restrict__ pr,
                                             const uint32_t *__restrict__ ps, uint64_t n, uint8_t *__restrict__ out,
                                             uint32_t *status, uint32_t *counters, uint32_t cta_threshold, uint2 *wbuf,
                                             uint4 *chunk_desc, uint32_t *chunk_k, uint32_t bars,
                                             uint32_t lane, uint32_t w0, uint32_t jo, uint32_t esc_windows, uint4 *esc,
                                             uint32_t esc_cap, const uint32_t *__restrict__ rest) {
    using C = GroupCfg<G>;
    const bool no_long = cta_threshold == kNoLongPairs;  // every pair is joined here; no binning kernel ran

    const uint32_t g = lane / G, t = lane % G, glead = g * G;
    const uint32_t gbits = (G == 32 ? kFull : ((1u << G) - 1u)) << glead;
    uint2 *xb = wbuf + g * 2 * C::BUF, *yb = xb + C::BUF;
    const uint32_t bar = bars + 8u * g;  // this group's mbarrier
    uint32_t phase = 0;
    // the warp's chunk of 32 pairs (from position `base` of the pair list or
    // of the triage's list): the pairs it takes are stored compacted, pair
    // chunk_k[i] with its two descriptors in chunk_desc[i] and
    // chunk_desc[32 + i]; entries [cur, cur + left) are still to be handed out
    uint32_t base = 0;
    uint32_t cur = 0, left = 0;
    bool exhausted = false;
    // this group's pair and join
    bool active = false;
    uint32_t k = 0;
    uint4 dr = make_uint4(0, 0, 0, 0), ds = make_uint4(0, 0, 0, 0);
    uint32_t stage = 0, i0 = 0, j0 = 0, w = w0;
    uint32_t nwin = 0;   // windows of the current join so far
    bool fresh = false;  // the join has just started: its start has not been searched yet
    uint32_t gal = 0, gt = 0;  // a galloping search due (bit 0: X, bit 1: Y) and its target
    using ListT = decltype(R.list(dr, false));
    ListT X = R.list(dr, false), Y = S.list(ds, false);

    for (;;) {
        // -------- hand pairs to idle groups
        uint32_t needg = __ballot_sync(kFull, !active) & C::LEADS;
        while (needg && !exhausted) {
            if (!left) {
                uint32_t c = 0;
                if (lane == 0) c = atomicAdd(&counters[C_CHUNK_HEAD], 1u);
                c = __shfl_sync(kFull, c, 0);
                // the pairs to join: all n, or the ones the triage listed (rest)
                const uint64_t nn = rest ? (uint64_t)*((volatile uint32_t *)&counters[C_REST_COUNT]) : n;
                if (c >= (nn + 31) / 32) {
                    exhausted = true;
                    break;
                }
                base = c * 32;  // n < 2^32 pairs
                const uint32_t qk = base + lane;
                bool take = false;
                __syncwarp();  // every group has read its descriptors from the previous chunk
                uint32_t kk = 0;
                uint4 qdr = make_uint4(0, 0, 0, 0), qds = qdr;
                if (qk < nn) {
                    kk = rest ? __ldg(rest + qk) : qk;
                    const uint32_t r = __ldg(pr + kk), s2 = __ldg(ps + kk);
                    if (r < R.n() && s2 < S.n()) {
                        qdr = R.load(r);
                        qds = S.load(s2);
                        take = no_long || (uint64_t)qdr.y + qds.y <= (uint64_t)cta_threshold;
                    } else if (no_long) {  // no binning kernel ran to report them
                        out[kk] = APRIL_VERDICT_ERROR;
                        atomicOr(status, ST_BAD_ID);
                    }
                }
                // the pairs this warp takes, compacted in order
                const uint32_t tb = __ballot_sync(kFull, take);
                if (take) {
                    const uint32_t pos = __popc(tb & ((1u << lane) - 1u));
                    chunk_k[pos] = kk;
                    chunk_desc[pos] = qdr;
                    chunk_desc[32 + pos] = qds;
                }
                cur = 0;
                left = __popc(tb);
                __syncwarp();
                continue;
            }
            const uint32_t cnt = min((uint32_t)__popc(needg), left);
            const uint32_t grank = __popc(needg & ((1u << glead) - 1u));
            const bool gets = ((needg >> glead) & 1u) && grank < cnt;
            if (gets) {
                const uint32_t src = cur + grank;
                k = chunk_k[src];
                dr = chunk_desc[src];
                ds = chunk_desc[32 + src];
                stage = 0;
                i0 = j0 = 0;
                w = w0;
                nwin = 0;
                fresh = true;
                int verdict = -1;  // steps with an empty list have no overlap
                while (!join_lists(R, S, dr, ds, stage, X, Y, jo))
                    if ((verdict = step_outcome(stage, false, jo)) >= 0) break;
                active = verdict < 0;
                if (!active && t == 0) out[k] = (uint8_t)verdict;
            }
            cur += cnt;
            left -= cnt;
            needg = __ballot_sync(kFull, !active) & C::LEADS;
        }
        if (!__any_sync(kFull, active)) break;  // only reachable once the pairs are exhausted

        // -------- a join that has just started skips, in each list longer
        // than a window, the intervals ending before the other list's first
        // start (they meet nothing; the merge would pass over them); a list
        // that the last window advanced alone skips those ending before the
        // other list's current start (galloping, see tile_join)
        if (__any_sync(kFull, active && (fresh || gal))) {
            const uint32_t smin = max(w0, kSearchMin);
            const uint32_t nd = !active ? 0u : fresh ? (uint32_t)(X.n > smin) | ((uint32_t)(Y.n > smin) << 1) : gal;
            dual_search<G>(X, Y, nd, fresh, gt, t, gbits, i0, j0);
        }
        fresh = false;
        gal = 0;
        const uint32_t nX = X.n, nY = Y.n;
        const bool ran_out = active && (i0 >= nX || j0 >= nY);  // the search passed a whole list

        // -------- one window of every active group's join: raw lists arrive
        // by two bulk copies on the group's mbarrier, compressed lists are
        // decoded by the group's lanes (one block each)
        uint32_t nx = 0, ny = 0, xa = 0, ya = 0;
        bool ok = true;
        if (active && !ran_out) {
            nx = min(w, nX - i0);
            ny = min(w, nY - j0);
            if constexpr (ListT::kBulk) {
                if constexpr (kStage2) {
                    // lane 0 copies X's window, lane 1 Y's; each arrives once
                    // with its own bytes on the group's mbarrier (count 2)
                    if (t < 2) {
                        fence_proxy_async();
                        const bool isy = t == 1;
                        const uint2 *src = isy ? Y.p + j0 : X.p + i0;
                        const uint2 *a;
                        uint32_t b, o;
                        bulk_span(src, isy ? ny : nx, a, b, o);
                        mbar_arrive_expect_tx(bar, b);
                        bulk_load(smem_addr(isy ? yb : xb), src - o, b, bar);
                    }
                } else if (t == 0) {
                    fence_proxy_async();
                    const uint2 *a;
                    uint32_t bx, by, ox, oy;
                    bulk_span(X.p + i0, nx, a, bx, ox);
                    bulk_span(Y.p + j0, ny, a, by, oy);
                    mbar_arrive_expect_tx(bar, bx + by);
                    bulk_load(smem_addr(xb), X.p + i0 - ox, bx, bar);
                    bulk_load(smem_addr(yb), Y.p + j0 - oy, by, bar);
                }
                ok = mbar_wait(bar, phase);
                phase ^= 1u;
            } else {
                X.template stage<G>(xb, i0, nx, t, gbits);
                Y.template stage<G>(yb, j0, ny, t, gbits);
            }
            xa = X.window(xb, i0);
            ya = Y.window(yb, j0);
        }
        if constexpr (!ListT::kBulk) __syncwarp();  // the decoded windows are visible to the group
        if (!__all_sync(kFull, ok)) {
            // a bounded wait ran out: once the copies in flight have landed
            // (bounded), mark the pairs this warp holds as errors, report
            // and stop this warp
            if (!ok) mbar_drain(bar, phase ^ 1u);
            if (active && t == 0) out[k] = APRIL_VERDICT_ERROR;
            if (lane < left) out[chunk_k[cur + lane]] = APRIL_VERDICT_ERROR;
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        bool found = false;
        uint32_t state = 0xffffffffu, D = 0, owner = 0;
        if (active && !ran_out) {
            D = min(w, nx + ny);
            const uint32_t per = w / G;  // a power of two
            owner = (D - 1) >> (__ffs(per) - 1);
            found = window_walk<C::WMAX / G>(xa, nx, ya, ny, w, D, per, t * per, state);
        }
        const uint32_t fmask = __ballot_sync(kFull, found);  // every read of the windows is done here
        const uint32_t split = __shfl_sync(kFull, state, glead + owner);
        if (active) {
            int res = -1;  // -1: join continues, 0: no overlap, 1: overlap
            if (ran_out) res = 0;
            else if (fmask & gbits) res = 1;
            else if (D == nx + ny || split == 0xffffffffu) res = 0;
            else {
                i0 += split;
                j0 += D - split;
                w = min(w * 2u, C::WMAX);
                // the windows stay intact until the next pass's staging,
                // which follows that pass's first warp vote
                if (split == 0 && nY - j0 > w) {
                    gal = 2u;
                    gt = lds1(xa);  // X's current start
                } else if (split == D && nX - i0 > w) {
                    gal = 1u;
                    gt = lds1(ya);  // Y's current start
                }
                if (esc_windows && ++nwin >= esc_windows) {
                    // a long join: hand it, at the position it reached, to a
                    // whole warp (k_long) and take the next pair, unless the
                    // queue is full
                    uint32_t slot = 0;
                    if (t == 0) slot = atomicAdd(&counters[C_ESC_COUNT], 1u);
                    slot = __shfl_sync(gbits, slot, glead);
                    if (slot < esc_cap) {
                        if (t == 0) esc[slot] = make_uint4(k, stage, i0, j0);
                        active = false;
                    } else {
                        nwin = 0;
                    }
                }
            }
            if (res >= 0) {
                int verdict = step_outcome(stage, res != 0, jo);
                while (verdict < 0) {
                    i0 = j0 = 0;
                    w = w0;
                    nwin = 0;
                    fresh = true;
                    if (join_lists(R, S, dr, ds, stage, X, Y, jo)) break;
                    verdict = step_outcome(stage, false, jo);
                }
                if (verdict >= 0) {
                    if (t == 0) out[k] = (uint8_t)verdict;
                    active = false;
                }
            }
        }
    }
}

// Phase 1 (only with a long-pair threshold): the long pairs, each joined by
// one warp (first window below 256) or by the whole CTA (the merge path of one
// join split over 256 threads).  Phase 2: the group engine on the other pairs
// (whole warps when G = 32), or on the pairs the triage left.
// Work is handed out by atomic counters; nothing waits on another CTA.
template <uint32_t G, class SetsT>
__global__ void APRIL_PERSISTENT_BOUNDS k_persistent(SetsT R, SetsT S,
                                                                         const uint32_t *__restrict__ pr,
                                                       const uint32_t *__restrict__ ps, uint64_t n,
                                                       uint8_t *__restrict__ out, uint32_t *status,
                                                       uint32_t cta_threshold, const uint32_t *__restrict__ big_list,
                                                       uint32_t *counters, uint32_t w0_group, uint32_t w0_cta,
                                                       uint32_t jo, uint32_t esc_windows, uint4 *esc, uint32_t esc_cap,
                                                       const uint32_t *__restrict__ rest) {
    using C = GroupCfg<G>;
    __shared__ __align__(16) uint2 sm[kWarpsPerBlock * C::SHARE];
    __shared__ uint32_t s_item, s_slot;
    __shared__ uint64_t bars[C::BARS];  // see GroupCfg
    __shared__ uint4 s_chunk[kWarpsPerBlock][64];     // group engine: each warp's chunk descriptors
    __shared__ uint32_t s_chunk_k[kWarpsPerBlock][32];    // and their pairs
    if constexpr (kStage2 && G < 32 && !SetsT::kPacked) {
        // the lane groups' mbarriers take two arrivals a window (see group_engine)
        for (uint32_t i = threadIdx.x; i < C::BARS; i += blockDim.x) {
            const bool grp = i >= 1 && i < 1 + kWarpsPerBlock * C::NG;
            mbar_init(smem_addr(bars + i), grp ? 2u : 1u);
        }
        if (threadIdx.x == 0) mbar_init_fence();
        __syncthreads();
    } else {
        init_barriers(bars, C::BARS);
    }
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nbig = *((volatile uint32_t *)&counters[C_BIG_COUNT]);
    uint2 *wbuf = sm + warp * C::SHARE;
    if (w0_cta < kBlock) {
        // long pairs one per warp (first window w0_cta): the CTA's warps work
        // on eight long pairs at once
        JoinSync ws{smem_addr(&bars[C::warp_bar(warp)]), 0u, false};
        for (;;) {
            uint32_t it = 0;
            if (lane == 0) it = atomicAdd(&counters[C_BIG_HEAD], 1u);
            it = __shfl_sync(kFull, it, 0);
            if (it >= nbig) break;
            const uint64_t k = big_list[it];
            const typename SetsT::Desc dr = R.load(__ldg(pr + k)), ds = S.load(__ldg(ps + k));
            const uint8_t v = warp_verdict(R, S, dr, ds, wbuf, wbuf + kWarpBuf, lane, w0_cta, ws, jo);
            if (lane == 0) out[k] = v;
            if (ws.timeout) {  // a bounded wait ran out: report and stop this warp
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
        }
        // no CTA barrier here: the warp's phase-2 buffers and mbarriers are
        // its own, so it starts on short pairs while its CTA's other warps
        // still join long ones
    } else {
        JoinSync cs{smem_addr(&bars[0]), 0u, false};
        for (;;) {
            if (tid == 0) s_item = atomicAdd(&counters[C_BIG_HEAD], 1u);
            __syncthreads();
            const uint32_t it = s_item;
            __syncthreads();
            if (it >= nbig) break;
            const uint64_t k = big_list[it];
            const typename SetsT::Desc dr = R.load(__ldg(pr + k)), ds = S.load(__ldg(ps + k));
            const uint8_t v = cta_verdict(R, S, dr, ds, sm, sm + kCtaBuf, &s_slot, tid, w0_cta, cs, jo);
            if (tid == 0) out[k] = v;
            if (cs.timeout) {  // a bounded wait ran out: report and stop this CTA
                if (tid == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
        }
        __syncthreads();
    }
    if constexpr (G == 32) {
        JoinSync js{smem_addr(&bars[C::group_bar(warp, 0)]), 0u, false};
        const uint64_t nchunks = (n + 31) / 32;
        for (;;) {
            uint32_t c = 0;
            if (lane == 0) c = atomicAdd(&counters[C_CHUNK_HEAD], 1u);
            c = __shfl_sync(kFull, c, 0);
            if (c >= nchunks) break;
            if (!warp_chunk(R, S, pr, ps, n, (uint64_t)c * 32, out, status, wbuf, wbuf + kWarpBuf, lane, w0_group,
                            cta_threshold, cta_threshold == kNoLongPairs, js, jo))
                return;
        }
    } else {
        group_engine<G>(R, S, pr, ps, n, out, status, counters, cta_threshold, wbuf, s_chunk[warp], s_chunk_k[warp],
                        smem_addr(&bars[C::group_bar(warp, 0)]), lane, w0_group, jo, esc_windows, esc, esc_cap,
                        rest);
    }
}

// ------------------------------ K3b: joins handed over by the lane groups
// Each warp takes the next queued join {pair, step, i0, j0} and finishes the
// pair by whole-warp joins: that step resumes at (i0, j0) with first window
// w0, the later steps of the join order start fresh.
template <class SetsT>
__global__ void __launch_bounds__(kBlock) k_long(SetsT R, SetsT S, const uint32_t *__restrict__ pr,
                                                 const uint32_t *__restrict__ ps, uint8_t *__restrict__ out,
                                                 uint32_t *status, const uint4 *__restrict__ esc, uint32_t *counters,
                                                 uint32_t esc_cap, uint32_t w0, uint32_t jo) {
    __shared__ __align__(16) uint2 sm[kWarpsPerBlock][2][kWarpBuf];
    __shared__ uint64_t bars[kWarpsPerBlock];
    init_barriers(bars, kWarpsPerBlock);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    JoinSync js{smem_addr(&bars[warp]), 0u, false};
    const uint32_t nesc = min(*((volatile uint32_t *)&counters[C_ESC_COUNT]), esc_cap);
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&counters[C_ESC_HEAD], 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= nesc) break;
        const uint4 rec = esc[it];
        const typename SetsT::Desc dr = R.load(__ldg(pr + rec.x)), ds = S.load(__ldg(ps + rec.x));
        const uint8_t v = warp_verdict(R, S, dr, ds, sm[warp][0], sm[warp][1], lane, w0, js, jo, rec.y, true, rec.z,
                                       rec.w);
        if (lane == 0) out[rec.x] = v;
        if (js.timeout) {  // a bounded wait ran out: report and stop this warp
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
    }
}

// -------------------------------- K7: filter variants (Sec. 4.3.2, Sec. 5.3)
// A plan is the decision sequence of one filter variant: each stage joins one
// list of r with one list of s under a predicate and either decides the
// verdict or moves to another stage.  The finer side's lists are coarsened
// on load when the two sets use grids of different order (Sec. 5.3).
struct Plan {
    uint8_t nst;
    uint8_t xf[3], yf[3];       // stage's list: 0 = A-list, 1 = F-list (r, s)
    uint8_t pred[3];            // kOverlap or kContain
    int8_t on_true[3], on_false[3];  // >= 0: next stage; < 0: verdict -(v + 1)
    uint8_t sx, sy;             // coarsening shifts of r's / s's intervals (bits)
};

template <class Scope, uint32_t NT, uint32_t WMAX>
__device__ __forceinline__ uint8_t plan_verdict(const Plan &P, const RawSets &R, const RawSets &S, const uint4 &dr,
                                                const uint4 &ds, uint2 *xs, uint2 *ys, uint32_t *slot, uint32_t tid,
                                                uint32_t w0, JoinSync &js) {
    int st = 0;
    for (int guard = 0; guard < 3; ++guard) {
        const RawList X = R.list(dr, P.xf[st] != 0), Y = S.list(ds, P.yf[st] != 0);
        const bool res =
            P.pred[st] == kContain
                ? tile_join<Scope, NT, WMAX, RawList, kContain>(X, Y, xs, ys, slot, tid, w0, js.bar, &js.phase,
                                                                &js.timeout, P.sx, P.sy)
                : tile_join<Scope, NT, WMAX, RawList, kOverlap>(X, Y, xs, ys, slot, tid, w0, js.bar, &js.phase,
                                                                &js.timeout, P.sx, P.sy);
        if (js.timeout) return APRIL_VERDICT_ERROR;
        const int nx = res ? P.on_true[st] : P.on_false[st];
        if (nx < 0) return (uint8_t)(-(nx + 1));
        st = nx;
    }
    return APRIL_VERDICT_ERROR;
}

// Same shape as K3 with 32-lane groups: long pairs by whole CTAs, the rest by
// warps taking 32-pair chunks.
// the variant kernel at four CTAs per SM (at most 64 registers a thread)
#ifndef APRIL_GENERAL_MIN_BLOCKS
#define APRIL_GENERAL_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(kBlock, APRIL_GENERAL_MIN_BLOCKS) k_general(Plan P, DevSet Rd, DevSet Sd, const uint32_t *__restrict__ pr,
                                                    const uint32_t *__restrict__ ps, uint64_t n,
                                                    uint8_t *__restrict__ out, uint32_t *status,
                                                    uint32_t cta_threshold, const uint32_t *__restrict__ big_list,
                                                    uint32_t *counters, uint32_t long_window,
                                                    const uint32_t *__restrict__ rest) {
    __shared__ __align__(16) uint2 sm[kSharedIv];
    __shared__ uint32_t s_item, s_slot;
    __shared__ uint64_t bars[1 + kWarpsPerBlock];
    init_barriers(bars, 1 + kWarpsPerBlock);
    const RawSets R{Rd}, S{Sd};
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nbig = *((volatile uint32_t *)&counters[C_BIG_COUNT]);
    uint2 *xs = sm + warp * kWarpShare, *ys = xs + kWarpBuf;
    JoinSync js{smem_addr(&bars[1 + warp]), 0u, false};
    if (long_window < kBlock) {  // long pairs one per warp
        for (;;) {
            uint32_t it = 0;
            if (lane == 0) it = atomicAdd(&counters[C_BIG_HEAD], 1u);
            it = __shfl_sync(kFull, it, 0);
            if (it >= nbig) break;
            const uint64_t k = big_list[it];
            const uint4 dr = R.load(__ldg(pr + k)), ds = S.load(__ldg(ps + k));
            const uint8_t v = plan_verdict<WarpScope, 32, kWarpWMax>(P, R, S, dr, ds, xs, ys, nullptr, lane,
                                                                      long_window, js);
            if (lane == 0) out[k] = v;
            if (js.timeout) break;
        }
        const bool dead = js.timeout;
        if (dead && lane == 0) atomicOr(status, ST_TIMEOUT);
        __syncthreads();
        if (dead) return;  // a bounded wait ran out: this warp stops (after the CTA's only barrier)
    } else {
        JoinSync cs{smem_addr(&bars[0]), 0u, false};
        for (;;) {
            if (tid == 0) s_item = atomicAdd(&counters[C_BIG_HEAD], 1u);
            __syncthreads();
            const uint32_t it = s_item;
            __syncthreads();
            if (it >= nbig) break;
            const uint64_t k = big_list[it];
            const uint4 dr = R.load(__ldg(pr + k)), ds = S.load(__ldg(ps + k));
            const uint8_t v = plan_verdict<CtaScope, kBlock, kCtaWMax>(P, R, S, dr, ds, sm, sm + kCtaBuf, &s_slot,
                                                                        tid, long_window, cs);
            if (tid == 0) out[k] = v;
            if (cs.timeout) {
                if (tid == 0) atomicOr(status, ST_TIMEOUT);
                return;
            }
        }
        __syncthreads();
    }
    // the pairs: all n, or the ones the coarse triage left (rest)
    const uint64_t nn = rest ? (uint64_t)*((volatile uint32_t *)&counters[C_REST_COUNT]) : n;
    const uint64_t nchunks = (nn + 31) / 32;
    for (;;) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&counters[C_CHUNK_HEAD], 1u);
        c = __shfl_sync(kFull, c, 0);
        if (c >= nchunks) break;
        const uint64_t q = (uint64_t)c * 32 + lane;
        const uint64_t k = q < nn ? (rest ? (uint64_t)__ldg(rest + q) : q) : n;
        uint4 dr = make_uint4(0, 0, 0, 0), ds = make_uint4(0, 0, 0, 0);
        bool take = false;
        if (k < n) {
            const uint32_t r = __ldg(pr + k), s2 = __ldg(ps + k);
            if (r < R.n() && s2 < S.n()) {
                dr = R.load(r);
                ds = S.load(s2);
                take = (uint64_t)dr.y + ds.y <= (uint64_t)cta_threshold;
            }
        }
        uint32_t todo = __ballot_sync(kFull, take);
        uint8_t mine = 0;
        while (todo) {
            const uint32_t t = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint8_t v = plan_verdict<WarpScope, 32, kWarpWMax>(P, R, S, shfl4(dr, t), shfl4(ds, t), xs, ys,
                                                                      nullptr, lane, 64u, js);
            if (lane == t) mine = v;
            if (js.timeout) {  // the pairs of the chunk not decided yet read as errors
                if (lane == 0) atomicOr(status, ST_TIMEOUT);
                if (take) out[k] = (lane == t || ((todo >> lane) & 1u)) ? (uint8_t)APRIL_VERDICT_ERROR : mine;
                return;
            }
        }
        if (take) out[k] = mine;
    }
}

// ----------------------------------------------- skip index of a set
// posts[q] = last cell of interval slot 16 q + 15 (see RawList::key).
__global__ void __launch_bounds__(256) k_posts(const uint2 *__restrict__ iv, uint64_t nposts,
                                               uint32_t *__restrict__ posts) {
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nposts;
         q += (uint64_t)gridDim.x * blockDim.x)
        posts[q] = __ldg(&iv[16 * q + 15].y) - 1u;
}

// ------------------------------------------- K6: partition routing (a-8)
// Sec. 5.2: a candidate pair is evaluated in the one partition that holds the
// lower-left corner of MBR(r) n MBR(s).  Writes the two entries (object
// approximations on that partition's grid) of every pair; an out-of-range id
// or a missing entry yields UINT32_MAX, which the filter reports as an error.
struct PartView {
    const int2 *ll;
    const uint32_t *obj_entry;
    const uint32_t *entry_pid;
    uint32_t n;
};

__device__ __forceinline__ uint32_t find_entry(const PartView &P, uint32_t obj, uint32_t pid) {
    const uint32_t e1 = __ldg(P.obj_entry + obj + 1);
    for (uint32_t e = __ldg(P.obj_entry + obj); e < e1; ++e)
        if (__ldg(P.entry_pid + e) == pid) return e;
    return 0xffffffffu;
}

__global__ void __launch_bounds__(256) k_route(PartView R, PartView S, uint32_t parts_log2,
                                               const uint32_t *__restrict__ pr, const uint32_t *__restrict__ ps,
                                               uint64_t n, uint32_t *__restrict__ er, uint32_t *__restrict__ es) {
    const uint32_t side_log2 = 24 - parts_log2, pmax = (1u << parts_log2) - 1u;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = __ldg(pr + k), s = __ldg(ps + k);
        uint32_t a = 0xffffffffu, b = 0xffffffffu;
        if (r < R.n && s < S.n) {
            const int2 lr = __ldg(R.ll + r), ls = __ldg(S.ll + s);
            const uint32_t x = (uint32_t)max(lr.x, ls.x), y = (uint32_t)max(lr.y, ls.y);
            const uint32_t pid = (min(y >> side_log2, pmax) << parts_log2) + min(x >> side_log2, pmax);
            a = find_entry(R, r, pid);
            b = find_entry(S, s, pid);
        }
        er[k] = a;
        es[k] = b;
    }
}

int g_num_sms = 0;

}  // namespace

int april_launch_posts(const uint32_t *iv, uint64_t iv_slots, uint32_t *posts, void *stream) {
    const uint64_t nposts = iv_slots / 16;
    if (nposts == 0) return (int)cudaSuccess;
    const unsigned grid = (unsigned)std::min<uint64_t>((nposts + 255) / 256, 152ull * 8);
    k_posts<<<grid, 256, 0, (cudaStream_t)stream>>>((const uint2 *)iv, nposts, posts);
    return (int)cudaGetLastError();
}

struct GraphKey {
    const void *r_desc, *r_iv, *s_desc, *s_iv, *r_posts, *s_posts;
    uint32_t rn, sn;
    const void *d_r, *d_s, *out, *scratch;
    uint64_t n;
    april_tune tune;
    unsigned grid_bin, grid_main;
    bool packed;
    uint32_t parts;
    const void *r_pdesc, *s_pdesc;
    const void *r_mbr, *s_mbr;
    int64_t r_ox, r_oy, s_ox, s_oy;
    uint32_t r_log2, s_log2, r_grid, s_grid;
    uint64_t r_gid, s_gid;
    const void *r_pgrid;
    bool operator==(const GraphKey &o) const {
        return packed == o.packed && parts == o.parts && r_pdesc == o.r_pdesc && s_pdesc == o.s_pdesc &&
               r_mbr == o.r_mbr && s_mbr == o.s_mbr && r_ox == o.r_ox && r_oy == o.r_oy && s_ox == o.s_ox &&
               s_oy == o.s_oy && r_log2 == o.r_log2 && s_log2 == o.s_log2 && r_grid == o.r_grid &&
               s_grid == o.s_grid && r_gid == o.r_gid && s_gid == o.s_gid && r_pgrid == o.r_pgrid &&
               tune.triage_off == o.tune.triage_off &&
               r_desc == o.r_desc && r_iv == o.r_iv && s_desc == o.s_desc && s_iv == o.s_iv &&
               r_posts == o.r_posts && s_posts == o.s_posts && rn == o.rn &&
               sn == o.sn && d_r == o.d_r && d_s == o.d_s && out == o.out && scratch == o.scratch && n == o.n &&
               tune.cta_threshold == o.tune.cta_threshold && tune.group_lanes == o.tune.group_lanes &&
               tune.group_window == o.tune.group_window && tune.cta_window == o.tune.cta_window &&
               tune.join_order == o.tune.join_order && tune.escalate_windows == o.tune.escalate_windows &&
               grid_bin == o.grid_bin && grid_main == o.grid_main;
    }
};

struct april_ctx {
    int device = 0;
    uint32_t *d_status = nullptr;  // 256-byte status block (word 0: ST_* bits)
    int num_sms = 0;
    // occupancy of k_persistent<4, 8, 16, 32> over raw lists, then over packed lists
    int persistent_blocks_per_sm[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    int long_blocks_per_sm = 1;  // occupancy of k_long (the larger of its two instances' limits)
    april_tune tune{};
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    // april_filter_pairs_host's pipeline (created on first use): streams for
    // the pair copies, two for the chunks' kernels, one for the verdict
    // copies, and events ordering them (start, end, per chunk: in, kernel)
    cudaStream_t pipe[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t pev[2 + 2 * 8] = {};
    cudaGraphExec_t graph = nullptr;    // the batched pipeline, captured once per argument set
    GraphKey key{};
    uint64_t graph_launches = 0;
    uint64_t graph_captures = 0;
};

using april::fail;

static april_status cuda_fail(cudaError_t e, const char *what) {
    return fail(APRIL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// index of a group size 4, 8, 16, 32 in the context's occupancy table
static int group_index(uint32_t g) { return g == 4 ? 0 : g == 8 ? 1 : g == 16 ? 2 : 3; }

static april_tune default_tune() {
    april_tune t{};
    // the shape the autotuner picks on the paper-scale, skewed and partitioned
    // workloads: every pair in groups of 4 lanes with full windows from the
    // start (with galloping, the lane groups also take the long pairs)
    t.cta_threshold = 0xffffffffu;
    t.group_lanes = 4;
    t.group_window = 32;
    t.cta_window = 128;      // with a threshold set: long pairs one per warp, first window 128
    t.join_order = kJoinOrderAuto;  // AA first after the triage, AF first otherwise
    t.escalate_windows = 0;  // lane groups finish every join they start
    t.triage_off = 0;        // the triage pass runs where it applies
    t.blocks_per_sm = 0;
    t.ms = 0.f;
    return t;
}

static april_status check_tune(const april_tune &t) {
    const uint32_t G = t.group_lanes;
    if (G != 4 && G != 8 && G != 16 && G != 32) return fail(APRIL_ERR_INVALID_ARG, "group_lanes must be 4, 8, 16 or 32");
    const uint32_t gmax = G == 32 ? kWarpWMax : kGroupPer * G;
    if (t.group_window < G || t.group_window > gmax || (t.group_window & (t.group_window - 1)))
        return fail(APRIL_ERR_INVALID_ARG, "group_window must be a power of two in [group_lanes, 8*group_lanes]");
    if (t.cta_window < 32 || t.cta_window > kCtaWMax || (t.cta_window & (t.cta_window - 1)))
        return fail(APRIL_ERR_INVALID_ARG, "cta_window must be a power of two in [32, 2048]");
    if (t.join_order > kJoinOrderAuto)
        return fail(APRIL_ERR_INVALID_ARG, "join_order must be 0 (AF AA FA), 1 (AA AF FA) or 2 (automatic)");
    if (t.escalate_windows > kMaxEscalateWindows) return fail(APRIL_ERR_INVALID_ARG, "escalate_windows must be 0..64");
    if (t.triage_off > 1) return fail(APRIL_ERR_INVALID_ARG, "triage_off must be 0 or 1");
    return APRIL_OK;
}

extern "C" april_status april_ctx_create(int device, april_ctx **out) {
    if (!out) return fail(APRIL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto *c = new april_ctx();
    c->device = device;
    c->tune = default_tune();
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
#define APRIL_OCC(I, G, SETS)                                                                                \
    if (e == cudaSuccess)                                                                                      \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->persistent_blocks_per_sm[I], k_persistent<G, SETS>, \
                                                          kBlock, 0)
    APRIL_OCC(0, 4, RawSets);
    APRIL_OCC(1, 8, RawSets);
    APRIL_OCC(2, 16, RawSets);
    APRIL_OCC(3, 32, RawSets);
    APRIL_OCC(4, 4, PackedSets);
    APRIL_OCC(5, 8, PackedSets);
    APRIL_OCC(6, 16, PackedSets);
    APRIL_OCC(7, 32, PackedSets);
#undef APRIL_OCC
    int occ_long_raw = 1, occ_long_packed = 1;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_long_raw, k_long<RawSets>, kBlock, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_long_packed, k_long<PackedSets>, kBlock, 0);
    c->long_blocks_per_sm = std::max(1, std::min(occ_long_raw, occ_long_packed));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, 256);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, 256);
    if (e != cudaSuccess) {
        if (c->d_status) cudaFree(c->d_status);
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        delete c;
        return cuda_fail(e, "april_ctx_create");
    }
    for (int &b : c->persistent_blocks_per_sm) b = b < 1 ? 1 : b;
    g_num_sms = c->num_sms;
    *out = c;
    return APRIL_OK;
}

extern "C" void april_ctx_destroy(april_ctx *ctx) {
    if (!ctx) return;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaStream_t &p : ctx->pipe)
        if (p) cudaStreamDestroy(p);
    for (cudaEvent_t &v : ctx->pev)
        if (v) cudaEventDestroy(v);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
}

extern "C" april_status april_set_tune(april_ctx *ctx, const april_tune *t) {
    if (!ctx || !t) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    april_status st = check_tune(*t);
    if (st) return st;
    ctx->tune = *t;
    return APRIL_OK;
}

extern "C" april_status april_ctx_graph_stats(const april_ctx *ctx, uint64_t *captures, uint64_t *launches) {
    if (!ctx) return fail(APRIL_ERR_INVALID_ARG, "NULL context");
    if (captures) *captures = ctx->graph_captures;
    if (launches) *launches = ctx->graph_launches;
    return APRIL_OK;
}

extern "C" april_status april_get_tune(const april_ctx *ctx, april_tune *t) {
    if (!ctx || !t) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    *t = ctx->tune;
    return APRIL_OK;
}

extern "C" april_status april_upload(const april_sets *S, void *dev_buf, size_t dev_bytes, void *stream,
                                     april_dev_sets *out) {
    if (!S || !dev_buf || !out) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)dev_buf) & 255u) return fail(APRIL_ERR_INVALID_ARG, "device buffer must be 256-byte aligned");
    const april_image_layout L = april_layout(*S);
    if (dev_bytes < L.total) return fail(APRIL_ERR_INVALID_ARG, "device buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)dev_buf;
    cudaError_t e = cudaSuccess;
    auto put = [&](uint64_t off, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    put(L.desc, S->desc.data(), S->desc.size() * 4);
    put(L.iv, S->iv.data(), S->iv.size() * 4);
    put(L.obj_ll, S->obj_ll.data(), S->obj_ll.size() * 4);
    put(L.obj_entry, S->obj_entry.data(), S->obj_entry.size() * 4);
    put(L.entry_pid, S->entry_pid.data(), S->entry_pid.size() * 4);
    put(L.pdesc, S->pdesc.data(), S->pdesc.size() * 4);
    put(L.anchors, S->anchors.data(), S->anchors.size() * 4);
    put(L.gaps, S->gaps.data(), S->gaps.size());
    put(L.mbr, S->mbr.data(), S->mbr.size() * 4);
    put(L.pgrid, S->part_grid.data(), S->part_grid.size() * 8);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(upload)");
    e = (cudaError_t)april_launch_posts((const uint32_t *)(base + L.iv), S->iv.size() / 2,
                                        (uint32_t *)(base + L.posts), stream);
    if (e != cudaSuccess) return cuda_fail(e, "building the skip index (upload)");
    *out = april_dev_sets{};
    out->desc = (const uint32_t *)(base + L.desc);
    out->iv = (const uint32_t *)(base + L.iv);
    out->n_objects = S->n;
    out->order = S->order;
    out->iv_slots = S->iv.size() / 2;
    out->n_entries = S->n_entries;
    out->parts = S->parts;
    out->mbr = S->mbr.empty() ? nullptr : (const int32_t *)(base + L.mbr);
    out->posts = (const uint32_t *)(base + L.posts);
    if (S->grid_known && !S->mbr.empty()) {
        out->grid_ox = S->grid_ox;
        out->grid_oy = S->grid_oy;
        out->grid_log2_cell = S->grid_log2_cell;
        out->grid_known = 1;
        out->grid_id = S->grid_id;
        if (S->parts) out->part_grid = (const int64_t *)(base + L.pgrid);
    }
    if (S->parts) {
        out->obj_ll = (const int32_t *)(base + L.obj_ll);
        out->obj_entry = (const uint32_t *)(base + L.obj_entry);
        out->entry_pid = (const uint32_t *)(base + L.entry_pid);
    }
    if (S->packed) {
        out->pdesc = (const uint32_t *)(base + L.pdesc);
        out->anchors = (const uint32_t *)(base + L.anchors);
        out->gaps = (const uint8_t *)(base + L.gaps);
    }
    return APRIL_OK;
}

static inline uint64_t round256(uint64_t b) { return (b + 255) / 256 * 256; }

extern "C" april_status april_filter_scratch_bytes(int mode, uint64_t n, size_t *bytes) {
    if (!bytes) return fail(APRIL_ERR_INVALID_ARG, "bytes is NULL");
    switch (mode) {
        case APRIL_MODE_PLAIN:
        case APRIL_MODE_WARP: *bytes = 0; return APRIL_OK;
        case APRIL_MODE_BATCHED:
        case APRIL_MODE_BATCHED_PACKED:
            *bytes = (size_t)(kCounterBytes + 3 * round256(4 * n) + round256(16 * esc_capacity(n)));
            return APRIL_OK;
        default: return fail(APRIL_ERR_INVALID_ARG, "unknown mode");
    }
}

// The filter reads sets as april_upload / april_build_sets_device lay them
// out: interval slots 256-byte aligned (a list's place among the skip
// index's 16-slot groups follows from its address) and the skip index.
static april_status check_layout(const april_dev_sets *d) {
    if (!d->desc || !d->iv || !d->posts || (((uintptr_t)d->iv) & 255u))
        return fail(APRIL_ERR_INVALID_ARG, "device sets not laid out by april_upload or april_build_sets_device");
    return APRIL_OK;
}

// The checks april_filter_pairs makes on its sets, size and mode.
static april_status check_filter_args(const april_dev_sets *R, const april_dev_sets *S, uint64_t n, int mode) {
    if (R->order != S->order || R->parts != S->parts)
        return fail(APRIL_ERR_INVALID_ARG, "R and S are on different grids");
    if (check_layout(R) || check_layout(S)) return APRIL_ERR_INVALID_ARG;
    if (n > 0xFFFFFFFFull) return fail(APRIL_ERR_INVALID_ARG, "at most 2^32-1 pairs per call");
    if (R->parts && mode != APRIL_MODE_BATCHED && mode != APRIL_MODE_BATCHED_PACKED)
        return fail(APRIL_ERR_INVALID_ARG, "partitioned sets need APRIL_MODE_BATCHED or APRIL_MODE_BATCHED_PACKED");
    if (mode == APRIL_MODE_BATCHED_PACKED && (!R->pdesc || !S->pdesc))
        return fail(APRIL_ERR_INVALID_ARG, "APRIL_MODE_BATCHED_PACKED needs sets compressed by april_sets_compress");
    return APRIL_OK;
}

static inline DevSet dev_set(const april_dev_sets *d) {
    return DevSet{(const uint4 *)d->desc, (const uint2 *)d->iv, d->n_entries ? d->n_entries : d->n_objects,
                  d->posts};
}

static inline PackedSets packed_set(const april_dev_sets *d) {
    return PackedSets{(const uint4 *)d->pdesc, (const uint2 *)d->anchors, d->gaps,
                      d->n_entries ? d->n_entries : d->n_objects};
}

static inline PartView part_view(const april_dev_sets *d) {
    return PartView{(const int2 *)d->obj_ll, d->obj_entry, d->entry_pid, d->n_objects};
}

// Enqueues the batched pipeline on `st`: counter reset, partition routing
// (partitioned sets only), K4 binning, K3 persistent filter, and, when the
// tuning escalates long joins, K3b for the joins the lane groups handed over.
// `esc_windows` overrides the tuning's escalate_windows (the allocation-free
// entry point has no room for the queue and passes 0).
// Whether the triage pass (K2) runs before the lane groups: raw sets built
// from polygons on the same grid(s) (equal fingerprints; for partitioned sets
// the same partition grids), and a tuning with every pair in lane groups of
// 4..16 lanes.
static bool triage_applies(const april_tune &t, const april_dev_sets *R, const april_dev_sets *S, bool packed) {
    if (t.triage_off || t.cta_threshold != kNoLongPairs || t.group_lanes >= 32) return false;
    if (packed && (!R->pdesc || !S->pdesc)) return false;
    if (!R->grid_known || !S->grid_known || !R->mbr || !S->mbr || R->order != S->order || R->grid_id != S->grid_id)
        return false;
    return !R->parts || (R->part_grid && R->entry_pid);
}

// The triage's grid: CTAs of 512 pairs a pass, at most
// APRIL_TRIAGE_GRID_PER_SM per SM.  Many more CTAs than fit at once (six per
// SM) balance the uneven cost of the pairs: CTAs that draw cheap pairs retire
// and make room for new ones.  Measured steps: a grid of exactly the resident
// CTAs ran 3-4% slower than 8 per SM, and 64 per SM ran 7% faster than 8 on
// 10M skewed pairs and on compressed lists (equal on the paper-scale pairs).
#ifndef APRIL_TRIAGE_GRID_PER_SM
#define APRIL_TRIAGE_GRID_PER_SM 64
#endif
static unsigned triage_grid(int num_sms, uint64_t n) {
    return (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((n + 511) / 512, (uint64_t)num_sms * APRIL_TRIAGE_GRID_PER_SM));
}

static TriageArgs triage_args(const april_dev_sets *R, const april_dev_sets *S, const uint32_t *er,
                              const uint32_t *es) {
    TriageArgs a{};
    a.mbr_r = (const int4 *)R->mbr;
    a.mbr_s = (const int4 *)S->mbr;
    a.g = TriageGrid{R->grid_ox, R->grid_oy, R->grid_log2_cell, R->order};
    a.part_grid = R->part_grid;
    a.entry_pid = R->entry_pid;
    a.er = er;
    a.es = es;
    return a;
}

static cudaError_t enqueue_groups(april_ctx *ctx, const april_dev_sets *Rd, const april_dev_sets *Sd,
                                  const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *out, void *scratch,
                                  bool packed, unsigned grid_main, cudaStream_t st, uint32_t *status,
                                  const uint32_t *rest);

static cudaError_t enqueue_batched(april_ctx *ctx, const april_dev_sets *Rd, const april_dev_sets *Sd,
                                   const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *out, void *scratch,
                                   bool packed, unsigned grid_bin, unsigned grid_main, cudaStream_t st,
                                   uint32_t *status = nullptr) {
    if (!status) status = ctx->d_status;
    uint32_t *counters = (uint32_t *)scratch;
    uint32_t *big_list = (uint32_t *)((char *)scratch + kCounterBytes);
    const april_tune &t = ctx->tune;
    const unsigned grid_tri = triage_grid(ctx->num_sms, n);
    cudaError_t e = cudaMemsetAsync(counters, 0, kCounterBytes, st);
    if (e != cudaSuccess) return e;
    const uint32_t *obj_r = d_r, *obj_s = d_s;  // the pairs' objects (their MBRs)
    if (Rd->parts) {
        uint32_t *er = (uint32_t *)((char *)scratch + kCounterBytes + round256(4 * n));
        uint32_t *es = (uint32_t *)((char *)scratch + kCounterBytes + 2 * round256(4 * n));
        uint32_t lg = 0;
        while ((1u << lg) < Rd->parts) ++lg;
        k_route<<<grid_bin, 256, 0, st>>>(part_view(Rd), part_view(Sd), lg, d_r, d_s, n, er, es);
        d_r = er;
        d_s = es;
    }
    const uint32_t *rest = nullptr;  // the pairs the lane groups join (nullptr: all)
    if (packed) {
        const PackedSets R = packed_set(Rd), S = packed_set(Sd);
        if (triage_applies(t, Rd, Sd, true)) {
            if (Rd->parts)
                k_triage<true, PackedSets><<<grid_tri, 256, 0, st>>>(R, S, triage_args(Rd, Sd, d_r, d_s), triage_lut(),
                                                                     obj_r, obj_s, n, out, status, big_list, counters,
                                                                     0u);
            else
                k_triage<false, PackedSets><<<grid_tri, 256, 0, st>>>(R, S, triage_args(Rd, Sd, nullptr, nullptr),
                                                                      triage_lut(), d_r, d_s, n, out, status, big_list,
                                                                      counters, 0u);
            rest = big_list;
        } else if (t.cta_threshold != kNoLongPairs) {
            k_bin<<<grid_bin, 256, 0, st>>>(R, S, d_r, d_s, n, out, status, t.cta_threshold, big_list, counters);
        }
        return enqueue_groups(ctx, Rd, Sd, d_r, d_s, n, out, scratch, true, grid_main, st, status, rest);
    }
    const RawSets R{dev_set(Rd)}, S{dev_set(Sd)};
    if (triage_applies(t, Rd, Sd, false)) {
        if (Rd->parts)
            k_triage<true, RawSets><<<grid_tri, 256, 0, st>>>(R, S, triage_args(Rd, Sd, d_r, d_s), triage_lut(), obj_r,
                                                              obj_s, n, out, status, big_list, counters, 0u);
        else
            k_triage<false, RawSets><<<grid_tri, 256, 0, st>>>(R, S, triage_args(Rd, Sd, nullptr, nullptr), triage_lut(),
                                                               d_r, d_s, n, out, status, big_list, counters, 0u);
        rest = big_list;
    } else if (t.cta_threshold != kNoLongPairs) {
        k_bin<<<grid_bin, 256, 0, st>>>(R, S, d_r, d_s, n, out, status, t.cta_threshold, big_list, counters);
    }
    return enqueue_groups(ctx, Rd, Sd, d_r, d_s, n, out, scratch, false, grid_main, st, status, rest);
}

// The lane-group stage of the batched pipeline (K3, then K3b when the tuning
// escalates long joins) over the pairs (d_r, d_s: routed entries for
// partitioned sets), or over the rest list a triage left.
static cudaError_t enqueue_groups(april_ctx *ctx, const april_dev_sets *Rd, const april_dev_sets *Sd,
                                  const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *out, void *scratch,
                                  bool packed, unsigned grid_main, cudaStream_t st, uint32_t *status,
                                  const uint32_t *rest) {
    uint32_t *counters = (uint32_t *)scratch;
    uint32_t *big_list = (uint32_t *)((char *)scratch + kCounterBytes);
    uint4 *esc = (uint4 *)((char *)scratch + kCounterBytes + 3 * round256(4 * n));
    const april_tune &t = ctx->tune;
    const uint32_t escw = t.group_lanes < 32 ? t.escalate_windows : 0u;
    const uint32_t w0_long = t.cta_window < kBlock ? std::min<uint32_t>(2 * t.cta_window, kWarpWMax) : 128u;
    const uint32_t esc_cap = (uint32_t)esc_capacity(n);
    const unsigned grid_long = (unsigned)std::max(1, ctx->num_sms * ctx->long_blocks_per_sm);
    const uint32_t jo = join_order_of(t.join_order, rest != nullptr);
    if (packed) {
        const PackedSets R = packed_set(Rd), S = packed_set(Sd);
#define APRIL_LAUNCH_PACKED(G)                                                                                  \
    k_persistent<G, PackedSets><<<grid_main, kBlock, 0, st>>>(R, S, d_r, d_s, n, out, status, t.cta_threshold,   \
                                                              big_list, counters, t.group_window, t.cta_window,   \
                                                              jo, escw, esc, esc_cap, rest)
        switch (t.group_lanes) {
            case 4: APRIL_LAUNCH_PACKED(4); break;
            case 8: APRIL_LAUNCH_PACKED(8); break;
            case 16: APRIL_LAUNCH_PACKED(16); break;
            default: APRIL_LAUNCH_PACKED(32); break;
        }
#undef APRIL_LAUNCH_PACKED
        if (escw)
            k_long<<<grid_long, kBlock, 0, st>>>(R, S, d_r, d_s, out, status, esc, counters, esc_cap, w0_long, jo);
        return cudaGetLastError();
    }
    const RawSets R{dev_set(Rd)}, S{dev_set(Sd)};
#define APRIL_LAUNCH_PERSISTENT(G)                                                                            \
    k_persistent<G, RawSets><<<grid_main, kBlock, 0, st>>>(R, S, d_r, d_s, n, out, status, t.cta_threshold,       \
                                                           big_list, counters, t.group_window, t.cta_window,      \
                                                           jo, escw, esc, esc_cap, rest)
    switch (t.group_lanes) {
        case 4: APRIL_LAUNCH_PERSISTENT(4); break;
        case 8: APRIL_LAUNCH_PERSISTENT(8); break;
        case 16: APRIL_LAUNCH_PERSISTENT(16); break;
        default: APRIL_LAUNCH_PERSISTENT(32); break;
    }
#undef APRIL_LAUNCH_PERSISTENT
    if (escw)
        k_long<<<grid_long, kBlock, 0, st>>>(R, S, d_r, d_s, out, status, esc, counters, esc_cap, w0_long, jo);
    return cudaGetLastError();
}

// The batched pipeline runs as one CUDA graph: captured on the context's
// private stream the first time an argument set is seen, then replayed on the
// caller's stream.
static april_status launch_batched(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                   const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *out,
                                   void *scratch, bool packed, cudaStream_t st) {
    const unsigned grid_bin = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 8);
    const uint32_t gl = ctx->tune.group_lanes;
    const int occ = ctx->persistent_blocks_per_sm[(packed ? 4 : 0) + group_index(gl)];
    const int bps = ctx->tune.blocks_per_sm ? (int)std::min<uint32_t>(ctx->tune.blocks_per_sm, (uint32_t)occ) : occ;
    const unsigned grid_main = (unsigned)std::max(1, ctx->num_sms * bps);
    GraphKey key{R->desc,         R->iv,          S->desc,          S->iv,          R->posts,       S->posts,
                 R->n_objects,    S->n_objects,   d_r,              d_s,            out,            scratch,
                 n,               ctx->tune,      grid_bin,         grid_main,      packed,         R->parts,
                 R->pdesc,        S->pdesc,       R->mbr,           S->mbr,         R->grid_ox,     R->grid_oy,
                 S->grid_ox,      S->grid_oy,     R->grid_log2_cell, S->grid_log2_cell, R->grid_known, S->grid_known,
                 R->grid_id,      S->grid_id,     R->part_grid};
    cudaError_t e;
    if (!ctx->graph || !(key == ctx->key)) {
        if (ctx->graph) {
            cudaGraphExecDestroy(ctx->graph);
            ctx->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        cudaError_t e1 = enqueue_batched(ctx, R, S, d_r, d_s, n, out, scratch, packed, grid_bin, grid_main,
                                         ctx->cap_stream);
        e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (e1 != cudaSuccess) e = e1;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->graph = nullptr;
            return cuda_fail(e, "capturing the batched pipeline");
        }
        ctx->key = key;
        ctx->graph_captures++;
    }
    e = cudaGraphLaunch(ctx->graph, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    ctx->graph_launches++;
    return APRIL_OK;
}

// Batched filter of one serving request (see server.cu): plain launches on
// `st` (no graph: every request has its own buffers), at most `max_ctas`
// persistent CTAs so that small requests leave SMs to the requests they
// overlap with, and a per-request status word.
april_status april_enqueue_request(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                   const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *d_verdict,
                                   void *d_scratch, uint32_t *d_status, unsigned max_ctas, void *stream) {
    if (n == 0) return APRIL_OK;
    if (check_layout(R) || check_layout(S)) return APRIL_ERR_INVALID_ARG;
    const bool packed = false;  // serving reads the raw lists
    const unsigned grid_bin = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 8));
    const uint32_t gl = ctx->tune.group_lanes;
    const int occ = ctx->persistent_blocks_per_sm[(packed ? 4 : 0) + group_index(gl)];
    unsigned grid_main = (unsigned)std::max(1, ctx->num_sms * occ);
    grid_main = std::min<unsigned>(grid_main, std::max<unsigned>(1, max_ctas));
    cudaError_t e = enqueue_batched(ctx, R, S, d_r, d_s, n, d_verdict, d_scratch, packed, grid_bin, grid_main,
                                    (cudaStream_t)stream, d_status);
    if (e != cudaSuccess) return cuda_fail(e, "enqueueing a serving request");
    return APRIL_OK;
}

int april_ctx_num_sms(const april_ctx *ctx) { return ctx->num_sms; }
int april_ctx_device(const april_ctx *ctx) { return ctx->device; }
uint32_t *april_ctx_status_word(april_ctx *ctx) { return ctx->d_status; }

extern "C" april_status april_filter_pairs(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                           const uint32_t *d_r, const uint32_t *d_s, uint64_t n,
                                           uint8_t *d_verdict, int mode, void *d_scratch, size_t scratch_bytes,
                                           void *stream) {
    if (!ctx || !R || !S) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return APRIL_OK;
    if (!d_r || !d_s || !d_verdict) return fail(APRIL_ERR_INVALID_ARG, "NULL pair or verdict array");
    const april_status chk = check_filter_args(R, S, n, mode);
    if (chk) return chk;
    cudaStream_t st = (cudaStream_t)stream;
    const DevSet dR = dev_set(R), dS = dev_set(S);
    const int sms = ctx->num_sms;
    switch (mode) {
        case APRIL_MODE_PLAIN: {
            uint64_t blocks = (n + 255) / 256;
            unsigned grid = (unsigned)std::min<uint64_t>(blocks, (uint64_t)sms * 8);
            k_plain<<<grid, 256, 0, st>>>(dR, dS, d_r, d_s, n, d_verdict, ctx->d_status);
            break;
        }
        case APRIL_MODE_WARP: {
            uint64_t blocks = (n + kBlock - 1) / kBlock;
            unsigned grid = (unsigned)std::min<uint64_t>(blocks, (uint64_t)sms * 16);
            k_warp<<<grid, kBlock, 0, st>>>(dR, dS, d_r, d_s, n, d_verdict, ctx->d_status, kWarpFirstWindow,
                                            join_order_of(ctx->tune.join_order, false));
            break;
        }
        case APRIL_MODE_BATCHED:
        case APRIL_MODE_BATCHED_PACKED: {
            size_t need = 0;
            april_filter_scratch_bytes(mode, n, &need);
            if (!d_scratch || scratch_bytes < need) return fail(APRIL_ERR_INVALID_ARG, "scratch missing or too small");
            if (((uintptr_t)d_scratch) & 255u) return fail(APRIL_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
            return launch_batched(ctx, R, S, d_r, d_s, n, d_verdict, d_scratch, mode == APRIL_MODE_BATCHED_PACKED, st);
        }
        default: return fail(APRIL_ERR_INVALID_ARG, "unknown mode");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return APRIL_OK;
}

// Decision plans (see K7).  Verdict v is encoded as -(v + 1).
static Plan make_plan(int predicate, uint32_t order_r, uint32_t order_s, uint32_t jo) {
    Plan P{};
    const int8_t TN = -1, TH = -2, INC = -3;
    if (predicate == APRIL_PREDICATE_WITHIN) {
        // Sec. 4.3.2: AA (no overlap: not within), then "every A(r) interval
        // lies in one F(s) interval" (yes: within; a violation: refine)
        P.nst = 2;
        P.xf[0] = 0; P.yf[0] = 0; P.pred[0] = kOverlap; P.on_true[0] = 1; P.on_false[0] = TN;
        P.xf[1] = 0; P.yf[1] = 1; P.pred[1] = kContain; P.on_true[1] = INC; P.on_false[1] = TH;
        return P;
    }
    // intersects in join order jo (step_outcome): 1 is Algorithm 2's AA AF FA
    // (for different granularity: AA, then the coarse side's F-list join)
    if (jo == 1) {
        P.xf[0] = 0; P.yf[0] = 0; P.pred[0] = kOverlap; P.on_true[0] = 1; P.on_false[0] = TN;
        if (order_r == order_s) {
            P.nst = 3;
            P.xf[1] = 0; P.yf[1] = 1; P.pred[1] = kOverlap; P.on_true[1] = TH; P.on_false[1] = 2;
            P.xf[2] = 1; P.yf[2] = 0; P.pred[2] = kOverlap; P.on_true[2] = TH; P.on_false[2] = INC;
        } else {
            P.nst = 2;
            const bool r_finer = order_r > order_s;
            P.sx = r_finer ? (uint8_t)(2 * (order_r - order_s)) : 0;
            P.sy = r_finer ? 0 : (uint8_t)(2 * (order_s - order_r));
            P.xf[1] = r_finer ? 0 : 1; P.yf[1] = r_finer ? 1 : 0; P.pred[1] = kOverlap;
            P.on_true[1] = TH; P.on_false[1] = INC;
        }
        return P;
    }
    if (order_r == order_s) {  // Algorithm 2's verdicts in the order AF, AA, FA
        P.nst = 3;
        P.xf[0] = 0; P.yf[0] = 1; P.pred[0] = kOverlap; P.on_true[0] = TH; P.on_false[0] = 1;
        P.xf[1] = 0; P.yf[1] = 0; P.pred[1] = kOverlap; P.on_true[1] = 2; P.on_false[1] = TN;
        P.xf[2] = 1; P.yf[2] = 0; P.pred[2] = kOverlap; P.on_true[2] = TH; P.on_false[2] = INC;
    } else if (order_r > order_s) {  // Sec. 5.3: coarsen r, use only the coarse side's F-list
        P.nst = 2;
        P.sx = (uint8_t)(2 * (order_r - order_s));
        P.xf[0] = 0; P.yf[0] = 1; P.pred[0] = kOverlap; P.on_true[0] = TH; P.on_false[0] = 1;
        P.xf[1] = 0; P.yf[1] = 0; P.pred[1] = kOverlap; P.on_true[1] = INC; P.on_false[1] = TN;
    } else {
        P.nst = 2;
        P.sy = (uint8_t)(2 * (order_s - order_r));
        P.xf[0] = 1; P.yf[0] = 0; P.pred[0] = kOverlap; P.on_true[0] = TH; P.on_false[0] = 1;
        P.xf[1] = 0; P.yf[1] = 0; P.pred[1] = kOverlap; P.on_true[1] = INC; P.on_false[1] = TN;
    }
    return P;
}

extern "C" april_status april_filter_pairs_ex(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                              const uint32_t *d_r, const uint32_t *d_s, uint64_t n,
                                              uint8_t *d_verdict, int predicate, void *d_scratch,
                                              size_t scratch_bytes, void *stream) {
    if (!ctx || !R || !S) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return APRIL_OK;
    if (!d_r || !d_s || !d_verdict) return fail(APRIL_ERR_INVALID_ARG, "NULL pair or verdict array");
    if (predicate != APRIL_PREDICATE_INTERSECTS && predicate != APRIL_PREDICATE_WITHIN)
        return fail(APRIL_ERR_INVALID_ARG, "unknown predicate");
    if (R->parts || S->parts) return fail(APRIL_ERR_INVALID_ARG, "april_filter_pairs_ex takes sets on one global grid");
    if (check_layout(R) || check_layout(S)) return APRIL_ERR_INVALID_ARG;
    if (predicate == APRIL_PREDICATE_WITHIN && R->order != S->order)
        return fail(APRIL_ERR_INVALID_ARG, "the within filter needs both sets on the same grid");
    if (n > 0xFFFFFFFFull) return fail(APRIL_ERR_INVALID_ARG, "at most 2^32-1 pairs per call");
    size_t need = 0;
    april_filter_scratch_bytes(APRIL_MODE_BATCHED, n, &need);
    if (!d_scratch || scratch_bytes < need) return fail(APRIL_ERR_INVALID_ARG, "scratch missing or too small");
    if (((uintptr_t)d_scratch) & 255u) return fail(APRIL_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *counters = (uint32_t *)d_scratch;
    uint32_t *big_list = (uint32_t *)((char *)d_scratch + kCounterBytes);
    const RawSets dR{dev_set(R)}, dS{dev_set(S)};
    const Plan P = make_plan(predicate, R->order, S->order, join_order_of(ctx->tune.join_order, false));
    const unsigned grid_bin = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)ctx->num_sms * 8);
    int bps = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_general, kBlock, 0);
    const unsigned grid_main = (unsigned)std::max(1, ctx->num_sms * std::max(bps, 1));
    cudaError_t e = cudaMemsetAsync(counters, 0, kCounterBytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    // the coarse triage (K2c): sets built from polygons on nested grids (same
    // origin and extent), no long-pair threshold
    const april_tune &t = ctx->tune;
    const bool coarse_triage = predicate == APRIL_PREDICATE_INTERSECTS && R->order != S->order && !t.triage_off &&
                               t.cta_threshold == kNoLongPairs && R->grid_known && S->grid_known && !R->parts && !S->parts && R->mbr &&
                               S->mbr && R->grid_ox == S->grid_ox && R->grid_oy == S->grid_oy &&
                               R->grid_log2_cell + R->order == S->grid_log2_cell + S->order;
    const uint32_t *rest = nullptr;
    if (coarse_triage) {
        const april_dev_sets *C = R->order < S->order ? R : S;
        const uint32_t sh = 2 * (R->order > S->order ? R->order - S->order : S->order - R->order);
        k_triage_coarse<<<grid_bin, 256, 0, st>>>(dR, dS, (const int4 *)R->mbr, (const int4 *)S->mbr,
                                                  TriageGrid{C->grid_ox, C->grid_oy, C->grid_log2_cell, C->order},
                                                  triage_lut(), sh, R->order > S->order, d_r, d_s, n, d_verdict,
                                                  ctx->d_status, big_list, counters);
        rest = big_list;
    } else {
        k_bin<<<grid_bin, 256, 0, st>>>(dR, dS, d_r, d_s, n, d_verdict, ctx->d_status, t.cta_threshold, big_list,
                                        counters);
    }
    k_general<<<grid_main, kBlock, 0, st>>>(P, dR.s, dS.s, d_r, d_s, n, d_verdict, ctx->d_status, t.cta_threshold,
                                            big_list, counters, t.cta_window, rest);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return APRIL_OK;
}

extern "C" april_status april_autotune(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                       const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *d_verdict,
                                       void *d_scratch, size_t scratch_bytes, void *stream, april_tune *out) {
    if (!ctx || !R || !S || !out) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) {
        *out = ctx->tune;
        return APRIL_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t thresholds[] = {2048, 4096, 8192, 16384, 0xffffffffu};
    const uint32_t groups[][2] = {{4, 8}, {4, 16}, {4, 32}, {8, 16}, {8, 32}, {8, 64}, {16, 32}, {16, 64}, {16, 128},
                                  {32, 64}};
    const april_tune saved = ctx->tune;
    april_tune best = saved;
    float best_ms = 1e30f;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    april_status rc = APRIL_OK;
    // times tuning t on the sample (best of three replays after the capture)
    auto time_tune = [&](const april_tune &t, float &best_here) -> april_status {
        ctx->tune = t;
        best_here = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaError_t e2 = cudaEventRecord(a, st);
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaEventRecord");
            april_status r2 = april_filter_pairs(ctx, R, S, d_r, d_s, n, d_verdict, APRIL_MODE_BATCHED, d_scratch,
                                                 scratch_bytes, stream);
            if (r2) return r2;
            e2 = cudaEventRecord(b, st);
            if (e2 == cudaSuccess) e2 = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e2 == cudaSuccess) e2 = cudaEventElapsedTime(&ms, a, b);
            if (e2 != cudaSuccess) return cuda_fail(e2, "timing an autotune candidate");
            if (rep > 0) best_here = std::min(best_here, ms);  // rep 0 captures the graph
        }
        return APRIL_OK;
    };
    // the context's tuning first: a candidate replaces it only if it is more
    // than 2% faster, so that the pick does not flip between shapes whose
    // times differ by noise
    float saved_ms = 1e30f;
    rc = time_tune(saved, saved_ms);
    // long pairs joined by one warp (first window 64 or 128) or by the whole CTA
    const uint32_t long_windows[] = {64u, 128u, saved.cta_window >= kBlock ? saved.cta_window : kBlock};
    for (uint32_t jo = 0; jo < 2 && rc == APRIL_OK; ++jo)
    for (uint32_t T : thresholds) {
        for (const auto &gw : groups)
        for (const uint32_t lw : long_windows) {
            if (T == 0xffffffffu && lw != long_windows[0]) continue;  // no long pairs: one scope is enough
            april_tune t = saved;
            t.cta_threshold = T;
            t.group_lanes = gw[0];
            t.group_window = gw[1];
            t.cta_window = lw;
            t.join_order = jo;
            float best_here = 1e30f;
            rc = time_tune(t, best_here);
            if (rc) break;
            if (best_here < best_ms) {
                best_ms = best_here;
                best = t;
            }
        }
        if (rc) break;
    }
    if (rc == APRIL_OK && saved_ms <= 1.02f * best_ms) {
        best = saved;
        best_ms = saved_ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) {
        ctx->tune = saved;
        return rc;
    }
    best.ms = best_ms;
    ctx->tune = best;
    *out = best;
    return APRIL_OK;
}

// april_filter_pairs_host in the batched modes pipelines the pairs in chunks
// of at least kPipeChunkMin pairs (at most kPipeMaxChunks): a chunk's pairs
// are copied in while the previous chunk is filtered, and its verdicts are
// copied out while the next one is.  Chunks alternate between two kernel
// streams, each with its own scratch, so that one chunk's tail overlaps the
// next chunk's start.  Each chunk costs a launch and a tail, which measured
// more than the copies it hides below 2^22 pairs (the end-to-end overhead is
// mostly fixed latency); 10M pairs in three chunks end 5% sooner than in one.
#ifndef APRIL_PIPE_CHUNK_LOG2
#define APRIL_PIPE_CHUNK_LOG2 22
#endif
constexpr uint64_t kPipeChunkMin = 1ull << APRIL_PIPE_CHUNK_LOG2;
constexpr uint32_t kPipeMaxChunks = 8;
static uint32_t pipe_chunks(uint64_t n) {
    return (uint32_t)std::min<uint64_t>(kPipeMaxChunks, std::max<uint64_t>(1, (n + kPipeChunkMin - 1) / kPipeChunkMin));
}
static uint64_t pipe_chunk_size(uint64_t n) {
    const uint32_t k = pipe_chunks(n);
    return ((n + k - 1) / k + 63) / 64 * 64;
}

// With the triage (K2), the pipeline is finer: the pairs are copied in
// chunks that double from kTriageChunk0 pairs up to kTriageChunkMax (at most
// kPipeMaxChunks, the last one taking what is left), and each chunk is
// triaged on one of two kernel streams as soon as it has arrived, while the
// next one is copied.  The triage appends to one rest list over all n pairs
// (indices plus the chunk's offset), so the lane groups then join it in one
// launch, with no chunk tails, and the verdicts are copied out.  The copies
// hide behind the triage, which reads about 3 pairs in the time the copy
// engine brings one in.
constexpr uint64_t kTriageChunk0 = 1ull << 18;
constexpr uint64_t kTriageChunkMax = 1ull << 21;

extern "C" april_status april_filter_host_work_bytes(int mode, uint64_t n, size_t *bytes) {
    if (!bytes) return fail(APRIL_ERR_INVALID_ARG, "bytes is NULL");
    size_t sb = 0;
    april_status st = april_filter_scratch_bytes(mode, n, &sb);
    if (st) return st;
    if (mode == APRIL_MODE_BATCHED || mode == APRIL_MODE_BATCHED_PACKED) {
        size_t sc = 0;  // per chunk, one region per kernel stream; the triage pipeline takes n's
        april_filter_scratch_bytes(mode, pipe_chunk_size(n), &sc);
        sb = std::max<size_t>(round256(sb), round256(sc) * (pipe_chunks(n) > 1 ? 2 : 1));
    }
    *bytes = (size_t)(round256(4 * n) * 2 + round256(n) + round256(sb));
    return APRIL_OK;
}

static april_status ensure_pipeline(april_ctx *ctx) {
    if (ctx->pipe[0]) return APRIL_OK;
    cudaError_t e = cudaSuccess;
    for (cudaStream_t &p : ctx->pipe)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p, cudaStreamNonBlocking);
    for (cudaEvent_t &v : ctx->pev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (cudaStream_t &p : ctx->pipe)
            if (p) cudaStreamDestroy(p), p = nullptr;
        for (cudaEvent_t &v : ctx->pev)
            if (v) cudaEventDestroy(v), v = nullptr;
        return cuda_fail(e, "creating the host pipeline's streams");
    }
    return APRIL_OK;
}

// The triage of pairs [off, off + cnt) of a call over n pairs (partition
// routing first for partitioned sets), appending to the call's rest list.
template <class SetsT>
static void enqueue_triage_chunk(april_ctx *ctx, const SetsT &R, const SetsT &S, const april_dev_sets *Rd,
                                 const april_dev_sets *Sd, const uint32_t *d_r, const uint32_t *d_s, uint64_t n,
                                 uint64_t off, uint64_t cnt, uint8_t *out, void *scratch, cudaStream_t st) {
    uint32_t *counters = (uint32_t *)scratch;
    uint32_t *big_list = (uint32_t *)((char *)scratch + kCounterBytes);
    const unsigned grid_bin = (unsigned)std::min<uint64_t>((cnt + 255) / 256, (uint64_t)ctx->num_sms * 8);
    const unsigned grid_tri = triage_grid(ctx->num_sms, cnt);
    if (Rd->parts) {
        uint32_t *er = (uint32_t *)((char *)scratch + kCounterBytes + round256(4 * n)) + off;
        uint32_t *es = (uint32_t *)((char *)scratch + kCounterBytes + 2 * round256(4 * n)) + off;
        uint32_t lg = 0;
        while ((1u << lg) < Rd->parts) ++lg;
        k_route<<<grid_bin, 256, 0, st>>>(part_view(Rd), part_view(Sd), lg, d_r + off, d_s + off, cnt, er, es);
        k_triage<true, SetsT><<<grid_tri, 256, 0, st>>>(R, S, triage_args(Rd, Sd, er, es), triage_lut(), d_r + off,
                                                        d_s + off, cnt, out + off, ctx->d_status, big_list, counters,
                                                        (uint32_t)off);
    } else {
        k_triage<false, SetsT><<<grid_tri, 256, 0, st>>>(R, S, triage_args(Rd, Sd, nullptr, nullptr), triage_lut(),
                                                         d_r + off, d_s + off, cnt, out + off, ctx->d_status, big_list,
                                                         counters, (uint32_t)off);
    }
}

static cudaError_t host_triage_pipeline(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                        const uint32_t *h_r, const uint32_t *h_s, uint64_t n, uint8_t *h_verdict,
                                        uint32_t *d_r, uint32_t *d_s, uint8_t *d_v, void *d_scr, bool packed,
                                        unsigned grid_main) {
    cudaStream_t s_in = ctx->pipe[0], k1 = ctx->pipe[1], k2 = ctx->pipe[2];
    cudaError_t e = cudaMemsetAsync(d_scr, 0, kCounterBytes, k1);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->pev[3], k1);  // the counters are reset
    if (e == cudaSuccess) e = cudaStreamWaitEvent(k2, ctx->pev[3], 0);
    uint64_t off = 0;
    for (uint32_t c = 0; off < n && e == cudaSuccess; ++c) {
        const uint64_t take = c + 1 == kPipeMaxChunks
                                  ? n - off
                                  : std::min<uint64_t>(std::min<uint64_t>(kTriageChunk0 << c, kTriageChunkMax), n - off);
        cudaStream_t ks = c & 1u ? k2 : k1;
        e = cudaMemcpyAsync(d_r + off, h_r + off, 4 * take, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_s + off, h_s + off, 4 * take, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->pev[2 + 2 * c], s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, ctx->pev[2 + 2 * c], 0);
        if (e == cudaSuccess) {
            if (packed)
                enqueue_triage_chunk(ctx, packed_set(R), packed_set(S), R, S, d_r, d_s, n, off, take, d_v, d_scr, ks);
            else
                enqueue_triage_chunk(ctx, RawSets{dev_set(R)}, RawSets{dev_set(S)}, R, S, d_r, d_s, n, off, take, d_v,
                                     d_scr, ks);
            e = cudaGetLastError();
        }
        off += take;
    }
    // the lane groups join the rest list once both kernel streams' triages are done
    if (e == cudaSuccess) e = cudaEventRecord(ctx->pev[5], k2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(k1, ctx->pev[5], 0);
    if (e == cudaSuccess) {
        const uint32_t *er = (const uint32_t *)((char *)d_scr + kCounterBytes + round256(4 * n));
        const uint32_t *es = (const uint32_t *)((char *)d_scr + kCounterBytes + 2 * round256(4 * n));
        e = enqueue_groups(ctx, R, S, R->parts ? er : d_r, R->parts ? es : d_s, n, d_v, d_scr, packed, grid_main, k1,
                           ctx->d_status, (const uint32_t *)((char *)d_scr + kCounterBytes));
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_verdict, d_v, n, cudaMemcpyDeviceToHost, k1);
    return e;
}

extern "C" april_status april_filter_pairs_host(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                                const uint32_t *h_r, const uint32_t *h_s, uint64_t n,
                                                uint8_t *h_verdict, int mode, void *d_work, size_t work_bytes,
                                                void *stream) {
    if (!ctx || !R || !S) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return APRIL_OK;
    if (!h_r || !h_s || !h_verdict || !d_work) return fail(APRIL_ERR_INVALID_ARG, "NULL host or work buffer");
    if (((uintptr_t)d_work) & 255u) return fail(APRIL_ERR_INVALID_ARG, "work buffer must be 256-byte aligned");
    size_t need = 0;
    april_status st = april_filter_host_work_bytes(mode, n, &need);
    if (st) return st;
    if (work_bytes < need) return fail(APRIL_ERR_INVALID_ARG, "work buffer too small");
    char *w = (char *)d_work;
    uint32_t *d_r = (uint32_t *)w;
    uint32_t *d_s = (uint32_t *)(w + round256(4 * n));
    uint8_t *d_v = (uint8_t *)(w + 2 * round256(4 * n));
    char *d_scr = w + 2 * round256(4 * n) + round256(n);
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e;
    if (mode != APRIL_MODE_BATCHED && mode != APRIL_MODE_BATCHED_PACKED) {
        // the one-pair-per-thread and per-warp modes: copy in, filter, copy out
        e = cudaMemcpyAsync(d_r, h_r, 4 * n, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, h_s, 4 * n, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(pairs)");
        st = april_filter_pairs(ctx, R, S, d_r, d_s, n, d_v, mode, nullptr, 0, stream);
        if (st) return st;
        e = cudaMemcpyAsync(h_verdict, d_v, n, cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(verdicts)");
        return april_sync_status(ctx, stream);
    }
    st = check_filter_args(R, S, n, mode);
    if (st) return st;
    st = ensure_pipeline(ctx);
    if (st) return st;
    const bool packed = mode == APRIL_MODE_BATCHED_PACKED;
    const uint32_t K = pipe_chunks(n);
    const uint64_t cs_n = pipe_chunk_size(n);
    size_t sb = 0;
    april_filter_scratch_bytes(mode, cs_n, &sb);
    sb = round256(sb);
    const uint32_t gl = ctx->tune.group_lanes;
    const int occ = ctx->persistent_blocks_per_sm[(packed ? 4 : 0) + group_index(gl)];
    const int bps = ctx->tune.blocks_per_sm ? (int)std::min<uint32_t>(ctx->tune.blocks_per_sm, (uint32_t)occ) : occ;
    const unsigned grid_main = (unsigned)std::max(1, ctx->num_sms * bps);
    cudaStream_t s_in = ctx->pipe[0], s_out = ctx->pipe[3];
    cudaEvent_t ev_start = ctx->pev[0], ev_end = ctx->pev[1];
    // the pipeline follows the work already queued on the caller's stream
    e = cudaEventRecord(ev_start, cs);
    for (cudaStream_t p : ctx->pipe)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p, ev_start, 0);
    const bool triaged = triage_applies(ctx->tune, R, S, packed);
    if (triaged && e == cudaSuccess)
        e = host_triage_pipeline(ctx, R, S, h_r, h_s, n, h_verdict, d_r, d_s, d_v, d_scr, packed, grid_main);
    for (uint32_t c = 0; c < K && e == cudaSuccess && !triaged; ++c) {
        const uint64_t off = c * cs_n;
        if (off >= n) break;
        const uint64_t cnt = std::min<uint64_t>(cs_n, n - off);
        cudaStream_t ks = ctx->pipe[1 + (c & 1u)];
        cudaEvent_t ev_in = ctx->pev[2 + 2 * c], ev_k = ctx->pev[3 + 2 * c];
        e = cudaMemcpyAsync(d_r + off, h_r + off, 4 * cnt, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_s + off, h_s + off, 4 * cnt, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in, s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, ev_in, 0);
        if (e == cudaSuccess) {
            const unsigned grid_bin = (unsigned)std::min<uint64_t>((cnt + 255) / 256, (uint64_t)ctx->num_sms * 8);
            e = enqueue_batched(ctx, R, S, d_r + off, d_s + off, cnt, d_v + off, d_scr + (K > 1 ? (c & 1u) * sb : 0),
                                packed, grid_bin, grid_main, ks);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_k, ks);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_k, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_verdict + off, d_v + off, cnt, cudaMemcpyDeviceToHost, s_out);
    }
    // the caller's stream waits for every stream of the pipeline
    for (uint32_t q = 0; q < 4 && e == cudaSuccess; ++q) {
        e = cudaEventRecord(ev_end, ctx->pipe[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_end, 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "april_filter_pairs_host pipeline");
    return april_sync_status(ctx, stream);
}

extern "C" april_status april_sync_status(april_ctx *ctx, void *stream) {
    if (!ctx) return fail(APRIL_ERR_INVALID_ARG, "ctx is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->d_status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "april_sync_status");
    if (h) {
        e = cudaMemsetAsync(ctx->d_status, 0, 4, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "april_sync_status(clear)");
    }
    if (h & ST_TIMEOUT) return fail(APRIL_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
    if (h & ST_BAD_ID) return fail(APRIL_ERR_OUT_OF_RANGE_ID, "a pair named an out-of-range object id");
    return APRIL_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// For callers that cannot allocate device memory on the call path -- for
// example code running where cudaMalloc is forbidden or would synchronize
// the device (inside a real-time serving loop, or a plugin whose host owns
// every allocation) -- the batched filter can run with its scratch in this
// file-scope device array instead of caller memory.  The array is part of
// the loaded module, so every GPU that loads libapril holds it (16 MiB +
// 512 bytes) until the process exits.  Layout: the batched pipeline's
// 256-byte counter block (cleared by every call), a 256-byte status block
// (word 0: the ST_* bits of every call since the last status query), then
// the list of long pairs, one uint32 per pair.
constexpr uint64_t kNoAllocMaxPairs = 4ull << 20;
constexpr uint32_t kNoAllocStatusWord = kCounterBytes / 4;
constexpr uint32_t kNoAllocListWord = 2 * kCounterBytes / 4;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocListWord + kNoAllocMaxPairs];

namespace {

struct NoAllocDevice {
    bool ready = false;
    int num_sms = 0;
    int blocks_per_sm = 1;
};
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

}  // namespace

// The persistent kernel instance for the default tuning's lane groups.
using PersistentRaw = void (*)(RawSets, RawSets, const uint32_t *, const uint32_t *, uint64_t, uint8_t *,
                               uint32_t *, uint32_t, const uint32_t *, uint32_t *, uint32_t, uint32_t, uint32_t,
                               uint32_t, uint4 *, uint32_t, const uint32_t *);
static PersistentRaw noalloc_kernel(uint32_t group_lanes) {
    switch (group_lanes) {
        case 4: return k_persistent<4, RawSets>;
        case 8: return k_persistent<8, RawSets>;
        case 16: return k_persistent<16, RawSets>;
        default: return k_persistent<32, RawSets>;
    }
}

// Device address of g_noalloc_scratch on the current device.  Host code
// cannot use the array's name as an address (it names a host-side stand-in),
// so the address is looked up on every call (no allocation; after the first
// call on a device the module is loaded and the lookup is cheap).
static april_status noalloc_scratch(uint32_t **ptr) {
    cudaError_t e = cudaGetSymbolAddress((void **)ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    return APRIL_OK;
}

extern "C" april_status april_filter_pairs_noalloc(const april_dev_sets *R, const april_dev_sets *S,
                                                   const uint32_t *d_r, const uint32_t *d_s, uint64_t n,
                                                   uint8_t *d_verdict, void *stream) {
    if (!R || !S) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return APRIL_OK;
    if (!d_r || !d_s || !d_verdict) return fail(APRIL_ERR_INVALID_ARG, "NULL pair or verdict array");
    if (R->order != S->order) return fail(APRIL_ERR_INVALID_ARG, "R and S are on different grids");
    if (R->parts || S->parts) return fail(APRIL_ERR_INVALID_ARG, "april_filter_pairs_noalloc takes unpartitioned sets");
    if (check_layout(R) || check_layout(S)) return APRIL_ERR_INVALID_ARG;
    if (n > kNoAllocMaxPairs)
        return fail(APRIL_ERR_INVALID_ARG, "april_filter_pairs_noalloc: n exceeds APRIL_NOALLOC_MAX_PAIRS (4194304); "
                                           "split the pairs or use april_filter_pairs with caller scratch");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(APRIL_ERR_INVALID_ARG, "device index out of range");
    const april_tune t = default_tune();
    uint32_t *scratch = nullptr;
    april_status rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    NoAllocDevice nd;
    {
        // first call on this device: the launch shape (the current device is
        // the one being set up)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoAllocDevice &slot = g_noalloc_dev[dev];
        if (!slot.ready) {
            int sms = 0, bps = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, noalloc_kernel(t.group_lanes), kBlock, 0);
            if (e != cudaSuccess) return cuda_fail(e, "april_filter_pairs_noalloc set-up");
            slot.num_sms = sms;
            slot.blocks_per_sm = bps < 1 ? 1 : bps;
            slot.ready = true;
        }
        nd = slot;
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *counters = scratch;
    uint32_t *status = scratch + kNoAllocStatusWord;
    uint32_t *big_list = scratch + kNoAllocListWord;
    // the array keeps the previous call's contents: reset the counters (the
    // status block keeps its bits until april_noalloc_sync_status reads them)
    e = cudaMemsetAsync(counters, 0, kCounterBytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(no-alloc counters)");
    const RawSets dR{dev_set(R)}, dS{dev_set(S)};
    const unsigned grid_bin = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)nd.num_sms * 8);
    const unsigned grid_main = (unsigned)std::max(1, nd.num_sms * nd.blocks_per_sm);
    const uint32_t *rest = nullptr;
    if (triage_applies(t, R, S, false)) {
        k_triage<false, RawSets><<<triage_grid(nd.num_sms, n), 256, 0, st>>>(
            dR, dS, triage_args(R, S, nullptr, nullptr), triage_lut(), d_r, d_s, n, d_verdict, status, big_list,
            counters, 0u);
        rest = big_list;
    } else if (t.cta_threshold != kNoLongPairs) {
        k_bin<<<grid_bin, 256, 0, st>>>(dR, dS, d_r, d_s, n, d_verdict, status, t.cta_threshold, big_list, counters);
    }
    // no escalation: the static array has no room for the queue of handed-over joins
    noalloc_kernel(t.group_lanes)<<<grid_main, kBlock, 0, st>>>(dR, dS, d_r, d_s, n, d_verdict, status,
                                                                t.cta_threshold, big_list, counters, t.group_window,
                                                                t.cta_window, join_order_of(t.join_order, rest != nullptr),
                                                                0u, nullptr, 0u, rest);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "april_filter_pairs_noalloc launch");
    return APRIL_OK;
}

extern "C" april_status april_noalloc_sync_status(void *stream) {
    uint32_t *scratch = nullptr;
    april_status rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t h = 0;  // pageable: the copy has completed when the call returns
    cudaError_t e = cudaMemcpyAsync(&h, scratch + kNoAllocStatusWord, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "april_noalloc_sync_status");
    if (h) {
        e = cudaMemsetAsync(scratch + kNoAllocStatusWord, 0, 4, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "april_noalloc_sync_status(clear)");
    }
    if (h & ST_TIMEOUT) return fail(APRIL_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
    if (h & ST_BAD_ID) return fail(APRIL_ERR_OUT_OF_RANGE_ID, "a pair named an out-of-range object id");
    return APRIL_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: the iteration limit of the filter kernels' bounded waits.
extern "C" april_status april_debug_set_wait_limit(uint32_t spins) {
    cudaError_t e = cudaMemcpyToSymbol(c_wait_limit, &spins, sizeof(spins));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(c_wait_limit)");
    return APRIL_OK;
}
