// Device-side interval joins of the APRIL filter (paper Sec. 4.2,
// Algorithm 2: IntervalJoin and its use in the AA, AF, FA sequence).
//
// Interval convention: [st, end) with end stored mod 2^32; comparisons use
// last = end - 1 in uint32, so an interval holding cell 2^32-1 (end 2^32,
// stored as 0) compares correctly.
//   X_i overlaps Y_j  <=>  X_i.st <= Y_j.last  and  Y_j.st <= X_i.last
//   merge step        :    advance X if X_i.last <= Y_j.last, else Y.
//
// Parallel join.  The sequential merge walks the merge path of X and Y
// ordered by `last` (ties: X first).  At diagonal d (d elements emitted) it
// sits at state (i, d - i) and tests X_i against Y_{d-i}.  "Some test
// succeeds" is the answer, so any split of the diagonals gives the same
// boolean.  A group (a warp or a CTA) stages a window of each list in shared
// memory, every thread finds the merge-path state at its first diagonal by
// binary search in the window and then walks a few diagonals serially, doing
// exactly the tests the sequential merge does there.  The group ORs the
// results, advances both lists by the split at the window's last diagonal,
// and doubles the window (up to a maximum) so that joins that stop early read
// little while long scans keep many bytes in flight.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace april_dev {

constexpr unsigned kFull = 0xffffffffu;

struct DevSet {
    const uint4 *desc;      // per object {a_off, a_len, f_off, f_len}
    const uint2 *iv;        // intervals {st, end}
    uint32_t n;
    const uint32_t *posts;  // skip index: last cell of interval slot 16 q + 15
};

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// IntervalJoin as written in Algorithm 2: one thread walks both lists.
__device__ __forceinline__ bool seq_join(const uint2 *__restrict__ X, uint32_t nx, const uint2 *__restrict__ Y,
                                         uint32_t ny) {
    if (nx == 0 || ny == 0) return false;
    uint32_t i = 0, j = 0;
    uint2 x = __ldg(X), y = __ldg(Y);
    for (;;) {
        const uint32_t xl = x.y - 1u, yl = y.y - 1u;
        if (x.x <= yl && y.x <= xl) return true;
        if (xl <= yl) {
            if (++i == nx) return false;
            x = __ldg(X + i);
        } else {
            if (++j == ny) return false;
            y = __ldg(Y + j);
        }
    }
}

// Shared-memory accesses on 32-bit shared-window addresses (the windows
// always live in shared memory; explicit ld.shared avoids generic addressing).
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint2 lds2(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ uint32_t lds1(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(a));
    return v;
}

// Merge-path split of the windows at shared addresses xa (nx intervals) and
// ya (ny intervals) at diagonal d: the number of X elements among the first
// d merged elements (X first on equal `last`).
#ifndef APRIL_SEARCH_FIXED
#define APRIL_SEARCH_FIXED 0
#endif
__device__ __forceinline__ uint32_t merge_split(uint32_t xa, uint32_t nx, uint32_t ya, uint32_t ny, uint32_t d) {
    uint32_t lo = d > ny ? d - ny : 0u, hi = min(d, nx);
    // compares X[mid].last <= Y[d-mid-1].last; the byte offsets of the two
    // `end` words move in opposite directions as mid changes
    const uint32_t yb = ya + 8u * (d - 1u) + 4u;
#if APRIL_SEARCH_FIXED
    // a fixed trip count (windows hold at most 2048 intervals): no divergence
#pragma unroll
    for (int it = 0; it < 12; ++it) {
        if (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            const uint32_t xl = lds1(xa + 8u * mid + 4u) - 1u;
            const uint32_t yl = lds1(yb - 8u * mid) - 1u;
            if (xl <= yl) lo = mid + 1;
            else hi = mid;
        }
    }
#else
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t xl = lds1(xa + 8u * mid + 4u) - 1u;
        const uint32_t yl = lds1(yb - 8u * mid) - 1u;
        if (xl <= yl) lo = mid + 1;
        else hi = mid;
    }
#endif
    return lo;
}

// Walks `steps` diagonals of the window from state (i, j): the tests of the
// sequential merge at those states.  `full` windows (neither list ends in
// them) need no bound checks.  Returns the OR of the tests; *state receives
// i after the last step, or 0xffffffff if a list ran out first.
// Predicates a join can test at each merge state (i, j):
//   kOverlap   X_i overlaps Y_j (Algorithm 2's IntervalJoin)
//   kContain   X_i is emitted here but Y_j does not start at or before it, so
//              Y_j (the first Y ending at or after X_i) cannot contain X_i --
//              a violation of "every X interval lies in one Y interval"
//              (the within-join variant of Sec. 4.3.2)
enum JoinPred : int { kOverlap = 0, kContain = 1 };

template <uint32_t PER, int PRED = kOverlap>
__device__ __forceinline__ bool walk_fixed(uint32_t xa, uint32_t ya, uint32_t i, uint32_t j, uint32_t &state) {
    uint2 x = lds2(xa + 8u * i), y = lds2(ya + 8u * j);
    bool found = false;
#pragma unroll
    for (uint32_t q = 0; q < PER; ++q) {
        const uint32_t xl = x.y - 1u, yl = y.y - 1u;
        const bool ax = xl <= yl;
        if (PRED == kOverlap) found |= (x.x <= yl) & (y.x <= xl);
        else found |= ax & (y.x > x.x);
        i += ax;
        j += !ax;
        if (q + 1 < PER) {
            const uint2 v = lds2(ax ? xa + 8u * i : ya + 8u * j);
            x = ax ? v : x;
            y = ax ? y : v;
        }
    }
    state = i;
    return found;
}

template <int PRED = kOverlap>
__device__ __forceinline__ bool walk_checked(uint32_t xa, uint32_t nx, uint32_t ya, uint32_t ny, uint32_t i,
                                             uint32_t j, uint32_t steps, uint32_t &state) {
    bool found = false;
    uint32_t q = 0;
    for (; q < steps && i < nx && j < ny; ++q) {
        const uint2 x = lds2(xa + 8u * i), y = lds2(ya + 8u * j);
        const uint32_t xl = x.y - 1u, yl = y.y - 1u;
        const bool ax = xl <= yl;
        if (PRED == kOverlap) found |= (x.x <= yl) & (y.x <= xl);
        else found |= ax & (y.x > x.x);
        i += ax;
        j += !ax;
    }
    // containment: Y ran out (this is its last window) while X elements remain
    if (PRED == kContain && q < steps && j >= ny && i < nx) found = true;
    state = (q == steps) ? i : 0xffffffffu;
    return found;
}

// The merge-path work of one thread in a window of D diagonals (w per list,
// nx/ny staged): diagonals [d0, d0 + per), per a power of two <= MAXPER.
template <uint32_t MAXPER, int PRED = kOverlap>
__device__ __forceinline__ bool window_walk(uint32_t xa, uint32_t nx, uint32_t ya, uint32_t ny, uint32_t w,
                                            uint32_t D, uint32_t per, uint32_t d0, uint32_t &state) {
    state = 0xffffffffu;
    if (d0 >= D) return false;
    const uint32_t i = merge_split(xa, nx, ya, ny, d0);
    const uint32_t j = d0 - i;
    if (nx == w && ny == w) {
        if constexpr (MAXPER >= 16) {
            switch (per) {
                case 1: return walk_fixed<1, PRED>(xa, ya, i, j, state);
                case 2: return walk_fixed<2, PRED>(xa, ya, i, j, state);
                case 4: return walk_fixed<4, PRED>(xa, ya, i, j, state);
                case 8: return walk_fixed<8, PRED>(xa, ya, i, j, state);
                default: return walk_fixed<16, PRED>(xa, ya, i, j, state);
            }
        } else {
            switch (per) {
                case 1: return walk_fixed<1, PRED>(xa, ya, i, j, state);
                case 2: return walk_fixed<2, PRED>(xa, ya, i, j, state);
                case 4: return walk_fixed<4, PRED>(xa, ya, i, j, state);
                default: return walk_fixed<8, PRED>(xa, ya, i, j, state);
            }
        }
    }
    return walk_checked<PRED>(xa, nx, ya, ny, i, j, min(per, D - d0), state);
}

// Coarsens a staged window in place (Sec. 5.3, joining approximations of
// different granularity): interval [st, end) of the finer grid becomes the
// interval of the coarser grid's cells that contain its cells,
// [st >> sh, ((end - 1) >> sh) + 1).  The result is sorted by start and by
// end but may overlap its neighbours, which the merge tolerates on this side.
template <uint32_t NT>
__device__ __forceinline__ void coarsen_window(uint32_t a, uint32_t cnt, uint32_t sh, uint32_t tid) {
    for (uint32_t k = tid; k < cnt; k += NT) {
        const uint2 v = lds2(a + 8u * k);
        const uint32_t st = v.x >> sh, en = ((v.y - 1u) >> sh) + 1u;
        asm volatile("st.shared.v2.u32 [%0], {%1, %2};\n" ::"r"(a + 8u * k), "r"(st), "r"(en));
    }
}

struct WarpScope {
    static __device__ __forceinline__ void sync() { __syncwarp(); }
    static __device__ __forceinline__ uint32_t sum(uint32_t v) { return __reduce_add_sync(kFull, v); }
    static __device__ __forceinline__ bool all(bool b) { return __all_sync(kFull, b) != 0; }
    static __device__ __forceinline__ uint32_t count(bool b) { return __popc(__ballot_sync(kFull, b)); }
    // OR of `b` over the group; `v` from thread `src` is returned to all.
    // Doubles as the point after which the window may be overwritten.
    static __device__ __forceinline__ bool vote(bool b, uint32_t &v, uint32_t src, uint32_t *) {
        v = __shfl_sync(kFull, v, src);
        return __any_sync(kFull, b) != 0;
    }
};

struct CtaScope {
    static __device__ __forceinline__ void sync() { __syncthreads(); }
    // sum of per-thread counts below 16 (bit by bit)
    static __device__ __forceinline__ uint32_t sum(uint32_t v) {
        return (uint32_t)__syncthreads_count(v & 1u) + 2u * (uint32_t)__syncthreads_count(v & 2u) +
               4u * (uint32_t)__syncthreads_count(v & 4u) + 8u * (uint32_t)__syncthreads_count(v & 8u);
    }
    static __device__ __forceinline__ bool all(bool b) { return __syncthreads_and(b) != 0; }
    static __device__ __forceinline__ uint32_t count(bool b) { return (uint32_t)__syncthreads_count(b); }
    static __device__ __forceinline__ bool vote(bool b, uint32_t &v, uint32_t src, uint32_t *slot) {
        if (threadIdx.x == src) *slot = v;
        const bool any = __syncthreads_or(b) != 0;
        v = *slot;
        return any;
    }
};

// ----- TMA bulk copies and mbarriers (sm_90+ PTX; used on sm_103a) -----
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

// Orders this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// One-dimensional bulk copy global -> shared; completes `bytes` on the mbarrier.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Spins on the mbarrier phase with an iteration limit; false if it ran out.
// The limit of the waits for window copies is c_wait_limit (default
// kMbarSpinLimit; a diagnostic setter lowers it, down to 0 = give up at once,
// so that the timeout path can run without any fault).  After a wait gave
// up, the copies it waited for may still be in flight: mbar_drain waits for
// them with the fixed limit kMbarDrainLimit before the join returns, so that
// no copy lands in shared memory the block no longer owns.
constexpr uint32_t kMbarSpinLimit = 1u << 24;
constexpr uint32_t kMbarDrainLimit = 1u << 24;
__constant__ uint32_t c_wait_limit = kMbarSpinLimit;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    const uint32_t lim = c_wait_limit;
    for (uint32_t k = 0; k < lim; ++k)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t phase) {
    for (uint32_t k = 0; k < kMbarDrainLimit; ++k)
        if (mbar_try_wait(bar, phase)) return;
}

// Window staging by bulk copy: the 16-byte aligned span around src[0..cnt)
// (src - 1 when src is odd, rounded up to an even count) is copied to buf;
// returns the shared address of src[0] inside buf and the byte count.  The
// device image ends with a 16-byte pad, so the rounding never leaves it.
__device__ __forceinline__ uint32_t bulk_span(const uint2 *src, uint32_t cnt, const uint2 *&a, uint32_t &bytes,
                                              uint32_t &odd) {
    odd = (uint32_t)(((uintptr_t)src >> 3) & 1u);
    a = src - odd;
    bytes = ((cnt + odd + 1) & ~1u) * 8u;
    return odd * 8u;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Copies src[0..cnt) into shared memory so that the returned pointer p has
// p[k] == src[k].  Lists start 16-byte aligned, so src - (src odd) is too;
// the copy runs in 16-byte pieces from there (buf holds WMAX + 2 intervals,
// 16-byte aligned).  Elements outside [src-1, src+cnt) are never read.
template <uint32_t NT>
__device__ __forceinline__ uint2 *stage_window(uint2 *buf, const uint2 *src, uint32_t cnt, uint32_t tid) {
    const uint32_t odd = (uint32_t)(((uintptr_t)src >> 3) & 1u);
    const uint2 *a = src - odd;
    const uint32_t tot = cnt + odd, full = tot >> 1;
    for (uint32_t c = tid; c < full; c += NT) cp_async16(buf + 2 * c, a + 2 * c);
    if ((tot & 1u) && tid == full % NT) cp_async8(buf + tot - 1, a + tot - 1);
    return buf + odd;
}

// A list as the joins read it.  RawList: intervals in global memory, staged
// into shared memory with 16-byte cp.async.  PackedList: the compressed form
// of Sec. 5.1 (blocks of 32 endpoints: a uint32 anchor and 31 uint16 or uint32
// gaps), decoded in registers by the staging threads (one block per thread,
// a running sum over the block) and stored to shared memory as intervals.
// Either way the window's intervals end up at the returned shared address.
struct RawList {
    static constexpr bool kBulk = true;
    static constexpr bool kRandomAccess = true;
    static constexpr uint32_t kKeyStride = 1;  // words per search key in keys()
    const uint2 *p;
    uint32_t n;
    const uint32_t *pk;  // the set's posts from the one that closes a slot of this list on
    template <uint32_t NT>
    __device__ __forceinline__ uint32_t stage(uint2 *buf, uint32_t i0, uint32_t cnt, uint32_t tid, uint32_t) const {
        return smem_addr(stage_window<NT>(buf, p + i0, cnt, tid));
    }
    // Bulk-copy form: called by the one issuing thread; returns bytes in flight.
    __device__ __forceinline__ uint32_t issue(uint2 *buf, uint32_t i0, uint32_t cnt, uint32_t bar) const {
        const uint2 *a;
        uint32_t bytes, odd;
        bulk_span(p + i0, cnt, a, bytes, odd);
        bulk_load(smem_addr(buf), a, bytes, bar);
        return bytes;
    }
    __device__ __forceinline__ uint32_t window(const uint2 *buf, uint32_t i0) const {
        return smem_addr(buf) + 8u * (uint32_t)(((uintptr_t)(p + i0) >> 3) & 1u);
    }
    __device__ __forceinline__ uint32_t first_start() const { return __ldg(&p->x); }
    // Start search over the skip index.  The set's post q is the last cell of
    // interval slot 16 q + 15; interval arrays start 256-byte aligned, so this
    // list's first post closes its interval pb = 15 - (slot % 16) and post k
    // closes interval pb + 16 k.  With c posts below the target, every
    // interval up to pb + 16 (c - 1) ends below it, and the join may start
    // right after that one: at most 16 intervals before the first that can
    // meet, all of which the merge passes over without a verdict.
    __device__ __forceinline__ uint32_t pb() const { return 15u - (uint32_t)(((uintptr_t)p >> 3) & 15u); }
    __device__ __forceinline__ uint32_t keys_n() const {
        const uint32_t b = pb();
        return n > b ? (n - 1 - b) / 16 + 1 : 0u;
    }
    __device__ __forceinline__ uint32_t key(uint32_t q) const { return __ldg(pk + q); }
    __device__ __forceinline__ const uint32_t *keys() const { return pk; }
    __device__ __forceinline__ uint32_t start_of(uint32_t c) const { return c ? pb() + 16u * (c - 1) + 1u : 0u; }
    // The largest post count c with start_of(c) <= j (j < n): a search from
    // merge position j counts the posts from there on.
    __device__ __forceinline__ uint32_t key_lo(uint32_t j) const {
        const uint32_t b = pb();
        return j > b ? (j - b - 1) / 16 + 1 : 0u;
    }
};

struct PackedList {
    static constexpr bool kBulk = false;
    static constexpr bool kRandomAccess = false;
    static constexpr uint32_t kKeyStride = 2;  // words per search key: the anchors of the block table
    const uint2 *blocks;  // per block {anchor, gap_off64 | wide << 31}
    const uint8_t *gaps;  // the set's gap stream
    uint32_t n;
    // Decodes the window [i0, i0 + cnt) into shared memory as intervals.  The
    // window's endpoints are split into slices of 8 (a quarter of a block),
    // one slice per thread per round: the thread loads its slice's gaps with
    // one 16-byte load (two for 32-bit gaps), sums them in registers, the 4
    // threads of a block add the totals of the slices before theirs (two
    // shuffle steps) and the block anchor, and every endpoint inside the
    // window is stored.  A block's slot 0 holds no gap (the anchor is its
    // endpoint 0) and reads as 0.  `mask` names the threads of this warp that
    // call stage together (whole groups of 4 consecutive lanes).
    template <uint32_t NT>
    __device__ __forceinline__ uint32_t stage(uint2 *buf, uint32_t i0, uint32_t cnt, uint32_t tid,
                                              uint32_t mask) const {
        static_assert(NT >= 4, "a block's four slices are decoded by four threads at once");
        const uint32_t base = smem_addr(buf);
        const uint32_t e0 = 2 * i0, e1 = 2 * (i0 + cnt);  // endpoint range of the window
        const uint32_t b0 = e0 >> 5, nsl = ((((e1 - 1) >> 5) - b0) + 1) * 4;
        for (uint32_t s0 = 0; s0 < nsl; s0 += NT) {
            const uint32_t sl = s0 + tid, q = sl & 3u;
            const bool on = sl < nsl;
            uint32_t g[8], anchor = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) g[k] = 0;
            if (on) {
                const uint2 meta = __ldg(blocks + b0 + (sl >> 2));
                anchor = meta.x;
                const uint8_t *gb = gaps + 64ull * (meta.y & 0x7FFFFFFFu);
                if (meta.y >> 31) {
                    const uint4 *p4 = (const uint4 *)(gb + 32u * q);
                    const uint4 u = __ldg(p4), v = __ldg(p4 + 1);
                    g[0] = u.x; g[1] = u.y; g[2] = u.z; g[3] = u.w;
                    g[4] = v.x; g[5] = v.y; g[6] = v.z; g[7] = v.w;
                } else {
                    const uint4 u = __ldg((const uint4 *)(gb + 16u * q));
                    g[0] = u.x & 0xFFFFu; g[1] = u.x >> 16; g[2] = u.y & 0xFFFFu; g[3] = u.y >> 16;
                    g[4] = u.z & 0xFFFFu; g[5] = u.z >> 16; g[6] = u.w & 0xFFFFu; g[7] = u.w >> 16;
                }
            }
#pragma unroll
            for (int k = 1; k < 8; ++k) g[k] += g[k - 1];
            // inclusive scan of the slice totals over the block's 4 threads
            uint32_t x = g[7];
            uint32_t y = __shfl_up_sync(mask, x, 1, 4);
            if (q >= 1) x += y;
            y = __shfl_up_sync(mask, x, 2, 4);
            if (q >= 2) x += y;
            const uint32_t v0 = anchor + x - g[7];
            const uint32_t ebase = 32u * (b0 + (sl >> 2)) + 8u * q;
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k) {
                const uint32_t e = ebase + k;
                if (on && e >= e0 && e < e1)
                    asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(base + 4 * (e - e0)), "r"(v0 + g[k]));
            }
        }
        return base;
    }
    __device__ __forceinline__ uint32_t issue(uint2 *, uint32_t, uint32_t, uint32_t) const { return 0; }
    __device__ __forceinline__ uint32_t window(const uint2 *buf, uint32_t) const { return smem_addr(buf); }
    __device__ __forceinline__ uint32_t first_start() const { return __ldg(&blocks->x); }
    // Start search over the block anchors: block b's anchor is the start of
    // its interval 16b, so with c blocks anchored below the target every
    // interval before 16 (c - 1) ends below it as well; the search starts at
    // that block boundary, at or before the first interval that can meet.
    __device__ __forceinline__ uint32_t keys_n() const { return (2 * n + 31) / 32; }
    __device__ __forceinline__ uint32_t key(uint32_t q) const { return __ldg(&blocks[q].x); }
    __device__ __forceinline__ const uint32_t *keys() const { return (const uint32_t *)blocks; }
    __device__ __forceinline__ uint32_t start_of(uint32_t c) const { return c ? 16u * (c - 1) : 0u; }
    __device__ __forceinline__ uint32_t key_lo(uint32_t j) const { return j / 16 + 1; }  // start_of(.) <= j < n
};

// The final round of a start search over sorted keys (a skip index, or block
// anchors at a stride of two words): the count of keys below t (after a
// right shift by sh) among keys [lo, hi) of `keys`, where hi - lo is at most
// P NT kPostVec - (P - 1) with P = 4 / STRIDE keys per 16-byte word.  Each
// thread loads kPostVec 16-byte words of keys (the group's loads cover one
// aligned run that holds [lo, hi)) and counts; the group sums.
#ifndef APRIL_POST_VEC
#define APRIL_POST_VEC 2
#endif
constexpr uint32_t kPostVec = APRIL_POST_VEC;
template <uint32_t STRIDE>  // words per key: 1 (posts) or 2 (block anchors, the first word of each pair)
__device__ __forceinline__ uint32_t post_count(const uint32_t *keys, uint32_t lo, uint32_t hi, uint32_t sh,
                                               uint32_t t, uint32_t tid, uint32_t nt) {
    constexpr int PER = 4 / STRIDE;  // keys per 16-byte word
    uint32_t c = 0;
    if (lo < hi) {
        const int mis = (int)(((uintptr_t)(keys + STRIDE * lo) >> 2) & 3u) / (int)STRIDE;
        // aligned down (signed: lo may be below mis), still inside the array
        const uint4 *base = (const uint4 *)(keys + (ptrdiff_t)STRIDE * ((ptrdiff_t)lo - mis));
        const int ilo = (int)lo, ihi = (int)hi;
#pragma unroll
        for (uint32_t j = 0; j < kPostVec; ++j) {
            const int v = (int)(tid + nt * j);  // 16-byte word of the run
            const int k0 = ilo - mis + PER * v;  // its first key (may lie before lo)
            if (k0 < ihi) {
                const uint4 q = __ldg(base + v);
                if (STRIDE == 1)
                    c += (k0 >= ilo && (q.x >> sh) < t) + (k0 + 1 >= ilo && k0 + 1 < ihi && (q.y >> sh) < t) +
                         (k0 + 2 >= ilo && k0 + 2 < ihi && (q.z >> sh) < t) + (k0 + 3 < ihi && (q.w >> sh) < t);
                else
                    c += (k0 >= ilo && (q.x >> sh) < t) + (k0 + 1 < ihi && (q.z >> sh) < t);
            }
        }
    }
    return c;
}

// Count of a list's search keys (the skip index's posts for raw lists, block
// anchors for compressed lists; sorted) that lie below t after a right shift
// by sh: an NT-ary search by the group.  Each round the NT threads probe
// evenly spaced keys and count those below t (a prefix, the keys being
// sorted), which leaves one gap of the spacing; with NT = 32 a list of 10^4
// keys takes three rounds.  Over a skip index the probing stops once the
// range fits one vector round (post_count), which ends the search.  Every
// thread of the group gets the same answer.  A search from a merge position
// j passes lo0 = L.key_lo(j) and counts the keys from there on (the keys
// before lo0 lie before j); the merge then resumes at the larger of j and
// L.start_of(answer).
template <class Scope, uint32_t NT, class ListT>
__device__ __forceinline__ uint32_t start_search(const ListT &L, uint32_t sh, uint32_t t, uint32_t tid,
                                                 uint32_t lo0 = 0) {
    constexpr uint32_t PER = 4 / ListT::kKeyStride;  // keys per 16-byte load
    constexpr uint32_t LIMIT = PER * NT * kPostVec - (PER - 1);
    uint32_t lo = lo0, hi = L.keys_n();  // the answer lies in [lo, hi]
    while (hi - lo > LIMIT) {
        const uint32_t step = (hi - lo + NT - 1) / NT;
        const uint32_t q = lo + (tid + 1) * step - 1;
        const bool below = q < hi && (L.key(q) >> sh) < t;
        const uint32_t c = Scope::count(below);
        // c below-probes leave the gap after the c-th probe, if that probe
        // exists (c < probes in [lo, hi)), else the tail after the last one
        if (lo + (c + 1) * step <= hi) hi = lo + (c + 1) * step - 1;
        lo += c * step;
    }
    lo += Scope::sum(post_count<ListT::kKeyStride>(L.keys(), lo, hi, sh, t, tid, NT));
    return lo;
}

// Any overlap between lists X and Y, by a group of NT threads (thread
// index tid) with shared buffers xb, yb of WMAX + 2 intervals each (16-byte
// aligned) and, for a CTA group, one shared word `slot`.  The first window
// holds w0 intervals per list (a multiple of NT); later windows double up to
// WMAX.  Every thread of the group must call it with the same arguments.
// For raw lists the window is staged by two bulk copies issued by thread 0
// and completed on the mbarrier `bar` (phase bit in *phase, flipped per
// window); a wait that runs out sets *timeout and ends the join.  A join
// handed over at merge position (ri, rj) of an earlier run (resume) starts
// there, without a search.
template <class Scope, uint32_t NT, uint32_t WMAX, class ListT, int PRED = kOverlap>
__device__ __noinline__ bool tile_join(const ListT X, const ListT Y, uint2 *xb, uint2 *yb, uint32_t *slot,
                                       uint32_t tid, uint32_t w0, uint32_t bar, uint32_t *phase, bool *timeout,
                                       uint32_t sx = 0, uint32_t sy = 0, bool resume = false, uint32_t ri = 0,
                                       uint32_t rj = 0) {
    const uint32_t n = X.n, m = Y.n;
    if (PRED == kContain && n > 0 && m == 0) return true;  // nothing can contain X
    uint32_t i0 = resume ? ri : 0u, j0 = resume ? rj : 0u, w = w0;
    // Start each list at (or, for compressed lists, at a block boundary
    // before) its first interval that can meet the other one: an interval of
    // Y ending before X's first start meets no interval of X (nor contains
    // one), and likewise for X against Y's first start.  The merge from
    // (0, 0) would pass over those intervals, and a merge started anywhere
    // before the first interval that can meet finds the same overlaps, so the
    // verdict is unchanged; only lists longer than a window search.  `need`
    // names the lists to search before the next window (bit 0: X, against
    // target tx; bit 1: Y, against ty).
    uint32_t need = 0, tx = 0, ty = 0;
    if (!resume && n && m && (n > w0 || m > w0)) {
        tx = Y.first_start() >> sy;
        ty = X.first_start() >> sx;
        if (PRED == kOverlap) {
            need = n > w0 ? 1u : 0u;
        } else {
            static_assert(PRED == kOverlap || ListT::kRandomAccess, "containment joins read raw lists");
            if constexpr (ListT::kRandomAccess)
                if (((__ldg(&X.p->y) - 1u) >> sx) < tx) return true;  // X's first interval ends before Y starts
        }
        if (m > w0) need |= 2u;
    }
    while (i0 < n && j0 < m) {
        // the searches, one call site for both lists (the group agrees on need)
#pragma unroll 1
        while (need) {
            const bool sideY = !(need & 1u);
            need &= need - 1u;
            const ListT L = sideY ? Y : X;
            const uint32_t pos = sideY ? j0 : i0;
            const uint32_t c = start_search<Scope, NT>(L, sideY ? sy : sx, sideY ? ty : tx, tid, L.key_lo(pos));
            const uint32_t at = max(pos, L.start_of(c));
            if (sideY) j0 = at;
            else i0 = at;
        }
        if (i0 >= n || j0 >= m) break;
        const uint32_t nx = min(w, n - i0), ny = min(w, m - j0);
        uint32_t xa, ya;
        if constexpr (ListT::kBulk) {
            if (tid == 0) {
                fence_proxy_async();
                const uint2 *a;
                uint32_t bx, by, ox, oy;
                bulk_span(X.p + i0, nx, a, bx, ox);
                bulk_span(Y.p + j0, ny, a, by, oy);
                mbar_arrive_expect_tx(bar, bx + by);
                X.issue(xb, i0, nx, bar);
                Y.issue(yb, j0, ny, bar);
            }
            const bool ok = Scope::all(mbar_wait(bar, *phase));
            if (!ok) {  // give up, once this window's copies have landed (bounded)
                mbar_drain(bar, *phase);
                *phase ^= 1u;
                *timeout = true;
                return false;
            }
            *phase ^= 1u;
            xa = X.window(xb, i0);
            ya = Y.window(yb, j0);
        } else {
            xa = X.template stage<NT>(xb, i0, nx, tid, kFull);
            ya = Y.template stage<NT>(yb, j0, ny, tid, kFull);
            cp_async_wait_all();
            Scope::sync();
        }
        if (sx | sy) {
            if (sx) coarsen_window<NT>(xa, nx, sx, tid);
            if (sy) coarsen_window<NT>(ya, ny, sy, tid);
            Scope::sync();
        }
        // D diagonals of the merge path lie in this window; thread tid walks
        // [d0, d0 + per).  No list can run out inside a full window.
        const uint32_t D = min(w, nx + ny);
        const uint32_t per = w / NT;                          // a power of two
        const uint32_t owner = (D - 1) >> (__ffs(per) - 1);  // walks the window's last diagonal
        uint32_t state;
        const bool found = window_walk<WMAX / NT, PRED>(xa, nx, ya, ny, w, D, per, tid * per, state);
        // the starts of the window's first intervals, read before the vote
        // (after it the next window may overwrite the buffers)
        const uint32_t xs0 = PRED == kOverlap ? lds1(xa) : 0u, ys0 = PRED == kOverlap ? lds1(ya) : 0u;
        if (Scope::vote(found, state, owner, slot)) return true;
        if (D == nx + ny || state == 0xffffffffu) return false;  // a list ran out (violations were seen in the walk)
        i0 += state;
        j0 += D - state;
        w = min(w * 2u, WMAX);
        if constexpr (PRED == kOverlap) {
            // Galloping: a window that advanced one list only (its every
            // interval ended before the other list's current one starts) is
            // likely followed by more of the same, as where a list of a few
            // intervals meets one of 10^5.  The lagging list then searches
            // from its merge position for its first interval that ends at or
            // after the other's current start; the ones it skips meet nothing
            // (the same argument as the start search), and a merge resumed
            // before the first that can meet finds the same overlaps.
            if (state == 0 && m - j0 > w) {
                need = 2u;
                ty = xs0;
            } else if (state == D && n - i0 > w) {
                need = 1u;
                tx = ys0;
            }
        }
    }
    return PRED == kContain && i0 < n;  // Y ended before X: the rest of X has no container
}

}  // namespace april_dev
