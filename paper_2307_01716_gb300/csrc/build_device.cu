// GPU construction of APRIL approximations: polygons in device memory in,
// a device image of their A- and F-lists (the layout the filter reads) out.
//
// The cells and lists are exactly the host builder's (build_sets.cpp): both
// take their arithmetic from geom.h, and the lists are canonical (maximal
// intervals of the A and F cell sets, Sec. 4.1), so the two agree list for
// list.  The steps follow the host builder (and Sec. 6):
//   count  (k_bcount, one warp per polygon): MBR, cell window, the number of
//          touched-cell incidences T (cells an edge meets, per edge) and of
//          centre-line incidences (rows an edge crosses at their centre);
//   scan   (k_bscan): per-polygon offsets into the work and image regions;
//          the host reads the totals once;
//   emit   (k_bemit, one CTA per polygon, persistent): every edge writes its
//          touched cells as keys (polygon << 33 | Hilbert id << 1 | crossed),
//          the crossed flag saying whether the edge enters the cell's open
//          square;
//   sort   (k_rs_*): one stable LSD radix sort of all keys of all polygons
//          (8-bit digits, the passes the key width needs), so that every
//          polygon's keys end up sorted in its own range;
//   build  (k_bconstruct, one CTA per polygon, persistent):
//     2. the sorted keys are reduced to one key per cell (crossed if any
//        edge crossed it);
//     3. the sorted crossings of every cell row's centre line (k_bemit writes
//        one key per edge and row it crosses: polygon, row, floor of the
//        crossing's x; the same radix sort orders them) give each row's
//        crossing list;
//     4. one point-in-polygon test at the first cell of every gap between
//        consecutive touched ids (a gap is wholly inside or outside: Sec.
//        6.2) and at every touched cell no edge crosses (Full when its
//        centre is inside): the parity of the row's crossings right of the
//        centre, by binary search;
//     5. the A- and F-intervals come out of block scans over the cells:
//        an A interval breaks at a non-empty gap outside the polygon, an F
//        interval runs over consecutive Full gaps and cells.
// Each polygon's lists go to a slot range sized from T (|A| <= T and
// |F| <= T + 1), so no second pass is needed; unused slots stay unused.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "april_internal.h"
#include "geom.h"

using april::fail;
using namespace april_geom;

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr unsigned kBB = 256;  // build CTA size
constexpr unsigned kBW = kBB / 32;

struct GridP {
    int64_t ox, oy, h, G;
    uint32_t order;
};

// Per polygon, written by k_bcount and k_bscan.
struct PolyMeta {
    uint64_t key_off;   // into the key and temp arrays (keys)
    uint64_t rb_off;    // into the row-start array (uint32, rows + 1)
    uint64_t cross_off; // into the crossing-key arrays (keys)
    uint64_t slot_off;  // into the image's interval slots
    uint32_t T;         // touched-cell incidences
    uint32_t inc;       // centre-line incidences
    int32_t wi0, wj0, wi1, wj1;
    int32_t mbr[4];
    uint32_t err;       // 0 ok; 1 fewer than 3 vertices; 2 outside the grid; 3 too large; 4 meets no cell
    uint32_t pad;
};

struct Totals {
    unsigned long long keys, rb, slots, cross;
    unsigned int n_err, first_err;
    unsigned int err_code, pad;
    unsigned int ctr_emit, ctr_build, ctr_cells, pad2;  // persistent kernels' polygon counters
};

// Crossing keys: polygon << 42 | (row - wj0) << 26 | (floor(x) - xmn), the x
// of an edge's crossing with the row's centre line (26 bits cover the
// lattice square and its margins).
constexpr uint32_t kCrossXBits = 26, kCrossRowBits = 16, kCrossPolyShift = kCrossXBits + kCrossRowBits;

__device__ __forceinline__ uint64_t even_up(uint64_t v) { return (v + 1) & ~1ull; }

__device__ __forceinline__ int2 vtx(const int2 *xy, uint64_t b, uint64_t nv, uint64_t k) {
    return xy[b + (k == nv ? 0 : k)];
}

// ------------------------------------------------------------------ count
__global__ void __launch_bounds__(256) k_bcount(const int2 *__restrict__ xy, const uint64_t *__restrict__ off,
                                                uint32_t n, GridP g, PolyMeta *meta, Totals *tot) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nw = gridDim.x * (blockDim.x / 32);
    for (uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nw) {
        const uint64_t b = off[p], e = off[p + 1];
        uint32_t err = 0;
        const uint64_t nv = e >= b ? e - b : 0;
        if (e < b || nv < 3) err = 1;
        int64_t xmn = INT64_MAX, ymn = INT64_MAX, xmx = INT64_MIN, ymx = INT64_MIN;
        if (!err)
            for (uint64_t k = lane; k < nv; k += 32) {
                const int2 v = xy[b + k];
                xmn = imin(xmn, v.x), xmx = imax(xmx, v.x), ymn = imin(ymn, v.y), ymx = imax(ymx, v.y);
            }
        for (int o = 16; o; o >>= 1) {
            xmn = imin(xmn, __shfl_xor_sync(kFull, xmn, o));
            ymn = imin(ymn, __shfl_xor_sync(kFull, ymn, o));
            xmx = imax(xmx, __shfl_xor_sync(kFull, xmx, o));
            ymx = imax(ymx, __shfl_xor_sync(kFull, ymx, o));
        }
        int64_t wi0 = 0, wj0 = 0, wi1 = -1, wj1 = -1;
        if (!err) {
            cell_window(xmn, ymn, xmx, ymx, g.ox, g.oy, g.h, g.G, wi0, wj0, wi1, wj1);
            if (wi0 > wi1 || wj0 > wj1) err = 2;
        }
        unsigned long long inc = 0;
        if (!err)
            for (uint64_t k = lane; k < nv; k += 32) {
                const int2 a = vtx(xy, b, nv, k), c = vtx(xy, b, nv, k + 1);
                int64_t r0, r1;
                centre_rows(edge_up(a.x, a.y, c.x, c.y), g.oy, g.h, wj0, wj1, r0, r1);
                if (r1 >= r0) inc += (unsigned long long)(r1 - r0 + 1);
            }
        for (int o = 16; o; o >>= 1) inc += __shfl_xor_sync(kFull, inc, o);
        if (!err && (inc > 0x7FFFFFFFull || xmx - xmn >= (1ll << kCrossXBits))) err = 3;
        if (lane == 0) {
            PolyMeta m{};
            m.T = 0;  // counted by k_bcells
            m.inc = err ? 0u : (uint32_t)inc;
            m.wi0 = (int32_t)wi0, m.wj0 = (int32_t)wj0, m.wi1 = (int32_t)wi1, m.wj1 = (int32_t)wj1;
            m.mbr[0] = (int32_t)xmn, m.mbr[1] = (int32_t)ymn, m.mbr[2] = (int32_t)xmx, m.mbr[3] = (int32_t)ymx;
            m.err = err;
            meta[p] = m;
            if (err) {
                atomicAdd(&tot->n_err, 1u);
                if (atomicMin(&tot->first_err, p) > p) atomicExch(&tot->err_code, err);
            }
        }
    }
}

// ------------------------------------------------------------------- scan
// Exclusive offsets of keys (T), row starts (rows + 1), slots
// (2 even(T + 1): |A| <= max(T, 1) and |F| <= T + 1) and crossing keys (inc)
// over the polygons, by one CTA in contiguous chunks.
constexpr unsigned kScanT = 1024;
__global__ void __launch_bounds__(kScanT) k_bscan(PolyMeta *meta, uint32_t n, Totals *tot) {
    __shared__ unsigned long long s_w[4][kScanT / 32];
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t chunk = (n + kScanT - 1) / kScanT;
    const uint32_t b = min(n, t * chunk), e = min(n, b + chunk);
    unsigned long long s[4] = {0, 0, 0, 0};
    auto amounts = [&](const PolyMeta &m, unsigned long long *a) {
        const unsigned long long rows = m.err ? 0 : (unsigned long long)(m.wj1 - m.wj0 + 1);
        a[0] = m.T;
        a[1] = m.err ? 0 : rows + 1;
        a[2] = 2 * even_up((uint64_t)m.T + 1);
        a[3] = m.inc;
    };
    for (uint32_t k = b; k < e; ++k) {
        unsigned long long a[4];
        amounts(meta[k], a);
        s[0] += a[0], s[1] += a[1], s[2] += a[2], s[3] += a[3];
    }
    unsigned long long incl[4];
    for (int f = 0; f < 4; ++f) {
        incl[f] = s[f];
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const unsigned long long v = __shfl_up_sync(kFull, incl[f], d);
            if (lane >= d) incl[f] += v;
        }
        if (lane == 31) s_w[f][warp] = incl[f];
    }
    __syncthreads();
    if (warp == 0)
        for (int f = 0; f < 4; ++f) {
            unsigned long long w = s_w[f][lane];
            for (uint32_t d = 1; d < 32; d <<= 1) {
                const unsigned long long v = __shfl_up_sync(kFull, w, d);
                if (lane >= d) w += v;
            }
            s_w[f][lane] = w;
        }
    __syncthreads();
    unsigned long long run[4];
    for (int f = 0; f < 4; ++f) run[f] = incl[f] - s[f] + (warp ? s_w[f][warp - 1] : 0ull);
    for (uint32_t k = b; k < e; ++k) {
        unsigned long long a[4];
        amounts(meta[k], a);
        meta[k].key_off = run[0];
        meta[k].rb_off = run[1];
        meta[k].slot_off = run[2];
        meta[k].cross_off = run[3];
        run[0] += a[0], run[1] += a[1], run[2] += a[2], run[3] += a[3];
    }
    if (t == kScanT - 1) {
        tot->keys = s_w[0][31];
        tot->rb = s_w[1][31];
        tot->slots = s_w[2][31];
        tot->cross = s_w[3][31];
    }
}

// ------------------------------------------------------------ CTA helpers
struct BuildShared {
    uint32_t warp_sum[kBW];
    uint32_t item;
    uint32_t k_count;
};

// Exclusive scan of one value per thread over the CTA; *total gets the sum.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t &total, BuildShared &sh) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh.warp_sum[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (uint32_t w = 0; w < kBW; ++w) {
        if (w < warp) before += sh.warp_sum[w];
        all += sh.warp_sum[w];
    }
    __syncthreads();
    total = all;
    return before + x - v;
}


// Point-in-polygon at the centre of cell (i, j), the host builder's rule: an
// upward edge toggles when the centre is strictly left of it, i.e. when its
// crossing x is greater than the centre's.  The centre is never on the
// boundary here (it lies in the open square of a cell the boundary does not
// enter), so x > xc is floor(x) >= xc, and the parity of the row's sorted
// crossings at or right of xc decides.  Cells outside the window are outside.
__device__ bool inside_cell(uint32_t i, uint32_t j, const PolyMeta &M, const GridP &g, const uint32_t *row_start,
                            const unsigned long long *cross) {
    if ((int64_t)i < M.wi0 || (int64_t)i > M.wi1 || (int64_t)j < M.wj0 || (int64_t)j > M.wj1) return false;
    const int64_t xc = g.ox + (int64_t)i * g.h + g.h / 2;
    const uint32_t r = j - (uint32_t)M.wj0;
    uint32_t lo = row_start[r];
    const uint32_t hi = row_start[r + 1];
    const int64_t xr = xc - M.mbr[0];
    if (xr > 0) {
        const unsigned long long xk = (unsigned long long)imin(xr, (1ll << kCrossXBits) - 1);
        uint32_t h2 = hi;
        while (lo < h2) {  // first crossing with floor(x) - xmn >= xc - xmn
            const uint32_t mid = (lo + h2) >> 1;
            if ((cross[mid] & ((1ull << kCrossXBits) - 1)) < xk) lo = mid + 1;
            else h2 = mid;
        }
    }
    return ((hi - lo) & 1u) != 0;
}

// ------------------------------------------------- (edge, row) work items
// The closed strips of cell rows an edge meets, flattened over a polygon's
// edges so that the CTA's threads share them evenly whatever the edges'
// lengths.  Edges are taken kChunkE at a time; for a chunk, pre[e] is the
// number of items before local edge e and j0[e] its first row.
constexpr uint32_t kChunkE = 1024;
struct EdgeChunk {
    uint32_t pre[kChunkE + 1];
    int32_t j0[kChunkE];
};

// Fills the chunk of edges [e_base, e_base + ne) and returns its item count.
__device__ uint32_t load_chunk(const int2 *xy, uint64_t b, uint64_t nv, uint64_t e_base, uint32_t ne, const GridP &g,
                               EdgeChunk &ch, BuildShared &sh) {
    constexpr uint32_t per = kChunkE / kBB;
    uint32_t cnt[per], sum = 0;
    for (uint32_t q = 0; q < per; ++q) {
        const uint32_t e = threadIdx.x * per + q;
        cnt[q] = 0;
        if (e < ne) {
            const int2 a = vtx(xy, b, nv, e_base + e), c = vtx(xy, b, nv, e_base + e + 1);
            int64_t j0, j1;
            edge_rows(edge_up(a.x, a.y, c.x, c.y), g.oy, g.h, g.G, j0, j1);
            ch.j0[e] = (int32_t)j0;
            cnt[q] = j1 >= j0 ? (uint32_t)(j1 - j0 + 1) : 0u;
        }
        sum += cnt[q];
    }
    uint32_t total;
    uint32_t run = block_scan(sum, total, sh);
    for (uint32_t q = 0; q < per; ++q) {
        const uint32_t e = threadIdx.x * per + q;
        if (e < kChunkE) ch.pre[e] = run;
        run += cnt[q];
    }
    if (threadIdx.x == 0) ch.pre[kChunkE] = total;
    __syncthreads();
    return total;
}

// The local edge of item q (the last e with pre[e] <= q) and its row.
__device__ __forceinline__ uint32_t item_edge(const EdgeChunk &ch, uint32_t ne, uint32_t q, int64_t &j) {
    uint32_t lo = 0, hi = ne - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (ch.pre[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    j = ch.j0[lo] + (int64_t)(q - ch.pre[lo]);
    return lo;
}

// Touched-cell incidences T of every polygon (one CTA per polygon); a
// polygon no edge touches holds the whole grid or misses it, which the
// centre of cell (0, 0) tells (crossing parity).
__global__ void __launch_bounds__(kBB) k_bcells(const int2 *__restrict__ xy, const uint64_t *__restrict__ off,
                                                uint32_t n, GridP g, PolyMeta *meta, Totals *tot, uint32_t *counter) {
    __shared__ BuildShared sh;
    __shared__ EdgeChunk ch;
    __shared__ unsigned long long s_red[kBW];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (;;) {
        if (tid == 0) sh.item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t p = sh.item;
        __syncthreads();
        if (p >= n) break;
        if (meta[p].err) continue;
        const uint64_t b = off[p], nv = off[p + 1] - b;
        unsigned long long T = 0;
        uint32_t par = 0;
        for (uint64_t e_base = 0; e_base < nv; e_base += kChunkE) {
            const uint32_t ne = (uint32_t)min((uint64_t)kChunkE, nv - e_base);
            const uint32_t R = load_chunk(xy, b, nv, e_base, ne, g, ch, sh);
            for (uint32_t q = tid; q < R; q += kBB) {
                int64_t j;
                const uint32_t e = item_edge(ch, ne, q, j);
                const int2 a = vtx(xy, b, nv, e_base + e), c = vtx(xy, b, nv, e_base + e + 1);
                int64_t i0, i1;
                if (edge_cells_in_row(edge_up(a.x, a.y, c.x, c.y), g.ox, g.oy, g.h, g.G, j, i0, i1))
                    T += (unsigned long long)(i1 - i0 + 1);
            }
            __syncthreads();
        }
        for (int o = 16; o; o >>= 1) T += __shfl_xor_sync(kFull, T, o);
        if (lane == 0) s_red[warp] = T;
        __syncthreads();
        T = 0;
        for (uint32_t w = 0; w < kBW; ++w) T += s_red[w];
        __syncthreads();
        uint32_t err = T > 0x7FFFFFFFull ? 3u : 0u;
        if (T == 0) {
            const int64_t xc = g.ox + g.h / 2, yc = g.oy + g.h / 2;
            for (uint64_t k = tid; k < nv; k += kBB) {
                const int2 a = vtx(xy, b, nv, k), c = vtx(xy, b, nv, k + 1);
                const EdgeUp ed = edge_up(a.x, a.y, c.x, c.y);
                if (ed.ay <= yc && yc < ed.by && turn(ed.ax, ed.ay, ed.bx, ed.by, xc, yc) > 0) par ^= 1u;
            }
            for (int o = 16; o; o >>= 1) par ^= __shfl_xor_sync(kFull, par, o);
            if (lane == 0) s_red[warp] = par;
            __syncthreads();
            par = 0;
            for (uint32_t w = 0; w < kBW; ++w) par ^= (uint32_t)s_red[w];
            __syncthreads();
            if (!par) err = 4;
        }
        if (tid == 0) {
            meta[p].T = err ? 0u : (uint32_t)T;
            if (err) {
                meta[p].err = err;
                atomicAdd(&tot->n_err, 1u);
                if (atomicMin(&tot->first_err, p) > p) atomicExch(&tot->err_code, err);
            }
        }
    }
}

// ------------------------------------------------------------------- sort
// Stable LSD radix sort of N 64-bit keys, 8 bits per pass.  A tile is 4096
// keys (256 threads x 16); per pass: k_rs_hist counts every tile's digits
// (digit-major table), k_rs_rows turns each digit's row into exclusive tile
// offsets and k_rs_digits the digit totals into digit bases, and
// k_rs_scatter moves every key to its digit base + tile offset + rank,
// ranking a tile's keys in order: 16 slices of 256, each ranked within its
// warp by match_any and across warps by per-warp digit counts.
constexpr unsigned kRsT = 256, kRsItems = 16, kRsTile = kRsT * kRsItems;

__global__ void __launch_bounds__(kRsT) k_rs_hist(const unsigned long long *__restrict__ src, uint64_t N,
                                                  uint32_t shift, uint32_t *hist, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    const uint32_t tid = threadIdx.x;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        h[tid] = 0;
        __syncthreads();
        for (uint32_t i = 0; i < kRsItems; ++i) {
            const uint64_t idx = (uint64_t)tile * kRsTile + i * kRsT + tid;
            if (idx < N) atomicAdd(&h[(uint32_t)(src[idx] >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[(uint64_t)tid * ntiles + tile] = h[tid];
        __syncthreads();
    }
}

constexpr unsigned kRsScanT = 1024;
__global__ void __launch_bounds__(kRsScanT) k_rs_rows(uint32_t *hist, uint32_t ntiles, uint32_t *totals) {
    __shared__ uint32_t s_w[kRsScanT / 32];
    uint32_t *row = hist + (uint64_t)blockIdx.x * ntiles;
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t chunk = (ntiles + kRsScanT - 1) / kRsScanT;
    const uint32_t b = min(ntiles, t * chunk), e = min(ntiles, b + chunk);
    uint32_t sum = 0;
    for (uint32_t k = b; k < e; ++k) sum += row[k];
    uint32_t incl = sum;
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_w[lane];
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, w, d);
            if (lane >= d) w += v;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    uint32_t run = incl - sum + (warp ? s_w[warp - 1] : 0u);
    for (uint32_t k = b; k < e; ++k) {
        const uint32_t c = row[k];
        row[k] = run;
        run += c;
    }
    if (t == kRsScanT - 1) totals[blockIdx.x] = s_w[31];
}

__global__ void __launch_bounds__(256) k_rs_digits(uint32_t *totals) {
    __shared__ uint32_t v[256];
    const uint32_t t = threadIdx.x;
    v[t] = totals[t];
    __syncthreads();
    if (t == 0) {
        uint32_t run = 0;
        for (int d = 0; d < 256; ++d) {
            const uint32_t c = v[d];
            v[d] = run;
            run += c;
        }
    }
    __syncthreads();
    totals[t] = v[t];
}

__global__ void __launch_bounds__(kRsT) k_rs_scatter(const unsigned long long *__restrict__ src,
                                                     unsigned long long *__restrict__ dst, uint64_t N, uint32_t shift,
                                                     const uint32_t *__restrict__ hist,
                                                     const uint32_t *__restrict__ dbase, uint32_t ntiles) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[kRsT / 32][256];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        run[tid] = dbase[tid] + hist[(uint64_t)tid * ntiles + tile];
        for (uint32_t w = 0; w < kRsT / 32; ++w) wc[w][tid] = 0;
        __syncthreads();
        for (uint32_t i = 0; i < kRsItems; ++i) {
            const uint64_t idx = (uint64_t)tile * kRsTile + i * kRsT + tid;
            const bool valid = idx < N;
            const unsigned long long key = valid ? src[idx] : 0ull;
            const uint32_t d = valid ? (uint32_t)(key >> shift) & 255u : 256u;
            const uint32_t peers = __match_any_sync(kFull, d);
            const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
            if (valid && rank == 0) wc[warp][d] = __popc(peers);
            __syncthreads();
            {  // thread tid: the start of every warp's keys of digit tid
                uint32_t r = run[tid];
                for (uint32_t w = 0; w < kRsT / 32; ++w) {
                    const uint32_t c = wc[w][tid];
                    wc[w][tid] = r;
                    r += c;
                }
                run[tid] = r;
            }
            __syncthreads();
            if (valid) dst[wc[warp][d] + rank] = key;
            __syncthreads();
            for (uint32_t w = 0; w < kRsT / 32; ++w) wc[w][tid] = 0;
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------- emit
constexpr uint32_t kKeyBits = 33;  // Hilbert id (32 bits at order 16) << 1 | crossed
__global__ void __launch_bounds__(kBB) k_bemit(const int2 *__restrict__ xy, const uint64_t *__restrict__ off,
                                               uint32_t n, GridP g, const PolyMeta *__restrict__ meta,
                                               unsigned long long *keys_all, unsigned long long *cross_all,
                                               uint32_t *counter) {
    __shared__ BuildShared sh;
    __shared__ EdgeChunk ch;
    const uint32_t tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh.item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t p = sh.item;
        __syncthreads();
        if (p >= n) break;
        const PolyMeta M = meta[p];
        const uint64_t b = off[p], nv = off[p + 1] - b;
        const uint32_t T = M.T;  // a polygon with no touched cell still writes its crossings
        unsigned long long *keys = keys_all + M.key_off, *cross = cross_all + M.cross_off;
        const unsigned long long tag = (unsigned long long)p << kKeyBits;
        const unsigned long long ctag = (unsigned long long)p << kCrossPolyShift;
        uint32_t carry = 0, ccarry = 0;
        for (uint64_t e_base = 0; e_base < nv; e_base += kChunkE) {
            const uint32_t ne = (uint32_t)min((uint64_t)kChunkE, nv - e_base);
            const uint32_t R = load_chunk(xy, b, nv, e_base, ne, g, ch, sh);
            for (uint32_t q0 = 0; q0 < R; q0 += kBB) {
                const uint32_t q = q0 + tid;
                EdgeUp ed{0, 0, 0, 0};
                int64_t j = 0, i0 = 0, i1 = -1, r0 = 0, r1 = -1;
                if (q < R) {
                    const uint32_t e = item_edge(ch, ne, q, j);
                    const int2 a = vtx(xy, b, nv, e_base + e), c = vtx(xy, b, nv, e_base + e + 1);
                    ed = edge_up(a.x, a.y, c.x, c.y);
                    if (!edge_cells_in_row(ed, g.ox, g.oy, g.h, g.G, j, i0, i1)) i1 = i0 - 1;
                    centre_rows(ed, g.oy, g.h, M.wj0, M.wj1, r0, r1);
                }
                const bool crosses = q < R && j >= r0 && j <= r1;  // the edge crosses row j's centre line
                uint32_t total, ctotal;
                uint32_t pos = carry + block_scan(i1 >= i0 ? (uint32_t)(i1 - i0 + 1) : 0u, total, sh);
                const uint32_t cpos = ccarry + block_scan(crosses ? 1u : 0u, ctotal, sh);
                carry += total;
                ccarry += ctotal;
                const int64_t Y0 = g.oy + j * g.h;
                for (int64_t i = i0; i <= i1; ++i) {
                    const bool crossed = enters_open_square(ed.ax, ed.ay, ed.bx, ed.by, g.ox + i * g.h, Y0, g.h);
                    const unsigned long long key =
                        tag | (hilbert_id(g.order, (uint32_t)i, (uint32_t)j) << 1) | (crossed ? 1ull : 0ull);
                    if (pos < T) keys[pos] = key;
                    ++pos;
                }
                if (crosses && cpos < M.inc) {
                    const int64_t yc = Y0 + g.h / 2, den = ed.by - ed.ay;
                    const int64_t xf = floor_div(ed.ax * den + (yc - ed.ay) * (ed.bx - ed.ax), den);
                    cross[cpos] = ctag | ((unsigned long long)(j - M.wj0) << kCrossXBits) |
                                  (unsigned long long)(xf - M.mbr[0]);
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ build
__global__ void __launch_bounds__(kBB) k_bconstruct(const int2 *__restrict__ xy, const uint64_t *__restrict__ off,
                                                    uint32_t n, GridP g, const PolyMeta *__restrict__ meta,
                                                    const unsigned long long *sorted_all, unsigned long long *other_all,
                                                    const unsigned long long *cross_all, uint8_t *flags_all,
                                                    uint32_t *rb_all, uint32_t *desc_out,
                                                    int4 *mbr_out, uint2 *iv_out, uint32_t *counter) {
    __shared__ BuildShared sh;
    const uint32_t tid = threadIdx.x;
    const uint64_t ncells = (uint64_t)g.G * (uint64_t)g.G;
    const unsigned long long kmask = (1ull << kKeyBits) - 1ull;
    for (;;) {
        if (tid == 0) sh.item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t p = sh.item;
        __syncthreads();
        if (p >= n) break;
        const PolyMeta M = meta[p];
        const uint32_t T = M.T;
        const unsigned long long *sorted = sorted_all + M.key_off;
        unsigned long long *U = other_all + M.key_off;
        uint8_t *flags = flags_all + M.key_off;
        const uint32_t rows = (uint32_t)(M.wj1 - M.wj0 + 1);
        uint32_t *row_start = rb_all + M.rb_off;
        const unsigned long long *cross = cross_all + M.cross_off;
        if (tid == 0) mbr_out[p] = make_int4(M.mbr[0], M.mbr[1], M.mbr[2], M.mbr[3]);
        if (T == 0) {  // the polygon holds the whole grid (the count pass checked)
            if (tid == 0) {
                uint2 *lists = iv_out + M.slot_off;
                lists[0] = make_uint2(0u, (uint32_t)ncells);  // 2^32 wraps to 0 by design
                lists[2] = make_uint2(0u, (uint32_t)ncells);
                uint32_t *dsc = desc_out + 4 * (size_t)p;
                dsc[0] = (uint32_t)M.slot_off, dsc[1] = 1u, dsc[2] = (uint32_t)(M.slot_off + 2), dsc[3] = 1u;
            }
            continue;
        }

        // 2. one key per cell (the last of a cell's run carries the crossed
        //    flag when any edge crossed it: (d << 1) | 1 sorts last)
        uint32_t carry = 0;
        for (uint32_t t0 = 0; t0 < T; t0 += kBB) {
            const uint32_t k = t0 + tid;
            bool last = false;
            unsigned long long key = 0;
            if (k < T) {
                key = sorted[k] & kmask;
                last = k + 1 == T || ((sorted[k + 1] & kmask) >> 1) != (key >> 1);
            }
            uint32_t total;
            const uint32_t pos = carry + block_scan(last ? 1u : 0u, total, sh);
            if (last) U[pos] = key;
            carry += total;
        }
        const uint32_t K = carry;

        // 3. row starts in the sorted crossings: row r's crossings are
        //    [row_start[r], row_start[r + 1]); every entry is written once, by
        //    the crossing that opens its row or the one that closes the list
        const uint32_t inc = M.inc;
        const unsigned long long rmask = (1ull << kCrossRowBits) - 1;
        if (inc == 0)
            for (uint32_t r = tid; r <= rows; r += kBB) row_start[r] = 0;
        for (uint32_t q = tid; q < inc; q += kBB) {
            const uint32_t r = (uint32_t)((cross[q] >> kCrossXBits) & rmask);
            const uint32_t rp = q ? (uint32_t)((cross[q - 1] >> kCrossXBits) & rmask) + 1u : 0u;
            for (uint32_t rr = rp; rr <= r; ++rr) row_start[rr] = q;
            if (q + 1 == inc)
                for (uint32_t rr = r + 1; rr <= rows; ++rr) row_start[rr] = inc;
        }
        __syncthreads();

        // 4. classification: bit 0 gap before the cell non-empty, bit 1 that
        //    gap Full, bit 2 the cell Full
        for (uint32_t u = tid; u < K; u += kBB) {
            const unsigned long long key = U[u];
            const uint64_t d = key >> 1;
            const uint64_t first_gap = u ? (U[u - 1] >> 1) + 1 : 0;
            uint8_t f = 0;
            uint32_t x, y;
            if (d > first_gap) {
                f |= 1;
                hilbert_cell(g.order, first_gap, x, y);
                if (inside_cell(x, y, M, g, row_start, cross)) f |= 2;
            }
            if (!(key & 1ull)) {
                hilbert_cell(g.order, d, x, y);
                if (inside_cell(x, y, M, g, row_start, cross)) f |= 4;
            }
            flags[u] = f;
        }
        if (tid == 0) {
            const uint64_t nxt = (U[K - 1] >> 1) + 1;
            bool tail = false;
            if (nxt < ncells) {
                uint32_t x, y;
                hilbert_cell(g.order, nxt, x, y);
                tail = inside_cell(x, y, M, g, row_start, cross);
            }
            sh.k_count = tail ? 1u : 0u;
        }
        __syncthreads();
        const bool tailF = sh.k_count != 0;

        // 5. intervals
        uint2 *Aout = iv_out + M.slot_off;
        uint2 *Fout = iv_out + M.slot_off + even_up((uint64_t)T + 1);
        uint32_t na = 0, nf = 0;
        {
            // A: a new interval at every cell after a non-empty gap that is not Full
            uint32_t ca = 0, cf = 0;
            for (uint32_t t0 = 0; t0 < K; t0 += kBB) {
                const uint32_t u = t0 + tid;
                const bool ok = u < K;
                const uint8_t f = ok ? flags[u] : 0;
                const uint64_t d = ok ? (U[u] >> 1) : 0;
                const uint64_t prev_end = (ok && u) ? (U[u - 1] >> 1) + 1 : 0;  // end of the previous cell
                const bool brk = ok && u > 0 && (f & 1) && !(f & 2);
                uint32_t ta;
                const uint32_t ia = ca + block_scan(brk ? 1u : 0u, ta, sh);
                if (brk) {
                    Aout[ia].y = (uint32_t)prev_end;  // the interval before closes
                    Aout[ia + 1].x = (uint32_t)d;
                }
                if (ok && u == 0) Aout[0].x = ((f & 1) && (f & 2)) ? 0u : (uint32_t)d;
                ca += ta;
                // F: slots gap(u) then cell(u); a run starts where an F slot
                // follows a non-F one and ends where a non-F one follows
                const bool gF = ok && (f & 2);
                const bool cF = ok && (f & 4);
                const bool prevCellF = ok && u > 0 && (flags[u - 1] & 4);
                const bool prev_of_cell = (f & 1) ? gF : prevCellF;
                bool next_of_cell = tailF;
                if (ok && u + 1 < K) {
                    const uint8_t fn = flags[u + 1];
                    next_of_cell = (fn & 1) ? (fn & 2) != 0 : (fn & 4) != 0;
                }
                const bool sg = gF && !prevCellF, sc = cF && !prev_of_cell;
                const bool eg = gF && !cF, ec = cF && !next_of_cell;
                uint32_t tf;
                const uint32_t i0 = cf + block_scan((sg ? 1u : 0u) + (sc ? 1u : 0u), tf, sh);
                if (sg) Fout[i0].x = (uint32_t)prev_end;                     // gap starts after the previous cell
                if (eg) Fout[i0 + (sg ? 1u : 0u) - 1u].y = (uint32_t)d;        // and ends at this cell
                if (sc) Fout[i0 + (sg ? 1u : 0u)].x = (uint32_t)d;
                if (ec) Fout[i0 + (sg ? 1u : 0u) + (sc ? 1u : 0u) - 1u].y = (uint32_t)(d + 1);
                cf += tf;
            }
            na = ca + 1;
            nf = cf;
            if (tid == 0) {
                const uint64_t last_end = (U[K - 1] >> 1) + 1;
                Aout[na - 1].y = (uint32_t)(tailF ? ncells : last_end);  // 2^32 wraps to 0 by design
                const bool lastCellF = (flags[K - 1] & 4) != 0;
                if (tailF) {
                    if (!lastCellF) Fout[nf].x = (uint32_t)last_end;
                    Fout[lastCellF ? nf - 1 : nf].y = (uint32_t)ncells;
                }
            }
            if (tailF && !(flags[K - 1] & 4)) nf += 1;
        }
        if (tid == 0) {
            uint32_t *dsc = desc_out + 4 * (size_t)p;
            dsc[0] = (uint32_t)M.slot_off;
            dsc[1] = na;
            dsc[2] = (uint32_t)(M.slot_off + even_up((uint64_t)T + 1));
            dsc[3] = nf;
        }
        __syncthreads();
    }
}

april_status cuda_fail(cudaError_t e, const char *what) {
    return fail(APRIL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline uint64_t r256(uint64_t b) { return april_round256(b); }

struct WorkLayout {
    uint64_t totals, meta, keys, tmp, flags, rb, cross, ctmp, hist, dbase, total;
};

inline uint32_t sort_tiles(uint64_t keys) { return (uint32_t)((keys + kRsTile - 1) / kRsTile); }

WorkLayout work_layout(uint32_t n, uint64_t keys, uint64_t rb, uint64_t cross) {
    WorkLayout L{};
    uint64_t o = 0;
    L.totals = o;
    o += 256;
    L.meta = o;
    o += r256((uint64_t)n * sizeof(PolyMeta));
    const uint64_t min_total = o;
    L.keys = o;
    o += r256(keys * 8);
    L.tmp = o;
    o += r256(keys * 8);
    L.flags = o;
    o += r256(keys);
    L.rb = o;
    o += r256(rb * 4);
    L.cross = o;
    o += r256(cross * 8);
    L.ctmp = o;
    o += r256(cross * 8);
    L.hist = o;
    o += r256((uint64_t)256 * sort_tiles(std::max(keys, cross)) * 4);
    L.dbase = o;
    o += 1024;
    L.total = keys || rb ? o : min_total;
    return L;
}

}  // namespace

extern "C" april_status april_build_sets_device(april_ctx *ctx, const int32_t *d_xy, const uint64_t *d_vert_off,
                                                uint32_t n_polys, const april_grid *grid, void *d_work,
                                                size_t work_bytes, void *d_image, size_t image_bytes,
                                                april_dev_sets *out, april_device_build_info *info, void *stream) {
    if (!ctx || !info || !out) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    *info = april_device_build_info{};
    GridP g{};
    april_status st = april::check_grid_params(grid, g.ox, g.oy, g.h, g.order, g.G);
    if (st) return st;
    if (n_polys == 0) return fail(APRIL_ERR_INVALID_ARG, "no polygons");
    if (!d_xy || !d_vert_off) return fail(APRIL_ERR_INVALID_ARG, "NULL polygon arrays");
    if ((((uintptr_t)d_xy) & 7u) || (((uintptr_t)d_vert_off) & 7u))
        return fail(APRIL_ERR_INVALID_ARG, "polygon arrays must be 8-byte aligned");
    const WorkLayout L0 = work_layout(n_polys, 0, 0, 0);
    info->work_bytes = L0.total;
    if (!d_work || work_bytes < L0.total) return fail(APRIL_ERR_OVER_BUDGET, "work buffer below the counting size");
    if (((uintptr_t)d_work) & 255u) return fail(APRIL_ERR_INVALID_ARG, "work buffer must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char *work = (char *)d_work;
    auto *tot = (Totals *)(work + L0.totals);
    auto *meta = (PolyMeta *)(work + L0.meta);
    cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(Totals), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&tot->first_err, 0xFF, 4, s);
    const int sms = april_ctx_num_sms(ctx);
    const unsigned gcount = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(((uint64_t)n_polys * 32 + 255) / 256, (uint64_t)sms * 8));
    if (e == cudaSuccess) {
        k_bcount<<<gcount, 256, 0, s>>>((const int2 *)d_xy, d_vert_off, n_polys, g, meta, tot);
        int occc = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occc, k_bcells, kBB, 0);
        const unsigned gcells = (unsigned)std::max<uint64_t>(
            1, std::min<uint64_t>(n_polys, (uint64_t)sms * (uint64_t)std::max(occc, 1)));
        k_bcells<<<gcells, kBB, 0, s>>>((const int2 *)d_xy, d_vert_off, n_polys, g, meta, tot, &tot->ctr_cells);
        k_bscan<<<1, kScanT, 0, s>>>(meta, n_polys, tot);
        e = cudaGetLastError();
    }
    Totals h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "counting cells on the device");
    if (h.n_err) {
        char m[160];
        const char *why = h.err_code == 1   ? "fewer than 3 vertices (or offsets not monotone)"
                          : h.err_code == 2 ? "outside the grid"
                          : h.err_code == 4 ? "meets no cell"
                                            : "too large (2^31 cells, or an MBR 2^26 lattice units wide)";
        std::snprintf(m, sizeof m, "polygon %u: %s (%u polygons rejected)", h.first_err, why, h.n_err);
        return fail(h.err_code == 3 ? APRIL_ERR_INVALID_ARG : APRIL_ERR_GEOMETRY, m);
    }
    const WorkLayout L = work_layout(n_polys, h.keys, h.rb, h.cross);
    const uint64_t desc_b = r256((uint64_t)n_polys * 16), mbr_b = r256((uint64_t)n_polys * 16);
    const uint64_t iv_b = r256(h.slots * 8 + 16), posts_b = r256(april_posts_words(h.slots) * 4);
    const uint64_t img = desc_b + mbr_b + iv_b + posts_b;
    info->touched_cells = h.keys;
    info->work_bytes = L.total;
    info->image_bytes = img;
    info->iv_slots = h.slots;
    if (h.slots > 0xFFFFFFF0ull) return fail(APRIL_ERR_INVALID_ARG, "more than 2^32 interval slots in one set");
    if (h.keys > 0xFFFFFFFFull || h.cross > 0xFFFFFFFFull || n_polys > (1u << 22))
        return fail(APRIL_ERR_INVALID_ARG, "more than 2^32 - 1 cells or crossings, or 2^22 polygons, in one build");
    if (work_bytes < L.total) return fail(APRIL_ERR_OVER_BUDGET, "work buffer too small");
    if (!d_image || image_bytes < img) return fail(APRIL_ERR_OVER_BUDGET, "image buffer too small");
    if (((uintptr_t)d_image) & 255u) return fail(APRIL_ERR_INVALID_ARG, "image buffer must be 256-byte aligned");
    char *image = (char *)d_image;
    e = cudaMemsetAsync(&tot->ctr_emit, 0, 8, s);  // both polygon counters
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bconstruct, kBB, 0);
    const unsigned gbuild = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(n_polys, (uint64_t)sms * (uint64_t)std::max(occ, 1)));
    auto *keys = (unsigned long long *)(work + L.keys), *tmp = (unsigned long long *)(work + L.tmp);
    if (e == cudaSuccess) {
        k_bemit<<<gbuild, kBB, 0, s>>>((const int2 *)d_xy, d_vert_off, n_polys, g, meta, keys,
                                       (unsigned long long *)(work + L.cross), &tot->ctr_emit);
        e = cudaGetLastError();
    }
    // one radix sort of all cell keys (the polygon id sits above the 33 key
    // bits) and one of all crossing keys (above row and x)
    uint32_t pbits = 0;
    while (pbits < 32 && (1ull << pbits) < n_polys) ++pbits;
    auto *hist = (uint32_t *)(work + L.hist), *dbase = (uint32_t *)(work + L.dbase);
    auto radix_sort = [&](unsigned long long *a, unsigned long long *t, uint64_t N, uint32_t bits) {
        const uint32_t passes = (bits + 7) / 8, ntiles = sort_tiles(N);
        const unsigned gs = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ntiles, (uint64_t)sms * 8));
        for (uint32_t pass = 0; pass < passes && N && e == cudaSuccess; ++pass) {
            k_rs_hist<<<gs, kRsT, 0, s>>>(a, N, 8 * pass, hist, ntiles);
            k_rs_rows<<<256, kRsScanT, 0, s>>>(hist, ntiles, dbase);
            k_rs_digits<<<1, 256, 0, s>>>(dbase);
            k_rs_scatter<<<gs, kRsT, 0, s>>>(a, t, N, 8 * pass, hist, dbase, ntiles);
            e = cudaGetLastError();
            std::swap(a, t);
        }
        return a;  // the buffer holding the sorted keys
    };
    unsigned long long *src = radix_sort(keys, tmp, h.keys, kKeyBits + pbits);
    unsigned long long *dst = src == keys ? tmp : keys;
    const unsigned long long *csorted = radix_sort((unsigned long long *)(work + L.cross),
                                                   (unsigned long long *)(work + L.ctmp), h.cross,
                                                   kCrossPolyShift + pbits);
    if (e == cudaSuccess) {
        k_bconstruct<<<gbuild, kBB, 0, s>>>((const int2 *)d_xy, d_vert_off, n_polys, g, meta, src, dst, csorted,
                                            (uint8_t *)(work + L.flags), (uint32_t *)(work + L.rb), (uint32_t *)image,
                                            (int4 *)(image + desc_b), (uint2 *)(image + desc_b + mbr_b),
                                            &tot->ctr_build);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)  // the skip index of the interval array
        e = (cudaError_t)april_launch_posts((const uint32_t *)(image + desc_b + mbr_b), h.slots,
                                            (uint32_t *)(image + desc_b + mbr_b + iv_b), s);
    if (e != cudaSuccess) return cuda_fail(e, "building lists on the device");
    *out = april_dev_sets{};
    out->desc = (const uint32_t *)image;
    out->iv = (const uint32_t *)(image + desc_b + mbr_b);
    out->mbr = (const int32_t *)(image + desc_b);
    out->posts = (const uint32_t *)(image + desc_b + mbr_b + iv_b);
    out->n_objects = n_polys;
    out->order = g.order;
    out->iv_slots = h.slots;
    out->n_entries = n_polys;
    out->grid_ox = g.ox;
    out->grid_oy = g.oy;
    out->grid_log2_cell = grid->log2_cell;
    out->grid_known = 1;
    out->grid_id = april_grid_id(g.ox, g.oy, grid->log2_cell, g.order);
    return APRIL_OK;
}
