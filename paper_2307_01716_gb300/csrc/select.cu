// Selection queries with APRIL as the intermediate filter (Sec. 4.3.1).
//
// The data polygons R are resident: their APRIL lists (april_upload) and a
// bucket index over their MBRs (built here on the host, uploaded once).  A
// batch of query polygons Q arrives with its own APRIL lists; one call finds
// every (r, q) whose closed MBRs meet (the MBR filter the paper delegates to
// an index) and runs the intermediate filter on those pairs with the batched
// kernels of filter.cu.
//
// The index is a uniform grid of 2^b x 2^b buckets over the lattice square;
// an object is listed in every bucket its MBR meets, in increasing object
// order.  A query scans the buckets its MBR meets, row by row; a pair is
// emitted only from the bucket holding the lower-left corner of
// MBR(r) n MBR(q) (the reference-point rule also used for partitions in
// Sec. 5.2), so each pair appears exactly once.  Pairs come out grouped by
// query, and within a query in bucket-row, bucket, object order: the
// same order on every run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "april_internal.h"

using april::fail;

struct april_index {
    uint32_t bits = 0;
    uint32_t n_objects = 0;
    std::vector<uint32_t> off;  // (2^bits)^2 + 1 bucket offsets
    std::vector<uint32_t> ent;  // object ids, bucket by bucket
    std::vector<uint16_t> ebx;  // the bucket column of every entry
};

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kLatticeBits = 24;
constexpr unsigned kSelBlock = 256;
constexpr uint32_t kMaxBucketBits = 12;

struct IndexLayout {
    uint64_t off, ent, ebx, total;
};

IndexLayout index_layout(const april_index &I) {
    IndexLayout L{};
    uint64_t o = 0;
    L.off = o;
    o += april_round256((uint64_t)I.off.size() * 4);
    L.ent = o;
    o += april_round256((uint64_t)I.ent.size() * 4);
    L.ebx = o;
    o += april_round256((uint64_t)I.ebx.size() * 2);
    L.total = o;
    return L;
}

inline uint32_t host_bucket(int64_t c, uint32_t bits) {
    const int64_t b = std::max<int64_t>(c, 0) >> (kLatticeBits - bits);
    return (uint32_t)std::min<int64_t>(b, ((int64_t)1 << bits) - 1);
}

april_status cuda_fail(cudaError_t e, const char *what) {
    return fail(APRIL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

__device__ __forceinline__ uint32_t bucket_of(int32_t c, uint32_t bits) {
    const uint32_t b = (uint32_t)max(c, 0) >> (kLatticeBits - bits);
    return min(b, (1u << bits) - 1u);
}

struct SelView {
    const uint32_t *off;
    const uint32_t *ent;
    const uint16_t *ebx;
    const int4 *rmbr;
    uint32_t bits;
};

// One warp per query.  Pass 1 (kFill = false) writes the query's pair count
// to qoff[q]; pass 2 writes the pairs at qoff[q] (then an exclusive offset)
// in the order described above, using ballots for an ordered compaction.
template <bool kFill>
__global__ void __launch_bounds__(kSelBlock) k_select(SelView I, const int4 *__restrict__ qmbr, uint32_t nq,
                                                      uint32_t *__restrict__ qoff, uint32_t *__restrict__ out_r,
                                                      uint32_t *__restrict__ out_q) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nw = gridDim.x * (kSelBlock / 32);
    for (uint32_t q = (blockIdx.x * kSelBlock + threadIdx.x) >> 5; q < nq; q += nw) {
        const int4 Q = __ldg(qmbr + q);
        const uint32_t bx0 = bucket_of(Q.x, I.bits), bx1 = bucket_of(Q.z, I.bits);
        const uint32_t by0 = bucket_of(Q.y, I.bits), by1 = bucket_of(Q.w, I.bits);
        const uint32_t base = kFill ? qoff[q] : 0u;
        uint32_t cnt = 0;
        for (uint32_t by = by0; by <= by1; ++by) {
            const uint32_t row = by << I.bits;
            const uint32_t p0 = __ldg(I.off + row + bx0), p1 = __ldg(I.off + row + bx1 + 1);
            for (uint32_t p = p0; p < p1; p += 32) {
                const uint32_t pp = p + lane;
                bool hit = false;
                uint32_t r = 0;
                if (pp < p1) {
                    r = __ldg(I.ent + pp);
                    const int4 M = __ldg(I.rmbr + r);
                    hit = M.x <= Q.z && Q.x <= M.z && M.y <= Q.w && Q.y <= M.w &&
                          (uint32_t)__ldg(I.ebx + pp) == max(bucket_of(M.x, I.bits), bx0) &&
                          by == max(bucket_of(M.y, I.bits), by0);
                }
                const uint32_t m = __ballot_sync(kFull, hit);
                if (kFill && hit) {
                    const uint32_t pos = base + cnt + __popc(m & ((1u << lane) - 1u));
                    out_r[pos] = r;
                    out_q[pos] = q;
                }
                cnt += __popc(m);
            }
        }
        if (!kFill && lane == 0) qoff[q] = cnt;
    }
}

// Exclusive prefix sum of the nq counts in place (one CTA of 1024 threads,
// each over a contiguous chunk); qoff[nq] and *total receive the sum.
constexpr unsigned kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan_counts(uint32_t *qoff, uint32_t nq,
                                                              unsigned long long *total) {
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    const uint32_t chunk = (nq + kScanThreads - 1) / kScanThreads;
    const uint32_t b = min(nq, t * chunk), e = min(nq, b + chunk);
    unsigned long long sum = 0;
    for (uint32_t k = b; k < e; ++k) sum += qoff[k];
    unsigned long long incl = sum;
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const unsigned long long v = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = s_warp[lane];
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const unsigned long long v = __shfl_up_sync(kFull, w, d);
            if (lane >= d) w += v;
        }
        s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long run = incl - sum + (warp ? s_warp[warp - 1] : 0ull);
    for (uint32_t k = b; k < e; ++k) {
        const uint32_t c = qoff[k];
        qoff[k] = (uint32_t)run;  // wraps only when the total overflows, which the host rejects
        run += c;
    }
    if (t == kScanThreads - 1) {
        const unsigned long long all = s_warp[31];
        qoff[nq] = (uint32_t)all;
        *total = all;
    }
}

}  // namespace

extern "C" april_status april_index_build(const april_sets *R, uint32_t bucket_bits, april_index **out) {
    if (!R || !out) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (R->parts) return fail(APRIL_ERR_INVALID_ARG, "the index takes sets built on one global grid");
    if (R->mbr.size() != 4 * (size_t)R->n) return fail(APRIL_ERR_INVALID_ARG, "sets carry no MBRs");
    uint32_t bits = bucket_bits;
    if (bits == 0) {  // about one object per bucket
        bits = 1;
        while (bits < kMaxBucketBits && ((uint64_t)1 << (2 * bits)) < R->n) ++bits;
    }
    if (bits > kMaxBucketBits) return fail(APRIL_ERR_INVALID_ARG, "bucket_bits must be at most 12");
    try {
        std::unique_ptr<april_index> I(new april_index());
        I->bits = bits;
        I->n_objects = R->n;
        const uint64_t B = (uint64_t)1 << bits;
        std::vector<uint64_t> cnt(B * B + 1, 0);
        for (uint32_t o = 0; o < R->n; ++o) {
            const int32_t *m = &R->mbr[4 * (size_t)o];
            const uint32_t x0 = host_bucket(m[0], bits), x1 = host_bucket(m[2], bits);
            const uint32_t y0 = host_bucket(m[1], bits), y1 = host_bucket(m[3], bits);
            for (uint32_t y = y0; y <= y1; ++y)
                for (uint32_t x = x0; x <= x1; ++x) ++cnt[((uint64_t)y << bits) + x];
        }
        uint64_t total = 0;
        for (uint64_t k = 0; k < B * B; ++k) {
            const uint64_t c = cnt[k];
            cnt[k] = total;
            total += c;
        }
        cnt[B * B] = total;
        if (total > 0xFFFFFFFFull) {
            return fail(APRIL_ERR_INVALID_ARG, "more than 2^32-1 index entries: use fewer buckets");
        }
        I->off.assign(cnt.begin(), cnt.end());
        I->ent.resize(total);
        I->ebx.resize(total);
        std::vector<uint64_t> pos(cnt.begin(), cnt.end() - 1);
        for (uint32_t o = 0; o < R->n; ++o) {
            const int32_t *m = &R->mbr[4 * (size_t)o];
            const uint32_t x0 = host_bucket(m[0], bits), x1 = host_bucket(m[2], bits);
            const uint32_t y0 = host_bucket(m[1], bits), y1 = host_bucket(m[3], bits);
            for (uint32_t y = y0; y <= y1; ++y)
                for (uint32_t x = x0; x <= x1; ++x) {
                    const uint64_t p = pos[((uint64_t)y << bits) + x]++;
                    I->ent[p] = o;
                    I->ebx[p] = (uint16_t)x;
                }
        }
        *out = I.release();
        return APRIL_OK;
    } catch (const std::bad_alloc &) {
        return fail(APRIL_ERR_NO_MEMORY, "host allocation failed while building the index");
    }
}

extern "C" void april_index_destroy(april_index *index) { delete index; }

extern "C" april_status april_index_get_info(const april_index *I, april_index_info *info) {
    if (!I || !info) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    info->bucket_bits = I->bits;
    info->n_objects = I->n_objects;
    info->n_entries = I->ent.size();
    info->device_bytes = index_layout(*I).total;
    return APRIL_OK;
}

extern "C" april_status april_index_upload(const april_index *I, void *dev_buf, size_t dev_bytes, void *stream,
                                           april_dev_index *out) {
    if (!I || !dev_buf || !out) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)dev_buf) & 255u) return fail(APRIL_ERR_INVALID_ARG, "device buffer must be 256-byte aligned");
    const IndexLayout L = index_layout(*I);
    if (dev_bytes < L.total) return fail(APRIL_ERR_INVALID_ARG, "device buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)dev_buf;
    cudaError_t e = cudaSuccess;
    auto put = [&](uint64_t off, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    put(L.off, I->off.data(), I->off.size() * 4);
    put(L.ent, I->ent.data(), I->ent.size() * 4);
    put(L.ebx, I->ebx.data(), I->ebx.size() * 2);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(index upload)");
    *out = april_dev_index{};
    out->off = (const uint32_t *)(base + L.off);
    out->ent = (const uint32_t *)(base + L.ent);
    out->ebx = (const uint16_t *)(base + L.ebx);
    out->bucket_bits = I->bits;
    out->n_objects = I->n_objects;
    out->n_entries = I->ent.size();
    return APRIL_OK;
}

extern "C" april_status april_select_scratch_bytes(uint64_t capacity, size_t *bytes) {
    if (!bytes) return fail(APRIL_ERR_INVALID_ARG, "bytes is NULL");
    size_t filt = 0;
    april_status s = april_filter_scratch_bytes(APRIL_MODE_BATCHED, std::max<uint64_t>(capacity, 1), &filt);
    if (s) return s;
    *bytes = 256 + april_round256(filt);
    return APRIL_OK;
}

extern "C" april_status april_select(april_ctx *ctx, const april_dev_index *I, const april_dev_sets *R,
                                     const april_dev_sets *Q, uint64_t capacity, uint32_t *d_r, uint32_t *d_q,
                                     uint8_t *d_verdict, uint32_t *d_query_off, uint64_t *n_pairs, void *d_scratch,
                                     size_t scratch_bytes, void *stream) {
    if (!ctx || !I || !R || !Q || !n_pairs || !d_query_off) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    *n_pairs = 0;
    if (R->parts || Q->parts) return fail(APRIL_ERR_INVALID_ARG, "selection takes sets built on one global grid");
    if (R->order != Q->order) return fail(APRIL_ERR_INVALID_ARG, "R and Q are on different grids");
    if (!R->mbr || !Q->mbr) return fail(APRIL_ERR_INVALID_ARG, "device sets carry no MBRs");
    if (I->n_objects != R->n_objects || I->bucket_bits == 0 || I->bucket_bits > kMaxBucketBits)
        return fail(APRIL_ERR_INVALID_ARG, "the index was not built over R");
    size_t need = 0;
    april_select_scratch_bytes(capacity, &need);
    if (!d_scratch || scratch_bytes < need) return fail(APRIL_ERR_INVALID_ARG, "scratch missing or too small");
    if (((uintptr_t)d_scratch) & 255u) return fail(APRIL_ERR_INVALID_ARG, "scratch must be 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nq = Q->n_objects;
    cudaError_t e;
    if (nq == 0) {
        e = cudaMemsetAsync(d_query_off, 0, 4, st);
        return e == cudaSuccess ? APRIL_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    const SelView V{I->off, I->ent, I->ebx, (const int4 *)R->mbr, I->bucket_bits};
    const int4 *qmbr = (const int4 *)Q->mbr;
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>(((uint64_t)nq * 32 + kSelBlock - 1) / kSelBlock, (uint64_t)april_ctx_num_sms(ctx) * 8));
    auto *total = (unsigned long long *)d_scratch;
    k_select<false><<<grid, kSelBlock, 0, st>>>(V, qmbr, nq, d_query_off, nullptr, nullptr);
    k_scan_counts<<<1, kScanThreads, 0, st>>>(d_query_off, nq, total);
    unsigned long long h_total = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_total, total, sizeof h_total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "counting selection candidates");
    *n_pairs = h_total;
    if (h_total > 0xFFFFFFFFull) return fail(APRIL_ERR_OVER_BUDGET, "more than 2^32-1 candidate pairs");
    if (!d_r && !d_q && !d_verdict) return APRIL_OK;  // count only
    if (!d_r || !d_q || !d_verdict) return fail(APRIL_ERR_INVALID_ARG, "NULL pair or verdict array");
    if (h_total > capacity) return fail(APRIL_ERR_OVER_BUDGET, "more candidate pairs than capacity");
    if (h_total == 0) return APRIL_OK;
    k_select<true><<<grid, kSelBlock, 0, st>>>(V, qmbr, nq, d_query_off, d_r, d_q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "selection candidates");
    return april_enqueue_request(ctx, R, Q, d_r, d_q, h_total, d_verdict, (char *)d_scratch + 256,
                                 april_ctx_status_word(ctx), 0xFFFFFFFFu, stream);
}
