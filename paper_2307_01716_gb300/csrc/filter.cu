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

#include <cstdio>
#include <string>

#include "april_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct DevSet {
    const uint4 *desc;  // {a_off, a_len, f_off, f_len}
    const uint2 *iv;    // {st, end}
    uint32_t n;
};

// status bits in the context's device status block
constexpr uint32_t ST_BAD_ID = 1u;
constexpr uint32_t ST_TIMEOUT = 2u;

__device__ __forceinline__ uint2 ld_iv(const uint2 *p) { return __ldg(p); }

// ------------------------------------------------------- K0: thread/pair
// IntervalJoin of Algorithm 2 as written: one thread walks both lists.
__device__ __forceinline__ bool seq_join(const uint2 *__restrict__ X, uint32_t nx, const uint2 *__restrict__ Y,
                                         uint32_t ny) {
    uint32_t i = 0, j = 0;
    if (nx == 0 || ny == 0) return false;
    uint2 x = ld_iv(X), y = ld_iv(Y);
    for (;;) {
        const uint32_t xl = x.y - 1u, yl = y.y - 1u;
        if (x.x <= yl && y.x <= xl) return true;
        if (xl <= yl) {
            if (++i == nx) return false;
            x = ld_iv(X + i);
        } else {
            if (++j == ny) return false;
            y = ld_iv(Y + j);
        }
    }
}

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

// -------------------------------------------------------- K1: warp/pair
// Number of elements among the first `cnt` lanes' values `v` (sorted
// ascending across lanes) that are < key (strict) or <= key (!strict).
template <bool kStrict>
__device__ __forceinline__ uint32_t warp_rank(uint32_t v, uint32_t cnt, uint32_t key) {
    uint32_t r = 0;
#pragma unroll
    for (uint32_t step = 16; step >= 1; step >>= 1) {
        const uint32_t probe = r + step - 1;
        const uint32_t pv = __shfl_sync(FULL, v, probe);
        const bool below = kStrict ? (pv < key) : (pv <= key);
        if (probe < cnt && below) r += step;
    }
    const uint32_t v31 = __shfl_sync(FULL, v, 31);
    const bool below31 = kStrict ? (v31 < key) : (v31 <= key);
    if (r == 31 && cnt == 32 && below31) r = 32;
    return r;
}

// Any overlap between X[0..n) and Y[0..m), one full warp, window of 32.
__device__ __noinline__ bool warp_join(const uint2 *__restrict__ X, uint32_t n, const uint2 *__restrict__ Y,
                                       uint32_t m, uint32_t lane) {
    uint32_t i0 = 0, j0 = 0;
    while (i0 < n && j0 < m) {
        const uint32_t nx = min(32u, n - i0), ny = min(32u, m - j0);
        uint2 x = make_uint2(0u, 0u), y = make_uint2(0u, 0u);
        if (lane < nx) x = ld_iv(X + i0 + lane);
        if (lane < ny) y = ld_iv(Y + j0 + lane);
        const uint32_t xl = x.y - 1u, yl = y.y - 1u;
        // X side: X_lane is emitted against Y_r
        const uint32_t r = warp_rank<true>(yl, ny, xl);
        const uint32_t ys = __shfl_sync(FULL, y.x, r & 31u), ylr = __shfl_sync(FULL, yl, r & 31u);
        bool hit = lane < nx && r < ny && ys <= xl && x.x <= ylr;
        // Y side: Y_lane is emitted against X_q
        const uint32_t q = warp_rank<false>(xl, nx, yl);
        const uint32_t xs = __shfl_sync(FULL, x.x, q & 31u), xlq = __shfl_sync(FULL, xl, q & 31u);
        hit |= lane < ny && q < nx && xs <= yl && y.x <= xlq;
        if (__any_sync(FULL, hit)) return true;
        i0 += __popc(__ballot_sync(FULL, lane < nx && lane + r < 32u));
        j0 += __popc(__ballot_sync(FULL, lane < ny && lane + q < 32u));
    }
    return false;
}

__global__ void __launch_bounds__(256) k_warp(DevSet R, DevSet S, const uint32_t *__restrict__ pr,
                                              const uint32_t *__restrict__ ps, uint64_t n,
                                              uint8_t *__restrict__ out, uint32_t *status) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t k = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n; k += warps) {
        const uint32_t r = __ldg(pr + k), s = __ldg(ps + k);
        if (r >= R.n || s >= S.n) {
            if (lane == 0) {
                out[k] = APRIL_VERDICT_ERROR;
                atomicOr(status, ST_BAD_ID);
            }
            continue;
        }
        const uint4 dr = __ldg(R.desc + r), ds = __ldg(S.desc + s);
        uint8_t v;
        if (!warp_join(R.iv + dr.x, dr.y, S.iv + ds.x, ds.y, lane)) v = APRIL_TRUE_NEGATIVE;
        else if (warp_join(R.iv + dr.x, dr.y, S.iv + ds.z, ds.w, lane)) v = APRIL_TRUE_HIT;
        else if (warp_join(R.iv + dr.z, dr.w, S.iv + ds.x, ds.y, lane)) v = APRIL_TRUE_HIT;
        else v = APRIL_INCONCLUSIVE;
        if (lane == 0) out[k] = v;
    }
}

int g_num_sms = 0;

}  // namespace

struct april_ctx {
    int device = 0;
    uint32_t *d_status = nullptr;  // 256-byte status block (word 0: ST_* bits)
    int num_sms = 0;
};

using april::fail;

static april_status cuda_fail(cudaError_t e, const char *what) {
    return fail(APRIL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" april_status april_ctx_create(int device, april_ctx **out) {
    if (!out) return fail(APRIL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto *c = new april_ctx();
    c->device = device;
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    e = cudaMalloc(&c->d_status, 256);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaMalloc(status)");
    }
    e = cudaMemset(c->d_status, 0, 256);
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return cuda_fail(e, "cudaMemset(status)");
    }
    g_num_sms = c->num_sms;
    *out = c;
    return APRIL_OK;
}

extern "C" void april_ctx_destroy(april_ctx *ctx) {
    if (!ctx) return;
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
}

extern "C" april_status april_upload(const april_sets *S, void *dev_buf, size_t dev_bytes, void *stream,
                                     april_dev_sets *out) {
    if (!S || !dev_buf || !out) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (((uintptr_t)dev_buf) & 255u) return fail(APRIL_ERR_INVALID_ARG, "device buffer must be 256-byte aligned");
    const uint64_t db = april_desc_bytes(S->n), ivb = (uint64_t)S->iv.size() * 4;
    if (dev_bytes < db + ivb) return fail(APRIL_ERR_INVALID_ARG, "device buffer too small");
    cudaStream_t st = (cudaStream_t)stream;
    char *base = (char *)dev_buf;
    cudaError_t e = cudaSuccess;
    if (S->n) e = cudaMemcpyAsync(base, S->desc.data(), (size_t)S->n * 16, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && ivb) e = cudaMemcpyAsync(base + db, S->iv.data(), ivb, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(upload)");
    out->desc = (const uint32_t *)base;
    out->iv = (const uint32_t *)(base + db);
    out->n_objects = S->n;
    out->order = S->order;
    out->iv_slots = S->iv.size() / 2;
    return APRIL_OK;
}

extern "C" april_status april_filter_scratch_bytes(int mode, uint64_t n, size_t *bytes) {
    if (!bytes) return fail(APRIL_ERR_INVALID_ARG, "bytes is NULL");
    (void)n;
    switch (mode) {
        case APRIL_MODE_PLAIN:
        case APRIL_MODE_WARP: *bytes = 0; return APRIL_OK;
        default: return fail(APRIL_ERR_INVALID_ARG, "unknown mode");
    }
}

static inline DevSet dev_set(const april_dev_sets *d) {
    return DevSet{(const uint4 *)d->desc, (const uint2 *)d->iv, d->n_objects};
}

extern "C" april_status april_filter_pairs(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                           const uint32_t *d_r, const uint32_t *d_s, uint64_t n,
                                           uint8_t *d_verdict, int mode, void *d_scratch, size_t scratch_bytes,
                                           void *stream) {
    if (!ctx || !R || !S) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return APRIL_OK;
    if (!d_r || !d_s || !d_verdict) return fail(APRIL_ERR_INVALID_ARG, "NULL pair or verdict array");
    if (R->order != S->order) return fail(APRIL_ERR_INVALID_ARG, "R and S are on different grids");
    (void)d_scratch;
    (void)scratch_bytes;
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
            uint64_t blocks = (n + 7) / 8;
            unsigned grid = (unsigned)std::min<uint64_t>(blocks, (uint64_t)sms * 8);
            k_warp<<<grid, 256, 0, st>>>(dR, dS, d_r, d_s, n, d_verdict, ctx->d_status);
            break;
        }
        default: return fail(APRIL_ERR_INVALID_ARG, "unknown mode");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return APRIL_OK;
}

static inline uint64_t round256(uint64_t b) { return (b + 255) / 256 * 256; }

extern "C" april_status april_filter_host_work_bytes(int mode, uint64_t n, size_t *bytes) {
    if (!bytes) return fail(APRIL_ERR_INVALID_ARG, "bytes is NULL");
    size_t sb = 0;
    april_status st = april_filter_scratch_bytes(mode, n, &sb);
    if (st) return st;
    *bytes = (size_t)(round256(4 * n) * 2 + round256(n) + round256(sb));
    return APRIL_OK;
}

extern "C" april_status april_filter_pairs_host(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                                const uint32_t *h_r, const uint32_t *h_s, uint64_t n,
                                                uint8_t *h_verdict, int mode, void *d_work, size_t work_bytes,
                                                void *stream) {
    if (!ctx || !R || !S) return fail(APRIL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return APRIL_OK;
    if (!h_r || !h_s || !h_verdict || !d_work) return fail(APRIL_ERR_INVALID_ARG, "NULL host or work buffer");
    if (((uintptr_t)d_work) & 255u) return fail(APRIL_ERR_INVALID_ARG, "work buffer must be 256-byte aligned");
    size_t need = 0, sb = 0;
    april_status st = april_filter_host_work_bytes(mode, n, &need);
    if (st) return st;
    if (work_bytes < need) return fail(APRIL_ERR_INVALID_ARG, "work buffer too small");
    april_filter_scratch_bytes(mode, n, &sb);
    char *w = (char *)d_work;
    uint32_t *d_r = (uint32_t *)w;
    uint32_t *d_s = (uint32_t *)(w + round256(4 * n));
    uint8_t *d_v = (uint8_t *)(w + 2 * round256(4 * n));
    void *d_scr = sb ? (void *)(w + 2 * round256(4 * n) + round256(n)) : nullptr;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_r, h_r, 4 * n, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, h_s, 4 * n, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(pairs)");
    st = april_filter_pairs(ctx, R, S, d_r, d_s, n, d_v, mode, d_scr, sb, stream);
    if (st) return st;
    e = cudaMemcpyAsync(h_verdict, d_v, n, cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(verdicts)");
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
