// Internal declarations shared by the host builder and the CUDA side of
// libapril.  Not part of the public ABI (include/april.h is).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/april.h"

namespace april {

// Records msg as the calling thread's last error and returns code.
april_status fail(april_status code, const std::string &msg);
// Validates a grid (as april_build_sets does) and returns its parameters.
april_status check_grid_params(const april_grid *grid, int64_t &ox, int64_t &oy, int64_t &h, uint32_t &order,
                               int64_t &G);

}  // namespace april

// Shared between filter.cu and server.cu (not exported).
april_status april_enqueue_request(april_ctx *ctx, const april_dev_sets *R, const april_dev_sets *S,
                                   const uint32_t *d_r, const uint32_t *d_s, uint64_t n, uint8_t *d_verdict,
                                   void *d_scratch, uint32_t *d_status, unsigned max_ctas, void *stream);
int april_ctx_num_sms(const april_ctx *ctx);
uint32_t *april_ctx_status_word(april_ctx *ctx);
int april_ctx_device(const april_ctx *ctx);

// Host-side sets: per-entry descriptors and the interval slots exactly as
// they are laid out in device memory by april_upload.  An entry is one
// object's approximation on one grid: for sets built on one global grid the
// entries are the objects; for partitioned sets (Sec. 5.2) an object has one
// entry per partition its MBR meets.
struct april_sets {
    uint32_t n = 0;          // objects
    uint32_t order = 0;
    uint32_t parts = 0;      // partitions per dimension (0: one global grid)
    uint32_t n_entries = 0;  // == n when parts == 0
    uint64_t a_total = 0;
    uint64_t f_total = 0;
    std::vector<uint32_t> desc;       // 4 per entry: a_off, a_len, f_off, f_len (in intervals)
    std::vector<uint32_t> iv;         // 2 per slot: st, end
    std::vector<int32_t> mbr;         // 4 per object: x0, y0, x1, y1 (lattice units, closed)
    std::vector<int32_t> obj_ll;      // parts > 0: 2 per object, lower-left corner of its MBR
    std::vector<uint32_t> obj_entry;  // parts > 0: n + 1 entry offsets (entries of an object are contiguous)
    std::vector<uint32_t> entry_pid;  // parts > 0: partition id of each entry (ascending within an object)
    std::vector<int64_t> part_grid;   // parts > 0: 4 per partition: ox, oy, log2_cell, used(0/1)
    // sets built from polygons: the grid of one-grid sets (parts == 0) as
    // lattice origin and log2 of the cell side (partitioned sets: part_grid),
    // with which the batched filter's triage maps an MBR point to its cell,
    // and a fingerprint of the grid(s) (april_grid_id / april_part_grid_id)
    bool grid_known = false;
    int64_t grid_ox = 0, grid_oy = 0;
    uint32_t grid_log2_cell = 0;
    uint64_t grid_id = 0;
    // compressed lists (Sec. 5.1), see april_sets_compress
    bool packed = false;
    std::vector<uint32_t> pdesc;      // 4 per entry: {a_block, a_len, f_block, f_len} (block-table indices)
    std::vector<uint32_t> anchors;    // block table, 2 per block: {anchor, gap_off64 | wide << 31}
    std::vector<uint8_t> gaps;        // per block 32 gap slots (slot 0 unused): 64 B (uint16) or 128 B (uint32)
};

inline uint64_t april_round256(uint64_t b) { return (b + 255) / 256 * 256; }

// Fingerprints of the grids sets were built on (FNV-1a over the defining
// integers): two sets may share the triage's cell mapping only when equal.
inline uint64_t april_fnv(uint64_t h, int64_t v) {
    for (int b = 0; b < 8; ++b) h = (h ^ (uint64_t)((v >> (8 * b)) & 0xFF)) * 1099511628211ull;
    return h;
}
inline uint64_t april_grid_id(int64_t ox, int64_t oy, uint32_t log2_cell, uint32_t order) {
    uint64_t h = 14695981039346656037ull;
    for (int64_t v : {ox, oy, (int64_t)log2_cell, (int64_t)order}) h = april_fnv(h, v);
    return h | 1;  // never 0
}
inline uint64_t april_part_grid_id(const std::vector<int64_t> &part_grid, uint32_t order, uint32_t parts) {
    uint64_t h = april_fnv(april_fnv(14695981039346656037ull, order), parts);
    for (int64_t v : part_grid) h = april_fnv(h, v);
    return h | 1;
}

// Skip index of a set's interval array ("posts"): posts[q] is the last cell
// (end - 1, in uint32) of interval slot 16 q + 15, one word per 16 slots; the
// filter's start searches read it instead of the intervals (see
// join_device.cuh).  Padded to whole 16-byte words for vector loads.
inline uint64_t april_posts_words(uint64_t iv_slots) { return (iv_slots / 16 + 3) / 4 * 4; }
// Fills posts from the device intervals iv (slots of {st, end}) on the CUDA
// stream `stream`; returns the launch's cudaError_t as an int.
int april_launch_posts(const uint32_t *iv, uint64_t iv_slots, uint32_t *posts, void *stream);

// Device image layout (each section starts 256-byte aligned):
//   desc (16 B/entry) | iv (8 B/slot, then a 16-byte pad) | posts (4 B per 16 slots) | obj_ll (8 B/object)
//   | obj_entry (4 B x (n+1)) | entry_pid (4 B/entry) | pdesc (16 B/entry) | block table (8 B/block) | gaps
//   | mbr (16 B/object) | part_grid (32 B/partition: ox, oy, log2_cell, used as int64)
struct april_image_layout {
    uint64_t desc, iv, posts, obj_ll, obj_entry, entry_pid, pdesc, anchors, gaps, mbr, pgrid, total;
};

inline april_image_layout april_layout(const april_sets &S) {
    april_image_layout L{};
    uint64_t o = 0;
    L.desc = o;
    o += april_round256((uint64_t)S.n_entries * 16);
    L.iv = o;
    o += april_round256((uint64_t)S.iv.size() * 4 + 16);  // 16-byte pad: bulk copies round spans up to 16 bytes
    L.posts = o;
    o += april_round256(april_posts_words(S.iv.size() / 2) * 4);
    L.obj_ll = o;
    o += april_round256((uint64_t)S.obj_ll.size() * 4);
    L.obj_entry = o;
    o += april_round256((uint64_t)S.obj_entry.size() * 4);
    L.entry_pid = o;
    o += april_round256((uint64_t)S.entry_pid.size() * 4);
    L.pdesc = o;
    o += april_round256((uint64_t)S.pdesc.size() * 4);
    L.anchors = o;
    o += april_round256((uint64_t)S.anchors.size() * 4);
    L.gaps = o;
    o += april_round256((uint64_t)S.gaps.size());
    L.mbr = o;
    o += april_round256((uint64_t)S.mbr.size() * 4);
    L.pgrid = o;
    o += april_round256((uint64_t)S.part_grid.size() * 8);
    L.total = o;
    return L;
}
