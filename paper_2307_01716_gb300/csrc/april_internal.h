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

}  // namespace april

// Host-side sets: per-object descriptors and the interval slots exactly as
// they are laid out in device memory by april_upload.
struct april_sets {
    uint32_t n = 0;
    uint32_t order = 0;
    uint64_t a_total = 0;
    uint64_t f_total = 0;
    std::vector<uint32_t> desc;  // 4 per object: a_off, a_len, f_off, f_len (in intervals)
    std::vector<uint32_t> iv;    // 2 per slot: st, end
};

// Device image layout: [desc (16 B per object)] [pad to 256 B] [iv (8 B per slot)]
inline uint64_t april_desc_bytes(uint32_t n) { return ((uint64_t)n * 16 + 255) / 256 * 256; }
