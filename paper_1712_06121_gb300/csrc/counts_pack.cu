// Section 2.1's compressed coarse density field: each cell's particle count
// in one byte, 255 marking a cell of 255 or more particles whose count is
// kept, in cell order, in a separate list of 4-byte integers.  Host code.
#include <cstdint>
#include <string>

#include "cube.h"

namespace cube {
cube_status served_fail(cube_status s, const char* msg);
}

extern "C" {

cube_status cube_counts_pack(const uint32_t* counts, int64_t n_cells, uint8_t* bytes, uint32_t* overflow,
                             int64_t overflow_cap, int64_t* n_overflow) {
    using cube::served_fail;
    if (!counts || !bytes || !n_overflow || n_cells < 0 || overflow_cap < 0)
        return served_fail(CUBE_E_ARG, "NULL argument or negative size");
    int64_t k = 0;
    for (int64_t i = 0; i < n_cells; ++i) {
        const uint32_t c = counts[i];
        if (c < 255u) {
            bytes[i] = (uint8_t)c;
        } else {
            bytes[i] = 255u;
            if (k < overflow_cap && overflow) overflow[k] = c;
            ++k;
        }
    }
    *n_overflow = k;                    // the list's length, also when it did not fit
    if (k > overflow_cap || (k && !overflow))
        return served_fail(CUBE_E_ARG, "overflow list too short (n_overflow holds the length needed)");
    return CUBE_OK;
}

cube_status cube_counts_unpack(const uint8_t* bytes, int64_t n_cells, const uint32_t* overflow, int64_t n_overflow,
                               uint32_t* counts) {
    using cube::served_fail;
    if (!bytes || !counts || n_cells < 0 || n_overflow < 0 || (n_overflow && !overflow))
        return served_fail(CUBE_E_ARG, "NULL argument or negative size");
    int64_t k = 0;
    for (int64_t i = 0; i < n_cells; ++i) {
        if (bytes[i] < 255u) {
            counts[i] = bytes[i];
        } else {
            if (k >= n_overflow) return served_fail(CUBE_E_ARG, "more 255 bytes than overflow entries");
            if (overflow[k] < 255u) return served_fail(CUBE_E_ARG, "an overflow entry below 255");
            counts[i] = overflow[k++];
        }
    }
    if (k != n_overflow) return served_fail(CUBE_E_ARG, "fewer 255 bytes than overflow entries");
    return CUBE_OK;
}

}  // extern "C"
