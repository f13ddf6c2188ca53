// Host-side helpers shared by the library's translation units: the error
// channel and the geometry handle.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/splitsart.h"

namespace splitsart {

// An NVTX range for the duration of a C-ABI call, so that a profiler's
// timeline shows the library's steps (fold, solve, recombine, ...). Without a
// tool attached a push/pop costs next to nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Record a failure for splitsart_last_error() and return `code`.
int fail(int code, const char* fmt, ...);

// First half (rows 0..Mh-1) of a matrix satisfying Eq. (2), in CSR form on the host.
struct HalfCsr {
    int64_t M = 0, N = 0;
    std::vector<int64_t> row_ptr;  // Mh + 1
    std::vector<int32_t> col;      // nnz, strictly increasing within a row
    std::vector<double> val;       // nnz
};

}  // namespace splitsart

struct splitsart_geometry {
    splitsart::HalfCsr half;
    bool has_params = false;
    splitsart_geometry_params params{};
};
