// Host-side helpers shared by the library's translation units: the error
// channel and the geometry handle.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <memory>
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
    std::vector<int32_t> col;      // nnz, strictly increasing within a row (empty if on the device)
    std::vector<double> val;       // nnz (empty if on the device)
};

// Columns and lengths traced on the device by one call, shared by the
// geometries of that call and freed with the last of them (geometry_gpu.cu).
struct DeviceRows {
    int32_t* col = nullptr;
    double* val = nullptr;
    ~DeviceRows();
};

// Copy a device-traced geometry's columns and lengths to host buffers (geometry_gpu.cu).
struct DeviceRowsView {
    const DeviceRows* rows;
    long long off, nnz;
};
int device_rows_to_host(const DeviceRowsView& v, int32_t* col, double* val);

// One slice's validated acquisition: sizes, and the source positions
// (source K-1-k is the exact mirror of source k). Shared by the host and
// device tracers, so that both trace from the same bits.
struct Acquisition {
    int64_t M = 0, N = 0, Mh = 0;
    std::vector<double> srcx, srcz;
};
int make_acquisition(const splitsart_geometry_params& p, Acquisition& a);

}  // namespace splitsart

struct splitsart_geometry {
    splitsart::HalfCsr half;  // row_ptr always on the host; col/val there unless `dev` holds them
    bool has_params = false;
    splitsart_geometry_params params{};
    std::shared_ptr<splitsart::DeviceRows> dev;  // device-traced rows: entries [dev_off, dev_off + nnz) of dev
    long long dev_off = 0;
};
