// C ABI: system lifetime, argument checks, error channel and exports.
// The operations themselves live in fold.cu (fold, vector kernels) and
// sart.cu (the persistent solve).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "system.h"

namespace splitsart {

namespace {
thread_local std::string g_last_error;

size_t pair_bytes(int dt) { return dt == SPLITSART_F64 ? 16 : (dt == SPLITSART_F32 ? 8 : 4); }
size_t norm_pair_bytes(int dt) { return dt == SPLITSART_F32 ? 8 : 16; }
size_t vec_pair_bytes(int dt) { return dt == SPLITSART_F64 ? 16 : 8; }
size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

int check_stream_ok(cudaStream_t st) {
    cudaError_t e = cudaStreamQuery(st);
    if (e == cudaSuccess || e == cudaErrorNotReady) return SPLITSART_OK;
    return cuda_fail(e, "stream");
}

float bf16_bits_to_float(uint16_t b) {
    uint32_t u = uint32_t(b) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// IEEE binary16 -> float, from the bit fields.
float f16_bits_to_float(uint16_t h) {
    const int sign = (h >> 15) & 1, ex = (h >> 10) & 31, man = h & 1023;
    double v;
    if (ex == 0) v = std::ldexp((double)man, -24);
    else if (ex == 31) v = man ? NAN : INFINITY;
    else v = std::ldexp((double)(man | 1024), ex - 25);
    return (float)(sign ? -v : v);
}

// Decode S stored pairs of `dtype` to double (dequantised with per-row scales if needed).
void decode_pairs(int dt, const std::vector<uint8_t>& raw, const std::vector<int32_t>& row_of,
                  const std::vector<float>& scale2, double* a1, double* a2, size_t S) {
    for (size_t e = 0; e < S; ++e) {
        double x1 = 0, x2 = 0;
        if (dt == SPLITSART_F64) {
            std::memcpy(&x1, &raw[e * 16], 8);
            std::memcpy(&x2, &raw[e * 16 + 8], 8);
        } else if (dt == SPLITSART_F32) {
            float f1, f2;
            std::memcpy(&f1, &raw[e * 8], 4);
            std::memcpy(&f2, &raw[e * 8 + 4], 4);
            x1 = f1;
            x2 = f2;
        } else {
            uint16_t h1, h2;
            std::memcpy(&h1, &raw[e * 4], 2);
            std::memcpy(&h2, &raw[e * 4 + 2], 2);
            const float c1 = dt == SPLITSART_BF16 ? bf16_bits_to_float(h1) : f16_bits_to_float(h1);
            const float c2 = dt == SPLITSART_BF16 ? bf16_bits_to_float(h2) : f16_bits_to_float(h2);
            const int32_t r = row_of[e];
            x1 = (double)scale2[2 * r] * (double)c1;
            x2 = (double)scale2[2 * r + 1] * (double)c2;
        }
        if (a1) a1[e] = x1;
        if (a2) a2[e] = x2;
    }
}

int64_t read_S(splitsart_system* s) {
    if (s->S >= 0) return s->S;
    cudaError_t e = cudaStreamSynchronize(s->last);
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    FoldStats fs;
    e = cudaMemcpy(&fs, s->stats, sizeof(fs), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read fold stats");
    s->S = s->Mh > 0 ? fs.S : 0;
    return s->S;
}

}  // namespace

int system_host_stats(splitsart_system* s, FoldStats* out) {
    if (!s->have_stats) {
        cudaError_t e = cudaStreamSynchronize(s->last);
        if (e != cudaSuccess) return cuda_fail(e, "sync");
        e = cudaMemcpy(&s->hstats, s->stats, sizeof(FoldStats), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read fold stats");
        if (s->Mh == 0) s->hstats = FoldStats{};
        s->have_stats = true;
    }
    *out = s->hstats;
    return SPLITSART_OK;
}

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(SPLITSART_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

}  // namespace splitsart

using namespace splitsart;

extern "C" int splitsart_solve_result_slices(splitsart_system* s, splitsart_solve_info* info, int n) {
    if (!s || !info || n < s->ns) return fail(SPLITSART_ERR_ARG, "solve_result_slices: NULL or short buffer");
    splitsart_solve_info agg;
    int rc = splitsart_solve_result(s, &agg);
    if (rc != SPLITSART_OK) {
        for (int k = 0; k < s->ns; ++k) info[k] = agg;
        return rc;
    }
    if (s->ns == 1) {
        info[0] = agg;
        return SPLITSART_OK;
    }
    std::vector<SliceSolve> v(s->ns);
    cudaError_t e = cudaMemcpy(v.data(), s->sl_solve, sizeof(SliceSolve) * s->ns, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "solve_result_slices: read");
    for (int k = 0; k < s->ns; ++k) {
        info[k].iters = v[k].iters;
        info[k].status = v[k].done ? SPLITSART_OK : SPLITSART_ERR_STATE;
        info[k].rho = v[k].rho;
        info[k].rr = v[k].rr;
        info[k].pp = v[k].pp;
    }
    return SPLITSART_OK;
}

extern "C" int splitsart_last_error(char* buf, size_t len) {
    if (buf && len) {
        std::strncpy(buf, g_last_error.c_str(), len - 1);
        buf[len - 1] = '\0';
    }
    return (int)g_last_error.size();
}

extern "C" const char* splitsart_version(void) { return "splitsart 0.1 (sm_103a)"; }

namespace {

// Build one device system from ns geometries (ns = 1: a single slice; more: a
// block-diagonal batch). Each slice keeps its own M_s, N_s and reflection.
int create_system(const splitsart_geometry* const* geoms, int ns, int dtype, cudaStream_t st, splitsart_system** out) {
    if (!geoms || !out || ns < 1) return fail(SPLITSART_ERR_ARG, "fold: NULL argument or no slices");
    *out = nullptr;
    if (dtype < SPLITSART_F64 || dtype > SPLITSART_F16) return fail(SPLITSART_ERR_ARG, "fold: bad dtype %d", dtype);
    std::vector<long long> rows(ns + 1, 0), cols(ns + 1, 0), Mo(ns + 1, 0), No(ns + 1, 0), nnzo(ns + 1, 0);
    std::vector<int> nxs(ns, 0), nzs(ns, 0);
    for (int k = 0; k < ns; ++k) {
        const splitsart_geometry* g = geoms[k];
        if (!g) return fail(SPLITSART_ERR_ARG, "fold: NULL geometry %d", k);
        const HalfCsr& h = g->half;
        rows[k + 1] = rows[k] + h.M / 2;
        cols[k + 1] = cols[k] + h.N / 2;
        Mo[k + 1] = Mo[k] + h.M;
        No[k + 1] = No[k] + h.N;
        nnzo[k + 1] = nnzo[k] + h.row_ptr.back();
        if (g->has_params) {
            nxs[k] = g->params.nx;
            nzs[k] = g->params.nz;
        }
    }
    const int64_t M = Mo[ns], N = No[ns], Mh = rows[ns], Nh = cols[ns], nnz = nnzo[ns];
    if (nnz >= INT32_MAX) return fail(SPLITSART_ERR_ARG, "fold: %lld half-row entries exceed int32", (long long)nnz);
    if (Mh >= INT32_MAX || Nh >= INT32_MAX) return fail(SPLITSART_ERR_ARG, "fold: dimensions exceed int32");
    int rc = check_stream_ok(st);
    if (rc) return rc;

    auto* s = new (std::nothrow) splitsart_system();
    if (!s) return fail(SPLITSART_ERR_NOMEM, "fold: out of host memory");
    s->M = M;
    s->N = N;
    s->Mh = Mh;
    s->Nh = Nh;
    s->nnz_half = nnz;
    s->dtype = dtype;
    s->last = st;
    s->ns = ns;
    s->h_rows = rows;
    s->h_cols = cols;
    s->h_M = Mo;
    s->h_N = No;
    s->h_nx = nxs;
    s->h_nz = nzs;
    if (ns == 1) {
        s->nx = nxs[0];
        s->nz = nzs[0];
        if (geoms[0]->has_params) s->nb = geoms[0]->params.nb;
    }
    const size_t pb = pair_bytes(dtype), nb = norm_pair_bytes(dtype), vb = vec_pair_bytes(dtype);
    const int64_t mx = (Mh > Nh ? Mh : Nh) + 1;
    const int64_t ntiles = (mx + 4095) / 4096 + 2;
    const bool quant = dtype == SPLITSART_BF16 || dtype == SPLITSART_F16;
    struct Item { void** ptr; size_t bytes; };
    std::vector<Item> items = {
        {(void**)&s->hrp, sizeof(int64_t) * (Mh + 1)},
        {(void**)&s->hcol, sizeof(int32_t) * nnz},
        {(void**)&s->hval, sizeof(double) * nnz},
        {(void**)&s->rp, sizeof(int32_t) * (Mh + 1)},
        {(void**)&s->col, sizeof(int32_t) * nnz},
        {(void**)&s->val, pb * nnz},
        {(void**)&s->cp, sizeof(int32_t) * (Nh + 1)},
        {(void**)&s->row, sizeof(int32_t) * nnz},
        {(void**)&s->valT, pb * nnz},
        {(void**)&s->Rsum, sizeof(double2) * Mh},
        {(void**)&s->Csum, sizeof(double2) * Nh},
        {(void**)&s->invR, nb * Mh},
        {(void**)&s->invC, nb * Nh},
        {(void**)&s->scale, quant ? sizeof(float2) * Mh : 0},
        {(void**)&s->wR, quant ? sizeof(float2) * Mh : 0},
        {(void**)&s->wC, quant ? sizeof(float2) * Nh : 0},
        {(void**)&s->nzr, sizeof(int32_t) * (Mh + 1)},
        {(void**)&s->nzrp, sizeof(int32_t) * (Mh + 1)},
        {(void**)&s->zr, sizeof(int32_t) * (Mh + 1)},
        {(void**)&s->nzc, sizeof(int32_t) * (Nh + 1)},
        {(void**)&s->nzcp, sizeof(int32_t) * (Nh + 1)},
        {(void**)&s->sl_rows, sizeof(long long) * (ns + 1)},
        {(void**)&s->sl_cols, sizeof(long long) * (ns + 1)},
        {(void**)&s->sl_M, sizeof(long long) * (ns + 1)},
        {(void**)&s->sl_N, sizeof(long long) * (ns + 1)},
        {(void**)&s->sl_nx, sizeof(int) * ns},
        {(void**)&s->sl_nz, sizeof(int) * ns},
        {(void**)&s->sl_solve, sizeof(SliceSolve) * ns},
        {(void**)&s->rr_row, ns > 1 ? sizeof(double) * Mh : 0},
        {(void**)&s->ndone, sizeof(int) * 4},
        {(void**)&s->cnt, sizeof(int32_t) * mx},
        {(void**)&s->flags, sizeof(int32_t) * mx},
        {(void**)&s->scan_tmp, sizeof(int32_t) * ntiles},
        {(void**)&s->stats, sizeof(FoldStats)},
        {(void**)&s->u12, vb * Mh},
        {(void**)&s->tmp_f12, vb * Nh},
        {(void**)&s->tmp_q12, vb * Mh},
        {(void**)&s->partials, sizeof(double) * 2 * kMaxCtas},
        {(void**)&s->ctl, sizeof(LaunchCtl)},
        {(void**)&s->result, sizeof(SolveResultDev)},
    };
    size_t total = 0;
    for (auto& it : items) total += align_up(it.bytes > 0 ? it.bytes : 1);
    cudaError_t e = cudaMalloc(&s->base, total);
    if (e != cudaSuccess) {
        delete s;
        cudaGetLastError();
        return fail(SPLITSART_ERR_NOMEM, "fold: cudaMalloc of %zu bytes failed (%s)", total, cudaGetErrorString(e));
    }
    s->device_bytes = (int64_t)total;
    size_t off = 0;
    for (auto& it : items) {
        *it.ptr = it.bytes > 0 ? (void*)((char*)s->base + off) : nullptr;
        off += align_up(it.bytes > 0 ? it.bytes : 1);
    }
    // Upload: one row-pointer array over all slices, then each slice's entries in place.
    std::vector<int64_t> hrp(Mh + 1);
    for (int k = 0; k < ns; ++k) {
        const HalfCsr& h = geoms[k]->half;
        for (int64_t i = 0; i < h.M / 2; ++i) hrp[rows[k] + i] = nnzo[k] + h.row_ptr[i];
    }
    hrp[Mh] = nnz;
    e = cudaMemcpyAsync(s->hrp, hrp.data(), sizeof(int64_t) * (Mh + 1), cudaMemcpyHostToDevice, st);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) {
        const splitsart_geometry* g = geoms[k];
        const int64_t n = nnzo[k + 1] - nnzo[k];
        if (n == 0) continue;
        // Rows traced on the device are copied there; host rows are uploaded.
        const int32_t* col = g->dev ? g->dev->col + g->dev_off : g->half.col.data();
        const double* val = g->dev ? g->dev->val + g->dev_off : g->half.val.data();
        const cudaMemcpyKind kind = g->dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        e = cudaMemcpyAsync(s->hcol + nnzo[k], col, sizeof(int32_t) * n, kind, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->hval + nnzo[k], val, sizeof(double) * n, kind, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sl_rows, rows.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sl_cols, cols.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sl_M, Mo.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sl_N, No.data(), sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sl_nx, nxs.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->sl_nz, nzs.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st);
    // The host vectors above are pageable: their copies complete before cudaMemcpyAsync
    // returns. Device-traced rows are copied on the stream; cudaFree, which releases
    // them with their geometries, waits for that copy.
    if (e != cudaSuccess) {
        splitsart_system_destroy(s);
        return cuda_fail(e, "fold: upload");
    }
    rc = run_fold(s, st);
    if (rc) {
        splitsart_system_destroy(s);
        return rc;
    }
    *out = s;
    return SPLITSART_OK;
}

}  // namespace

extern "C" int splitsart_fold_system(const splitsart_geometry* g, int dtype, void* stream, splitsart_system** out) {
    splitsart::NvtxRange nvtx_range("splitsart_fold_system");
    if (!g) return fail(SPLITSART_ERR_ARG, "fold_system: NULL geometry");
    return create_system(&g, 1, dtype, (cudaStream_t)stream, out);
}

extern "C" int splitsart_fold_batch(const splitsart_geometry* const* geoms, int nslices, int dtype, void* stream,
                                    splitsart_system** out) {
    splitsart::NvtxRange nvtx_range("splitsart_fold_batch");
    return create_system(geoms, nslices, dtype, (cudaStream_t)stream, out);
}

extern "C" int splitsart_system_slices(const splitsart_system* s, int64_t* M_off, int64_t* N_off, int64_t* Mh_off,
                                       int64_t* Nh_off) {
    if (!s) return fail(SPLITSART_ERR_ARG, "system_slices: NULL system");
    for (int k = 0; k <= s->ns; ++k) {
        if (M_off) M_off[k] = s->h_M[k];
        if (N_off) N_off[k] = s->h_N[k];
        if (Mh_off) Mh_off[k] = s->h_rows[k];
        if (Nh_off) Nh_off[k] = s->h_cols[k];
    }
    return SPLITSART_OK;
}

extern "C" int splitsart_refold(splitsart_system* s, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_refold");
    if (!s) return fail(SPLITSART_ERR_ARG, "refold: NULL system");
    s->last = (cudaStream_t)stream;
    s->S = -1;
    return run_fold(s, (cudaStream_t)stream);
}

extern "C" void splitsart_system_destroy(splitsart_system* s) {
    if (!s) return;
    if (s->base || s->res_alloc || s->os_alloc || s->cg_alloc || s->st[0].alloc || s->st[1].alloc)
        cudaStreamSynchronize(s->last);
    for (auto& f : s->st) {
        if (f.alloc) cudaFree(f.alloc);
        if (f.ring_alloc) cudaFree(f.ring_alloc);
    }
    if (s->base) cudaFree(s->base);
    if (s->res_alloc) cudaFree(s->res_alloc);
    if (s->os_alloc) cudaFree(s->os_alloc);
    if (s->cg_alloc) cudaFree(s->cg_alloc);
    delete s;
}

extern "C" int splitsart_system_info_get(splitsart_system* s, splitsart_system_info* info) {
    if (!s || !info) return fail(SPLITSART_ERR_ARG, "system_info: NULL argument");
    const int64_t S = read_S(s);
    if (S < 0) return (int)S;
    FoldStats fs{};
    cudaError_t e = cudaMemcpy(&fs, s->stats, sizeof(fs), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "system_info");
    info->M = s->M;
    info->N = s->N;
    info->Mh = s->Mh;
    info->Nh = s->Nh;
    info->nnz_half = s->nnz_half;
    info->S = S;
    info->empty_rows = s->Mh > 0 ? fs.empty_rows : 0;
    info->exact_zeros = s->Mh > 0 ? fs.exact_zeros : 0;
    info->dtype = s->dtype;
    info->nx = s->nx;
    info->nz = s->nz;
    info->device_bytes = s->device_bytes;
    info->nslices = s->ns;
    info->reserved = 0;
    return SPLITSART_OK;
}

extern "C" int splitsart_system_export(splitsart_system* s, int64_t* rp_h, int32_t* col_h, double* a1_h, double* a2_h,
                                       double* R_h, double* C_h) {
    if (!s || !rp_h || !col_h) return fail(SPLITSART_ERR_ARG, "system_export: NULL argument");
    const int64_t S = read_S(s);
    if (S < 0) return (int)S;
    const int64_t Mh = s->Mh;
    std::vector<int32_t> rp(Mh + 1);
    std::vector<uint8_t> raw(pair_bytes(s->dtype) * S);
    std::vector<float> sc(2 * Mh);
    cudaError_t e;
    if ((e = cudaMemcpy(rp.data(), s->rp, sizeof(int32_t) * (Mh + 1), cudaMemcpyDeviceToHost)) ||
        (S && (e = cudaMemcpy(col_h, s->col, sizeof(int32_t) * S, cudaMemcpyDeviceToHost))) ||
        (S && (e = cudaMemcpy(raw.data(), s->val, raw.size(), cudaMemcpyDeviceToHost))) ||
        (s->scale && Mh && (e = cudaMemcpy(sc.data(), s->scale, sizeof(float) * 2 * Mh, cudaMemcpyDeviceToHost))) ||
        (R_h && Mh && (e = cudaMemcpy(R_h, s->Rsum, sizeof(double2) * Mh, cudaMemcpyDeviceToHost))) ||
        (C_h && s->Nh && (e = cudaMemcpy(C_h, s->Csum, sizeof(double2) * s->Nh, cudaMemcpyDeviceToHost))))
        return cuda_fail(e, "system_export");
    std::vector<int32_t> row_of(S);
    for (int64_t i = 0; i < Mh; ++i) {
        rp_h[i] = rp[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) row_of[k] = (int32_t)i;
    }
    rp_h[Mh] = rp[Mh];
    decode_pairs(s->dtype, raw, row_of, sc, a1_h, a2_h, (size_t)S);
    return SPLITSART_OK;
}

extern "C" int splitsart_system_export_csc(splitsart_system* s, int64_t* cp_h, int32_t* row_h, double* a1_h,
                                           double* a2_h) {
    if (!s || !cp_h || !row_h) return fail(SPLITSART_ERR_ARG, "system_export_csc: NULL argument");
    const int64_t S = read_S(s);
    if (S < 0) return (int)S;
    const int64_t Nh = s->Nh, Mh = s->Mh;
    std::vector<int32_t> cp(Nh + 1);
    std::vector<uint8_t> raw(pair_bytes(s->dtype) * S);
    std::vector<float> sc(2 * Mh);
    cudaError_t e;
    if ((e = cudaMemcpy(cp.data(), s->cp, sizeof(int32_t) * (Nh + 1), cudaMemcpyDeviceToHost)) ||
        (S && (e = cudaMemcpy(row_h, s->row, sizeof(int32_t) * S, cudaMemcpyDeviceToHost))) ||
        (S && (e = cudaMemcpy(raw.data(), s->valT, raw.size(), cudaMemcpyDeviceToHost))) ||
        (s->scale && Mh && (e = cudaMemcpy(sc.data(), s->scale, sizeof(float) * 2 * Mh, cudaMemcpyDeviceToHost))))
        return cuda_fail(e, "system_export_csc");
    for (int64_t j = 0; j <= Nh; ++j) cp_h[j] = cp[j];
    std::vector<int32_t> row_of(row_h, row_h + S);
    decode_pairs(s->dtype, raw, row_of, sc, a1_h, a2_h, (size_t)S);
    return SPLITSART_OK;
}

extern "C" int splitsart_fold_rhs(const splitsart_system* s, const void* p, void* p12, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_fold_rhs");
    if (!s || (s->Mh > 0 && (!p || !p12))) return fail(SPLITSART_ERR_ARG, "fold_rhs: NULL argument");
    const_cast<splitsart_system*>(s)->last = (cudaStream_t)stream;
    return run_fold_rhs(s, p, p12, (cudaStream_t)stream);
}

static int check_layout(const splitsart_system* s, int layout, const char* who) {
    if (layout == SPLITSART_LAYOUT_SNAKE) return SPLITSART_OK;
    if (layout == SPLITSART_LAYOUT_IMAGE) {
        for (int k = 0; k < s->ns; ++k)
            if (s->h_nx[k] <= 0 || s->h_nz[k] <= 0)
                return fail(SPLITSART_ERR_ARG, "%s: image layout needs geometries built from parameters", who);
        return SPLITSART_OK;
    }
    return fail(SPLITSART_ERR_ARG, "%s: unknown layout %d", who, layout);
}

extern "C" int splitsart_fold_image(const splitsart_system* s, const void* f, int layout, void* f12, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_fold_image");
    if (!s || (s->Nh > 0 && (!f || !f12))) return fail(SPLITSART_ERR_ARG, "fold_image: NULL argument");
    int rc = check_layout(s, layout, "fold_image");
    if (rc) return rc;
    const_cast<splitsart_system*>(s)->last = (cudaStream_t)stream;
    return run_fold_image(s, f, layout, f12, (cudaStream_t)stream);
}

extern "C" int splitsart_recombine(const splitsart_system* s, const void* f12, void* f, int layout, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_recombine");
    if (!s || (s->Nh > 0 && (!f || !f12))) return fail(SPLITSART_ERR_ARG, "recombine: NULL argument");
    int rc = check_layout(s, layout, "recombine");
    if (rc) return rc;
    const_cast<splitsart_system*>(s)->last = (cudaStream_t)stream;
    return run_recombine(s, f12, f, layout, (cudaStream_t)stream);
}

extern "C" int splitsart_project(splitsart_system* s, const void* f, int layout, void* p, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_project");
    if (!s || !f || !p) return fail(SPLITSART_ERR_ARG, "project: NULL argument");
    int rc = check_layout(s, layout, "project");
    if (rc) return rc;
    s->last = (cudaStream_t)stream;
    return run_project(s, f, layout, p, (cudaStream_t)stream);
}

extern "C" int splitsart_solve(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts* o,
                               void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_solve");
    if (!s || !o) return fail(SPLITSART_ERR_ARG, "solve: NULL argument");
    if ((s->Mh > 0 && !p12) || (s->Nh > 0 && !f12)) return fail(SPLITSART_ERR_ARG, "solve: NULL vector");
    if (o->max_iters < 0 || o->max_iters > 500000)
        return fail(SPLITSART_ERR_ARG, "solve: max_iters must be in [0, 500000]");
    if (o->kernel < 0 || o->kernel > 8) return fail(SPLITSART_ERR_ARG, "solve: kernel must be in [0, 8]");
    if (o->tile_entries != 0 && (o->tile_entries % 1024 != 0 || o->tile_entries < 1024 || o->tile_entries > 16384))
        return fail(SPLITSART_ERR_ARG, "solve: tile_entries must be 0 or a multiple of 1024 in [1024, 16384]");
    if (!(o->lambda > 0.0) || !std::isfinite(o->lambda)) return fail(SPLITSART_ERR_ARG, "solve: lambda must be > 0");
    if (!(o->tol >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve: tol must be >= 0");
    if (o->check_every < 0) return fail(SPLITSART_ERR_ARG, "solve: check_every must be >= 0");
    if (!(o->timeout_ms >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve: timeout_ms must be >= 0");
    s->last = (cudaStream_t)stream;
    if (o->kernel == 5 || o->kernel == 6) return run_solve_stream(s, p12, f12, *o, (cudaStream_t)stream);
    if (o->kernel == 7 || o->kernel == 8) return run_solve_ring(s, p12, f12, *o, (cudaStream_t)stream);
    return run_solve(s, p12, f12, *o, (cudaStream_t)stream);
}

extern "C" int splitsart_solve_os(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts* o,
                                  const splitsart_os_opts* os, void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_solve_os");
    if (!s || !o || !os) return fail(SPLITSART_ERR_ARG, "solve_os: NULL argument");
    if ((s->Mh > 0 && !p12) || (s->Nh > 0 && !f12)) return fail(SPLITSART_ERR_ARG, "solve_os: NULL vector");
    if (o->max_iters < 0 || o->max_iters > 500000)
        return fail(SPLITSART_ERR_ARG, "solve_os: max_iters must be in [0, 500000]");
    if (!(o->lambda > 0.0) || !std::isfinite(o->lambda)) return fail(SPLITSART_ERR_ARG, "solve_os: lambda must be > 0");
    if (!(o->tol >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve_os: tol must be >= 0");
    if (o->check_every < 0) return fail(SPLITSART_ERR_ARG, "solve_os: check_every must be >= 0");
    if (!(o->timeout_ms >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve_os: timeout_ms must be >= 0");
    s->last = (cudaStream_t)stream;
    return run_solve_os(s, p12, f12, *o, *os, (cudaStream_t)stream);
}

extern "C" int splitsart_solve_cgls(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts* o,
                                    void* stream) {
    splitsart::NvtxRange nvtx_range("splitsart_solve_cgls");
    if (!s || !o) return fail(SPLITSART_ERR_ARG, "solve_cgls: NULL argument");
    if ((s->Mh > 0 && !p12) || (s->Nh > 0 && !f12)) return fail(SPLITSART_ERR_ARG, "solve_cgls: NULL vector");
    if (o->max_iters < 0 || o->max_iters > 500000)
        return fail(SPLITSART_ERR_ARG, "solve_cgls: max_iters must be in [0, 500000]");
    if (!(o->tol >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve_cgls: tol must be >= 0");
    if (o->check_every < 0) return fail(SPLITSART_ERR_ARG, "solve_cgls: check_every must be >= 0");
    if (!(o->timeout_ms >= 0.0)) return fail(SPLITSART_ERR_ARG, "solve_cgls: timeout_ms must be >= 0");
    s->last = (cudaStream_t)stream;
    return run_solve_cgls(s, p12, f12, *o, (cudaStream_t)stream);
}

extern "C" int splitsart_solve_result(splitsart_system* s, splitsart_solve_info* info) {
    if (!s || !info) return fail(SPLITSART_ERR_ARG, "solve_result: NULL argument");
    cudaError_t e = cudaStreamSynchronize(s->last);
    if (e != cudaSuccess) return cuda_fail(e, "solve_result: sync");
    LaunchCtl ctl;
    SolveResultDev r;
    if ((e = cudaMemcpy(&ctl, s->ctl, sizeof ctl, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(&r, s->result, sizeof r, cudaMemcpyDeviceToHost)))
        return cuda_fail(e, "solve_result: read");
    info->iters = r.iters;
    info->rho = r.rho;
    info->rr = r.rr;
    info->pp = r.pp;
    info->status = ctl.err != 0 ? ctl.err : r.status;
    if (ctl.err != 0) {
        info->iters = -1;
        return fail(ctl.err, "solve: a grid-barrier wait ran out (barrier %d); the result is invalid", ctl.err_where);
    }
    return SPLITSART_OK;
}
