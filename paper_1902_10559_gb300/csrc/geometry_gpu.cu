// Device geometry: the first Mh rows of A for many slices at once, traced on
// the GPU with one thread per ray.
//
// The rays, cells and lengths are those of the host tracer (geometry.cpp),
// bit for bit (Section 2: symmetric sources, vertical snake numbering; only
// rows i < M/2 are traced, Eq. (2) gives the rest):
// - the acquisition (sizes, source positions) comes from the same host
//   function, so both tracers start from the same bits;
// - this file is compiled with -fmad=false, so every FP64 expression rounds
//   like the host's (compiled with -ffp-contract=off); the only functions used
//   are floor, lround and sqrt, which are exact or correctly rounded;
// - each ray's crossings are generated in the host's order and merged by the
//   same two-way rule; a piece's cell is the cell of its midpoint.
// Rows are then put in (index, length) order and equal indices merged, as the
// host does after its sort.
//
// Passes: count (trace without writing), an exclusive scan on the host,
// fill (trace and write, in traversal order), order-and-merge per row, and a
// compaction that runs only when a merge removed entries. The columns and
// lengths stay in device memory, shared by the call's geometries; their row
// pointers go to the host. The fold copies the rows on the device, and
// splitsart_geometry_export copies them to the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "host_common.h"

namespace splitsart {

int cuda_fail(cudaError_t e, const char* what);

namespace {

struct SliceGeo {
    int nx, nz, nb, K;
    double W, H, z0, ddx, ddz, D;
    long long ray0;  // first ray of this slice in the global ray numbering
    int src0;        // first source of this slice in the source arrays
    int pad;
};

// std::min / std::max semantics (the first argument on ties).
__device__ __forceinline__ double dmin(double a, double b) { return b < a ? b : a; }
__device__ __forceinline__ double dmax(double a, double b) { return a < b ? b : a; }
__device__ __forceinline__ int clampi(double v, int hi) {
    const int k = static_cast<int>(floor(v));
    return k < 0 ? 0 : (k > hi ? hi : k);
}
__device__ __forceinline__ double xplane(const SliceGeo& g, int c) { return (2.0 * c - g.nx) * g.W / (2.0 * g.nx); }
__device__ __forceinline__ double zplane(const SliceGeo& g, int r) { return g.z0 + r * g.ddz; }
__device__ __forceinline__ int32_t snake(const SliceGeo& g, int c, int r) {
    return c * g.nz + ((c & 1) ? (g.nz - 1 - r) : r);
}

// Trace S -> T; emit(j, length) for each piece, in traversal order.
template <class Emit>
__device__ void trace_ray(const SliceGeo& g, double sx, double sz, double tx, double tz, Emit& emit) {
    const double dx = tx - sx, dz = tz - sz;
    const double L = sqrt(dx * dx + dz * dz);
    const double xlo = xplane(g, 0), xhi = xplane(g, g.nx);
    const double zlo = zplane(g, 0), zhi = zplane(g, g.nz);

    double amin, amax;
    const double az0 = (zlo - sz) / dz, az1 = (zhi - sz) / dz;
    if (dx == 0.0) {
        if (sx < xlo || sx > xhi) return;
        amin = dmax(0.0, dmin(az0, az1));
        amax = dmin(1.0, dmax(az0, az1));
    } else {
        const double ax0 = (xlo - sx) / dx, ax1 = (xhi - sx) / dx;
        amin = dmax(dmax(0.0, dmin(ax0, ax1)), dmin(az0, az1));
        amax = dmin(dmin(1.0, dmax(ax0, ax1)), dmax(az0, az1));
    }
    if (!(amax > amin)) return;

    // Crossings strictly inside (amin, amax), in increasing a: the planes in
    // ascending order, or descending when the direction is negative. The host
    // tests every plane. Here a is the same expression, and it is monotone
    // along that order (each step of it rounds monotonically), so the planes
    // with a > amin are a suffix, found by bisection, and those with a < amax
    // a prefix: the walk starts at the suffix and ends at the first a >= amax.
    // The crossings are the host's, in the host's order, with fewer divisions.
    const int stx = dx < 0.0 ? -1 : 1, stz = dz < 0.0 ? -1 : 1;
    const int cx0 = dx < 0.0 ? g.nx : 0, rz0 = dz < 0.0 ? g.nz : 0;
    auto a_x = [&](int q) { return (xplane(g, cx0 + stx * q) - sx) / dx; };
    auto a_z = [&](int q) { return (zplane(g, rz0 + stz * q) - sz) / dz; };
    auto first_above = [&](auto&& a_of, int n) {  // first q in [0, n) with a_of(q) > amin, or n
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a_of(mid) > amin) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    };
    const int nqx = dx != 0.0 ? g.nx + 1 : 0, nqz = g.nz + 1;
    int qx = first_above(a_x, nqx), qz = first_above(a_z, nqz);
    double ax = 0.0, az = 0.0;
    auto next_x = [&]() {
        if (qx >= nqx) return false;
        const double a = a_x(qx++);
        if (!(a < amax)) {
            qx = nqx;
            return false;
        }
        ax = a;
        return true;
    };
    auto next_z = [&]() {
        if (qz >= nqz) return false;
        const double a = a_z(qz++);
        if (!(a < amax)) {
            qz = nqz;
            return false;
        }
        az = a;
        return true;
    };

    // A vertical ray on a boundary plane gives half its length to each side.
    bool on_plane = false;
    int split_lo = 0;
    if (dx == 0.0) {
        const int cb = static_cast<int>(lround((sx - xlo) / g.ddx));
        if (cb >= 0 && cb <= g.nx && xplane(g, cb) == sx) {
            on_plane = true;
            split_lo = cb - 1;
        }
    }

    bool hx = next_x(), hz = next_z();
    double a0 = amin;
    for (;;) {
        double a1;
        if (hx && hz) {
            if (ax < az) {
                a1 = ax;
                hx = next_x();
            } else if (az < ax) {
                a1 = az;
                hz = next_z();
            } else {  // through a cell corner: one breakpoint
                a1 = ax;
                hx = next_x();
                hz = next_z();
            }
        } else if (hx) {
            a1 = ax;
            hx = next_x();
        } else if (hz) {
            a1 = az;
            hz = next_z();
        } else {
            a1 = amax;
        }
        const double da = a1 - a0;
        if (da > 0.0) {
            const double mid = 0.5 * (a1 + a0);
            const double zm = sz + mid * dz;
            const int r = clampi((zm - zlo) / g.ddz, g.nz - 1);
            const double len = da * L;
            if (on_plane) {
                for (int c = split_lo; c <= split_lo + 1; ++c)
                    if (c >= 0 && c < g.nx) emit(snake(g, c, r), 0.5 * len);
            } else {
                const double xm = sx + mid * dx;
                const int c = clampi((xm - xlo) / g.ddx, g.nx - 1);
                emit(snake(g, c, r), len);
            }
        }
        if (a1 == amax) break;
        a0 = a1;
    }
}

// The slice of global ray r (largest s with ray0[s] <= r).
__device__ __forceinline__ int slice_of(const long long* ray0, int ns, long long r) {
    int lo = 0, hi = ns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(ray0 + mid) <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <class Emit>
__device__ void trace_global_ray(const SliceGeo* geo, const long long* ray0, int ns, const double* srcx,
                                 const double* srcz, long long r, Emit& emit) {
    const SliceGeo g = geo[slice_of(ray0, ns, r)];
    const long long i = r - g.ray0;
    const int k = static_cast<int>(i / g.nb), b = static_cast<int>(i % g.nb);
    const double u = g.D * double(2 * b + 1 - g.nb) / (2.0 * g.nb);
    trace_ray(g, srcx[g.src0 + k], srcz[g.src0 + k], u, 0.0, emit);
}

struct CountEmit {
    int n = 0;
    __device__ void operator()(int32_t, double) { ++n; }
};
struct FillEmit {
    int32_t* col;
    double* val;
    long long o, end;  // the row's slot [o, end), sized by the count pass
    __device__ void operator()(int32_t j, double len) {
        if (o < end) {
            col[o] = j;
            val[o] = len;
        }
        ++o;
    }
};

__global__ void trace_count_kernel(const SliceGeo* geo, const long long* ray0, int ns, const double* srcx,
                                   const double* srcz, long long R, int32_t* cnt) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    CountEmit e;
    trace_global_ray(geo, ray0, ns, srcx, srcz, r, e);
    cnt[r] = e.n;
}

__global__ void trace_fill_kernel(const SliceGeo* geo, const long long* ray0, int ns, const double* srcx,
                                  const double* srcz, long long R, const long long* off, int32_t* col, double* val) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    FillEmit e{col, val, off[r], off[r + 1]};
    trace_global_ray(geo, ray0, ns, srcx, srcz, r, e);
}

// Put one row in (index, length) order and merge equal indices, in place.
// The ray walks the cell columns in one direction and, within a column, the
// cells in one direction, so two reversals leave a sorted row; the insertion
// sort that follows is then a single comparison per entry, and still sorts
// any other row exactly (a vertical ray on a cell boundary alternates two
// columns).
__global__ void order_merge_kernel(const SliceGeo* geo, const long long* ray0, int ns, long long R,
                                   const long long* off, const int32_t* cnt, int32_t* col, double* val,
                                   int32_t* mcnt) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int nz = geo[slice_of(ray0, ns, r)].nz;
    const int n = cnt[r];
    int32_t* c = col + off[r];
    double* v = val + off[r];
    auto reverse = [&](int a, int b) {  // [a, b)
        for (--b; a < b; ++a, --b) {
            const int32_t tc = c[a];
            c[a] = c[b];
            c[b] = tc;
            const double tv = v[a];
            v[a] = v[b];
            v[b] = tv;
        }
    };
    if (n > 1) {
        if (c[0] / nz > c[n - 1] / nz) reverse(0, n);
        for (int a = 0; a < n;) {
            const int cc = c[a] / nz;
            int b = a + 1;
            while (b < n && c[b] / nz == cc) ++b;
            if (b - a > 1 && c[a] > c[b - 1]) reverse(a, b);
            a = b;
        }
        for (int e = 1; e < n; ++e) {
            const int32_t kc = c[e];
            const double kv = v[e];
            int q = e - 1;
            while (q >= 0 && (c[q] > kc || (c[q] == kc && v[q] > kv))) {
                c[q + 1] = c[q];
                v[q + 1] = v[q];
                --q;
            }
            c[q + 1] = kc;
            v[q + 1] = kv;
        }
    }
    int m = 0;
    for (int e = 0; e < n; ++e) {
        if (m > 0 && c[m - 1] == c[e]) {
            v[m - 1] += v[e];
        } else {
            c[m] = c[e];
            v[m] = v[e];
            ++m;
        }
    }
    mcnt[r] = m;
}

__global__ void compact_rows_kernel(long long R, const long long* off, const long long* moff, const int32_t* col,
                                    const double* val, int32_t* col_out, double* val_out) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const long long src = off[r], dst = moff[r], n = moff[r + 1] - moff[r];
    for (long long e = 0; e < n; ++e) {
        col_out[dst + e] = col[src + e];
        val_out[dst + e] = val[src + e];
    }
}

// Device buffers of one call, freed on every exit unless released.
struct DevBufs {
    std::vector<void*> ptrs;
    ~DevBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
    void release(const void* p) {
        for (auto& q : ptrs)
            if (q == p) q = nullptr;
    }
    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// Exclusive scan of int32 counts into int64 offsets (n + 1 entries).
std::vector<long long> scan_counts(const std::vector<int32_t>& cnt) {
    std::vector<long long> off(cnt.size() + 1, 0);
    for (size_t i = 0; i < cnt.size(); ++i) off[i + 1] = off[i] + cnt[i];
    return off;
}

int trace_on_device(const splitsart_geometry_params* params, int n, cudaStream_t st,
                    std::vector<splitsart_geometry*>& geoms) {
    std::vector<SliceGeo> geo(n);
    std::vector<long long> ray0(n + 1, 0);
    std::vector<double> srcx, srcz;
    for (int s = 0; s < n; ++s) {
        const splitsart_geometry_params& p = params[s];
        Acquisition acq;
        const int rc = make_acquisition(p, acq);
        if (rc) return rc;
        SliceGeo& g = geo[s];
        g.nx = p.nx;
        g.nz = p.nz;
        g.nb = p.nb;
        g.K = p.K;
        g.W = p.W;
        g.H = p.H;
        g.z0 = p.z0;
        g.ddx = p.W / p.nx;
        g.ddz = p.H / p.nz;
        g.D = p.D;
        g.ray0 = ray0[s];
        g.src0 = (int)srcx.size();
        g.pad = 0;
        ray0[s + 1] = ray0[s] + acq.Mh;
        srcx.insert(srcx.end(), acq.srcx.begin(), acq.srcx.end());
        srcz.insert(srcz.end(), acq.srcz.begin(), acq.srcz.end());
        auto* h = new (std::nothrow) splitsart_geometry();
        if (!h) return fail(SPLITSART_ERR_NOMEM, "make_geometries_device: out of host memory");
        geoms.push_back(h);
        h->half.M = acq.M;
        h->half.N = acq.N;
        h->has_params = true;
        h->params = p;
    }
    const long long R = ray0[n];
    const unsigned threads = 128, blocks = (unsigned)((R + threads - 1) / threads);

    DevBufs d;
    SliceGeo* d_geo;
    long long *d_ray0, *d_off, *d_moff = nullptr;
    double *d_srcx, *d_srcz, *d_val, *d_val2 = nullptr;
    int32_t *d_cnt, *d_mcnt, *d_col, *d_col2 = nullptr;
    cudaError_t e;
    if ((e = d.alloc(&d_geo, n)) || (e = d.alloc(&d_ray0, n + 1)) || (e = d.alloc(&d_srcx, srcx.size())) ||
        (e = d.alloc(&d_srcz, srcz.size())) || (e = d.alloc(&d_cnt, R)) || (e = d.alloc(&d_mcnt, R)) ||
        (e = d.alloc(&d_off, R + 1)))
        return cuda_fail(e, "make_geometries_device: cudaMalloc");
    if ((e = cudaMemcpyAsync(d_geo, geo.data(), sizeof(SliceGeo) * n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(d_ray0, ray0.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(d_srcx, srcx.data(), sizeof(double) * srcx.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(d_srcz, srcz.data(), sizeof(double) * srcz.size(), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "make_geometries_device: upload");

    trace_count_kernel<<<blocks, threads, 0, st>>>(d_geo, d_ray0, n, d_srcx, d_srcz, R, d_cnt);
    if ((e = cudaGetLastError())) return cuda_fail(e, "make_geometries_device: count launch");
    std::vector<int32_t> cnt(R);
    if ((e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "make_geometries_device: read the counts");
    const std::vector<long long> off = scan_counts(cnt);
    const long long total = off[R];
    if ((e = d.alloc(&d_col, total)) || (e = d.alloc(&d_val, total)))
        return cuda_fail(e, "make_geometries_device: cudaMalloc of the rows");
    if ((e = cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (R + 1), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "make_geometries_device: upload the offsets");
    trace_fill_kernel<<<blocks, threads, 0, st>>>(d_geo, d_ray0, n, d_srcx, d_srcz, R, d_off, d_col, d_val);
    order_merge_kernel<<<blocks, threads, 0, st>>>(d_geo, d_ray0, n, R, d_off, d_cnt, d_col, d_val, d_mcnt);
    if ((e = cudaGetLastError())) return cuda_fail(e, "make_geometries_device: fill launch");
    std::vector<int32_t> mcnt(R);
    if ((e = cudaMemcpyAsync(mcnt.data(), d_mcnt, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "make_geometries_device: read the merged counts");
    const std::vector<long long> moff = scan_counts(mcnt);
    int32_t* col = d_col;
    double* val = d_val;
    if (moff[R] != total) {  // a merge removed entries: close the gaps
        if ((e = d.alloc(&d_moff, R + 1)) || (e = d.alloc(&d_col2, moff[R])) || (e = d.alloc(&d_val2, moff[R])))
            return cuda_fail(e, "make_geometries_device: cudaMalloc of the compacted rows");
        if ((e = cudaMemcpyAsync(d_moff, moff.data(), sizeof(long long) * (R + 1), cudaMemcpyHostToDevice, st)))
            return cuda_fail(e, "make_geometries_device: upload the merged offsets");
        compact_rows_kernel<<<blocks, threads, 0, st>>>(R, d_off, d_moff, d_col, d_val, d_col2, d_val2);
        if ((e = cudaGetLastError())) return cuda_fail(e, "make_geometries_device: compact launch");
        col = d_col2;
        val = d_val2;
    }
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "make_geometries_device: synchronise");
    auto rows = std::make_shared<DeviceRows>();
    rows->col = col;
    rows->val = val;
    d.release(col);
    d.release(val);
    for (int s = 0; s < n; ++s) {
        HalfCsr& h = geoms[s]->half;
        const long long r0 = ray0[s], r1 = ray0[s + 1], e0 = moff[r0], nnz = moff[r1] - e0;
        if (nnz >= INT32_MAX) return fail(SPLITSART_ERR_ARG, "make_geometries_device: slice %d has too many entries", s);
        h.row_ptr.resize(r1 - r0 + 1);
        for (long long i = r0; i <= r1; ++i) h.row_ptr[i - r0] = moff[i] - e0;
        geoms[s]->dev = rows;
        geoms[s]->dev_off = e0;
    }
    return SPLITSART_OK;
}

}  // namespace

DeviceRows::~DeviceRows() {
    cudaFree(col);
    cudaFree(val);
}

int device_rows_to_host(const DeviceRowsView& v, int32_t* col, double* val) {
    if (v.nnz == 0) return SPLITSART_OK;
    cudaError_t e;
    if ((e = cudaMemcpy(col, v.rows->col + v.off, sizeof(int32_t) * v.nnz, cudaMemcpyDeviceToHost)) ||
        (e = cudaMemcpy(val, v.rows->val + v.off, sizeof(double) * v.nnz, cudaMemcpyDeviceToHost)))
        return cuda_fail(e, "geometry_export: read the device rows");
    return SPLITSART_OK;
}

}  // namespace splitsart

using namespace splitsart;

extern "C" int splitsart_make_geometries_device(const splitsart_geometry_params* params, int n, void* stream,
                                                splitsart_geometry** out) {
    NvtxRange nvtx_range("splitsart_make_geometries_device");
    if (!params || !out || n < 1) return fail(SPLITSART_ERR_ARG, "make_geometries_device: NULL argument or n < 1");
    for (int s = 0; s < n; ++s) out[s] = nullptr;
    std::vector<splitsart_geometry*> geoms;
    int rc;
    try {
        rc = trace_on_device(params, n, (cudaStream_t)stream, geoms);
    } catch (const std::bad_alloc&) {
        rc = fail(SPLITSART_ERR_NOMEM, "make_geometries_device: out of host memory");
    }
    if (rc != SPLITSART_OK) {
        for (auto* g : geoms) delete g;
        return rc;
    }
    for (int s = 0; s < n; ++s) out[s] = geoms[s];
    return SPLITSART_OK;
}
