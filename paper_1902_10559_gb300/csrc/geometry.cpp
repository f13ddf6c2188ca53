// Host geometry: symmetric acquisition and Siddon intersection lengths.
//
// Section 2 of the paper:
// - the sources are pairwise symmetric about OZ;
// - the voxels are numbered by the vertical snake rule;
// - together these give w_{i,j} = w_{M-i+1,N-j+1} (Eq. 2).
// Only rows i < M/2 are traced. Eq. (2) makes the others redundant, and the
// fold never reads them.
//
// Ray model: Siddon's exact radiological path. The segment S + a (T - S),
// a in [0, 1], is cut at every cell boundary it crosses. The crossings are
// two monotone sequences, one for x-boundaries and one for z-boundaries, and
// a two-way merge walks them. The midpoint of each piece gives its cell.
// A ray lying exactly on a vertical boundary gives half its length to each
// of the two adjacent cells.
//
// Host code compiles with -ffp-contract=off, so that x86 and Arm give the
// same bits.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <thread>
#include <utility>

#include "host_common.h"

namespace splitsart {

namespace {

struct Grid {
    int nx, nz;
    double W, H, z0, ddx, ddz;
    double xplane(int c) const { return (2.0 * c - nx) * W / (2.0 * nx); }
    double zplane(int r) const { return z0 + r * ddz; }
    int32_t snake(int c, int r) const { return c * nz + ((c & 1) ? (nz - 1 - r) : r); }
};

inline int clampi(double v, int hi) {
    int k = static_cast<int>(std::floor(v));
    return k < 0 ? 0 : (k > hi ? hi : k);
}

// Trace S->T. Append (snake index, length) pairs to `out`, unsorted.
void trace(const Grid& g, double sx, double sz, double tx, double tz,
           std::vector<std::pair<int32_t, double>>& out, std::vector<double>& ax,
           std::vector<double>& az) {
    const double dx = tx - sx, dz = tz - sz;
    // A plain correctly rounded square root: the device tracer computes the
    // same expression and gets the same bits.
    const double L = std::sqrt(dx * dx + dz * dz);
    const double xlo = g.xplane(0), xhi = g.xplane(g.nx);
    const double zlo = g.zplane(0), zhi = g.zplane(g.nz);

    double amin, amax;
    const double az0 = (zlo - sz) / dz, az1 = (zhi - sz) / dz;  // dz != 0: sources lie above z = 0
    if (dx == 0.0) {
        if (sx < xlo || sx > xhi) return;
        amin = std::max(0.0, std::min(az0, az1));
        amax = std::min(1.0, std::max(az0, az1));
    } else {
        const double ax0 = (xlo - sx) / dx, ax1 = (xhi - sx) / dx;
        amin = std::max(std::max(0.0, std::min(ax0, ax1)), std::min(az0, az1));
        amax = std::min(std::min(1.0, std::max(ax0, ax1)), std::max(az0, az1));
    }
    if (!(amax > amin)) return;

    // Crossings strictly inside (amin, amax), in increasing order of a.
    ax.clear();
    az.clear();
    if (dx != 0.0) {
        for (int c = 0; c <= g.nx; ++c) {
            const double a = (g.xplane(c) - sx) / dx;
            if (a > amin && a < amax) ax.push_back(a);
        }
        if (dx < 0) std::reverse(ax.begin(), ax.end());
    }
    for (int r = 0; r <= g.nz; ++r) {
        const double a = (g.zplane(r) - sz) / dz;
        if (a > amin && a < amax) az.push_back(a);
    }
    if (dz < 0) std::reverse(az.begin(), az.end());

    // A vertical ray on a boundary plane gives half its length to each side.
    bool on_plane = false;
    int split_lo = 0;
    if (dx == 0.0) {
        const int cb = static_cast<int>(std::lround((sx - xlo) / g.ddx));
        if (cb >= 0 && cb <= g.nx && g.xplane(cb) == sx) {
            on_plane = true;
            split_lo = cb - 1;
        }
    }

    double a0 = amin;
    size_t ix = 0, iz = 0;
    for (;;) {
        double a1;
        const bool hx = ix < ax.size(), hz = iz < az.size();
        if (hx && hz) {
            if (ax[ix] < az[iz]) a1 = ax[ix++];
            else if (az[iz] < ax[ix]) a1 = az[iz++];
            else { a1 = ax[ix++]; ++iz; }  // through a cell corner: one breakpoint
        } else if (hx) {
            a1 = ax[ix++];
        } else if (hz) {
            a1 = az[iz++];
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
                    if (c >= 0 && c < g.nx) out.emplace_back(g.snake(c, r), 0.5 * len);
            } else {
                const double xm = sx + mid * dx;
                const int c = clampi((xm - xlo) / g.ddx, g.nx - 1);
                out.emplace_back(g.snake(c, r), len);
            }
        }
        if (a1 == amax) break;
        a0 = a1;
    }
}

}  // namespace

int make_acquisition(const splitsart_geometry_params& p, Acquisition& a) {
    if (p.nx <= 0 || p.nz <= 0 || p.K < 2 || p.nb <= 0 || !(p.W > 0) || !(p.H > 0) || !(p.R > 0) ||
        !(p.D > 0) || !(p.gamma_deg >= 0))
        return fail(SPLITSART_ERR_ARG, "make_geometry: sizes must be positive and K >= 2");
    if (p.nx % 2 != 0)
        return fail(SPLITSART_ERR_ODD_DIM, "make_geometry: nx=%d is odd; the snake mirror j <-> N-1-j needs nx even",
                    p.nx);
    const int64_t M = int64_t(p.K) * p.nb;
    if (M % 2 != 0)
        return fail(SPLITSART_ERR_ODD_DIM, "make_geometry: M = K*nb = %lld is odd; a ray would be its own mirror",
                    (long long)M);
    const int64_t N = int64_t(p.nx) * p.nz;
    if (N > INT32_MAX) return fail(SPLITSART_ERR_ARG, "make_geometry: N too large for int32 column indices");
    a.M = M;
    a.N = N;
    a.Mh = M / 2;
    // Sources: source K-1-k is the exact mirror of source k.
    a.srcx.assign(p.K, 0.0);
    a.srcz.assign(p.K, 0.0);
    const double gam = p.gamma_deg * (M_PI / 180.0);
    for (int k = 0; 2 * k + 1 <= p.K; ++k) {
        const double th = gam * (2 * k + 1 - p.K) / (p.K - 1);
        a.srcx[k] = p.R * std::sin(th);
        a.srcz[k] = p.R * std::cos(th);
        a.srcx[p.K - 1 - k] = -a.srcx[k];
        a.srcz[p.K - 1 - k] = a.srcz[k];
    }
    return SPLITSART_OK;
}

int build_half_rows(const splitsart_geometry_params& p, HalfCsr& h) {
    Acquisition acq;
    const int rc = make_acquisition(p, acq);
    if (rc) return rc;
    const int64_t M = acq.M, N = acq.N, Mh = acq.Mh;
    const std::vector<double>& srcx = acq.srcx;
    const std::vector<double>& srcz = acq.srcz;
    Grid g{p.nx, p.nz, p.W, p.H, p.z0, p.W / p.nx, p.H / p.nz};

    unsigned nthr = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (Mh < 4096) nthr = 1;
    std::vector<std::vector<int64_t>> cnt(nthr);
    std::vector<std::vector<int32_t>> cols(nthr);
    std::vector<std::vector<double>> vals(nthr);
    auto work = [&](unsigned t) {
        const int64_t i0 = Mh * t / nthr, i1 = Mh * (t + 1) / nthr;
        std::vector<std::pair<int32_t, double>> row;
        std::vector<double> ax, az;
        for (int64_t i = i0; i < i1; ++i) {
            const int k = static_cast<int>(i / p.nb), b = static_cast<int>(i % p.nb);
            const double u = p.D * double(2 * b + 1 - p.nb) / (2.0 * p.nb);
            row.clear();
            trace(g, srcx[k], srcz[k], u, 0.0, row, ax, az);
            std::sort(row.begin(), row.end());
            // Merge equal indices (never produced by a straight ray, kept for safety).
            int64_t n = 0;
            for (size_t e = 0; e < row.size(); ++e) {
                if (n > 0 && cols[t].back() == row[e].first) {
                    vals[t].back() += row[e].second;
                } else {
                    cols[t].push_back(row[e].first);
                    vals[t].push_back(row[e].second);
                    ++n;
                }
            }
            cnt[t].push_back(n);
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nthr; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();

    h.M = M;
    h.N = N;
    h.row_ptr.assign(1, 0);
    h.row_ptr.reserve(Mh + 1);
    size_t total = 0;
    for (unsigned t = 0; t < nthr; ++t) total += cols[t].size();
    h.col.clear();
    h.val.clear();
    h.col.reserve(total);
    h.val.reserve(total);
    for (unsigned t = 0; t < nthr; ++t) {
        for (int64_t c : cnt[t]) h.row_ptr.push_back(h.row_ptr.back() + c);
        h.col.insert(h.col.end(), cols[t].begin(), cols[t].end());
        h.val.insert(h.val.end(), vals[t].begin(), vals[t].end());
    }
    return SPLITSART_OK;
}

int check_half_csr(int64_t M, int64_t N, const int64_t* rp, const int32_t* col, const double* val) {
    if (M <= 0 || N <= 0) return fail(SPLITSART_ERR_ARG, "from_csr: M and N must be positive");
    if (M % 2 || N % 2) return fail(SPLITSART_ERR_ODD_DIM, "from_csr: M and N must be even (Section 2)");
    if (N > INT32_MAX) return fail(SPLITSART_ERR_ARG, "from_csr: N too large for int32 column indices");
    if (!rp || (rp[M / 2] > 0 && (!col || !val))) return fail(SPLITSART_ERR_ARG, "from_csr: NULL array");
    if (rp[0] != 0) return fail(SPLITSART_ERR_ARG, "from_csr: row_ptr[0] must be 0");
    for (int64_t i = 0; i < M / 2; ++i) {
        if (rp[i + 1] < rp[i]) return fail(SPLITSART_ERR_ARG, "from_csr: row_ptr decreases at row %lld", (long long)i);
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (col[e] < 0 || col[e] >= N)
                return fail(SPLITSART_ERR_ARG, "from_csr: column %d out of range in row %lld", col[e], (long long)i);
            if (e > rp[i] && col[e] <= col[e - 1])
                return fail(SPLITSART_ERR_ARG, "from_csr: columns not strictly increasing in row %lld", (long long)i);
            if (!std::isfinite(val[e]))
                return fail(SPLITSART_ERR_NONFINITE, "from_csr: non-finite value in row %lld", (long long)i);
        }
    }
    return SPLITSART_OK;
}

}  // namespace splitsart

using namespace splitsart;

extern "C" int splitsart_make_geometry(const splitsart_geometry_params* params, splitsart_geometry** out) {
    if (!params || !out) return fail(SPLITSART_ERR_ARG, "make_geometry: NULL argument");
    *out = nullptr;
    auto* g = new (std::nothrow) splitsart_geometry();
    if (!g) return fail(SPLITSART_ERR_NOMEM, "make_geometry: out of host memory");
    int st;
    try {
        st = build_half_rows(*params, g->half);
    } catch (const std::bad_alloc&) {
        st = fail(SPLITSART_ERR_NOMEM, "make_geometry: out of host memory");
    }
    if (st != SPLITSART_OK) {
        delete g;
        return st;
    }
    g->has_params = true;
    g->params = *params;
    *out = g;
    return SPLITSART_OK;
}

extern "C" int splitsart_make_geometry_from_csr(int64_t M, int64_t N, const int64_t* row_ptr_host,
                                                const int32_t* col_host, const double* val_host,
                                                splitsart_geometry** out) {
    if (!out) return fail(SPLITSART_ERR_ARG, "from_csr: NULL out");
    *out = nullptr;
    int st = check_half_csr(M, N, row_ptr_host, col_host, val_host);
    if (st != SPLITSART_OK) return st;
    auto* g = new (std::nothrow) splitsart_geometry();
    if (!g) return fail(SPLITSART_ERR_NOMEM, "from_csr: out of host memory");
    const int64_t Mh = M / 2, nnz = row_ptr_host[Mh];
    try {
        g->half.M = M;
        g->half.N = N;
        g->half.row_ptr.assign(row_ptr_host, row_ptr_host + Mh + 1);
        g->half.col.assign(col_host, col_host + nnz);
        g->half.val.assign(val_host, val_host + nnz);
    } catch (const std::bad_alloc&) {
        delete g;
        return fail(SPLITSART_ERR_NOMEM, "from_csr: out of host memory");
    }
    *out = g;
    return SPLITSART_OK;
}

extern "C" int splitsart_geometry_info(const splitsart_geometry* g, int64_t* M, int64_t* N, int64_t* nnz_half) {
    if (!g) return fail(SPLITSART_ERR_ARG, "geometry_info: NULL geometry");
    if (M) *M = g->half.M;
    if (N) *N = g->half.N;
    if (nnz_half) *nnz_half = g->half.row_ptr.back();
    return SPLITSART_OK;
}

extern "C" int splitsart_geometry_export(const splitsart_geometry* g, int64_t* rp, int32_t* col, double* val) {
    if (!g || !rp || !col || !val) return fail(SPLITSART_ERR_ARG, "geometry_export: NULL argument");
    std::memcpy(rp, g->half.row_ptr.data(), g->half.row_ptr.size() * sizeof(int64_t));
    if (g->dev) return device_rows_to_host(DeviceRowsView{g->dev.get(), g->dev_off, g->half.row_ptr.back()}, col, val);
    std::memcpy(col, g->half.col.data(), g->half.col.size() * sizeof(int32_t));
    std::memcpy(val, g->half.val.data(), g->half.val.size() * sizeof(double));
    return SPLITSART_OK;
}

extern "C" void splitsart_geometry_destroy(splitsart_geometry* g) { delete g; }
