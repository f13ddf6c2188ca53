// Internal layout of a folded system on the device. Shared by the library's
// translation units; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "host_common.h"

namespace splitsart {

struct LaunchCtl;

// Device-side counters written by the fold.
struct FoldStats {
    long long S;            // folded pattern size
    long long empty_rows;   // folded rows without entries
    long long exact_zeros;  // a1 == 0 by cancellation
    long long pad;
    int n_nzr;              // rows with entries
    int n_nzc;              // columns with entries
    int n_zr;               // rows without entries
    int max_row;            // longest folded row
    int max_col;            // longest folded column
    int pad3[3];
};

// Result of one solve, written by CTA 0 of the persistent launch.
struct SolveResultDev {
    int iters;
    int status;
    double rho, rr, pp;
};

// Upper bound on grid-reduction partials (CTAs of one persistent launch).
constexpr int kMaxCtas = 4096;

// Where each slice of a system lives in the global index spaces. A system
// built from one geometry has one slice. A batch concatenates several
// independent slices into one block-diagonal folded system.
struct SliceMap {
    int ns;
    const long long* rows;  // [ns+1] prefix of Mh_s: folded rows
    const long long* cols;  // [ns+1] prefix of Nh_s: folded columns
    const long long* M;     // [ns+1] prefix of M_s: full projection vectors
    const long long* N;     // [ns+1] prefix of N_s: full images
    const int* nx;          // [ns] 0 when the slice came from a CSR
    const int* nz;          // [ns]
};

// A folded system re-indexed for the pipelined streaming solve (stream.cu):
// rows and columns are renumbered in compacted order (only those with
// entries), so the hot loop never looks an index up. Two storages:
// - explicit: the folded CSR/CSC pairs (a1, a2) themselves, 12 bytes per entry
//   per pass in FP32;
// - implicit: each entry of the half rows of A stored once, as the compacted
//   folded column (row) with A1's sign in bit 31 and its one length w:
//   a1 = +-w, a2 = w, 8 bytes per entry per pass in FP32. A ray and its mirror
//   through the same folded cell give two entries (+w, then -w').
struct StreamFmt {
    int built = 0;
    void* alloc = nullptr;
    int32_t* rp = nullptr;   // [n_nzr + 1] compacted-row pointers
    int32_t* ci = nullptr;   // CSR indices: compacted columns (implicit: A1's sign in bit 31)
    const void* cv = nullptr;  // CSR values: pairs (explicit) or single values (implicit)
    int32_t* cp = nullptr;   // [n_nzc + 1] compacted-column pointers
    int32_t* ri = nullptr;   // CSC indices: compacted rows (implicit: A1's sign in bit 31)
    const void* rv = nullptr;  // CSC values
    void* ir = nullptr;      // [n_nzr] 1/R as applied, compacted
    float2* sc = nullptr;    // [n_nzr] row scales of BF16/FP16 codes, compacted
    void* ic = nullptr;      // [n_nzc] 1/C as applied, compacted
    void* pc = nullptr;      // [n_nzr] pairs: p of the launch, compacted
    void* uc = nullptr;      // [n_nzr] pairs: u
    void* fc = nullptr;      // [n_nzc] pairs: f of the launch, compacted
    double* rr = nullptr;    // [n_nzr] per-row residual^2 (batch stop tests)
    int32_t* qs = nullptr;   // [ns + 1] first compacted row of each slice
    int32_t* cs = nullptr;   // [n_nzc] slice of each compacted column
    double* pz = nullptr;    // [ns] ||p||^2 of each slice's empty rows (per launch)
    // Chunk plans of the ring kernels (ring.cu), made on their first use for a
    // chunk entry target: chunk c of pass k is rows (k = 0) or columns (k = 1)
    // [desc[k][c].x, desc[k][c + 1].x), whose entries start at desc[k][c].y.
    int ring_E = 0;                  // entry target of the plans (0: none yet)
    int ring_nch[2] = {0, 0};        // chunks per pass
    int ring_len[2] = {0, 0};        // longest row, longest column
    int2* ring_desc[2] = {nullptr, nullptr};
    void* ring_alloc = nullptr;
};

// Per-slice solve state of a batch launch.
struct SliceSolve {
    int iters;
    int done;
    double rho, rr, pp;
};

}  // namespace splitsart

struct splitsart_system {
    int64_t M = 0, N = 0, Mh = 0, Nh = 0, nnz_half = 0;
    int ns = 1;  // slices
    std::vector<long long> h_rows, h_cols, h_M, h_N;  // host copies of the slice prefixes
    std::vector<int> h_nx, h_nz;
    int dtype = 0;
    int nx = 0, nz = 0;
    int64_t S = -1;  // host copy, read lazily
    int64_t device_bytes = 0;
    cudaStream_t last = nullptr;
    bool have_stats = false;  // host copy of the fold statistics (identical across refolds)
    splitsart::FoldStats hstats{};

    // Uploaded first-half rows of A (FP64).
    int64_t* hrp = nullptr;
    int32_t* hcol = nullptr;
    double* hval = nullptr;

    // Folded CSR (capacity nnz_half; used length S).
    int32_t* rp = nullptr;   // Mh + 1
    int32_t* col = nullptr;  // S
    void* val = nullptr;     // S pairs, storage by dtype
    // Folded CSC.
    int32_t* cp = nullptr;   // Nh + 1
    int32_t* row = nullptr;  // S
    void* valT = nullptr;    // S pairs
    // Normalisers: raw absolute sums (double2) and reciprocals (storage by dtype).
    double2* Rsum = nullptr;  // Mh
    double2* Csum = nullptr;  // Nh
    void* invR = nullptr;     // Mh pairs
    void* invC = nullptr;     // Nh pairs
    float2* scale = nullptr;  // Mh (BF16/F16 only)
    float2* wR = nullptr;     // Mh (BF16/F16 only): fl32(scale / R), as the iteration applies it
    float2* wC = nullptr;     // Nh (BF16/F16 only): fl32(1 / C)

    // Compacted index lists (entries of empty rows/columns are skipped by the solve).
    int32_t* nzr = nullptr;   // rows with entries, increasing (n_nzr)
    int32_t* nzrp = nullptr;  // rp of those rows, plus S at the end (n_nzr + 1)
    int32_t* zr = nullptr;    // rows without entries (n_zr)
    int32_t* nzc = nullptr;   // columns with entries (n_nzc)
    int32_t* nzcp = nullptr;  // cp of those columns, plus S at the end (n_nzc + 1)

    // Slice map (device).
    long long* sl_rows = nullptr;
    long long* sl_cols = nullptr;
    long long* sl_M = nullptr;
    long long* sl_N = nullptr;
    int* sl_nx = nullptr;
    int* sl_nz = nullptr;
    splitsart::SliceSolve* sl_solve = nullptr;  // [ns]
    double* rr_row = nullptr;                   // [Mh] per-row residual^2 (batch solves)
    int* ndone = nullptr;                       // slices finished (batch solves)

    // Scratch.
    int32_t* cnt = nullptr;          // max(Mh, Nh) + 1 counters
    int32_t* flags = nullptr;        // max(Mh, Nh) + 1 scan scratch
    int32_t* scan_tmp = nullptr;     // block sums of the scan
    splitsart::FoldStats* stats = nullptr;
    void* u12 = nullptr;             // Mh pairs (vector type)
    void* tmp_f12 = nullptr;         // Nh pairs (vector type), projection
    void* tmp_q12 = nullptr;         // Mh pairs (vector type), projection
    double* partials = nullptr;      // 2 * kMaxCtas
    splitsart::LaunchCtl* ctl = nullptr;
    splitsart::SolveResultDev* result = nullptr;
    void* base = nullptr;            // single device allocation holding all of the above

    // Row plan of the shared-memory-resident solve, built on its first use for a
    // grid of res_G CTAs and a row weight (the rows do not change across refolds).
    int res_G = 0;
    int res_weight = -1;
    std::vector<int32_t> res_ptr;  // host copy of the compacted row pointers
    int32_t* res_rows = nullptr;   // [n_nzr] compacted row positions, in CTA order
    int32_t* res_off = nullptr;    // [G + 1] start of each CTA's group in res_rows
    int32_t* res_loc = nullptr;    // [n_nzr + G] per group: local entry offsets of its rows, then its total
    long long res_row_bytes = 0;   // the largest CTA's shared-memory bytes for its rows
    void* res_alloc = nullptr;     // device allocation of the plan

    // Detector bins of a single-slice system folded from acquisition parameters
    // (0 otherwise): the rows of one folded view pair.
    int nb = 0;

    // Ordered-subsets tables (os_sart.cu), built on the first ordered-subsets
    // solve for a subset size and kept: a refold rebuilds the same pattern and
    // values from the same uploaded half rows.
    int os_rows = 0;                // folded rows per subset of the tables below (0: none yet)
    int os_T = 0;                   // subsets
    int32_t* os_qr = nullptr;       // [T + 1] compacted-row range of each subset
    int32_t* os_off = nullptr;      // [(T + 1) x n_nzc] start of each subset's entries in each compacted column
    void* os_invC = nullptr;        // [T x n_nzc] pairs 1/C_t (vector type), 0 where C_t = 0
    void* os_alloc = nullptr;       // device allocation of the tables

    // Conjugate-gradient work vectors (cgls.cu), allocated on the first CGLS solve.
    void* cg_alloc = nullptr;

    // Compacted streaming formats (stream.cu): [0] explicit, [1] implicit,
    // each built on its first use and kept.
    splitsart::StreamFmt st[2];
};

namespace splitsart {
// The iterations at which a solve tests rho: every check_every-th (0 means 1).
// With tol = 0 only an exactly zero residual could stop the solve before
// max_iters, and from then on f no longer changes, so rho is tested only at
// k = 0 (where p = 0 still stops at once) and at k = max_iters.
inline int effective_check_every(const splitsart_solve_opts& o) {
    if (o.tol == 0.0 && o.max_iters > 0) return o.max_iters;
    return o.check_every > 0 ? o.check_every : 1;
}
inline SliceMap slice_map(const splitsart_system* s) {
    return SliceMap{s->ns, s->sl_rows, s->sl_cols, s->sl_M, s->sl_N, s->sl_nx, s->sl_nz};
}
// Defined in fold.cu.
int run_fold(splitsart_system* s, cudaStream_t st);
int run_fold_rhs(const splitsart_system* s, const void* p, void* p12, cudaStream_t st);
int run_fold_image(const splitsart_system* s, const void* f, int layout, void* f12, cudaStream_t st);
int run_recombine(const splitsart_system* s, const void* f12, void* f, int layout, cudaStream_t st);
int run_project(splitsart_system* s, const void* f, int layout, void* p, cudaStream_t st);
// Defined in sart.cu.
int run_solve(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st);
int cuda_fail(cudaError_t e, const char* what);
// Defined in api.cu: the fold statistics on the host (one synchronisation on first use).
int system_host_stats(splitsart_system* s, FoldStats* out);
// Defined in os_sart.cu and cgls.cu.
int run_solve_os(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o,
                 const splitsart_os_opts& os, cudaStream_t st);
int run_solve_cgls(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st);
int run_solve_stream(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st);
// Defined in stream.cu: build compacted format `kind` (0 explicit, 1 implicit) of s once.
int stream_format(splitsart_system* s, int kind, cudaStream_t st);
// Defined in ring.cu: solve kernels 7 and 8.
int run_solve_ring(splitsart_system* s, const void* p12, void* f12, const splitsart_solve_opts& o, cudaStream_t st);
// Defined in fold.cu: the implicit fold of the half rows (entry d of half row i
// at hrp[i] + d, in the fold's merged column order), as global folded columns
// with A1's sign in bit 31 and FP64 or FP32 lengths.
int run_implicit_rows(const splitsart_system* s, bool fp64, int32_t* col, void* val, cudaStream_t st);
// Defined in fold.cu: exclusive scan of in[0..n) into out[0..n] (out[n] = total);
// tile_sums holds n / 4096 + 2 ints.
int scan_exclusive(const int32_t* in, int32_t* out, int32_t* tile_sums, int64_t n, cudaStream_t st);
}  // namespace splitsart
