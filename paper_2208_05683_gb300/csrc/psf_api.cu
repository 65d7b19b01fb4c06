// psf_api.cu -- C ABI (include/psf.h) and the host orchestration of one
// evaluation of Algorithm 2 on the GPU.
//
// An evaluation keeps every intermediate matrix in one device pool of
// (column, value) entries; each row reserves its exact entry count with one
// atomic add, so rows of a matrix are contiguous but not ordered in the pool
// (row r spans [rb[r], re[r])).  The host synchronizes twice: after the
// norms ||Z^i||_1 (the plan needs them) and at the end (to size the result).
// A pool that turns out too small is detected on the device; the phase is
// then repeated with the capacity the device asked for.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "psf_internal.h"

using namespace psf;
using namespace psf::host;

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

namespace psf {
namespace host {
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

// the device memory pool's release threshold is raised once per device
constexpr int kMaxPoolDevices = 64;
bool g_pool_configured[kMaxPoolDevices] = {};
std::mutex g_pool_mu;
Profile g_prof;
// Default: the bitmap map for every step.  psf_autotune measured it faster
// than the column table on the 2D Laplacian (exp, cos) and banded workloads,
// giant steps included, where its 24 resident warps per SM hide the gather
// latency better than the table map's 14.
std::atomic<double> g_table_crossover{1e300};
std::atomic<bool> g_batch_graph{true};
std::atomic<bool> g_batch_reuse{true};
std::atomic<int> g_far_shift{6};
std::atomic<long long> g_fail_admission{0};
std::atomic<double> g_dense_xover{kDenseXoverDefault};
std::atomic<int> g_row_bitmaps{1};
thread_local TuneRecorder* g_tune_rec = nullptr;

cudaError_t configure_mempool() {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool_configured[dev]) return cudaSuccess;
    cudaMemPool_t pool;
    err = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (err != cudaSuccess) return err;
    unsigned long long thr = ~0ull;  // keep freed blocks for reuse
    err = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (err != cudaSuccess) return err;
    g_pool_configured[dev] = true;
    return cudaSuccess;
}

int lsb_for_bound_host(double x) {
    unsigned long long bits;
    std::memcpy(&bits, &x, sizeof bits);
    int E = (int)((bits >> 52) & 0x7ff);
    int eref = E ? E - 1023 + 1 : -1022;
    int lsb = eref - kWindow;
    return lsb < kMinLsb ? kMinLsb : lsb;
}

RowView view_of(const psf_csr_t& m) { return RowView{m.rowptr, m.rowptr + 1, m.col, m.val}; }

int check_csr(const psf_csr_t* m, int n, const char* what) {
    if (!m) return fail(PSF_EINVAL, "%s: null matrix", what);
    if (m->n != n || m->n < 0 || m->nnz < 0) return fail(PSF_EINVAL, "%s: bad size n=%d nnz=%d", what, m->n, m->nnz);
    if (!m->rowptr || (m->nnz > 0 && (!m->col || !m->val)))
        return fail(PSF_EINVAL, "%s: null device array", what);
    return PSF_OK;
}


// ---- mailboxes of the read-backs (see psf_internal.h)
static std::mutex g_mbox_mu;
static std::vector<std::pair<void*, void*>> g_mbox_free;
std::pair<void*, void*> mailbox_take() {
    {
        std::lock_guard<std::mutex> g(g_mbox_mu);
        if (!g_mbox_free.empty()) {
            auto m = g_mbox_free.back();
            g_mbox_free.pop_back();
            return m;
        }
    }
    void* h = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&h, kMboxBytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return {nullptr, nullptr};
    }
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h);
        return {nullptr, nullptr};
    }
    return {h, d};
}
void mailbox_give(std::pair<void*, void*> m) {
    std::lock_guard<std::mutex> g(g_mbox_mu);
    g_mbox_free.push_back(m);
}
// Step records (bytes of device memory at src) to dst on the host, after
// the stream's work: through the mailbox when they fit, else a copy.
int read_stats(Work& w, void* dst, const void* src, size_t bytes) {
    if (w.mbox.first && bytes % 4 == 0 && bytes <= kMboxBytes - kMboxStats) {
        w.mbox_pending = true;
        CU(launch_export(src, static_cast<char*>(w.mbox.second) + kMboxStats, bytes, w.st));
        CU(cudaStreamSynchronize(w.st));
        w.mbox_pending = false;
        memcpy(dst, static_cast<char*>(w.mbox.first) + kMboxStats, bytes);
        return PSF_OK;
    }
    CU(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return PSF_OK;
}

// The control block (and the norm slots) to the host, after the stream's work.
int read_back(Work& w, Ctl& c, NormSlot* slots) {
    if (w.mbox.first) {
        char* hd = static_cast<char*>(w.mbox.second);
        w.mbox_pending = true;
        CU(launch_export(w.ctl.p, hd, sizeof(Ctl), w.st));
        if (slots) CU(launch_export(w.slots.p, hd + kMboxSlots, sizeof(NormSlot) * kMaxNorms, w.st));
        CU(cudaStreamSynchronize(w.st));
        w.mbox_pending = false;
        const char* hh = static_cast<const char*>(w.mbox.first);
        memcpy(&c, hh, sizeof(Ctl));
        if (slots) memcpy(slots, hh + kMboxSlots, sizeof(NormSlot) * kMaxNorms);
        return PSF_OK;
    }
    CU(cudaMemcpyAsync(&c, w.ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, w.st));
    if (slots) CU(cudaMemcpyAsync(slots, w.slots.p, sizeof(NormSlot) * kMaxNorms, cudaMemcpyDeviceToHost, w.st));
    CU(cudaStreamSynchronize(w.st));
    return PSF_OK;
}

// A phase whose pool overflowed is discarded and run again with a larger
// pool, so only the bits that hold whatever the pool size are reported then.
int status_to_code(int st) {
    if (st & kDevBadInput) return fail(PSF_EINVAL, "malformed CSR input (row pointers, column order or range, or non-finite value)");
    if (st & kDevTimeout) return fail(PSF_ETIMEOUT, "a bounded device wait expired");
    if (st & kDevPoolFull) return PSF_OK;
    if (st & kDevInternal) return fail(PSF_ECUDA, "internal error: a pool entry held a column outside the matrix");
    if (st & kDevNotConv) return fail(PSF_ENOTCONV, "Algorithm 1 reached its pass cap");
    return PSF_OK;
}

// Validate input matrices on the device and wait for the outcome: nothing
// indexes with an input's columns before this returns PSF_OK.
int validate_inputs(Work& w, std::initializer_list<const psf_csr_t*> ms) {
    for (const psf_csr_t* m : ms)
        if (m) CU(launch_validate(m->n, m->nnz, m->rowptr, m->col, m->val, w.C(), w.st));
    Ctl c;
    int rc = read_back(w, c, nullptr);
    if (rc) return rc;
    return status_to_code(c.status);
}


// Pool entries a warp takes at a time: about eight rows of the expected size.
unsigned long long arena_for(double row_len) {
    double a = 8.0 * row_len;
    if (a < 32.0) a = 32.0;
    if (a > 512.0) a = 512.0;
    return ((unsigned long long)a + 3ull) & ~3ull;
}

// Launch one product step into matrix slot `slot`, with Algorithm 1 when
// threshold > 0.
// wide_window: the previous evaluation's rows of this step spanned more
// columns than one bitmap chunk (kBitmapColumns), so the bitmap map's wide
// window is used.
// reuse_k > 0: the step is baby step k and row slot `slot` still holds the
// norm phase's Z^k; while no entry has been dropped (a device flag), the
// product is skipped and k_reuse_pass1 does the step on those rows.
int run_step(Work& w, const RowView* A, const RowView* B, const std::vector<AddTerm>& add,
             double threshold, double e_r, int maxit, int stat_index, size_t slot, RowView* out,
             NormSlot* absmax_slot = nullptr, double blen = 0.0, double alen = 0.0, int reuse_k = 0,
             unsigned long long reuse_fma = 0, double out_len = 0.0, bool wide_window = false,
             double fma_hint = 0.0) {
    if (add.size() > (size_t)kMaxAdd) return fail(PSF_ETOOBIG, "%zu addend terms (max %d)", add.size(), kMaxAdd);
    int *rb, *re;
    int rc = w.rows_for(slot, &rb, &re);
    if (rc) return rc;
    ProductArgs P{};
    P.n = w.n;
    if (A) {
        P.A = *A;
        P.B = *B;
    }
    P.nadd = (int)add.size();
    for (size_t t = 0; t < add.size(); ++t) P.add[t] = add[t];
    P.out_rb = rb;
    P.out_re = re;
    P.pool_col = w.pcol();
    P.pool_val = w.pval();
    P.ctl = w.C();
    const bool filt = threshold > 0.0;
    const double eps_g = filt ? threshold / (1.0 + e_r) : 0.0;
    P.filtering = filt ? 1 : 0;
    P.eps_g = eps_g;
    P.e_lsb = lsb_for_bound_host(eps_g);
    P.words = w.words.as<unsigned long long>();
    P.sticky = w.sticky.as<unsigned>();
    P.stat = stat_index >= 0 ? w.stats.as<StepStat>() + stat_index : nullptr;
    P.absmax_slot = absmax_slot;
    P.chunk_cols = w.chunk_cols;
    P.chunk_slots = w.chunk_slots;
    P.arena = arena_for(alen > 0.0 ? alen * (blen > 1.0 ? blen : 1.0) : 8.0 * (add.size() + 1));
    if (filt) {
        P.cand_col = w.cand_col.as<int>();
        P.cand_x = w.cand_x.as<unsigned long long>();
        P.cand_cap = w.ccap;
        P.cand_chunk = w.cand_chunk();
    }
    if (P.stat) CU(cudaMemcpyAsync(&P.stat->pool_start, &w.C()->pool_used, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToDevice, w.st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = g_prof.on || g_tune_rec;
    if (timed) {
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        CU(cudaEventRecord(e0, w.st));
    }
    // table map when a row folds many products (the crossover is tunable)
    const double work = alen > 0.0 ? alen * blen : 0.0;
    const bool table = use_table(w.slot_map, work);
    if (reuse_k > 0) P.skip_unless = &w.C()->dropped;
    // dense tiles for a product with at least dense_xover n^3 multiply-adds:
    // every product step when the crossover is 0; otherwise a step whose count
    // is known (the same step of the previous evaluation, or a single product
    // whose operands' mean row lengths give its expected count) and n >= 512
    // (below that either form takes a few tens of microseconds, and the dense
    // form's extra launches dominate)
    const double nd = (double)w.n;
    const double fma_est = fma_hint > 0.0 ? fma_hint : (w.dense_estimate ? work * nd : 0.0);
    const bool dense = A && reuse_k == 0 && w.n > 0 && w.n <= kDenseMaxN &&
                       (w.dense_xover == 0.0 ||
                        (w.n >= kDenseMinN && fma_est > 0.0 && fma_est >= w.dense_xover * nd * nd * nd));
    if (dense) {
        const size_t bytes = sizeof(double) * (size_t)w.n * (size_t)w.n;
        for (DevBuf& d : w.dense)
            if (!d.p) CU(d.alloc(bytes, w.st));
        CU(launch_dense_product(P, w.dense[0].as<double>(), w.dense[1].as<double>(), w.dense[2].as<double>(), w.st));
    } else {
        // the bitmap map marks B rows from their column bitmaps (built here,
        // one launch over B); the chunked test settings keep the column marks
        const int bm = g_row_bitmaps.load();
        if (A && !table && bm > 0 && w.bits_cap >= w.cap && w.chunk_cols <= 0 && w.chunk_slots <= 0 &&
            (bm == 2 || (alen >= kBitmapMinA && blen >= kBitmapMinB))) {
            CU(launch_row_bitmaps(w.n, *B, w.bhdr.as<int2>(), w.pool_bits.as<unsigned>(), w.st));
            P.bhdr = w.bhdr.as<int2>();
            P.bbits = w.pool_bits.as<unsigned>();
        }
        const bool cta = A && !table && (w.slot_map == 4 || (w.slot_map == 0 && use_cta(w.n, alen, blen)));
        CU(launch_product(P, table, w.st, out_len, wide_window || w.slot_map == 3, cta));
    }
    if (reuse_k > 0) {
        ReuseArgs R{};
        R.n = w.n;
        R.rb = rb;
        R.re = re;
        R.col = w.pcol();
        R.val = w.pval();
        R.k = reuse_k;
        R.eps_g = eps_g;
        R.e_lsb = P.e_lsb;
        R.fma = reuse_fma;
        R.words = P.words;
        R.sticky = P.sticky;
        R.cand_col = P.cand_col;
        R.cand_x = P.cand_x;
        R.cand_cap = P.cand_cap;
        R.cand_chunk = P.cand_chunk;
        R.ctl = w.C();
        R.stat = P.stat;
        CU(launch_reuse_pass1(R, w.st));
    }
    if (timed) {
        CU(cudaEventRecord(e1, w.st));
        if (g_tune_rec) {
            g_tune_rec->work.push_back(work);
            g_tune_rec->ev.emplace_back(e0, e1);
        } else {
            g_prof.ev.emplace_back(e0, e1);
        }
    }
    if (filt) {
        Alg1Args a{};
        a.n = w.n;
        a.rb = rb;
        a.re = re;
        a.col = w.pcol();
        a.val = w.pval();
        a.eps_g = eps_g;
        a.bound = eps_g * (1.0 + e_r);
        a.maxit = maxit;
        a.e_lsb = P.e_lsb;
        a.words = P.words;
        a.sticky = P.sticky;
        a.ctl = w.C();
        a.stat = P.stat;
        a.cand_col = P.cand_col;
        a.cand_x = P.cand_x;
        a.far_shift = g_far_shift.load(std::memory_order_relaxed);
        CU(launch_alg1(a, w.st));
    }
    *out = w.pooled(rb, re);
    return PSF_OK;
}

// Copy a canonical CSR input into the pool (4-entry aligned rows), as row
// slot `slot`; the product kernels read every B row and addend row there.
int pool_copy(Work& w, const psf_csr_t& m, size_t slot, RowView* out) {
    int *rb, *re;
    int rc = w.rows_for(slot, &rb, &re);
    if (rc) return rc;
    CU(launch_copy_rows(m.n, m.rowptr, m.col, m.val, rb, re, w.pcol(), w.pval(), w.C(),
                        arena_for(m.n > 0 ? (double)m.nnz / m.n : 1.0), w.st));
    *out = w.pooled(rb, re);
    return PSF_OK;
}

constexpr size_t kSlotZp = 60;  // row slot of the pooled copy of Z
constexpr size_t kSlotW = 61;   // row slot of W = Z Z (PSF_Z_SQUARE) when computed in the PS phase

// ctl->mark[i] <- the pool counter, in stream order
int mark_pool(Work& w, int i) {
    CU(cudaMemcpyAsync(&w.C()->mark[i], &w.C()->pool_used, sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                       w.st));
    return PSF_OK;
}

int make_result(Work& w, const RowView& M, psf_result_t* out, psf_result_s** made) {
    psf_result_s* r = new (std::nothrow) psf_result_s();
    if (!r) return fail(PSF_ENOMEM, "host allocation");
    r->n = w.n;
    r->stream = w.st;
    int rc = PSF_OK;
    do {
        cudaError_t e = cudaMallocAsync((void**)&r->rowptr, sizeof(int) * ((size_t)w.n + 1), w.st);
        if (e != cudaSuccess) {
            rc = fail(PSF_ENOMEM, "result rowptr: %s", cudaGetErrorString(e));
            break;
        }
        if (w.n > 0) {
            e = launch_scan_rows(w.n, M.rb, M.re, r->rowptr, w.C(), w.scan.as<long long>(), w.st);
        } else {
            e = cudaMemsetAsync(r->rowptr, 0, sizeof(int), w.st);
        }
        if (e != cudaSuccess) {
            rc = fail(PSF_ECUDA, "scan: %s", cudaGetErrorString(e));
            break;
        }
    } while (0);
    if (rc) {
        if (r->rowptr) cudaFreeAsync(r->rowptr, w.st);
        delete r;
        return rc;
    }
    *made = r;
    *out = r;
    return PSF_OK;
}

// Second half of make_result, after the host has read nnz_total.
int finish_result(Work& w, const RowView& M, psf_result_s* r, unsigned long long nnz) {
    if (nnz > (unsigned long long)INT32_MAX) return fail(PSF_ETOOBIG, "result has %llu entries (>= 2^31)", nnz);
    r->nnz = (long long)nnz;
    CU(cudaMallocAsync((void**)&r->col, sizeof(int) * (nnz ? nnz : 1), w.st));
    CU(cudaMallocAsync((void**)&r->val, sizeof(double) * (nnz ? nnz : 1), w.st));
    if (w.n > 0 && nnz) CU(launch_gather(w.n, M, r->rowptr, r->col, r->val, w.st));
    r->info.nnz = (int64_t)nnz;
    return PSF_OK;
}

void destroy_result(psf_result_s* r) {
    if (!r) return;
    if (r->owner) {  // views into a batch's storage, freed with its last result
        delete r;
        return;
    }
    if (r->rowptr) cudaFreeAsync(r->rowptr, r->stream);
    if (r->col) cudaFreeAsync(r->col, r->stream);
    if (r->val) cudaFreeAsync(r->val, r->stream);
    delete r;
}

int prepare(cudaStream_t st) {
    (void)st;
    CU(kernels_init());
    CU(configure_mempool());
    return PSF_OK;
}

}  // namespace host
}  // namespace psf

using namespace psf::host;

// ---------------------------------------------------------------- ABI
extern "C" {

int psf_version(void) { return (0 << 16) | 1; }

const char* psf_last_error(void) { return g_last_error.c_str(); }

int psf_series_create(const double* coeffs, int64_t m, int32_t s, double tol, uint32_t flags,
                      psf_series_t* out) {
    if (!out) return fail(PSF_EINVAL, "out is null");
    *out = nullptr;
    if (!coeffs || m < 1) return fail(PSF_EINVAL, "need at least one coefficient");
    if (m > 100000) return fail(PSF_ETOOBIG, "m = %lld coefficients (max 100000)", (long long)m);
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PSF_EINVAL, "tol must be finite and > 0");
    if (flags & ~(PSF_POLY | PSF_NOFILTER | PSF_Z_SUBMULT | PSF_Z_ESTIMATE | PSF_Z_SQUARE))
        return fail(PSF_EINVAL, "unknown flags 0x%x", flags);
    if ((flags & PSF_Z_SUBMULT) && (flags & PSF_Z_ESTIMATE))
        return fail(PSF_EINVAL, "PSF_Z_SUBMULT and PSF_Z_ESTIMATE exclude each other");
    if (s < 0 || s > PSF_MAX_Q) return fail(PSF_EINVAL, "s = %d out of [0, %d]", s, PSF_MAX_Q);
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(coeffs[i])) return fail(PSF_EINVAL, "coefficient %lld is not finite", (long long)i);
    psf_series_s* p = new (std::nothrow) psf_series_s();
    if (!p) return fail(PSF_ENOMEM, "host allocation");
    p->a.assign(coeffs, coeffs + m);
    if ((flags & PSF_Z_SQUARE) && split_even_odd(p->a, p->c, p->odd)) {
        delete p;
        return fail(PSF_EINVAL, "PSF_Z_SQUARE needs a series of only even or only odd powers");
    }
    p->tol = tol;
    p->flags = flags;
    p->s = s;
    *out = p;
    return PSF_OK;
}

int psf_series_set_param(psf_series_t series, int32_t key, double value) {
    if (!series) return fail(PSF_EINVAL, "null series");
    switch (key) {
        case PSF_PARAM_ER:
            if (!(value > 0.0) || !std::isfinite(value)) return fail(PSF_EINVAL, "e_r must be finite and > 0");
            series->e_r = value;
            return PSF_OK;
        case PSF_PARAM_ALG1_MAXIT:
            if (!(value >= 1.0) || value > 1e9) return fail(PSF_EINVAL, "maxit must be in [1, 1e9]");
            series->maxit = (int)value;
            return PSF_OK;
        case PSF_PARAM_KERNEL:
            if (!(value == 0.0 || value == 1.0 || value == 2.0 || value == 3.0 || value == 4.0))
                return fail(PSF_EINVAL, "kernel must be 0, 1, 2, 3 or 4");
            series->kernel = (int)value;
            return PSF_OK;
        case PSF_PARAM_CHUNK_COLS:
            if (!(value >= 0.0) || value > 1e9) return fail(PSF_EINVAL, "chunk columns out of range");
            series->chunk_cols = value > 0.0 && value < 32.0 ? 32 : (int)value;
            return PSF_OK;
        case PSF_PARAM_CHUNK_SLOTS:
            if (!(value >= 0.0) || value > 1e9) return fail(PSF_EINVAL, "chunk slots out of range");
            series->chunk_slots = (int)value;
            return PSF_OK;
        case PSF_PARAM_DENSE_XOVER:
            if (!(value == -1.0 || value >= 0.0)) return fail(PSF_EINVAL, "dense crossover must be -1 or >= 0");
            series->dense_xover = value;
            return PSF_OK;
        case PSF_PARAM_POOL_ENTRIES:
            if (!(value >= 0.0) || value > (double)INT32_MAX) return fail(PSF_EINVAL, "pool entries out of range");
            series->pool_hint = (unsigned long long)value;
            return PSF_OK;
        default:
            return fail(PSF_EINVAL, "unknown parameter key %d", key);
    }
}

int psf_series_destroy(psf_series_t series) {
    delete series;
    return PSF_OK;
}

int psf_plan(const double* coeffs, int64_t m, int32_t s, double tol, uint32_t flags, const double* norms,
             psf_info_t* info, double* zeta, double* sigma) {
    if (!coeffs || m < 1 || !norms || !info) return fail(PSF_EINVAL, "null argument or m < 1");
    if (m > 100000) return fail(PSF_ETOOBIG, "m = %lld coefficients (max 100000)", (long long)m);
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(PSF_EINVAL, "tol must be finite and > 0");
    if (s < 0 || s > PSF_MAX_Q) return fail(PSF_EINVAL, "s out of range");
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(coeffs[i])) return fail(PSF_EINVAL, "coefficient %lld is not finite", (long long)i);
    for (int i = 0; i <= ((flags & PSF_Z_SUBMULT) ? 1 : 10); ++i)
        if (!(norms[i] >= 0.0) || !std::isfinite(norms[i])) return fail(PSF_EINVAL, "norm z_%d must be finite and >= 0", i);
    std::vector<double> a(coeffs, coeffs + m);
    const bool square = flags & PSF_Z_SQUARE;
    bool odd = false;
    if (square) {
        std::vector<double> c;
        if (split_even_odd(a, c, odd))
            return fail(PSF_EINVAL, "PSF_Z_SQUARE needs a series of only even or only odd powers");
        a.swap(c);
        if (odd) tol = tol / norms[1];  // IEEE: infinite for ||Z||_1 = 0
    }
    Plan p;
    if (make_plan(a, tol, flags & PSF_POLY, flags & PSF_Z_SUBMULT, s, norms, p, square ? 2 : 1))
        return fail(PSF_ENOTCONV, "no truncation length within %zu coefficients (Eq. 34)", a.size());
    // the thresholds go to indices 2..q and 1+g..b-1 of arrays of
    // PSF_MAX_Q + 2 entries
    if ((zeta && p.q > PSF_MAX_Q + 1) || (sigma && p.b > PSF_MAX_Q + 2))
        return fail(PSF_ETOOBIG, "q = %d, b = %d: the thresholds do not fit arrays of PSF_MAX_Q + 2 entries "
                    "(pass NULL zeta and sigma for the rest of the plan)", p.q, p.b);
    std::memset(info, 0, sizeof *info);
    info->N = p.N;
    info->q = p.q;
    info->b = p.b;
    info->g = p.g;
    info->products = p.products + (square ? 1 + (int)odd : 0);
    for (int i = 0; i <= 10; ++i) info->z[i] = p.zz[(size_t)i];
    info->alpha10 = p.alpha10;
    info->trunc = p.trunc;
    info->budget = p.budget;
    if (zeta)
        for (int k = 0; k < PSF_MAX_Q + 2; ++k) zeta[k] = (k >= 2 && k <= p.q) ? p.zeta[(size_t)k] : 0.0;
    if (sigma)
        for (int j = 0; j < PSF_MAX_Q + 2; ++j) sigma[j] = (j >= 1 + p.g && j < p.b) ? p.sigma[(size_t)j] : 0.0;
    return PSF_OK;
}

int psf_norm1(const psf_csr_t* M, void* stream, double* out) {
    if (!M || !out) return fail(PSF_EINVAL, "null argument");
    int rc = check_csr(M, M->n, "M");
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = prepare(st))) return rc;
    if (M->n == 0) {
        *out = 0.0;
        return PSF_OK;
    }
    Work w;
    if ((rc = w.init(M->n, st, 1))) return rc;
    if ((rc = validate_inputs(w, {M}))) return rc;
    if ((rc = w.reset_pool((unsigned long long)M->nnz + 4ull * M->n + 2048ull * num_sms() * 8))) return rc;
    RowView v;
    if ((rc = mark_pool(w, 0)) || (rc = pool_copy(w, *M, 0, &v)) || (rc = mark_pool(w, 1))) return rc;
    NormSlot* slots = w.slots.as<NormSlot>();
    CU(launch_absmax(w.pval(), w.C(), 0, slots + 0, st));
    NormArgs na{};
    na.n = M->n;
    na.count = 1;
    na.pool_col = w.pcol();
    na.pool_val = w.pval();
    na.slots = slots;
    na.words = w.words.as<unsigned long long>();
    na.sticky = w.sticky.as<unsigned>();
    na.ctl = w.C();
    CU(launch_norms(na, st));
    Ctl c;
    NormSlot hs[kMaxNorms];
    if ((rc = read_back(w, c, hs))) return rc;
    if ((rc = status_to_code(c.status))) return rc;
    unsigned long long b = hs[0].result;
    std::memcpy(out, &b, sizeof b);
    return PSF_OK;
}

int psf_product_filter(const psf_csr_t* A, const psf_csr_t* B, int32_t nadd, const double* alphas,
                       const psf_csr_t* const* addends, double threshold, double e_r, int32_t maxit,
                       void* stream, psf_result_t* out) {
    if (!out) return fail(PSF_EINVAL, "out is null");
    *out = nullptr;
    if ((A == nullptr) != (B == nullptr)) return fail(PSF_EINVAL, "A and B must both be given or both be null");
    if (nadd < 0 || nadd > kMaxAdd) return fail(PSF_EINVAL, "nadd = %d out of [0, %d]", nadd, kMaxAdd);
    if (nadd > 0 && (!alphas || !addends)) return fail(PSF_EINVAL, "null addend arrays");
    if (!(threshold >= 0.0) || !std::isfinite(threshold)) return fail(PSF_EINVAL, "threshold must be finite and >= 0");
    if (threshold > 0.0 && (!(e_r > 0.0) || !std::isfinite(e_r))) return fail(PSF_EINVAL, "e_r must be > 0");
    if (maxit < 1) return fail(PSF_EINVAL, "maxit must be >= 1");
    int n = -1;
    if (A) n = A->n;
    for (int t = 0; t < nadd && n < 0; ++t)
        if (addends[t]) n = addends[t]->n;
    if (n < 0) return fail(PSF_EINVAL, "cannot infer n: no matrix given");
    int rc;
    if (A && ((rc = check_csr(A, n, "A")) || (rc = check_csr(B, n, "B")))) return rc;
    for (int t = 0; t < nadd; ++t) {
        if (addends[t] && (rc = check_csr(addends[t], n, "addend"))) return rc;
        if (!std::isfinite(alphas[t])) return fail(PSF_EINVAL, "alpha %d not finite", t);
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = prepare(st))) return rc;
    Work w;
    if ((rc = w.init(n, st, 1))) return rc;
    w.dense_xover = g_dense_xover.load();
    w.dense_estimate = true;  // one product: the operands' mean row lengths give its expected count
    CU(cudaMemsetAsync(w.stats.p, 0, sizeof(StepStat), st));
    if ((rc = validate_inputs(w, {A, B}))) return rc;
    for (int t = 0; t < nadd; ++t)
        if (addends[t] && (rc = validate_inputs(w, {addends[t]}))) return rc;
    const double blen = B && n > 0 ? (double)B->nnz / n : 0.0;
    unsigned long long est = (unsigned long long)n * 8ull + 16;
    for (int t = 0; t < nadd; ++t)
        if (addends[t]) est += (unsigned long long)addends[t]->nnz * 2ull + 4ull * n;
    if (A) {
        est += (unsigned long long)B->nnz + 4ull * n;
        est += (unsigned long long)A->nnz * (2ull + (unsigned long long)B->nnz / (unsigned long long)(n > 0 ? n : 1)) * 2ull;
    }
    RowView va, vb, res;
    if (A) va = view_of(*A);
    unsigned long long cap = est < kMaxPool ? est : kMaxPool;
    psf_result_s* r = nullptr;
    for (int attempt = 0;; ++attempt) {
        if ((rc = w.reset_pool(cap))) return rc;
        CU(cudaMemsetAsync(w.stats.p, 0, sizeof(StepStat), st));
        // B and the addend matrices are read from pooled copies
        std::vector<AddTerm> add;
        for (int t = 0; t < nadd; ++t) {
            AddTerm T{};
            T.alpha = alphas[t];
            if (addends[t]) {
                RowView mv;
                if ((rc = pool_copy(w, *addends[t], 2 + (size_t)t, &mv))) return rc;
                T.rb = mv.rb;
                T.re = mv.re;
                T.col = mv.col;
                T.val = mv.val;
            }
            add.push_back(T);
        }
        if (A && (rc = pool_copy(w, *B, 1, &vb))) return rc;
        if ((rc = run_step(w, A ? &va : nullptr, A ? &vb : nullptr, add, threshold, e_r, maxit, 0, 0, &res,
                           nullptr, blen, A && n > 0 ? (double)A->nnz / n : 0.0)))
            return rc;
        Ctl c;
        if ((rc = read_back(w, c, nullptr))) return rc;
        if ((rc = status_to_code(c.status))) return rc;
        if (c.status & kDevPoolFull) {
            if ((rc = w.clear_sums())) return rc;
            if (attempt > 8) return fail(PSF_ENOMEM, "pool kept overflowing");
            if (cap >= kMaxPool) return fail(PSF_ETOOBIG, "the step needs more than 2^31 - 2^20 pool entries");
            unsigned long long need = c.pool_used + c.pool_used / 4 + 1024;
            cap = need > 2 * cap ? need : 2 * cap;
            if (cap > kMaxPool) cap = kMaxPool;
            continue;
        }
        break;
    }
    psf_result_t handle;
    if ((rc = make_result(w, res, &handle, &r))) return rc;
    Ctl c;
    StepStat ss{};
    if ((rc = read_back(w, c, nullptr))) {
        destroy_result(r);
        return rc;
    }
    if (read_stats(w, &ss, w.stats.p, sizeof ss) != PSF_OK) {
        destroy_result(r);
        return fail(PSF_ECUDA, "stats read-back");
    }
    if ((rc = finish_result(w, res, r, c.nnz_total))) {
        destroy_result(r);
        return rc;
    }
    psf_step_info_t si{};
    si.kind = A ? 0 : 2;
    si.index = 0;
    si.threshold = threshold;
    si.nnz_pre = (int64_t)ss.nnz_pre;
    si.nnz_post = threshold > 0.0 ? (int64_t)ss.nnz_post : (int64_t)ss.nnz_pre;
    si.eps_f = threshold > 0.0 ? ss.eps_f : 0.0;
    si.iters = threshold > 0.0 ? ss.iters : 0;
    si.dropped = threshold > 0.0 ? ss.dropped : 0.0;
    si.fma = (int64_t)ss.fma;
    r->info.fma = (int64_t)ss.fma;
    if (g_prof.on) g_prof.fma += (double)ss.fma;
    r->steps.push_back(si);
    r->info.nsteps = 1;
    *out = r;
    return PSF_OK;
}

int psf_eval(psf_series_t series, const psf_csr_t* Z, void* stream, psf_result_t* out) {
    if (!out) return fail(PSF_EINVAL, "out is null");
    *out = nullptr;
    if (!series) return fail(PSF_EINVAL, "null series");
    int rc = check_csr(Z, Z ? Z->n : 0, "Z");
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = prepare(st))) return rc;
    const int n = Z->n;
    const bool submult = series->flags & PSF_Z_SUBMULT;
    const bool poly = series->flags & PSF_POLY;
    const bool nofilter = series->flags & PSF_NOFILTER;
    // PSF_Z_SQUARE: Algorithm 2 runs on W = Z Z with g's coefficients, and an
    // odd series ends with F = Z G-hat
    const bool square = series->flags & PSF_Z_SQUARE;
    const bool odd = square && series->odd;
    const int stride = square ? 2 : 1;
    const std::vector<double>& a = square ? series->c : series->a;

    Work w;
    if ((rc = w.init(n, st, 16))) return rc;
    if ((rc = validate_inputs(w, {Z}))) return rc;
    w.slot_map = series->kernel;
    w.dense_xover = series->dense_xover >= 0.0 ? series->dense_xover : g_dense_xover.load();
    // the column windows the series' previous evaluation measured (batches on
    // other threads may update them)
    std::vector<unsigned> span_z, span_baby, span_giant;
    {
        std::lock_guard<std::mutex> lock(series->span_mu);
        span_z = series->span_z;
        span_baby = series->span_baby;
        span_giant = series->span_giant;
    }
    w.chunk_cols = series->chunk_cols;
    w.chunk_slots = series->chunk_slots;
    const RowView vz = view_of(*Z);
    const double zlen = n > 0 ? (double)Z->nnz / n : 0.0;
    double znnz[kMaxNorms] = {0.0};  // nnz(Z^i) of this evaluation
    znnz[1] = (double)Z->nnz;
    NormSlot* slots = w.slots.as<NormSlot>();
    if (n > 0) {
        const size_t nb = sizeof(unsigned long long) * (size_t)kNormPieces * (size_t)n * 10;
        CU(w.nwords.alloc(nb, st));
        CU(cudaMemsetAsync(w.nwords.p, 0, nb, st));
    }

    // ---- Alg. 2 step 1: norms ||Z^i||_1, i <= 10 (Eq. 37): exact (the powers
    // Z^2..Z^10 are computed), or ||Z||^i, or ||Z||_1 exact and the others
    // estimated (a column of Z too long for the estimator: exact)
    double norms[kMaxNorms];
    norms[0] = 1.0;
    bool chain = !submult && n > 0;
    if ((series->flags & PSF_Z_ESTIMATE) && n > 0) {
        bool fallback = false;
        if ((rc = estimate_power_norms(w, *Z, norms, &fallback))) return rc;
        chain = fallback;
    }
    unsigned long long zcap = series->pool_hint;
    if (zcap < series->z_need + series->z_need / 8) zcap = series->z_need + series->z_need / 8;
    unsigned long long z_used = 0, z_fma = 0;
    // Once the series knows what its PS phase needs, the pool holds both
    // phases: the PS phase continues after the powers Z^2..Z^10, whose
    // leading ones double as baby steps while nothing is dropped.
    const unsigned long long ps_reserve =
        (series->ps_need > 0 && chain) ? series->ps_need + series->ps_need / 8 + 4096 : 0;
    RowView zp{}, zsq{};  // the pooled Z and, when the chain ran, Z^2
    unsigned long long zfma[kMaxNorms] = {0ull};  // multiply-adds of Z^i in the norm phase
    {
        unsigned long long est = (unsigned long long)Z->nnz * 256ull + (unsigned long long)n * 64ull + 4096ull;
        if (series->z_need == 0 && zcap < est) zcap = est;
        if (zcap > kMaxPool) zcap = kMaxPool;
        for (int attempt = 0;; ++attempt) {
            CU(cudaMemsetAsync(slots, 0, sizeof(NormSlot) * kMaxNorms, st));
            // the pooled Z and Z^2 .. Z^10, each delimited in the pool by counter
            // snapshots (the marks also give baby steps their powers' ranges)
            if (n > 0) {
                unsigned long long total = zcap + ps_reserve;
                if (total > kMaxPool) total = kMaxPool;
                if ((rc = w.reset_pool(total))) return rc;
                CU(cudaMemsetAsync(w.stats.p, 0, sizeof(StepStat) * 16, st));
                if ((rc = mark_pool(w, 0)) || (rc = pool_copy(w, *Z, kSlotZp, &zp)) || (rc = mark_pool(w, 1)))
                    return rc;
                CU(launch_absmax(w.pval(), w.C(), 0, slots + 1, st));
                // norms by row tiles: matrix 0 is the pooled Z, matrix i-1 is Z^i
                NormRowsArgs nr{};
                nr.n = n;
                nr.count = 1;
                nr.rb[0] = zp.rb;
                nr.re[0] = zp.re;
                nr.col = w.pcol();
                nr.val = w.pval();
                nr.slots = slots + 1;
                nr.words = w.nwords.as<unsigned long long>();
                nr.sticky = w.sticky.as<unsigned>();
                nr.ctl = w.C();
                if (chain) {
                    RowView prev = zp;
                    for (int i = 2; i <= 10; ++i) {
                        RowView cur;
                        double blen = (size_t)(i - 2) < series->len_z.size() ? series->len_z[(size_t)(i - 2)]
                                                                              : zlen * (i - 1) * (i - 1);
                        const bool wz = (size_t)(i - 2) < span_z.size() && span_z[(size_t)(i - 2)] > kBitmapColumns;
                        if ((rc = run_step(w, &vz, &prev, {}, 0.0, 0.0, 1, i - 2, (size_t)(i - 2), &cur,
                                           slots + i, blen, zlen, 0, 0ull, 0.0, wz)))
                            return rc;
                        if ((rc = mark_pool(w, i))) return rc;
                        if (i == 2) zsq = cur;
                        nr.rb[i - 1] = cur.rb;
                        nr.re[i - 1] = cur.re;
                        prev = cur;
                    }
                    nr.count = 10;
                }
                CU(launch_norms_rows(nr, st));
            }
            Ctl c;
            NormSlot hs[kMaxNorms];
            if ((rc = read_back(w, c, hs))) return rc;
            if ((rc = status_to_code(c.status))) return rc;
            if (c.status & kDevPoolFull) {
                if ((rc = w.clear_sums())) return rc;
                if (attempt > 8 || zcap >= kMaxPool)
                    return fail(PSF_ETOOBIG, "the powers Z^2..Z^10 need more than 2^31 - 2^20 pool entries; use PSF_Z_SUBMULT or PSF_Z_ESTIMATE");
                unsigned long long need = c.pool_used + c.pool_used / 4 + 4096;
                zcap = need > 2 * zcap ? need : 2 * zcap;
                if (zcap > kMaxPool) zcap = kMaxPool;
                continue;
            }
            z_used = c.pool_used;
            z_fma = c.fma_total;
            if (z_used > series->z_need) series->z_need = z_used;
            if (chain) {
                StepStat zs[9];
                if (read_stats(w, zs, w.stats.p, sizeof zs) != PSF_OK)
                    return fail(PSF_ECUDA, "stats read-back");
                series->len_z.assign(9, 0.0);
                std::vector<unsigned> sz(9, 0u);
                for (int i = 2; i <= 10; ++i) {
                    znnz[i] = (double)zs[i - 2].nnz_pre;
                    zfma[i] = zs[i - 2].fma;
                    series->len_z[(size_t)(i - 2)] = znnz[i - 1] / n;
                    sz[(size_t)(i - 2)] = zs[i - 2].span_max;
                }
                std::lock_guard<std::mutex> lock(series->span_mu);
                series->span_z = sz;
            }
            // ||Z||_1 always; Z^2..Z^10 when the chain ran (else estimated above)
            for (int i = 1; i <= (chain || submult ? 10 : 1); ++i) {
                unsigned long long bits = hs[i].result;
                std::memcpy(&norms[i], &bits, sizeof bits);
            }
            break;
        }
    }

    // ---- Alg. 2 steps 2-3 and the thresholds
    Plan p;
    // an odd series: ||f(Z) - Z G-hat||_1 <= ||Z||_1 ||g(W) - G-hat||_1 (IEEE: 1/0 = inf)
    const double tol_g = odd ? series->tol / norms[1] : series->tol;
    if (make_plan(a, tol_g, poly, submult, series->s, norms, p, stride))
        return fail(PSF_ENOTCONV, "no truncation length within %zu coefficients (Eq. 34)", a.size());
    if (p.q > PSF_MAX_Q) return fail(PSF_ETOOBIG, "q = %d exceeds %d", p.q, PSF_MAX_Q);
    const int N = p.N, q = p.q, b = p.b, g = p.g;
    const int stat_cap = q + b + 4;
    CU(w.stats.alloc(sizeof(StepStat) * (size_t)stat_cap, st));
    auto coef = [&](int idx) { return (idx < N && idx < (int)a.size()) ? a[(size_t)idx] : 0.0; };

    psf_result_s* r = nullptr;
    psf_result_t handle;
    RowView F;
    std::vector<psf_step_info_t> steps;
    unsigned long long eval_fma = z_fma;
    // mean row length of the k-th power of the matrix the scheme multiplies by
    auto pow_len = [&](int k) {
        const int e = k * stride;
        return (e <= 10 && znnz[e] > 0.0) ? znnz[e] / n : zlen * e * e;
    };
    if ((N == 1 && !odd) || n == 0) {
        // f(Z) ~ a_0 I: no product (Eq. 5)
        r = new (std::nothrow) psf_result_s();
        if (!r) return fail(PSF_ENOMEM, "host allocation");
        r->n = n;
        r->stream = st;
        long long nnz = (a[0] != 0.0) ? n : 0;
        bool ok = cudaMallocAsync((void**)&r->rowptr, sizeof(int) * ((size_t)n + 1), st) == cudaSuccess &&
                  cudaMallocAsync((void**)&r->col, sizeof(int) * (size_t)(n > 0 ? n : 1), st) == cudaSuccess &&
                  cudaMallocAsync((void**)&r->val, sizeof(double) * (size_t)(n > 0 ? n : 1), st) == cudaSuccess;
        if (!ok) {
            destroy_result(r);
            return fail(PSF_ENOMEM, "result allocation");
        }
        if (nnz) {
            CU(launch_identity(n, a[0], r->rowptr, r->col, r->val, st));
        } else {
            CU(cudaMemsetAsync(r->rowptr, 0, sizeof(int) * ((size_t)n + 1), st));
        }
        r->nnz = nnz;
        handle = r;
    } else {
        // ---- steps 4-14 in one pool
        unsigned long long cap = series->pool_hint;
        if (cap < series->ps_need + series->ps_need / 8) cap = series->ps_need + series->ps_need / 8;
        unsigned long long est = 4ull * z_used + (unsigned long long)Z->nnz * 64ull + (unsigned long long)n * 64ull;
        if (series->ps_need == 0 && cap < est) cap = est;
        if (cap > kMaxPool) cap = kMaxPool;
        for (int attempt = 0;; ++attempt) {
            // attempt 0 continues in the norm phase's pool when it reserved
            // room; a retry after an overflow starts from an empty pool
            const bool reuse = attempt == 0 && ps_reserve > 0;
            const unsigned long long used_before = reuse ? z_used : 0ull;
            if (!reuse && (rc = w.reset_pool(cap))) return rc;
            CU(cudaMemsetAsync(w.stats.p, 0, sizeof(StepStat) * (size_t)stat_cap, st));
            steps.clear();
            int si = 0;
            std::vector<RowView> Zh((size_t)q + 2);
            if (reuse) {
                Zh[1] = zp;  // Z-hat_(1) = Z, pooled by the norm phase
            } else if ((rc = pool_copy(w, *Z, kSlotZp, &Zh[1]))) {
                return rc;
            }
            // the left factor of the baby steps: Z, or W = Z Z (unfiltered;
            // the norm phase's Z^2 when this pool still holds it)
            RowView vm = vz;
            if (square) {
                if (reuse) {
                    vm = zsq;
                } else if ((rc = run_step(w, &vz, &Zh[1], {}, 0.0, 0.0, 1, -1, kSlotW, &vm, nullptr, zlen, zlen))) {
                    return rc;
                }
                Zh[1] = vm;
            }
            // square mode keeps the norm phase's row slots 0..8 (W is slot 0)
            size_t slot = square ? 9 : 0;
            // baby steps: Z-hat_(k+1) = filter(Z Z-hat_(k)), threshold zeta_{k+1}
            for (int k = 1; k < q; ++k) {
                double thr = nofilter ? 0.0 : p.zeta[(size_t)k + 1];
                double blen = (size_t)(k - 1) < series->len_baby.size() ? series->len_baby[(size_t)(k - 1)]
                                                                         : pow_len(k);
                // baby step k + 1 writes row slot k - 1, the slot of the norm phase's Z^(k+1)
                const int rk = (reuse && !square && k + 1 <= 10 && slot == (size_t)(k - 1)) ? k + 1 : 0;
                const bool wb = (size_t)(k - 1) < span_baby.size() && span_baby[(size_t)(k - 1)] > kBitmapColumns;
                if ((rc = run_step(w, &vm, &Zh[(size_t)k], {}, thr, series->e_r, series->maxit, si, slot++,
                                   &Zh[(size_t)k + 1], nullptr, blen, pow_len(1), rk, rk ? zfma[rk] : 0ull, 0.0, wb)))
                    return rc;
                psf_step_info_t s{};
                s.kind = 0;
                s.index = k + 1;
                s.threshold = thr;
                steps.push_back(s);
                ++si;
            }
            auto block = [&](int i) {
                std::vector<AddTerm> add;
                if (q == 0 && coef(0) != 0.0) {  // N = 1 (odd series only): c_0 I
                    AddTerm T{};
                    T.alpha = coef(0);
                    add.push_back(T);
                }
                for (int j = 0; j < q; ++j) {
                    double alpha = coef(i * q + j);
                    if (alpha == 0.0) continue;
                    AddTerm T{};
                    T.alpha = alpha;
                    if (j >= 1) {
                        T.rb = Zh[(size_t)j].rb;
                        T.re = Zh[(size_t)j].re;
                        T.col = Zh[(size_t)j].col;
                        T.val = Zh[(size_t)j].val;
                    }
                    add.push_back(T);
                }
                return add;
            };
            // S-hat_0 = B-hat_{b-1} (not needed when g = 1: S_1 is a plain add)
            RowView S{};
            size_t sslot[2] = {slot, slot + 1};
            int cur = 0;
            if (g == 0) {
                if ((rc = run_step(w, nullptr, nullptr, block(b - 1), 0.0, 0.0, 1, si, sslot[cur], &S))) return rc;
                psf_step_info_t s{};
                s.kind = 2;
                s.index = 0;
                steps.push_back(s);
                ++si;
            }
            for (int i = 1; i < b; ++i) {
                std::vector<AddTerm> add = block(b - 1 - i);
                RowView nxt;
                int nslot = cur ^ 1;
                psf_step_info_t s{};
                s.index = i;
                if (g == 1 && i == 1) {
                    // B_{b-1} = a_{(b-1)q} I: S_1 = B-hat_{b-2} + a_{(b-1)q} Z-hat_(q), unfiltered
                    double alpha = coef((b - 1) * q);
                    if (alpha != 0.0) {
                        AddTerm T{};
                        T.alpha = alpha;
                        T.rb = Zh[(size_t)q].rb;
                        T.re = Zh[(size_t)q].re;
                        T.col = Zh[(size_t)q].col;
                        T.val = Zh[(size_t)q].val;
                        add.push_back(T);
                    }
                    if ((rc = run_step(w, nullptr, nullptr, add, 0.0, 0.0, 1, si, sslot[nslot], &nxt))) return rc;
                    s.kind = 2;
                } else {
                    double thr = nofilter ? 0.0 : p.sigma[(size_t)i];
                    double blen = (size_t)(i - 1) < series->len_giant.size()
                                      ? series->len_giant[(size_t)(i - 1)]
                                      : (znnz[10] > 0.0 ? znnz[10] / n : zlen * 100.0);
                    const double alen = pow_len(q);
                    const double olen =
                        (size_t)(i - 1) < series->out_giant.size() ? series->out_giant[(size_t)(i - 1)] : 0.0;
                    const bool wg = (size_t)(i - 1) < span_giant.size() && span_giant[(size_t)(i - 1)] > kBitmapColumns;
                    const double fh =
                        (size_t)(i - 1) < series->fma_giant.size() ? series->fma_giant[(size_t)(i - 1)] : 0.0;
                    if ((rc = run_step(w, &Zh[(size_t)q], &S, add, thr, series->e_r, series->maxit, si, sslot[nslot],
                                       &nxt, nullptr, blen, alen, 0, 0ull, olen, wg, fh)))
                        return rc;
                    s.kind = 1;
                    s.threshold = thr;
                }
                steps.push_back(s);
                ++si;
                S = nxt;
                cur = nslot;
            }
            if (odd) {
                // F = Z G-hat, unfiltered
                psf_step_info_t s{};
                s.kind = 3;
                s.index = 1;
                RowView G = S;
                const double glen = series->len_odd > 0.0 ? series->len_odd : pow_len(N - 1);
                if ((rc = run_step(w, &vz, &G, {}, 0.0, 0.0, 1, si, sslot[cur ^ 1], &S, nullptr, glen, zlen)))
                    return rc;
                steps.push_back(s);
                ++si;
            }
            F = S;
            if ((rc = make_result(w, F, &handle, &r))) return rc;
            Ctl c;
            if ((rc = read_back(w, c, nullptr))) {
                destroy_result(r);
                return rc;
            }
            if ((rc = status_to_code(c.status))) {
                destroy_result(r);
                return rc;
            }
            if (c.status & kDevPoolFull) {
                destroy_result(r);
                r = nullptr;
                if ((rc = w.clear_sums())) return rc;
                if (attempt > 8 || cap >= kMaxPool)
                    return fail(PSF_ETOOBIG, "evaluation needs more than 2^31 - 2^20 pool entries");
                unsigned long long need = c.pool_used + c.pool_used / 4 + 4096;
                cap = need > 2 * cap ? need : 2 * cap;
                if (cap > kMaxPool) cap = kMaxPool;
                continue;
            }
            std::vector<StepStat> ss(steps.size());
            if (!ss.empty()) {
                if (read_stats(w, ss.data(), w.stats.p, sizeof(StepStat) * ss.size()) != PSF_OK) {
                    destroy_result(r);
                    return fail(PSF_ECUDA, "stats read-back");
                }
            }
            for (size_t i = 0; i < steps.size(); ++i) {
                steps[i].nnz_pre = (int64_t)ss[i].nnz_pre;
                bool filt = steps[i].threshold > 0.0;
                steps[i].nnz_post = filt ? (int64_t)ss[i].nnz_post : (int64_t)ss[i].nnz_pre;
                steps[i].eps_f = filt ? ss[i].eps_f : 0.0;
                steps[i].iters = filt ? ss[i].iters : 0;
                steps[i].dropped = filt ? ss[i].dropped : 0.0;
                steps[i].fma = (int64_t)ss[i].fma;
            }
            // B-operand row lengths of this evaluation, for the next one
            series->len_baby.assign((size_t)(q > 1 ? q - 1 : 0), 0.0);
            series->len_giant.assign((size_t)(b > 1 ? b - 1 : 0), 0.0);
            series->fma_giant.assign((size_t)(b > 1 ? b - 1 : 0), 0.0);
            series->out_giant.assign((size_t)(b > 1 ? b - 1 : 0), 0.0);
            std::vector<unsigned> sb((size_t)(q > 1 ? q - 1 : 0), 0u), sg((size_t)(b > 1 ? b - 1 : 0), 0u);
            {
                double prev_len = pow_len(1);  // Z-hat_(1) = Z or W
                size_t idx = 0;
                for (int k = 1; k < q; ++k, ++idx) {
                    series->len_baby[(size_t)(k - 1)] = prev_len;
                    sb[(size_t)(k - 1)] = ss[idx].span_max;
                    prev_len = (double)steps[idx].nnz_post / n;
                }
                double s_len = 0.0;
                if (g == 0) s_len = (double)steps[idx++].nnz_post / n;  // S-hat_0
                for (int i = 1; i < b; ++i, ++idx) {
                    series->len_giant[(size_t)(i - 1)] = s_len;
                    sg[(size_t)(i - 1)] = ss[idx].span_max;
                    series->out_giant[(size_t)(i - 1)] = (double)steps[idx].nnz_pre / n;
                    series->fma_giant[(size_t)(i - 1)] = (double)steps[idx].fma;
                    s_len = (double)steps[idx].nnz_post / n;
                }
                if (odd) series->len_odd = s_len;  // G-hat, the right factor of F = Z G-hat
            }
            {
                std::lock_guard<std::mutex> lock(series->span_mu);
                series->span_baby = sb;
                series->span_giant = sg;
            }
            if ((rc = finish_result(w, F, r, c.nnz_total))) {
                destroy_result(r);
                return rc;
            }
            eval_fma = c.fma_total;
            if (c.pool_used - used_before > series->ps_need) series->ps_need = c.pool_used - used_before;
            break;
        }
    }
    r->steps = steps;
    psf_info_t& inf = r->info;
    inf.N = N;
    inf.q = q;
    inf.b = b;
    inf.g = g;
    inf.products = p.products + (square ? 1 + (int)odd : 0);
    inf.nsteps = (int32_t)steps.size();
    for (int i = 0; i <= 10; ++i) inf.z[i] = p.zz[(size_t)i];
    inf.alpha10 = p.alpha10;
    inf.trunc = p.trunc;
    inf.budget = p.budget;
    inf.nnz = r->nnz;
    inf.fma = (int64_t)eval_fma;
    if (g_prof.on) g_prof.fma += (double)eval_fma;
    *out = handle;
    return PSF_OK;
}

int psf_tune_set(int32_t key, double value) {
    switch (key) {
        case PSF_TUNE_TABLE_CROSSOVER:
            if (!(value >= 0.0)) return fail(PSF_EINVAL, "crossover must be >= 0");
            g_table_crossover.store(value);
            return PSF_OK;
        case PSF_TUNE_BATCH_GRAPH:
            if (!(value == 0.0 || value == 1.0)) return fail(PSF_EINVAL, "batch graph must be 0 or 1");
            g_batch_graph.store(value != 0.0);
            return PSF_OK;
        case PSF_TUNE_BATCH_REUSE:
            if (!(value == 0.0 || value == 1.0)) return fail(PSF_EINVAL, "batch reuse must be 0 or 1");
            g_batch_reuse.store(value != 0.0);
            return PSF_OK;
        case PSF_TUNE_ALG1_FAR_SHIFT:
            if (!(value >= 0.0 && value <= 2047.0 && value == (double)(int)value))
                return fail(PSF_EINVAL, "far shift must be an integer in [0, 2047]");
            g_far_shift.store((int)value);
            return PSF_OK;
        case PSF_TUNE_BARRIER_BUDGET_NS:
            if (!(value >= 0.0 && value <= 6e10 && value == std::floor(value)))
                return fail(PSF_EINVAL, "barrier budget must be an integer number of ns in [0, 6e10]");
            set_barrier_budget_ns((unsigned long long)value);
            return PSF_OK;
        case PSF_TUNE_FAIL_ADMISSION:
            if (!(value >= 0.0 && value <= 1e15 && value == std::floor(value)))
                return fail(PSF_EINVAL, "admission count must be a non-negative integer");
            g_fail_admission.store((long long)value);
            return PSF_OK;
        case PSF_TUNE_DENSE_XOVER:
            if (!(value >= 0.0)) return fail(PSF_EINVAL, "dense crossover must be >= 0");
            g_dense_xover.store(value);
            return PSF_OK;
        case PSF_TUNE_ROW_BITMAPS:
            if (!(value == 0.0 || value == 1.0 || value == 2.0)) return fail(PSF_EINVAL, "row bitmaps must be 0, 1 or 2");
            g_row_bitmaps.store((int)value);
            return PSF_OK;
        default:
            return fail(PSF_EINVAL, "unknown tuning key %d", key);
    }
}

int psf_tune_get(int32_t key, double* value) {
    if (!value) return fail(PSF_EINVAL, "null argument");
    switch (key) {
        case PSF_TUNE_TABLE_CROSSOVER:
            *value = g_table_crossover.load();
            return PSF_OK;
        case PSF_TUNE_BATCH_GRAPH:
            *value = g_batch_graph.load() ? 1.0 : 0.0;
            return PSF_OK;
        case PSF_TUNE_BATCH_REUSE:
            *value = g_batch_reuse.load() ? 1.0 : 0.0;
            return PSF_OK;
        case PSF_TUNE_ALG1_FAR_SHIFT:
            *value = (double)g_far_shift.load();
            return PSF_OK;
        case PSF_TUNE_BARRIER_BUDGET_NS:
            *value = (double)barrier_budget_ns();
            return PSF_OK;
        case PSF_TUNE_FAIL_ADMISSION:
            *value = (double)g_fail_admission.load();
            return PSF_OK;
        case PSF_TUNE_DENSE_XOVER:
            *value = g_dense_xover.load();
            return PSF_OK;
        case PSF_TUNE_ROW_BITMAPS:
            *value = (double)g_row_bitmaps.load();
            return PSF_OK;
        default:
            return fail(PSF_EINVAL, "unknown tuning key %d", key);
    }
}

// Evaluate the series once with each slot map, timing every product launch,
// and keep the crossover (work per row) that minimises the summed time: the
// launches are the same in both runs (same plan, same steps), only the map
// differs, and both maps give bitwise identical results.
int psf_autotune(psf_series_t series, const psf_csr_t* Z, void* stream, double* crossover, double* saved_ms) {
    if (!series || !Z || !crossover) return fail(PSF_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    psf_result_t r = nullptr;
    int rc = psf_eval(series, Z, stream, &r);  // warm-up: pool sizes are learnt
    if (rc) return rc;
    psf_result_destroy(r);
    const int saved_map = series->kernel;
    std::vector<double> work[2];
    std::vector<double> ms[2];
    for (int m = 0; m < 2; ++m) {
        TuneRecorder rec;
        series->kernel = m == 0 ? 1 : 2;
        g_tune_rec = &rec;
        rc = psf_eval(series, Z, stream, &r);
        g_tune_rec = nullptr;
        series->kernel = saved_map;
        if (rc == PSF_OK) {
            psf_result_destroy(r);
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = fail(PSF_ECUDA, "autotune sync");
        }
        for (auto& pr : rec.ev) {
            float t = 0.0f;
            if (rc == PSF_OK && cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess)
                rc = fail(PSF_ECUDA, "autotune timing");
            ms[m].push_back(t);
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        work[m] = rec.work;
        if (rc) return rc;
    }
    if (work[0] != work[1]) return fail(PSF_ECUDA, "autotune: the two runs launched different products");
    // candidate crossovers: every work level, plus "never table"
    std::vector<double> cand(work[0]);
    cand.push_back(std::numeric_limits<double>::infinity());
    double best_t = std::numeric_limits<double>::infinity(), best_c = g_table_crossover.load(), cur_t = 0.0;
    const double cur_c = g_table_crossover.load();
    for (size_t i = 0; i < work[0].size(); ++i) cur_t += work[0][i] >= cur_c ? ms[0][i] : ms[1][i];
    for (double c : cand) {
        double t = 0.0;
        for (size_t i = 0; i < work[0].size(); ++i) t += work[0][i] >= c ? ms[0][i] : ms[1][i];
        if (t < best_t || (t == best_t && c > best_c)) {
            best_t = t;
            best_c = c;
        }
    }
    if (std::isinf(best_c)) best_c = 1e300;
    g_table_crossover.store(best_c);
    *crossover = best_c;
    if (saved_ms) *saved_ms = cur_t - best_t;
    return PSF_OK;
}

int psf_fp64_peak(void* stream, double* tflops) {
    if (!tflops) return fail(PSF_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    CU(kernels_init());
    const int blocks = fp64_probe_blocks(), iters = 8192;
    DevBuf out;
    CU(out.alloc(sizeof(double) * (size_t)blocks * 256, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    double best = 0.0;
    // three warm-up launches (about 50 ms: the clocks rise from idle), then
    // the best of five
    for (int rep = 0; rep < 8 && err == cudaSuccess; ++rep) {
        err = cudaEventRecord(e0, st);
        if (err == cudaSuccess) err = launch_fp64_probe(iters, out.as<double>(), st);
        if (err == cudaSuccess) err = cudaEventRecord(e1, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        const double flop = 2.0 * 8.0 * iters * 256.0 * blocks;
        if (err == cudaSuccess && rep >= 3 && ms > 0.0f) best = std::max(best, flop / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    out.release();
    if (err != cudaSuccess) return fail(PSF_ECUDA, "fp64 probe: %s", cudaGetErrorString(err));
    *tflops = best;
    return PSF_OK;
}

int psf_launch_count(int64_t* count) {
    if (!count) return fail(PSF_EINVAL, "null argument");
    *count = (int64_t)launch_count();
    return PSF_OK;
}

int psf_profile(int32_t enable) {
    g_prof.on = enable != 0;
    return PSF_OK;
}

int psf_profile_read(int64_t* launches, double* ms, double* fma, int32_t reset) {
    double total = 0.0;
    for (auto& pr : g_prof.ev) {
        CU(cudaEventSynchronize(pr.second));
        float t = 0.0f;
        CU(cudaEventElapsedTime(&t, pr.first, pr.second));
        total += t;
    }
    if (launches) *launches = (int64_t)g_prof.ev.size();
    if (ms) *ms = total;
    if (fma) *fma = g_prof.fma;
    if (reset) {
        for (auto& pr : g_prof.ev) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        g_prof.ev.clear();
        g_prof.fma = 0.0;
    }
    return PSF_OK;
}

int psf_result_csr(psf_result_t r, psf_csr_t* view) {
    if (!r || !view) return fail(PSF_EINVAL, "null argument");
    view->n = r->n;
    view->nnz = (int32_t)r->nnz;
    view->rowptr = r->rowptr;
    view->col = r->col;
    view->val = r->val;
    return PSF_OK;
}

int psf_result_copy(psf_result_t r, int32_t* rowptr, int32_t* col, double* val, void* stream) {
    if (!r) return fail(PSF_EINVAL, "null result");
    cudaStream_t st = (cudaStream_t)stream;
    // cudaMemcpyDefault: the destination may be device or host memory
    if (rowptr) CU(cudaMemcpyAsync(rowptr, r->rowptr, sizeof(int) * ((size_t)r->n + 1), cudaMemcpyDefault, st));
    if (col && r->nnz) CU(cudaMemcpyAsync(col, r->col, sizeof(int) * (size_t)r->nnz, cudaMemcpyDefault, st));
    if (val && r->nnz) CU(cudaMemcpyAsync(val, r->val, sizeof(double) * (size_t)r->nnz, cudaMemcpyDefault, st));
    return PSF_OK;
}

int psf_eval_from_host(psf_series_t series, const psf_csr_t* Z, void* stream, psf_result_t* out) {
    if (!out) return fail(PSF_EINVAL, "out is null");
    *out = nullptr;
    if (!series) return fail(PSF_EINVAL, "null series");
    int rc = check_csr(Z, Z ? Z->n : 0, "Z");
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = prepare(st))) return rc;
    // a stream-ordered device copy of Z, released after the evaluation's work
    DevBuf rp, ci, v;
    CU(rp.alloc(sizeof(int) * ((size_t)Z->n + 1), st));
    CU(ci.alloc(sizeof(int) * (size_t)Z->nnz, st));
    CU(v.alloc(sizeof(double) * (size_t)Z->nnz, st));
    CU(cudaMemcpyAsync(rp.p, Z->rowptr, sizeof(int) * ((size_t)Z->n + 1), cudaMemcpyDefault, st));
    if (Z->nnz) {
        CU(cudaMemcpyAsync(ci.p, Z->col, sizeof(int) * (size_t)Z->nnz, cudaMemcpyDefault, st));
        CU(cudaMemcpyAsync(v.p, Z->val, sizeof(double) * (size_t)Z->nnz, cudaMemcpyDefault, st));
    }
    psf_csr_t Zd{Z->n, Z->nnz, rp.as<int>(), ci.as<int>(), v.as<double>()};
    return psf_eval(series, &Zd, stream, out);
}

int psf_result_info(psf_result_t r, psf_info_t* info) {
    if (!r || !info) return fail(PSF_EINVAL, "null argument");
    *info = r->info;
    return PSF_OK;
}

int psf_result_step(psf_result_t r, int32_t i, psf_step_info_t* step) {
    if (!r || !step) return fail(PSF_EINVAL, "null argument");
    if (i < 0 || i >= (int32_t)r->steps.size()) return fail(PSF_EINVAL, "step %d out of range", i);
    *step = r->steps[(size_t)i];
    return PSF_OK;
}

int psf_result_destroy(psf_result_t r) {
    destroy_result(r);
    return PSF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- norm without allocation
// psf_norm1_noalloc works in one scratch region compiled into the library
// instead of a per-call workspace: some callers cannot allocate at the moment
// they need a norm (their device memory is committed to other work, or the
// implicit device-wide synchronisation of freeing memory would stall their
// other streams).  The region holds the control block, the norm slot and the
// fixed-point column sums of up to PSF_NORM1_NOALLOC_MAX_N columns; the
// matrix's own (col, val) arrays serve as the flat entry range the norm
// kernels scan, so nothing is copied.
namespace {

constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kNaMaxN = PSF_NORM1_NOALLOC_MAX_N;
constexpr size_t kNaCtl = 0;
constexpr size_t kNaSlot = kNaCtl + round256(sizeof(Ctl));
constexpr size_t kNaSticky = kNaSlot + round256(sizeof(NormSlot));
constexpr size_t kNaWords = kNaSticky + round256(sizeof(unsigned) * kNaMaxN);
constexpr size_t kNaBytes = kNaWords + sizeof(unsigned long long) * kChunks * kNaMaxN;

// psf.h states this size; a change to the control block, kChunks or the
// column limit must update it there too.
static_assert(kNaBytes == 4456960, "the scratch size stated in psf.h");
static __device__ __align__(256) unsigned char g_norm1_scratch[kNaBytes];

// Device address of the scratch region, looked up once per device (with
// that device current) and kept for the life of the process (a
// cudaDeviceReset would make it stale); the lookup is the call that may load
// the module, which is why the first call belongs before any stream capture.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mu;
void* g_na_ptr[kNaMaxDevices] = {};

int noalloc_scratch(unsigned char** out) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(PSF_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        CU(cudaGetSymbolAddress(&p, g_norm1_scratch));
        if (!p) return fail(PSF_ECUDA, "scratch region has no device address");
        g_na_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_na_ptr[dev]);
    return PSF_OK;
}

}  // namespace

extern "C" int psf_norm1_noalloc(const psf_csr_t* M, void* stream, double* out) {
    if (!M || !out) return fail(PSF_EINVAL, "null argument");
    int rc = check_csr(M, M->n, "M");
    if (rc) return rc;
    if ((size_t)M->n > kNaMaxN)
        return fail(PSF_ETOOBIG, "psf_norm1_noalloc: n = %d exceeds its static scratch limit of %d columns", M->n,
                    (int)kNaMaxN);
    if (M->n == 0) {
        *out = 0.0;
        return PSF_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CU(kernels_init());
    unsigned char* base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;
    Ctl* ctl = reinterpret_cast<Ctl*>(base + kNaCtl);
    NormSlot* slot = reinterpret_cast<NormSlot*>(base + kNaSlot);
    unsigned* sticky = reinterpret_cast<unsigned*>(base + kNaSticky);
    unsigned long long* words = reinterpret_cast<unsigned long long*>(base + kNaWords);
    // clear what must start at zero, check the input (its outcome is read
    // with the result; the norm kernels never index with a column outside
    // [0, n)), then max |x| and the exact column sums over M's entries
    CU(launch_norm_scratch_init(ctl, slot, words, sticky, M->n, M->nnz, st));
    CU(launch_validate(M->n, M->nnz, M->rowptr, M->col, M->val, ctl, st));
    CU(launch_absmax(M->val, ctl, 0, slot, st));
    NormArgs na{};
    na.n = M->n;
    na.count = 1;
    na.pool_col = M->col;
    na.pool_val = M->val;
    na.slots = slot;
    na.words = words;
    na.sticky = sticky;
    na.ctl = ctl;
    CU(launch_norms(na, st));
    int status = 0;
    unsigned long long bits = 0ull;
    CU(cudaMemcpyAsync(&status, &ctl->status, sizeof status, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&bits, &slot->result, sizeof bits, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if ((rc = status_to_code(status))) return rc;
    std::memcpy(out, &bits, sizeof bits);
    return PSF_OK;
}
