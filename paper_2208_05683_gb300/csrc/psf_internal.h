// psf_internal.h -- host-side internals shared by the translation units of
// the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/psf.h"
#include "psf_kernels.h"
#include "psf_plan.h"

// ---------------------------------------------------------------- objects
struct psf_series_s {
    std::vector<double> a;
    // PSF_Z_SQUARE: the coefficients c_k of g (f(Z) = g(Z^2) or Z g(Z^2))
    std::vector<double> c;
    bool odd = false;
    double tol = 0.0;
    uint32_t flags = 0;
    int s = 0;
    double e_r = 0.1;
    int maxit = 1000;
    unsigned long long pool_hint = 0;  // user-set initial capacity (entries)
    unsigned long long z_need = 0;     // largest pool the norm phase has needed
    unsigned long long ps_need = 0;    // largest pool the PS phase has needed
    // B-operand mean row lengths seen by the previous evaluation, per step:
    // they pick the thread-group size of the product kernel (tuning only)
    std::vector<double> len_z, len_baby, len_giant;
    // mean output row length before the filter of each giant step (the
    // product kernel's accumulator variant for long rows)
    std::vector<double> out_giant;
    double len_odd = 0.0;  // row length of G-hat in F = Z G-hat (odd series, PSF_Z_SQUARE)
    // widest column window of each step's rows (the bitmap map's wide window
    // is used where it exceeded kBitmapColumns); batches, which may run
    // concurrently on one series, read and write them under span_mu
    std::vector<unsigned> span_z, span_baby, span_giant;
    std::mutex span_mu;
    int kernel = 0;       // PSF_PARAM_KERNEL
    int chunk_cols = 0;   // PSF_PARAM_CHUNK_COLS
    int chunk_slots = 0;  // PSF_PARAM_CHUNK_SLOTS
    double dense_xover = -1.0;  // PSF_PARAM_DENSE_XOVER (-1: the process-wide PSF_TUNE_DENSE_XOVER)
    // multiply-adds of each giant step in the previous evaluation (the
    // dense-tile choice of the next one)
    std::vector<double> fma_giant;
};

struct psf_result_s {
    int n = 0;
    long long nnz = 0;
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
    cudaStream_t stream = nullptr;
    psf_info_t info{};
    std::vector<psf_step_info_t> steps;
    // set when rowptr/col/val point into storage shared by several results
    // (a batch); the storage is released with the last of them
    std::shared_ptr<void> owner;
};

namespace psf {
namespace host {

// Record a failure message for psf_last_error and return `code`.
int fail(int code, const char* fmt, ...);

#define CU(expr)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? PSF_ENOMEM : PSF_ECUDA, "%s: %s (%s:%d)", \
                        #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

// Stream-ordered device buffer released on the stream it was made on.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    cudaError_t alloc(size_t bytes, cudaStream_t s) {
        release();
        st = s;
        if (bytes == 0) bytes = 16;
        return cudaMallocAsync(&p, bytes, s);
    }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
    }
    template <class T>
    T* as() const {
        return static_cast<T*>(p);
    }
};

// Optional event timing of the product kernel (psf_profile).
struct Profile {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    double fma = 0.0;
};
extern Profile g_prof;

// Largest entry pool: pool positions are 32-bit in the kernels, and loops
// step at most a row (plus a few hundred entries) past a row's end, so the
// capacity stays 2^20 below 2^31 and no position plus offset overflows.
constexpr unsigned long long kMaxPool = (1ull << 31) - (1ull << 20);

// Mailboxes: pinned host buffers mapped into the device's address space,
// {host, device} pointers, into which k_export writes the control block
// (offset 0), the norm slots (kMboxSlots) and the step records (kMboxStats)
// that the host reads back.  A kernel's stores take no copy engine, so these
// reads do not wait behind a large device-to-host copy in flight on another
// stream (a user copying one result out while the next evaluation runs).
// Each evaluation's workspace takes one from a process-wide free list and
// gives it back; they are kept for the life of the process (which must not
// outlive a cudaDeviceReset).  {nullptr, nullptr} if none could be made: the
// read-backs then use copies.
constexpr size_t kMboxBytes = 64 * 1024, kMboxSlots = 4096, kMboxStats = 8192;
static_assert(sizeof(Ctl) % 4 == 0 && sizeof(Ctl) <= kMboxSlots, "control block in its mailbox part");
static_assert(sizeof(NormSlot) * kMaxNorms % 4 == 0 && kMboxSlots + sizeof(NormSlot) * kMaxNorms <= kMboxStats,
              "norm slots in their mailbox part");
std::pair<void*, void*> mailbox_take();
void mailbox_give(std::pair<void*, void*> m);

// Device workspace shared by the phases of one evaluation.
// products mark their output pattern from column bitmaps of B's rows
// (PSF_TUNE_ROW_BITMAPS: 0 never, 1 when A's rows average at least
// kBitmapMinA entries and B's kBitmapMinB, 2 always)
extern std::atomic<int> g_row_bitmaps;
constexpr double kBitmapMinA = 12.0;
constexpr double kBitmapMinB = 32.0;

struct Work {
    int n = 0;
    cudaStream_t st = nullptr;
    DevBuf ctl, stats, slots, words, sticky, pool_col, pool_val, cand_col, cand_x, scan;
    DevBuf nwords;  // 24-bit-piece column sums of the norm phase (zero between uses)
    DevBuf dense[3];  // the dense-tile path's A, B and C (n^2 doubles each), allocated on first use
    DevBuf bhdr, pool_bits;  // column bitmaps of a product's B rows: n headers, a word per pool entry
    double dense_xover = 1e300;  // dense tiles for a step with at least this many multiply-adds per n^3
    bool dense_estimate = false;  // a step without a recorded count may use the row-length estimate
    unsigned long long cap = 0, ccap = 0, bits_cap = 0;
    std::vector<DevBuf*> rows;  // 2n ints each: rb then re
    int slot_map = 0;            // 0 auto (by products per row), 1 table, 2 bitmap, 3 wide window, 4 CTA per row
    int chunk_cols = 0, chunk_slots = 0;

    std::pair<void*, void*> mbox{nullptr, nullptr};
    bool mbox_pending = false;  // an export into the mailbox may still be in flight
    ~Work() {
        for (DevBuf* b : rows) delete b;
        if (mbox.first) {
            // (an error path can leave an export unsynchronised: let it land
            // before another evaluation takes the mailbox)
            if (mbox_pending) cudaStreamSynchronize(st);
            mailbox_give(mbox);
        }
    }
    Ctl* C() const { return ctl.as<Ctl>(); }
    int init(int n_, cudaStream_t s, int nstats) {
        n = n_;
        st = s;
        if (!mbox.first) mbox = mailbox_take();
        CU(ctl.alloc(sizeof(Ctl), st));
        CU(cudaMemsetAsync(ctl.p, 0, sizeof(Ctl), st));
        CU(stats.alloc(sizeof(StepStat) * (size_t)(nstats > 0 ? nstats : 1), st));
        CU(slots.alloc(sizeof(NormSlot) * kMaxNorms, st));
        CU(cudaMemsetAsync(slots.p, 0, sizeof(NormSlot) * kMaxNorms, st));
        size_t nn = (size_t)(n > 0 ? n : 1);
        CU(words.alloc(sizeof(unsigned long long) * kChunks * nn * kMaxNorms, st));
        CU(cudaMemsetAsync(words.p, 0, sizeof(unsigned long long) * kChunks * nn * kMaxNorms, st));
        CU(sticky.alloc(sizeof(unsigned) * nn * kMaxNorms, st));
        CU(cudaMemsetAsync(sticky.p, 0, sizeof(unsigned) * nn * kMaxNorms, st));
        CU(scan.alloc(sizeof(long long) * scan_scratch_len(n_), st));
        CU(bhdr.alloc(sizeof(int2) * nn, st));
        return PSF_OK;
    }
    // (re)allocate the entry pool and reset the device control block
    int reset_pool(unsigned long long entries) {
        if (entries > kMaxPool) return fail(PSF_ETOOBIG, "pool of %llu entries exceeds 2^31 - 2^20", entries);
        if (entries > cap) {
            CU(pool_col.alloc(sizeof(int) * entries, st));
            CU(pool_val.alloc(sizeof(double) * entries, st));
            cap = entries;
            // two Algorithm 1 candidate lists of half the pool each (a step
            // whose candidates do not fit falls back to full scans)
            ccap = cap / 2 > 1024 ? cap / 2 : 1024;
            CU(cand_col.alloc(sizeof(int) * 2 * ccap, st));
            CU(cand_x.alloc(sizeof(unsigned long long) * 2 * ccap, st));
        }
        if (g_row_bitmaps.load() > 0 && bits_cap < cap) {
            CU(pool_bits.alloc(sizeof(unsigned) * cap, st));
            bits_cap = cap;
        }
        Ctl h{};
        h.pool_cap = cap;
        h.cand_cap = ccap;
        h.cand_chunk = cand_chunk();
        CU(cudaMemcpyAsync(ctl.p, &h, offsetof(Ctl, bar_count), cudaMemcpyHostToDevice, st));
        return PSF_OK;
    }
    // Entries a warp reserves in a candidate list at a time: up to 128, so
    // that about 12k warps' unused chunk ends take at most a quarter of it.
    unsigned cand_chunk() const {
        unsigned long long c = ccap / (4ull * 12288ull);
        c = c < 32ull ? 32ull : (c > 128ull ? 128ull : c);
        return (unsigned)(c & ~31ull);
    }
    // Column-sum accumulators are zero between steps; a phase cut short by a
    // pool overflow can leave some set, so they are cleared before its retry.
    int clear_sums() {
        size_t nn = (size_t)(n > 0 ? n : 1);
        CU(cudaMemsetAsync(words.p, 0, sizeof(unsigned long long) * kChunks * nn * kMaxNorms, st));
        CU(cudaMemsetAsync(sticky.p, 0, sizeof(unsigned) * nn * kMaxNorms, st));
        return PSF_OK;
    }
    // row arrays of matrix slot i
    int rows_for(size_t i, int** rb, int** re) {
        while (rows.size() <= i) rows.push_back(new DevBuf());
        if (!rows[i]->p) CU(rows[i]->alloc(sizeof(int) * 2 * (size_t)(n > 0 ? n : 1), st));
        *rb = rows[i]->as<int>();
        *re = *rb + n;
        return PSF_OK;
    }
    RowView pooled(int* rb, int* re) const { return RowView{rb, re, pool_col.as<int>(), pool_val.as<double>()}; }
    int* pcol() const { return pool_col.as<int>(); }
    double* pval() const { return pool_val.as<double>(); }
};

// Process-wide tuning (psf_tune_*, psf_autotune): the products per output
// row from which the product kernel uses the column-table slot map.
extern std::atomic<double> g_table_crossover;
// the PS phase of a batch runs as one captured CUDA graph (PSF_TUNE_BATCH_GRAPH)
extern std::atomic<bool> g_batch_graph;
// batched baby steps copy the norm phase's powers while nothing was dropped (PSF_TUNE_BATCH_REUSE)
extern std::atomic<bool> g_batch_reuse;
// Algorithm 1 sets candidates at or below eps_g / 2^g_far_shift apart (PSF_TUNE_ALG1_FAR_SHIFT)
extern std::atomic<int> g_far_shift;
// fault injection: the k-th server admission from now fails (PSF_TUNE_FAIL_ADMISSION)
extern std::atomic<long long> g_fail_admission;
// the dense-tile crossover in multiply-adds per n^3 (PSF_TUNE_DENSE_XOVER)
constexpr double kDenseXoverDefault = 0.15;
constexpr int kDenseMinN = 512;  // the automatic choice leaves smaller products sparse
extern std::atomic<double> g_dense_xover;
// slot_map 1: table, 2: bitmap, 0: by the work per row and the crossover
inline bool use_table(int slot_map, double work_per_row) {
    return slot_map == 1 || (slot_map == 0 && work_per_row >= g_table_crossover.load(std::memory_order_relaxed));
}

// One output row per block of four warps (k_product_cta) for a product of
// the single-matrix path when its rows fit one wave of blocks (7 per SM), so
// that warps would otherwise sit idle, and its B rows average at least 16
// entries (they are shared by the block's 128 threads); PSF_PARAM_KERNEL 4
// forces it.  Measured on GB300: the banded N(0, 1) family at n = 1000 runs
// 1.3-1.6x faster from bandwidth 8 on; at n = 4096 and above the warp per row
// is faster (1.4-2.7x).
inline bool use_cta(int n, double alen, double blen) {
    (void)alen;
    return n > 0 && n <= 7 * num_sms() && blen >= 16.0;
}

// Recorder of product launches for psf_autotune (set on the calling thread
// only): each launch's work per row and its event pair.
struct TuneRecorder {
    std::vector<double> work;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};
extern thread_local TuneRecorder* g_tune_rec;

int lsb_for_bound_host(double x);
RowView view_of(const psf_csr_t& m);
int check_csr(const psf_csr_t* m, int n, const char* what);
int read_back(Work& w, Ctl& c, NormSlot* slots);
int status_to_code(int st);
unsigned long long arena_for(double row_len);
int mark_pool(Work& w, int i);
void destroy_result(psf_result_s* r);
int prepare(cudaStream_t st);
// Estimates of ||Z^k||_1, k = 2..10, into norms[2..10] (psf_normest.cu);
// *fallback: a column of Z is too long for the estimator, nothing computed.
int estimate_power_norms(Work& w, const psf_csr_t& Z, double* norms, bool* fallback);

}  // namespace host
}  // namespace psf
