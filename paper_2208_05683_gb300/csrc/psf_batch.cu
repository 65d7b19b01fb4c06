// psf_batch.cu -- psf_eval_batch: Algorithm 2 for many (series, Z) instances
// at once.
//
// The instances of a batch form one block-diagonal matrix: instance i owns the
// global rows and columns [off_i, off_i + n_i).  Products of block-diagonal
// matrices stay block-diagonal and every output row is computed exactly as
// in a single evaluation (same terms, same fold order), so one launch of the
// product kernel serves every instance of a step, whatever their sizes.  The
// instances differ only in small per-instance tables: what a step does to the
// instance (its mode), its coefficients and its Algorithm 1 threshold.
//
// Steps of a batch (S = the stage counter):
//   z chain   Z^2..Z^10 of all instances (exact norms, Eq. 37), then one
//             norm launch; the host plans every instance (one sync)
//   baby k    k = 2..max q_i: Z-hat_(k) = filter(Z Z-hat_(k-1)) for q_i >= k;
//             an instance that has dropped no entry yet copies its Z^k from
//             the norm phase instead (the same entries, k <= 10)
//   S_0       B-hat_{b_i - 1} (addends only) for instances with g_i = 0
//   giant j   j = 1..max b_i - 1: S-hat_j = filter(B-hat + Z-hat_(q_i) S-hat_{j-1})
//             for j <= b_i - 1; finished instances pass their rows through
// then the result is split into one CSR per instance (second sync).  The
// number of launches depends on max q_i and max b_i, not on the batch size.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <vector>

#include "psf_internal.h"

using namespace psf;
using namespace psf::host;

namespace {

constexpr size_t kRowsZ = 60;        // pooled block-diagonal Z
constexpr size_t kRowsZq = 61;       // composite Z-hat_(q_i)
constexpr size_t kRowsBaby = 0;      // + k: baby step k (k = 2..23)
constexpr size_t kRowsS = 30;        // + (stage & 1): giant-step outputs
constexpr size_t kRowsPow = 40;      // + k - 2: the norm phase's Z^k (k = 2..10)
constexpr size_t kRowsW = 62;        // W = Z Z of the PSF_Z_SQUARE instances
constexpr size_t kRowsLeft = 63;     // composite left factor of the baby steps: Z, or W
constexpr int kMaxBatchRows = 1 << 24;  // column-sum words: 704 B per row

// Device storage shared by the results of one batch.
struct BatchStorage {
    int* rowptr = nullptr;
    int* col = nullptr;
    double* val = nullptr;
    cudaStream_t st = nullptr;
    ~BatchStorage() {
        if (rowptr) cudaFreeAsync(rowptr, st);
        if (col) cudaFreeAsync(col, st);
        if (val) cudaFreeAsync(val, st);
    }
};

// Pool sizing learnt from earlier batches (entries per row of the batch).
std::atomic<double> g_z_per_row{0.0}, g_ps_per_row{0.0};

void raise_to(std::atomic<double>& a, double v) {
    double cur = a.load();
    while (v > cur && !a.compare_exchange_weak(cur, v)) {
    }
}

struct InstPlan {
    bool trivial = false;  // N = 1 (f = a_0 I, not an odd series) or n = 0
    bool sq = false;       // PSF_Z_SQUARE: the scheme runs on W = Z Z
    bool odd = false;      // ... and ends with F = Z G-hat
    Plan p;
    std::vector<double> znnz;  // nnz(Z^k), k = 0..10 (0 where not computed)
};

// the coefficients the scheme runs on: a, or g's c_k with PSF_Z_SQUARE
const std::vector<double>& coeffs_of(const psf_series_s* s) { return (s->flags & PSF_Z_SQUARE) ? s->c : s->a; }

double coef_of(const psf_series_s* s, const Plan& p, int idx) {
    const std::vector<double>& a = coeffs_of(s);
    return (idx < p.N && idx < (int)a.size()) ? a[(size_t)idx] : 0.0;
}

// Host tables of one stage: what every instance does, and the coefficients
// of the addend terms (term t: Z-hat_(t) for t < tz, Z-hat_(q_i) for t = tz).
struct StageTab {
    std::vector<BatchStep> step;
    std::vector<double> alpha;  // [t * ninst + i]
    bool any_filter = false;
    bool any_product = false;
    bool any_reuse = false;  // some instance may take the norm phase's Z^k
    bool wide = false;       // some instance's rows spanned more than one bitmap chunk last time
    int nadd = 0;
    double reuse_rows = 0.0, reuse_nnz = 0.0;  // size of those powers (arena estimate)
    double work_rows = 0.0, work_fma = 0.0;  // estimates for the slot map and arenas
};

BatchStep step_of(int mode, double thr, double e_r, int maxit) {
    BatchStep b{};
    b.mode = mode;
    b.maxit = maxit;
    if (thr > 0.0) {
        b.eps_g = thr / (1.0 + e_r);
        b.bound = b.eps_g * (1.0 + e_r);
        b.e_lsb = lsb_for_bound_host(b.eps_g);
    }
    return b;
}

// A non-blocking stream of the calling thread on the current device, on
// which batch graphs are recorded (never executed).  It is destroyed when
// the thread exits (server workers come and go with their servers).
struct CaptureStream {
    cudaStream_t stream = nullptr;
    int dev = -1;
    ~CaptureStream() {
        if (stream) cudaStreamDestroy(stream);  // may fail harmlessly at process exit
    }
};

int capture_stream(cudaStream_t* out) {
    static thread_local CaptureStream t;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (!t.stream || t.dev != dev) {
        if (t.stream) {
            // the previous device's stream: destroyed on that device
            int cur = dev;
            CU(cudaSetDevice(t.dev));
            cudaStreamDestroy(t.stream);
            t.stream = nullptr;
            CU(cudaSetDevice(cur));
        }
        CU(cudaStreamCreateWithFlags(&t.stream, cudaStreamNonBlocking));
        t.dev = dev;
    }
    *out = t.stream;
    return PSF_OK;
}

int eval_group(const psf_series_t* series, const psf_csr_t* Zs, int count, cudaStream_t st, psf_result_t* outs) {
    int rc = PSF_OK;
    // ---- offsets of the block-diagonal matrix
    std::vector<int> off((size_t)count + 1, 0);
    long long ntot = 0, nnz_tot = 0;
    for (int i = 0; i < count; ++i) {
        off[(size_t)i] = (int)ntot;
        ntot += Zs[i].n;
        nnz_tot += Zs[i].nnz;
    }
    off[(size_t)count] = (int)ntot;
    const int n = (int)ntot;
    const psf_series_s* s0 = series[0];

    Work w;
    if ((rc = w.init(n, st, 1))) return rc;
    w.slot_map = s0->kernel;
    w.chunk_cols = s0->chunk_cols;
    w.chunk_slots = s0->chunk_slots;

    // ---- per-instance descriptors, instance table, validation (sync)
    DevBuf d_off, d_src, d_nnz, d_inst, d_slots;
    CU(d_off.alloc(sizeof(int) * ((size_t)count + 1), st));
    CU(d_src.alloc(sizeof(BatchSrc) * (size_t)count, st));
    CU(d_nnz.alloc(sizeof(int) * (size_t)count, st));
    CU(d_inst.alloc(sizeof(int) * (size_t)(n > 0 ? n : 1), st));
    CU(d_slots.alloc(sizeof(NormSlot) * kMaxNorms * (size_t)count, st));
    if (n > 0) {
        const size_t nb = sizeof(unsigned long long) * (size_t)kNormPieces * (size_t)n * 10;
        CU(w.nwords.alloc(nb, st));
        CU(cudaMemsetAsync(w.nwords.p, 0, nb, st));
    }
    std::vector<BatchSrc> src((size_t)count);
    std::vector<int> nnz((size_t)count);
    for (int i = 0; i < count; ++i) {
        src[(size_t)i] = BatchSrc{Zs[i].rowptr, Zs[i].col, Zs[i].val, Zs[i].n, off[(size_t)i]};
        nnz[(size_t)i] = Zs[i].nnz;
    }
    CU(cudaMemcpyAsync(d_off.p, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_src.p, src.data(), sizeof(BatchSrc) * src.size(), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_nnz.p, nnz.data(), sizeof(int) * nnz.size(), cudaMemcpyHostToDevice, st));
    const int* inst = d_inst.as<int>();
    const BatchSrc* dsrc = d_src.as<BatchSrc>();
    NormSlot* slots = d_slots.as<NormSlot>();
    CU(launch_inst_table(n, count, d_off.as<int>(), d_inst.as<int>(), st));
    CU(launch_validate_batch(n, inst, dsrc, d_nnz.as<int>(), w.C(), st));
    {
        Ctl c;
        if ((rc = read_back(w, c, nullptr))) return rc;
        if (c.status & kDevBadInput) return fail(PSF_EINVAL, "a batch input is malformed (row pointers, column order "
                                                            "or range, or non-finite value)");
    }
    const double zlen_all = n > 0 ? (double)nnz_tot / n : 0.0;
    const unsigned long long arena_z = arena_for(zlen_all > 0.0 ? zlen_all : 1.0);

    // ---- z chain: Z^2..Z^10 of every instance that needs exact norms
    std::vector<InstPlan> ip((size_t)count);
    std::vector<char> chain((size_t)count);
    bool any_chain = false;
    for (int i = 0; i < count; ++i) {
        chain[(size_t)i] = !(series[i]->flags & PSF_Z_SUBMULT) && Zs[i].n > 0;
        any_chain = any_chain || chain[(size_t)i];
    }
    // the column windows each series' previous evaluation measured, per step
    // (read under the series' lock: batches on other threads may share it)
    std::vector<std::vector<unsigned>> span_z((size_t)count), span_baby((size_t)count), span_giant((size_t)count);
    for (int i = 0; i < count; ++i) {
        std::lock_guard<std::mutex> lock(series[i]->span_mu);
        span_z[(size_t)i] = series[i]->span_z;
        span_baby[(size_t)i] = series[i]->span_baby;
        span_giant[(size_t)i] = series[i]->span_giant;
    }
    auto wide_of = [](const std::vector<unsigned>& v, int idx) {
        return idx >= 0 && (size_t)idx < v.size() && v[(size_t)idx] > (unsigned)kBitmapColumns;
    };
    std::vector<StepStat> zst;  // 9 * count
    unsigned long long z_fma_tot = 0;
    {
        DevBuf d_zstep, d_zstat;
        std::vector<BatchStep> zstep((size_t)count);
        for (int i = 0; i < count; ++i) zstep[(size_t)i] = step_of(chain[(size_t)i] ? kBatchProduct : kBatchSkip, 0.0, 0.0, 1);
        CU(d_zstep.alloc(sizeof(BatchStep) * (size_t)count, st));
        CU(cudaMemcpyAsync(d_zstep.p, zstep.data(), sizeof(BatchStep) * zstep.size(), cudaMemcpyHostToDevice, st));
        CU(d_zstat.alloc(sizeof(StepStat) * 9 * (size_t)count, st));
        unsigned long long zcap = (unsigned long long)(g_z_per_row.load() * 1.25 * n) + 4096ull;
        unsigned long long est = (unsigned long long)nnz_tot * (any_chain ? 128ull : 2ull) + (unsigned long long)n * 8ull +
                                 4096ull * 64ull;
        if (g_z_per_row.load() == 0.0 && zcap < est) zcap = est;
        if (zcap > kMaxPool) zcap = kMaxPool;
        for (int attempt = 0;; ++attempt) {
            CU(cudaMemsetAsync(slots, 0, sizeof(NormSlot) * kMaxNorms * (size_t)count, st));
            CU(cudaMemsetAsync(d_zstat.p, 0, sizeof(StepStat) * 9 * (size_t)count, st));
            if ((rc = w.reset_pool(zcap))) return rc;
            int *zrb, *zre;
            if ((rc = w.rows_for(kRowsZ, &zrb, &zre))) return rc;
            if ((rc = mark_pool(w, 0))) return rc;
            CU(launch_copy_rows_batch(n, inst, dsrc, zrb, zre, w.pcol(), w.pval(), w.C(), arena_z, slots + 1,
                                      kMaxNorms, st));
            if ((rc = mark_pool(w, 1))) return rc;
            const RowView zp = w.pooled(zrb, zre);
            // norms by row tiles: matrix 0 is the pooled Z, matrix k-1 is Z^k
            NormRowsArgs nr{};
            nr.n = n;
            nr.count = 1;
            nr.rb[0] = zrb;
            nr.re[0] = zre;
            nr.col = w.pcol();
            nr.val = w.pval();
            nr.slots = slots + 1;
            nr.slot_stride = kMaxNorms;
            nr.inst = inst;
            nr.words = w.nwords.as<unsigned long long>();
            nr.sticky = w.sticky.as<unsigned>();
            nr.ctl = w.C();
            if (any_chain) {
                RowView prev = zp;
                for (int k = 2; k <= 10; ++k) {
                    int *rb, *re;
                    if ((rc = w.rows_for(kRowsPow + (size_t)(k - 2), &rb, &re))) return rc;
                    nr.rb[k - 1] = rb;
                    nr.re[k - 1] = re;
                    ProductArgs P{};
                    P.n = n;
                    P.A = zp;
                    P.B = prev;
                    P.out_rb = rb;
                    P.out_re = re;
                    P.pool_col = w.pcol();
                    P.pool_val = w.pval();
                    P.ctl = w.C();
                    P.words = w.words.as<unsigned long long>();
                    P.sticky = w.sticky.as<unsigned>();
                    P.inst = inst;
                    P.inst_off = d_off.as<int>();
                    P.bstep = d_zstep.as<BatchStep>();
                    P.ninst = count;
                    P.absmax_slot = slots + k;
                    P.absmax_stride = kMaxNorms;
                    P.stat_tab = d_zstat.as<StepStat>() + (size_t)(k - 2) * count;
                    P.chunk_cols = w.chunk_cols;
                    P.chunk_slots = w.chunk_slots;
                    const double blen = zlen_all * (k - 1) * (k - 1);
                    P.arena = arena_for(zlen_all * blen);
                    const bool table = use_table(w.slot_map, zlen_all * blen);
                    bool wz = false;
                    for (int i = 0; i < count && !wz; ++i) wz = chain[(size_t)i] && wide_of(span_z[(size_t)i], k - 2);
                    cudaEvent_t t0 = nullptr, t1 = nullptr;
                    if (g_tune_rec) {
                        CU(cudaEventCreate(&t0));
                        CU(cudaEventCreate(&t1));
                        CU(cudaEventRecord(t0, st));
                    }
                    CU(launch_product(P, table, st, 0.0, wz));
                    if (g_tune_rec) {
                        CU(cudaEventRecord(t1, st));
                        g_tune_rec->work.push_back(zlen_all * blen);
                        g_tune_rec->ev.emplace_back(t0, t1);
                    }
                    if ((rc = mark_pool(w, k))) return rc;
                    prev = w.pooled(rb, re);
                }
                nr.count = 10;
            }
            CU(launch_norms_rows(nr, st));
            Ctl c;
            if ((rc = read_back(w, c, nullptr))) return rc;
            if ((rc = status_to_code(c.status))) return rc;
            if (c.status & kDevPoolFull) {
                if ((rc = w.clear_sums())) return rc;
                if (attempt > 8 || zcap >= kMaxPool)
                    return fail(PSF_ETOOBIG, "the powers Z^2..Z^10 of the batch need more than 2^31 - 2^20 pool entries");
                unsigned long long need = c.pool_used + c.pool_used / 4 + 4096;
                zcap = need > 2 * zcap ? need : 2 * zcap;
                if (zcap > kMaxPool) zcap = kMaxPool;
                continue;
            }
            if (n > 0) raise_to(g_z_per_row, (double)c.pool_used / n);
            break;
        }
        std::vector<NormSlot> hs(kMaxNorms * (size_t)count);
        zst.resize(9 * (size_t)count);
        CU(cudaMemcpyAsync(hs.data(), slots, sizeof(NormSlot) * hs.size(), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(zst.data(), d_zstat.p, sizeof(StepStat) * zst.size(), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        // ---- plans (Alg. 2 steps 1-3)
        for (int i = 0; i < count; ++i) {
            const psf_series_s* S = series[i];
            InstPlan& P = ip[(size_t)i];
            double norms[kMaxNorms];
            norms[0] = 1.0;
            for (int k = 1; k <= 10; ++k) {
                unsigned long long bits = hs[(size_t)i * kMaxNorms + (size_t)k].result;
                std::memcpy(&norms[k], &bits, sizeof bits);
            }
            const bool submult = S->flags & PSF_Z_SUBMULT;
            P.sq = S->flags & PSF_Z_SQUARE;
            P.odd = P.sq && S->odd;
            // an odd series: ||f(Z) - Z G-hat||_1 <= ||Z||_1 ||g(W) - G-hat||_1 (IEEE: 1/0 = inf)
            const double tol_g = P.odd ? S->tol / norms[1] : S->tol;
            if (make_plan(coeffs_of(S), tol_g, S->flags & PSF_POLY, submult, S->s, norms, P.p, P.sq ? 2 : 1))
                return fail(PSF_ENOTCONV, "batch instance %d: no truncation length within %zu coefficients (Eq. 34)", i,
                            coeffs_of(S).size());
            if (P.p.q > PSF_MAX_Q) return fail(PSF_ETOOBIG, "batch instance %d: q = %d exceeds %d", i, P.p.q, PSF_MAX_Q);
            // an odd series with N = 1 still forms F = Z (c_0 I)
            P.trivial = (P.p.N == 1 && !P.odd) || Zs[i].n == 0;
            P.znnz.assign(11, 0.0);
            P.znnz[1] = (double)Zs[i].nnz;
            for (int k = 2; k <= 10; ++k) {
                const StepStat& z = zst[(size_t)(k - 2) * count + (size_t)i];
                P.znnz[(size_t)k] = (double)z.nnz_pre;
                z_fma_tot += z.fma;
            }
        }
    }

    // ---- the norm phase's powers stay in their pool for the baby steps: while
    // an instance has dropped no entry, its baby step k is its Z^k
    bool keep_powers = false;
    for (int i = 0; i < count && g_batch_reuse.load(); ++i)
        if (chain[(size_t)i] && !ip[(size_t)i].trivial && ip[(size_t)i].p.q >= 2 && !ip[(size_t)i].sq)
            keep_powers = true;
    DevBuf zk_col, zk_val;  // that pool; the PS phase gets a new one
    if (keep_powers) {
        std::swap(zk_col.p, w.pool_col.p);
        std::swap(zk_col.st, w.pool_col.st);
        std::swap(zk_val.p, w.pool_val.p);
        std::swap(zk_val.st, w.pool_val.st);
        w.cap = 0;
    }

    // ---- stage schedule of the PS phase
    int qmax = 1, bmax = 1;
    for (int i = 0; i < count; ++i)
        if (!ip[(size_t)i].trivial) {
            qmax = std::max(qmax, ip[(size_t)i].p.q);
            bmax = std::max(bmax, ip[(size_t)i].p.b);
        }
    const int tz = qmax;          // term index of Z-hat_(q_i)
    const int nadd = qmax + 1;    // addend terms of S_0 and giant stages
    if (nadd > kMaxAdd) return fail(PSF_ETOOBIG, "q = %d exceeds %d", qmax, kMaxAdd - 1);
    // stage list: [W = Z Z], baby k = 2..qmax, S_0, giant j = 1..bmax-1, [F = Z G-hat]
    bool any_sq = false, any_odd = false;
    for (int i = 0; i < count; ++i) {
        any_sq = any_sq || (ip[(size_t)i].sq && !ip[(size_t)i].trivial);
        any_odd = any_odd || (ip[(size_t)i].odd && !ip[(size_t)i].trivial);
    }
    struct StageDesc {
        int kind;   // 0 baby, 2 S_0, 1 giant, 3 W = Z Z, 4 F = Z G-hat (PSF_Z_SQUARE)
        int index;  // k or j
    };
    std::vector<StageDesc> stages;
    if (any_sq) stages.push_back({3, 0});
    for (int k = 2; k <= qmax; ++k) stages.push_back({0, k});
    stages.push_back({2, 0});
    for (int j = 1; j < bmax; ++j) stages.push_back({1, j});
    if (any_odd) stages.push_back({4, 1});
    auto slot_of = [&](size_t si) {
        const int k = stages[si].kind;
        return k == 0 ? kRowsBaby + (size_t)stages[si].index : (k == 3 ? kRowsW : kRowsS + (si & 1));
    };
    const size_t nst = stages.size();
    std::vector<StageTab> tabs(nst);
    for (size_t si = 0; si < nst; ++si) {
        StageTab& T = tabs[si];
        const StageDesc& D = stages[si];
        T.step.resize((size_t)count);
        T.nadd = (D.kind == 1 || D.kind == 2) ? nadd : 0;  // products alone: baby steps, W, Z G-hat
        T.alpha.assign((size_t)T.nadd * count, 0.0);
        for (int i = 0; i < count; ++i) {
            const psf_series_s* S = series[i];
            const InstPlan& P = ip[(size_t)i];
            const Plan& p = P.p;
            const bool nofilter = S->flags & PSF_NOFILTER;
            const int ni = Zs[i].n;
            BatchStep& B = T.step[(size_t)i];
            B = step_of(kBatchSkip, 0.0, 0.0, 1);
            auto set_alpha = [&](int t, double a) {
                if (a != 0.0) T.alpha[(size_t)t * count + (size_t)i] = a;  // +0 marks an absent term
            };
            auto block = [&](int blk) {
                for (int j = 0; j < p.q; ++j) set_alpha(j, coef_of(S, p, blk * p.q + j));
            };
            if (ni == 0) continue;
            const double zl = (double)Zs[i].nnz / ni;
            if (P.trivial) {
                if (D.kind == 2) {
                    B = step_of(kBatchAddOnly, 0.0, 0.0, 1);
                    set_alpha(0, coeffs_of(S)[0]);
                } else if (D.kind == 1 || D.kind == 4) {
                    B = step_of(kBatchPass, 0.0, 0.0, 1);
                }
                continue;
            }
            if (D.kind == 3) {
                // W = Z Z, unfiltered (other instances leave the rows empty)
                if (P.sq) {
                    B = step_of(kBatchProduct, 0.0, 0.0, 1);
                    T.work_rows += ni;
                    T.work_fma += ni * zl * zl;
                }
            } else if (D.kind == 4) {
                // F = Z G-hat of an odd series, unfiltered; the others pass through
                if (P.odd) {
                    B = step_of(kBatchProduct, 0.0, 0.0, 1);
                    T.work_rows += ni;
                    T.work_fma += ni * zl * (P.znnz[10] > 0.0 ? P.znnz[10] / ni : zl * 100.0);
                } else {
                    B = step_of(kBatchPass, 0.0, 0.0, 1);
                }
            } else if (D.kind == 0) {
                if (D.index <= p.q) {
                    const double thr = nofilter ? 0.0 : p.zeta[(size_t)D.index];
                    B = step_of(kBatchProduct, thr, S->e_r, S->maxit);
                    if (keep_powers && chain[(size_t)i] && D.index <= 10 && !P.sq) {
                        B.reuse = 1;
                        T.any_reuse = true;
                        T.reuse_rows += ni;
                        T.reuse_nnz += P.znnz[(size_t)D.index];
                    }
                    // the power of the left factor (Z, or W = Z^2) the step multiplies
                    const int e = (P.sq ? 2 : 1) * (D.index - 1);
                    const double bl = e <= 10 && P.znnz[(size_t)e] > 0.0 ? P.znnz[(size_t)e] / ni : zl * e * e;
                    const double al = P.sq && P.znnz[2] > 0.0 ? P.znnz[2] / ni : zl;
                    T.work_rows += ni;
                    T.work_fma += ni * al * bl;
                }
            } else if (D.kind == 2) {
                if (p.g == 0) {
                    B = step_of(kBatchAddOnly, 0.0, 0.0, 1);
                    block(p.b - 1);
                    if (p.q == 0) set_alpha(0, coef_of(S, p, 0));  // N = 1 of an odd series: c_0 I
                }
            } else {
                const int j = D.index;
                if (j <= p.b - 1) {
                    if (p.g == 1 && j == 1) {
                        // S_1 = B-hat_{b-2} + a_{(b-1)q} Z-hat_(q), unfiltered
                        B = step_of(kBatchAddOnly, 0.0, 0.0, 1);
                        block(p.b - 2);
                        set_alpha(tz, coef_of(S, p, (p.b - 1) * p.q));
                    } else {
                        const double thr = nofilter ? 0.0 : p.sigma[(size_t)j];
                        B = step_of(kBatchProduct, thr, S->e_r, S->maxit);
                        block(p.b - 1 - j);
                        const double al = (p.q <= 10 && P.znnz[(size_t)p.q] > 0.0) ? P.znnz[(size_t)p.q] / ni
                                                                                   : zl * p.q * p.q;
                        const double bl = P.znnz[10] > 0.0 ? P.znnz[10] / ni : zl * 100.0;
                        T.work_rows += ni;
                        T.work_fma += ni * al * bl;
                    }
                } else {
                    B = step_of(kBatchPass, 0.0, 0.0, 1);
                }
            }
            T.any_filter = T.any_filter || B.eps_g > 0.0;
            T.any_product = T.any_product || B.mode == kBatchProduct;
            if (B.mode == kBatchProduct && !P.trivial)
                T.wide = T.wide || (D.kind == 0 && wide_of(span_baby[(size_t)i], D.index - 2)) ||
                         (D.kind == 1 && wide_of(span_giant[(size_t)i], D.index - 1));
        }
    }
    // device copies of the stage tables, one upload
    DevBuf d_tab, d_stat, d_sel, d_cslot, d_pstart, d_dropped;
    std::vector<size_t> step_off(nst), alpha_off(nst);
    size_t bytes = 0;
    for (size_t si = 0; si < nst; ++si) {
        step_off[si] = bytes;
        bytes += sizeof(BatchStep) * (size_t)count;
        alpha_off[si] = bytes;
        bytes += sizeof(double) * tabs[si].alpha.size();
        bytes = (bytes + 15) & ~(size_t)15;
    }
    std::vector<unsigned char> htab(bytes > 0 ? bytes : 16);
    for (size_t si = 0; si < nst; ++si) {
        std::memcpy(htab.data() + step_off[si], tabs[si].step.data(), sizeof(BatchStep) * (size_t)count);
        if (!tabs[si].alpha.empty())
            std::memcpy(htab.data() + alpha_off[si], tabs[si].alpha.data(), sizeof(double) * tabs[si].alpha.size());
    }
    CU(d_tab.alloc(htab.size(), st));
    CU(cudaMemcpyAsync(d_tab.p, htab.data(), htab.size(), cudaMemcpyHostToDevice, st));
    CU(d_stat.alloc(sizeof(StepStat) * nst * (size_t)count, st));
    CU(d_cslot.alloc(sizeof(unsigned long long) * 2 * (size_t)count, st));
    CU(d_pstart.alloc(sizeof(unsigned long long) * (nst + 1), st));
    CU(d_dropped.alloc(sizeof(int) * (size_t)count, st));
    // the norm phase's Z^k (k = 2..10) in its kept pool
    RowView zpow[11] = {};
    if (keep_powers)
        for (int k = 2; k <= 10; ++k) {
            int *rb, *re;
            if ((rc = w.rows_for(kRowsPow + (size_t)(k - 2), &rb, &re))) return rc;
            zpow[k] = RowView{rb, re, zk_col.as<int>(), zk_val.as<double>()};
        }
    std::vector<int> sel((size_t)count);
    for (int i = 0; i < count; ++i) sel[(size_t)i] = ip[(size_t)i].trivial ? 1 : ip[(size_t)i].p.q;
    CU(d_sel.alloc(sizeof(int) * (size_t)count, st));
    CU(cudaMemcpyAsync(d_sel.p, sel.data(), sizeof(int) * sel.size(), cudaMemcpyHostToDevice, st));
    // the baby steps' left factor per instance: 0 for Z, 1 for W (PSF_Z_SQUARE)
    DevBuf d_lsel;
    if (any_sq) {
        std::vector<int> lsel((size_t)count);
        for (int i = 0; i < count; ++i) lsel[(size_t)i] = ip[(size_t)i].sq ? 1 : 0;
        CU(d_lsel.alloc(sizeof(int) * (size_t)count, st));
        CU(cudaMemcpyAsync(d_lsel.p, lsel.data(), sizeof(int) * lsel.size(), cudaMemcpyHostToDevice, st));
    }

    // ---- PS phase in one pool
    unsigned long long cap = (unsigned long long)(g_ps_per_row.load() * 1.25 * n) + 4096ull;
    {
        unsigned long long est = (unsigned long long)nnz_tot * 64ull + (unsigned long long)n * 64ull + 4096ull * 64ull;
        for (int i = 0; i < count; ++i) est += (unsigned long long)(4.0 * ip[(size_t)i].znnz[10]);
        if (g_ps_per_row.load() == 0.0 && cap < est) cap = est;
        if (cap > kMaxPool) cap = kMaxPool;
    }
    DevBuf d_rowptr, d_bounds;
    CU(d_rowptr.alloc(sizeof(int) * ((size_t)n + 1), st));
    CU(d_bounds.alloc(sizeof(int) * ((size_t)count + 1), st));
    std::vector<int> bounds((size_t)count + 1);
    std::vector<StepStat> pst(nst * (size_t)count);
    RowView F{};
    Ctl cfin{};
    for (int attempt = 0;; ++attempt) {
        if ((rc = w.reset_pool(cap))) return rc;
        int *zrb, *zre, *qrb, *qre;
        if ((rc = w.rows_for(kRowsZ, &zrb, &zre)) || (rc = w.rows_for(kRowsZq, &qrb, &qre))) return rc;
        // every row slot of the stages exists before the launches are enqueued
        // (a captured graph must not allocate)
        for (size_t si = 0; si < nst; ++si) {
            int *rb0, *re0;
            if ((rc = w.rows_for(slot_of(si), &rb0, &re0))) return rc;
        }
        int *lrb = nullptr, *lre = nullptr;
        if (any_sq && (rc = w.rows_for(kRowsLeft, &lrb, &lre))) return rc;
        // the whole PS phase: pool copy of Z, every stage, the row-length scan
        auto enqueue = [&](cudaStream_t st) -> int {
        CU(cudaMemsetAsync(d_stat.p, 0, sizeof(StepStat) * nst * (size_t)count, st));
        CU(cudaMemsetAsync(d_dropped.p, 0, sizeof(int) * (size_t)count, st));

        CU(launch_copy_rows_batch(n, inst, dsrc, zrb, zre, w.pcol(), w.pval(), w.C(), arena_z, nullptr, 0, st));
        const RowView zp = w.pooled(zrb, zre);
        std::vector<RowView> baby((size_t)qmax + 1);
        baby[1] = zp;
        RowView left = zp;  // the baby steps' left factor (Z, or W per instance)
        RowView S{};
        bool zq_done = false;
        for (size_t si = 0; si < nst; ++si) {
            const StageDesc& D = stages[si];
            const StageTab& T = tabs[si];
            if ((D.kind == 1 || D.kind == 2) && !zq_done) {
                // Z-hat_(q_i) of every instance, for the giant steps and the g = 1 step
                const int* rbs[kMaxAdd + 2];
                const int* res[kMaxAdd + 2];
                for (int k = 0; k <= qmax; ++k) {
                    rbs[k] = baby[(size_t)(k >= 1 ? k : 1)].rb;
                    res[k] = baby[(size_t)(k >= 1 ? k : 1)].re;
                }
                CU(launch_compose_rows(n, inst, d_sel.as<int>(), rbs, res, qmax + 1, qrb, qre, st));
                zq_done = true;
            }
            int *rb, *re;
            if ((rc = w.rows_for(slot_of(si), &rb, &re))) return rc;
            ProductArgs P{};
            P.n = n;
            const RowView zq = w.pooled(qrb, qre);
            if (D.kind == 0) {
                P.A = left;
                P.B = baby[(size_t)D.index - 1];
            } else if (D.kind == 1 || D.kind == 4) {
                P.A = D.kind == 1 ? zq : zp;  // Z-hat_(q_i) S-hat, or Z G-hat
                P.B = S;  // also the source of pass-through rows
            } else if (D.kind == 3) {
                P.A = zp;
                P.B = zp;
            }
            P.nadd = T.nadd;
            for (int t = 0; t < T.nadd; ++t) {
                AddTerm A{};
                const RowView* v = nullptr;
                if (t == tz) v = &zq;
                else if (t >= 1) v = &baby[(size_t)t];
                if (v) {
                    A.rb = v->rb;
                    A.re = v->re;
                    A.col = v->col;
                    A.val = v->val;
                }
                P.add[t] = A;
            }
            P.out_rb = rb;
            P.out_re = re;
            P.pool_col = w.pcol();
            P.pool_val = w.pval();
            P.ctl = w.C();
            P.words = w.words.as<unsigned long long>();
            P.sticky = w.sticky.as<unsigned>();
            P.inst = inst;
            P.inst_off = d_off.as<int>();
            P.bstep = reinterpret_cast<const BatchStep*>(d_tab.as<unsigned char>() + step_off[si]);
            P.alpha_tab = reinterpret_cast<const double*>(d_tab.as<unsigned char>() + alpha_off[si]);
            P.ninst = count;
            P.stat_tab = d_stat.as<StepStat>() + si * (size_t)count;
            P.chunk_cols = w.chunk_cols;
            P.chunk_slots = w.chunk_slots;
            P.inst_dropped = d_dropped.as<int>();
            if (T.any_filter) {
                P.cand_col = w.cand_col.as<int>();
                P.cand_x = w.cand_x.as<unsigned long long>();
                P.cand_cap = w.ccap;
                P.cand_chunk = w.cand_chunk();
            }
            const double fma_row = T.work_rows > 0.0 ? T.work_fma / T.work_rows : 8.0 * (T.nadd + 1);
            P.arena = arena_for(fma_row);
            CU(cudaMemcpyAsync(d_pstart.as<unsigned long long>() + si, &w.C()->pool_used, sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, st));
            const bool table = use_table(w.slot_map, fma_row);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (g_prof.on || g_tune_rec) {
                CU(cudaEventCreate(&e0));
                CU(cudaEventCreate(&e1));
                CU(cudaEventRecord(e0, st));
            }
            // giant stages mark their rows from column bitmaps of S's rows
            // (each S row is read by every row of Z-hat_(q) that needs it)
            const int bm = g_row_bitmaps.load();
            if (D.kind == 1 && !table && !T.wide && bm > 0 && w.bits_cap >= w.cap && w.chunk_cols <= 0 &&
                w.chunk_slots <= 0 && (bm == 2 || fma_row >= kBitmapMinA * kBitmapMinB)) {
                CU(launch_row_bitmaps(n, P.B, w.bhdr.as<int2>(), w.pool_bits.as<unsigned>(), st));
                P.bhdr = w.bhdr.as<int2>();
                P.bbits = w.pool_bits.as<unsigned>();
            }
            CU(launch_product(P, table, st, 0.0, T.wide));
            if (g_tune_rec) {
                CU(cudaEventRecord(e1, st));
                g_tune_rec->work.push_back(fma_row);
                g_tune_rec->ev.emplace_back(e0, e1);
            } else if (g_prof.on) {
                CU(cudaEventRecord(e1, st));
                g_prof.ev.emplace_back(e0, e1);
            }
            if (T.any_reuse) {
                ProductArgs C = P;
                C.power = zpow[D.index];
                C.arena = arena_for(T.reuse_nnz / T.reuse_rows);
                CU(launch_reuse_copy_batch(C, st));
            }
            if (T.any_filter) {
                Alg1BatchArgs a{};
                a.n = n;
                a.ninst = count;
                a.inst = inst;
                a.bstep = P.bstep;
                a.rb = rb;
                a.re = re;
                a.col = w.pcol();
                a.val = w.pval();
                a.words = P.words;
                a.sticky = P.sticky;
                a.cslot = d_cslot.as<unsigned long long>();
                a.pool_start = d_pstart.as<unsigned long long>() + si;
                a.ctl = w.C();
                a.stat_tab = P.stat_tab;
                a.cand_col = P.cand_col;
                a.cand_x = P.cand_x;
                a.inst_dropped = d_dropped.as<int>();
                a.far_shift = g_far_shift.load(std::memory_order_relaxed);
                CU(launch_alg1_batch(a, st));
            }
            const RowView out = w.pooled(rb, re);
            if (D.kind == 0) {
                baby[(size_t)D.index] = out;
            } else if (D.kind == 3) {
                // each instance's left factor and Z-hat_(1): Z, or its W
                const int* rbs[2] = {zp.rb, out.rb};
                const int* res[2] = {zp.re, out.re};
                CU(launch_compose_rows(n, inst, d_lsel.as<int>(), rbs, res, 2, lrb, lre, st));
                left = w.pooled(lrb, lre);
                baby[1] = left;
            } else {
                S = out;
            }
        }
        F = S;
        CU(launch_scan_rows(n, F.rb, F.re, d_rowptr.as<int>(), w.C(), w.scan.as<long long>(), st));
        CU(launch_bounds(count, d_off.as<int>(), d_rowptr.as<int>(), d_bounds.as<int>(), st));
        return PSF_OK;
        };
        // captured into a CUDA graph and launched as one unit (no host work
        // between its ~2 launches per stage); direct launches while the
        // product kernel is being profiled, or when graphs are switched off
        const bool use_graph = !g_prof.on && !g_tune_rec && g_batch_graph.load();
        cudaGraphExec_t exec = nullptr;
        if (use_graph) {
            // recorded on a stream of the library (capture is not allowed on
            // the legacy default stream), launched on the caller's stream
            cudaStream_t cs = nullptr;
            if ((rc = capture_stream(&cs))) return rc;
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            rc = enqueue(cs);
            const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
            if (rc == PSF_OK && ec != cudaSuccess) rc = fail(PSF_ECUDA, "batch graph capture: %s", cudaGetErrorString(ec));
            if (rc == PSF_OK) {
                const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
                if (ei != cudaSuccess) rc = fail(PSF_ECUDA, "batch graph instantiation: %s", cudaGetErrorString(ei));
            }
            if (graph) cudaGraphDestroy(graph);
            if (rc == PSF_OK) {
                const cudaError_t el = cudaGraphLaunch(exec, st);
                if (el != cudaSuccess) rc = fail(PSF_ECUDA, "batch graph launch: %s", cudaGetErrorString(el));
            }
            if (rc) {
                if (exec) cudaGraphExecDestroy(exec);
                return rc;
            }
        } else if ((rc = enqueue(st))) {
            return rc;
        }
        CU(cudaMemcpyAsync(bounds.data(), d_bounds.p, sizeof(int) * bounds.size(), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(pst.data(), d_stat.p, sizeof(StepStat) * pst.size(), cudaMemcpyDeviceToHost, st));
        rc = read_back(w, cfin, nullptr);
        if (exec) cudaGraphExecDestroy(exec);  // the stream has drained
        if (rc) return rc;
        if ((rc = status_to_code(cfin.status))) return rc;
        if (cfin.status & kDevPoolFull) {
            if ((rc = w.clear_sums())) return rc;
            if (attempt > 8 || cap >= kMaxPool)
                return fail(PSF_ETOOBIG, "the batch needs more than 2^31 - 2^20 pool entries");
            unsigned long long need = cfin.pool_used + cfin.pool_used / 4 + 4096;
            cap = need > 2 * cap ? need : 2 * cap;
            if (cap > kMaxPool) cap = kMaxPool;
            continue;
        }
        if (n > 0) raise_to(g_ps_per_row, (double)cfin.pool_used / n);
        break;
    }
    const unsigned long long nnz_out = cfin.nnz_total;
    if (nnz_out > (unsigned long long)INT32_MAX) return fail(PSF_ETOOBIG, "batch result has %llu entries", nnz_out);

    // ---- results: shared storage, one CSR view per instance
    auto store = std::make_shared<BatchStorage>();
    store->st = st;
    CU(cudaMallocAsync((void**)&store->rowptr, sizeof(int) * ((size_t)n + (size_t)count), st));
    CU(cudaMallocAsync((void**)&store->col, sizeof(int) * (nnz_out ? nnz_out : 1), st));
    CU(cudaMallocAsync((void**)&store->val, sizeof(double) * (nnz_out ? nnz_out : 1), st));
    CU(launch_gather_batch(n, count, inst, d_off.as<int>(), F, d_rowptr.as<int>(), store->rowptr, store->col,
                           store->val, st));
    for (int i = 0; i < count; ++i) {
        const psf_series_s* S = series[i];
        const InstPlan& P = ip[(size_t)i];
        const Plan& p = P.p;
        psf_result_s* r = new (std::nothrow) psf_result_s();
        if (!r) return fail(PSF_ENOMEM, "host allocation");
        r->owner = store;
        r->stream = st;
        r->n = Zs[i].n;
        r->nnz = bounds[(size_t)i + 1] - bounds[(size_t)i];
        r->rowptr = store->rowptr + off[(size_t)i] + i;
        r->col = store->col + bounds[(size_t)i];
        r->val = store->val + bounds[(size_t)i];
        unsigned long long fma = 0;
        for (int k = 2; k <= 10; ++k) fma += zst[(size_t)(k - 2) * count + (size_t)i].fma;
        // per-step statistics in the order of a single evaluation
        if (!P.trivial) {
            for (size_t si = 0; si < nst; ++si) {
                const StageDesc& D = stages[si];
                const BatchStep& B = tabs[si].step[(size_t)i];
                if (B.mode != kBatchProduct && B.mode != kBatchAddOnly) continue;
                const StepStat& ss = pst[si * (size_t)count + (size_t)i];
                if (D.kind == 3) {  // W = Z Z: counted, not a step record (as in psf_eval)
                    fma += ss.fma;
                    continue;
                }
                psf_step_info_t s{};
                s.kind = B.mode == kBatchAddOnly ? 2 : (D.kind == 0 ? 0 : (D.kind == 4 ? 3 : 1));
                s.index = D.index;
                const bool filt = B.eps_g > 0.0;
                s.threshold = filt ? (S->flags & PSF_NOFILTER ? 0.0
                                                              : (D.kind == 0 ? p.zeta[(size_t)D.index]
                                                                             : p.sigma[(size_t)D.index]))
                                   : 0.0;
                s.nnz_pre = (int64_t)ss.nnz_pre;
                s.nnz_post = filt ? (int64_t)ss.nnz_post : (int64_t)ss.nnz_pre;
                s.eps_f = filt ? ss.eps_f : 0.0;
                s.iters = filt ? ss.iters : 0;
                s.dropped = filt ? ss.dropped : 0.0;
                s.fma = (int64_t)ss.fma;
                fma += ss.fma;
                r->steps.push_back(s);
            }
        }
        // the column windows of this evaluation's steps, for the series' next one
        {
            std::vector<unsigned> sz, sb((size_t)(p.q > 1 ? p.q - 1 : 0), 0u),
                sg((size_t)(p.b > 1 ? p.b - 1 : 0), 0u);
            if (chain[(size_t)i]) {
                sz.assign(9, 0u);
                for (int k = 2; k <= 10; ++k) sz[(size_t)(k - 2)] = zst[(size_t)(k - 2) * count + (size_t)i].span_max;
            }
            for (size_t si = 0; si < nst && !P.trivial; ++si) {
                const StageDesc& D = stages[si];
                if (tabs[si].step[(size_t)i].mode != kBatchProduct) continue;
                const unsigned sp = pst[si * (size_t)count + (size_t)i].span_max;
                if (D.kind == 0 && D.index - 2 >= 0 && (size_t)(D.index - 2) < sb.size()) sb[(size_t)(D.index - 2)] = sp;
                if (D.kind == 1 && D.index - 1 >= 0 && (size_t)(D.index - 1) < sg.size()) sg[(size_t)(D.index - 1)] = sp;
            }
            std::lock_guard<std::mutex> lock(series[i]->span_mu);
            if (chain[(size_t)i]) series[i]->span_z = sz;
            series[i]->span_baby = sb;
            series[i]->span_giant = sg;
        }
        psf_info_t& inf = r->info;
        inf.N = p.N;
        inf.q = p.q;
        inf.b = p.b;
        inf.g = p.g;
        inf.products = p.products + (P.sq ? 1 + (int)P.odd : 0);
        inf.nsteps = (int32_t)r->steps.size();
        for (int k = 0; k <= 10; ++k) inf.z[k] = k < (int)p.zz.size() ? p.zz[(size_t)k] : 0.0;
        inf.alpha10 = p.alpha10;
        inf.trunc = p.trunc;
        inf.budget = p.budget;
        inf.nnz = r->nnz;
        inf.fma = (int64_t)fma;
        if (g_prof.on) g_prof.fma += (double)fma;
        outs[i] = r;
    }
    (void)z_fma_tot;
    return PSF_OK;
}

}  // namespace

extern "C" int psf_eval_batch(const psf_series_t* series, const psf_csr_t* Zs, int32_t count, void* stream,
                              psf_result_t* outs) {
    if (count < 0 || (count > 0 && (!series || !Zs || !outs))) return fail(PSF_EINVAL, "bad batch arguments");
    for (int i = 0; i < count; ++i) outs[i] = nullptr;
    if (count == 0) return PSF_OK;
    for (int i = 0; i < count; ++i) {
        if (!series[i]) return fail(PSF_EINVAL, "batch instance %d: null series", i);
        if (series[i]->flags & PSF_Z_ESTIMATE)
            return fail(PSF_EINVAL, "batch instance %d: PSF_Z_ESTIMATE is for psf_eval only", i);
        int rc = check_csr(&Zs[i], Zs[i].n, "Z");
        if (rc) return rc;
        if (Zs[i].n == 0 && Zs[i].nnz != 0) return fail(PSF_EINVAL, "batch instance %d: n = 0 with entries", i);
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = prepare(st);
    if (rc) return rc;
    // groups of at most kMaxBatchInst instances and kMaxBatchRows rows
    int start = 0;
    while (start < count) {
        int end = start;
        long long rows = 0;
        while (end < count && end - start < kMaxBatchInst && (end == start || rows + Zs[end].n <= kMaxBatchRows)) {
            rows += Zs[end].n;
            ++end;
        }
        if (rows > INT32_MAX / 2) {
            rc = fail(PSF_ETOOBIG, "batch instance %d: n = %d too large", start, Zs[start].n);
        } else {
            rc = eval_group(series + start, Zs + start, end - start, st, outs + start);
        }
        if (rc) {
            for (int i = 0; i < count; ++i) {
                if (outs[i]) destroy_result(outs[i]);
                outs[i] = nullptr;
            }
            return rc;
        }
        start = end;
    }
    return PSF_OK;
}

// ---- psf_autotune_batch

namespace {

// One psf_eval_batch, its results released.
int run_batch_once(const psf_series_t* series, const psf_csr_t* Z, int32_t count, void* stream) {
    std::vector<psf_result_t> outs((size_t)count, nullptr);
    const int rc = psf_eval_batch(series, Z, count, stream, outs.data());
    for (psf_result_t r : outs)
        if (r) psf_result_destroy(r);
    return rc;
}

// Median event-timed milliseconds of `reps` psf_eval_batch calls.
int time_batch(const psf_series_t* series, const psf_csr_t* Z, int32_t count, void* stream, int reps, double* ms) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    std::vector<double> t;
    int rc = err == cudaSuccess ? PSF_OK : fail(PSF_ECUDA, "autotune events: %s", cudaGetErrorString(err));
    for (int i = 0; i < reps && rc == PSF_OK; ++i) {
        float v = 0.0f;
        if ((err = cudaEventRecord(e0, st)) != cudaSuccess) break;
        if ((rc = run_batch_once(series, Z, count, stream))) break;
        if ((err = cudaEventRecord(e1, st)) != cudaSuccess || (err = cudaEventSynchronize(e1)) != cudaSuccess ||
            (err = cudaEventElapsedTime(&v, e0, e1)) != cudaSuccess)
            break;
        t.push_back(v);
    }
    if (rc == PSF_OK && err != cudaSuccess) rc = fail(PSF_ECUDA, "autotune timing: %s", cudaGetErrorString(err));
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return PSF_OK;
}

// The batch once with the slot-map crossover `c`, every product launch timed.
int time_launches(const psf_series_t* series, const psf_csr_t* Z, int32_t count, void* stream, double c,
                  std::vector<double>& work, std::vector<double>& ms) {
    TuneRecorder rec;
    const double saved = g_table_crossover.load();
    g_table_crossover.store(c);
    g_tune_rec = &rec;
    int rc = run_batch_once(series, Z, count, stream);
    g_tune_rec = nullptr;
    g_table_crossover.store(saved);
    if (rc == PSF_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        rc = fail(PSF_ECUDA, "autotune sync");
    for (auto& pr : rec.ev) {
        float t = 0.0f;
        if (rc == PSF_OK && cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess)
            rc = fail(PSF_ECUDA, "autotune timing");
        ms.push_back(t);
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    work = rec.work;
    return rc;
}

}  // namespace

extern "C" int psf_autotune_batch(const psf_series_t* series, const psf_csr_t* Z, int32_t count, void* stream,
                                  psf_batch_tune_t* out) {
    if (!series || !Z || !out || count <= 0) return fail(PSF_EINVAL, "null argument or empty batch");
    *out = psf_batch_tune_t{};
    const double c0 = g_table_crossover.load();
    const int bm0 = g_row_bitmaps.load();
    const bool reuse0 = g_batch_reuse.load();
    int rc = run_batch_once(series, Z, count, stream);  // warm-up: sizes are learnt
    if (rc == PSF_OK) rc = time_batch(series, Z, count, stream, 3, &out->ms_before);
    if (rc) return rc;
    // the slot map per launch: the table everywhere, then the bitmap everywhere
    std::vector<double> work[2], ms[2];
    rc = time_launches(series, Z, count, stream, 0.0, work[0], ms[0]);
    if (rc == PSF_OK) rc = time_launches(series, Z, count, stream, 1e300, work[1], ms[1]);
    if (rc) return rc;
    if (work[0] != work[1]) return fail(PSF_ECUDA, "autotune: the two runs launched different products");
    double best_c = 1e300, best_t = 0.0;
    for (double v : ms[1]) best_t += v;  // never the table
    for (double c : work[0]) {
        double t = 0.0;
        for (size_t i = 0; i < work[0].size(); ++i) t += work[0][i] >= c ? ms[0][i] : ms[1][i];
        if (t < best_t || (t == best_t && c > best_c)) {
            best_t = t;
            best_c = c;
        }
    }
    out->launches = (int32_t)work[0].size();
    // row bitmaps and baby-step reuse, as whole batches with that crossover
    double best_ms = std::numeric_limits<double>::infinity();
    int best_bm = bm0;
    bool best_reuse = reuse0;
    g_table_crossover.store(best_c);
    for (int bm = 0; bm <= 1 && rc == PSF_OK; ++bm) {
        for (int ru = 0; ru <= 1 && rc == PSF_OK; ++ru) {
            g_row_bitmaps.store(bm);
            g_batch_reuse.store(ru != 0);
            double t = 0.0;
            rc = run_batch_once(series, Z, count, stream);  // the pool for this setting
            if (rc == PSF_OK) rc = time_batch(series, Z, count, stream, 3, &t);
            ++out->configs;
            if (rc == PSF_OK && t < best_ms) {
                best_ms = t;
                best_bm = bm;
                best_reuse = ru != 0;
            }
        }
    }
    if (rc) {
        g_table_crossover.store(c0);
        g_row_bitmaps.store(bm0);
        g_batch_reuse.store(reuse0);
        return rc;
    }
    g_row_bitmaps.store(best_bm);
    g_batch_reuse.store(best_reuse);
    out->table_crossover = best_c;
    out->row_bitmaps = best_bm;
    out->batch_reuse = best_reuse ? 1 : 0;
    out->ms_after = best_ms;
    return PSF_OK;
}
