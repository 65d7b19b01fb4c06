// psf_normest.cu -- deterministic estimates of ||Z^k||_1, k = 2..10, on the
// device (series flag PSF_Z_ESTIMATE; Sec. 3.2.2, Eq. 37).
//
// The paper takes ||Z^i||, i <= 10, from Higham's normest1.  This is the
// deterministic single-vector core of that method: Hager's 1-norm power
// iteration with Higham's stopping rules and alternating test vector.  For
// A = Z^k:
//   1. x = (1/n, ..., 1/n); v = A x; best = ||v||_1 (n = 1: done).
//   2. s = sgn(v); w = A^T s.
//   3. Repeat: j = the smallest index maximising |w_j|; stop if the previous
//      index p has |w_p| = |w_j|, or after five products with A; v = A e_j,
//      e = ||v||_1, s' = sgn(v); if e <= best or s' = s, best = max(best, e)
//      and stop; else best = e, s = s', w = A^T s, p = j.
//   4. b_i = (-1)^i (1 + i/(n-1)); the estimate is max(best, 2||A b||_1/(3n)).
// Every operation is fixed so that the result does not depend on the launch:
// A is applied as k products with Z and A^T as k products with Z^T, each row
// of a product a chain of fma over the row's entries in stored order from +0
// (Z^T's rows in ascending row order of Z); ||v||_1 is the exactly rounded
// sum (24-bit pieces, as the norm phase); sgn(t) = -1 for t < 0, else +1.
//
// The nine powers run in lock step, one column each of an n x 9 block of
// vectors: a product phase is ten launches, column c (power c + 2) taking
// part in the last c + 2 of them, so every column sees exactly its power.
// The host drives the iteration from a few scalars per column and round.
#include <climits>
#include <cstddef>
#include <cstring>
#include <vector>

#include "psf_internal.h"

namespace psf {
namespace {

constexpr int kCols = 9;            // powers 2..10
constexpr int kSteps = 10;          // products per phase (the largest power)
constexpr int kMaxColumn = 4096;    // longest column of Z the transposition orders
constexpr int kMaxProducts = 5;     // products with A in the power iteration
constexpr int kThreads = 256;

// entries per column of Z
__global__ void k_col_counts(int nnz, const int* col, int* counts) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += gridDim.x * blockDim.x)
        atomicAdd(&counts[col[p]], 1);
}

__global__ void k_max_count(int n, const int* counts, int* out) {
    int m = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) m = max(m, counts[c]);
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// Z^T, unordered: row c of Z^T gets the entries of column c of Z in any order
__global__ void k_transpose_fill(int n, const int* rowptr, const int* col, const double* val, const int* rpt,
                                 int* cursor, int* tcol, double* tval) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
            const int c = col[p];
            const int pos = rpt[c] + atomicAdd(&cursor[c], 1);
            tcol[pos] = r;
            tval[pos] = val[p];
        }
}

// Put every row of Z^T in ascending row order of Z: one warp per row; an
// entry's place is the number of the row's entries with a smaller key (the
// keys, Z's row indices, are distinct within a row).
__global__ void k_transpose_order(int n, const int* rpt, const int* scol, const double* sval, int* tcol,
                                  double* tval) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += nw) {
        const int s = rpt[c], e = rpt[c + 1];
        for (int i0 = s; i0 < e; i0 += 32) {
            const int i = i0 + lane;
            const int key = i < e ? scol[i] : INT_MAX;
            int rank = 0;
            for (int q0 = s; q0 < e; q0 += 32) {
                const int other = q0 + lane < e ? scol[q0 + lane] : INT_MAX;
                for (int t = 0; t < 32; ++t) rank += __shfl_sync(kFull, other, t) < key ? 1 : 0;
            }
            if (i < e) {
                tcol[s + rank] = key;
                tval[s + rank] = sval[i];
            }
        }
    }
}

// Y = M X for the columns c >= c_lo of the n x kCols block (row-major);
// the other columns pass through unchanged.
__global__ void k_spmv_block(int n, const int* rowptr, const int* col, const double* val, int c_lo,
                             const double* X, double* Y) {
    const long long total = (long long)n * kCols;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(u / kCols), c = (int)(u % kCols);
        if (c < c_lo) {
            Y[u] = X[u];
            continue;
        }
        double acc = 0.0;
        for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) acc = __fma_rn(val[p], X[(size_t)col[p] * kCols + c], acc);
        Y[u] = acc;
    }
}

// Test vectors: kind 0 x = 1/n, kind 1 x = e_j, kind 2 the alternating b.
__global__ void k_set_x(int n, const int* kind, const int* j, double* X) {
    const long long total = (long long)n * kCols;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(u / kCols), c = (int)(u % kCols);
        double x;
        if (kind[c] == 0) {
            x = 1.0 / (double)n;
        } else if (kind[c] == 1) {
            x = r == j[c] ? 1.0 : 0.0;
        } else {
            x = 1.0 + (double)r / (double)(n - 1);
            if (r & 1) x = -x;
        }
        X[u] = x;
    }
}

// Scalars of the iteration, per column (device side; the host reads them
// back each round).
struct EstScal {
    unsigned long long maxbits[kCols];  // max |x| (bits) of a column
    unsigned long long wprev[kCols];    // |w_p| (bits) at the previous index p
    double sums[kCols];                 // ||v||_1, exactly rounded
    int jmin[kCols];                    // smallest index maximising |w_j|
    int changed[kCols];                 // sgn(v) differs from the current signs
    int kind[kCols];                    // test vector of the next forward phase
    int j[kCols];
    int prev[kCols];                    // previous index p (-1: none)
    unsigned sticky[kCols];
    int maxcnt;                         // longest column of Z
};

// max |x| per column, and |w_p| at the previous index of each column
__global__ void k_col_absmax(int n, const double* V, EstScal* sc) {
    __shared__ unsigned long long m[kCols];
    if (threadIdx.x < kCols) m[threadIdx.x] = 0ull;
    __syncthreads();
    const long long total = (long long)n * kCols;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(u / kCols), c = (int)(u % kCols);
        const unsigned long long xb = mag_bits(V[u]);
        if (xb) atomicMax(&m[c], xb);
        if (r == sc->prev[c]) sc->wprev[c] = xb;
    }
    __syncthreads();
    if (threadIdx.x < kCols && m[threadIdx.x]) atomicMax(&sc->maxbits[threadIdx.x], m[threadIdx.x]);
}

// smallest index whose |x| is the column's maximum
__global__ void k_col_argmax(int n, const double* V, EstScal* sc) {
    const long long total = (long long)n * kCols;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(u / kCols), c = (int)(u % kCols);
        if (mag_bits(V[u]) == sc->maxbits[c]) atomicMin(&sc->jmin[c], r);
    }
}

// Exact sum of |x| per column: each block sums its rows in 24-bit pieces in
// shared memory (at most kThreads rows: a 32-bit word cannot overflow) and
// adds them to the column's global pieces once.
__global__ void __launch_bounds__(kThreads) k_col_asum(int n, const double* V, EstScal* sc,
                                                      unsigned long long* words) {
    __shared__ unsigned piece[kCols][kNormPieces];
    __shared__ unsigned st[kCols];
    for (int i = threadIdx.x; i < kCols * kNormPieces; i += blockDim.x) piece[i / kNormPieces][i % kNormPieces] = 0u;
    if (threadIdx.x < kCols) st[threadIdx.x] = 0u;
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        for (int c = 0; c < kCols; ++c) {
            const unsigned long long xb = mag_bits(V[(size_t)r * kCols + c]);
            if (!xb) continue;
            unsigned pc[4];
            bool lost;
            const int L = split24(xb, lsb_for_bound(sc->maxbits[c]), pc, lost);
            for (int q = 0; q < 4; ++q)
                if (pc[q]) atomicAdd(&piece[c][L + q], pc[q]);
            if (lost) atomicAdd(&st[c], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCols * kNormPieces; i += blockDim.x) {
        const unsigned v = piece[i / kNormPieces][i % kNormPieces];
        if (v) atomicAdd(&words[i], (unsigned long long)v);
    }
    if (threadIdx.x < kCols && st[threadIdx.x]) atomicAdd(&sc->sticky[threadIdx.x], st[threadIdx.x]);
}

__global__ void k_col_round(EstScal* sc, unsigned long long* words) {
    const int c = threadIdx.x;
    if (c < kCols)
        sc->sums[c] = round24(words + (size_t)c * kNormPieces, 1, &sc->sticky[c], lsb_for_bound(sc->maxbits[c]));
}

// S_new = sgn(V); flag the columns whose signs differ from S_cur
__global__ void k_signs(int n, const double* V, const double* S_cur, double* S_new, EstScal* sc) {
    __shared__ int ch[kCols];
    if (threadIdx.x < kCols) ch[threadIdx.x] = 0;
    __syncthreads();
    const long long total = (long long)n * kCols;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        const double s = V[u] < 0.0 ? -1.0 : 1.0;
        S_new[u] = s;
        if (s != S_cur[u]) ch[(int)(u % kCols)] = 1;
    }
    __syncthreads();
    if (threadIdx.x < kCols && ch[threadIdx.x]) atomicOr(&sc->changed[threadIdx.x], 1);
}

}  // namespace
}  // namespace psf

namespace psf {
namespace host {

int estimate_power_norms(Work& w, const psf_csr_t& Z, double* norms, bool* fallback) {
    *fallback = false;
    const int n = Z.n, nnz = Z.nnz;
    cudaStream_t st = w.st;
    if (n == 0) {
        for (int k = 2; k <= 10; ++k) norms[k] = 0.0;
        return PSF_OK;
    }
    const size_t nb = (size_t)n * kCols;
    DevBuf counts, cursor, zeros, rpt, scol, sval, tcol, tval, X, Y, Sg, Sn, scb, words;
    CU(counts.alloc(sizeof(int) * (size_t)n, st));
    CU(cursor.alloc(sizeof(int) * (size_t)n, st));
    CU(zeros.alloc(sizeof(int) * (size_t)n, st));
    CU(rpt.alloc(sizeof(int) * ((size_t)n + 1), st));
    CU(scol.alloc(sizeof(int) * (size_t)nnz, st));
    CU(sval.alloc(sizeof(double) * (size_t)nnz, st));
    CU(tcol.alloc(sizeof(int) * (size_t)nnz, st));
    CU(tval.alloc(sizeof(double) * (size_t)nnz, st));
    CU(X.alloc(sizeof(double) * nb, st));
    CU(Y.alloc(sizeof(double) * nb, st));
    CU(Sg.alloc(sizeof(double) * nb, st));
    CU(Sn.alloc(sizeof(double) * nb, st));
    CU(scb.alloc(sizeof(EstScal), st));
    CU(words.alloc(sizeof(unsigned long long) * kCols * kNormPieces, st));
    CU(cudaMemsetAsync(counts.p, 0, sizeof(int) * (size_t)n, st));
    CU(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (size_t)n, st));
    CU(cudaMemsetAsync(zeros.p, 0, sizeof(int) * (size_t)n, st));
    CU(cudaMemsetAsync(scb.p, 0, sizeof(EstScal), st));
    CU(cudaMemsetAsync(words.p, 0, sizeof(unsigned long long) * kCols * kNormPieces, st));
    EstScal* sc = scb.as<EstScal>();
    EstScal h{};
    int launches = 0;
    const int sms = num_sms();
    auto grid = [&](long long items) {
        long long g = (items + kThreads - 1) / kThreads;
        if (g > (long long)sms * 8) g = (long long)sms * 8;
        return (unsigned)(g > 0 ? g : 1);
    };
    auto launched = [&]() -> int {
        ++launches;
        CU(cudaGetLastError());
        return PSF_OK;
    };
    auto read = [&]() -> int {
        CU(cudaMemcpyAsync(&h, sc, sizeof h, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        return PSF_OK;
    };
    auto upload_choice = [&]() -> int {  // kind, j and prev, contiguous in EstScal
        CU(cudaMemcpyAsync(reinterpret_cast<char*>(sc) + offsetof(EstScal, kind), &h.kind,
                           sizeof(int) * 3 * kCols, cudaMemcpyHostToDevice, st));
        return PSF_OK;
    };
    int rc;

    // ---- Z^T with every row in ascending row order of Z
    k_col_counts<<<grid(nnz), kThreads, 0, st>>>(nnz, Z.col, counts.as<int>());
    if ((rc = launched())) return rc;
    k_max_count<<<grid(n), kThreads, 0, st>>>(n, counts.as<int>(), &sc->maxcnt);
    if ((rc = launched()) || (rc = read())) return rc;
    if (h.maxcnt > kMaxColumn) {
        count_launches(launches);
        *fallback = true;
        return PSF_OK;
    }
    CU(launch_scan_rows(n, zeros.as<int>(), counts.as<int>(), rpt.as<int>(), w.C(), w.scan.as<long long>(), st));
    k_transpose_fill<<<grid(n), kThreads, 0, st>>>(n, Z.rowptr, Z.col, Z.val, rpt.as<int>(), cursor.as<int>(),
                                                   scol.as<int>(), sval.as<double>());
    if ((rc = launched())) return rc;
    k_transpose_order<<<grid((long long)n * 32), kThreads, 0, st>>>(n, rpt.as<int>(), scol.as<int>(),
                                                                   sval.as<double>(), tcol.as<int>(),
                                                                   tval.as<double>());
    if ((rc = launched())) return rc;

    // ---- building blocks
    double* Xp = X.as<double>();
    double* Yp = Y.as<double>();
    // ten products: column c takes part in the last c + 2; the result ends in X
    auto phase = [&](const int* rp, const int* ci, const double* v) -> int {
        double* a = Xp;
        double* b = Yp;
        for (int t = 1; t <= kSteps; ++t) {
            const int c_lo = kCols - t > 0 ? kCols - t : 0;
            k_spmv_block<<<grid((long long)nb), kThreads, 0, st>>>(n, rp, ci, v, c_lo, a, b);
            int e = launched();
            if (e) return e;
            std::swap(a, b);
        }
        return PSF_OK;  // an even number of swaps: the result is in X
    };
    auto forward = [&]() -> int {
        int e = upload_choice();
        if (e) return e;
        k_set_x<<<grid((long long)nb), kThreads, 0, st>>>(n, sc->kind, sc->j, Xp);
        if ((e = launched())) return e;
        return phase(Z.rowptr, Z.col, Z.val);
    };
    auto transposed = [&](const double* S) -> int {
        CU(cudaMemcpyAsync(Xp, S, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
        return phase(rpt.as<int>(), tcol.as<int>(), tval.as<double>());
    };
    auto col_sums = [&]() -> int {  // exact ||X[:, c]||_1 into sums
        CU(cudaMemsetAsync(sc->maxbits, 0, sizeof(h.maxbits), st));
        CU(cudaMemsetAsync(sc->sticky, 0, sizeof(h.sticky), st));
        k_col_absmax<<<grid((long long)nb), kThreads, 0, st>>>(n, Xp, sc);
        int e = launched();
        if (e) return e;
        k_col_asum<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(n, Xp, sc, words.as<unsigned long long>());
        if ((e = launched())) return e;
        k_col_round<<<1, 32, 0, st>>>(sc, words.as<unsigned long long>());
        return launched();
    };
    auto argmax = [&]() -> int {  // of |X[:, c]|, and |X[p_c, c]|
        int e = upload_choice();
        if (e) return e;
        CU(cudaMemsetAsync(sc->maxbits, 0, sizeof(h.maxbits), st));
        CU(cudaMemsetAsync(sc->jmin, 0x7f, sizeof(h.jmin), st));
        k_col_absmax<<<grid((long long)nb), kThreads, 0, st>>>(n, Xp, sc);
        if ((e = launched())) return e;
        k_col_argmax<<<grid((long long)nb), kThreads, 0, st>>>(n, Xp, sc);
        if ((e = launched())) return e;
        return read();
    };

    // ---- 1-2: x = e/n, best = ||A x||_1, s = sgn(A x), w = A^T s
    double best[kCols];
    int products[kCols];
    bool run[kCols];
    for (int c = 0; c < kCols; ++c) {
        h.kind[c] = 0;
        h.j[c] = 0;
        h.prev[c] = -1;
        products[c] = 1;
        run[c] = true;
    }
    double* sg = Sg.as<double>();
    double* sn = Sn.as<double>();
    if ((rc = forward()) || (rc = col_sums())) return rc;
    k_signs<<<grid((long long)nb), kThreads, 0, st>>>(n, Xp, sg, sg, sc);
    if ((rc = launched()) || (rc = read())) return rc;
    for (int c = 0; c < kCols; ++c) best[c] = h.sums[c];
    if (n > 1) {
        if ((rc = transposed(sg)) || (rc = argmax())) return rc;
        // ---- 3: the power iteration
        for (;;) {
            bool any = false;
            for (int c = 0; c < kCols; ++c) {
                h.kind[c] = 0;
                if (!run[c]) continue;
                if ((h.prev[c] >= 0 && h.wprev[c] == h.maxbits[c]) || products[c] == kMaxProducts) {
                    run[c] = false;
                    continue;
                }
                h.kind[c] = 1;
                h.j[c] = h.jmin[c];
                any = true;
            }
            if (!any) break;
            if ((rc = forward()) || (rc = col_sums())) return rc;
            CU(cudaMemsetAsync(sc->changed, 0, sizeof(h.changed), st));
            k_signs<<<grid((long long)nb), kThreads, 0, st>>>(n, Xp, sg, sn, sc);
            if ((rc = launched()) || (rc = read())) return rc;
            bool more = false;
            for (int c = 0; c < kCols; ++c) {
                if (h.kind[c] != 1) continue;
                ++products[c];
                const double e = h.sums[c];
                if (e <= best[c] || !h.changed[c]) {
                    best[c] = e > best[c] ? e : best[c];
                    run[c] = false;
                } else {
                    best[c] = e;
                    h.prev[c] = h.j[c];
                    more = true;
                }
            }
            if (!more) break;
            std::swap(sg, sn);  // the continuing columns' new signs become current
            if ((rc = transposed(sg)) || (rc = argmax())) return rc;
        }
        // ---- 4: the alternating test vector
        for (int c = 0; c < kCols; ++c) h.kind[c] = 2;
        if ((rc = forward()) || (rc = col_sums()) || (rc = read())) return rc;
        for (int c = 0; c < kCols; ++c) {
            const double alt = (2.0 * h.sums[c]) / (3.0 * (double)n);
            if (alt > best[c]) best[c] = alt;
        }
    }
    for (int c = 0; c < kCols; ++c) norms[c + 2] = best[c];
    count_launches(launches);
    return PSF_OK;
}

}  // namespace host
}  // namespace psf
