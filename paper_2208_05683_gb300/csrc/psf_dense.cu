// psf_dense.cu -- the dense-tile form of one product step,
//   C = sum_t alpha_t M_t + A B,
// for products whose operands have filled in: the step runs as an FP64 dense
// tile product instead of the row-by-row sparse kernel once its multiply-adds
// per n^2 output entries pass a measured crossover.
//
//  k_dense_rows    pooled CSR rows -> a dense row-major n x n matrix
//  k_dense_addends the weighted sum of the addends, t ascending, as dense
//                  rows: the accumulator's starting values
//  k_dense_gemm    c_ij = fma(a_ik, b_kj, c_ij) for k = 0, 1, .., n - 1 in
//                  order, 64 x 64 output tiles, 16-deep k slices staged in
//                  shared memory, 4 x 4 outputs per thread
//  k_dense_out     the nonzero entries of each row into the pool, in column
//                  order, with Algorithm 1's first pass (exact column sums
//                  and the candidate list of the entries |x| <= eps_g), as
//                  the sparse kernel's write-back
//
// Rounding order.  The sparse kernel folds each output entry as: start from
// 0, the addends in order t = 0, 1, ..., then a_rk b_kj for k ascending over
// A's row.  The dense fold visits the same terms in the same order and in
// between adds products in which a factor is zero: fma(0, b, c) and
// fma(a, 0, c) return c unchanged for any finite c other than a signed zero,
// and a zero result is never stored, so the stored entries are bit for bit
// those of the sparse kernel.
#include "psf_device.cuh"
#include "psf_kernels.h"

namespace psf {

// ---------------------------------------------------------------- k_dense_rows
// One warp per row: D[r][col] = val for the row's entries (D zero before).
__global__ void k_dense_rows(int n, RowView M, double* D) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < n; r += nw) {
        double* row = D + (size_t)r * n;
        const int s = M.rb[r], e = M.re[r];
        for (int q = s + lane; q < e; q += 32) {
            const double v = M.val[q];
            if (mag_bits(v) != 0ull) row[M.col[q]] = v;  // the pool's padding holds zeros
        }
    }
}

// ---------------------------------------------------------------- k_dense_addends
// One warp per row: the addends folded in order t = 0, 1, ... as
// D[r][j] = fma(alpha_t, m_rj, D[r][j]) (D zero before), the identity as m_rr = 1.
struct DenseAddArgs {
    int n;
    int nadd;
    AddTerm add[kMaxAdd];
};

__global__ void k_dense_addends(DenseAddArgs A, double* D) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < A.n; r += nw) {
        double* row = D + (size_t)r * A.n;
        for (int t = 0; t < A.nadd; ++t) {
            const AddTerm& T = A.add[t];
            if (!T.rb) {
                if (lane == 0) row[r] = __fma_rn(T.alpha, 1.0, row[r]);
            } else {
                for (int q = T.rb[r] + lane; q < T.re[r]; q += 32) {
                    const double v = T.val[q];
                    if (mag_bits(v) != 0ull) row[T.col[q]] = __fma_rn(T.alpha, v, row[T.col[q]]);
                }
            }
            __syncwarp();  // term t + 1 may touch the columns term t touched
        }
    }
}

// ---------------------------------------------------------------- k_dense_gemm
// C = C + A B with every output entry folded k = 0, 1, ..., n - 1 in order.
// 256 threads own a 64 x 64 tile of C, thread (tx, ty) the rows ty + 16 i and
// columns tx + 16 j, i, j < 4.  Slices of 16 k are staged in shared memory
// (A transposed), the next slice's global loads in registers while the
// current one is folded.  Out-of-range rows, columns and k read as zeros.
constexpr int kDT = 64;   // output tile
constexpr int kDK = 16;   // k slice

__global__ void __launch_bounds__(256) k_dense_gemm(int n, const double* __restrict__ A, const double* __restrict__ B,
                                                    double* C) {
    __shared__ double As[2][kDK][kDT + 1];  // padded: the transposing stores hit distinct banks
    __shared__ double Bs[2][kDK][kDT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * kDT, j0 = blockIdx.x * kDT;
    // each thread loads 4 A and 4 B values per slice: A rows i0 + (t >> 4) +
    // 16 u, k offset t & 15; B row k0 + (t >> 6) + 4 u, column j0 + (t & 63)
    const int t = threadIdx.x;
    double ra[4], rb[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ia = i0 + (t >> 4) + 16 * u, ka = k0 + (t & 15);
            ra[u] = (ia < n && ka < n) ? A[(size_t)ia * n + ka] : 0.0;
            const int kb = k0 + (t >> 6) + 4 * u, jb = j0 + (t & 63);
            rb[u] = (kb < n && jb < n) ? B[(size_t)kb * n + jb] : 0.0;
        }
    };
    auto stage = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            As[buf][t & 15][(t >> 4) + 16 * u] = ra[u];
            Bs[buf][(t >> 6) + 4 * u][t & 63] = rb[u];
        }
    };
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
            acc[i][j] = (r < n && c < n) ? C[(size_t)r * n + c] : 0.0;
        }
    load(0);
    stage(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < n; k0 += kDK) {
        const bool more = k0 + kDK < n;
        if (more) load(k0 + kDK);
#pragma unroll
        for (int k = 0; k < kDK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[buf][k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[buf][k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = __fma_rn(a[i], b[j], acc[i][j]);
        }
        if (more) {
            stage(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
            if (r < n && c < n) C[(size_t)r * n + c] = acc[i][j];
        }
}

// ---------------------------------------------------------------- k_dense_out
// One warp per row of the dense C: count its nonzero entries, reserve them in
// the pool, write them in column order; entries with |x| <= eps_g enter
// Algorithm 1's first pass.  The step statistics are those of the sparse
// kernel, multiply-adds included (sum over A's row of B's row lengths plus
// the addend entries: the work of the method, not of the dense tiles).
__global__ void __launch_bounds__(256) k_dense_out(ProductArgs P, const double* __restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n = P.n;
    const unsigned long long eps_bits = (unsigned long long)__double_as_longlong(P.eps_g);
    const bool filt = P.filtering != 0;
    unsigned long long my_written = 0ull, my_cand = 0ull, my_absmax = 0ull, my_fma = 0ull;
    Arena arena;
    CandArena carena;
    for (int r = gw; r < n; r += nw) {
        const double* row = C + (size_t)r * n;
        if (P.A.rb)
            for (int p = P.A.rb[r] + lane; p < P.A.re[r]; p += 32) {
                const int k = P.A.col[p];
                my_fma += (unsigned long long)(P.B.re[k] - P.B.rb[k]);
            }
        if (lane == 0)
            for (int t = 0; t < P.nadd; ++t)
                my_fma += P.add[t].rb ? (unsigned long long)(P.add[t].re[r] - P.add[t].rb[r]) : 1ull;
        int cnt = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            cnt += __popc(__ballot_sync(kFull, j < n && mag_bits(row[j]) != 0ull));
        }
        if (cnt == 0) {
            if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
            continue;
        }
        const unsigned long long span = ((unsigned long long)cnt + 3ull) & ~3ull;
        const long long base = arena_take(arena, span, P.arena, P.ctl, P.pool_val, lane);
        if (base < 0) {
            if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
            continue;
        }
        int written = 0;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            const double x = j < n ? row[j] : 0.0;
            const unsigned long long xb = mag_bits(x);
            const bool nz = xb != 0ull;
            const unsigned m = __ballot_sync(kFull, nz);
            if (!m) continue;
            const bool cand = nz && filt && xb <= eps_bits;
            if (nz) {
                const long long pos = base + written + __popc(m & lanemask_lt());
                P.pool_col[pos] = j;
                P.pool_val[pos] = x;
                my_absmax = xb > my_absmax ? xb : my_absmax;
                if (cand) {
                    exact_add(P.words + j, (size_t)n, P.sticky + j, xb, P.e_lsb);
                    ++my_cand;
                }
            }
            if (P.cand_col)
                cand_push(carena, cand, j, xb, P.cand_col, P.cand_x, &P.ctl->cand_cnt[0], P.cand_cap, P.cand_chunk,
                          &P.ctl->cand_over, lane);
            written += __popc(m);
        }
        for (long long q = base + cnt + lane; q < base + (long long)span; q += 32) P.pool_val[q] = 0.0;
        if (lane == 0) {
            P.out_rb[r] = (int)base;
            P.out_re[r] = (int)(base + cnt);
            my_written += (unsigned long long)cnt;
        }
    }
    arena_close(arena, P.pool_val, lane);
    if (P.cand_col) cand_close(carena, P.cand_x, lane);
    my_cand = (unsigned long long)warp_sum((int)my_cand);
    my_absmax = warp_max_u64(my_absmax);
    for (int o = 16; o; o >>= 1) my_fma += __shfl_xor_sync(kFull, my_fma, o);
    if (lane == 0) {
        if (my_fma) atomicAdd(&P.ctl->fma_total, my_fma);
        if (P.stat) {
            if (my_fma) atomicAdd(&P.stat->fma, my_fma);
            if (my_written) atomicAdd(&P.stat->nnz_pre, my_written);
            if (my_cand) atomicAdd(&P.stat->ncand, my_cand);
        }
        if (P.absmax_slot && my_absmax) atomicMax(&P.absmax_slot->absmax, my_absmax);
    }
}

// ---------------------------------------------------------------- launcher
cudaError_t launch_dense_product(const ProductArgs& P, double* Ad, double* Bd, double* Cd, cudaStream_t st) {
    const int n = P.n;
    if (n <= 0) return cudaSuccess;
    const size_t bytes = sizeof(double) * (size_t)n * (size_t)n;
    const int rows_blocks = (n + 7) / 8;  // 8 warps (rows) per block
    cudaError_t err = cudaMemsetAsync(Cd, 0, bytes, st);
    if (err != cudaSuccess) return err;
    DenseAddArgs D{};
    D.n = n;
    D.nadd = P.nadd;
    for (int t = 0; t < P.nadd; ++t) D.add[t] = P.add[t];
    if (P.nadd > 0) {
        k_dense_addends<<<rows_blocks, 256, 0, st>>>(D, Cd);
        count_launches(1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (P.A.rb) {
        if ((err = cudaMemsetAsync(Ad, 0, bytes, st)) != cudaSuccess) return err;
        if ((err = cudaMemsetAsync(Bd, 0, bytes, st)) != cudaSuccess) return err;
        k_dense_rows<<<rows_blocks, 256, 0, st>>>(n, P.A, Ad);
        k_dense_rows<<<rows_blocks, 256, 0, st>>>(n, P.B, Bd);
        const dim3 grid((unsigned)((n + kDT - 1) / kDT), (unsigned)((n + kDT - 1) / kDT));
        k_dense_gemm<<<grid, 256, 0, st>>>(n, Ad, Bd, Cd);
        count_launches(3);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // every row reserves exactly its own (rounded) entry count
    ProductArgs Q = P;
    Q.arena = 4;
    k_dense_out<<<rows_blocks, 256, 0, st>>>(Q, Cd);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace psf
