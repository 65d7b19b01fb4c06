// psf_kernels.cu -- CUDA kernels of the filtered Paterson-Stockmeyer
// evaluator (sm_103a, FP64 throughout).
//
//  k_product      one fused step C = sum_t alpha_t M_t + A B: column window,
//                 bitmap of the output pattern, exact per-row reservation in
//                 the pool, FP64 accumulation in shared memory, write-back of
//                 the nonzero entries, and the first pass of Algorithm 1
//                 (exact column sums of the entries |x| <= eps_g).
//  k_alg1         the remaining passes of Algorithm 1 (Sec. 3.1.1) and the
//                 final in-place compaction, one cooperative launch.
//  k_norms        exact 1-norms of up to 11 matrices (Eq. 37's z_i).
//  k_absmax, k_validate, k_scan_rows, k_gather, k_identity: plumbing.
#include <atomic>
#include <climits>

#include "psf_device.cuh"
#include "psf_kernels.h"

namespace psf {

// ---------------------------------------------------------------- k_product
// One warp computes one output row.  Shared memory per warp:
//   bm[kBmWords]      bitmap of output columns in the chunk [c0, c0 + 32 kBmWords)
//   prefix[kBmWords]  number of set bits before each bitmap word
//   colbuf[kAccCap]   column of each accumulator slot (ascending)
//   acc[kAccCap]      FP64 accumulators, slot = rank of the column in the chunk
// A row whose pattern exceeds a chunk (wider than the bitmap or with more
// than kAccCap entries) is processed in several chunks.
constexpr int kBmWords = 256;
constexpr int kBmBits = kBmWords * 32;
constexpr int kAccCap = 1024;
constexpr int kProdWarps = 4;

struct WarpSmem {
    unsigned bm[kBmWords];
    int prefix[kBmWords];
    int colbuf[kAccCap];
    double acc[kAccCap];
};

size_t product_smem_bytes() { return sizeof(WarpSmem) * kProdWarps + sizeof(AddTerm) * kMaxAdd; }
int product_warps_per_block() { return kProdWarps; }

__device__ __forceinline__ void bm_set(WarpSmem& S, int off) {
    atomicOr(&S.bm[off >> 5], 1u << (off & 31));
}

__device__ __forceinline__ int slot_of(const WarpSmem& S, int off) {
    int w = off >> 5, b = off & 31;
    return S.prefix[w] + __popc(S.bm[w] & ((1u << b) - 1u));
}

// first position in [s, e) with col >= c (col ascending)
__device__ __forceinline__ int lower_bound_col(const int* col, int s, int e, int c) {
    while (s < e) {
        int mid = (s + e) >> 1;
        if (col[mid] < c) s = mid + 1;
        else e = mid;
    }
    return s;
}

// Set the bitmap bits of every candidate output column in [c0, cend) of row r.
__device__ void build_bitmap(const ProductArgs& P, const AddTerm* add, int r, int c0, int cend,
                             int pa0, int pa1, int lane, WarpSmem& S) {
    for (int w = lane; w < kBmWords; w += 32) S.bm[w] = 0u;
    __syncwarp();
    for (int t = 0; t < P.nadd; ++t) {
        const AddTerm& T = add[t];
        if (!T.rb) {
            if (lane == 0 && r >= c0 && r < cend) bm_set(S, r - c0);
        } else {
            int s = T.rb[r], e = T.re[r];
            for (int q = s + lane; q < e; q += 32) {
                int c = T.col[q];
                if (c >= c0 && c < cend) bm_set(S, c - c0);
            }
        }
    }
    for (int p = pa0; p < pa1; ++p) {
        int k = P.A.col[p];
        int s = P.B.rb[k], e = P.B.re[k];
        for (int q = s + lane; q < e; q += 32) {
            int c = P.B.col[q];
            if (c >= c0 && c < cend) bm_set(S, c - c0);
        }
    }
    __syncwarp();
}

// prefix[] from bm[]; returns the number of set bits.
__device__ int scan_bitmap(int lane, WarpSmem& S) {
    constexpr int per = kBmWords / 32;
    int base = lane * per, s = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) s += __popc(S.bm[base + i]);
    int run = warp_excl_scan(s, lane);
    int total = __shfl_sync(kFull, run + s, 31);
#pragma unroll
    for (int i = 0; i < per; ++i) {
        S.prefix[base + i] = run;
        run += __popc(S.bm[base + i]);
    }
    __syncwarp();
    return total;
}

__device__ int count_bitmap(int lane, const WarpSmem& S) {
    int s = 0;
    for (int w = lane; w < kBmWords; w += 32) s += __popc(S.bm[w]);
    return warp_sum(s);
}

// Column at which the chunk must stop so that it holds exactly kAccCap
// entries (called when the chunk holds more).
__device__ int cut_column(int lane, const WarpSmem& S, int c0) {
    int found = INT_MAX;
    for (int w = lane; w < kBmWords; w += 32) {
        int pc = __popc(S.bm[w]);
        if (S.prefix[w] <= kAccCap && kAccCap < S.prefix[w] + pc) {
            int need = kAccCap - S.prefix[w];  // set bits of this word inside the chunk
            unsigned bits = S.bm[w];
            for (int i = 0; i < need; ++i) bits &= bits - 1u;  // drop the lowest `need`
            found = c0 + w * 32 + (__ffs(bits) - 1);
        }
    }
    return warp_min(found);
}

__global__ void __launch_bounds__(kProdWarps * 32) k_product(ProductArgs P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AddTerm* add = reinterpret_cast<AddTerm*>(smem_raw);
    WarpSmem* warps = reinterpret_cast<WarpSmem*>(smem_raw + sizeof(AddTerm) * kMaxAdd);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < P.nadd; t += blockDim.x) add[t] = P.add[t];
    __shared__ unsigned long long blk_written, blk_cand, blk_absmax, blk_fma;
    if (threadIdx.x == 0) {
        blk_fma = 0ull;
        blk_written = 0ull;
        blk_cand = 0ull;
        blk_absmax = 0ull;
    }
    __syncthreads();
    WarpSmem& S = warps[wib];
    const int r = blockIdx.x * kProdWarps + wib;
    unsigned long long my_written = 0ull, my_cand = 0ull, my_absmax = 0ull, my_fma = 0ull;

    if (r < P.n) {
        // ---- column window of row r
        int lo = INT_MAX, hi = -1;
        for (int t = 0; t < P.nadd; ++t) {
            const AddTerm& T = add[t];
            if (!T.rb) {
                lo = min(lo, r);
                hi = max(hi, r);
            } else {
                int s = T.rb[r], e = T.re[r];
                if (s < e) {
                    lo = min(lo, T.col[s]);
                    hi = max(hi, T.col[e - 1]);
                }
            }
        }
        int pa0 = 0, pa1 = 0;
        if (P.A.rb) {
            pa0 = P.A.rb[r];
            pa1 = P.A.re[r];
        }
        for (int p = pa0 + lane; p < pa1; p += 32) {
            int k = P.A.col[p];
            int s = P.B.rb[k], e = P.B.re[k];
            my_fma += (unsigned long long)(e - s);
            if (s < e) {
                lo = min(lo, P.B.col[s]);
                hi = max(hi, P.B.col[e - 1]);
            }
        }
        if (lane == 0)
            for (int t = 0; t < P.nadd; ++t)
                my_fma += add[t].rb ? (unsigned long long)(add[t].re[r] - add[t].rb[r]) : 1ull;
        lo = warp_min(lo);
        hi = warp_max(hi);

        if (hi < lo) {
            if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
        } else {
            // ---- exact entry count of the row, reserve it in the pool
            long long total = 0;
            bool reuse = false;
            int chunk_total = 0;
            if (hi - lo + 1 <= kBmBits) {
                build_bitmap(P, add, r, lo, hi + 1, pa0, pa1, lane, S);
                chunk_total = scan_bitmap(lane, S);
                total = chunk_total;
                reuse = true;
            } else {
                for (long long c0 = lo; c0 <= hi; c0 += kBmBits) {
                    int cend = (int)min((long long)hi + 1, c0 + kBmBits);
                    build_bitmap(P, add, r, (int)c0, cend, pa0, pa1, lane, S);
                    total += count_bitmap(lane, S);
                }
            }
            unsigned long long base = 0ull;
            if (lane == 0) base = atomicAdd(&P.ctl->pool_used, (unsigned long long)total);
            base = __shfl_sync(kFull, base, 0);
            if (base + (unsigned long long)total > P.ctl->pool_cap) {
                if (lane == 0) {
                    atomicOr(&P.ctl->status, kDevPoolFull);
                    P.out_rb[r] = P.out_re[r] = 0;
                }
            } else {
                const bool single = reuse && chunk_total <= kAccCap;
                int written = 0;
                int c0 = lo;
                while (c0 <= hi) {
                    int cend = (int)min((long long)hi + 1, (long long)c0 + kBmBits);
                    if (!reuse) {
                        build_bitmap(P, add, r, c0, cend, pa0, pa1, lane, S);
                        chunk_total = scan_bitmap(lane, S);
                    }
                    reuse = false;
                    int c1 = cend, cnt = chunk_total;
                    if (chunk_total > kAccCap) {
                        c1 = cut_column(lane, S, c0);
                        cnt = kAccCap;
                    }
                    // slot -> column, zero the accumulators
                    for (int w = lane; w < kBmWords; w += 32) {
                        unsigned bits = S.bm[w];
                        int idx = S.prefix[w];
                        while (bits) {
                            int b = __ffs(bits) - 1;
                            int c = c0 + w * 32 + b;
                            if (c < c1) S.colbuf[idx] = c;
                            ++idx;
                            bits &= bits - 1u;
                        }
                    }
                    for (int i = lane; i < cnt; i += 32) S.acc[i] = 0.0;
                    __syncwarp();

                    // ---- weighted sum of the addends, t ascending
                    for (int t = 0; t < P.nadd; ++t) {
                        const AddTerm& T = add[t];
                        const double alpha = T.alpha;
                        if (!T.rb) {
                            if (lane == 0 && r >= c0 && r < c1) {
                                int i = slot_of(S, r - c0);
                                S.acc[i] = __fma_rn(alpha, 1.0, S.acc[i]);
                            }
                        } else {
                            int s = T.rb[r], e = T.re[r];
                            for (int q = s + lane; q < e; q += 32) {
                                int c = T.col[q];
                                if (c >= c0 && c < c1) {
                                    int i = slot_of(S, c - c0);
                                    S.acc[i] = __fma_rn(alpha, T.val[q], S.acc[i]);
                                }
                            }
                        }
                        __syncwarp();
                    }

                    // ---- product A B: k of row r ascending, one B row per step.
                    // The (k, a, B-row range) of 32 A entries are held one per
                    // lane; the next 32-entry piece of B is loaded while the
                    // current one is folded in.
                    for (int seg = pa0; seg < pa1; seg += 32) {
                        const int cntseg = min(32, pa1 - seg);
                        int mys = 0, mye = 0;
                        double mya = 0.0;
                        if (lane < cntseg) {
                            int k = P.A.col[seg + lane];
                            mya = P.A.val[seg + lane];
                            mys = P.B.rb[k];
                            mye = P.B.re[k];
                            if (!single) {
                                int s2 = lower_bound_col(P.B.col, mys, mye, c0);
                                mye = lower_bound_col(P.B.col, s2, mye, c1);
                                mys = s2;
                            }
                        }
                        int kk = 0;
                        int bq = __shfl_sync(kFull, mys, 0), be = __shfl_sync(kFull, mye, 0);
                        double a = __shfl_sync(kFull, mya, 0);
                        while (kk < cntseg && bq >= be) {
                            ++kk;
                            int src = kk < cntseg ? kk : 0;
                            bq = __shfl_sync(kFull, mys, src);
                            be = __shfl_sync(kFull, mye, src);
                            a = __shfl_sync(kFull, mya, src);
                        }
                        int c = 0;
                        double v = 0.0;
                        bool have = false;
                        if (kk < cntseg && bq + lane < be) {
                            have = true;
                            c = P.B.col[bq + lane];
                            v = P.B.val[bq + lane];
                        }
                        while (kk < cntseg) {
                            int nk = kk, nq = bq + 32, ne = be;
                            double na = a;
                            bool newk = false;
                            if (nq >= ne) {
                                newk = true;
                                do {
                                    ++nk;
                                    int src = nk < cntseg ? nk : 0;
                                    nq = __shfl_sync(kFull, mys, src);
                                    ne = __shfl_sync(kFull, mye, src);
                                    na = __shfl_sync(kFull, mya, src);
                                } while (nk < cntseg && nq >= ne);
                            }
                            int c2 = 0;
                            double v2 = 0.0;
                            bool have2 = false;
                            if (nk < cntseg && nq + lane < ne) {
                                have2 = true;
                                c2 = P.B.col[nq + lane];
                                v2 = P.B.val[nq + lane];
                            }
                            if (have) {
                                int i = slot_of(S, c - c0);
                                S.acc[i] = __fma_rn(a, v, S.acc[i]);
                            }
                            if (newk) __syncwarp();
                            kk = nk;
                            bq = nq;
                            be = ne;
                            a = na;
                            c = c2;
                            v = v2;
                            have = have2;
                        }
                        __syncwarp();
                    }

                    // ---- write back the nonzero entries in column order; the
                    // entries with |x| <= eps_g enter the column sums of the
                    // first pass of Algorithm 1
                    for (int i0 = 0; i0 < cnt; i0 += 32) {
                        int i = i0 + lane;
                        double x = 0.0;
                        int c = 0;
                        if (i < cnt) {
                            x = S.acc[i];
                            c = S.colbuf[i];
                        }
                        bool nz = i < cnt && x != 0.0;
                        unsigned m = __ballot_sync(kFull, nz);
                        if (nz) {
                            long long pos = (long long)base + written + __popc(m & lanemask_lt());
                            P.pool_col[pos] = c;
                            P.pool_val[pos] = x;
                            double ax = fabs(x);
                            unsigned long long axb = (unsigned long long)__double_as_longlong(ax);
                            my_absmax = axb > my_absmax ? axb : my_absmax;
                            if (P.filtering && ax <= P.eps_g) {
                                exact_add(P.limbs + c, (size_t)P.n, P.sticky + c, ax, P.e_lsb);
                                ++my_cand;
                            }
                        }
                        written += __popc(m);
                    }
                    __syncwarp();
                    c0 = c1;
                }
                if (lane == 0) {
                    P.out_rb[r] = (int)base;
                    P.out_re[r] = (int)(base + written);
                    my_written = (unsigned long long)written;
                }
            }
        }
    }
    // ---- block totals for the step statistics
    my_cand = (unsigned long long)warp_sum((int)my_cand);
    my_absmax = warp_max_u64(my_absmax);
    for (int o = 16; o; o >>= 1) my_fma += __shfl_xor_sync(kFull, my_fma, o);
    if (lane == 0) {
        atomicAdd(&blk_fma, my_fma);
        atomicAdd(&blk_written, my_written);
        atomicAdd(&blk_cand, my_cand);
        atomicMax(&blk_absmax, my_absmax);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_fma) atomicAdd(&P.ctl->fma_total, blk_fma);
        if (P.stat) {
            if (blk_fma) atomicAdd(&P.stat->fma, blk_fma);
            if (blk_written) atomicAdd(&P.stat->nnz_pre, blk_written);
            if (blk_cand) atomicAdd(&P.stat->ncand, blk_cand);
        }
        if (P.absmax_slot && blk_absmax) atomicMax(&P.absmax_slot->absmax, blk_absmax);
    }
}

// ---------------------------------------------------------------- k_alg1
// Passes 2, 3, ... of Algorithm 1 and the compaction, as one cooperative
// launch.  On entry the column sums of pass 1 (entries |x| <= eps_g) are in
// the limbs and both cslot words are 0.  Every block evaluates the same
// scalar recurrence from the same global values, so all blocks take the same
// decisions without further communication.
constexpr int kAlg1Threads = 256;
constexpr unsigned long long kBarrierBudgetNs = 2000000000ull;  // 2 s

__global__ void __launch_bounds__(kAlg1Threads) k_alg1(Alg1Args A) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    __shared__ unsigned long long red[kAlg1Threads / 32];

    double eps_f = A.eps_g, c = 0.0;
    int it = 0;
    bool alive = true;
    for (;;) {
        // finalize: round each column sum, clear the accumulator, max
        unsigned long long local = 0ull;
        for (int j = gt; j < A.n; j += nthreads) {
            unsigned long long w[kLimbs];
#pragma unroll
            for (int l = 0; l < kLimbs; ++l) {  // L2 reads: other SMs' atomics
                w[l] = __ldcg(&A.limbs[(size_t)l * A.n + j]);
                A.limbs[(size_t)l * A.n + j] = 0ull;
            }
            bool st = __ldcg(&A.sticky[j]) != 0u;
            A.sticky[j] = 0u;
            double s = exact_round(w, st, A.e_lsb);
            unsigned long long sb = (unsigned long long)__double_as_longlong(s);
            local = sb > local ? sb : local;
        }
        local = warp_max_u64(local);
        if (lane == 0) red[threadIdx.x >> 5] = local;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
            v = warp_max_u64(v);
            if (threadIdx.x == 0) {
                if (v) atomicMax(&A.ctl->cslot[it & 1], v);
                if (blockIdx.x == 0) A.ctl->cslot[(it + 1) & 1] = 0ull;
            }
        }
        if (!grid_barrier(A.ctl, kBarrierBudgetNs)) {
            alive = false;
            break;
        }
        c = __longlong_as_double((long long)__ldcg(&A.ctl->cslot[it & 1]));
        double m = c / eps_f;
        ++it;
        if (!(c > A.bound)) break;
        if (it >= A.maxit) {
            if (gt == 0) atomicOr(&A.ctl->status, kDevNotConv);
            break;
        }
        eps_f = A.eps_g / m;
        // accumulate the entries still below the threshold
        for (int r = gw; r < A.n; r += nwarps) {
            int s = A.rb[r], e = A.re[r];
            for (int q = s + lane; q < e; q += 32) {
                double ax = fabs(A.val[q]);
                if (ax <= eps_f) exact_add(A.limbs + A.col[q], (size_t)A.n, A.sticky + A.col[q], ax, A.e_lsb);
            }
        }
        if (!grid_barrier(A.ctl, kBarrierBudgetNs)) {
            alive = false;
            break;
        }
    }
    if (!alive) return;

    // compaction: keep |x| > eps_f, in place, column order preserved
    unsigned long long kept = 0ull;
    for (int r = gw; r < A.n; r += nwarps) {
        int s = A.rb[r], e = A.re[r];
        int w = s;
        for (int q0 = s; q0 < e; q0 += 32) {
            int q = q0 + lane;
            int col = 0;
            double x = 0.0;
            bool keep = false;
            if (q < e) {
                col = A.col[q];
                x = A.val[q];
                keep = fabs(x) > eps_f;
            }
            __syncwarp();
            unsigned m = __ballot_sync(kFull, keep);
            if (keep) {
                int pos = w + __popc(m & lanemask_lt());
                A.col[pos] = col;
                A.val[pos] = x;
            }
            w += __popc(m);
            __syncwarp();
        }
        if (lane == 0) {
            A.re[r] = w;
            kept += (unsigned long long)(w - s);
        }
    }
    if (lane == 0 && kept) atomicAdd(&A.stat->nnz_post, kept);
    if (gt == 0) {
        A.stat->eps_f = eps_f;
        A.stat->iters = it;
        A.stat->dropped = c;
    }
}

// ---------------------------------------------------------------- k_norms
// Exact ||M||_1 of up to kMaxNorms matrices whose max |x| is already in
// slots[i].absmax: accumulate every |x| into per-column fixed-point sums,
// barrier, round and take the maximum into slots[i].result.
constexpr int kNormThreads = 256;

__global__ void __launch_bounds__(kNormThreads) k_norms(NormArgs A) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const size_t n = (size_t)A.n;
    for (long long u = gw; u < (long long)A.count * A.n; u += nwarps) {
        int mi = (int)(u / A.n), r = (int)(u % A.n);
        const RowView& M = A.m[mi];
        int lsb = lsb_for_bound(A.slots[mi].absmax);
        unsigned long long* limbs = A.limbs + (size_t)mi * kLimbs * n;
        unsigned* sticky = A.sticky + (size_t)mi * n;
        int s = M.rb[r], e = M.re[r];
        for (int q = s + lane; q < e; q += 32) {
            int c = M.col[q];
            exact_add(limbs + c, n, sticky + c, fabs(M.val[q]), lsb);
        }
    }
    if (!grid_barrier(A.ctl, kBarrierBudgetNs)) return;
    for (long long u = gt; u < (long long)A.count * A.n; u += nthreads) {
        int mi = (int)(u / A.n), j = (int)(u % A.n);
        int lsb = lsb_for_bound(A.slots[mi].absmax);
        unsigned long long* limbs = A.limbs + (size_t)mi * kLimbs * n;
        unsigned long long w[kLimbs];
#pragma unroll
        for (int l = 0; l < kLimbs; ++l) {  // L2 reads: other SMs' atomics
            w[l] = __ldcg(&limbs[(size_t)l * n + j]);
            limbs[(size_t)l * n + j] = 0ull;
        }
        bool st = __ldcg(&A.sticky[(size_t)mi * n + j]) != 0u;
        A.sticky[(size_t)mi * n + j] = 0u;
        double sum = exact_round(w, st, lsb);
        unsigned long long sb = (unsigned long long)__double_as_longlong(sum);
        if (sb) atomicMax(&A.slots[mi].result, sb);
    }
}

// ---------------------------------------------------------------- plumbing
__global__ void k_absmax(int n, RowView M, NormSlot* slot) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long mx = 0ull;
    for (int r = gw; r < n; r += nwarps)
        for (int q = M.rb[r] + lane; q < M.re[r]; q += 32) {
            unsigned long long b = (unsigned long long)__double_as_longlong(fabs(M.val[q]));
            mx = b > mx ? b : mx;
        }
    mx = warp_max_u64(mx);
    if (lane == 0 && mx) atomicMax(&slot->absmax, mx);
}

// Check a canonical CSR input: row pointers non-decreasing from 0 to nnz,
// columns in range and strictly increasing per row, values finite.
__global__ void k_validate(int n, int nnz, const int* rowptr, const int* col, const double* val,
                           Ctl* ctl) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    bool bad = false;
    if (r == 0 && rowptr[0] != 0) bad = true;
    if (r == n) {
        if (rowptr[n] != nnz) bad = true;
    } else {
        int s = rowptr[r], e = rowptr[r + 1];
        if (s > e || s < 0 || e > nnz) {
            bad = true;
        } else {
            int prev = -1;
            for (int q = s; q < e; ++q) {
                int c = col[q];
                double v = val[q];
                if (c <= prev || c >= n || !isfinite(v)) {
                    bad = true;
                    break;
                }
                prev = c;
            }
        }
    }
    if (bad) atomicOr(&ctl->status, kDevBadInput);
}

// Exclusive scan of row lengths re - rb into rowptr (n + 1 entries); one
// block of kScanThreads threads, each owning a contiguous range of rows.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_rows(int n, const int* rb, const int* re,
                                                             int* rowptr, Ctl* ctl) {
    __shared__ long long part[kScanThreads];
    const int t = threadIdx.x;
    const long long per = ((long long)n + kScanThreads - 1) / kScanThreads;
    const long long r0 = t * per, r1 = min((long long)n, r0 + per);
    long long s = 0;
    for (long long r = r0; r < r1; ++r) s += re[r] - rb[r];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        long long v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (long long r = r0; r < r1; ++r) {
        rowptr[r] = (int)run;
        run += re[r] - rb[r];
    }
    if (t == kScanThreads - 1) {
        rowptr[n] = (int)part[t];
        ctl->nnz_total = (unsigned long long)part[t];
    }
}

__global__ void k_gather(int n, RowView src, const int* rowptr, int* col, double* val) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < n; r += nwarps) {
        int s = src.rb[r], e = src.re[r], d = rowptr[r];
        for (int q = lane; q < e - s; q += 32) {
            col[d + q] = src.col[s + q];
            val[d + q] = src.val[s + q];
        }
    }
}

__global__ void k_identity(int n, double alpha, int* rowptr, int* col, double* val) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        rowptr[r] = r;
        col[r] = r;
        val[r] = alpha;
    }
    if (r == n) rowptr[n] = n;
}

__global__ void k_csr_to_rows(int n, const int* rowptr, int* rb, int* re) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        rb[r] = rowptr[r];
        re[r] = rowptr[r + 1];
    }
}

// ---------------------------------------------------------------- launchers
static int g_sms = 0, g_alg1_blocks = 0, g_norm_blocks = 0;
static std::atomic<long long> g_launches{0};

long long launch_count() { return g_launches.load(); }

cudaError_t kernels_init() {
    if (g_sms) return cudaSuccess;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_product, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)product_smem_bytes());
    if (err != cudaSuccess) return err;
    int per = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_alg1, kAlg1Threads, 0);
    if (err != cudaSuccess) return err;
    g_alg1_blocks = g_sms * (per < 2 ? per : 2);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_norms, kNormThreads, 0);
    if (err != cudaSuccess) return err;
    g_norm_blocks = g_sms * (per < 2 ? per : 2);
    if (g_alg1_blocks <= 0 || g_norm_blocks <= 0) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

int num_sms() { return g_sms; }

cudaError_t launch_product(const ProductArgs& P, cudaStream_t st) {
    if (P.n <= 0) return cudaSuccess;
    int blocks = (P.n + kProdWarps - 1) / kProdWarps;
    k_product<<<blocks, kProdWarps * 32, product_smem_bytes(), st>>>(P);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_alg1(const Alg1Args& A, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(&A.ctl->cslot[0], 0, sizeof(A.ctl->cslot), st);
    if (err != cudaSuccess) return err;
    Alg1Args a = A;
    void* args[] = {&a};
    ++g_launches;
    return cudaLaunchCooperativeKernel((const void*)k_alg1, dim3(g_alg1_blocks), dim3(kAlg1Threads), args,
                                       0, st);
}

cudaError_t launch_norms(const NormArgs& A, cudaStream_t st) {
    NormArgs a = A;
    void* args[] = {&a};
    ++g_launches;
    return cudaLaunchCooperativeKernel((const void*)k_norms, dim3(g_norm_blocks), dim3(kNormThreads), args,
                                       0, st);
}

cudaError_t launch_absmax(int n, const RowView& M, NormSlot* slot, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > g_sms * 8) blocks = g_sms * 8;
    k_absmax<<<blocks, 256, 0, st>>>(n, M, slot);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_validate(int n, int nnz, const int* rowptr, const int* col, const double* val, Ctl* ctl,
                            cudaStream_t st) {
    int blocks = (n + 1 + 255) / 256;
    k_validate<<<blocks, 256, 0, st>>>(n, nnz, rowptr, col, val, ctl);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_scan_rows(int n, const int* rb, const int* re, int* rowptr, Ctl* ctl, cudaStream_t st) {
    k_scan_rows<<<1, kScanThreads, 0, st>>>(n, rb, re, rowptr, ctl);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_gather(int n, const RowView& src, const int* rowptr, int* col, double* val,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > g_sms * 16) blocks = g_sms * 16;
    k_gather<<<blocks, 256, 0, st>>>(n, src, rowptr, col, val);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_identity(int n, double alpha, int* rowptr, int* col, double* val, cudaStream_t st) {
    k_identity<<<(n + 1 + 255) / 256, 256, 0, st>>>(n, alpha, rowptr, col, val);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_csr_to_rows(int n, const int* rowptr, int* rb, int* re, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_csr_to_rows<<<(n + 255) / 256, 256, 0, st>>>(n, rowptr, rb, re);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace psf
