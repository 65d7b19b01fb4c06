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
//   kb/kl/ka/ke       B-row begin, length, a_rk and element prefix of up to 32
//                     entries k of A's row (one segment)
//   sc/sv             kStages staged 32-entry pieces of B rows (cp.async ring)
// A row whose pattern exceeds a chunk (wider than the bitmap or with more
// than kAccCap entries) is processed in several column chunks.
constexpr int kBmWords = 256;
constexpr int kBmBits = kBmWords * 32;
constexpr int kAccCap = 1024;
constexpr int kProdWarps = 4;
constexpr int kStages = 8;

struct WarpSmem {
    unsigned bm[kBmWords];
    int prefix[kBmWords];
    int colbuf[kAccCap];
    double acc[kAccCap];
    double ka[32];
    int kb[32];
    int kl[32];
    int ke[33];
    int sc[kStages][32];
    double sv[kStages][32];
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

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Load the segment [seg, seg + cnt) of A's row: k, a_rk and the range of B's
// row k restricted to columns [c0, c1) (the whole row when `whole`).
__device__ void load_segment(const ProductArgs& P, int seg, int cnt, bool whole, int c0, int c1, int lane,
                             WarpSmem& S) {
    int len = 0;
    if (lane < cnt) {
        int k = P.A.col[seg + lane];
        int b = P.B.rb[k], e = P.B.re[k];
        if (!whole) {
            int b2 = lower_bound_col(P.B.col, b, e, c0);
            e = lower_bound_col(P.B.col, b2, e, c1);
            b = b2;
        }
        S.ka[lane] = P.A.val[seg + lane];
        S.kb[lane] = b;
        S.kl[lane] = e - b;
        len = e - b;
    }
    int ex = warp_excl_scan(len, lane);
    S.ke[lane] = ex;
    if (lane == 31) S.ke[32] = ex + len;
    __syncwarp();
}

// Set the bitmap bits of every output column in [c0, cend) of row r.  The
// B rows of a segment are walked as one flattened sequence of entries, so
// every lane has an independent load in each step.
__device__ void build_bitmap(const ProductArgs& P, const AddTerm* add, int nadd, int r, int c0, int cend,
                             int pa0, int pa1, bool whole, int lane, WarpSmem& S) {
    for (int w = lane; w < kBmWords; w += 32) S.bm[w] = 0u;
    __syncwarp();
    for (int t = 0; t < nadd; ++t) {
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
    for (int seg = pa0; seg < pa1; seg += 32) {
        const int cnt = min(32, pa1 - seg);
        load_segment(P, seg, cnt, whole, c0, cend, lane, S);
        const int F = S.ke[cnt];
        constexpr int U = 4;
        for (int f0 = 0; f0 < F; f0 += 32 * U) {
            int cols[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int f = f0 + u * 32 + lane;
                cols[u] = -1;
                if (f < F) {
                    int lo = 0, hi = cnt - 1;  // last i with ke[i] <= f
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (S.ke[mid] <= f) lo = mid;
                        else hi = mid - 1;
                    }
                    cols[u] = P.B.col[S.kb[lo] + (f - S.ke[lo])];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (cols[u] >= c0 && cols[u] < cend) bm_set(S, cols[u] - c0);
        }
        __syncwarp();
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

// Next (segment entry, 32-entry piece) of the flattened B-row sequence.
__device__ __forceinline__ void next_piece(const WarpSmem& S, int cnt, int& i, int& ch) {
    ++ch;
    if (ch * 32 >= S.kl[i]) {
        ch = 0;
        do {
            ++i;
        } while (i < cnt && S.kl[i] == 0);
    }
}

__device__ __forceinline__ void issue_piece(const ProductArgs& P, WarpSmem& S, int cnt, int i, int ch, int slot,
                                            int lane) {
    if (i < cnt) {
        int off = ch * 32 + lane;
        if (off < S.kl[i]) {
            int q = S.kb[i] + off;
            cp_async4(&S.sc[slot][lane], P.B.col + q);
            cp_async8(&S.sv[slot][lane], P.B.val + q);
        }
    }
    cp_async_commit();
}

// acc[slot(j)] = fma(a_rk, b_kj, acc[slot(j)]) for k of the segment in
// order; B pieces arrive through a kStages-deep cp.async ring.
__device__ void accumulate_segment(const ProductArgs& P, int cnt, int c0, int lane, WarpSmem& S) {
    int ci = 0, cch = 0;
    while (ci < cnt && S.kl[ci] == 0) ++ci;
    int ii = ci, ich = 0;
#pragma unroll 1
    for (int s = 0; s < kStages - 1; ++s) {
        issue_piece(P, S, cnt, ii, ich, s, lane);
        if (ii < cnt) next_piece(S, cnt, ii, ich);
    }
    int slot = 0;
    while (ci < cnt) {
        cp_async_wait<kStages - 2>();
        int off = cch * 32 + lane;
        if (off < S.kl[ci]) {
            int c = S.sc[slot][lane];
            double v = S.sv[slot][lane];
            int i = slot_of(S, c - c0);
            S.acc[i] = __fma_rn(S.ka[ci], v, S.acc[i]);
        }
        int pi = ci;
        next_piece(S, cnt, ci, cch);
        if (ci != pi) __syncwarp();
        // refill the slot consumed one piece ago
        issue_piece(P, S, cnt, ii, ich, (slot + kStages - 1) % kStages, lane);
        if (ii < cnt) next_piece(S, cnt, ii, ich);
        slot = (slot + 1) % kStages;
    }
    cp_async_wait<0>();
    __syncwarp();
}

__global__ void __launch_bounds__(kProdWarps * 32) k_product(ProductArgs P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AddTerm* add = reinterpret_cast<AddTerm*>(smem_raw);
    WarpSmem* warps = reinterpret_cast<WarpSmem*>(smem_raw + sizeof(AddTerm) * kMaxAdd);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nadd = P.nadd;
    for (int t = threadIdx.x; t < nadd; t += blockDim.x) add[t] = P.add[t];
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
    const unsigned long long eps_bits = (unsigned long long)__double_as_longlong(P.eps_g);
    unsigned long long my_written = 0ull, my_cand = 0ull, my_absmax = 0ull, my_fma = 0ull;

    if (r < P.n) {
        // ---- column window of row r and the row's multiply-add count
        int lo = INT_MAX, hi = -1;
        for (int t = 0; t < nadd; ++t) {
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
            for (int t = 0; t < nadd; ++t)
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
                build_bitmap(P, add, nadd, r, lo, hi + 1, pa0, pa1, true, lane, S);
                chunk_total = scan_bitmap(lane, S);
                total = chunk_total;
                reuse = true;
            } else {
                for (long long c0 = lo; c0 <= hi; c0 += kBmBits) {
                    int cend = (int)min((long long)hi + 1, c0 + kBmBits);
                    build_bitmap(P, add, nadd, r, (int)c0, cend, pa0, pa1, false, lane, S);
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
                        build_bitmap(P, add, nadd, r, c0, cend, pa0, pa1, false, lane, S);
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
                    for (int t = 0; t < nadd; ++t) {
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

                    // ---- product A B: k of row r ascending
                    for (int seg = pa0; seg < pa1; seg += 32) {
                        const int cnt_seg = min(32, pa1 - seg);
                        load_segment(P, seg, cnt_seg, single, c0, c1, lane, S);
                        accumulate_segment(P, cnt_seg, c0, lane, S);
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
                        unsigned long long xb = mag_bits(x);
                        bool nz = i < cnt && xb != 0ull;
                        unsigned m = __ballot_sync(kFull, nz);
                        if (nz) {
                            long long pos = (long long)base + written + __popc(m & lanemask_lt());
                            P.pool_col[pos] = c;
                            P.pool_val[pos] = x;
                            my_absmax = xb > my_absmax ? xb : my_absmax;
                            if (P.filtering && xb <= eps_bits) {
                                exact_add(P.words + c, (size_t)P.n, P.sticky + c, xb, P.e_lsb);
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

// ---------------------------------------------------------------- k_product_win
// Row-group kernel with a dense column-window accumulator.  A group of G
// threads (G = 32..256, several groups per block) computes one output row at
// a time: acc[c - c0] holds column c of the chunk [c0, c0 + cap) of the row's
// window, so no symbolic pass and no slot lookup is needed.  The addend
// terms are folded in order t = 0, 1, ... and the B rows in ascending k, with
// a group barrier between consecutive k: every output entry sees exactly the
// fixed fma order of the product definition.  B rows reach shared memory in
// pieces of G * kWinE entries through a kWinStages-deep cp.async ring; each
// thread copies and later reads only its own elements.  Rows whose window
// exceeds `cap` are processed in several column chunks (their pool space is
// reserved up front from an upper bound); other rows reserve their exact
// entry count after accumulation.
constexpr int kWinThreads = 256;
constexpr int kWinStages = 4;
constexpr int kWinE = 2;

template <int G>
struct WinGroup {
    static constexpr int NG = kWinThreads / G;
    static constexpr int NW = G / 32;
    static constexpr int PIECE = G * kWinE;
    // per-group layout after acc[cap]
    int sc[kWinStages][PIECE];
    double sv[kWinStages][PIECE];
    double ka[G];
    int kb[G];
    int kl[G];
    long long red[NW];
    int misc[4];
};

template <int G>
__host__ __device__ size_t win_group_bytes(int cap) {
    return ((size_t)cap * sizeof(double) + sizeof(WinGroup<G>) + 15) & ~(size_t)15;
}

template <int G>
size_t win_smem_bytes(int cap) {
    return sizeof(AddTerm) * kMaxAdd + win_group_bytes<G>(cap) * WinGroup<G>::NG;
}

template <int G>
__device__ __forceinline__ void group_sync(int g) {
    if constexpr (G == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(G) : "memory");
    }
}

// group-wide reductions through the per-group scratch (all G threads call)
template <int G>
__device__ __forceinline__ long long group_sum(long long v, WinGroup<G>& S, int g, int gt) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if constexpr (G == 32) {
        return v;
    } else {
        group_sync<G>(g);
        if ((gt & 31) == 0) S.red[gt >> 5] = v;
        group_sync<G>(g);
        long long t = 0;
#pragma unroll
        for (int w = 0; w < WinGroup<G>::NW; ++w) t += S.red[w];
        return t;
    }
}
template <int G>
__device__ __forceinline__ int group_min(int v, WinGroup<G>& S, int g, int gt) {
    v = warp_min(v);
    if constexpr (G == 32) {
        return v;
    } else {
        group_sync<G>(g);
        if ((gt & 31) == 0) S.red[gt >> 5] = v;
        group_sync<G>(g);
        long long t = S.red[0];
#pragma unroll
        for (int w = 1; w < WinGroup<G>::NW; ++w) t = min(t, S.red[w]);
        return (int)t;
    }
}
template <int G>
__device__ __forceinline__ int group_max(int v, WinGroup<G>& S, int g, int gt) {
    v = warp_max(v);
    if constexpr (G == 32) {
        return v;
    } else {
        group_sync<G>(g);
        if ((gt & 31) == 0) S.red[gt >> 5] = v;
        group_sync<G>(g);
        long long t = S.red[0];
#pragma unroll
        for (int w = 1; w < WinGroup<G>::NW; ++w) t = max(t, S.red[w]);
        return (int)t;
    }
}

template <int G>
__device__ __forceinline__ void win_next(const WinGroup<G>& S, int cnt, int& i, int& off) {
    off += WinGroup<G>::PIECE;
    if (off >= S.kl[i]) {
        off = 0;
        do {
            ++i;
        } while (i < cnt && S.kl[i] == 0);
    }
}

template <int G>
__device__ __forceinline__ void win_issue(const ProductArgs& P, WinGroup<G>& S, int cnt, int i, int off, int stage,
                                          int gt) {
    if (i < cnt) {
#pragma unroll
        for (int e = 0; e < kWinE; ++e) {
            int o = off + gt + e * G;
            if (o < S.kl[i]) {
                int q = S.kb[i] + o;
                cp_async4(&S.sc[stage][gt + e * G], P.B.col + q);
                cp_async8(&S.sv[stage][gt + e * G], P.B.val + q);
            }
        }
    }
    cp_async_commit();
}

template <int G>
__global__ void __launch_bounds__(kWinThreads) k_product_win(ProductArgs P, int cap) {
    constexpr int NG = WinGroup<G>::NG;
    constexpr int NW = WinGroup<G>::NW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AddTerm* add = reinterpret_cast<AddTerm*>(smem_raw);
    const int g = threadIdx.x / G, gt = threadIdx.x % G, lane = threadIdx.x & 31, gw = gt >> 5;
    unsigned char* gbase = smem_raw + sizeof(AddTerm) * kMaxAdd + win_group_bytes<G>(cap) * g;
    double* acc = reinterpret_cast<double*>(gbase);
    WinGroup<G>& S = *reinterpret_cast<WinGroup<G>*>(gbase + (size_t)cap * sizeof(double));
    const int nadd = P.nadd;
    for (int t = threadIdx.x; t < nadd; t += blockDim.x) add[t] = P.add[t];
    __syncthreads();
    const unsigned long long eps_bits = (unsigned long long)__double_as_longlong(P.eps_g);
    unsigned long long my_written = 0ull, my_cand = 0ull, my_absmax = 0ull, my_fma = 0ull;

    for (int r = blockIdx.x * NG + g; r < P.n; r += gridDim.x * NG) {
        // ---- window [lo, hi] of row r and its multiply-add count
        int lo = INT_MAX, hi = -1;
        long long ub = 0;  // entry upper bound: products plus addend entries
        if (gt == 0)
            for (int t = 0; t < nadd; ++t) {
                const AddTerm& T = add[t];
                if (!T.rb) {
                    lo = min(lo, r);
                    hi = max(hi, r);
                    ub += 1;
                } else {
                    int s = T.rb[r], e = T.re[r];
                    ub += e - s;
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
        for (int p = pa0 + gt; p < pa1; p += G) {
            int k = P.A.col[p];
            int s = P.B.rb[k], e = P.B.re[k];
            ub += e - s;
            if (s < e) {
                lo = min(lo, P.B.col[s]);
                hi = max(hi, P.B.col[e - 1]);
            }
        }
        lo = group_min<G>(lo, S, g, gt);
        hi = group_max<G>(hi, S, g, gt);
        ub = group_sum<G>(ub, S, g, gt);
        if (gt == 0) my_fma += (unsigned long long)ub;
        if (hi < lo) {
            if (gt == 0) P.out_rb[r] = P.out_re[r] = 0;
            group_sync<G>(g);
            continue;
        }
        const long long W = (long long)hi - lo + 1;
        const bool single = W <= cap;
        long long base = 0;
        bool ok = true;
        if (!single) {
            // reserve the upper bound min(W, products + addend entries) now
            long long need = min(W, ub);
            if (gt == 0) {
                unsigned long long b = atomicAdd(&P.ctl->pool_used, (unsigned long long)need);
                if (b + (unsigned long long)need > P.ctl->pool_cap) {
                    atomicOr(&P.ctl->status, kDevPoolFull);
                    S.misc[0] = 0;
                } else {
                    S.misc[0] = 1;
                }
                S.misc[1] = (int)(b & 0x7fffffff);
            }
            group_sync<G>(g);
            ok = S.misc[0] != 0;
            base = S.misc[1];
            group_sync<G>(g);
        }
        long long written = 0;
        for (long long c0l = lo; c0l <= hi && ok; c0l += cap) {
            const int c0 = (int)c0l;
            const int wlen = (int)min((long long)cap, (long long)hi - c0 + 1);
            const int c1 = c0 + wlen;
            for (int i = gt; i < wlen; i += G) acc[i] = 0.0;
            group_sync<G>(g);
            // ---- weighted sum of the addends, t ascending
            for (int t = 0; t < nadd; ++t) {
                const AddTerm& T = add[t];
                const double alpha = T.alpha;
                if (!T.rb) {
                    if (gt == 0 && r >= c0 && r < c1) acc[r - c0] = __fma_rn(alpha, 1.0, acc[r - c0]);
                } else {
                    int s = T.rb[r], e = T.re[r];
                    for (int q = s + gt; q < e; q += G) {
                        int c = T.col[q];
                        if (c >= c0 && c < c1) acc[c - c0] = __fma_rn(alpha, T.val[q], acc[c - c0]);
                    }
                }
                group_sync<G>(g);
            }
            // ---- product: k of row r ascending
            for (int seg = pa0; seg < pa1; seg += G) {
                const int cnt = min(G, pa1 - seg);
                if (gt < cnt) {
                    int k = P.A.col[seg + gt];
                    int b = P.B.rb[k], e = P.B.re[k];
                    if (!single) {
                        int b2 = lower_bound_col(P.B.col, b, e, c0);
                        e = lower_bound_col(P.B.col, b2, e, c1);
                        b = b2;
                    }
                    S.ka[gt] = P.A.val[seg + gt];
                    S.kb[gt] = b;
                    S.kl[gt] = e - b;
                }
                group_sync<G>(g);
                int ci = 0, coff = 0;
                while (ci < cnt && S.kl[ci] == 0) ++ci;
                int ii = ci, ioff = 0;
#pragma unroll 1
                for (int st = 0; st < kWinStages - 1; ++st) {
                    win_issue<G>(P, S, cnt, ii, ioff, st, gt);
                    if (ii < cnt) win_next<G>(S, cnt, ii, ioff);
                }
                int stage = 0;
                while (ci < cnt) {
                    cp_async_wait<kWinStages - 2>();
                    const double a = S.ka[ci];
                    const int len = S.kl[ci];
#pragma unroll
                    for (int e = 0; e < kWinE; ++e) {
                        int o = coff + gt + e * G;
                        if (o < len) {
                            int c = S.sc[stage][gt + e * G];
                            double v = S.sv[stage][gt + e * G];
                            acc[c - c0] = __fma_rn(a, v, acc[c - c0]);
                        }
                    }
                    int pi = ci;
                    win_next<G>(S, cnt, ci, coff);
                    if (ci != pi) group_sync<G>(g);
                    win_issue<G>(P, S, cnt, ii, ioff, (stage + kWinStages - 1) % kWinStages, gt);
                    if (ii < cnt) win_next<G>(S, cnt, ii, ioff);
                    stage = (stage + 1) % kWinStages;
                }
                cp_async_wait<0>();
                group_sync<G>(g);
            }
            // ---- write-back: each warp sweeps a contiguous part of the window
            const int part = ((wlen + NW * 32 - 1) / (NW * 32)) * 32;
            const int p0 = gw * part, p1 = min(wlen, p0 + part);
            int mycount = 0;
            for (int i0 = p0; i0 < p1; i0 += 32) {
                int i = i0 + lane;
                bool nz = i < p1 && mag_bits(acc[i]) != 0ull;
                mycount += __popc(__ballot_sync(kFull, nz));
            }
            // exclusive prefix of the warp counts within the group
            int before = 0, total = mycount;
            if constexpr (G > 32) {
                if (lane == 0) S.red[gw] = mycount;
                group_sync<G>(g);
                total = 0;
                for (int w = 0; w < NW; ++w) {
                    int cw = (int)S.red[w];
                    if (w < gw) before += cw;
                    total += cw;
                }
                group_sync<G>(g);
            }
            if (single) {
                if (gt == 0) {
                    unsigned long long b = atomicAdd(&P.ctl->pool_used, (unsigned long long)total);
                    if (b + (unsigned long long)total > P.ctl->pool_cap) {
                        atomicOr(&P.ctl->status, kDevPoolFull);
                        S.misc[0] = 0;
                    } else {
                        S.misc[0] = 1;
                    }
                    S.misc[1] = (int)(b & 0x7fffffff);
                }
                group_sync<G>(g);
                ok = S.misc[0] != 0;
                base = S.misc[1];
                group_sync<G>(g);
                if (!ok) break;
            }
            long long pos0 = base + written + before;
            for (int i0 = p0; i0 < p1; i0 += 32) {
                int i = i0 + lane;
                double x = i < p1 ? acc[i] : 0.0;
                unsigned long long xb = mag_bits(x);
                bool nz = i < p1 && xb != 0ull;
                unsigned m = __ballot_sync(kFull, nz);
                if (nz) {
                    long long pos = pos0 + __popc(m & lanemask_lt());
                    int c = c0 + i;
                    P.pool_col[pos] = c;
                    P.pool_val[pos] = x;
                    my_absmax = xb > my_absmax ? xb : my_absmax;
                    if (P.filtering && xb <= eps_bits) {
                        exact_add(P.words + c, (size_t)P.n, P.sticky + c, xb, P.e_lsb);
                        ++my_cand;
                    }
                }
                pos0 += __popc(m);
            }
            written += total;
            group_sync<G>(g);
        }
        if (gt == 0) {
            if (ok) {
                P.out_rb[r] = (int)base;
                P.out_re[r] = (int)(base + written);
                my_written += (unsigned long long)written;
            } else {
                P.out_rb[r] = P.out_re[r] = 0;
            }
        }
        group_sync<G>(g);
    }
    // ---- block totals for the step statistics
    __shared__ unsigned long long blk[4];
    if (threadIdx.x < 4) blk[threadIdx.x] = 0ull;
    __syncthreads();
    my_cand = (unsigned long long)warp_sum((int)my_cand);
    my_absmax = warp_max_u64(my_absmax);
    for (int o = 16; o; o >>= 1) {
        my_fma += __shfl_xor_sync(kFull, my_fma, o);
        my_written += __shfl_xor_sync(kFull, my_written, o);
    }
    if (lane == 0) {
        if (my_fma) atomicAdd(&blk[0], my_fma);
        if (my_written) atomicAdd(&blk[1], my_written);
        if (my_cand) atomicAdd(&blk[2], my_cand);
        if (my_absmax) atomicMax(&blk[3], my_absmax);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk[0]) atomicAdd(&P.ctl->fma_total, blk[0]);
        if (P.stat) {
            if (blk[0]) atomicAdd(&P.stat->fma, blk[0]);
            if (blk[1]) atomicAdd(&P.stat->nnz_pre, blk[1]);
            if (blk[2]) atomicAdd(&P.stat->ncand, blk[2]);
        }
        if (P.absmax_slot && blk[3]) atomicMax(&P.absmax_slot->absmax, blk[3]);
    }
}

// ---------------------------------------------------------------- k_alg1
// Passes 2, 3, ... of Algorithm 1 and the compaction, as one cooperative
// launch.  On entry the column sums of pass 1 (entries |x| <= eps_g) are in
// the chunk words and both cslot words are 0.  Every block evaluates the same
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
    const size_t n = (size_t)A.n;
    __shared__ unsigned long long red[kAlg1Threads / 32];

    double eps_f = A.eps_g, c = 0.0;
    int it = 0;
    bool alive = true;
    for (;;) {
        // finalize: round each column sum, clear the accumulator, max
        unsigned long long local = 0ull;
        for (int j = gt; j < A.n; j += nthreads) {
            double s = chunk_round(A.words + j, n, A.sticky + j, A.e_lsb);
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
        const unsigned long long fb = (unsigned long long)__double_as_longlong(eps_f);
        // accumulate the entries still below the threshold
        for (int r = gw; r < A.n; r += nwarps) {
            int s = A.rb[r], e = A.re[r];
            for (int q = s + lane; q < e; q += 32) {
                unsigned long long xb = mag_bits(A.val[q]);
                if (xb <= fb) {
                    int col = A.col[q];
                    exact_add(A.words + col, n, A.sticky + col, xb, A.e_lsb);
                }
            }
        }
        if (!grid_barrier(A.ctl, kBarrierBudgetNs)) {
            alive = false;
            break;
        }
    }
    if (!alive) return;

    // compaction: keep |x| > eps_f, in place, column order preserved
    const unsigned long long fb = (unsigned long long)__double_as_longlong(eps_f);
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
                keep = mag_bits(x) > fb;
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
        unsigned long long* words = A.words + (size_t)mi * kChunks * n;
        unsigned* sticky = A.sticky + (size_t)mi * n;
        int s = M.rb[r], e = M.re[r];
        for (int q = s + lane; q < e; q += 32) {
            int c = M.col[q];
            exact_add(words + c, n, sticky + c, mag_bits(M.val[q]), lsb);
        }
    }
    if (!grid_barrier(A.ctl, kBarrierBudgetNs)) return;
    for (long long u = gt; u < (long long)A.count * A.n; u += nthreads) {
        int mi = (int)(u / A.n), j = (int)(u % A.n);
        int lsb = lsb_for_bound(A.slots[mi].absmax);
        unsigned long long* words = A.words + (size_t)mi * kChunks * n;
        double sum = chunk_round(words + j, n, A.sticky + (size_t)mi * n + j, lsb);
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
            unsigned long long b = mag_bits(M.val[q]);
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
            if (s < e) atomicMax(&ctl->maxwin, col[e - 1] - col[s] + 1);
            for (int q = s; q < e; ++q) {
                int c = col[q];
                double v = val[q];
                bool finite = (mag_bits(v) >> 52) != 0x7ffull;
                if (c <= prev || c >= n || !finite) {
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

// smem budget of one k_product_win block: three blocks fit on one SM
constexpr size_t kWinBlockBudget = 74 * 1024;

template <int G>
static int win_cap() {
    size_t fixed = sizeof(AddTerm) * kMaxAdd + sizeof(WinGroup<G>) * WinGroup<G>::NG + 16 * WinGroup<G>::NG;
    size_t per = (kWinBlockBudget - fixed) / WinGroup<G>::NG / sizeof(double);
    return (int)(per & ~(size_t)31);
}

template <int G>
static cudaError_t win_init() {
    return cudaFuncSetAttribute(k_product_win<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)win_smem_bytes<G>(win_cap<G>()));
}

template <int G>
static cudaError_t win_launch(const ProductArgs& P, int cap_limit, cudaStream_t st) {
    const int full = win_cap<G>();
    const int cap = (cap_limit > 0 && cap_limit < full) ? cap_limit : full;
    long long blocks = ((long long)P.n + WinGroup<G>::NG - 1) / WinGroup<G>::NG;
    if (blocks > 65535LL * 64) blocks = 65535LL * 64;
    k_product_win<G><<<(unsigned)blocks, kWinThreads, win_smem_bytes<G>(full), st>>>(P, cap);
    ++g_launches;
    return cudaGetLastError();
}

int product_win_cap(int group) {
    switch (group) {
        case 32: return win_cap<32>();
        case 64: return win_cap<64>();
        case 128: return win_cap<128>();
        default: return win_cap<256>();
    }
}

cudaError_t launch_product_win(const ProductArgs& P, int group, int cap_limit, cudaStream_t st) {
    if (P.n <= 0) return cudaSuccess;
    switch (group) {
        case 32: return win_launch<32>(P, cap_limit, st);
        case 64: return win_launch<64>(P, cap_limit, st);
        case 128: return win_launch<128>(P, cap_limit, st);
        default: return win_launch<256>(P, cap_limit, st);
    }
}

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
    if ((err = win_init<32>()) != cudaSuccess) return err;
    if ((err = win_init<64>()) != cudaSuccess) return err;
    if ((err = win_init<128>()) != cudaSuccess) return err;
    if ((err = win_init<256>()) != cudaSuccess) return err;
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
