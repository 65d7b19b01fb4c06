// psf_kernels.cu -- CUDA kernels of the filtered Paterson-Stockmeyer
// evaluator (sm_103a, FP64 throughout).
//
//  k_product      one fused step C = sum_t alpha_t M_t + A B: output pattern
//                 and slot map of each row, exact row reservation in the
//                 pool, FP64 accumulation in shared memory, write-back of the
//                 nonzero entries, and the first pass of Algorithm 1 (exact
//                 column sums and the candidate list of the entries
//                 |x| <= eps_g); a batch instantiation reads per-row
//                 instance parameters.
//  k_product_cta  the same step with one output row per block of four warps
//                 (matrices of at most one wave of rows with long B rows).
//  k_row_bitmaps  column bitmaps of B's rows for the symbolic pass.
//  k_reuse_pass1  a baby step equal to a power of the norm phase: the first
//                 pass of Algorithm 1 on that power's rows.
//  k_reuse_copy_batch  the same for the instances of a batch: those rows
//                 copied into the step's pool range, with that first pass.
//  k_alg1         the remaining passes of Algorithm 1 (Sec. 3.1.1) and the
//  k_alg1_batch   final in-place compaction, one cooperative launch (single
//                 instance, or every filtered instance of a batched step).
//  k_norms_rows   exact 1-norms of Z^1..Z^10 (Eq. 37's z_i) by row tiles,
//  k_norms_finish column sums in shared memory; rounding and maxima.
//  k_norms        exact 1-norms from flat pool ranges (psf_norm1 and its
//                 allocation-free variant).
//  k_export       small device records written into pinned, device-mapped
//                 host memory (the host's read-backs take no copy engine).
//  k_absmax, k_validate*, k_copy_rows*, k_scan_*, k_gather*, k_identity,
//  k_inst_table, k_compose_rows, k_bounds: plumbing.
#include <atomic>
#include <climits>
#include <mutex>

#include "psf_device.cuh"
#include "psf_kernels.h"

namespace psf {

// ---------------------------------------------------------------- k_product
// Compact-accumulator kernel: one warp computes one output row, with no
// block-level synchronisation.  The row's output pattern is found first (the
// symbolic pass), each output column gets an accumulator slot (its rank in
// the pattern), then the products are folded in (the numeric pass).  Two
// ways to map a column offset o = c - c0 to its slot, a template parameter:
//
//  table  (TAB = true)   tab[o] (16 bit) holds first a flag, set by plain
//         stores of every contributing entry, then the slot, after a ballot
//         scan.  O(window) set-up per row, one load per lookup: for rows with
//         many products per column of the window.
//  bitmap (TAB = false)  pm[o / 32] holds a 32-column bitmap word, set by
//         atomic ORs (one per run of columns a lane meets), and the number of
//         set bits before it; slot = prefix + popcount of the lower bits.
//         O(window / 32) set-up per row: for thin rows.
//
// Numeric pass: the addends in order, then the B rows in ascending k, each
// entry folded as acc[slot] = fma(a, b, acc[slot]); a warp barrier separates
// consecutive rows (the fixed rounding order of the product).  B rows are
// read in 128-entry chunks (four 32-entry pieces; the entries of a chunk
// have distinct columns, so its four read-modify-writes are independent).
// A row whose pattern exceeds the chunk (wider than the map or with more
// than kAccCap entries) is processed in several column chunks.
constexpr int kTabCap = 4160;  // columns of the table map
constexpr int kBmWords = 144;  // bitmap words of the bitmap map (4608 columns)
constexpr int kBmBits = kBmWords * 32;
// The wide-window bitmap (16384 columns) for steps whose rows span more
// columns than kBmBits (a grid of side M spreads a row over about 2rM
// columns for a pattern of radius r): one column chunk instead of several,
// at 5 blocks per SM instead of 7.
constexpr int kBmWordsBig = 512;
static_assert(kBmBits == kBitmapColumns, "the host's notion of the bitmap window");
// Accumulator slots; with 7 bitmap blocks of 4 warps per SM shared memory is
// full.  The bitmap map keeps a segment's a_rk in the last 32 slots, so a row
// has kAccCap - 32 of them; its WIDE instantiation, for steps whose rows are
// long, reads a_rk from A's row instead and gives a row every slot (a row of
// up to kAccCap entries then takes one pass, not two column chunks).
constexpr int kAccCap = 640;

template <bool TAB, int W = kBmWords>
struct ProdSmem;

template <>
struct ProdSmem<true, kBmWords> {
    static constexpr int kCols = kTabCap;
    static constexpr int kWarps = 2;
    static constexpr int kBlocksPerSm = 7;
    unsigned short tab[kTabCap];
    double acc[kAccCap];
    double ka[32];
    int kb[32];
    int kl[32];
    unsigned short colbuf[kAccCap];
};

template <int W>
struct ProdSmem<false, W> {
    static constexpr int kCols = W * 32;
    static constexpr int kWarps = 4;
    // 28 warps: registers (72) and shared memory; 20 with the wide window
    static constexpr int kBlocksPerSm = W > kBmWords ? 5 : 7;
    uint2 pm[W];  // .x = set bits before the word, .y = bitmap word
    double acc[kAccCap];  // the last 32 hold a_rk of the segment (not in WIDE)
    int kb[32];
    int kl[32];
    unsigned short colbuf[kAccCap];
};

template <bool TAB, int W = kBmWords>
size_t prod_smem_bytes() {
    return sizeof(ProdSmem<TAB, W>) * ProdSmem<TAB, W>::kWarps + sizeof(AddTerm) * kMaxAdd;
}

// first position in [s, e) with col >= c (col ascending).  Pool positions
// reach 2^31 - 2^20, so the midpoint is s + (e - s) / 2: s + e would overflow.
__device__ __forceinline__ int lower_bound_col(const int* col, int s, int e, int c) {
    while (s < e) {
        const int mid = s + ((e - s) >> 1);
        if (col[mid] < c) s = mid + 1;
        else e = mid;
    }
    return s;
}

// slot of column offset o (o inside the current chunk's pattern)
__device__ __forceinline__ int slot_lookup(const ProdSmem<true>& S, int o) { return S.tab[o]; }
// (o's own bit is set: the set bits at or below it, shifted to the top,
// count one more than the bits below it)
template <int W>
__device__ __forceinline__ int slot_lookup(const ProdSmem<false, W>& S, int o) {
    const uint2 e = S.pm[o >> 5];
    return (int)e.x + __popc(e.y << (~o & 31)) - 1;
}

// where a segment's a_rk are kept
__device__ __forceinline__ double* ka_of(ProdSmem<true>& S) { return S.ka; }
template <int W>
__device__ __forceinline__ double* ka_of(ProdSmem<false, W>& S) { return S.acc + (kAccCap - 32); }

// Load the segment [seg, seg + cnt) of A's row: a_rk (unless `store_a` is
// false) and the range of B's row k restricted to columns [c0, c1) (the
// whole row when `whole`).
template <bool TAB, int W>
__device__ __forceinline__ void load_segment(const ProductArgs& P, int seg, int cnt, bool whole, int c0, int c1,
                                             int lane, ProdSmem<TAB, W>& S, bool store_a,
                                             unsigned long long* fma = nullptr, int* kwn = nullptr) {
    if (lane < cnt) {
        int k = P.A.col[seg + lane];
        int b = P.B.rb[k], e = P.B.re[k];
        if (fma) *fma += (unsigned long long)(e - b);
        if (kwn) {
            // B row k's bitmap: its first word's offset in the window (c0 is a
            // multiple of 32 and the window holds the whole row) and its words
            const int2 h = P.bhdr[k];
            kwn[lane] = h.y > 0 ? ((h.x - (c0 >> 5)) << 16) | h.y : 0;
        }
        if (!whole) {
            int b2 = lower_bound_col(P.B.col, b, e, c0);
            e = lower_bound_col(P.B.col, b2, e, c1);
            b = b2;
        }
        if (store_a) ka_of(S)[lane] = P.A.val[seg + lane];
        S.kb[lane] = b;
        S.kl[lane] = e - b;
    }
    __syncwarp();
}

// ---- symbolic pass, table map: plain flag stores, four pieces per step
__device__ __forceinline__ void mark_row(const int* __restrict__ col, int s, int e, int c0, int cend, int lane,
                                         ProdSmem<true>& S) {
    for (int q0 = s; q0 < e; q0 += 128) {
        int cs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * 32 + lane;
            cs[u] = q < e ? col[q] : INT_MIN;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (cs[u] >= c0 && cs[u] < cend) S.tab[cs[u] - c0] = 1;
    }
}
__device__ __forceinline__ void mark_one(int o, ProdSmem<true>& S) { S.tab[o] = 1; }
__device__ __forceinline__ void clear_map(int wlen, int lane, ProdSmem<true>& S) {
    uint4* t4 = reinterpret_cast<uint4*>(S.tab);
    const int n16 = (wlen + 7) >> 3;
    for (int i = lane; i < n16; i += 32) t4[i] = make_uint4(0u, 0u, 0u, 0u);
}

// ---- symbolic pass, bitmap map: lane l walks a contiguous slice of the row
// and ORs whole runs of columns into a bitmap word at a time.  CHK: test
// each column against [c0, cend); a B row needs no test, since
// load_segment has already clipped it to that range (or, for a row that
// takes one chunk, the range spans every B column of the row).
template <bool CHK, int W>
__device__ __forceinline__ void mark_row(const int* __restrict__ col, int s, int e, int c0, int cend, int lane,
                                         ProdSmem<false, W>& S) {
    const int m = (e - s + 31) >> 5;
    const int q0 = s + lane * m, q1 = min(e, q0 + m);
    unsigned curw = 0xffffffffu, mask = 0u;
    for (int q = q0; q < q1; q += 4) {
        int cs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cs[u] = q + u < q1 ? col[q + u] : INT_MIN;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int c = cs[u];
            if (CHK ? (c < c0 || c >= cend) : (q + u >= q1)) continue;
            unsigned off = (unsigned)(c - c0), w = off >> 5;
            if (w != curw) {
                if (mask) atomicOr(&S.pm[curw].y, mask);
                curw = w;
                mask = 0u;
            }
            mask |= 1u << (off & 31);
        }
    }
    if (mask) atomicOr(&S.pm[curw].y, mask);
}
// Two B rows at once, each as mark_row<false> marks it (lane l walks its
// contiguous slice of each row): the column loads of both rows are issued
// before either row's columns are ORed in, so the second row's loads do not
// wait for the first row's marking.  The rows are clipped to the window.
template <int W>
__device__ __forceinline__ void mark_row_pair(const int* __restrict__ col, int sa, int ea, int sb, int eb, int c0,
                                              int lane, ProdSmem<false, W>& S) {
    const int ma = (ea - sa + 31) >> 5, mb = (eb - sb + 31) >> 5;
    int qa = sa + lane * ma, qb = sb + lane * mb;
    const int qa1 = min(ea, qa + ma), qb1 = min(eb, qb + mb);
    unsigned wa = 0xffffffffu, ka = 0u, wb = 0xffffffffu, kb = 0u;
    while (qa < qa1 || qb < qb1) {
        int cs[2][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            cs[0][u] = qa + u < qa1 ? col[qa + u] : 0;
            cs[1][u] = qb + u < qb1 ? col[qb + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (qa + u >= qa1) continue;
            const unsigned off = (unsigned)(cs[0][u] - c0), w = off >> 5;
            if (w != wa) {
                if (ka) atomicOr(&S.pm[wa].y, ka);
                wa = w;
                ka = 0u;
            }
            ka |= 1u << (off & 31);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (qb + u >= qb1) continue;
            const unsigned off = (unsigned)(cs[1][u] - c0), w = off >> 5;
            if (w != wb) {
                if (kb) atomicOr(&S.pm[wb].y, kb);
                wb = w;
                kb = 0u;
            }
            kb |= 1u << (off & 31);
        }
        qa += 4;
        qb += 4;
    }
    if (ka) atomicOr(&S.pm[wa].y, ka);
    if (kb) atomicOr(&S.pm[wb].y, kb);
}
// Short B rows (at most 32 entries each): lane i marks the segment's B row i,
// so the rows' column loads are in flight together instead of one row after
// the other.  The rows are clipped to [c0, cend) (see mark_row).
template <int W>
__device__ __forceinline__ void mark_rows_short(const int* __restrict__ col, int cnt, int c0, int cend, int lane,
                                                ProdSmem<false, W>& S, bool active = true) {
    if (lane >= cnt || !active) return;
    const int s = S.kb[lane], e = s + S.kl[lane];
    unsigned curw = 0xffffffffu, mask = 0u;
#pragma unroll 2
    for (int q = s; q < e; q += 4) {
        int cs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cs[u] = q + u < e ? col[q + u] : INT_MIN;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = cs[u];
            if (q + u >= e) continue;
            const unsigned off = (unsigned)(c - c0), w = off >> 5;
            if (w != curw) {
                if (mask) atomicOr(&S.pm[curw].y, mask);
                curw = w;
                mask = 0u;
            }
            mask |= 1u << (off & 31);
        }
    }
    if (mask) atomicOr(&S.pm[curw].y, mask);
}
template <int W>
__device__ __forceinline__ void mark_one(int o, ProdSmem<false, W>& S) { atomicOr(&S.pm[o >> 5].y, 1u << (o & 31)); }
template <int W>
__device__ __forceinline__ void clear_map(int wlen, int lane, ProdSmem<false, W>& S) {
    const int nw = (wlen + 31) >> 5;
    for (int w = lane; w < nw; w += 32) S.pm[w].y = 0u;
}

// The B rows of A's row [pa0, pa1) into the bitmap, for a row that takes one
// chunk whose first column c0 is a multiple of 32: a B row with a bitmap
// (bhdr) is ORed in a word at a time, lane l collecting the window words
// l, l + 32, ... in registers (coalesced loads, no shared-memory traffic
// until the end); the others are marked column by column as in build_map.
template <int W>
__device__ __forceinline__ void mark_from_bitmaps(const ProductArgs& P, int pa0, int pa1, int c0, int cend, int lane,
                                                  ProdSmem<false, W>& S, bool store_a, unsigned long long* fma) {
    constexpr int R = (W + 31) / 32;
    unsigned reg[R];
#pragma unroll
    for (int u = 0; u < R; ++u) reg[u] = 0u;
    int* kwn = reinterpret_cast<int*>(S.colbuf);  // free until the slots are assigned
    const unsigned* __restrict__ bits = P.bbits;
    for (int seg = pa0; seg < pa1; seg += 32) {
        const int cnt = min(32, pa1 - seg);
        load_segment<false>(P, seg, cnt, true, c0, cend, lane, S, store_a, fma, kwn);
        // rows without a bitmap: short ones one per lane, long ones by the warp
        const int my = lane < cnt && kwn[lane] == 0 ? S.kl[lane] : 0;
        mark_rows_short(P.B.col, cnt, c0, cend, lane, S, my > 0 && my <= 32);
        unsigned longm = __ballot_sync(kFull, my > 32);
        while (longm) {
            const int i = __ffs(longm) - 1;
            longm &= longm - 1u;
            mark_row<false>(P.B.col, S.kb[i], S.kb[i] + S.kl[i], c0, cend, lane, S);
        }
        // U B rows at a time (4; 2 for the wide window's 16 words per lane):
        // their words are loaded before any is ORed in, so the loads of
        // consecutive rows are in flight together
        constexpr int U = R <= 5 ? 4 : 2;
        for (int i = 0; i < cnt; i += U) {
            unsigned t[U][R];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int h = i + j < cnt ? kwn[i + j] : 0;
                const int kw = h >> 16, kn = h & 0xffff;
                const int base = S.kb[i + j < cnt ? i + j : i] - kw;  // bits[base + w]: window word w
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    const int w = lane + 32 * u;
                    t[j][u] = h != 0 && w >= kw && w < kw + kn ? bits[base + w] : 0u;
                }
            }
#pragma unroll
            for (int j = 0; j < U; ++j)
#pragma unroll
                for (int u = 0; u < R; ++u) reg[u] |= t[j][u];
        }
        __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int w = lane + 32 * u;
        if (w < W && reg[u]) S.pm[w].y |= reg[u];
    }
    __syncwarp();
}

// Mark every output column of row r in [c0, cend) (cend - c0 <= kCols).
// BMP: B row bitmaps may be used (not in the batch kernel's wide window).
// PAIR: long B rows are marked two at a time (not in the batch kernel, which
// runs at its register limit).
template <bool TAB, bool BMP = false, bool PAIR = false, int W>
__device__ __forceinline__ void build_map(const ProductArgs& P, const AddTerm* add, int nadd, unsigned tmask, int r,
                                          int c0, int cend, int pa0, int pa1, bool whole, int lane, ProdSmem<TAB, W>& S,
                                          bool store_a, int ab, int ae, unsigned long long* fma = nullptr) {
    clear_map(cend - c0, lane, S);
    __syncwarp();
    for (int t = 0; t < nadd; ++t) {
        if (!((tmask >> t) & 1u)) continue;
        const AddTerm& T = add[t];
        if (!T.rb) {
            if (lane == 0 && r >= c0 && r < cend) mark_one(r - c0, S);
        } else {
            // (term t's row range is in lane t)
            const int s = __shfl_sync(kFull, ab, t), e = __shfl_sync(kFull, ae, t);
            if constexpr (TAB) mark_row(T.col, s, e, c0, cend, lane, S);
            else mark_row<true>(T.col, s, e, c0, cend, lane, S);
        }
    }
    if constexpr (!TAB && BMP) {
        if (whole && P.bhdr) {
            mark_from_bitmaps(P, pa0, pa1, c0, cend, lane, S, store_a, fma);
            return;
        }
    }
    for (int seg = pa0; seg < pa1; seg += 32) {
        const int cnt = min(32, pa1 - seg);
        load_segment<TAB>(P, seg, cnt, whole, c0, cend, lane, S, store_a, fma);
        if constexpr (!TAB) {
            if (warp_max(lane < cnt ? S.kl[lane] : 0) <= 32) {
                mark_rows_short(P.B.col, cnt, c0, cend, lane, S);
                __syncwarp();
                continue;
            }
        }
        if constexpr (TAB) {
            for (int i = 0; i < cnt; ++i) mark_row(P.B.col, S.kb[i], S.kb[i] + S.kl[i], c0, cend, lane, S);
        } else {
            int i = 0;
            if constexpr (PAIR)
                for (; i + 1 < cnt; i += 2)
                    mark_row_pair(P.B.col, S.kb[i], S.kb[i] + S.kl[i], S.kb[i + 1], S.kb[i + 1] + S.kl[i + 1], c0,
                                  lane, S);
            for (; i < cnt; ++i) mark_row<false>(P.B.col, S.kb[i], S.kb[i] + S.kl[i], c0, cend, lane, S);
        }
        __syncwarp();
    }
    __syncwarp();
}

// number of marked columns in [0, wlen)
__device__ __forceinline__ int count_marks(int wlen, int lane, const ProdSmem<true>& S) {
    int total = 0;
    for (int i0 = 0; i0 < wlen; i0 += 32) {
        int i = i0 + lane;
        total += __popc(__ballot_sync(kFull, i < wlen && S.tab[i] != 0));
    }
    return total;
}
template <int W>
__device__ __forceinline__ int count_marks(int wlen, int lane, const ProdSmem<false, W>& S) {
    int s = 0;
    for (int w = lane; w < ((wlen + 31) >> 5); w += 32) s += __popc(S.pm[w].y);
    return warp_sum(s);
}

// Number the marked columns of [0, wlen) in ascending order and fill
// colbuf.  Only the first kAccCap get a slot; returns their count and sets
// *cut to the offset of the first column without one (wlen if all fit).
__device__ __forceinline__ int assign_slots(int wlen, int cap, int lane, ProdSmem<true>& S, int* cut) {
    int run = 0, cutoff = wlen;
    for (int i0 = 0; i0 < wlen; i0 += 32) {
        const int i = i0 + lane;
        const bool f = i < wlen && S.tab[i] != 0;
        const unsigned m = __ballot_sync(kFull, f);
        const int slot = run + __popc(m & lanemask_lt());
        if (f && slot < cap) {
            S.tab[i] = (unsigned short)slot;
            S.colbuf[slot] = (unsigned short)i;
        }
        if (run <= cap && run + __popc(m) > cap) {
            const unsigned fo = __ballot_sync(kFull, f && slot == cap);
            cutoff = i0 + __ffs(fo) - 1;
        }
        run += __popc(m);
        if (cutoff < wlen) break;
    }
    __syncwarp();
    *cut = cutoff;
    return min(run, cap);
}
template <int W>
__device__ __forceinline__ int assign_slots(int wlen, int cap, int lane, ProdSmem<false, W>& S, int* cut) {
    constexpr int per = (W + 31) / 32;  // words per lane (the last lanes' partly past nw)
    const int nw = (wlen + 31) >> 5;
    const int base = lane * per;
    int s = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) s += base + i < nw ? __popc(S.pm[base + i].y) : 0;
    int run = warp_excl_scan(s, lane);
    const int total = __shfl_sync(kFull, run + s, 31);
#pragma unroll
    for (int i = 0; i < per; ++i) {
        if (base + i < nw) {
            S.pm[base + i].x = (unsigned)run;
            run += __popc(S.pm[base + i].y);
        }
    }
    __syncwarp();
    int cutoff = wlen;
    if (total > cap) {
        int found = INT_MAX;
        for (int w = lane; w < nw; w += 32) {
            const int pc = __popc(S.pm[w].y), pre = (int)S.pm[w].x;
            if (pre <= cap && cap < pre + pc) {
                unsigned bits = S.pm[w].y;
                for (int i = 0; i < cap - pre; ++i) bits &= bits - 1u;  // drop the lowest ones
                found = w * 32 + (__ffs(bits) - 1);
            }
        }
        cutoff = warp_min(found);
    }
    if (nw <= 8) {
        // a few words: lane l takes bit l of one word at a time (no lane
        // walks a word's set bits alone)
        for (int w = 0; w < nw; ++w) {
            const unsigned bits = S.pm[w].y;
            if ((bits >> lane) & 1u) {
                const int o = w * 32 + lane;
                if (o < cutoff) S.colbuf[(int)S.pm[w].x + __popc(bits & lanemask_lt())] = (unsigned short)o;
            }
        }
    } else {
        for (int w = lane; w < nw; w += 32) {
            unsigned bits = S.pm[w].y;
            int idx = (int)S.pm[w].x;
            while (bits) {
                const int o = w * 32 + __ffs(bits) - 1;
                if (o < cutoff) S.colbuf[idx] = (unsigned short)o;
                ++idx;
                bits &= bits - 1u;
            }
        }
    }
    __syncwarp();
    *cut = cutoff;
    return min(total, cap);
}

// The 128 entries [off, off + 128) of B row kk of the segment, four 32-entry
// pieces, one element of each per lane (column -1: no element).
struct Chunk {
    int c[4];
    double v[4];
};

template <bool TAB, int W>
__device__ __forceinline__ void chunk_load(const int* __restrict__ bcol, const double* __restrict__ bval,
                                           const ProdSmem<TAB, W>& S, int kk, int off, int lane, Chunk& ch) {
    const int len = S.kl[kk];
    const int* rc = bcol + S.kb[kk] + lane;
    const double* rv = bval + S.kb[kk] + lane;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int q = off + u * 32;
        ch.c[u] = -1;
        if (q + lane < len) {
            ch.c[u] = rc[q];
            ch.v[u] = rv[q];
        }
    }
}

template <bool TAB, int W>
__device__ __forceinline__ void chunk_next(const ProdSmem<TAB, W>& S, int cnt, int& kk, int& off) {
    off += 128;
    if (off >= S.kl[kk]) {
        off = 0;
        do {
            ++kk;
        } while (kk < cnt && S.kl[kk] == 0);
    }
}

// Fold a chunk in: its columns are distinct, so the four read-modify-writes
// are independent and are interleaved.  `np` (the same in every lane) is the
// number of pieces holding entries: a DFMA occupies the FP64 pipe for the
// whole warp, so the empty pieces at a row's end are branched over.
template <bool TAB, int W>
__device__ __forceinline__ void chunk_fold(ProdSmem<TAB, W>& S, const Chunk& ch, double a, int c0, int np = 4) {
    int i[4];
    double x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) i[u] = ch.c[u] >= 0 ? slot_lookup(S, ch.c[u] - c0) : -1;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (i[u] >= 0) x[u] = S.acc[i[u]];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (u >= np) break;
        if (i[u] >= 0) S.acc[i[u]] = __fma_rn(a, ch.v[u], x[u]);
    }
}

// acc[slot(j)] = fma(a_rk, b_kj, acc[slot(j)]) for the segment's k in order.
// Table map: chunks stream through three register sets (the loads of the
// next two are in flight while one is folded in).  Bitmap map (more warps,
// fewer registers): one chunk at a time.  A warp barrier separates
// consecutive B rows (the order of the fma chain).
template <bool WIDE>
__device__ __forceinline__ void accumulate_segment(const ProductArgs& P, int /*seg*/, int cnt, int c0, int lane,
                                                   ProdSmem<true>& S, bool /*wide_row*/) {
    const int* __restrict__ bcol = P.B.col;
    const double* __restrict__ bval = P.B.val;
    int k0 = 0, o0 = 0;
    while (k0 < cnt && S.kl[k0] == 0) ++k0;
    if (k0 >= cnt) return;
    Chunk A, B, C;
    chunk_load<true>(bcol, bval, S, k0, o0, lane, A);
    int k1 = k0, o1 = o0;
    chunk_next<true>(S, cnt, k1, o1);
    int k2 = k1, o2 = o1;
    if (k1 < cnt) {
        chunk_load<true>(bcol, bval, S, k1, o1, lane, B);
        chunk_next<true>(S, cnt, k2, o2);
    }
    auto step = [&](Chunk& X, Chunk& Z) -> bool {
        if (k2 < cnt) chunk_load<true>(bcol, bval, S, k2, o2, lane, Z);
        chunk_fold<true>(S, X, S.ka[k0], c0);
        if (k1 >= cnt) return false;
        if (k1 != k0) __syncwarp();
        k0 = k1;
        o0 = o1;
        k1 = k2;
        o1 = o2;
        if (k2 < cnt) chunk_next<true>(S, cnt, k2, o2);
        return true;
    };
    for (;;) {
        if (!step(A, C)) break;
        if (!step(B, A)) break;
        if (!step(C, B)) break;
    }
    __syncwarp();
}
// One 32-lane piece of short B row kk (at most 32 entries): column -1 where
// there is none.
template <int W>
__device__ __forceinline__ void short_load(const int* __restrict__ bcol, const double* __restrict__ bval,
                                           const ProdSmem<false, W>& S, int cnt, int kk, int lane, int& c, double& v) {
    c = -1;
    v = 0.0;
    if (kk < cnt && lane < S.kl[kk]) {
        const int q = S.kb[kk] + lane;
        c = bcol[q];
        v = bval[q];
    }
}
template <int W>
__device__ __forceinline__ void short_fold(ProdSmem<false, W>& S, int c, double v, double a, int c0) {
    if (c >= 0) {
        const int i = slot_lookup(S, c - c0);
        S.acc[i] = __fma_rn(a, v, S.acc[i]);
    }
}

template <bool WIDE, int W>
__device__ __forceinline__ void accumulate_segment(const ProductArgs& P, int seg, int cnt, int c0, int lane,
                                                   ProdSmem<false, W>& S, bool wide_row) {
    const int* __restrict__ bcol = P.B.col;
    const double* __restrict__ bval = P.B.val;
    const double* ka = ka_of(S);
    // a_rk of row kk: kept in the accumulator's last slots, or (WIDE, or a
    // row that takes every slot) read from A's row (the same address in
    // every lane)
    const bool a_global = WIDE || wide_row;
    auto a_of = [&](int kk) { return a_global ? P.A.val[seg + kk] : ka[kk]; };
    if (warp_max(lane < cnt ? S.kl[lane] : 0) <= 32) {
        // every B row is one piece: the pieces of the next three rows are
        // loaded while one is folded (rows in k order, a warp barrier between)
        int ca, cb, cc, cd;
        double va, vb, vc, vd;
        short_load(bcol, bval, S, cnt, 0, lane, ca, va);
        short_load(bcol, bval, S, cnt, 1, lane, cb, vb);
        short_load(bcol, bval, S, cnt, 2, lane, cc, vc);
        for (int kk = 0; kk < cnt; kk += 4) {
            short_load(bcol, bval, S, cnt, kk + 3, lane, cd, vd);
            short_fold(S, ca, va, a_of(kk), c0);
            __syncwarp();
            if (kk + 1 >= cnt) break;
            short_load(bcol, bval, S, cnt, kk + 4, lane, ca, va);
            short_fold(S, cb, vb, a_of(kk + 1), c0);
            __syncwarp();
            if (kk + 2 >= cnt) break;
            short_load(bcol, bval, S, cnt, kk + 5, lane, cb, vb);
            short_fold(S, cc, vc, a_of(kk + 2), c0);
            __syncwarp();
            if (kk + 3 >= cnt) break;
            short_load(bcol, bval, S, cnt, kk + 6, lane, cc, vc);
            short_fold(S, cd, vd, a_of(kk + 3), c0);
            __syncwarp();
        }
        return;
    }
    for (int kk = 0; kk < cnt; ++kk) {
        const int len = S.kl[kk];
        if (len == 0) continue;
        const double a = a_of(kk);
        if (len <= 32) {
            // a short B row fills one piece: fold only that one (a DFMA
            // occupies the FP64 pipe for the whole warp, active lanes or not)
            if (lane < len) {
                const int q = S.kb[kk] + lane;
                const int i = slot_lookup(S, bcol[q] - c0);
                S.acc[i] = __fma_rn(a, bval[q], S.acc[i]);
            }
        } else {
            // whole 128-entry chunks: four full pieces, no per-lane tests
            const int* __restrict__ rc = bcol + S.kb[kk] + lane;
            const double* __restrict__ rv = bval + S.kb[kk] + lane;
            int off = 0;
            for (; off + 128 <= len; off += 128) {
                int j[4];
                double v[4], x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    j[u] = rc[off + 32 * u];
                    v[u] = rv[off + 32 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) j[u] = slot_lookup(S, j[u] - c0);
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = S.acc[j[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) S.acc[j[u]] = __fma_rn(a, v[u], x[u]);
            }
            // the rest (up to four pieces, the last one partial), two pieces
            // at a time with their read-modify-writes interleaved
            for (; off < len; off += 64) {
                const bool in0 = off + lane < len;
                const bool two = off + 32 < len;  // (the same in every lane)
                const bool in1 = two && off + 32 + lane < len;
                int j0 = 0, j1 = 0;
                double v0 = 0.0, v1 = 0.0, x0 = 0.0, x1 = 0.0;
                if (in0) {
                    j0 = rc[off];
                    v0 = rv[off];
                }
                if (in1) {
                    j1 = rc[off + 32];
                    v1 = rv[off + 32];
                }
                if (in0) j0 = slot_lookup(S, j0 - c0);
                if (in1) j1 = slot_lookup(S, j1 - c0);
                if (in0) x0 = S.acc[j0];
                if (in1) x1 = S.acc[j1];
                if (in0) S.acc[j0] = __fma_rn(a, v0, x0);
                if (two && in1) S.acc[j1] = __fma_rn(a, v1, x1);
            }
        }
        __syncwarp();
    }
}

// Statistics of one row of a batched step, added to its instance's record:
// multiply-adds (per-lane partial counts), Algorithm 1 candidates (per lane),
// entries written and the largest |x| (per lane).
__device__ __forceinline__ void row_stats_batch(const ProductArgs& P, int inst, unsigned long long fma,
                                                unsigned long long cand, int written, unsigned long long absmax,
                                                int lane, int span = 0) {
    for (int o = 16; o; o >>= 1) {
        fma += __shfl_xor_sync(kFull, fma, o);
        cand += __shfl_xor_sync(kFull, cand, o);
    }
    absmax = warp_max_u64(absmax);
    if (lane == 0) {
        if (P.stat_tab) {
            StepStat* st = P.stat_tab + inst;
            if (fma) atomicAdd(&st->fma, fma);
            if (written) atomicAdd(&st->nnz_pre, (unsigned long long)written);
            if (cand) atomicAdd(&st->ncand, cand);
            if (span > 0) atomicMax(&st->span_max, (unsigned)span);
        }
        if (P.absmax_slot && absmax) atomicMax(&(P.absmax_slot + (size_t)inst * P.absmax_stride)->absmax, absmax);
    }
}

// Per-warp state of the product kernel across the rows a warp processes.
struct RowState {
    unsigned long long written = 0ull, cand = 0ull, absmax = 0ull, fma = 0ull;
    int span = 0;  // widest column window of this warp's rows
    Arena arena;
    CandArena carena;
};

// One output row r of C = sum_t alpha_t M_t + A B (see k_product), processed
// by one warp with the slot map S.
template <bool TAB, bool BATCH, bool WIDE, int W>
__device__ __forceinline__ void product_row(const ProductArgs& P, const AddTerm* add, ProdSmem<TAB, W>& S,
                                            RowState& st, int r, int lane) {
    using Smem = ProdSmem<TAB, W>;
    // columns and slots of one chunk (lowered only to exercise chunking)
    const int kCols = P.chunk_cols > 0 && P.chunk_cols < Smem::kCols ? P.chunk_cols : Smem::kCols;
    constexpr int kCapN = (TAB || WIDE) ? kAccCap : kAccCap - 32;  // a row's slots
    const int kSlots = P.chunk_slots > 0 && P.chunk_slots < kCapN ? P.chunk_slots : kCapN;
    const int nadd = P.nadd;
    const unsigned long long eps_bits = (unsigned long long)__double_as_longlong(P.eps_g);
    unsigned long long& my_written = st.written;
    unsigned long long& my_cand = st.cand;
    unsigned long long& my_absmax = st.absmax;
    unsigned long long& my_fma = st.fma;
    int& my_span = st.span;
    Arena& arena = st.arena;
    CandArena& carena = st.carena;


    // ---- the row's terms: single instance, every term and the product;
    // batch, what the row's instance does in this step
    bool prod = P.A.rb != nullptr;
    unsigned tmask = kFull;  // terms present in this row (batch: coefficient != 0)
    int r_inst = 0;
    if constexpr (BATCH) {
        r_inst = P.inst[r];
        const BatchStep bs = P.bstep[r_inst];
        // the row equals the norm phase's power: k_reuse_copy_batch writes it
        if (bs.reuse && __ldcg(P.inst_dropped + r_inst) == 0) return;
        if (bs.mode == kBatchSkip || bs.mode == kBatchPass) {
            if (lane == 0) {
                P.out_rb[r] = bs.mode == kBatchPass ? P.B.rb[r] : 0;
                P.out_re[r] = bs.mode == kBatchPass ? P.B.re[r] : 0;
            }
            return;
        }
        prod = bs.mode == kBatchProduct;
        const double a_lane = lane < nadd ? P.alpha_tab[(size_t)lane * P.ninst + r_inst] : 0.0;
        tmask = __ballot_sync(kFull, __double_as_longlong(a_lane) != 0ll);
    }
    // batch: the counters are per row (reported per instance after each
    // row); single: running totals, reported per block at the end
    if constexpr (BATCH) {
        my_fma = 0ull;
        my_cand = 0ull;
    }
    const unsigned long long fma0 = BATCH ? 0ull : my_fma, cand0 = BATCH ? 0ull : my_cand;
    // ---- column window of row r and the row's multiply-add count.  A
    // matrix (or a batch instance) of at most one map's columns is its own
    // window: no loads to find the row's, and the B row lengths are counted
    // while the map is built
    int lo = INT_MAX, hi = -1;
    bool fixed = false;
    int fixed_span = 0;
    if constexpr (!TAB) {
        int w0 = 0, w1 = P.n;
        if constexpr (BATCH) {
            w1 = -1;
            if (P.inst_off) {
                w0 = P.inst_off[r_inst];
                w1 = P.inst_off[r_inst + 1];
            }
        }
        // with B row bitmaps the window starts at a multiple of 32 columns
        const int a0 = P.bhdr ? (w0 & ~31) : w0;
        if (w1 > w0 && w1 - a0 <= kCols) {
            lo = a0;
            hi = w1 - 1;
            fixed = true;
            fixed_span = w1 - w0;
        }
    }
    // addend term t's row range, in lane t (the terms' loads in parallel;
    // the loops over the terms below take it with a shuffle)
    int ab = 0, ae = 0;
    const bool my_term = lane < nadd && ((tmask >> lane) & 1u);
    if (my_term && add[lane].rb) {
        ab = add[lane].rb[r];
        ae = add[lane].re[r];
    }
    if (!fixed && my_term) {
        const AddTerm& T = add[lane];
        if (!T.rb) {
            lo = min(lo, r);
            hi = max(hi, r);
        } else if (ab < ae) {
            lo = min(lo, T.col[ab]);
            hi = max(hi, T.col[ae - 1]);
        }
    }
    int pa0 = 0, pa1 = 0;
    if (prod) {
        pa0 = P.A.rb[r];
        pa1 = P.A.re[r];
    }
    for (int p = pa0 + lane; p < pa1 && !fixed; p += 32) {
        int k = P.A.col[p];
        int s = P.B.rb[k], e = P.B.re[k];
        my_fma += (unsigned long long)(e - s);
        if (s < e) {
            lo = min(lo, P.B.col[s]);
            hi = max(hi, P.B.col[e - 1]);
        }
    }
    if (my_term) my_fma += add[lane].rb ? (unsigned long long)(ae - ab) : 1ull;
    lo = warp_min(lo);
    hi = warp_max(hi);
    const int row_span = fixed ? fixed_span : hi - lo + 1;  // the statistic: before any alignment
    my_span = max(my_span, row_span);
    if (hi < lo) {
        if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
        if constexpr (BATCH) row_stats_batch(P, r_inst, my_fma - fma0, 0ull, 0, 0ull, lane);
        return;
    }
    if constexpr (!TAB) {
        if (P.bhdr) lo &= ~31;
    }

    // ---- exact entry count of the row, reserve it in the pool
    long long total = 0;
    bool reuse = false;
    if (hi - lo + 1 <= kCols) {
        build_map<TAB, (!BATCH || W == kBmWords), !BATCH>(P, add, nadd, tmask, r, lo, hi + 1, pa0, pa1, true, lane, S,
                                                   !WIDE, ab, ae, fixed ? &my_fma : nullptr);
        total = count_marks(hi - lo + 1, lane, S);
        reuse = true;
    } else {
        for (long long c0 = lo; c0 <= hi; c0 += kCols) {
            int cend = (int)min((long long)hi + 1, c0 + kCols);
            build_map<TAB, false, !BATCH>(P, add, nadd, tmask, r, (int)c0, cend, pa0, pa1, false, lane, S, !WIDE, ab,
                                          ae);
            total += count_marks(cend - (int)c0, lane, S);
        }
    }
    const long long base = arena_take(arena, (unsigned long long)((total + 3) & ~3LL), P.arena, P.ctl, P.pool_val, lane);
    if (base < 0) {
        if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
        return;
    }
    // a row of the narrow accumulator that fits every slot (kAccCap) in one
    // chunk takes them all and reads a_rk from A's row, as WIDE does,
    // instead of two column chunks (single-matrix kernels: the batch kernel
    // runs at its register limit)
    bool wide_row = WIDE;
    int slots = kSlots;
    if constexpr (!TAB && !WIDE && !BATCH) {
        if (reuse && total > kSlots && total <= kAccCap && P.chunk_slots <= 0) {
            wide_row = true;
            slots = kAccCap;
        }
    }
    const bool single = reuse && total <= slots;
    int written = 0;
    int c0 = lo;
    while (c0 <= hi) {
        int cend = (int)min((long long)hi + 1, (long long)c0 + kCols);
        if (!reuse)
            build_map<TAB, false, !BATCH>(P, add, nadd, tmask, r, c0, cend, pa0, pa1, false, lane, S, !WIDE, ab, ae);
        reuse = false;
        int cut;
        const int cnt = assign_slots(cend - c0, slots, lane, S, &cut);
        const int c1 = c0 + cut;
        for (int i = lane; i < cnt; i += 32) S.acc[i] = 0.0;
        __syncwarp();

        // ---- weighted sum of the addends, t ascending
        for (int t = 0; t < nadd; ++t) {
            if (!((tmask >> t) & 1u)) continue;
            const AddTerm& T = add[t];
            // batch: the row's instance's coefficient (a small, cached table)
            const double alpha = BATCH ? P.alpha_tab[(size_t)t * P.ninst + r_inst] : T.alpha;
            if (!T.rb) {
                if (lane == 0 && r >= c0 && r < c1) {
                    int i = slot_lookup(S, r - c0);
                    S.acc[i] = __fma_rn(alpha, 1.0, S.acc[i]);
                }
            } else {
                const int s = __shfl_sync(kFull, ab, t), e = __shfl_sync(kFull, ae, t);
                for (int q = s + lane; q < e; q += 32) {
                    int c = T.col[q];
                    if (c >= c0 && c < c1) {
                        int i = slot_lookup(S, c - c0);
                        S.acc[i] = __fma_rn(alpha, T.val[q], S.acc[i]);
                    }
                }
            }
            __syncwarp();
        }

        // ---- product A B: k of row r ascending
        for (int seg = pa0; seg < pa1; seg += 32) {
            const int cnt_seg = min(32, pa1 - seg);
            load_segment<TAB>(P, seg, cnt_seg, single, c0, c1, lane, S, !wide_row);
            accumulate_segment<WIDE>(P, seg, cnt_seg, c0, lane, S, wide_row);
        }

        // ---- write back the nonzero entries in column order; the entries
        // with |x| <= eps_g enter the column sums of Algorithm 1's first pass
        // (batch: the filter of the row's instance, read here rather than
        // held in registers through the row)
        unsigned long long r_eps = eps_bits;
        int r_lsb = P.e_lsb;
        bool r_filt = P.filtering != 0;
        if constexpr (BATCH) {
            const BatchStep& bs = P.bstep[r_inst];
            r_filt = bs.eps_g > 0.0;
            r_eps = (unsigned long long)__double_as_longlong(bs.eps_g);
            r_lsb = bs.e_lsb;
        }
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            int i = i0 + lane;
            double x = 0.0;
            int c = 0;
            if (i < cnt) {
                x = S.acc[i];
                c = c0 + (int)S.colbuf[i];
            }
            unsigned long long xb = mag_bits(x);
            bool nz = i < cnt && xb != 0ull;
            unsigned m = __ballot_sync(kFull, nz);
            const bool cand = nz && r_filt && xb <= r_eps;
            if (nz) {
                long long pos = (long long)base + written + __popc(m & lanemask_lt());
                P.pool_col[pos] = c;
                P.pool_val[pos] = x;
                my_absmax = xb > my_absmax ? xb : my_absmax;
                if (cand) {
                    exact_add(P.words + c, (size_t)P.n, P.sticky + c, xb, r_lsb);
                    ++my_cand;
                }
            }
            if (P.cand_col)
                cand_push(carena, cand, c, xb, P.cand_col, P.cand_x, &P.ctl->cand_cnt[0], P.cand_cap,
                          P.cand_chunk, &P.ctl->cand_over, lane);
            written += __popc(m);
        }
        __syncwarp();
        c0 = c1;
    }
    // the row's unused reserved slots read as exact zeros (never candidates)
    const long long rend = base + ((total + 3) & ~3LL);
    for (long long q = base + written + lane; q < rend; q += 32) P.pool_val[q] = 0.0;
    if (lane == 0) {
        P.out_rb[r] = (int)base;
        P.out_re[r] = (int)(base + written);
    }
    if constexpr (BATCH) {
        row_stats_batch(P, r_inst, my_fma - fma0, my_cand - cand0, written, my_absmax, lane, row_span);
        my_absmax = 0ull;
    } else if (lane == 0) {
        my_written += (unsigned long long)written;
    }
}

template <bool TAB, bool BATCH, bool WIDE, int W = kBmWords>
__global__ void __launch_bounds__(ProdSmem<TAB, W>::kWarps * 32, ProdSmem<TAB, W>::kBlocksPerSm)
    k_product(ProductArgs P) {
    // a baby step whose product equals an already computed power (no entry
    // dropped so far) is done by k_reuse_pass1 instead (same value in all blocks)
    if (P.skip_unless && __ldcg(P.skip_unless) == 0) return;
    using Smem = ProdSmem<TAB, W>;
    constexpr int kWarps = Smem::kWarps;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AddTerm* add = reinterpret_cast<AddTerm*>(smem_raw);
    Smem* warps = reinterpret_cast<Smem*>(smem_raw + sizeof(AddTerm) * kMaxAdd);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nadd = P.nadd;
    for (int t = threadIdx.x; t < nadd; t += blockDim.x) add[t] = P.add[t];
    __shared__ unsigned long long blk_written, blk_cand, blk_absmax, blk_fma, blk_arena;
    __shared__ int blk_span;
    if (threadIdx.x == 0) {
        // the block's warps take their first pool arenas with one atomic: at
        // the launch every warp wants one at once, on the same counter
        blk_arena = atomicAdd(&P.ctl->pool_used, (unsigned long long)kWarps * P.arena);
        blk_span = 0;
        blk_fma = 0ull;
        blk_written = 0ull;
        blk_cand = 0ull;
        blk_absmax = 0ull;
    }
    __syncthreads();
    Smem& S = warps[wib];
    RowState st;
    // (past the pool's capacity the first row's arena_take reports the overflow)
    if (blk_arena + (unsigned long long)kWarps * P.arena <= P.ctl->pool_cap) {
        st.arena.next = blk_arena + (unsigned long long)wib * P.arena;
        st.arena.end = st.arena.next + P.arena;
    }
    for (int r = blockIdx.x * kWarps + wib; r < P.n; r += gridDim.x * kWarps)
        product_row<TAB, BATCH, WIDE, W>(P, add, S, st, r, lane);
    // the unused end of this warp's arena reads as exact zeros too, and the
    // unused end of its candidate chunk as holes
    arena_close(st.arena, P.pool_val, lane);
    if (P.cand_col) cand_close(st.carena, P.cand_x, lane);
    if constexpr (BATCH) return;
    // ---- block totals for the step statistics
    st.cand = (unsigned long long)warp_sum((int)st.cand);
    st.absmax = warp_max_u64(st.absmax);
    for (int o = 16; o; o >>= 1) st.fma += __shfl_xor_sync(kFull, st.fma, o);
    if (lane == 0) {
        atomicAdd(&blk_fma, st.fma);
        atomicAdd(&blk_written, st.written);
        atomicAdd(&blk_cand, st.cand);
        atomicMax(&blk_absmax, st.absmax);
        atomicMax(&blk_span, st.span);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_fma) atomicAdd(&P.ctl->fma_total, blk_fma);
        if (P.stat) {
            if (blk_span > 0) atomicMax(&P.stat->span_max, (unsigned)blk_span);
            if (blk_fma) atomicAdd(&P.stat->fma, blk_fma);
            if (blk_written) atomicAdd(&P.stat->nnz_pre, blk_written);
            if (blk_cand) atomicAdd(&P.stat->ncand, blk_cand);
        }
        if (P.absmax_slot && blk_absmax) atomicMax(&P.absmax_slot->absmax, blk_absmax);
    }
}


// Keep the entries of row [s, e) with |x| > fb (bits), in place and in
// column order; the dropped tail is cleared to exact zeros.  Returns the new
// end.  Rounds of 128 entries, software-pipelined: the loads of round i + 1
// are issued before the writes of round i.  Entries only move left, so the
// writes of round i stay below its end and never reach round i + 1's
// entries, which were read before the warp barrier that ends round i.
__device__ __forceinline__ void compact_load(const int* col, const double* val, int q0, int e, int lane, int c[4],
                                             double x[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * 32 + lane;
        c[u] = 0;
        x[u] = 0.0;
        if (q < e) {
            c[u] = col[q];
            x[u] = val[q];
        }
    }
}

__device__ __forceinline__ int compact_row(int* col, double* val, int s, int e, unsigned long long fb, int lane) {
    int w = s;
    int c[4];
    double x[4];
    compact_load(col, val, s, e, lane, c, x);
    for (int q0 = s; q0 < e; q0 += 128) {
        int cn[4];
        double xn[4];
        compact_load(col, val, q0 + 128, e, lane, cn, xn);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool keep = q0 + u * 32 + lane < e && mag_bits(x[u]) > fb;
            const unsigned m = __ballot_sync(kFull, keep);
            if (keep) {
                const int pos = w + __popc(m & lanemask_lt());
                col[pos] = c[u];
                val[pos] = x[u];
            }
            w += __popc(m);
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = cn[u];
            x[u] = xn[u];
        }
    }
    for (int q = w + lane; q < e; q += 32) val[q] = 0.0;
    return w;
}

// ---------------------------------------------------------------- k_product_cta
// One output row per block of four warps: for matrices with fewer rows than
// the warp-per-row kernel has resident warps, whose B rows are long.  The
// block's warps share one bitmap slot map over the row's window (up to 4608
// columns) and kCtaCap accumulator slots:
//  - symbolic pass: each warp marks the B rows of every fourth 32-entry
//    segment of A's row (from their bitmaps when the step has them), ORing
//    into the shared map; a block-wide scan numbers the columns;
//  - numeric pass: the addends in order, then the B rows in k order, each B
//    row's entries spread over the block's 128 threads (four independent
//    read-modify-writes per thread: a B row's entries have distinct
//    columns), with a block barrier after each B row, so that every slot is
//    folded in the order of k_product (addends t ascending, then k
//    ascending) and the results are bitwise the same;
//  - write-back: each warp takes a quarter of the slots in column order,
//    positions from a block-wide count, Algorithm 1's first pass as in
//    k_product.
// A row whose window or pattern does not fit is computed by the block's
// first warp with the warp-per-row code (bitmap map, every accumulator
// slot) in the same shared memory, the other warps waiting.
constexpr int kCtaWarps = 4;
constexpr int kCtaCap = 2560;

struct CtaSmem {
    uint2 pm[kBmWords];  // the first member, as in ProdSmem<false, kBmWords> (mark_row uses only pm)
    double acc[kCtaCap];
    unsigned short colbuf[kCtaCap];
    int kb[kCtaWarps][32];
    int kl[kCtaWarps][32];
    int kwn[kCtaWarps][32];
    double ka[32];
    int wcnt[kCtaWarps];
    int lo, hi, total, fits;
    long long base;
};
static_assert(sizeof(ProdSmem<false, kBmWords>) <= sizeof(CtaSmem), "the warp-per-row fallback fits");

size_t cta_smem_bytes() { return sizeof(CtaSmem) + sizeof(AddTerm) * kMaxAdd; }

// block-wide exclusive scan of one int per thread; *total gets the sum
__device__ __forceinline__ int cta_excl_scan(int v, int tid, int* wsum, int* total) {
    const int lane = tid & 31, wib = tid >> 5;
    const int x = warp_excl_scan(v, lane);
    if (lane == 31) wsum[wib] = x + v;
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kCtaWarps; ++w) {
        before += w < wib ? wsum[w] : 0;
        all += wsum[w];
    }
    *total = all;
    __syncthreads();
    return before + x;
}

__device__ __forceinline__ void cta_row(const ProductArgs& P, const AddTerm* add, CtaSmem& S, RowState& st, int r,
                                        int tid) {
    const int lane = tid & 31, wib = tid >> 5;
    constexpr int kT = kCtaWarps * 32;
    const int nadd = P.nadd;
    const bool prod = P.A.rb != nullptr;
    int pa0 = 0, pa1 = 0;
    if (prod) {
        pa0 = P.A.rb[r];
        pa1 = P.A.re[r];
    }
    // ---- column window: the matrix itself when it is at most one map wide
    int lo = INT_MAX, hi = -1;
    int row_span = 0;
    if (P.n <= kBmBits) {
        lo = 0;
        hi = P.n - 1;
        row_span = P.n;
    } else {
        if (tid == 0)
            for (int t = 0; t < nadd; ++t) {
                const AddTerm& T = add[t];
                if (!T.rb) {
                    lo = min(lo, r);
                    hi = max(hi, r);
                } else if (T.rb[r] < T.re[r]) {
                    lo = min(lo, T.col[T.rb[r]]);
                    hi = max(hi, T.col[T.re[r] - 1]);
                }
            }
        for (int p = pa0 + tid; p < pa1; p += kT) {
            const int k = P.A.col[p];
            const int s = P.B.rb[k], e = P.B.re[k];
            if (s < e) {
                lo = min(lo, P.B.col[s]);
                hi = max(hi, P.B.col[e - 1]);
            }
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) {
            S.kb[wib][0] = lo;
            S.kl[wib][0] = hi;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kCtaWarps; ++w) {
            lo = min(lo, S.kb[w][0]);
            hi = max(hi, S.kl[w][0]);
        }
        __syncthreads();
        row_span = hi - lo + 1;
    }
    if (hi < lo) {  // no entry at all
        if (tid == 0) P.out_rb[r] = P.out_re[r] = 0;
        return;
    }
    st.span = max(st.span, row_span);
    if (P.bhdr) lo &= ~31;
    const int wlen = hi - lo + 1;
    const int nw = (wlen + 31) >> 5;
    if (wlen > kBmBits) {
        // wider than the map: the first warp computes the row alone
        if (wib == 0)
            product_row<false, false, true, kBmWords>(P, add, *reinterpret_cast<ProdSmem<false, kBmWords>*>(&S), st,
                                                      r, lane);
        __syncthreads();
        return;
    }
    // ---- symbolic pass
    for (int w = tid; w < nw; w += kT) S.pm[w].y = 0u;
    __syncthreads();
    ProdSmem<false, kBmWords>& M = *reinterpret_cast<ProdSmem<false, kBmWords>*>(&S);  // its pm is S.pm
    if (wib == 0) {
        for (int t = 0; t < nadd; ++t) {
            const AddTerm& T = add[t];
            if (!T.rb) {
                if (lane == 0 && r >= lo && r <= hi) mark_one(r - lo, M);
            } else {
                mark_row<true>(T.col, T.rb[r], T.re[r], lo, hi + 1, lane, M);
            }
        }
    }
    unsigned long long rf = 0ull;  // this thread's share of the row's multiply-adds
    constexpr int R = (kBmWords + 31) / 32;
    unsigned reg[R];
#pragma unroll
    for (int u = 0; u < R; ++u) reg[u] = 0u;
    for (int seg = pa0 + 32 * wib; seg < pa1; seg += 32 * kCtaWarps) {
        const int cnt = min(32, pa1 - seg);
        if (lane < cnt) {
            const int k = P.A.col[seg + lane];
            const int b = P.B.rb[k], e = P.B.re[k];
            rf += (unsigned long long)(e - b);
            S.kb[wib][lane] = b;
            S.kl[wib][lane] = e - b;
            int h = 0;
            if (P.bhdr) {
                const int2 bh = P.bhdr[k];
                h = bh.y > 0 ? ((bh.x - (lo >> 5)) << 16) | bh.y : 0;
            }
            S.kwn[wib][lane] = h;
        }
        __syncwarp();
        // rows without a bitmap: short ones one per lane, long ones by the warp
        const int my = lane < cnt && S.kwn[wib][lane] == 0 ? S.kl[wib][lane] : 0;
        if (my > 0 && my <= 32) {
            const int s0 = S.kb[wib][lane];
            unsigned curw = 0xffffffffu, mask = 0u;
            for (int q = s0; q < s0 + my; ++q) {
                const unsigned off = (unsigned)(P.B.col[q] - lo), w = off >> 5;
                if (w != curw) {
                    if (mask) atomicOr(&S.pm[curw].y, mask);
                    curw = w;
                    mask = 0u;
                }
                mask |= 1u << (off & 31);
            }
            if (mask) atomicOr(&S.pm[curw].y, mask);
        }
        unsigned longm = __ballot_sync(kFull, my > 32);
        while (longm) {
            const int i = __ffs(longm) - 1;
            longm &= longm - 1u;
            mark_row<false>(P.B.col, S.kb[wib][i], S.kb[wib][i] + S.kl[wib][i], lo, hi + 1, lane, M);
        }
        for (int i = 0; i < cnt; ++i) {
            const int h = S.kwn[wib][i];
            if (h == 0) continue;
            const int kw = h >> 16, kn = h & 0xffff;
            const int base = S.kb[wib][i] - kw;  // bits[base + w]: window word w
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int w = lane + 32 * u;
                if (w >= kw && w < kw + kn) reg[u] |= P.bbits[base + w];
            }
        }
        __syncwarp();
    }
    if (wib == 0 && lane == 0)
        for (int t = 0; t < nadd; ++t) rf += add[t].rb ? (unsigned long long)(add[t].re[r] - add[t].rb[r]) : 1ull;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int w = lane + 32 * u;
        if (w < kBmWords && reg[u]) atomicOr(&S.pm[w].y, reg[u]);
    }
    __syncthreads();
    // ---- number the columns: thread t takes words 2t and 2t + 1 (in order)
    static_assert(2 * kCtaWarps * 32 >= kBmWords, "two words per thread cover the map");
    int total = 0;
    {
        const int w0 = 2 * tid, w1 = 2 * tid + 1;
        const int c0 = w0 < nw ? __popc(S.pm[w0].y) : 0;
        const int c1 = w1 < nw ? __popc(S.pm[w1].y) : 0;
        const int ex = cta_excl_scan(c0 + c1, tid, S.wcnt, &total);
        if (w0 < nw) S.pm[w0].x = (unsigned)ex;
        if (w1 < nw) S.pm[w1].x = (unsigned)(ex + c0);
    }
    if (total > kCtaCap) {
        // more entries than slots: the first warp computes the row alone
        // (with its own counts; this pass's are dropped), once every thread
        // is done with the map
        __syncthreads();
        if (wib == 0)
            product_row<false, false, true, kBmWords>(P, add, *reinterpret_cast<ProdSmem<false, kBmWords>*>(&S), st,
                                                      r, lane);
        __syncthreads();
        return;
    }
    st.fma += rf;
    if (wib == 0) {
        const long long b = arena_take(st.arena, (unsigned long long)((total + 3) & ~3), P.arena, P.ctl, P.pool_val,
                                       lane);
        if (lane == 0) S.base = b;
    }
    // the column list: each thread fills the two words whose prefixes it wrote
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int w = 2 * tid + k;
        if (w < nw) {
            unsigned bits = S.pm[w].y;
            int idx = (int)S.pm[w].x;
            while (bits) {
                S.colbuf[idx++] = (unsigned short)(w * 32 + __ffs(bits) - 1);
                bits &= bits - 1u;
            }
        }
    }
    for (int i = tid; i < total; i += kT) S.acc[i] = 0.0;
    __syncthreads();
    const long long base = S.base;
    if (base < 0) {
        if (tid == 0) P.out_rb[r] = P.out_re[r] = 0;
        return;
    }
    // ---- numeric pass: the addends, t ascending
    for (int t = 0; t < nadd; ++t) {
        const AddTerm& T = add[t];
        if (!T.rb) {
            if (tid == 0) {
                const int i = slot_lookup(M, r - lo);
                S.acc[i] = __fma_rn(T.alpha, 1.0, S.acc[i]);
            }
        } else {
            for (int q = T.rb[r] + tid; q < T.re[r]; q += kT) {
                const int i = slot_lookup(M, T.col[q] - lo);
                S.acc[i] = __fma_rn(T.alpha, T.val[q], S.acc[i]);
            }
        }
        __syncthreads();
    }
    // ---- the B rows, k ascending, a block barrier after each
    const int* __restrict__ bcol = P.B.col;
    const double* __restrict__ bval = P.B.val;
    for (int seg = pa0; seg < pa1; seg += 32) {
        const int cnt = min(32, pa1 - seg);
        __syncthreads();  // every thread is done with the last segment (its last rows may be empty)
        if (wib == 0 && lane < cnt) {
            const int k = P.A.col[seg + lane];
            const int b = P.B.rb[k];
            S.kb[0][lane] = b;
            S.kl[0][lane] = P.B.re[k] - b;
            S.ka[lane] = P.A.val[seg + lane];
        }
        __syncthreads();
        for (int kk = 0; kk < cnt; ++kk) {
            const int len = S.kl[0][kk];
            if (len == 0) continue;
            const double a = S.ka[kk];
            const int* __restrict__ rc = bcol + S.kb[0][kk];
            const double* __restrict__ rv = bval + S.kb[0][kk];
            int off = tid;
            for (; off + 3 * kT < len; off += 4 * kT) {
                int j[4];
                double v[4], x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    j[u] = rc[off + u * kT];
                    v[u] = rv[off + u * kT];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) j[u] = slot_lookup(M, j[u] - lo);
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = S.acc[j[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) S.acc[j[u]] = __fma_rn(a, v[u], x[u]);
            }
            for (; off < len; off += kT) {
                const int j = slot_lookup(M, rc[off] - lo);
                S.acc[j] = __fma_rn(a, rv[off], S.acc[j]);
            }
            __syncthreads();
        }
    }
    // ---- write-back: warp w takes slots [w Q, (w + 1) Q) in column order
    const int Q = ((total + kCtaWarps - 1) / kCtaWarps + 31) & ~31;
    const int s0 = min(total, wib * Q), s1 = min(total, s0 + Q);
    int mine = 0;
    for (int i0 = s0; i0 < s1; i0 += 32) {
        const int i = i0 + lane;
        mine += __popc(__ballot_sync(kFull, i < s1 && mag_bits(S.acc[i]) != 0ull));
    }
    int written = 0;
    const int before = cta_excl_scan(lane == 0 ? mine : 0, tid, S.wcnt, &written);
    const long long wbase = base + __shfl_sync(kFull, before, 0);
    const bool filt = P.filtering != 0;
    const unsigned long long r_eps = (unsigned long long)__double_as_longlong(P.eps_g);
    int w_off = 0;
    for (int i0 = s0; i0 < s1; i0 += 32) {
        const int i = i0 + lane;
        double x = 0.0;
        int c = 0;
        if (i < s1) {
            x = S.acc[i];
            c = lo + (int)S.colbuf[i];
        }
        const unsigned long long xb = mag_bits(x);
        const bool nz = i < s1 && xb != 0ull;
        const unsigned m = __ballot_sync(kFull, nz);
        const bool cand = nz && filt && xb <= r_eps;
        if (nz) {
            const long long pos = wbase + w_off + __popc(m & lanemask_lt());
            P.pool_col[pos] = c;
            P.pool_val[pos] = x;
            st.absmax = xb > st.absmax ? xb : st.absmax;
            if (cand) {
                exact_add(P.words + c, (size_t)P.n, P.sticky + c, xb, P.e_lsb);
                ++st.cand;
            }
        }
        if (P.cand_col)
            cand_push(st.carena, cand, c, xb, P.cand_col, P.cand_x, &P.ctl->cand_cnt[0], P.cand_cap, P.cand_chunk,
                      &P.ctl->cand_over, lane);
        w_off += __popc(m);
    }
    // the row's unused reserved slots read as exact zeros (never candidates)
    const long long rend = base + ((total + 3) & ~3);
    for (long long q = base + written + tid; q < rend; q += kT) P.pool_val[q] = 0.0;
    if (tid == 0) {
        P.out_rb[r] = (int)base;
        P.out_re[r] = (int)(base + written);
        st.written += (unsigned long long)written;
    }
    __syncthreads();  // the map and the accumulator are free for the next row
}

__global__ void __launch_bounds__(kCtaWarps * 32, 7) k_product_cta(ProductArgs P) {
    if (P.skip_unless && __ldcg(P.skip_unless) == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AddTerm* add = reinterpret_cast<AddTerm*>(smem_raw);
    CtaSmem& S = *reinterpret_cast<CtaSmem*>(smem_raw + sizeof(AddTerm) * kMaxAdd);
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    for (int t = tid; t < P.nadd; t += blockDim.x) add[t] = P.add[t];
    __syncthreads();
    RowState st;
    for (int r = blockIdx.x; r < P.n; r += gridDim.x) cta_row(P, add, S, st, r, tid);
    if (wib == 0) arena_close(st.arena, P.pool_val, lane);
    if (P.cand_col) cand_close(st.carena, P.cand_x, lane);
    st.cand = (unsigned long long)warp_sum((int)st.cand);
    st.absmax = warp_max_u64(st.absmax);
    for (int o = 16; o; o >>= 1) st.fma += __shfl_xor_sync(kFull, st.fma, o);
    st.written = __shfl_sync(kFull, st.written, 0);
    st.span = warp_max(st.span);
    if (lane == 0) {
        if (st.fma) atomicAdd(&P.ctl->fma_total, st.fma);
        if (P.stat) {
            if (st.span > 0) atomicMax(&P.stat->span_max, (unsigned)st.span);
            if (st.fma) atomicAdd(&P.stat->fma, st.fma);
            if (st.written) atomicAdd(&P.stat->nnz_pre, st.written);
            if (st.cand) atomicAdd(&P.stat->ncand, st.cand);
        }
        if (P.absmax_slot && st.absmax) atomicMax(&P.absmax_slot->absmax, st.absmax);
    }
}

// ---------------------------------------------------------------- k_reuse_pass1
// A baby step Z-hat_(k) = filter(Z Z-hat_(k-1)) while no earlier step has
// dropped an entry: Z-hat_(k-1) is then the power Z^(k-1) of the norm phase,
// so the product is that phase's Z^k, entry for entry, and its rows are kept
// as they are.  What the product's write-back would have done remains:
// Algorithm 1's first pass (exact column sums and the candidate list of the
// entries 0 < |x| <= eps_g) and the step statistics.  The power's pool range
// is [mark[k-1], mark[k]).  Does nothing once an entry has been dropped (the
// product kernel then runs instead).

__global__ void __launch_bounds__(256) k_reuse_pass1(ReuseArgs R) {
    if (__ldcg(&R.ctl->dropped) != 0) return;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned long long eb = (unsigned long long)__double_as_longlong(R.eps_g);
    unsigned long long nnz = 0ull, cand = 0ull;
    CandArena ca;
    for (int r = gw; r < R.n; r += nwarps) {
        const int s = R.rb[r], e = R.re[r];
        for (int q0 = s; q0 < e; q0 += 32) {
            const int q = q0 + lane;
            const bool in = q < e;
            const unsigned long long xb = in ? mag_bits(R.val[q]) : 0ull;
            const int c = in ? R.col[q] : 0;
            const bool is_cand = xb != 0ull && xb <= eb;
            if (is_cand) {
                exact_add_checked(R.words, R.sticky, c, R.n, xb, R.e_lsb, R.ctl);
                ++cand;
            }
            if (xb) ++nnz;
            cand_push(ca, is_cand, c, xb, R.cand_col, R.cand_x, &R.ctl->cand_cnt[0], R.cand_cap, R.cand_chunk,
                      &R.ctl->cand_over, lane);
        }
    }
    cand_close(ca, R.cand_x, lane);
    // the counts go to the step's record once per block: one atomic per warp
    // on the same two words queued behind one another at the launch's end
    __shared__ unsigned long long blk_nnz, blk_cand;
    if (threadIdx.x == 0) {
        blk_nnz = 0ull;
        blk_cand = 0ull;
    }
    __syncthreads();
    nnz = (unsigned long long)warp_sum((int)nnz);
    cand = (unsigned long long)warp_sum((int)cand);
    if (lane == 0) {
        if (nnz) atomicAdd(&blk_nnz, nnz);
        if (cand) atomicAdd(&blk_cand, cand);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_nnz) atomicAdd(&R.stat->nnz_pre, blk_nnz);
        if (blk_cand) atomicAdd(&R.stat->ncand, blk_cand);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        R.stat->fma = R.fma;
        R.stat->pool_start = R.ctl->mark[R.k - 1];
        R.stat->pool_end = R.ctl->mark[R.k];
    }
}

// ---------------------------------------------------------------- k_reuse_copy_batch
// Batched baby step k for the instances that have dropped no entry so far:
// their Z-hat_(k-1) is the norm phase's Z^(k-1), so the product Z Z-hat_(k-1)
// is that phase's Z^k, entry for entry (the same terms in the same order).
// Each such row is copied from the norm phase's pool (P.power) into the
// step's own pool range, and what the product's write-back does besides is
// done on the way: Algorithm 1's first pass (column sums and candidate list
// of the entries 0 < |x| <= eps_g) and the row statistics, with the
// product's multiply-add count (the B row lengths summed over row r of A).
// The product kernel skips these rows.
__global__ void __launch_bounds__(256) k_reuse_copy_batch(ProductArgs P) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    Arena arena;
    CandArena carena;
    for (int r = gw; r < P.n; r += nwarps) {
        const int i = P.inst[r];
        const BatchStep bs = P.bstep[i];
        if (!bs.reuse || __ldcg(P.inst_dropped + i) != 0) continue;
        unsigned long long fma = 0ull;
        for (int p = P.A.rb[r] + lane; p < P.A.re[r]; p += 32) {
            const int k = P.A.col[p];
            fma += (unsigned long long)(P.B.re[k] - P.B.rb[k]);
        }
        const int s = P.power.rb[r], len = P.power.re[r] - s;
        if (len <= 0) {
            if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
            row_stats_batch(P, i, fma, 0ull, 0, 0ull, lane);
            continue;
        }
        const unsigned long long span = ((unsigned long long)len + 3ull) & ~3ull;
        const long long base = arena_take(arena, span, P.arena, P.ctl, P.pool_val, lane);
        if (base < 0) {
            if (lane == 0) P.out_rb[r] = P.out_re[r] = 0;
            continue;
        }
        const bool filt = bs.eps_g > 0.0;
        const unsigned long long eb = (unsigned long long)__double_as_longlong(bs.eps_g);
        unsigned long long cand = 0ull;
        for (int q0 = 0; q0 < len; q0 += 32) {
            const int q = q0 + lane;
            const bool in = q < len;
            const double x = in ? P.power.val[s + q] : 0.0;
            const int c = in ? P.power.col[s + q] : 0;
            const unsigned long long xb = mag_bits(x);
            const bool is_cand = filt && xb != 0ull && xb <= eb;
            if (in) {
                P.pool_col[base + q] = c;
                P.pool_val[base + q] = x;
            }
            if (is_cand) {
                exact_add(P.words + c, (size_t)P.n, P.sticky + c, xb, bs.e_lsb);
                ++cand;
            }
            if (P.cand_col)
                cand_push(carena, is_cand, c, xb, P.cand_col, P.cand_x, &P.ctl->cand_cnt[0], P.cand_cap, P.cand_chunk,
                          &P.ctl->cand_over, lane);
        }
        for (long long q = base + len + lane; q < base + (long long)span; q += 32) P.pool_val[q] = 0.0;
        if (lane == 0) {
            P.out_rb[r] = (int)base;
            P.out_re[r] = (int)(base + len);
        }
        row_stats_batch(P, i, fma, cand, len, 0ull, lane);
    }
    arena_close(arena, P.pool_val, lane);
    if (P.cand_col) cand_close(carena, P.cand_x, lane);
}

// ---------------------------------------------------------------- k_alg1
// Passes 2, 3, ... of Algorithm 1 and the compaction, as one cooperative
// launch.  On entry the column sums of pass 1 (entries |x| <= eps_g) are in
// the chunk words and both cslot words are 0.  Every block evaluates the same
// scalar recurrence from the same global values, so all blocks take the same
// decisions without further communication.
constexpr int kAlg1Threads = 1024;  // one block per SM: few grid-barrier arrivals
constexpr int kAlg1BlocksPerSm = 1;

__global__ void __launch_bounds__(kAlg1Threads, kAlg1BlocksPerSm) k_alg1(Alg1Args A) {
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
    // the step's pool range; the counter runs past the capacity on overflow
    const unsigned long long p0 = min(__ldcg(&A.stat->pool_start), A.ctl->pool_cap);
    const unsigned long long pe = __ldcg(&A.stat->pool_end);
    const unsigned long long p1 = min(pe ? pe : __ldcg(&A.ctl->pool_used), A.ctl->pool_cap);
    // a phase whose pool overflowed is discarded: its pool range is not
    // complete, so there is nothing to filter (every block reads the same
    // status, set by an earlier launch)
    if (__ldcg(&A.ctl->status) & kDevPoolFull) return;
    bool over = __ldcg(&A.ctl->cand_over) != 0 || A.cand_col == nullptr;
    const unsigned long long ccap = A.ctl->cand_cap;
    const unsigned cchunk = A.ctl->cand_chunk;
    const unsigned long long split = far_split(A.eps_g, A.far_shift);
    if (__ldcg(&A.stat->ncand) == 0ull) {
        // the product left no entry with |x| <= eps_g: the first pass finds an
        // empty candidate matrix (c = 0), nothing is dropped
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            A.stat->eps_f = eps_f;
            A.stat->iters = 1;
            A.stat->dropped = 0.0;
            A.stat->nnz_post = A.stat->nnz_pre;
        }
        return;
    }
    bool dirty = false;  // the column sums were left in place by the last finalize
    for (;;) {
        // finalize: round each column sum, take the max.  The sums are kept
        // for an incremental (list) pass and cleared for a full pool scan.
        unsigned long long local = 0ull;
        dirty = !over;
        for (int j = gt; j < A.n; j += nthreads) {
            double s = chunk_round(A.words + j, n, A.sticky + j, A.e_lsb, over);
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
                if (blockIdx.x == 0) {
                    A.ctl->cslot[(it + 1) & 1] = 0ull;
                    if (it == 0) A.ctl->cand_cnt[1] = 0ull;  // the first rescan's output list
                }
            }
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) {
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
        if (!over) {
            // The first rescan reads the product's candidates (list 0) and
            // writes those still at or below eps_f to list 1: the near ones
            // (above eps_g / 2^far_shift, default 2^6) to its front half, the
            // far ones to its back half.  The far ones cannot leave while
            // eps_f stays above that bound; later rescans read the near
            // ones in place, subtracting and clearing (|x| = 0: a hole) those
            // that leave, and read the far half (in place) only once eps_f
            // falls below the bound.
            const bool first = it == 1;
            const unsigned long long half = ccap / 2;
            int* fcol = A.cand_col + ccap + half;
            unsigned long long* fx = A.cand_x + ccap + half;
            const unsigned long long nt = (unsigned long long)nthreads;
            if (!first) {
                const unsigned long long cnt = min(__ldcg(&A.ctl->cand_cnt[1]), half);
                const int* ic = A.cand_col + ccap;
                unsigned long long* ix = A.cand_x + ccap;
                for (unsigned long long q0 = (unsigned long long)gt; q0 < cnt; q0 += 4ull * nt) {
                    unsigned long long xb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const unsigned long long q = q0 + (unsigned long long)u * nt;
                        xb[u] = q < cnt ? __ldcg(ix + q) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (xb[u] > fb) {  // 0 (a hole) never
                            const unsigned long long q = q0 + (unsigned long long)u * nt;
                            exact_sub_checked(A.words, A.sticky, __ldcg(ic + q), A.n, xb[u], A.e_lsb, A.ctl);
                            ix[q] = 0ull;
                        }
                    }
                }
            }
            const unsigned long long cnt = first ? min(__ldcg(&A.ctl->cand_cnt[0]), ccap) : 0ull;
            const int* ic = A.cand_col;
            const unsigned long long* ix = A.cand_x;
            const int bo = 1;
            CandArena ca, cf;
            // four candidates per thread at a time, all loads issued first
            for (unsigned long long q0 = (unsigned long long)(gt & ~31); q0 < cnt; q0 += 4ull * nt) {
                unsigned long long xb[4];
                int col[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned long long q = q0 + (unsigned long long)u * nt + (unsigned long long)lane;
                    xb[u] = q < cnt ? __ldcg(ix + q) : 0ull;
                    col[u] = q < cnt ? __ldcg(ic + q) : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool keep = xb[u] != 0ull && xb[u] <= fb;
                    // an entry that leaves the list leaves the column sums
                    if (xb[u] != 0ull && !keep)
                        exact_sub_checked(A.words, A.sticky, col[u], A.n, xb[u], A.e_lsb, A.ctl);
                    const bool far = first && keep && xb[u] <= split;
                    cand_push(ca, keep && !far, col[u], xb[u], A.cand_col + (size_t)bo * ccap,
                              A.cand_x + (size_t)bo * ccap, &A.ctl->cand_cnt[bo], half, cchunk, &A.ctl->cand_over,
                              lane);
                    if (first)
                        cand_push(cf, far, col[u], xb[u], fcol, fx, &A.ctl->cand_far, half, cchunk, &A.ctl->cand_over,
                                  lane);
                }
            }
            cand_close(ca, A.cand_x + (size_t)bo * ccap, lane);
            if (first) cand_close(cf, fx, lane);
            if (!first && fb < split) {
                // eps_f is below the far candidates' bound: those above it leave
                const unsigned long long nf = min(__ldcg(&A.ctl->cand_far), half);
                for (unsigned long long q = (unsigned long long)gt; q < nf; q += nt) {
                    const unsigned long long xb = __ldcg(fx + q);
                    if (xb > fb) {
                        exact_sub_checked(A.words, A.sticky, __ldcg(fcol + q), A.n, xb, A.e_lsb, A.ctl);
                        fx[q] = 0ull;
                    }
                }
            }
            if (!grid_barrier(A.ctl, A.budget_ns)) {
                alive = false;
                break;
            }
            // a list that overflowed is incomplete: scan the pool from now on
            // (the flag is read after the barrier, so every block agrees)
            over = __ldcg(&A.ctl->cand_over) != 0;
            continue;
        }
        // accumulate the entries still below the threshold: one streaming
        // pass over the step's pool range (its gaps hold exact zeros)
        for (unsigned long long q0 = p0 + (unsigned long long)gt; q0 < p1; q0 += 4ull * nthreads) {
            unsigned long long xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned long long q = q0 + (unsigned long long)u * nthreads;
                xb[u] = q < p1 ? mag_bits(__ldcg(A.val + q)) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (xb[u] != 0ull && xb[u] <= fb) {
                    const int col = A.col[q0 + (unsigned long long)u * nthreads];
                    exact_add_checked(A.words, A.sticky, col, A.n, xb[u], A.e_lsb, A.ctl);
                }
            }
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) {
            alive = false;
            break;
        }
    }
    if (!alive) return;
    if (gt == 0) {  // the lists are empty for the next step
        A.ctl->cand_cnt[0] = A.ctl->cand_cnt[1] = A.ctl->cand_far = 0ull;
        A.ctl->cand_over = 0;
    }
    if (dirty) clear_sums(A.words, A.sticky, A.n, gt, nthreads);  // zero for the next step
    if (!sum_is_exact(c, A.e_lsb)) {
        // every candidate is tiny against eps_g and c may have lost bits
        // below the LSB: count the final candidates again with the LSB of
        // the largest one.  cslot[it & 1] is 0 (cleared by the last
        // finalize), cslot[(it - 1) & 1] holds the c every block has read
        // once all blocks reach the first barrier.
        const unsigned long long fb = (unsigned long long)__double_as_longlong(eps_f);
        const int sx = it & 1, sc = (it - 1) & 1;
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        if (gt == 0) A.ctl->cslot[sc] = 0ull;
        unsigned long long mx = 0ull;
        for (unsigned long long q = p0 + (unsigned long long)gt; q < p1; q += (unsigned long long)nthreads) {
            const unsigned long long xb = mag_bits(__ldcg(A.val + q));
            if (xb <= fb && xb > mx) mx = xb;
        }
        mx = warp_max_u64(mx);
        if (lane == 0 && mx) atomicMax(&A.ctl->cslot[sx], mx);
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        const int lsb = lsb_for_bound(__ldcg(&A.ctl->cslot[sx]));
        for (unsigned long long q = p0 + (unsigned long long)gt; q < p1; q += (unsigned long long)nthreads) {
            const unsigned long long xb = mag_bits(__ldcg(A.val + q));
            if (xb != 0ull && xb <= fb) exact_add_checked(A.words, A.sticky, A.col[q], A.n, xb, lsb, A.ctl);
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        unsigned long long local = 0ull;
        for (int j = gt; j < A.n; j += nthreads) {
            const double s = chunk_round(A.words + j, n, A.sticky + j, lsb, true);
            const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
            local = sb > local ? sb : local;
        }
        local = warp_max_u64(local);
        if (lane == 0 && local) atomicMax(&A.ctl->cslot[sc], local);
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        c = __longlong_as_double((long long)__ldcg(&A.ctl->cslot[sc]));
    }
    if (!(c > 0.0)) {
        // nothing was dropped: the matrix stays as the product wrote it
        if (gt == 0) {
            A.stat->eps_f = eps_f;
            A.stat->iters = it;
            A.stat->dropped = c;
            A.stat->nnz_post = __ldcg(&A.stat->nnz_pre);
        }
        return;
    }

    if (gt == 0) A.ctl->dropped = 1;
    // compaction: keep |x| > eps_f, in place, column order preserved
    const unsigned long long fb = (unsigned long long)__double_as_longlong(eps_f);
    unsigned long long kept = 0ull;
    for (int r = gw; r < A.n; r += nwarps) {
        const int s = A.rb[r], e = A.re[r];
        const int w = compact_row(A.col, A.val, s, e, fb, lane);
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

// ---------------------------------------------------------------- k_alg1_batch
// Algorithm 1 for every filtered instance of a batched step, one cooperative
// launch.  The instances run the recurrence of k_alg1 side by side: column
// sums belong to the instance owning the column, each instance has its own
// c, eps_f and pass count, and a pass streams the step's whole pool range
// once for all instances still iterating.  Every block keeps the per-instance
// state in shared memory and updates it from the same global column-sum
// maxima, so all blocks take the same decisions.
constexpr int kMaxBatch = 1024;  // instances of one batched launch

__global__ void __launch_bounds__(kAlg1Threads, kAlg1BlocksPerSm) k_alg1_batch(Alg1BatchArgs A) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const size_t n = (size_t)A.n;
    __shared__ double s_eps[kMaxBatch];  // eps_f
    __shared__ double s_c[kMaxBatch];    // last column-sum maximum c
    __shared__ int s_it[kMaxBatch];
    // 0 iterating, 1 finished, 2 not filtered here, 3 finished without
    // candidates, 4 finished with a c to count again (see below)
    __shared__ unsigned char s_state[kMaxBatch];
    __shared__ int s_left;
    if (__ldcg(&A.ctl->status) & kDevPoolFull) return;  // discarded phase (same for all blocks)
    if (threadIdx.x == 0) s_left = 0;
    __syncthreads();
    int left = 0;
    for (int i = threadIdx.x; i < A.ninst; i += blockDim.x) {
        const BatchStep bs = A.bstep[i];
        const bool filt = (bs.mode == kBatchProduct || bs.mode == kBatchAddOnly) && bs.eps_g > 0.0;
        s_eps[i] = bs.eps_g;
        s_c[i] = 0.0;
        s_it[i] = 0;
        // an instance without candidates finds c = 0 in its first pass
        const bool empty = filt && __ldcg(&A.stat_tab[i].ncand) == 0ull;
        s_state[i] = !filt ? 2 : (empty ? 3 : 0);
        if (empty) s_it[i] = 1;
        left += (filt && !empty) ? 1 : 0;
    }
    atomicAdd(&s_left, left);
    __syncthreads();
    const unsigned long long cap = A.ctl->pool_cap;
    const unsigned long long p0 = min(__ldcg(A.pool_start), cap);
    const unsigned long long p1 = min(__ldcg(&A.ctl->pool_used), cap);
    bool over = __ldcg(&A.ctl->cand_over) != 0 || A.cand_col == nullptr;
    const unsigned long long ccap = A.ctl->cand_cap;
    const unsigned cchunk = A.ctl->cand_chunk;
    bool alive = true;
    bool dirty = false;  // some column sums were left in place
    int pass = 0;
    while (s_left > 0) {
        // finalize the column sums of the iterating instances (kept for an
        // incremental list pass, cleared for a full pool scan)
        if (!over) dirty = true;
        for (int j = gt; j < A.n; j += nthreads) {
            const int i = A.inst[j];
            if (s_state[i] != 0) continue;
            double v = chunk_round(A.words + j, n, A.sticky + j, A.bstep[i].e_lsb, over);
            unsigned long long vb = (unsigned long long)__double_as_longlong(v);
            if (vb) atomicMax(&A.cslot[2 * i + (pass & 1)], vb);
        }
        if (blockIdx.x == 0) {
            for (int i = threadIdx.x; i < A.ninst; i += blockDim.x) A.cslot[2 * i + ((pass + 1) & 1)] = 0ull;
            if (threadIdx.x == 0 && pass == 0) A.ctl->cand_cnt[1] = 0ull;  // the first rescan's output list
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) {
            alive = false;
            break;
        }
        // the recurrence of every iterating instance (identical in all blocks)
        __syncthreads();
        if (threadIdx.x == 0) s_left = 0;
        __syncthreads();
        left = 0;
        for (int i = threadIdx.x; i < A.ninst; i += blockDim.x) {
            if (s_state[i] != 0) continue;
            const BatchStep bs = A.bstep[i];
            const double c = __longlong_as_double((long long)__ldcg(&A.cslot[2 * i + (pass & 1)]));
            const double m = c / s_eps[i];
            const int it = ++s_it[i];
            s_c[i] = c;
            if (!(c > bs.bound)) {
                s_state[i] = 1;
            } else if (it >= bs.maxit) {
                s_state[i] = 1;
                if (blockIdx.x == 0) atomicOr(&A.ctl->status, kDevNotConv);
            } else {
                s_eps[i] = bs.eps_g / m;
                ++left;
            }
        }
        atomicAdd(&s_left, left);
        __syncthreads();
        if (s_left == 0) break;
        if (!over) {
            // the first rescan reads the product's candidates (list 0) into
            // list 1, each instance's candidates at or below its eps_g /
            // 2^far_shift in its back half; later rescans read the front half
            // in place (as in k_alg1), clearing the entries that leave and
            // those of instances that have finished
            const bool first = pass == 0;
            const unsigned long long half = ccap / 2;
            int* fcol = A.cand_col + ccap + half;
            unsigned long long* fx = A.cand_x + ccap + half;
            const unsigned long long nt = (unsigned long long)nthreads;
            if (!first) {
                const unsigned long long cnt = min(__ldcg(&A.ctl->cand_cnt[1]), half);
                const int* ic = A.cand_col + ccap;
                unsigned long long* ix = A.cand_x + ccap;
                for (unsigned long long q0 = (unsigned long long)gt; q0 < cnt; q0 += 4ull * nt) {
                    unsigned long long xb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const unsigned long long q = q0 + (unsigned long long)u * nt;
                        xb[u] = q < cnt ? __ldcg(ix + q) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (!xb[u]) continue;
                        const unsigned long long q = q0 + (unsigned long long)u * nt;
                        const int cq = __ldcg(ic + q);
                        if ((unsigned)cq >= (unsigned)A.n) {
                            atomicOr(&A.ctl->status, kDevInternal);
                            continue;
                        }
                        const int i = A.inst[cq];
                        if (s_state[i] != 0) {
                            ix[q] = 0ull;
                        } else if (xb[u] > (unsigned long long)__double_as_longlong(s_eps[i])) {
                            // an entry that leaves the list leaves the column sums
                            exact_sub(A.words + cq, n, A.sticky + cq, xb[u], A.bstep[i].e_lsb);
                            ix[q] = 0ull;
                        }
                    }
                }
            }
            const unsigned long long cnt = first ? min(__ldcg(&A.ctl->cand_cnt[0]), ccap) : 0ull;
            const int* ic = A.cand_col;
            const unsigned long long* ix = A.cand_x;
            const int bo = 1;
            CandArena ca, cf;
            // four candidates per thread at a time, all loads issued first
            for (unsigned long long q0 = (unsigned long long)(gt & ~31); q0 < cnt; q0 += 4ull * nt) {
                unsigned long long xb[4];
                int col[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned long long q = q0 + (unsigned long long)u * nt + (unsigned long long)lane;
                    xb[u] = q < cnt ? __ldcg(ix + q) : 0ull;
                    col[u] = q < cnt ? __ldcg(ic + q) : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    bool keep = false, far = false;
                    if (xb[u]) {
                        if ((unsigned)col[u] >= (unsigned)A.n) {
                            atomicOr(&A.ctl->status, kDevInternal);
                        } else {
                            const int i = A.inst[col[u]];
                            if (s_state[i] == 0) {
                                keep = xb[u] <= (unsigned long long)__double_as_longlong(s_eps[i]);
                                // an entry that leaves the list leaves the column sums
                                if (!keep) exact_sub(A.words + col[u], n, A.sticky + col[u], xb[u], A.bstep[i].e_lsb);
                                far = first && keep && xb[u] <= far_split(A.bstep[i].eps_g, A.far_shift);
                            }
                        }
                    }
                    cand_push(ca, keep && !far, col[u], xb[u], A.cand_col + (size_t)bo * ccap,
                              A.cand_x + (size_t)bo * ccap, &A.ctl->cand_cnt[bo], half, cchunk, &A.ctl->cand_over,
                              lane);
                    if (first)
                        cand_push(cf, far, col[u], xb[u], fcol, fx, &A.ctl->cand_far, half, cchunk, &A.ctl->cand_over,
                                  lane);
                }
            }
            cand_close(ca, A.cand_x + (size_t)bo * ccap, lane);
            if (first) cand_close(cf, fx, lane);
            // an instance whose eps_f fell below its far bound: its far
            // candidates above eps_f leave, in place (the same test in all blocks)
            int below = 0;
            if (!first)
                for (int i = threadIdx.x; i < A.ninst; i += blockDim.x)
                    if (s_state[i] == 0 &&
                        (unsigned long long)__double_as_longlong(s_eps[i]) < far_split(A.bstep[i].eps_g, A.far_shift))
                        below = 1;
            if (__syncthreads_or(below)) {
                const unsigned long long nf = min(__ldcg(&A.ctl->cand_far), half);
                for (unsigned long long q = (unsigned long long)gt; q < nf; q += nt) {
                    const unsigned long long xq = __ldcg(fx + q);
                    if (xq == 0ull) continue;
                    const int cq = __ldcg(fcol + q);
                    if ((unsigned)cq >= (unsigned)A.n) continue;
                    const int i = A.inst[cq];
                    if (s_state[i] == 0 && xq > (unsigned long long)__double_as_longlong(s_eps[i])) {
                        exact_sub(A.words + cq, n, A.sticky + cq, xq, A.bstep[i].e_lsb);
                        fx[q] = 0ull;
                    }
                }
            }
            if (!grid_barrier(A.ctl, A.budget_ns)) {
                alive = false;
                break;
            }
            over = __ldcg(&A.ctl->cand_over) != 0;  // read after the barrier: every block agrees
            ++pass;
            continue;
        }
        // accumulate the entries still below their instance's threshold
        for (unsigned long long q0 = p0 + (unsigned long long)gt; q0 < p1; q0 += 4ull * nthreads) {
            unsigned long long xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned long long q = q0 + (unsigned long long)u * nthreads;
                xb[u] = q < p1 ? mag_bits(__ldcg(A.val + q)) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (xb[u] == 0ull) continue;
                const int col = A.col[q0 + (unsigned long long)u * nthreads];
                if ((unsigned)col >= (unsigned)A.n) {
                    atomicOr(&A.ctl->status, kDevInternal);
                    continue;
                }
                const int i = A.inst[col];
                if (s_state[i] != 0) continue;
                if (xb[u] <= (unsigned long long)__double_as_longlong(s_eps[i]))
                    exact_add(A.words + col, n, A.sticky + col, xb[u], A.bstep[i].e_lsb);
            }
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) {
            alive = false;
            break;
        }
        ++pass;
    }
    if (!alive) return;
    if (gt == 0) {  // the lists are empty for the next step
        A.ctl->cand_cnt[0] = A.ctl->cand_cnt[1] = A.ctl->cand_far = 0ull;
        A.ctl->cand_over = 0;
    }
    if (dirty) clear_sums(A.words, A.sticky, A.n, gt, nthreads);  // zero for the next step
    // an instance whose candidates are all tiny against its eps_g may have
    // lost bits of c below the LSB: its final candidates are counted again
    // with the LSB of its largest one (the same instances in every block)
    int nfix = 0;
    for (int i = threadIdx.x; i < A.ninst; i += blockDim.x)
        if (s_state[i] == 1 && !sum_is_exact(s_c[i], A.bstep[i].e_lsb)) {
            s_state[i] = 4;
            ++nfix;
        }
    if (__syncthreads_or(nfix)) {
        __shared__ int s_lsb[kMaxBatch];
        // every block has read the maxima: slot 2i takes the largest
        // candidate, slot 2i + 1 the new c
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        if (blockIdx.x == 0)
            for (int i = threadIdx.x; i < A.ninst; i += blockDim.x)
                if (s_state[i] == 4) A.cslot[2 * i] = A.cslot[2 * i + 1] = 0ull;
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        for (unsigned long long q = p0 + (unsigned long long)gt; q < p1; q += (unsigned long long)nthreads) {
            const unsigned long long xb = mag_bits(__ldcg(A.val + q));
            if (xb == 0ull) continue;
            const int col = A.col[q];
            if ((unsigned)col >= (unsigned)A.n) continue;
            const int i = A.inst[col];
            if (s_state[i] == 4 && xb <= (unsigned long long)__double_as_longlong(s_eps[i]))
                atomicMax(&A.cslot[2 * i], xb);
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        for (int i = threadIdx.x; i < A.ninst; i += blockDim.x)
            if (s_state[i] == 4) s_lsb[i] = lsb_for_bound(__ldcg(&A.cslot[2 * i]));
        __syncthreads();
        for (unsigned long long q = p0 + (unsigned long long)gt; q < p1; q += (unsigned long long)nthreads) {
            const unsigned long long xb = mag_bits(__ldcg(A.val + q));
            if (xb == 0ull) continue;
            const int col = A.col[q];
            if ((unsigned)col >= (unsigned)A.n) continue;
            const int i = A.inst[col];
            if (s_state[i] == 4 && xb <= (unsigned long long)__double_as_longlong(s_eps[i]))
                exact_add(A.words + col, n, A.sticky + col, xb, s_lsb[i]);
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        for (int j = gt; j < A.n; j += nthreads) {
            const int i = A.inst[j];
            if (s_state[i] != 4) continue;
            const double v = chunk_round(A.words + j, n, A.sticky + j, s_lsb[i], true);
            const unsigned long long vb = (unsigned long long)__double_as_longlong(v);
            if (vb) atomicMax(&A.cslot[2 * i + 1], vb);
        }
        if (!grid_barrier(A.ctl, A.budget_ns)) return;
        for (int i = threadIdx.x; i < A.ninst; i += blockDim.x)
            if (s_state[i] == 4) {
                s_c[i] = __longlong_as_double((long long)__ldcg(&A.cslot[2 * i + 1]));
                s_state[i] = 1;
            }
        __syncthreads();
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < A.ninst; i += blockDim.x) {
            if (s_state[i] == 2) continue;
            A.stat_tab[i].eps_f = s_eps[i];
            A.stat_tab[i].iters = s_it[i];
            A.stat_tab[i].dropped = s_c[i];
            if (!(s_c[i] > 0.0)) A.stat_tab[i].nnz_post = __ldcg(&A.stat_tab[i].nnz_pre);  // nothing dropped
            else if (A.inst_dropped) A.inst_dropped[i] = 1;
        }
    // compaction of the instances that dropped entries: keep |x| > eps_f of
    // the row's instance, in place
    for (int r = gw; r < A.n; r += nwarps) {
        const int i = A.inst[r];
        if (s_state[i] != 1 || !(s_c[i] > 0.0)) continue;
        const unsigned long long fb = (unsigned long long)__double_as_longlong(s_eps[i]);
        const int s = A.rb[r], e = A.re[r];
        const int w = compact_row(A.col, A.val, s, e, fb, lane);
        if (lane == 0) {
            A.re[r] = w;
            if (w > s) atomicAdd(&A.stat_tab[i].nnz_post, (unsigned long long)(w - s));
        }
    }
}

// ---------------------------------------------------------------- k_norms
// Exact ||M||_1 of up to kMaxNorms matrices whose max |x| is already in
// slots[i].absmax: accumulate every |x| into per-column fixed-point sums,
// barrier, round and take the maximum into slots[i].result.
constexpr int kNormThreads = 256;

__global__ void __launch_bounds__(kNormThreads) k_norms(NormArgs A) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const size_t n = (size_t)A.n;
    // a phase whose pool overflowed is discarded (all blocks read the same
    // status, set by an earlier launch)
    if (__ldcg(&A.ctl->status) & kDevPoolFull) return;
    // every |x| of every matrix into per-column fixed-point sums: streaming
    // passes over the matrices' pool ranges
    for (int mi = 0; mi < A.count; ++mi) {
        // the counter keeps counting past the capacity when the pool overflows
        const unsigned long long cap = A.ctl->pool_cap;
        const unsigned long long p0 = min(__ldcg(&A.ctl->mark[mi]), cap);
        const unsigned long long p1 = min(__ldcg(&A.ctl->mark[mi + 1]), cap);
        unsigned long long* words = A.words + (size_t)mi * kChunks * n;
        unsigned* sticky = A.sticky + (size_t)mi * n;
        if (A.inst) {
            // batch: the fixed point of each column follows its instance's max
            // |x|; four entries per thread at a time, so that their dependent
            // loads (column, instance, max) overlap
            for (unsigned long long q0 = p0 + (unsigned long long)gt; q0 < p1; q0 += 4ull * nthreads) {
                unsigned long long xb[4];
                int c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const unsigned long long q = q0 + (unsigned long long)u * nthreads;
                    xb[u] = q < p1 ? mag_bits(A.pool_val[q]) : 0ull;
                    c[u] = xb[u] ? A.pool_col[q] : 0;
                }
                int lsb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    lsb[u] = 0;
                    if (xb[u] && (unsigned)c[u] < (unsigned)A.n)
                        lsb[u] = lsb_for_bound(A.slots[(size_t)A.inst[c[u]] * A.slot_stride + mi].absmax);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (!xb[u]) continue;
                    if ((unsigned)c[u] >= (unsigned)A.n) {
                        atomicOr(&A.ctl->status, kDevInternal);
                        continue;
                    }
                    exact_add(words + c[u], n, sticky + c[u], xb[u], lsb[u]);
                }
            }
            continue;
        }
        const int lsb = lsb_for_bound(A.slots[mi].absmax);
        for (unsigned long long q0 = p0 + (unsigned long long)gt; q0 < p1; q0 += 4ull * nthreads) {
            unsigned long long xb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned long long q = q0 + (unsigned long long)u * nthreads;
                xb[u] = q < p1 ? mag_bits(A.pool_val[q]) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (xb[u] != 0ull) {
                    const int c = A.pool_col[q0 + (unsigned long long)u * nthreads];
                    exact_add_checked(words, sticky, c, A.n, xb[u], lsb, A.ctl);
                }
            }
        }
    }
    if (!grid_barrier(A.ctl, A.budget_ns)) return;
    const int lane = threadIdx.x & 31;
    for (int mi = 0; mi < A.count; ++mi) {
        unsigned long long* words = A.words + (size_t)mi * kChunks * n;
        unsigned long long mx = 0ull;
        for (int j = gt; j < A.n; j += nthreads) {
            NormSlot* slot = A.inst ? A.slots + (size_t)A.inst[j] * A.slot_stride + mi : A.slots + mi;
            const int lsb = lsb_for_bound(slot->absmax);
            const double sum = chunk_round(words + j, n, A.sticky + (size_t)mi * n + j, lsb);
            const unsigned long long sb = (unsigned long long)__double_as_longlong(sum);
            if (A.inst) {
                if (sb) atomicMax(&slot->result, sb);  // columns of one warp may belong to several instances
            } else {
                mx = sb > mx ? sb : mx;
            }
        }
        if (!A.inst) {
            mx = warp_max_u64(mx);  // one reduction per warp, not per column
            if (lane == 0 && mx) atomicMax(&A.slots[mi].result, mx);
        }
    }
}

// ---------------------------------------------------------------- k_norms_rows
// The same norms, by tiles of consecutive rows: for banded and grid matrices
// a tile's entries fall in a narrow window of columns, so a block sums its
// tile exactly in shared memory (24-bit pieces in 32-bit words: a tile of at
// most 255 rows cannot overflow them) and adds the window to the global sums
// once, instead of one global reduction per piece of every entry.  A tile
// whose window is wider than kNormWin takes the global path entry by entry.
// One block per (tile, matrix); k_norms_finish rounds and takes the maxima.
constexpr int kNormTile = 128;
constexpr int kNormWin = 3072;
constexpr int kNormRowsThreads = 1024;
static_assert(kNormTile <= 255, "shared 24-bit pieces of a tile must not overflow");

size_t norms_rows_smem_bytes() { return sizeof(unsigned) * (size_t)(kNormPieces + 1) * kNormWin; }

__global__ void __launch_bounds__(kNormRowsThreads) k_norms_rows(NormRowsArgs A) {
    extern __shared__ unsigned nsm[];  // [kNormPieces][kNormWin] pieces, then [kNormWin] sticky counts
    __shared__ int s_lo[kNormRowsThreads / 32], s_hi[kNormRowsThreads / 32];
    if (__ldcg(&A.ctl->status) & kDevPoolFull) return;  // discarded phase
    const int mi = blockIdx.y;
    const int n = A.n;
    const int r0 = blockIdx.x * kNormTile, r1 = min(n, r0 + kNormTile);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int* rb = A.rb[mi];
    const int* re = A.re[mi];
    const int lsb0 = A.inst ? 0 : lsb_for_bound(A.slots[mi].absmax);
    unsigned long long* words = A.words + (size_t)mi * kNormPieces * n;
    unsigned* sticky = A.sticky + (size_t)mi * n;
    // the tile's column window (rows are sorted)
    int lo = INT_MAX, hi = -1;
    for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) {
        const int s = rb[r], e = re[r];
        if (s < e) {
            lo = min(lo, A.col[s]);
            hi = max(hi, A.col[e - 1]);
        }
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) {
        s_lo[wid] = lo;
        s_hi[wid] = hi;
    }
    __syncthreads();
    lo = INT_MAX;
    hi = -1;
    for (int i = 0; i < nw; ++i) {
        lo = min(lo, s_lo[i]);
        hi = max(hi, s_hi[i]);
    }
    if (hi < lo) return;  // an empty tile (same in all threads)
    if (lo < 0 || hi >= n) {
        if (threadIdx.x == 0) atomicOr(&A.ctl->status, kDevInternal);
        return;
    }
    const int wlen = hi - lo + 1;
    const bool local = wlen <= kNormWin;
    unsigned* wst = nsm + (size_t)kNormPieces * kNormWin;
    if (local) {
        for (int i = threadIdx.x; i < wlen; i += blockDim.x) {
#pragma unroll
            for (int p = 0; p < kNormPieces; ++p) nsm[p * kNormWin + i] = 0u;
            wst[i] = 0u;
        }
        __syncthreads();
    }
    for (int r = r0 + wid; r < r1; r += nw) {
        const int s = rb[r], e = re[r];
        // batch: the fixed point of a column follows its instance's max |x|;
        // a row's columns all belong to the row's instance (block diagonal)
        const int lsb = A.inst ? lsb_for_bound(A.slots[(size_t)A.inst[r] * A.slot_stride + mi].absmax) : lsb0;
        // 128 entries per round, all loads issued first
        for (int q0 = s; q0 < e; q0 += 128) {
            unsigned long long xs[4];
            int cs[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u * 32 + lane;
                xs[u] = q < e ? mag_bits(A.val[q]) : 0ull;
                cs[u] = q < e ? A.col[q] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned long long xb = xs[u];
                if (xb == 0ull) continue;
                const int c = cs[u];
                if ((unsigned)c >= (unsigned)n) {
                    atomicOr(&A.ctl->status, kDevInternal);
                    continue;
                }
                unsigned pc[4];
                bool lost;
                const int L = split24(xb, lsb, pc, lost);
                if (local) {
                    const int o = c - lo;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (pc[j]) atomicAdd(&nsm[(L + j) * kNormWin + o], pc[j]);
                    if (lost) atomicAdd(&wst[o], 1u);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (pc[j]) atomicAdd(&words[(size_t)(L + j) * n + c], (unsigned long long)pc[j]);
                    if (lost) atomicAdd(&sticky[c], 1u);
                }
            }
        }
    }
    if (!local) return;
    __syncthreads();
    for (int i = threadIdx.x; i < wlen; i += blockDim.x) {
#pragma unroll
        for (int p = 0; p < kNormPieces; ++p) {
            const unsigned v = nsm[p * kNormWin + i];
            if (v) atomicAdd(&words[(size_t)p * n + lo + i], (unsigned long long)v);
        }
        if (wst[i]) atomicAdd(&sticky[lo + i], wst[i]);
    }
}

__global__ void k_norms_finish(int n, int count, NormSlot* slots, unsigned long long* words, unsigned* sticky,
                               const Ctl* ctl, const int* inst, int slot_stride) {
    if (__ldcg(&ctl->status) & kDevPoolFull) return;
    // one thread per (matrix, column); the column count is padded to whole
    // warps so that a warp's columns belong to one matrix and it reduces
    // them before the single atomic
    const long long npad = ((long long)n + 31) & ~31LL;
    const long long nt = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < (long long)count * npad; u += nt) {
        const int mi = (int)(u / npad), j = (int)(u % npad);
        unsigned long long vb = 0ull;
        NormSlot* slot = slots + mi;
        if (j < n) {
            if (inst) slot = slots + (size_t)inst[j] * slot_stride + mi;
            const int lsb = lsb_for_bound(slot->absmax);
            const double v = round24(words + (size_t)mi * kNormPieces * n + j, (size_t)n, sticky + (size_t)mi * n + j, lsb);
            vb = (unsigned long long)__double_as_longlong(v);
        }
        if (inst) {
            // a warp's columns are consecutive, so their instances form
            // contiguous runs: a segmented reduction leaves each run's
            // maximum in its first lane
            const int ti = j < n ? inst[j] : -1;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long w = __shfl_down_sync(kFull, vb, o);
                const int tj = __shfl_down_sync(kFull, ti, o);
                if (lane + o < 32 && tj == ti) vb = w > vb ? w : vb;
            }
            const int tp = __shfl_up_sync(kFull, ti, 1);
            const bool first = lane == 0 || tp != ti;
            if (first && ti >= 0 && vb) atomicMax(&slot->result, vb);
        } else {
            vb = warp_max_u64(vb);
            if (lane == 0 && vb) atomicMax(&slot->result, vb);
        }
    }
}

// ---------------------------------------------------------------- k_export
// Copy nwords 32-bit words of a device record (the control block, norm slots,
// step records) into pinned host memory mapped into the device's address
// space.  The host reads the words after synchronising with the stream.  A
// kernel's stores take no copy engine, so these small read-backs do not
// queue behind a large device-to-host copy that another stream has in
// flight (a result being copied out while the next evaluation runs).
__global__ void k_export(const unsigned* src, unsigned* dst, int nwords) {
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = __ldcg(src + i);
}

// ---------------------------------------------------------------- k_row_bitmaps
// Column bitmap of every row of B for the product's symbolic pass: hdr[r] =
// {first column / 32, words}, the words at bits[rb[r]] on.  A row gets one
// only if it needs no more words than it has entries (so they fit its own
// pool range) and no more than one window's; otherwise words = 0.  One warp
// per row: each 32-entry piece ORs runs of lanes with the same word (the
// columns ascend) and the first lane of a run adds it to the word.
__global__ void k_row_bitmaps(int n, RowView B, int2* hdr, unsigned* bits) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
        const int s = B.rb[r], e = B.re[r];
        int2 h = make_int2(0, 0);
        if (e > s) {
            const int w0 = B.col[s] >> 5;
            const int nw = (B.col[e - 1] >> 5) - w0 + 1;
            h.x = w0;
            if (nw <= e - s && nw <= kBmWordsBig) {
                h.y = nw;
                for (int j = lane; j < nw; j += 32) bits[s + j] = 0u;
                __syncwarp();
                for (int q0 = s; q0 < e; q0 += 32) {
                    const int q = q0 + lane;
                    const bool in = q < e;
                    const int c = in ? B.col[q] : 0;
                    const int wi = in ? (c >> 5) - w0 : -1 - lane;
                    unsigned v = in ? 1u << (c & 31) : 0u;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const unsigned v2 = __shfl_down_sync(kFull, v, d);
                        const int w2 = __shfl_down_sync(kFull, wi, d);
                        if (lane + d < 32 && w2 == wi) v |= v2;
                    }
                    const int wp = __shfl_up_sync(kFull, wi, 1);
                    if (in && (lane == 0 || wp != wi)) atomicOr(bits + s + wi, v);
                }
            }
        }
        if (lane == 0) hdr[r] = h;
    }
}

// ---------------------------------------------------------------- plumbing
// max |x| over the pool entries [mark[i], mark[i+1])
__global__ void k_absmax(const double* pool_val, const Ctl* ctl, int i, NormSlot* slot) {
    const int lane = threadIdx.x & 31;
    const unsigned long long cap = ctl->pool_cap;  // counters may run past it on overflow
    const unsigned long long p0 = min(__ldcg(&ctl->mark[i]), cap), p1 = min(__ldcg(&ctl->mark[i + 1]), cap);
    unsigned long long mx = 0ull;
    for (unsigned long long q = p0 + blockIdx.x * blockDim.x + threadIdx.x; q < p1;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned long long b = mag_bits(pool_val[q]);
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

// Exclusive scan of row lengths re - rb into rowptr (n + 1 entries), in
// three launches over tiles of kScanTile rows: tile sums, a scan of the tile
// sums (one block), and the scan inside each tile plus its tile's offset.
// `sums` holds ceil(n / kScanTile) + 1 values.
constexpr int kScanTile = 1024;

__device__ __forceinline__ long long block_excl_scan(long long v, long long* part, long long* total) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) part[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = (int)(blockDim.x >> 5);
        long long p = lane < nw ? part[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, p, o);
            if (lane >= o) p += y;
        }
        if (lane < nw) part[lane] = p;  // inclusive warp totals
    }
    __syncthreads();
    const long long before = wid ? part[wid - 1] : 0;
    *total = part[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanTile) k_scan_tile_sums(int n, const int* rb, const int* re, long long* sums) {
    __shared__ long long part[32];
    const long long r = (long long)blockIdx.x * kScanTile + threadIdx.x;
    const long long len = r < n ? (long long)(re[r] - rb[r]) : 0;
    long long total;
    block_excl_scan(len, part, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanTile) k_scan_tiles(int ntiles, long long* sums, Ctl* ctl) {
    __shared__ long long part[32];
    // each thread owns a contiguous run of tiles
    const int per = (ntiles + kScanTile - 1) / kScanTile;
    const int t0 = threadIdx.x * per, t1 = min(ntiles, t0 + per);
    long long s = 0;
    for (int t = t0; t < t1; ++t) s += sums[t];
    long long total;
    long long run = block_excl_scan(s, part, &total);
    for (int t = t0; t < t1; ++t) {
        const long long v = sums[t];
        sums[t] = run;
        run += v;
    }
    if (threadIdx.x == 0) {
        sums[ntiles] = total;
        ctl->nnz_total = (unsigned long long)total;
    }
}

__global__ void __launch_bounds__(kScanTile) k_scan_apply(int n, const int* rb, const int* re, const long long* sums,
                                                           int* rowptr) {
    __shared__ long long part[32];
    const long long r = (long long)blockIdx.x * kScanTile + threadIdx.x;
    const long long len = r < n ? (long long)(re[r] - rb[r]) : 0;
    long long total;
    const long long ex = block_excl_scan(len, part, &total) + sums[blockIdx.x];
    if (r < n) rowptr[r] = (int)ex;  // the host rejects totals of 2^31 and more
    if (r == n - 1 || (n == 0 && r == 0)) rowptr[n] = (int)sums[gridDim.x];
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

// Copy a canonical CSR matrix into the pool: each row gets a 4-entry aligned
// slot of round-up(len, 4) entries (rows start 16-byte aligned, like the
// product kernel's rows).
__global__ void k_copy_rows(int n, const int* rowptr, const int* col, const double* val, int* rb, int* re,
                            int* pool_col, double* pool_val, Ctl* ctl, unsigned long long arena_size) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    Arena arena;
    for (int r = gw; r < n; r += nwarps) {
        int s = rowptr[r], e = rowptr[r + 1];
        const long long base = arena_take(arena, (unsigned long long)((e - s + 3) & ~3), arena_size, ctl, pool_val, lane);
        if (base < 0) {
            if (lane == 0) rb[r] = re[r] = 0;
            continue;
        }
        const int padded = (e - s + 3) & ~3;
        for (int q = lane; q < padded; q += 32) {
            pool_col[base + q] = q < e - s ? col[s + q] : 0;
            pool_val[base + q] = q < e - s ? val[s + q] : 0.0;
        }
        if (lane == 0) {
            rb[r] = (int)base;
            re[r] = (int)base + (e - s);
        }
    }
    arena_close(arena, pool_val, lane);
}

// Reset a caller-provided norm workspace for one matrix of n columns and
// nnz entries read in place: clear the control block, the norm slot and the
// column-sum words, and let the matrix's entries [0, nnz) be norm matrix 0.
__global__ void k_norm_scratch_init(Ctl* ctl, NormSlot* slot, unsigned long long* words, unsigned* sticky, int n,
                                    long long nnz) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nt = (long long)gridDim.x * blockDim.x;
    for (long long i = t; i < (long long)kChunks * n; i += nt) words[i] = 0ull;
    for (long long i = t; i < n; i += nt) sticky[i] = 0u;
    if (t == 0) {
        Ctl c{};
        c.pool_cap = (unsigned long long)nnz;
        c.pool_used = (unsigned long long)nnz;
        c.mark[0] = 0ull;
        c.mark[1] = (unsigned long long)nnz;
        *ctl = c;
        slot->absmax = 0ull;
        slot->result = 0ull;
    }
}

// ---- batches: the instance of every row (binary search over the row
// offsets off[0..ninst], off[ninst] = n)
__global__ void k_inst_table(int n, int ninst, const int* off, int* inst) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int lo = 0, hi = ninst - 1;  // largest i with off[i] <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    inst[r] = lo;
}

// Check every input of a batch like k_validate: thread per global row.
__global__ void k_validate_batch(int n, const int* inst, const BatchSrc* src, const int* nnz, Ctl* ctl) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int i = inst[r];
    const BatchSrc S = src[i];
    const int l = r - S.off;
    bool bad = false;
    const int s = S.rowptr[l], e = S.rowptr[l + 1];
    if (l == 0 && s != 0) bad = true;
    if (l == S.n - 1 && e != nnz[i]) bad = true;
    if (s > e || s < 0 || e > nnz[i]) {
        bad = true;
    } else {
        int prev = -1;
        for (int q = s; q < e; ++q) {
            const int c = S.col[q];
            const bool finite = (mag_bits(S.val[q]) >> 52) != 0x7ffull;
            if (c <= prev || c >= S.n || !finite) {
                bad = true;
                break;
            }
            prev = c;
        }
    }
    if (bad) atomicOr(&ctl->status, kDevBadInput);
}

// Copy the inputs of a batch into the pool as the block-diagonal matrix
// (columns shifted to global), rows padded to 4 entries; records each
// instance's max |x| in absmax[i * stride].
__global__ void k_copy_rows_batch(int n, const int* inst, const BatchSrc* src, int* rb, int* re, int* pool_col,
                                  double* pool_val, Ctl* ctl, unsigned long long arena_size, NormSlot* absmax,
                                  int stride) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    Arena arena;
    for (int r = gw; r < n; r += nwarps) {
        const int i = inst[r];
        const BatchSrc S = src[i];
        const int l = r - S.off;
        const int s = S.rowptr[l], e = S.rowptr[l + 1];
        const long long base = arena_take(arena, (unsigned long long)((e - s + 3) & ~3), arena_size, ctl, pool_val, lane);
        if (base < 0) {
            if (lane == 0) rb[r] = re[r] = 0;
            continue;
        }
        const int padded = (e - s + 3) & ~3;
        unsigned long long mx = 0ull;
        for (int q = lane; q < padded; q += 32) {
            const bool in = q < e - s;
            const double v = in ? S.val[s + q] : 0.0;
            pool_col[base + q] = in ? S.col[s + q] + S.off : 0;
            pool_val[base + q] = v;
            const unsigned long long b = mag_bits(v);
            mx = b > mx ? b : mx;
        }
        mx = warp_max_u64(mx);
        if (lane == 0) {
            rb[r] = (int)base;
            re[r] = (int)base + (e - s);
            if (absmax && mx) atomicMax(&absmax[(size_t)i * stride].absmax, mx);
        }
    }
    arena_close(arena, pool_val, lane);
}

// out rows <- the rows of matrix sel[inst[r]] of a table of row arrays.
struct RowTable {
    const int* rb[kMaxAdd + 2];
    const int* re[kMaxAdd + 2];
};
__global__ void k_compose_rows(int n, const int* inst, const int* sel, RowTable T, int* out_rb, int* out_re) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int k = sel[inst[r]];
    out_rb[r] = T.rb[k][r];
    out_re[r] = T.re[k][r];
}

// Split the block-diagonal result (global row pointers rowptr) into the
// instances' CSR: instance i's row pointers start at out_rp + off_i + i
// (n_i + 1 entries, rebased to 0), its entries at rowptr[off_i] with local
// columns.
__global__ void k_gather_batch(int n, int ninst, const int* inst, const int* off, RowView src, const int* rowptr,
                               int* out_rp, int* col, double* val) {
    const int lane = threadIdx.x & 31;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int gw = gt >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = gt; i < ninst; i += gridDim.x * blockDim.x)
        out_rp[off[i + 1] + i] = rowptr[off[i + 1]] - rowptr[off[i]];
    for (int r = gw; r < n; r += nwarps) {
        const int i = inst[r];
        const int o = off[i];
        const int s = src.rb[r], e = src.re[r], d = rowptr[r];
        if (lane == 0) out_rp[r + i] = d - rowptr[o];
        for (int q = lane; q < e - s; q += 32) {
            col[d + q] = src.col[s + q] - o;
            val[d + q] = src.val[s + q];
        }
    }
}

// bounds[i] = rowptr[off[i]], i = 0..ninst
__global__ void k_bounds(int ninst, const int* off, const int* rowptr, int* bounds) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= ninst) bounds[i] = rowptr[off[i]];
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

// ---------------------------------------------------------------- launchers
// Launch configuration, per device (set up once by kernels_init, guarded by
// a mutex; a device's entry is published through `ready`).
struct DevCfg {
    int sms = 0, alg1_blocks = 0, alg1b_blocks = 0, norm_blocks = 0;
    std::atomic<bool> ready{false};
};
constexpr int kMaxDevices = 64;
static DevCfg g_dev[kMaxDevices];
// wait limit of every grid barrier (PSF_TUNE_BARRIER_BUDGET_NS)
static std::atomic<unsigned long long> g_barrier_budget_ns{kBarrierBudgetDefaultNs};
void set_barrier_budget_ns(unsigned long long ns) { g_barrier_budget_ns.store(ns); }
unsigned long long barrier_budget_ns() { return g_barrier_budget_ns.load(); }
static std::mutex g_init_mu;
static std::atomic<long long> g_launches{0};

long long launch_count() { return g_launches.load(); }
void count_launches(int k) { g_launches += k; }

static const DevCfg& dcfg();
static int sms_now();
static const DevCfg& dcfg() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    return g_dev[dev];
}

cudaError_t kernels_init() {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    DevCfg& c = g_dev[dev];
    if (c.ready.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_init_mu);
    if (c.ready.load(std::memory_order_acquire)) return cudaSuccess;
    int sms = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    const void* prods[7] = {(const void*)k_product<true, false, false>, (const void*)k_product<false, false, false>,
                            (const void*)k_product<true, true, false>, (const void*)k_product<false, true, false>,
                            (const void*)k_product<false, false, true>,
                            (const void*)k_product<false, false, true, kBmWordsBig>,
                            (const void*)k_product<false, true, false, kBmWordsBig>};
    const int psmem[7] = {(int)prod_smem_bytes<true>(), (int)prod_smem_bytes<false>(), (int)prod_smem_bytes<true>(),
                          (int)prod_smem_bytes<false>(), (int)prod_smem_bytes<false>(),
                          (int)prod_smem_bytes<false, kBmWordsBig>(), (int)prod_smem_bytes<false, kBmWordsBig>()};
    for (int i = 0; i < 7; ++i) {
        err = cudaFuncSetAttribute(prods[i], cudaFuncAttributeMaxDynamicSharedMemorySize, psmem[i]);
        if (err != cudaSuccess) return err;
    }
    err = cudaFuncSetAttribute((const void*)k_product_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)cta_smem_bytes());
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute((const void*)k_norms_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)norms_rows_smem_bytes());
    if (err != cudaSuccess) return err;
    int per = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_alg1, kAlg1Threads, 0);
    if (err != cudaSuccess) return err;
    c.alg1_blocks = sms * (per < kAlg1BlocksPerSm ? per : kAlg1BlocksPerSm);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_alg1_batch, kAlg1Threads, 0);
    if (err != cudaSuccess) return err;
    c.alg1b_blocks = sms * (per < 4 ? per : 4);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_norms, kNormThreads, 0);
    if (err != cudaSuccess) return err;
    c.norm_blocks = sms * (per < 2 ? per : 2);
    if (c.alg1_blocks <= 0 || c.alg1b_blocks <= 0 || c.norm_blocks <= 0) return cudaErrorInvalidConfiguration;
    c.sms = sms;
    c.ready.store(true, std::memory_order_release);
    return cudaSuccess;
}

int num_sms() { return dcfg().sms; }
static int sms_now() { return dcfg().sms; }

template <bool TAB, bool BATCH, bool WIDE, int W = kBmWords>
static cudaError_t prod_launch(const ProductArgs& P, cudaStream_t st) {
    constexpr int kWarps = ProdSmem<TAB, W>::kWarps;
    // one wave of resident blocks, rows strided over the warps (each warp
    // keeps one pool arena)
    long long blocks = ((long long)P.n + kWarps - 1) / kWarps;
    const long long cap = (long long)sms_now() * ProdSmem<TAB, W>::kBlocksPerSm;
    if (blocks > cap) blocks = cap;
    k_product<TAB, BATCH, WIDE, W><<<(unsigned)blocks, kWarps * 32, prod_smem_bytes<TAB, W>(), st>>>(P);
    ++g_launches;
    return cudaGetLastError();
}

static cudaError_t cta_launch(const ProductArgs& P, cudaStream_t st) {
    long long blocks = P.n;
    const long long cap = (long long)sms_now() * 7;
    if (blocks > cap) blocks = cap;
    k_product_cta<<<(unsigned)blocks, kCtaWarps * 32, cta_smem_bytes(), st>>>(P);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_product(const ProductArgs& P, bool table, cudaStream_t st, double out_len, bool wide_window,
                           bool cta) {
    if (P.n <= 0) return cudaSuccess;
    if (cta && !table && !P.inst && P.chunk_cols <= 0 && P.chunk_slots <= 0) return cta_launch(P, st);
    if (P.inst) {
        if (table) return prod_launch<true, true, false>(P, st);
        return wide_window ? prod_launch<false, true, false, kBmWordsBig>(P, st) : prod_launch<false, true, false>(P, st);
    }
    if (table) return prod_launch<true, false, false>(P, st);
    // rows expected to span more columns than the bitmap covers: the wide
    // window (with every accumulator slot, as WIDE)
    if (wide_window) return prod_launch<false, false, true, kBmWordsBig>(P, st);
    // rows expected near or above the bitmap map's kAccCap - 32 slots: WIDE
    if (out_len > 0.9 * (kAccCap - 32)) return prod_launch<false, false, true>(P, st);
    return prod_launch<false, false, false>(P, st);
}

cudaError_t launch_row_bitmaps(int n, const RowView& B, int2* hdr, unsigned* bits, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long blocks = ((long long)n + 7) / 8;
    const long long cap = (long long)sms_now() * 8;
    if (blocks > cap) blocks = cap;
    k_row_bitmaps<<<(unsigned)blocks, 256, 0, st>>>(n, B, hdr, bits);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_alg1(const Alg1Args& A, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(&A.ctl->cslot[0], 0, sizeof(A.ctl->cslot), st);
    if (err != cudaSuccess) return err;
    Alg1Args a = A;
    a.budget_ns = barrier_budget_ns();
    void* args[] = {&a};
    ++g_launches;
    return cudaLaunchCooperativeKernel((const void*)k_alg1, dim3(dcfg().alg1_blocks), dim3(kAlg1Threads), args,
                                       0, st);
}

cudaError_t launch_norms(const NormArgs& A, cudaStream_t st) {
    NormArgs a = A;
    a.budget_ns = barrier_budget_ns();
    void* args[] = {&a};
    ++g_launches;
    return cudaLaunchCooperativeKernel((const void*)k_norms, dim3(dcfg().norm_blocks), dim3(kNormThreads), args,
                                       0, st);
}

cudaError_t launch_absmax(const double* pool_val, const Ctl* ctl, int i, NormSlot* slot, cudaStream_t st) {
    k_absmax<<<sms_now() * 4, 256, 0, st>>>(pool_val, ctl, i, slot);
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

size_t scan_scratch_len(int n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 2; }

cudaError_t launch_scan_rows(int n, const int* rb, const int* re, int* rowptr, Ctl* ctl, long long* sums,
                             cudaStream_t st) {
    const int ntiles = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
    if (n > 0) {
        k_scan_tile_sums<<<ntiles, kScanTile, 0, st>>>(n, rb, re, sums);
        ++g_launches;
    } else {
        cudaError_t err = cudaMemsetAsync(sums, 0, sizeof(long long), st);
        if (err != cudaSuccess) return err;
    }
    k_scan_tiles<<<1, kScanTile, 0, st>>>(ntiles, sums, ctl);
    ++g_launches;
    k_scan_apply<<<ntiles, kScanTile, 0, st>>>(n, rb, re, sums, rowptr);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_gather(int n, const RowView& src, const int* rowptr, int* col, double* val,
                          cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > sms_now() * 16) blocks = sms_now() * 16;
    k_gather<<<blocks, 256, 0, st>>>(n, src, rowptr, col, val);
    ++g_launches;
    return cudaGetLastError();
}

// FP64 rate probe: every thread runs eight independent chains of fused
// multiply-adds (enough in flight to fill the pipe); the result is stored so
// that none of the work can be dropped.
// (Measured on GB300: this form reaches 1.257 TFLOP/s at 2070 MHz, 99.9 %
// of the unit count; a form with __fma_rn and the output pointer last was
// scheduled differently and reached only 1.01-1.06.)
__global__ void k_fp64_probe(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

int fp64_probe_blocks() { return sms_now() * 4; }

cudaError_t launch_fp64_probe(int iters, double* out, cudaStream_t st) {
    k_fp64_probe<<<fp64_probe_blocks(), 256, 0, st>>>(out, iters, 0.999999, 1e-7);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_identity(int n, double alpha, int* rowptr, int* col, double* val, cudaStream_t st) {
    k_identity<<<(n + 1 + 255) / 256, 256, 0, st>>>(n, alpha, rowptr, col, val);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_copy_rows(int n, const int* rowptr, const int* col, const double* val, int* rb, int* re,
                             int* pool_col, double* pool_val, Ctl* ctl, unsigned long long arena_size,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // about four rows per warp: each row is a dependent load pair, so the
    // copy is latency-bound and wants many warps in flight
    long long blocks = ((long long)n + 31) / 32;
    if (blocks > (long long)sms_now() * 8) blocks = (long long)sms_now() * 8;
    k_copy_rows<<<(unsigned)blocks, 256, 0, st>>>(n, rowptr, col, val, rb, re, pool_col, pool_val, ctl, arena_size);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_norm_scratch_init(Ctl* ctl, NormSlot* slot, unsigned long long* words, unsigned* sticky, int n,
                                     long long nnz, cudaStream_t st) {
    int blocks = (int)(((long long)kChunks * n + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > sms_now() * 4) blocks = sms_now() * 4;
    k_norm_scratch_init<<<blocks, 256, 0, st>>>(ctl, slot, words, sticky, n, nnz);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_alg1_batch(const Alg1BatchArgs& A, cudaStream_t st) {
    if (A.ninst > kMaxBatch) return cudaErrorInvalidValue;
    cudaError_t err = cudaMemsetAsync(A.cslot, 0, sizeof(unsigned long long) * 2 * (size_t)A.ninst, st);
    if (err != cudaSuccess) return err;
    Alg1BatchArgs a = A;
    a.budget_ns = barrier_budget_ns();
    void* args[] = {&a};
    ++g_launches;
    return cudaLaunchCooperativeKernel((const void*)k_alg1_batch, dim3(dcfg().alg1b_blocks), dim3(kAlg1Threads), args,
                                       0, st);
}

cudaError_t launch_inst_table(int n, int ninst, const int* off, int* inst, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_inst_table<<<(n + 255) / 256, 256, 0, st>>>(n, ninst, off, inst);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_validate_batch(int n, const int* inst, const BatchSrc* src, const int* nnz, Ctl* ctl,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_validate_batch<<<(n + 255) / 256, 256, 0, st>>>(n, inst, src, nnz, ctl);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_copy_rows_batch(int n, const int* inst, const BatchSrc* src, int* rb, int* re, int* pool_col,
                                   double* pool_val, Ctl* ctl, unsigned long long arena_size, NormSlot* absmax,
                                   int stride, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > sms_now() * 8) blocks = sms_now() * 8;
    k_copy_rows_batch<<<blocks, 256, 0, st>>>(n, inst, src, rb, re, pool_col, pool_val, ctl, arena_size, absmax,
                                              stride);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_compose_rows(int n, const int* inst, const int* sel, const int* const* rbs, const int* const* res,
                                int count, int* out_rb, int* out_re, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (count > kMaxAdd + 2) return cudaErrorInvalidValue;
    RowTable T{};
    for (int k = 0; k < count; ++k) {
        T.rb[k] = rbs[k];
        T.re[k] = res[k];
    }
    k_compose_rows<<<(n + 255) / 256, 256, 0, st>>>(n, inst, sel, T, out_rb, out_re);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_gather_batch(int n, int ninst, const int* inst, const int* off, const RowView& src,
                                const int* rowptr, int* out_rp, int* col, double* val, cudaStream_t st) {
    int blocks = (n + 7) / 8;
    if (blocks < 1) blocks = 1;
    if (blocks > sms_now() * 16) blocks = sms_now() * 16;
    k_gather_batch<<<blocks, 256, 0, st>>>(n, ninst, inst, off, src, rowptr, out_rp, col, val);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_bounds(int ninst, const int* off, const int* rowptr, int* bounds, cudaStream_t st) {
    k_bounds<<<(ninst + 1 + 255) / 256, 256, 0, st>>>(ninst, off, rowptr, bounds);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_reuse_copy_batch(const ProductArgs& P, cudaStream_t st) {
    if (P.n <= 0) return cudaSuccess;
    long long blocks = ((long long)P.n + 7) / 8;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_reuse_copy_batch<<<(unsigned)blocks, 256, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_export(const void* src, void* dst, size_t bytes, cudaStream_t st) {
    k_export<<<1, 256, 0, st>>>(static_cast<const unsigned*>(src), static_cast<unsigned*>(dst), (int)(bytes / 4));
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_reuse_pass1(const ReuseArgs& R, cudaStream_t st) {
    if (R.n <= 0) return cudaSuccess;
    int blocks = (R.n + 7) / 8;
    if (blocks > sms_now() * 8) blocks = sms_now() * 8;
    k_reuse_pass1<<<blocks, 256, 0, st>>>(R);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_norms_rows(const NormRowsArgs& A, cudaStream_t st) {
    if (A.n <= 0 || A.count <= 0) return cudaSuccess;
    dim3 grid((unsigned)((A.n + kNormTile - 1) / kNormTile), (unsigned)A.count);
    k_norms_rows<<<grid, kNormRowsThreads, norms_rows_smem_bytes(), st>>>(A);
    ++g_launches;
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const long long total = (long long)A.count * (((long long)A.n + 31) & ~31LL);
    long long blocks = (total + 255) / 256;  // one (matrix, column) per thread
    if (blocks > 65535LL * 64) blocks = 65535LL * 64;
    k_norms_finish<<<(unsigned)blocks, 256, 0, st>>>(A.n, A.count, A.slots, A.words, A.sticky, A.ctl, A.inst,
                                                     A.slot_stride);
    ++g_launches;
    return cudaGetLastError();
}


}  // namespace psf
