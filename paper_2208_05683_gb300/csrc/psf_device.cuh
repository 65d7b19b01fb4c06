// psf_device.cuh -- device-side data structures and helpers shared by the
// CUDA kernels of the filtered PS evaluator.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace psf {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kChunks = 8;    // exact column sums: 8 x 32-bit chunks = 256-bit fixed point
constexpr int kWindow = 190;  // bits between the fixed point's LSB and 2^E_ref
constexpr int kMinLsb = -1074;  // the LSB of the subnormals: nothing below it
constexpr int kExactBits = 96;  // a rounded column sum at or above 2^(e_lsb + 96) is exact
constexpr int kMaxAdd = 24;   // addend terms of one product (PSF_MAX_Q + 1)
constexpr int kMaxNorms = 11; // ||Z^i||_1, i = 0..10

// Device status bits (Ctl::status).
enum : int {
    kDevOk = 0,
    kDevBadInput = 1,
    kDevPoolFull = 2,
    kDevNotConv = 4,
    kDevTimeout = 8,
    kDevInternal = 16,  // a pool entry held a column outside [0, n) (skipped)
};

// Control block of one evaluation, in device memory.
struct Ctl {
    unsigned long long pool_used;  // pool entries reserved (keeps counting past capacity)
    unsigned long long pool_cap;
    unsigned long long cslot[2];   // Algorithm 1 column-sum maxima (bits of doubles >= 0)
    unsigned long long nnz_total;  // row-length scan result
    int status;
    int pad2;
    // Algorithm 1 candidate lists (two buffers of cand_cap entries): entry
    // counts, and a flag set when the product's list overflowed
    unsigned long long cand_cnt[2];
    // entries in the far half of list 1 (candidates below eps_g / 64, set
    // apart by Algorithm 1's first rescan)
    unsigned long long cand_far;
    unsigned long long cand_cap;
    int cand_over;
    unsigned cand_chunk;  // entries a warp reserves at a time (32..128)
    int dropped;          // set once Algorithm 1 has dropped an entry (baby steps reuse powers until then)
    int pad1;
    unsigned bar_count;  // fields from here on survive a pool reset
    unsigned bar_gen;
    int pad;
    unsigned long long fma_total;  // algorithmic multiply-adds of all products
    unsigned long long mark[kMaxNorms + 1];  // pool counter snapshots delimiting the norm matrices
};

// Device half of psf_step_info_t.
struct StepStat {
    unsigned long long pool_start;  // pool counter before the step's product
    unsigned long long pool_end;    // 0: the step's entries end at the pool counter
    unsigned long long nnz_pre, nnz_post, ncand, fma;
    double eps_f, dropped;
    int iters;
    unsigned span_max;  // widest column window of the product's rows (hi - lo + 1)
};

// Per-matrix norm slot for the exact 1-norm kernel.
struct NormSlot {
    unsigned long long absmax;  // bits of max |x|
    unsigned long long result;  // bits of the 1-norm
};

// Row view of a matrix: row r spans [rb[r], re[r]) of col/val.
struct RowView {
    const int* rb;
    const int* re;
    const int* col;
    const double* val;
};

// One term alpha * M of a weighted sum; rb == nullptr means M = I.
struct AddTerm {
    const int* rb;
    const int* re;
    const int* col;
    const double* val;
    double alpha;
};

// A batch of instances is one block-diagonal matrix: instance i owns the
// rows and columns [off_i, off_i + n_i).  What a step does to an instance's
// rows is one of these modes.
enum : int {
    kBatchSkip = 0,     // no output rows
    kBatchProduct = 1,  // sum of the addends + A B (and Algorithm 1 pass 1)
    kBatchPass = 2,     // rows of B passed through unchanged (no work)
    kBatchAddOnly = 3,  // sum of the addends only
};

// Per-instance parameters of one batched step.
struct BatchStep {
    double eps_g;  // > 0: Algorithm 1 on this instance with eps_g and bound
    double bound;  // eps_g (1 + e_r)
    int e_lsb;     // LSB exponent of the column-sum fixed point
    int maxit;     // Algorithm 1 pass cap
    int mode;
    int reuse;     // baby step k <= 10 of an instance whose norm phase computed Z^k
};

// C = sum_t add[t].alpha * M_t + A * B, rows written to the pool.
struct ProductArgs {
    int n;
    RowView A;  // A.rb == nullptr: no product term
    RowView B;
    int nadd;
    AddTerm add[kMaxAdd];
    int* out_rb;
    int* out_re;
    int* pool_col;
    double* pool_val;
    Ctl* ctl;
    int filtering;  // 1: first pass of Algorithm 1 on |x| <= eps_g
    double eps_g;
    int e_lsb;
    unsigned long long* words;  // kChunks * n, column-sum chunks
    unsigned* sticky;           // n
    StepStat* stat;
    NormSlot* absmax_slot;      // optional: record max |x|
    int chunk_cols;             // > 0: fewer columns per chunk (exercises chunking)
    int chunk_slots;            // > 0: fewer accumulator slots per chunk
    unsigned long long arena;   // pool entries a warp takes at a time (multiple of 4)
    // Algorithm 1 candidates (0 < |x| <= eps_g) appended to list 0 (nullptr: none)
    int* cand_col;
    unsigned long long* cand_x;  // |x| bits
    unsigned long long cand_cap;
    unsigned cand_chunk;
    const int* skip_unless;     // non-null: the launch does nothing while *skip_unless == 0
    // batch (inst == nullptr: one instance, the fields above apply to all rows)
    const int* inst;            // instance of each row, n entries
    const int* inst_off;        // first row (= column) of each instance, ninst + 1 entries (optional)
    const BatchStep* bstep;     // per instance
    const double* alpha_tab;    // [t * ninst + i]: coefficient of term t for instance i (+0: absent)
    int ninst;
    int absmax_stride;          // absmax slot of instance i: absmax_slot + i * absmax_stride
    StepStat* stat_tab;         // per instance (nullptr: no statistics)
    // batched baby steps: instances with bstep.reuse whose flag here is 0
    // (no entry dropped so far) take their rows from `power` (the norm
    // phase's Z^k) instead of the product
    const int* inst_dropped;
    RowView power;
    // column bitmaps of B's rows (nullptr: none): bhdr[k] = {first column of
    // row k / 32, words}, the words at bbits[B.rb[k]] on (0 words: row k has
    // no bitmap)
    const int2* bhdr;
    const unsigned* bbits;
};

// Algorithm 1 passes 2, 3, ... and compaction for every filtered instance of
// a batched step.
struct Alg1BatchArgs {
    int n;  // rows = columns of the block-diagonal batch
    int ninst;
    const int* inst;
    const BatchStep* bstep;
    int* rb;
    int* re;
    int* col;
    double* val;
    unsigned long long* words;
    unsigned* sticky;
    unsigned long long* cslot;             // 2 * ninst column-sum maxima (bits)
    const unsigned long long* pool_start;  // pool counter before the step's product
    Ctl* ctl;
    StepStat* stat_tab;  // per instance
    int* cand_col;       // two candidate lists of ctl->cand_cap entries each
    unsigned long long* cand_x;
    int* inst_dropped;   // optional: set to 1 for the instances that dropped entries
    int far_shift;       // as in Alg1Args
    unsigned long long budget_ns;  // grid-barrier wait limit (set by the launcher)
};

// One input matrix of a batch (device CSR, 0-based local columns).
struct BatchSrc {
    const int* rowptr;
    const int* col;
    const double* val;
    int n;
    int off;  // first global row / column
};

struct Alg1Args {
    int n;
    int* rb;
    int* re;
    int* col;
    double* val;
    double eps_g, bound;
    int maxit, e_lsb;
    unsigned long long* words;
    unsigned* sticky;
    Ctl* ctl;
    StepStat* stat;
    int* cand_col;               // two candidate lists of ctl->cand_cap entries each
    unsigned long long* cand_x;
    int far_shift;               // candidates at or below eps_g / 2^far_shift are set apart
    unsigned long long budget_ns;  // grid-barrier wait limit (set by the launcher)
};

// Arguments of k_reuse_pass1 (a baby step that equals a power of the norm
// phase).
struct ReuseArgs {
    int n;
    const int* rb;
    const int* re;
    const int* col;
    const double* val;
    int k;  // power
    double eps_g;
    int e_lsb;
    unsigned long long fma;  // the power's multiply-adds in the norm phase
    unsigned long long* words;
    unsigned* sticky;
    int* cand_col;
    unsigned long long* cand_x;
    unsigned long long cand_cap;
    unsigned cand_chunk;
    Ctl* ctl;
    StepStat* stat;
};

// Exact ||M_i||_1 of up to kMaxNorms matrices given by their rows (row r of
// matrix i spans [rb[i][r], re[i][r]) of col/val); max |x| of matrix i is in
// slots[i].absmax.
struct NormRowsArgs {
    int n;
    int count;
    const int* rb[kMaxNorms];
    const int* re[kMaxNorms];
    const int* col;
    const double* val;
    NormSlot* slots;
    unsigned long long* words;  // count * kNormPieces * n, zero on entry
    unsigned* sticky;           // count * n, zero on entry
    Ctl* ctl;
    const int* inst;            // batch: instance of each column; matrix i of instance t: slots[t * slot_stride + i]
    int slot_stride;
};

// Matrix i of the norm kernel occupies the pool entries [mark[i], mark[i+1])
// (gaps read as exact zeros).
struct NormArgs {
    int n;
    int count;  // matrices
    const int* pool_col;
    const double* pool_val;
    NormSlot* slots;            // count (instance i of a batch: slots + i * slot_stride)
    unsigned long long* words;  // count * kChunks * n
    unsigned* sticky;           // count * n
    Ctl* ctl;
    const int* inst;            // batch: instance of each column (nullptr: one instance)
    int slot_stride;
    unsigned long long budget_ns;  // grid-barrier wait limit (set by the launcher)
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int warp_min(int v) {
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x - v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// E_ref - kWindow clamped: the LSB exponent of the column-sum fixed point for
// summands below 2^E_ref, where E_ref is the smallest e with x < 2^e.
__device__ __forceinline__ int lsb_for_bound(unsigned long long xbits) {
    int E = (int)((xbits >> 52) & 0x7ff);
    int eref = E ? E - 1023 + 1 : -1022;
    int lsb = eref - kWindow;
    return lsb < kMinLsb ? kMinLsb : lsb;
}

// Is a column sum rounded from the fixed point with LSB 2^e_lsb the exact
// sum rounded?  The truncated remainder is below 2^(e_lsb + 32) (at most
// 2^31 summands), so it only acts as a sticky bit when the sum's leading bit
// is 54 + 32 or more bits above the LSB; an LSB at the subnormal LSB
// truncates nothing.
__device__ __forceinline__ bool sum_is_exact(double c, int e_lsb) {
    const int E = (int)(((unsigned long long)__double_as_longlong(c) >> 52) & 0x7ff);
    return e_lsb <= kMinLsb || (E != 0 && E - 1023 >= e_lsb + kExactBits);
}

// |x| as the bit pattern of a non-negative double: for such patterns the
// unsigned integer order is the order of the values, so magnitude tests need
// no floating-point instruction.
__device__ __forceinline__ unsigned long long mag_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Exact column sums with deferred carries.  A column's fixed-point value is
//   sum_c  w[c] * 2^(32 c + e_lsb),  c = 0 .. kChunks-1,
// where every 64-bit word w[c] only ever receives addends of magnitude below
// 2^32, added or subtracted (two's complement): a word absorbs 2^31
// operations without overflow, operations need no carry handling and are
// fire-and-forget reductions; carries are propagated once, when the column
// is read (chunk_round).  Bits below 2^e_lsb are truncated; *sticky counts
// the summands whose truncated part is nonzero (it is decremented when such
// a summand is subtracted), so the remainder is zero iff the count is.

// Split v (0 <= v < 2^(e_lsb + kWindow)) into its chunk pieces: returns the
// first chunk index, and the three 32-bit pieces (possibly 0).
__device__ __forceinline__ int exact_split(unsigned long long vbits, int e_lsb, unsigned long long& p0,
                                           unsigned long long& p1, unsigned long long& p2, bool& lost) {
    int E = (int)(vbits >> 52);
    unsigned long long M = vbits & ((1ull << 52) - 1);
    int e;
    if (E) {
        M |= (1ull << 52);
        e = E - 1075;
    } else {
        e = -1074;
    }
    p0 = p1 = p2 = 0ull;
    lost = false;
    if (M == 0ull) return 0;
    int o = e - e_lsb;
    if (o < 0) {
        int sh = -o;
        lost = (sh >= 64 ? M : (M & ((1ull << sh) - 1))) != 0ull;
        M = sh >= 64 ? 0ull : (M >> sh);
        if (M == 0ull) return 0;
        o = 0;
    }
    const int L = o >> 5, s = o & 31;
    const unsigned long long lo = M << s;  // bits [0, 64) of M * 2^s
    p0 = lo & 0xffffffffull;
    p1 = lo >> 32;
    p2 = s ? (M >> (64 - s)) : 0ull;  // bits [64, 85)
    return L;
}

// Add v to the column whose chunk 0 is at w (chunk stride `stride`).
__device__ __forceinline__ void exact_add(unsigned long long* w, size_t stride, unsigned* sticky,
                                          unsigned long long vbits, int e_lsb) {
    unsigned long long p0, p1, p2;
    bool lost;
    const int L = exact_split(vbits, e_lsb, p0, p1, p2, lost);
    if (lost) atomicAdd(sticky, 1u);
    if (p0) atomicAdd(w + (size_t)L * stride, p0);
    if (p1) atomicAdd(w + (size_t)(L + 1) * stride, p1);
    if (p2) atomicAdd(w + (size_t)(L + 2) * stride, p2);
}

// Subtract v (added before with the same e_lsb) from the column.
__device__ __forceinline__ void exact_sub(unsigned long long* w, size_t stride, unsigned* sticky,
                                          unsigned long long vbits, int e_lsb) {
    unsigned long long p0, p1, p2;
    bool lost;
    const int L = exact_split(vbits, e_lsb, p0, p1, p2, lost);
    if (lost) atomicSub(sticky, 1u);
    if (p0) atomicAdd(w + (size_t)L * stride, 0ull - p0);
    if (p1) atomicAdd(w + (size_t)(L + 1) * stride, 0ull - p1);
    if (p2) atomicAdd(w + (size_t)(L + 2) * stride, 0ull - p2);
}

// Round the non-negative integer limb[0..3] (256 bits, little endian) times
// 2^e_lsb to the nearest double, ties to even; `st` flags a positive
// remainder below the LSB (it breaks ties upward).
__device__ __forceinline__ double round_limbs(const unsigned long long limb[4], bool st, int e_lsb) {
    int top = -1;
    for (int i = 3; i >= 0; --i)
        if (limb[i]) {
            top = i * 64 + 63 - __clzll((long long)limb[i]);
            break;
        }
    if (top < 0) return 0.0;
    if (top <= 52) return ldexp((double)limb[0], e_lsb);  // < 2^53: exact
    int shift = top - 52;
    int wi = shift >> 6, ws = shift & 63;
    unsigned long long M = limb[wi] >> ws;
    if (ws && wi + 1 < 4) M |= limb[wi + 1] << (64 - ws);
    M &= (1ull << 53) - 1;
    int rpos = shift - 1;
    int rbit = (int)((limb[rpos >> 6] >> (rpos & 63)) & 1ull);
    if (!st) {
        int sw = rpos >> 6, sb = rpos & 63;
        if (sb && (limb[sw] & ((1ull << sb) - 1))) st = true;
        for (int i = 0; i < sw && !st; ++i) st = limb[i] != 0ull;
    }
    if (rbit && (st || (M & 1ull))) {
        ++M;
        if (M == (1ull << 53)) {
            M >>= 1;
            ++shift;
        }
    }
    return ldexp((double)M, shift + e_lsb);
}

// Read a column's chunks (L2 reads: they were written by other SMs'
// reductions), clear them if `clear`, propagate the (signed) carries and
// round the non-negative value to the nearest double, ties to even (a
// truncated positive remainder, flagged by a nonzero sticky count, breaks
// ties upward).
__device__ __forceinline__ double chunk_round(unsigned long long* w, size_t stride, unsigned* sticky, int e_lsb,
                                              bool clear = true) {
    unsigned long long limb[4] = {0ull, 0ull, 0ull, 0ull};
    long long carry = 0;
    // all chunks are loaded before any is cleared, so the loads are in
    // flight together
    unsigned long long raw[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) raw[c] = __ldcg(w + (size_t)c * stride);
    const bool st = __ldcg(sticky) != 0u;
    if (clear) {
#pragma unroll
        for (int c = 0; c < kChunks; ++c) w[(size_t)c * stride] = 0ull;
        *sticky = 0u;
    }
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
        const long long t = (long long)raw[c] + carry;
        limb[c >> 1] |= ((unsigned long long)t & 0xffffffffull) << (32 * (c & 1));
        carry = t >> 32;
    }
    return round_limbs(limb, st, e_lsb);
}

// Column sums of the norm kernel in 24-bit pieces: a column's value is
//   sum_p w[p] * 2^(24 p + e_lsb),  p = 0 .. kNormPieces-1  (240 bits),
// each word receiving addends below 2^32 (a tile's shared-memory piece, or
// one 24-bit piece of a summand).  Summands are below 2^(e_lsb + kWindow).
constexpr int kNormPieces = 10;

// Split v into 24-bit pieces at offset e_lsb: returns the first piece index;
// p[0..3] are the pieces (possibly 0); `lost` flags truncated nonzero bits.
__device__ __forceinline__ int split24(unsigned long long vbits, int e_lsb, unsigned p[4], bool& lost) {
    int E = (int)(vbits >> 52);
    unsigned long long M = vbits & ((1ull << 52) - 1);
    int e;
    if (E) {
        M |= (1ull << 52);
        e = E - 1075;
    } else {
        e = -1074;
    }
    p[0] = p[1] = p[2] = p[3] = 0u;
    lost = false;
    if (M == 0ull) return 0;
    int o = e - e_lsb;
    if (o < 0) {
        const int sh = -o;
        lost = (sh >= 64 ? M : (M & ((1ull << sh) - 1))) != 0ull;
        M = sh >= 64 ? 0ull : (M >> sh);
        if (M == 0ull) return 0;
        o = 0;
    }
    const int L = o / 24, s = o - L * 24;
    const unsigned long long lo = M << s;                 // bits [0, 64) of M * 2^s
    const unsigned long long hi = s ? (M >> (64 - s)) : 0ull;  // bits [64, 77)
    p[0] = (unsigned)(lo & 0xffffffull);
    p[1] = (unsigned)((lo >> 24) & 0xffffffull);
    p[2] = (unsigned)(((lo >> 48) | (hi << 16)) & 0xffffffull);
    p[3] = (unsigned)((hi >> 8) & 0xffffffull);
    return L;
}

// Read, clear and round a column of 24-bit pieces.
__device__ __forceinline__ double round24(unsigned long long* w, size_t stride, unsigned* sticky, int e_lsb) {
    unsigned long long limb[4] = {0ull, 0ull, 0ull, 0ull};
    unsigned long long carry = 0ull;
    // every piece is loaded before any is cleared: the loads are in flight
    // together (a store between them would order each after the last)
    unsigned long long raw[kNormPieces];
#pragma unroll
    for (int p = 0; p < kNormPieces; ++p) raw[p] = __ldcg(w + (size_t)p * stride);
    const bool st = __ldcg(sticky) != 0u;
#pragma unroll
    for (int p = 0; p < kNormPieces; ++p) w[(size_t)p * stride] = 0ull;
    *sticky = 0u;
#pragma unroll
    for (int p = 0; p < kNormPieces; ++p) {
        const unsigned long long t = raw[p] + carry;
        const unsigned long long piece = t & 0xffffffull;
        carry = t >> 24;
        const int bit = 24 * p, li = bit >> 6, sh = bit & 63;
        limb[li] |= piece << sh;
        if (sh > 40) limb[li + 1] |= piece >> (64 - sh);
    }
    return round_limbs(limb, st, e_lsb);
}

// Per-warp sub-allocator of the entry pool: a warp takes `size` entries (or
// the request, if larger) from the shared counter with one atomic and carves
// its rows out of them, so rows cost no contended atomic.  Every request and
// arena is a multiple of 4 entries (rows start 16-byte aligned).  Returns
// the row's first entry, or -1 when the pool is full (recorded in status);
// the counter then keeps counting past the capacity.  The flat scans over a
// step's pool range read every entry of it, so the unused tail of an arena
// is cleared to exact zeros when the warp moves on (arena_close at the end).
struct Arena {
    unsigned long long next = 0, end = 0;
};

__device__ __forceinline__ void arena_close(Arena& a, double* pool_val, int lane) {
    for (unsigned long long q = a.next + lane; q < a.end; q += 32) pool_val[q] = 0.0;
    a.next = a.end = 0;
}

__device__ __forceinline__ long long arena_take(Arena& a, unsigned long long need, unsigned long long size, Ctl* ctl,
                                                double* pool_val, int lane) {
    if (a.next + need > a.end) {
        arena_close(a, pool_val, lane);
        const unsigned long long chunk = need > size ? need : size;
        unsigned long long b = 0ull;
        if (lane == 0) b = atomicAdd(&ctl->pool_used, chunk);
        b = __shfl_sync(kFull, b, 0);
        if (b + chunk > ctl->pool_cap) {
            if (lane == 0) atomicOr(&ctl->status, kDevPoolFull);
            return -1;
        }
        a.next = b;
        a.end = b + chunk;
    }
    const unsigned long long r = a.next;
    a.next += need;
    return (long long)r;
}

// Clear the column sums of columns [j0, n) with stride `step` (all chunks
// and the sticky count).
__device__ __forceinline__ void clear_sums(unsigned long long* words, unsigned* sticky, int n, int j0, int step) {
    for (int j = j0; j < n; j += step) {
#pragma unroll
        for (int c = 0; c < kChunks; ++c) words[(size_t)c * n + j] = 0ull;
        sticky[j] = 0u;
    }
}

// Column sums of a flat scan: an entry whose column lies outside [0, n)
// cannot come from a correct pool; it is skipped and flagged, never used as
// an index.
__device__ __forceinline__ void exact_add_checked(unsigned long long* words, unsigned* sticky, int col, int n,
                                                  unsigned long long vbits, int e_lsb, Ctl* ctl) {
    if ((unsigned)col < (unsigned)n) {
        exact_add(words + col, (size_t)n, sticky + col, vbits, e_lsb);
    } else {
        atomicOr(&ctl->status, kDevInternal);
    }
}
__device__ __forceinline__ void exact_sub_checked(unsigned long long* words, unsigned* sticky, int col, int n,
                                                  unsigned long long vbits, int e_lsb, Ctl* ctl) {
    if ((unsigned)col < (unsigned)n) {
        exact_sub(words + col, (size_t)n, sticky + col, vbits, e_lsb);
    } else {
        atomicOr(&ctl->status, kDevInternal);
    }
}

// Candidate lists of Algorithm 1.  A list holds the entries that can still
// be dropped, and the exact column sums hold exactly the list's entries:
// pass 1 (in the product's write-back) appends and adds every entry with
// 0 < |x| <= eps_g; a later pass with threshold eps_f keeps the entries with
// |x| <= eps_f and subtracts the others from the sums (an entry above eps_f
// stays in the matrix for good, since eps_f only decreases).  A warp reserves
// list space `chunk` entries at a time (one atomic per chunk, so the counter
// is not contended) and clears the unused end of a chunk when it takes the
// next one or finishes: a list entry with |x| bits 0 is a hole.  A list that
// runs out of space sets the overflow flag; its consumer then scans the
// step's pool range instead.

struct CandArena {
    unsigned long long next = 0, end = 0;
};

__device__ __forceinline__ void cand_close(CandArena& a, unsigned long long* out_x, int lane) {
    for (unsigned long long q = a.next + lane; q < a.end; q += 32) out_x[q] = 0ull;
    a.next = a.end = 0;
}

__device__ __forceinline__ void cand_push(CandArena& a, bool keep, int col, unsigned long long xb, int* out_col,
                                          unsigned long long* out_x, unsigned long long* counter,
                                          unsigned long long cap, unsigned chunk, int* over, int lane) {
    const unsigned km = __ballot_sync(kFull, keep);
    if (!km) return;
    const unsigned k = (unsigned)__popc(km);
    if (a.next + k > a.end) {
        cand_close(a, out_x, lane);
        unsigned long long b = 0ull;
        if (lane == 0) b = atomicAdd(counter, (unsigned long long)chunk);
        b = __shfl_sync(kFull, b, 0);
        if (b + chunk > cap) {  // full: the consumer scans the pool instead
            if (lane == 0) *over = 1;
            return;
        }
        a.next = b;
        a.end = b + chunk;
    }
    if (keep) {
        const unsigned long long i = a.next + (unsigned)__popc(km & lanemask_lt());
        out_col[i] = col;
        out_x[i] = xb;
    }
    a.next += k;
}

// Candidates at or below this (bits), eps_g / 2^shift, cannot leave
// Algorithm 1's list while eps_f stays at or above it (0: none are set
// apart).  Exact for normal eps_g: only the exponent changes.
__device__ __forceinline__ unsigned long long far_split(double eps_g, int shift) {
    const unsigned long long gb = (unsigned long long)__double_as_longlong(eps_g);
    return (gb >> 52) > (unsigned long long)shift ? gb - ((unsigned long long)shift << 52) : 0ull;
}

// Grid-wide barrier for cooperative launches, with a bounded wait: after
// `budget_ns` it records kDevTimeout and returns false (a budget of 0 gives
// up at once unless the barrier is already complete: a test of that path).
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned long long budget_ns) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = &ctl->bar_gen;
        unsigned g = *gen;
        __threadfence();
        unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (budget_ns == 0ull || global_ns() - t0 > budget_ns) {
                    atomicOr(&ctl->status, kDevTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace psf
