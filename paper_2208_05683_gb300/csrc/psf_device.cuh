// psf_device.cuh -- device-side data structures and helpers shared by the
// CUDA kernels of the filtered PS evaluator.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace psf {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLimbs = 4;     // exact column sums: 256-bit fixed point per column
constexpr int kWindow = 190;  // bits between the fixed point's LSB and 2^E_ref
constexpr int kMinLsb = -1000;
constexpr int kMaxAdd = 24;   // addend terms of one product (PSF_MAX_Q + 1)
constexpr int kMaxNorms = 11; // ||Z^i||_1, i = 0..10

// Device status bits (Ctl::status).
enum : int {
    kDevOk = 0,
    kDevBadInput = 1,
    kDevPoolFull = 2,
    kDevNotConv = 4,
    kDevTimeout = 8,
};

// Control block of one evaluation, in device memory.
struct Ctl {
    unsigned long long pool_used;  // pool entries reserved (keeps counting past capacity)
    unsigned long long pool_cap;
    unsigned long long cslot[2];   // Algorithm 1 column-sum maxima (bits of doubles >= 0)
    unsigned long long nnz_total;  // row-length scan result
    int status;
    unsigned bar_count;  // fields from here on survive a pool reset
    unsigned bar_gen;
    int pad;
    unsigned long long fma_total;  // algorithmic multiply-adds of all products
};

// Device half of psf_step_info_t.
struct StepStat {
    unsigned long long nnz_pre, nnz_post, ncand, fma;
    double eps_f, dropped;
    int iters, pad;
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
    unsigned long long* limbs;  // kLimbs * n
    unsigned* sticky;           // n
    StepStat* stat;
    NormSlot* absmax_slot;      // optional: record max |x|
};

struct Alg1Args {
    int n;
    int* rb;
    int* re;
    int* col;
    double* val;
    double eps_g, bound;
    int maxit, e_lsb;
    unsigned long long* limbs;
    unsigned* sticky;
    Ctl* ctl;
    StepStat* stat;
};

struct NormArgs {
    int n;
    int count;  // matrices
    RowView m[kMaxNorms];
    NormSlot* slots;            // count
    unsigned long long* limbs;  // count * kLimbs * n
    unsigned* sticky;           // count * n
    Ctl* ctl;
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

// Add x at 64-bit limb L of a column whose limbs are `stride` apart, with
// carry propagation.  Concurrent callers may interleave: every carry out of a
// limb is added to the next one exactly once.
__device__ __forceinline__ void limb_add(unsigned long long* limbs, size_t stride, int L,
                                         unsigned long long x) {
    while (x != 0ull && L < kLimbs) {
        unsigned long long old = atomicAdd(limbs + (size_t)L * stride, x);
        x = (old + x < old) ? 1ull : 0ull;
        ++L;
    }
}

// Exact accumulation of v >= 0 (v < 2^(e_lsb + kWindow)) into the column
// whose first limb is at `limbs` (limb stride `stride`).  Bits below 2^e_lsb
// are truncated and noted in `sticky`.
__device__ __forceinline__ void exact_add(unsigned long long* limbs, size_t stride, unsigned* sticky,
                                          double v, int e_lsb) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    int E = (int)(bits >> 52);
    unsigned long long M = bits & ((1ull << 52) - 1);
    int e;
    if (E) {
        M |= (1ull << 52);
        e = E - 1075;
    } else {
        e = -1074;
    }
    if (M == 0ull) return;
    int o = e - e_lsb;
    if (o < 0) {
        int sh = -o;
        unsigned long long lost = sh >= 64 ? M : (M & ((1ull << sh) - 1));
        M = sh >= 64 ? 0ull : (M >> sh);
        if (lost) atomicOr(sticky, 1u);
        if (M == 0ull) return;
        o = 0;
    }
    int L = o >> 6, s = o & 63;
    unsigned long long lo = M << s;
    unsigned long long hi = s ? (M >> (64 - s)) : 0ull;
    limb_add(limbs, stride, L, lo);
    if (hi) limb_add(limbs, stride, L + 1, hi);
}

// Round the fixed-point value sum_l w[l] 2^(64 l + e_lsb) (plus a truncated
// positive remainder when `sticky`) to the nearest double, ties to even.
__device__ __forceinline__ double exact_round(const unsigned long long w[kLimbs], bool sticky,
                                              int e_lsb) {
    int top = -1;
    for (int i = kLimbs - 1; i >= 0; --i)
        if (w[i]) {
            top = i * 64 + 63 - __clzll((long long)w[i]);
            break;
        }
    if (top < 0) return 0.0;
    if (top <= 52) return ldexp((double)w[0], e_lsb);  // < 2^53: exact
    int shift = top - 52;
    int wi = shift >> 6, ws = shift & 63;
    unsigned long long M = w[wi] >> ws;
    if (ws && wi + 1 < kLimbs) M |= w[wi + 1] << (64 - ws);
    M &= (1ull << 53) - 1;
    int rpos = shift - 1;
    int rbit = (int)((w[rpos >> 6] >> (rpos & 63)) & 1ull);
    bool st = sticky;
    if (!st) {
        int sw = rpos >> 6, sb = rpos & 63;
        if (sb && (w[sw] & ((1ull << sb) - 1))) st = true;
        for (int i = 0; i < sw && !st; ++i) st = w[i] != 0ull;
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

// Grid-wide barrier for cooperative launches, with a bounded wait: after
// `budget_ns` it records kDevTimeout and returns false.
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
                if (global_ns() - t0 > budget_ns) {
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
