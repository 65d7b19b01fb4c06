// psf_kernels.h -- host-side launchers of the CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "psf_device.cuh"

namespace psf {

cudaError_t kernels_init();
// wait limit of the cooperative kernels' grid barriers (default 2 s); a wait
// that runs out records kDevTimeout, and the call reports PSF_ETIMEOUT
constexpr unsigned long long kBarrierBudgetDefaultNs = 2000000000ull;
void set_barrier_budget_ns(unsigned long long ns);
unsigned long long barrier_budget_ns();
int num_sms();
long long launch_count();
void count_launches(int k);  // kernels launched by other translation units

// out_len: the expected mean output row length (0: unknown), which picks the
// bitmap map's wide-accumulator instantiation for long rows; wide_window:
// rows are expected to span more columns than the bitmap map covers, which
// picks its wide-window instantiation (16384 columns)
// columns one chunk of the bitmap map covers (the wide window: 16384)
constexpr int kBitmapColumns = 4608;
// cta: one row per block of four warps (k_product_cta), for single-matrix
// steps with long B rows and fewer rows than resident warps
cudaError_t launch_product(const ProductArgs& P, bool table, cudaStream_t st, double out_len = 0.0,
                           bool wide_window = false, bool cta = false);
// column bitmaps of B's rows for the product's symbolic pass
// (ProductArgs::bhdr, bbits); bits has one word per entry of B's index space
cudaError_t launch_row_bitmaps(int n, const RowView& B, int2* hdr, unsigned* bits, cudaStream_t st);
// bytes (a multiple of 4) of device memory at src to dst, the device address
// of pinned, mapped host memory, by a kernel on st (k_export)
cudaError_t launch_export(const void* src, void* dst, size_t bytes, cudaStream_t st);
cudaError_t launch_alg1(const Alg1Args& A, cudaStream_t st);
cudaError_t launch_norms(const NormArgs& A, cudaStream_t st);
cudaError_t launch_absmax(const double* pool_val, const Ctl* ctl, int i, NormSlot* slot, cudaStream_t st);
cudaError_t launch_validate(int n, int nnz, const int* rowptr, const int* col, const double* val, Ctl* ctl,
                            cudaStream_t st);
size_t scan_scratch_len(int n);  // long longs of scratch launch_scan_rows needs
cudaError_t launch_scan_rows(int n, const int* rb, const int* re, int* rowptr, Ctl* ctl, long long* sums,
                             cudaStream_t st);
cudaError_t launch_gather(int n, const RowView& src, const int* rowptr, int* col, double* val,
                          cudaStream_t st);
cudaError_t launch_identity(int n, double alpha, int* rowptr, int* col, double* val, cudaStream_t st);
cudaError_t launch_copy_rows(int n, const int* rowptr, const int* col, const double* val, int* rb, int* re,
                             int* pool_col, double* pool_val, Ctl* ctl, unsigned long long arena_size,
                             cudaStream_t st);
cudaError_t launch_norm_scratch_init(Ctl* ctl, NormSlot* slot, unsigned long long* words, unsigned* sticky, int n,
                                     long long nnz, cudaStream_t st);
// batches (block-diagonal matrix of instances)
constexpr int kMaxBatchInst = 1024;
cudaError_t launch_alg1_batch(const Alg1BatchArgs& A, cudaStream_t st);
cudaError_t launch_inst_table(int n, int ninst, const int* off, int* inst, cudaStream_t st);
cudaError_t launch_validate_batch(int n, const int* inst, const BatchSrc* src, const int* nnz, Ctl* ctl,
                                  cudaStream_t st);
cudaError_t launch_copy_rows_batch(int n, const int* inst, const BatchSrc* src, int* rb, int* re, int* pool_col,
                                   double* pool_val, Ctl* ctl, unsigned long long arena_size, NormSlot* absmax,
                                   int stride, cudaStream_t st);
cudaError_t launch_compose_rows(int n, const int* inst, const int* sel, const int* const* rbs, const int* const* res,
                                int count, int* out_rb, int* out_re, cudaStream_t st);
cudaError_t launch_gather_batch(int n, int ninst, const int* inst, const int* off, const RowView& src,
                                const int* rowptr, int* out_rp, int* col, double* val, cudaStream_t st);
cudaError_t launch_bounds(int ninst, const int* off, const int* rowptr, int* bounds, cudaStream_t st);
cudaError_t launch_reuse_pass1(const ReuseArgs& R, cudaStream_t st);
cudaError_t launch_reuse_copy_batch(const ProductArgs& P, cudaStream_t st);
cudaError_t launch_norms_rows(const NormRowsArgs& A, cudaStream_t st);  // then rounds (k_norms_finish)
// Dense-tile form of a product step (psf_dense.cu): the same output rows,
// statistics and Algorithm 1 first pass as launch_product, through dense
// n x n buffers Ad, Bd, Cd (each n^2 doubles, device).
constexpr int kDenseMaxN = 16384;
cudaError_t launch_dense_product(const ProductArgs& P, double* Ad, double* Bd, double* Cd, cudaStream_t st);
// FP64 rate probe: fp64_probe_blocks() blocks of 256 threads, 8 x iters
// fused multiply-adds per thread, one double per thread written to out
int fp64_probe_blocks();
cudaError_t launch_fp64_probe(int iters, double* out, cudaStream_t st);

}  // namespace psf
