/* Prints the size and field offsets of the header's structs, one
 * "struct field offset" line per field (and "struct - size"), for the
 * binding's layout test. */
#include <stddef.h>
#include <stdio.h>

#include "psf.h"

#define F(T, f) printf("%s %s %zu\n", #T, #f, offsetof(T, f))
#define S(T) printf("%s - %zu\n", #T, sizeof(T))

int main(void) {
    S(psf_csr_t); F(psf_csr_t, n); F(psf_csr_t, nnz); F(psf_csr_t, rowptr); F(psf_csr_t, col); F(psf_csr_t, val);
    S(psf_info_t); F(psf_info_t, N); F(psf_info_t, q); F(psf_info_t, b); F(psf_info_t, g);
    F(psf_info_t, products); F(psf_info_t, nsteps); F(psf_info_t, z); F(psf_info_t, alpha10);
    F(psf_info_t, trunc); F(psf_info_t, budget); F(psf_info_t, nnz); F(psf_info_t, fma);
    S(psf_step_info_t); F(psf_step_info_t, kind); F(psf_step_info_t, index); F(psf_step_info_t, threshold);
    F(psf_step_info_t, nnz_pre); F(psf_step_info_t, nnz_post); F(psf_step_info_t, eps_f);
    F(psf_step_info_t, iters); F(psf_step_info_t, dropped); F(psf_step_info_t, fma);
    S(psf_server_config_t); F(psf_server_config_t, workers); F(psf_server_config_t, max_batch);
    F(psf_server_config_t, hbm_budget);
    S(psf_completion_t); F(psf_completion_t, tag); F(psf_completion_t, status); F(psf_completion_t, batch_size);
    F(psf_completion_t, result); F(psf_completion_t, queue_ms); F(psf_completion_t, latency_ms);
    S(psf_server_stats_t); F(psf_server_stats_t, submitted); F(psf_server_stats_t, completed);
    F(psf_server_stats_t, failed); F(psf_server_stats_t, batches); F(psf_server_stats_t, max_concurrent);
    F(psf_server_stats_t, pending); F(psf_server_stats_t, budget_peak);
    F(psf_server_stats_t, cancelled);
    S(psf_batch_tune_t); F(psf_batch_tune_t, table_crossover); F(psf_batch_tune_t, row_bitmaps);
    F(psf_batch_tune_t, batch_reuse); F(psf_batch_tune_t, configs); F(psf_batch_tune_t, launches);
    F(psf_batch_tune_t, ms_before); F(psf_batch_tune_t, ms_after);
    return 0;
}
