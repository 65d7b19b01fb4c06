/* A C99 caller of the library's host-side entry points (no GPU needed):
 * the header compiles as C, the symbols link, the planner of the 2D
 * Laplacian's exp series gives N = 28, q = 5, b = 6 (Eqs. 6, 34 with
 * z_i = 4^i), and a bad argument returns PSF_EINVAL with a message. */
#include <stdio.h>
#include <string.h>

#include "psf.h"

static int fail(const char* what) {
    printf("FAIL %s: %s\n", what, psf_last_error());
    return 1;
}

int main(void) {
    double a[40], norms[11], zeta[PSF_MAX_Q + 2], sigma[PSF_MAX_Q + 2], v = 0.0, f = 1.0;
    psf_info_t info;
    psf_series_t s = NULL;
    int i;
    if (psf_version() < 1) return fail("version");
    for (i = 0; i < 40; ++i) {  /* 1 / i! */
        a[i] = 1.0 / f;
        f *= (double)(i + 1);
    }
    norms[0] = 1.0;
    for (i = 1; i <= 10; ++i) norms[i] = norms[i - 1] * 4.0;
    if (psf_plan(a, 40, 0, 1e-12, PSF_SERIES, norms, &info, zeta, sigma) != PSF_OK) return fail("plan");
    if (info.N != 28 || info.q != 5 || info.b != 6 || info.products != 9) return fail("plan values");
    if (!(info.budget > 0.0 && info.budget < 1e-12) || !(sigma[1] > 0.0)) return fail("budget and thresholds");
    if (psf_series_create(a, 40, 0, 1e-12, PSF_SERIES, &s) != PSF_OK || s == NULL) return fail("create");
    if (psf_series_set_param(s, PSF_PARAM_ER, 0.2) != PSF_OK) return fail("set_param");
    if (psf_series_destroy(s) != PSF_OK) return fail("destroy");
    if (psf_series_create(a, 40, 0, 0.0, PSF_SERIES, &s) != PSF_EINVAL || s != NULL) return fail("bad tol accepted");
    if (strlen(psf_last_error()) == 0) return fail("no message");
    if (psf_tune_get(PSF_TUNE_ALG1_FAR_SHIFT, &v) != PSF_OK || v != 6.0) return fail("tune_get");
    printf("ok N=%d q=%d b=%d products=%d\n", info.N, info.q, info.b, info.products);
    return 0;
}
