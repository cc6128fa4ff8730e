/* A plain C client of include/dmcr.h, compiled and run by test_c_abi_cpu.py: the header
 * compiles as C, the library links without C++ or CUDA headers, and the host-side calls
 * (no device work) behave as documented.  It prints the size and field offsets of every
 * struct of the header, so that a binding can check its own layout against the C one. */
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "dmcr.h"

#define SIZE(T) printf("size %s %zu\n", #T, sizeof(T))
#define OFF(T, f) printf("offset %s.%s %zu\n", #T, #f, offsetof(T, f))

static dmcr_params params_2d(int64_t n0, int64_t n1, int p0, int p1, int levels) {
    dmcr_params p;
    memset(&p, 0, sizeof(p));
    p.ndim = 2;
    p.n[0] = n0;
    p.n[1] = n1;
    p.window[0] = p0;
    p.window[1] = p1;
    p.levels = levels;
    p.threshold = DMCR_SOFT;
    p.alpha = 10.f;
    p.level_weight_exp = -1.f;
    p.path = DMCR_PATH_AUTO;
    p.descriptor = DMCR_DESC_S2;
    p.phases = 1;
    return p;
}

int main(void) {
    SIZE(dmcr_params);
    OFF(dmcr_params, ndim);
    OFF(dmcr_params, n);
    OFF(dmcr_params, window);
    OFF(dmcr_params, levels);
    OFF(dmcr_params, threshold);
    OFF(dmcr_params, alpha);
    OFF(dmcr_params, level_weight_exp);
    OFF(dmcr_params, path);
    OFF(dmcr_params, tune);
    OFF(dmcr_params, descriptor);
    OFF(dmcr_params, phases);
    SIZE(dmcr_loss_opts);
    OFF(dmcr_loss_opts, mode);
    OFF(dmcr_loss_opts, lambda0);
    OFF(dmcr_loss_opts, bc_on);
    SIZE(dmcr_recon_opts);
    OFF(dmcr_recon_opts, max_iters);
    OFF(dmcr_recon_opts, tol_rel);
    OFF(dmcr_recon_opts, lr);
    OFF(dmcr_recon_opts, beta1);
    OFF(dmcr_recon_opts, beta2);
    OFF(dmcr_recon_opts, eps);
    OFF(dmcr_recon_opts, loss);
    OFF(dmcr_recon_opts, init);
    OFF(dmcr_recon_opts, seed);
    OFF(dmcr_recon_opts, check_every);
    OFF(dmcr_recon_opts, report_rounded);
    SIZE(dmcr_adam_state);
    OFF(dmcr_adam_state, m);
    OFF(dmcr_adam_state, v);
    OFF(dmcr_adam_state, step);
    SIZE(dmcr_recon_report);
    OFF(dmcr_recon_report, iterations);
    OFF(dmcr_recon_report, converged);
    OFF(dmcr_recon_report, loss);
    OFF(dmcr_recon_report, status);
    OFF(dmcr_recon_report, rounded_rel_err);

    printf("version %d\n", dmcr_version());
    /* the 64 x 64, +-16 problem: K_half = (33 * 33 + 1) / 2 = 545 */
    dmcr_params p = params_2d(64, 64, 16, 16, 1);
    int64_t len = -1;
    dmcr_status st = dmcr_descriptor_length(&p, &len);
    printf("length_64_16 %d %lld\n", (int)st, (long long)len);
    /* 512 x 512, +-64, three levels: 3 x 8321 */
    p = params_2d(512, 512, 64, 64, 3);
    st = dmcr_descriptor_length(&p, &len);
    printf("length_512_64_3 %d %lld\n", (int)st, (long long)len);
    size_t ws = 0;
    st = dmcr_workspace_size(&p, &ws);
    printf("workspace_512_64_3 %d %zu\n", (int)st, ws);
    /* a window wider than half the field: EINVAL with a reason */
    p = params_2d(64, 64, 40, 16, 1);
    st = dmcr_descriptor_length(&p, &len);
    printf("invalid %d %d\n", (int)st, (int)(strlen(dmcr_last_error()) > 0));
    /* NULL params */
    st = dmcr_descriptor_length(NULL, &len);
    printf("null_params %d\n", (int)st);
    /* a descriptor call without a workspace is rejected before any launch */
    p = params_2d(64, 64, 4, 4, 1);
    st = dmcr_descriptor(&p, (const float*)0x1000, (float*)0x2000, NULL, 0, NULL);
    printf("null_workspace %d\n", (int)st);
    return 0;
}
