// Host-only check of how a reconstruction's device scalars become a report and a call
// status (paper_2103_09686_gb300/csrc/scalars.h, the code dmcr_reconstruct and
// dmcr_reconstruct_batched run after copying the scalars back).  The error word a bounded
// tensor-core wait sets on the device is preset here, with no GPU involved.  Prints one
// line per case; exits 1 on the first mismatch.
#include <stdio.h>
#include <string.h>

#include "scalars.h"

static int fails = 0;

static void expect(const char* what, long got, long want) {
    printf("%s: %ld (want %ld)\n", what, got, want);
    if (got != want) fails = 1;
}

int main() {
    using dmcr::Scalars;
    Scalars s[3];
    memset(s, 0, sizeof(s));
    for (int i = 0; i < 3; ++i) {
        s[i].adam_step = 40 + i;
        s[i].done = 3;                 // iteration budget spent
        for (int k = 0; k < 6; ++k) s[i].loss[k] = 0.5f * (float)(k + 1);
    }
    s[1].err = 1;                      // instance 1: a bounded wait gave up
    s[2].done = 2;                     // instance 2: non-finite loss
    dmcr_recon_report r;
    memset(&r, 0, sizeof(r));
    dmcr::fill_report(s[1], 10, &r);
    expect("timeout instance status", r.status, DMCR_ETIMEOUT);
    expect("timeout instance iterations", r.iterations, 31);
    expect("timeout instance loss[4] x 2", (long)(2 * r.loss[4]), 5);
    dmcr::fill_report(s[2], 0, &r);
    expect("non-finite instance status", r.status, DMCR_ENONFINITE);
    s[2].err = 1;                      // both: the timed-out wait ranks first
    expect("both", dmcr::instance_status(s[2]), DMCR_ETIMEOUT);
    s[2].err = 0;
    dmcr::fill_report(s[0], 40, &r);
    expect("clean instance status", r.status, DMCR_OK);
    expect("clean instance converged", r.converged, 0);
    int which = -1;
    expect("single call status", dmcr::call_status(s, 3, false, &which), DMCR_ETIMEOUT);
    expect("single call failing instance", which, 1);
    expect("batched call status", dmcr::call_status(s, 3, true, &which), DMCR_OK);
    expect("single call, clean instance only", dmcr::call_status(s, 1, false, &which), DMCR_OK);
    s[0].done = 1;
    dmcr::fill_report(s[0], 40, &r);
    expect("converged instance", r.converged, 1);
    return fails;
}
