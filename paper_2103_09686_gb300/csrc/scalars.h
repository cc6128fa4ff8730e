// Per-instance device scalars of an evaluation or reconstruction, and how the host turns
// the ones it copies back into a dmcr_recon_report and a call status.  Plain C++ with no
// CUDA dependency, so the mapping can be compiled and checked by a host-only program.
#pragma once
#include <stdint.h>

#include "dmcr.h"

namespace dmcr {

// Device-side scalars of one evaluation / reconstruction.
struct Scalars {
    float loss[6];        // E, E2, Ebc, lambda, L, rel_err
    float gscale;         // dL/dD = gscale * rho
    float pen_coef;       // penalty gradient coefficient: pen_coef * ex * dex
    float lr_t;           // Adam step size of the current iteration
    int done;             // 0 running, 1 converged, 2 non-finite loss, 3 iteration budget spent
    int iter;             // iterations evaluated in this call
    int64_t adam_step;    // Adam steps taken (global, for bias correction)
    double b1t, b2t;      // beta1^adam_step, beta2^adam_step (running products)
    int err;              // set when a bounded tensor-core wait timed out (any kernel of the instance)
};

// Status of one instance after a run: a timed-out bounded wait outranks a non-finite loss
// (the loss of an instance whose wait gave up is not trustworthy).
inline dmcr_status instance_status(const Scalars& s) {
    if (s.err) return DMCR_ETIMEOUT;
    if (s.done == 2) return DMCR_ENONFINITE;
    return DMCR_OK;
}

// Report of one instance from its scalars copied back after the run; step0 is the Adam
// step count before the call.  rounded_rel_err is filled in separately.
inline void fill_report(const Scalars& s, int64_t step0, dmcr_recon_report* r) {
    r->iterations = (int)(s.adam_step - step0);
    r->converged = s.done == 1;
    for (int k = 0; k < DMCR_OUT_COUNT; ++k) r->loss[k] = s.loss[k];
    r->status = instance_status(s);
}

// Status of a whole call over `count` instances: with per_instance set (the batched
// reconstruction) each instance carries its own status and the call succeeds; otherwise
// the first failing instance's status is the call's (its index goes to *which).
inline dmcr_status call_status(const Scalars* s, int count, bool per_instance, int* which) {
    if (per_instance) return DMCR_OK;
    for (int i = 0; i < count; ++i) {
        const dmcr_status st = instance_status(s[i]);
        if (st != DMCR_OK) {
            if (which != nullptr) *which = i;
            return st;
        }
    }
    return DMCR_OK;
}

}  // namespace dmcr
