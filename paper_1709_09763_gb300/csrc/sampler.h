// Per-handle sampler state (internal): the particles, potentials and scratch on the device, and
// the update scheme's host-side state (controller.cpp; also advanced by the batched sampler).
#pragma once

#include <vector>

#include "handle.h"
#include "smc_device.h"

namespace mls2mc {

struct Sampler {
    int J = 0, K = 0;
    double *theta = nullptr, *theta_p = nullptr, *theta_t = nullptr;
    double *phi_c = nullptr, *phi_f = nullptr, *phi_cp = nullptr, *phi_fp = nullptr;
    double *phi_t0 = nullptr, *phi_t1 = nullptr;
    double *a = nullptr, *cdf = nullptr, *scal = nullptr, *mom = nullptr;
    int *anc = nullptr, *iters = nullptr;
    unsigned long long* n_acc = nullptr;
    IncWork inc;
    // delayed acceptance: surrogate potentials of current particles (s) and proposals (sp),
    // compacted survivors of stage 1, observations of exact solves (training pairs)
    double *G_buf = nullptr, *ps_c = nullptr, *ps_f = nullptr, *psp_c = nullptr, *psp_f = nullptr;
    double *theta_s = nullptr, *phi_cs = nullptr, *phi_fs = nullptr;
    int *surv_idx = nullptr, *n_surv = nullptr, *da_pass = nullptr;
    // covariance-shaped random walk: population mean, covariance partials, covariance, its factor
    double *cmean = nullptr, *cpart = nullptr, *cov = nullptr, *chol = nullptr;
    long long pairs_new[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long da_proposals = 0, da_pass1 = 0;
    // host-side state
    bool started = false;
    int level = 0;
    double beta = 0.0, log_z = 0.0;
    bool prev_lu = true;
    bool terminated = false;   // scheme u': stopped on a level below the finest
    long long stage = 0, mcmc_event = 0;
    double step = 0.0;                 // the Markov kernel's step s for the next update
    long long evals[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<smc_stage_info> path;
};

}  // namespace mls2mc
