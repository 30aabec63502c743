// Launch-shape autotuner (see lqcd_tune.cu).
#pragma once

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "lqcd_internal.cuh"

struct TuneChoice {
    int variant = 0;   // kernel instantiation (occupancy bound)
    int tx = 128, ty = 1;
    float us = 0;      // measured time of the choice
    int nr = 1;        // fields per thread (register-blocked kernels)
    int kind = 0;      // kernel form (family specific)
};

std::string tune_key(const lqcd_ctx *c, const char *kernel, int mode, int prec, int nrhs);
bool tune_lookup(const std::string &key, TuneChoice *out);
void tune_store(const std::string &key, const TuneChoice &t);
bool tune_enabled();
bool tune_verbose();   // LQCD_TUNE_VERBOSE=1: report every timed candidate on stderr
lqcd_status tune_time(lqcd_ctx *c, const std::function<lqcd_status()> &launch, int reps, float *us);
