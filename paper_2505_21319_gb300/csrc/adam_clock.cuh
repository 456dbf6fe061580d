// Adam's step state kept in device memory, for fitting steps that are
// replayed from a CUDA graph: a replayed launch repeats its arguments, so the
// step number t, the bias corrections 1 - beta^t (Sec. 3.4, Adam) and the
// row of the per-step statistics come from this block instead.
#pragma once

#include "common.cuh"

namespace efunc {

struct AdamClock {
    int64_t t;               // step number of the next Adam step (1-based)
    int64_t t_first;         // first step of the call: statistics row t - t_first
    double beta1, beta2, lr;
    double b1t, b2t;         // beta1^t, beta2^t
    float step_size;         // lr / (1 - beta1^t)
    float inv_sqrt_bc2;      // 1 / sqrt(1 - beta2^t)
    unsigned int done;       // blocks of the current Adam launch that have finished
};

// Host-side initial state for step t_first, formed in FP64 exactly as the
// per-launch constants of adam_args are.
AdamClock adam_clock_init(double lr, double beta1, double beta2, int64_t t_first);

// Writes the initial state to clk [device] (one thread).
cudaError_t launch_adam_clock_seed(AdamClock *clk, const AdamClock &init, cudaStream_t s);

// The Adam step of launch_adam with step_size / inv_sqrt_bc2 read from clk;
// when a.stats is set, writes the statistics to a.stats[2 (t - t_first) + 0..1];
// the last block to finish advances clk to step t + 1 (running products
// beta^t in FP64).
cudaError_t launch_adam_clocked(const AdamArgs &a, AdamClock *clk, cudaStream_t s);

}  // namespace efunc
