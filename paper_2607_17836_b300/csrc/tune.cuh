// The autotuner's timing helpers and search, shared by single flows (api.cu)
// and batches (batch.cu).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "common.cuh"

namespace el {

// Milliseconds per step of `window` steps after two untimed ones, with
// CUDA events on `stream` (re-binning included where it falls due).
template <class StepFn>
el_status time_steps(StepFn step, cudaStream_t stream, int window, double* ms, char* why) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return EL_ECUDA;
    el_status s = step(2);
    if (s == EL_OK) {
        cudaEventRecord(a, stream);
        s = step(window);
        cudaEventRecord(b, stream);
    }
    if (s == EL_OK && cudaEventSynchronize(b) == cudaSuccess) {
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        *ms = t / window;
    } else if (s == EL_OK) {
        s = EL_ECUDA;
        snprintf(why, 128, "event synchronize failed");
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return s;
}

// Event time in ms of whatever fn() enqueues on `stream`.
template <class Fn>
el_status time_call(Fn fn, cudaStream_t stream, double* ms) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return EL_ECUDA;
    cudaEventRecord(a, stream);
    el_status s = fn();
    cudaEventRecord(b, stream);
    if (s == EL_OK && cudaEventSynchronize(b) == cudaSuccess) {
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        *ms = t;
    } else if (s == EL_OK) {
        s = EL_ECUDA;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return s;
}

// The autotuner (shared by single flows and batches).  None of its choices
// changes any result, so its trial windows are ordinary steps.
//  1. block size of the particle step: the fastest of {128, 256, 512} over
//     `trial` steps, each started right after a re-binning, and with the
//     cubic schemes (`cubic`) for each stencil gather (registers, shared);
//  2. re-binning tile: the fastest of {1, 2, 4} cells per side, counting the
//     re-binning cost spread over 40 steps;
//  3. re-binning cadence from a measured model: particles drift out of cell
//     order, so the step time grows about linearly after a re-binning,
//     t(k) = t0 + a k; with re-binning cost c every S steps the mean step time
//     is t0 + a S / 2 + c / S, least at S = sqrt(2 c / a).  t0 and t(W) are
//     timed right after a re-binning and W steps later, c directly.
template <class StepFn, class ApplyFn, class SortFn>
el_status autotune_model(StepFn step, ApplyFn apply, SortFn sort_all, cudaStream_t stream,
                         el_tuning start, int trial, el_tuning* best_out, int n, bool cubic) {
    char why[128] = {0};
    el_tuning best = start;
    best.sort_every = 0;  // the trials below place their own re-binnings
    double best_ms = 1e30;
    const el_tuning base = best;
    for (int g : {EL_GATHER_REGISTERS, EL_GATHER_SHARED}) {
        if (!cubic && g != EL_GATHER_REGISTERS) continue;
        for (int th : {128, 256, 512}) {
            el_tuning t = base;
            t.rk4_threads = th;
            t.gather = cubic ? g : base.gather;
            EL_TRY(apply(t));
            EL_TRY(sort_all());
            double ms = 0.0;
            EL_TRY(time_steps(step, stream, trial, &ms, why));
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    double best_cost = 1e30, sort_ms = 0.0;
    for (int sh : {0, 1, 2}) {
        if ((1 << sh) > n / 4) continue;
        el_tuning t = best;
        t.sort_shift = sh;
        EL_TRY(apply(t));
        double c = 0.0, ms = 0.0;
        EL_TRY(time_call(sort_all, stream, &c));
        EL_TRY(time_steps(step, stream, trial, &ms, why));
        if (ms + c / 40.0 < best_cost) {
            best_cost = ms + c / 40.0;
            best = t;
            sort_ms = c;
        }
    }
    EL_TRY(apply(best));
    const int W = std::max(200, 10 * trial), probe = std::max(10, trial);
    double t0 = 0.0, tw = 0.0;
    EL_TRY(sort_all());
    EL_TRY(time_steps(step, stream, probe, &t0, why));
    EL_TRY(step(W));
    EL_TRY(time_steps(step, stream, probe, &tw, why));
    const double slope = (tw - t0) / (double)(W + probe + 2);
    if (slope > 1e-9 && sort_ms > 0.0) {
        double S = std::sqrt(2.0 * sort_ms / slope);
        best.sort_every = (int)std::min(1000.0, std::max(5.0, std::round(S)));
        best.ms_per_step = t0 + slope * best.sort_every / 2.0 + sort_ms / best.sort_every;
    } else {
        best.sort_every = 0;  // no measurable drift: re-binning never pays
        best.ms_per_step = t0;
    }
    EL_TRY(apply(best));
    *best_out = best;
    return EL_OK;
}

}  // namespace el
