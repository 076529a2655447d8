// Internal interface between the library's translation units (not exported).
#pragma once
#include <cuda_runtime.h>

#include "pit.h"

// The problem a context holds, for helpers that build a related problem from it.
struct PitProblemView {
    pit_grid grid;
    int M;
    double dt;
    pit_params params;
    pit_options opt;
    const double* u0;  // [Ns] device
    const double* bc;  // [M][2nx+2ny] device, or nullptr for zero Dirichlet data
    const double* q;   // [M][Ns] device, or nullptr for no source
    cudaStream_t stream;
    int wave_teams;      // Newton iterations in flight in pit_solve's wavefront (0: per-stage launches)
    int wave_team_ctas;  // CTAs per wavefront team
};

__attribute__((visibility("hidden"))) void pit_internal_view(const pit_ctx* ctx, PitProblemView* v);
// Record a formatted message as the context's last error and return s.
__attribute__((visibility("hidden"))) pit_status pit_internal_fail(pit_ctx* ctx, pit_status s, const char* fmt, ...);
