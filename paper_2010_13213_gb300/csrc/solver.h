// solver.h -- host drivers of the Poisson solve and the heat apply (not part of the ABI).
#pragma once
#include "internal.h"

namespace lgf {

Workspace *workspace_for(lgf_table *t, cudaStream_t st);

int solve_poisson(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                  const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st);
int solve_multi(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *phi, int dtype,
                const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st, const lgf_indicator *ind);
int solve_projection(lgf_table *t, const lgf_mesh *m, const void *r, void *u, void *p, int dtype, double alpha,
                     const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st);
int solve_heat(lgf_table *t, const lgf_mesh *m, int ncomp, const void *f, void *g, int dtype,
               double alpha_finest, const lgf_solve_opts &o, lgf_report *rep, cudaStream_t st);

// Phase timer: CUDA events on the call's stream, read back at the end (only when opts.timing).
struct PhaseTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[160];
  int phase_of[160];
  int n = 0;
  void start(bool enable, cudaStream_t s) {
    on = enable;
    st = s;
    n = 0;
    if (on) mark(-1);
  }
  void mark(int phase) {
    if (!on || n >= 160) return;
    cudaEventCreate(&ev[n]);
    cudaEventRecord(ev[n], st);
    phase_of[n] = phase;
    ++n;
  }
  void finish(lgf_report *rep) {
    if (!on) return;
    cudaEventSynchronize(ev[n - 1]);
    if (rep) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[0], ev[n - 1]);
      rep->ms_total = ms;
      for (int i = 1; i < n; ++i) {
        cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
        if (phase_of[i] >= 0 && phase_of[i] < 8) rep->ms_phase[phase_of[i]] += ms;
      }
    }
    for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
    n = 0;
  }
};

inline void phase_mark_cb(void *ctx, int phase) { ((PhaseTimer *)ctx)->mark(phase); }

enum Phase { PH_RESTRICT = 0, PH_CORRECT, PH_FORWARD, PH_MAC, PH_INVERSE, PH_INTERP, PH_RESIDUAL, PH_HEAT };

}  // namespace lgf
