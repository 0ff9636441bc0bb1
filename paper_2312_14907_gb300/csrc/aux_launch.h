// aux_launch.h -- launchers of the per-pixel and reduction kernels.
#pragma once
#include "mpbp_internal.h"

namespace mpbp {

struct StepArgs {
  float* rho;
  float* u;
  float* alpha;
  const float* g_rho;
  const float* g_u;
  const double* g_alpha;
  float* rho_base;
  float* u_base;
  float* alpha_base;
  float* g_rho_base;
  float* g_u_base;
  double* g_alpha_base;
  const mpbp_step_state* st;
  long long npix;
  int C, D;
  int alpha_from;
};

cudaError_t launch_object_build(const ObjectArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_frame_transpose(const float* in, float* out, long long nframes, int m,
                                   bool take_sqrt, cudaStream_t s);
int finish_grid(long long npix, int num_sms);
// gradient assembly, then (last block to finish) the reductions and decision
cudaError_t launch_finish(const FinishArgs& a, const ReduceArgs& r, int grid, cudaStream_t s);
cudaError_t launch_step_update(const StepArgs& a, int num_sms, cudaStream_t s);

}  // namespace mpbp
