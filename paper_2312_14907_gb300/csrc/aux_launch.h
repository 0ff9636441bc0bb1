// aux_launch.h -- launchers of the per-pixel and reduction kernels.
#pragma once
#include "mpbp_internal.h"

namespace mpbp {

// Alg. 1 (Adam in the auxiliary variables of Eq. 8), mpbp_alg1.cu
struct AdamArgs {
  float* chi;           // [npix] log density (updated)
  float* u;             // [C][npix] (updated)
  float* alpha_t;       // [D] log peak scalings, entry 0 unused (updated)
  const float* mask;    // [npix] support, or nullptr
  float* rho_x;         // [npix] mask * e^chi (written by prep)
  float* alpha_x;       // [D] (1, e^alpha_t[1..]) (written by prep)
  const float* g_rho;   // df/drho, df/du, df/dalpha of the minibatch
  const float* g_u;
  const double* g_alpha;
  float* m_chi;         // Adam moments
  float* v_chi;
  float* m_u;
  float* v_u;
  double* m_a;
  double* v_a;
  mpbp_adam_state* st;  // parameters, step count, bias corrections
  long long npix;
  int C, D;
};
cudaError_t launch_adam_prep(const AdamArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_adam_update(const AdamArgs& a, int num_sms, cudaStream_t s);

// illumination map: sum over frames of |P_m(r - s_j)|^2 (mpbp_alg1.cu)
struct IllumArgs {
  const cf* probe;       // [Dp][M][M]
  const int2* scan;      // [J]
  float* out;            // [n1][n2], zeroed before the launch
  int nframes, J, m, n1, n2;
  long long probe_stride;   // M*M per peak, or 0; kProbePerScan / kProbePerFrame
                            // (one probe per scan position / per frame)
};
cudaError_t launch_illumination(const IllumArgs& a, int num_sms, cudaStream_t s);

// Probes for scan positions off the pixel grid: out[i] = P_src(i)(k - d_j(i)),
// the band-limited (DFT) interpolation of the source probe, for i = 0 ..
// nout - 1 with j(i) = i mod J and source probe i / J when per_peak (out
// holds D*J probes), else j = i and the single source probe (J probes).
struct ProbeShiftArgs {
  const cf* src;        // [1 or D][M][M]
  cf* out;              // [nout][M][M]
  const float2* d;      // [J] offsets (row, col), |d| <= 1/2
  int nout, J, m;
  bool per_peak;
};
bool probe_shift_prepare(int m);
cudaError_t launch_probe_shift(const ProbeShiftArgs& a, cudaStream_t s);

cudaError_t launch_object_build(const ObjectArgs& a, int num_sms, cudaStream_t s);
// out[i] = in[i] for n 16-bit counts
cudaError_t launch_counts16(const unsigned short* in, float* out, long long n, int num_sms, cudaStream_t s);
cudaError_t launch_frame_transpose(const float* in, float* out, long long nframes, int m,
                                   bool take_sqrt, cudaStream_t s);
int finish_grid(long long npix, int num_sms);
// gradient assembly, then (last block to finish) the reductions and decision;
// with r.step set (and r.st), also the optimizer update of mpbp_step
cudaError_t launch_finish(const FinishArgs& a, const ReduceArgs& r, int grid, cudaStream_t s);
// loss = fixed-order sum of n per-block loss partials (one warp); err gets
// the non-finite bit
cudaError_t launch_loss_reduce(const double* part, long long n, double* loss, int* err, cudaStream_t s);
// the deterministic gradient: acc [D][n1][n2] = per pixel, the fixed-order
// sum of the plan's pieces covering it (pieces w columns wide; plan in
// device memory)
cudaError_t launch_det_reduce(const DetPlan* plan, cf* acc, int D, int n1, int n2, int w, int num_sms,
                              cudaStream_t s);

}  // namespace mpbp
