// mpbp_internal.h -- structures shared by the host API and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "fft_reg.cuh"
#include "mpbp.h"

namespace mpbp {

constexpr int kMaxPeaks = 16;
constexpr int kMaxComp = 3;

// device error word bits (the same values as the MPBP_DEVERR_* of mpbp.h)
constexpr int kErrBounds = MPBP_DEVERR_BOUNDS;
constexpr int kErrNonfinite = MPBP_DEVERR_NONFINITE;
constexpr int kErrTimeout = MPBP_DEVERR_TIMEOUT;   // a bounded wait on the GPU ran out

// FrameArgs::probe_stride codes for probes that vary with the scan position
constexpr int kProbePerScan = -1;
constexpr int kProbePerFrame = -2;

// Checks of a problem's geometry, shared by every entry point that takes an
// mpbp_problem: sizes in range, G and phase_scale finite, the pixel and frame
// counts within the kernels' 32-bit indexing.  MPBP_ERR_UNSUPPORTED for a
// frame side the kernels do not cover.
inline mpbp_status validate_problem(const mpbp_problem* pr) {
  if (!pr || !pr->G || !pr->scan) return MPBP_ERR_INVALID_ARG;
  if (pr->n1 < 1 || pr->n2 < 1 || pr->ncomp < 1 || pr->ncomp > kMaxComp || pr->npeaks < 1 ||
      pr->npeaks > kMaxPeaks || pr->nscan < 1 || !std::isfinite(pr->phase_scale))
    return MPBP_ERR_INVALID_ARG;
  if ((long long)pr->n1 * pr->n2 > (1LL << 31) / 16) return MPBP_ERR_INVALID_ARG;
  if ((long long)pr->npeaks * pr->nscan > (1LL << 31) - 1) return MPBP_ERR_INVALID_ARG;
  for (int i = 0; i < pr->npeaks * pr->ncomp; ++i)
    if (!std::isfinite(pr->G[i])) return MPBP_ERR_INVALID_ARG;
  if (pr->m != 8 && pr->m != 16 && pr->m != 32 && pr->m != 64 && pr->m != 128) return MPBP_ERR_UNSUPPORTED;
  return MPBP_OK;
}

// Arguments of the fused per-frame kernel (A2..A7 of the hot path).
struct FrameArgs {
  const cf* O;          // [D][n1][n2] objects O_m
  const cf* probe;      // [Dp][M][M]
  const float* aT;      // [D*J][M][M] sqrt(y), each frame stored transposed [q1][q0]
  const float* bgT;     // same layout as aT, or nullptr
  const int2* scan;     // [J] top-left (row, col)
  const int* frames;    // frame list or nullptr
  cf* acc;              // [D][n1][n2] sum_j P conj(ghat_j), patch-aligned
  double* loss_part;    // [gridDim.x] per-block loss partials
  float* I_out;         // forward mode: [D*J][M][M]
  int* err;             // device error word
  unsigned* arrivals;   // block counter of the gradient assembly that follows;
                        // cleared here, before that kernel can start
  long long obj_stride; // n1*n2
  int nframes;          // frames to process
  int frame0;           // without a frame list: frames frame0 .. frame0 + nframes - 1
  int nframes_total;    // D*J (bound for frame indices)
  int n1, n2, J;
  int probe_stride;     // M*M when one probe per peak, 0 when one for all;
                        // kProbePerScan / kProbePerFrame: one per scan
                        // position j / per frame f, M*M apart (scan
                        // positions off the pixel grid)
  // raw-data variant of the gradient kernel (M >= 32): the measured counts
  // y (natural layout [q0][q1], frame f at yraw + f*M*M) are read instead of
  // the context's sqrt(y), and sqrt(y) is written to aT_w in the context's
  // transposed layout on the way
  const float* yraw;
  float* aT_w;
  // deterministic gradient (M = 128 exchange kernel, every frame of the
  // context in column-strip order): where the gradient window writes back,
  // or nullptr for red.global.add into acc
  const struct DetPlan* det;
};

// One piece of the deterministic gradient: a run of frames of one block that
// share peak and first column (a column strip, or the part of one that a
// block takes).  Its rows [row0, row0 + rows) x columns [y, y + 128) sit at
// pool + off, row-major; the block that owns it adds into it with plain
// loads and stores.
struct DetPiece {
  long long off;   // complex elements into the pool
  int row0, rows;
  int mpk, y;
};

// The deterministic gradient's plan for one grid size: pieces in order,
// each block's first piece, and per (peak, column, band of w rows) the
// pieces reaching into it (CSR: col_start[D * n2 * bands + 1],
// col_piece[...]) in piece order.
struct DetPlan {
  cf* pool;
  const DetPiece* pieces;
  const int* block_piece0;
  const int* col_start;
  const int* col_piece;
};

// Per-pixel coefficients of phi_m = phase_scale * G_m . u.
struct PhaseCoef {
  float kpi[kMaxPeaks][kMaxComp];  // phase_scale * G / pi  (argument of sincospif)
  float kps[kMaxPeaks][kMaxComp];  // phase_scale * G       (d phi_m / d u_c)
};

struct ObjectArgs {
  const float* rho;
  const float* u;
  const float* phi;     // per-peak phases [D][npix] in place of u (or nullptr)
  const float* alpha;
  cf* O;
  long long npix;
  int D, C;
  PhaseCoef pc;
};

// Per-pixel gradient assembly (A6/A7 tail) and its partial sums.
struct FinishArgs {
  const float* rho;
  const float* u;
  const float* phi;     // per-peak phases [D][npix] in place of u (or nullptr):
  float* g_phi;         // then df/dphi_m [D][npix] is written in place of g_u
  const float* alpha;
  cf* acc;              // read, then cleared for the next evaluation
  float* g_rho;
  float* g_u;
  double* part;         // [gridDim.x][D + 3]: df/dalpha_m partials, |g_rho|^2, |g_u|^2, loss
  unsigned* arrivals;   // blocks done (the last one runs the final reduction)
  const double* loss_part;  // the frame kernel's loss partials, summed by slices
  long long n_loss_part;
  long long npix;
  int D, C;
  PhaseCoef pc;
};

// The optimizer update of mpbp_step, applied by the gradient assembly itself:
// x = x_base - t w g_base, where on acceptance the current point and its
// gradient become the base (rho, u, alpha are the iterate, updated in place).
struct StepPtrs {
  float* rho;
  float* u;
  float* alpha;
  float* rho_base;
  float* u_base;
  float* alpha_base;
  float* g_rho_base;
  float* g_u_base;
  double* g_alpha_base;
};

struct ReduceArgs {
  const double* part;
  int n_part;
  int D;
  double* loss_out;
  double* g_alpha_out;  // nullable
  double* g_alpha_ws;   // workspace copy for the optimizer (nullable)
  int* err;
  mpbp_step_state* st;  // nullable: decide an optimizer step
  int alpha_from;       // first alpha index that is a variable (1)
  StepPtrs step;        // with st: the iterate and base point to update
};

}  // namespace mpbp
