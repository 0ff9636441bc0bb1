// unwrap_launch.h -- the phase unwrapper and the projector Pi_U (mpbp_unwrap.cu).
#pragma once
#include "mpbp_internal.h"

namespace mpbp {

// one cooperative launch over D maps of n1 x n2 pixels (nodes = D * npix)
struct UnwrapArgs {
  const float* wrapped;   // [nodes] wrapped phases in [-pi, pi)
  const float* mask;      // [npix] nonzero = inside, or nullptr
  float* out;             // [nodes] unwrapped phases
  float* rel;             // [nodes] pixel reliabilities
  int* parent;            // forest, double-buffered
  int* off;               //   multiple of 2 pi relative to the parent
  int* parent2;
  int* off2;
  int* hook_parent;       // [nodes] the current Boruvka round's hooks of the roots
  int* hook_off;
  int* minnode;           // [nodes] lowest node of each group (at its root)
  unsigned long long* best;   // [nodes] heaviest incident edge of each root
  unsigned long long* ekey;   // [2 nodes] key of edge e = 2 v + dir (0: no edge)
  int* flags;             // [3] rotating "something changed" flags, zeroed before launch
  unsigned* bar_count;    // grid barrier, zeroed before launch
  unsigned* bar_gen;
  int* err;               // kErrTimeout if a barrier wait runs out
  long long npix, nodes;
  int n1, n2;
  int max_rounds;
  int test_stall;         // != 0: block 0 never arrives at a grid barrier (test
                          // of the bounded waits; the result is meaningless)
};

struct ProjectArgs {
  float* u;               // [C][npix], corrected in place
  const float* mask;      // [npix] or nullptr
  float* phi;             // [D][npix] phase_scale G_m . u
  float* wrapped;         // [D][npix] W(phi)
  const float* unwrapped; // [D][npix]
  float g_scaled[kMaxPeaks * kMaxComp];      // phase_scale G[m][c]
  float pinv_scaled[kMaxComp * kMaxPeaks];   // pinv(G)[c][m] / phase_scale
  long long npix;
  int C, D;
};

bool unwrap_prepare(int num_sms, int* grid);
cudaError_t unwrap_launch(const UnwrapArgs& a, int grid, cudaStream_t s);
cudaError_t project_phase_launch(const ProjectArgs& a, int num_sms, cudaStream_t s);
cudaError_t project_correct_launch(const ProjectArgs& a, int num_sms, cudaStream_t s);

}  // namespace mpbp
