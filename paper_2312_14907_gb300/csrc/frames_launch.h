// frames_launch.h -- host entry points of the per-M fused frame kernels.
#pragma once
#include "mpbp_internal.h"

namespace mpbp {

struct FrameKernelInfo {
  int threads;          // threads per block
  int smem;             // dynamic shared memory per block (bytes)
  int frames_per_block; // frames in flight per block
  int blocks_per_sm;    // occupancy limit on the current device
};

// Prepares the kernels of frame side m on the current device (shared-memory
// carve-out) and reports their launch shape.  Returns false for unsupported m.
bool frames_prepare(int m, FrameKernelInfo* info);

// Enqueues the fused kernel for frame side m: forward mode writes I_out,
// otherwise loss partials and the gradient accumulator.
cudaError_t frames_launch(int m, const FrameArgs& a, int grid, bool forward, cudaStream_t s);

}  // namespace mpbp
