// frames_launch.h -- host entry points of the per-M fused frame kernels.
#pragma once
#include "bulk.cuh"
#include "mpbp_internal.h"

namespace mpbp {

struct FrameKernelInfo {
  int threads;          // threads per block
  int smem;             // dynamic shared memory per block (bytes)
  int frames_per_block; // frames in flight per block
  int blocks_per_sm;    // occupancy limit on the current device
  int tile_w_grad;      // box width (columns) of the objects' tensor map for the
  int tile_w_fwd;       //   gradient / forward kernels' tile copies; 0: none
};

//
// Several problems in one persistent launch.  A work item is one block's worth
// of frames of one problem: 1 frame of M = 128, 2 of M = 64 or 4 of M = 32,
// each on its own group of 2M threads.  Items are taken round-robin; when a
// block's next item has the same frame side its inputs are prefetched during
// the current item, as in the single-problem kernel.  Each warp writes its
// loss partial per frame (fixed slots, so the per-problem sums are
// deterministic).
//
constexpr int kBatchThreads = 256;
constexpr int kBatchWarpSlots = kBatchThreads / 32;   // loss partials per frame
constexpr int kBatchSmem = 128 * 129 * 8 + 128 * 128 * 4;   // the M = 128 frame buffers

// Per-problem arguments travel in the launch's parameter space (constant
// bank), like the single-problem kernel's, so reading them costs no
// registers across a frame; larger batches are split into several launches.
constexpr int kBatchMaxProbs = 48;

struct BatchArgs {
  FrameArgs probs[kBatchMaxProbs];       // per-problem arguments (frames == nullptr)
  int prob_m[kBatchMaxProbs];            // frame side
  long long frame_base[kBatchMaxProbs];  // first slot of the problem in frame_part
  const TmaMap* tmaps;                   // per-side launches with tile copies: [nprob]
                                         // tensor maps (device memory), else nullptr
  const int2* items;                     // [nitems] (problem, first frame)
  double* frame_part;                    // [frames][kBatchWarpSlots] loss partials,
                                         // zeroed before the launch
  int nitems;
  int nprob;
};

// Prepares the batched kernel on the current device; reports its occupancy.
bool batched_prepare(int* blocks_per_sm);
cudaError_t batched_launch(const BatchArgs& b, int grid, cudaStream_t s);

// One launch per frame side: items are single frames of problems with side m.
// tma (m = 32, 64): the inputs by tile and bulk copies, b.tmaps set.
bool batched_m_prepare(int m, bool tma, int* blocks_per_sm);
cudaError_t batched_m_launch(int m, bool tma, const BatchArgs& b, int grid, cudaStream_t s);

// Layout of the M = 128 loss-and-gradient kernel (ignored for other sides):
// radix-2 stages of each 128-point line across four threads by shuffles
// (frames_t4.cuh), or 32 x 4 column and 8 x 16 row factorisations in three
// register layouts joined by shared-memory exchanges (frames_x3.cuh).
enum FrameLayout { kLayoutShuffle = MPBP_FFT_SHUFFLE, kLayoutExchange = MPBP_FFT_EXCHANGE };
constexpr int kLayoutDefault = kLayoutExchange;

// Prepares the kernels of frame side m on the current device (shared-memory
// carve-out) and reports their launch shape.  Returns false for unsupported m.
bool frames_prepare(int m, FrameKernelInfo* info);

// Enqueues the fused kernel for frame side m: forward mode writes I_out,
// otherwise loss partials and the gradient accumulator.  tm: the objects'
// tensor map with the box width the kernel reports (tile_w_*), or nullptr
// for the cp.async copies.
cudaError_t frames_launch(int m, const FrameArgs& a, int grid, bool forward, cudaStream_t s,
                          const TmaMap* tm = nullptr, int layout = kLayoutDefault);

// The loss alone (Eq. 4 over the frames of a, no adjoint and no scatter-add):
// per-block partials in a.loss_part.  tm as for the gradient kernel.
cudaError_t frames_launch_loss(int m, const FrameArgs& a, int grid, cudaStream_t s, const TmaMap* tm = nullptr,
                               int layout = kLayoutDefault);

// Raw-data gradient kernel (a.yraw: counts in their natural layout, device
// memory; sqrt(y) written to a.aT_w).  Frame sides 32, 64, 128.
bool frames_raw_supported(int m);
// tm: tensor maps of the objects and of the staged counts (TmaMap::ymap),
// or nullptr for the cp.async copies.  y16: the staged counts are 16-bit
// unsigned integers (tile copies only; frame sides 64 and 128).
bool frames_raw16_supported(int m);
cudaError_t frames_launch_raw(int m, const FrameArgs& a, int grid, cudaStream_t s, const TmaMap* tm = nullptr,
                              bool y16 = false);

// Tensor-core variant of the gradient kernel for m = 32, 64, 128
// (frames_tc.cu): the DFT passes as split-FP16 GEMMs on tcgen05.  Two 64 x 64
// tiles in flight per 256-thread block: one frame each (m = 64), four
// 32 x 32 frames each (m = 32, with the block-diagonal pair of 32-point DFT
// matrices), or one 128 x 128 frame per tile as four 64 x 64 sub-transforms
// after a radix-2 x 2 step on the CUDA cores (m = 128).
constexpr int kTcThreads = 256;
inline int tc_frames_per_block(int m) { return m == 32 ? 8 : 2; }
constexpr size_t kTcSplitBytes = 2 * 128 * 128 * 2;   // W hi + lo, FP16

// W hi and lo in the kernel's tensor-memory layout (kTcSplitBytes / 4 words,
// host): the 64-point DFT (n = 64) or diag(W32, W32) (n = 32)
void tc_split_dft(uint32_t* out, int n);
// Prepares the kernel on the current device: shared memory, occupancy.
bool tc_prepare(int* blocks_per_sm, int* smem_bytes);
// wsplit: device copy of tc_split_dft's table for frame side m (16-byte aligned).
// test_stall: no MMA is issued and none is committed, so the bounded wait for
// its completion runs out (test of the timeout path; results meaningless).
cudaError_t tc_launch(int m, const FrameArgs& a, const void* wsplit, int grid, cudaStream_t s,
                      bool test_stall = false);

}  // namespace mpbp
