// frames_dispatch.cu -- run-time dispatch over the compiled frame sides.
#include "frames_launch.h"

namespace mpbp {

bool frames_prepare_m8(FrameKernelInfo*);
bool frames_prepare_m16(FrameKernelInfo*);
bool frames_prepare_m32(FrameKernelInfo*);
bool frames_prepare_m64(FrameKernelInfo*);
bool frames_prepare_m128(FrameKernelInfo*);
cudaError_t frames_launch_m8(const FrameArgs&, int, bool, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_m16(const FrameArgs&, int, bool, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_m32(const FrameArgs&, int, bool, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_m64(const FrameArgs&, int, bool, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_m128(const FrameArgs&, int, bool, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_loss_m8(const FrameArgs&, int, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_loss_m16(const FrameArgs&, int, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_loss_m32(const FrameArgs&, int, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_loss_m64(const FrameArgs&, int, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_loss_m128(const FrameArgs&, int, cudaStream_t, const TmaMap*, int);
cudaError_t frames_launch_raw_m32(const FrameArgs&, int, cudaStream_t, const TmaMap*, bool);
cudaError_t frames_launch_raw_m64(const FrameArgs&, int, cudaStream_t, const TmaMap*, bool);
cudaError_t frames_launch_raw_m128(const FrameArgs&, int, cudaStream_t, const TmaMap*, bool);

bool frames_prepare(int m, FrameKernelInfo* info) {
  switch (m) {
    case 8: return frames_prepare_m8(info);
    case 16: return frames_prepare_m16(info);
    case 32: return frames_prepare_m32(info);
    case 64: return frames_prepare_m64(info);
    case 128: return frames_prepare_m128(info);
    default: return false;
  }
}

cudaError_t frames_launch(int m, const FrameArgs& a, int grid, bool forward, cudaStream_t s, const TmaMap* tm,
                          int layout) {
  switch (m) {
    case 8: return frames_launch_m8(a, grid, forward, s, tm, layout);
    case 16: return frames_launch_m16(a, grid, forward, s, tm, layout);
    case 32: return frames_launch_m32(a, grid, forward, s, tm, layout);
    case 64: return frames_launch_m64(a, grid, forward, s, tm, layout);
    case 128: return frames_launch_m128(a, grid, forward, s, tm, layout);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t frames_launch_loss(int m, const FrameArgs& a, int grid, cudaStream_t s, const TmaMap* tm, int layout) {
  switch (m) {
    case 8: return frames_launch_loss_m8(a, grid, s, tm, layout);
    case 16: return frames_launch_loss_m16(a, grid, s, tm, layout);
    case 32: return frames_launch_loss_m32(a, grid, s, tm, layout);
    case 64: return frames_launch_loss_m64(a, grid, s, tm, layout);
    case 128: return frames_launch_loss_m128(a, grid, s, tm, layout);
    default: return cudaErrorInvalidValue;
  }
}

// M = 128 takes the staged counts through the transpose kernel and the
// four-threads-per-line kernels (faster than the pair layout's raw-data
// variant, whose 64 values a thread spill)
bool frames_raw_supported(int m) { return m == 32 || m == 64; }

bool frames_raw16_supported(int m) { return m == 64; }

cudaError_t frames_launch_raw(int m, const FrameArgs& a, int grid, cudaStream_t s, const TmaMap* tm,
                              bool y16) {
  switch (m) {
    case 32: return frames_launch_raw_m32(a, grid, s, tm, y16);
    case 64: return frames_launch_raw_m64(a, grid, s, tm, y16);
    case 128: return frames_launch_raw_m128(a, grid, s, tm, y16);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace mpbp
