// frames_inst.cuh -- prepare/launch functions of the fused frame kernel for
// one frame side M, in the layout chosen for that M:
//   one thread per line (frames_t1) for M <= 16; a thread pair per line
//   (frames_t2) for M >= 32, which halves the registers a line needs and
//   doubles the warps in flight (measured faster from M = 32 up).
#pragma once
#include "frames.cuh"
#include "frames_launch.h"

namespace mpbp {

template <int M>
struct UsePairs {
  static constexpr bool value = M >= 32;
};

template <int M, bool PAIRS = UsePairs<M>::value>
struct FramesKernel;

template <int M>
struct FramesKernel<M, false> {
  using C = T1Cfg<M>;
  static constexpr int T = C::T, SMEM = C::SMEM, NG = C::NG;
  static auto fn(bool fwd) { return fwd ? frames_t1<M, true> : frames_t1<M, false>; }
  static constexpr bool kRaw = false;
  static auto fn_raw() { return frames_t1<M, false>; }
};

template <int M>
struct FramesKernel<M, true> {
  using C = T2Cfg<M>;
  static constexpr int T = C::T, SMEM = C::SMEM, NG = 1;
  static auto fn(bool fwd) { return fwd ? frames_t2<M, true> : frames_t2<M, false>; }
  static constexpr bool kRaw = true;
  static auto fn_raw() { return frames_t2<M, false, true>; }
};

template <int M>
bool frames_prepare_impl(FrameKernelInfo* info) {
  using K = FramesKernel<M>;
  cudaFuncSetAttribute(K::fn(false), cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  cudaFuncSetAttribute(K::fn(true), cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  if (K::kRaw) cudaFuncSetAttribute(K::fn_raw(), cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  info->threads = K::T;
  info->smem = K::SMEM;
  info->frames_per_block = K::NG;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, K::fn(false), K::T, K::SMEM) != cudaSuccess)
    return false;
  info->blocks_per_sm = nb;
  return nb > 0;
}

template <int M>
cudaError_t frames_launch_impl(const FrameArgs& a, int grid, bool forward, cudaStream_t s) {
  using K = FramesKernel<M>;
  K::fn(forward)<<<grid, K::T, K::SMEM, s>>>(a);
  return cudaGetLastError();
}

// the raw-data gradient kernel (FrameArgs::yraw); thread-pair sides only
template <int M>
cudaError_t frames_launch_raw_impl(const FrameArgs& a, int grid, cudaStream_t s) {
  using K = FramesKernel<M>;
  if (!K::kRaw) return cudaErrorNotSupported;
  K::fn_raw()<<<grid, K::T, K::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mpbp

#define MPBP_DEFINE_FRAMES(M)                                                              \
  namespace mpbp {                                                                         \
  bool frames_prepare_m##M(FrameKernelInfo* info) { return frames_prepare_impl<M>(info); } \
  cudaError_t frames_launch_m##M(const FrameArgs& a, int grid, bool forward, cudaStream_t s) { \
    return frames_launch_impl<M>(a, grid, forward, s);                                     \
  }                                                                                        \
  cudaError_t frames_launch_raw_m##M(const FrameArgs& a, int grid, cudaStream_t s) {       \
    return frames_launch_raw_impl<M>(a, grid, s);                                          \
  }                                                                                        \
  }
