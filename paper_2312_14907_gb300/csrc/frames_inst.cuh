// frames_inst.cuh -- prepare/launch functions of the fused frame kernel for
// one frame side M, in the layout chosen for that M:
//   one thread per line (frames_t1) for M <= 16; a thread pair per line
//   (frames_t2) for M >= 32, which halves the registers a line needs and
//   doubles the warps in flight (measured faster from M = 32 up); for the
//   loss and gradient at M = 128, four threads per line (frames_t4), whose
//   32 values a thread fit in registers where the pair's 64 spill.
#pragma once
#include "frames.cuh"
#include "frames_launch.h"
#include "frames_t4.cuh"

namespace mpbp {

template <int M>
struct UsePairs {
  static constexpr bool value = M >= 32;
};

template <int M>
struct UseQuads {
#ifdef MPBP_QUADS_FROM
  static constexpr bool value = M >= MPBP_QUADS_FROM;
#else
  static constexpr bool value = M >= 128;
#endif
};

template <int M, bool PAIRS = UsePairs<M>::value>
struct FramesKernel;

// T, SMEM: the loss-and-gradient kernel; TF, SMEM_F: the forward and the
// raw-data kernels
template <int M>
struct FramesKernel<M, false> {
  using C = T1Cfg<M>;
  static constexpr int T = C::T, SMEM = C::SMEM, NG = C::NG;
  static constexpr int TF = T, SMEM_F = SMEM;
  static auto fn(bool fwd) { return fwd ? frames_t1<M, true> : frames_t1<M, false>; }
  static constexpr bool kRaw = false;
  static auto fn_raw() { return frames_t1<M, false>; }
};

template <int M>
struct FramesKernel<M, true> {
  using C = T2Cfg<M>;
  static constexpr bool kQuads = UseQuads<M>::value;
  using GC = std::conditional_t<kQuads, T4Cfg<M>, T2Cfg<M>>;
  static constexpr int T = GC::T, SMEM = GC::SMEM;
  static constexpr int NG = 1;
  static constexpr int TF = C::T, SMEM_F = C::SMEM;
  static auto fn(bool fwd) {
    if constexpr (kQuads) return fwd ? frames_t2<M, true> : frames_t4<M>;
    else return fwd ? frames_t2<M, true> : frames_t2<M, false>;
  }
  static constexpr bool kRaw = true;
  static auto fn_raw() { return frames_t2<M, false, true>; }
};

template <int M>
bool frames_prepare_impl(FrameKernelInfo* info) {
  using K = FramesKernel<M>;
  cudaFuncSetAttribute(K::fn(false), cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  cudaFuncSetAttribute(K::fn(true), cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM_F);
  if (K::kRaw) cudaFuncSetAttribute(K::fn_raw(), cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM_F);
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
  if (forward) K::fn(true)<<<grid, K::TF, K::SMEM_F, s>>>(a);
  else K::fn(false)<<<grid, K::T, K::SMEM, s>>>(a);
  return cudaGetLastError();
}

// the raw-data gradient kernel (FrameArgs::yraw); thread-pair sides only
template <int M>
cudaError_t frames_launch_raw_impl(const FrameArgs& a, int grid, cudaStream_t s) {
  using K = FramesKernel<M>;
  if (!K::kRaw) return cudaErrorNotSupported;
  K::fn_raw()<<<grid, K::TF, K::SMEM_F, s>>>(a);
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
