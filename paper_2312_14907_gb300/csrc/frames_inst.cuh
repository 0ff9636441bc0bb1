// frames_inst.cuh -- prepare/launch functions of the fused frame kernel for
// one frame side M, in the layout chosen for that M:
//   one thread per line (frames_t1) for M <= 16; a thread pair per line
//   (frames_t2) for M >= 32, which halves the registers a line needs and
//   doubles the warps in flight (measured faster from M = 32 up); for the
//   loss and gradient at M = 128, four threads per line (frames_t4), whose
//   32 values a thread fit in registers where the pair's 64 spill.
#pragma once
#include <algorithm>

#include "frames.cuh"
#include "frames_launch.h"
#include "frames_t4.cuh"
#include "frames_x3.cuh"

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

// The kernels of one frame side: loss and gradient, forward, raw-data
// gradient; the first two also as tile-copy (TMA) instances where the layout
// has one (tile width > 0).
struct KernelShape {
  void (*fn)(const FrameArgs, const TmaMap);
  int threads;
  int smem;
  int tmem_cols = 0;   // tensor-memory columns a block allocates, where the
                       // schedule has to count them (occupancy below)
};

// Resident blocks per SM of kernel k.  For a kernel that allocates a part of
// tensor memory the runtime's calculator answers one block per SM whatever
// the part (measured: four such blocks of 128 columns run together), so the
// count is formed here from its registers (in units of 256 a warp), shared
// memory (with the per-block reservation), threads and columns.
inline bool occupancy(const KernelShape& k, int* blocks) {
  if (k.tmem_cols == 0)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k.fn, k.threads, k.smem) == cudaSuccess;
  cudaFuncAttributes a{};
  int dev = 0, regs = 0, smem = 0, resv = 0, thr = 0, blk = 0;
  if (cudaFuncGetAttributes(&a, k.fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess)
    return false;
  const int warps = (k.threads + 31) / 32;
  const int regs_warp = (a.numRegs * 32 + 255) / 256 * 256;
  const int smem_block = ((int)a.sharedSizeBytes + k.smem + 127) / 128 * 128 + resv;
  int b = regs_warp > 0 ? regs / (warps * regs_warp) : blk;
  b = std::min(b, smem / smem_block);
  b = std::min(b, thr / k.threads);
  b = std::min(b, blk);
  b = std::min(b, 512 / k.tmem_cols);
  *blocks = b;
  return true;
}

// M = 128 loss-and-gradient layouts (FrameLayout): radix-2 stages across
// threads by shuffles (frames_t4) or three register layouts joined by
// shared-memory exchanges (frames_x3)
template <int M>
struct FramesKernel<M, false> {
  using C = T1Cfg<M>;
  static constexpr int NG = C::NG;
  static constexpr int kTileGrad = 0, kTileFwd = 0;
  static KernelShape grad(bool, bool = false, int = 0, bool = false, bool = false) {
    return {frames_t1<M, false>, C::T, C::SMEM};
  }
  static KernelShape fwd(bool) { return {frames_t1<M, true>, C::T, C::SMEM}; }
  static KernelShape loss(bool, bool = false, int = 0, bool = false) {
    return {frames_t1<M, false, true>, C::T, C::SMEM};
  }
  static constexpr bool kRaw = false;
  static constexpr bool kRaw16 = false;
  static KernelShape raw(bool, bool = false) { return grad(false); }
};

template <int M>
struct FramesKernel<M, true> {
  using C = T2Cfg<M>;
  static constexpr bool kQuads = UseQuads<M>::value;
  static constexpr int NG = 1;
  static constexpr int kTileFwd = C::PW;
  static constexpr int kTileGrad = kQuads ? T4Cfg<M>::PW : (C::SWZ ? 0 : C::PW);
  // tpr: the probe stays in tensor memory (four threads per line; probes
  // shared by the frames of a peak)
  static KernelShape grad(bool tma, bool tpr = false, int layout = kLayoutDefault, bool bg = false,
                          bool det = false) {
    if constexpr (kQuads) {
      if (layout == kLayoutExchange && det) {   // deterministic gradient: tile copies only
        return {bg ? frames_x3<true, false, true, true> : frames_x3<true, false, false, true>, X3Cfg::T, X3Cfg::SMEM};
      }
      if (layout == kLayoutExchange) {   // the probe always in tensor memory
        if (bg) return {tma ? frames_x3<true, false, true> : frames_x3<false, false, true>, X3Cfg::T, X3Cfg::SMEM};
        return {tma ? frames_x3<true> : frames_x3<false>, X3Cfg::T, X3Cfg::SMEM};
      }
      if (tpr)
        return {tma ? frames_t4<M, true, false, true> : frames_t4<M, false, false, true>, T4Cfg<M>::T, T4Cfg<M>::SMEM};
      return {tma ? frames_t4<M, true> : frames_t4<M, false>, T4Cfg<M>::T, T4Cfg<M>::SMEM};
    } else if constexpr (C::SWZ) {
      return {frames_t2<M, false>, C::T, C::SMEM};
    } else if constexpr (M == 64) {
      // tile copies: the probe in tensor memory; deterministic gradient: its
      // window beside it (tile copies only)
      if (det) return {frames_t2<M, false, false, true, false, false, true, true>, C::T, C::SMEM_TMA, 2 * M};
      return tma ? KernelShape{frames_t2<M, false, false, true, false, false, true>, C::T, C::SMEM_TMA, M}
                 : KernelShape{frames_t2<M, false>, C::T, C::SMEM};
    } else {
      return tma ? KernelShape{frames_t2<M, false, false, true>, C::T, C::SMEM_TMA}
                 : KernelShape{frames_t2<M, false>, C::T, C::SMEM};
    }
  }
  static KernelShape fwd(bool tma) {
    return tma ? KernelShape{frames_t2<M, true, false, true>, C::T, C::SMEM_TMA}
               : KernelShape{frames_t2<M, true>, C::T, C::SMEM};
  }
  // the loss alone, in the gradient kernel's layout (same tile width)
  static KernelShape loss(bool tma, bool tpr = false, int layout = kLayoutDefault, bool bg = false) {
    if constexpr (kQuads) {
      if (layout == kLayoutExchange) {
        if (bg) return {tma ? frames_x3<true, true, true> : frames_x3<false, true, true>, X3Cfg::T, X3Cfg::SMEM};
        return {tma ? frames_x3<true, true> : frames_x3<false, true>, X3Cfg::T, X3Cfg::SMEM};
      }
      if (tpr)
        return {tma ? frames_t4<M, true, true, true> : frames_t4<M, false, true, true>, T4Cfg<M>::T, T4Cfg<M>::SMEM};
      return {tma ? frames_t4<M, true, true> : frames_t4<M, false, true>, T4Cfg<M>::T, T4Cfg<M>::SMEM};
    } else if constexpr (C::SWZ) {
      return {frames_t2<M, false, false, false, false, true>, C::T, C::SMEM};
    } else {
      return tma ? KernelShape{frames_t2<M, false, false, true, false, true>, C::T, C::SMEM_TMA}
                 : KernelShape{frames_t2<M, false, false, false, false, true>, C::T, C::SMEM};
    }
  }
  // raw-data variants for M = 32, 64 (M = 128 host chunks go through the
  // transpose kernel and the four-threads-per-line kernels)
  static constexpr bool kRaw = M < 128;
  static constexpr bool kRaw16 = M == 64;   // 16-bit counts by tile copies
  static KernelShape raw(bool tma, bool y16 = false) {
    if constexpr (!kRaw) {
      return grad(tma);
    } else {
      if constexpr (kRaw16) {
        if (y16) return {frames_t2<M, false, true, true, true>, C::T, C::SMEM_RAW_TMA};
      }
      return tma ? KernelShape{frames_t2<M, false, true, true>, C::T, C::SMEM_RAW_TMA}
                 : KernelShape{frames_t2<M, false, true>, C::T, C::SMEM};
    }
  }
};

inline bool set_smem(const KernelShape& k) {
  return cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) == cudaSuccess;
}

template <int M>
bool frames_prepare_impl(FrameKernelInfo* info) {
  using K = FramesKernel<M>;
  bool ok = true;
  for (int t = 0; t < 32; ++t)
    ok = set_smem(K::grad(t & 1, (t >> 1) & 1, (t >> 2) & 1, (t >> 3) & 1, t >> 4)) && set_smem(K::fwd(t & 1)) &&
         set_smem(K::loss(t & 1, (t >> 1) & 1, (t >> 2) & 1, (t >> 3) & 1)) && ok;
  if (K::kRaw) ok = set_smem(K::raw(false)) && set_smem(K::raw(true)) && ok;
  if (K::kRaw16) ok = set_smem(K::raw(true, true)) && ok;
  if (!ok) return false;
  info->threads = K::grad(false).threads;
  info->smem = K::grad(false).smem;
  info->frames_per_block = K::NG;
  info->tile_w_grad = K::kTileGrad;
  info->tile_w_fwd = K::kTileFwd;
  // the schedule's blocks per SM must hold for both copy variants and layouts
  int nb = 1 << 20;
  for (int t = 0; t < 4; ++t) {
    const KernelShape k = K::grad(t & 1, false, t >> 1);
    int b = 0;
    if (!occupancy(k, &b)) return false;
    nb = b < nb ? b : nb;
  }
  info->blocks_per_sm = nb;
  return nb > 0;
}

template <int M>
cudaError_t frames_launch_impl(const FrameArgs& a, int grid, bool forward, cudaStream_t s, const TmaMap* tm,
                               int layout) {
  using K = FramesKernel<M>;
  static const TmaMap kNone{};
  const bool tile = tm != nullptr && (forward ? K::kTileFwd : K::kTileGrad) > 0;
  const KernelShape k = forward ? K::fwd(tile)
                                : K::grad(tile, a.probe_stride >= 0, layout, a.bgT != nullptr, a.det != nullptr);
  k.fn<<<grid, k.threads, k.smem, s>>>(a, tile ? *tm : kNone);
  return cudaGetLastError();
}

// the loss alone (no adjoint, no scatter-add)
template <int M>
cudaError_t frames_launch_loss_impl(const FrameArgs& a, int grid, cudaStream_t s, const TmaMap* tm, int layout) {
  using K = FramesKernel<M>;
  static const TmaMap kNone{};
  const bool tile = tm != nullptr && K::kTileGrad > 0;
  const KernelShape k = K::loss(tile, a.probe_stride >= 0, layout, a.bgT != nullptr);
  k.fn<<<grid, k.threads, k.smem, s>>>(a, tile ? *tm : kNone);
  return cudaGetLastError();
}

// the raw-data gradient kernel (FrameArgs::yraw); thread-pair sides only
template <int M>
cudaError_t frames_launch_raw_impl(const FrameArgs& a, int grid, cudaStream_t s, const TmaMap* tm, bool y16) {
  using K = FramesKernel<M>;
  if (!K::kRaw || (y16 && (!K::kRaw16 || !tm))) return cudaErrorNotSupported;
  static const TmaMap kNone{};
  const KernelShape k = K::raw(tm != nullptr, y16);
  k.fn<<<grid, k.threads, k.smem, s>>>(a, tm ? *tm : kNone);
  return cudaGetLastError();
}

}  // namespace mpbp

#define MPBP_DEFINE_FRAMES(M)                                                              \
  namespace mpbp {                                                                         \
  bool frames_prepare_m##M(FrameKernelInfo* info) { return frames_prepare_impl<M>(info); } \
  cudaError_t frames_launch_m##M(const FrameArgs& a, int grid, bool forward, cudaStream_t s, \
                                 const TmaMap* tm, int layout) {                           \
    return frames_launch_impl<M>(a, grid, forward, s, tm, layout);                         \
  }                                                                                        \
  cudaError_t frames_launch_raw_m##M(const FrameArgs& a, int grid, cudaStream_t s,        \
                                     const TmaMap* tm, bool y16) {                         \
    return frames_launch_raw_impl<M>(a, grid, s, tm, y16);                                 \
  }                                                                                        \
  cudaError_t frames_launch_loss_m##M(const FrameArgs& a, int grid, cudaStream_t s,       \
                                      const TmaMap* tm, int layout) {                      \
    return frames_launch_loss_impl<M>(a, grid, s, tm, layout);                             \
  }                                                                                        \
  }
