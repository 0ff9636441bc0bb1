// frames_batched.cu -- the fused frame kernel over several problems in one
// persistent launch (frame sides 32, 64 and 128).
#include "frames.cuh"
#include "frames_launch.h"

namespace mpbp {

static_assert(kBatchSmem == T2Cfg<128>::SMEM, "batched kernel sized for the M = 128 buffers");

// copy one problem's arguments into shared memory (word by word, by the
// first threads of the block)
MPBP_DI void stage_args(FrameArgs* dst, const FrameArgs* src) {
  constexpr int W = (int)(sizeof(FrameArgs) / sizeof(unsigned));
  static_assert(sizeof(FrameArgs) % sizeof(unsigned) == 0, "word copy");
  if (threadIdx.x < W)
    reinterpret_cast<unsigned*>(dst)[threadIdx.x] = reinterpret_cast<const unsigned*>(src)[threadIdx.x];
}

template <int M>
MPBP_DI void batch_item(const BatchArgs& b, int it, int2 item, bool prefetched,
                        unsigned char* smem, bool& next_prefetched) {
  constexpr int GT = 2 * M;                      // threads per frame
  constexpr int NG = kBatchThreads / GT;         // frames per item
  const int gi = threadIdx.x / GT;
  const T2Group<M> g = T2Group<M>::make(threadIdx.x % GT, NG == 1 ? 0 : 1 + gi,
                                        smem + gi * T2Cfg<M>::SMEM);
  const FrameArgs& p = b.probs[item.x];
  const FrameRef cur = frame_ref(p, item.y + gi);
  if (!prefetched) {
    t2_fetch<M, false>(p, g, cur);
    cp_async_commit();
  }
  // the next item of this block, if it has the same frame side
  const int it2 = it + gridDim.x;
  int2 item2 = make_int2(0, 0);
  bool same = false;
  if (it2 < b.nitems) {
    item2 = b.items[it2];
    same = b.prob_m[item2.x] == M;
  }
  next_prefetched = same;
  const long long slot = (b.frame_base[item.x] + item.y + gi) * kBatchWarpSlots;
  t2_frame<M, false>(
      p, g, cur,
      [&](const FrameArgs*& pn, const TmaMap*&) {
        if (same) {
          pn = &b.probs[item2.x];
          return frame_ref(*pn, item2.y + gi);
        }
        pn = &p;
        return frame_ref(p, p.nframes);   // nothing to fetch
      },
      [&](float fl) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fl += __shfl_xor_sync(0xffffffffu, fl, o);
        if ((g.tid & 31) == 0 && cur.valid) b.frame_part[slot + (g.tid >> 5)] = (double)fl;
      });
}

__global__ void __launch_bounds__(kBatchThreads, 1) frames_batched(const __grid_constant__ BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < b.nprob; i += blockDim.x)
      if (b.probs[i].arrivals) *b.probs[i].arrivals = 0u;
  bool prefetched = false;
  for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
    const int2 item = b.items[it];
    bool nxt = false;
    switch (b.prob_m[item.x]) {
      case 128: batch_item<128>(b, it, item, prefetched, smem_raw, nxt); break;
      case 64: batch_item<64>(b, it, item, prefetched, smem_raw, nxt); break;
      case 32: batch_item<32>(b, it, item, prefetched, smem_raw, nxt); break;
      default: break;
    }
    prefetched = nxt;
    __syncthreads();   // the next item may lay its groups out differently
  }
  cp_async_wait_all();
}

// One persistent launch over the frames of every problem with frame side M
// (items are single frames); the block shape and occupancy are those of the
// single-problem kernel for M.  TMA: the inputs by tile and bulk copies as in
// the single-problem kernel, each problem's objects through its own tensor
// map (b.tmaps, device memory), on the block's mbarrier with the same bounded
// wait; else per-element cp.async.
template <int M, bool TMA>
__global__ void __launch_bounds__(T2Cfg<M>::T, T2Cfg<M>::MINB) frames_batched_m(const __grid_constant__ BatchArgs b) {
  using C = T2Cfg<M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // arguments of the frames' problems, three-way rotated: the slot written at
  // the top of an iteration was last read two frames earlier, and a thread
  // can only be here after every thread has passed that frame's barriers
  __shared__ FrameArgs sp[3];
  __shared__ __align__(8) uint64_t mbar;
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < b.nprob; i += blockDim.x)
      if (b.probs[i].arrivals) *b.probs[i].arrivals = 0u;
  unsigned char* smem = TMA ? smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u) : smem_raw;
  const T2Group<M> g = T2Group<M>::make(threadIdx.x, 0, smem, TMA ? C::TBUF : C::BUF);
  BulkState bs{smem_addr(&mbar), 0u, true};
  int it = blockIdx.x;
  if (it >= b.nitems) return;
  int cs = 0;   // which of sp[] holds the current problem
  FrameRef cur;
  {
    const int2 item = b.items[it];
    stage_args(&sp[0], &b.probs[item.x]);
    if (TMA && threadIdx.x == 0) mbar_init(bs.bar, 1);
    __syncthreads();
    cur = frame_ref(sp[0], item.y);
    t2_fetch<M, false, false, TMA>(sp[0], g, cur, &bs, TMA ? &b.tmaps[item.x] : nullptr);
  }
  if constexpr (!TMA) cp_async_commit();
  for (; it < b.nitems; it += gridDim.x) {
    const int2 item = b.items[it];
    const int it2 = it + gridDim.x;
    const int2 item2 = it2 < b.nitems ? b.items[it2] : make_int2(item.x, 1 << 30);
    const long long slot = (b.frame_base[item.x] + item.y) * kBatchWarpSlots;
    const int ns = cs == 2 ? 0 : cs + 1;
    // visible after the barrier that opens t2_frame
    stage_args(&sp[ns], &b.probs[item2.x]);
    cur = t2_frame<M, false, false, TMA>(
        sp[cs], g, cur,
        [&](const FrameArgs*& pn, const TmaMap*& tmn) {
          pn = &sp[ns];
          if (TMA) tmn = &b.tmaps[item2.x];
          return frame_ref(*pn, item2.y);
        },
        [&](float fl) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) fl += __shfl_xor_sync(0xffffffffu, fl, o);
          if ((g.tid & 31) == 0) b.frame_part[slot + (g.tid >> 5)] = (double)fl;
        },
        &bs, TMA ? &b.tmaps[item.x] : nullptr);
    if (TMA && !bs.ok) {
      if (threadIdx.x == 0) atomicOr(sp[cs].err, kErrTimeout);
      break;
    }
    cs = ns;
  }
  cp_async_wait_all();
}

bool batched_m_prepare(int m, bool tma, int* blocks_per_sm) {
  auto prep = [&](auto kern, int threads, int smem) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return false;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, threads, smem) ==
               cudaSuccess && *blocks_per_sm > 0;
  };
  switch (m) {
    case 32:
      return tma ? prep(frames_batched_m<32, true>, T2Cfg<32>::T, T2Cfg<32>::SMEM_TMA)
                 : prep(frames_batched_m<32, false>, T2Cfg<32>::T, T2Cfg<32>::SMEM);
    case 64:
      return tma ? prep(frames_batched_m<64, true>, T2Cfg<64>::T, T2Cfg<64>::SMEM_TMA)
                 : prep(frames_batched_m<64, false>, T2Cfg<64>::T, T2Cfg<64>::SMEM);
    case 128: return !tma && prep(frames_batched_m<128, false>, T2Cfg<128>::T, T2Cfg<128>::SMEM);
    default: return false;
  }
}

cudaError_t batched_m_launch(int m, bool tma, const BatchArgs& b, int grid, cudaStream_t s) {
  switch (m) {
    case 32:
      if (tma) frames_batched_m<32, true><<<grid, T2Cfg<32>::T, T2Cfg<32>::SMEM_TMA, s>>>(b);
      else frames_batched_m<32, false><<<grid, T2Cfg<32>::T, T2Cfg<32>::SMEM, s>>>(b);
      break;
    case 64:
      if (tma) frames_batched_m<64, true><<<grid, T2Cfg<64>::T, T2Cfg<64>::SMEM_TMA, s>>>(b);
      else frames_batched_m<64, false><<<grid, T2Cfg<64>::T, T2Cfg<64>::SMEM, s>>>(b);
      break;
    case 128:
      if (tma) return cudaErrorInvalidValue;
      frames_batched_m<128, false><<<grid, T2Cfg<128>::T, T2Cfg<128>::SMEM, s>>>(b);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool batched_prepare(int* blocks_per_sm) {
  if (cudaFuncSetAttribute(frames_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem) !=
      cudaSuccess)
    return false;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, frames_batched, kBatchThreads,
                                                       kBatchSmem) == cudaSuccess &&
         *blocks_per_sm > 0;
}

cudaError_t batched_launch(const BatchArgs& b, int grid, cudaStream_t s) {
  frames_batched<<<grid, kBatchThreads, kBatchSmem, s>>>(b);
  return cudaGetLastError();
}

}  // namespace mpbp
