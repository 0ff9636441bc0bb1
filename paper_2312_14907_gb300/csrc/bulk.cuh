// bulk.cuh -- the frame kernels' input copies through the tensor memory
// accelerator: the object patch of a frame as one 2-D tile load
// (cp.async.bulk.tensor; rows or columns outside the grid arrive as zeros),
// its sqrt(y) tile as plain bulk copies (or, in the raw-data variant, its
// staged counts as swizzled 2-D tiles), all completing on one mbarrier of
// the block.  One thread issues them; every thread waits with a time limit.
#pragma once
#include <cuda.h>

#include "mpbp_internal.h"

namespace mpbp {

// Tensor map of the objects O [D][n1][n2] (8-byte elements; dimensions n2,
// n1, D), box (w, M, 1).  A tile starts at an even column (16-byte rule of
// the innermost coordinate), so a box is w >= M + 2 columns wide and the
// kernel reads it from column s.y & 1 on.
struct TmaMap {
  CUtensorMap map;
  // raw-data variant: the staged counts of the launch's chunk, [rows][M]
  // floats (16-bit counts), boxes of 32 (64) columns x M rows -- 128 bytes
  // a box row -- with the 128-byte swizzle
  CUtensorMap ymap;
  // bytes announced on a tile-copy barrier beyond what the copies deliver
  // (0; > 0 only to test the bounded wait, which then runs out)
  unsigned tx_extra;
};

constexpr unsigned long long kBulkWaitNs = 200ull * 1000 * 1000;   // 0.2 s

MPBP_DI uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

MPBP_DI unsigned long long timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

MPBP_DI void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the issuing thread's arrival, announcing `bytes` of copies on this phase
MPBP_DI void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

MPBP_DI uint32_t mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done;
}

MPBP_DI void tile_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

MPBP_DI void tile_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// contiguous copy: both addresses 16-byte aligned, bytes a multiple of 16
MPBP_DI void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// a contiguous copy of data read once per evaluation (the frames' sqrt(y)):
// as bulk_load, with an L2 evict-first policy, so that the stream does not
// push the objects and the gradient accumulator out of L2
MPBP_DI void bulk_load_stream(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}

// generic-proxy accesses of shared memory (ordered before this point by a
// barrier) before the asynchronous copies that follow
MPBP_DI void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Every thread of the block: wait (at most kBulkWaitNs) for the phase with
// the given parity; block-uniform result, false if the copies did not land.
MPBP_DI bool bulk_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = mbar_test(bar, parity);
  if (!done) {
    const unsigned long long t0 = timer_ns();
    while (!(done = mbar_test(bar, parity)) && timer_ns() - t0 < kBulkWaitNs) {
    }
  }
  return __syncthreads_and((int)done) != 0;
}

// a block's input copies: its mbarrier and the phase it waits for next
struct BulkState {
  uint32_t bar;      // mbarrier (shared address)
  uint32_t parity;   // phase the next wait is for
  bool ok;           // false once a wait ran out
};

}  // namespace mpbp
