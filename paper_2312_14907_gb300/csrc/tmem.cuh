// tmem.cuh -- tensor memory (TMEM) as per-thread storage beside the register
// file: allocation by one warp, 32-bit loads and stores of a thread's own
// lane (the 32x32b shape: thread i of a warp reaches lane 32 (warp mod 4) + i
// of the SM's 128 lanes), and the waits and fences that order them.
//
// A warp may only touch the lane quarter of its index modulo 4, so the warps
// w, w + 4, w + 8, ... share lanes and are given disjoint column ranges.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_reg.cuh"

namespace mpbp {

// one warp: allocate ncols columns (a power of two >= 32) and write the base
// address to the shared-memory word at smem_dst; then give up the right to
// allocate more, so that other blocks on the SM are not kept waiting
MPBP_DI void tmem_alloc(uint32_t smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_dst), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// one warp: free what tmem_alloc allocated
MPBP_DI void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

MPBP_DI void tmem_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
MPBP_DI void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// address of lane `lane`, column `col` relative to base
MPBP_DI uint32_t tmem_addr(uint32_t base, uint32_t lane, uint32_t col) { return base + (lane << 16) + col; }

// 16 consecutive columns of the thread's lane (whole warp, converged)
MPBP_DI void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

MPBP_DI void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// 2 consecutive columns (one complex value) of the thread's lane (whole
// warp, converged; taddr's column even)
MPBP_DI void tmem_ld2(uint32_t taddr, uint32_t (&v)[2]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(taddr));
}

MPBP_DI void tmem_st2(uint32_t taddr, uint32_t v0, uint32_t v1) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(v0), "r"(v1) : "memory");
}

// the thread's earlier tcgen05.ld / tcgen05.st have completed
MPBP_DI void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
MPBP_DI void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// eight complex values (16 columns) of the thread's lane
MPBP_DI void tmem_ld_cf8(uint32_t taddr, cf (&out)[8]) {
  uint32_t w[16];
  tmem_ld16(taddr, w);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 8; ++j) out[j] = cf{__uint_as_float(w[2 * j]), __uint_as_float(w[2 * j + 1])};
}

}  // namespace mpbp
