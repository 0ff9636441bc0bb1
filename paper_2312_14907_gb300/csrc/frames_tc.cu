// frames_tc.cu -- the fused per-frame kernel for M = 64 with the 2-D DFT of
// Eq. 2 computed on the tensor cores (tcgen05.mma, accumulators in TMEM).
//
// Each 1-D pass of the 2-D transform is one real GEMM
//   D[r][n] = sum_K W[r][K] X[n][K],    r = row (q, po),  K = 64 pi + k,
//   W[(q, 0)][k] = cos,  W[(q, 0)][64 + k] = sin,
//   W[(q, 1)][k] = -sin, W[(q, 1)][64 + k] = cos     (theta = 2 pi q k / 64),
// with M = 128 (64 complex outputs, a real and an imaginary row each),
// N = 64 (the other index of the frame) and K = 128 (the real parts of the 64
// inputs, then their imaginary parts).  W is a constant held in tensor memory
// as the A operand; the data X is the B operand in shared memory.  Both are
// split into FP16 hi + lo parts (the data after a per-frame power-of-two
// scaling that brings its maximum into [2^13, 2^14)) and
// D = Wh Xh + Wh Xl + Wl Xh is accumulated in FP32, which keeps about 22
// significant bits of each operand.
//
// Because an accumulator row (q, po) of one pass is the operand row q (part
// po) of the next, each thread writes the next operand straight from its own
// accumulator row (thread t reads TMEM lane t); only the residual and the
// scatter, which need both parts of one value, trade halves with the partner
// lane.  The rows of W, and so the TMEM lanes, are ordered so that lane t
// holds transform row q(t) = (t mod 16) + 16 (t div 32), part po(t) =
// (t div 16) mod 2: the partner is lane t ^ 16 of the same warp, and eight
// neighbouring lanes write eight different operand rows (no bank conflicts).
// Passes:
//   forward   X[k1][k0]  = psi(k0, k1)            -> D = F_0 psi     [(q0,po)][k1]
//             X[q0][k1]  = D                      -> D = Psi         [(q1,po)][q0]
//   residual  (A4) on Psi; its conj(chi) becomes the next operand
//   adjoint   X[q1][q0]  = conj(chi)(q0, q1)      -> D = F_0 conj(chi) [(k0,po)][q1]
//             X[k0][q1]  = D                      -> D = Z           [(k1,po)][k0]
//   scatter   acc_m(s_j + (k0, k1)) += P(k0, k1) Z(k0, k1)      (A6 + A7)
// with Z = F conj(chi) = conj(F^H chi), exactly as in the FFT kernels.
//
// A block runs two frame groups of 128 threads that share W; each has its
// own operand tiles, accumulator columns and completion barrier, so one
// group's CUDA-core work overlaps the other's tensor-core passes.  The next
// frame's object patch and sqrt(y) tile are fetched into shared memory with
// cp.async while the current frame is transformed.
//
// Waits on the MMA completion barriers are bounded in time (0.2 s): when one
// runs out the group records kErrTimeout, skips the rest of its frames and
// the block still frees its tensor memory.
#include <cuda_fp16.h>

#include <cmath>

#include "frames.cuh"
#include "frames_launch.h"

namespace mpbp {

namespace {

constexpr int TM = 64;                  // frame side
constexpr int TK = 128;                 // GEMM K and M: 64 complex values
constexpr int GT = 128;                 // threads per frame group
constexpr int NGROUPS = 2;
constexpr int TC_THREADS = GT * NGROUPS;
constexpr int B_BYTES = TM * TK * 2;    // one FP16 operand tile (16 KB)
constexpr int PATCH_BYTES = TM * TM * 8;
constexpr int AT_BYTES = TM * TM * 4;
constexpr int G_BYTES = 2 * B_BYTES + PATCH_BYTES + AT_BYTES;   // 80 KB per group
constexpr int TC_SMEM = NGROUPS * G_BYTES;
constexpr int W_COLS = TK / 2;          // TMEM columns of one W copy (2 FP16 per column)
constexpr int TMEM_COLS = 256;          // W hi, W lo, one 64-column accumulator per group
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;   // 0.2 s per MMA wait

MPBP_DI uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row r, column k) of a K-major operand without
// swizzle: 8-row x 16-byte core matrices, neighbours along K 128 B apart
// (leading byte offset), row groups TK * 16 B apart (stride byte offset).
MPBP_DI int cm_off(int r, int k) { return ((r >> 3) * (TK / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2; }

MPBP_DI uint64_t smem_desc(uint32_t addr) {
  constexpr uint32_t lbo = 128, sbo = TK * 16;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 D, FP16 A and B (both K-major),
// N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(TM >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

// D (tmem) (+)= A (tmem) * B (smem)
MPBP_DI void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

// 2^e as a float, e in [-126, 127]
MPBP_DI float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// exponent s with mx * 2^s in [2^13, 2^14) for a normal positive mx
// (0 for zero, subnormal or non-finite maxima, which need no rescaling)
MPBP_DI int scale_exp(float mx) {
  const int E = (__float_as_int(mx) >> 23) & 0xff;   // mx >= 0
  if (E == 0 || E == 255) return 0;
  const int s = 140 - E;                             // mx < 2^(E - 126)
  return s > 100 ? 100 : (s < -100 ? -100 : s);
}

// eight consecutive K values of operand row n, scaled by s and split into the
// hi and lo tiles
MPBP_DI void split_store8(unsigned char* bh, unsigned char* bl, int n, int k, const float* v, float s) {
  __align__(16) __half2 h[4];
  __align__(16) __half2 l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 x = make_float2(v[2 * i] * s, v[2 * i + 1] * s);
    h[i] = __float22half2_rn(x);
    const float2 hb = __half22float2(h[i]);
    l[i] = __float22half2_rn(make_float2(x.x - hb.x, x.y - hb.y));
  }
  *reinterpret_cast<uint4*>(bh + cm_off(n, k)) = *reinterpret_cast<const uint4*>(h);
  *reinterpret_cast<uint4*>(bl + cm_off(n, k)) = *reinterpret_cast<const uint4*>(l);
}

// the 64 accumulator columns of this thread's TMEM lane
MPBP_DI void tmem_row64(uint32_t taddr, float (&d)[64]) {
#pragma unroll
  for (int c0 = 0; c0 < 64; c0 += 16) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr + (uint32_t)c0));
#pragma unroll
    for (int j = 0; j < 16; ++j) d[c0 + j] = __uint_as_float(v[j]);
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Partner lanes t and t ^ 16 (accumulator rows (i, 0) and (i, 1): real and
// imaginary part of transform row i) trade halves.  Afterwards the lane of
// part po holds both parts of columns 32 po .. 32 po + 31: re[j], im[j] of
// column 32 po + j.
MPBP_DI void pair_columns(const float (&d)[64], int po, float (&re)[32], float (&im)[32]) {
  const bool hi = po != 0;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float keep = hi ? d[32 + j] : d[j];
    const float send = hi ? d[j] : d[32 + j];
    const float recv = __shfl_xor_sync(0xffffffffu, send, 16);
    re[j] = hi ? recv : keep;
    im[j] = hi ? keep : recv;
  }
}

MPBP_DI float abs_max(float m, float x) { return fmaxf(m, fabsf(x)); }

MPBP_DI void group_bar(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(GT) : "memory"); }

// group barrier that also returns whether v != 0 in every thread of the group
MPBP_DI int group_bar_and(int id, int v) {
  int r;
  asm volatile(
      "{\n.reg .pred q, a;\nsetp.ne.s32 q, %1, 0;\nbar.red.and.pred a, %2, %3, q;\nselp.s32 %0, 1, 0, a;\n}"
      : "=r"(r)
      : "r"(v), "r"(id), "r"(GT)
      : "memory");
  return r;
}

// maximum of non-negative floats over the group (one barrier; slot sets
// alternate between the two uses per frame)
MPBP_DI float group_max(float v, float* red4, int id) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red4[(threadIdx.x >> 5) & 3] = v;
  group_bar(id);
  return fmaxf(fmaxf(red4[0], red4[1]), fmaxf(red4[2], red4[3]));
}

MPBP_DI uint32_t try_wait(uint32_t mbar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(mbar), "r"(phase)
      : "memory");
  return done;
}

MPBP_DI unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// cp.async of 16 bytes, zero-filled when !valid
MPBP_DI void cp_async16z(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

// patch element (k0, k1) in the staging buffer: the column index is XORed
// with 8 for k0 >= 32, so that the two row halves a warp reads at once sit in
// different banks
MPBP_DI int patch_idx(int k0, int k1) { return k0 * TM + (k1 ^ (((k0 >> 5) & 1) << 3)); }
// sqrt(y) tile element (q1, q0) (16-byte chunks of a row XORed with q1 mod 8)
MPBP_DI int at_idx(int q1, int q0) { return q1 * TM + ((((q0 >> 2) ^ (q1 & 7)) << 2) | (q0 & 3)); }

struct TcGroup {
  int id;           // named barrier
  int t;            // thread within the group
  uint32_t dcol;    // TMEM address of the group's accumulator (lane 0)
  uint32_t lane;    // this warp's TMEM lane offset (bits 16+)
  uint32_t wcol;    // TMEM address of W hi (W lo at + W_COLS)
  uint32_t mbar;
  uint32_t phase;
  int ok;           // group-uniform; 0 once a wait has run out
  unsigned char* bh;
  unsigned char* bl;
  cf* patch;
  float* at;
};

// next frame's object patch and sqrt(y) tile into the staging buffers
MPBP_DI void fetch_patch(const FrameArgs& p, const TcGroup& G, const FrameRef& r) {
  const cf* obj = p.O + r.mpk * p.obj_stride;
#pragma unroll 4
  for (int i = 0; i < TM * TM / GT; ++i) {
    const int e = G.t + i * GT;
    const int k0 = e >> 6, k1 = e & 63;
    const int row = r.s.x + k0, col = r.s.y + k1;
    const bool ok = r.valid && row >= 0 && row < p.n1 && col >= 0 && col < p.n2;
    cp_async8(G.patch + patch_idx(k0, k1), ok ? obj + (long long)row * p.n2 + col : obj, ok);
  }
  cp_async_commit();
}

MPBP_DI void fetch_at(const FrameArgs& p, const TcGroup& G, const FrameRef& r) {
  const float* src = p.aT + (long long)r.f * TM * TM;
#pragma unroll
  for (int i = 0; i < TM * TM / 4 / GT; ++i) {
    const int c = G.t + i * GT;   // 16-byte chunk: row c / 16, chunk c % 16
    const int q1 = c >> 4, ch = c & 15;
    cp_async16z(G.at + q1 * TM + ((ch ^ (q1 & 7)) << 2), src + 4 * c, r.valid);
  }
  cp_async_commit();
}

// ---- four 32 x 32 frames per 64 x 64 tile (frame side 32).  With the
// block-diagonal pair diag(W32, W32) in place of W64, each pass transforms
// the tile's four quadrants independently, so frame f = 2 b0 + b1 occupies
// rows 32 b0 .. and columns 32 b1 .. of the tile (b0: the block of k0 / q0,
// b1: the block of k1 / q1).  A thread (column or row rq, part po) always
// touches frame 2 po + (rq >> 5).

// the four frames' object patches into the staging tile
MPBP_DI void fetch_patch4(const FrameArgs& p, const TcGroup& G, const FrameRef (&r)[4]) {
#pragma unroll 4
  for (int i = 0; i < TM * TM / GT; ++i) {
    const int e = G.t + i * GT;
    const int k0 = e >> 6, k1 = e & 63;
    const FrameRef& fr = r[2 * (k0 >> 5) + (k1 >> 5)];
    const cf* obj = p.O + fr.mpk * p.obj_stride;
    const int row = fr.s.x + (k0 & 31), col = fr.s.y + (k1 & 31);
    const bool ok = fr.valid && row >= 0 && row < p.n1 && col >= 0 && col < p.n2;
    cp_async8(G.patch + patch_idx(k0, k1), ok ? obj + (long long)row * p.n2 + col : obj, ok);
  }
  cp_async_commit();
}

// the four frames' sqrt(y) tiles ([q1][q0], 32 x 32 each) into the staging tile
MPBP_DI void fetch_at4(const FrameArgs& p, const TcGroup& G, const FrameRef (&r)[4]) {
#pragma unroll
  for (int i = 0; i < TM * TM / 4 / GT; ++i) {
    const int c = G.t + i * GT;   // 16-byte chunk: row q1 = c / 16, q0 = 4 (c % 16)
    const int q1 = c >> 4, ch = c & 15;
    const FrameRef& fr = r[2 * (ch >> 3) + (q1 >> 5)];
    const float* src = p.aT + (long long)fr.f * 32 * 32 + (q1 & 31) * 32 + 4 * (ch & 7);
    cp_async16z(G.at + q1 * TM + ((ch ^ (q1 & 7)) << 2), src, fr.valid);
  }
  cp_async_commit();
}

// maximum of non-negative floats over the 32 threads of each frame (one
// barrier; slot sets alternate between the two uses per frame): lanes 0..15
// and 16..31 of a warp are parts po = 0, 1, warps 0-1 / 2-3 column blocks
MPBP_DI float group_max4(float v, float* red8, int id, int t) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((t & 15) == 0) red8[(t >> 4) & 7] = v;
  group_bar(id);
  const int po = (t >> 4) & 1, wb = (t >> 6) * 2;
  return fmaxf(red8[wb * 2 + po], red8[(wb + 1) * 2 + po]);
}

// D = Wh Xh + Wh Xl + Wl Xh from the group's operand tiles, then wait
// (bounded) until the accumulator holds it
MPBP_DI void tc_pass(TcGroup& G, int* err, bool stall) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operand stores -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  G.ok = group_bar_and(G.id, G.ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (G.t == 0 && G.ok && !stall) {
    const uint32_t bh = smem_u32(G.bh), bl = smem_u32(G.bl);
#pragma unroll
    for (int prod = 0; prod < 3; ++prod) {
      const uint32_t a = G.wcol + (prod == 2 ? W_COLS : 0);
      const uint32_t b = prod == 1 ? bl : bh;
#pragma unroll
      for (int c = 0; c < TK / 16; ++c)
        mma_ts(G.dcol, a + 8 * c, smem_desc(b + c * 256), (prod > 0 || c > 0) ? 1u : 0u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(G.mbar)
                 : "memory");
  }
}

// one warp polls the completion barrier; the others sleep in the group barrier
MPBP_DI void tc_wait(TcGroup& G, int* err) {
  uint32_t done = 1u;
  if (G.t < 32 && G.ok) {
    done = try_wait(G.mbar, G.phase);
    if (!done) {
      const unsigned long long t0 = global_ns();
      while (!(done = try_wait(G.mbar, G.phase)) && global_ns() - t0 < kWaitNs) {
      }
    }
  }
  G.phase ^= 1u;
  const int ok = group_bar_and(G.id, G.ok && done);
  if (G.ok && !ok && G.t == 0) atomicOr(err, kErrTimeout);
  G.ok = ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

}  // namespace

// W hi (group 0) and W lo (group 1) into TMEM: lane r = W row r
MPBP_DI void tc_load_w(const uint32_t* __restrict__ wsplit, int gi, const TcGroup& G, uint32_t tbase) {
  const uint32_t* src = wsplit + (size_t)gi * TK * W_COLS + (size_t)G.t * W_COLS;
  const uint32_t dst = tbase + G.lane + (uint32_t)(gi * W_COLS);
#pragma unroll
  for (int c0 = 0; c0 < W_COLS; c0 += 16) {
    uint32_t v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __ldg(src + c0 + j);
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            dst + (uint32_t)c0),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// stall != 0: no MMA is issued (test of the bounded completion waits).
// Q4: frame side 32, four frames per group tile (wsplit: diag(W32, W32)).
template <bool Q4>
__global__ void __launch_bounds__(TC_THREADS, 1)
    frames_tc64(const FrameArgs p, const uint32_t* __restrict__ wsplit, int stall) {
  constexpr int FPG = Q4 ? 4 : 1;     // frames per group tile
  constexpr int FS = Q4 ? 32 : TM;    // frame side
  extern __shared__ __align__(16) unsigned char smem_tc[];
  __shared__ uint32_t taddr_holder;
  __shared__ __align__(8) uint64_t mbar[NGROUPS];
  __shared__ float redf[NGROUPS][2][8];
  __shared__ double red[TC_THREADS / 32];
  const int tid = threadIdx.x;
  const int gi = tid / GT;
  if (blockIdx.x == 0 && tid == 0 && p.arrivals) *p.arrivals = 0u;

  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int g = 0; g < NGROUPS; ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[g])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = taddr_holder;

  TcGroup G;
  G.id = 1 + gi;
  G.t = tid % GT;
  G.lane = (uint32_t)((G.t >> 5) * 32) << 16;
  G.wcol = tbase;
  G.dcol = tbase + 2 * W_COLS + TM * gi;
  G.mbar = smem_u32(&mbar[gi]);
  G.phase = 0u;
  G.ok = 1;
  G.bh = smem_tc + gi * G_BYTES;
  G.bl = G.bh + B_BYTES;
  G.patch = reinterpret_cast<cf*>(G.bl + B_BYTES);
  G.at = reinterpret_cast<float*>(G.bh + 2 * B_BYTES + PATCH_BYTES);

  tc_load_w(wsplit, gi, G, tbase);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const int t = G.t;
  const int rq = (t & 15) | ((t >> 5) << 4);   // transform row of this thread's TMEM lane
  const int po = (t >> 4) & 1;                  // its part
  const uint32_t dlane = G.dcol + G.lane;
  double lsum = 0.0;
  float d[64], cre[32], cim[32];

  const int stride = NGROUPS * gridDim.x * FPG;
  int it = (NGROUPS * blockIdx.x + gi) * FPG;
  // the group's frames; this thread's one (fme) and its column within it
  FrameRef curs[FPG];
  for (int f = 0; f < FPG; ++f) curs[f] = frame_ref(p, it + f);
  const int fme = Q4 ? 2 * po + (rq >> 5) : 0;
  const int lc = Q4 ? (rq & 31) : rq;
  if (it < p.nframes) {
    if constexpr (Q4) {
      fetch_patch4(p, G, curs);
      fetch_at4(p, G, curs);
    } else {
      fetch_patch(p, G, curs[0]);
      fetch_at(p, G, curs[0]);
    }
  }
  for (; it < p.nframes && G.ok; it += stride) {
    FrameRef nxts[FPG];
    for (int f = 0; f < FPG; ++f) nxts[f] = frame_ref(p, it + stride + f);
    const bool has_next = it + stride < p.nframes;
    const FrameRef cur = curs[fme];
    const cf* P = frame_probe(p, cur, FS * FS);
    cp_async_wait_all();
    group_bar(G.id);

    // A2: thread (column k1 = rq, half po) forms psi(k0, k1) = P(k0, k1) O_m(s + k)
    // for k0 = 32 po + j and writes operand row k1 (real block, imaginary block)
    int e1;
    {
      float mx = 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int k0 = 32 * po + j;
        const cf v = cmul(ldg_cf(P + (Q4 ? j : k0) * FS + lc), G.patch[patch_idx(k0, rq)]);
        cre[j] = v.x;
        cim[j] = v.y;
        mx = abs_max(abs_max(mx, v.x), v.y);
      }
      e1 = scale_exp(Q4 ? group_max4(mx, redf[gi][0], G.id, t) : group_max(mx, redf[gi][0], G.id));
      const float s = pow2f(e1);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        split_store8(G.bh, G.bl, rq, 32 * po + 8 * c, cre + 8 * c, s);
        split_store8(G.bh, G.bl, rq, 64 + 32 * po + 8 * c, cim + 8 * c, s);
      }
    }
    tc_pass(G, p.err, stall);   // [(q0, po)][k1] = 2^e1 F_0 psi
    if (has_next) {   // every thread is past its patch reads
      if constexpr (Q4) fetch_patch4(p, G, nxts);
      else fetch_patch(p, G, nxts[0]);
    }
    tc_wait(G, p.err);

    // operand row q0 = rq, block po: 2^-6 of the first pass (stays below 2^15)
    if (G.ok) tmem_row64(dlane, d);
#pragma unroll
    for (int c = 0; c < 8; ++c) split_store8(G.bh, G.bl, rq, 64 * po + 8 * c, d + 8 * c, pow2f(-6));
    tc_pass(G, p.err, stall);   // [(q1, po)][q0] = 2^(e1 - 6) Psi
    tc_wait(G, p.err);

    // A4: row q1 = rq of Psi; after the pairing this thread has q0 = 32 po + j
    int e3;
    {
      if (G.ok) tmem_row64(dlane, d);
      pair_columns(d, po, cre, cim);
      const float un = pow2f(6 - e1);
      const float* bg = p.bgT ? (Q4 ? p.bgT + (long long)cur.f * FS * FS + lc * FS
                                    : p.bgT + (long long)cur.f * TM * TM + rq * TM + 32 * po)
                              : nullptr;
      float av[32];
#pragma unroll
      for (int i = 0; i < 8; ++i) {   // q0 = 32 po + 4i .. + 3
        const float4 v = *reinterpret_cast<const float4*>(G.at + at_idx(rq, 32 * po + 4 * i));
        av[4 * i] = v.x;
        av[4 * i + 1] = v.y;
        av[4 * i + 2] = v.z;
        av[4 * i + 3] = v.w;
      }
      float fl = 0.0f, mx = 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float bv = bg ? __ldg(bg + j) : 0.0f;
        const cf z = residual(cf{cre[j] * un, cim[j] * un}, av[j], bv, fl);
        cre[j] = z.x;
        cim[j] = z.y;
        mx = abs_max(abs_max(mx, z.x), z.y);
      }
      if (cur.valid) lsum += 0.5 * (double)fl;
      e3 = scale_exp(Q4 ? group_max4(mx, redf[gi][1], G.id, t) : group_max(mx, redf[gi][1], G.id));
      const float s = pow2f(e3);
#pragma unroll
      for (int c = 0; c < 4; ++c) {   // operand row q1: conj(chi) at q0
        split_store8(G.bh, G.bl, rq, 32 * po + 8 * c, cre + 8 * c, s);
        split_store8(G.bh, G.bl, rq, 64 + 32 * po + 8 * c, cim + 8 * c, s);
      }
    }
    tc_pass(G, p.err, stall);   // [(k0, po)][q1] = 2^e3 F_0 conj(chi)
    if (has_next) {   // every thread is past its sqrt(y) reads
      if constexpr (Q4) fetch_at4(p, G, nxts);
      else fetch_at(p, G, nxts[0]);
    }
    tc_wait(G, p.err);

    if (G.ok) tmem_row64(dlane, d);
#pragma unroll
    for (int c = 0; c < 8; ++c) split_store8(G.bh, G.bl, rq, 64 * po + 8 * c, d + 8 * c, pow2f(-6));
    tc_pass(G, p.err, stall);   // [(k1, po)][k0] = 2^(e3 - 6) Z
    // the probe values of the scatter load while the pass runs
    cf pv[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) pv[j] = ldg_cf(P + (Q4 ? j : 32 * po + j) * FS + lc);
    tc_wait(G, p.err);

    // A6 + A7: Z(k0, k1) for k1 = rq, k0 = 32 po + j
    if (G.ok) {
      tmem_row64(dlane, d);
      pair_columns(d, po, cre, cim);
      const float uz = pow2f(6 - e3);
      const int col = cur.s.y + lc;
      cf* acc = p.acc + cur.mpk * p.obj_stride;
      if (cur.valid && col >= 0 && col < p.n2) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int r = cur.s.x + (Q4 ? 0 : 32 * po) + j;
          if (r >= 0 && r < p.n1) red_add_v2(acc + (long long)r * p.n2 + col, cmul(pv[j], cf{cre[j] * uz, cim[j] * uz}));
        }
      }
    }
    for (int f = 0; f < FPG; ++f) curs[f] = nxts[f];
  }
  cp_async_wait_all();   // copies of a frame this group no longer processes

  const double tot = block_sum_d<TC_THREADS>(lsum, red);
  if (tid == 0) p.loss_part[blockIdx.x] = tot;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

// ----------------------------------------------------------------------------
// Frame side 128: each 2-D transform by one radix-2 x 2 step on the CUDA cores
// and four 64 x 64 tensor-core transforms.  With W = exp(-2 pi i / 128),
// sub-frame (a, b) in {0, 1}^2 and n0, n1, k0, k1 < 64:
//   y_ab(n0, n1) = W^(a n0 + b n1) sum_{i,j} (-1)^(a i + b j) psi(n0 + 64 i, n1 + 64 j)
//   Psi(2 k0 + a, 2 k1 + b) = F64x64[y_ab](k0, k1)
// and for the adjoint, with G_ab = F64x64[conj(chi)(2 k0 + a, 2 k1 + b)],
//   Z(n0 + 64 i, n1 + 64 j) = sum_ab (-1)^(a i + b j) W^(a n0 + b n1) G_ab(n0, n1).
// A group takes one frame and its four sub-frames in turn, each through the
// four passes of the 64 x 64 kernel (W64 in tensor memory); psi is formed
// from the probe and the objects in global memory (L2), the sub-frame's
// sqrt(y) values are gathered with stride 2, and each sub-frame's share of Z
// is scattered to the four quadrants.
// ----------------------------------------------------------------------------
constexpr int T8_G_BYTES = 2 * B_BYTES + AT_BYTES;   // operands + the sub-frame's sqrt(y)
constexpr int TC128_SMEM = NGROUPS * T8_G_BYTES;

// sqrt(y) of sub-frame (a, b): element (q1, q0) of the staging tile = the
// frame's sqrt(y) at (2 q0 + a, 2 q1 + b) (stored [Q1][Q0], 128 x 128)
MPBP_DI void fetch_at_sub(const FrameArgs& p, const TcGroup& G, const FrameRef& r, int a, int b) {
  const float* src = p.aT + (long long)r.f * 128 * 128;
#pragma unroll 4
  for (int i = 0; i < TM * TM / GT; ++i) {
    const int e = G.t + i * GT;
    const int q1 = e >> 6, q0 = e & 63;
    const unsigned d = (unsigned)__cvta_generic_to_shared(G.at + q1 * TM + ((((q0 >> 2) ^ (q1 & 7)) << 2) | (q0 & 3)));
    const float* sp = r.valid ? src + (2 * q1 + b) * 128 + 2 * q0 + a : src;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(sp), "r"(r.valid ? 4 : 0) : "memory");
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    frames_tc128(const FrameArgs p, const uint32_t* __restrict__ wsplit, int stall) {
  constexpr int FS = 128;
  extern __shared__ __align__(16) unsigned char smem_tc[];
  __shared__ uint32_t taddr_holder;
  __shared__ __align__(8) uint64_t mbar[NGROUPS];
  __shared__ float redf[NGROUPS][2][8];
  __shared__ double red[TC_THREADS / 32];
  __shared__ cf w128[FS];   // W^j
  const int tid = threadIdx.x;
  const int gi = tid / GT;
  if (blockIdx.x == 0 && tid == 0 && p.arrivals) *p.arrivals = 0u;
  if (tid < FS) {
    float sn, cs;
    sincospif((float)tid / 64.0f, &sn, &cs);
    w128[tid] = cf{cs, -sn};
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int g = 0; g < NGROUPS; ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[g])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = taddr_holder;

  TcGroup G;
  G.id = 1 + gi;
  G.t = tid % GT;
  G.lane = (uint32_t)((G.t >> 5) * 32) << 16;
  G.wcol = tbase;
  G.dcol = tbase + 2 * W_COLS + TM * gi;
  G.mbar = smem_u32(&mbar[gi]);
  G.phase = 0u;
  G.ok = 1;
  G.bh = smem_tc + gi * T8_G_BYTES;
  G.bl = G.bh + B_BYTES;
  G.patch = nullptr;
  G.at = reinterpret_cast<float*>(G.bh + 2 * B_BYTES);
  tc_load_w(wsplit, gi, G, tbase);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  const int t = G.t;
  const int rq = (t & 15) | ((t >> 5) << 4);   // transform row of this thread's TMEM lane
  const int po = (t >> 4) & 1;                  // its part
  const uint32_t dlane = G.dcol + G.lane;
  double lsum = 0.0;
  float d[64], cre[32], cim[32];

  const int stride = NGROUPS * gridDim.x;
  for (int it = NGROUPS * blockIdx.x + gi; it < p.nframes && G.ok; it += stride) {
    const FrameRef cur = frame_ref(p, it);
    const cf* P = frame_probe(p, cur, FS * FS);
    const cf* obj = p.O + cur.mpk * p.obj_stride;
    for (int ab = 0; ab < 4 && G.ok; ++ab) {
      const int a = ab >> 1, b = ab & 1;
      group_bar(G.id);   // the staging tile's last reads (previous residual) are done
      fetch_at_sub(p, G, cur, a, b);

      // A2: thread (column n1 = rq, half po) forms y_ab(n0, n1), n0 = 32 po + j
      int e1;
      {
        float mx = 0.0f;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
          const int n0 = 32 * po + j;
          cf sum = cf{0.0f, 0.0f};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = q >> 1, jj = q & 1;
            const int r0 = n0 + 64 * i, c0 = rq + 64 * jj;
            const int row = cur.s.x + r0, col = cur.s.y + c0;
            cf psi = cf{0.0f, 0.0f};
            if (cur.valid && row >= 0 && row < p.n1 && col >= 0 && col < p.n2)
              psi = cmul(ldg_cf(P + r0 * FS + c0), ldg_cf(obj + (long long)row * p.n2 + col));
            if ((a * i + b * jj) & 1) sum = csub(sum, psi);
            else sum = cadd(sum, psi);
          }
          const cf v = cmul(sum, w128[(a * n0 + b * rq) & (FS - 1)]);
          cre[j] = v.x;
          cim[j] = v.y;
          mx = abs_max(abs_max(mx, v.x), v.y);
        }
        e1 = scale_exp(group_max(mx, redf[gi][0], G.id));
        const float s = pow2f(e1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          split_store8(G.bh, G.bl, rq, 32 * po + 8 * c, cre + 8 * c, s);
          split_store8(G.bh, G.bl, rq, 64 + 32 * po + 8 * c, cim + 8 * c, s);
        }
      }
      tc_pass(G, p.err, stall);   // [(k0, po)][n1] = 2^e1 F_0 y_ab
      tc_wait(G, p.err);
      if (G.ok) tmem_row64(dlane, d);
#pragma unroll
      for (int c = 0; c < 8; ++c) split_store8(G.bh, G.bl, rq, 64 * po + 8 * c, d + 8 * c, pow2f(-6));
      tc_pass(G, p.err, stall);   // [(k1, po)][k0] = 2^(e1 - 6) Psi(2 k0 + a, 2 k1 + b)
      tc_wait(G, p.err);

      // A4 on Psi(2 q0 + a, 2 q1 + b), q1 = rq, q0 = 32 po + j
      int e3;
      {
        if (G.ok) tmem_row64(dlane, d);
        pair_columns(d, po, cre, cim);
        cp_async_wait_all();
        group_bar(G.id);   // the sub-frame's sqrt(y) values are staged
        const float un = pow2f(6 - e1);
        const float* bg = p.bgT ? p.bgT + (long long)cur.f * FS * FS + (2 * rq + b) * FS + a : nullptr;
        float av[32];
#pragma unroll
        for (int i = 0; i < 8; ++i) {   // q0 = 32 po + 4i .. + 3
          const float4 v = *reinterpret_cast<const float4*>(G.at + at_idx(rq, 32 * po + 4 * i));
          av[4 * i] = v.x;
          av[4 * i + 1] = v.y;
          av[4 * i + 2] = v.z;
          av[4 * i + 3] = v.w;
        }
        float fl = 0.0f, mx = 0.0f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float bv = bg ? __ldg(bg + 2 * (32 * po + j)) : 0.0f;
          const cf z = residual(cf{cre[j] * un, cim[j] * un}, av[j], bv, fl);
          cre[j] = z.x;
          cim[j] = z.y;
          mx = abs_max(abs_max(mx, z.x), z.y);
        }
        if (cur.valid) lsum += 0.5 * (double)fl;
        e3 = scale_exp(group_max(mx, redf[gi][1], G.id));
        const float s = pow2f(e3);
#pragma unroll
        for (int c = 0; c < 4; ++c) {   // operand row q1: conj(chi) at q0
          split_store8(G.bh, G.bl, rq, 32 * po + 8 * c, cre + 8 * c, s);
          split_store8(G.bh, G.bl, rq, 64 + 32 * po + 8 * c, cim + 8 * c, s);
        }
      }
      tc_pass(G, p.err, stall);   // [(n0, po)][q1] = 2^e3 F_0 conj(chi)_ab
      tc_wait(G, p.err);
      if (G.ok) tmem_row64(dlane, d);
#pragma unroll
      for (int c = 0; c < 8; ++c) split_store8(G.bh, G.bl, rq, 64 * po + 8 * c, d + 8 * c, pow2f(-6));
      tc_pass(G, p.err, stall);   // [(n1, po)][n0] = 2^(e3 - 6) G_ab
      tc_wait(G, p.err);

      // A6 + A7: G_ab(n0, n1), n1 = rq, n0 = 32 po + j, to the four quadrants
      if (G.ok) {
        tmem_row64(dlane, d);
        pair_columns(d, po, cre, cim);
        const float uz = pow2f(6 - e3);
        cf* acc = p.acc + cur.mpk * p.obj_stride;
        if (cur.valid) {
#pragma unroll 2
          for (int j = 0; j < 32; ++j) {
            const int n0 = 32 * po + j;
            const cf g = cmul(cf{cre[j] * uz, cim[j] * uz}, w128[(a * n0 + b * rq) & (FS - 1)]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int i = q >> 1, jj = q & 1;
              const int r0 = n0 + 64 * i, c0 = rq + 64 * jj;
              const int row = cur.s.x + r0, col = cur.s.y + c0;
              if (row >= 0 && row < p.n1 && col >= 0 && col < p.n2) {
                const cf z = ((a * i + b * jj) & 1) ? cf{-g.x, -g.y} : g;
                red_add_v2(acc + (long long)row * p.n2 + col, cmul(ldg_cf(P + r0 * FS + c0), z));
              }
            }
          }
        }
      }
    }
  }
  cp_async_wait_all();

  const double tot = block_sum_d<TC_THREADS>(lsum, red);
  if (tid == 0) p.loss_part[blockIdx.x] = tot;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

// W hi and lo as the A operand in tensor memory: [2][128 rows][64 columns],
// column c of a row holding elements 2c (low half) and 2c + 1 (high half);
// row r is transform row (r mod 16) + 16 (r div 32), part (r div 16) mod 2.
// n = 64: the 64-point DFT; n = 32: the block-diagonal pair diag(W32, W32)
// (rows and columns of the two 32-blocks, zero between them).
void tc_split_dft(uint32_t* out, int n) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int r = 0; r < TK; ++r) {
    const int q = (r & 15) | ((r >> 5) << 4), po = (r >> 4) & 1;
    for (int c = 0; c < W_COLS; ++c) {
      uint16_t hv[2], lv[2];
      for (int e = 0; e < 2; ++e) {
        const int K = 2 * c + e, pi = K >> 6, k = K & 63;
        const bool same_block = n == TM || (q >> 5) == (k >> 5);
        const int qq = q % n, kk = k % n;
        const double th = two_pi * (double)((qq * kk) % n) / n;
        const double cs = std::cos(th), sn = std::sin(th);
        const double v0 = po == 0 ? (pi == 0 ? cs : sn) : (pi == 0 ? -sn : cs);
        const double v = same_block ? v0 : 0.0;
        const __half h = __double2half(v);
        const __half l = __double2half(v - (double)__half2float(h));
        hv[e] = __half_as_ushort(h);
        lv[e] = __half_as_ushort(l);
      }
      out[r * W_COLS + c] = (uint32_t)hv[1] << 16 | hv[0];
      out[TK * W_COLS + r * W_COLS + c] = (uint32_t)lv[1] << 16 | lv[0];
    }
  }
}

bool tc_prepare(int* blocks_per_sm, int* smem_bytes) {
  *smem_bytes = TC_SMEM;
  for (auto kern : {frames_tc64<false>, frames_tc64<true>})
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
      return false;
  if (cudaFuncSetAttribute(frames_tc128, cudaFuncAttributeMaxDynamicSharedMemorySize, TC128_SMEM) != cudaSuccess ||
      cudaFuncSetAttribute(frames_tc128, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return false;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, frames_tc64<false>, TC_THREADS, TC_SMEM) !=
      cudaSuccess)
    return false;
  // the tensor memory of every resident block must fit the SM's 512 columns
  if (*blocks_per_sm * TMEM_COLS > 512) *blocks_per_sm = 512 / TMEM_COLS;
  return *blocks_per_sm > 0;
}

cudaError_t tc_launch(int m, const FrameArgs& a, const void* wsplit, int grid, cudaStream_t s, bool test_stall) {
  if (m == 128)
    frames_tc128<<<grid, TC_THREADS, TC128_SMEM, s>>>(a, static_cast<const uint32_t*>(wsplit), test_stall ? 1 : 0);
  else if (m == 32)
    frames_tc64<true><<<grid, TC_THREADS, TC_SMEM, s>>>(a, static_cast<const uint32_t*>(wsplit), test_stall ? 1 : 0);
  else
    frames_tc64<false><<<grid, TC_THREADS, TC_SMEM, s>>>(a, static_cast<const uint32_t*>(wsplit), test_stall ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace mpbp
