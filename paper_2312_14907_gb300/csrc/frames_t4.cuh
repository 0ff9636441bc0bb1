// frames_t4.cuh -- the fused frame kernel (A2-A7 of frames.cuh) with four
// threads per line (fft_quad.cuh): M/4 values per thread, 4M threads and one
// frame per block.
//
// A warp holds eight lines: lane = 8 h + (ln mod 8), so the four threads of a
// line are lanes l, l^8, l^16, l^24 and every exchange of the line FFTs is a
// shuffle.  The exchange buffer has no padding; the column index of row r is
// XOR-swizzled with
//   sw(r) = (r & 6) | 8 (bit 0 of r  XOR  bit b of r),   b = log2(M/4),
// which keeps every 16-lane half of a warp on distinct 8-byte
// banks for the three access patterns the kernel has:
//   column ln, rows 4n + h    (the patch, the dec4 input of a column pass),
//   column ln, rows Q g + t   (the blk4 output of a column pass: the rows of
//                              the two halves differ by M/4, bit b),
//   row ln, columns 4n + h    (the transposed dec4 input of a row pass).
// The sqrt(y) tile [q1][q0] is staged with its 16-byte chunks XORed with
// 2 ((q1 / Q) mod 4), so the four rows Q g + t that one warp reads at eight
// consecutive q0 fall in different banks.
#pragma once
#include "fft_quad.cuh"
#include "frames.cuh"

namespace mpbp {

template <int M>
struct T4Cfg {
  static constexpr int T = 4 * M;     // threads per block (one frame)
  static constexpr int H = M / 4;     // values per thread
  static constexpr int Q = M / 8;
  static constexpr int B = ct::ilog2(M / 4);
  static constexpr int BUF = M * M * (int)sizeof(cf);
  static constexpr int ABUF = M * M * (int)sizeof(float);
  static constexpr int SMEM = BUF + ABUF;
  static_assert(M == 32 || M == 64 || M == 128, "four threads per line: M = 32, 64 or 128");
};

MPBP_DI cf xchg8(cf v) {
  return cf{__shfl_xor_sync(0xffffffffu, v.x, 8), __shfl_xor_sync(0xffffffffu, v.y, 8)};
}

template <int M>
MPBP_DI int t4_at(int r, int c) {
  constexpr int B = T4Cfg<M>::B;
  return r * M + (c ^ ((r & 6) | (((r ^ (r >> B)) & 1) << 3)));
}

// the frame's sqrt(y) tile, 16-byte chunks swizzled by row band
template <int M>
MPBP_DI void t4_fetch_amp(const PatchSrc& q, int t, float* dst) {
  if (!q.amp) return;
  constexpr int CH = M * M / 4, CPR = M / 4, NT = T4Cfg<M>::T, QQ = T4Cfg<M>::Q;
  static_assert(CH % NT == 0, "tile chunks must divide among the threads");
#pragma unroll
  for (int i = 0; i < CH / NT; ++i) {
    const int c = t + i * NT;
    const int row = c / CPR, cc = c - row * CPR;
    cp_async16(dst + 4 * (row * CPR + (cc ^ (2 * ((row / QQ) & 3)))), q.amp + 4 * c);
  }
}

template <int M>
MPBP_DI float t4_amp_at(const float* abuf, int q1, int q0) {
  constexpr int QQ = T4Cfg<M>::Q;
  return abuf[q1 * M + 4 * ((q0 >> 2) ^ (2 * ((q1 / QQ) & 3))) + (q0 & 3)];
}

template <int M>
struct T4Group {
  int tid;
  int ln;          // line (column or row) index
  int h, h0, h1;   // quarter of the line: h = 2 h1 + h0
  cf* buf;         // exchange buffer [M][M], swizzled
  float* abuf;     // sqrt(y) staging [M][M], swizzled
  MPBP_DI static T4Group make(int tid, unsigned char* smem) {
    T4Group g;
    g.tid = tid;
    const int lane = tid & 31;
    g.ln = (tid >> 5) * 8 + (lane & 7);
    g.h = lane >> 3;
    g.h0 = g.h & 1;
    g.h1 = g.h >> 1;
    g.buf = reinterpret_cast<cf*>(smem);
    g.abuf = reinterpret_cast<float*>(smem + T4Cfg<M>::BUF);
    return g;
  }
  // index of blk4 slot i (compile-time i)
  MPBP_DI int blk(int i) const {
    constexpr int Q = T4Cfg<M>::Q;
    const int g = 2 * h0 + h1;
    return i < Q ? Q * g + i : M / 2 + Q * g + (i - Q);
  }
};

template <int M>
MPBP_DI void t4_fetch(const FrameArgs& p, const T4Group<M>& g, const FrameRef& r) {
  const PatchSrc q = patch_src<M>(p, r);
  sfor<0, T4Cfg<M>::H>([&](auto n_) {
    constexpr int n = decltype(n_)::value;
    const int k0 = 4 * n + g.h;
    fetch_patch_elem(q, k0, g.ln, g.buf + t4_at<M>(k0, g.ln));
  });
  t4_fetch_amp<M>(q, g.tid, g.abuf);
}

// One frame's loss and gradient (inputs in flight, committed); fetches the
// next frame's inputs as soon as their buffers are free.
template <int M, typename AddLoss>
MPBP_DI FrameRef t4_frame(const FrameArgs& p, const T4Group<M>& g, const FrameRef& cur, const FrameRef& nxt,
                          AddLoss&& add_loss) {
  using C = T4Cfg<M>;
  constexpr int H = C::H;
  cf* buf = g.buf;
  const int ln = g.ln, h = g.h;
  auto x8 = [](cf v) { return xchg8(v); };
  auto x16 = [](cf v) { return xchg16(v); };
  const cf* P = p.probe + cur.mpk * p.probe_stride;
  const int col = cur.s.y + ln;
  const bool cok = cur.valid && col >= 0 && col < p.n2;
  cp_async_wait_all();
  __syncthreads();

  // A2: column ln, rows 4n + h
  cf v[H];
  sfor<0, H>([&](auto n_) {
    constexpr int n = decltype(n_)::value;
    const int k0 = 4 * n + h;
    v[n] = cmul(ldg_cf(P + k0 * M + ln), buf[t4_at<M>(k0, ln)]);
  });

  // A3: columns, transpose, rows
  fft_quad_dec_to_blk<M>(v, g.h0, g.h1, x8, x16);
  __syncwarp();   // the other three threads of the line read the rows this thread writes
  sfor<0, H>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    buf[t4_at<M>(g.blk(i), ln)] = v[i];
  });
  __syncthreads();
  sfor<0, H>([&](auto n_) {
    constexpr int n = decltype(n_)::value;
    v[n] = buf[t4_at<M>(ln, 4 * n + h)];
  });
  fft_quad_dec_to_blk<M>(v, g.h0, g.h1, x8, x16);
  // row ln: Psi[ln][blk(i)] in slot i

  // A4
  const float* b = p.bgT ? p.bgT + (long long)cur.f * M * M : nullptr;
  float fl = 0.0f;
  sfor<0, H>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const int q1 = g.blk(i);
    const float bv = b ? b[q1 * M + ln] : 0.0f;
    v[i] = residual(v[i], t4_amp_at<M>(g.abuf, q1, ln), bv, fl);
  });
  add_loss(cur.valid ? fl : 0.0f);

  // A5: rows (blk4 -> dec4), transpose, columns; the exchange buffer's last
  // reads (the transposed row input above) are behind this barrier
  fft_quad_blk_to_dec<M>(v, g.h0, g.h1, x8, x16);   // Z'[ln][4k + h] in slot brev(k)
  __syncthreads();
  sfor<0, H>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    buf[t4_at<M>(ln, 4 * k + h)] = v[ct::brev<H>(k)];
  });
  __syncthreads();
  const PatchSrc q = patch_src<M>(p, nxt);
  t4_fetch_amp<M>(q, g.tid, g.abuf);   // every thread is past its residual
  sfor<0, H>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    v[i] = buf[t4_at<M>(g.blk(i), ln)];
  });
  __syncthreads();
  // the exchange buffer is free again; a rolled loop here keeps the copies'
  // addresses out of the registers the values need (unrolled, they spill)
#pragma unroll 2
  for (int n = 0; n < H; ++n) {
    const int k0 = 4 * n + h;
    fetch_patch_elem(q, k0, ln, buf + t4_at<M>(k0, ln));
  }
  cp_async_commit();
  fft_quad_blk_to_dec<M>(v, g.h0, g.h1, x8, x16);   // Z[4k + h][ln] in slot brev(k)

  // A6 + A7
  cf* acc = p.acc + cur.mpk * p.obj_stride;
  sfor<0, H>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    const int k0 = 4 * k + h;
    const int row = cur.s.x + k0;
    if (cok && row >= 0 && row < p.n1) {
      const cf w = cmul(ldg_cf(P + k0 * M + ln), v[ct::brev<H>(k)]);
      red_add_v2(acc + (long long)row * p.n2 + col, w);
    }
  });
  return nxt;
}

// loss and gradient: one frame per block, frames round-robin over a
// persistent grid
template <int M>
__global__ void __launch_bounds__(T4Cfg<M>::T, 1) frames_t4(FrameArgs p) {
  using C = T4Cfg<M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[C::T / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.arrivals) *p.arrivals = 0u;
  const T4Group<M> g = T4Group<M>::make(threadIdx.x, smem_raw);
  double lsum = 0.0;
  int it = blockIdx.x;
  FrameRef cur = frame_ref(p, it);
  t4_fetch<M>(p, g, cur);
  cp_async_commit();
  for (; it < p.nframes; it += gridDim.x) {
    const FrameRef nxt = frame_ref(p, it + gridDim.x);
    cur = t4_frame<M>(p, g, cur, nxt, [&](float fl) { lsum += (double)fl; });
  }
  cp_async_wait_all();
  const double tot = block_sum_d<C::T>(lsum, red);
  if (threadIdx.x == 0) p.loss_part[blockIdx.x] = tot;
}

}  // namespace mpbp
