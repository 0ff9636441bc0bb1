// frames_t4.cuh -- the fused frame kernel (A2-A7 of frames.cuh) with four
// threads per line (fft_quad.cuh): M/4 values per thread, 4M threads and one
// frame per block.
//
// A warp holds eight lines: lane = 8 h + (ln mod 8), so the four threads of a
// line are lanes l, l^8, l^16, l^24 and every exchange of the line FFTs is a
// shuffle.  Each phase of a frame lays the shared buffers out for its own
// access pattern (a buffer is fully consumed before the next phase writes
// it), with paddings that keep every 16-lane half of a warp on distinct
// 8-byte banks and every address a per-thread base plus a constant:
//   patch     [k0][PW], PW = M + 8: column ln, rows 4n + h (the two row
//             parities of a half-warp 8 banks apart); a tile starts at an
//             even column, read from column s.y & 1 on
//   transpose [r][TW] + 8 (r / (M/4)), TW = M + 2: column ln, rows Q g + t
//             (the two halves' rows M/4 apart: 8 banks apart) and row ln,
//             columns 4n + h (eight rows 2 banks apart)
//   sqrt(y)   [q1][M] + 8 (q1 / Q) floats: the four rows Q g + t a warp reads
//             at eight consecutive q0 fall in different bank octets; 16-row
//             bands of M floats, one bulk copy each.
//
// The probe (TPR): the 32 probe values a thread multiplies, P(4n + h, ln)
// for n = 0 .. 31, are the same in A2 and A6 and for every frame of the
// block's peak, so they are kept in tensor memory, in 64 columns of the
// thread's own TMEM lane (warps w, w + 4, w + 8, w + 12 share a lane quarter
// and take columns 64 (w / 4) on), and read with tcgen05.ld instead of twice
// per frame from L2 (128 KB per probe does not fit in L1 beside the shared
// buffers).  They are reloaded when the frame's probe changes (a new peak with
// one probe per peak).  Probes that change with every scan position take the
// global loads (TPR = false).
#pragma once
#include "fft_quad.cuh"
#include "frames.cuh"
#include "tmem.cuh"

namespace mpbp {

template <int M>
struct T4Cfg {
  static constexpr int T = 4 * M;     // threads per block (one frame)
  static constexpr int H = M / 4;     // values per thread
  static constexpr int Q = M / 8;
  static constexpr int PW = M + 8;    // patch row
  static constexpr int TW = M + 2;    // transpose row
  static constexpr int TB = M / 4;    // rows per transpose band (8 cf padding after each)
  static constexpr int AB = Q;        // sqrt(y) rows per band (8 floats padding after each)
  static constexpr int PATCH = M * PW * (int)sizeof(cf);
  static constexpr int TRANS = (M * TW + 4 * 8) * (int)sizeof(cf);
  static constexpr int BUF = PATCH > TRANS ? PATCH : TRANS;
  static constexpr int ABAND = (AB * M + 8) * (int)sizeof(float);
  static constexpr int ABUF = (M / AB) * ABAND;
  static constexpr int SMEM = BUF + ABUF + 128;   // + alignment of the tile destination
  static constexpr int MINB = M >= 128 ? 1 : 3;   // blocks per SM the registers must allow
  static_assert(M == 32 || M == 64 || M == 128, "four threads per line: M = 32, 64 or 128");
  static_assert(BUF % 16 == 0 && ABAND % 16 == 0, "bulk copy alignment");
};

MPBP_DI cf xchg8(cf v) {
  return cf{__shfl_xor_sync(0xffffffffu, v.x, 8), __shfl_xor_sync(0xffffffffu, v.y, 8)};
}

template <int M>
MPBP_DI int t4_tr(int r, int c) {
  using C = T4Cfg<M>;
  return r * C::TW + (r / C::TB) * 8 + c;
}

template <int M>
MPBP_DI int t4_amp(int q1, int q0) {
  using C = T4Cfg<M>;
  return q1 * M + (q1 / C::AB) * 8 + q0;
}

// the frame's sqrt(y) tile by cp.async, into the banded layout
template <int M>
MPBP_DI void t4_fetch_amp(const PatchSrc& q, int t, float* dst) {
  if (!q.amp) return;
  constexpr int CH = M * M / 4, CPR = M / 4, NT = T4Cfg<M>::T;
  static_assert(CH % NT == 0, "tile chunks must divide among the threads");
#pragma unroll
  for (int i = 0; i < CH / NT; ++i) {
    const int c = t + i * NT;
    const int row = c / CPR, cc = c - row * CPR;
    cp_async16(dst + t4_amp<M>(row, 4 * cc), q.amp + 4 * c);
  }
}

template <int M>
struct T4Group {
  int tid;
  int ln;          // line (column or row) index
  int h, h0, h1;   // quarter of the line: h = 2 h1 + h0
  cf* buf;         // patch / transpose buffer
  float* abuf;     // sqrt(y) staging
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

// The inputs of frame r: TMA (thread 0 issues a tile load of the patch and
// one bulk copy per sqrt(y) band on the block's mbarrier), else cp.async by
// every thread (not committed).  Called after the barrier that freed the
// buffers.
template <int M, bool TMA>
MPBP_DI void t4_fetch(const FrameArgs& p, const T4Group<M>& g, const FrameRef& r, const BulkState& bs,
                      const TmaMap* tm) {
  using C = T4Cfg<M>;
  if constexpr (TMA) {
    if (g.tid == 0) {
      constexpr uint32_t kPatch = M * C::PW * (uint32_t)sizeof(cf);
      constexpr uint32_t kBand = C::AB * M * (uint32_t)sizeof(float);
      fence_async_smem();
      mbar_arrive_tx(bs.bar, (r.valid ? kPatch + (M / C::AB) * kBand : 0u) + tm->tx_extra);
      if (r.valid) {
        tile_load_3d(smem_addr(g.buf), &tm->map, r.s.y - (r.s.y & 1), r.s.x, r.mpk, bs.bar);
        const float* src = p.aT + (long long)r.f * M * M;
        const uint32_t dst = smem_addr(g.abuf);
#pragma unroll 1
        for (int b = 0; b < M / C::AB; ++b) bulk_load_stream(dst + b * C::ABAND, src + b * C::AB * M, kBand, bs.bar);
      }
    }
  } else {
    const PatchSrc q = patch_src<M>(p, r);
    // a rolled loop keeps the copies' addresses out of the registers the
    // values need (unrolled, they spill)
#pragma unroll 2
    for (int n = 0; n < C::H; ++n) {
      const int k0 = 4 * n + g.h;
      fetch_patch_elem(q, k0, g.ln, g.buf + k0 * C::PW + g.ln);
    }
    t4_fetch_amp<M>(q, g.tid, g.abuf);
  }
}

// One frame's loss and gradient (inputs in flight); fetches the next frame's
// inputs as soon as their buffers are free.  TMA: a wait that runs out clears
// bs.ok and returns at once.
// TMEM columns of the resident probe: 32 complex values a thread, four
// threads (warps w, w + 4, w + 8, w + 12) per lane
constexpr uint32_t kT4ProbeCols = 256;

// the thread's 32 probe values P(4n + h, ln) of probe P into its TMEM words
template <int M>
MPBP_DI void t4_probe_to_tmem(const cf* P, const T4Group<M>& g, uint32_t tp) {
  static_assert(T4Cfg<M>::H == 32, "the resident probe holds 32 values a thread");
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t w[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const cf v = ldg_cf(P + (4 * (8 * c + j) + g.h) * M + g.ln);
      w[2 * j] = __float_as_uint(v.x);
      w[2 * j + 1] = __float_as_uint(v.y);
    }
    tmem_st16(tp + 16 * c, w);
  }
  tmem_wait_st();
}

template <int M, bool TMA, bool LOSS, bool TPR, typename AddLoss>
MPBP_DI void t4_frame(const FrameArgs& p, const T4Group<M>& g, const FrameRef& cur, const FrameRef& nxt,
                      AddLoss&& add_loss, BulkState& bs, const TmaMap* tm, uint32_t tp) {
  using C = T4Cfg<M>;
  constexpr int H = C::H, PW = C::PW;
  cf* buf = g.buf;
  const int ln = g.ln, h = g.h;
  auto x8 = [](cf v) { return xchg8(v); };
  auto x16 = [](cf v) { return xchg16(v); };
  const cf* P = frame_probe(p, cur, M * M);
  const int col = cur.s.y + ln;
  const bool cok = cur.valid && col >= 0 && col < p.n2;
  if constexpr (TMA) {
    bs.ok = bulk_wait(bs.bar, bs.parity);
    bs.parity ^= 1u;
    if (!bs.ok) return;
  } else {
    cp_async_wait_all();
    __syncthreads();
  }
  const int dlt = TMA ? (cur.s.y & 1) : 0;   // a tile starts at an even column

  // A2: column ln, rows 4n + h
  cf v[H];
  if constexpr (TPR) {
    uint32_t w[4][16];
    sfor<0, 4>([&](auto c_) { tmem_ld16(tp + 16 * decltype(c_)::value, w[decltype(c_)::value]); });
    tmem_wait_ld();
    sfor<0, H>([&](auto n_) {
      constexpr int n = decltype(n_)::value;
      const int k0 = 4 * n + h;
      const cf pv = cf{__uint_as_float(w[n / 8][2 * (n % 8)]), __uint_as_float(w[n / 8][2 * (n % 8) + 1])};
      v[n] = cmul(pv, buf[k0 * PW + ln + dlt]);
    });
  } else {
    sfor<0, H>([&](auto n_) {
      constexpr int n = decltype(n_)::value;
      const int k0 = 4 * n + h;
      v[n] = cmul(ldg_cf(P + k0 * M + ln), buf[k0 * PW + ln + dlt]);
    });
  }

  // A3: columns, transpose, rows; the barrier orders the patch reads above
  // before the transpose writes of other threads
  fft_quad_dec_to_blk<M>(v, g.h0, g.h1, x8, x16);
  __syncthreads();
  sfor<0, H>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    buf[t4_tr<M>(g.blk(i), ln)] = v[i];
  });
  __syncthreads();
  sfor<0, H>([&](auto n_) {
    constexpr int n = decltype(n_)::value;
    v[n] = buf[t4_tr<M>(ln, 4 * n + h)];
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
    v[i] = residual(v[i], g.abuf[t4_amp<M>(q1, ln)], bv, fl);
  });
  add_loss(cur.valid ? 0.5f * fl : 0.0f);
  if constexpr (LOSS) {
    // loss only: the buffers are free once every thread is past its residual
    __syncthreads();
    t4_fetch<M, TMA>(p, g, nxt, bs, tm);
    if constexpr (!TMA) cp_async_commit();
    return;
  }

  // A5: rows (blk4 -> dec4), transpose, columns; the exchange buffer's last
  // reads (the transposed row input above) are behind this barrier
  fft_quad_blk_to_dec<M>(v, g.h0, g.h1, x8, x16);   // Z'[ln][4k + h] in slot brev(k)
  __syncthreads();
  sfor<0, H>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    buf[t4_tr<M>(ln, 4 * k + h)] = v[ct::brev<H>(k)];
  });
  __syncthreads();
  if constexpr (!TMA) t4_fetch_amp<M>(patch_src<M>(p, nxt), g.tid, g.abuf);   // every thread is past its residual
  sfor<0, H>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    v[i] = buf[t4_tr<M>(g.blk(i), ln)];
  });
  __syncthreads();   // both buffers are free
  if constexpr (TMA) {
    t4_fetch<M, true>(p, g, nxt, bs, tm);
  } else {
    const PatchSrc q = patch_src<M>(p, nxt);
#pragma unroll 2
    for (int n = 0; n < H; ++n) {
      const int k0 = 4 * n + h;
      fetch_patch_elem(q, k0, ln, buf + k0 * PW + ln);
    }
    cp_async_commit();
  }
  fft_quad_blk_to_dec<M>(v, g.h0, g.h1, x8, x16);   // Z[4k + h][ln] in slot brev(k)

  // A6 + A7
  // one running address and row, 4 rows a step
  int row = cur.s.x + h;
  cf* a = p.acc + cur.mpk * p.obj_stride + (long long)row * p.n2 + col;
  const long long step = 4LL * p.n2;
  const unsigned n1 = (unsigned)p.n1;
  if constexpr (TPR) {
    // probe values by chunks of eight, the next chunk's load in flight while
    // the current one is used
    uint32_t w[2][16];
    tmem_ld16(tp, w[0]);
    tmem_wait_ld();
    sfor<0, 4>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      if constexpr (c + 1 < 4) tmem_ld16(tp + 16 * (c + 1), w[(c + 1) & 1]);
      sfor<0, 8>([&](auto j_) {
        constexpr int j = decltype(j_)::value, k = 8 * c + j;
        const cf pv = cf{__uint_as_float(w[c & 1][2 * j]), __uint_as_float(w[c & 1][2 * j + 1])};
        const cf wv = cmul(pv, v[ct::brev<H>(k)]);
        red_add_v2_if(a, wv, cok && (unsigned)row < n1);
        a += step;
        row += 4;
      });
      if constexpr (c + 1 < 4) tmem_wait_ld();
    });
  } else {
    sfor<0, H>([&](auto k_) {
      constexpr int k = decltype(k_)::value;
      const cf w = cmul(ldg_cf(P + (4 * k + h) * M + ln), v[ct::brev<H>(k)]);
      if (cok && (unsigned)row < n1) red_add_v2(a, w);
      a += step;
      row += 4;
    });
  }
}

// loss and gradient (LOSS: loss only): one frame per block, frames
// round-robin over a persistent grid; TMA: inputs by tile and bulk copies
// (tm: the objects' tensor map), else by cp.async
// TPR: the probe resident in tensor memory (probes shared by all frames of a
// peak: FrameArgs::probe_stride >= 0)
template <int M, bool TMA, bool LOSS = false, bool TPR = false>
__global__ void __launch_bounds__(T4Cfg<M>::T, T4Cfg<M>::MINB)
    frames_t4(const FrameArgs p, const __grid_constant__ TmaMap tm) {
  using C = T4Cfg<M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[C::T / 32];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.arrivals) *p.arrivals = 0u;
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  const T4Group<M> g = T4Group<M>::make(threadIdx.x, smem);
  BulkState bs{smem_addr(&mbar), 0u, true};
  const int warp = threadIdx.x >> 5;
  if constexpr (TPR) {
    if (warp == 0) tmem_alloc(smem_addr(&tmem_base), kT4ProbeCols);
  }
  if constexpr (TMA) {
    if (threadIdx.x == 0) mbar_init(bs.bar, 1);
  }
  if constexpr (TMA || TPR) {
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
  }
  // this thread's 64 probe columns: lane 32 (warp mod 4) + lane id, columns
  // 64 (warp / 4) on
  const uint32_t tp = TPR ? tmem_addr(tmem_base, 32u * (warp & 3), 64u * (warp >> 2)) : 0u;
  const cf* tp_src = nullptr;   // the probe held in tensor memory (block-uniform)
  double lsum = 0.0;
  int it = blockIdx.x;
  FrameRef cur = frame_ref(p, it);
  t4_fetch<M, TMA>(p, g, cur, bs, &tm);
  if constexpr (!TMA) cp_async_commit();
  for (; it < p.nframes; it += gridDim.x) {
    const FrameRef nxt = frame_ref(p, it + gridDim.x);
    if constexpr (TPR) {
      const cf* P = frame_probe(p, cur, M * M);
      if (P != tp_src) {
        t4_probe_to_tmem<M>(P, g, tp);
        tp_src = P;
      }
    }
    t4_frame<M, TMA, LOSS, TPR>(p, g, cur, nxt, [&](float fl) { lsum += (double)fl; }, bs, &tm, tp);
    if (TMA && !bs.ok) {
      if (threadIdx.x == 0) atomicOr(p.err, kErrTimeout);
      break;
    }
    cur = nxt;
  }
  cp_async_wait_all();
  const double tot = block_sum_d<C::T>(lsum, red);
  if (threadIdx.x == 0) p.loss_part[blockIdx.x] = tot;
  if constexpr (TPR) {
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem_base, kT4ProbeCols);
  }
}

}  // namespace mpbp
