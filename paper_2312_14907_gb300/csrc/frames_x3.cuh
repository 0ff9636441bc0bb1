// frames_x3.cuh -- the fused frame kernel for M = 128 (A2-A7 of frames.cuh)
// with each 2-D transform computed in three register layouts joined by two
// shared-memory exchanges, in place of the radix-2 stages across threads
// (warp shuffles and selects) of frames_t4.cuh.
//
// Index split (W = exp(-2 pi i / 128); 512 threads, 32 values each):
//   rows    r = 4 n + h,          q0 = k' + 32 k''   (n, k' < 32; h, k'' < 4)
//   columns c = c_r + 16 c_a,     q1 = m' + 8 m''    (c_r, m'' < 16; c_a, m' < 8)
// and the forward transform Psi = F psi of Eq. 2 as
//   X1(q0, c)  = sum_h  W4^(k'' h) W^(k' h) [sum_n W32^(n k') psi(4n + h, c)]
//   Psi(q0,q1) = sum_c_r W16^(m'' c_r) W^(m' c_r) [sum_c_a W8^(m' c_a) X1(q0, c_r + 16 c_a)]
// Layouts (register index -> thread index):
//   L1  n (32)                    | c, h        lane = c mod 32, warp = 4 h + c / 32
//   L2  h or k'' (4) x c_a or m'  | k', c_r     lane = c_r + 16 (k' mod 2), warp = k' / 2
//   L3  c_r or m'' (16) x m_r (2) | q0, m_t     lane = k', warp = 4 k'' + m_t;  m' = m_t + 4 m_r
// L1: the 32-point transforms over n.  L2: twiddle W^(k' h), 4-point
// transforms over h, 8-point over c_a, twiddle W^(m' c_r).  L3: 16-point
// transforms over c_r; the residual (A4) reads sqrt(y)[q1][q0] with 32
// consecutive q0 per warp.  The adjoint Z = F conj(chi) (A5) runs the same
// factorisation backwards (16-point over m'' in L3, twiddle W^(m' c_r) and
// 8-point over m' in L2, 4-point over k'' and twiddle W^(k' h) in L2, 32-point
// over k' in L1) and ends in L1, the columns layout of the scatter (A6, A7).
// The twiddles W^(h k'), h = 1..3, and W^(m' c_r), m' = 1..7, are formed once
// per block into a 1.7 KB shared table.
//
// Gradient accumulation (A7).  A block takes a contiguous range of the
// frames in the order it is given; the host orders them by peak, scan column
// and scan row, so that a block's consecutive frames mostly share their
// columns and overlap in rows.  Tensor memory holds the probe (columns
// 0..255) and, in columns 256..511, the gradient of a 128-row window of the
// block's current column strip: TMEM lane c is column c of the frame (the
// four warps of L1 that hold column c share that lane), and absolute row R
// sits in slot R mod 128.  A frame adds P conj(F^H chi) into the slots of its
// rows; when the next frame of the strip starts d rows lower, the d rows that
// leave the window are added to the object-sized accumulator with
// red.global.add and their slots cleared, so the rows shared by successive
// frames cross to global memory once.  A frame in another strip (another
// column, peak, or a row outside the window) writes the whole window back
// first; the block writes back what is left at its end.
//
// Shared layouts (complex values), every 16-lane half-warp on 16 distinct
// 8-byte banks:
//   A  [h][k'][c ^ 8 (h mod 2)]       (L1 <-> L2), 16,384 values
//   B  [m'][q0][17] (c_r or m'')      (L2 <-> L3), 17,408 values
//   the patch tile [k0][M + 8] as in frames_t4.cuh, and sqrt(y) [q1][q0].
#pragma once
#include "frames_t4.cuh"
#include "tmem.cuh"

#include <climits>

namespace mpbp {

struct X3Cfg {
  static constexpr int M = 128;
  static constexpr int T = 512;
  static constexpr int PW = M + 8;                               // patch row (the tile copy's box width)
  static constexpr int A_VALS = 4 * 32 * 128;                    // layout A
  static constexpr int B_VALS = 8 * 128 * 17;                    // layout B
  static constexpr int PATCH_VALS = M * PW;
  static constexpr int BUF = (B_VALS > PATCH_VALS ? B_VALS : PATCH_VALS) * (int)sizeof(cf);
  static constexpr int ABUF = M * M * (int)sizeof(float);       // sqrt(y) [q1][q0]
  static constexpr int SMEM = BUF + ABUF + 128;                  // + alignment of the tile destination
  static constexpr uint32_t TMEM_COLS = 512;                     // probe (0..255), gradient window (256..)
  static constexpr uint32_t ACC_COL = 256;
  static_assert(A_VALS <= B_VALS && BUF % 16 == 0, "layouts");
};

// a thread's indices in the three layouts
struct X3Roles {
  int tid;
  // L1
  int c, h;
  // L2
  int kp, cr;
  // L3
  int q0, mt;
  MPBP_DI static X3Roles make(int tid) {
    X3Roles r;
    r.tid = tid;
    const int w = tid >> 5, l = tid & 31;
    r.c = 32 * (w & 3) + l;   // a warp holds 32 consecutive columns of one row h
    r.h = w >> 2;
    r.kp = 2 * w + (l >> 4);
    r.cr = l & 15;
    r.q0 = l + 32 * (w >> 2);
    r.mt = w & 3;
    return r;
  }
};

MPBP_DI int x3_a(int h, int kp, int c) { return (h * 32 + kp) * 128 + (c ^ ((h & 1) << 3)); }
MPBP_DI int x3_b(int mp, int q0, int i) { return (mp * 128 + q0) * 17 + i; }

// W^j = exp(-2 pi i j / 128)
MPBP_DI cf x3_w128(int j) {
  float sn, cs;
  sincospif((float)(j & 127) / 64.0f, &sn, &cs);
  return cf{cs, -sn};
}

// the twiddles of L2: th[h - 1][k'] = W^(h k'), um[m' - 1][c_r] = W^(m' c_r)
struct X3Tables {
  cf th[3][32];
  cf um[7][16];
};

// every thread of the block (before a barrier)
MPBP_DI void x3_tables_init(X3Tables& t) {
  const int i = threadIdx.x;
  if (i < 96) t.th[i / 32][i % 32] = x3_w128((i / 32 + 1) * (i % 32));
  else if (i < 96 + 112) t.um[(i - 96) / 16][(i - 96) % 16] = x3_w128(((i - 96) / 16 + 1) * ((i - 96) % 16));
}

struct X3Tw {
  cf th[4];   // th[h] = W^(h k'), th[0] unused
  cf um[8];   // um[m'] = W^(m' c_r), um[0] unused
};

MPBP_DI void x3_twiddles(const X3Tables& t, const X3Roles& r, X3Tw& tw) {
#pragma unroll
  for (int h = 1; h < 4; ++h) tw.th[h] = t.th[h - 1][r.kp];
#pragma unroll
  for (int m = 1; m < 8; ++m) tw.um[m] = t.um[m - 1][r.cr];
}

// the gradient window of a block: strip (peak, first column) and its first
// row; with a deterministic plan, the block's current piece and the hull
// [wlo, whi) of the rows written into it so far
struct X3Win {
  bool ok;
  int mpk, y, x;
  int piece;
  int wlo, whi;
};

// Add rows [x0, x0 + d) of the window to the accumulator (A7) and, if zero,
// clear their slots; thread (c, h) takes rows x0 + h + 4 i.  Whole block,
// converged; ta: the thread's lane at the window's first column.  With a
// deterministic plan the rows go to the block's current piece instead:
// rows outside the hull of those written so far are stored, the others
// loaded, added and stored (the piece has no other writer, it starts
// cleared, and successive write-backs of a row are separated by block
// barriers); on a strip the window slides down, so every row is a store.
template <bool DET>
MPBP_DI void x3_flush(const FrameArgs& p, const X3Roles& r, const X3Win& w, int x0, int d, uint32_t ta,
                      bool zero) {
  const int col = w.y + r.c;
  const bool cok = col >= 0 && col < p.n2;
  cf* const base = p.acc + (long long)w.mpk * p.obj_stride + col;
  const unsigned n1 = (unsigned)p.n1;
  cf* pbase = nullptr;   // the piece's column c at row 0
  if constexpr (DET) {
    const DetPiece pc = p.det->pieces[w.piece];
    pbase = p.det->pool + pc.off - (long long)pc.row0 * X3Cfg::M + r.c;
  }
  const int cnt = d > r.h ? (d - r.h + 3) / 4 : 0;   // warp-uniform
  for (int i0 = 0; i0 < cnt; i0 += 8) {
    uint32_t v[8][2];
    sfor<0, 8>([&](auto j_) {
      constexpr int j = decltype(j_)::value;
      if (i0 + j < cnt) tmem_ld2(ta + 2u * (uint32_t)((x0 + r.h + 4 * (i0 + j)) & 127), v[j]);
    });
    tmem_wait_ld();
    sfor<0, 8>([&](auto j_) {
      constexpr int j = decltype(j_)::value;
      if (i0 + j < cnt) {
        const int row = x0 + r.h + 4 * (i0 + j);
        const cf g = cf{__uint_as_float(v[j][0]), __uint_as_float(v[j][1])};
        if constexpr (DET) {
          cf* q = pbase + (long long)row * X3Cfg::M;
          if (row >= w.wlo && row < w.whi) {   // warp-uniform
            const cf o = *q;
            *q = cf{o.x + g.x, o.y + g.y};
          } else {
            *q = g;
          }
        } else {
          red_add_v2_if(base + (long long)row * p.n2, g, cok && (unsigned)row < n1);
        }
        if (zero) tmem_st2(ta + 2u * (uint32_t)(row & 127), 0u, 0u);
      }
    });
  }
}

// the thread's 32 probe values P(4 n + h, c) (its L1 role) into its TMEM
// words, in four chunks of 16 words: chunk n mod 4 holds n = n mod 4 + 4 m,
// m = 0..7, the order in which the last transform's outputs are scattered
MPBP_DI void x3_probe_to_tmem(const cf* P, const X3Roles& r, uint32_t tp) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t w[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const cf v = ldg_cf(P + (4 * (4 * j + c) + r.h) * X3Cfg::M + r.c);
      w[2 * j] = __float_as_uint(v.x);
      w[2 * j + 1] = __float_as_uint(v.y);
    }
    tmem_st16(tp + 16 * c, w);
  }
  tmem_wait_st();
}

// TMA, in two parts on one mbarrier phase: the sqrt(y) tile of frame fr as
// soon as the residual has read the staging buffer (thread 0 announces both
// copies' bytes), the patch tile once the exchanges have freed theirs
MPBP_DI void x3_fetch_amp_tma(const FrameArgs& p, const X3Roles& r, const FrameRef& fr, float* abuf,
                              const BulkState& bs, const TmaMap* tm) {
  constexpr int M = X3Cfg::M;
  if (r.tid == 0) {
    constexpr uint32_t kPatch = M * X3Cfg::PW * (uint32_t)sizeof(cf);
    constexpr uint32_t kAmp = M * M * (uint32_t)sizeof(float);
    fence_async_smem();
    mbar_arrive_tx(bs.bar, (fr.valid ? kPatch + kAmp : 0u) + tm->tx_extra);
    if (fr.valid) bulk_load_stream(smem_addr(abuf), p.aT + (long long)fr.f * M * M, kAmp, bs.bar);
  }
}

MPBP_DI void x3_fetch_patch_tma(const X3Roles& r, const FrameRef& fr, cf* buf, const BulkState& bs,
                                const TmaMap* tm) {
  if (r.tid == 0 && fr.valid) {
    fence_async_smem();
    tile_load_3d(smem_addr(buf), &tm->map, fr.s.y - (fr.s.y & 1), fr.s.x, fr.mpk, bs.bar);
  }
}

// inputs of frame fr: the patch tile and sqrt(y) [q1][q0] (64 KB); TMA: one
// thread issues a tile load and one bulk copy on the block's mbarrier, after
// the barrier that freed the buffers; else cp.async by every thread
template <bool TMA>
MPBP_DI void x3_fetch(const FrameArgs& p, const X3Roles& r, const FrameRef& fr, cf* buf, float* abuf,
                      const BulkState& bs, const TmaMap* tm) {
  using C = X3Cfg;
  constexpr int M = C::M;
  if constexpr (TMA) {
    if (r.tid == 0) {
      constexpr uint32_t kPatch = M * C::PW * (uint32_t)sizeof(cf);
      constexpr uint32_t kAmp = M * M * (uint32_t)sizeof(float);
      fence_async_smem();
      mbar_arrive_tx(bs.bar, (fr.valid ? kPatch + kAmp : 0u) + tm->tx_extra);
      if (fr.valid) {
        tile_load_3d(smem_addr(buf), &tm->map, fr.s.y - (fr.s.y & 1), fr.s.x, fr.mpk, bs.bar);
        bulk_load_stream(smem_addr(abuf), p.aT + (long long)fr.f * M * M, kAmp, bs.bar);
      }
    }
  } else {
    const PatchSrc q = patch_src<M>(p, fr);
#pragma unroll 2
    for (int n = 0; n < 32; ++n) {
      const int k0 = 4 * n + r.h;
      fetch_patch_elem(q, k0, r.c, buf + k0 * C::PW + r.c);
    }
    if (q.amp) {
#pragma unroll
      for (int i = 0; i < M * M / 4 / C::T; ++i) {
        const int ch = r.tid + i * C::T;
        cp_async16(abuf + 4 * ch, q.amp + 4 * ch);
      }
    }
  }
}

// One frame's loss and gradient (inputs in flight); fetches the next frame's
// inputs as soon as their buffers are free.  TMA: a wait that runs out clears
// bs.ok and returns at once.
template <bool TMA, bool LOSS, bool BG, bool DET, typename AddLoss>
MPBP_DI void x3_frame(const FrameArgs& p, const X3Roles& r, const FrameRef& cur, const FrameRef& nxt,
                      AddLoss&& add_loss, BulkState& bs, const TmaMap* tm, cf* buf, float* abuf, uint32_t tp,
                      uint32_t ta, const X3Tables& tab, X3Win& win) {
  using C = X3Cfg;
  constexpr int M = C::M, PW = C::PW;
  // the probe values of A2 load from tensor memory while the inputs land
  uint32_t w[4][16];
  sfor<0, 4>([&](auto c_) { tmem_ld16(tp + 16 * decltype(c_)::value, w[decltype(c_)::value]); });
  if constexpr (TMA) {
    bs.ok = bulk_wait(bs.bar, bs.parity);
    bs.parity ^= 1u;
    if (!bs.ok) {
      tmem_wait_ld();
      return;
    }
  } else {
    cp_async_wait_all();
    __syncthreads();
  }
  tmem_fence_after_sync();   // the previous frame's window updates
  const int dlt = TMA ? (cur.s.y & 1) : 0;   // a tile starts at an even column

  // ---- A2 + the 32-point transforms over n (L1)
  cf v[32];
  tmem_wait_ld();
  sfor<0, 32>([&](auto n_) {
    constexpr int n = decltype(n_)::value;
    const cf pv = cf{__uint_as_float(w[n % 4][2 * (n / 4)]), __uint_as_float(w[n % 4][2 * (n / 4) + 1])};
    v[n] = cmul(pv, buf[(4 * n + r.h) * PW + r.c + dlt]);
  });
  fft_line<32>(v);   // Y(h, k', c) in slot brev(k')
  __syncthreads();   // the patch reads are done
  sfor<0, 32>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    buf[x3_a(r.h, k, r.c)] = v[ct::brev<32>(k)];
  });
  cf x[32];
  {
  X3Tw tw;
  x3_twiddles(tab, r, tw);   // the table is constant: read ahead of the barrier
  __syncthreads();

  // ---- L2: twiddle, 4-point over h, 8-point over c_a, twiddle
  sfor<0, 4>([&](auto h_) {
    constexpr int hh = decltype(h_)::value;
    sfor<0, 8>([&](auto a_) {
      constexpr int ca = decltype(a_)::value;
      x[hh * 8 + ca] = buf[x3_a(hh, r.kp, r.cr + 16 * ca)];
    });
  });
  sfor<0, 8>([&](auto a_) {
    constexpr int ca = decltype(a_)::value;
    cf t4[4];
    t4[0] = x[ca];
    sfor<1, 4>([&](auto h_) {
      constexpr int hh = decltype(h_)::value;
      t4[hh] = cmul(x[hh * 8 + ca], tw.th[hh]);
    });
    fft_line<4>(t4);
    sfor<0, 4>([&](auto k_) {
      constexpr int kk = decltype(k_)::value;
      x[kk * 8 + ca] = t4[ct::brev<4>(kk)];   // x[8 k'' + c_a]
    });
  });
  sfor<0, 4>([&](auto k_) {
    constexpr int kk = decltype(k_)::value;
    cf t8[8];
    sfor<0, 8>([&](auto a_) { t8[decltype(a_)::value] = x[kk * 8 + decltype(a_)::value]; });
    fft_line<8>(t8);
    x[kk * 8] = t8[0];
    sfor<1, 8>([&](auto m_) {
      constexpr int mp = decltype(m_)::value;
      x[kk * 8 + mp] = cmul(t8[ct::brev<8>(mp)], tw.um[mp]);   // x[8 k'' + m']
    });
  });
  }
  __syncthreads();   // every layout-A read is done
  sfor<0, 4>([&](auto k_) {
    constexpr int kk = decltype(k_)::value;
    sfor<0, 8>([&](auto m_) {
      constexpr int mp = decltype(m_)::value;
      buf[x3_b(mp, r.kp + 32 * kk, r.cr)] = x[kk * 8 + mp];
    });
  });
  __syncthreads();

  // ---- L3: 16-point over c_r; A4 on row q0
  sfor<0, 2>([&](auto m_) {
    constexpr int mr = decltype(m_)::value;
    sfor<0, 16>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      v[mr * 16 + i] = buf[x3_b(r.mt + 4 * mr, r.q0, i)];
    });
  });
  sfor<0, 2>([&](auto m_) {
    constexpr int mr = decltype(m_)::value;
    cf t16[16];
    sfor<0, 16>([&](auto i_) { t16[decltype(i_)::value] = v[mr * 16 + decltype(i_)::value]; });
    fft_line<16>(t16);
    sfor<0, 16>([&](auto i_) {
      constexpr int mm = decltype(i_)::value;
      v[mr * 16 + mm] = t16[ct::brev<16>(mm)];   // Psi(q0, m' + 8 m'') at v[16 m_r + m'']
    });
  });
  float fl = 0.0f;
  // BG: the background b of Eq. 2 (a kernel of its own, so that the common
  // case carries no per-value test)
  const float* bg = BG ? p.bgT + (long long)cur.f * M * M : nullptr;
  sfor<0, 2>([&](auto m_) {
    constexpr int mr = decltype(m_)::value;
    sfor<0, 16>([&](auto i_) {
      constexpr int mm = decltype(i_)::value;
      const int q1 = r.mt + 4 * mr + 8 * mm;
      const float bv = BG ? bg[q1 * M + r.q0] : 0.0f;
      v[mr * 16 + mm] = residual(v[mr * 16 + mm], abuf[q1 * M + r.q0], bv, fl);
    });
  });
  add_loss(cur.valid ? 0.5f * fl : 0.0f);
  if constexpr (LOSS) {
    __syncthreads();   // every read of the buffers is done
    x3_fetch<TMA>(p, r, nxt, buf, abuf, bs, tm);
    if constexpr (!TMA) cp_async_commit();
    return;
  }

  // ---- A5: Z = F conj(chi), L3: 16-point over m''
  sfor<0, 2>([&](auto m_) {
    constexpr int mr = decltype(m_)::value;
    cf t16[16];
    sfor<0, 16>([&](auto i_) { t16[decltype(i_)::value] = v[mr * 16 + decltype(i_)::value]; });
    fft_line<16>(t16);   // T(m', kr) in slot brev(kr)
    sfor<0, 16>([&](auto i_) {
      constexpr int kr = decltype(i_)::value;
      v[mr * 16 + kr] = t16[ct::brev<16>(kr)];
    });
  });
  __syncthreads();   // every layout-B read is done
  sfor<0, 2>([&](auto m_) {
    constexpr int mr = decltype(m_)::value;
    sfor<0, 16>([&](auto i_) {
      constexpr int kr = decltype(i_)::value;
      buf[x3_b(r.mt + 4 * mr, r.q0, kr)] = v[mr * 16 + kr];
    });
  });
  // the residual's reads of the sqrt(y) buffer are behind the barrier above:
  // the next frame's tile can land there now
  if constexpr (TMA) x3_fetch_amp_tma(p, r, nxt, abuf, bs, tm);
  X3Tw tw;
  x3_twiddles(tab, r, tw);
  __syncthreads();

  // ---- L2: twiddle, 8-point over m', 4-point over k'', twiddle
  sfor<0, 4>([&](auto k_) {
    constexpr int kk = decltype(k_)::value;
    cf t8[8];
    t8[0] = buf[x3_b(0, r.kp + 32 * kk, r.cr)];
    sfor<1, 8>([&](auto m_) {
      constexpr int mp = decltype(m_)::value;
      t8[mp] = cmul(buf[x3_b(mp, r.kp + 32 * kk, r.cr)], tw.um[mp]);
    });
    fft_line<8>(t8);
    sfor<0, 8>([&](auto a_) {
      constexpr int ka = decltype(a_)::value;
      x[kk * 8 + ka] = t8[ct::brev<8>(ka)];   // x[8 k'' + k_a]
    });
  });
  sfor<0, 8>([&](auto a_) {
    constexpr int ka = decltype(a_)::value;
    cf t4[4];
    sfor<0, 4>([&](auto k_) { t4[decltype(k_)::value] = x[decltype(k_)::value * 8 + ka]; });
    fft_line<4>(t4);
    x[ka] = t4[0];
    sfor<1, 4>([&](auto h_) {
      constexpr int hh = decltype(h_)::value;
      x[hh * 8 + ka] = cmul(t4[ct::brev<4>(hh)], tw.th[hh]);   // x[8 h' + k_a]
    });
  });
  __syncthreads();   // every layout-B read is done
  sfor<0, 4>([&](auto h_) {
    constexpr int hh = decltype(h_)::value;
    sfor<0, 8>([&](auto a_) {
      constexpr int ka = decltype(a_)::value;
      buf[x3_a(hh, r.kp, r.cr + 16 * ka)] = x[hh * 8 + ka];
    });
  });
  __syncthreads();

  // ---- L1: 32-point over k'; A6 + A7
  sfor<0, 32>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    v[k] = buf[x3_a(r.h, k, r.c)];
  });
  // the window moves to this frame's rows: rows that leave it go out
  if (cur.valid) {
    const bool slide = win.ok && cur.mpk == win.mpk && cur.s.y == win.y && cur.s.x >= win.x &&
                       cur.s.x - win.x < X3Cfg::M;
    const int dd = slide ? cur.s.x - win.x : X3Cfg::M;
    if (win.ok) x3_flush<DET>(p, r, win, win.x, dd, ta, true);
    // a new strip starts the block's next piece (the host splits them there)
    const bool strip = !win.ok || cur.mpk != win.mpk || cur.s.y != win.y;
    int wlo = win.wlo, whi = win.whi;
    if (win.ok && dd > 0) {
      wlo = min(wlo, win.x);
      whi = max(whi, win.x + dd);
    }
    if (strip) {
      wlo = INT_MAX;
      whi = INT_MIN;
    }
    win = X3Win{true, cur.mpk, cur.s.y, cur.s.x, win.piece + (strip ? 1 : 0), wlo, whi};
  }
  tmem_wait_st();
  tmem_fence_before_sync();
  __syncthreads();   // both buffers are free; the slots the window left are clear
  tmem_fence_after_sync();
  if constexpr (TMA) {
    x3_fetch_patch_tma(r, nxt, buf, bs, tm);
  } else {
    x3_fetch<false>(p, r, nxt, buf, abuf, bs, tm);
    cp_async_commit();
  }
  if (!cur.valid) return;
  // the 32-point transform over k' split by frequency, n = 4 m + r:
  //   Z(n) = sum_j W8^(j m) [W32^(j r) sum_s W4^(s r) v(j + 8 s)],
  // a radix-4 step, then one 8-point transform per r, whose outputs are
  // multiplied by the probe (A6) and added into the window's slots of rows
  // s.x + h + 4 n
  sfor<0, 8>([&](auto j_) {
    constexpr int j = decltype(j_)::value;
    cf t4[4] = {v[j], v[j + 8], v[j + 16], v[j + 24]};
    fft_line<4>(t4);
    sfor<0, 4>([&](auto r_) {
      constexpr int rr = decltype(r_)::value;
      v[j + 8 * rr] = twmul<j * rr, 32>(t4[ct::brev<4>(rr)]);   // u_r(j) at v[j + 8 r]
    });
  });
  const int b0 = cur.s.x + r.h;   // row of n = 0
  sfor<0, 4>([&](auto r_) {
    constexpr int rr = decltype(r_)::value;
    uint32_t pw[16], o[8][2];
    tmem_ld16(tp + 16 * rr, pw);   // P at n = 4 m + r, m = 0..7
    sfor<0, 8>([&](auto m_) {
      constexpr int m = decltype(m_)::value;
      tmem_ld2(ta + 2u * (uint32_t)((b0 + 4 * (4 * m + rr)) & 127), o[m]);
    });
    cf t8[8];
    sfor<0, 8>([&](auto j_) { t8[decltype(j_)::value] = v[decltype(j_)::value + 8 * rr]; });
    fft_line<8>(t8);   // Z(4 m + r) in slot brev(m)
    tmem_wait_ld();
    sfor<0, 8>([&](auto m_) {
      constexpr int m = decltype(m_)::value;
      const cf pv = cf{__uint_as_float(pw[2 * m]), __uint_as_float(pw[2 * m + 1])};
      const cf z = t8[ct::brev<8>(m)];
      const float gx = fmaf(pv.x, z.x, fmaf(-pv.y, z.y, __uint_as_float(o[m][0])));
      const float gy = fmaf(pv.x, z.y, fmaf(pv.y, z.x, __uint_as_float(o[m][1])));
      tmem_st2(ta + 2u * (uint32_t)((b0 + 4 * (4 * m + rr)) & 127), __float_as_uint(gx), __float_as_uint(gy));
    });
  });
  tmem_wait_st();
  tmem_fence_before_sync();
}

// loss and gradient (LOSS: loss only; BG: with the background of Eq. 2;
// DET: the gradient through the deterministic plan p.det): a
// persistent grid, block b taking frames [N b / G, N (b + 1) / G) of the
// order given (p.frames, else 0..N-1); TMA: inputs by tile and bulk copies
// (tm: the objects' tensor map), else by cp.async.  The probe values of a
// thread sit in tensor memory and are reloaded when the frame's probe
// changes: once per block for one probe, per peak for one probe per peak,
// per frame for probes shifted per scan position.
template <bool TMA, bool LOSS = false, bool BG = false, bool DET = false>
__global__ void __launch_bounds__(X3Cfg::T, 1) frames_x3(const FrameArgs p, const __grid_constant__ TmaMap tm) {
  using C = X3Cfg;
  constexpr int M = C::M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[C::T / 32];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ X3Tables tab;
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.arrivals) *p.arrivals = 0u;
  unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  cf* buf = reinterpret_cast<cf*>(smem);
  float* abuf = reinterpret_cast<float*>(smem + C::BUF);
  const X3Roles r = X3Roles::make(threadIdx.x);
  BulkState bs{smem_addr(&mbar), 0u, true};
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tmem_alloc(smem_addr(&tmem_base), C::TMEM_COLS);
  if (TMA && threadIdx.x == 0) mbar_init(bs.bar, 1);
  x3_tables_init(tab);
  tmem_fence_before_sync();
  __syncthreads();
  tmem_fence_after_sync();
  // this thread's lane is 32 (warp mod 4) + lane id = its column c; its probe
  // words are columns 64 (warp / 4) .. + 63; the window's slot s of column c
  // is columns 256 + 2 s, + 1 (every warp holding column c reaches them)
  const uint32_t tp = tmem_addr(tmem_base, 32u * (warp & 3), 64u * (warp >> 2));
  const uint32_t ta = tmem_addr(tmem_base, 32u * (warp & 3), C::ACC_COL);
  if constexpr (!LOSS) {
    // clear the window: warp w the slots 32 (w / 4) .. + 31 of its lanes
    const uint32_t z[16] = {};
    sfor<0, 4>([&](auto k_) { tmem_st16(ta + 64u * (warp >> 2) + 16u * decltype(k_)::value, z); });
    tmem_wait_st();
    tmem_fence_before_sync();   // ordered before the first frame's barriers
  }
  X3Win win{false, 0, 0, 0, DET ? p.det->block_piece0[blockIdx.x] - 1 : 0, INT_MAX, INT_MIN};
  const cf* tp_src = nullptr;   // the probe held in tensor memory (block-uniform)
  double lsum = 0.0;
  const int lo = (int)((long long)p.nframes * blockIdx.x / gridDim.x);
  const int hi = (int)((long long)p.nframes * (blockIdx.x + 1) / gridDim.x);
  const FrameRef none = frame_ref(p, p.nframes);   // not valid: nothing to fetch
  FrameRef cur = lo < hi ? frame_ref(p, lo) : none;
  x3_fetch<TMA>(p, r, cur, buf, abuf, bs, &tm);
  if constexpr (!TMA) cp_async_commit();
  // frame indices are read one frame ahead of their scan positions, so that
  // neither global load waits on the other
  int f1 = lo + 1 < hi ? frame_at(p, lo + 1) : 0;
  for (int it = lo; it < hi; ++it) {
    const int f2 = it + 2 < hi ? frame_at(p, it + 2) : 0;
    const FrameRef nxt = it + 1 < hi ? frame_ref_of(p, f1) : none;
    f1 = f2;
    {
      const cf* P = frame_probe(p, cur, M * M);
      if (P != tp_src) {
        x3_probe_to_tmem(P, r, tp);
        tp_src = P;
      }
    }
    x3_frame<TMA, LOSS, BG, DET>(p, r, cur, nxt, [&](float fl) { lsum += (double)fl; }, bs, &tm, buf, abuf, tp, ta,
                            tab, win);
    if (TMA && !bs.ok) {
      if (threadIdx.x == 0) atomicOr(p.err, kErrTimeout);
      break;
    }
    cur = nxt;
  }
  cp_async_wait_all();
  if constexpr (!LOSS) {
    if (bs.ok && win.ok) {   // what is left of the window
      __syncthreads();
      tmem_fence_after_sync();
      x3_flush<DET>(p, r, win, win.x, M, ta, false);
    }
  }
  const double tot = block_sum_d<C::T>(lsum, red);
  if (threadIdx.x == 0) p.loss_part[blockIdx.x] = tot;
  tmem_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_base, C::TMEM_COLS);
}

}  // namespace mpbp
