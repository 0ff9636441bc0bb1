// fft_pair.cuh -- L-point FFT lines split over a pair of threads.
//
// A line of L complex values (L = 64 or 128) is shared by two threads (lanes
// l and l^16 of one warp, h = 0 / 1), H = L/2 values each, which meet once per
// line through a warp shuffle.  With Q = L/4:
//   "dec" layout: thread h holds x[2n + h], n = 0..H-1
//   "blk" layout: thread h holds x[Q h + i] in slot i and x[H + Q h + i] in
//                 slot Q + i, i = 0..Q-1
// dec -> blk is decimation in time: an H-point FFT per thread, then the last
// radix-2 stage across the pair.  blk -> dec is decimation in frequency: the
// first radix-2 stage across the pair, then an H-point FFT per thread, whose
// result X[2k + h] sits in slot brev_H(k).  The twiddle of index Q h + i is
// W_L^i (W_L^Q)^h = W_L^i (-i)^h.
// `Xchg` returns the value the partner lane passed in (a warp shuffle on the
// GPU).
#pragma once
#include "fft_reg.cuh"

namespace mpbp {

MPBP_DI cf cadd(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
MPBP_DI cf csub(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
MPBP_DI cf csel(bool c, cf a, cf b) { return cf{c ? a.x : b.x, c ? a.y : b.y}; }

template <int L, typename Xchg>
MPBP_DI void fft_pair_dec_to_blk(cf (&v)[L / 2], int h, Xchg&& xchg) {
  constexpr int H = L / 2, Q = L / 4;
  fft_line<H>(v);  // Y_h[k] in slot brev_H(k)
  cf out[H];
  const bool hi = h != 0;
  sfor<0, Q>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    constexpr int lo_slot = ct::brev<H>(i), hi_slot = ct::brev<H>(Q + i);
    const cf recv = xchg(csel(hi, v[lo_slot], v[hi_slot]));   // Y_{1-h}[Q h + i]
    cf a = csel(hi, recv, v[lo_slot]);                          // Y_0[Q h + i]
    // (-i)^h Y_1[Q h + i]: the twiddle W_L^{Q h + i} = (-i)^h W_L^i
    cf b = cf{hi ? v[hi_slot].y : recv.x, hi ? -v[hi_slot].x : recv.y};
    bfly<i, L>(a, b);                                           // a + W_L^i b, a - W_L^i b
    out[i] = a;
    out[Q + i] = b;
  });
  sfor<0, H>([&](auto i_) { v[decltype(i_)::value] = out[decltype(i_)::value]; });
}

template <int L, typename Xchg>
MPBP_DI void fft_pair_blk_to_dec(cf (&v)[L / 2], int h, Xchg&& xchg) {
  constexpr int H = L / 2, Q = L / 4;
  cf w[H];
  const bool hi = h != 0;
  sfor<0, Q>([&](auto i_) {
    constexpr int i = decltype(i_)::value;
    const cf a = cadd(v[i], v[Q + i]);                    // x[n] + x[n+H], n = Q h + i
    const cf b = twmul<i, L>(csub(v[i], v[Q + i]));       // (x[n] - x[n+H]) W_L^i; times (-i)^h below
    const cf recv = xchg(csel(hi, a, b));                 // the low thread keeps the sums
    w[i] = csel(hi, recv, a);
    w[Q + i] = cf{hi ? b.y : recv.x, hi ? -b.x : recv.y};
  });
  fft_line<H>(w);
  sfor<0, H>([&](auto i_) { v[decltype(i_)::value] = w[decltype(i_)::value]; });
}

}  // namespace mpbp
