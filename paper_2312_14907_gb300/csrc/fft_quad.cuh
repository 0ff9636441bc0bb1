// fft_quad.cuh -- L-point FFT lines split over four threads (h = 2 h1 + h0;
// the h0 partner is lane ^ 8, the h1 partner lane ^ 16), L/4 values each.
//
// With Q = L/8 and g = 2 h0 + h1:
//   "dec4" layout: thread h holds x[4n + h] in slot n, n = 0..L/4-1
//   "blk4" layout: thread holds X[Q g + t] in slot t and X[L/2 + Q g + t] in
//                  slot Q + t, t = 0..Q-1
// dec4 -> blk4 is decimation in time: each h0-subsequence x[2n' + h0] is an
// (L/2)-point line over the h1 pair (fft_pair.cuh), then the last radix-2
// stage runs across h0.  blk4 -> dec4 is decimation in frequency: the first
// radix-2 stage across h0 (no data move is needed to form it: a thread holds
// both X[n] and X[n + L/2]), then an (L/2)-point pair line across h1, whose
// output X[4k + h] sits in slot brev_{L/4}(k).  The twiddle of index Q g + t
// is W_L^t (a compile-time constant) times W_8^g (one per thread).
#pragma once
#include "fft_pair.cuh"

namespace mpbp {

// W_8^h1 for h1 in {0, 1}: the per-thread factor of the cross-thread twiddle
// W_L^{Q g + t} = W_L^t W_8^h1 (-i)^h0 (g = 2 h0 + h1; (-i)^h0 is folded into
// the selects)
MPBP_DI cf w8_h1(int h1) {
  return cf{h1 ? ct::Tw<1, 8>::re : 1.0f, h1 ? ct::Tw<1, 8>::im : 0.0f};
}

template <int L, typename X8, typename X16>
MPBP_DI void fft_quad_dec_to_blk(cf (&v)[L / 4], int h0, int h1, X8&& xchg8, X16&& xchg16) {
  constexpr int Q = L / 8;
  fft_pair_dec_to_blk<L / 2>(v, h1, xchg16);   // E_h0[k] for k = Q h1 + i, L/4 + Q h1 + i
  const bool hi = h0 != 0;
  const cf c1 = w8_h1(h1);
  cf out[L / 4];
  sfor<0, Q>([&](auto t_) {
    constexpr int t = decltype(t_)::value;
    const cf recv = xchg8(csel(hi, v[t], v[Q + t]));   // E_{1-h0}[Q g + t]
    cf a = csel(hi, recv, v[t]);                        // E_0[Q g + t]
    cf b = cf{hi ? v[Q + t].y : recv.x, hi ? -v[Q + t].x : recv.y};   // (-i)^h0 E_1[Q g + t]
    b = cmul(b, c1);
    bfly<t, L>(a, b);                                   // a + W_L^t b, a - W_L^t b
    out[t] = a;
    out[Q + t] = b;
  });
  sfor<0, L / 4>([&](auto i_) { v[decltype(i_)::value] = out[decltype(i_)::value]; });
}

template <int L, typename X8, typename X16>
MPBP_DI void fft_quad_blk_to_dec(cf (&v)[L / 4], int h0, int h1, X8&& xchg8, X16&& xchg16) {
  constexpr int Q = L / 8;
  const bool hi = h0 != 0;
  const cf c1 = w8_h1(h1);
  cf w[L / 4];
  sfor<0, Q>([&](auto t_) {
    constexpr int t = decltype(t_)::value;
    const cf a = cadd(v[t], v[Q + t]);                                  // even outputs
    const cf b = cmul(twmul<t, L>(csub(v[t], v[Q + t])), c1);          // odd: W_L^t W_8^h1; (-i)^h0 below
    const cf recv = xchg8(csel(hi, a, b));                              // the h0 = 0 thread keeps the sums
    w[t] = csel(hi, recv, a);
    w[Q + t] = cf{hi ? b.y : recv.x, hi ? -b.x : recv.y};
  });
  fft_pair_blk_to_dec<L / 2>(w, h1, xchg16);
  sfor<0, L / 4>([&](auto i_) { v[decltype(i_)::value] = w[decltype(i_)::value]; });
}

}  // namespace mpbp
