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

// W_8^g, g in 0..3
MPBP_DI cf w8_pow(int g) {
  const float re = g == 0 ? 1.0f : g == 1 ? ct::Tw<1, 8>::re : g == 2 ? ct::Tw<2, 8>::re : ct::Tw<3, 8>::re;
  const float im = g == 0 ? 0.0f : g == 1 ? ct::Tw<1, 8>::im : g == 2 ? ct::Tw<2, 8>::im : ct::Tw<3, 8>::im;
  return cf{re, im};
}

template <int L, typename X8, typename X16>
MPBP_DI void fft_quad_dec_to_blk(cf (&v)[L / 4], int h0, int h1, X8&& xchg8, X16&& xchg16) {
  constexpr int Q = L / 8;
  fft_pair_dec_to_blk<L / 2>(v, h1, xchg16);   // E_h0[k] for k = Q h1 + i, L/4 + Q h1 + i
  const bool hi = h0 != 0;
  const cf cg = w8_pow(2 * h0 + h1);
  cf out[L / 4];
  sfor<0, Q>([&](auto t_) {
    constexpr int t = decltype(t_)::value;
    const cf mine = csel(hi, v[Q + t], v[t]);   // E_h0[Q g + t]
    const cf send = csel(hi, v[t], v[Q + t]);   // what the partner keeps
    const cf recv = xchg8(send);
    const cf e0 = csel(hi, recv, mine);
    const cf e1 = csel(hi, mine, recv);
    const cf tw = cmul(twmul<t, L>(e1), cg);    // W_L^{Q g + t} E_1
    out[t] = cadd(e0, tw);
    out[Q + t] = csub(e0, tw);
  });
  sfor<0, L / 4>([&](auto i_) { v[decltype(i_)::value] = out[decltype(i_)::value]; });
}

template <int L, typename X8, typename X16>
MPBP_DI void fft_quad_blk_to_dec(cf (&v)[L / 4], int h0, int h1, X8&& xchg8, X16&& xchg16) {
  constexpr int Q = L / 8;
  const bool hi = h0 != 0;
  const cf cg = w8_pow(2 * h0 + h1);
  cf w[L / 4];
  sfor<0, Q>([&](auto t_) {
    constexpr int t = decltype(t_)::value;
    const cf a = cadd(v[t], v[Q + t]);                          // even outputs
    const cf b = cmul(twmul<t, L>(csub(v[t], v[Q + t])), cg);   // odd outputs, W_L^{Q g + t}
    const cf keep = csel(hi, b, a);
    const cf recv = xchg8(csel(hi, a, b));
    w[t] = csel(hi, recv, keep);
    w[Q + t] = csel(hi, keep, recv);
  });
  fft_pair_blk_to_dec<L / 2>(w, h1, xchg16);
  sfor<0, L / 4>([&](auto i_) { v[decltype(i_)::value] = w[decltype(i_)::value]; });
}

}  // namespace mpbp
