// fft_reg.cuh -- register-resident radix-2 FFT lines for the far-field
// transform F of Eq. 2 (unnormalised, kernel exp(-2 pi i q k / L)).
//
// One thread holds one line of L complex values in registers.  Every index is
// a compile-time constant after unrolling, so the bit-reversed storage order
// costs nothing: the result X[k] lives in register slot brev(k).  Twiddles are
// compile-time constants evaluated by constexpr trigonometry (octant reduction
// of the exact dyadic angle plus a Taylor series in double), so they become
// immediate operands of FFMA instead of loads.
#pragma once

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define MPBP_HD __host__ __device__
#define MPBP_DI __device__ __forceinline__
#else
#define MPBP_HD
#define MPBP_DI inline
#endif

#include <type_traits>

namespace mpbp {

// ----------------------------------------------------------------------------
// compile-time trigonometry on turns (angle = 2 pi p)
// ----------------------------------------------------------------------------
namespace ct {
constexpr double kTwoPi = 6.28318530717958647692528676655900577;

MPBP_HD constexpr double sin_series(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int n = 1; n < 16; ++n) {
    term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
MPBP_HD constexpr double cos_series(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int n = 1; n < 16; ++n) {
    term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
MPBP_HD constexpr double sin_turn(double p);
// cos(2 pi p) for p in [0, 1); p is a dyadic rational, so every reduction
// below is exact and the series only sees angles up to pi/4.
MPBP_HD constexpr double cos_turn(double p) {
  return p >= 0.5    ? -cos_turn(p - 0.5)
         : p > 0.25  ? -sin_turn(p - 0.25)
         : p > 0.125 ? sin_turn(0.25 - p)
                     : cos_series(kTwoPi * p);
}
MPBP_HD constexpr double sin_turn(double p) {
  return p >= 0.5    ? -sin_turn(p - 0.5)
         : p > 0.25  ? cos_turn(p - 0.25)
         : p > 0.125 ? cos_turn(0.25 - p)
                     : sin_series(kTwoPi * p);
}
// W_N^K = exp(-2 pi i K / N)
template <int K, int N>
struct Tw {
  static constexpr int k = ((K % N) + N) % N;
  static constexpr float re = static_cast<float>(cos_turn(double(k) / double(N)));
  static constexpr float im = static_cast<float>(-sin_turn(double(k) / double(N)));
};

MPBP_HD constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }
template <int L>
MPBP_HD constexpr int brev(int i) {
  int r = 0;
  for (int b = 1; b < L; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}
}  // namespace ct

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, typename F>
MPBP_DI void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

struct alignas(8) cf {
  float x, y;
};

MPBP_DI cf mk(float a, float b) { return cf{a, b}; }
MPBP_DI cf cmul(cf a, cf b) {
  return cf{fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}

// radix-2 butterfly with a compile-time twiddle w = W_N^K:
//   a' = a + w b,  b' = a - w b  (b' formed as 2a - a' with one FFMA each)
template <int K, int N>
MPBP_DI void bfly(cf& a, cf& b) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    cf t = b;
    b = cf{a.x - t.x, a.y - t.y};
    a = cf{a.x + t.x, a.y + t.y};
  } else if constexpr (4 * k == N) {  // w = -i
    cf t = cf{b.y, -b.x};
    b = cf{a.x - t.x, a.y - t.y};
    a = cf{a.x + t.x, a.y + t.y};
  } else if constexpr (2 * k == N) {  // w = -1
    cf t = b;
    b = cf{a.x + t.x, a.y + t.y};
    a = cf{a.x - t.x, a.y - t.y};
  } else if constexpr (4 * k == 3 * N) {  // w = +i
    cf t = cf{-b.y, b.x};
    b = cf{a.x - t.x, a.y - t.y};
    a = cf{a.x + t.x, a.y + t.y};
  } else {
    constexpr float wr = ct::Tw<K, N>::re, wi = ct::Tw<K, N>::im;
    float r = fmaf(wr, b.x, fmaf(-wi, b.y, a.x));
    float i = fmaf(wr, b.y, fmaf(wi, b.x, a.y));
    b = cf{fmaf(2.0f, a.x, -r), fmaf(2.0f, a.y, -i)};
    a = cf{r, i};
  }
}

// In-place L-point forward DFT of x[0..L) (natural order in).  Decimation in
// time on the bit-reversed view of the array: afterwards X[k] = x[brev(k)].
template <int L>
MPBP_DI void fft_line(cf (&x)[L]) {
  constexpr int LOG = ct::ilog2(L);
  sfor<0, LOG>([&](auto s_) {
    constexpr int span = 1 << decltype(s_)::value;
    sfor<0, L / 2>([&](auto b_) {
      constexpr int b = decltype(b_)::value;
      constexpr int grp = b / span, k = b % span;
      constexpr int i0 = ct::brev<L>(grp * 2 * span + k);
      constexpr int i1 = ct::brev<L>(grp * 2 * span + k + span);
      bfly<k, 2 * span>(x[i0], x[i1]);
    });
  });
}

// multiply by a compile-time twiddle W_N^K
template <int K, int N>
MPBP_DI cf twmul(cf v) {
  constexpr int k = ((K % N) + N) % N;
  if constexpr (k == 0) {
    return v;
  } else if constexpr (4 * k == N) {
    return cf{v.y, -v.x};
  } else if constexpr (2 * k == N) {
    return cf{-v.x, -v.y};
  } else if constexpr (4 * k == 3 * N) {
    return cf{-v.y, v.x};
  } else {
    constexpr float wr = ct::Tw<K, N>::re, wi = ct::Tw<K, N>::im;
    return cf{fmaf(wr, v.x, -wi * v.y), fmaf(wr, v.y, wi * v.x)};
  }
}

}  // namespace mpbp
