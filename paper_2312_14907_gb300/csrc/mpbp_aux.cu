// mpbp_aux.cu -- per-pixel and reduction kernels around the fused frame kernel:
//   A1  object synthesis O_m = alpha_m rho exp(i phi_m)          (Eq. 1, Eq. 3)
//   data layout: a = sqrt(y) stored transposed per frame
//   A6/A7 tail: gradient assembly from the patch accumulator
//   A8  fixed-order FP64 reductions, the line-search decision and the update
//       of mpbp_step (applied by the gradient assembly, pixel by pixel)
#include "aux_launch.h"

#include <algorithm>

namespace mpbp {

// ----------------------------------------------------------------------------
// A1: objects
// ----------------------------------------------------------------------------
// PHI: the phases phi_m are given per peak (the per-peak-phase variables of
// the paper's two-step reconstruction) instead of derived from u
template <bool PHI>
__global__ void object_build_kernel(ObjectArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < a.npix; p += stride) {
    const float r = a.rho[p];
    float uc[kMaxComp];
#pragma unroll
    for (int c = 0; c < kMaxComp; ++c) uc[c] = !PHI && c < a.C ? a.u[c * a.npix + p] : 0.f;
#pragma unroll
    for (int m = 0; m < kMaxPeaks; ++m) {
      if (m < a.D) {
        float sn, cs;
        if constexpr (PHI) {
          sincosf(a.phi[m * a.npix + p], &sn, &cs);
        } else {
          float arg = 0.f;
#pragma unroll
          for (int c = 0; c < kMaxComp; ++c) arg = fmaf(a.pc.kpi[m][c], uc[c], arg);
          sincospif(arg, &sn, &cs);   // exp(i phi), phi = pi * arg
        }
        const float amp = a.alpha[m] * r;
        reinterpret_cast<float2*>(a.O)[m * a.npix + p] = make_float2(amp * cs, amp * sn);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// 16-bit photon counts to floats (exact), for the paths that read floats
// ----------------------------------------------------------------------------
__global__ void counts16_kernel(const unsigned short* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// ----------------------------------------------------------------------------
// data: out[f][q1][q0] = g(in[f][q0][q1]), g = sqrt or identity
// ----------------------------------------------------------------------------
template <bool SQRT>
__global__ void frame_transpose_kernel(const float* __restrict__ in, float* __restrict__ out,
                                       int m, int ts, long long nblocks_per_frame_side) {
  __shared__ float tile[32][33];
  const long long tiles_per_frame = nblocks_per_frame_side * nblocks_per_frame_side;
  const long long b = blockIdx.x;
  const long long f = b / tiles_per_frame;
  const int tb = (int)(b - f * tiles_per_frame);
  const int t0 = (tb / (int)nblocks_per_frame_side) * ts;  // tile row origin (q0)
  const int t1 = (tb % (int)nblocks_per_frame_side) * ts;  // tile col origin (q1)
  const float* src = in + f * m * m;
  float* dst = out + f * m * m;
  for (int i = threadIdx.y; i < ts; i += blockDim.y) {
    for (int j = threadIdx.x; j < ts; j += blockDim.x) {
      float v = src[(long long)(t0 + i) * m + t1 + j];
      tile[i][j] = SQRT ? sqrtf(v) : v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < ts; i += blockDim.y) {
    for (int j = threadIdx.x; j < ts; j += blockDim.x) {
      dst[(long long)(t1 + i) * m + t0 + j] = tile[j][i];
    }
  }
}

// ----------------------------------------------------------------------------
// gradient assembly.  With T_m = E_m acc_m (E_m = exp(i phi_m)):
//   df/drho = sum_m alpha_m Re T_m,  df/dphi_m = -alpha_m rho Im T_m,
//   df/du_c = sum_m phase_scale G_{m,c} df/dphi_m,  df/dalpha_m = sum_r rho Re T_m.
// acc is cleared behind the read so the next evaluation starts from zero.
// ----------------------------------------------------------------------------

// ----------------------------------------------------------------------------
// A8: fixed-order FP64 reductions and the optional line-search decision, run
// by the last block of the gradient-assembly grid to finish (one warp per
// reduced quantity, partials read in a fixed order, so the result does not
// depend on which block finishes last)
// ----------------------------------------------------------------------------
constexpr int kReduceLoads = 20;   // partials per lane issued together (up to 640 blocks)

// One lane's share of a fixed-order sum over n partials p[i * stride]: the
// lane adds i = lane, lane + 32, ... in index order (all its loads in flight
// at once when n <= 32 kReduceLoads).  Followed by a shuffle tree, the same
// partials give the same bits in every block that sums them.
__device__ __forceinline__ double warp_slice_sum(const double* p, long long n, long long stride, int lane) {
  double v = 0.0;
  if (n <= 32 * kReduceLoads) {
    double xv[kReduceLoads];
#pragma unroll
    for (int k = 0; k < kReduceLoads; ++k) {
      const int i = lane + 32 * k;
      xv[k] = i < n ? __ldcg(p + i * stride) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < kReduceLoads; ++k)
      if (lane + 32 * k < n) v += xv[k];
  } else {
    for (long long i = lane; i < n; i += 32) v += __ldcg(p + i * stride);
  }
  return v;
}

// The optimizer state as one thread reads it: every field loaded at once, so
// the reads cost one round trip and can be issued long before they are used.
struct StepView {
  double f_prev, gn2_prev, t, c_armijo, grow, shrink, w_rho, w_u, w_alpha;
  int k, n_accept, n_reject;
};

__device__ __forceinline__ StepView load_state(const mpbp_step_state* st) {
  StepView v;
  v.f_prev = __ldcg(&st->f_prev);
  v.gn2_prev = __ldcg(&st->gn2_prev);
  v.t = __ldcg(&st->t);
  v.c_armijo = __ldcg(&st->c_armijo);
  v.grow = __ldcg(&st->grow);
  v.shrink = __ldcg(&st->shrink);
  v.w_rho = __ldcg(&st->w_rho);
  v.w_u = __ldcg(&st->w_u);
  v.w_alpha = __ldcg(&st->w_alpha);
  v.k = __ldcg(&st->k);
  v.n_accept = __ldcg(&st->n_accept);
  v.n_reject = __ldcg(&st->n_reject);
  return v;
}

// The lagged Armijo test of an optimizer step: a pure function of the state
// and the loss at the trial point, so every block of the gradient assembly
// reaches the same decision as the block that records it.
struct StepDecision {
  bool accept;
  double t_new;   // step length of the next trial
};

__device__ StepDecision step_decide(const StepView& st, double loss) {
  const bool finite = isfinite(loss);
  StepDecision d;
  if (st.k == 0) d.accept = finite;
  else d.accept = finite && (loss <= st.f_prev - st.c_armijo * st.t * st.gn2_prev);
  d.t_new = d.accept ? (st.k > 0 ? st.t * st.grow : st.t) : st.t * st.shrink;
  return d;
}

// STEP: the loss is the block's own fixed-order sum of all frame-kernel
// partials (loss_all), and the alpha update of the step follows the decision
// (thread m updates alpha_m).  The state and the alpha values are read
// before the partials, so their latency overlaps the partial sums.
template <int T, bool STEP>
__device__ void final_reduce(const ReduceArgs& a, double loss_all) {
  __shared__ double vals[kMaxPeaks + 3];
  __shared__ int s_accept;
  __shared__ double s_step;   // t_new * w_alpha
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  mpbp_step_state* st = a.st;
  StepView sv{};
  if (st && threadIdx.x == 0) sv = load_state(st);
  const StepPtrs& x = a.step;
  float al = 0.f, alb = 0.f;
  double galb = 0.0;
  if (STEP && threadIdx.x < a.D) {
    al = __ldcg(x.alpha + threadIdx.x);
    alb = __ldcg(x.alpha_base + threadIdx.x);
    galb = __ldcg(x.g_alpha_base + threadIdx.x);
  }
  const int nq = a.D + 3;   // loss, df/dalpha_m (D), |g_rho|^2, |g_u|^2
  for (int q = (STEP ? 1 : 0) + w; q < nq; q += T / 32) {
    // per-block partials: column D + 2 is the loss, columns 0..D+1 as named
    const int col = q == 0 ? a.D + 2 : q - 1;
    double v = warp_slice_sum(a.part + col, a.n_part, a.D + 3, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) vals[q] = v;
  }
  __syncthreads();
  const double* galpha = vals + 1;
  if (threadIdx.x == 0) {
    const double loss = STEP ? loss_all : vals[0];
    const bool finite = isfinite(loss);
    if (!finite) atomicOr(a.err, kErrNonfinite);
    if (a.loss_out) *a.loss_out = loss;
    for (int m = 0; m < a.D; ++m) {
      if (a.g_alpha_out) a.g_alpha_out[m] = galpha[m];
      if (a.g_alpha_ws) a.g_alpha_ws[m] = galpha[m];
    }
    if (st) {
      // lagged Armijo decision in FP64; weighted squared norm of the descent
      // direction (alpha_0 is not a variable)
      double gn2 = sv.w_rho * galpha[a.D] + sv.w_u * galpha[a.D + 1];
      for (int m = a.alpha_from; m < a.D; ++m) gn2 += sv.w_alpha * galpha[m] * galpha[m];
      const StepDecision d = step_decide(sv, loss);
      if (d.accept) {
        st->f_prev = loss;
        st->gn2_prev = gn2;
        st->n_accept = sv.n_accept + 1;
      } else {
        st->n_reject = sv.n_reject + 1;
      }
      st->t = d.t_new;
      st->accepted = d.accept ? 1 : 0;
      st->f_last = loss;
      st->k = sv.k + 1;
      s_accept = d.accept ? 1 : 0;
      s_step = d.t_new * sv.w_alpha;
    }
  }
  if constexpr (STEP) {
    // alpha = alpha_base - t w g_alpha_base, alpha_0 held fixed; every block
    // has finished reading alpha
    __syncthreads();
    const int m = threadIdx.x;
    if (m < a.D) {
      double base, gbase;
      if (s_accept) {
        base = al;
        gbase = galpha[m];
        x.alpha_base[m] = al;
        x.g_alpha_base[m] = gbase;
      } else {
        base = alb;
        gbase = galb;
      }
      x.alpha[m] = m < a.alpha_from ? (float)base : (float)(base - s_step * gbase);
    }
  }
}

constexpr int kFinishThreads = 256;
constexpr int kFinishPixelsPerThread = 1;   // latency-bound: many warps, few pixels each

// the loads of one pixel, issued together before its phase arithmetic
template <bool PHI>
struct PixelIn {
  float r;
  float uc[kMaxComp];
  float2 Am[kMaxPeaks];
};

template <bool PHI>
__device__ __forceinline__ void pixel_load(const FinishArgs& a, long long p, PixelIn<PHI>& in) {
  const float2* acc = reinterpret_cast<const float2*>(a.acc);
  in.r = a.rho[p];
#pragma unroll
  for (int c = 0; c < kMaxComp; ++c) in.uc[c] = !PHI && c < a.C ? a.u[c * a.npix + p] : 0.f;
#pragma unroll
  for (int m = 0; m < kMaxPeaks; ++m) in.Am[m] = m < a.D ? __ldcg(acc + m * a.npix + p) : make_float2(0.f, 0.f);
}

// STEP: mpbp_step's update x = x_base - t w g_base is applied here, pixel by
// pixel, after a decision that every block takes from the same fixed-order
// loss sum; the last block updates alpha and records the state.
template <bool PHI, bool STEP>
__global__ void __launch_bounds__(kFinishThreads) finish_kernel(FinishArgs a, ReduceArgs ra) {
  constexpr int NW = kFinishThreads / 32;
  constexpr int NQ = kMaxPeaks + 3;
  __shared__ double wsum[NW][NQ];
  __shared__ double s_loss;
  __shared__ float s_w[2];
  __shared__ int s_accept;
  __shared__ bool last;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float ap[kMaxPeaks];   // df/dalpha_m partials of this thread
#pragma unroll
  for (int m = 0; m < kMaxPeaks; ++m) ap[m] = 0.f;
  float n_rho = 0.f, n_u = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long p0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // the frame kernel's loss partials (FP64), issued first: this block's
  // slice of them, or with STEP all of them in a fixed order
  double lp = 0.0;
  StepView sv{};
  if constexpr (STEP) {
    // warp 0 sums all of them (the FP64 pipe is narrow; one warp's share
    // of the adds and one shuffle tree)
    if (threadIdx.x == 0) sv = load_state(ra.st);
    if (w == 0) lp = warp_slice_sum(a.loss_part, a.n_loss_part, 1, lane);
  } else {
    for (long long i = p0; i < a.n_loss_part; i += stride) lp += __ldcg(a.loss_part + i);
  }
  PixelIn<PHI> in;
  if (p0 < a.npix) pixel_load<PHI>(a, p0, in);
  if (!STEP || w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, o);
  }
  bool accept = false;
  float wr = 0.f, wu = 0.f;
  if constexpr (STEP) {
    if (threadIdx.x == 0) {
      const StepDecision d = step_decide(sv, lp);
      s_loss = lp;
      s_accept = d.accept ? 1 : 0;
      s_w[0] = (float)(d.t_new * sv.w_rho);
      s_w[1] = (float)(d.t_new * sv.w_u);
    }
    __syncthreads();
    accept = s_accept != 0;
    wr = s_w[0];
    wu = s_w[1];
  }
  float2* acc = reinterpret_cast<float2*>(a.acc);
  for (long long p = p0; p < a.npix; p += stride) {
    const float r = in.r;
    float gr = 0.f, gphi2 = 0.f;
    float gu[kMaxComp] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m < kMaxPeaks; ++m) {
      if (m < a.D) {
        float sn, cs;
        if constexpr (PHI) {
          sincosf(a.phi[m * a.npix + p], &sn, &cs);
        } else {
          float arg = 0.f;
#pragma unroll
          for (int c = 0; c < kMaxComp; ++c) arg = fmaf(a.pc.kpi[m][c], in.uc[c], arg);
          sincospif(arg, &sn, &cs);
        }
        const float2 A = in.Am[m];
        acc[m * a.npix + p] = make_float2(0.f, 0.f);
        const float Tr = fmaf(cs, A.x, -sn * A.y);
        const float Ti = fmaf(cs, A.y, sn * A.x);
        const float am = a.alpha[m];
        gr = fmaf(am, Tr, gr);
        const float dphi = -am * r * Ti;
        if constexpr (PHI) {
          a.g_phi[m * a.npix + p] = dphi;
          gphi2 = fmaf(dphi, dphi, gphi2);
        } else {
#pragma unroll
          for (int c = 0; c < kMaxComp; ++c) gu[c] = fmaf(a.pc.kps[m][c], dphi, gu[c]);
        }
        ap[m] = fmaf(r, Tr, ap[m]);
      }
    }
    a.g_rho[p] = gr;
    float su = gphi2;   // |g_phi|^2 in the phase form, |g_u|^2 otherwise
    if constexpr (!PHI) {
#pragma unroll
      for (int c = 0; c < kMaxComp; ++c) {
        if (c < a.C) {
          a.g_u[c * a.npix + p] = gu[c];
          su = fmaf(gu[c], gu[c], su);
        }
      }
    }
    if constexpr (STEP) {
      const StepPtrs& x = ra.step;
      float base, gbase;
      if (accept) {
        base = r;
        gbase = gr;
        x.rho_base[p] = base;
        x.g_rho_base[p] = gbase;
      } else {
        base = x.rho_base[p];
        gbase = x.g_rho_base[p];
      }
      x.rho[p] = fmaf(-wr, gbase, base);
#pragma unroll
      for (int c = 0; c < kMaxComp; ++c) {
        if (c < a.C) {
          const long long i = c * a.npix + p;
          if (accept) {
            base = in.uc[c];
            gbase = gu[c];
            x.u_base[i] = base;
            x.g_u_base[i] = gbase;
          } else {
            base = x.u_base[i];
            gbase = x.g_u_base[i];
          }
          x.u[i] = fmaf(-wu, gbase, base);
        }
      }
    }
    n_rho = fmaf(gr, gr, n_rho);
    n_u += su;
    if (p + stride < a.npix) pixel_load<PHI>(a, p + stride, in);
  }
  // partial sums: FP32 within the warp (a few pixels per lane), FP64 across
  // warps and blocks; one barrier for all D + 3 quantities
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (q < a.D + 2) {
      float v = q < a.D ? ap[q < kMaxPeaks ? q : 0] : (q == a.D ? n_rho : n_u);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[w][q] = (double)v;
    }
  }
  if (lane == 0) wsum[w][a.D + 2] = lp;
  __syncthreads();
  double* out = a.part + (long long)blockIdx.x * (a.D + 3);
  if (w == 0 && lane < a.D + 3) {
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < NW; ++i) t += wsum[i][lane];
    out[lane] = t;
    __threadfence();   // publish this block's partials before counting it in
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.arrivals, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  final_reduce<kFinishThreads, STEP>(ra, STEP ? s_loss : 0.0);
}

// The loss alone (mpbp_loss): one warp sums the frame kernel's per-block
// partials in a fixed order (the same bits as the gradient assembly's
// sum of them) and flags a non-finite result.
__global__ void loss_reduce_kernel(const double* __restrict__ part, long long n, double* loss, int* err) {
  const int lane = threadIdx.x & 31;
  double v = warp_slice_sum(part, n, 1, lane);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    *loss = v;
    if (!isfinite(v)) atomicOr(err, kErrNonfinite);
  }
}

// ----------------------------------------------------------------------------
// The deterministic gradient (A7): acc_m(row, col) = the sum, in piece
// order, of the pieces covering that pixel (a piece holds the gradient rows
// one block wrote back for a run of frames of one column strip; DetPlan),
// the candidates listed per (peak, column, band of w rows).
// One thread per pixel of the D object-sized accumulators, consecutive
// threads on consecutive columns; every pixel is written, so acc needs no
// clearing before.
// ----------------------------------------------------------------------------
constexpr int kDetThreads = 256;

__global__ void __launch_bounds__(kDetThreads) det_reduce_kernel(const DetPlan* __restrict__ plan, cf* acc, int D,
                                                                  int n1, int n2, int w) {
  const long long npix = (long long)n1 * n2;
  const int nband = (n1 + w - 1) / w;
  const cf* pool = plan->pool;
  const DetPiece* pieces = plan->pieces;
  const int* col_start = plan->col_start;
  const int* col_piece = plan->col_piece;
  for (long long i = blockIdx.x * (long long)kDetThreads + threadIdx.x; i < npix * D;
       i += (long long)gridDim.x * kDetThreads) {
    const int m = (int)(i / npix);
    const long long rc = i - m * npix;
    const int row = (int)(rc / n2), col = (int)(rc - (long long)row * n2);
    const long long key = ((long long)m * n2 + col) * nband + row / w;
    const int k0 = col_start[key], k1 = col_start[key + 1];
    float sx = 0.0f, sy = 0.0f;
    for (int k = k0; k < k1; ++k) {
      const DetPiece pc = pieces[col_piece[k]];
      const int r = row - pc.row0;
      if (r >= 0 && r < pc.rows) {
        const cf v = pool[pc.off + (long long)r * w + (col - pc.y)];
        sx += v.x;
        sy += v.y;
      }
    }
    acc[i] = cf{sx, sy};
  }
}

cudaError_t launch_det_reduce(const DetPlan* plan, cf* acc, int D, int n1, int n2, int w, int num_sms,
                              cudaStream_t s) {
  const long long n = (long long)D * n1 * n2;
  const long long need = (n + kDetThreads - 1) / kDetThreads;
  const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms * 8));
  det_reduce_kernel<<<grid, kDetThreads, 0, s>>>(plan, acc, D, n1, n2, w);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Probes for scan positions off the pixel grid (Eq. 2's shift S_j at a real
// position s_j = n_j + d_j): frame j keeps the integer window n_j and takes
// P(k - d_j).  With the frequencies of each axis in [-M/2, M/2) the
// band-limited interpolation is separable,
//   P_d(k0, k1) = sum_{k0', k1'} D(k0 - k0' - d0) D(k1 - k1' - d1) P(k0', k1'),
//   D(y) = (1/M) sum_q exp(2 pi i q y / M) = sin(pi y) / (M sin(pi y / M)) exp(-i pi y / M),
// D(0) = 1 and D(n) = 0 at the other integers.  One block per output probe:
// the probe in shared memory, one pass along k1 (a warp per row), one along
// k0 (a warp per column), each output a length-M sum in FP32.
// ----------------------------------------------------------------------------
constexpr int kShiftThreads = 256;

__device__ float2 interp_weight(float y, int m) {
  if (y == 0.0f) return make_float2(1.0f, 0.0f);
  const float a = sinpif(y) / ((float)m * sinpif(y / (float)m));
  float sn, cs;
  sincospif(-y / (float)m, &sn, &cs);
  return make_float2(a * cs, a * sn);
}

__device__ __forceinline__ float2 cfma(float2 w, float2 v, float2 acc) {
  acc.x = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc.x));
  acc.y = fmaf(w.x, v.y, fmaf(w.y, v.x, acc.y));
  return acc;
}

__global__ void __launch_bounds__(kShiftThreads) probe_shift_kernel(ProbeShiftArgs a) {
  extern __shared__ float2 sm[];   // w0 [2M], w1 [2M], buf [M][M + 1]
  const int m = a.m, ld = m + 1;
  const int i = blockIdx.x;
  const int j = a.per_peak ? i % a.J : i;
  const int src = a.per_peak ? i / a.J : 0;
  float2* w0 = sm;
  float2* w1 = sm + 2 * m;
  float2* buf = sm + 4 * m;
  const float2 d = a.d[j];
  for (int t = threadIdx.x; t < 2 * m - 1; t += blockDim.x) {
    const float x = (float)(t - (m - 1));   // k - k'
    w0[t] = interp_weight(x - d.x, m);
    w1[t] = interp_weight(x - d.y, m);
  }
  const float2* P = reinterpret_cast<const float2*>(a.src) + (size_t)src * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) buf[(e / m) * ld + e % m] = P[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  // along k1: warp per row, lane outputs k1 = lane + 32 u (M <= 128)
  for (int r = warp; r < m; r += nw) {
    float2 o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = lane + 32 * u;
      float2 acc = make_float2(0.0f, 0.0f);
      if (c < m)
        for (int cp = 0; cp < m; ++cp) acc = cfma(w1[c - cp + m - 1], buf[r * ld + cp], acc);
      o[u] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (lane + 32 * u < m) buf[r * ld + lane + 32 * u] = o[u];
    __syncwarp();
  }
  __syncthreads();
  // along k0: warp per column
  for (int c = warp; c < m; c += nw) {
    float2 o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = lane + 32 * u;
      float2 acc = make_float2(0.0f, 0.0f);
      if (r < m)
        for (int rp = 0; rp < m; ++rp) acc = cfma(w0[r - rp + m - 1], buf[rp * ld + c], acc);
      o[u] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (lane + 32 * u < m) buf[(lane + 32 * u) * ld + c] = o[u];
    __syncwarp();
  }
  __syncthreads();
  float2* out = reinterpret_cast<float2*>(a.out) + (size_t)i * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) out[e] = buf[(e / m) * ld + e % m];
}

static int probe_shift_smem(int m) { return (int)sizeof(float2) * (4 * m + m * (m + 1)); }

bool probe_shift_prepare(int m) {
  if (m < 1 || m > 128) return false;
  return cudaFuncSetAttribute(probe_shift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              probe_shift_smem(m)) == cudaSuccess;
}

cudaError_t launch_probe_shift(const ProbeShiftArgs& a, cudaStream_t s) {
  if (a.m < 1 || a.m > 128 || a.nout < 0) return cudaErrorInvalidValue;
  if (a.nout == 0) return cudaSuccess;
  probe_shift_kernel<<<a.nout, kShiftThreads, probe_shift_smem(a.m), s>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
static int grid_for(long long n, int threads, int cap) {
  long long g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_object_build(const ObjectArgs& a, int num_sms, cudaStream_t s) {
  if (a.phi) object_build_kernel<true><<<grid_for(a.npix, 256, num_sms * 8), 256, 0, s>>>(a);
  else object_build_kernel<false><<<grid_for(a.npix, 256, num_sms * 8), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_counts16(const unsigned short* in, float* out, long long n, int num_sms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  counts16_kernel<<<grid_for(n, 256, num_sms * 8), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_frame_transpose(const float* in, float* out, long long nframes, int m,
                                   bool take_sqrt, cudaStream_t s) {
  const int ts = m < 32 ? m : 32;
  const long long side = m / ts;
  const long long nb = nframes * side * side;
  if (nb == 0) return cudaSuccess;
  dim3 block(ts, ts < 8 ? ts : 8);
  if (take_sqrt) frame_transpose_kernel<true><<<(unsigned)nb, block, 0, s>>>(in, out, m, ts, side);
  else frame_transpose_kernel<false><<<(unsigned)nb, block, 0, s>>>(in, out, m, ts, side);
  return cudaGetLastError();
}

int finish_grid(long long npix, int num_sms) {
  return grid_for((npix + kFinishPixelsPerThread - 1) / kFinishPixelsPerThread, kFinishThreads,
                  num_sms * 4);
}

cudaError_t launch_loss_reduce(const double* part, long long n, double* loss, int* err, cudaStream_t s) {
  loss_reduce_kernel<<<1, 32, 0, s>>>(part, n, loss, err);
  return cudaGetLastError();
}

cudaError_t launch_finish(const FinishArgs& a, const ReduceArgs& r, int grid, cudaStream_t s) {
  if (a.phi) {
    if (r.step.rho) return cudaErrorInvalidValue;   // the step updates u, not per-peak phases
    finish_kernel<true, false><<<grid, kFinishThreads, 0, s>>>(a, r);
  } else if (r.step.rho) {
    if (!r.st) return cudaErrorInvalidValue;
    finish_kernel<false, true><<<grid, kFinishThreads, 0, s>>>(a, r);
  } else {
    finish_kernel<false, false><<<grid, kFinishThreads, 0, s>>>(a, r);
  }
  return cudaGetLastError();
}

}  // namespace mpbp
