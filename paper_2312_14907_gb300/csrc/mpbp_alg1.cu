// mpbp_alg1.cu -- the element-wise kernels of the paper's minibatch optimizer
// (Alg. 1 without its projector line):
//   prep    rho = mask * e^{chi}, alpha_0 = 1, alpha_m = e^{alpha_t[m]}   (Eq. 8)
//           and the step count with its bias corrections
//   update  the chain rule to the auxiliary variables, g_chi = rho df/drho,
//           g_alpha_t[m] = alpha_m df/dalpha_m, then Adam (Kingma and Ba) on
//           chi, u and alpha_t[1..D-1], moments in FP32 per pixel and FP64
//           per peak, bias corrections in FP64
// The loss and gradient in between are the fused path of every other entry
// point, evaluated on the minibatch's frame list.
#include <cmath>

#include "aux_launch.h"

namespace mpbp {

namespace {

__global__ void adam_prep_kernel(AdamArgs a) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.npix; i += stride)
    a.rho_x[i] = (a.mask ? a.mask[i] : 1.0f) * expf(a.chi[i]);
  if (blockIdx.x == 0) {
    if (threadIdx.x < a.D) a.alpha_x[threadIdx.x] = threadIdx.x == 0 ? 1.0f : expf(a.alpha_t[threadIdx.x]);
    if (threadIdx.x == 0) {
      mpbp_adam_state* st = a.st;
      st->t += 1;
      st->bc1 = 1.0 - pow(st->beta1, (double)st->t);
      st->bc2 = 1.0 - pow(st->beta2, (double)st->t);
    }
  }
}

__global__ void adam_update_kernel(AdamArgs a) {
  const mpbp_adam_state* st = a.st;
  const float b1 = (float)st->beta1, b2 = (float)st->beta2, eps = (float)st->eps;
  const float ic1 = (float)(1.0 / st->bc1), ic2 = (float)(1.0 / st->bc2);
  const float lr_chi = (float)st->lr_chi, lr_u = (float)st->lr_u;
  const long long n = a.npix * (1 + a.C);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const bool is_chi = i < a.npix;
    const long long j = is_chi ? i : i - a.npix;
    const float g = is_chi ? a.rho_x[j] * a.g_rho[j] : a.g_u[j];
    float* x = is_chi ? a.chi + j : a.u + j;
    float* mo = is_chi ? a.m_chi + j : a.m_u + j;
    float* ve = is_chi ? a.v_chi + j : a.v_u + j;
    const float m = fmaf(b1, *mo, (1.0f - b1) * g);
    const float v = fmaf(b2, *ve, (1.0f - b2) * g * g);
    *mo = m;
    *ve = v;
    *x -= (is_chi ? lr_chi : lr_u) * (m * ic1) / (sqrtf(v * ic2) + eps);
  }
  // alpha_t[0] is not a variable (alpha_0 = 1): its gradient is 0 and it
  // never moves, so it is left alone
  if (blockIdx.x == 0 && threadIdx.x >= 1 && threadIdx.x < a.D) {
    const int mk = threadIdx.x;
    const double g = (double)a.alpha_x[mk] * a.g_alpha[mk];
    const double m = st->beta1 * a.m_a[mk] + (1.0 - st->beta1) * g;
    const double v = st->beta2 * a.v_a[mk] + (1.0 - st->beta2) * g * g;
    a.m_a[mk] = m;
    a.v_a[mk] = v;
    a.alpha_t[mk] = (float)((double)a.alpha_t[mk] -
                            st->lr_alpha * (m / st->bc1) / (sqrt(v / st->bc2) + st->eps));
  }
}

int grid_of(long long n, int num_sms) {
  const long long b = (n + 255) / 256;
  const long long cap = (long long)num_sms * 8;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace

cudaError_t launch_adam_prep(const AdamArgs& a, int num_sms, cudaStream_t s) {
  adam_prep_kernel<<<grid_of(a.npix, num_sms), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adam_update(const AdamArgs& a, int num_sms, cudaStream_t s) {
  adam_update_kernel<<<grid_of(a.npix * (1 + a.C), num_sms), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mpbp

namespace mpbp {

namespace {

// one thread per (frame, frame pixel): out(s_j + k) += |P_m(k)|^2
__global__ void illumination_kernel(IllumArgs a) {
  const long long mm = (long long)a.m * a.m;
  const long long n = (long long)a.nframes * mm;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / mm, k = i - f * mm;
    const int mk = (int)(f / a.J), j = (int)(f - (long long)mk * a.J);
    const int k0 = (int)(k / a.m), k1 = (int)(k - (long long)k0 * a.m);
    const int r0 = a.scan[j].x + k0, r1 = a.scan[j].y + k1;
    if (r0 < 0 || r0 >= a.n1 || r1 < 0 || r1 >= a.n2) continue;
    const long long pi = a.probe_stride >= 0 ? mk * a.probe_stride
                         : (a.probe_stride == kProbePerFrame ? f : j) * mm;
    const float2 P = reinterpret_cast<const float2*>(a.probe)[pi + k];
    atomicAdd(a.out + (long long)r0 * a.n2 + r1, P.x * P.x + P.y * P.y);
  }
}

}  // namespace

cudaError_t launch_illumination(const IllumArgs& a, int num_sms, cudaStream_t s) {
  const long long n = (long long)a.nframes * a.m * a.m;
  const long long b = (n + 255) / 256;
  illumination_kernel<<<(int)(b < num_sms * 16 ? b : num_sms * 16), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mpbp
