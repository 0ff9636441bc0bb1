// mpbp_noalloc.cu -- loss and gradient without any device allocation.
//
// Some callers cannot allocate device memory: code running inside another
// runtime's memory pool or allocator hooks, plugins that must not grow the
// process footprint after start-up, or callers that have reserved all of the
// GPU's memory for themselves.  mpbp_create allocates a workspace, so they
// cannot use the context API.  This entry point runs the same kernels with its
// scratch (scan table, objects, gradient accumulator, sqrt(y) tiles, partial
// sums) in a fixed-size array that is part of the library's device image:
// every GPU that loads the library holds it until the process exits.
#include <mutex>

#include "aux_launch.h"
#include "frames_launch.h"

using namespace mpbp;

namespace {

constexpr size_t kScratchBytes = 16u << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  void* scratch = nullptr;   // device address of g_scratch on this device
  int num_sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Once per device, with that device current: the device address of the
// scratch array (its name is only a host-side stand-in in host code).
mpbp_status device_setup(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= kMaxDevices) return MPBP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return MPBP_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return MPBP_ERR_CUDA;
    s.scratch = p;
    s.num_sms = sms;
    s.done = true;
  }
  *out = &s;
  return MPBP_OK;
}

}  // namespace

extern "C" mpbp_status mpbp_loss_grad_noalloc(const mpbp_problem* pr, const float* probe,
                                              const float* y, const float* rho, const float* u,
                                              const float* alpha, double* loss, float* g_rho,
                                              float* g_u, double* g_alpha, int32_t* dev_err,
                                              void* stream) {
  if (!probe || !y || !rho || !u || !alpha || !loss || !g_rho || !g_u) return MPBP_ERR_INVALID_ARG;
  const mpbp_status vs = validate_problem(pr);
  if (vs != MPBP_OK) return vs;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPBP_ERR_CUDA;
  DeviceSetup* ds = nullptr;
  mpbp_status st = device_setup(dev, &ds);
  if (st != MPBP_OK) return st;
  FrameKernelInfo fk{};
  if (!frames_prepare(pr->m, &fk)) return MPBP_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  const long long npix = (long long)pr->n1 * pr->n2;
  const long long nframes = (long long)pr->npeaks * pr->nscan;
  const long long mm = (long long)pr->m * pr->m;
  const int grid_cap = ds->num_sms * fk.blocks_per_sm;
  const long long need = (nframes + fk.frames_per_block - 1) / fk.frames_per_block;
  const int fgrid = (int)(need < grid_cap ? need : grid_cap);
  const int pgrid = finish_grid(npix, ds->num_sms);

  // carve the scratch array; reject problems that do not fit
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = align256(off);
    off = o + bytes;
    return o;
  };
  const size_t oScan = take(sizeof(int2) * pr->nscan);
  const size_t oO = take(sizeof(cf) * npix * pr->npeaks);
  const size_t oAcc = take(sizeof(cf) * npix * pr->npeaks);
  const size_t oA = take(sizeof(float) * nframes * mm);
  const size_t oLP = take(sizeof(double) * (fgrid > 0 ? fgrid : 1));
  const size_t oPart = take(sizeof(double) * pgrid * (pr->npeaks + 3));
  const size_t oErr = take(sizeof(int));   // used when the caller passes no error word
  const size_t oArr = take(sizeof(unsigned));
  if (off > kScratchBytes) return MPBP_ERR_UNSUPPORTED;
  char* b = static_cast<char*>(ds->scratch);
  int2* scan = reinterpret_cast<int2*>(b + oScan);
  cf* O = reinterpret_cast<cf*>(b + oO);
  cf* acc = reinterpret_cast<cf*>(b + oAcc);
  float* aT = reinterpret_cast<float*>(b + oA);
  double* loss_part = reinterpret_cast<double*>(b + oLP);
  double* part = reinterpret_cast<double*>(b + oPart);
  // the device error bits of this call go to the caller's word when given
  int* err = dev_err ? reinterpret_cast<int*>(dev_err) : reinterpret_cast<int*>(b + oErr);
  unsigned* arrivals = reinterpret_cast<unsigned*>(b + oArr);

  PhaseCoef pc{};
  for (int m = 0; m < pr->npeaks; ++m)
    for (int k = 0; k < kMaxComp; ++k) {
      const double g = k < pr->ncomp ? pr->G[m * pr->ncomp + k] : 0.0;
      pc.kpi[m][k] = (float)(pr->phase_scale * g / 3.14159265358979323846);
      pc.kps[m][k] = (float)(pr->phase_scale * g);
    }

  // the array keeps the previous call's contents: clear what must start at 0
  // (the accumulator, the error word; the arrival counter is cleared by the
  // frame kernel) and load this call's scan table, copied from the caller's
  // host array on the stream
  if (cudaMemcpyAsync(scan, pr->scan, sizeof(int2) * pr->nscan, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(acc, 0, sizeof(cf) * npix * pr->npeaks, s) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess)
    return MPBP_ERR_CUDA;
  if (launch_frame_transpose(y, aT, nframes, pr->m, true, s) != cudaSuccess) return MPBP_ERR_CUDA;

  ObjectArgs oa{};
  oa.rho = rho;
  oa.u = u;
  oa.alpha = alpha;
  oa.O = O;
  oa.npix = npix;
  oa.D = pr->npeaks;
  oa.C = pr->ncomp;
  oa.pc = pc;
  if (launch_object_build(oa, ds->num_sms, s) != cudaSuccess) return MPBP_ERR_CUDA;

  FrameArgs fa{};
  fa.O = O;
  fa.probe = reinterpret_cast<const cf*>(probe);
  fa.aT = aT;
  fa.bgT = nullptr;
  fa.scan = scan;
  fa.frames = nullptr;
  fa.acc = acc;
  fa.loss_part = loss_part;
  fa.I_out = nullptr;
  fa.err = err;
  fa.arrivals = arrivals;
  fa.obj_stride = npix;
  fa.nframes = (int)nframes;
  fa.frame0 = 0;
  fa.nframes_total = (int)nframes;
  fa.n1 = pr->n1;
  fa.n2 = pr->n2;
  fa.J = pr->nscan;
  fa.probe_stride = pr->probe_per_peak ? (int)mm : 0;
  if (frames_launch(pr->m, fa, fgrid > 0 ? fgrid : 1, false, s) != cudaSuccess) return MPBP_ERR_CUDA;

  FinishArgs fi{};
  fi.rho = rho;
  fi.u = u;
  fi.alpha = alpha;
  fi.acc = acc;
  fi.g_rho = g_rho;
  fi.g_u = g_u;
  fi.part = part;
  fi.arrivals = arrivals;
  fi.npix = npix;
  fi.D = pr->npeaks;
  fi.C = pr->ncomp;
  fi.pc = pc;
  fi.loss_part = loss_part;
  fi.n_loss_part = fgrid > 0 ? fgrid : 1;
  ReduceArgs ra{};
  ra.part = part;
  ra.n_part = pgrid;
  ra.D = pr->npeaks;
  ra.loss_out = loss;
  ra.g_alpha_out = g_alpha;
  ra.g_alpha_ws = nullptr;
  ra.err = err;
  ra.st = nullptr;
  ra.alpha_from = 1;
  if (launch_finish(fi, ra, pgrid, s) != cudaSuccess) return MPBP_ERR_CUDA;
  return MPBP_OK;
}
