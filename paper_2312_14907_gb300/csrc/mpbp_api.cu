// mpbp_api.cu -- the C ABI declared in include/mpbp.h: context, workspace,
// argument checks and the launch sequence of each entry point.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <new>
#include <string>
#include <vector>

#include "aux_launch.h"
#include "frames_launch.h"
#include "unwrap_launch.h"

using namespace mpbp;

constexpr int kStageSlots = 3;   // staging buffers of the host-buffer entry point

struct mpbp_ctx {
  unsigned long long serial = 0;   // unique per context created in this process
  int device = 0;
  int num_sms = 0;
  // problem
  int n1 = 0, n2 = 0, C = 0, D = 0, M = 0, J = 0;
  int probe_per_peak = 0;
  double phase_scale = 0.0;
  long long npix = 0;
  long long nframes = 0;  // D * J
  PhaseCoef pc{};
  std::vector<double> G;   // [D][C] scattering vectors
  // kernel schedule
  FrameKernelInfo fk{};       // the gradient kernel in use
  FrameKernelInfo fk_fft{};   // the FFT kernels (forward mode always uses them)
  // tensor maps of O for the FFT kernels' tile copies (box widths from fk_fft)
  TmaMap tm_grad{}, tm_fwd{};
  bool tile_grad = false, tile_fwd = false;
  unsigned test_tx_extra = 0;   // mpbp_set_test_stall
  // host path: tensor maps of the staged counts, one per staging slot
  CUtensorMap ymap[kStageSlots];
  long long ymap_per = 0;       // frames per slot they were encoded for (0: none)
  // host path with 16-bit counts: their staging slots and tensor maps
  unsigned short* stage16 = nullptr;
  size_t stage16_elems = 0;
  CUtensorMap ymap16[kStageSlots];
  long long ymap16_per = 0;
  int precision = MPBP_PRECISION_FP32;
  int fft_schedule = kLayoutDefault;   // M = 128: FrameLayout of the gradient kernel
  void* tc_w = nullptr;       // split DFT matrix of the tensor-core kernel
  int blocks_per_sm = 0;  // schedule in use
  int frames_grid_cap = 0;
  int finish_grid = 0;
  // device workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cf* O = nullptr;
  cf* acc = nullptr;
  cf* probe = nullptr;
  int2* scan = nullptr;
  int* strip_order = nullptr;   // [nframes] frames by peak, scan column, scan row
  float* aT = nullptr;
  float* bgT = nullptr;
  double* loss_part = nullptr;
  double* part = nullptr;
  double* loss_ws = nullptr;
  float* g_rho_ws = nullptr;
  float* g_u_ws = nullptr;
  double* g_alpha_ws = nullptr;
  float* rho_base = nullptr;
  float* u_base = nullptr;
  float* alpha_base = nullptr;
  float* g_rho_base = nullptr;
  float* g_u_base = nullptr;
  double* g_alpha_base = nullptr;
  int* err = nullptr;
  unsigned* arrivals = nullptr;
  // lazily allocated tables of a batched launch led by this context
  void* batch_ws = nullptr;
  size_t batch_ws_bytes = 0;
  int batch_order = 0;    // 0: items grouped by frame side, 1: problems interleaved
  int batch_mode = 1;     // 0: one launch for every frame side, 1: one launch per side,
                          // 2: as 1 but M = 128 problems launched one by one,
                          // 3: every problem launched on its own
  std::vector<long long> batch_key;   // the batch whose plan is cached below
  struct PlanLaunch {
    int m;          // frame side, or 0 for the single launch over every side
    int grid;
    bool tma;       // per-side launch with tile copies (args.tmaps set)
    BatchArgs args;
  };
  std::vector<PlanLaunch> batch_plan;
  std::vector<long long> batch_base;  // first loss slot of each fused problem
  std::vector<int> batch_fused;       // batch positions of the fused problems
  long long batch_frames = 0;
  unsigned long long version = 0;     // bumped when probe or data change
  // lazily allocated for the host-buffer entry point: inputs, two staging
  // buffers for chunks of y, a copy stream and events for the pipeline
  float* io_x = nullptr;
  float* stage = nullptr;
  size_t stage_elems = 0;   // per staging buffer
  cudaStream_t copy_stream = nullptr;
  cudaStream_t chunk_stream[2] = {nullptr, nullptr};   // alternating chunk launches
  cudaEvent_t ev_ready = nullptr;          // caller's stream reached the frame launches
  cudaEvent_t ev_x = nullptr;              // rho, u, alpha are on the device
  cudaEvent_t ev_copied[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_consumed[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_done[2] = {nullptr, nullptr};
  bool has_probe = false, has_data = false;
  bool acc_dirty = false;
  // scan positions off the pixel grid (mpbp_set_scan_offsets): the offsets
  // d_j (empty: integer positions) and the probes shifted by them, one per
  // scan position (shared probe) or per frame (one probe per peak)
  std::vector<float2> scan_off_h;
  float2* scan_off = nullptr;   // [J]
  cf* probe_scan = nullptr;     // [J or D*J][M][M]
  bool shift_ready = false;
  // optional event timing of the fused frame kernel
  bool timing = false;
  // Alg. 1: Adam moments and the materialised rho, alpha (mpbp_adam_init)
  void* adam_buf = nullptr;
  float *m_chi = nullptr, *v_chi = nullptr, *m_u = nullptr, *v_u = nullptr;
  double *m_a = nullptr, *v_a = nullptr;
  float *rho_x = nullptr, *alpha_x = nullptr;
  // phase unwrapping / projector workspace (lazily allocated)
  void* uw_buf = nullptr;
  UnwrapArgs uw{};
  float *pj_phi = nullptr, *pj_wrapped = nullptr;
  int uw_grid = 0;
  // one optimizer step captured as a CUDA graph (mpbp_step_capture)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  // the deterministic gradient (mpbp_set_deterministic): host copies of the
  // scan and of the column-strip order, and the plan for grid det_grid
  std::vector<int2> scan_h;
  std::vector<int> order_h;
  bool det = false;
  int det_grid = 0;
  void* det_meta = nullptr;   // pieces, block starts, column lists, the DetPlan
  cf* det_pool = nullptr;
  size_t det_pool_elems = 0, det_pool_cap = 0;
  const DetPlan* det_plan = nullptr;
  std::vector<void*> det_old;   // earlier plans' buffers a captured step may still use
  std::string last_error;
};

namespace {

const char* kStatusNames[] = {"MPBP_OK",          "MPBP_ERR_INVALID_ARG", "MPBP_ERR_UNSUPPORTED",
                              "MPBP_ERR_CUDA",    "MPBP_ERR_NONFINITE",   "MPBP_ERR_TIMEOUT",
                              "MPBP_ERR_BOUNDS",  "MPBP_ERR_OOM",         "MPBP_ERR_NO_DATA"};

mpbp_status fail(mpbp_ctx* c, mpbp_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

#define MPBP_CUDA(ctx, call)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return fail(ctx, MPBP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                     \
  } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Carver {
  size_t off = 0;
  template <typename T>
  size_t take(size_t n) {
    size_t o = align_up(off, 256);
    off = o + n * sizeof(T);
    return o;
  }
};

// whether problems of frame side m go through the batched kernel in `mode`
bool batch_fused_side(int mode, int m) {
  if (m < 32 || mode == 3) return false;
  return mode != 2 || m < 128;
}

// frame-range launches of one host-path evaluation (each writes its own
// slice of the loss partials)
constexpr int kMaxHostChunks = 8;

// device address of page-locked (CUDA-registered) host memory, else NULL
void* mapped_host(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int frames_grid_for(const mpbp_ctx* c, long long nframes) {
  const long long need = (nframes + c->fk.frames_per_block - 1) / c->fk.frames_per_block;
  long long g = std::min<long long>(need, c->frames_grid_cap);
  return (int)std::max<long long>(g, 1);
}

// grid of the forward-mode FFT kernel: occupancy maximum
int frames_grid_fft(const mpbp_ctx* c, long long nframes) {
  const long long need = (nframes + c->fk_fft.frames_per_block - 1) / c->fk_fft.frames_per_block;
  long long g = std::min<long long>(need, (long long)c->num_sms * c->fk_fft.blocks_per_sm);
  return (int)std::max<long long>(g, 1);
}

// a launch over every frame of the context from its own data and objects
bool full_launch(const mpbp_ctx* c, const FrameArgs& fa) {
  return !fa.frames && fa.frame0 == 0 && fa.nframes == c->nframes && fa.aT == c->aT && fa.O == c->O;
}

// The deterministic gradient's plan for a grid of `grid` blocks (host work
// and synchronous uploads: called outside any stream capture).  Block b
// takes positions [N b / G, N (b + 1) / G) of the strip order; its run is cut
// into pieces where the peak or the first column changes, as the kernel's
// window does.  A piece spans its frames' rows plus a frame, 128 columns.
mpbp_status det_prepare(mpbp_ctx* c, int grid) {
  if (c->det_grid == grid && c->det_plan) return MPBP_OK;
  const int W = c->M;
  const long long N = c->nframes;
  std::vector<DetPiece> pieces;
  std::vector<int> b0(grid);
  for (int b = 0; b < grid; ++b) {
    const long long lo = N * b / grid, hi = N * (b + 1) / grid;
    b0[b] = (int)pieces.size();
    for (long long it = lo; it < hi; ++it) {
      const int f = c->order_h[(size_t)it];
      const int m = f / c->J;
      const int2 sp = c->scan_h[f - m * c->J];
      if (it == lo || m != pieces.back().mpk || sp.y != pieces.back().y) {
        pieces.push_back(DetPiece{0, sp.x, sp.x, m, sp.y});   // rows: the last row start, for now
      } else {
        DetPiece& pc = pieces.back();
        pc.row0 = std::min(pc.row0, sp.x);
        pc.rows = std::max(pc.rows, sp.x);
      }
    }
  }
  long long off = 0;
  for (DetPiece& pc : pieces) {
    pc.rows = pc.rows - pc.row0 + W;
    pc.off = off;
    off += (long long)pc.rows * W;
  }
  // per (peak, column, band of W rows): the pieces that reach into it, in
  // piece order (a pixel's candidates; the sum takes those covering it)
  const int nband = (c->n1 + W - 1) / W;
  const long long nkey = (long long)c->D * c->n2 * nband;
  std::vector<int> cnt((size_t)nkey + 1, 0);
  auto each_key = [&](const DetPiece& pc, auto&& fn) {
    const int b0 = std::max(pc.row0, 0) / W, b1 = (std::min(pc.row0 + pc.rows, c->n1) - 1) / W;
    if (std::min(pc.row0 + pc.rows, c->n1) <= std::max(pc.row0, 0)) return;
    for (int col = std::max(pc.y, 0); col < std::min(pc.y + W, c->n2); ++col)
      for (int b = b0; b <= b1; ++b) fn(((long long)pc.mpk * c->n2 + col) * nband + b);
  };
  for (const DetPiece& pc : pieces) each_key(pc, [&](long long k) { cnt[(size_t)k + 1]++; });
  for (long long i = 0; i < nkey; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i];
  std::vector<int> lists((size_t)cnt[(size_t)nkey]);
  {
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (size_t p = 0; p < pieces.size(); ++p)
      each_key(pieces[p], [&](long long k) { lists[(size_t)fill[(size_t)k]++] = (int)p; });
  }
  // device copies: one block of tables, and the pool (kept if large enough)
  Carver cv;
  const size_t oP = cv.take<DetPiece>(pieces.size());
  const size_t oB = cv.take<int>(b0.size());
  const size_t oS = cv.take<int>(cnt.size());
  const size_t oL = cv.take<int>(std::max<size_t>(lists.size(), 1));
  const size_t oD = cv.take<DetPlan>(1);
  // an earlier plan's buffers: freed now (cudaFree waits for the work that
  // uses them), or kept while a captured step may still point at them
  auto retire = [c](void* q) {
    if (!q) return;
    if (c->step_exec) c->det_old.push_back(q);
    else cudaFree(q);
  };
  retire(c->det_meta);
  c->det_meta = nullptr;
  c->det_plan = nullptr;
  c->det_grid = 0;
  if (cudaMalloc(&c->det_meta, cv.off) != cudaSuccess) {
    cudaGetLastError();
    c->det_meta = nullptr;
    return fail(c, MPBP_ERR_OOM, "deterministic gradient: tables");
  }
  if ((size_t)off > c->det_pool_cap) {
    retire(c->det_pool);
    c->det_pool = nullptr;
    c->det_pool_cap = 0;
    if (cudaMalloc(&c->det_pool, sizeof(cf) * (size_t)off) != cudaSuccess) {
      cudaGetLastError();
      c->det_pool = nullptr;
      return fail(c, MPBP_ERR_OOM, "deterministic gradient: pieces");
    }
    c->det_pool_cap = (size_t)off;
  }
  c->det_pool_elems = (size_t)off;
  char* m = static_cast<char*>(c->det_meta);
  DetPlan plan{c->det_pool, reinterpret_cast<DetPiece*>(m + oP), reinterpret_cast<int*>(m + oB),
               reinterpret_cast<int*>(m + oS), reinterpret_cast<int*>(m + oL)};
  if (cudaMemcpy(m + oP, pieces.data(), sizeof(DetPiece) * pieces.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m + oB, b0.data(), sizeof(int) * b0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m + oS, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      (!lists.empty() &&
       cudaMemcpy(m + oL, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(m + oD, &plan, sizeof(plan), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(c, MPBP_ERR_CUDA, "deterministic gradient: upload");
  c->det_plan = reinterpret_cast<const DetPlan*>(m + oD);
  c->det_grid = grid;
  return MPBP_OK;
}

// the gradient-mode frame kernel of the context's precision
cudaError_t launch_frames(const mpbp_ctx* c, const FrameArgs& fa, int grid, cudaStream_t s) {
  if (c->det) {
    // only launches over every frame with the plan's grid get here (the
    // entry points refuse the others); anything else is a library bug
    if (!full_launch(c, fa) || grid != c->det_grid || !c->det_plan || c->precision != MPBP_PRECISION_FP32 ||
        (c->M == 128 && c->fft_schedule != kLayoutExchange) || !c->tile_grad)
      return cudaErrorNotSupported;
  } else if (c->precision == MPBP_PRECISION_TC_SPLIT16) {
    return tc_launch(c->M, fa, c->tc_w, grid, s, c->test_tx_extra != 0);
  }
  FrameArgs f2 = fa;
  // every frame of the context: the exchange kernel at M = 128 takes them in
  // column strips (any order gives the same sums up to rounding)
  if (((c->M == 128 && c->fft_schedule == kLayoutExchange) || c->det) && !fa.frames && fa.frame0 == 0 &&
      fa.nframes == c->nframes && fa.aT == c->aT)
    f2.frames = c->strip_order;
  if (c->det) {
    f2.det = c->det_plan;
    cudaError_t e = cudaMemsetAsync(c->det_pool, 0, sizeof(cf) * c->det_pool_elems, s);
    if (e != cudaSuccess) return e;
    TmaMap tm = c->tm_grad;
    tm.tx_extra = c->test_tx_extra;
    e = frames_launch(c->M, f2, grid, false, s, &tm, c->fft_schedule);
    if (e != cudaSuccess) return e;
    return launch_det_reduce(c->det_plan, c->acc, c->D, c->n1, c->n2, c->M, c->num_sms, s);
  }
  if (!c->tile_grad || fa.O != c->O) return frames_launch(c->M, f2, grid, false, s, nullptr, c->fft_schedule);
  TmaMap tm = c->tm_grad;
  tm.tx_extra = c->test_tx_extra;
  return frames_launch(c->M, f2, grid, false, s, &tm, c->fft_schedule);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the CUDA driver API's tensor-map encoder, looked up once through the runtime
EncodeTiledFn encode_tiled_fn() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor map of one staging slot of counts, [per M rows][M] floats, in boxes
// of 32 columns x M rows with the 128-byte swizzle (the raw-data kernel's
// shared-memory layout).
// (y16: 16-bit counts, boxes of 64 columns; the same 128 bytes a box row)
bool encode_counts_map(const mpbp_ctx* c, const void* base, long long per, bool y16, CUtensorMap* out) {
  const EncodeTiledFn fn = encode_tiled_fn();
  const int eb = y16 ? 2 : 4;
  if (!fn || c->M * eb < 128 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)c->M, (cuuint64_t)(per * c->M)};
  const cuuint64_t stride[1] = {(cuuint64_t)c->M * eb};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)c->M};
  const cuuint32_t estride[2] = {1u, 1u};
  return fn(out, y16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dim,
            stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the objects O [D][n1][n2] (8-byte elements) for tiles of
// w columns and M rows; false where the layout admits none (rows of O not a
// multiple of 16 bytes) or the encoder is unavailable, and the kernels then
// copy with cp.async.
bool encode_objects_map(const mpbp_ctx* c, int w, TmaMap* out) {
  if (w <= 0 || w > 256 || (c->n2 * sizeof(cf)) % 16 != 0 || (reinterpret_cast<uintptr_t>(c->O) & 15) != 0)
    return false;
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)c->n2, (cuuint64_t)c->n1, (cuuint64_t)c->D};
  const cuuint64_t stride[2] = {(cuuint64_t)c->n2 * sizeof(cf), (cuuint64_t)c->npix * sizeof(cf)};
  const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)c->M, 1u};
  const cuuint32_t estride[3] = {1u, 1u, 1u};
  return fn(&out->map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, c->O, dim, stride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

FrameArgs frame_args(mpbp_ctx* c, const int* frames, int nframes) {
  FrameArgs a{};
  a.O = c->O;
  a.probe = c->probe;
  a.aT = c->aT;
  a.bgT = c->bgT;
  a.scan = c->scan;
  a.frames = frames;
  a.acc = c->acc;
  a.loss_part = c->loss_part;
  a.I_out = nullptr;
  a.err = c->err;
  a.arrivals = c->arrivals;
  a.obj_stride = c->npix;
  a.nframes = nframes;
  a.frame0 = 0;
  a.nframes_total = (int)c->nframes;
  a.n1 = c->n1;
  a.n2 = c->n2;
  a.J = c->J;
  a.probe_stride = c->probe_per_peak ? c->M * c->M : 0;
  if (!c->scan_off_h.empty()) {
    a.probe = c->probe_scan;
    a.probe_stride = c->probe_per_peak ? kProbePerFrame : kProbePerScan;
  }
  return a;
}

// the probes of the context's scan offsets from its probe (after either changed)
mpbp_status enqueue_probe_shift(mpbp_ctx* c, cudaStream_t s) {
  if (c->scan_off_h.empty() || !c->has_probe) return MPBP_OK;
  const long long n = c->probe_per_peak ? c->nframes : c->J;
  if (!c->probe_scan) {
    if (cudaMalloc(&c->scan_off, sizeof(float2) * c->J) != cudaSuccess ||
        cudaMalloc(&c->probe_scan, sizeof(cf) * n * c->M * c->M) != cudaSuccess) {
      cudaGetLastError();
      if (c->scan_off) cudaFree(c->scan_off);
      if (c->probe_scan) cudaFree(c->probe_scan);
      c->scan_off = nullptr;
      c->probe_scan = nullptr;
      c->scan_off_h.clear();
      return fail(c, MPBP_ERR_OOM, "probes of the scan offsets");
    }
  }
  if (!c->shift_ready) c->shift_ready = probe_shift_prepare(c->M);
  ProbeShiftArgs a{};
  a.src = c->probe;
  a.out = c->probe_scan;
  a.d = c->scan_off;
  a.nout = (int)n;
  a.J = c->J;
  a.m = c->M;
  a.per_peak = c->probe_per_peak != 0;
  if (!c->shift_ready ||
      cudaMemcpyAsync(c->scan_off, c->scan_off_h.data(), sizeof(float2) * c->J, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      launch_probe_shift(a, s) != cudaSuccess) {
    // no shifted probes: back to the integer positions rather than stale probes
    cudaGetLastError();
    c->scan_off_h.clear();
    return fail(c, MPBP_ERR_CUDA, "shifting the probe for the scan offsets");
  }
  return MPBP_OK;
}

mpbp_status enqueue_object_build(mpbp_ctx* c, const float* rho, const float* u,
                                 const float* alpha, cf* out, cudaStream_t s,
                                 const float* phi = nullptr) {
  ObjectArgs oa{};
  oa.rho = rho;
  oa.u = u;
  oa.phi = phi;
  oa.alpha = alpha;
  oa.O = out;
  oa.npix = c->npix;
  oa.D = c->D;
  oa.C = c->C;
  oa.pc = c->pc;
  MPBP_CUDA(c, launch_object_build(oa, c->num_sms, s));
  return MPBP_OK;
}

// A1..A8: objects, fused frames, gradient assembly, reductions.  st != nullptr
// adds the line-search decision, and step (with st) the optimizer update.
mpbp_status enqueue_loss_grad(mpbp_ctx* c, const float* rho, const float* u, const float* alpha,
                              const int32_t* frames, int32_t nframes, double* loss,
                              float* g_rho, float* g_u, double* g_alpha,
                              mpbp_step_state* st, cudaStream_t s,
                              const float* phi = nullptr, float* g_phi = nullptr,
                              const StepPtrs* step = nullptr) {
  if (c->det && frames)
    return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient is for evaluations over every frame");
  if (c->acc_dirty) {
    MPBP_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(cf) * c->npix * c->D, s));
    c->acc_dirty = false;
  }
  mpbp_status r = enqueue_object_build(c, rho, u, alpha, c->O, s, phi);
  if (r != MPBP_OK) return r;
  const int nf = frames ? nframes : (int)c->nframes;
  FrameArgs fa = frame_args(c, frames, nf);
  const int grid = frames_grid_for(c, nf);
  c->acc_dirty = true;
  cudaEvent_t ev1 = nullptr;
  if (c->timing) {
    if (c->ev_used == c->ev_pool.size()) {
      cudaEvent_t a, b;
      MPBP_CUDA(c, cudaEventCreate(&a));
      MPBP_CUDA(c, cudaEventCreate(&b));
      c->ev_pool.emplace_back(a, b);
    }
    MPBP_CUDA(c, cudaEventRecord(c->ev_pool[c->ev_used].first, s));
    ev1 = c->ev_pool[c->ev_used].second;
    c->ev_used++;
  }
  MPBP_CUDA(c, launch_frames(c, fa, grid, s));
  if (ev1) MPBP_CUDA(c, cudaEventRecord(ev1, s));

  FinishArgs fi{};
  fi.rho = rho;
  fi.u = u;
  fi.alpha = alpha;
  fi.acc = c->acc;
  fi.g_rho = g_rho;
  fi.g_u = g_u;
  fi.phi = phi;
  fi.g_phi = g_phi;
  fi.part = c->part;
  fi.npix = c->npix;
  fi.D = c->D;
  fi.C = c->C;
  fi.pc = c->pc;
  fi.arrivals = c->arrivals;
  fi.loss_part = c->loss_part;
  fi.n_loss_part = grid;

  ReduceArgs ra{};
  ra.part = c->part;
  ra.n_part = c->finish_grid;
  ra.D = c->D;
  ra.loss_out = loss;
  ra.g_alpha_out = g_alpha;
  ra.g_alpha_ws = c->g_alpha_ws;
  ra.err = c->err;
  ra.st = st;
  ra.alpha_from = 1;
  if (step) ra.step = *step;
  MPBP_CUDA(c, launch_finish(fi, ra, c->finish_grid, s));
  c->acc_dirty = false;
  return MPBP_OK;
}

}  // namespace

extern "C" {

const char* mpbp_status_string(mpbp_status s) {
  int i = (int)s;
  if (i < 0 || i >= (int)(sizeof(kStatusNames) / sizeof(kStatusNames[0]))) return "MPBP_ERR_UNKNOWN";
  return kStatusNames[i];
}

const char* mpbp_last_error(const mpbp_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

mpbp_status mpbp_create(const mpbp_problem* pr, mpbp_ctx** out) {
  if (!out) return MPBP_ERR_INVALID_ARG;
  *out = nullptr;
  const mpbp_status vs = validate_problem(pr);
  if (vs != MPBP_OK) return vs;

  mpbp_ctx* c = new (std::nothrow) mpbp_ctx();
  if (!c) return MPBP_ERR_OOM;
  static std::atomic<unsigned long long> next_serial{1};
  c->serial = next_serial.fetch_add(1);
  auto bail = [&](mpbp_status s) {
    if (c->ws) cudaFree(c->ws);
    delete c;
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(MPBP_ERR_CUDA);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
    return bail(MPBP_ERR_CUDA);
  c->n1 = pr->n1;
  c->n2 = pr->n2;
  c->C = pr->ncomp;
  c->D = pr->npeaks;
  c->M = pr->m;
  c->J = pr->nscan;
  c->probe_per_peak = pr->probe_per_peak ? 1 : 0;
  c->phase_scale = pr->phase_scale;
  c->npix = (long long)pr->n1 * pr->n2;
  c->nframes = (long long)pr->npeaks * pr->nscan;
  for (int m = 0; m < c->D; ++m)
    for (int k = 0; k < kMaxComp; ++k) {
      const double g = k < c->C ? pr->G[m * c->C + k] : 0.0;
      if (k < c->C) c->G.push_back(g);
      c->pc.kpi[m][k] = (float)(pr->phase_scale * g / 3.14159265358979323846);
      c->pc.kps[m][k] = (float)(pr->phase_scale * g);
    }
  if (!frames_prepare(c->M, &c->fk)) return bail(MPBP_ERR_CUDA);
  c->fk_fft = c->fk;
  c->blocks_per_sm = c->fk.blocks_per_sm;
  c->frames_grid_cap = c->num_sms * c->blocks_per_sm;
  c->finish_grid = finish_grid(c->npix, c->num_sms);

  const long long mm = (long long)c->M * c->M;
  const int Dp = c->probe_per_peak ? c->D : 1;
  const int max_frames_grid = c->num_sms * 64 * kMaxHostChunks;
  Carver cv;
  size_t oO = cv.take<cf>(c->npix * c->D);
  size_t oAcc = cv.take<cf>(c->npix * c->D);
  size_t oProbe = cv.take<cf>(Dp * mm);
  size_t oScan = cv.take<int2>(c->J);
  size_t oOrd = cv.take<int>(c->nframes);
  size_t oAT = cv.take<float>(c->nframes * mm);
  size_t oLP = cv.take<double>(max_frames_grid);
  size_t oPart = cv.take<double>((size_t)c->finish_grid * (c->D + 3));
  size_t oLoss = cv.take<double>(1);
  size_t oGR = cv.take<float>(c->npix);
  size_t oGU = cv.take<float>(c->npix * c->C);
  size_t oGA = cv.take<double>(c->D);
  size_t oRB = cv.take<float>(c->npix);
  size_t oUB = cv.take<float>(c->npix * c->C);
  size_t oAB = cv.take<float>(c->D);
  size_t oGRB = cv.take<float>(c->npix);
  size_t oGUB = cv.take<float>(c->npix * c->C);
  size_t oGAB = cv.take<double>(c->D);
  size_t oErr = cv.take<int>(1);
  size_t oArr = cv.take<unsigned>(1);
  c->ws_bytes = align_up(cv.off, 256);
  cudaError_t e = cudaMalloc(&c->ws, c->ws_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    return bail(e == cudaErrorMemoryAllocation ? MPBP_ERR_OOM : MPBP_ERR_CUDA);
  }
  char* b = static_cast<char*>(c->ws);
  c->O = reinterpret_cast<cf*>(b + oO);
  c->acc = reinterpret_cast<cf*>(b + oAcc);
  c->probe = reinterpret_cast<cf*>(b + oProbe);
  c->scan = reinterpret_cast<int2*>(b + oScan);
  c->strip_order = reinterpret_cast<int*>(b + oOrd);
  c->aT = reinterpret_cast<float*>(b + oAT);
  c->loss_part = reinterpret_cast<double*>(b + oLP);
  c->part = reinterpret_cast<double*>(b + oPart);
  c->loss_ws = reinterpret_cast<double*>(b + oLoss);
  c->g_rho_ws = reinterpret_cast<float*>(b + oGR);
  c->g_u_ws = reinterpret_cast<float*>(b + oGU);
  c->g_alpha_ws = reinterpret_cast<double*>(b + oGA);
  c->rho_base = reinterpret_cast<float*>(b + oRB);
  c->u_base = reinterpret_cast<float*>(b + oUB);
  c->alpha_base = reinterpret_cast<float*>(b + oAB);
  c->g_rho_base = reinterpret_cast<float*>(b + oGRB);
  c->g_u_base = reinterpret_cast<float*>(b + oGUB);
  c->g_alpha_base = reinterpret_cast<double*>(b + oGAB);
  c->err = reinterpret_cast<int*>(b + oErr);
  c->arrivals = reinterpret_cast<unsigned*>(b + oArr);
  c->tile_grad = encode_objects_map(c, c->fk_fft.tile_w_grad, &c->tm_grad);
  c->tile_fwd = encode_objects_map(c, c->fk_fft.tile_w_fwd, &c->tm_fwd);

  std::vector<int2> sc(c->J);
  for (int j = 0; j < c->J; ++j) sc[j] = make_int2(pr->scan[2 * j], pr->scan[2 * j + 1]);
  // column strips: a block of the M = 128 exchange kernel takes a contiguous
  // run of this order, so that its successive frames overlap in rows
  std::vector<int> ord((size_t)c->nframes);
  for (long long f = 0; f < c->nframes; ++f) ord[(size_t)f] = (int)f;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    const int pa = a / c->J, pb = b / c->J;
    const int2 sa = sc[a - pa * c->J], sb = sc[b - pb * c->J];
    if (pa != pb) return pa < pb;
    if (sa.y != sb.y) return sa.y < sb.y;
    return sa.x < sb.x;
  });
  c->scan_h = sc;
  c->order_h = ord;
  if (cudaMemcpy(c->scan, sc.data(), sizeof(int2) * c->J, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->strip_order, ord.data(), sizeof(int) * ord.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->acc, 0, sizeof(cf) * c->npix * c->D) != cudaSuccess ||
      cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(c->arrivals, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return bail(MPBP_ERR_CUDA);
  *out = c;
  return MPBP_OK;
}

void mpbp_destroy(mpbp_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (auto& e : c->ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (c->ws) cudaFree(c->ws);
  if (c->io_x) cudaFree(c->io_x);
  if (c->scan_off) cudaFree(c->scan_off);
  if (c->probe_scan) cudaFree(c->probe_scan);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  if (c->ev_x) cudaEventDestroy(c->ev_x);
  for (int i = 0; i < kStageSlots; ++i) {
    if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
    if (c->ev_consumed[i]) cudaEventDestroy(c->ev_consumed[i]);
  }
  for (int i = 0; i < 2; ++i) {
    if (c->chunk_stream[i]) cudaStreamDestroy(c->chunk_stream[i]);
    if (c->ev_done[i]) cudaEventDestroy(c->ev_done[i]);
  }
  if (c->batch_ws) cudaFree(c->batch_ws);
  if (c->stage) cudaFree(c->stage);
  if (c->stage16) cudaFree(c->stage16);
  if (c->bgT) cudaFree(c->bgT);
  if (c->tc_w) cudaFree(c->tc_w);
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->adam_buf) cudaFree(c->adam_buf);
  if (c->uw_buf) cudaFree(c->uw_buf);
  if (c->det_meta) cudaFree(c->det_meta);
  if (c->det_pool) cudaFree(c->det_pool);
  for (void* q : c->det_old) cudaFree(q);
  delete c;
}

mpbp_status mpbp_get_info(const mpbp_ctx* c, mpbp_info* info) {
  if (!c || !info) return MPBP_ERR_INVALID_ARG;
  info->workspace_bytes = (int64_t)c->ws_bytes;
  info->frames_grid = frames_grid_for(c, c->nframes);
  info->frames_block = c->fk.threads;
  info->frames_smem = c->fk.smem;
  info->blocks_per_sm = c->blocks_per_sm;
  info->num_sms = c->num_sms;
  // object build, frames, gradient assembly + reductions (the assembly also
  // applies the step's update); deterministic: + the pieces' clearing and sum
  info->launches_loss_grad = c->det ? 5 : 3;
  info->launches_step = c->det ? 5 : 3;
  info->precision = c->precision;
  info->tile_copies = (c->tile_grad ? 1 : 0) | (c->tile_fwd ? 2 : 0);
  info->fft_schedule = c->fft_schedule;
  info->deterministic = c->det ? 1 : 0;
  return MPBP_OK;
}

mpbp_status mpbp_set_deterministic(mpbp_ctx* c, int32_t on) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  if (!on) {
    c->det = false;
    return MPBP_OK;
  }
  if (c->M != 64 && c->M != 128)
    return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient needs frame side 64 or 128");
  if (c->precision != MPBP_PRECISION_FP32 || (c->M == 128 && c->fft_schedule != kLayoutExchange))
    return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient needs FP32 FFTs (at 128: the exchange schedule)");
  if (!c->tile_grad)
    return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient needs tile copies (rows of O a multiple of 16 bytes)");
  const mpbp_status r = det_prepare(c, frames_grid_for(c, c->nframes));
  if (r != MPBP_OK) return r;
  c->det = true;
  return MPBP_OK;
}

mpbp_status mpbp_set_fft_schedule(mpbp_ctx* c, int32_t schedule) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  if (schedule != MPBP_FFT_SHUFFLE && schedule != MPBP_FFT_EXCHANGE)
    return fail(c, MPBP_ERR_INVALID_ARG, "unknown FFT schedule");
  if (c->det && c->M == 128 && schedule != MPBP_FFT_EXCHANGE)
    return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient runs on the exchange schedule");
  c->fft_schedule = schedule;
  return MPBP_OK;
}

mpbp_status mpbp_set_precision(mpbp_ctx* c, int32_t mode) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  if (mode != MPBP_PRECISION_FP32 && mode != MPBP_PRECISION_TC_SPLIT16)
    return fail(c, MPBP_ERR_INVALID_ARG, "unknown precision mode");
  if (c->det && mode != MPBP_PRECISION_FP32)
    return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient runs on the FP32 FFTs");
  if (mode == MPBP_PRECISION_FP32) {
    c->fk = c->fk_fft;
  } else {
    if (c->M != 32 && c->M != 64 && c->M != 128)
      return fail(c, MPBP_ERR_UNSUPPORTED, "tensor-core DFTs need frame side 32, 64 or 128");
    int bps = 0, smem = 0;
    if (!tc_prepare(&bps, &smem)) return fail(c, MPBP_ERR_CUDA, "tensor-core kernel cannot run here");
    if (!c->tc_w) {
      std::vector<uint32_t> w(kTcSplitBytes / 4);
      tc_split_dft(w.data(), c->M == 32 ? 32 : 64);   // M = 128: four 64 x 64 sub-transforms
      MPBP_CUDA(c, cudaDeviceSynchronize());
      void* d = nullptr;
      if (cudaMalloc(&d, kTcSplitBytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MPBP_ERR_OOM, "cudaMalloc of the DFT table failed");
      }
      c->tc_w = d;
      MPBP_CUDA(c, cudaMemcpy(d, w.data(), kTcSplitBytes, cudaMemcpyHostToDevice));
    }
    c->fk = FrameKernelInfo{kTcThreads, smem, tc_frames_per_block(c->M), bps};
  }
  c->precision = mode;
  c->batch_key.clear();
  return mpbp_set_schedule(c, 0);
}

mpbp_status mpbp_set_schedule(mpbp_ctx* c, int32_t blocks_per_sm) {
  if (!c || blocks_per_sm < 0) return fail(c, MPBP_ERR_INVALID_ARG, "blocks_per_sm < 0");
  int b = blocks_per_sm == 0 ? c->fk.blocks_per_sm : std::min<int>(blocks_per_sm, c->fk.blocks_per_sm);
  c->blocks_per_sm = std::max(b, 1);
  c->frames_grid_cap = std::min(c->num_sms * c->blocks_per_sm, c->num_sms * 64);
  if (c->det) return det_prepare(c, frames_grid_for(c, c->nframes));   // the plan follows the grid
  return MPBP_OK;
}

mpbp_status mpbp_set_batch_schedule(mpbp_ctx* c, int32_t mode, int32_t order) {
  if (!c || mode < 0 || mode > 3 || order < 0 || order > 1)
    return fail(c, MPBP_ERR_INVALID_ARG, "batch schedule out of range");
  c->batch_key.clear();
  c->batch_mode = mode;
  c->batch_order = order;
  return MPBP_OK;
}

mpbp_status mpbp_set_probe(mpbp_ctx* c, const float* probe, void* stream) {
  if (!c || !probe) return fail(c, MPBP_ERR_INVALID_ARG, "null probe");
  const int Dp = c->probe_per_peak ? c->D : 1;
  MPBP_CUDA(c, cudaMemcpyAsync(c->probe, probe, sizeof(cf) * Dp * c->M * c->M,
                               cudaMemcpyDeviceToDevice, S(stream)));
  c->has_probe = true;
  c->version++;
  return enqueue_probe_shift(c, S(stream));
}

mpbp_status mpbp_set_scan_offsets(mpbp_ctx* c, const double* d, void* stream) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  if (!d) {
    c->scan_off_h.clear();
    c->version++;
    return MPBP_OK;
  }
  std::vector<float2> h(c->J);
  for (int j = 0; j < c->J; ++j) {
    const double a = d[2 * j], b = d[2 * j + 1];
    if (!(std::fabs(a) <= 0.5) || !(std::fabs(b) <= 0.5))
      return fail(c, MPBP_ERR_INVALID_ARG, "scan offsets must lie in [-1/2, 1/2]");
    h[j] = make_float2((float)a, (float)b);
  }
  c->scan_off_h.swap(h);
  c->version++;
  return enqueue_probe_shift(c, S(stream));
}

mpbp_status mpbp_shift_probe(const float* probe, int32_t m, const double* d, int32_t n, float* out,
                             void* stream) {
  if (!probe || !d || !out || n < 0 || m < 1 || m > 128) return MPBP_ERR_INVALID_ARG;
  if (n == 0) return MPBP_OK;
  std::vector<float2> h(n);
  for (int j = 0; j < n; ++j) {
    if (!(std::fabs(d[2 * j]) <= 0.5) || !(std::fabs(d[2 * j + 1]) <= 0.5)) return MPBP_ERR_INVALID_ARG;
    h[j] = make_float2((float)d[2 * j], (float)d[2 * j + 1]);
  }
  float2* dd = nullptr;
  if (cudaMalloc(&dd, sizeof(float2) * n) != cudaSuccess) {
    cudaGetLastError();
    return MPBP_ERR_OOM;
  }
  cudaStream_t s = S(stream);
  ProbeShiftArgs a{};
  a.src = reinterpret_cast<const cf*>(probe);
  a.out = reinterpret_cast<cf*>(out);
  a.d = dd;
  a.nout = n;
  a.J = n;
  a.m = m;
  a.per_peak = false;
  const bool ok = cudaMemcpyAsync(dd, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                  probe_shift_prepare(m) && launch_probe_shift(a, s) == cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  cudaFree(dd);
  if (!ok) {
    cudaGetLastError();
    return MPBP_ERR_CUDA;
  }
  return MPBP_OK;
}

mpbp_status mpbp_set_data(mpbp_ctx* c, const float* y, const float* bg, void* stream) {
  if (!c || !y) return fail(c, MPBP_ERR_INVALID_ARG, "null data");
  MPBP_CUDA(c, launch_frame_transpose(y, c->aT, c->nframes, c->M, true, S(stream)));
  if (bg) {
    if (!c->bgT) {
      cudaError_t e = cudaMalloc(&c->bgT, sizeof(float) * c->nframes * c->M * c->M);
      if (e != cudaSuccess) {
        cudaGetLastError();
        c->bgT = nullptr;
        return fail(c, MPBP_ERR_OOM, "background buffer");
      }
    }
    MPBP_CUDA(c, launch_frame_transpose(bg, c->bgT, c->nframes, c->M, false, S(stream)));
  } else if (c->bgT) {
    MPBP_CUDA(c, cudaStreamSynchronize(S(stream)));
    cudaFree(c->bgT);
    c->bgT = nullptr;
  }
  c->has_data = true;
  c->version++;
  return MPBP_OK;
}

mpbp_status mpbp_object_build(mpbp_ctx* c, const float* rho, const float* u, const float* alpha,
                              float* O_out, void* stream) {
  if (!c || !rho || !u || !alpha || !O_out) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  return enqueue_object_build(c, rho, u, alpha, reinterpret_cast<cf*>(O_out), S(stream));
}

mpbp_status mpbp_forward(mpbp_ctx* c, const float* rho, const float* u, const float* alpha,
                         float* I_out, void* stream) {
  if (!c || !rho || !u || !alpha || !I_out) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->has_probe) return fail(c, MPBP_ERR_NO_DATA, "probe not set");
  mpbp_status r = enqueue_object_build(c, rho, u, alpha, c->O, S(stream));
  if (r != MPBP_OK) return r;
  FrameArgs fa = frame_args(c, nullptr, (int)c->nframes);
  fa.I_out = I_out;
  fa.arrivals = nullptr;
  MPBP_CUDA(c, frames_launch(c->M, fa, frames_grid_fft(c, c->nframes), true, S(stream),
                             c->tile_fwd ? &c->tm_fwd : nullptr));
  return MPBP_OK;
}

mpbp_status mpbp_loss_grad(mpbp_ctx* c, const float* rho, const float* u, const float* alpha,
                           const int32_t* frames, int32_t nframes, double* loss, float* g_rho,
                           float* g_u, double* g_alpha, void* stream) {
  if (!c || !rho || !u || !alpha || !loss) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (frames && nframes < 0) return fail(c, MPBP_ERR_INVALID_ARG, "nframes < 0");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  return enqueue_loss_grad(c, rho, u, alpha, frames, nframes, loss, g_rho ? g_rho : c->g_rho_ws,
                           g_u ? g_u : c->g_u_ws, g_alpha, nullptr, S(stream));
}

mpbp_status mpbp_loss(mpbp_ctx* c, const float* rho, const float* u, const float* alpha,
                      const int32_t* frames, int32_t nframes, double* loss, void* stream) {
  if (!c || !rho || !u || !alpha || !loss) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (frames && nframes < 0) return fail(c, MPBP_ERR_INVALID_ARG, "nframes < 0");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  cudaStream_t s = S(stream);
  mpbp_status r = enqueue_object_build(c, rho, u, alpha, c->O, s);
  if (r != MPBP_OK) return r;
  const int nf = frames ? nframes : (int)c->nframes;
  FrameArgs fa = frame_args(c, frames, nf);
  fa.arrivals = nullptr;   // no gradient assembly follows
  const int grid = frames_grid_fft(c, nf);
  if (c->tile_grad) {
    TmaMap tm = c->tm_grad;
    tm.tx_extra = c->test_tx_extra;
    MPBP_CUDA(c, frames_launch_loss(c->M, fa, grid, s, &tm, c->fft_schedule));
  } else {
    MPBP_CUDA(c, frames_launch_loss(c->M, fa, grid, s, nullptr, c->fft_schedule));
  }
  MPBP_CUDA(c, launch_loss_reduce(c->loss_part, grid, loss, c->err, s));
  return MPBP_OK;
}

}  // extern "C"

namespace {

// The host-buffer evaluation; y: float counts, or (y16) 16-bit counts.
mpbp_status loss_grad_host_impl(mpbp_ctx* c, const void* y, bool y16, const float* rho, const float* u,
                                const float* alpha, double* loss, float* g_rho, float* g_u,
                                double* g_alpha, void* stream) {
  if (!c || !rho || !u || !alpha || !loss) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->has_probe) return fail(c, MPBP_ERR_NO_DATA, "probe not set");
  if (!y && !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "data not set");
  if (c->det) return fail(c, MPBP_ERR_UNSUPPORTED, "the deterministic gradient takes device-resident data");
  cudaStream_t s = S(stream);
  const long long nx = c->npix * (1 + c->C) + c->D;
  const long long mm = (long long)c->M * c->M;
  if (!c->io_x) {
    cudaError_t e = cudaMalloc(&c->io_x, sizeof(float) * nx + sizeof(double) * 2);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->io_x = nullptr;
      return fail(c, MPBP_ERR_OOM, "host-path buffers");
    }
  }
  float* drho = c->io_x;
  float* du = drho + c->npix;
  float* dalpha = du + c->npix * c->C;
  double* dloss = reinterpret_cast<double*>(c->io_x + align_up(nx, 2));
  // Frames in chunks.  Chunk k of y is copied by the copy engine into one of
  // kStageSlots staging buffers while earlier chunks are evaluated.  On the
  // thread-pair frame sides (FP32 precision) the frame kernel reads the
  // staged counts in their natural layout and writes sqrt(y) into the
  // context's layout itself, and the chunk launches alternate between two
  // streams so that one chunk's last frames overlap the next chunk's first;
  // otherwise each chunk is transposed into the context's layout and
  // evaluated on the caller's stream.  The gradient accumulator sums over the
  // chunk launches, each with its own slice of loss partials.
  const bool raw = y && c->precision == MPBP_PRECISION_FP32 && frames_raw_supported(c->M);
  // 16-bit counts read by the raw-data kernel itself (tile copies), or
  // widened to floats on the device first (the other paths)
  const bool fast16 = y16 && raw && c->tile_fwd && frames_raw16_supported(c->M);
  int nchunks = 1;
  // (about 512 frames a chunk: fewer chunks leave less overlap, more chunks
  // cost more per-chunk launch and copy overhead; measured)
  if (y) nchunks = (int)std::min<long long>(kMaxHostChunks, std::max<long long>(1, c->nframes / 512));
  // chunk k holds frames [bound[k], bound[k+1]) (equal chunks: measured as
  // fast as chunks shrinking towards the end)
  long long bound[kMaxHostChunks + 1];
  for (int k = 0; k <= nchunks; ++k) bound[k] = c->nframes * k / nchunks;
  long long per = 0;
  for (int k = 0; k < nchunks; ++k) per = std::max(per, bound[k + 1] - bound[k]);
  if (y) {
    if (!c->copy_stream) {
      bool ok = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&c->ev_x, cudaEventDisableTiming) == cudaSuccess;
      for (int i = 0; i < 2 && ok; ++i)
        ok = cudaStreamCreateWithFlags(&c->chunk_stream[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_done[i], cudaEventDisableTiming) == cudaSuccess;
      for (int i = 0; i < kStageSlots && ok; ++i)
        ok = cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_consumed[i], cudaEventDisableTiming) == cudaSuccess;
      if (!ok) return fail(c, MPBP_ERR_CUDA, "host-path streams");
    }
    if (!fast16 && (size_t)(per * mm) > c->stage_elems) {
      MPBP_CUDA(c, cudaStreamSynchronize(s));
      MPBP_CUDA(c, cudaStreamSynchronize(c->copy_stream));
      if (c->stage) cudaFree(c->stage);
      c->stage = nullptr;
      c->stage_elems = 0;
      cudaError_t e = cudaMalloc(&c->stage, sizeof(float) * kStageSlots * per * mm);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MPBP_ERR_OOM, "host-path staging buffers");
      }
      c->stage_elems = per * mm;
      c->ymap_per = 0;
    }
    if (y16 && (size_t)(per * mm) > c->stage16_elems) {
      MPBP_CUDA(c, cudaStreamSynchronize(s));
      MPBP_CUDA(c, cudaStreamSynchronize(c->copy_stream));
      if (c->stage16) cudaFree(c->stage16);
      c->stage16 = nullptr;
      c->stage16_elems = 0;
      cudaError_t e = cudaMalloc(&c->stage16, sizeof(unsigned short) * kStageSlots * per * mm);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MPBP_ERR_OOM, "host-path staging buffers");
      }
      c->stage16_elems = per * mm;
      c->ymap16_per = 0;
    }
  }
  // tile copies for the raw-data kernel: the objects' map of the pair layout
  // (the forward kernel's box) and one counts map per staging slot
  bool raw_tiles = raw && c->tile_fwd;
  if (raw_tiles && !fast16 && c->ymap_per != per) {
    for (int i = 0; i < kStageSlots && raw_tiles; ++i)
      raw_tiles = encode_counts_map(c, c->stage + i * c->stage_elems, per, false, &c->ymap[i]);
    c->ymap_per = raw_tiles ? per : 0;
  }
  if (fast16 && c->ymap16_per != per) {
    bool ok = true;
    for (int i = 0; i < kStageSlots && ok; ++i)
      ok = encode_counts_map(c, c->stage16 + i * c->stage16_elems, per, true, &c->ymap16[i]);
    if (!ok) return fail(c, MPBP_ERR_CUDA, "tensor map of the 16-bit counts");
    c->ymap16_per = per;
  }
  auto copy_chunk = [&](int k) -> mpbp_status {
    const int slot = k % kStageSlots;
    const long long f0 = bound[k];
    const long long nf = bound[k + 1] - f0;
    if (k >= kStageSlots) MPBP_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_consumed[slot], 0));
    if (y16)
      MPBP_CUDA(c, cudaMemcpyAsync(c->stage16 + slot * c->stage16_elems,
                                   static_cast<const unsigned short*>(y) + f0 * mm,
                                   sizeof(unsigned short) * nf * mm, cudaMemcpyHostToDevice, c->copy_stream));
    else
      MPBP_CUDA(c, cudaMemcpyAsync(c->stage + slot * c->stage_elems, static_cast<const float*>(y) + f0 * mm,
                                   sizeof(float) * nf * mm, cudaMemcpyHostToDevice, c->copy_stream));
    MPBP_CUDA(c, cudaEventRecord(c->ev_copied[slot], c->copy_stream));
    return MPBP_OK;
  };

  // The host link carries rho, u, alpha first, then the first chunks of y.
  // io_x and the staging buffers are used by this function alone, and its
  // last call released them before it returned, so these copies need not
  // wait for anything.
  cudaStream_t xs = y ? c->copy_stream : s;
  MPBP_CUDA(c, cudaMemcpyAsync(drho, rho, sizeof(float) * c->npix, cudaMemcpyHostToDevice, xs));
  MPBP_CUDA(c, cudaMemcpyAsync(du, u, sizeof(float) * c->npix * c->C, cudaMemcpyHostToDevice, xs));
  MPBP_CUDA(c, cudaMemcpyAsync(dalpha, alpha, sizeof(float) * c->D, cudaMemcpyHostToDevice, xs));
  if (y) {
    MPBP_CUDA(c, cudaEventRecord(c->ev_x, c->copy_stream));
    for (int k = 0; k < nchunks && k < kStageSlots; ++k) {
      mpbp_status rc = copy_chunk(k);
      if (rc != MPBP_OK) return rc;
    }
    MPBP_CUDA(c, cudaStreamWaitEvent(s, c->ev_x, 0));
  }
  if (c->acc_dirty) {
    MPBP_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(cf) * c->npix * c->D, s));
    c->acc_dirty = false;
  }
  mpbp_status r = enqueue_object_build(c, drho, du, dalpha, c->O, s);
  if (r != MPBP_OK) return r;
  // the frame launches follow the object build and any earlier work of the
  // caller's stream (which may still read the data being replaced)
  if (y) MPBP_CUDA(c, cudaEventRecord(c->ev_ready, s));
  c->acc_dirty = true;
  int nparts = 0;
  for (int k = 0; k < nchunks; ++k) {
    const long long f0 = bound[k];
    const long long nf = bound[k + 1] - f0;
    if (nf <= 0) continue;
    FrameArgs fa = frame_args(c, nullptr, (int)nf);
    fa.frame0 = (int)f0;
    fa.loss_part = c->loss_part + nparts;
    fa.arrivals = k == 0 ? c->arrivals : nullptr;
    const int grid = frames_grid_for(c, nf);
    if (y) {
      const int slot = k % kStageSlots;
      float* st = fast16 ? nullptr : c->stage + slot * c->stage_elems;
      if (k >= kStageSlots) {
        mpbp_status rc = copy_chunk(k);
        if (rc != MPBP_OK) return rc;
      }
      // 16-bit counts for a path that reads floats: widen them first
      auto widen = [&](cudaStream_t ws) -> mpbp_status {
        if (y16 && !fast16)
          MPBP_CUDA(c, launch_counts16(c->stage16 + slot * c->stage16_elems, st, nf * mm, c->num_sms, ws));
        return MPBP_OK;
      };
      if (raw) {
        // the last chunk runs on the caller's stream, right before the finish
        const bool last = k == nchunks - 1;
        cudaStream_t cs = last ? s : c->chunk_stream[k & 1];
        if (k < 2 && !last) MPBP_CUDA(c, cudaStreamWaitEvent(cs, c->ev_ready, 0));
        MPBP_CUDA(c, cudaStreamWaitEvent(cs, c->ev_copied[slot], 0));
        mpbp_status wr = widen(cs);
        if (wr != MPBP_OK) return wr;
        fa.yraw = st ? st - f0 * mm : nullptr;   // indexed by absolute frame number
        fa.aT_w = c->aT;
        if (fast16) {
          TmaMap tm = c->tm_fwd;
          tm.ymap = c->ymap16[slot];
          tm.tx_extra = 0;
          MPBP_CUDA(c, frames_launch_raw(c->M, fa, grid, cs, &tm, true));
        } else if (raw_tiles) {
          TmaMap tm = c->tm_fwd;
          tm.ymap = c->ymap[slot];
          tm.tx_extra = 0;
          MPBP_CUDA(c, frames_launch_raw(c->M, fa, grid, cs, &tm));
        } else {
          MPBP_CUDA(c, frames_launch_raw(c->M, fa, grid, cs));
        }
        MPBP_CUDA(c, cudaEventRecord(c->ev_consumed[slot], cs));
      } else {
        MPBP_CUDA(c, cudaStreamWaitEvent(s, c->ev_copied[slot], 0));
        mpbp_status wr = widen(s);
        if (wr != MPBP_OK) return wr;
        MPBP_CUDA(c, launch_frame_transpose(st, c->aT + f0 * mm, nf, c->M, true, s));
        MPBP_CUDA(c, cudaEventRecord(c->ev_consumed[slot], s));
        MPBP_CUDA(c, launch_frames(c, fa, grid, s));
      }
    } else {
      MPBP_CUDA(c, launch_frames(c, fa, grid, s));
    }
    nparts += grid;
  }
  if (raw) {
    for (int i = 0; i < 2 && i < nchunks - 1; ++i) {
      MPBP_CUDA(c, cudaEventRecord(c->ev_done[i], c->chunk_stream[i]));
      MPBP_CUDA(c, cudaStreamWaitEvent(s, c->ev_done[i], 0));
    }
  }
  if (y) c->has_data = true;

  FinishArgs fi{};
  fi.rho = drho;
  fi.u = du;
  fi.alpha = dalpha;
  fi.acc = c->acc;
  fi.g_rho = c->g_rho_ws;
  fi.g_u = c->g_u_ws;
  fi.part = c->part;
  fi.npix = c->npix;
  fi.D = c->D;
  fi.C = c->C;
  fi.pc = c->pc;
  fi.arrivals = c->arrivals;
  fi.loss_part = c->loss_part;
  fi.n_loss_part = nparts;
  ReduceArgs ra{};
  ra.part = c->part;
  ra.n_part = c->finish_grid;
  ra.D = c->D;
  ra.loss_out = dloss;
  ra.g_alpha_out = nullptr;
  ra.g_alpha_ws = c->g_alpha_ws;
  ra.err = c->err;
  ra.st = nullptr;
  ra.alpha_from = 1;
  // Page-locked outputs are written by the gradient assembly itself, through
  // their device mapping; otherwise they are copied back from the workspace.
  void* m_loss = mapped_host(loss);
  void* m_rho = g_rho ? mapped_host(g_rho) : nullptr;
  void* m_u = g_u ? mapped_host(g_u) : nullptr;
  void* m_alpha = g_alpha ? mapped_host(g_alpha) : nullptr;
  const bool direct = m_loss && (!g_rho || m_rho) && (!g_u || m_u) && (!g_alpha || m_alpha);
  if (direct) {
    if (m_rho) fi.g_rho = static_cast<float*>(m_rho);
    if (m_u) fi.g_u = static_cast<float*>(m_u);
    ra.loss_out = static_cast<double*>(m_loss);
    ra.g_alpha_out = static_cast<double*>(m_alpha);
  }
  MPBP_CUDA(c, launch_finish(fi, ra, c->finish_grid, s));
  c->acc_dirty = false;
  if (direct) {
    MPBP_CUDA(c, cudaStreamSynchronize(s));
    return MPBP_OK;
  }

  MPBP_CUDA(c, cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (g_rho)
    MPBP_CUDA(c, cudaMemcpyAsync(g_rho, c->g_rho_ws, sizeof(float) * c->npix, cudaMemcpyDeviceToHost, s));
  if (g_u)
    MPBP_CUDA(c, cudaMemcpyAsync(g_u, c->g_u_ws, sizeof(float) * c->npix * c->C,
                                 cudaMemcpyDeviceToHost, s));
  if (g_alpha)
    MPBP_CUDA(c, cudaMemcpyAsync(g_alpha, c->g_alpha_ws, sizeof(double) * c->D,
                                 cudaMemcpyDeviceToHost, s));
  MPBP_CUDA(c, cudaStreamSynchronize(s));
  return MPBP_OK;
}

}  // namespace

extern "C" {

mpbp_status mpbp_loss_grad_host(mpbp_ctx* c, const float* y, const float* rho, const float* u,
                                const float* alpha, double* loss, float* g_rho, float* g_u,
                                double* g_alpha, void* stream) {
  return loss_grad_host_impl(c, y, false, rho, u, alpha, loss, g_rho, g_u, g_alpha, stream);
}

mpbp_status mpbp_loss_grad_host_counts16(mpbp_ctx* c, const uint16_t* y, const float* rho, const float* u,
                                         const float* alpha, double* loss, float* g_rho, float* g_u,
                                         double* g_alpha, void* stream) {
  if (!y) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  return loss_grad_host_impl(c, y, true, rho, u, alpha, loss, g_rho, g_u, g_alpha, stream);
}

mpbp_status mpbp_step_init(mpbp_ctx* c, const mpbp_step_params* prm, mpbp_step_state* st,
                           void* stream) {
  if (!c || !prm || !st) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!(prm->t0 > 0) || !(prm->grow >= 1) || !(prm->shrink > 0 && prm->shrink < 1) ||
      !(prm->c_armijo >= 0) || !(prm->w_rho >= 0) || !(prm->w_u >= 0) || !(prm->w_alpha >= 0))
    return fail(c, MPBP_ERR_INVALID_ARG, "step parameters out of range");
  mpbp_step_state h{};
  h.t = prm->t0;
  h.c_armijo = prm->c_armijo;
  h.grow = prm->grow;
  h.shrink = prm->shrink;
  h.w_rho = prm->w_rho;
  h.w_u = prm->w_u;
  h.w_alpha = prm->w_alpha;
  MPBP_CUDA(c, cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, S(stream)));
  MPBP_CUDA(c, cudaStreamSynchronize(S(stream)));
  return MPBP_OK;
}

mpbp_status mpbp_step(mpbp_ctx* c, float* rho, float* u, float* alpha, mpbp_step_state* st,
                      void* stream) {
  if (!c || !rho || !u || !alpha || !st) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  cudaStream_t s = S(stream);
  StepPtrs sp{};
  sp.rho = rho;
  sp.u = u;
  sp.alpha = alpha;
  sp.rho_base = c->rho_base;
  sp.u_base = c->u_base;
  sp.alpha_base = c->alpha_base;
  sp.g_rho_base = c->g_rho_base;
  sp.g_u_base = c->g_u_base;
  sp.g_alpha_base = c->g_alpha_base;
  return enqueue_loss_grad(c, rho, u, alpha, nullptr, 0, c->loss_ws, c->g_rho_ws, c->g_u_ws, nullptr,
                           st, s, nullptr, nullptr, &sp);
}

mpbp_status mpbp_adam_init(mpbp_ctx* c, const mpbp_adam_params* prm, mpbp_adam_state* st,
                           void* stream) {
  if (!c || !prm || !st) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!(prm->lr_u >= 0) || !(prm->lr_chi >= 0) || !(prm->lr_alpha >= 0) || !(prm->beta1 >= 0 && prm->beta1 < 1) ||
      !(prm->beta2 >= 0 && prm->beta2 < 1) || !(prm->eps >= 0))
    return fail(c, MPBP_ERR_INVALID_ARG, "Adam parameters out of range");
  cudaStream_t s = S(stream);
  const long long np = c->npix, nu = c->npix * c->C;
  if (!c->adam_buf) {
    Carver cv;
    const size_t o_mc = cv.take<float>(np), o_vc = cv.take<float>(np), o_mu = cv.take<float>(nu),
                 o_vu = cv.take<float>(nu), o_ma = cv.take<double>(c->D), o_va = cv.take<double>(c->D),
                 o_rx = cv.take<float>(np), o_ax = cv.take<float>(c->D);
    void* b = nullptr;
    MPBP_CUDA(c, cudaStreamSynchronize(s));
    if (cudaMalloc(&b, align_up(cv.off, 256)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MPBP_ERR_OOM, "Adam moment buffers");
    }
    c->adam_buf = b;
    char* p = static_cast<char*>(b);
    c->m_chi = reinterpret_cast<float*>(p + o_mc);
    c->v_chi = reinterpret_cast<float*>(p + o_vc);
    c->m_u = reinterpret_cast<float*>(p + o_mu);
    c->v_u = reinterpret_cast<float*>(p + o_vu);
    c->m_a = reinterpret_cast<double*>(p + o_ma);
    c->v_a = reinterpret_cast<double*>(p + o_va);
    c->rho_x = reinterpret_cast<float*>(p + o_rx);
    c->alpha_x = reinterpret_cast<float*>(p + o_ax);
  }
  MPBP_CUDA(c, cudaMemsetAsync(c->m_chi, 0, sizeof(float) * np, s));
  MPBP_CUDA(c, cudaMemsetAsync(c->v_chi, 0, sizeof(float) * np, s));
  MPBP_CUDA(c, cudaMemsetAsync(c->m_u, 0, sizeof(float) * nu, s));
  MPBP_CUDA(c, cudaMemsetAsync(c->v_u, 0, sizeof(float) * nu, s));
  MPBP_CUDA(c, cudaMemsetAsync(c->m_a, 0, sizeof(double) * c->D, s));
  MPBP_CUDA(c, cudaMemsetAsync(c->v_a, 0, sizeof(double) * c->D, s));
  mpbp_adam_state h{};
  h.lr_u = prm->lr_u;
  h.lr_chi = prm->lr_chi;
  h.lr_alpha = prm->lr_alpha;
  h.beta1 = prm->beta1;
  h.beta2 = prm->beta2;
  h.eps = prm->eps;
  h.bc1 = h.bc2 = 1.0;
  MPBP_CUDA(c, cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  MPBP_CUDA(c, cudaStreamSynchronize(s));
  return MPBP_OK;
}

mpbp_status mpbp_adam_step(mpbp_ctx* c, const int32_t* frames, int32_t nframes, float* chi, float* u,
                           float* alpha_t, const float* mask, mpbp_adam_state* st, void* stream) {
  if (!c || !chi || !u || !alpha_t || !st) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (frames && nframes < 0) return fail(c, MPBP_ERR_INVALID_ARG, "nframes < 0");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  if (!c->adam_buf) return fail(c, MPBP_ERR_NO_DATA, "mpbp_adam_init first");
  cudaStream_t s = S(stream);
  AdamArgs a{};
  a.chi = chi;
  a.u = u;
  a.alpha_t = alpha_t;
  a.mask = mask;
  a.rho_x = c->rho_x;
  a.alpha_x = c->alpha_x;
  a.g_rho = c->g_rho_ws;
  a.g_u = c->g_u_ws;
  a.g_alpha = c->g_alpha_ws;
  a.m_chi = c->m_chi;
  a.v_chi = c->v_chi;
  a.m_u = c->m_u;
  a.v_u = c->v_u;
  a.m_a = c->m_a;
  a.v_a = c->v_a;
  a.st = st;
  a.npix = c->npix;
  a.C = c->C;
  a.D = c->D;
  MPBP_CUDA(c, launch_adam_prep(a, c->num_sms, s));
  mpbp_status r = enqueue_loss_grad(c, c->rho_x, u, c->alpha_x, frames, frames ? nframes : 0, &st->f_last,
                                    c->g_rho_ws, c->g_u_ws, nullptr, nullptr, s);
  if (r != MPBP_OK) return r;
  MPBP_CUDA(c, launch_adam_update(a, c->num_sms, s));
  return MPBP_OK;
}

mpbp_status mpbp_adam_get_state(mpbp_ctx* c, float* m_chi, float* v_chi, float* m_u, float* v_u,
                                double* m_alpha, double* v_alpha, void* stream) {
  if (!c || !m_chi || !v_chi || !m_u || !v_u || !m_alpha || !v_alpha)
    return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->adam_buf) return fail(c, MPBP_ERR_NO_DATA, "mpbp_adam_init first");
  cudaStream_t s = S(stream);
  const long long np = c->npix, nu = c->npix * c->C;
  MPBP_CUDA(c, cudaMemcpyAsync(m_chi, c->m_chi, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(v_chi, c->v_chi, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(m_u, c->m_u, sizeof(float) * nu, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(v_u, c->v_u, sizeof(float) * nu, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(m_alpha, c->m_a, sizeof(double) * c->D, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(v_alpha, c->v_a, sizeof(double) * c->D, cudaMemcpyDeviceToDevice, s));
  return MPBP_OK;
}

mpbp_status mpbp_adam_set_state(mpbp_ctx* c, const float* m_chi, const float* v_chi, const float* m_u,
                                const float* v_u, const double* m_alpha, const double* v_alpha,
                                void* stream) {
  if (!c || !m_chi || !v_chi || !m_u || !v_u || !m_alpha || !v_alpha)
    return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->adam_buf) return fail(c, MPBP_ERR_NO_DATA, "mpbp_adam_init first");
  cudaStream_t s = S(stream);
  const long long np = c->npix, nu = c->npix * c->C;
  MPBP_CUDA(c, cudaMemcpyAsync(c->m_chi, m_chi, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(c->v_chi, v_chi, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(c->m_u, m_u, sizeof(float) * nu, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(c->v_u, v_u, sizeof(float) * nu, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(c->m_a, m_alpha, sizeof(double) * c->D, cudaMemcpyDeviceToDevice, s));
  MPBP_CUDA(c, cudaMemcpyAsync(c->v_a, v_alpha, sizeof(double) * c->D, cudaMemcpyDeviceToDevice, s));
  return MPBP_OK;
}

mpbp_status mpbp_loss_grad_phases(mpbp_ctx* c, const float* rho, const float* phi, const float* alpha,
                                  const int32_t* frames, int32_t nframes, double* loss, float* g_rho,
                                  float* g_phi, double* g_alpha, void* stream) {
  if (!c || !rho || !phi || !alpha || !loss || !g_rho || !g_phi)
    return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (frames && nframes < 0) return fail(c, MPBP_ERR_INVALID_ARG, "nframes < 0");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  return enqueue_loss_grad(c, rho, nullptr, alpha, frames, frames ? nframes : 0, loss, g_rho, nullptr,
                           g_alpha, nullptr, S(stream), phi, g_phi);
}

// the unwrapper's workspace for the context's D maps
mpbp_status unwrap_setup(mpbp_ctx* c, cudaStream_t s) {
  if (c->uw_buf) return MPBP_OK;
  if (!unwrap_prepare(c->num_sms, &c->uw_grid)) return fail(c, MPBP_ERR_CUDA, "unwrap kernel cannot run here");
  const long long nodes = c->npix * c->D;
  Carver cv;
  const size_t o_rel = cv.take<float>(nodes), o_p = cv.take<int>(nodes), o_o = cv.take<int>(nodes),
               o_p2 = cv.take<int>(nodes), o_o2 = cv.take<int>(nodes), o_hp = cv.take<int>(nodes),
               o_ho = cv.take<int>(nodes), o_mn = cv.take<int>(nodes),
               o_b = cv.take<unsigned long long>(nodes), o_ek = cv.take<unsigned long long>(2 * nodes),
               o_f = cv.take<int>(3), o_bc = cv.take<unsigned>(2),
               o_phi = cv.take<float>(nodes), o_w = cv.take<float>(nodes);
  void* b = nullptr;
  MPBP_CUDA(c, cudaStreamSynchronize(s));
  if (cudaMalloc(&b, align_up(cv.off, 256)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MPBP_ERR_OOM, "unwrap workspace");
  }
  c->uw_buf = b;
  char* p = static_cast<char*>(b);
  UnwrapArgs& a = c->uw;
  a.rel = reinterpret_cast<float*>(p + o_rel);
  a.parent = reinterpret_cast<int*>(p + o_p);
  a.off = reinterpret_cast<int*>(p + o_o);
  a.parent2 = reinterpret_cast<int*>(p + o_p2);
  a.off2 = reinterpret_cast<int*>(p + o_o2);
  a.hook_parent = reinterpret_cast<int*>(p + o_hp);
  a.hook_off = reinterpret_cast<int*>(p + o_ho);
  a.minnode = reinterpret_cast<int*>(p + o_mn);
  a.best = reinterpret_cast<unsigned long long*>(p + o_b);
  a.ekey = reinterpret_cast<unsigned long long*>(p + o_ek);
  a.flags = reinterpret_cast<int*>(p + o_f);
  a.bar_count = reinterpret_cast<unsigned*>(p + o_bc);
  a.bar_gen = a.bar_count + 1;
  a.err = c->err;
  a.npix = c->npix;
  a.nodes = nodes;
  a.n1 = c->n1;
  a.n2 = c->n2;
  int rounds = 2;
  while ((1ll << rounds) < nodes) ++rounds;
  a.max_rounds = rounds + 2;
  c->pj_phi = reinterpret_cast<float*>(p + o_phi);
  c->pj_wrapped = reinterpret_cast<float*>(p + o_w);
  return MPBP_OK;
}

mpbp_status enqueue_unwrap(mpbp_ctx* c, const float* wrapped, const float* mask, float* out, cudaStream_t s) {
  UnwrapArgs a = c->uw;
  a.wrapped = wrapped;
  a.mask = mask;
  a.out = out;
  a.test_stall = c->test_tx_extra != 0 ? 1 : 0;
  MPBP_CUDA(c, cudaMemsetAsync(a.flags, 0, sizeof(int) * 3, s));
  MPBP_CUDA(c, cudaMemsetAsync(a.bar_count, 0, sizeof(unsigned) * 2, s));
  MPBP_CUDA(c, unwrap_launch(a, c->uw_grid, s));
  return MPBP_OK;
}

// Moore-Penrose pseudo-inverse [C][D] of G [D][C] (C <= 3) as the limit of
// (G^T G + delta I)^{-1} G^T: delta = 1e-12 trace(G^T G) leaves full-rank
// cases exact to ~1e-12 and maps directions no G_m reaches to zero.
void pseudo_inverse(int D, int C, const std::vector<double>& G, double* pinv) {
  double A[3][3] = {{0}};
  double tr = 0.0;
  for (int a = 0; a < C; ++a)
    for (int b = 0; b < C; ++b) {
      for (int m = 0; m < D; ++m) A[a][b] += G[m * C + a] * G[m * C + b];
    }
  for (int a = 0; a < C; ++a) tr += A[a][a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      if (a >= C || b >= C) A[a][b] = (a == b) ? 1.0 : 0.0;
      else if (a == b) A[a][b] += 1e-12 * tr;
    }
  // 3 x 3 inverse by cofactors
  double inv[3][3];
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
  inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
  inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
  inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
  for (int a = 0; a < C; ++a)
    for (int m = 0; m < D; ++m) {
      double v = 0.0;
      for (int b = 0; b < C; ++b) v += inv[a][b] * G[m * C + b];
      pinv[a * D + m] = v;
    }
}

mpbp_status mpbp_unwrap_phases(mpbp_ctx* c, const float* wrapped, const float* mask, float* out, void* stream) {
  if (!c || !wrapped || !out) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = S(stream);
  mpbp_status r = unwrap_setup(c, s);
  if (r != MPBP_OK) return r;
  return enqueue_unwrap(c, wrapped, mask, out, s);
}

mpbp_status mpbp_project_displacement(mpbp_ctx* c, float* u, const float* mask, void* stream) {
  if (!c || !u) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = S(stream);
  mpbp_status r = unwrap_setup(c, s);
  if (r != MPBP_OK) return r;
  ProjectArgs pa{};
  pa.u = u;
  pa.mask = mask;
  pa.phi = c->pj_phi;
  pa.wrapped = c->pj_wrapped;
  pa.unwrapped = c->pj_wrapped;   // unwrapped in place of the wrapped copy
  pa.npix = c->npix;
  pa.C = c->C;
  pa.D = c->D;
  double pinv[kMaxComp * kMaxPeaks];
  pseudo_inverse(c->D, c->C, c->G, pinv);
  for (int m = 0; m < c->D; ++m)
    for (int k = 0; k < c->C; ++k) {
      pa.g_scaled[m * kMaxComp + k] = (float)(c->phase_scale * c->G[m * c->C + k]);
      pa.pinv_scaled[k * kMaxPeaks + m] = (float)(pinv[k * c->D + m] / c->phase_scale);
    }
  MPBP_CUDA(c, project_phase_launch(pa, c->num_sms, s));
  r = enqueue_unwrap(c, c->pj_wrapped, mask, c->pj_wrapped, s);
  if (r != MPBP_OK) return r;
  MPBP_CUDA(c, project_correct_launch(pa, c->num_sms, s));
  return MPBP_OK;
}

mpbp_status mpbp_illumination(mpbp_ctx* c, float* out, void* stream) {
  if (!c || !out) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->has_probe) return fail(c, MPBP_ERR_NO_DATA, "probe not set");
  cudaStream_t s = S(stream);
  MPBP_CUDA(c, cudaMemsetAsync(out, 0, sizeof(float) * c->npix, s));
  IllumArgs a{};
  a.probe = c->probe;
  a.scan = c->scan;
  a.out = out;
  a.nframes = (int)c->nframes;
  a.J = c->J;
  a.m = c->M;
  a.n1 = c->n1;
  a.n2 = c->n2;
  a.probe_stride = c->probe_per_peak ? (long long)c->M * c->M : 0;
  if (!c->scan_off_h.empty()) {
    a.probe = c->probe_scan;
    a.probe_stride = c->probe_per_peak ? kProbePerFrame : kProbePerScan;
  }
  MPBP_CUDA(c, launch_illumination(a, c->num_sms, s));
  return MPBP_OK;
}

mpbp_status mpbp_step_capture(mpbp_ctx* c, float* rho, float* u, float* alpha, mpbp_step_state* st) {
  if (!c || !rho || !u || !alpha || !st) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  if (c->timing) return fail(c, MPBP_ERR_INVALID_ARG, "frame-kernel timing must be off while capturing");
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    return fail(c, MPBP_ERR_CUDA, "capture stream");
  }
  // the graph starts from a clear gradient accumulator, as every step leaves it
  if (c->acc_dirty) {
    MPBP_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(cf) * c->npix * c->D, c->cap_stream));
    MPBP_CUDA(c, cudaStreamSynchronize(c->cap_stream));
    c->acc_dirty = false;
  }
  MPBP_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const mpbp_status r = mpbp_step(c, rho, u, alpha, st, c->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  c->acc_dirty = false;   // the captured step ends by clearing the accumulator
  if (r != MPBP_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return r != MPBP_OK ? r : fail(c, MPBP_ERR_CUDA, "stream capture of the step failed");
  }
  cudaGraphExec_t x = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MPBP_ERR_CUDA, "graph instantiation failed");
  }
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  c->step_exec = x;
  return MPBP_OK;
}

mpbp_status mpbp_step_replay(mpbp_ctx* c, void* stream) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  if (!c->step_exec) return fail(c, MPBP_ERR_INVALID_ARG, "no step captured");
  cudaStream_t s = S(stream);
  if (c->acc_dirty) {
    MPBP_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(cf) * c->npix * c->D, s));
    c->acc_dirty = false;
  }
  MPBP_CUDA(c, cudaGraphLaunch(c->step_exec, s));
  return MPBP_OK;
}

mpbp_status mpbp_loss_grad_batched(int32_t n, mpbp_ctx* const* ctxs, const float* const* rho,
                                   const float* const* u, const float* const* alpha,
                                   double* const* loss, float* const* g_rho, float* const* g_u,
                                   double* const* g_alpha, void* stream) {
  if (n < 0 || (n > 0 && (!ctxs || !rho || !u || !alpha || !loss || !g_rho || !g_u)))
    return MPBP_ERR_INVALID_ARG;
  if (n == 0) return MPBP_OK;
  mpbp_ctx* lead = ctxs[0];
  if (!lead) return MPBP_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (ctxs[i] && ctxs[i]->det)
      return fail(lead, MPBP_ERR_UNSUPPORTED, "batched evaluations use the atomic gradient (a problem is deterministic)");
  cudaStream_t s = S(stream);
  for (int i = 0; i < n; ++i) {
    mpbp_ctx* c = ctxs[i];
    if (!c || !rho[i] || !u[i] || !alpha[i] || !loss[i] || !g_rho[i] || !g_u[i])
      return fail(lead, MPBP_ERR_INVALID_ARG, "null argument in batch");
    if (c->device != lead->device) return fail(lead, MPBP_ERR_INVALID_ARG, "batch spans devices");
    if (!c->has_probe || !c->has_data) return fail(lead, MPBP_ERR_NO_DATA, "probe or data not set");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == c) return fail(lead, MPBP_ERR_INVALID_ARG, "a context appears twice in a batch");
  }
  // problems with M in {32, 64, 128} share the batched kernel: one launch for
  // all sides (mode 0) or one per side (mode 1), at most kBatchMaxProbs
  // problems per launch.  The plan (item table, launch arguments) is built
  // once per batch composition and kept in the lead context.
  std::vector<long long> key = {lead->batch_mode, lead->batch_order, n};
  for (int i = 0; i < n; ++i) {
    key.push_back((long long)ctxs[i]->serial);
    key.push_back((long long)ctxs[i]->version);
  }
  if (key != lead->batch_key || !lead->batch_ws) {
    lead->batch_key.clear();
    lead->batch_plan.clear();
    std::vector<int> fused;
    for (int i = 0; i < n; ++i)
      if (batch_fused_side(lead->batch_mode, ctxs[i]->M)) fused.push_back(i);
    const int nf = (int)fused.size();
    std::vector<long long> base(nf);
    long long total_frames = 0;
    for (int k = 0; k < nf; ++k) {
      base[k] = total_frames;
      total_frames += ctxs[fused[k]]->nframes;
    }
    // frames per work item: a 256-thread block's worth in the single launch
    // over every side (mode 0), one frame in the per-side launches
    auto per_item = [&](int m) {
      if (lead->batch_mode != 0) return 1;
      return m >= 128 ? 1 : (m == 64 ? 2 : 4);
    };
    struct Launch {
      int m;
      std::vector<int> probs;   // indices into `fused`
      size_t first, count;      // item range
    };
    std::vector<Launch> launches;
    std::vector<int2> items;    // (problem index within its launch, first frame)
    auto add_launch = [&](int m, const std::vector<int>& probs) {
      Launch L{m, probs, items.size(), 0};
      const int np = (int)probs.size();
      for (int side : {128, 64, 32}) {
        if (lead->batch_order == 0) {
          for (int k = 0; k < np; ++k) {
            mpbp_ctx* c = ctxs[fused[probs[k]]];
            if (c->M != side) continue;
            for (long long f = 0; f < c->nframes; f += per_item(side)) items.push_back(make_int2(k, (int)f));
          }
        } else {
          std::vector<long long> next(np, 0);
          bool any = true;
          while (any) {
            any = false;
            for (int k = 0; k < np; ++k) {
              mpbp_ctx* c = ctxs[fused[probs[k]]];
              if (c->M != side || next[k] >= c->nframes) continue;
              items.push_back(make_int2(k, (int)next[k]));
              next[k] += per_item(side);
              any = true;
            }
          }
        }
      }
      L.count = items.size() - L.first;
      if (L.count) launches.push_back(L);
    };
    for (int side : {0, 128, 64, 32}) {
      if ((lead->batch_mode == 0) != (side == 0)) continue;
      std::vector<int> group;
      for (int k = 0; k < nf; ++k) {
        if (side != 0 && ctxs[fused[k]]->M != side) continue;
        group.push_back(k);
        if ((int)group.size() == kBatchMaxProbs) {
          add_launch(side, group);
          group.clear();
        }
      }
      if (!group.empty()) add_launch(side, group);
    }
    // device tables in the lead context's batch buffer
    // per-side launches of frame sides 32 and 64 whose problems all have
    // tile copies (rows of 16-byte multiples) take their inputs by TMA, each
    // problem through its own tensor map in the batch buffer
    std::vector<char> launch_tma(launches.size(), 0);
    size_t ntm = 0;
    for (size_t l = 0; l < launches.size(); ++l) {
      const Launch& L = launches[l];
      if (L.m != 32 && L.m != 64) continue;
      bool all = true;
      for (int k : L.probs) all = all && ctxs[fused[k]]->tile_grad;
      launch_tma[l] = all;
      if (all) ntm += L.probs.size();
    }
    Carver cv;
    const size_t oI = cv.take<int2>(items.empty() ? 1 : items.size());
    const size_t oFP = cv.take<double>((size_t)(total_frames > 0 ? total_frames : 1) * kBatchWarpSlots);
    const size_t oTM = cv.take<TmaMap>(ntm > 0 ? ntm : 1);
    const size_t need = align_up(cv.off, 256);
    if (need > lead->batch_ws_bytes) {
      MPBP_CUDA(lead, cudaStreamSynchronize(s));
      if (lead->batch_ws) cudaFree(lead->batch_ws);
      lead->batch_ws = nullptr;
      lead->batch_ws_bytes = 0;
      cudaError_t e = cudaMalloc(&lead->batch_ws, need);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(lead, MPBP_ERR_OOM, "batch tables");
      }
      lead->batch_ws_bytes = need;
    }
    char* wb = static_cast<char*>(lead->batch_ws);
    if (!items.empty())
      MPBP_CUDA(lead, cudaMemcpyAsync(wb + oI, items.data(), sizeof(int2) * items.size(),
                                      cudaMemcpyHostToDevice, s));
    double* frame_part = reinterpret_cast<double*>(wb + oFP);
    std::vector<TmaMap> tms(ntm > 0 ? ntm : 1);
    size_t tm_next = 0;
    for (size_t l = 0; l < launches.size(); ++l) {
      const Launch& L = launches[l];
      mpbp_ctx::PlanLaunch P{};
      P.m = L.m;
      P.tma = launch_tma[l] != 0;
      if (P.tma) P.args.tmaps = reinterpret_cast<const TmaMap*>(wb + oTM) + tm_next;
      for (size_t k = 0; k < L.probs.size(); ++k) {
        mpbp_ctx* c = ctxs[fused[L.probs[k]]];
        P.args.probs[k] = frame_args(c, nullptr, (int)c->nframes);
        P.args.prob_m[k] = c->M;
        P.args.frame_base[k] = base[L.probs[k]];
        if (P.tma) {
          tms[tm_next] = c->tm_grad;
          tms[tm_next].tx_extra = c->test_tx_extra;
          ++tm_next;
        }
      }
      P.args.nprob = (int)L.probs.size();
      P.args.items = reinterpret_cast<const int2*>(wb + oI) + L.first;
      P.args.nitems = (int)L.count;
      P.args.frame_part = frame_part;
      int bps = 1;
      const bool ok = L.m == 0 ? batched_prepare(&bps) : batched_m_prepare(L.m, P.tma, &bps);
      if (!ok) return fail(lead, MPBP_ERR_CUDA, "batched kernel setup");
      P.grid = (int)std::min<long long>((long long)L.count, (long long)lead->num_sms * bps);
      lead->batch_plan.push_back(P);
    }
    if (ntm > 0)
      MPBP_CUDA(lead, cudaMemcpyAsync(wb + oTM, tms.data(), sizeof(TmaMap) * ntm, cudaMemcpyHostToDevice, s));
    lead->batch_base = base;
    lead->batch_fused = fused;
    lead->batch_frames = total_frames;
    lead->batch_key = key;
  }
  const std::vector<long long>& base = lead->batch_base;
  const std::vector<int>& fused = lead->batch_fused;
  const int nf = (int)fused.size();

  // A1 for every problem
  for (int i = 0; i < n; ++i) {
    mpbp_ctx* c = ctxs[i];
    if (c->acc_dirty) {
      MPBP_CUDA(c, cudaMemsetAsync(c->acc, 0, sizeof(cf) * c->npix * c->D, s));
      c->acc_dirty = false;
    }
    mpbp_status r = enqueue_object_build(c, rho[i], u[i], alpha[i], c->O, s);
    if (r != MPBP_OK) return r;
  }
  // A2..A7: the batched launches, then the usual kernel for M <= 16
  double* frame_part = nullptr;
  if (!lead->batch_plan.empty()) {
    frame_part = lead->batch_plan[0].args.frame_part;
    MPBP_CUDA(lead, cudaMemsetAsync(frame_part, 0, sizeof(double) * lead->batch_frames * kBatchWarpSlots, s));
  }
  for (int k = 0; k < nf; ++k) ctxs[fused[k]]->acc_dirty = true;
  for (const auto& P : lead->batch_plan) {
    if (P.m == 0) MPBP_CUDA(lead, batched_launch(P.args, P.grid, s));
    else MPBP_CUDA(lead, batched_m_launch(P.m, P.tma, P.args, P.grid, s));
  }
  std::vector<int> grid_of(n, 0);
  for (int i = 0; i < n; ++i) {
    mpbp_ctx* c = ctxs[i];
    if (batch_fused_side(lead->batch_mode, c->M)) continue;
    FrameArgs fa = frame_args(c, nullptr, (int)c->nframes);
    grid_of[i] = frames_grid_for(c, c->nframes);
    c->acc_dirty = true;
    MPBP_CUDA(c, launch_frames(c, fa, grid_of[i], s));
  }
  // A6/A7 tail and A8 reductions per problem
  int k = 0;
  for (int i = 0; i < n; ++i) {
    mpbp_ctx* c = ctxs[i];
    FinishArgs fi{};
    fi.rho = rho[i];
    fi.u = u[i];
    fi.alpha = alpha[i];
    fi.acc = c->acc;
    fi.g_rho = g_rho[i];
    fi.g_u = g_u[i];
    fi.part = c->part;
    fi.arrivals = c->arrivals;
    fi.npix = c->npix;
    fi.D = c->D;
    fi.C = c->C;
    fi.pc = c->pc;
    ReduceArgs ra{};
    if (batch_fused_side(lead->batch_mode, c->M)) {
      fi.loss_part = frame_part + base[k] * kBatchWarpSlots;
      fi.n_loss_part = c->nframes * kBatchWarpSlots;
      ++k;
    } else {
      fi.loss_part = c->loss_part;
      fi.n_loss_part = grid_of[i];
    }
    ra.part = c->part;
    ra.n_part = c->finish_grid;
    ra.D = c->D;
    ra.loss_out = loss[i];
    ra.g_alpha_out = g_alpha ? g_alpha[i] : nullptr;
    ra.g_alpha_ws = c->g_alpha_ws;
    ra.err = c->err;
    ra.st = nullptr;
    ra.alpha_from = 1;
    MPBP_CUDA(c, launch_finish(fi, ra, c->finish_grid, s));
    c->acc_dirty = false;
  }
  return MPBP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// autotuning: time each candidate schedule on the caller's data, keep the
// fastest, optionally remember it in a JSON-lines cache file
// ---------------------------------------------------------------------------
namespace {

std::string gpu_name(int dev) {
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string n(prop.name);
  for (char& ch : n)
    if (ch == '"' || ch == '\\') ch = '_';
  return n;
}

// value of "field": <number> in a cache line whose "key" is `key` (-1: none)
double cache_lookup(const char* path, const std::string& key, const char* field) {
  if (!path) return -1.0;
  std::ifstream in(path);
  std::string line, want = "\"key\": \"" + key + "\"";
  double found = -1.0;
  while (std::getline(in, line)) {
    if (line.find(want) == std::string::npos) continue;
    const std::string f = std::string("\"") + field + "\": ";
    const size_t p = line.find(f);
    if (p == std::string::npos) continue;
    found = std::atof(line.c_str() + p + f.size());   // the last matching line wins
  }
  return found;
}

void cache_store(const char* path, const std::string& key, const std::string& fields) {
  if (!path) return;
  std::ofstream out(path, std::ios::app);
  out << "{\"key\": \"" << key << "\", " << fields << "}\n";
}

template <typename F>
double time_ms(cudaStream_t s, int reps, F&& run, mpbp_status* st) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    *st = MPBP_ERR_CUDA;
    return 0.0;
  }
  *st = run();   // warm-up
  if (*st == MPBP_OK) cudaEventRecord(a, s);
  for (int r = 0; r < reps && *st == MPBP_OK; ++r) *st = run();
  float ms = 0.f;
  if (*st == MPBP_OK) {
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess)
      *st = MPBP_ERR_CUDA;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

extern "C" {

mpbp_status mpbp_autotune(mpbp_ctx* c, const float* rho, const float* u, const float* alpha,
                          double* loss, float* g_rho, float* g_u, const char* cache_path,
                          void* stream) {
  if (!c || !rho || !u || !alpha || !loss || !g_rho || !g_u)
    return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  if (!c->has_probe || !c->has_data) return fail(c, MPBP_ERR_NO_DATA, "probe or data not set");
  if (c->det) return fail(c, MPBP_ERR_UNSUPPORTED, "the autotuner's candidates include atomic schedules");
  std::ostringstream k;
  k << gpu_name(c->device) << "|single|m" << c->M << "|d" << c->D << "|n" << c->n1 << "x" << c->n2 << "|f"
    << c->nframes;
  const double cached = cache_lookup(cache_path, k.str(), "blocks_per_sm");
  if (cached >= 1.0) {
    const double prec = cache_lookup(cache_path, k.str(), "precision");
    if (prec >= 0.0 && (int)prec != c->precision) {
      const mpbp_status ps = mpbp_set_precision(c, (int32_t)prec);
      if (ps != MPBP_OK) return ps;
    }
    const double sched = cache_lookup(cache_path, k.str(), "fft_schedule");
    if (sched >= 0.0) c->fft_schedule = (int)sched;
    return mpbp_set_schedule(c, (int32_t)cached);
  }
  cudaStream_t s = S(stream);
  // candidates: the DFT arithmetic (frame sides 32, 64, 128: FP32 FFTs or the
  // split tensor-core DFTs, both within the same error bounds) x (M = 128,
  // FP32) the FFT schedule x resident blocks per SM
  std::vector<int> precs = {MPBP_PRECISION_FP32};
  if (c->M >= 32) precs.push_back(MPBP_PRECISION_TC_SPLIT16);
  int best = 1, best_sched = c->fft_schedule, best_prec = c->precision;
  double best_ms = 1e30;
  for (int prec : precs) {
    mpbp_status ps = mpbp_set_precision(c, prec);
    if (ps != MPBP_OK) return ps;
    const int nsched = (c->M == 128 && prec == MPBP_PRECISION_FP32) ? 2 : 1;
    for (int sc = 0; sc < nsched; ++sc) {
      if (nsched > 1) c->fft_schedule = sc;
      for (int b = 1; b <= c->fk.blocks_per_sm; ++b) {
        mpbp_set_schedule(c, b);
        mpbp_status st = MPBP_OK;
        const double ms = time_ms(s, 3, [&]() {
          return mpbp_loss_grad(c, rho, u, alpha, nullptr, 0, loss, g_rho, g_u, nullptr, stream);
        }, &st);
        if (st != MPBP_OK) return st;
        if (ms < best_ms) {
          best_ms = ms;
          best = b;
          best_sched = c->fft_schedule;
          best_prec = prec;
        }
      }
    }
  }
  mpbp_status ps = mpbp_set_precision(c, best_prec);
  if (ps != MPBP_OK) return ps;
  c->fft_schedule = best_sched;
  mpbp_set_schedule(c, best);
  std::ostringstream f;
  f << "\"blocks_per_sm\": " << best << ", \"fft_schedule\": " << best_sched << ", \"precision\": " << best_prec
    << ", \"ms\": " << best_ms;
  cache_store(cache_path, k.str(), f.str());
  return MPBP_OK;
}

mpbp_status mpbp_autotune_batched(int32_t n, mpbp_ctx* const* ctxs, const float* const* rho,
                                  const float* const* u, const float* const* alpha,
                                  double* const* loss, float* const* g_rho, float* const* g_u,
                                  const char* cache_path, void* stream) {
  if (n < 1 || !ctxs || !ctxs[0]) return MPBP_ERR_INVALID_ARG;
  mpbp_ctx* lead = ctxs[0];
  std::ostringstream k;
  k << gpu_name(lead->device) << "|batch";
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(lead, MPBP_ERR_INVALID_ARG, "null context");
    k << "|m" << ctxs[i]->M << "d" << ctxs[i]->D << "n" << ctxs[i]->n1 << "x" << ctxs[i]->n2 << "f"
      << ctxs[i]->nframes;
  }
  const double cm = cache_lookup(cache_path, k.str(), "mode");
  const double co = cache_lookup(cache_path, k.str(), "order");
  if (cm >= 0.0 && co >= 0.0) return mpbp_set_batch_schedule(lead, (int32_t)cm, (int32_t)co);
  cudaStream_t s = S(stream);
  int best_m = lead->batch_mode, best_o = lead->batch_order;
  double best_ms = 1e30;
  for (int mode = 0; mode <= 3; ++mode) {
    for (int order = 0; order <= 1; ++order) {
      mpbp_set_batch_schedule(lead, mode, order);
      mpbp_status st = MPBP_OK;
      const double ms = time_ms(s, 3, [&]() {
        return mpbp_loss_grad_batched(n, ctxs, rho, u, alpha, loss, g_rho, g_u, nullptr, stream);
      }, &st);
      if (st != MPBP_OK) return st;
      if (ms < best_ms) {
        best_ms = ms;
        best_m = mode;
        best_o = order;
      }
    }
  }
  mpbp_set_batch_schedule(lead, best_m, best_o);
  std::ostringstream f;
  f << "\"mode\": " << best_m << ", \"order\": " << best_o << ", \"ms\": " << best_ms;
  cache_store(cache_path, k.str(), f.str());
  return MPBP_OK;
}

mpbp_status mpbp_frames_timing(mpbp_ctx* c, int32_t enable) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  c->timing = enable != 0;
  return MPBP_OK;
}

mpbp_status mpbp_frames_timing_read(mpbp_ctx* c, double* total_ms, int32_t* count) {
  if (!c || !total_ms || !count) return fail(c, MPBP_ERR_INVALID_ARG, "null argument");
  double tot = 0.0;
  for (size_t i = 0; i < c->ev_used; ++i) {
    MPBP_CUDA(c, cudaEventSynchronize(c->ev_pool[i].second));
    float ms = 0.f;
    MPBP_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[i].first, c->ev_pool[i].second));
    tot += ms;
  }
  *total_ms = tot;
  *count = (int32_t)c->ev_used;
  c->ev_used = 0;
  return MPBP_OK;
}

mpbp_status mpbp_set_test_stall(mpbp_ctx* c, int32_t on) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  c->test_tx_extra = on ? 16u : 0u;
  c->version++;   // batched plans copy the tensor maps with the hook
  return MPBP_OK;
}

mpbp_status mpbp_sync_status(mpbp_ctx* c, void* stream) {
  if (!c) return MPBP_ERR_INVALID_ARG;
  MPBP_CUDA(c, cudaStreamSynchronize(S(stream)));
  int h = 0;
  MPBP_CUDA(c, cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) MPBP_CUDA(c, cudaMemset(c->err, 0, sizeof(int)));
  // a wait that ran out leaves the evaluation's results undefined (a
  // non-finite loss among them), so it is reported ahead of the loss check
  if (h & kErrBounds) return fail(c, MPBP_ERR_BOUNDS, "frame index out of range");
  if (h & kErrTimeout) return fail(c, MPBP_ERR_TIMEOUT, "a bounded wait on the GPU ran out");
  if (h & kErrNonfinite) return fail(c, MPBP_ERR_NONFINITE, "non-finite loss");
  return MPBP_OK;
}

}  // extern "C"
