// mpbp_unwrap.cu -- the projector Pi_U of Eq. 10 on the GPU: the phases
// Phi_m = phase_scale G_m . u, wrapped (Eq. 9's W), unwrapped by
// reliability-ordered path following (Herraez et al., Appl. Opt. 2002), and
// mapped back to u with the pseudo-inverse of G.
//
// Path-following unwrappers merge pixel groups along edges taken in order of
// decreasing reliability, i.e. they integrate the wrapped phase differences
// along the maximum spanning forest of the pixel grid (edge weight = the sum
// of its pixels' reliabilities, ties broken by the edge number so that the
// order is strict and the forest unique).  Here that forest is built in
// parallel by Boruvka rounds instead of a sorted sweep:
//   - every component takes its heaviest incident edge (64-bit atomicMax of
//     (weight bits, ~edge number)); a root whose choice is shared with the
//     component on the other side keeps its place if its index is the lower;
//   - each other root hooks under the component across its edge with the
//     multiple of 2 pi that brings the phase difference across the edge into
//     [-pi, pi) (its offset relative to its new parent);
//   - pointer jumping compresses the forest, adding offsets along the way,
//     until every pixel points at its root with its offset to it.
// The rounds repeat until no root hooks; each group is then shifted so that
// its lowest-numbered pixel keeps its wrapped value.  The D phase maps form
// one graph with D disconnected parts.
//
// All of it runs in one cooperative launch (every block resident), with grid
// barriers that are bounded in time: if one runs out, the block records
// kErrTimeout and leaves, and the rest run out at their next barrier.
#include <cmath>
#include <climits>

#include "unwrap_launch.h"

namespace mpbp {

namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr unsigned long long kBarrierNs = 100ull * 1000 * 1000;   // 0.1 s per barrier
constexpr int kUnwrapThreads = 256;

__device__ __forceinline__ float wrapf(float x) { return x - kTwoPi * floorf(x / kTwoPi + 0.5f); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Sense by generation: the last block to arrive resets the count and bumps
// the generation; the others wait (bounded) for the generation to change.
// Returns false (in every thread of the block) if this block's wait ran out.
// With a.test_stall block 0 leaves without arriving, so the others' waits
// run out.
__device__ bool grid_sync(UnwrapArgs& a) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* genp = a.bar_gen;
    const unsigned g = *genp;
    __threadfence();
    if (a.test_stall && blockIdx.x == 0) {
      atomicOr(a.err, kErrTimeout);
      ok = 0;
    } else if (atomicAdd(a.bar_count, 1u) == gridDim.x - 1) {
      *a.bar_count = 0u;
      __threadfence();
      atomicAdd(a.bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*genp == g) {
        __nanosleep(32);
        if (global_ns() - t0 > kBarrierNs) {
          atomicOr(a.err, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__device__ __forceinline__ bool in_mask(const UnwrapArgs& a, long long r) { return !a.mask || a.mask[r] != 0.0f; }

// reliability of node v: 1 / sqrt(H^2 + V^2 + D1^2 + D2^2) when all eight
// neighbours are in the grid and the mask, else 0
__device__ float reliability(const UnwrapArgs& a, long long v) {
  const long long m = v / a.npix, r = v - m * a.npix;
  const int i = (int)(r / a.n2), j = (int)(r - (long long)i * a.n2);
  if (i < 1 || j < 1 || i > a.n1 - 2 || j > a.n2 - 2) return 0.0f;
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj)
      if (!in_mask(a, r + (long long)di * a.n2 + dj)) return 0.0f;
  const float* w = a.wrapped + m * a.npix;
  auto P = [&](int ii, int jj) { return w[(long long)ii * a.n2 + jj]; };
  const float c = P(i, j);
  const float h = wrapf(P(i, j - 1) - c) - wrapf(c - P(i, j + 1));
  const float vv = wrapf(P(i - 1, j) - c) - wrapf(c - P(i + 1, j));
  const float d1 = wrapf(P(i - 1, j - 1) - c) - wrapf(c - P(i + 1, j + 1));
  const float d2 = wrapf(P(i - 1, j + 1) - c) - wrapf(c - P(i + 1, j - 1));
  const float dd = sqrtf(h * h + vv * vv + d1 * d1 + d2 * d2);
  return 1.0f / fmaxf(dd, 1e-30f);
}

// the other end of edge e = 2 v + dir (dir 0: right, 1: down), or -1
__device__ __forceinline__ long long edge_other(const UnwrapArgs& a, long long e) {
  const long long v = e >> 1;
  const long long r = v % a.npix;
  const int i = (int)(r / a.n2), j = (int)(r - (long long)i * a.n2);
  long long q;
  if (e & 1) {
    if (i + 1 >= a.n1) return -1;
    q = v + a.n2;
  } else {
    if (j + 1 >= a.n2) return -1;
    q = v + 1;
  }
  if (!in_mask(a, r) || !in_mask(a, q % a.npix)) return -1;
  return q;
}

__device__ __forceinline__ unsigned long long edge_key(float w, long long e) {
  return ((unsigned long long)__float_as_uint(w) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)e);
}

// Local contraction.  In every 16 x 16 tile of a map, Boruvka rounds over the
// tile in shared memory hook a component only when the heaviest edge incident
// to it -- edges that leave the tile included -- lies inside the tile.  By the
// cut property such an edge belongs to the maximum spanning forest, so the
// global rounds continue from a forest of the same tree, with about one
// component per tile left instead of one per pixel.  Writes parent and off
// (multiple of 2 pi relative to the tile-local root) of every node.
constexpr int kTile = 16;
static_assert(kTile * kTile == kUnwrapThreads, "one node per thread");

__device__ void local_contract(const UnwrapArgs& a) {
  __shared__ int lp[kUnwrapThreads], lo[kUnwrapThreads], gid[kUnwrapThreads];
  __shared__ float wv[kUnwrapThreads];
  __shared__ unsigned long long bk[kUnwrapThreads];
  const int t = threadIdx.x, ti = t / kTile, tj = t % kTile;
  const int n1 = a.n1, n2 = a.n2;
  const int tpr = (n2 + kTile - 1) / kTile, tpc = (n1 + kTile - 1) / kTile;
  const int tiles_per_map = tpr * tpc;
  const int ntiles = (int)(a.nodes / a.npix) * tiles_per_map;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int m = tile / tiles_per_map, rem = tile - m * tiles_per_map;
    const int i0 = rem / tpr * kTile, j0 = rem % tpr * kTile;
    const int i = i0 + ti, j = j0 + tj;
    const bool in = i < n1 && j < n2;
    const long long base = (long long)m * a.npix;
    const long long v = in ? base + (long long)i * n2 + j : -1;
    // the node's edges (keys never change): right and down ones, inside the
    // tile or leaving it; left and up ones only where they leave it
    unsigned long long kr = 0, kd = 0, kl = 0, ku = 0;
    if (in) {
      kr = a.ekey[2 * v];
      kd = a.ekey[2 * v + 1];
      if (tj == 0 && j > 0) kl = a.ekey[2 * (v - 1)];
      if (ti == 0 && i > 0) ku = a.ekey[2 * (v - n2) + 1];
    }
    const bool r_in = tj + 1 < kTile, d_in = ti + 1 < kTile;
    gid[t] = (int)v;
    lp[t] = t;
    lo[t] = 0;
    wv[t] = in ? a.wrapped[v] : 0.0f;
    for (int round = 0; round < 2 * kTile; ++round) {
      bk[t] = 0ull;
      __syncthreads();
      const int r = lp[t];
      if (kr) {
        const int rq = r_in ? lp[t + 1] : -1;
        if (rq != r) {
          atomicMax(&bk[r], kr);
          if (rq >= 0) atomicMax(&bk[rq], kr);
        }
      }
      if (kd) {
        const int rq = d_in ? lp[t + kTile] : -1;
        if (rq != r) {
          atomicMax(&bk[r], kd);
          if (rq >= 0) atomicMax(&bk[rq], kd);
        }
      }
      if (kl) atomicMax(&bk[r], kl);
      if (ku) atomicMax(&bk[r], ku);
      __syncthreads();
      // hooks of the roots whose heaviest edge stays inside the tile
      int hook_p = -1, hook_o = 0;
      if (in && r == t && bk[t] != 0ull) {
        const long long e = 0xFFFFFFFFll - (long long)(bk[t] & 0xFFFFFFFFull);
        const long long pg = (e >> 1) - base;   // the edge's first end, within the map
        const int pi = (int)(pg / n2), pj = (int)(pg - (long long)pi * n2);
        const int qi = pi + (int)(e & 1), qj = pj + (int)(1 - (e & 1));
        if (pi >= i0 && pj >= j0 && qi < i0 + kTile && qj < j0 + kTile) {
          const int pl = (pi - i0) * kTile + (pj - j0), ql = (qi - i0) * kTile + (qj - j0);
          const bool p_in_r = lp[pl] == t;
          const int lr = p_in_r ? pl : ql, ls = p_in_r ? ql : pl;
          const int sr = lp[ls];
          if (!(bk[sr] == bk[t] && gid[t] < gid[sr])) {   // the shared edge: sr hooks under t
            const float d = (wv[lr] + kTwoPi * (float)lo[lr]) - (wv[ls] + kTwoPi * (float)lo[ls]);
            hook_p = sr;
            hook_o = -(int)floorf(d / kTwoPi + 0.5f);
          }
        }
      }
      if (!__syncthreads_or(hook_p >= 0)) break;
      if (hook_p >= 0) {
        lp[t] = hook_p;
        lo[t] = hook_o;
      }
      __syncthreads();
      // pointer jumping to the roots (a forest of 256 nodes: at most 9 passes)
      for (int jump = 0; jump < 2 * kTile; ++jump) {
        const int p = lp[t], pp = lp[p];
        const int no = lo[t] + (pp != p ? lo[p] : 0);
        __syncthreads();
        if (pp != p) {
          lp[t] = pp;
          lo[t] = no;
        }
        if (!__syncthreads_or(pp != p)) break;
      }
    }
    if (in) {
      a.parent[v] = gid[lp[t]];
      a.off[v] = lo[t];
    }
    __syncthreads();   // the next tile reuses the shared arrays
  }
}

__global__ void __launch_bounds__(kUnwrapThreads) unwrap_kernel(UnwrapArgs a) {
  const long long n = a.nodes;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int* par[2] = {a.parent, a.parent2};
  int* off[2] = {a.off, a.off2};
  int cur = 0;   // which buffer holds the forest

  for (long long v = tid; v < n; v += stride) {
    a.rel[v] = reliability(a, v);
    a.best[v] = 0ull;
    a.minnode[v] = INT_MAX;   // read only by the closing phase
  }
  if (!grid_sync(a)) return;
  // edge keys (0: no edge), computed once
  for (long long e = tid; e < 2 * n; e += stride) {
    const long long q = edge_other(a, e);
    a.ekey[e] = q < 0 ? 0ull : edge_key(a.rel[e >> 1] + a.rel[q], e);
  }
  if (!grid_sync(a)) return;
  local_contract(a);   // writes parent and off of every node
  if (!grid_sync(a)) return;

  int flag_it = 0;   // flags rotate over 3 slots (see next_flag)
  auto next_flag = [&]() {
    // the slot of the next use is cleared now; it was last read two uses ago
    if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[(flag_it + 1) % 3] = 0;
  };

  for (int round = 0; round < a.max_rounds; ++round) {
    int* P = par[cur];
    int* O = off[cur];
    // heaviest incident edge of every component (best[] is all zero here)
    for (long long e = tid; e < 2 * n; e += stride) {
      const unsigned long long key = a.ekey[e];
      if (!key) continue;
      const long long p = e >> 1, q = p + ((e & 1) ? a.n2 : 1);
      const int rp = P[p], rq = P[q];
      if (rp == rq) continue;
      atomicMax(&a.best[rp], key);
      atomicMax(&a.best[rq], key);
    }
    if (!grid_sync(a)) return;
    // hooks, decided from a consistent snapshot
    const int fs = flag_it % 3;
    for (long long r = tid; r < n; r += stride) {
      a.hook_parent[r] = -1;
      if (P[r] != (int)r || a.best[r] == 0ull) continue;
      const long long e = 0xFFFFFFFFll - (long long)(a.best[r] & 0xFFFFFFFFull);
      const long long p = e >> 1, q = p + ((e & 1) ? a.n2 : 1);
      const bool p_in_r = P[p] == (int)r;
      const long long pr = p_in_r ? p : q, ps = p_in_r ? q : p;
      const int s = P[ps];
      if (a.best[s] == a.best[r] && r < s) continue;   // the shared edge: s hooks under r
      const float d = (a.wrapped[pr] + kTwoPi * (float)O[pr]) - (a.wrapped[ps] + kTwoPi * (float)O[ps]);
      a.hook_parent[r] = s;
      a.hook_off[r] = -(int)floorf(d / kTwoPi + 0.5f);
      a.flags[fs] = 1;
    }
    next_flag();
    if (!grid_sync(a)) return;
    const bool any = *(volatile int*)&a.flags[fs] != 0;
    ++flag_it;
    if (!any) break;
    // pointer jumping until every node points at its root, four hops a pass
    // (the depth shrinks fourfold per pass; an acyclic forest of n nodes
    // needs at most log4(n) + 1 passes, the cap only guards against a forest
    // that is not), stopping after the pass that leaves every node under a
    // root.  The first pass reads the forest with the Boruvka round's hooks
    // applied (a hooked root's parent and offset from hook_parent/hook_off)
    // and clears best[]: every decision that read it is behind the barrier.
    for (int jump = 0;; ++jump) {
      if (jump > 64) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.err, kErrTimeout);
        break;
      }
      const bool first = jump == 0;
      const int* Pi = par[cur];
      const int* Oi = off[cur];
      int* Po = par[cur ^ 1];
      int* Oo = off[cur ^ 1];
      auto up = [&](int x, int& o) {   // parent of x, o = x's offset to it
        if (first) {
          const int h = a.hook_parent[x];
          if (h >= 0) {
            o = a.hook_off[x];
            return h;
          }
        }
        o = Oi[x];
        return Pi[x];
      };
      const int fj = flag_it % 3;
      for (long long v = tid; v < n; v += stride) {
        int o1, o2, o3, o4;
        const int p1 = up((int)v, o1);
        const int p2 = up(p1, o2);
        const int p3 = up(p2, o3);
        const int p4 = up(p3, o4);
        int ov = o1;
        if (p2 != p1) ov += o2;
        if (p3 != p2) ov += o3;
        if (p4 != p3) ov += o4;
        Po[v] = p4;
        Oo[v] = ov;
        // another pass only if the new parent is not a root (a root stays one)
        int o5;
        if (up(p4, o5) != p4) a.flags[fj] = 1;
        if (first) a.best[v] = 0ull;
      }
      next_flag();
      if (!grid_sync(a)) return;
      const bool changed = *(volatile int*)&a.flags[fj] != 0;
      ++flag_it;
      cur ^= 1;
      if (!changed) break;
    }
  }

  // each group's lowest-numbered node keeps its wrapped value
  int* P = par[cur];
  int* O = off[cur];
  for (long long v = tid; v < n; v += stride) atomicMin(&a.minnode[P[v]], (int)v);
  if (!grid_sync(a)) return;
  for (long long v = tid; v < n; v += stride) {
    const int mn = a.minnode[P[v]];
    a.out[v] = a.wrapped[v] + kTwoPi * (float)(O[v] - O[mn]);
  }
}

// Phi_m = phase_scale G_m . u, wrapped
__global__ void project_phase_kernel(ProjectArgs a) {
  const long long n = a.npix * a.D;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / a.npix);
    const long long r = i - (long long)m * a.npix;
    float ph = 0.0f;
    for (int c = 0; c < a.C; ++c) ph = fmaf(a.g_scaled[m * kMaxComp + c], a.u[c * a.npix + r], ph);
    a.phi[i] = ph;
    a.wrapped[i] = wrapf(ph);
  }
}

// u += (Phi' - Phi) pinv^T / phase_scale inside the mask
__global__ void project_correct_kernel(ProjectArgs a) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < a.npix;
       r += (long long)gridDim.x * blockDim.x) {
    if (a.mask && a.mask[r] == 0.0f) continue;
    for (int c = 0; c < a.C; ++c) {
      float s = 0.0f;
      for (int m = 0; m < a.D; ++m) s = fmaf(a.pinv_scaled[c * kMaxPeaks + m], a.unwrapped[m * a.npix + r] - a.phi[m * a.npix + r], s);
      a.u[c * a.npix + r] += s;
    }
  }
}

}  // namespace

bool unwrap_prepare(int num_sms, int* grid) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unwrap_kernel, kUnwrapThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return false;
  *grid = num_sms * (per_sm < 2 ? per_sm : 2);   // 2 per SM: measured fastest (fewer barrier arrivals)
  return true;
}

cudaError_t unwrap_launch(const UnwrapArgs& a, int grid, cudaStream_t s) {
  void* args[] = {const_cast<UnwrapArgs*>(&a)};
  return cudaLaunchCooperativeKernel((const void*)unwrap_kernel, dim3(grid), dim3(kUnwrapThreads), args, 0, s);
}

cudaError_t project_phase_launch(const ProjectArgs& a, int num_sms, cudaStream_t s) {
  const long long n = a.npix * a.D;
  const long long b = (n + 255) / 256;
  project_phase_kernel<<<(int)(b < num_sms * 8 ? b : num_sms * 8), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t project_correct_launch(const ProjectArgs& a, int num_sms, cudaStream_t s) {
  const long long b = (a.npix + 255) / 256;
  project_correct_kernel<<<(int)(b < num_sms * 8 ? b : num_sms * 8), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mpbp
