// Graph-side kernels of one rank-one update: old-S row gathers, gamma
// assembly (Thm 3, Thm 9, Table 2), CSR patching (Thm 1), the xi/eta
// recurrence on the new graph (Eq. 16a) with fused affected-area masks
// (Thm 4), and the affected tile-pair list.
#include <algorithm>

#include "sr_internal.h"

namespace sr {

namespace {

template <typename T>
__device__ __forceinline__ double ld_s(const T* p) { return (double)__ldg(p); }
// S[r, c] as a double, reading the mirror of a lower tile when upper != 0
template <typename T>
__device__ __forceinline__ double ld_sym(const T* S, int64_t ld, int64_t r, int64_t c, int upper) {
  return (upper && (r / PT) > (c / PT)) ? (double)__ldg(S + c * ld + r)
                                        : (double)__ldg(S + r * ld + c);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block 0 also forms w_j = (1/delta) [Q]_{j,*} S_{*,I} on the old graph
// (= (1/(delta d_j)) sum_{b in I(j)} sum_t S[I[t], b]) for lambda (Eq. 29b).
template <typename T>
__global__ void k_gather_rows(const T* __restrict__ S, int64_t ld, const int32_t* __restrict__ I,
                              int delta, int j, int n_pad, DevAdj in, double* __restrict__ sI,
                              double* __restrict__ sJ, double* __restrict__ scal, int upper) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n_pad) {
    double acc = 0.0;
    for (int t = 0; t < delta; ++t) acc += ld_sym(S, ld, I[t], a, upper);
    sI[a] = acc;
    sJ[a] = ld_sym(S, ld, j, a, upper);
  }
  if (blockIdx.x == 0) {
    __shared__ double red[2][32];
    double acc = 0.0;
    for (int t = 0; t < delta; ++t)
      for (int u = threadIdx.x; u < delta; u += blockDim.x) acc += ld_sym(S, ld, I[t], I[u], upper);
    const int64_t js = in.start[j];
    const int jl = in.len[j];
    double wj = 0.0;
    for (int t = 0; t < delta; ++t) {
#pragma unroll 8
      for (int u = threadIdx.x; u < jl; u += blockDim.x)
        wj += ld_sym(S, ld, I[t], in.col[js + u], upper);
    }
    acc = warp_sum(acc);
    wj = warp_sum(wj);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = acc;
      red[1][threadIdx.x >> 5] = wj;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = (threadIdx.x < (blockDim.x >> 5)) ? red[0][threadIdx.x] : 0.0;
      double w = (threadIdx.x < (blockDim.x >> 5)) ? red[1][threadIdx.x] : 0.0;
      v = warp_sum(v);
      w = warp_sum(w);
      if (threadIdx.x == 0) {
        scal[0] = v;
        scal[1] = ld_sym(S, ld, j, j, upper);
        scal[2] = (jl > 0) ? w / ((double)delta * (double)jl) : 0.0;
      }
    }
  }
}

// Rows of the current S when G earlier updates are still pending (their
// panels not yet added to S): for x in {I_0..I_{delta-1}} and j,
//   S_cur[x, a] = S[x, a] + sum_{u < np} sum_k xi^u_k[x] eta^u_k[a] + eta^u_k[x] xi^u_k[a]
// with the pending panels Pp stored tile-blocked [T][which][G*K1][128] (FP32,
// term = u * K1 + k).  sI[a] = sum_t S_cur[I_t, a], sJ[a] = S_cur[j, a].
template <typename T>
__global__ void __launch_bounds__(256) k_gather_rows_pending(
    const T* __restrict__ S, int64_t ld, const int32_t* __restrict__ I, int delta, int j, int n_pad,
    const float* __restrict__ Pp, int GK1, int nterms, double* __restrict__ sI,
    double* __restrict__ sJ, int upper) {
  // coefficients: [2 vectors (I-sum, j)][2 (xi, eta)][nterms]
  extern __shared__ double coef[];
  __shared__ double red[8][32][2];
  for (int q = threadIdx.x; q < nterms; q += blockDim.x) {
    double cx = 0.0, ce = 0.0;
    for (int t = 0; t < delta; ++t) {
      const int64_t x = I[t];
      const int64_t base = ((x / PT) * 2) * (int64_t)GK1 * PT + (int64_t)q * PT + (x % PT);
      cx += (double)Pp[base];
      ce += (double)Pp[base + (int64_t)GK1 * PT];
    }
    const int64_t base = ((int64_t)(j / PT) * 2) * GK1 * PT + (int64_t)q * PT + (j % PT);
    coef[0 * nterms + q] = cx;
    coef[1 * nterms + q] = ce;
    coef[2 * nterms + q] = (double)Pp[base];
    coef[3 * nterms + q] = (double)Pp[base + (int64_t)GK1 * PT];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a = blockIdx.x * 32 + lane;  // 32 consecutive rows share one tile
  double accI = 0.0, accJ = 0.0;
  if (a < n_pad) {
    const int64_t ba = ((int64_t)(a / PT) * 2) * GK1 * PT + (a % PT);
    for (int q = warp; q < nterms; q += 8) {
      const double xa = (double)Pp[ba + (int64_t)q * PT];
      const double ea = (double)Pp[ba + (int64_t)(GK1 + q) * PT];
      accI += coef[0 * nterms + q] * ea + coef[1 * nterms + q] * xa;
      accJ += coef[2 * nterms + q] * ea + coef[3 * nterms + q] * xa;
    }
    if (warp == 0) {
      for (int t = 0; t < delta; ++t) accI += ld_sym(S, ld, I[t], a, upper);
      accJ += ld_sym(S, ld, j, a, upper);
    }
  }
  red[warp][lane][0] = accI;
  red[warp][lane][1] = accJ;
  __syncthreads();
  if (warp == 0 && a < n_pad) {
    double vI = 0.0, vJ = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      vI += red[w][lane][0];
      vJ += red[w][lane][1];
    }
    sI[a] = vI;
    sJ[a] = vJ;
  }
}

// scal[0] = S_II = sum_t sI[I_t], scal[1] = S_jj = sJ[j],
// scal[2] = w_j = (1/(delta d_j)) sum_{b in I(j)} sI[b] on the graph `in` (old)
__global__ void k_scalars_from_rows(DevAdj in, const double* __restrict__ sI,
                                    const double* __restrict__ sJ, const int32_t* __restrict__ I,
                                    int delta, int j, double* __restrict__ scal) {
  __shared__ double red[2][32];
  const int64_t st = in.start[j];
  const int len = in.len[j];
  double w = 0.0, sii = 0.0;
  for (int e = threadIdx.x; e < len; e += blockDim.x) w += sI[in.col[st + e]];
  for (int t = threadIdx.x; t < delta; t += blockDim.x) sii += sI[I[t]];
  w = warp_sum(w);
  sii = warp_sum(sii);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = w;
    red[1][threadIdx.x >> 5] = sii;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ws = 0.0, ss = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      ws += red[0][q];
      ss += red[1][q];
    }
    scal[0] = ss;
    scal[1] = sJ[j];
    scal[2] = len > 0 ? ws / ((double)delta * (double)len) : 0.0;
  }
}

// tile-level "any term non-zero" masks of the pending updates
__global__ void k_or_any(const uint64_t* __restrict__ mXi, const uint64_t* __restrict__ mEta,
                         int nT, uint64_t* __restrict__ pXi, uint64_t* __restrict__ pEta) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T < nT) {
    if (mXi[T]) pXi[T] = 1ull;
    if (mEta[T]) pEta[T] = 1ull;
  }
}

// Per-tile sparse gather used by the gamma and chain kernels.  One CTA owns
// the 128 rows of tile T; the nonzeros of those rows are flattened (row
// offsets by an exclusive scan in shared memory) and split into contiguous
// runs, one per thread, so rows of any length - including hub rows with
// thousands of in-neighbours - are spread over the whole CTA.  Each thread
// sums its run in registers and flushes one partial sum per row it touches
// into shared accumulators.  NV = number of gathered vectors (1 or 2).
constexpr int GT = 512;  // threads of a gather CTA
constexpr int CHAIN_ITEM = 16 * GT;  // nonzeros per work item of k_chain_step_items

struct TileRows {
  int64_t start[PT];
  int len[PT];
  int off[PT + 1];
};

__device__ __forceinline__ void tile_rows_load(const DevAdj& in, int T, TileRows& tr) {
  const int tid = threadIdx.x;
  if (tid < PT) {
    tr.start[tid] = in.start[T * PT + tid];
    tr.len[tid] = in.len[T * PT + tid];
  }
  __syncthreads();
  if (tid < 32) {
    // exclusive scan of 128 lengths by one warp (4 per lane)
    int v[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = tr.len[tid * 4 + q];
      sum += v[q];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    int run = incl - sum;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      tr.off[tid * 4 + q] = run;
      run += v[q];
    }
    if (tid == 31) tr.off[PT] = incl;
  }
  __syncthreads();
}

// Adds val into acc[key] once per run of equal keys across the lanes of a
// warp (keys are non-decreasing with the lane index; key < 0 = nothing):
// a segmented suffix sum by shuffles, then one atomic per segment head.
template <int NV>
__device__ __forceinline__ void warp_segment_flush(int key, double (&val)[NV], double (*acc)[PT]) {
  const int lane = threadIdx.x & 31;
  // only as many rounds as the longest run of equal keys needs (GB300 issues
  // each FP64 addition at 1/64 of the FP32 rate, predicated lanes included)
  const unsigned same = __match_any_sync(0xffffffffu, key);
  const int span = (int)__reduce_max_sync(0xffffffffu, key >= 0 ? (unsigned)__popc(same) : 1u);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= span) break;
    const int k2 = __shfl_down_sync(0xffffffffu, key, o);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double x = __shfl_down_sync(0xffffffffu, val[v], o);
      if (lane + o < 32 && k2 == key) val[v] += x;
    }
  }
  const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kprev != key)) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (val[v] != 0.0) atomicAdd(&acc[v][key], val[v]);
  }
}

// acc[v][r] = sum over nonzeros b of row r of X_v[b], X_v given by gather(v, b).
// Thread t owns the contiguous run of flattened nonzeros [t*per, (t+1)*per):
// rows that start and end inside its run are stored directly (no other
// thread touches them); its first and last row may be shared with the
// neighbouring runs and are combined by warp_segment_flush.
// With g1 >= 0 only the flattened nonzeros [g0, g1) of the tile are gathered
// (one work item of a tile split over several CTAs): acc then holds this
// item's partial sums of the rows it touches.
template <int NV, typename G>
__device__ __forceinline__ void tile_gather(const DevAdj& in, const TileRows& tr, G gather,
                                            double (*acc)[PT], int g0 = 0, int g1 = -1) {
  const int tid = threadIdx.x;
  for (int r = tid; r < PT; r += GT)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v][r] = 0.0;
  __syncthreads();
  const int total = g1 >= 0 ? g1 : tr.off[PT];
  const int per = (total - g0 + GT - 1) / GT;
  const int e0 = g0 + tid * per;
  const int e1 = min(total, e0 + per);
  int r_first = -1, r_last = -1;
  double pf[NV], pl[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) pf[v] = pl[v] = 0.0;
  if (e0 < e1) {
    int lo = 0, hi = PT;  // find r with off[r] <= e0 < off[r+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tr.off[mid] <= e0) lo = mid; else hi = mid;
    }
    int r = lo;
    r_first = r;
    double part[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v] = 0.0;
    // batches of 8 nonzeros: all column loads, then all gathers, are independent
    constexpr int B = 8;
    for (int e = e0; e < e1; e += B) {
      int rr[B], bb[B];
      int rc = r;
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int ee = e + q;
        if (ee < e1) {
          while (ee >= tr.off[rc + 1]) ++rc;
          rr[q] = rc;
          bb[q] = in.col[tr.start[rc] + (ee - tr.off[rc])];
        } else {
          rr[q] = -1;
          bb[q] = 0;
        }
      }
      double xv[NV][B];
#pragma unroll
      for (int q = 0; q < B; ++q)
#pragma unroll
        for (int v = 0; v < NV; ++v) xv[v][q] = (rr[q] >= 0) ? gather(v, bb[q]) : 0.0;
#pragma unroll
      for (int q = 0; q < B; ++q) {
        if (rr[q] < 0) break;
        if (rr[q] != r) {
          if (r == r_first) {
#pragma unroll
            for (int v = 0; v < NV; ++v) pf[v] = part[v];
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v][r] = part[v];  // row wholly inside this run
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) part[v] = 0.0;
          r = rr[q];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) part[v] += xv[v][q];
      }
    }
    if (r == r_first) {
#pragma unroll
      for (int v = 0; v < NV; ++v) pf[v] = part[v];
    } else {
      r_last = r;
#pragma unroll
      for (int v = 0; v < NV; ++v) pl[v] = part[v];
    }
  }
  warp_segment_flush<NV>(r_first, pf, acc);
  warp_segment_flush<NV>(r_last, pl, acc);
  __syncthreads();
}

// gamma of Thm 3 (insert), Thm 9 (delete) and Table 2 (sink blocks) for the
// rows of tile T, on the OLD graph: w = (1/delta) Q S_{*,I}, lambda from
// Eq. 29b with w_j (row j recomputed by every CTA), then the gamma branch.
__global__ void __launch_bounds__(GT) k_gamma(DevAdj in, const double* __restrict__ sI,
                                              const double* __restrict__ sJ,
                                              const double* __restrict__ scal, int j, int delta,
                                              int op, int d_j, double C, int K1,
                                              double* __restrict__ P64, float* __restrict__ P32,
                                              uint64_t* __restrict__ mXi,
                                              uint64_t* __restrict__ mEta) {
  __shared__ TileRows tr;
  __shared__ double acc[1][PT];
  __shared__ int any_eta;
  const int tid = threadIdx.x;
  const int T = blockIdx.x;
  if (tid == 0) any_eta = 0;
  tile_rows_load(in, T, tr);  // contains __syncthreads
  const double dl = (double)delta;
  const double S_II = scal[0], S_jj = scal[1], wj = scal[2];
  const double lam = S_II / (dl * dl) + S_jj / C - 2.0 * wj - 1.0 / C + 1.0;
  tile_gather<1>(in, tr, [&](int, int b) { return sI[b]; }, acc);
  if (tid < PT) {
    const int r = tid;
    const int ai = T * PT + r;
    const int len = tr.len[r];
    const double w = (len > 0) ? acc[0][r] / (dl * (double)len) : 0.0;
    const double ej = (ai == j) ? 1.0 : 0.0;
    double g;
    if (op > 0) {
      if (d_j == 0) {
        g = w + S_II / (2.0 * dl * dl) * ej;
      } else {
        const double dd = (double)d_j + dl;
        g = (dl / dd) * (w - sJ[ai] / C + (lam * dl / (2.0 * dd) + 1.0 / C - 1.0) * ej);
      }
    } else {
      if (d_j == delta) {
        g = -w + S_II / (2.0 * dl * dl) * ej;
      } else {
        const double dd = (double)d_j - dl;
        g = (dl / dd) * (sJ[ai] / C - w + (lam * dl / (2.0 * dd) - 1.0 / C + 1.0) * ej);
      }
    }
    const int64_t bx = ((int64_t)T * 2 + 0) * K1 * PT + r;  // xi_0 entry
    const int64_t be = ((int64_t)T * 2 + 1) * K1 * PT + r;  // eta_0 entry
    const double x0 = (ai == j) ? C : 0.0;
    P64[bx] = x0;
    P64[be] = g;
    if (P32) {
      P32[bx] = (float)x0;
      P32[be] = (float)g;
    }
    if (g != 0.0) any_eta = 1;
  }
  __syncthreads();
  if (tid == 0) {
    mXi[T] = (T == j / PT) ? 1ull : 0ull;
    mEta[T] = any_eta ? 1ull : 0ull;
  }
}

__global__ void k_patch(const PatchOp* __restrict__ ops, int64_t begin, int64_t end, DevAdj in,
                        DevAdj out) {
  for (int64_t o = begin; o < end; ++o) {
    const PatchOp op = ops[o];
    if (op.kind == PK_IN_COPY || op.kind == PK_OUT_COPY) {
      int32_t* c = (op.kind == PK_IN_COPY) ? in.col : out.col;
      for (int e = threadIdx.x; e < op.v; e += blockDim.x) c[op.a + e] = c[op.b + e];
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      switch (op.kind) {
        case PK_IN_COL: in.col[op.a] = op.v; break;
        case PK_OUT_COL: out.col[op.a] = op.v; break;
        case PK_IN_LEN: in.len[op.a] = op.v; break;
        case PK_OUT_LEN: out.len[op.a] = op.v; break;
        case PK_IN_START: in.start[op.a] = op.b; break;
        case PK_OUT_START: out.start[op.a] = op.b; break;
        default: break;
      }
    }
    __syncthreads();
  }
}

// xi_{k+1}[a] = C * mean_{b in I(a)} xi_k[b], eta_{k+1}[a] = mean_{b in I(a)} eta_k[b]
// on the patched (new) CSR; one CTA per 128-row tile (Eq. 16a).
__global__ void __launch_bounds__(GT) k_chain_step(DevAdj in, int k, double C, int K1,
                                                   double* __restrict__ P64,
                                                   float* __restrict__ P32,
                                                   uint64_t* __restrict__ mXi,
                                                   uint64_t* __restrict__ mEta) {
  __shared__ TileRows tr;
  __shared__ double acc[2][PT];
  __shared__ int any_x, any_e;
  const int tid = threadIdx.x;
  const int T = blockIdx.x;
  if (tid == 0) {
    any_x = 0;
    any_e = 0;
  }
  tile_rows_load(in, T, tr);
  const double* __restrict__ src = P64;
  tile_gather<2>(in, tr,
                 [&](int v, int b) {
                   return src[(((int64_t)(b / PT) * 2 + v) * K1 + k) * PT + (b % PT)];
                 },
                 acc);
  if (tid < PT) {
    const int r = tid;
    const int len = tr.len[r];
    const double inv = (len > 0) ? 1.0 / (double)len : 0.0;
    const double x = C * acc[0][r] * inv;
    const double y = acc[1][r] * inv;
    const int64_t bx = ((int64_t)T * 2 + 0) * K1 * PT + (int64_t)(k + 1) * PT + r;
    const int64_t be = bx + (int64_t)K1 * PT;
    P64[bx] = x;
    P64[be] = y;
    if (P32) {
      P32[bx] = (float)x;
      P32[be] = (float)y;
    }
    if (x != 0.0) any_x = 1;
    if (y != 0.0) any_e = 1;
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned long long bit = 1ull << ((k + 1) & 63);
    if (any_x) atomicOr((unsigned long long*)&mXi[T], bit);
    if (any_e) atomicOr((unsigned long long*)&mEta[T], bit);
  }
}

// The same step with the tiles cut into work items of at most CHAIN_ITEM
// nonzeros (item q: tile item_tile[q], nonzeros [item_sub[q] * CHAIN_ITEM,
// ...) of its flattened in-lists): a hub tile no longer holds one CTA for the
// whole step.  The items of a tile with several add their partial row sums
// into gacc[T]; the item that arrives last (counter tile_count[T]) finishes
// the tile and clears gacc[T] and its counter for the next step.
__global__ void __launch_bounds__(GT) k_chain_step_items(
    DevAdj in, const int* __restrict__ item_tile, const int* __restrict__ item_sub,
    const int* __restrict__ tile_items, int k, double C, int K1, double* __restrict__ P64,
    float* __restrict__ P32, uint64_t* __restrict__ mXi, uint64_t* __restrict__ mEta,
    double* __restrict__ gacc, unsigned int* __restrict__ tile_count) {
  __shared__ TileRows tr;
  __shared__ double acc[2][PT];
  __shared__ int any_x, any_e, last;
  const int tid = threadIdx.x;
  const int q = blockIdx.x;
  const int T = item_tile[q];
  const int parts = tile_items[T];
  if (tid == 0) {
    any_x = 0;
    any_e = 0;
    last = 1;
  }
  tile_rows_load(in, T, tr);
  const int g0 = item_sub[q] * CHAIN_ITEM;
  const int g1 = min(tr.off[PT], g0 + CHAIN_ITEM);
  const double* __restrict__ src = P64;
  tile_gather<2>(in, tr,
                 [&](int v, int b) {
                   return src[(((int64_t)(b / PT) * 2 + v) * K1 + k) * PT + (b % PT)];
                 },
                 acc, g0, g1);
  double* ga = gacc + (int64_t)T * 2 * PT;
  if (parts > 1) {
    if (tid < PT) {
      if (acc[0][tid] != 0.0) atomicAdd(&ga[tid], acc[0][tid]);
      if (acc[1][tid] != 0.0) atomicAdd(&ga[PT + tid], acc[1][tid]);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&tile_count[T], 1u) == (unsigned int)(parts - 1)) ? 1 : 0;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid < PT) {
      acc[0][tid] = __ldcg(&ga[tid]);
      acc[1][tid] = __ldcg(&ga[PT + tid]);
      ga[tid] = 0.0;
      ga[PT + tid] = 0.0;
    }
    if (tid == 0) tile_count[T] = 0u;
    __syncthreads();
  }
  if (tid < PT) {
    const int r = tid;
    const int len = tr.len[r];
    const double inv = (len > 0) ? 1.0 / (double)len : 0.0;
    const double x = C * acc[0][r] * inv;
    const double y = acc[1][r] * inv;
    const int64_t bx = ((int64_t)T * 2 + 0) * K1 * PT + (int64_t)(k + 1) * PT + r;
    const int64_t be = bx + (int64_t)K1 * PT;
    P64[bx] = x;
    P64[be] = y;
    if (P32) {
      P32[bx] = (float)x;
      P32[be] = (float)y;
    }
    if (x != 0.0) any_x = 1;
    if (y != 0.0) any_e = 1;
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned long long bit = 1ull << ((k + 1) & 63);
    if (any_x) atomicOr((unsigned long long*)&mXi[T], bit);
    if (any_e) atomicOr((unsigned long long*)&mEta[T], bit);
  }
}

__global__ void k_tile_list(const uint64_t* __restrict__ mXi, const uint64_t* __restrict__ mEta,
                            int nT, int aff, uint32_t* __restrict__ tiles,
                            int* __restrict__ ntiles) {
  const int I = blockIdx.y;
  const int J = I + blockIdx.x * blockDim.x + threadIdx.x;
  bool act = false;
  if (J < nT) {
    act = aff ? (((mXi[I] & mEta[J]) | (mEta[I] & mXi[J])) != 0ull) : true;
  }
  const unsigned mask = __ballot_sync(0xffffffffu, act);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(ntiles, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (act) tiles[base + __popc(mask & ((1u << lane) - 1u))] = ((uint32_t)I << 16) | (uint32_t)J;
}

}  // namespace

void launch_gather_rows(const void* S, int s_prec, int64_t ld, const int32_t* I, int delta, int j,
                        int n_pad, const DevAdj& in, double* sI, double* sJ, double* scal,
                        cudaStream_t st, int upper) {
  const int threads = 256;
  const int blocks = (n_pad + threads - 1) / threads;
  if (s_prec == 64)
    k_gather_rows<double><<<blocks, threads, 0, st>>>((const double*)S, ld, I, delta, j, n_pad, in,
                                                      sI, sJ, scal, upper);
  else
    k_gather_rows<float><<<blocks, threads, 0, st>>>((const float*)S, ld, I, delta, j, n_pad, in,
                                                     sI, sJ, scal, upper);
}

void launch_gather_rows_pending(const void* S, int s_prec, int64_t ld, const int32_t* I, int delta,
                                int j, int n_pad, const float* Pp, int GK1, int nterms, double* sI,
                                double* sJ, cudaStream_t st, int upper) {
  const int threads = 256;
  const int blocks = (n_pad + 31) / 32;
  const size_t smem = (size_t)4 * nterms * sizeof(double);
  if (s_prec == 64) {
    cudaFuncSetAttribute(k_gather_rows_pending<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_gather_rows_pending<double><<<blocks, threads, smem, st>>>((const double*)S, ld, I, delta, j,
                                                                 n_pad, Pp, GK1, nterms, sI, sJ,
                                                                 upper);
  } else {
    cudaFuncSetAttribute(k_gather_rows_pending<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_gather_rows_pending<float><<<blocks, threads, smem, st>>>((const float*)S, ld, I, delta, j,
                                                                n_pad, Pp, GK1, nterms, sI, sJ,
                                                                 upper);
  }
}

void launch_scalars_from_rows(const DevAdj& in, const double* sI, const double* sJ, const int32_t* I,
                              int delta, int j, double* scal, cudaStream_t st) {
  k_scalars_from_rows<<<1, 256, 0, st>>>(in, sI, sJ, I, delta, j, scal);
}

void launch_or_any(const uint64_t* mXi, const uint64_t* mEta, int nT, uint64_t* pXi, uint64_t* pEta,
                   cudaStream_t st) {
  k_or_any<<<(nT + 127) / 128, 128, 0, st>>>(mXi, mEta, nT, pXi, pEta);
}

void launch_gamma(const DevAdj& in, const double* sI, const double* sJ, const double* scal, int j,
                  int delta, int op, int d_j, double C, int nT, int K1, double* P64, float* P32,
                  uint64_t* mXi, uint64_t* mEta, cudaStream_t st) {
  k_gamma<<<nT, GT, 0, st>>>(in, sI, sJ, scal, j, delta, op, d_j, C, K1, P64, P32, mXi, mEta);
}

void launch_patch(const PatchOp* ops, int64_t begin, int64_t end, DevAdj in, DevAdj out,
                  cudaStream_t st) {
  if (end > begin) k_patch<<<1, 256, 0, st>>>(ops, begin, end, in, out);
}

void launch_chain_step(const DevAdj& in, int k, double C, int nT, int K1, double* P64, float* P32,
                       uint64_t* mXi, uint64_t* mEta, cudaStream_t st) {
  k_chain_step<<<nT, GT, 0, st>>>(in, k, C, K1, P64, P32, mXi, mEta);
}

void launch_chain_step_items(const DevAdj& in, const int* item_tile, const int* item_sub,
                             const int* tile_items, int n_items, int k, double C, int K1,
                             double* P64, float* P32, uint64_t* mXi, uint64_t* mEta, double* gacc,
                             unsigned int* tile_count, cudaStream_t st) {
  k_chain_step_items<<<n_items, GT, 0, st>>>(in, item_tile, item_sub, tile_items, k, C, K1, P64,
                                             P32, mXi, mEta, gacc, tile_count);
}

int chain_item_size() { return CHAIN_ITEM; }

void launch_tile_list(const uint64_t* mXi, const uint64_t* mEta, int nT, int aff, uint32_t* tiles,
                      int* ntiles, cudaStream_t st) {
  const int threads = 128;
  dim3 grid((nT + threads - 1) / threads, nT);
  k_tile_list<<<grid, threads, 0, st>>>(mXi, mEta, nT, aff, tiles, ntiles);
}

}  // namespace sr
