// Graph-side kernels of one rank-one update: old-S row gathers, gamma
// assembly (Thm 3, Thm 9, Table 2), CSR patching (Thm 1), the xi/eta
// recurrence on the new graph (Eq. 16a) with fused affected-area masks
// (Thm 4), and the affected tile-pair list.
#include "sr_internal.h"

namespace sr {

namespace {

template <typename T>
__device__ __forceinline__ double ld_s(const T* p) { return (double)__ldg(p); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void k_gather_rows(const T* __restrict__ S, int64_t ld, const int32_t* __restrict__ I,
                              int delta, int j, int n_pad, double* __restrict__ sI,
                              double* __restrict__ sJ, double* __restrict__ scal) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n_pad) {
    double acc = 0.0;
    for (int t = 0; t < delta; ++t) acc += ld_s(S + (int64_t)I[t] * ld + a);
    sI[a] = acc;
    sJ[a] = ld_s(S + (int64_t)j * ld + a);
  }
  if (blockIdx.x == 0) {
    __shared__ double red[32];
    double acc = 0.0;
    const int64_t tot = (int64_t)delta * delta;
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      const int t = (int)(e / delta), u = (int)(e % delta);
      acc += ld_s(S + (int64_t)I[t] * ld + I[u]);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0) {
        scal[0] = v;
        scal[1] = ld_s(S + (int64_t)j * ld + j);
      }
    }
  }
}

// One CTA per 128-row tile; 16 warps x 8 rows.  Every CTA first recomputes
// w_j = (1/delta) [Q]_{j,*} S_{*,I} (needed by lambda, Eq. 29b) from row j
// of the old CSR, then each warp forms w_a = (1/delta) [Q]_{a,*} S_{*,I} for
// its rows and the gamma entry of the branch (op, d_j).
__global__ void __launch_bounds__(512) k_gamma(DevAdj in, const double* __restrict__ sI,
                                               const double* __restrict__ sJ,
                                               const double* __restrict__ scal, int j, int delta,
                                               int op, int d_j, double C, int K1,
                                               double* __restrict__ P64, float* __restrict__ P32,
                                               uint64_t* __restrict__ mXi,
                                               uint64_t* __restrict__ mEta) {
  __shared__ double red[16];
  __shared__ int any_eta;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) any_eta = 0;
  // w_j over row j of the old graph
  double acc = 0.0;
  const int64_t js = in.start[j];
  const int jl = in.len[j];
  for (int e = threadIdx.x; e < jl; e += blockDim.x) acc += sI[in.col[js + e]];
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  double wj = 0.0;
  for (int w = 0; w < 16; ++w) wj += red[w];
  wj = (jl > 0) ? wj / ((double)delta * (double)jl) : 0.0;
  const double S_II = scal[0], S_jj = scal[1];
  const double dl = (double)delta;
  const double lam = S_II / (dl * dl) + S_jj / C - 2.0 * wj - 1.0 / C + 1.0;

  const int T = blockIdx.x;
  bool nz = false;
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    const int a = T * PT + r;
    const int64_t st = in.start[a];
    const int len = in.len[a];
    double s = 0.0;
    for (int e = lane; e < len; e += 32) s += sI[in.col[st + e]];
    s = warp_sum(s);
    const double w = (len > 0) ? s / (dl * (double)len) : 0.0;
    const double ej = (a == j) ? 1.0 : 0.0;
    double g;
    if (op > 0) {
      if (d_j == 0) {
        g = w + S_II / (2.0 * dl * dl) * ej;
      } else {
        const double dd = (double)d_j + dl;
        g = (dl / dd) * (w - sJ[a] / C + (lam * dl / (2.0 * dd) + 1.0 / C - 1.0) * ej);
      }
    } else {
      if (d_j == delta) {
        g = -w + S_II / (2.0 * dl * dl) * ej;
      } else {
        const double dd = (double)d_j - dl;
        g = (dl / dd) * (sJ[a] / C - w + (lam * dl / (2.0 * dd) - 1.0 / C + 1.0) * ej);
      }
    }
    if (lane == 0) {
      const int64_t bx = ((int64_t)T * 2 + 0) * K1 * PT + r;  // xi_0 entry
      const int64_t be = ((int64_t)T * 2 + 1) * K1 * PT + r;  // eta_0 entry
      const double x0 = (a == j) ? C : 0.0;
      P64[bx] = x0;
      P64[be] = g;
      if (P32) {
        P32[bx] = (float)x0;
        P32[be] = (float)g;
      }
      nz = nz || (g != 0.0);
    }
  }
  if (lane == 0 && nz) any_eta = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
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
// on the patched (new) CSR; one CTA per 128-row tile.
__global__ void __launch_bounds__(512) k_chain_step(DevAdj in, int k, double C, int K1,
                                                    double* __restrict__ P64,
                                                    float* __restrict__ P32,
                                                    uint64_t* __restrict__ mXi,
                                                    uint64_t* __restrict__ mEta) {
  __shared__ int any_x, any_e;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    any_x = 0;
    any_e = 0;
  }
  __syncthreads();
  const int T = blockIdx.x;
  bool nzx = false, nze = false;
  for (int rr = 0; rr < 8; ++rr) {
    const int r = warp * 8 + rr;
    const int a = T * PT + r;
    const int64_t st = in.start[a];
    const int len = in.len[a];
    double sx = 0.0, se = 0.0;
    for (int e = lane; e < len; e += 32) {
      const int b = in.col[st + e];
      const int64_t base = ((int64_t)(b / PT) * 2) * K1 * PT + (int64_t)k * PT + (b % PT);
      sx += P64[base];
      se += P64[base + (int64_t)K1 * PT];
    }
    sx = warp_sum(sx);
    se = warp_sum(se);
    if (lane == 0) {
      const double inv = (len > 0) ? 1.0 / (double)len : 0.0;
      const double x = C * sx * inv;
      const double y = se * inv;
      const int64_t bx = ((int64_t)T * 2 + 0) * K1 * PT + (int64_t)(k + 1) * PT + r;
      const int64_t be = bx + (int64_t)K1 * PT;
      P64[bx] = x;
      P64[be] = y;
      if (P32) {
        P32[bx] = (float)x;
        P32[be] = (float)y;
      }
      nzx = nzx || (x != 0.0);
      nze = nze || (y != 0.0);
    }
  }
  if (lane == 0) {
    if (nzx) any_x = 1;
    if (nze) any_e = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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
                        int n_pad, double* sI, double* sJ, double* scal, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (n_pad + threads - 1) / threads;
  if (s_prec == 64)
    k_gather_rows<double><<<blocks, threads, 0, st>>>((const double*)S, ld, I, delta, j, n_pad, sI,
                                                      sJ, scal);
  else
    k_gather_rows<float><<<blocks, threads, 0, st>>>((const float*)S, ld, I, delta, j, n_pad, sI,
                                                     sJ, scal);
}

void launch_gamma(const DevAdj& in, const double* sI, const double* sJ, const double* scal, int j,
                  int delta, int op, int d_j, double C, int nT, int K1, double* P64, float* P32,
                  uint64_t* mXi, uint64_t* mEta, cudaStream_t st) {
  k_gamma<<<nT, 512, 0, st>>>(in, sI, sJ, scal, j, delta, op, d_j, C, K1, P64, P32, mXi, mEta);
}

void launch_patch(const PatchOp* ops, int64_t begin, int64_t end, DevAdj in, DevAdj out,
                  cudaStream_t st) {
  if (end > begin) k_patch<<<1, 256, 0, st>>>(ops, begin, end, in, out);
}

void launch_chain_step(const DevAdj& in, int k, double C, int nT, int K1, double* P64, float* P32,
                       uint64_t* mXi, uint64_t* mEta, cudaStream_t st) {
  k_chain_step<<<nT, 512, 0, st>>>(in, k, C, K1, P64, P32, mXi, mEta);
}

void launch_tile_list(const uint64_t* mXi, const uint64_t* mEta, int nT, int aff, uint32_t* tiles,
                      int* ntiles, cudaStream_t st) {
  const int threads = 128;
  dim3 grid((nT + threads - 1) / threads, nT);
  k_tile_list<<<grid, threads, 0, st>>>(mXi, mEta, nT, aff, tiles, ntiles);
}

}  // namespace sr
