// Gradient of a pair loss L = sum_p (S_K[a_p, b_p] - t_p)^2 with respect to
// the edge weights, for the K-truncated series S_K = (1-C) sum_{k<=K} C^k Q^k Q^kT
// (Eq. 17) of the weighted Q[a][b] = w_ba / sum_x w_xa.  With
// g_p = 2 (S_K[a_p, b_p] - t_p), psi^x = sum_{p: a_p = x} g_p e_{b_p} + sum_{p: b_p = x} g_p e_{a_p},
// F^x_l = (Q^T)^l e_x and y^x_l = C^{l+1} (Q^T)^{l+1} psi^x + Q y^x_{l+1} (y^x_K = 0):
//   dL/dQ[u][v] = (1-C) sum_x sum_{l<K} F^x_l[u] y^x_l[v],
// needed only at the edges (an SDDMM), then the chain rule through the row
// normalisation.  The series vectors are recomputed per block of endpoints.
#include "sr_internal.h"

namespace sr {

namespace {

// one CTA per chunk of an in-list row u; warp w handles entries w, w + 8, ...
__global__ void k_adj_sddmm(const RowChunk* __restrict__ chunks, const int32_t* __restrict__ col,
                            const double* __restrict__ F, const double* __restrict__ Y, int B,
                            double scale, double* __restrict__ G) {
  const RowChunk ch = chunks[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* fu = F + (int64_t)ch.row * B;
  for (int e = warp; e < ch.len; e += (int)(blockDim.x >> 5)) {
    const int v = col[ch.start + e];
    const double* yv = Y + (int64_t)v * B;
    double acc = 0.0;
    for (int x = lane; x < B; x += 32) acc += fu[x] * yv[x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) G[ch.start + e] += scale * acc;
  }
}

__global__ void k_adj_scatter(const int32_t* __restrict__ node, const int32_t* __restrict__ c,
                              const double* __restrict__ coef, int64_t count, int B,
                              double* __restrict__ X) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) atomicAdd(&X[(int64_t)node[t] * B + c[t]], coef[t]);
}

__global__ void k_adj_pairs(const double* __restrict__ Y, int B, const int32_t* __restrict__ row,
                            const int32_t* __restrict__ c, int64_t count, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) out[t] = Y[(int64_t)row[t] * B + c[t]];
}

// one warp per in-list row a
__global__ void k_adj_weights(DevAdj in, WeightView wv, int n_rows, const double* __restrict__ G,
                              double* __restrict__ dW) {
  const int lane = threadIdx.x & 31;
  const int a = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (a >= n_rows) return;
  const int64_t st = in.start[a];
  const int len = in.len[a];
  if (len == 0) return;
  const double W = wv.wsum ? wv.wsum[a] : (double)len;
  double s = 0.0;
  for (int e = lane; e < len; e += 32) {
    const double w = wv.in_w ? (double)wv.in_w[st + e] : 1.0;
    s += G[st + e] * w / W;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  for (int e = lane; e < len; e += 32) dW[st + e] = (G[st + e] - s) / W;
}

}  // namespace

void launch_adj_sddmm(const ChunkList& hor, const int32_t* in_col, const double* F, const double* Y,
                      int B, double scale, double* G, cudaStream_t st) {
  if (hor.count > 0) k_adj_sddmm<<<(unsigned)hor.count, 256, 0, st>>>(hor.chunks, in_col, F, Y, B, scale, G);
}

void launch_adj_scatter(const int32_t* node, const int32_t* c, const double* coef, int64_t count,
                        int B, double* X, cudaStream_t st) {
  if (count > 0) k_adj_scatter<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(node, c, coef, count, B, X);
}

void launch_adj_pairs(const double* Y, int B, const int32_t* row, const int32_t* c, int64_t count,
                      double* out, cudaStream_t st) {
  if (count > 0) k_adj_pairs<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(Y, B, row, c, count, out);
}

void launch_adj_weights(const DevAdj& in, const WeightView& wv, int n_rows, const double* G,
                        double* dW, cudaStream_t st) {
  const int64_t threads = (int64_t)n_rows * 32;
  k_adj_weights<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(in, wv, n_rows, G, dW);
}

}  // namespace sr
