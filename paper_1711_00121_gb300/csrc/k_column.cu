// Column mode (§7): SimRank columns without a dense S, in O(Kn + m) memory
// per column.
//  - Procedure 1 (PartialSim) on a block of B columns: forward steps
//    X_t = Q^T X_{t-1} over the out-lists (row b of Q^T X sums X[a,:] / d_a
//    over the out-neighbours a of b), stored for t = 0..K, then the Horner
//    steps Y <- X_{K-t} + C Q Y over the in-lists; result (1-C) Y.
//  - The change of a column through the stored updates (Eq. 70-71):
//    Y[a, c] += sum_k xi_k[a] eta_k[x_c] + eta_k[a] xi_k[x_c].
// Blocks are row-major [node][B]; the arithmetic is in the storage
// precision (FP32 or FP64).  With FP32 the change through the stored updates
// is one dense product per block: Y += A G with A = [xi_k, eta_k of every
// update] (n x 2 U (K+1), straight from the tile-blocked panels) and G the
// matching values at the block's columns.
#include <algorithm>

#include "sr_internal.h"

namespace sr {

namespace {

// X0[x_c][c] = 1 (the other entries are zero beforehand)
template <typename T>
__global__ void k_col_unit(const int32_t* __restrict__ cols, int B, T* __restrict__ X0) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < B) X0[(int64_t)cols[c] * B + c] = (T)1;
}

// Column 0 of X0 = the indicator of the distinct ids cols[0 .. g0), column c
// (1 <= c < B) = e_{cols[g0 + c - 1]}: Procedure 1 is linear in its start
// vector, so column 0 of its result is the sum of the g0 columns.
template <typename T>
__global__ void k_col_unit_grouped(const int32_t* __restrict__ cols, int g0, int B,
                                   T* __restrict__ X0) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < g0) X0[(int64_t)cols[q] * B] = (T)1;
  else if (q < g0 + B - 1) X0[(int64_t)cols[q] * B + (q - g0 + 1)] = (T)1;
}

// Y[a][c] = s * X[a][c] (X may be null: Y = 0), a < n_rows, c < B
template <typename T>
__global__ void k_col_fill(const T* __restrict__ X, double s, T* __restrict__ Y, int64_t count) {
  const T sv = (T)s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = X ? sv * X[e] : (T)0;
}

// One row chunk (at most CHUNK nonzeros of one adjacency row) per CTA and
// 128 columns per thread block column:
//   Y[row][c] += row_scale * sum_{e in chunk} w_e X[col_e][c]
// forward (Q^T, out-lists): w_e = 1 / d_{col_e}, row_scale = 1
// Horner  (Q,   in-lists):  w_e = 1,            row_scale = scale / d_row
// Long rows are split over many chunks, whose partial sums meet in atomics.
template <typename T, bool FORWARD>
__global__ void k_col_chunk(const RowChunk* __restrict__ chunks, const int32_t* __restrict__ col,
                            const float* __restrict__ ew, const int32_t* __restrict__ in_len,
                            const double* __restrict__ wsum, const T* __restrict__ X,
                            T* __restrict__ Y, int B, double scale) {
  // weighted Q (wsum != null): Q[a][b] = w(b -> a) / wsum[a]; ew = weight of each
  // adjacency entry (by pool position), null = 1
  const RowChunk ch = chunks[blockIdx.x];
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= B) return;
  T acc = T(0);
#pragma unroll 8
  for (int e = 0; e < ch.len; ++e) {
    const int a = col[ch.start + e];
    T x = X[(int64_t)a * B + c];
    if (ew) x *= (T)ew[ch.start + e];
    if (FORWARD) x /= wsum ? (T)wsum[a] : (T)in_len[a];
    acc += x;
  }
  const T rs = FORWARD ? T(1) : (T)scale / (wsum ? (T)wsum[ch.row] : (T)in_len[ch.row]);
  atomicAdd(&Y[(int64_t)ch.row * B + c], rs * acc);
}

// The same for FP32 blocks with B a multiple of 4: each thread takes four
// adjacent columns (one 16-byte gather per nonzero, one weight per nonzero
// for the four) and adds its partial sums with one vector atomic.
template <bool FORWARD>
__global__ void k_col_chunk4(const RowChunk* __restrict__ chunks, const int32_t* __restrict__ col,
                             const float* __restrict__ ew, const int32_t* __restrict__ in_len,
                             const double* __restrict__ wsum, const float* __restrict__ X,
                             float* __restrict__ Y, int B4, double scale) {
  const RowChunk ch = chunks[blockIdx.x];
  const int c4 = blockIdx.y * blockDim.x + threadIdx.x;
  if (c4 >= B4) return;
  const float4* __restrict__ X4 = reinterpret_cast<const float4*>(X);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
  for (int e = 0; e < ch.len; ++e) {
    const int a = col[ch.start + e];
    float w = ew ? ew[ch.start + e] : 1.f;
    if (FORWARD) w /= wsum ? (float)wsum[a] : (float)in_len[a];
    const float4 x = X4[(int64_t)a * B4 + c4];
    acc.x += w * x.x;
    acc.y += w * x.y;
    acc.z += w * x.z;
    acc.w += w * x.w;
  }
  const float rs =
      FORWARD ? 1.f : (float)scale / (wsum ? (float)wsum[ch.row] : (float)in_len[ch.row]);
  atomicAdd(reinterpret_cast<float4*>(Y) + (int64_t)ch.row * B4 + c4,
            make_float4(rs * acc.x, rs * acc.y, rs * acc.z, rs * acc.w));
}

int num_sms_for_narrow() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;
}

// Narrow blocks (B = BW <= 4 columns, e.g. the two old columns of one update):
// persistent warps, each taking four row chunks at a time (a chunk has at
// most 32 nonzeros): an 8-lane group per chunk, up to four nonzeros per lane
// gathered at once, the group's sums combined by shuffles within the group
// and added by its first lane.  The forward step reads X already divided by
// the in-degree (or in-weight) of each row (k_col_prescale).
template <typename T, bool FORWARD, int BW>
__global__ void __launch_bounds__(256) k_col_chunk_narrow(
    const RowChunk* __restrict__ chunks, int64_t count, const int32_t* __restrict__ col,
    const float* __restrict__ ew, const int32_t* __restrict__ in_len,
    const double* __restrict__ wsum, const T* __restrict__ X, T* __restrict__ Y, double scale) {
  const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // the loop bound depends on the warp only: every lane runs every shuffle
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 4 < count;
       w += nwarps) {
    const int64_t q = w * 4 + g;
    RowChunk ch;
    ch.row = 0;
    ch.len = 0;
    ch.start = 0;
    if (q < count) ch = chunks[q];
    int a[4];
    T wt[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = gl + 8 * u;
      a[u] = (e < ch.len) ? col[ch.start + e] : -1;
      wt[u] = (e < ch.len && ew) ? (T)ew[ch.start + e] : T(1);
    }
    T acc[BW];
#pragma unroll
    for (int c = 0; c < BW; ++c) acc[c] = T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (a[u] >= 0) {
#pragma unroll
        for (int c = 0; c < BW; ++c) acc[c] += wt[u] * X[(int64_t)a[u] * BW + c];
      }
#pragma unroll
    for (int c = 0; c < BW; ++c)
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, 8);
    if (gl == 0 && ch.len > 0) {
      const T rs = FORWARD ? T(1) : (T)scale / (wsum ? (T)wsum[ch.row] : (T)in_len[ch.row]);
#pragma unroll
      for (int c = 0; c < BW; ++c) atomicAdd(&Y[(int64_t)ch.row * BW + c], rs * acc[c]);
    }
  }
}

// Z[a][c] = X[a][c] / (in-degree of a, or its in-weight), a < n_rows, c < B
template <typename T>
__global__ void k_col_prescale(const T* __restrict__ X, const int32_t* __restrict__ in_len,
                               const double* __restrict__ wsum, int B, int64_t count,
                               T* __restrict__ Z) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / B;
    const T d = wsum ? (T)wsum[a] : (T)in_len[a];
    Z[e] = d != T(0) ? X[e] / d : T(0);
  }
}

// Y[a][c] += sum_k xi_k[a] eta_k[x_c] + eta_k[a] xi_k[x_c] for one stored
// update (tile-blocked panels P[T][which][k][128]); the panel values at the
// block's columns are staged in shared memory.
template <typename T, typename TP>
__global__ void k_col_apply(const TP* __restrict__ P, int K1, const int32_t* __restrict__ cols,
                            int B, int n_rows, T* __restrict__ Y) {
  extern __shared__ double sg[];  // [B][2*K1]: xi_k[x_c], eta_k[x_c]
  for (int e = threadIdx.x; e < B * K1; e += blockDim.x) {
    const int c = e / K1, k = e % K1;
    const int64_t x = cols[c];
    const int64_t base = ((x / PT) * 2) * (int64_t)K1 * PT + (int64_t)k * PT + (x % PT);
    sg[c * 2 * K1 + k] = (double)P[base];
    sg[c * 2 * K1 + K1 + k] = (double)P[base + (int64_t)K1 * PT];
  }
  __syncthreads();
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_rows) return;
  const int64_t ba = ((a / PT) * 2) * (int64_t)K1 * PT + (a % PT);
  for (int c = 0; c < B; ++c) {
    const double* g = sg + c * 2 * K1;
    double acc = 0.0;
    for (int k = 0; k < K1; ++k)
      acc += (double)P[ba + (int64_t)k * PT] * g[K1 + k] +
             (double)P[ba + (int64_t)(K1 + k) * PT] * g[k];
    Y[a * B + c] = (T)((double)Y[a * B + c] + acc);
  }
}

// G[u][r][c] for the FP32 product: r = which * K1 + k, the value of the
// OTHER vector of term k of update u at column x_c (eta_k[x_c] pairs with
// xi_k[a], xi_k[x_c] with eta_k[a]); c < B, zero for c in [B, Bp).
__global__ void k_col_gvals(const float* const* __restrict__ hist, int K1,
                            const int32_t* __restrict__ cols, int B, int Bp,
                            float* __restrict__ G) {
  const int u = blockIdx.y;
  const float* P = hist[u];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * K1 * Bp; e += gridDim.x * blockDim.x) {
    const int r = e / Bp, c = e % Bp;
    const int which = r / K1, k = r % K1;
    float v = 0.f;
    if (c < B) {
      const int64_t x = cols[c];
      v = P[(((x / PT) * 2 + (1 - which)) * (int64_t)K1 + k) * PT + (x % PT)];
    }
    G[((int64_t)u * 2 * K1 + r) * Bp + c] = v;
  }
}

// Y[a][c] += sum_u sum_r A_u[a][r] G[u][r][c] for the 128 rows of tile
// blockIdx.x and the 128 columns of group blockIdx.y (256 threads, an 8 x 8
// block of outputs each; the r-chunks of A and G are staged in shared memory:
// A_u's tile-blocked panel slice [r][128 rows] is already in that layout).
constexpr int CG_KC = 16;
__global__ void __launch_bounds__(256) k_col_corr(const float* const* __restrict__ hist, int U,
                                                  int K1, const float* __restrict__ G, int Bp,
                                                  int B, int n_rows, float* __restrict__ Y) {
  __shared__ __align__(16) float sA[CG_KC][PT];
  __shared__ __align__(16) float sG[CG_KC][PT];
  const int T = blockIdx.x, c0 = blockIdx.y * PT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  const int R = 2 * K1;
  for (int u = 0; u < U; ++u) {
    const float* Pt = hist[u] + (int64_t)T * 2 * K1 * PT;  // [r][128], r = which * K1 + k
    const float* Gu = G + (int64_t)u * R * Bp;
    for (int r0 = 0; r0 < R; r0 += CG_KC) {
      const int kc = min(CG_KC, R - r0);
      __syncthreads();
      for (int e = tid; e < kc * PT / 4; e += 256) {
        const int rr = e / (PT / 4), q = e % (PT / 4);
        reinterpret_cast<float4*>(sA[rr])[q] =
            reinterpret_cast<const float4*>(Pt + (int64_t)(r0 + rr) * PT)[q];
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        const int cc = c0 + 4 * q;
        if (cc < Bp) g = *reinterpret_cast<const float4*>(Gu + (int64_t)(r0 + rr) * Bp + cc);
        reinterpret_cast<float4*>(sG[rr])[q] = g;
      }
      __syncthreads();
      for (int rr = 0; rr < kc; ++rr) {
        float a[8], g[8];
        const float4 a0 = reinterpret_cast<const float4*>(sA[rr])[ty];
        const float4 a1 = reinterpret_cast<const float4*>(sA[rr])[16 + ty];
        const float4 g0 = reinterpret_cast<const float4*>(sG[rr])[tx];
        const float4 g1 = reinterpret_cast<const float4*>(sG[rr])[16 + tx];
        a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
        a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
        g[0] = g0.x; g[1] = g0.y; g[2] = g0.z; g[3] = g0.w;
        g[4] = g1.x; g[5] = g1.y; g[6] = g1.z; g[7] = g1.w;
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], g[c], acc[r][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t row = (int64_t)T * PT + ((r < 4) ? ty * 4 + r : 64 + ty * 4 + (r - 4));
    if (row >= n_rows) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = c0 + ((c < 4) ? tx * 4 + c : 64 + tx * 4 + (c - 4));
      if (col < B) Y[row * B + col] += acc[r][c];
    }
  }
}

// scal[0] = x_i[i], scal[1] = x_j[j], scal[2] = (1/d_j) sum_{b in I(j)} x_i[b]
// (columns i and j of S as FP64 vectors, old graph)
__global__ void k_col_scalars(DevAdj in, const double* __restrict__ si, const double* __restrict__ sj,
                              int i, int j, double* __restrict__ scal) {
  __shared__ double red[32];
  const int64_t st = in.start[j];
  const int len = in.len[j];
  double acc = 0.0;
  for (int e = threadIdx.x; e < len; e += blockDim.x) acc += si[in.col[st + e]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) w += red[q];
    scal[0] = si[i];
    scal[1] = sj[j];
    scal[2] = len > 0 ? w / (double)len : 0.0;
  }
}

// out[c * n + a] = Y[a][c] (column-major output, optional FP32)
template <typename T, typename TO>
__global__ void k_col_out(const T* __restrict__ Y, int B, int n, TO* __restrict__ out) {
  const int c = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) out[(int64_t)c * n + a] = (TO)Y[(int64_t)a * B + c];
}

// column c of a row-major [n][B] block into a contiguous FP64 vector
template <typename T>
__global__ void k_col_extract(const T* __restrict__ Y, int B, int c, int n, double* __restrict__ v) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) v[a] = (double)Y[(int64_t)a * B + c];
}

}  // namespace

template <typename T>
static void partial_sim_block_t(const ChunkList& fwd, const ChunkList& hor, const int32_t* out_col,
                                const int32_t* in_col, const WeightView& wv, const int32_t* in_len,
                                const int32_t* cols, int B, int n_rows, int K, double C, T* xs, T* y0,
                                T* y1, T* result, cudaStream_t st, int group0) {
  const int64_t blk = (int64_t)n_rows * B;
  const int fill_blocks = 4096;
  k_col_fill<T><<<fill_blocks, 256, 0, st>>>(nullptr, 0.0, xs, blk);
  if (group0 > 1)
    k_col_unit_grouped<T><<<(group0 + B + 126) / 128, 128, 0, st>>>(cols, group0, B, xs);
  else
    k_col_unit<T><<<(B + 127) / 128, 128, 0, st>>>(cols, B, xs);
  const int ygroups = (B + 127) / 128;
  const int tpb = B >= 128 ? 128 : (B + 31) / 32 * 32;
  // FP32 blocks of a multiple of 4 columns: four columns per thread
  const bool vec4 = sizeof(T) == 4 && B % 4 == 0;
  const int B4 = B / 4;
  const int tpb4 = B4 >= 256 ? 256 : (B4 + 31) / 32 * 32;
  const int ygroups4 = (B4 + tpb4 - 1) / tpb4;
  // narrow blocks: one warp per chunk; the forward input divided once per row
  const bool narrow = B <= 4;
  auto narrow_step = [&](const ChunkList& L, const int32_t* adj, const float* w, bool forward,
                         const T* X, T* Y, double scale) {
    // persistent: at most 8 CTAs of 8 warps per SM, four chunks per warp at a time
    const int64_t want = (L.count + 31) / 32;
    const unsigned grid = (unsigned)std::min<int64_t>(want, (int64_t)num_sms_for_narrow() * 8);
#define SR_NARROW(BW)                                                                          \
  do {                                                                                         \
    if (forward)                                                                               \
      k_col_chunk_narrow<T, true, BW><<<grid, 256, 0, st>>>(L.chunks, L.count, adj, w, in_len,  \
                                                            wv.wsum, X, Y, scale);             \
    else                                                                                       \
      k_col_chunk_narrow<T, false, BW><<<grid, 256, 0, st>>>(L.chunks, L.count, adj, w, in_len, \
                                                             wv.wsum, X, Y, scale);            \
  } while (0)
    switch (B) {
      case 1: SR_NARROW(1); break;
      case 2: SR_NARROW(2); break;
      case 3: SR_NARROW(3); break;
      default: SR_NARROW(4); break;
    }
#undef SR_NARROW
  };
  auto chunk_step = [&](const ChunkList& L, const int32_t* adj, const float* w, bool forward,
                        const T* X, T* Y, double scale) {
    if (L.count <= 0) return;
    if (narrow) {
      if (forward) {
        // y0 is free until the Horner steps: it holds X divided by the row degrees
        k_col_prescale<T><<<fill_blocks, 256, 0, st>>>(X, in_len, wv.wsum, B, blk, y0);
        narrow_step(L, adj, w, true, y0, Y, scale);
      } else {
        narrow_step(L, adj, w, false, X, Y, scale);
      }
    } else if (vec4) {
      if (forward)
        k_col_chunk4<true><<<dim3((unsigned)L.count, ygroups4), tpb4, 0, st>>>(
            L.chunks, adj, w, in_len, wv.wsum, (const float*)X, (float*)Y, B4, scale);
      else
        k_col_chunk4<false><<<dim3((unsigned)L.count, ygroups4), tpb4, 0, st>>>(
            L.chunks, adj, w, in_len, wv.wsum, (const float*)X, (float*)Y, B4, scale);
    } else if (forward) {
      k_col_chunk<T, true><<<dim3((unsigned)L.count, ygroups), tpb, 0, st>>>(
          L.chunks, adj, w, in_len, wv.wsum, X, Y, B, scale);
    } else {
      k_col_chunk<T, false><<<dim3((unsigned)L.count, ygroups), tpb, 0, st>>>(
          L.chunks, adj, w, in_len, wv.wsum, X, Y, B, scale);
    }
  };
  for (int t = 1; t <= K; ++t) {
    T* dst = xs + (int64_t)t * blk;
    k_col_fill<T><<<fill_blocks, 256, 0, st>>>(nullptr, 0.0, dst, blk);
    chunk_step(fwd, out_col, wv.out_w, true, xs + (int64_t)(t - 1) * blk, dst, 1.0);
  }
  // Horner: y = x_K; y <- x_{K-t} + C Q y; result (1-C) y (the last step folds the scale)
  const T* y = xs + (int64_t)K * blk;
  T* bufs[2] = {y0, y1};
  if (K == 0) {
    k_col_fill<T><<<fill_blocks, 256, 0, st>>>(xs, 1.0 - C, result, blk);
    return;
  }
  for (int t = 1; t <= K; ++t) {
    T* dst = (t == K) ? result : bufs[t & 1];
    const double s = (t == K) ? 1.0 - C : 1.0;
    k_col_fill<T><<<fill_blocks, 256, 0, st>>>(xs + (int64_t)(K - t) * blk, s, dst, blk);
    chunk_step(hor, in_col, wv.in_w, false, y, dst, s * C);
    y = dst;
  }
}

void launch_partial_sim_block(const ChunkList& fwd, const ChunkList& hor, const int32_t* out_col,
                              const int32_t* in_col, const int32_t* in_len, const int32_t* cols,
                              int B, int n_rows, int K, double C, int prec, void* xs, void* y0,
                              void* y1, void* result, cudaStream_t st, const WeightView& wv,
                              int group0) {
  if (prec == 64)
    partial_sim_block_t<double>(fwd, hor, out_col, in_col, wv, in_len, cols, B, n_rows, K, C,
                                (double*)xs, (double*)y0, (double*)y1, (double*)result, st, group0);
  else
    partial_sim_block_t<float>(fwd, hor, out_col, in_col, wv, in_len, cols, B, n_rows, K, C,
                               (float*)xs, (float*)y0, (float*)y1, (float*)result, st, group0);
}

// Y = Q^T X (FP64 blocks [n_rows][B])
void launch_col_forward64(const ChunkList& fwd, const int32_t* out_col, const WeightView& wv,
                          const int32_t* in_len, const double* X, double* Y, int B, int n_rows,
                          cudaStream_t st) {
  const int64_t blk = (int64_t)n_rows * B;
  k_col_fill<double><<<4096, 256, 0, st>>>(nullptr, 0.0, Y, blk);
  const int tpb = B >= 128 ? 128 : (B + 31) / 32 * 32;
  if (fwd.count > 0)
    k_col_chunk<double, true><<<dim3((unsigned)fwd.count, (B + 127) / 128), tpb, 0, st>>>(
        fwd.chunks, out_col, wv.out_w, in_len, wv.wsum, X, Y, B, 1.0);
}

// Yn = add_scale * Xadd + scale * Q Y (FP64 blocks [n_rows][B])
void launch_col_horner64(const ChunkList& hor, const int32_t* in_col, const WeightView& wv,
                         const int32_t* in_len, const double* Xadd, double add_scale,
                         const double* Y, double* Yn, int B, int n_rows, double scale,
                         cudaStream_t st) {
  const int64_t blk = (int64_t)n_rows * B;
  k_col_fill<double><<<4096, 256, 0, st>>>(Xadd, add_scale, Yn, blk);
  const int tpb = B >= 128 ? 128 : (B + 31) / 32 * 32;
  if (hor.count > 0)
    k_col_chunk<double, false><<<dim3((unsigned)hor.count, (B + 127) / 128), tpb, 0, st>>>(
        hor.chunks, in_col, wv.in_w, in_len, wv.wsum, Y, Yn, B, scale);
}

void launch_col_apply(const void* P, int p_prec, int K1, const int32_t* cols, int B, int n_rows,
                      int prec, void* Y, cudaStream_t st) {
  const size_t smem = (size_t)B * 2 * K1 * sizeof(double);
  const int threads = 128;
  const int blocks = (n_rows + threads - 1) / threads;
#define SR_COL_APPLY(T, TP)                                                                  \
  do {                                                                                       \
    cudaFuncSetAttribute(k_col_apply<T, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                         (int)smem);                                                         \
    k_col_apply<T, TP><<<blocks, threads, smem, st>>>((const TP*)P, K1, cols, B, n_rows, (T*)Y); \
  } while (0)
  if (prec == 64 && p_prec == 64)
    SR_COL_APPLY(double, double);
  else if (prec == 64)
    SR_COL_APPLY(double, float);
  else if (p_prec == 64)
    SR_COL_APPLY(float, double);
  else
    SR_COL_APPLY(float, float);
#undef SR_COL_APPLY
}

void launch_col_corr(const float* const* hist, int U, int K1, const int32_t* cols, int B,
                     int n_rows, float* G, float* Y, cudaStream_t st) {
  if (U <= 0 || B <= 0) return;
  const int Bp = (B + 3) / 4 * 4;
  k_col_gvals<<<dim3((2 * K1 * Bp + 255) / 256, U), 256, 0, st>>>(hist, K1, cols, B, Bp, G);
  k_col_corr<<<dim3(n_rows / PT, (B + PT - 1) / PT), 256, 0, st>>>(hist, U, K1, G, Bp, B, n_rows,
                                                                   Y);
}

void launch_col_scalars(const DevAdj& in, const double* si, const double* sj, int i, int j,
                        double* scal, cudaStream_t st) {
  k_col_scalars<<<1, 256, 0, st>>>(in, si, sj, i, j, scal);
}

void launch_col_out(const void* Y, int prec, int B, int n, void* out, int out_fp64,
                    cudaStream_t st) {
  dim3 grid((n + 255) / 256, B);
  if (prec == 64) {
    if (out_fp64)
      k_col_out<double, double><<<grid, 256, 0, st>>>((const double*)Y, B, n, (double*)out);
    else
      k_col_out<double, float><<<grid, 256, 0, st>>>((const double*)Y, B, n, (float*)out);
  } else {
    if (out_fp64)
      k_col_out<float, double><<<grid, 256, 0, st>>>((const float*)Y, B, n, (double*)out);
    else
      k_col_out<float, float><<<grid, 256, 0, st>>>((const float*)Y, B, n, (float*)out);
  }
}

void launch_col_extract(const void* Y, int prec, int B, int c, int n, double* v, cudaStream_t st) {
  if (prec == 64)
    k_col_extract<double><<<(n + 255) / 256, 256, 0, st>>>((const double*)Y, B, c, n, v);
  else
    k_col_extract<float><<<(n + 255) / 256, 256, 0, st>>>((const float*)Y, B, c, n, v);
}

}  // namespace sr
