// One-shot batch update (rank-2r Sylvester form).  For a whole batch,
// dQ = U V^T with U = [e_{j_1} .. e_{j_r}] (the r distinct sinks) and
// V_t = Q_new[j_t,:]^T - Q[j_t,:]^T.  The proof of Thm 2 (Eq. 23-28) carries
// over column by column: Delta S = sum_k C^{k+1} Q_new^k T Q_new^kT with
// T = U W^T + W U^T, W = Q S V + U Lambda / 2, Lambda = V^T S V.  With
// V_t = a_t Q[j_t,:]^T + b_t e_{D_t} (e_{D_t} = inserted minus deleted sources
// of sink j_t) and Eq. 33 (Q S Q[j,:]^T = (S_{*,j} - (1-C) e_j) / C), W and
// Lambda need only the S rows of the batch's endpoints.  These kernels build
// W and Lambda, the panels Xi_k = C^{k+1} Q_new^k U, H_k = Q_new^k W, and the
// operand layouts of the two S-update kernels.
#include <cuda_fp16.h>

#include "sr_internal.h"

namespace sr {

namespace {

// Zc[t][a] = sum_{e in [off[t], off[t+1])} sign[e] * S[src[e], a]
template <typename T>
__global__ void k_signed_rows(const T* __restrict__ S, int64_t ld, const int32_t* __restrict__ src,
                              const int8_t* __restrict__ sign, const int64_t* __restrict__ off,
                              int n_pad, double* __restrict__ Zc, int upper) {
  const int t = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_pad) return;
  double acc = 0.0;
  for (int64_t e = off[t]; e < off[t + 1]; ++e) {
    const double v = (double)s_at(S, ld, src[e], a, upper != 0);
    acc += sign[e] > 0 ? v : -v;
  }
  Zc[(int64_t)t * n_pad + a] = acc;
}

// B[c * ldb + r] = A[r * lda + c] for r < rows, c < cols (32 x 32 tiles)
__global__ void k_transpose_rect(const double* __restrict__ A, int64_t lda, double* __restrict__ B,
                                 int64_t ldb, int rows, int cols) {
  __shared__ double tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int r = r0 + q, c = c0 + threadIdx.x;
    tile[q][threadIdx.x] = (r < rows && c < cols) ? A[(int64_t)r * lda + c] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += 8) {
    const int c = c0 + q, r = r0 + threadIdx.x;
    if (c < cols && r < rows) B[(int64_t)c * ldb + r] = tile[threadIdx.x][q];
  }
}

// Lambda[t][u] = V_t^T S V_u with V_t = a_t Q[j_t,:]^T + b_t e_{D_t}:
//   a_t a_u (S[j_t, j_u] - (1-C) [t == u]) / C      (Eq. 33-34)
// + a_t b_u Y[j_t][u] + b_t a_u Y[j_u][t]           (Y = Q Z, row-major)
// + b_t b_u sum_{e in D_t} sign_e Z[src_e][u]       (Z row-major)
template <typename T>
__global__ void k_lambda(const T* __restrict__ S, int64_t ld, const int32_t* __restrict__ sinks,
                         const double* __restrict__ av, const double* __restrict__ bv,
                         const double* __restrict__ Y, const double* __restrict__ Z, int64_t ldz,
                         const int32_t* __restrict__ src, const int8_t* __restrict__ sign,
                         const int64_t* __restrict__ off, int r, double C,
                         double* __restrict__ Lam, int upper) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = blockIdx.y;
  if (u >= r) return;
  const int jt = sinks[t], ju = sinks[u];
  const double at = av[t], au = av[u], bt = bv[t], bu = bv[u];
  double v = at * au * ((double)s_at(S, ld, jt, ju, upper != 0) - (t == u ? 1.0 - C : 0.0)) / C;
  v += at * bu * Y[(int64_t)jt * ldz + u] + bt * au * Y[(int64_t)ju * ldz + t];
  double d = 0.0;
  for (int64_t e = off[t]; e < off[t + 1]; ++e) {
    const double z = Z[(int64_t)src[e] * ldz + u];
    d += sign[e] > 0 ? z : -z;
  }
  v += bt * bu * d;
  Lam[(int64_t)t * r + u] = v;
}

// Wc[t][a] = a_t (S[j_t, a] - (1-C) [a == j_t]) / C + b_t Yc[t][a]
template <typename T>
__global__ void k_w_assemble(const T* __restrict__ S, int64_t ld, const int32_t* __restrict__ sinks,
                             const double* __restrict__ av, const double* __restrict__ bv,
                             const double* __restrict__ Yc, int n_pad, double C,
                             double* __restrict__ Wc, int upper) {
  const int t = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_pad) return;
  const int jt = sinks[t];
  const double s = (double)s_at(S, ld, jt, a, upper != 0) - (a == jt ? 1.0 - C : 0.0);
  Wc[(int64_t)t * n_pad + a] = av[t] * s / C + bv[t] * Yc[(int64_t)t * n_pad + a];
}

// Wc[t][j_u] += Lambda[u][t] / 2  (the U Lambda / 2 term of W; sinks are distinct)
__global__ void k_w_lambda(const int32_t* __restrict__ sinks, const double* __restrict__ Lam, int r,
                           int n_pad, double* __restrict__ Wc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int u = blockIdx.y;
  if (t >= r) return;
  Wc[(int64_t)t * n_pad + sinks[u]] += 0.5 * Lam[(int64_t)u * r + t];
}

// X0 (row-major, ldx): X0[j_t][t] = C for the xi half (columns [0, r))
__global__ void k_xi0(const int32_t* __restrict__ sinks, int r, double C, double* __restrict__ X0,
                      int64_t ldx) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < r) X0[(int64_t)sinks[t] * ldx + t] = C;
}

// Panels for the CUDA-core S update from X_k (row-major FP64, xi half at
// column 0, eta half at column rh): term = slot * r + t of the tile-blocked
// layout P[T][which][term][128] with `terms` terms; ORs AFF bits (term % 64).
template <typename TP>
__global__ void k_pack_ffma(const double* __restrict__ X, int64_t ldx, int rh, int r, int slot,
                            int terms, int nT, TP* __restrict__ Pn, uint64_t* __restrict__ mXi,
                            uint64_t* __restrict__ mEta) {
  // block: 128 rows of tile T, threads over (row, t) with row fastest
  const int T = blockIdx.x;
  const int t = blockIdx.y * 2 + (threadIdx.x >> 7);
  const int row = threadIdx.x & 127;
  __shared__ int anyx[2], anye[2];
  if (threadIdx.x < 2) {
    anyx[threadIdx.x] = 0;
    anye[threadIdx.x] = 0;
  }
  __syncthreads();
  if (t < r) {
    const int64_t a = (int64_t)T * PT + row;
    const double x = X[a * ldx + t];
    const double e = X[a * ldx + rh + t];
    const int term = slot * r + t;
    Pn[(((int64_t)T * 2 + 0) * terms + term) * PT + row] = (TP)x;
    Pn[(((int64_t)T * 2 + 1) * terms + term) * PT + row] = (TP)e;
    if (x != 0.0) anyx[threadIdx.x >> 7] = 1;
    if (e != 0.0) anye[threadIdx.x >> 7] = 1;
  }
  __syncthreads();
  if (threadIdx.x < 2 && blockIdx.y * 2 + threadIdx.x < r) {
    const int term = slot * r + blockIdx.y * 2 + threadIdx.x;
    const unsigned long long bit = 1ull << (term & 63);
    if (anyx[threadIdx.x]) atomicOr((unsigned long long*)&mXi[T], bit);
    if (anye[threadIdx.x]) atomicOr((unsigned long long*)&mEta[T], bit);
  }
}

// Round to TF32 (10 explicit mantissa bits), round-to-nearest-even on the
// dropped 13 bits; the result is an FP32 value whose low 13 bits are zero.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // inf / nan unchanged
  const uint32_t lsb = (u >> 13) & 1u;
  u += 0x0fffu + lsb;
  u &= 0xffffe000u;
  return __uint_as_float(u);
}

// Operands of the tensor-core S update from X_k: row-major A_hi, A_lo with
// kd columns; xi terms at column slot * r + t, eta terms at rg + slot * r + t.
// A value x is split as hi = tf32(x), lo = tf32(x - hi).
__global__ void k_pack_tc(const double* __restrict__ X, int64_t ldx, int rh, int r, int slot,
                          int rg, int n_rows, float* __restrict__ Ahi, float* __restrict__ Alo,
                          int64_t kd) {
  const int64_t a = blockIdx.x;
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  if (t >= r || a >= n_rows) return;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float x = (float)X[a * ldx + h * rh + t];
    const float hi = tf32_round(x);
    const float lo = tf32_round(x - hi);
    const int64_t c = (int64_t)h * rg + (int64_t)slot * r + t;
    Ahi[a * kd + c] = hi;
    Alo[a * kd + c] = lo;
  }
}

// Tensor-core operands from tile-blocked FP32 panels [T][which][GK1][128]:
// row a of A gets xi terms at columns q < nterms and eta terms at rg + q; the
// other columns of the row are zero.  x = hi + lo, hi = tf32(x), lo = tf32(x - hi).
__global__ void k_pack_tc_tiles(const float* __restrict__ Pp, int GK1, int nterms, int rg,
                                int n_rows, float* __restrict__ Ahi, float* __restrict__ Alo,
                                int64_t kd) {
  const int64_t a = blockIdx.x;
  const int64_t ba = ((a / PT) * 2) * (int64_t)GK1 * PT + (a % PT);
  for (int c = threadIdx.x; c < kd; c += blockDim.x) {
    const int h = c >= rg ? 1 : 0;
    const int q = c - h * rg;
    float x = 0.f;
    if (q < nterms) x = Pp[ba + (int64_t)(h * GK1 + q) * PT];
    const float hi = tf32_round(x);
    Ahi[a * kd + c] = hi;
    Alo[a * kd + c] = tf32_round(x - hi);
  }
}

// Largest |value| of each pending term: maxes[which][q] over all rows (the
// bits of a non-negative float order like the float).  Block (T, which, z)
// takes terms z * 32 + [0, 32) of tile T, one warp per term at a time.
constexpr int TM_TERMS = 32;
__global__ void k_term_max(const float* __restrict__ Pp, int GK1, int nterms,
                           unsigned int* __restrict__ maxes) {
  const int T = blockIdx.x, which = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q1 = min(nterms, (int)(blockIdx.z + 1) * TM_TERMS);
  for (int q = blockIdx.z * TM_TERMS + warp; q < q1; q += blockDim.x >> 5) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(
        Pp + (((int64_t)T * 2 + which) * GK1 + q) * PT) + lane);
    float m = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > 0.f) atomicMax(&maxes[which * nterms + q], __float_as_uint(m));
  }
}

// FP16 tensor-core operands from tile-blocked FP32 panels: as k_pack_tc_tiles,
// after scaling term q's xi column by 2^e_q and its eta column by 2^-e_q,
// e_q = (exponent of max|eta_q| - exponent of max|xi_q|) / 2.  The product
// xi_q eta_q^T is unchanged by the scaling (powers of two are exact) and both
// scaled columns share one magnitude, which keeps them in FP16's normal range.
// x = hi + lo, hi = fp16(x), lo = fp16(x - hi).
// Bhi / Blo (optional): the same rows with their two halves swapped, for a
// pass whose operand rows are too narrow to swap the halves by TMA box.
// Block (T, z) transposes operand columns [64 z, 64 z + 64) of the 128 rows of
// tile T through shared memory: each panel column is read as one contiguous
// 512-byte run, each operand row segment written as one 128-byte run.
constexpr int PK_COLS = 64;
__global__ void __launch_bounds__(256) k_pack_f16_tiles(
    const float* __restrict__ Pp, int GK1, int nterms, int rg, const unsigned int* __restrict__ maxes,
    __half* __restrict__ Ahi, __half* __restrict__ Alo, __half* __restrict__ Bhi,
    __half* __restrict__ Blo, int64_t kd) {
  __shared__ float tile[PK_COLS][PT + 1];
  const int T = blockIdx.x;
  const int c0 = blockIdx.y * PK_COLS;  // rg is a multiple of 32
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cc = warp; cc < PK_COLS; cc += 8) {
    const int h = c0 + cc >= rg ? 1 : 0;
    const int q = c0 + cc - h * rg;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < nterms) {
      v = __ldcs(reinterpret_cast<const float4*>(Pp + (((int64_t)T * 2 + h) * GK1 + q) * PT) +
                 lane);
      const float mx = __uint_as_float(maxes[q]), me = __uint_as_float(maxes[nterms + q]);
      if (mx > 0.f && me > 0.f) {
        const int e = (ilogbf(me) - ilogbf(mx)) / 2;
        const int sh = h ? -e : e;
        v.x = ldexpf(v.x, sh);
        v.y = ldexpf(v.y, sh);
        v.z = ldexpf(v.z, sh);
        v.w = ldexpf(v.w, sh);
      }
    }
    tile[cc][4 * lane + 0] = v.x;
    tile[cc][4 * lane + 1] = v.y;
    tile[cc][4 * lane + 2] = v.z;
    tile[cc][4 * lane + 3] = v.w;
  }
  __syncthreads();
  // warp w writes rows w, w + 8, ...: lane l the columns 2l, 2l + 1
  for (int r = warp; r < PT; r += 8) {
    const float x0 = tile[2 * lane][r], x1 = tile[2 * lane + 1][r];
    const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
    const __half l0 = __float2half_rn(x0 - __half2float(h0));
    const __half l1 = __float2half_rn(x1 - __half2float(h1));
    const int c = c0 + 2 * lane;
    const int64_t o = ((int64_t)T * PT + r) * kd;
    *reinterpret_cast<__half2*>(Ahi + o + c) = __halves2half2(h0, h1);
    *reinterpret_cast<__half2*>(Alo + o + c) = __halves2half2(l0, l1);
    if (Bhi) {
      const int cb = c < rg ? c + rg : c - rg;  // rg is even: the pair stays in one half
      *reinterpret_cast<__half2*>(Bhi + o + cb) = __halves2half2(h0, h1);
      *reinterpret_cast<__half2*>(Blo + o + cb) = __halves2half2(l0, l1);
    }
  }
}

}  // namespace

void launch_signed_rows(const void* S, int s_prec, int64_t ld, const int32_t* src, const int8_t* sign,
                        const int64_t* off, int r, int n_pad, double* Zc, cudaStream_t st,
                        int upper) {
  dim3 grid((n_pad + 255) / 256, r);
  if (s_prec == 64)
    k_signed_rows<double><<<grid, 256, 0, st>>>((const double*)S, ld, src, sign, off, n_pad, Zc, upper);
  else
    k_signed_rows<float><<<grid, 256, 0, st>>>((const float*)S, ld, src, sign, off, n_pad, Zc, upper);
}

void launch_transpose_rect(const double* A, int64_t lda, double* B, int64_t ldb, int rows, int cols,
                           cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  k_transpose_rect<<<grid, block, 0, st>>>(A, lda, B, ldb, rows, cols);
}

void launch_lambda(const void* S, int s_prec, int64_t ld, const int32_t* sinks, const double* av,
                   const double* bv, const double* Y, const double* Z, int64_t ldz,
                   const int32_t* src, const int8_t* sign, const int64_t* off, int r, double C,
                   double* Lam, cudaStream_t st, int upper) {
  dim3 grid((r + 127) / 128, r);
  if (s_prec == 64)
    k_lambda<double><<<grid, 128, 0, st>>>((const double*)S, ld, sinks, av, bv, Y, Z, ldz, src, sign,
                                          off, r, C, Lam, upper);
  else
    k_lambda<float><<<grid, 128, 0, st>>>((const float*)S, ld, sinks, av, bv, Y, Z, ldz, src, sign,
                                         off, r, C, Lam, upper);
}

void launch_w_assemble(const void* S, int s_prec, int64_t ld, const int32_t* sinks, const double* av,
                       const double* bv, const double* Yc, const double* Lam, int r, int n_pad,
                       double C, double* Wc, cudaStream_t st, int upper) {
  dim3 grid((n_pad + 255) / 256, r);
  if (s_prec == 64)
    k_w_assemble<double><<<grid, 256, 0, st>>>((const double*)S, ld, sinks, av, bv, Yc, n_pad, C, Wc, upper);
  else
    k_w_assemble<float><<<grid, 256, 0, st>>>((const float*)S, ld, sinks, av, bv, Yc, n_pad, C, Wc, upper);
  dim3 g2((r + 127) / 128, r);
  k_w_lambda<<<g2, 128, 0, st>>>(sinks, Lam, r, n_pad, Wc);
}

void launch_xi0(const int32_t* sinks, int r, double C, double* X0, int64_t ldx, cudaStream_t st) {
  k_xi0<<<(r + 127) / 128, 128, 0, st>>>(sinks, r, C, X0, ldx);
}

void launch_pack_ffma(const double* X, int64_t ldx, int rh, int r, int slot, int terms, int nT,
                      void* Pn, int p_prec, uint64_t* mXi, uint64_t* mEta, cudaStream_t st) {
  dim3 grid(nT, (r + 1) / 2);
  if (p_prec == 64)
    k_pack_ffma<double><<<grid, 256, 0, st>>>(X, ldx, rh, r, slot, terms, nT, (double*)Pn, mXi, mEta);
  else
    k_pack_ffma<float><<<grid, 256, 0, st>>>(X, ldx, rh, r, slot, terms, nT, (float*)Pn, mXi, mEta);
}

void launch_pack_tc_tiles(const float* Pp, int GK1, int nterms, int rg, int n_rows, float* Ahi,
                          float* Alo, int64_t kd, cudaStream_t st) {
  k_pack_tc_tiles<<<n_rows, 256, 0, st>>>(Pp, GK1, nterms, rg, n_rows, Ahi, Alo, kd);
}

void launch_pack_f16_tiles(const float* Pp, int GK1, int nterms, int rg, int n_rows,
                           unsigned int* maxes, void* Ahi, void* Alo, void* Bhi, void* Blo,
                           int64_t kd, cudaStream_t st) {
  const int nT = n_rows / PT;
  cudaMemsetAsync(maxes, 0, 2 * (size_t)nterms * sizeof(unsigned int), st);
  k_term_max<<<dim3(nT, 2, (nterms + TM_TERMS - 1) / TM_TERMS), 256, 0, st>>>(Pp, GK1, nterms,
                                                                             maxes);
  k_pack_f16_tiles<<<dim3(nT, (unsigned)(kd / PK_COLS)), 256, 0, st>>>(
      Pp, GK1, nterms, rg, maxes, (__half*)Ahi, (__half*)Alo, (__half*)Bhi, (__half*)Blo, kd);
}

void launch_pack_tc(const double* X, int64_t ldx, int rh, int r, int slot, int rg, int n_rows,
                    float* Ahi, float* Alo, int64_t kd, cudaStream_t st) {
  dim3 grid(n_rows, (r + 127) / 128);
  k_pack_tc<<<grid, 128, 0, st>>>(X, ldx, rh, r, slot, rg, n_rows, Ahi, Alo, kd);
}

}  // namespace sr

namespace sr {
namespace {

// Y[row][c] += scale / len(row) * sum_{e in chunk} X[col_e][c] (Q times a
// block of columns, in FP64), for the column quads c = 4 q < ncols; Y zeroed by
// the caller.  A group of LPC lanes takes one row chunk (at most kChunk
// nonzeros), lane l of the group the quad blockIdx.y * LPC + l, so a long row
// is spread over many groups and meets in atomics.
template <int LPC>
__global__ void __launch_bounds__(256) k_spmm_chunks64(const RowChunk* __restrict__ chunks,
                                                       int64_t count,
                                                       const int32_t* __restrict__ col,
                                                       const int32_t* __restrict__ len,
                                                       const double* __restrict__ X, int64_t ldx,
                                                       double* __restrict__ Y, int64_t ldy,
                                                       int ncols, double scale) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPC;
  const int c0 = 4 * ((int)blockIdx.y * LPC + (int)(threadIdx.x % LPC));
  if (q >= count || c0 >= ncols) return;
  const RowChunk ch = chunks[q];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int e = 0;
  for (; e + 2 <= ch.len; e += 2) {
    const int b0 = __ldg(col + ch.start + e), b1 = __ldg(col + ch.start + e + 1);
    const double2* p0 = reinterpret_cast<const double2*>(X + (int64_t)b0 * ldx + c0);
    const double2* p1 = reinterpret_cast<const double2*>(X + (int64_t)b1 * ldx + c0);
    const double2 u0 = p0[0], v0 = p0[1], u1 = p1[0], v1 = p1[1];
    a0 += u0.x + u1.x;
    a1 += u0.y + u1.y;
    a2 += v0.x + v1.x;
    a3 += v0.y + v1.y;
  }
  if (e < ch.len) {
    const int b0 = __ldg(col + ch.start + e);
    const double2* p0 = reinterpret_cast<const double2*>(X + (int64_t)b0 * ldx + c0);
    const double2 u0 = p0[0], v0 = p0[1];
    a0 += u0.x;
    a1 += u0.y;
    a2 += v0.x;
    a3 += v0.y;
  }
  const double rs = scale / (double)len[ch.row];
  double* y = Y + (int64_t)ch.row * ldy + c0;
  atomicAdd(y + 0, rs * a0);
  atomicAdd(y + 1, rs * a1);
  atomicAdd(y + 2, rs * a2);
  atomicAdd(y + 3, rs * a3);
}

// Largest |value| of every term column of the one-shot block X (FP64
// [n_rows][ldx]): maxes[c] for xi column c < r, maxes[r + c] for the W column
// rh + c, as the bits of an FP32 magnitude (non-negative floats order like
// their bits).  Block (32, 8): a lane per column, 8 row phases.
__global__ void __launch_bounds__(256) k_oneshot_max(const double* __restrict__ X, int64_t ldx,
                                                     int rh, int r, int n_rows,
                                                     unsigned int* __restrict__ maxes) {
  __shared__ float red[8][32];
  const int c2 = blockIdx.x * 32 + threadIdx.x;
  float m = 0.f;
  if (c2 < 2 * r) {
    const int which = c2 >= r ? 1 : 0;
    const int64_t col = (int64_t)which * rh + (c2 - which * r);
    for (int64_t a = (int64_t)blockIdx.y * 8 + threadIdx.y; a < n_rows; a += (int64_t)gridDim.y * 8)
      m = fmaxf(m, (float)fabs(X[a * ldx + col]));
  }
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && c2 < 2 * r) {
#pragma unroll
    for (int y = 1; y < 8; ++y) m = fmaxf(m, red[y][threadIdx.x]);
    if (m > 0.f) atomicMax(&maxes[c2], __float_as_uint(m));
  }
}

// FP16 tensor-core operands of the one-shot update from X_k: term t of the
// slot (xi column t, W column rh + t) goes to columns slot * r + t and
// rg + slot * r + t of A_hi / A_lo, after scaling the xi column by 2^e and the
// W column by 2^-e, e = (exponent of max |W_t| - exponent of max |xi_t|) / 2:
// their product is unchanged (powers of two are exact) and both share one
// magnitude inside FP16's range.  x = hi + lo, hi = fp16(x), lo = fp16(x - hi).
__global__ void k_pack_f16_oneshot(const double* __restrict__ X, int64_t ldx, int rh, int r,
                                   int slot, int rg, int n_rows,
                                   const unsigned int* __restrict__ maxes,
                                   __half* __restrict__ Ahi, __half* __restrict__ Alo, int64_t kd) {
  const int64_t a = blockIdx.x;
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  if (t >= r || a >= n_rows) return;
  const float mx = __uint_as_float(maxes[t]), me = __uint_as_float(maxes[r + t]);
  const int e = (mx > 0.f && me > 0.f) ? (ilogbf(me) - ilogbf(mx)) / 2 : 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double x = ldexp(X[a * ldx + (int64_t)h * rh + t], h ? -e : e);
    const __half hi = __double2half(x);
    const __half lo = __double2half(x - (double)__half2float(hi));
    const int64_t c = (int64_t)h * rg + (int64_t)slot * r + t;
    Ahi[a * kd + c] = hi;
    Alo[a * kd + c] = lo;
  }
}

template <int LPC>
void spmm_chunks64_t(const RowChunk* chunks, int64_t count, const int32_t* col,
                     const int32_t* len, const double* X, int64_t ldx, double* Y, int64_t ldy,
                     int ncols, double scale, cudaStream_t st) {
  const int quads = ncols / 4;
  const dim3 grid((unsigned)((count * LPC + 255) / 256), (unsigned)((quads + LPC - 1) / LPC));
  k_spmm_chunks64<LPC><<<grid, 256, 0, st>>>(chunks, count, col, len, X, ldx, Y, ldy, ncols,
                                              scale);
}

}  // namespace

void launch_pack_f16_oneshot(const double* X, int64_t ldx, int rh, int r, int slot, int rg,
                             int n_rows, unsigned int* maxes, void* Ahi, void* Alo, int64_t kd,
                             cudaStream_t st) {
  cudaMemsetAsync(maxes, 0, 2 * (size_t)r * sizeof(unsigned int), st);
  const dim3 mg((unsigned)((2 * r + 31) / 32), 64), mb(32, 8);
  k_oneshot_max<<<mg, mb, 0, st>>>(X, ldx, rh, r, n_rows, maxes);
  const dim3 grid((unsigned)n_rows, (unsigned)((r + 127) / 128));
  k_pack_f16_oneshot<<<grid, 128, 0, st>>>(X, ldx, rh, r, slot, rg, n_rows, maxes, (__half*)Ahi,
                                           (__half*)Alo, kd);
}

int launch_spmm_chunks64(const RowChunk* chunks, int64_t count, const int32_t* col,
                         const int32_t* len, const double* X, int64_t ldx, double* Y, int64_t ldy,
                         int ncols, double scale, cudaStream_t st) {
  if (ncols % 4 || ldx % 2 || ldy % 2 || ((uintptr_t)X & 15)) return 1;
  if (count <= 0 || ncols <= 0) return 0;
  const int quads = ncols / 4;
  if (quads <= 8)
    spmm_chunks64_t<8>(chunks, count, col, len, X, ldx, Y, ldy, ncols, scale, st);
  else if (quads <= 16)
    spmm_chunks64_t<16>(chunks, count, col, len, X, ldx, Y, ldy, ncols, scale, st);
  else
    spmm_chunks64_t<32>(chunks, count, col, len, X, ldx, Y, ldy, ncols, scale, st);
  return 0;
}

}  // namespace sr
