// Batch SimRank on the GPU: Jacobi sweeps of Eq. 1,
//   S <- C Q S Q^T + (1 - C) I,
// computed as X = Q S (row gathers), X^T (tiled transpose), S' = C Q X^T + (1-C) I.
// Since S is symmetric, Q S Q^T = Q (Q S)^T.  Used at init and to re-anchor S
// after long FP32 update streams.  Also the column copy used by
// simrank_columns.
#include "sr_internal.h"

namespace sr {

namespace {

template <typename T>
struct Ld4;
template <>
struct Ld4<float> {
  static __device__ __forceinline__ void load(const float* p, double* v) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
  static __device__ __forceinline__ void store(float* p, const double* v) {
    *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  }
};
template <>
struct Ld4<double> {
  static __device__ __forceinline__ void load(const double* p, double* v) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p));
    const double2 y = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = y.x;
    v[3] = y.y;
  }
  static __device__ __forceinline__ void store(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// Y[a, c] = scale * sum_{b in I(a)} q_ab X[b, c] + diag [a == c and a < n_diag]
// for a < n_rows, c < ncols (multiple of 4); q_ab = 1/len(a) or w_ba / wsum_a.
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) k_spmm_rows(DevAdj in, const float* __restrict__ w,
                                                   const double* __restrict__ wsum,
                                                   const TX* __restrict__ X, int64_t ldx,
                                                   TY* __restrict__ Y, int64_t ldy, int ncols,
                                                   double scale, double diag, int n_diag) {
  const int a = blockIdx.x;
  const int c0 = (blockIdx.y * 256 + threadIdx.x) * 4;
  if (c0 >= ncols) return;
  const int64_t st = in.start[a];
  const int len = in.len[a];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int e = 0;
  for (; e + 1 < len; e += 2) {
    const int b0 = in.col[st + e], b1 = in.col[st + e + 1];
    double v0[4], v1[4];
    Ld4<TX>::load(X + (int64_t)b0 * ldx + c0, v0);
    Ld4<TX>::load(X + (int64_t)b1 * ldx + c0, v1);
    const double q0 = w ? (double)w[st + e] : 1.0;
    const double q1 = w ? (double)w[st + e + 1] : 1.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += q0 * v0[q] + q1 * v1[q];
  }
  if (e < len) {
    const int b0 = in.col[st + e];
    double v0[4];
    Ld4<TX>::load(X + (int64_t)b0 * ldx + c0, v0);
    const double q0 = w ? (double)w[st + e] : 1.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += q0 * v0[q];
  }
  double norm = 0.0;
  if (len > 0) norm = w ? 1.0 / wsum[a] : 1.0 / (double)len;
  double out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    out[q] = scale * norm * acc[q];
    if (c0 + q == a && a < n_diag) out[q] += diag;
  }
  Ld4<TY>::store(Y + (int64_t)a * ldy + c0, out);
}

template <typename T>
__global__ void k_transpose(const T* __restrict__ A, T* __restrict__ B, int64_t ld) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8)
    tile[r][threadIdx.x] = A[(int64_t)(by + r) * ld + bx + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8)
    B[(int64_t)(bx + r) * ld + by + threadIdx.x] = tile[threadIdx.x][r];
}

template <typename T>
__global__ void k_symmetrize(T* __restrict__ A, int64_t ld) {
  // one CTA per 32 x 32 block pair (bi <= bj)
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj < bi) return;
  __shared__ T t1[32][33], t2[32][33];
  for (int r = threadIdx.y; r < 32; r += 8) {
    t1[r][threadIdx.x] = A[(int64_t)(bi * 32 + r) * ld + bj * 32 + threadIdx.x];
    t2[r][threadIdx.x] = A[(int64_t)(bj * 32 + r) * ld + bi * 32 + threadIdx.x];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const T v = (T)0.5 * (t1[r][threadIdx.x] + t2[threadIdx.x][r]);
    A[(int64_t)(bi * 32 + r) * ld + bj * 32 + threadIdx.x] = v;
  }
  __syncthreads();
  if (bi != bj) {
    for (int r = threadIdx.y; r < 32; r += 8) {
      const T v = (T)0.5 * (t2[r][threadIdx.x] + t1[threadIdx.x][r]);
      A[(int64_t)(bj * 32 + r) * ld + bi * 32 + threadIdx.x] = v;
    }
  }
}

template <typename T>
__global__ void k_maxdiff(const T* __restrict__ A, const T* __restrict__ B, int n, int64_t ld,
                          unsigned long long* out) {
  double m = 0.0;
  const int64_t tot = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, c = e % n;
    const double d = fabs((double)A[r * ld + c] - (double)B[r * ld + c]);
    m = fmax(m, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

template <typename T>
__global__ void k_set_diag(T* A, int from, int to, int64_t ld, double value) {
  const int x = from + blockIdx.x * blockDim.x + threadIdx.x;
  if (x < to) A[(int64_t)x * ld + x] = (T)value;
}

template <typename TA, typename TB>
__global__ void k_convert(const TA* __restrict__ A, TB* __restrict__ B, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    B[e] = (TB)A[e];
}

// out[c * n + a] = S[cols[c], perm[a]] (perm = caller id -> storage id, or identity)
template <typename TS, typename TO>
__global__ void k_copy_cols(const TS* __restrict__ S, int64_t ld, const int32_t* __restrict__ cols,
                            const int32_t* __restrict__ perm, int n, TO* __restrict__ out,
                            int upper) {
  const int c = blockIdx.y;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) {
    const int p = perm ? perm[a] : a;
    out[(int64_t)c * n + a] = (TO)s_at(S, ld, cols[c], p, upper != 0);
  }
}

// Lower tiles := the transposes of their mirrors (S[J, I] = S[I, J]^T for
// 128-tiles I < J), one CTA per 32 x 32 block of the upper triangle.
template <typename T>
__global__ void k_mirror_lower(T* __restrict__ A, int64_t ld) {
  const int bi = blockIdx.y, bj = blockIdx.x;  // 32-blocks
  if ((bi * 32) / PT >= (bj * 32) / PT) return;
  __shared__ T t[32][33];
  for (int r = threadIdx.y; r < 32; r += 8)
    t[r][threadIdx.x] = A[(int64_t)(bi * 32 + r) * ld + bj * 32 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8)
    A[(int64_t)(bj * 32 + r) * ld + bi * 32 + threadIdx.x] = t[threadIdx.x][r];
}

}  // namespace

// Example 2 (§1): on a forest of arborescences (every node has at most one
// in-neighbour, its parent) Eq. 1 has the closed form
//   S(a, b) = C^lam (1 - C^(H - lam + 1))
// when a and b are on the same level H of the same tree, lam being the number
// of edges from their lowest common ancestor down to a (or b); S(a, b) = 0
// when they are on different levels or in different trees.  (Row a of Q is
// e_parent(a), so S(a, b) = C S(p(a), p(b)) for a != b and
// S(a, a) = C S(p(a), p(a)) + 1 - C, with S(r, x) = (1 - C) [r == x] at a root.)
// One CTA per 128 x 128 tile (tiles I <= J only when `upper`); thread t owns
// column t % 128 and every other row.  powC[k] = C^k for k <= max level + 1.
template <typename T>
__global__ void __launch_bounds__(256) k_forest_init(T* __restrict__ S, int64_t ld,
                                                     const int32_t* __restrict__ parent,
                                                     const int32_t* __restrict__ level,
                                                     const double* __restrict__ powC, int n,
                                                     int nT, int upper) {
  const int I = blockIdx.y, J = blockIdx.x;
  if (upper && I > J) return;
  const int c = threadIdx.x & (PT - 1);
  const int b = J * PT + c;
  const int lb = b < n ? __ldg(level + b) : -1;
  for (int r = threadIdx.x >> 7; r < PT; r += 2) {
    const int a = I * PT + r;
    T v = T(0);
    if (a < n && lb >= 0 && __ldg(level + a) == lb) {
      int x = a, y = b, lam = 0;
      while (x != y && x >= 0 && lam <= lb) {
        x = __ldg(parent + x);
        y = __ldg(parent + y);
        ++lam;
      }
      if (x >= 0 && x == y) v = (T)(powC[lam] * (1.0 - powC[lb - lam + 1]));
    }
    S[(int64_t)a * ld + b] = v;
  }
}

void launch_forest_init(void* S, int prec, int64_t ld, const int32_t* parent, const int32_t* level,
                        const double* powC, int n, int nT, int upper, cudaStream_t st) {
  dim3 grid(nT, nT);
  if (prec == 64)
    k_forest_init<double><<<grid, 256, 0, st>>>((double*)S, ld, parent, level, powC, n, nT, upper);
  else
    k_forest_init<float><<<grid, 256, 0, st>>>((float*)S, ld, parent, level, powC, n, nT, upper);
}

void launch_spmm_rows(const DevAdj& in, const float* w, const double* wsum, const void* X,
                      int x_prec, int64_t ldx, void* Y, int y_prec, int64_t ldy, int n_rows,
                      int ncols, double scale, double diag, int n_diag, cudaStream_t st) {
  dim3 grid(n_rows, (ncols / 4 + 255) / 256);
  if (x_prec == 64 && y_prec == 64)
    k_spmm_rows<double, double><<<grid, 256, 0, st>>>(in, w, wsum, (const double*)X, ldx,
                                                      (double*)Y, ldy, ncols, scale, diag, n_diag);
  else if (x_prec == 32 && y_prec == 32)
    k_spmm_rows<float, float><<<grid, 256, 0, st>>>(in, w, wsum, (const float*)X, ldx, (float*)Y,
                                                    ldy, ncols, scale, diag, n_diag);
  else if (x_prec == 64 && y_prec == 32)
    k_spmm_rows<double, float><<<grid, 256, 0, st>>>(in, w, wsum, (const double*)X, ldx,
                                                     (float*)Y, ldy, ncols, scale, diag, n_diag);
  else
    k_spmm_rows<float, double><<<grid, 256, 0, st>>>(in, w, wsum, (const float*)X, ldx,
                                                     (double*)Y, ldy, ncols, scale, diag, n_diag);
}

void launch_transpose(const void* A, void* B, int prec, int n_pad, int64_t ld, cudaStream_t st) {
  dim3 grid(n_pad / 32, n_pad / 32), block(32, 8);
  if (prec == 64)
    k_transpose<double><<<grid, block, 0, st>>>((const double*)A, (double*)B, ld);
  else
    k_transpose<float><<<grid, block, 0, st>>>((const float*)A, (float*)B, ld);
}

void launch_maxdiff(const void* A, const void* B, int prec, int n, int64_t ld,
                    unsigned long long* out_bits, cudaStream_t st) {
  const int blocks = 4096;
  if (prec == 64)
    k_maxdiff<double><<<blocks, 256, 0, st>>>((const double*)A, (const double*)B, n, ld, out_bits);
  else
    k_maxdiff<float><<<blocks, 256, 0, st>>>((const float*)A, (const float*)B, n, ld, out_bits);
}

void launch_symmetrize(void* A, int prec, int n_pad, int64_t ld, cudaStream_t st) {
  dim3 grid(n_pad / 32, n_pad / 32), block(32, 8);
  if (prec == 64)
    k_symmetrize<double><<<grid, block, 0, st>>>((double*)A, ld);
  else
    k_symmetrize<float><<<grid, block, 0, st>>>((float*)A, ld);
}

void launch_mirror_lower(void* A, int prec, int n_pad, int64_t ld, cudaStream_t st) {
  dim3 grid(n_pad / 32, n_pad / 32), block(32, 8);
  if (prec == 64)
    k_mirror_lower<double><<<grid, block, 0, st>>>((double*)A, ld);
  else
    k_mirror_lower<float><<<grid, block, 0, st>>>((float*)A, ld);
}

void launch_set_diag(void* A, int prec, int from, int to, int64_t ld, double value,
                     cudaStream_t st) {
  if (to <= from) return;
  const int blocks = (to - from + 255) / 256;
  if (prec == 64)
    k_set_diag<double><<<blocks, 256, 0, st>>>((double*)A, from, to, ld, value);
  else
    k_set_diag<float><<<blocks, 256, 0, st>>>((float*)A, from, to, ld, value);
}

void launch_convert(const void* A, int a_prec, void* B, int b_prec, int64_t count, cudaStream_t st) {
  const int blocks = 8192;
  if (a_prec == 64 && b_prec == 32)
    k_convert<double, float><<<blocks, 256, 0, st>>>((const double*)A, (float*)B, count);
  else if (a_prec == 32 && b_prec == 64)
    k_convert<float, double><<<blocks, 256, 0, st>>>((const float*)A, (double*)B, count);
  else if (a_prec == 64)
    k_convert<double, double><<<blocks, 256, 0, st>>>((const double*)A, (double*)B, count);
  else
    k_convert<float, float><<<blocks, 256, 0, st>>>((const float*)A, (float*)B, count);
}

void launch_copy_cols(const void* S, int s_prec, int64_t ld, const int32_t* cols, const int32_t* perm,
                      int ncols, int n, void* out, int out_fp64, cudaStream_t st, int upper) {
  if (ncols <= 0 || n <= 0) return;
  dim3 grid((n + 255) / 256, ncols);
  if (s_prec == 64) {
    if (out_fp64)
      k_copy_cols<double, double><<<grid, 256, 0, st>>>((const double*)S, ld, cols, perm, n, (double*)out, upper);
    else
      k_copy_cols<double, float><<<grid, 256, 0, st>>>((const double*)S, ld, cols, perm, n, (float*)out, upper);
  } else {
    if (out_fp64)
      k_copy_cols<float, double><<<grid, 256, 0, st>>>((const float*)S, ld, cols, perm, n, (double*)out, upper);
    else
      k_copy_cols<float, float><<<grid, 256, 0, st>>>((const float*)S, ld, cols, perm, n, (float*)out, upper);
  }
}

}  // namespace sr
