// Fused S update (Alg 1 final step, Alg 2 with Thm 4 pruning):
//   S <- S + M_K + M_K^T,  M_K = sum_{k=0}^{K} xi_k eta_k^T,
// applied as one read-modify-write pass per affected tile pair (I <= J): the
// CTA forms Delta_IJ = sum_k xi_k[I] eta_k[J]^T + eta_k[I] xi_k[J]^T once and
// adds it to S[I,J] and, transposed, to S[J,I] (Delta S is symmetric), so
// each entry of the upper triangle costs 2(K+1) FMAs for two S entries.
#include "sr_internal.h"

namespace sr {

namespace {

// 256 threads as 16 x 16; thread (tx, ty) owns rows {ty*4+q, 64+ty*4+q} and
// columns {tx*4+q, 64+tx*4+q}, q < 4, of the 128 x 128 tile, so every
// float4 access of a warp covers 256 contiguous bytes.
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4;
};

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
  const typename Vec4<T>::type x = *reinterpret_cast<const typename Vec4<T>::type*>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
template <typename T>
__device__ __forceinline__ void ld4p(const T* p, T* v) {
  const typename Vec4<T>::type x = *reinterpret_cast<const typename Vec4<T>::type*>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
  typename Vec4<T>::type x;
  x.x = v[0];
  x.y = v[1];
  x.z = v[2];
  x.w = v[3];
  *reinterpret_cast<typename Vec4<T>::type*>(p) = x;
}

// Row pitch (elements) of the Delta tile staged in shared memory; odd, so
// that both a row sweep and a column sweep of a warp hit 32 distinct banks.
constexpr int DP = PT + 1;

// One affected tile pair of one graph: where its S and panels live, and the
// AFF words of the two cross terms (bit k % 64: xi_k[I] eta_k[J]^T resp.
// eta_k[I] xi_k[J]^T can be nonzero).
template <typename T>
struct TileRef {
  T* S;
  int64_t ld;
  const T* P;
  int I, J, n;
  uint64_t a1, a2;
  bool mirror;  // also apply Delta^T to S[J, I] (both triangles kept)
};

// Tile source of one graph: a list of (I << 16 | J) pairs.
template <typename T>
struct OneGraphTiles {
  T* S;
  int64_t ld;
  const T* P;
  const uint32_t* tiles;
  const uint64_t* mXi;
  const uint64_t* mEta;
  int use_masks, n, mirror;
  __device__ __forceinline__ TileRef<T> get(int t) const {
    const uint32_t pr = tiles[t];
    const int I = (int)(pr >> 16), J = (int)(pr & 0xffffu);
    TileRef<T> r{S, ld, P, I, J, n, ~0ull, ~0ull, mirror != 0};
    if (use_masks) {
      r.a1 = mXi[I] & mEta[J];
      r.a2 = mEta[I] & mXi[J];
    }
    return r;
  }
};

// Tile source of many graphs: (g << 32 | I << 16 | J) entries and one
// descriptor per graph.
template <typename T>
struct ManyGraphTiles {
  const MultiGraphDesc* d;
  const uint64_t* tiles;
  __device__ __forceinline__ TileRef<T> get(int t) const {
    const uint64_t e = tiles[t];
    const int g = (int)(e >> 32), I = (int)((e >> 16) & 0xffffu), J = (int)(e & 0xffffu);
    const MultiGraphDesc& q = d[g];
    return TileRef<T>{(T*)q.S,         q.ld, (const T*)q.P, I, J, q.n, q.mXi[I] & q.mEta[J],
                      q.mEta[I] & q.mXi[J], q.upper == 0};
  }
};

template <typename T, int KC, int MINB, typename Src>
__global__ void __launch_bounds__(256, MINB)
    k_s_update(Src src, int K1, const int* __restrict__ ntiles, int k0g, int k1g,
               unsigned long long* __restrict__ counters) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sXiI = reinterpret_cast<T*>(smem_raw);
  T* sEtaI = sXiI + KC * PT;
  T* sXiJ = sEtaI + KC * PT;
  T* sEtaJ = sXiJ + KC * PT;
  T* sD = sEtaJ + KC * PT;  // [PT][DP] Delta tile
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int nt = *ntiles;
  unsigned long long my_tiles = 0, my_bytes = 0;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const TileRef<T> tr = src.get(t);
    T* __restrict__ S = tr.S;
    const T* __restrict__ P = tr.P;
    const int64_t ld = tr.ld;
    const int I = tr.I, J = tr.J, n = tr.n;
    const uint64_t a1 = tr.a1;  // xi_I eta_J^T
    const uint64_t a2 = tr.a2;  // eta_I xi_J^T
    T acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = T(0);

    // ---- phase 1: Delta_IJ = sum_k xi_k[I] eta_k[J]^T + eta_k[I] xi_k[J]^T (registers)
    for (int kb = k0g; kb < k1g; kb += KC) {
      const int kc = min(KC, k1g - kb);
      uint64_t chunk = 0;
      for (int kk = 0; kk < kc; ++kk) chunk |= 1ull << ((kb + kk) & 63);
      if (((a1 | a2) & chunk) == 0) continue;  // no active term in this chunk
      __syncthreads();  // previous chunk fully consumed
      const int nvec = kc * PT / 4;
      const T* gXiI = P + ((int64_t)I * 2 + 0) * K1 * PT + (int64_t)kb * PT;
      const T* gEtaI = P + ((int64_t)I * 2 + 1) * K1 * PT + (int64_t)kb * PT;
      const T* gXiJ = P + ((int64_t)J * 2 + 0) * K1 * PT + (int64_t)kb * PT;
      const T* gEtaJ = P + ((int64_t)J * 2 + 1) * K1 * PT + (int64_t)kb * PT;
      using V = typename Vec4<T>::type;
      for (int e = tid; e < nvec; e += 256) {
        reinterpret_cast<V*>(sXiI)[e] = reinterpret_cast<const V*>(gXiI)[e];
        reinterpret_cast<V*>(sEtaI)[e] = reinterpret_cast<const V*>(gEtaI)[e];
        reinterpret_cast<V*>(sXiJ)[e] = reinterpret_cast<const V*>(gXiJ)[e];
        reinterpret_cast<V*>(sEtaJ)[e] = reinterpret_cast<const V*>(gEtaJ)[e];
      }
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
        const uint64_t bit = 1ull << ((kb + kk) & 63);
        const bool p1 = (a1 & bit) != 0, p2 = (a2 & bit) != 0;
        if (!(p1 || p2)) continue;
        T rx[8], re[8], cx[8], ce[8];
        ld4p(sXiI + kk * PT + ty * 4, &rx[0]);
        ld4p(sXiI + kk * PT + 64 + ty * 4, &rx[4]);
        ld4p(sEtaI + kk * PT + ty * 4, &re[0]);
        ld4p(sEtaI + kk * PT + 64 + ty * 4, &re[4]);
        ld4p(sXiJ + kk * PT + tx * 4, &cx[0]);
        ld4p(sXiJ + kk * PT + 64 + tx * 4, &cx[4]);
        ld4p(sEtaJ + kk * PT + tx * 4, &ce[0]);
        ld4p(sEtaJ + kk * PT + 64 + tx * 4, &ce[4]);
        if (p1) {
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = fma(rx[r], ce[c], acc[r][c]);
        }
        if (p2) {
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = fma(re[r], cx[c], acc[r][c]);
        }
      }
    }

    // ---- phase 2: stage Delta in shared memory
    __syncthreads();  // previous tile's phase 3/4 readers are done with sD
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = (r < 4) ? ty * 4 + r : 64 + ty * 4 + (r - 4);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int col = (c < 4) ? tx * 4 + c : 64 + tx * 4 + (c - 4);
        sD[row * DP + col] = acc[r][c];
      }
    }
    __syncthreads();

    // ---- phase 3: S[I, J] += Delta, one 512-byte row segment per warp access
    {
      constexpr int NQ = PT * PT / 4 / 256;  // 16 vectors of 4 per thread
      T v[NQ][4];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int idx = tid + 256 * q;
        const int row = idx >> 5, c4 = (idx & 31) * 4;
        ld4p(S + (int64_t)(I * PT + row) * ld + (int64_t)J * PT + c4, v[q]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int idx = tid + 256 * q;
        const int row = idx >> 5, c4 = (idx & 31) * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) v[q][e] += sD[row * DP + c4 + e];
        st4(S + (int64_t)(I * PT + row) * ld + (int64_t)J * PT + c4, v[q]);
      }
    }
    // ---- phase 4: S[J, I] += Delta^T; a warp covers one 512-byte row segment
    // (lane -> 4 consecutive columns), 16 vector loads in flight per thread
    if (I != J && tr.mirror) {
      constexpr int NQ = PT * PT / 4 / 256;
      const int lane = tid & 31, warp = tid >> 5;
      T v[NQ][4];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = warp + 8 * q;
        ld4p(S + (int64_t)(J * PT + c) * ld + (int64_t)I * PT + lane * 4, v[q]);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int c = warp + 8 * q;
#pragma unroll
        for (int e = 0; e < 4; ++e) v[q][e] += sD[(lane * 4 + e) * DP + c];
        st4(S + (int64_t)(J * PT + c) * ld + (int64_t)I * PT + lane * 4, v[q]);
      }
    }
    if (tid == 0) {
      const long long vr = max(0, min(PT, n - I * PT)), vc = max(0, min(PT, n - J * PT));
      my_tiles += 1;
      my_bytes += (unsigned long long)(vr * vc) * 2ull * sizeof(T) *
                  ((I == J || !tr.mirror) ? 1ull : 2ull);
    }
  }
  if (tid == 0 && my_tiles) {
    atomicAdd(&counters[CNT_TILES_TOUCHED], my_tiles);
    atomicAdd(&counters[CNT_S_BYTES], my_bytes);
    atomicAdd(&counters[CNT_PANEL_BYTES],
              my_tiles * 4ull * (unsigned long long)(k1g - k0g) * PT * sizeof(T));
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised FP32 version: 8 math warps form Delta of tile pair i in
// shared buffer i % 2 while 8 memory warps apply Delta of tile pair i - 1 to
// S[I,J] and S[J,I], so the HBM stream never waits for the FMAs.  Hand-off
// by mbarriers; every wait is bounded and sets a status word on timeout.
// ---------------------------------------------------------------------------
constexpr int WS_KC = 16;
constexpr int WS_THREADS = 512;

__device__ __forceinline__ uint32_t ws_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ws_bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ws_smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void ws_bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ws_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool ws_bar_wait(uint64_t* bar, uint32_t parity, long long limit,
                                            volatile int* abort_flag) {
  const uint32_t a = ws_smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  return false;
}
// barrier among the 256 math threads only (hardware barrier 1)
__device__ __forceinline__ void ws_math_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// true on every one of the 256 threads of hardware barrier `id` iff `pred` is
// true on all of them: the two roles take each decision to stop together
__device__ __forceinline__ bool ws_all(int id, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, 256, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(WS_THREADS, 1)
    k_s_update_ws(float* __restrict__ S, int64_t ld, const float* __restrict__ P, int K1,
                  const uint32_t* __restrict__ tiles, const int* __restrict__ ntiles,
                  const uint64_t* __restrict__ mXi, const uint64_t* __restrict__ mEta, int k0g,
                  int k1g, int use_masks, int n, int mirror, long long wait_limit,
                  unsigned long long* __restrict__ counters) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* sXiI = reinterpret_cast<float*>(smem_raw);
  float* sEtaI = sXiI + WS_KC * PT;
  float* sXiJ = sEtaI + WS_KC * PT;
  float* sEtaJ = sXiJ + WS_KC * PT;
  float* sDbuf = sEtaJ + WS_KC * PT;  // 2 x [PT][DP]
  __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2];
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x;
  const int nt = *ntiles;
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < 2; ++b) {
      ws_bar_init(&bar_full[b], 256);
      ws_bar_init(&bar_empty[b], 256);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = true;
  if (tid < 256) {
    // ---------------- math warps
    const int tx = tid & 15, ty = tid >> 4;
    int i = 0;
    for (int t = blockIdx.x; t < nt; t += gridDim.x, ++i) {
      const uint32_t pr = tiles[t];
      const int I = (int)(pr >> 16), J = (int)(pr & 0xffffu);
      const uint64_t a1 = use_masks ? (mXi[I] & mEta[J]) : ~0ull;
      const uint64_t a2 = use_masks ? (mEta[I] & mXi[J]) : ~0ull;
      float acc[8][8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
      for (int kb = k0g; kb < k1g; kb += WS_KC) {
        const int kc = min(WS_KC, k1g - kb);
        uint64_t chunk = 0;
        for (int kk = 0; kk < kc; ++kk) chunk |= 1ull << ((kb + kk) & 63);
        if (((a1 | a2) & chunk) == 0) continue;
        ws_math_sync();
        const int nvec = kc * PT / 4;
        const float4* gXiI = reinterpret_cast<const float4*>(P + ((int64_t)I * 2 + 0) * K1 * PT + (int64_t)kb * PT);
        const float4* gEtaI = reinterpret_cast<const float4*>(P + ((int64_t)I * 2 + 1) * K1 * PT + (int64_t)kb * PT);
        const float4* gXiJ = reinterpret_cast<const float4*>(P + ((int64_t)J * 2 + 0) * K1 * PT + (int64_t)kb * PT);
        const float4* gEtaJ = reinterpret_cast<const float4*>(P + ((int64_t)J * 2 + 1) * K1 * PT + (int64_t)kb * PT);
        for (int e = tid; e < nvec; e += 256) {
          reinterpret_cast<float4*>(sXiI)[e] = __ldg(gXiI + e);
          reinterpret_cast<float4*>(sEtaI)[e] = __ldg(gEtaI + e);
          reinterpret_cast<float4*>(sXiJ)[e] = __ldg(gXiJ + e);
          reinterpret_cast<float4*>(sEtaJ)[e] = __ldg(gEtaJ + e);
        }
        ws_math_sync();
        for (int kk = 0; kk < kc; ++kk) {
          const uint64_t bit = 1ull << ((kb + kk) & 63);
          const bool p1 = (a1 & bit) != 0, p2 = (a2 & bit) != 0;
          if (!(p1 || p2)) continue;
          float rx[8], re[8], cx[8], ce[8];
          ld4p(sXiI + kk * PT + ty * 4, &rx[0]);
          ld4p(sXiI + kk * PT + 64 + ty * 4, &rx[4]);
          ld4p(sEtaI + kk * PT + ty * 4, &re[0]);
          ld4p(sEtaI + kk * PT + 64 + ty * 4, &re[4]);
          ld4p(sXiJ + kk * PT + tx * 4, &cx[0]);
          ld4p(sXiJ + kk * PT + 64 + tx * 4, &cx[4]);
          ld4p(sEtaJ + kk * PT + tx * 4, &ce[0]);
          ld4p(sEtaJ + kk * PT + 64 + tx * 4, &ce[4]);
          if (p1) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
              for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(rx[r], ce[c], acc[r][c]);
          }
          if (p2) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
              for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(re[r], cx[c], acc[r][c]);
          }
        }
      }
      const int b = i & 1;
      const bool got = ws_bar_wait(&bar_empty[b], ((i >> 1) & 1) ^ 1u, wait_limit, &abort_flag);
      if (!ws_all(1, got)) {
        ok = false;
        break;
      }
      float* sD = sDbuf + b * PT * DP;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = (r < 4) ? ty * 4 + r : 64 + ty * 4 + (r - 4);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int col = (c < 4) ? tx * 4 + c : 64 + tx * 4 + (c - 4);
          sD[row * DP + col] = acc[r][c];
        }
      }
      ws_bar_arrive(&bar_full[b]);
    }
  } else {
    // ---------------- memory warps: 8 warps, one 512-byte row segment per access
    const int mt = tid - 256;
    const int lane = mt & 31, warp = mt >> 5;
    int i = 0;
    unsigned long long my_tiles = 0, my_bytes = 0;
    for (int t = blockIdx.x; t < nt; t += gridDim.x, ++i) {
      const uint32_t pr = tiles[t];
      const int I = (int)(pr >> 16), J = (int)(pr & 0xffffu);
      const int b = i & 1;
      const bool got = ws_bar_wait(&bar_full[b], (i >> 1) & 1, wait_limit, &abort_flag);
      if (!ws_all(2, got)) {
        ok = false;
        break;
      }
      const float* sD = sDbuf + b * PT * DP;
      constexpr int NQ = PT / 8;  // 16 rows per warp
      {
        float v[NQ][4];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int row = warp + 8 * q;
          ld4p(S + (int64_t)(I * PT + row) * ld + (int64_t)J * PT + lane * 4, v[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int row = warp + 8 * q;
#pragma unroll
          for (int e = 0; e < 4; ++e) v[q][e] += sD[row * DP + lane * 4 + e];
          st4(S + (int64_t)(I * PT + row) * ld + (int64_t)J * PT + lane * 4, v[q]);
        }
      }
      if (I != J && mirror) {
        float v[NQ][4];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int c = warp + 8 * q;
          ld4p(S + (int64_t)(J * PT + c) * ld + (int64_t)I * PT + lane * 4, v[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int c = warp + 8 * q;
#pragma unroll
          for (int e = 0; e < 4; ++e) v[q][e] += sD[(lane * 4 + e) * DP + c];
          st4(S + (int64_t)(J * PT + c) * ld + (int64_t)I * PT + lane * 4, v[q]);
        }
      }
      ws_bar_arrive(&bar_empty[b]);
      if (mt == 0) {
        const long long vr = max(0, min(PT, n - I * PT)), vc = max(0, min(PT, n - J * PT));
        my_tiles += 1;
        my_bytes += (unsigned long long)(vr * vc) * 8ull * ((I == J || !mirror) ? 1ull : 2ull);
      }
    }
    if (mt == 0 && my_tiles) {
      atomicAdd(&counters[CNT_TILES_TOUCHED], my_tiles);
      atomicAdd(&counters[CNT_S_BYTES], my_bytes);
      atomicAdd(&counters[CNT_PANEL_BYTES],
                my_tiles * 4ull * (unsigned long long)(k1g - k0g) * PT * sizeof(float));
    }
  }
  if (!ok) abort_flag = 1;
  __syncthreads();
  if (tid == 0 && abort_flag)
    atomicExch(&counters[CNT_STATUS], (unsigned long long)SR_ERR_TIMEOUT);
}

constexpr int KC_F32 = 16;
constexpr int KC_F64 = 16;

}  // namespace

int s_update_grid(int s_prec, int num_sms, bool ws) {
  return num_sms * ((s_prec == 64 || ws) ? 1 : 2);
}

void launch_s_update(void* S, int s_prec, int64_t ld, const void* P, int K1, const uint32_t* tiles,
                     const int* ntiles, const uint64_t* mXi, const uint64_t* mEta, int k0, int k1,
                     int use_masks, int n, int64_t* counters, int grid, cudaStream_t st,
                     long long ws_wait_limit, int upper) {
  const int mirror = upper ? 0 : 1;
  if (s_prec == 64) {
    const size_t smem = (4ull * KC_F64 * PT + (size_t)PT * DP) * sizeof(double);
    static std::atomic<unsigned long long> attr64{0};
    smem_attr_once((const void*)k_s_update<double, KC_F64, 1, OneGraphTiles<double>>, (int)smem, attr64);
    OneGraphTiles<double> src{(double*)S, ld,        (const double*)P, tiles, mXi,
                              mEta,       use_masks, n,                mirror};
    k_s_update<double, KC_F64, 1><<<grid, 256, smem, st>>>(src, K1, ntiles, k0, k1,
                                                             (unsigned long long*)counters);
  } else if (ws_wait_limit > 0) {
    const size_t smem = (4ull * WS_KC * PT + 2ull * PT * DP) * sizeof(float);
    static std::atomic<unsigned long long> attr_ws{0};
    smem_attr_once((const void*)k_s_update_ws, (int)smem, attr_ws);
    k_s_update_ws<<<grid, WS_THREADS, smem, st>>>((float*)S, ld, (const float*)P, K1, tiles, ntiles,
                                                  mXi, mEta, k0, k1, use_masks, n, mirror,
                                                  ws_wait_limit,
                                                  (unsigned long long*)counters);
  } else {
    const size_t smem = (4ull * KC_F32 * PT + (size_t)PT * DP) * sizeof(float);
    static std::atomic<unsigned long long> attr32{0};
    smem_attr_once((const void*)k_s_update<float, KC_F32, 2, OneGraphTiles<float>>, (int)smem, attr32);
    OneGraphTiles<float> src{(float*)S, ld, (const float*)P, tiles, mXi, mEta, use_masks, n, mirror};
    k_s_update<float, KC_F32, 2><<<grid, 256, smem, st>>>(src, K1, ntiles, k0, k1,
                                                            (unsigned long long*)counters);
  }
}

void launch_s_update_multi(int s_prec, const MultiGraphDesc* descs, const uint64_t* tiles,
                           const int* ntiles, int K1, int64_t* counters, int grid,
                           cudaStream_t st) {
  if (s_prec == 64) {
    const size_t smem = (4ull * KC_F64 * PT + (size_t)PT * DP) * sizeof(double);
    static std::atomic<unsigned long long> attr{0};
    smem_attr_once((const void*)k_s_update<double, KC_F64, 1, ManyGraphTiles<double>>, (int)smem, attr);
    ManyGraphTiles<double> src{descs, tiles};
    k_s_update<double, KC_F64, 1><<<grid, 256, smem, st>>>(src, K1, ntiles, 0, K1,
                                                             (unsigned long long*)counters);
  } else {
    const size_t smem = (4ull * KC_F32 * PT + (size_t)PT * DP) * sizeof(float);
    static std::atomic<unsigned long long> attr{0};
    smem_attr_once((const void*)k_s_update<float, KC_F32, 2, ManyGraphTiles<float>>, (int)smem, attr);
    ManyGraphTiles<float> src{descs, tiles};
    k_s_update<float, KC_F32, 2><<<grid, 256, smem, st>>>(src, K1, ntiles, 0, K1,
                                                            (unsigned long long*)counters);
  }
}

}  // namespace sr
