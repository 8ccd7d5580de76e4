// Everything one rank-one (sink-block) update does before its S pass, in one
// cooperative launch:
//   phase 0  graph patch (Thm 1: row j of the in-adjacency gains / loses the
//            sources I), and the rows of the current S that gamma reads,
//            sI = sum_t S[I_t, *] and sJ = S[j, *], with the panels of updates
//            whose S pass is still pending added in;
//   phase 1  gamma (Thm 3 insert, Thm 9 delete, Table 2 sink blocks) written
//            as eta_0, with xi_0 = C e_j;
//   phase 2  the K steps of the recurrence on the new graph (Eq. 16a),
//            xi_{k+1} = C Q xi_k, eta_{k+1} = Q eta_k;
//   phase 3  the affected-area mask words of every tile (Thm 4) and the list
//            of affected tile pairs of the S pass.
// Phases are separated by a bounded grid barrier.  Each CTA owns the tiles
// blockIdx.x + t * gridDim.x; their row extents and up to `cap` column
// indices stay in shared memory for all K steps, so a step is one gather of
// the previous column plus one barrier.  Arithmetic is in the precision of S:
// FP64 work on GB300 runs at a small fraction of the FP32 rate, and the FP32
// path stores S and the panels in FP32 anyway.
//
// gamma needs w = (1/delta) Q_old S_{*,I}; only row j of Q changes, so the
// kernel gathers on the patched graph and corrects row j by the sources it
// gained or lost: sum over old in-neighbours = sum over new - op * S_II.
#include <algorithm>

#include "sr_internal.h"

namespace sr {

namespace {

constexpr int PG = 512;     // threads of a prep CTA
constexpr int PREP_MT = 8;  // tiles one CTA may own

struct alignas(16) PrepTile {
  int64_t start[PT];
  int len[PT];
  int off[PT + 1];
  int cbase;          // first cached column index of this tile in the CTA's cache
  int clen;           // flattened nonzeros [0, clen) of the tile are cached
  int pad_;
  uint64_t mask[2];   // this update's AFF words: bit k % 64 set if xi_k / eta_k has a
                      // nonzero in the tile
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on a monotonically increasing arrival counter: barrier number
// b of a launch returns once b * gridDim.x arrivals are visible.  Bounded:
// false after `limit` polls.
__device__ __forceinline__ bool prep_barrier(unsigned int* count, unsigned int target,
                                             long long limit, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    int ok = 1;
    long long it = 0;
    while (ld_acquire(count) < target) {
      if (++it > limit) {
        ok = 0;
        break;
      }
      __nanosleep(16);
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

template <int NV, typename V>
__device__ __forceinline__ void seg_flush(int key, V (&val)[NV], V (*acc)[PT]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int k2 = __shfl_down_sync(0xffffffffu, key, o);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const V x = __shfl_down_sync(0xffffffffu, val[v], o);
      if (lane + o < 32 && k2 == key) val[v] += x;
    }
  }
  const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kprev != key)) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      if (val[v] != V(0)) atomicAdd(&acc[v][key], val[v]);
  }
}

// acc[v][r] = sum over the in-neighbours b of row r of tile `tr` of gather(v, b).
// The tile's nonzeros are flattened and split into one contiguous run per
// thread (hub rows spread over the whole CTA); rows wholly inside a run are
// stored directly, the first and last row of a run are combined across lanes
// by seg_flush.  Column indices come from the shared cache where cached.
template <int NV, typename V, typename Gf>
__device__ __forceinline__ void prep_gather(const PrepTile& tr, const int* __restrict__ cc,
                                            const int32_t* __restrict__ col, Gf gather,
                                            V (*acc)[PT]) {
  const int tid = threadIdx.x;
  if (tid < PT) {
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v][tid] = V(0);
  }
  __syncthreads();
  const int total = tr.off[PT];
  const int per = (total + PG - 1) / PG;
  const int e0 = tid * per;
  const int e1 = min(total, e0 + per);
  int r_first = -1, r_last = -1;
  V pf[NV], pl[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) pf[v] = pl[v] = V(0);
  if (e0 < e1) {
    int lo = 0, hi = PT;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tr.off[mid] <= e0) lo = mid; else hi = mid;
    }
    int r = lo;
    r_first = r;
    V part[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v] = V(0);
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
          bb[q] = (ee < tr.clen) ? cc[tr.cbase + ee]
                                 : __ldcg(col + tr.start[rc] + (ee - tr.off[rc]));
        } else {
          rr[q] = -1;
          bb[q] = 0;
        }
      }
      V xv[NV][B];
#pragma unroll
      for (int q = 0; q < B; ++q)
#pragma unroll
        for (int v = 0; v < NV; ++v) xv[v][q] = (rr[q] >= 0) ? gather(v, bb[q]) : V(0);
#pragma unroll
      for (int q = 0; q < B; ++q) {
        if (rr[q] < 0) break;
        if (rr[q] != r) {
          if (r == r_first) {
#pragma unroll
            for (int v = 0; v < NV; ++v) pf[v] = part[v];
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v][r] = part[v];
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) part[v] = V(0);
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
  seg_flush<NV, V>(r_first, pf, acc);
  seg_flush<NV, V>(r_last, pl, acc);
  __syncthreads();
}

__device__ void prep_patch(const PatchOp* __restrict__ ops, int64_t begin, int64_t end,
                           const DevAdj& in, const DevAdj& out) {
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

template <typename V>
__global__ void __launch_bounds__(PG, 1) k_prep(PrepParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ V acc[2][PT];
  __shared__ V red[4][2][PT];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int nT = p.nT;
  const int mt = (nT + G - 1) / G;
  PrepTile* tr = reinterpret_cast<PrepTile*>(dsm);
  int* cc = reinterpret_cast<int*>(tr + mt);
  V* coef = reinterpret_cast<V*>(cc + p.cap);
  const V* __restrict__ S = static_cast<const V*>(p.S);
  V* P = static_cast<V*>(p.P);
  V* sI = static_cast<V*>(p.sI);
  V* sJ = static_cast<V*>(p.sJ);
  const int64_t ldk = p.ldk;
  auto pidx = [ldk](int64_t a, int which, int k) -> int64_t {
    return (((a / PT) * 2 + which) * ldk + k) * PT + (a % PT);
  };
  const int np = p.npend;
  const int koff = p.koff;
  const V Cv = (V)p.C;
  unsigned int nb = 0;
  bool alive = true;

  // ---- phase 0: patch (CTA 0) and the rows sI, sJ of the current S
  if (blockIdx.x == 0) {
    if (p.op_end > p.op_begin) prep_patch(p.ops, p.op_begin, p.op_end, p.in, p.out);
    if (tid == 0 && p.tiles) *p.ntiles = 0;
  }
  if (np > 0) {
    // c_x[q] = sum_t xi_q[I_t], c_e[q] = sum_t eta_q[I_t]; the same at j
    for (int q = tid; q < np; q += PG) {
      V cx = V(0), ce = V(0);
      for (int t = 0; t < p.delta; ++t) {
        const int64_t x = p.I[t];
        cx += P[pidx(x, 0, q)];
        ce += P[pidx(x, 1, q)];
      }
      coef[q] = cx;
      coef[np + q] = ce;
      coef[2 * np + q] = P[pidx(p.j, 0, q)];
      coef[3 * np + q] = P[pidx(p.j, 1, q)];
    }
    __syncthreads();
  }
  {
    const int r = tid & (PT - 1), part = tid >> 7;
    for (int t = 0; t < mt; ++t) {
      const int T = blockIdx.x + t * G;
      if (T >= nT) break;
      const int64_t a = (int64_t)T * PT + r;
      V vI = V(0), vJ = V(0);
      for (int u = part; u < p.delta; u += 4) vI += S[(int64_t)p.I[u] * p.ld + a];
      if (part == 3) vJ = S[(int64_t)p.j * p.ld + a];
      // S_cur[x, a] = S[x, a] + sum_q xi_q[x] eta_q[a] + eta_q[x] xi_q[a]
      for (int q = part; q < np; q += 4) {
        const V xa = P[pidx(a, 0, q)];
        const V ea = P[pidx(a, 1, q)];
        vI += coef[q] * ea + coef[np + q] * xa;
        vJ += coef[2 * np + q] * ea + coef[3 * np + q] * xa;
      }
      red[part][0][r] = vI;
      red[part][1][r] = vJ;
      __syncthreads();
      if (tid < PT) {
        sI[a] = (red[0][0][r] + red[1][0][r]) + (red[2][0][r] + red[3][0][r]);
        sJ[a] = (red[0][1][r] + red[1][1][r]) + (red[2][1][r] + red[3][1][r]);
      }
      __syncthreads();
    }
  }
  alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);

  // ---- phase 1: tile rows of the new graph, column cache, gamma
  if (alive) {
    int cbase = 0;
    for (int t = 0; t < mt; ++t) {
      const int T = blockIdx.x + t * G;
      if (T >= nT) break;
      PrepTile& tt = tr[t];
      if (tid < PT) {
        tt.start[tid] = __ldcg(p.in.start + (int64_t)T * PT + tid);
        tt.len[tid] = __ldcg(p.in.len + (int64_t)T * PT + tid);
      }
      __syncthreads();
      if (tid < 32) {
        int v[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] = tt.len[tid * 4 + q];
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
          tt.off[tid * 4 + q] = run;
          run += v[q];
        }
        if (tid == 31) {
          tt.off[PT] = incl;
          tt.cbase = cbase;
          tt.clen = max(0, min(incl, p.cap - cbase));
          tt.mask[0] = tt.mask[1] = 0ull;
        }
      }
      __syncthreads();
      const int clen = tt.clen;
      {
        const int lane = tid & 31, warp = tid >> 5;
        for (int r = warp; r < PT; r += PG / 32) {
          const int o = tt.off[r];
          if (o >= clen) break;
          const int L = min(tt.len[r], clen - o);
          for (int e = lane; e < L; e += 32) cc[cbase + o + e] = __ldcg(p.in.col + tt.start[r] + e);
        }
      }
      cbase += clen;
      __syncthreads();
      prep_gather<1, V>(tt, cc, p.in.col, [&](int, int b) { return __ldcg(sI + b); }, acc);
      int pe = 0;
      if (tid < PT) {
        const int64_t a = (int64_t)T * PT + tid;
        const int len = tt.len[tid];
        const double dl = (double)p.delta;
        V g;
        if (a == p.j) {
          // row j: lambda (Eq. 29b) and w_j on the old row j, in FP64
          double S_II = 0.0;
          for (int u = 0; u < p.delta; ++u) S_II += (double)__ldcg(sI + p.I[u]);
          const double S_jj = (double)__ldcg(sJ + p.j);
          const double C = p.C;
          const double wj =
              (p.d_j > 0) ? ((double)acc[0][tid] - (double)p.op * S_II) / (dl * (double)p.d_j)
                          : 0.0;
          const double lam = S_II / (dl * dl) + S_jj / C - 2.0 * wj - 1.0 / C + 1.0;
          double gd;
          if (p.op > 0) {
            if (p.d_j == 0) {
              gd = wj + S_II / (2.0 * dl * dl);
            } else {
              const double dd = (double)p.d_j + dl;
              gd = (dl / dd) * (wj - S_jj / C + lam * dl / (2.0 * dd) + 1.0 / C - 1.0);
            }
          } else {
            if (p.d_j == p.delta) {
              gd = -wj + S_II / (2.0 * dl * dl);
            } else {
              const double dd = (double)p.d_j - dl;
              gd = (dl / dd) * (S_jj / C - wj + lam * dl / (2.0 * dd) - 1.0 / C + 1.0);
            }
          }
          g = (V)gd;
        } else {
          const V w = (len > 0) ? acc[0][tid] / ((V)p.delta * (V)len) : V(0);
          const V sJa = __ldcg(sJ + a);
          if (p.op > 0) {
            if (p.d_j == 0) {
              g = w;
            } else {
              const V dd = (V)(p.d_j + p.delta);
              g = ((V)p.delta / dd) * (w - sJa / Cv);
            }
          } else {
            if (p.d_j == p.delta) {
              g = -w;
            } else {
              const V dd = (V)(p.d_j - p.delta);
              g = ((V)p.delta / dd) * (sJa / Cv - w);
            }
          }
        }
        P[pidx(a, 0, koff)] = (a == p.j) ? Cv : V(0);
        P[pidx(a, 1, koff)] = g;
        pe = (g != V(0));
      }
      const int any_e = __syncthreads_or(pe);
      if (tid == 0) {
        tt.mask[0] = (T == p.j / PT) ? 1ull : 0ull;
        tt.mask[1] = any_e ? 1ull : 0ull;
      }
    }
    if (p.K > 0) alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
  }

  // ---- phase 2: K steps of the recurrence on the new graph
  for (int k = 0; alive && k < p.K; ++k) {
    const int kc = koff + k;
    for (int t = 0; t < mt; ++t) {
      const int T = blockIdx.x + t * G;
      if (T >= nT) break;
      PrepTile& tt = tr[t];
      prep_gather<2, V>(tt, cc, p.in.col,
                        [&](int v, int b) { return __ldcg(P + pidx(b, v, kc)); }, acc);
      int px = 0, pe = 0;
      if (tid < PT) {
        const int len = tt.len[tid];
        const V inv = (len > 0) ? V(1) / (V)len : V(0);
        const V x = Cv * acc[0][tid] * inv;
        const V y = acc[1][tid] * inv;
        const int64_t a = (int64_t)T * PT + tid;
        P[pidx(a, 0, kc + 1)] = x;
        P[pidx(a, 1, kc + 1)] = y;
        px = (x != V(0));
        pe = (y != V(0));
      }
      const int ax = __syncthreads_or(px);
      const int ae = __syncthreads_or(pe);
      if (tid == 0) {
        const uint64_t bit = 1ull << ((k + 1) & 63);
        if (ax) tt.mask[0] |= bit;
        if (ae) tt.mask[1] |= bit;
      }
    }
    if (k + 1 < p.K) alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
  }

  // ---- phase 3: mask words and the affected tile pairs
  if (alive) {
    __syncthreads();
    if (tid == 0) {
      for (int t = 0; t < mt; ++t) {
        const int T = blockIdx.x + t * G;
        if (T >= nT) break;
        p.mXi[T] = tr[t].mask[0];
        p.mEta[T] = tr[t].mask[1];
        if (p.pXi) {
          if (tr[t].mask[0]) p.pXi[T] = 1ull;
          if (tr[t].mask[1]) p.pEta[T] = 1ull;
        }
      }
    }
    if (p.tiles) {
      alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
      if (alive) {
        const unsigned long long* mx = reinterpret_cast<const unsigned long long*>(p.mXi);
        const unsigned long long* me = reinterpret_cast<const unsigned long long*>(p.mEta);
        const int lane = tid & 31;
        for (int I = blockIdx.x; I < nT; I += G) {
          const unsigned long long xi = __ldcg(mx + I), ei = __ldcg(me + I);
          for (int J0 = I; J0 < nT; J0 += PG) {
            const int J = J0 + tid;
            bool act = false;
            if (J < nT) act = (p.tile_mode == 0) || (((xi & __ldcg(me + J)) | (ei & __ldcg(mx + J))) != 0ull);
            const unsigned mask = __ballot_sync(0xffffffffu, act);
            if (mask == 0) continue;
            const int leader = __ffs(mask) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(p.ntiles, __popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (act)
              p.tiles[base + __popc(mask & ((1u << lane) - 1u))] = ((uint32_t)I << 16) | (uint32_t)J;
          }
        }
      }
    }
  }

  // every CTA has left every barrier once all have arrived here: the last
  // one resets the barrier state for the next launch
  __syncthreads();
  if (tid == 0) {
    if (!alive) atomicExch(&p.counters[CNT_STATUS], (unsigned long long)SR_ERR_TIMEOUT);
    __threadfence();
    const unsigned int e = atomicAdd(p.bar + 1, 1u) + 1u;
    if (e == (unsigned int)G) {
      atomicExch(p.bar, 0u);
      atomicExch(p.bar + 1, 0u);
    }
  }
}

template <typename V>
size_t prep_smem(int mt, int cap, int npend_max) {
  return (size_t)mt * sizeof(PrepTile) + (size_t)cap * sizeof(int) +
         (size_t)4 * npend_max * sizeof(V);
}

}  // namespace

int launch_prep(const PrepParams& prm, int s_prec, int npend_max, int num_sms, int max_ctas,
                cudaStream_t st) {
  if (prm.nT <= 0) return 0;
  const size_t smem = (s_prec == 64) ? prep_smem<double>(PREP_MT, prm.cap, npend_max)
                                     : prep_smem<float>(PREP_MT, prm.cap, npend_max);
  const void* fn = (s_prec == 64) ? (const void*)k_prep<double> : (const void*)k_prep<float>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PG, smem) != cudaSuccess ||
      per_sm <= 0)
    return 1;
  int grid = std::min(prm.nT, per_sm * num_sms);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  if ((prm.nT + grid - 1) / grid > PREP_MT) return 2;
  if (prm.npend > npend_max) return 1;
  PrepParams a = prm;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel(fn, grid, PG, args, smem, st) != cudaSuccess) return 1;
  return 0;
}

}  // namespace sr
