// Many independent graphs advanced together.  A round applies one rank-one
// update (Alg 1 with the cases of Thm 3 / Thm 9) to every graph that has one
// left: k_multi_prep runs one CTA per graph and does everything before the S
// pass - the graph patch (Thm 1), the rows of S that gamma reads, gamma, the
// K steps of the recurrence on the new graph (Eq. 16a), the affected-area
// masks (Thm 4) and the graph's affected tile pairs - with only CTA-level
// synchronisation, so graphs of any size progress independently; one S pass
// (k_supdate.cu, ManyGraphTiles) then covers the tile pairs of all graphs.
// Arithmetic is in the precision of S (row j of gamma in FP64).
#include "sr_internal.h"

namespace sr {

namespace {

constexpr int MT = 512;    // threads of a CTA
constexpr int RB = MT;     // rows per gathered block (one row per thread)
constexpr int MNT = 512;   // tiles a graph may have (n <= 65536)
constexpr int NW = MT / 32;

template <typename V>
struct MultiSmem {
  int64_t start[RB];
  int len[RB];
  int off[RB + 1];
  int wsum[NW];
  V acc[2][RB];
  unsigned long long mx[MNT];
  unsigned long long me[MNT];
};

// Rows [row0, row0 + RB) of the in-adjacency: extents and the exclusive scan
// of their lengths (rows at or beyond nrows are empty).
template <typename V>
__device__ __forceinline__ void block_rows_load(const DevAdj& in, int row0, int nrows,
                                                MultiSmem<V>& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int a = row0 + tid;
  int L = 0;
  int64_t st = 0;
  if (a < nrows) {
    st = __ldcg(in.start + a);
    L = __ldcg(in.len + a);
  }
  sm.start[tid] = st;
  sm.len[tid] = L;
  int incl = L;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sm.wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int v = (lane < NW) ? sm.wsum[lane] : 0;
    int w = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) sm.wsum[lane] = w - v;
    if (lane == NW - 1) sm.off[RB] = w;
  }
  __syncthreads();
  sm.off[tid] = sm.wsum[warp] + incl - L;
  __syncthreads();
}

template <int NV, typename V>
__device__ __forceinline__ void mseg_flush(int key, V (&val)[NV], V (*acc)[RB]) {
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

// sm.acc[v][r] = sum over the in-neighbours b of block row r of gather(v, b):
// the block's nonzeros are flattened and split into one contiguous run per
// thread; rows inside a run are stored directly, the first and last row of a
// run are combined across lanes.
template <int NV, typename V, typename Gf>
__device__ __forceinline__ void rows_gather(MultiSmem<V>& sm, const int32_t* __restrict__ col,
                                            Gf gather) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int v = 0; v < NV; ++v) sm.acc[v][tid] = V(0);
  __syncthreads();
  const int total = sm.off[RB];
  const int per = (total + MT - 1) / MT;
  const int e0 = tid * per;
  const int e1 = min(total, e0 + per);
  int r_first = -1, r_last = -1;
  V pf[NV], pl[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) pf[v] = pl[v] = V(0);
  if (e0 < e1) {
    int lo = 0, hi = RB;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (sm.off[mid] <= e0) lo = mid; else hi = mid;
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
          while (ee >= sm.off[rc + 1]) ++rc;
          rr[q] = rc;
          bb[q] = __ldcg(col + sm.start[rc] + (ee - sm.off[rc]));
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
            for (int v = 0; v < NV; ++v) sm.acc[v][r] = part[v];
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
  mseg_flush<NV, V>(r_first, pf, sm.acc);
  mseg_flush<NV, V>(r_last, pl, sm.acc);
  __syncthreads();
}

__device__ void multi_patch(const PatchOp* __restrict__ ops, int64_t begin, int64_t end,
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

// ORs `bit` into the mask word of the tile of this warp's 32 rows when any of
// them has pred set (row0 is a multiple of 32, so a warp's rows share a tile).
__device__ __forceinline__ void warp_mask(bool pred, int a, unsigned long long bit,
                                          unsigned long long* words) {
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if ((threadIdx.x & 31) == 0 && b) atomicOr(&words[a / PT], bit);
}

template <typename V>
__global__ void __launch_bounds__(MT, 2)
    k_multi_prep(const MultiGraphDesc* __restrict__ descs, const MultiStep* __restrict__ steps,
                 const int* __restrict__ count, const int32_t* __restrict__ srcs,
                 const PatchOp* __restrict__ ops, double C, int K, int aff,
                 uint64_t* __restrict__ tiles, int* __restrict__ ntiles) {
  __shared__ MultiSmem<V> sm;
  if ((int)blockIdx.x >= *count) return;
  const int tid = threadIdx.x;
  const MultiStep stp = steps[blockIdx.x];
  const MultiGraphDesc q = descs[stp.g];
  const int K1 = K + 1;
  const int nT = (stp.n_after + PT - 1) / PT;
  const int nrows = nT * PT;
  const V* __restrict__ S = static_cast<const V*>(q.S);
  V* P = static_cast<V*>(q.P);
  V* sI = static_cast<V*>(q.sI);
  V* sJ = static_cast<V*>(q.sJ);
  const int32_t* __restrict__ I = srcs + stp.src_off;
  const int j = stp.j, delta = stp.delta, op = stp.op, d_j = stp.d_j;
  const V Cv = (V)C;
  auto pidx = [K1](int64_t a, int which, int k) -> int64_t {
    return (((a / PT) * 2 + which) * (int64_t)K1 + k) * PT + (a % PT);
  };

  multi_patch(ops, stp.op_begin, stp.op_end, q.in, q.out);
  // rows of the current S that gamma reads
  for (int a = tid; a < nrows; a += MT) {
    V vI = V(0);
    for (int t = 0; t < delta; ++t) vI += S[(int64_t)I[t] * q.ld + a];
    sI[a] = vI;
    sJ[a] = S[(int64_t)j * q.ld + a];
  }
  for (int T = tid; T < nT; T += MT) sm.mx[T] = sm.me[T] = 0ull;
  __syncthreads();

  // gamma on the new graph, row j corrected to the old row (see k_prep.cu)
  for (int row0 = 0; row0 < nrows; row0 += RB) {
    block_rows_load(q.in, row0, nrows, sm);
    rows_gather<1, V>(sm, q.in.col, [&](int, int b) { return __ldcg(sI + b); });
    const int a = row0 + tid;
    bool nz = false;
    if (a < nrows) {
      const int len = sm.len[tid];
      const double dl = (double)delta;
      V g;
      if (a == j) {
        double S_II = 0.0;
        for (int u = 0; u < delta; ++u) S_II += (double)__ldcg(sI + I[u]);
        const double S_jj = (double)__ldcg(sJ + j);
        const double wj =
            (d_j > 0) ? ((double)sm.acc[0][tid] - (double)op * S_II) / (dl * (double)d_j) : 0.0;
        const double lam = S_II / (dl * dl) + S_jj / C - 2.0 * wj - 1.0 / C + 1.0;
        double gd;
        if (op > 0) {
          if (d_j == 0) {
            gd = wj + S_II / (2.0 * dl * dl);
          } else {
            const double dd = (double)d_j + dl;
            gd = (dl / dd) * (wj - S_jj / C + lam * dl / (2.0 * dd) + 1.0 / C - 1.0);
          }
        } else {
          if (d_j == delta) {
            gd = -wj + S_II / (2.0 * dl * dl);
          } else {
            const double dd = (double)d_j - dl;
            gd = (dl / dd) * (S_jj / C - wj + lam * dl / (2.0 * dd) - 1.0 / C + 1.0);
          }
        }
        g = (V)gd;
      } else {
        const V w = (len > 0) ? sm.acc[0][tid] / ((V)delta * (V)len) : V(0);
        const V sJa = __ldcg(sJ + a);
        if (op > 0) {
          g = (d_j == 0) ? w : ((V)delta / (V)(d_j + delta)) * (w - sJa / Cv);
        } else {
          g = (d_j == delta) ? -w : ((V)delta / (V)(d_j - delta)) * (sJa / Cv - w);
        }
      }
      P[pidx(a, 0, 0)] = (a == j) ? Cv : V(0);
      P[pidx(a, 1, 0)] = g;
      nz = (g != V(0));
    }
    warp_mask(nz, a, 1ull, sm.me);
    __syncthreads();
  }
  if (tid == 0) sm.mx[j / PT] |= 1ull;
  __syncthreads();

  // K steps: xi_{k+1} = C Q xi_k, eta_{k+1} = Q eta_k
  for (int k = 0; k < K; ++k) {
    const unsigned long long bit = 1ull << ((k + 1) & 63);
    for (int row0 = 0; row0 < nrows; row0 += RB) {
      block_rows_load(q.in, row0, nrows, sm);
      rows_gather<2, V>(sm, q.in.col, [&](int v, int b) { return __ldcg(P + pidx(b, v, k)); });
      const int a = row0 + tid;
      bool nx = false, ne = false;
      if (a < nrows) {
        const int len = sm.len[tid];
        const V inv = (len > 0) ? V(1) / (V)len : V(0);
        const V x = Cv * sm.acc[0][tid] * inv;
        const V y = sm.acc[1][tid] * inv;
        P[pidx(a, 0, k + 1)] = x;
        P[pidx(a, 1, k + 1)] = y;
        nx = (x != V(0));
        ne = (y != V(0));
      }
      warp_mask(nx, a, bit, sm.mx);
      warp_mask(ne, a, bit, sm.me);
      __syncthreads();
    }
  }

  for (int T = tid; T < nT; T += MT) {
    q.mXi[T] = sm.mx[T];
    q.mEta[T] = sm.me[T];
  }
  // this graph's tile pairs
  const int lane = tid & 31;
  const uint64_t gk = (uint64_t)(uint32_t)stp.g << 32;
  for (int Ti = 0; Ti < nT; ++Ti) {
    const unsigned long long xi = sm.mx[Ti], ei = sm.me[Ti];
    for (int J0 = Ti; J0 < nT; J0 += MT) {
      const int Tj = J0 + tid;
      bool act = false;
      if (Tj < nT) act = !aff || (((xi & sm.me[Tj]) | (ei & sm.mx[Tj])) != 0ull);
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if (m == 0) continue;
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(ntiles, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (act)
        tiles[base + __popc(m & ((1u << lane) - 1u))] =
            gk | ((uint64_t)Ti << 16) | (uint64_t)Tj;
    }
  }
}

}  // namespace

void launch_multi_prep(int s_prec, const MultiGraphDesc* descs, const MultiStep* steps,
                       const int* count, int grid, const int32_t* srcs, const PatchOp* ops,
                       double C, int K, int aff, uint64_t* tiles, int* ntiles, cudaStream_t st) {
  if (grid <= 0) return;
  if (s_prec == 64)
    k_multi_prep<double><<<grid, MT, 0, st>>>(descs, steps, count, srcs, ops, C, K, aff, tiles,
                                              ntiles);
  else
    k_multi_prep<float><<<grid, MT, 0, st>>>(descs, steps, count, srcs, ops, C, K, aff, tiles,
                                             ntiles);
}

}  // namespace sr
