// Many independent graphs advanced together.  A round applies one rank-one
// update (Alg 1 with the cases of Thm 3 / Thm 9) to every graph that has one
// left: k_multi_prep runs one CTA per graph and does everything before the S
// pass - the graph patch (Thm 1), the rows of S that gamma reads, gamma, the
// K steps of the recurrence on the new graph (Eq. 16a), the affected-area
// masks (Thm 4) and the graph's affected tile pairs - with only CTA-level
// synchronisation, so graphs of any size progress independently; one S pass
// (k_supdate.cu, ManyGraphTiles) then covers the tile pairs of all graphs.
//
// Graphs whose (xi, eta) vectors fit in shared memory keep them there: a
// step gathers from shared memory (rows of up to LONG nonzeros one per
// thread with 16-byte column loads, longer rows one per warp) and writes the
// next vectors there and into the panels.  Larger graphs gather from the
// panels in global memory in blocks of rows.
// Arithmetic is in the precision of S (lambda and row j of gamma in FP64).
#include "sr_internal.h"

namespace sr {

namespace {

constexpr int MT = 1024;   // threads of a CTA
constexpr int RB = MT;     // rows per gathered block of the global path
constexpr int MNT = 512;   // tiles a graph may have (n <= 65536)
constexpr int NW = MT / 32;
constexpr int LONG = 32;   // longer rows are gathered by a whole warp
constexpr int SMEM_BYTES = 200 * 1024;  // dynamic shared memory of a CTA

template <typename V>
struct V2 {
  V x, y;
};

template <typename V>
struct MultiSmem {
  int64_t start[RB];
  int len[RB];
  int off[RB + 1];
  int wsum[NW];
  V acc[2][RB];
};

// rows of the shared-memory path: two (xi, eta) vectors and the row extents
template <typename V>
constexpr int smem_rows() {
  return (SMEM_BYTES / (2 * (int)sizeof(V2<V>) + 8)) / PT * PT;
}

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
// them has pred set (a warp's rows are 32 consecutive rows of one tile).
__device__ __forceinline__ void warp_mask(bool pred, int a, unsigned long long bit,
                                          unsigned long long* words) {
  const unsigned b = __ballot_sync(0xffffffffu, pred);
  if ((threadIdx.x & 31) == 0 && b) atomicOr(&words[a / PT], bit);
}

// One update's constants.
struct StepConst {
  int j, delta, op, d_j;
  double C;
};

// gamma_a (Thm 3 / Thm 9 / Table 2) from y = sum over the NEW in-neighbours
// of a of sI, len = new in-degree of a, sJa = S[j, a]; S_II for row j.
template <typename V>
__device__ __forceinline__ V gamma_row(const StepConst& c, int a, V y, int len, V sJa,
                                       double S_II) {
  const double dl = (double)c.delta;
  if (a == c.j) {
    const double S_jj = (double)sJa;
    const double C = c.C;
    const double wj =
        (c.d_j > 0) ? ((double)y - (double)c.op * S_II) / (dl * (double)c.d_j) : 0.0;
    const double lam = S_II / (dl * dl) + S_jj / C - 2.0 * wj - 1.0 / C + 1.0;
    double gd;
    if (c.op > 0) {
      if (c.d_j == 0) {
        gd = wj + S_II / (2.0 * dl * dl);
      } else {
        const double dd = (double)c.d_j + dl;
        gd = (dl / dd) * (wj - S_jj / C + lam * dl / (2.0 * dd) + 1.0 / C - 1.0);
      }
    } else {
      if (c.d_j == c.delta) {
        gd = -wj + S_II / (2.0 * dl * dl);
      } else {
        const double dd = (double)c.d_j - dl;
        gd = (dl / dd) * (S_jj / C - wj + lam * dl / (2.0 * dd) - 1.0 / C + 1.0);
      }
    }
    return (V)gd;
  }
  const V Cv = (V)c.C;
  const V w = (len > 0) ? y / ((V)c.delta * (V)len) : V(0);
  if (c.op > 0) return (c.d_j == 0) ? w : ((V)c.delta / (V)(c.d_j + c.delta)) * (w - sJa / Cv);
  return (c.d_j == c.delta) ? -w : ((V)c.delta / (V)(c.d_j - c.delta)) * (sJa / Cv - w);
}

// Shared-memory path: for every row a < nrows, out(a, kind, active, sx, sy)
// with (sx, sy) = the sum over the in-neighbours b of a of vec[b].  Rows of
// at most LONG nonzeros: one thread each, two rows at a time, the first 8
// columns by two 16-byte loads (rows start 16-byte aligned in the pool);
// every lane of the warp calls out with kind 0 (active = the lane owns a
// short row).  Longer rows: one warp each; the warp calls out with kind 1,
// active on lane 0 only.  Every row is active exactly once.
template <typename V, typename Out>
__device__ __forceinline__ void smem_pass(const V2<V>* vec, const int* st32, const int* ln,
                                          const int32_t* __restrict__ col, int nrows, Out out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int a0 = tid; a0 < nrows; a0 += 2 * MT) {
    int L[2], s[2];
    int4 c0[2], c1[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int a = a0 + g * MT;
      L[g] = (a < nrows) ? ln[a] : 0;
      s[g] = (a < nrows) ? st32[a] : 0;
      if (L[g] > LONG) L[g] = -1;
      if (L[g] > 0) c0[g] = __ldcg(reinterpret_cast<const int4*>(col + s[g]));
      if (L[g] > 4) c1[g] = __ldcg(reinterpret_cast<const int4*>(col + s[g] + 4));
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int a = a0 + g * MT;
      V sx = V(0), sy = V(0);
      if (L[g] > 0) {
        const int cs[8] = {c0[g].x, c0[g].y, c0[g].z, c0[g].w, c1[g].x, c1[g].y, c1[g].z, c1[g].w};
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (e < L[g]) {
            const V2<V> v = vec[cs[e]];
            sx += v.x;
            sy += v.y;
          }
        for (int e0 = 8; e0 < L[g]; e0 += 4) {
          const int4 c = __ldcg(reinterpret_cast<const int4*>(col + s[g] + e0));
          const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (e0 + e < L[g]) {
              const V2<V> v = vec[cc[e]];
              sx += v.x;
              sy += v.y;
            }
        }
      }
      out(a, 0, a < nrows && L[g] >= 0, sx, sy);
    }
  }
  // long rows: one warp each
  for (int a = warp; a < nrows; a += NW) {
    const int L = ln[a];
    if (L <= LONG) continue;
    const int s = st32[a];
    V sx = V(0), sy = V(0);
    for (int e0 = 4 * lane; e0 < L; e0 += 128) {
      const int4 c = __ldcg(reinterpret_cast<const int4*>(col + s + e0));
      const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e0 + e < L) {
          const V2<V> v = vec[cc[e]];
          sx += v.x;
          sy += v.y;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    out(a, 1, lane == 0, sx, sy);
  }
}

template <typename V>
__global__ void __launch_bounds__(MT, 1)
    k_multi_prep(const MultiGraphDesc* __restrict__ descs, const MultiStep* __restrict__ steps,
                 const int* __restrict__ count, const int32_t* __restrict__ srcs,
                 const PatchOp* __restrict__ ops, double C, int K, int aff,
                 uint64_t* __restrict__ tiles, int* __restrict__ ntiles) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ unsigned long long mx[MNT], me[MNT];
  __shared__ double s_SII;
  if ((int)blockIdx.x >= *count) return;
  const int tid = threadIdx.x;
  const MultiStep stp = steps[blockIdx.x];
  const MultiGraphDesc q = descs[stp.g];
  const int K1 = K + 1;
  const int nT = (stp.n_after + PT - 1) / PT;
  const int nrows = nT * PT;
  const V* __restrict__ S = static_cast<const V*>(q.S);
  V* P = static_cast<V*>(q.P);
  const int32_t* __restrict__ I = srcs + stp.src_off;
  const StepConst sc{stp.j, stp.delta, stp.op, stp.d_j, C};
  const V Cv = (V)C;
  auto pidx = [K1](int64_t a, int which, int k) -> int64_t {
    return (((a / PT) * 2 + which) * (int64_t)K1 + k) * PT + (a % PT);
  };

  multi_patch(ops, stp.op_begin, stp.op_end, q.in, q.out);
  for (int T = tid; T < nT; T += MT) mx[T] = me[T] = 0ull;
  if (tid == 0) mx[sc.j / PT] = 1ull;  // xi_0 = C e_j

  if (nrows <= smem_rows<V>()) {
    // ---------------- vectors in shared memory
    V2<V>* vA = reinterpret_cast<V2<V>*>(dsm);
    V2<V>* vB = vA + nrows;
    int* st32 = reinterpret_cast<int*>(vB + nrows);
    int* ln = st32 + nrows;
    for (int a = tid; a < nrows; a += MT) {
      st32[a] = (int)__ldcg(q.in.start + a);
      ln[a] = __ldcg(q.in.len + a);
      V vI = V(0);
      for (int t = 0; t < sc.delta; ++t) vI += s_at(S, q.ld, I[t], a, q.upper != 0);
      vA[a] = V2<V>{vI, s_at(S, q.ld, sc.j, a, q.upper != 0)};  // (sI, sJ)
    }
    __syncthreads();
    if (tid == 0) {
      double sii = 0.0;
      for (int t = 0; t < sc.delta; ++t) sii += (double)vA[I[t]].x;
      s_SII = sii;
    }
    __syncthreads();
    const double S_II = s_SII;
    // gamma: W[0] = (C e_j, gamma) into vB and the panels
    smem_pass<V>(vA, st32, ln, q.in.col, nrows, [&](int a, int kind, bool act, V y, V) {
      bool nz = false;
      if (act) {
        const V g = gamma_row<V>(sc, a, y, ln[a], vA[a].y, S_II);
        const V x0 = (a == sc.j) ? Cv : V(0);
        vB[a] = V2<V>{x0, g};
        P[pidx(a, 0, 0)] = x0;
        P[pidx(a, 1, 0)] = g;
        nz = (g != V(0));
        if (kind == 1 && nz) atomicOr(&me[a / PT], 1ull);
      }
      if (kind == 0) warp_mask(nz, a, 1ull, me);
    });
    __syncthreads();
    V2<V>* cur = vB;
    V2<V>* nxt = vA;
    for (int k = 0; k < K; ++k) {
      const unsigned long long bit = 1ull << ((k + 1) & 63);
      smem_pass<V>(cur, st32, ln, q.in.col, nrows, [&](int a, int kind, bool act, V sx, V sy) {
        bool nx = false, ne = false;
        if (act) {
          const int L = ln[a];
          const V inv = (L > 0) ? V(1) / (V)L : V(0);
          const V x = Cv * sx * inv, y = sy * inv;
          nxt[a] = V2<V>{x, y};
          P[pidx(a, 0, k + 1)] = x;
          P[pidx(a, 1, k + 1)] = y;
          nx = (x != V(0));
          ne = (y != V(0));
          if (kind == 1) {
            if (nx) atomicOr(&mx[a / PT], bit);
            if (ne) atomicOr(&me[a / PT], bit);
          }
        }
        if (kind == 0) {
          warp_mask(nx, a, bit, mx);
          warp_mask(ne, a, bit, me);
        }
      });
      __syncthreads();
      V2<V>* t = cur;
      cur = nxt;
      nxt = t;
    }
  } else {
    // ---------------- vectors in global memory, rows in blocks of RB
    MultiSmem<V>& sm = *reinterpret_cast<MultiSmem<V>*>(dsm);
    V* sI = static_cast<V*>(q.sI);
    V* sJ = static_cast<V*>(q.sJ);
    for (int a = tid; a < nrows; a += MT) {
      V vI = V(0);
      for (int t = 0; t < sc.delta; ++t) vI += s_at(S, q.ld, I[t], a, q.upper != 0);
      sI[a] = vI;
      sJ[a] = s_at(S, q.ld, sc.j, a, q.upper != 0);
    }
    __syncthreads();
    double S_II = 0.0;
    for (int u = 0; u < sc.delta; ++u) S_II += (double)__ldcg(sI + I[u]);
    for (int row0 = 0; row0 < nrows; row0 += RB) {
      block_rows_load(q.in, row0, nrows, sm);
      rows_gather<1, V>(sm, q.in.col, [&](int, int b) { return __ldcg(sI + b); });
      const int a = row0 + tid;
      bool nz = false;
      if (a < nrows) {
        const V g = gamma_row<V>(sc, a, sm.acc[0][tid], sm.len[tid], __ldcg(sJ + a), S_II);
        P[pidx(a, 0, 0)] = (a == sc.j) ? Cv : V(0);
        P[pidx(a, 1, 0)] = g;
        nz = (g != V(0));
      }
      warp_mask(nz, a, 1ull, me);
      __syncthreads();
    }
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
        warp_mask(nx, a, bit, mx);
        warp_mask(ne, a, bit, me);
        __syncthreads();
      }
    }
  }
  __syncthreads();

  for (int T = tid; T < nT; T += MT) {
    q.mXi[T] = mx[T];
    q.mEta[T] = me[T];
  }
  // this graph's tile pairs
  const int lane = tid & 31;
  const uint64_t gk = (uint64_t)(uint32_t)stp.g << 32;
  for (int Ti = 0; Ti < nT; ++Ti) {
    const unsigned long long xi = mx[Ti], ei = me[Ti];
    for (int J0 = Ti; J0 < nT; J0 += MT) {
      const int Tj = J0 + tid;
      bool act = false;
      if (Tj < nT) act = !aff || (((xi & me[Tj]) | (ei & mx[Tj])) != 0ull);
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if (m == 0) continue;
      const int leader = __ffs(m) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(ntiles, __popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (act)
        tiles[base + __popc(m & ((1u << lane) - 1u))] = gk | ((uint64_t)Ti << 16) | (uint64_t)Tj;
    }
  }
}

// Tensor-core operands of one 128-row tile of a graph of this round: row a
// of the graph is row row_off + a of A_hi / A_lo, with xi terms in columns
// [0, K1) and eta terms in [rg, rg + K1), split as x = hi + lo in TF32.
__global__ void k_multi_pack_tc(const MultiGraphDesc* __restrict__ descs,
                                const MultiStep* __restrict__ steps,
                                const int* __restrict__ count, int K1, int rg,
                                float* __restrict__ Ahi, float* __restrict__ Alo, int64_t kd) {
  if ((int)blockIdx.x >= *count) return;
  const MultiStep stp = steps[blockIdx.x];
  const int T = blockIdx.y;
  if (T >= (stp.n_after + PT - 1) / PT) return;
  const MultiGraphDesc& q = descs[stp.g];
  const float* __restrict__ P = static_cast<const float*>(q.P);
  const int64_t row0 = q.row_off + (int64_t)T * PT;
  for (int64_t e = threadIdx.x; e < (int64_t)PT * kd; e += blockDim.x) {
    const int r = (int)(e / kd), c = (int)(e % kd);
    const int h = c >= rg ? 1 : 0;
    const int k = c - h * rg;
    const float x = (k < K1) ? P[((int64_t)(T * 2 + h) * K1 + k) * PT + r] : 0.f;
    const float hi = tf32_rne(x);
    Ahi[(row0 + r) * kd + c] = hi;
    Alo[(row0 + r) * kd + c] = tf32_rne(x - hi);
  }
}

}  // namespace

void launch_multi_pack_tc(const MultiGraphDesc* descs, const MultiStep* steps, const int* count,
                          int grid, int max_tiles, int K1, int rg, float* Ahi, float* Alo,
                          int64_t kd, cudaStream_t st) {
  if (grid <= 0 || max_tiles <= 0) return;
  k_multi_pack_tc<<<dim3(grid, max_tiles), 256, 0, st>>>(descs, steps, count, K1, rg, Ahi, Alo,
                                                         kd);
}

void launch_multi_prep(int s_prec, const MultiGraphDesc* descs, const MultiStep* steps,
                       const int* count, int grid, const int32_t* srcs, const PatchOp* ops,
                       double C, int K, int aff, uint64_t* tiles, int* ntiles, cudaStream_t st) {
  if (grid <= 0) return;
  static std::atomic<unsigned long long> attr64{0}, attr32{0};
  smem_attr_once((const void*)k_multi_prep<double>, SMEM_BYTES, attr64);
  smem_attr_once((const void*)k_multi_prep<float>, SMEM_BYTES, attr32);
  if (s_prec == 64)
    k_multi_prep<double><<<grid, MT, SMEM_BYTES, st>>>(descs, steps, count, srcs, ops, C, K, aff,
                                                       tiles, ntiles);
  else
    k_multi_prep<float><<<grid, MT, SMEM_BYTES, st>>>(descs, steps, count, srcs, ops, C, K, aff,
                                                      tiles, ntiles);
}

}  // namespace sr
