// Everything one rank-one (sink-block) update does before its S pass, in one
// cooperative launch:
//   phase 0  graph patch (Thm 1: row j of the in-adjacency gains / loses the
//            sources I); the rows of the current S that gamma reads,
//            sI = sum_t S[I_t, *] and sJ = S[j, *], with the panels of updates
//            whose S pass is still pending added in; per-tile nonzero counts;
//   phase 1  w = Q sI (the SpMV of Thm 3's preprocessing), then gamma (Thm 3
//            insert, Thm 9 delete, Table 2 sink blocks) as eta_0, with
//            xi_0 = C e_j;
//   phase 2  the K steps of the recurrence on the new graph (Eq. 16a),
//            xi_{k+1} = C Q xi_k, eta_{k+1} = Q eta_k;
//   phase 3  the affected-area mask words of every tile (Thm 4) and the list
//            of affected tile pairs of the S pass.
// Phases and steps are separated by a bounded grid barrier.
//
// Work split.  A gather of one scattered vector element per nonzero is bound
// by the L1 throughput of the SM that issues it, and on GB300 the FP64 form
// by the FP64 issue rate of the SM, so the nonzeros, not the rows, are spread
// evenly.  Flat split (default): the in-lists of all rows, flattened in row
// order, are cut into equal contiguous ranges, one per CTA, two nonzeros per
// thread, located once per launch from the tile offsets and the in-tile row
// offsets that phase 0 writes.  Item split (a set `item`, or too many
// nonzeros for two per thread): every 128-row tile is cut into items of at
// most `item` flattened nonzeros, and items go round-robin to the CTAs (a hub
// row with thousands of in-neighbours spreads over many SMs); each CTA keeps
// the row extents and column indices of its first items in shared memory for
// all K steps.  Partial row sums are combined within a warp and added to the next
// column with global atomics.  xi_k and eta_k are kept interleaved in the
// working buffer W[k][a] (one 8- or 16-byte load per nonzero).  Row-wise work
// (gamma; after the last step, the copy of the columns into the tile-blocked
// panels that the S pass reads, with the masks) goes by tiles, round-robin.
//
// gamma needs w on the OLD graph; only row j of Q changes, so the kernel
// gathers on the patched graph and corrects row j: the sum over the old
// in-neighbours = the sum over the new ones - op * S_II.
//
// The vectors and the arithmetic are FP64 (vec64 = 1, or S in FP64) or FP32;
// the panels the S pass reads have the precision of S, and lambda and row j
// of gamma are always FP64.  The correction of the rows of S by pending
// panels is summed in the precision of S (those panels are stored in it).
// GB300 issues FP64 instructions at 1/64 of the FP32 rate, so the FP64 form
// keeps per-row factors in shared memory, tests for zero on the integer pipe
// and leaves the additions of the atomics to L2.  The atomic accumulation
// makes the last bit of a result depend on the order of the additions.
#include <algorithm>

#include "fx64.h"
#include "sr_internal.h"

namespace sr {

namespace {

constexpr int PG = 512;     // threads of a prep CTA
constexpr int PREP_MT = 8;  // tiles one CTA may own for row-wise work
constexpr int MAXI = 6;     // items whose row extents stay in shared memory

template <typename V>
struct V2 {
  V x, y;
};

struct alignas(16) PrepItem {
  int64_t start[PT];
  int len[PT];
  int off[PT + 1];
  int T;       // tile
  int e0, e1;  // flattened nonzeros [e0, e1) of the tile
  int cbase;   // nonzeros [e0, e0 + clen) have their column index at cc[cbase ...]
  int clen;
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on a monotonically increasing arrival counter: barrier number
// b of a launch returns once b * gridDim.x arrivals are visible.  Bounded:
// false after `limit` polls.  The arrival is a release reduction (it orders
// the CTA's earlier writes, made visible to thread 0 by the CTA barrier, before
// it) and the polls are acquire loads, so after the final CTA barrier plain
// (L1-cached) loads of every thread see every CTA's writes from before the
// barrier.
__device__ __forceinline__ bool prep_barrier(unsigned int* count, unsigned int target,
                                             long long limit, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    int ok = 1;
    long long it = 0;
    while (ld_acquire(count) < target) {
      if (++it > limit) {
        ok = 0;
        break;
      }
      __nanosleep(16);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add2(V2<float>* p, float x, float y) {
  asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x), "f"(y)
               : "memory");
}
__device__ __forceinline__ void red_add2(V2<double>* p, double x, double y) {
  red_add(&p->x, x);
  red_add(&p->y, y);
}
// x != 0 on the integer pipe (GB300 issues FP64 compares at the FP64 rate)
__device__ __forceinline__ bool nz(float x) { return (__float_as_uint(x) << 1) != 0u; }
__device__ __forceinline__ bool nz(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}
// Gathers of the working vectors go through L1: a column with a large
// out-degree is read by many rows of the same CTA.  Each W[k] is written (by
// atomics, in L2) only in the step before the one that reads it, with a grid
// barrier between, so no L1 line can be stale.
__device__ __forceinline__ V2<float> ld_v2(const V2<float>* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return V2<float>{v.x, v.y};
}
__device__ __forceinline__ V2<double> ld_v2(const V2<double>* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return V2<double>{v.x, v.y};
}

__device__ __forceinline__ V2<float> ld_v2cg(const V2<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return V2<float>{v.x, v.y};
}
__device__ __forceinline__ V2<double> ld_v2cg(const V2<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return V2<double>{v.x, v.y};
}

// Row extents of tile T (after the patch) and the exclusive scan of their lengths.
__device__ __forceinline__ void item_rows_load(const DevAdj& in, int T, PrepItem& it) {
  const int tid = threadIdx.x;
  if (tid < PT) {
    it.start[tid] = __ldcg(in.start + (int64_t)T * PT + tid);
    it.len[tid] = __ldcg(in.len + (int64_t)T * PT + tid);
  }
  __syncthreads();
  if (tid < 32) {
    int v[4], sum = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = it.len[tid * 4 + q];
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
      it.off[tid * 4 + q] = run;
      run += v[q];
    }
    if (tid == 31) it.off[PT] = incl;
  }
  __syncthreads();
}

// Item q of the launch: its tile (the last T with ioff[T] <= q) and range.
__device__ __forceinline__ void item_locate(const DevAdj& in, const int* ioff, int nT, int q,
                                            int item, PrepItem& it) {
  int lo = 0, hi = nT;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ioff[mid] <= q) lo = mid; else hi = mid;
  }
  item_rows_load(in, lo, it);
  if (threadIdx.x == 0) {
    it.T = lo;
    it.e0 = (q - ioff[lo]) * item;
    it.e1 = min(it.off[PT], it.e0 + item);
    it.cbase = 0;
    it.clen = 0;
  }
  __syncthreads();
}

// Combines per-lane partials of equal row keys across a warp (keys are
// non-decreasing with the lane; key < 0 = nothing) and hands each segment's
// nonzero total to emit(key, a, b) once.
template <typename V, typename Emit>
__device__ __forceinline__ void seg_emit(int key, V a, V b, Emit emit) {
  const int lane = threadIdx.x & 31;
  // only as many rounds as the longest run of equal keys needs
  const unsigned same = __match_any_sync(0xffffffffu, key);
  const int span = (int)__reduce_max_sync(0xffffffffu, key >= 0 ? (unsigned)__popc(same) : 1u);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= span) break;
    const int k2 = __shfl_down_sync(0xffffffffu, key, o);
    const V xa = __shfl_down_sync(0xffffffffu, a, o);
    const V xb = __shfl_down_sync(0xffffffffu, b, o);
    if (lane + o < 32 && k2 == key) {
      a += xa;
      b += xb;
    }
  }
  const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
  if (key >= 0 && (lane == 0 || kprev != key) && (nz(a) || nz(b))) emit(key, a, b);
}

// One thread's contiguous run [e0, e1) of an item's nonzeros (flattened order
// of the tile) and the row r holding e0 (r = -1: empty run).  The same for
// every step, so the step loop computes it once for the CTA's first item.
struct Run {
  int e0, e1, r;
};

__device__ __forceinline__ Run item_run(const PrepItem& it) {
  const int n_e = it.e1 - it.e0;
  const int per = (n_e + PG - 1) / PG;
  Run u;
  u.e0 = it.e0 + (int)threadIdx.x * per;
  u.e1 = min(it.e1, u.e0 + per);
  u.r = -1;
  if (u.e0 < u.e1) {
    int lo = 0, hi = PT;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (it.off[mid] <= u.e0) lo = mid; else hi = mid;
    }
    u.r = lo;
  }
  return u;
}

// Sums gather(b) over the nonzeros of the item's tile, per row, and calls
// emit(r, a, b) with each row's (partial) sums.  Each thread takes its run; a
// row wholly inside one run is emitted by that thread, the first and last row
// of a run go through seg_emit.
template <typename V, typename Gf, typename Emit>
__device__ __forceinline__ void item_gather(const PrepItem& it, const Run& run,
                                            const int* __restrict__ cc,
                                            const int32_t* __restrict__ col, Gf gather,
                                            Emit emit) {
  const int e0 = run.e0, e1 = run.e1;
  int r_first = -1, r_last = -1;
  V fa = V(0), fb = V(0), la = V(0), lb = V(0);
  if (run.r >= 0) {
    int r = run.r;
    r_first = r;
    V pa = V(0), pb = V(0);
    constexpr int B = sizeof(V) == 8 ? 4 : 8;
    for (int e = e0; e < e1; e += B) {
      int rr[B], bb[B];
      int rc = r;
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int ee = e + q;
        if (ee < e1) {
          while (ee >= it.off[rc + 1]) ++rc;
          rr[q] = rc;
          const int ce = ee - it.e0;
          bb[q] = (ce < it.clen) ? cc[it.cbase + ce]
                                 : __ldcg(col + it.start[rc] + (ee - it.off[rc]));
        } else {
          rr[q] = -1;
          bb[q] = 0;
        }
      }
      V2<V> xv[B];
#pragma unroll
      for (int q = 0; q < B; ++q) xv[q] = (rr[q] >= 0) ? gather(bb[q]) : V2<V>{V(0), V(0)};
#pragma unroll
      for (int q = 0; q < B; ++q) {
        if (rr[q] < 0) break;
        if (rr[q] != r) {
          if (r == r_first) {
            fa = pa;
            fb = pb;
          } else if (nz(pa) || nz(pb)) {
            emit(r, pa, pb);  // row wholly inside this run
          }
          pa = pb = V(0);
          r = rr[q];
        }
        pa += xv[q].x;
        pb += xv[q].y;
      }
    }
    if (r == r_first) {
      fa = pa;
      fb = pb;
    } else {
      r_last = r;
      la = pa;
      lb = pb;
    }
  }
  seg_emit<V>(r_first, fa, fb, emit);
  seg_emit<V>(r_last, la, lb, emit);
}

// A step over an item of at most 2 * PG nonzeros gives each thread at most two
// of them, so a thread's part of every step is fixed by the graph: its columns,
// the rows they fall in (head = row of the first; tail = row of the second
// when it differs) and the shuffle pattern of the warp that adds up the rows
// spread over several lanes.  StepPair holds that, set up once per launch.
template <typename V>
struct StepPair {
  int ca, cb;    // columns of the nonzeros (-1: none)
  int kh, kt;    // head / tail row in the tile (-1: none)
  int span;      // warp-uniform: the longest run of lanes sharing a head row
  unsigned fl;   // bits 0-4: take lane + 2^b's head sum; 5: add lane - 1's tail;
                 // 6: emit the head sum; 7: emit the tail sum; 8-12: the first lane
                 // of the head row's run of lanes
};

template <typename V>
__device__ __forceinline__ void pair_pattern(StepPair<V>& q);

template <typename V>
__device__ __forceinline__ StepPair<V> pair_setup(const PrepItem& it, const int* __restrict__ cc,
                                                  const int32_t* __restrict__ col) {
  const Run run = item_run(it);
  StepPair<V> q;
  q.ca = q.cb = q.kh = q.kt = -1;
  auto column = [&](int e, int r) {
    const int ce = e - it.e0;
    return (ce < it.clen) ? cc[it.cbase + ce] : __ldcg(col + it.start[r] + (e - it.off[r]));
  };
  if (run.r >= 0) {
    q.kh = run.r;
    q.ca = column(run.e0, q.kh);
    if (run.e1 - run.e0 == 2) {
      int r2 = q.kh;
      while (run.e0 + 1 >= it.off[r2 + 1]) ++r2;
      q.cb = column(run.e0 + 1, r2);
      if (r2 != q.kh) q.kt = r2;
    }
  }
  pair_pattern(q);
  return q;
}

// The warp-wide pattern of a step for threads whose (ca, cb, kh, kt) are set:
// row keys must not decrease with the lane.
template <typename V>
__device__ __forceinline__ void pair_pattern(StepPair<V>& q) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // every lane takes part in the warp-wide intrinsics below
  const unsigned same = __match_any_sync(full, q.kh);
  const int seg = (q.kh >= 0) ? __popc(same) : 1;
  q.span = __reduce_max_sync(full, (unsigned)seg);
  // a segment's lanes are consecutive (row keys do not decrease with the lane):
  // a tree over the segment that leaves the total in its first lane only adds,
  // in round b, the partial of lane + 2^b into the lanes at positions 0 mod
  // 2^(b+1), so a segment of s lanes costs s - 1 additions
  const int pos = lane - (__ffs(same) - 1);
  q.fl = (unsigned)(__ffs(same) - 1) << 8;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const int k2 = __shfl_down_sync(full, q.kh, 1 << b);
    if (lane + (1 << b) < 32 && k2 == q.kh && q.kh >= 0 && (pos & ((2 << b) - 1)) == 0)
      q.fl |= 1u << b;
  }
  const int kt_prev = __shfl_up_sync(full, q.kt, 1);
  const int kh_prev = __shfl_up_sync(full, q.kh, 1);
  const int kh_next = __shfl_down_sync(full, q.kh, 1);
  if (lane > 0 && q.kh >= 0 && kt_prev == q.kh) q.fl |= 1u << 5;
  if (q.kh >= 0 && (lane == 0 || kh_prev != q.kh)) q.fl |= 1u << 6;
  if (q.kt >= 0 && !(lane < 31 && kh_next == q.kt)) q.fl |= 1u << 7;
}

// One step of the recurrence for a thread set up by pair_setup: gathers its
// (xi_k, eta_k) entries, adds the rows up across the warp and emits each row's
// sum (times C / in-degree for xi, 1 / in-degree for eta; rc / ri hold those
// factors per row of the item's tile) into W[k + 1].
template <typename Gf, typename Emit>
__device__ __forceinline__ void pair_step_fx(const StepPair<double>& q, Gf gather, Emit emit);

template <typename V, typename Gf, typename Emit>
__device__ __forceinline__ void pair_step(const StepPair<V>& q, Gf gather, Emit emit) {
  if constexpr (sizeof(V) == 8) {
    pair_step_fx(q, gather, emit);
    return;
  }
  const unsigned full = 0xffffffffu;
  V ha = V(0), hb = V(0), ta = V(0), tb = V(0);
  if (q.ca >= 0) {
    const V2<V> v = gather(q.ca);
    ha = v.x;
    hb = v.y;
  }
  if (q.cb >= 0) {
    const V2<V> v = gather(q.cb);
    if (q.kt >= 0) {
      ta = v.x;
      tb = v.y;
    } else {
      ha += v.x;
      hb += v.y;
    }
  }
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if ((1 << b) >= q.span) break;
    const V xa = __shfl_down_sync(full, ha, 1 << b);
    const V xb = __shfl_down_sync(full, hb, 1 << b);
    if (q.fl & (1u << b)) {
      ha += xa;
      hb += xb;
    }
  }
  const V pa = __shfl_up_sync(full, ta, 1);
  const V pb = __shfl_up_sync(full, tb, 1);
  if (q.fl & (1u << 5)) {
    ha += pa;
    hb += pb;
  }
  if ((q.fl & (1u << 6)) && (nz(ha) || nz(hb))) emit(q.kh, ha, hb);
  if ((q.fl & (1u << 7)) && (nz(ta) || nz(tb))) emit(q.kt, ta, tb);
}

// Exact row sums of FP64 values on the integer pipe (fx64.h): the values of
// one row's run of lanes (at most 65: two per lane and an incoming tail, so
// below 2^63 in total) are turned into 64-bit fixed-point numbers with 55
// fraction bits below the run's largest binary exponent, added exactly, and
// the total is rounded to FP64 once.  The error stays below 65 * 2^-55 of the
// largest value, where FP64 additions in any order can lose (n - 1) 2^-53 of
// the sum of the magnitudes.
// pair_step for FP64 vectors with the row sums formed exactly as above: the
// run's largest exponent goes through the same shuffle tree (integer max) and
// back to every lane of the run from its first lane, then the fixed-point
// values through the tree (integer adds).  A tail that ends its row in this
// lane is one value and is emitted as it is.
template <typename Gf, typename Emit>
__device__ __forceinline__ void pair_step_fx(const StepPair<double>& q, Gf gather, Emit emit) {
  const unsigned full = 0xffffffffu;
  double h1x = 0.0, h1y = 0.0, h2x = 0.0, h2y = 0.0, tx = 0.0, ty = 0.0;
  if (q.ca >= 0) {
    const V2<double> v = gather(q.ca);
    h1x = v.x;
    h1y = v.y;
  }
  if (q.cb >= 0) {
    const V2<double> v = gather(q.cb);
    if (q.kt >= 0) {
      tx = v.x;
      ty = v.y;
    } else {
      h2x = v.x;
      h2y = v.y;
    }
  }
  // lane - 1's tail, added into this lane's head row (bit 5)
  double px = __shfl_up_sync(full, tx, 1), py = __shfl_up_sync(full, ty, 1);
  if (!(q.fl & (1u << 5))) px = py = 0.0;
  int ex = max(max(fx_exp(h1x), fx_exp(h2x)), fx_exp(px));
  int ey = max(max(fx_exp(h1y), fx_exp(h2y)), fx_exp(py));
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if ((1 << b) >= q.span) break;
    const int xe = __shfl_down_sync(full, ex, 1 << b);
    const int ye = __shfl_down_sync(full, ey, 1 << b);
    if (q.fl & (1u << b)) {
      ex = max(ex, xe);
      ey = max(ey, ye);
    }
  }
  const int first = (int)((q.fl >> 8) & 31u);
  ex = __shfl_sync(full, ex, first);
  ey = __shfl_sync(full, ey, first);
  long long fx = fx_of(h1x, ex) + fx_of(h2x, ex) + fx_of(px, ex);
  long long fy = fx_of(h1y, ey) + fx_of(h2y, ey) + fx_of(py, ey);
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if ((1 << b) >= q.span) break;
    const long long xa = __shfl_down_sync(full, fx, 1 << b);
    const long long xb = __shfl_down_sync(full, fy, 1 << b);
    if (q.fl & (1u << b)) {
      fx += xa;
      fy += xb;
    }
  }
  if ((q.fl & (1u << 6)) && (fx != 0 || fy != 0)) emit(q.kh, fx_value(fx, ex), fx_value(fy, ey));
  if ((q.fl & (1u << 7)) && (nz(tx) || nz(ty))) emit(q.kt, tx, ty);
}

// The flat split: CTA c takes the nonzeros [c E, (c + 1) E) of the in-lists of
// all rows flattened in row order, E = ceil(nnz / CTAs), two per thread, so
// every CTA gets the same number whatever the tiles hold.  Nonzero e is found
// by its tile (tile offsets toff, shared) and its row in the tile (in-tile row
// offsets loff, global); rows are keyed by their global index.
__device__ __forceinline__ void flat_locate(const int* toff, int nT, const int* __restrict__ loff,
                                            const DevAdj& in, int e, int& row, int& col) {
  int lo = 0, hi = nT;  // the last tile T with toff[T] <= e
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (toff[mid] <= e) lo = mid; else hi = mid;
  }
  const int l = e - toff[lo];
  const int* lt = loff + (int64_t)lo * PT;
  int a = 0, b = PT;  // the last row of the tile with loff <= l
  while (b - a > 1) {
    const int mid = (a + b) >> 1;
    if (__ldcg(lt + mid) <= l) a = mid; else b = mid;
  }
  row = lo * PT + a;
  col = __ldcg(in.col + __ldcg(in.start + row) + (l - __ldcg(lt + a)));
}

template <typename V>
__device__ __forceinline__ StepPair<V> flat_setup(const int* toff, int nT, const int* loff,
                                                  const DevAdj& in, int e0, int e1) {
  StepPair<V> q;
  q.ca = q.cb = q.kh = q.kt = -1;
  const int e = e0 + 2 * (int)threadIdx.x;
  if (e < e1) {
    flat_locate(toff, nT, loff, in, e, q.kh, q.ca);
    if (e + 1 < e1) {
      int r2;
      flat_locate(toff, nT, loff, in, e + 1, r2, q.cb);
      if (r2 != q.kh) q.kt = r2;
    }
  }
  pair_pattern(q);
  return q;
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

// V: arithmetic and vector precision; TS: storage precision of S and the panels
template <typename V, typename TS>
__global__ void __launch_bounds__(PG, 2) k_prep(PrepParams p) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ V red[4][2][PT];
  __shared__ V rrc[PT], rri[PT];  // C / in-degree and 1 / in-degree of the rows of item 0
  __shared__ V2<V> fsh[PG][2];      // flat split: the same for each thread's head / tail row
  __shared__ unsigned long long mk[PREP_MT][2];
  __shared__ int wsum[PG / 32];
  __shared__ int s_ok, s_div;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int nT = p.nT;
  const int mt = p.mt;
  // dynamic shared memory: item slots, column cache, item offsets, pending coefficients
  PrepItem* items = reinterpret_cast<PrepItem*>(dsm);
  int* cc = reinterpret_cast<int*>(items + (MAXI + 1));
  int* ioff = cc + p.cap;  // [nT + 1]
  // the pending correction of the rows of S is summed in the storage precision of S
  TS* coef = reinterpret_cast<TS*>(ioff + ((p.nT_cap + 1 + 3) & ~3));
  const TS* __restrict__ S = static_cast<const TS*>(p.S);
  TS* P = static_cast<TS*>(p.P);
  V* sI = static_cast<V*>(p.sI);
  V* sJ = static_cast<V*>(p.sJ);
  V2<V>* W = static_cast<V2<V>*>(p.W);
  V2<V>* rinv = static_cast<V2<V>*>(p.rinv);  // (C / in-degree, 1 / in-degree) per row
  const int64_t ldk = p.ldk;
  auto pidx = [ldk](int64_t a, int which, int k) -> int64_t {
    return (((a / PT) * 2 + which) * ldk + k) * PT + (a % PT);
  };
  const int np = p.npend;
  const int koff = p.koff;
  const V Cv = (V)p.C;
  const int K = p.K;
  const int new_len_j = p.d_j + p.op * p.delta;
  unsigned int nb = 0;
  bool alive = true;

  // ---- phase 0: patch (CTA 0), zero W, rows sI / sJ, tile nonzero counts
  if (blockIdx.x == 0) {
    if (p.op_end > p.op_begin) prep_patch(p.ops, p.op_begin, p.op_end, p.in, p.out);
    if (tid == 0 && p.tiles) *p.ntiles = 0;
  }
  {
    // W[0 .. K] over all n_pad rows, 16 bytes per store (n_pad is a multiple of 128)
    uint4* w16 = reinterpret_cast<uint4*>(W);
    const int64_t total = (int64_t)(K + 1) * p.n_pad * (int64_t)sizeof(V2<V>) / 16;
    for (int64_t e = (int64_t)blockIdx.x * PG + tid; e < total; e += (int64_t)G * PG)
      w16[e] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (np > 0) {
    // c_x[q] = sum_t xi_q[I_t], c_e[q] = sum_t eta_q[I_t]; the same at j
    for (int q = tid; q < np; q += PG) {
      TS cx = TS(0), ce = TS(0);
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
  for (int t = 0; t < mt; ++t) {
    const int T = blockIdx.x + t * G;
    if (T >= nT) break;
    const int r = tid & (PT - 1), part = tid >> 7;
    const int64_t a = (int64_t)T * PT + r;
    V vI = V(0), vJ = V(0);
    for (int u = part; u < p.delta; u += 4) vI += (V)s_at(S, p.ld, p.I[u], a, p.upper != 0);
    if (part == 3) vJ = (V)s_at(S, p.ld, p.j, a, p.upper != 0);
    // S_cur[x, a] = S[x, a] + sum_q xi_q[x] eta_q[a] + eta_q[x] xi_q[a]: the
    // pending terms are FP32 panels of an FP32 S, so they are added in FP32
    // (on GB300 an FP64 FMA issues at 1/64 of the FP32 rate)
    TS cI = TS(0), cJ = TS(0);
    for (int q = part; q < np; q += 4) {
      const TS xa = P[pidx(a, 0, q)];
      const TS ea = P[pidx(a, 1, q)];
      cI += coef[q] * ea + coef[np + q] * xa;
      cJ += coef[2 * np + q] * ea + coef[3 * np + q] * xa;
    }
    vI += (V)cI;
    vJ += (V)cJ;
    red[part][0][r] = vI;
    red[part][1][r] = vJ;
    // nonzeros of the tile after the patch (row j is being patched by CTA 0:
    // it counts with its new length; no other row's length changes)
    int L = 0;
    if (part == 0) L = (a == p.j) ? new_len_j : p.in.len[a];
    // inclusive scan of the row lengths over the tile (warps 0..3 hold its rows)
    int incl = L;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (tid < PT) {
      sI[a] = (red[0][0][r] + red[1][0][r]) + (red[2][0][r] + red[3][0][r]);
      sJ[a] = (red[0][1][r] + red[1][1][r]) + (red[2][1][r] + red[3][1][r]);
      int base = 0;
      for (int w = 0; w < warp; ++w) base += wsum[w];
      p.loff[a] = base + incl - L;  // nonzeros of the tile before row a
    }
    if (tid == 0) p.tile_nnz[T] = (wsum[0] + wsum[1]) + (wsum[2] + wsum[3]);
    __syncthreads();
  }
  alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);

  // ---- phase 1: the split of the nonzeros over the CTAs; w = Q sI summed by
  // atomics into W[0].x
  int my_items = 0;
  bool flat = false;
  StepPair<V> q0;
  if (alive) {
    // ioff[T] = the units of the tiles before T: their nonzeros (flat split,
    // tried first when allowed) or their items of at most `item` nonzeros
    for (int pass = p.flat ? 0 : 1; pass < 2; ++pass) {
      const int div = pass == 0 ? 1 : p.item;
      const int per = (nT + PG - 1) / PG;
      const int t0 = min(nT, tid * per), t1 = min(nT, t0 + per);
      int s = 0;
      for (int T = t0; T < t1; ++T) {
        const int c = __ldcg(p.tile_nnz + T);
        s += div == 1 ? c : (c + div - 1) / div;
      }
      int incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) wsum[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        const int v = (lane < PG / 32) ? wsum[lane] : 0;
        int w = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, w, o);
          if (lane >= o) w += y;
        }
        if (lane < PG / 32) wsum[lane] = w - v;
        if (lane == PG / 32 - 1) {
          ioff[nT] = w;
          // the CTA's share, by one thread (a division would be issued by
          // every thread): nonzeros per CTA (flat pass) or this CTA's items
          const int b = (int)blockIdx.x;
          s_div = pass == 0 ? (w + G - 1) / G : (w > b ? (w - b + G - 1) / G : 0);
        }
      }
      __syncthreads();
      int run = wsum[warp] + incl - s;
      for (int T = t0; T < t1; ++T) {
        ioff[T] = run;
        const int c = __ldcg(p.tile_nnz + T);
        run += div == 1 ? c : (c + div - 1) / div;
      }
      __syncthreads();
      if (pass == 0) {
        // every CTA computes the same nnz, so the choice is uniform over the grid
        const int nnz = ioff[nT];
        const int per_cta = (nnz + G - 1) / G;
        if (per_cta <= 2 * PG) {
          flat = true;
          const int e0 = min(nnz, (int)blockIdx.x * per_cta), e1 = min(nnz, e0 + per_cta);
          q0 = flat_setup<V>(ioff, nT, p.loff, p.in, e0, e1);
          break;
        }
        __syncthreads();  // ioff is rewritten by the item pass
      }
    }
  }
  if (alive && flat) {
    pair_step<V>(q0, [&](int b) { return V2<V>{sI[b], V(0)}; },
                 [&](int r, V a, V) { red_add(&W[r].x, a); });
    alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
  } else if (alive) {
    my_items = s_div;
    int cbase = 0;
    for (int u = 0; u < my_items; ++u) {
      PrepItem& it = items[min(u, MAXI)];
      item_locate(p.in, ioff, nT, blockIdx.x + u * G, p.item, it);
      if (u < MAXI) {
        const int clen = max(0, min(it.e1 - it.e0, p.cap - cbase));
        // cache the column indices of [e0, e0 + clen), one nonzero per thread
        // (a row of the item may hold all of them)
#pragma unroll 2
        for (int e = it.e0 + tid; e < it.e0 + clen; e += PG) {
          int lo = 0, hi = PT;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (it.off[mid] <= e) lo = mid; else hi = mid;
          }
          cc[cbase + (e - it.e0)] = __ldcg(p.in.col + it.start[lo] + (e - it.off[lo]));
        }
        __syncthreads();
        if (tid == 0) {
          it.cbase = cbase;
          it.clen = clen;
        }
        cbase += clen;
        __syncthreads();
      }
      const int64_t rb = (int64_t)it.T * PT;
      item_gather<V>(it, item_run(it), cc, p.in.col, [&](int b) { return V2<V>{sI[b], V(0)}; },
                     [&](int r, V a, V) { red_add(&W[rb + r].x, a); });
      __syncthreads();
    }
    alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
  }

  // ---- phase 1b: gamma per row (tiles round-robin); W[0] = (xi_0, eta_0)
  if (alive) {
    for (int t = 0; t < mt; ++t) {
      const int T = blockIdx.x + t * G;
      if (T >= nT) break;
      int pe = 0;
      if (tid < PT) {
        const int64_t a = (int64_t)T * PT + tid;
        const int len = __ldcg(p.in.len + a);
        // the factors of row a of Q on the new graph, for every step below
        const V inv = len > 0 ? V(1) / (V)len : V(0);
        const V y = __ldcg(&W[a].x);
        const double dl = (double)p.delta;
        V g;
        if (a == p.j) {
          // row j: lambda (Eq. 29b) and w_j on the old row j, in FP64
          double S_II = 0.0;
          for (int u = 0; u < p.delta; ++u) S_II += (double)__ldcg(sI + p.I[u]);
          const double S_jj = (double)__ldcg(sJ + p.j);
          const double C = p.C;
          const double wj =
              (p.d_j > 0) ? ((double)y - (double)p.op * S_II) / (dl * (double)p.d_j) : 0.0;
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
          const V w = y * inv * (V)p.inv_delta;
          const V sJa = __ldcg(sJ + a);
          const V sc = sJa * (V)p.inv_C;
          if (p.op > 0) {
            g = (p.d_j == 0) ? w : (V)p.gq * (w - sc);
          } else {
            g = (p.d_j == p.delta) ? -w : (V)p.gq * (sc - w);
          }
        }
        const V x0 = (a == p.j) ? Cv : V(0);
        W[a] = V2<V>{x0, g};
        rinv[a] = V2<V>{Cv * inv, inv};
        P[pidx(a, 0, koff)] = (TS)x0;
        P[pidx(a, 1, koff)] = (TS)g;
        pe = nz(g);
      }
      const int any_e = __syncthreads_or(pe);
      if (tid == 0) {
        mk[t][0] = (T == p.j / PT) ? 1ull : 0ull;
        mk[t][1] = any_e ? 1ull : 0ull;
      }
    }
    if (K > 0) alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
  }

  // ---- phase 2: K steps
  // the CTA's first item takes the fixed per-thread form when it can
  const bool pair0 = !flat && my_items > 0 && items[0].e1 - items[0].e0 <= 2 * PG;
  int64_t rb0 = 0;
  if (flat) {
    // flat split: the factors of each thread's head and tail rows
    fsh[tid][0] = q0.kh >= 0 ? ld_v2cg(rinv + q0.kh) : V2<V>{V(0), V(0)};
    fsh[tid][1] = q0.kt >= 0 ? ld_v2cg(rinv + q0.kt) : V2<V>{V(0), V(0)};
  }
  if (pair0) {
    q0 = pair_setup<V>(items[0], cc, p.in.col);
    rb0 = (int64_t)items[0].T * PT;
    if (tid < PT) {
      const V2<V> f = ld_v2cg(rinv + rb0 + tid);
      rrc[tid] = f.x;
      rri[tid] = f.y;
    }
    __syncthreads();
  }
  for (int k = 0; alive && k < K; ++k) {
    const V2<V>* Wk = W + (int64_t)k * p.n_pad;
    V2<V>* Wn = W + (int64_t)(k + 1) * p.n_pad;
    if (flat)
      pair_step<V>(q0, [&](int b) { return ld_v2(Wk + b); }, [&](int r, V a, V b) {
        const V2<V> f = fsh[tid][r == q0.kh ? 0 : 1];
        red_add2(Wn + r, a * f.x, b * f.y);
      });
    for (int u = 0; u < my_items; ++u) {
      if (u == 0 && pair0) {
        pair_step<V>(q0, [&](int b) { return ld_v2(Wk + b); },
                     [&](int r, V a, V b) { red_add2(Wn + rb0 + r, a * rrc[r], b * rri[r]); });
        continue;
      }
      PrepItem& it = items[min(u, MAXI)];
      if (u >= MAXI) item_locate(p.in, ioff, nT, blockIdx.x + u * G, p.item, it);
      const int64_t rb = (int64_t)it.T * PT;
      item_gather<V>(it, item_run(it), cc, p.in.col,
                     [&](int b) { return ld_v2(Wk + b); },
                     [&](int r, V a, V b) {
                       const V2<V> f = ld_v2cg(rinv + rb + r);
                       red_add2(Wn + rb + r, a * f.x, b * f.y);
                     });
      __syncthreads();
    }
    alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
  }

  // ---- columns 1..K of the owned tiles into the panels, with their mask bits
  if (alive && K > 0) {
    for (int t = 0; t < mt; ++t) {
      const int T = blockIdx.x + t * G;
      if (T >= nT) break;
      // warp w copies columns k = 1 + w, 1 + w + 16, ...
      for (int k = 1 + warp; k <= K; k += PG / 32) {
        const V2<V>* Wk = W + (int64_t)k * p.n_pad;
        bool nx = false, ne = false;
#pragma unroll
        for (int q = 0; q < PT / 32; ++q) {
          const int64_t a = (int64_t)T * PT + q * 32 + lane;
          const V2<V> v = ld_v2(Wk + a);
          // the mask bits follow the stored panel values (a value that rounds
          // to zero in the precision of S adds nothing to S)
          const TS px = (TS)v.x, pe = (TS)v.y;
          P[pidx(a, 0, koff + k)] = px;
          P[pidx(a, 1, koff + k)] = pe;
          nx |= nz(px);
          ne |= nz(pe);
        }
        const unsigned bx = __ballot_sync(0xffffffffu, nx), be = __ballot_sync(0xffffffffu, ne);
        const unsigned long long bit = 1ull << (k & 63);
        if (lane == 0) {
          if (bx) atomicOr(&mk[t][0], bit);
          if (be) atomicOr(&mk[t][1], bit);
        }
      }
    }
  }

  // ---- phase 3: mask words and the affected tile pairs
  if (alive) {
    __syncthreads();
    if (tid == 0) {
      for (int t = 0; t < mt; ++t) {
        const int T = blockIdx.x + t * G;
        if (T >= nT) break;
        p.mXi[T] = mk[t][0];
        p.mEta[T] = mk[t][1];
        if (p.pXi) {
          if (mk[t][0]) p.pXi[T] = 1ull;
          if (mk[t][1]) p.pEta[T] = 1ull;
        }
      }
    }
    if (p.tiles) {
      alive = prep_barrier(p.bar, ++nb * G, p.limit, &s_ok);
      if (alive) {
        const unsigned long long* mx = reinterpret_cast<const unsigned long long*>(p.mXi);
        const unsigned long long* me = reinterpret_cast<const unsigned long long*>(p.mEta);
        for (int I = blockIdx.x; I < nT; I += G) {
          const unsigned long long xi = __ldcg(mx + I), ei = __ldcg(me + I);
          for (int J0 = I; J0 < nT; J0 += PG) {
            const int J = J0 + tid;
            bool act = false;
            if (J < nT)
              act = (p.tile_mode == 0) ||
                    (((xi & __ldcg(me + J)) | (ei & __ldcg(mx + J))) != 0ull);
            const unsigned mask = __ballot_sync(0xffffffffu, act);
            if (mask == 0) continue;
            const int leader = __ffs(mask) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(p.ntiles, __popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (act)
              p.tiles[base + __popc(mask & ((1u << lane) - 1u))] =
                  ((uint32_t)I << 16) | (uint32_t)J;
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

template <typename TS>
size_t prep_smem(int cap, int nT_cap, int npend_max) {
  return (size_t)(MAXI + 1) * sizeof(PrepItem) + (size_t)cap * sizeof(int) +
         (size_t)((nT_cap + 1 + 3) & ~3) * sizeof(int) + (size_t)4 * npend_max * sizeof(TS);
}

}  // namespace

int launch_prep(const PrepParams& prm, int s_prec, int vec64, int npend_max, int num_sms,
                int max_ctas, int64_t nnz_bound, cudaStream_t st) {
  if (prm.nT <= 0) return 0;
  if (prm.item < 0 || prm.cap < 0 || (prm.cap & 3)) return 1;
  const size_t smem = (s_prec == 64) ? prep_smem<double>(prm.cap, prm.nT_cap, npend_max)
                                     : prep_smem<float>(prm.cap, prm.nT_cap, npend_max);
  const void* fn = (s_prec == 64) ? (const void*)k_prep<double, double>
                   : vec64        ? (const void*)k_prep<double, float>
                                  : (const void*)k_prep<float, float>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PG, smem) != cudaSuccess)
    return 1;
  if (per_sm <= 0) return 2;
  // one CTA per item (at most nT + nnz / item of them), at most all
  // co-resident CTAs
  const int full = per_sm * num_sms;
  int grid = full;
  const int item = prm.item > 0 ? prm.item : 1024;
  grid = (int)std::min<int64_t>((int64_t)prm.nT + nnz_bound / item + 1, full);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  grid = std::max(grid, 1);
  if ((prm.nT + grid - 1) / grid > PREP_MT) return 2;
  if (prm.npend > npend_max) return 1;
  PrepParams a = prm;
  if (a.item == 0) a.item = 1024;
  a.mt = (prm.nT + grid - 1) / grid;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel(fn, grid, PG, args, smem, st) != cudaSuccess) return 1;
  return 0;
}

}  // namespace sr
