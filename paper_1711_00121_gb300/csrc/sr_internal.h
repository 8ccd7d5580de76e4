// Internal declarations of libsimrank (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/simrank.h"

namespace sr {

// Edge of an S tile and height of a panel block.  S is padded to a multiple
// of PT in both dimensions; panels are stored tile-blocked:
//   panel[((T * 2 + which) * K1 + k) * PT + r]   for node a = T * PT + r,
// which = 0 for xi_k, 1 for eta_k, k = 0..K (K1 = K + 1 terms).
constexpr int PT = 128;

// Element (r, c) of S when only the tiles on or above the block diagonal are
// kept (upper = true): an element of a lower tile is read from its mirror.
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ T s_at(const T* S, int64_t ld, int64_t r, int64_t c, bool upper) {
  return (upper && (r / PT) > (c / PT)) ? S[c * ld + r] : S[r * ld + c];
}
#endif

#ifdef __CUDACC__
// x rounded to TF32 (10 explicit mantissa bits), to nearest, ties to even
__device__ __forceinline__ float tf32_rne(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // inf / nan unchanged
  u += 0x0fffu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xffffe000u);
}
#endif

inline int64_t panel_index(int64_t node, int which, int k, int K1) {
  return (((node / PT) * 2 + which) * (int64_t)K1 + k) * PT + (node % PT);
}

// Graph patch operation applied on the device in order (exact integer work).
struct PatchOp {
  int32_t kind;  // see PatchKind
  int32_t v;     // value (col id, length) or copy length
  int64_t a;     // destination index
  int64_t b;     // source index / start value
};
enum PatchKind : int32_t {
  PK_IN_COL = 0,    // in_col[a] = v
  PK_OUT_COL = 1,   // out_col[a] = v
  PK_IN_LEN = 2,    // in_len[a] = v
  PK_OUT_LEN = 3,   // out_len[a] = v
  PK_IN_START = 4,  // in_start[a] = b
  PK_OUT_START = 5, // out_start[a] = b
  PK_IN_COPY = 6,   // in_col[a .. a+v) = in_col[b .. b+v)
  PK_OUT_COPY = 7,  // out_col[a .. a+v) = out_col[b .. b+v)
};

// Adjacency lists with per-row slack, mirrored bit-for-bit on host and device.
struct HostAdj {
  std::vector<int64_t> start;
  std::vector<int32_t> len, cap;
  std::vector<int32_t> pool;
  int64_t used = 0;
};

struct DevAdj {
  int64_t* start = nullptr;
  int32_t* len = nullptr;
  int32_t* col = nullptr;
  int64_t pool_cap = 0;
};

// Device counters (int64): see Counter.
enum Counter : int {
  CNT_TILES_TOUCHED = 0,
  CNT_S_BYTES = 1,
  CNT_PANEL_BYTES = 2,
  CNT_STATUS = 3,
  CNT_N = 8
};

// Sets the message that simrank_last_error(NULL) returns on this thread.
void set_global_error(const std::string& msg);

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All are asynchronous on `st`.
// ---------------------------------------------------------------------------

// sI[a] = sum_t S[I[t], a], sJ[a] = S[j, a] (a < n_pad, FP64);
// scal[0] = sum_{t,t'} S[I[t], I[t']], scal[1] = S[j, j],
// scal[2] = w_j = (1/delta) [Q]_{j,*} S_{*,I} on the graph `in` (the old one).
void launch_gather_rows(const void* S, int s_prec, int64_t ld, const int32_t* I, int delta, int j,
                        int n_pad, const DevAdj& in, double* sI, double* sJ, double* scal,
                        cudaStream_t st, int upper = 0);

// gamma of Thm 3 / Thm 9 / Table 2 on the OLD graph; writes xi_0 = C e_j and
// eta_0 = gamma into the panels (FP64 and, for FP32 S, FP32) and writes the
// k = 0 AFF mask words of tiles [0, nT).
void launch_gamma(const DevAdj& in, const double* sI, const double* sJ, const double* scal, int j,
                  int delta, int op, int d_j, double C, int nT, int K1, double* P64, float* P32,
                  uint64_t* mXi, uint64_t* mEta, cudaStream_t st);

// Deferred S updates: rows of the current S = S + the pending panels Pp
// (tile-blocked FP32 [T][which][GK1][128], nterms used terms).
void launch_gather_rows_pending(const void* S, int s_prec, int64_t ld, const int32_t* I, int delta,
                                int j, int n_pad, const float* Pp, int GK1, int nterms, double* sI,
                                double* sJ, cudaStream_t st, int upper = 0);
// scal[0] = sum_t sI[I_t], scal[1] = sJ[j], scal[2] = (1/(delta d_j)) sum_{b in I(j)} sI[b]
void launch_scalars_from_rows(const DevAdj& in, const double* sI, const double* sJ, const int32_t* I,
                              int delta, int j, double* scal, cudaStream_t st);
// pXi[T] = 1 if mXi[T] != 0 (and the same for eta); other entries unchanged
void launch_or_any(const uint64_t* mXi, const uint64_t* mEta, int nT, uint64_t* pXi, uint64_t* pEta,
                   cudaStream_t st);
// tensor-core operands (row-major hi/lo, kd columns) from tile-blocked FP32 panels
void launch_pack_tc_tiles(const float* Pp, int GK1, int nterms, int rg, int n_rows, float* Ahi,
                          float* Alo, int64_t kd, cudaStream_t st);

// Apply patch ops [begin, end) to the device adjacency (one CTA, in order).
void launch_patch(const PatchOp* ops, int64_t begin, int64_t end, DevAdj in, DevAdj out,
                  cudaStream_t st);

// One step of the xi/eta recurrence on the NEW graph (Eq. 16a):
// xi_{k+1} = C Q xi_k, eta_{k+1} = Q eta_k; ORs bit (k+1) % 64 into the AFF masks.
void launch_chain_step(const DevAdj& in, int k, double C, int nT, int K1, double* P64, float* P32,
                       uint64_t* mXi, uint64_t* mEta, cudaStream_t st);

// Everything a rank-one update does before its S pass, in one cooperative
// launch (k_prep.cu): patch ops [op_begin, op_end), the rows sI, sJ of the
// current S (panel terms [0, npend) of P not yet in S are added in), gamma
// into term koff of P, K recurrence steps into terms koff+1 .. koff+K, the
// mask words mXi/mEta of tiles [0, nT) (ORed as 0/1 into pXi/pEta when
// those are set) and, when `tiles` is set, the tile-pair list (tile_mode 0 =
// all pairs, 1 = AFF-pruned).  P is tile-blocked [T][which][ldk][128] in the
// precision of S; sI, sJ hold n_pad values of the vector precision (FP64 when
// vec64 or S is FP64, else FP32); W is the working buffer [K+1][n_pad] of
// (xi, eta) pairs of the vector precision; tile_nnz holds nT_cap ints.  Gathers are split into items of at most `item`
// nonzeros; `cap` column indices are cached per CTA (a multiple of 4).
// bar: two zeroed unsigned ints, left zeroed.  nnz_bound bounds the edges of
// the new graph (it sizes the grid).  Returns 0 on launch, 2 when the graph
// has more tiles than the co-resident CTAs can own (use the per-step path),
// 1 on a launch error.
struct PrepParams {
  DevAdj in, out;
  const PatchOp* ops;
  int64_t op_begin, op_end;
  const void* S;
  int64_t ld;
  const int32_t* I;
  int delta, j, op, d_j;
  double C;
  // quotients that are the same for every row, computed once on the host (a
  // division in the kernel would be issued by every thread): 1 / C, 1 / delta
  // and delta / (d_j + op delta) (0 when that sum is 0)
  double inv_C, inv_delta, gq;
  int mt;  // tiles per CTA, ceil(nT / grid) (set by launch_prep)
  int K;
  int nT;
  void* P;
  int ldk, koff, npend;
  void* sI;
  void* sJ;
  uint64_t *mXi, *mEta, *pXi, *pEta;
  uint32_t* tiles;
  int* ntiles;
  int tile_mode;
  int upper;  // 1: only tiles on or above the block diagonal of S are kept
  int cap;
  int item;
  int n_pad, nT_cap;
  void* W;
  void* rinv;  // per row: (C / in-degree, 1 / in-degree) in the vector precision, n_pad pairs
  int* loff;   // per row: nonzeros of its tile before it (n_pad)
  int flat;    // 1: split the nonzeros evenly over the CTAs when two per thread suffice
  int* tile_nnz;
  unsigned int* bar;
  long long limit;
  unsigned long long* counters;
};
int launch_prep(const PrepParams& p, int s_prec, int vec64, int npend_max, int num_sms,
                int max_ctas, int64_t nnz_bound, cudaStream_t st);

// ---------------------------------------------------------------------------
// Many independent graphs advanced together (k_multi.cu).
// ---------------------------------------------------------------------------
// One graph: its dense S (precision of the handle), tile-blocked panels
// [T][which][K1][128] in the same precision, AFF words, adjacency, and the
// sI/sJ scratch rows (n_pad values each).
struct MultiGraphDesc {
  void* S;
  int64_t ld;
  void* P;
  uint64_t* mXi;
  uint64_t* mEta;
  DevAdj in, out;
  void* sI;
  void* sJ;
  int n;      // current node count (byte counters)
  int upper;  // 1: only tiles on or above the block diagonal are kept
  int64_t row_off;  // first row of this graph in the shared tensor-core operands
};
// One rank-one update of graph g in a round: sources srcs[src_off ..
// src_off + delta) into sink j, op = +1/-1, old in-degree d_j, patch ops
// [op_begin, op_end), node count after the update n_after.
struct MultiStep {
  int32_t g, j, op, d_j, delta, n_after;
  int64_t src_off, op_begin, op_end;
};
// Rank-one work before the S pass for steps[0 .. *count) (one CTA each, grid
// >= *count): patch, rows of S, gamma, K recurrence steps, masks, and the
// tile pairs (g << 32 | I << 16 | J) appended to tiles / *ntiles.
void launch_multi_prep(int s_prec, const MultiGraphDesc* descs, const MultiStep* steps,
                       const int* count, int grid, const int32_t* srcs, const PatchOp* ops,
                       double C, int K, int aff, uint64_t* tiles, int* ntiles, cudaStream_t st);
// S pass over the tile pairs of many graphs (single-role CUDA-core kernel).
void launch_s_update_multi(int s_prec, const MultiGraphDesc* descs, const uint64_t* tiles,
                           const int* ntiles, int K1, int64_t* counters, int grid,
                           cudaStream_t st);

// Affected tile pairs (I <= J) of Thm 4 at tile granularity.
// The chain step with tiles cut into items of at most chain_item_size()
// nonzeros (item_tile / item_sub per item, tile_items per tile); gacc (2 * 128
// doubles per tile) and tile_count (per tile) must start at zero and are left
// at zero.
void launch_chain_step_items(const DevAdj& in, const int* item_tile, const int* item_sub,
                             const int* tile_items, int n_items, int k, double C, int K1,
                             double* P64, float* P32, uint64_t* mXi, uint64_t* mEta, double* gacc,
                             unsigned int* tile_count, cudaStream_t st);
int chain_item_size();
void launch_tile_list(const uint64_t* mXi, const uint64_t* mEta, int nT, int aff, uint32_t* tiles,
                      int* ntiles, cudaStream_t st);

// S[I,J] += sum_{k in [k0,k1)} xi_k[I] eta_k[J]^T + eta_k[I] xi_k[J]^T, and the
// mirrored tile S[J,I], over the tile list.  n = current node count (for the
// algorithmic byte counters).
// Raises a kernel's dynamic shared-memory limit once per device: the attribute
// belongs to the current device's context, so each device of the process needs
// its own call (bit d of `done` records device d; devices past 63 set it on
// every launch).  Two threads may both set it; that is harmless.
inline cudaError_t smem_attr_once(const void* fn, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// With S in FP32 and ws_wait_limit > 0 the warp-specialised kernel runs (its
// mbarrier waits are bounded by ws_wait_limit iterations); otherwise the
// single-role kernel.
void launch_s_update(void* S, int s_prec, int64_t ld, const void* P, int K1, const uint32_t* tiles,
                     const int* ntiles, const uint64_t* mXi, const uint64_t* mEta, int k0, int k1,
                     int use_masks, int n, int64_t* counters, int grid, cudaStream_t st,
                     long long ws_wait_limit = 0, int upper = 0);
// Persistent grid for launch_s_update on this device (ws: warp-specialised).
int s_update_grid(int s_prec, int num_sms, bool ws = false);

// Jacobi sweep pieces for Eq. 1 (init / re-anchor).
// Y[a, :] = scale * sum_b Q[a, b] X[b, :] + diag * e_a (the diagonal term only
// for a < n_diag), rows a < n_rows, columns < ncols (a multiple of 4).
void launch_spmm_rows(const DevAdj& in, const float* w, const double* wsum, const void* X,
                      int x_prec, int64_t ldx, void* Y, int y_prec, int64_t ldy, int n_rows,
                      int ncols, double scale, double diag, int n_diag, cudaStream_t st);
void launch_transpose(const void* A, void* B, int prec, int n_pad, int64_t ld, cudaStream_t st);
// *out_bits = max(*out_bits, max |A - B|) over the n x n block (as double bits)
void launch_maxdiff(const void* A, const void* B, int prec, int n, int64_t ld,
                    unsigned long long* out_bits, cudaStream_t st);
// S[J, I] = S[I, J]^T for all 128-tiles I < J (restores the lower triangle)
void launch_mirror_lower(void* A, int prec, int n_pad, int64_t ld, cudaStream_t st);
void launch_symmetrize(void* A, int prec, int n_pad, int64_t ld, cudaStream_t st);
// B[e] = A[e] for e < count, converting between FP32 and FP64.
void launch_convert(const void* A, int a_prec, void* B, int b_prec, int64_t count, cudaStream_t st);
void launch_set_diag(void* A, int prec, int from, int to, int64_t ld, double value, cudaStream_t st);
// S of a forest of arborescences in closed form (Example 2): parent[x] (-1 at
// a root) and level[x] for x < n, powC[k] = C^k; S is ld-pitched, nT tiles a side.
void launch_forest_init(void* S, int prec, int64_t ld, const int32_t* parent, const int32_t* level,
                        const double* powC, int n, int nT, int upper, cudaStream_t st);

// out[c * n + a] = S[cols[c], perm[a]]  (column c of the symmetric S in caller
// order; perm maps caller ids to storage ids, nullptr = identity)
void launch_copy_cols(const void* S, int s_prec, int64_t ld, const int32_t* cols, const int32_t* perm,
                      int ncols, int n, void* out, int out_fp64, cudaStream_t st, int upper = 0);

// ---- one-shot batch (rank-2r) pieces, k_batch.cu
// Zc[t][a] = sum_{e in block t} sign[e] * S[src[e], a], a < n_pad
void launch_signed_rows(const void* S, int s_prec, int64_t ld, const int32_t* src, const int8_t* sign,
                        const int64_t* off, int r, int n_pad, double* Zc, cudaStream_t st, int upper = 0);
// B[c * ldb + r] = A[r * lda + c]
void launch_transpose_rect(const double* A, int64_t lda, double* B, int64_t ldb, int rows, int cols,
                           cudaStream_t st);
// Lambda = V^T S V (r x r) from S rows of the sinks, Y = Q Z and Z (row-major, ldz)
void launch_lambda(const void* S, int s_prec, int64_t ld, const int32_t* sinks, const double* av,
                   const double* bv, const double* Y, const double* Z, int64_t ldz,
                   const int32_t* src, const int8_t* sign, const int64_t* off, int r, double C,
                   double* Lam, cudaStream_t st, int upper = 0);
// Wc[t][a] = a_t (S[j_t,a] - (1-C)[a==j_t]) / C + b_t Yc[t][a] + Lambda[u][t]/2 [a == j_u]
void launch_w_assemble(const void* S, int s_prec, int64_t ld, const int32_t* sinks, const double* av,
                       const double* bv, const double* Yc, const double* Lam, int r, int n_pad,
                       double C, double* Wc, cudaStream_t st, int upper = 0);
void launch_xi0(const int32_t* sinks, int r, double C, double* X0, int64_t ldx, cudaStream_t st);
void launch_pack_ffma(const double* X, int64_t ldx, int rh, int r, int slot, int terms, int nT,
                      void* Pn, int p_prec, uint64_t* mXi, uint64_t* mEta, cudaStream_t st);
void launch_pack_tc(const double* X, int64_t ldx, int rh, int r, int slot, int rg, int n_rows,
                    float* Ahi, float* Alo, int64_t kd, cudaStream_t st);
// The same operands in FP16 with each term balanced by a power of two
// (maxes: 2 r unsigned ints of scratch).
void launch_pack_f16_oneshot(const double* X, int64_t ldx, int rh, int r, int slot, int rg,
                             int n_rows, unsigned int* maxes, void* Ahi, void* Alo, int64_t kd,
                             cudaStream_t st);
// Operand rows at least this wide (bytes) make the tensor-core S pass bound by
// the tensor cores rather than by the S stream.
constexpr int64_t TC_WIDE_K_BYTES = 1024;
// tcgen05 symmetric update S += A B^T (B = A with halves swapped), 3-term
// split (TF32, or FP16 when f16); returns 0 on launch, 1 for a bad shape, 2 if
// no tensor map could be encoded.  Bhi / Blo: B stored on its own (kd a
// multiple of 128 bytes), else B is read from A by swapping the two halves'
// TMA boxes (kd a multiple of 256 bytes).
// tiles[0 .. nt): tile pairs (I << 16 | J) in the order CTAs take them; a
// pair is skipped when use_masks and (mX[I] & mE[J]) | (mE[I] & mX[J]) == 0.
// jobs[0 .. nj) (may be null): the same pairs, two per job where they share I
// (I << 32 | J1 << 16 | J2, J2 = 0xffff for one), taken instead of tiles when
// only upper tiles are kept and the operands are at least 1 KB wide.
int launch_s_update_tc(float* S, int64_t ld, const void* Ahi, const void* Alo, int64_t n_rows,
                       int64_t kd, const uint32_t* tiles, int nt, const uint64_t* jobs, int nj,
                       const uint64_t* mX, const uint64_t* mE, int use_masks, int n,
                       int64_t* counters, int grid, long long wait_limit, cudaStream_t st,
                       int upper = 0, int f16 = 0, const void* Bhi = nullptr,
                       const void* Blo = nullptr);
// The same pass over the tile pairs (g << 32 | I << 16 | J) of many graphs,
// *ntiles of them; graph g's operand rows start at descs[g].row_off of the
// shared operands A_hi / A_lo ([rows][kd]).
int launch_s_update_tc_multi(const void* Ahi, const void* Alo, int64_t rows, int64_t kd,
                             const MultiGraphDesc* descs, const uint64_t* tiles, const int* ntiles,
                             int64_t* counters, int grid, long long wait_limit, cudaStream_t st,
                             int f16, int upper);
// Tensor-core operands of the graphs of steps[0 .. *count) from their
// tile-blocked panels (K1 terms, TF32 split, rg columns per half): rows
// descs[g].row_off + a for a < nT_g * 128.  max_tiles bounds nT_g.
void launch_multi_pack_tc(const MultiGraphDesc* descs, const MultiStep* steps, const int* count,
                          int grid, int max_tiles, int K1, int rg, float* Ahi, float* Alo,
                          int64_t kd, cudaStream_t st);
// FP16 operands (row-major [n_rows][kd] hi/lo) from tile-blocked FP32 pending
// panels, each term scaled by 2^(+-e_q) (exact); maxes: 2 * nterms scratch uints.
void launch_pack_f16_tiles(const float* Pp, int GK1, int nterms, int rg, int n_rows,
                           unsigned int* maxes, void* Ahi, void* Alo, void* Bhi, void* Blo,
                           int64_t kd, cudaStream_t st);

// ---- column mode (§7), k_column.cu
// A piece of one adjacency row: row id, count (<= kChunk) and pool offset.
struct RowChunk {
  int32_t row;
  int32_t len;
  int64_t start;
};
constexpr int kChunk = 32;
struct ChunkList {
  RowChunk* chunks = nullptr;  // device
  int64_t count = 0;
};
// Y[a][c] += scale / len(a) * sum over a's in-list of X[b][c], columns c <
// ncols (a multiple of 4), by row chunks (FP64 atomics into Y, which the
// caller zeroes); X 16-byte aligned with even ldx.  Returns 1 for a bad shape.
int launch_spmm_chunks64(const RowChunk* chunks, int64_t count, const int32_t* col,
                         const int32_t* len, const double* X, int64_t ldx, double* Y, int64_t ldy,
                         int ncols, double scale, cudaStream_t st);
// Edge weights of a weighted Q (all null: Q[a][b] = 1 / in-degree(a)):
// out_w / in_w give the weight of each out-list / in-list entry by pool
// position, wsum[a] the total in-weight of a.
struct WeightView {
  const float* out_w = nullptr;
  const float* in_w = nullptr;
  const double* wsum = nullptr;
};
// Procedure 1 on B columns `cols` (device) of the graph whose out-lists
// (fwd chunks over out_col) and in-lists (hor chunks over in_col) are given;
// in_len = in-degrees.  xs holds (K+1) row-major [n_rows][B] blocks, y0 / y1
// are scratch blocks, result receives (1-C) sum_k C^k Q^k (Q^T)^k e_cols.
void launch_partial_sim_block(const ChunkList& fwd, const ChunkList& hor, const int32_t* out_col,
                              const int32_t* in_col, const int32_t* in_len, const int32_t* cols,
                              int B, int n_rows, int K, double C, int prec, void* xs, void* y0,
                              void* y1, void* result, cudaStream_t st,
                              const WeightView& wv = WeightView(), int group0 = 1);
void launch_col_forward64(const ChunkList& fwd, const int32_t* out_col, const WeightView& wv,
                          const int32_t* in_len, const double* X, double* Y, int B, int n_rows,
                          cudaStream_t st);
void launch_col_horner64(const ChunkList& hor, const int32_t* in_col, const WeightView& wv,
                         const int32_t* in_len, const double* Xadd, double add_scale,
                         const double* Y, double* Yn, int B, int n_rows, double scale,
                         cudaStream_t st);
// Y[a][c] += sum_k xi_k[a] eta_k[cols[c]] + eta_k[a] xi_k[cols[c]] (panels P, FP32/64)
// FP32 blocks: Y[a][c] += sum over the U stored updates (device array of
// their panel pointers, tile-blocked FP32) of xi_k[a] eta_k[x_c] +
// eta_k[a] xi_k[x_c], as one product; G: scratch of U * 2 * K1 * round4(B)
// floats.  n_rows is a multiple of 128.
void launch_col_corr(const float* const* hist, int U, int K1, const int32_t* cols, int B,
                     int n_rows, float* G, float* Y, cudaStream_t st);
void launch_col_apply(const void* P, int p_prec, int K1, const int32_t* cols, int B, int n_rows,
                      int prec, void* Y, cudaStream_t st);
// scal[0] = si[i], scal[1] = sj[j], scal[2] = (1/d_j) sum_{b in I(j)} si[b]
void launch_col_scalars(const DevAdj& in, const double* si, const double* sj, int i, int j,
                        double* scal, cudaStream_t st);
void launch_col_out(const void* Y, int prec, int B, int n, void* out, int out_fp64, cudaStream_t st);
void launch_col_extract(const void* Y, int prec, int B, int c, int n, double* v, cudaStream_t st);

// ---- adjoint (k_adjoint.cu)
// G[e] += scale * sum_{x < B} F[u][x] Y[v][x] for every in-list entry e (row u,
// in-neighbour v = col[e]) covered by the chunks
void launch_adj_sddmm(const ChunkList& hor, const int32_t* in_col, const double* F, const double* Y,
                      int B, double scale, double* G, cudaStream_t st);
// X[node[t]][c[t]] += coef[t] for t < count (X zeroed before)
void launch_adj_scatter(const int32_t* node, const int32_t* c, const double* coef, int64_t count,
                        int B, double* X, cudaStream_t st);
// out[t] = Y[row[t]][c[t]]
void launch_adj_pairs(const double* Y, int B, const int32_t* row, const int32_t* c, int64_t count,
                      double* out, cudaStream_t st);
// chain rule Q[a][b] = w_ba / wsum_a: dW[e] = (G[e] - sum_{e' in row a} G[e'] Q[e']) / wsum_a
void launch_adj_weights(const DevAdj& in, const WeightView& wv, int n_rows, const double* G,
                        double* dW, cudaStream_t st);

}  // namespace sr
