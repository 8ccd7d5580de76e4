// C ABI of libsimrank and its host engine: validation, graph bookkeeping
// (mirrored CSR/CSC with per-row slack, exact integer patches), batch
// planning (§8 net update and similar-sink partition), and the stream-ordered
// launch sequence of each rank-one update.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "sr_internal.h"

using namespace sr;

namespace {

thread_local std::string g_init_error;

}  // namespace

namespace sr {
void set_global_error(const std::string& msg) { g_init_error = msg; }
}  // namespace sr

struct simrank_ctx {
  simrank_config cfg{};
  cudaStream_t st = nullptr;
  int device = 0;
  int num_sms = 0;
  int n_cur = 0, n_cap = 0, n_pad = 0, nT_cap = 0, K1 = 0;
  int64_t since_anchor = 0;  // updates since the last automatic re-anchor
  int64_t ld = 0;
  bool weighted = false;
  // caller id <-> storage id (identity unless cfg.relabel)
  bool relabeled = false;
  std::vector<int32_t> ext2int, int2ext;
  int32_t* d_ext2int = nullptr;
  // host mirror of the graph (storage ids)
  HostAdj hin, hout;
  std::unordered_set<uint64_t> edges;
  // device graph
  DevAdj din, dout;
  float* d_in_w = nullptr;
  float* d_out_w = nullptr;
  double* d_wsum = nullptr;
  std::vector<int32_t> init_src, init_dst;  // initial edges in storage ids, caller order
  // dense S and panels
  void* S = nullptr;
  double* P64 = nullptr;
  float* P32 = nullptr;
  uint64_t* mXi = nullptr;
  uint64_t* mEta = nullptr;
  uint32_t* tiles = nullptr;
  int* ntiles = nullptr;
  double* sI = nullptr;
  double* sJ = nullptr;
  double* scal = nullptr;
  int64_t* counters = nullptr;
  unsigned long long* diffbits = nullptr;
  unsigned int* gbar = nullptr;  // grid barrier state of the cooperative pre-update kernel
  uint32_t* d_order = nullptr;   // all tile pairs I <= J in band order (tensor-core S pass)
  uint32_t* d_order_row = nullptr;  // the same pairs in row-major order (narrow operands)
  int order_nT = -1;
  int order_n = 0;
  uint64_t* d_jobs = nullptr;    // the same pairs, two per job where they share I
  int jobs_n = 0;
  void* W = nullptr;              // (xi, eta) working columns of the pre-update kernel
  void* rinv = nullptr;           // its per-row (C / in-degree, 1 / in-degree)
  int32_t* loff = nullptr;        // its per-row offsets inside the tile
  int* tile_nnz = nullptr;       // per-tile nonzeros (scratch of the pre-update kernel)
  // per-call staging
  int32_t* d_srcs = nullptr;
  int64_t srcs_cap = 0;
  PatchOp* d_ops = nullptr;
  int64_t ops_cap = 0;
  int32_t* d_cols = nullptr;
  int64_t cols_cap = 0;
  // column mode (§7): snapshot of the initial graph and the stored updates
  bool column = false;
  int32_t* g0_in_col = nullptr;
  int32_t* g0_out_col = nullptr;
  int32_t* g0_in_len = nullptr;
  ChunkList g0_fwd, g0_hor, cur_fwd, cur_hor;
  int64_t cur_fwd_cap = 0, cur_hor_cap = 0;
  // column mode: host copies of cur_fwd / cur_hor with the first chunk of
  // every row, kept current row by row between updates
  std::vector<RowChunk> hfwd, hhor;
  std::vector<int64_t> ffwd, fhor;
  bool col_chunks_ok = false;
  std::vector<int32_t> col_last_srcs;  // sources and sink of the last stored update
  int col_last_j = -1;
  std::vector<void*> hist;  // per-update panel snapshots (tile-blocked, S precision)
  // one-shot batch scratch (grow-only)
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  } ob[28];
  // column mode: per-tile nonzeros of the in-lists (host), the work-item table
  // of the chain steps and its partial-sum accumulators (device)
  std::vector<int64_t> col_tnnz;
  int32_t* col_items = nullptr;  // item_tile | item_sub | tile_items
  int64_t col_items_cap = 0;
  double* col_gacc = nullptr;    // 2 x 128 doubles per tile, kept at zero between steps
  unsigned int* col_tcount = nullptr;
  // deferred S updates: pending panels [T][which][G*K1][128] (FP32), count, tile masks
  float* Pp = nullptr;
  int np = 0;
  uint64_t* pXi = nullptr;
  uint64_t* pEta = nullptr;
  // profiling
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  size_t events_used = 0;
  double prof_ms = 0.0;
  std::vector<std::array<cudaEvent_t, 5>> phase_ev;
  size_t phase_used = 0;
  double phase_ms[4] = {0, 0, 0, 0};
  int64_t prof_launches = 0;
  int64_t launches = 0;  // every kernel launch of this handle
  // stats
  simrank_stats stats{};
  std::string err;
};

namespace {

simrank_status fail(simrank_ctx* h, simrank_status s, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_init_error = msg;
  return s;
}

#define CUDA_TRY(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess)                                                                \
      return fail((h), e__ == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e__));                    \
  } while (0)

#define LAUNCH_CHECK(h)                                                                    \
  do {                                                                                     \
    cudaError_t e__ = cudaGetLastError();                                                  \
    if (e__ != cudaSuccess)                                                                \
      return fail((h), SR_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e__)); \
  } while (0)

inline uint64_t ekey(int32_t s, int32_t d) { return ((uint64_t)(uint32_t)s << 32) | (uint32_t)d; }

inline int elem_bytes(const simrank_ctx* h) { return h->cfg.s_precision == 64 ? 8 : 4; }

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

// Builds adjacency lists (rows indexed by `key`, entries `val`) with per-row
// slack.  Row capacities are multiples of 4, so every row starts on a 16-byte
// boundary of the pool (vector loads of whole rows).
void build_adj(HostAdj& A, int n_rows, const std::vector<std::vector<int32_t>>& rows) {
  A.start.assign(n_rows, 0);
  A.len.assign(n_rows, 0);
  A.cap.assign(n_rows, 0);
  int64_t used = 0;
  for (int a = 0; a < n_rows; ++a) {
    const int len = (int)rows[a].size();
    const int cap = (len + std::max(4, len / 4) + 3) & ~3;
    A.start[a] = used;
    A.len[a] = len;
    A.cap[a] = cap;
    used += cap;
  }
  A.pool.assign((size_t)(used + used / 4 + 65536), 0);
  for (int a = 0; a < n_rows; ++a)
    std::copy(rows[a].begin(), rows[a].end(), A.pool.begin() + A.start[a]);
  A.used = used;
}

// Appends `v` to row r of the mirror, recording the device patch ops.
void adj_append(HostAdj& A, int r, int32_t v, std::vector<PatchOp>& ops, bool is_in) {
  if (A.len[r] == A.cap[r]) {
    const int new_cap = (2 * A.len[r] + 4 + 3) & ~3;
    const int64_t ns = A.used;
    if ((int64_t)A.pool.size() < ns + new_cap) A.pool.resize((size_t)(2 * (ns + new_cap)), 0);
    std::copy(A.pool.begin() + A.start[r], A.pool.begin() + A.start[r] + A.len[r],
              A.pool.begin() + ns);
    ops.push_back({is_in ? PK_IN_COPY : PK_OUT_COPY, A.len[r], ns, A.start[r]});
    ops.push_back({is_in ? PK_IN_START : PK_OUT_START, 0, (int64_t)r, ns});
    A.start[r] = ns;
    A.cap[r] = new_cap;
    A.used += new_cap;
  }
  const int64_t pos = A.start[r] + A.len[r];
  A.pool[pos] = v;
  A.len[r] += 1;
  ops.push_back({is_in ? PK_IN_COL : PK_OUT_COL, v, pos, 0});
  ops.push_back({is_in ? PK_IN_LEN : PK_OUT_LEN, A.len[r], (int64_t)r, 0});
}

// Removes `v` from row r (swap with the last entry), recording the patch ops.
void adj_remove(HostAdj& A, int r, int32_t v, std::vector<PatchOp>& ops, bool is_in) {
  const int64_t s = A.start[r];
  const int len = A.len[r];
  int p = -1;
  for (int e = 0; e < len; ++e)
    if (A.pool[s + e] == v) {
      p = e;
      break;
    }
  if (p < 0) return;  // validated earlier; cannot happen
  const int last = len - 1;
  if (p != last) {
    A.pool[s + p] = A.pool[s + last];
    ops.push_back({is_in ? PK_IN_COL : PK_OUT_COL, A.pool[s + p], s + p, 0});
  }
  A.len[r] = last;
  ops.push_back({is_in ? PK_IN_LEN : PK_OUT_LEN, last, (int64_t)r, 0});
}

// ---------------------------------------------------------------------------
// Batch planning (§8): net update, sign split, similar-sink partition.
// ---------------------------------------------------------------------------
struct Block {
  int32_t sink;
  int32_t op;
  std::vector<int32_t> srcs;
};

simrank_status plan_blocks(const simrank_update* u, int64_t count, int32_t n_old,
                           std::vector<Block>& out, std::string& msg) {
  std::unordered_map<uint64_t, int> cnt;
  std::vector<uint64_t> order;
  cnt.reserve((size_t)count * 2);
  for (int64_t t = 0; t < count; ++t) {
    const uint64_t k = ekey(u[t].src, u[t].dst);
    auto it = cnt.find(k);
    if (it == cnt.end()) {
      cnt.emplace(k, 0);
      order.push_back(k);
    }
    cnt[k] += (u[t].op > 0) ? 1 : -1;
  }
  std::map<int32_t, std::vector<int32_t>> plus, minus;
  for (uint64_t k : order) {
    const int c = cnt[k];
    const int32_t s = (int32_t)(k >> 32), d = (int32_t)(k & 0xffffffffu);
    if (c == 1)
      plus[d].push_back(s);
    else if (c == -1)
      minus[d].push_back(s);
    else if (c != 0) {
      msg = "net count " + std::to_string(c) + " for edge (" + std::to_string(s) + "," +
            std::to_string(d) + ")";
      return SR_ERR_ARG;
    }
  }
  out.clear();
  for (auto& kv : minus) {
    std::vector<int32_t> s = kv.second;
    std::sort(s.begin(), s.end());
    out.push_back({kv.first, -1, s});
  }
  // Insertion sub-blocks: per sink (ascending) the sources in the old V, then
  // the new ones.  A sub-block is split again by the node set at the time it
  // runs (sources that an earlier sub-block of this batch created come first),
  // so every block is one of the cases C0..C3 of §8 when it is applied.
  std::unordered_set<int32_t> created;
  auto exists = [&](int32_t x) { return x < n_old || created.count(x) != 0; };
  for (auto& kv : plus) {
    std::vector<int32_t> olds, news;
    for (int32_t s : kv.second) (s < n_old ? olds : news).push_back(s);
    std::sort(olds.begin(), olds.end());
    std::sort(news.begin(), news.end());
    for (const std::vector<int32_t>* sub : {&olds, &news}) {
      if (sub->empty()) continue;
      std::vector<int32_t> have, fresh;
      for (int32_t s : *sub) (exists(s) ? have : fresh).push_back(s);
      if (!have.empty()) out.push_back({kv.first, +1, have});
      if (!fresh.empty()) out.push_back({kv.first, +1, fresh});
      for (int32_t s : *sub) created.insert(s);
      created.insert(kv.first);
    }
  }
  return SR_OK;
}

// Sequential validation of a batch against the current graph (no mutation).
// New nodes are the ids >= n_cur that the batch names; as a set they must be
// exactly n_cur, n_cur + 1, ... (in any order of appearance) and stay below
// n_capacity.  An edge may be deleted only if present at that point of the
// sequence.
simrank_status validate(simrank_ctx* h, const simrank_update* u, int64_t count, int* n_after) {
  std::unordered_map<uint64_t, char> overlay;
  int max_id = h->n_cur - 1;
  std::unordered_set<int32_t> fresh;
  for (int64_t t = 0; t < count; ++t) {
    const int32_t s = u[t].src, d = u[t].dst;
    const std::string at = " (update " + std::to_string(t) + ": " + std::to_string(s) + " -> " +
                           std::to_string(d) + ")";
    if (u[t].op != 1 && u[t].op != -1) return fail(h, SR_ERR_ARG, "op must be +1 or -1" + at);
    if (s < 0 || d < 0) return fail(h, SR_ERR_ARG, "negative node id" + at);
    if (s == d) return fail(h, SR_ERR_EDGE_EXISTS, "self-loop" + at);
    for (int32_t x : {s, d}) {
      if (x >= h->n_cur) {
        if (x >= h->n_cap) return fail(h, SR_ERR_CAPACITY, "n_capacity exceeded" + at);
        fresh.insert(x);
        max_id = std::max(max_id, (int)x);
      }
    }
    const uint64_t k = ekey(s, d);
    bool present;
    auto it = overlay.find(k);
    if (it != overlay.end())
      present = it->second != 0;
    else
      present = h->edges.count(k) != 0;
    if (u[t].op > 0) {
      if (present) return fail(h, SR_ERR_EDGE_EXISTS, "inserting an existing edge" + at);
      overlay[k] = 1;
    } else {
      if (!present) return fail(h, SR_ERR_EDGE_MISSING, "deleting an absent edge" + at);
      overlay[k] = 0;
    }
  }
  if ((int64_t)fresh.size() != (int64_t)max_id + 1 - h->n_cur)
    return fail(h, SR_ERR_ARG, "new node ids must be contiguous from n_cur = " +
                                   std::to_string(h->n_cur));
  *n_after = max_id + 1;
  return SR_OK;
}

simrank_status ensure_dev_capacity(simrank_ctx* h, int64_t nsrc, int64_t nops) {
  if (nsrc > h->srcs_cap) {
    if (h->d_srcs) cudaFree(h->d_srcs);
    h->srcs_cap = std::max<int64_t>(nsrc, 2 * h->srcs_cap);
    CUDA_TRY(h, dev_alloc(&h->d_srcs, (size_t)h->srcs_cap));
  }
  if (nops > h->ops_cap) {
    if (h->d_ops) cudaFree(h->d_ops);
    h->ops_cap = std::max<int64_t>(nops, 2 * h->ops_cap);
    CUDA_TRY(h, dev_alloc(&h->d_ops, (size_t)h->ops_cap));
  }
  return SR_OK;
}

// Grows a device column pool to hold the host mirror's pool (rare).
simrank_status grow_pool(simrank_ctx* h, DevAdj& D, const HostAdj& A) {
  if (A.used <= D.pool_cap) return SR_OK;
  const int64_t cap = std::max<int64_t>((int64_t)A.pool.size(), A.used * 2);
  int32_t* np = nullptr;
  CUDA_TRY(h, dev_alloc(&np, (size_t)cap));
  CUDA_TRY(h, cudaMemcpyAsync(np, D.col, (size_t)D.pool_cap * sizeof(int32_t),
                              cudaMemcpyDeviceToDevice, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  cudaFree(D.col);
  D.col = np;
  D.pool_cap = cap;
  return SR_OK;
}

// Iteration bound of every device-side wait of this handle.
long long wait_limit(const simrank_ctx* h) {
  return h->cfg.timeout_iters > 0 ? h->cfg.timeout_iters : (1ll << 24);
}

std::pair<cudaEvent_t, cudaEvent_t>* next_event_pair(simrank_ctx* h) {
  if (h->events_used == h->events.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&b) != cudaSuccess) return nullptr;
    h->events.push_back({a, b});
  }
  return &h->events[h->events_used++];
}

void harvest_events(simrank_ctx* h) {
  for (size_t e = 0; e < h->events_used; ++e) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->events[e].first, h->events[e].second) == cudaSuccess)
      h->prof_ms += ms;
  }
  h->events_used = 0;
  for (size_t e = 0; e < h->phase_used; ++e)
    for (int q = 0; q < 4; ++q) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->phase_ev[e][q], h->phase_ev[e][q + 1]) == cudaSuccess)
        h->phase_ms[q] += ms;
    }
  h->phase_used = 0;
}

// Events at the phase boundaries of one rank-one update (profile = 1 only).
cudaEvent_t* next_phase_events(simrank_ctx* h) {
  if (h->phase_used == h->phase_ev.size()) {
    std::array<cudaEvent_t, 5> a;
    for (auto& e : a)
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->phase_ev.push_back(a);
  }
  return h->phase_ev[h->phase_used++].data();
}

// 1 when only the tiles of S on or above the block diagonal are kept
int upper(const simrank_ctx* h) { return (h->cfg.upper_only && !h->column) ? 1 : 0; }

void* panel_for_s(simrank_ctx* h) {
  return h->cfg.s_precision == 64 ? (void*)h->P64 : (void*)h->P32;
}

simrank_status s_update_launch(simrank_ctx* h, int k0, int k1, int use_masks) {
  std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
  if (h->cfg.profile) {
    if (h->events_used >= 4096) {
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      harvest_events(h);
    }
    ev = next_event_pair(h);
    if (!ev) return fail(h, SR_ERR_CUDA, "cudaEventCreate failed");
    CUDA_TRY(h, cudaEventRecord(ev->first, h->st));
  }
  const bool ws = h->cfg.s_precision == 32 && h->cfg.s_kernel == 0;
  launch_s_update(h->S, h->cfg.s_precision, h->ld, panel_for_s(h), h->K1, h->tiles, h->ntiles,
                  h->mXi, h->mEta, k0, k1, use_masks, h->n_cur, h->counters,
                  s_update_grid(h->cfg.s_precision, h->num_sms, ws), h->st,
                  ws ? wait_limit(h) : 0, upper(h));
  LAUNCH_CHECK(h);
  if (ev) CUDA_TRY(h, cudaEventRecord(ev->second, h->st));
  h->prof_launches += 1;
  h->launches += 1;
  return SR_OK;
}

simrank_status ob_ensure(simrank_ctx* h, int slot, size_t bytes);

// Updates go through the pending-panel buffer: G > 1 pending updates share
// one S pass, or (tc = 1) each update's S pass runs on the tensor cores.
bool deferring(const simrank_ctx* h) {
  return (h->cfg.defer > 1 || h->cfg.tc) && h->cfg.s_precision == 32 && !h->column &&
         h->cfg.s_update == SR_SUPDATE_FUSED && h->cfg.apply != SR_APPLY_ONE_SHOT;
}
// Updates per pending group (1 when tensor cores apply each update at once).
int group(const simrank_ctx* h) { return std::max(1, (int)h->cfg.defer); }

// All tile pairs (I <= J) of nT tiles, in the orders the tensor-core S passes
// take them.  Band order: bands of 8 tile rows; within a band, J ascending
// and, for each J, the band's rows I <= J.  Concurrent CTAs then work on a few
// row bands and a few column tiles, so their operand rows are shared through
// L2 (what counts for wide operands).  Row-major order: concurrent CTAs
// stream adjacent 512-byte segments of the same S rows (what counts when the
// operands are narrow and stay in L2 anyway).
simrank_status ensure_order(simrank_ctx* h, int nT) {
  if (h->order_nT == nT) return SR_OK;
  std::vector<uint32_t> v, vr;
  v.reserve((size_t)nT * (nT + 1) / 2);
  vr.reserve((size_t)nT * (nT + 1) / 2);
  for (int I = 0; I < nT; ++I)
    for (int J = I; J < nT; ++J) vr.push_back(((uint32_t)I << 16) | (uint32_t)J);
  constexpr int BAND = 8;
  std::vector<uint64_t> jb;
  jb.reserve((size_t)nT * (nT + 1) / 4 + nT);
  for (int b0 = 0; b0 < nT; b0 += BAND) {
    for (int J = b0; J < nT; ++J)
      for (int I = b0; I < std::min(b0 + BAND, J + 1); ++I)
        v.push_back(((uint32_t)I << 16) | (uint32_t)J);
    // jobs: column tiles in pairs (J, J + 1), each with the band's row tiles I <= J + 1
    for (int J = b0; J < nT; J += 2) {
      const int J2 = J + 1 < nT ? J + 1 : -1;
      for (int I = b0; I < std::min(b0 + BAND, (J2 >= 0 ? J2 : J) + 1); ++I) {
        const bool p1 = I <= J, p2 = J2 >= 0 && I <= J2;
        const int a = p1 ? J : J2, c = (p1 && p2) ? J2 : 0xffff;
        jb.push_back(((uint64_t)I << 32) | ((uint64_t)a << 16) | (uint64_t)c);
      }
    }
  }
  if (h->d_order) cudaFree(h->d_order);
  h->d_order = nullptr;
  if (h->d_order_row) cudaFree(h->d_order_row);
  h->d_order_row = nullptr;
  if (h->d_jobs) cudaFree(h->d_jobs);
  h->d_jobs = nullptr;
  h->order_nT = -1;
  CUDA_TRY(h, dev_alloc(&h->d_order, v.size()));
  CUDA_TRY(h, cudaMemcpy(h->d_order, v.data(), v.size() * sizeof(uint32_t),
                         cudaMemcpyHostToDevice));
  CUDA_TRY(h, dev_alloc(&h->d_order_row, vr.size()));
  CUDA_TRY(h, cudaMemcpy(h->d_order_row, vr.data(), vr.size() * sizeof(uint32_t),
                         cudaMemcpyHostToDevice));
  CUDA_TRY(h, dev_alloc(&h->d_jobs, jb.size()));
  CUDA_TRY(h, cudaMemcpy(h->d_jobs, jb.data(), jb.size() * sizeof(uint64_t),
                         cudaMemcpyHostToDevice));
  h->order_nT = nT;
  h->order_n = (int)v.size();
  h->jobs_n = (int)jb.size();
  return SR_OK;
}

// The tile order for operand rows of kd_bytes (ensure_order has run).
const uint32_t* tile_order(const simrank_ctx* h, int64_t kd_bytes) {
  return kd_bytes < TC_WIDE_K_BYTES ? h->d_order_row : h->d_order;
}

// Applies the pending updates' panels to S in one pass (rank 2 * np * K1).
simrank_status flush_pending(simrank_ctx* h) {
  if (h->np == 0) return SR_OK;
  const int nT = (h->n_cur + PT - 1) / PT;
  cudaEvent_t* pe = nullptr;
  if (h->cfg.profile) {
    if (h->phase_used >= 2048) {
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      harvest_events(h);
    }
    pe = next_phase_events(h);
    if (!pe) return fail(h, SR_ERR_CUDA, "cudaEventCreate failed");
    for (int q = 0; q < 3; ++q) CUDA_TRY(h, cudaEventRecord(pe[q], h->st));
  }
  const int GK1 = group(h) * h->K1;
  const int nterms = h->np * h->K1;
  simrank_status s;
  if (h->cfg.tc) {
    if ((s = ensure_order(h, nT)) != SR_OK) return s;
  } else {
    CUDA_TRY(h, cudaMemsetAsync(h->ntiles, 0, sizeof(int), h->st));
    launch_tile_list(h->pXi, h->pEta, nT, h->cfg.aff ? 1 : 0, h->tiles, h->ntiles, h->st);
  }
  std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
  if (h->cfg.profile) {
    ev = next_event_pair(h);
    if (!ev) return fail(h, SR_ERR_CUDA, "cudaEventCreate failed");
  }
  if (h->cfg.tc) {
    // tc = 2: FP16 operands, terms rounded up to 64 (B read from A by
    // swapping 128-byte boxes), or to 32 with B stored on its own when that
    // saves a k-block of a narrow pass; tc = 1: TF32, terms rounded up to 32
    const bool f16 = h->cfg.tc == 2;
    int rg = f16 ? (nterms + 63) / 64 * 64 : (nterms + 31) / 32 * 32;
    const int rg32 = (nterms + 31) / 32 * 32;
    const bool own_b = f16 && rg32 != rg && 2 * (int64_t)rg32 * 2 < TC_WIDE_K_BYTES;
    if (own_b) rg = rg32;
    const int64_t kd = 2 * (int64_t)rg;
    const size_t eb = f16 ? 2 : 4;
    if ((s = ob_ensure(h, 12, (size_t)h->n_pad * kd * eb)) != SR_OK) return s;
    if ((s = ob_ensure(h, 13, (size_t)h->n_pad * kd * eb)) != SR_OK) return s;
    if (own_b) {
      if ((s = ob_ensure(h, 24, (size_t)h->n_pad * kd * eb)) != SR_OK) return s;
      if ((s = ob_ensure(h, 25, (size_t)h->n_pad * kd * eb)) != SR_OK) return s;
    }
    void* bhi = own_b ? h->ob[24].p : nullptr;
    void* blo = own_b ? h->ob[25].p : nullptr;
    if (f16) {
      if ((s = ob_ensure(h, 19, 2 * (size_t)nterms * sizeof(unsigned int))) != SR_OK) return s;
      launch_pack_f16_tiles(h->Pp, GK1, nterms, rg, nT * PT, (unsigned int*)h->ob[19].p,
                            h->ob[12].p, h->ob[13].p, bhi, blo, kd, h->st);
      h->launches += 2;
    } else {
      launch_pack_tc_tiles(h->Pp, GK1, nterms, rg, nT * PT, (float*)h->ob[12].p,
                           (float*)h->ob[13].p, kd, h->st);
    }
    if (ev) CUDA_TRY(h, cudaEventRecord(ev->first, h->st));
    const int rc = launch_s_update_tc((float*)h->S, h->ld, h->ob[12].p, h->ob[13].p, h->n_pad,
                                      kd, tile_order(h, kd * (int64_t)eb), h->order_n,
                                      h->d_jobs, h->jobs_n,
                                      h->pXi, h->pEta,
                                      h->cfg.aff ? 1 : 0, h->n_cur, h->counters, h->num_sms,
                                      wait_limit(h), h->st, upper(h), f16 ? 1 : 0, bhi, blo);
    if (rc != 0) return fail(h, SR_ERR_CUDA, "tensor-core S update: launch setup failed");
    h->launches += 2;
  } else {
    if (ev) CUDA_TRY(h, cudaEventRecord(ev->first, h->st));
    const bool ws = h->cfg.s_kernel == 0;
    launch_s_update(h->S, 32, h->ld, h->Pp, GK1, h->tiles, h->ntiles, h->pXi, h->pEta, 0, nterms,
                    0, h->n_cur, h->counters, s_update_grid(32, h->num_sms, ws), h->st,
                    ws ? wait_limit(h) : 0, upper(h));
    h->launches += 1;
  }
  LAUNCH_CHECK(h);
  if (ev) CUDA_TRY(h, cudaEventRecord(ev->second, h->st));
  h->prof_launches += 1;
  h->launches += 1;
  h->stats.tiles_total += (int64_t)nT * (nT + 1) / 2;
  CUDA_TRY(h, cudaMemsetAsync(h->pXi, 0, h->nT_cap * sizeof(uint64_t), h->st));
  CUDA_TRY(h, cudaMemsetAsync(h->pEta, 0, h->nT_cap * sizeof(uint64_t), h->st));
  if (pe) {
    CUDA_TRY(h, cudaEventRecord(pe[3], h->st));
    CUDA_TRY(h, cudaEventRecord(pe[4], h->st));
  }
  h->np = 0;
  return SR_OK;
}

// One rank-one update of the current S for the sink block (srcs at d_srcs +
// src_off, delta of them) into sink j, op = +1/-1, old in-degree d_j; the
// graph patch ops [op_begin, op_end) turn the old graph into the new one.
// chain = 0 runs everything before the S pass in one cooperative launch
// (k_prep.cu, arithmetic in the precision of S); chain = 1, or a graph with
// more tiles than the co-resident CTAs can own, takes the per-step kernels
// (FP64 vectors).
simrank_status run_rank_one(simrank_ctx* h, int64_t src_off, int delta, int j, int op, int d_j,
                            int64_t op_begin, int64_t op_end) {
  const int nT = (h->n_cur + PT - 1) / PT;
  const double C = h->cfg.C;
  cudaEvent_t* pe = nullptr;
  if (h->cfg.profile) {
    if (h->phase_used >= 2048) {
      CUDA_TRY(h, cudaStreamSynchronize(h->st));
      harvest_events(h);
    }
    pe = next_phase_events(h);
    if (!pe) return fail(h, SR_ERR_CUDA, "cudaEventCreate failed");
    CUDA_TRY(h, cudaEventRecord(pe[0], h->st));
  }
  const bool defer = deferring(h);
  if (defer && !h->Pp) {
    const size_t pb = (size_t)h->nT_cap * 2 * group(h) * h->K1 * PT * sizeof(float);
    CUDA_TRY(h, cudaMalloc(&h->Pp, pb));
    CUDA_TRY(h, cudaMemsetAsync(h->Pp, 0, pb, h->st));
    CUDA_TRY(h, dev_alloc(&h->pXi, (size_t)h->nT_cap));
    CUDA_TRY(h, dev_alloc(&h->pEta, (size_t)h->nT_cap));
    CUDA_TRY(h, cudaMemsetAsync(h->pXi, 0, h->nT_cap * sizeof(uint64_t), h->st));
    CUDA_TRY(h, cudaMemsetAsync(h->pEta, 0, h->nT_cap * sizeof(uint64_t), h->st));
  }
  const bool plain = h->cfg.s_update == SR_SUPDATE_PLAIN;
  bool fused = false;
  if (h->cfg.chain == 0) {
    PrepParams pp{};
    pp.in = h->din;
    pp.out = h->dout;
    pp.ops = h->d_ops;
    pp.op_begin = op_begin;
    pp.op_end = op_end;
    pp.S = h->S;
    pp.ld = h->ld;
    pp.I = h->d_srcs + src_off;
    pp.delta = delta;
    pp.j = j;
    pp.op = op;
    pp.d_j = d_j;
    pp.C = C;
    pp.inv_C = 1.0 / C;
    pp.inv_delta = 1.0 / (double)delta;
    pp.gq = (d_j + op * delta) != 0 ? (double)delta / (double)(d_j + op * delta) : 0.0;
    pp.K = h->cfg.K;
    pp.nT = nT;
    if (defer) {
      pp.P = h->Pp;
      pp.ldk = group(h) * h->K1;
      pp.koff = h->np * h->K1;
      pp.npend = h->np * h->K1;
      pp.pXi = h->pXi;
      pp.pEta = h->pEta;
    } else {
      pp.P = panel_for_s(h);
      pp.ldk = h->K1;
      pp.tiles = h->tiles;
      pp.ntiles = h->ntiles;
      pp.tile_mode = (plain || !h->cfg.aff) ? 0 : 1;
    }
    pp.upper = upper(h);
    pp.sI = h->sI;
    pp.sJ = h->sJ;
    pp.mXi = h->mXi;
    pp.mEta = h->mEta;
    pp.cap = h->cfg.prep_cache > 0 ? h->cfg.prep_cache : 8192;
    pp.item = h->cfg.prep_item;
    pp.n_pad = h->n_pad;
    pp.nT_cap = h->nT_cap;
    if (!h->W) {
      CUDA_TRY(h, cudaMalloc(&h->W, (size_t)h->K1 * h->n_pad * 2 * sizeof(double)));
      CUDA_TRY(h, cudaMalloc(&h->rinv, (size_t)h->n_pad * 2 * sizeof(double)));
      CUDA_TRY(h, dev_alloc(&h->loff, (size_t)h->n_pad));
      CUDA_TRY(h, dev_alloc(&h->tile_nnz, (size_t)h->nT_cap));
    }
    pp.W = h->W;
    pp.rinv = h->rinv;
    pp.loff = h->loff;
    pp.flat = h->cfg.prep_item == 0 ? 1 : 0;
    pp.tile_nnz = h->tile_nnz;
    pp.bar = h->gbar + 2;
    pp.limit = wait_limit(h);
    pp.counters = (unsigned long long*)h->counters;
    const int rc = launch_prep(pp, h->cfg.s_precision, h->cfg.vec_fp64 ? 1 : 0,
                               defer ? group(h) * h->K1 : 0,
                               h->num_sms, h->cfg.prep_ctas, (int64_t)h->edges.size() + delta,
                               h->st);
    if (rc == 1) return fail(h, SR_ERR_CUDA, "fused pre-update launch failed");
    fused = (rc == 0);
    if (fused) {
      LAUNCH_CHECK(h);
      h->launches += 1;
      if (pe) {
        CUDA_TRY(h, cudaEventRecord(pe[1], h->st));
        CUDA_TRY(h, cudaEventRecord(pe[2], h->st));
        CUDA_TRY(h, cudaEventRecord(pe[3], h->st));
      }
    }
  }
  if (!fused) {
    if (defer) {
      // rows i (summed over the block) and j of the current S = S + pending panels
      launch_gather_rows_pending(h->S, 32, h->ld, h->d_srcs + src_off, delta, j, nT * PT, h->Pp,
                                 group(h) * h->K1, h->np * h->K1, h->sI, h->sJ, h->st,
                                 upper(h));
      launch_scalars_from_rows(h->din, h->sI, h->sJ, h->d_srcs + src_off, delta, j, h->scal, h->st);
      h->launches += 1;
    } else {
      launch_gather_rows(h->S, h->cfg.s_precision, h->ld, h->d_srcs + src_off, delta, j, nT * PT,
                         h->din, h->sI, h->sJ, h->scal, h->st, upper(h));
    }
    launch_gamma(h->din, h->sI, h->sJ, h->scal, j, delta, op, d_j, C, nT, h->K1, h->P64,
                 h->cfg.s_precision == 64 ? nullptr : h->P32, h->mXi, h->mEta, h->st);
    if (pe) CUDA_TRY(h, cudaEventRecord(pe[1], h->st));
    launch_patch(h->d_ops, op_begin, op_end, h->din, h->dout, h->st);
    float* p32 = h->cfg.s_precision == 64 ? nullptr : h->P32;
    for (int k = 0; k < h->cfg.K; ++k)
      launch_chain_step(h->din, k, C, nT, h->K1, h->P64, p32, h->mXi, h->mEta, h->st);
    h->launches += 2 + (op_end > op_begin ? 1 : 0) + h->cfg.K;
    LAUNCH_CHECK(h);
    if (pe) CUDA_TRY(h, cudaEventRecord(pe[2], h->st));
    if (defer) {
      // append this update's panels as pending terms np*K1 .. np*K1 + K (FP32)
      const size_t w = (size_t)h->K1 * PT * sizeof(float);
      const size_t dpitch = (size_t)group(h) * w;
      CUDA_TRY(h, cudaMemcpy2DAsync((unsigned char*)h->Pp + (size_t)h->np * w, dpitch, h->P32, w,
                                    w, (size_t)nT * 2, cudaMemcpyDeviceToDevice, h->st));
      launch_or_any(h->mXi, h->mEta, nT, h->pXi, h->pEta, h->st);
      h->launches += 1;
    } else {
      CUDA_TRY(h, cudaMemsetAsync(h->ntiles, 0, sizeof(int), h->st));
      launch_tile_list(h->mXi, h->mEta, nT, (plain || !h->cfg.aff) ? 0 : 1, h->tiles, h->ntiles,
                       h->st);
      LAUNCH_CHECK(h);
      h->launches += 1;
    }
    if (pe) CUDA_TRY(h, cudaEventRecord(pe[3], h->st));
  }
  if (defer) {
    h->np += 1;
    if (pe) CUDA_TRY(h, cudaEventRecord(pe[4], h->st));
    h->stats.rank_one_updates += 1;
    if (h->np == group(h)) return flush_pending(h);
    return SR_OK;
  }
  simrank_status s;
  if (plain) {
    for (int k = 0; k < h->K1; ++k)
      if ((s = s_update_launch(h, k, k + 1, 0)) != SR_OK) return s;
  } else {
    if ((s = s_update_launch(h, 0, h->K1, h->cfg.aff ? 1 : 0)) != SR_OK) return s;
  }
  if (pe) CUDA_TRY(h, cudaEventRecord(pe[4], h->st));
  h->stats.rank_one_updates += 1;
  h->stats.tiles_total += (int64_t)nT * (nT + 1) / 2;
  return SR_OK;
}

// Jacobi sweeps of Eq. 1 starting from the current S, in FP64 work buffers
// when three of them fit in `fp64_budget` bytes (or S itself is FP64), else
// in FP32 storage with FP64 accumulation.  Stops when a sweep changes S by
// less than `tol` (max-abs) or after max_sweeps; S is symmetrised at the end.
simrank_status jacobi_sweeps(simrank_ctx* h, int max_sweeps, double tol, double* last_diff,
                             int* sweeps_done, double* tol_used = nullptr,
                             double* first_diff = nullptr) {
  const int sp = h->cfg.s_precision;
  const size_t elems = (size_t)h->n_pad * h->ld;
  const size_t fp64_budget = (size_t)48 << 30;
  const int wp = (sp == 64 || 3 * elems * 8 <= fp64_budget) ? 64 : 32;
  const size_t bytes = elems * (wp == 64 ? 8 : 4);
  // sweeps stored in FP32 cannot change S by much less than its rounding
  // (about 6e-8 relative): their stopping test is floored at 1e-7, and below
  // 3e-7 they also stop once three sweeps in a row changed S no less than the
  // sweep before (the change has reached the rounding noise)
  if (wp == 32) tol = std::max(tol, 1e-7);
  int flat_sweeps = 0;
  double prev = INFINITY;
  void* bufs[3] = {nullptr, nullptr, nullptr};
  const bool alias = (wp == sp);
  for (int b = (alias ? 1 : 0); b < 3; ++b) {
    if (cudaMalloc(&bufs[b], bytes) != cudaSuccess) {
      for (void* p : bufs)
        if (p) cudaFree(p);
      return fail(h, SR_ERR_OOM, "cudaMalloc of Jacobi buffers failed");
    }
  }
  if (alias)
    bufs[0] = h->S;
  else
    launch_convert(h->S, sp, bufs[0], wp, (int64_t)elems, h->st);
  cudaMemsetAsync(bufs[1], 0, bytes, h->st);
  cudaMemsetAsync(bufs[2], 0, bytes, h->st);
  void *A = bufs[0], *B = bufs[1], *T = bufs[2];
  double diff = INFINITY;
  int it = 0;
  cudaError_t e = cudaGetLastError();
  const float* w = h->weighted ? h->d_in_w : nullptr;
  while (e == cudaSuccess && it < max_sweeps) {
    launch_spmm_rows(h->din, w, h->d_wsum, A, wp, h->ld, B, wp, h->ld, h->n_pad, h->n_pad, 1.0,
                     0.0, 0, h->st);
    launch_transpose(B, T, wp, h->n_pad, h->ld, h->st);
    launch_spmm_rows(h->din, w, h->d_wsum, T, wp, h->ld, B, wp, h->ld, h->n_pad, h->n_pad,
                     h->cfg.C, 1.0 - h->cfg.C, h->n_cap, h->st);
    cudaMemsetAsync(h->diffbits, 0, sizeof(unsigned long long), h->st);
    launch_maxdiff(A, B, wp, h->n_pad, h->ld, h->diffbits, h->st);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    std::swap(A, B);
    ++it;
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, h->diffbits, sizeof(bits), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) break;
    std::memcpy(&diff, &bits, sizeof(diff));
    if (it == 1 && first_diff) *first_diff = diff;
    if (diff < tol) break;
    if (wp == 32) {
      flat_sweeps = diff >= prev ? flat_sweeps + 1 : 0;
      prev = diff;
      if (diff < 3e-7 && flat_sweeps >= 3) {
        tol = diff * 1.0000001;  // converged to the rounding noise of FP32 storage
        break;
      }
    }
  }
  if (e == cudaSuccess) {
    launch_symmetrize(A, wp, h->n_pad, h->ld, h->st);
    if (!alias) launch_convert(A, wp, h->S, sp, (int64_t)elems, h->st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  // bufs[] holds three distinct buffers (bufs[0] is the old S when aliasing);
  // keep the result as S when aliasing and free every other buffer once.
  if (alias && e == cudaSuccess) h->S = A;
  for (int b = 0; b < 3; ++b)
    if (bufs[b] && bufs[b] != h->S) cudaFree(bufs[b]);
  if (e != cudaSuccess)
    return fail(h, SR_ERR_CUDA, std::string("Jacobi sweep: ") + cudaGetErrorString(e));
  *last_diff = diff;
  *sweeps_done = it;
  if (tol_used) *tol_used = tol;
  return SR_OK;
}

// Drift correction: Jacobi sweeps of Eq. 1 started from the current S (its
// lower tiles restored from their mirrors first when only the upper ones are
// kept), until a sweep changes S by less than tol or after `sweeps` sweeps.
// The first sweep's change is the residual max |C Q S Q^T + (1-C) I - S| of
// the S it started from.
simrank_status reanchor_run(simrank_ctx* h, int sweeps, double tol, double* first, double* last,
                            int* done) {
  if (upper(h)) {
    launch_mirror_lower(h->S, h->cfg.s_precision, h->n_pad, h->ld, h->st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, SR_ERR_CUDA, cudaGetErrorString(e));
  }
  return jacobi_sweeps(h, sweeps, tol, last, done, nullptr, first);
}

// Counts accepted rank-one work towards the automatic re-anchor
// (cfg.reanchor_every) and runs it when due; pending panels are applied first.
simrank_status maybe_reanchor(simrank_ctx* h, int64_t updates) {
  if (h->column || h->cfg.reanchor_every <= 0) return SR_OK;
  h->since_anchor += updates;
  if (h->since_anchor < h->cfg.reanchor_every) return SR_OK;
  h->since_anchor = 0;
  simrank_status s = flush_pending(h);
  if (s != SR_OK) return s;
  double first = 0.0, last = 0.0;
  int done = 0;
  if ((s = reanchor_run(h, h->cfg.reanchor_sweeps, h->cfg.init_tol, &first, &last, &done)) != SR_OK)
    return s;
  h->stats.reanchors += 1;
  h->stats.reanchor_residual = first;
  h->stats.reanchor_change = last;
  return SR_OK;
}

simrank_status ob_ensure(simrank_ctx* h, int slot, size_t bytes) {
  auto& b = h->ob[slot];
  if (b.bytes >= bytes) return SR_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  CUDA_TRY(h, cudaMalloc(&b.p, std::max<size_t>(bytes, 256)));
  b.bytes = bytes;
  return SR_OK;
}

void build_chunks(const HostAdj& A, int n_rows, std::vector<RowChunk>& out,
                  std::vector<int64_t>* first);

// The whole batch as one rank-2r update (proof of Thm 2 with dQ = U V^T over
// the r distinct sinks).  `plus` / `minus` hold the net insertions and
// deletions per sink (storage ids); `ops` turn the old graph into the new one.
simrank_status run_one_shot(simrank_ctx* h, const std::map<int32_t, std::vector<int32_t>>& plus,
                            const std::map<int32_t, std::vector<int32_t>>& minus,
                            const std::vector<PatchOp>& ops) {
  std::map<int32_t, std::pair<std::vector<int32_t>, std::vector<int32_t>>> sinks;
  for (auto& kv : plus) sinks[kv.first].first = kv.second;
  for (auto& kv : minus) sinks[kv.first].second = kv.second;
  const int r = (int)sinks.size();
  if (r == 0) return SR_OK;
  const double C = h->cfg.C;
  const int sp = h->cfg.s_precision;
  std::vector<int32_t> sink_id, src;
  std::vector<int8_t> sign;
  std::vector<int64_t> off{0};
  std::vector<double> av, bv;
  for (auto& kv : sinks) {
    const int32_t j = kv.first;
    const auto& ins = kv.second.first;
    const auto& del = kv.second.second;
    // old in-degree: the mirror already holds the new graph, undo the net change
    const int d_new = h->hin.len[j];
    const int d_old = d_new - (int)ins.size() + (int)del.size();
    double a, b;
    if (d_old == 0) {
      a = 0.0;
      b = 1.0 / d_new;
    } else if (d_new == 0) {
      a = -1.0;
      b = 0.0;
    } else {
      a = (double)d_old / d_new - 1.0;
      b = 1.0 / d_new;
    }
    sink_id.push_back(j);
    av.push_back(a);
    bv.push_back(b);
    for (int32_t x : ins) {
      src.push_back(x);
      sign.push_back(1);
    }
    if (d_new > 0)
      for (int32_t x : del) {
        src.push_back(x);
        sign.push_back(-1);
      }
    off.push_back((int64_t)src.size());
  }
  const int n_pad = h->n_pad;
  const int rp = (r + 3) / 4 * 4;
  const int64_t nr = (int64_t)n_pad * rp;
  simrank_status s;
  // 0: small host->device arrays, 1: Zc / Yc, 2: Z, 3: Y, 4: Wc, 5: Lambda, 6/7: X ping-pong
  const size_t small = (size_t)r * (4 + 8 + 8 + 8) + src.size() * 5 + 1024;
  if ((s = ob_ensure(h, 0, small)) != SR_OK) return s;
  if ((s = ob_ensure(h, 1, (size_t)nr * 8)) != SR_OK) return s;
  if ((s = ob_ensure(h, 2, (size_t)nr * 8)) != SR_OK) return s;
  if ((s = ob_ensure(h, 3, (size_t)nr * 8)) != SR_OK) return s;
  if ((s = ob_ensure(h, 4, (size_t)nr * 8)) != SR_OK) return s;
  if ((s = ob_ensure(h, 5, (size_t)r * r * 8)) != SR_OK) return s;
  if ((s = ob_ensure(h, 6, (size_t)nr * 2 * 8)) != SR_OK) return s;
  if ((s = ob_ensure(h, 7, (size_t)nr * 2 * 8)) != SR_OK) return s;
  unsigned char* sm = (unsigned char*)h->ob[0].p;
  int32_t* d_sinks = (int32_t*)sm;
  double* d_av = (double*)(sm + (((size_t)r * 4 + 7) / 8) * 8);
  double* d_bv = d_av + r;
  int64_t* d_off = (int64_t*)(d_bv + r);
  int32_t* d_src = (int32_t*)(d_off + r + 1);
  int8_t* d_sign = (int8_t*)(d_src + src.size());
  CUDA_TRY(h, cudaMemcpyAsync(d_sinks, sink_id.data(), r * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d_av, av.data(), r * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d_bv, bv.data(), r * 8, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d_off, off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, h->st));
  if (!src.empty()) {
    CUDA_TRY(h, cudaMemcpyAsync(d_src, src.data(), src.size() * 4, cudaMemcpyHostToDevice, h->st));
    CUDA_TRY(h, cudaMemcpyAsync(d_sign, sign.data(), src.size(), cudaMemcpyHostToDevice, h->st));
  }
  double* Zc = (double*)h->ob[1].p;
  double* Z = (double*)h->ob[2].p;
  double* Y = (double*)h->ob[3].p;
  double* Wc = (double*)h->ob[4].p;
  double* Lam = (double*)h->ob[5].p;
  double* X = (double*)h->ob[6].p;
  double* Xn = (double*)h->ob[7].p;
  CUDA_TRY(h, cudaMemsetAsync(Z, 0, (size_t)nr * 8, h->st));
  CUDA_TRY(h, cudaMemsetAsync(Y, 0, (size_t)nr * 8, h->st));
  // Z = sum of signed source rows, Y = Q Z on the OLD graph
  launch_signed_rows(h->S, sp, h->ld, d_src, d_sign, d_off, r, n_pad, Zc, h->st, upper(h));
  launch_transpose_rect(Zc, n_pad, Z, rp, r, n_pad, h->st);
  launch_spmm_rows(h->din, nullptr, nullptr, Z, 64, rp, Y, 64, rp, n_pad, rp, 1.0, 0.0, 0, h->st);
  launch_transpose_rect(Y, rp, Zc, n_pad, n_pad, r, h->st);  // Yc into buffer 1
  launch_lambda(h->S, sp, h->ld, d_sinks, d_av, d_bv, Y, Z, rp, d_src, d_sign, d_off, r, C, Lam,
                h->st, upper(h));
  launch_w_assemble(h->S, sp, h->ld, d_sinks, d_av, d_bv, Zc, Lam, r, n_pad, C, Wc, h->st,
                    upper(h));
  LAUNCH_CHECK(h);
  h->launches += 7;
  // the graph becomes the new one
  CUDA_TRY(h, cudaMemcpyAsync(h->d_ops, ops.data(), ops.size() * sizeof(PatchOp),
                              cudaMemcpyHostToDevice, h->st));
  launch_patch(h->d_ops, 0, (int64_t)ops.size(), h->din, h->dout, h->st);
  // X_0 = [C U | W] (row-major, 2 rp columns)
  const int64_t ldx = 2 * rp;
  CUDA_TRY(h, cudaMemsetAsync(X, 0, (size_t)nr * 2 * 8, h->st));
  CUDA_TRY(h, cudaMemsetAsync(Xn, 0, (size_t)nr * 2 * 8, h->st));
  launch_xi0(d_sinks, r, C, X, ldx, h->st);
  launch_transpose_rect(Wc, n_pad, X + rp, ldx, r, n_pad, h->st);
  LAUNCH_CHECK(h);
  h->launches += 3;
  // the steps below gather by row chunks of the new graph (the host mirror
  // holds it), so that a hub row spreads over many warps
  std::vector<RowChunk> chv;
  build_chunks(h->hin, n_pad, chv, nullptr);
  if ((s = ob_ensure(h, 26, std::max<size_t>(1, chv.size()) * sizeof(RowChunk))) != SR_OK) return s;
  const RowChunk* d_chunks = (const RowChunk*)h->ob[26].p;
  if (!chv.empty())
    CUDA_TRY(h, cudaMemcpyAsync(h->ob[26].p, chv.data(), chv.size() * sizeof(RowChunk),
                                cudaMemcpyHostToDevice, h->st));

  // k-groups: as many terms per S pass as fit an operand budget
  // tc = 2: FP16 split, terms balanced by powers of two (rg a multiple of 64);
  // tc = 1: TF32 split (rg a multiple of 32)
  const bool tc = h->cfg.tc != 0 && sp == 32;
  const bool f16 = tc && h->cfg.tc == 2;
  const int ra = f16 ? 64 : 32;
  const size_t eb = f16 ? 2 : 4;
  const int nT = (h->n_cur + PT - 1) / PT;
  const size_t budget = (size_t)8 << 30;
  const size_t per_k = tc ? (size_t)n_pad * 2 * (size_t)((r + ra - 1) / ra * ra) * eb * 2
                          : (size_t)n_pad * 2 * (size_t)r * (sp == 64 ? 8 : 4);
  const int g = (int)std::max<size_t>(1, std::min<size_t>((size_t)h->K1, budget / per_k));
  const int rg = tc ? ((g * r + ra - 1) / ra) * ra : g * r;
  const int64_t kd = 2 * (int64_t)rg;
  if (tc) {
    if ((s = ob_ensure(h, 8, (size_t)n_pad * kd * eb)) != SR_OK) return s;
    if ((s = ob_ensure(h, 9, (size_t)n_pad * kd * eb)) != SR_OK) return s;
    if (f16 && (s = ob_ensure(h, 27, 2 * (size_t)r * sizeof(unsigned int))) != SR_OK) return s;
  } else {
    if ((s = ob_ensure(h, 8, (size_t)h->nT_cap * 2 * (size_t)(g * r) * PT * (sp == 64 ? 8 : 4))) !=
        SR_OK)
      return s;
  }
  const long long wait_limit = ::wait_limit(h);
  int slot = 0;
  for (int k = 0; k <= h->cfg.K; ++k) {
    if (k > 0) {
      CUDA_TRY(h, cudaMemsetAsync(Xn, 0, (size_t)nr * 2 * 8, h->st));
      if (launch_spmm_chunks64(d_chunks, (int64_t)chv.size(), h->din.col, h->din.len, X, ldx, Xn,
                               ldx, rp, C, h->st) != 0 ||
          launch_spmm_chunks64(d_chunks, (int64_t)chv.size(), h->din.col, h->din.len, X + rp,
                               ldx, Xn + rp, ldx, rp, 1.0, h->st) != 0)
        return fail(h, SR_ERR_CUDA, "chunked SpMM: bad shape");
      std::swap(X, Xn);
      h->launches += 2;
    }
    if (slot == 0) {
      if (tc) {
        CUDA_TRY(h, cudaMemsetAsync(h->ob[8].p, 0, (size_t)n_pad * kd * eb, h->st));
        CUDA_TRY(h, cudaMemsetAsync(h->ob[9].p, 0, (size_t)n_pad * kd * eb, h->st));
      } else {
        CUDA_TRY(h, cudaMemsetAsync(h->mXi, 0, h->nT_cap * sizeof(uint64_t), h->st));
        CUDA_TRY(h, cudaMemsetAsync(h->mEta, 0, h->nT_cap * sizeof(uint64_t), h->st));
      }
    }
    if (f16)
      launch_pack_f16_oneshot(X, ldx, rp, r, slot, rg, n_pad, (unsigned int*)h->ob[27].p,
                              h->ob[8].p, h->ob[9].p, kd, h->st);
    else if (tc)
      launch_pack_tc(X, ldx, rp, r, slot, rg, n_pad, (float*)h->ob[8].p, (float*)h->ob[9].p, kd,
                     h->st);
    else
      launch_pack_ffma(X, ldx, rp, r, slot, g * r, nT, h->ob[8].p, sp, h->mXi, h->mEta, h->st);
    LAUNCH_CHECK(h);
    h->launches += 1;
    ++slot;
    if (slot == g || k == h->cfg.K) {
      if (tc) {
        if ((s = ensure_order(h, nT)) != SR_OK) return s;
      } else {
        CUDA_TRY(h, cudaMemsetAsync(h->ntiles, 0, sizeof(int), h->st));
        launch_tile_list(h->mXi, h->mEta, nT, h->cfg.aff ? 1 : 0, h->tiles, h->ntiles, h->st);
        h->launches += 1;
      }
      std::pair<cudaEvent_t, cudaEvent_t>* ev = nullptr;
      if (h->cfg.profile) {
        ev = next_event_pair(h);
        if (!ev) return fail(h, SR_ERR_CUDA, "cudaEventCreate failed");
        CUDA_TRY(h, cudaEventRecord(ev->first, h->st));
      }
      if (tc) {
        const int rc = launch_s_update_tc((float*)h->S, h->ld, h->ob[8].p, h->ob[9].p, n_pad,
                                          kd, tile_order(h, kd * (int64_t)eb), h->order_n,
                                          nullptr, 0, h->mXi, h->mEta, 0, h->n_cur, h->counters,
                                          h->num_sms, wait_limit, h->st, upper(h), f16 ? 1 : 0);
        if (rc != 0) return fail(h, SR_ERR_CUDA, "tensor-core S update: launch setup failed");
      } else {
        const bool ws = sp == 32 && h->cfg.s_kernel == 0;
        launch_s_update(h->S, sp, h->ld, h->ob[8].p, g * r, h->tiles, h->ntiles, h->mXi, h->mEta,
                        0, slot * r, h->cfg.aff ? 1 : 0, h->n_cur, h->counters,
                        s_update_grid(sp, h->num_sms, ws), h->st, ws ? wait_limit : 0,
                        upper(h));
      }
      LAUNCH_CHECK(h);
      if (ev) CUDA_TRY(h, cudaEventRecord(ev->second, h->st));
      h->launches += 1;
      h->prof_launches += 1;
      h->stats.tiles_total += (int64_t)nT * (nT + 1) / 2;
      slot = 0;
    }
  }
  h->stats.rank_one_updates += 0;
  // keep host staging alive until the copies above have run
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  return SR_OK;
}

// Row chunks (at most kChunk nonzeros each) of the adjacency rows [0, n_rows);
// first (optional) gets the index of each row's first chunk (n_rows + 1).
void build_chunks(const HostAdj& A, int n_rows, std::vector<RowChunk>& out,
                  std::vector<int64_t>* first = nullptr) {
  out.clear();
  int64_t total = 0;
  for (int a = 0; a < n_rows; ++a) total += (A.len[a] + kChunk - 1) / kChunk;
  out.reserve((size_t)total);
  if (first) first->assign((size_t)n_rows + 1, 0);
  for (int a = 0; a < n_rows; ++a) {
    if (first) (*first)[a] = (int64_t)out.size();
    for (int off = 0; off < A.len[a]; off += kChunk)
      out.push_back({a, std::min(kChunk, A.len[a] - off), A.start[a] + off});
  }
  if (first) (*first)[n_rows] = (int64_t)out.size();
}

// Rewrites row a's chunks of a list built by build_chunks (with first) after
// a change of that row, on the host and on the device; false if the row's
// number of chunks changed (the list must be rebuilt).
bool patch_row_chunks(simrank_ctx* h, const HostAdj& A, int a, std::vector<RowChunk>& v,
                      const std::vector<int64_t>& first, ChunkList& L) {
  const int64_t c0 = first[a], nc = first[a + 1] - c0;
  if ((A.len[a] + kChunk - 1) / kChunk != nc) return false;
  for (int64_t c = 0; c < nc; ++c)
    v[c0 + c] = {a, std::min(kChunk, A.len[a] - (int)(c * kChunk)), A.start[a] + c * kChunk};
  if (nc > 0 && cudaMemcpyAsync(L.chunks + c0, v.data() + c0, nc * sizeof(RowChunk),
                                cudaMemcpyHostToDevice, h->st) != cudaSuccess)
    return false;
  return true;
}

simrank_status upload_chunks(simrank_ctx* h, const std::vector<RowChunk>& v, ChunkList& L,
                             int64_t* cap) {
  if ((int64_t)v.size() > *cap) {
    if (L.chunks) cudaFree(L.chunks);
    L.chunks = nullptr;
    *cap = std::max<int64_t>((int64_t)v.size(), 2 * *cap);
    CUDA_TRY(h, dev_alloc(&L.chunks, (size_t)*cap));
  }
  L.count = (int64_t)v.size();
  if (!v.empty())
    CUDA_TRY(h, cudaMemcpyAsync(L.chunks, v.data(), v.size() * sizeof(RowChunk),
                                cudaMemcpyHostToDevice, h->st));
  return SR_OK;
}

// One update in column mode (Alg 7 with new nodes as isolated nodes): the
// old columns S_{*,i}, S_{*,j} by Procedure 1 on the current graph, gamma,
// the graph patch, the xi/eta recurrence, and a snapshot of the panels.
// One stored update of column mode (Alg 7): a unit update or, with
// SR_APPLY_SINK_BLOCKS, a sink block of delta sources into j (Table 2, the
// batch scheme of §8 that the closing remark of §7 combines with Alg 7).  The
// old columns S_{*,i} (i in I) and S_{*,j} come from Procedure 1 on the
// current graph; Table 2 needs only the sum of the sources' columns and S_II,
// and Procedure 1 started from the indicator of the sources gives that sum as
// one column, so memory stays O(Kn + m) for any delta.  d_cols holds the
// delta sources then j (device).
simrank_status run_column_update(simrank_ctx* h, const std::vector<int32_t>& srcs, int j, int op,
                                 int d_j, int64_t op_begin, int64_t op_end, int32_t* d_cols) {
  const int K = h->cfg.K, n_pad = h->n_pad, nT = (h->n_cur + PT - 1) / PT;
  const int delta = (int)srcs.size();
  simrank_status s;
  std::vector<int32_t> cols(srcs);
  cols.push_back(j);
  CUDA_TRY(h, cudaMemcpyAsync(d_cols, cols.data(), cols.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, h->st));
  // one Procedure-1 block of two columns: column 0 starts from the
  // indicator of the sources (Procedure 1 is linear, so it yields
  // sum_i S_{*,i} directly), column 1 from e_j
  const size_t blk = (size_t)n_pad * 2 * sizeof(double);
  if ((s = ob_ensure(h, 10, blk * (K + 1))) != SR_OK) return s;
  if ((s = ob_ensure(h, 11, blk * 3)) != SR_OK) return s;
  unsigned char* w = (unsigned char*)h->ob[11].p;
  launch_partial_sim_block(h->cur_fwd, h->cur_hor, h->dout.col, h->din.col, h->din.len, d_cols, 2,
                           n_pad, K, h->cfg.C, 64, h->ob[10].p, w, w + blk, w + 2 * blk, h->st,
                           WeightView(), delta);
  launch_col_extract(w + 2 * blk, 64, 2, 0, n_pad, h->sI, h->st);
  launch_col_extract(w + 2 * blk, 64, 2, 1, n_pad, h->sJ, h->st);
  h->launches += 2 * K + 5;
  // S_II and w_j = (1/delta) (Q S_{*,I})_j on the graph before the update
  launch_scalars_from_rows(h->din, h->sI, h->sJ, d_cols, delta, j, h->scal, h->st);
  const bool f32 = h->cfg.s_precision == 32;
  launch_gamma(h->din, h->sI, h->sJ, h->scal, j, delta, op, d_j, h->cfg.C, nT, h->K1, h->P64,
               f32 ? h->P32 : nullptr, h->mXi, h->mEta, h->st);
  launch_patch(h->d_ops, op_begin, op_end, h->din, h->dout, h->st);
  // the K steps on the new graph, tiles cut into work items of at most
  // chain_item_size() nonzeros (the host mirror already holds the new graph)
  if (h->col_tnnz.empty()) {
    h->col_tnnz.assign(h->nT_cap, 0);
    for (int a = 0; a < h->n_pad; ++a) h->col_tnnz[a / PT] += h->hin.len[a];
  } else {
    int64_t s_j = 0;
    for (int a = (j / PT) * PT; a < (j / PT + 1) * PT; ++a) s_j += h->hin.len[a];
    h->col_tnnz[j / PT] = s_j;
  }
  const int64_t item = chain_item_size();
  std::vector<int32_t> it_tile, it_sub, t_items(nT);
  for (int T = 0; T < nT; ++T) {
    const int parts = (int)std::max<int64_t>(1, (h->col_tnnz[T] + item - 1) / item);
    t_items[T] = parts;
    for (int q = 0; q < parts; ++q) {
      it_tile.push_back(T);
      it_sub.push_back(q);
    }
  }
  const int64_t n_items = (int64_t)it_tile.size();
  const int64_t need = 2 * n_items + h->nT_cap;
  if (need > h->col_items_cap) {
    if (h->col_items) cudaFree(h->col_items);
    h->col_items = nullptr;
    CUDA_TRY(h, dev_alloc(&h->col_items, (size_t)need));
    h->col_items_cap = need;
  }
  if (!h->col_gacc) {
    CUDA_TRY(h, dev_alloc(&h->col_gacc, (size_t)h->nT_cap * 2 * PT));
    CUDA_TRY(h, dev_alloc(&h->col_tcount, (size_t)h->nT_cap));
    CUDA_TRY(h, cudaMemsetAsync(h->col_gacc, 0, (size_t)h->nT_cap * 2 * PT * sizeof(double), h->st));
    CUDA_TRY(h, cudaMemsetAsync(h->col_tcount, 0, (size_t)h->nT_cap * sizeof(unsigned int), h->st));
  }
  int32_t* d_tile = h->col_items;
  int32_t* d_sub = d_tile + n_items;
  int32_t* d_titems = d_sub + n_items;
  CUDA_TRY(h, cudaMemcpyAsync(d_tile, it_tile.data(), n_items * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d_sub, it_sub.data(), n_items * 4, cudaMemcpyHostToDevice, h->st));
  CUDA_TRY(h, cudaMemcpyAsync(d_titems, t_items.data(), nT * 4, cudaMemcpyHostToDevice, h->st));
  for (int k = 0; k < K; ++k)
    launch_chain_step_items(h->din, d_tile, d_sub, d_titems, (int)n_items, k, h->cfg.C, h->K1,
                            h->P64, f32 ? h->P32 : nullptr, h->mXi, h->mEta, h->col_gacc,
                            h->col_tcount, h->st);
  LAUNCH_CHECK(h);
  h->launches += 3 + K;
  const size_t pbytes = (size_t)h->nT_cap * 2 * h->K1 * PT * (f32 ? 4 : 8);
  void* snap = nullptr;
  CUDA_TRY(h, cudaMallocAsync(&snap, pbytes, h->st));
  h->hist.push_back(snap);
  CUDA_TRY(h, cudaMemcpyAsync(snap, f32 ? (void*)h->P32 : (void*)h->P64, pbytes,
                              cudaMemcpyDeviceToDevice, h->st));
  // the chunk lists of this update must not change before its kernels ran
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  h->stats.rank_one_updates += 1;
  return SR_OK;
}

// Columns in column mode: Procedure 1 on the initial graph plus, for every
// stored update, Eq. 70-71's column of M_K + M_K^T.
simrank_status column_mode_columns(simrank_ctx* h, const int32_t* cols, int ncols, void* out,
                                   int out_on_device, int out_fp64) {
  const int prec = h->cfg.s_precision, K = h->cfg.K, n_pad = h->n_pad;
  const size_t eb = prec == 64 ? 8 : 4;
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(h, cudaMemGetInfo(&free_b, &total_b));
  const size_t per_col = (size_t)n_pad * eb * (K + 4);
  int Bmax = (int)std::min<size_t>(1024, std::max<size_t>(1, (size_t)(0.6 * free_b) / per_col));
  simrank_status s;
  if ((s = ob_ensure(h, 10, per_col * Bmax)) != SR_OK) return s;
  if (ncols > h->cols_cap) {
    if (h->d_cols) cudaFree(h->d_cols);
    h->d_cols = nullptr;
    h->cols_cap = ncols;
    CUDA_TRY(h, dev_alloc(&h->d_cols, (size_t)ncols));
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_cols, cols, ncols * sizeof(int32_t), cudaMemcpyHostToDevice,
                              h->st));
  const size_t ob = (size_t)h->n_cur * ncols * (out_fp64 ? 8 : 4);
  void* dst = out;
  void* tmp = nullptr;
  if (!out_on_device) {
    CUDA_TRY(h, cudaMalloc(&tmp, ob));
    dst = tmp;
  }
  for (int c0 = 0; c0 < ncols; c0 += Bmax) {
    const int B = std::min(Bmax, ncols - c0);
    const int32_t* bc = h->d_cols + c0;
    unsigned char* base = (unsigned char*)h->ob[10].p;
    const size_t blkb = (size_t)n_pad * B * eb;
    void* xs = base;
    void* y0 = base + blkb * (K + 1);
    void* y1 = base + blkb * (K + 2);
    void* res = base + blkb * (K + 3);
    launch_partial_sim_block(h->g0_fwd, h->g0_hor, h->g0_out_col, h->g0_in_col, h->g0_in_len, bc,
                             B, n_pad, K, h->cfg.C, prec, xs, y0, y1, res, h->st);
    if (prec == 32 && !h->hist.empty()) {
      // all stored updates in one FP32 product
      const int U = (int)h->hist.size();
      const size_t gbytes = (size_t)U * 2 * h->K1 * ((B + 3) / 4 * 4) * sizeof(float);
      if ((s = ob_ensure(h, 17, U * sizeof(void*))) != SR_OK) return s;
      if ((s = ob_ensure(h, 18, gbytes)) != SR_OK) return s;
      CUDA_TRY(h, cudaMemcpyAsync(h->ob[17].p, h->hist.data(), U * sizeof(void*),
                                  cudaMemcpyHostToDevice, h->st));
      launch_col_corr((const float* const*)h->ob[17].p, U, h->K1, bc, B, n_pad,
                      (float*)h->ob[18].p, (float*)res, h->st);
    } else {
      for (void* P : h->hist) launch_col_apply(P, prec, h->K1, bc, B, n_pad, prec, res, h->st);
    }
    launch_col_out(res, prec, B, h->n_cur,
                   (unsigned char*)dst + (size_t)c0 * h->n_cur * (out_fp64 ? 8 : 4), out_fp64, h->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      if (tmp) cudaFree(tmp);
      return fail(h, SR_ERR_CUDA, std::string("column mode: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaSuccess;
  if (!out_on_device) e = cudaMemcpyAsync(out, tmp, ob, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return fail(h, SR_ERR_CUDA, std::string("column mode: ") + cudaGetErrorString(e));
  return SR_OK;
}

void free_ctx(simrank_ctx* h) {
  if (!h) return;
  if (h->d_out_w) cudaFree(h->d_out_w);
  void* ptrs[] = {h->din.start, h->din.len,  h->din.col,   h->dout.start, h->dout.len,
                  h->dout.col,  h->d_in_w,   h->d_wsum,    h->S,          h->P64,
                  h->P32,       h->mXi,      h->mEta,      h->tiles,      h->ntiles,
                  h->sI,        h->sJ,       h->scal,      h->counters,   h->diffbits,
                  h->gbar,      h->W,        h->rinv,       h->loff,     h->tile_nnz,  h->d_order,    h->d_order_row, h->d_jobs,
                  h->d_srcs,    h->d_ops,    h->d_cols,     h->d_ext2int, h->col_items,
                  h->col_gacc,  h->col_tcount};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& b : h->ob)
    if (b.p) cudaFree(b.p);
  if (h->Pp) cudaFree(h->Pp);
  if (h->pXi) cudaFree(h->pXi);
  if (h->pEta) cudaFree(h->pEta);
  void* colptrs[] = {h->g0_in_col, h->g0_out_col, h->g0_in_len, h->g0_fwd.chunks,
                     h->g0_hor.chunks, h->cur_fwd.chunks, h->cur_hor.chunks};
  for (void* p : colptrs)
    if (p) cudaFree(p);
  // the panel snapshots come from the stream-ordered allocator
  for (void* p : h->hist)
    if (p) cudaFreeAsync(p, h->st);
  if (!h->hist.empty()) cudaStreamSynchronize(h->st);
  for (auto& e : h->events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& a : h->phase_ev)
    for (auto& e : a) cudaEventDestroy(e);
  delete h;
}

}  // namespace

extern "C" {

simrank_status simrank_default_config(simrank_config* cfg) {
  if (!cfg) return SR_ERR_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->C = 0.6;
  cfg->K = 15;
  cfg->s_precision = 32;
  cfg->mode = SR_MODE_DENSE;
  cfg->n_capacity = 0;
  cfg->aff = 1;
  cfg->apply = SR_APPLY_UNIT;
  cfg->s_update = SR_SUPDATE_FUSED;
  cfg->tc = 0;
  cfg->init_max_sweeps = 400;
  cfg->init_tol = 0.0;  // 0 = precision default
  cfg->profile = 0;
  cfg->relabel = 1;
  cfg->upper_only = 1;
  cfg->timeout_iters = 0;
  cfg->cuda_stream = nullptr;
  return SR_OK;
}

simrank_status simrank_init(const simrank_config* cfg_in, int32_t n, int64_t m, const int32_t* src,
                            const int32_t* dst, const float* weight, const void* S0,
                            simrank_t* out) {
  if (!cfg_in || !out) return fail(nullptr, SR_ERR_ARG, "null config or output handle");
  *out = nullptr;
  simrank_config cfg = *cfg_in;
  if (!(cfg.C > 0.0 && cfg.C < 1.0)) return fail(nullptr, SR_ERR_ARG, "C must be in (0, 1)");
  if (cfg.K < 0 || cfg.K > 1023) return fail(nullptr, SR_ERR_ARG, "K must be in [0, 1023]");
  if (cfg.s_precision != 32 && cfg.s_precision != 64)
    return fail(nullptr, SR_ERR_ARG, "s_precision must be 32 or 64");
  if (cfg.mode != SR_MODE_DENSE && cfg.mode != SR_MODE_COLUMN)
    return fail(nullptr, SR_ERR_ARG, "mode must be SR_MODE_DENSE or SR_MODE_COLUMN");
  if (cfg.mode == SR_MODE_COLUMN) {
    if (S0) return fail(nullptr, SR_ERR_ARG, "column mode keeps no dense S: S0 must be NULL");
    if (cfg.apply == SR_APPLY_ONE_SHOT)
      return fail(nullptr, SR_ERR_UNSUPPORTED,
                  "column mode applies unit updates or sink blocks (Alg 7, §8)");
    cfg.relabel = 0;
  }
  if (n < 1 || m < 0) return fail(nullptr, SR_ERR_ARG, "need n >= 1 and m >= 0");
  if (m > 0 && (!src || !dst)) return fail(nullptr, SR_ERR_ARG, "null edge arrays");
  if (cfg.n_capacity == 0) cfg.n_capacity = n;
  if (cfg.n_capacity < n) return fail(nullptr, SR_ERR_ARG, "n_capacity < n");
  if ((int64_t)cfg.n_capacity > (int64_t)65535 * PT)
    return fail(nullptr, SR_ERR_ARG, "n_capacity too large for 16-bit tile indices");
  if (cfg.apply < 0 || cfg.apply > 2) return fail(nullptr, SR_ERR_ARG, "bad apply mode");
  if (cfg.prep_ctas < 0 || cfg.prep_cache < 0 || cfg.prep_cache > 16384 || cfg.prep_cache % 4 ||
      cfg.prep_item < 0)
    return fail(nullptr, SR_ERR_ARG,
                "prep_ctas, prep_item >= 0; prep_cache a multiple of 4 in [0, 16384]");
  if (cfg.defer < 0 || (cfg.defer > 1 && (int64_t)cfg.defer * (cfg.K + 1) > 4096))
    return fail(nullptr, SR_ERR_ARG, "defer * (K + 1) must be at most 4096");
  if (cfg.tc < 0 || cfg.tc > 2) return fail(nullptr, SR_ERR_ARG, "tc must be 0, 1 or 2");
  if (cfg.tc && cfg.s_precision != 32)
    return fail(nullptr, SR_ERR_ARG, "the tensor-core update needs s_precision = 32");
  if (cfg.init_tol <= 0.0) cfg.init_tol = 1e-13;
  if (cfg.init_max_sweeps <= 0) cfg.init_max_sweeps = 400;
  if (cfg.init_form < SR_INIT_SWEEPS || cfg.init_form > SR_INIT_COMPONENTS)
    return fail(nullptr, SR_ERR_ARG,
                "init_form must be SR_INIT_SWEEPS, SR_INIT_FOREST or SR_INIT_COMPONENTS");
  if (cfg.init_form != SR_INIT_SWEEPS && (cfg.mode != SR_MODE_DENSE || S0))
    return fail(nullptr, SR_ERR_ARG, "init_form computes the dense S: dense mode, S0 = NULL");
  if (cfg.init_form == SR_INIT_COMPONENTS && weight)
    return fail(nullptr, SR_ERR_UNSUPPORTED, "SR_INIT_COMPONENTS on a weighted graph");
  if (cfg.reanchor_every < 0 || cfg.reanchor_sweeps < 0)
    return fail(nullptr, SR_ERR_ARG, "reanchor_every and reanchor_sweeps must be >= 0");
  if (cfg.reanchor_sweeps == 0) cfg.reanchor_sweeps = 4;

  simrank_ctx* h = new (std::nothrow) simrank_ctx();
  if (!h) return fail(nullptr, SR_ERR_OOM, "host allocation failed");
  h->cfg = cfg;
  h->st = (cudaStream_t)cfg.cuda_stream;
  h->n_cur = n;
  h->n_cap = cfg.n_capacity;
  h->n_pad = ((cfg.n_capacity + PT - 1) / PT) * PT;
  h->nT_cap = h->n_pad / PT;
  h->ld = h->n_pad;
  h->K1 = cfg.K + 1;
  h->weighted = weight != nullptr;

  auto bail = [&](simrank_status s) {
    g_init_error = h->err;
    free_ctx(h);
    return s;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    return bail(fail(h, SR_ERR_CUDA, "no CUDA device"));

  // --- caller id -> storage id: with relabel, nodes that have in-degree 0
  // go after all others (their rows and columns of S are outside every
  // affected area, Thm 4), keeping ascending order inside both groups.
  h->ext2int.resize(h->n_cap);
  h->int2ext.resize(h->n_cap);
  for (int x = 0; x < h->n_cap; ++x) h->ext2int[x] = h->int2ext[x] = x;
  if (cfg.relabel && m > 0 && cfg.init_form != SR_INIT_COMPONENTS) {
    std::vector<char> has_in(n, 0);
    for (int64_t e = 0; e < m; ++e)
      if (dst[e] >= 0 && dst[e] < n) has_in[dst[e]] = 1;
    int next = 0;
    for (int pass = 1; pass >= 0; --pass)
      for (int x = 0; x < n; ++x)
        if (has_in[x] == pass) h->ext2int[x] = next++;
    for (int x = 0; x < n; ++x) h->int2ext[h->ext2int[x]] = x;
    h->relabeled = true;
  }
  // Example 1: weakly connected components stored one after another, grouped
  // into bins of at most 4096 nodes (a larger component is a bin of its own);
  // each bin's diagonal block of S gets its own Jacobi sweeps
  std::vector<std::pair<int, int>> bins;  // (first storage id, size)
  if (cfg.init_form == SR_INIT_COMPONENTS) {
    std::vector<int> root(n);
    for (int x = 0; x < n; ++x) root[x] = x;
    auto find = [&](int x) {
      while (root[x] != x) x = root[x] = root[root[x]];
      return x;
    };
    for (int64_t e = 0; e < m; ++e) {
      if (src[e] < 0 || dst[e] < 0 || src[e] >= n || dst[e] >= n) continue;  // rejected below
      const int a = find(src[e]), b = find(dst[e]);
      if (a != b) root[std::max(a, b)] = std::min(a, b);
    }
    std::vector<std::vector<int>> comp(n);
    for (int x = 0; x < n; ++x) comp[find(x)].push_back(x);
    int next = 0, bin_start = 0, bin_size = 0;
    for (int r = 0; r < n; ++r) {
      if (comp[r].empty()) continue;
      const int sz = (int)comp[r].size();
      if (bin_size > 0 && bin_size + sz > 4096) {
        bins.push_back({bin_start, bin_size});
        bin_start = next;
        bin_size = 0;
      }
      for (int x : comp[r]) h->ext2int[x] = next++;
      bin_size += sz;
    }
    if (bin_size > 0) bins.push_back({bin_start, bin_size});
    for (int x = 0; x < n; ++x) h->int2ext[h->ext2int[x]] = x;
    h->relabeled = true;
  }
  if (h->relabeled) {
    if (dev_alloc(&h->d_ext2int, (size_t)h->n_cap) != cudaSuccess ||
        cudaMemcpy(h->d_ext2int, h->ext2int.data(), h->n_cap * sizeof(int32_t),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(h, SR_ERR_OOM, "cudaMalloc of the id map failed"));
  }

  // --- host graph (storage ids), validated
  std::vector<std::vector<int32_t>> in_rows(h->n_pad), out_rows(h->n_pad);
  std::vector<std::vector<float>> in_w(h->weighted ? h->n_pad : 0), out_w(h->weighted ? h->n_pad : 0);
  h->edges.reserve((size_t)m * 2 + 16);
  for (int64_t e = 0; e < m; ++e) {
    const int32_t s = src[e], d = dst[e];
    if (s < 0 || d < 0 || s >= n || d >= n)
      return bail(fail(h, SR_ERR_ARG, "edge " + std::to_string(e) + " has an id outside [0, n)"));
    if (s == d) return bail(fail(h, SR_ERR_EDGE_EXISTS, "self-loop at edge " + std::to_string(e)));
    if (!h->edges.insert(ekey(s, d)).second)
      return bail(fail(h, SR_ERR_EDGE_EXISTS, "duplicate edge " + std::to_string(e)));
    if (h->weighted && !(weight[e] > 0.0f))
      return bail(fail(h, SR_ERR_ARG, "edge weights must be > 0"));
    const int32_t si = h->ext2int[s], di = h->ext2int[d];
    in_rows[di].push_back(si);
    out_rows[si].push_back(di);
    if (h->weighted) {
      in_w[di].push_back(weight[e]);
      out_w[si].push_back(weight[e]);
    }
    h->init_src.push_back(si);
    h->init_dst.push_back(di);
  }
  if (h->relabeled) {
    // the duplicate check above ran on caller ids; keep the edge set in storage ids
    std::unordered_set<uint64_t> mapped;
    mapped.reserve(h->edges.size() * 2 + 16);
    for (uint64_t k : h->edges)
      mapped.insert(ekey(h->ext2int[(int32_t)(k >> 32)], h->ext2int[(int32_t)(k & 0xffffffffu)]));
    h->edges.swap(mapped);
  }
  build_adj(h->hin, h->n_pad, in_rows);
  build_adj(h->hout, h->n_pad, out_rows);

  // --- forest form of the initial S (Example 2): each node's parent (its one
  // in-neighbour) and level; nodes beyond n are isolated roots
  std::vector<int32_t> f_parent, f_level;
  int f_top = 0;
  if (cfg.init_form == SR_INIT_FOREST) {
    f_parent.assign(h->n_cap, -1);
    f_level.assign(h->n_cap, -1);
    for (int x = 0; x < n; ++x) {
      if (in_rows[x].size() > 1)
        return bail(fail(h, SR_ERR_ARG, "SR_INIT_FOREST needs every in-degree <= 1 (node " +
                                            std::to_string(h->int2ext[x]) + ")"));
      if (!in_rows[x].empty()) f_parent[x] = in_rows[x][0];
    }
    std::vector<int32_t> path;
    for (int x = 0; x < h->n_cap; ++x) {
      path.clear();
      int y = x;
      while (y >= 0 && f_level[y] < 0) {
        path.push_back(y);
        if ((int)path.size() > n + 1)
          return bail(fail(h, SR_ERR_ARG, "SR_INIT_FOREST: the initial graph has a cycle"));
        y = f_parent[y];
      }
      int lv = y < 0 ? -1 : f_level[y];
      for (auto it = path.rbegin(); it != path.rend(); ++it) f_level[*it] = ++lv;
      f_top = std::max(f_top, lv);
    }
  }

  // --- device graph
  auto upload_adj = [&](DevAdj& D, const HostAdj& A) -> simrank_status {
    D.pool_cap = (int64_t)A.pool.size();
    CUDA_TRY(h, dev_alloc(&D.start, (size_t)h->n_pad));
    CUDA_TRY(h, dev_alloc(&D.len, (size_t)h->n_pad));
    CUDA_TRY(h, dev_alloc(&D.col, (size_t)D.pool_cap));
    CUDA_TRY(h, cudaMemcpy(D.start, A.start.data(), A.start.size() * sizeof(int64_t),
                           cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(D.len, A.len.data(), A.len.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(D.col, A.pool.data(), A.pool.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice));
    return SR_OK;
  };
  simrank_status s;
  if ((s = upload_adj(h->din, h->hin)) != SR_OK) return bail(s);
  if ((s = upload_adj(h->dout, h->hout)) != SR_OK) return bail(s);
  if (h->weighted) {
    std::vector<float> wpool(h->hin.pool.size(), 0.f), opool(h->hout.pool.size(), 0.f);
    std::vector<double> wsum(h->n_pad, 0.0);
    for (int a = 0; a < h->n_pad; ++a) {
      for (size_t e = 0; e < in_w[a].size(); ++e) {
        wpool[h->hin.start[a] + e] = in_w[a][e];
        wsum[a] += in_w[a][e];
      }
      for (size_t e = 0; e < out_w[a].size(); ++e) opool[h->hout.start[a] + e] = out_w[a][e];
    }
    if (cudaMalloc(&h->d_in_w, wpool.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_out_w, opool.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&h->d_wsum, wsum.size() * sizeof(double)) != cudaSuccess)
      return bail(fail(h, SR_ERR_OOM, "cudaMalloc of weights failed"));
    cudaMemcpy(h->d_in_w, wpool.data(), wpool.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(h->d_out_w, opool.data(), opool.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(h->d_wsum, wsum.data(), wsum.size() * sizeof(double), cudaMemcpyHostToDevice);
  }

  // --- S, panels, masks
  h->column = cfg.mode == SR_MODE_COLUMN;
  const size_t eb = (size_t)elem_bytes(h);
  const size_t s_bytes = h->column ? 256 : (size_t)h->n_pad * h->ld * eb;
  if (cudaMalloc(&h->S, s_bytes) != cudaSuccess)
    return bail(fail(h, SR_ERR_OOM, "cudaMalloc of S (" + std::to_string(s_bytes) + " bytes) failed"));
  const size_t panel_elems = (size_t)h->nT_cap * 2 * h->K1 * PT;
  if (dev_alloc(&h->P64, panel_elems) != cudaSuccess ||
      (cfg.s_precision == 32 && dev_alloc(&h->P32, panel_elems) != cudaSuccess) ||
      dev_alloc(&h->mXi, (size_t)h->nT_cap) != cudaSuccess ||
      dev_alloc(&h->mEta, (size_t)h->nT_cap) != cudaSuccess ||
      dev_alloc(&h->tiles, (size_t)h->nT_cap * (h->nT_cap + 1) / 2) != cudaSuccess ||
      dev_alloc(&h->ntiles, 1) != cudaSuccess || dev_alloc(&h->sI, (size_t)h->n_pad) != cudaSuccess ||
      dev_alloc(&h->sJ, (size_t)h->n_pad) != cudaSuccess || dev_alloc(&h->scal, 8) != cudaSuccess ||
      dev_alloc(&h->counters, CNT_N) != cudaSuccess || dev_alloc(&h->diffbits, 1) != cudaSuccess ||
      dev_alloc(&h->gbar, 4) != cudaSuccess)
    return bail(fail(h, SR_ERR_OOM, "cudaMalloc of work buffers failed"));
  cudaMemsetAsync(h->P64, 0, panel_elems * sizeof(double), h->st);
  if (h->P32) cudaMemsetAsync(h->P32, 0, panel_elems * sizeof(float), h->st);
  cudaMemsetAsync(h->mXi, 0, h->nT_cap * sizeof(uint64_t), h->st);
  cudaMemsetAsync(h->mEta, 0, h->nT_cap * sizeof(uint64_t), h->st);
  cudaMemsetAsync(h->counters, 0, CNT_N * sizeof(int64_t), h->st);
  cudaMemsetAsync(h->gbar, 0, 4 * sizeof(unsigned int), h->st);
  cudaMemsetAsync(h->S, 0, s_bytes, h->st);

  if (h->column) {
    // snapshot of the initial graph for the base columns (Procedure 1)
    std::vector<RowChunk> ch;
    if (dev_alloc(&h->g0_in_col, (size_t)h->din.pool_cap) != cudaSuccess ||
        dev_alloc(&h->g0_out_col, (size_t)h->dout.pool_cap) != cudaSuccess ||
        dev_alloc(&h->g0_in_len, (size_t)h->n_pad) != cudaSuccess)
      return bail(fail(h, SR_ERR_OOM, "cudaMalloc of the graph snapshot failed"));
    cudaMemcpyAsync(h->g0_in_col, h->din.col, h->din.pool_cap * 4, cudaMemcpyDeviceToDevice, h->st);
    cudaMemcpyAsync(h->g0_out_col, h->dout.col, h->dout.pool_cap * 4, cudaMemcpyDeviceToDevice,
                    h->st);
    cudaMemcpyAsync(h->g0_in_len, h->din.len, (size_t)h->n_pad * 4, cudaMemcpyDeviceToDevice, h->st);
    int64_t cap_f = 0, cap_h = 0;
    build_chunks(h->hout, h->n_pad, ch);
    if ((s = upload_chunks(h, ch, h->g0_fwd, &cap_f)) != SR_OK) return bail(s);
    build_chunks(h->hin, h->n_pad, ch);
    if ((s = upload_chunks(h, ch, h->g0_hor, &cap_h)) != SR_OK) return bail(s);
    if (cudaStreamSynchronize(h->st) != cudaSuccess)
      return bail(fail(h, SR_ERR_CUDA, "init synchronisation failed"));
  } else if (S0) {
    const void* src_S = S0;
    std::vector<unsigned char> perm_S;
    if (h->relabeled) {
      perm_S.resize((size_t)n * n * eb);
      for (int r = 0; r < n; ++r) {
        const unsigned char* row = (const unsigned char*)S0 + (size_t)h->int2ext[r] * n * eb;
        unsigned char* dstrow = perm_S.data() + (size_t)r * n * eb;
        for (int c = 0; c < n; ++c)
          std::memcpy(dstrow + (size_t)c * eb, row + (size_t)h->int2ext[c] * eb, eb);
      }
      src_S = perm_S.data();
    }
    cudaError_t e = cudaMemcpy2DAsync(h->S, h->ld * eb, src_S, (size_t)n * eb, (size_t)n * eb, n,
                                      cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return bail(fail(h, SR_ERR_CUDA, "upload of S0 failed"));
    launch_set_diag(h->S, cfg.s_precision, n, h->n_cap, h->ld, 1.0 - cfg.C, h->st);
    if (cudaStreamSynchronize(h->st) != cudaSuccess)
      return bail(fail(h, SR_ERR_CUDA, "init synchronisation failed"));
  } else if (cfg.init_form == SR_INIT_FOREST) {
    std::vector<double> powC(f_top + 2, 1.0);
    for (size_t k = 1; k < powC.size(); ++k) powC[k] = powC[k - 1] * cfg.C;
    int32_t *d_par = nullptr, *d_lev = nullptr;
    double* d_pow = nullptr;
    cudaError_t e = dev_alloc(&d_par, (size_t)h->n_cap);
    if (e == cudaSuccess) e = dev_alloc(&d_lev, (size_t)h->n_cap);
    if (e == cudaSuccess) e = dev_alloc(&d_pow, powC.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(d_par, f_parent.data(), h->n_cap * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d_lev, f_level.data(), h->n_cap * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(d_pow, powC.data(), powC.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      launch_forest_init(h->S, cfg.s_precision, h->ld, d_par, d_lev, d_pow, h->n_cap, h->nT_cap,
                         upper(h) ? 1 : 0, h->st);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    cudaFree(d_par);
    cudaFree(d_lev);
    cudaFree(d_pow);
    if (e != cudaSuccess)
      return bail(fail(h, SR_ERR_CUDA, std::string("forest init: ") + cudaGetErrorString(e)));
    h->stats.init_residual = 0.0;
    h->stats.init_sweeps = 0;
  } else if (cfg.init_form == SR_INIT_COMPONENTS) {
    // every bin's S by the batch algorithm on its own subgraph, copied into
    // its diagonal block; the blocks between bins stay zero
    launch_set_diag(h->S, cfg.s_precision, 0, h->n_cap, h->ld, 1.0 - cfg.C, h->st);
    std::vector<int32_t> bin_of(n);
    for (size_t b = 0; b < bins.size(); ++b)
      for (int x = bins[b].first; x < bins[b].first + bins[b].second; ++x) bin_of[x] = (int)b;
    std::vector<std::vector<int32_t>> bsrc(bins.size()), bdst(bins.size());
    for (size_t e = 0; e < h->init_src.size(); ++e) {
      const int b = bin_of[h->init_src[e]];
      bsrc[b].push_back(h->init_src[e] - bins[b].first);
      bdst[b].push_back(h->init_dst[e] - bins[b].first);
    }
    double worst = 0.0;
    int most = 0;
    for (size_t b = 0; b < bins.size(); ++b) {
      if (bsrc[b].empty()) continue;  // isolated nodes: S_xx = 1 - C is set
      simrank_config sc = cfg;
      sc.init_form = SR_INIT_SWEEPS;
      sc.relabel = 0;
      sc.upper_only = 0;
      sc.n_capacity = 0;
      sc.reanchor_every = 0;
      simrank_t sub = nullptr;
      s = simrank_init(&sc, bins[b].second, (int64_t)bsrc[b].size(), bsrc[b].data(),
                       bdst[b].data(), nullptr, nullptr, &sub);
      if (s != SR_OK) return bail(fail(h, s, "component init: " + g_init_error));
      const int64_t r0 = bins[b].first, sz = bins[b].second;
      cudaError_t e = cudaMemcpy2DAsync((unsigned char*)h->S + (r0 * h->ld + r0) * eb, h->ld * eb,
                                        sub->S, sub->ld * eb, sz * eb, sz,
                                        cudaMemcpyDeviceToDevice, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      worst = std::max(worst, sub->stats.init_residual);
      most = std::max(most, sub->stats.init_sweeps);
      simrank_destroy(sub);
      if (e != cudaSuccess)
        return bail(fail(h, SR_ERR_CUDA, std::string("component copy: ") + cudaGetErrorString(e)));
    }
    h->stats.init_residual = worst;
    h->stats.init_sweeps = most;
  } else {
    // start from (1 - C) I on the whole capacity
    launch_set_diag(h->S, cfg.s_precision, 0, h->n_cap, h->ld, 1.0 - cfg.C, h->st);
    double diff = 0.0, tol_used = cfg.init_tol;
    int sweeps = 0;
    if ((s = jacobi_sweeps(h, cfg.init_max_sweeps, cfg.init_tol, &diff, &sweeps, &tol_used)) !=
        SR_OK)
      return bail(s);
    h->stats.init_residual = diff;
    h->stats.init_sweeps = sweeps;
    if (!(diff < tol_used))
      return bail(fail(h, SR_ERR_NOT_CONVERGED,
                       "Jacobi init stopped at max-abs change " + std::to_string(diff)));
  }
  *out = h;
  return SR_OK;
}

simrank_status simrank_apply_updates(simrank_t h, const simrank_update* u, int64_t count) {
  if (!h) return fail(nullptr, SR_ERR_ARG, "null handle");
  if (count < 0 || (count > 0 && !u)) return fail(h, SR_ERR_ARG, "bad update array");
  if (count == 0) return SR_OK;
  if (h->weighted) return fail(h, SR_ERR_UNSUPPORTED, "updates on a weighted graph");
  // caller ids -> storage ids (new ids >= n_cur map to themselves)
  std::vector<simrank_update> um(u, u + count);
  auto to_int = [&](int32_t x) { return (x >= 0 && x < h->n_cap) ? h->ext2int[x] : x; };
  if (h->relabeled)
    for (auto& v : um) {
      v.src = to_int(v.src);
      v.dst = to_int(v.dst);
    }
  int n_after = h->n_cur;
  simrank_status s = validate(h, um.data(), count, &n_after);
  if (s != SR_OK) return s;

  // Plan the rank-one updates: (sink, op, sources, d_j, patch op range).
  struct R1 {
    int32_t sink, op, d_j, delta;
    int64_t src_off, op_begin, op_end;
  };
  std::vector<R1> plan;
  std::vector<int32_t> srcs;
  std::vector<PatchOp> ops;
  const int n_old = h->n_cur;
  auto add_r1 = [&](int32_t j, int32_t op, const std::vector<int32_t>& I) {
    R1 r;
    r.sink = j;
    r.op = op;
    r.d_j = h->hin.len[j];
    r.delta = (int)I.size();
    r.src_off = (int64_t)srcs.size();
    r.op_begin = (int64_t)ops.size();
    for (int32_t i : I) {
      srcs.push_back(i);
      if (op > 0) {
        adj_append(h->hin, j, i, ops, true);
        adj_append(h->hout, i, j, ops, false);
        h->edges.insert(ekey(i, j));
      } else {
        adj_remove(h->hin, j, i, ops, true);
        adj_remove(h->hout, i, j, ops, false);
        h->edges.erase(ekey(i, j));
      }
    }
    r.op_end = (int64_t)ops.size();
    plan.push_back(r);
  };
  if (h->column) {
    // Alg 7: one stored update at a time (a unit update, or with
    // SR_APPLY_SINK_BLOCKS a similar-sink block of the net batch, §8); the old
    // columns come from the graph before that update, so each one is planned
    // right before it runs
    std::vector<Block> blocks;
    if (h->cfg.apply == SR_APPLY_SINK_BLOCKS) {
      std::string msg;
      if ((s = plan_blocks(um.data(), count, n_old, blocks, msg)) != SR_OK) return fail(h, s, msg);
    } else {
      for (int64_t t = 0; t < count; ++t) blocks.push_back(Block{um[t].dst, um[t].op, {um[t].src}});
    }
    h->n_cur = n_after;
    for (const Block& b : blocks) {
      const int32_t j = b.sink, op = b.op;
      // chunk lists of the graph before this update: the previous one changed
      // the out-rows of its sources and the in-row of its sink only
      bool ok_f = h->col_chunks_ok && !h->col_last_srcs.empty();
      for (int32_t i : h->col_last_srcs)
        ok_f = ok_f && patch_row_chunks(h, h->hout, i, h->hfwd, h->ffwd, h->cur_fwd);
      bool ok_h = h->col_chunks_ok && h->col_last_j >= 0 &&
                  patch_row_chunks(h, h->hin, h->col_last_j, h->hhor, h->fhor, h->cur_hor);
      if (!ok_f) {
        build_chunks(h->hout, h->n_pad, h->hfwd, &h->ffwd);
        if ((s = upload_chunks(h, h->hfwd, h->cur_fwd, &h->cur_fwd_cap)) != SR_OK) return s;
      }
      if (!ok_h) {
        build_chunks(h->hin, h->n_pad, h->hhor, &h->fhor);
        if ((s = upload_chunks(h, h->hhor, h->cur_hor, &h->cur_hor_cap)) != SR_OK) return s;
      }
      h->col_chunks_ok = true;
      h->col_last_srcs = b.srcs;
      h->col_last_j = j;
      std::vector<PatchOp> ops1;
      const int d_j = h->hin.len[j];
      for (int32_t i : b.srcs) {
        if (op > 0) {
          adj_append(h->hin, j, i, ops1, true);
          adj_append(h->hout, i, j, ops1, false);
          h->edges.insert(ekey(i, j));
        } else {
          adj_remove(h->hin, j, i, ops1, true);
          adj_remove(h->hout, i, j, ops1, false);
          h->edges.erase(ekey(i, j));
        }
      }
      if ((s = grow_pool(h, h->din, h->hin)) != SR_OK) return s;
      if ((s = grow_pool(h, h->dout, h->hout)) != SR_OK) return s;
      if ((s = ensure_dev_capacity(h, (int64_t)b.srcs.size() + 1, (int64_t)ops1.size())) != SR_OK)
        return s;
      CUDA_TRY(h, cudaMemcpyAsync(h->d_ops, ops1.data(), ops1.size() * sizeof(PatchOp),
                                  cudaMemcpyHostToDevice, h->st));
      if ((s = run_column_update(h, b.srcs, j, op, d_j, 0, (int64_t)ops1.size(), h->d_srcs)) !=
          SR_OK)
        return s;
    }
    h->stats.updates += count;
    return SR_OK;
  }
  if (h->cfg.apply == SR_APPLY_ONE_SHOT) {
    // net update per sink, in storage ids; then one rank-2r update
    std::vector<Block> blocks;
    std::string msg;
    if ((s = plan_blocks(um.data(), count, n_old, blocks, msg)) != SR_OK) return fail(h, s, msg);
    std::map<int32_t, std::vector<int32_t>> plus, minus;
    for (const Block& b : blocks) {
      auto& dstv = (b.op > 0 ? plus : minus)[b.sink];
      dstv.insert(dstv.end(), b.srcs.begin(), b.srcs.end());
      for (int32_t i : b.srcs) {
        if (b.op > 0) {
          adj_append(h->hin, b.sink, i, ops, true);
          adj_append(h->hout, i, b.sink, ops, false);
          h->edges.insert(ekey(i, b.sink));
        } else {
          adj_remove(h->hin, b.sink, i, ops, true);
          adj_remove(h->hout, i, b.sink, ops, false);
          h->edges.erase(ekey(i, b.sink));
        }
      }
    }
    h->n_cur = n_after;
    if ((s = grow_pool(h, h->din, h->hin)) != SR_OK) return s;
    if ((s = grow_pool(h, h->dout, h->hout)) != SR_OK) return s;
    if ((s = ensure_dev_capacity(h, 1, (int64_t)ops.size())) != SR_OK) return s;
    if ((s = run_one_shot(h, plus, minus, ops)) != SR_OK) return s;
    h->stats.updates += count;
    return maybe_reanchor(h, count);
  }
  if (h->cfg.apply == SR_APPLY_UNIT) {
    for (int64_t t = 0; t < count; ++t) add_r1(um[t].dst, um[t].op, {um[t].src});
  } else {
    // the canonical block order is defined on caller ids
    std::vector<Block> blocks;
    std::string msg;
    if ((s = plan_blocks(u, count, n_old, blocks, msg)) != SR_OK) return fail(h, s, msg);
    for (Block& b : blocks) {
      for (int32_t& x : b.srcs) x = to_int(x);
      add_r1(to_int(b.sink), b.op, b.srcs);
    }
  }
  h->n_cur = n_after;
  if ((s = grow_pool(h, h->din, h->hin)) != SR_OK) return s;
  if ((s = grow_pool(h, h->dout, h->hout)) != SR_OK) return s;
  if ((s = ensure_dev_capacity(h, (int64_t)srcs.size() + 2, (int64_t)ops.size())) != SR_OK) return s;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_srcs, srcs.data(), srcs.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, h->st));
  if (!ops.empty())
    CUDA_TRY(h, cudaMemcpyAsync(h->d_ops, ops.data(), ops.size() * sizeof(PatchOp),
                                cudaMemcpyHostToDevice, h->st));
  // the staging vectors must outlive the asynchronous copies
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  for (const R1& r : plan) {
    if ((s = run_rank_one(h, r.src_off, r.delta, r.sink, r.op, r.d_j, r.op_begin, r.op_end)) !=
        SR_OK)
      return s;
    // every rank-one update (a unit update or a sink block) counts its edges
    if ((s = maybe_reanchor(h, r.delta)) != SR_OK) return s;
  }
  if ((s = flush_pending(h)) != SR_OK) return s;
  h->stats.updates += count;
  return SR_OK;
}

simrank_status simrank_columns(simrank_t h, const int32_t* cols, int32_t ncols, void* out,
                               int32_t out_on_device, int32_t out_fp64) {
  if (!h) return fail(nullptr, SR_ERR_ARG, "null handle");
  if (ncols < 0 || (ncols > 0 && (!cols || !out))) return fail(h, SR_ERR_ARG, "bad column request");
  for (int c = 0; c < ncols; ++c)
    if (cols[c] < 0 || cols[c] >= h->n_cur) return fail(h, SR_ERR_ARG, "column id out of range");
  if (ncols == 0) return SR_OK;
  if (h->column) return column_mode_columns(h, cols, ncols, out, out_on_device, out_fp64);
  std::vector<int32_t> icols(cols, cols + ncols);
  for (int32_t& x : icols) x = h->ext2int[x];
  cols = icols.data();
  const int32_t* perm = h->relabeled ? h->d_ext2int : nullptr;
  if (ncols > h->cols_cap) {
    if (h->d_cols) cudaFree(h->d_cols);
    h->cols_cap = ncols;
    CUDA_TRY(h, dev_alloc(&h->d_cols, (size_t)ncols));
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_cols, cols, ncols * sizeof(int32_t), cudaMemcpyHostToDevice,
                              h->st));
  const size_t ob = (size_t)h->n_cur * ncols * (out_fp64 ? 8 : 4);
  if (out_on_device) {
    launch_copy_cols(h->S, h->cfg.s_precision, h->ld, h->d_cols, perm, ncols, h->n_cur, out,
                     out_fp64, h->st, upper(h));
    LAUNCH_CHECK(h);
    CUDA_TRY(h, cudaStreamSynchronize(h->st));  // cols staging reuse safety
    return SR_OK;
  }
  void* tmp = nullptr;
  CUDA_TRY(h, cudaMalloc(&tmp, ob));
  launch_copy_cols(h->S, h->cfg.s_precision, h->ld, h->d_cols, perm, ncols, h->n_cur, tmp,
                   out_fp64, h->st, upper(h));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, ob, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(h, SR_ERR_CUDA, std::string("columns: ") + cudaGetErrorString(e));
  return SR_OK;
}

int32_t simrank_num_nodes(simrank_t h) { return h ? h->n_cur : -1; }

const char* simrank_last_error(simrank_t h) { return h ? h->err.c_str() : g_init_error.c_str(); }

simrank_status simrank_sync(simrank_t h) {
  if (!h) return fail(nullptr, SR_ERR_ARG, "null handle");
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  int64_t status = 0;
  CUDA_TRY(h, cudaMemcpy(&status, h->counters + CNT_STATUS, sizeof(status), cudaMemcpyDeviceToHost));
  if (status != 0) return fail(h, (simrank_status)status, "a bounded device wait ran out");
  return SR_OK;
}

void simrank_destroy(simrank_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  free_ctx(h);
}

simrank_status simrank_get_stats(simrank_t h, simrank_stats* out) {
  if (!h || !out) return fail(h, SR_ERR_ARG, "null argument");
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  harvest_events(h);
  int64_t c[CNT_N];
  CUDA_TRY(h, cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
  simrank_stats r = h->stats;
  r.tiles_touched = c[CNT_TILES_TOUCHED];
  r.s_bytes = c[CNT_S_BYTES];
  r.panel_bytes = c[CNT_PANEL_BYTES];
  r.s_update_launches = h->prof_launches;
  r.kernel_launches = h->launches;
  r.s_update_ms = h->prof_ms;
  for (int q = 0; q < 4; ++q) r.phase_ms[q] = h->phase_ms[q];
  *out = r;
  return SR_OK;
}

simrank_status simrank_set_launch(simrank_t h, const simrank_config* knobs) {
  if (!h || !knobs) return fail(h, SR_ERR_ARG, "null argument");
  const simrank_config& k = *knobs;
  if (k.prep_ctas < 0 || k.prep_cache < 0 || k.prep_cache > 16384 || k.prep_cache % 4 ||
      k.prep_item < 0)
    return fail(h, SR_ERR_ARG, "prep_ctas, prep_item >= 0; prep_cache a multiple of 4 in [0, 16384]");
  if (k.defer < 0 || (k.defer > 1 && (int64_t)k.defer * h->K1 > 4096))
    return fail(h, SR_ERR_ARG, "defer * (K + 1) must be at most 4096");
  if (k.tc < 0 || k.tc > 2) return fail(h, SR_ERR_ARG, "tc must be 0, 1 or 2");
  if (k.tc && h->cfg.s_precision != 32)
    return fail(h, SR_ERR_ARG, "the tensor-core update needs s_precision = 32");
  if (k.s_kernel < 0 || k.s_kernel > 1) return fail(h, SR_ERR_ARG, "s_kernel must be 0 or 1");
  // pending updates are applied under the old group size, whose buffers go
  simrank_status s = flush_pending(h);
  if (s != SR_OK) return s;
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  if (h->Pp && std::max(1, (int)k.defer) != group(h)) {
    cudaFree(h->Pp);
    cudaFree(h->pXi);
    cudaFree(h->pEta);
    h->Pp = nullptr;
    h->pXi = h->pEta = nullptr;
  }
  h->cfg.defer = k.defer;
  h->cfg.tc = k.tc;
  h->cfg.prep_ctas = k.prep_ctas;
  h->cfg.prep_cache = k.prep_cache;
  h->cfg.prep_item = k.prep_item;
  h->cfg.s_kernel = k.s_kernel;
  return SR_OK;
}

simrank_status simrank_reanchor(simrank_t h, int32_t sweeps, double* max_change) {
  if (!h) return fail(nullptr, SR_ERR_ARG, "null handle");
  if (h->column) return fail(h, SR_ERR_UNSUPPORTED, "column mode keeps no dense S to re-anchor");
  if (sweeps <= 0) return fail(h, SR_ERR_ARG, "sweeps must be positive");
  double first = 0.0, diff = 0.0;
  int done = 0;
  simrank_status s = reanchor_run(h, sweeps, 0.0, &first, &diff, &done);
  if (s != SR_OK) return s;
  h->stats.init_residual = diff;
  h->stats.init_sweeps = done;
  if (max_change) *max_change = diff;
  return SR_OK;
}

simrank_status simrank_grad(simrank_t h, const int32_t* pa, const int32_t* pb, const double* target,
                            int64_t npairs, double* loss, double* grad_weight) {
  if (!h) return fail(nullptr, SR_ERR_ARG, "null handle");
  if (npairs < 0 || (npairs > 0 && (!pa || !pb || !target)) || !loss || !grad_weight)
    return fail(h, SR_ERR_ARG, "bad pair arrays");
  if (h->stats.updates > 0)
    return fail(h, SR_ERR_UNSUPPORTED, "simrank_grad needs the graph as initialised (no updates)");
  const int n_pad = h->n_pad, K = h->cfg.K;
  const double C = h->cfg.C;
  for (int64_t p = 0; p < npairs; ++p)
    if (pa[p] < 0 || pb[p] < 0 || pa[p] >= h->n_cur || pb[p] >= h->n_cur)
      return fail(h, SR_ERR_ARG, "pair id out of range");
  simrank_status s;
  std::vector<RowChunk> ch;
  build_chunks(h->hout, n_pad, ch);
  if ((s = upload_chunks(h, ch, h->cur_fwd, &h->cur_fwd_cap)) != SR_OK) return s;
  build_chunks(h->hin, n_pad, ch);
  if ((s = upload_chunks(h, ch, h->cur_hor, &h->cur_hor_cap)) != SR_OK) return s;
  h->col_chunks_ok = false;
  WeightView wv;
  if (h->weighted) {
    wv.in_w = h->d_in_w;
    wv.out_w = h->d_out_w;
    wv.wsum = h->d_wsum;
  }
  std::vector<int32_t> A(npairs), Bv(npairs);
  for (int64_t p = 0; p < npairs; ++p) {
    A[p] = h->ext2int[pa[p]];
    Bv[p] = h->ext2int[pb[p]];
  }
  // endpoint block size from free memory: F and F_psi (K+1 blocks each), 2 y blocks
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(h, cudaMemGetInfo(&free_b, &total_b));
  const size_t per_col = (size_t)n_pad * 8 * (2 * (K + 1) + 2);
  const int Eb = (int)std::max<size_t>(1, std::min<size_t>(1024, (size_t)(0.5 * free_b) / per_col));
  const size_t blkb = (size_t)n_pad * Eb * 8;
  if ((s = ob_ensure(h, 14, blkb * (K + 1))) != SR_OK) return s;
  if ((s = ob_ensure(h, 15, blkb * (K + 1))) != SR_OK) return s;
  if ((s = ob_ensure(h, 16, blkb)) != SR_OK) return s;
  if ((s = ob_ensure(h, 17, blkb)) != SR_OK) return s;
  const int64_t pool = h->din.pool_cap;
  if ((s = ob_ensure(h, 18, (size_t)pool * 8 * 2)) != SR_OK) return s;
  double* F = (double*)h->ob[14].p;
  double* Fp = (double*)h->ob[15].p;
  double* y0 = (double*)h->ob[16].p;
  double* y1 = (double*)h->ob[17].p;
  double* G = (double*)h->ob[18].p;
  double* dW = G + pool;
  auto upload_i32 = [&](int slot, const std::vector<int32_t>& v) -> simrank_status {
    simrank_status r = ob_ensure(h, slot, std::max<size_t>(v.size(), 1) * 4);
    if (r != SR_OK) return r;
    if (!v.empty())
      CUDA_TRY(h, cudaMemcpyAsync(h->ob[slot].p, v.data(), v.size() * 4, cudaMemcpyHostToDevice, h->st));
    return SR_OK;
  };
  auto upload_f64 = [&](int slot, const std::vector<double>& v) -> simrank_status {
    simrank_status r = ob_ensure(h, slot, std::max<size_t>(v.size(), 1) * 8);
    if (r != SR_OK) return r;
    if (!v.empty())
      CUDA_TRY(h, cudaMemcpyAsync(h->ob[slot].p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, h->st));
    return SR_OK;
  };

  // ---- pass 1: S_K[a_p, b_p] from Procedure 1 on the distinct b's
  std::vector<int32_t> bcols(Bv);
  std::sort(bcols.begin(), bcols.end());
  bcols.erase(std::unique(bcols.begin(), bcols.end()), bcols.end());
  std::vector<double> sval(npairs, 0.0);
  for (size_t c0 = 0; c0 < bcols.size(); c0 += Eb) {
    const int B = (int)std::min<size_t>(Eb, bcols.size() - c0);
    std::vector<int32_t> cols(bcols.begin() + c0, bcols.begin() + c0 + B);
    std::vector<int32_t> rows, cidx;
    std::vector<int64_t> who;
    for (int64_t p = 0; p < npairs; ++p) {
      auto it = std::lower_bound(cols.begin(), cols.end(), Bv[p]);
      if (it != cols.end() && *it == Bv[p]) {
        rows.push_back(A[p]);
        cidx.push_back((int32_t)(it - cols.begin()));
        who.push_back(p);
      }
    }
    if ((s = upload_i32(19, cols)) != SR_OK) return s;
    if ((s = upload_i32(20, rows)) != SR_OK) return s;
    if ((s = upload_i32(21, cidx)) != SR_OK) return s;
    if ((s = ob_ensure(h, 22, std::max<size_t>(rows.size(), 1) * 8)) != SR_OK) return s;
    launch_partial_sim_block(h->cur_fwd, h->cur_hor, h->dout.col, h->din.col, h->din.len,
                             (const int32_t*)h->ob[19].p, B, n_pad, K, C, 64, F, y0, y1, Fp, h->st,
                             wv);
    launch_adj_pairs(Fp, B, (const int32_t*)h->ob[20].p, (const int32_t*)h->ob[21].p,
                     (int64_t)rows.size(), (double*)h->ob[22].p, h->st);
    std::vector<double> got(rows.size());
    if (!rows.empty())
      CUDA_TRY(h, cudaMemcpyAsync(got.data(), h->ob[22].p, rows.size() * 8, cudaMemcpyDeviceToHost,
                                  h->st));
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
    for (size_t q = 0; q < who.size(); ++q) sval[who[q]] = got[q];
  }
  double L = 0.0;
  std::vector<double> g(npairs);
  for (int64_t p = 0; p < npairs; ++p) {
    const double r = sval[p] - target[p];
    L += r * r;
    g[p] = 2.0 * r;
  }
  *loss = L;

  // ---- pass 2: dL/dQ at the edges, per block of endpoints
  std::vector<int32_t> ends(A);
  ends.insert(ends.end(), Bv.begin(), Bv.end());
  std::sort(ends.begin(), ends.end());
  ends.erase(std::unique(ends.begin(), ends.end()), ends.end());
  std::vector<std::vector<std::pair<int32_t, double>>> psi(ends.size());
  for (int64_t p = 0; p < npairs; ++p) {
    const size_t ia = std::lower_bound(ends.begin(), ends.end(), A[p]) - ends.begin();
    const size_t ib = std::lower_bound(ends.begin(), ends.end(), Bv[p]) - ends.begin();
    psi[ia].push_back({Bv[p], g[p]});
    psi[ib].push_back({A[p], g[p]});
  }
  CUDA_TRY(h, cudaMemsetAsync(G, 0, (size_t)pool * 8, h->st));
  for (size_t c0 = 0; c0 < ends.size(); c0 += Eb) {
    const int B = (int)std::min<size_t>(Eb, ends.size() - c0);
    std::vector<int32_t> un, uc, pn, pc;
    std::vector<double> ucoef, pcoef;
    for (int c = 0; c < B; ++c) {
      un.push_back(ends[c0 + c]);
      uc.push_back(c);
      ucoef.push_back(1.0);
      for (auto& nv : psi[c0 + c]) {
        pn.push_back(nv.first);
        pc.push_back(c);
        pcoef.push_back(nv.second);
      }
    }
    if ((s = upload_i32(19, un)) != SR_OK) return s;
    if ((s = upload_i32(20, uc)) != SR_OK) return s;
    if ((s = upload_f64(22, ucoef)) != SR_OK) return s;
    if ((s = upload_i32(21, pn)) != SR_OK) return s;
    if ((s = upload_i32(23, pc)) != SR_OK) return s;
    std::vector<double>* keep = &pcoef;
    if ((s = ob_ensure(h, 13, std::max<size_t>(keep->size(), 1) * 8)) != SR_OK) return s;
    if (!keep->empty())
      CUDA_TRY(h, cudaMemcpyAsync(h->ob[13].p, keep->data(), keep->size() * 8,
                                  cudaMemcpyHostToDevice, h->st));
    const int64_t blk = (int64_t)n_pad * B;
    CUDA_TRY(h, cudaMemsetAsync(F, 0, (size_t)blk * 8, h->st));
    CUDA_TRY(h, cudaMemsetAsync(Fp, 0, (size_t)blk * 8, h->st));
    launch_adj_scatter((const int32_t*)h->ob[19].p, (const int32_t*)h->ob[20].p,
                       (const double*)h->ob[22].p, B, B, F, h->st);
    launch_adj_scatter((const int32_t*)h->ob[21].p, (const int32_t*)h->ob[23].p,
                       (const double*)h->ob[13].p, (int64_t)pn.size(), B, Fp, h->st);
    for (int l = 1; l <= K; ++l) {
      launch_col_forward64(h->cur_fwd, h->dout.col, wv, h->din.len, F + (l - 1) * blk, F + l * blk,
                           B, n_pad, h->st);
      launch_col_forward64(h->cur_fwd, h->dout.col, wv, h->din.len, Fp + (l - 1) * blk,
                           Fp + l * blk, B, n_pad, h->st);
    }
    CUDA_TRY(h, cudaMemsetAsync(y0, 0, (size_t)blk * 8, h->st));
    double* y = y0;
    double* yn = y1;
    for (int l = K - 1; l >= 0; --l) {
      launch_col_horner64(h->cur_hor, h->din.col, wv, h->din.len, Fp + (l + 1) * blk,
                          std::pow(C, l + 1), y, yn, B, n_pad, 1.0, h->st);
      launch_adj_sddmm(h->cur_hor, h->din.col, F + l * blk, yn, B, 1.0 - C, G, h->st);
      std::swap(y, yn);
    }
    LAUNCH_CHECK(h);
    // the host vectors above must outlive their copies
    CUDA_TRY(h, cudaStreamSynchronize(h->st));
  }
  launch_adj_weights(h->din, wv, n_pad, G, dW, h->st);
  LAUNCH_CHECK(h);
  std::vector<double> dwh((size_t)pool);
  CUDA_TRY(h, cudaMemcpyAsync(dwh.data(), dW, (size_t)pool * 8, cudaMemcpyDeviceToHost, h->st));
  CUDA_TRY(h, cudaStreamSynchronize(h->st));
  // map the caller's edge order to pool positions (rows are as initialised)
  std::vector<int32_t> cnt(n_pad, 0);
  for (size_t e = 0; e < h->init_src.size(); ++e) {
    const int32_t d = h->init_dst[e];
    grad_weight[e] = dwh[(size_t)(h->hin.start[d] + cnt[d]++)];
  }
  return SR_OK;
}

simrank_status simrank_plan_batch(const simrank_update* u, int64_t count, int32_t n_old,
                                  int32_t max_blocks, int32_t* nblocks, int32_t* block_sink,
                                  int32_t* block_op, int64_t* block_off, int32_t* block_src) {
  if (count < 0 || (count > 0 && !u) || !nblocks) return SR_ERR_ARG;
  std::vector<Block> blocks;
  std::string msg;
  simrank_status s = plan_blocks(u, count, n_old, blocks, msg);
  if (s != SR_OK) {
    g_init_error = msg;
    return s;
  }
  *nblocks = (int32_t)blocks.size();
  if ((int32_t)blocks.size() > max_blocks) return SR_ERR_ARG;
  int64_t off = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    block_sink[b] = blocks[b].sink;
    block_op[b] = blocks[b].op;
    block_off[b] = off;
    for (int32_t x : blocks[b].srcs) block_src[off++] = x;
  }
  block_off[blocks.size()] = off;
  return SR_OK;
}

}  // extern "C"

// ===========================================================================
// Many independent graphs (simrank_multi_*).  Each graph is a simrank_ctx of
// its own (S, adjacency, ids, validation and bookkeeping as for one graph);
// the multi handle plans all graphs' updates on the host, uploads one step
// table, and queues per launch l: one prep launch over the steps of l (one
// CTA each) and one S pass over the tile pairs they list.  In the batched
// form launch l is round l (every graph's l-th update); in the per-graph
// form every step is a launch of its own, graph by graph.
// ===========================================================================
struct simrank_multi {
  simrank_config cfg{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::vector<simrank_ctx*> g;
  MultiGraphDesc* d_desc = nullptr;
  MultiStep* d_steps = nullptr;
  int64_t steps_cap = 0;
  int* d_count = nullptr;  // [launch] number of steps
  int* d_ntiles = nullptr; // [launch] tile pairs listed
  int64_t launch_cap = 0;
  uint64_t* d_tiles = nullptr;
  int64_t tiles_cap = 0;
  int32_t* d_srcs = nullptr;
  int64_t srcs_cap = 0;
  PatchOp* d_ops = nullptr;
  int64_t ops_cap = 0;
  int64_t* counters = nullptr;
  // tensor-core S pass (cfg.tc != 0, FP32 S): all graphs' operands in one
  // row-major pair [op_rows][kd], graph g from row row_off[g]
  float* Ahi = nullptr;
  float* Alo = nullptr;
  int64_t op_rows = 0, kd = 0;
  int rg = 0, max_tiles = 0;
  std::vector<int64_t> row_off;
  // host staging of the last call (uploaded, then the stream is synchronised)
  std::vector<MultiGraphDesc> h_desc;
  std::vector<MultiStep> h_steps;
  std::vector<int> h_count;
  std::vector<int32_t> h_srcs;
  std::vector<PatchOp> h_ops;
  // CUDA graph of the last launch sequence, reused while its shape and
  // buffers are unchanged
  cudaGraphExec_t exec = nullptr;
  std::vector<int> exec_count;
  std::vector<const void*> exec_ptrs;
  // stats
  simrank_stats stats{};
  std::vector<std::array<cudaEvent_t, 3>> ev;
  size_t ev_used = 0;
  double prep_ms = 0.0, sup_ms = 0.0;
  int64_t sup_launches = 0, launches = 0;
  std::string err;
};

namespace {

simrank_status mfail(simrank_multi* h, simrank_status s, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_init_error = msg;
  return s;
}

#define MCUDA_TRY(h, call)                                                                 \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess)                                                                \
      return mfail((h), e__ == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA,       \
                   std::string(#call) + ": " + cudaGetErrorString(e__));                   \
  } while (0)

template <typename T>
cudaError_t grow_dev(T** p, int64_t* cap, int64_t need) {
  if (need <= *cap) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = std::max<int64_t>(need, 2 * *cap);
  return dev_alloc(p, (size_t)*cap);
}

void multi_free(simrank_multi* h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  for (void* p : {(void*)h->d_desc, (void*)h->d_steps, (void*)h->d_count, (void*)h->d_ntiles,
                  (void*)h->d_tiles, (void*)h->d_srcs, (void*)h->d_ops, (void*)h->counters,
                  (void*)h->Ahi, (void*)h->Alo})
    if (p) cudaFree(p);
  for (auto& e : h->ev)
    for (cudaEvent_t x : e) cudaEventDestroy(x);
  for (simrank_ctx* c : h->g)
    if (c) {
      cudaStreamSynchronize(c->st);
      free_ctx(c);
    }
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
}

void multi_harvest(simrank_multi* h) {
  for (size_t e = 0; e < h->ev_used; ++e) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, h->ev[e][0], h->ev[e][1]) == cudaSuccess) h->prep_ms += a;
    if (cudaEventElapsedTime(&b, h->ev[e][1], h->ev[e][2]) == cudaSuccess) h->sup_ms += b;
  }
  h->ev_used = 0;
}

// The S pass of launch l: on the tensor cores (operands packed from the
// panels of this launch's graphs) or on the CUDA cores.
void multi_s_pass(simrank_multi* h, int l, int64_t off, int cnt) {
  const int sp = h->cfg.s_precision;
  if (h->Ahi) {
    launch_multi_pack_tc(h->d_desc, h->d_steps + off, h->d_count + l, cnt, h->max_tiles,
                         h->cfg.K + 1, h->rg, h->Ahi, h->Alo, h->kd, h->st);
    const long long lim = h->cfg.timeout_iters > 0 ? h->cfg.timeout_iters : (1ll << 24);
    launch_s_update_tc_multi(h->Ahi, h->Alo, h->op_rows, h->kd, h->d_desc, h->d_tiles,
                             h->d_ntiles + l, h->counters, h->num_sms, lim, h->st, 0,
                             h->cfg.upper_only ? 1 : 0);
  } else {
    launch_s_update_multi(sp, h->d_desc, h->d_tiles, h->d_ntiles + l, h->cfg.K + 1, h->counters,
                          h->num_sms * (sp == 64 ? 1 : 2), h->st);
  }
}

// Queues launch l: the prep of steps [off, off + cnt) and the S pass.
void multi_enqueue(simrank_multi* h, int l, int64_t off, int cnt) {
  const int sp = h->cfg.s_precision;
  launch_multi_prep(sp, h->d_desc, h->d_steps + off, h->d_count + l, cnt, h->d_srcs, h->d_ops,
                    h->cfg.C, h->cfg.K, h->cfg.aff ? 1 : 0, h->d_tiles, h->d_ntiles + l, h->st);
  multi_s_pass(h, l, off, cnt);
}

}  // namespace

extern "C" {

simrank_status simrank_multi_init(const simrank_config* cfg_in, int32_t ngraphs, const int32_t* n,
                                  const int32_t* n_capacity, const int64_t* edge_offsets,
                                  const int32_t* src, const int32_t* dst, simrank_multi_t* out) {
  if (!cfg_in || !out || !n || !edge_offsets) return mfail(nullptr, SR_ERR_ARG, "null argument");
  *out = nullptr;
  if (ngraphs < 1) return mfail(nullptr, SR_ERR_ARG, "ngraphs must be >= 1");
  const simrank_config& cfg = *cfg_in;
  if (cfg.mode != SR_MODE_DENSE || cfg.apply != SR_APPLY_UNIT || cfg.defer > 1 ||
      cfg.s_update != SR_SUPDATE_FUSED)
    return mfail(nullptr, SR_ERR_UNSUPPORTED,
                 "many graphs: dense mode, unit apply, fused S update, defer 0 or 1");
  if (cfg.multi_launch != 0 && cfg.multi_launch != 1)
    return mfail(nullptr, SR_ERR_ARG, "multi_launch must be 0 or 1");
  for (int g = 0; g < ngraphs; ++g) {
    const int cap = n_capacity ? n_capacity[g] : n[g];
    if (n[g] < 1 || cap < n[g] || cap > 65536)
      return mfail(nullptr, SR_ERR_ARG,
                   "graph " + std::to_string(g) + ": need 1 <= n <= n_capacity <= 65536");
    if (edge_offsets[g + 1] < edge_offsets[g])
      return mfail(nullptr, SR_ERR_ARG, "edge_offsets must be non-decreasing");
  }
  simrank_multi* h = new (std::nothrow) simrank_multi();
  if (!h) return mfail(nullptr, SR_ERR_OOM, "host allocation failed");
  h->cfg = cfg;
  h->st = (cudaStream_t)cfg.cuda_stream;
  if (!h->st) {
    // stream capture needs a stream other than the legacy default stream
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return mfail(nullptr, SR_ERR_CUDA, "cudaStreamCreate failed");
    }
    h->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  h->g.assign(ngraphs, nullptr);
  for (int g = 0; g < ngraphs; ++g) {
    simrank_config c = cfg;
    c.n_capacity = n_capacity ? n_capacity[g] : n[g];
    c.cuda_stream = h->st;
    const int64_t e0 = edge_offsets[g], m = edge_offsets[g + 1] - edge_offsets[g];
    simrank_t ctx = nullptr;
    const simrank_status s = simrank_init(&c, n[g], m, src ? src + e0 : nullptr,
                                          dst ? dst + e0 : nullptr, nullptr, nullptr, &ctx);
    if (s != SR_OK) {
      const std::string msg = "graph " + std::to_string(g) + ": " + g_init_error;
      multi_free(h);
      return mfail(nullptr, s, msg);
    }
    h->g[g] = ctx;
  }
  if (dev_alloc(&h->d_desc, (size_t)ngraphs) != cudaSuccess ||
      dev_alloc(&h->counters, (size_t)CNT_N) != cudaSuccess) {
    multi_free(h);
    return mfail(nullptr, SR_ERR_OOM, "cudaMalloc failed");
  }
  h->row_off.resize(ngraphs);
  for (int g = 0; g < ngraphs; ++g) {
    h->row_off[g] = h->op_rows;
    h->op_rows += h->g[g]->n_pad;
    h->max_tiles = std::max(h->max_tiles, h->g[g]->n_pad / PT);
  }
  if (cfg.tc && cfg.s_precision == 32) {
    h->rg = (cfg.K + 1 + 31) / 32 * 32;
    h->kd = 2 * (int64_t)h->rg;
    if (h->op_rows >= ((int64_t)1 << 31) ||
        dev_alloc(&h->Ahi, (size_t)(h->op_rows * h->kd)) != cudaSuccess ||
        dev_alloc(&h->Alo, (size_t)(h->op_rows * h->kd)) != cudaSuccess) {
      multi_free(h);
      return mfail(nullptr, SR_ERR_OOM, "tensor-core operand allocation failed");
    }
  }
  cudaMemsetAsync(h->counters, 0, CNT_N * sizeof(int64_t), h->st);
  h->h_desc.resize(ngraphs);
  if (cudaStreamSynchronize(h->st) != cudaSuccess) {
    multi_free(h);
    return mfail(nullptr, SR_ERR_CUDA, "initialisation failed on the GPU");
  }
  *out = h;
  return SR_OK;
}

simrank_status simrank_multi_apply(simrank_multi_t h, const simrank_update* u,
                                   const int64_t* update_offsets) {
  if (!h) return mfail(nullptr, SR_ERR_ARG, "null handle");
  if (!update_offsets) return mfail(h, SR_ERR_ARG, "null update_offsets");
  const int G = (int)h->g.size();
  // caller ids -> storage ids, then validation of every graph before any change
  std::vector<std::vector<simrank_update>> um(G);
  std::vector<int> n_after(G);
  int64_t total = 0;
  int R = 0;
  for (int g = 0; g < G; ++g) {
    const int64_t c = update_offsets[g + 1] - update_offsets[g];
    if (c < 0) return mfail(h, SR_ERR_ARG, "update_offsets must be non-decreasing");
    if (c > 0 && !u) return mfail(h, SR_ERR_ARG, "null update array");
    simrank_ctx* x = h->g[g];
    um[g].assign(u + update_offsets[g], u + update_offsets[g] + c);
    if (x->relabeled)
      for (auto& v : um[g]) {
        if (v.src >= 0 && v.src < x->n_cap) v.src = x->ext2int[v.src];
        if (v.dst >= 0 && v.dst < x->n_cap) v.dst = x->ext2int[v.dst];
      }
    n_after[g] = x->n_cur;
    const simrank_status s = validate(x, um[g].data(), c, &n_after[g]);
    if (s != SR_OK) return mfail(h, s, "graph " + std::to_string(g) + ": " + x->err);
    total += c;
    R = std::max<int>(R, (int)c);
  }
  if (total == 0) return SR_OK;
  // plan: per graph its steps, in order (host mirrors and patch ops)
  h->h_srcs.clear();
  h->h_ops.clear();
  std::vector<std::vector<MultiStep>> per(G);
  for (int g = 0; g < G; ++g) {
    simrank_ctx* x = h->g[g];
    int n_run = x->n_cur;
    for (const simrank_update& v : um[g]) {
      const int32_t i = v.src, j = v.dst;
      n_run = std::max(n_run, std::max(i, j) + 1);
      MultiStep s{};
      s.g = g;
      s.j = j;
      s.op = v.op;
      s.d_j = x->hin.len[j];
      s.delta = 1;
      s.src_off = (int64_t)h->h_srcs.size();
      h->h_srcs.push_back(i);
      s.op_begin = (int64_t)h->h_ops.size();
      if (v.op > 0) {
        adj_append(x->hin, j, i, h->h_ops, true);
        adj_append(x->hout, i, j, h->h_ops, false);
        x->edges.insert(ekey(i, j));
      } else {
        adj_remove(x->hin, j, i, h->h_ops, true);
        adj_remove(x->hout, i, j, h->h_ops, false);
        x->edges.erase(ekey(i, j));
      }
      s.op_end = (int64_t)h->h_ops.size();
      s.n_after = n_run;
      per[g].push_back(s);
    }
    x->n_cur = n_after[g];
    simrank_status s;
    if ((s = grow_pool(x, x->din, x->hin)) != SR_OK || (s = grow_pool(x, x->dout, x->hout)) != SR_OK)
      return mfail(h, s, "graph " + std::to_string(g) + ": " + x->err);
    x->stats.updates += (int64_t)um[g].size();
    x->stats.rank_one_updates += (int64_t)um[g].size();
    MultiGraphDesc& d = h->h_desc[g];
    d.S = x->S;
    d.ld = x->ld;
    d.P = x->cfg.s_precision == 64 ? (void*)x->P64 : (void*)x->P32;
    d.mXi = x->mXi;
    d.mEta = x->mEta;
    d.in = x->din;
    d.out = x->dout;
    d.sI = x->sI;
    d.sJ = x->sJ;
    d.n = x->n_cur;
    d.upper = upper(x);
    d.row_off = h->row_off[g];
  }
  // launch table
  h->h_steps.clear();
  h->h_count.clear();
  std::vector<int64_t> loff;
  int64_t tiles_need = 0;
  auto pairs = [](int n_after) {
    const int64_t nT = (n_after + PT - 1) / PT;
    return nT * (nT + 1) / 2;
  };
  if (h->cfg.multi_launch == 0) {
    for (int r = 0; r < R; ++r) {
      loff.push_back((int64_t)h->h_steps.size());
      int64_t tp = 0;
      for (int g = 0; g < G; ++g)
        if ((int)per[g].size() > r) {
          h->h_steps.push_back(per[g][r]);
          tp += pairs(per[g][r].n_after);
        }
      h->h_count.push_back((int)(h->h_steps.size() - loff.back()));
      tiles_need = std::max(tiles_need, tp);
    }
  } else {
    for (int g = 0; g < G; ++g)
      for (const MultiStep& s : per[g]) {
        loff.push_back((int64_t)h->h_steps.size());
        h->h_steps.push_back(s);
        h->h_count.push_back(1);
        tiles_need = std::max(tiles_need, pairs(s.n_after));
      }
  }
  const int L = (int)h->h_count.size();
  MCUDA_TRY(h, grow_dev(&h->d_steps, &h->steps_cap, (int64_t)h->h_steps.size()));
  if (L > h->launch_cap) {
    if (h->d_count) cudaFree(h->d_count);
    if (h->d_ntiles) cudaFree(h->d_ntiles);
    h->d_count = nullptr;
    h->d_ntiles = nullptr;
    h->launch_cap = std::max<int64_t>(L, 2 * h->launch_cap);
    MCUDA_TRY(h, dev_alloc(&h->d_count, (size_t)h->launch_cap));
    MCUDA_TRY(h, dev_alloc(&h->d_ntiles, (size_t)h->launch_cap));
  }
  MCUDA_TRY(h, grow_dev(&h->d_tiles, &h->tiles_cap, tiles_need));
  MCUDA_TRY(h, grow_dev(&h->d_srcs, &h->srcs_cap, (int64_t)h->h_srcs.size()));
  MCUDA_TRY(h, grow_dev(&h->d_ops, &h->ops_cap, (int64_t)h->h_ops.size()));
  MCUDA_TRY(h, cudaMemcpyAsync(h->d_desc, h->h_desc.data(), G * sizeof(MultiGraphDesc),
                               cudaMemcpyHostToDevice, h->st));
  MCUDA_TRY(h, cudaMemcpyAsync(h->d_steps, h->h_steps.data(), h->h_steps.size() * sizeof(MultiStep),
                               cudaMemcpyHostToDevice, h->st));
  MCUDA_TRY(h, cudaMemcpyAsync(h->d_count, h->h_count.data(), L * sizeof(int),
                               cudaMemcpyHostToDevice, h->st));
  MCUDA_TRY(h, cudaMemcpyAsync(h->d_srcs, h->h_srcs.data(), h->h_srcs.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, h->st));
  if (!h->h_ops.empty())
    MCUDA_TRY(h, cudaMemcpyAsync(h->d_ops, h->h_ops.data(), h->h_ops.size() * sizeof(PatchOp),
                                 cudaMemcpyHostToDevice, h->st));
  // the staging vectors may change once the copies are done
  MCUDA_TRY(h, cudaStreamSynchronize(h->st));

  if (h->cfg.profile) {
    multi_harvest(h);
    MCUDA_TRY(h, cudaMemsetAsync(h->d_ntiles, 0, L * sizeof(int), h->st));
    for (int l = 0; l < L; ++l) {
      if (h->ev_used == h->ev.size()) {
        std::array<cudaEvent_t, 3> a{};
        for (auto& x : a) MCUDA_TRY(h, cudaEventCreate(&x));
        h->ev.push_back(a);
      }
      auto& e = h->ev[h->ev_used++];
      const int sp = h->cfg.s_precision;
      MCUDA_TRY(h, cudaEventRecord(e[0], h->st));
      launch_multi_prep(sp, h->d_desc, h->d_steps + loff[l], h->d_count + l, h->h_count[l],
                        h->d_srcs, h->d_ops, h->cfg.C, h->cfg.K, h->cfg.aff ? 1 : 0, h->d_tiles,
                        h->d_ntiles + l, h->st);
      MCUDA_TRY(h, cudaEventRecord(e[1], h->st));
      multi_s_pass(h, l, loff[l], h->h_count[l]);
      MCUDA_TRY(h, cudaEventRecord(e[2], h->st));
    }
  } else {
    const std::vector<const void*> ptrs = {h->d_desc, h->d_steps, h->d_count, h->d_ntiles,
                                           h->d_tiles, h->d_srcs, h->d_ops, h->counters};
    if (!h->exec || h->exec_count != h->h_count || h->exec_ptrs != ptrs) {
      if (h->exec) cudaGraphExecDestroy(h->exec);
      h->exec = nullptr;
      cudaGraph_t graph = nullptr;
      MCUDA_TRY(h, cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
      cudaMemsetAsync(h->d_ntiles, 0, L * sizeof(int), h->st);
      for (int l = 0; l < L; ++l) multi_enqueue(h, l, loff[l], h->h_count[l]);
      const cudaError_t ce = cudaStreamEndCapture(h->st, &graph);
      if (ce != cudaSuccess) return mfail(h, SR_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(ce));
      const cudaError_t ie = cudaGraphInstantiate(&h->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) {
        h->exec = nullptr;
        return mfail(h, SR_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
      }
      h->exec_count = h->h_count;
      h->exec_ptrs = ptrs;
    }
    MCUDA_TRY(h, cudaGraphLaunch(h->exec, h->st));
  }
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return mfail(h, SR_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(le));
  h->launches += 2 * (int64_t)L;
  h->sup_launches += L;
  h->stats.updates += total;
  h->stats.rank_one_updates += total;
  return SR_OK;
}

simrank_status simrank_multi_columns(simrank_multi_t h, int32_t g, const int32_t* cols,
                                     int32_t ncols, void* out, int32_t out_on_device,
                                     int32_t out_fp64) {
  if (!h) return mfail(nullptr, SR_ERR_ARG, "null handle");
  if (g < 0 || g >= (int)h->g.size()) return mfail(h, SR_ERR_ARG, "graph index out of range");
  const simrank_status s = simrank_columns(h->g[g], cols, ncols, out, out_on_device, out_fp64);
  if (s != SR_OK) return mfail(h, s, "graph " + std::to_string(g) + ": " + h->g[g]->err);
  return SR_OK;
}

int32_t simrank_multi_num_graphs(simrank_multi_t h) { return h ? (int32_t)h->g.size() : -1; }

int32_t simrank_multi_num_nodes(simrank_multi_t h, int32_t g) {
  if (!h || g < 0 || g >= (int)h->g.size()) return -1;
  return h->g[g]->n_cur;
}

simrank_status simrank_multi_sync(simrank_multi_t h) {
  if (!h) return mfail(nullptr, SR_ERR_ARG, "null handle");
  MCUDA_TRY(h, cudaStreamSynchronize(h->st));
  int64_t status = 0;
  MCUDA_TRY(h, cudaMemcpy(&status, h->counters + CNT_STATUS, sizeof(status), cudaMemcpyDeviceToHost));
  if (status != 0) return mfail(h, (simrank_status)status, "a bounded device wait ran out");
  return SR_OK;
}

simrank_status simrank_multi_get_stats(simrank_multi_t h, simrank_stats* out) {
  if (!h || !out) return mfail(h, SR_ERR_ARG, "null argument");
  MCUDA_TRY(h, cudaStreamSynchronize(h->st));
  multi_harvest(h);
  int64_t c[CNT_N];
  MCUDA_TRY(h, cudaMemcpy(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost));
  simrank_stats r = h->stats;
  r.tiles_touched = c[CNT_TILES_TOUCHED];
  r.s_bytes = c[CNT_S_BYTES];
  r.panel_bytes = c[CNT_PANEL_BYTES];
  r.kernel_launches = h->launches;
  r.s_update_launches = h->sup_launches;
  r.s_update_ms = h->sup_ms;
  r.phase_ms[0] = h->prep_ms;
  r.phase_ms[3] = h->sup_ms;
  *out = r;
  return SR_OK;
}

const char* simrank_multi_last_error(simrank_multi_t h) {
  return h ? h->err.c_str() : g_init_error.c_str();
}

void simrank_multi_destroy(simrank_multi_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  multi_free(h);
}

}  // extern "C"
