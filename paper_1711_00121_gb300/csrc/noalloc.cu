// simrank_update_noalloc: one edge update of a caller-owned S and graph that
// allocates nothing.  Its scratch (panels, masks, tile list, gathered rows)
// lives in one fixed-size __device__ array of this library; the per-edge
// kernels are the ones simrank_apply_updates uses.  The paper has no
// counterpart: this entry point exists for callers that cannot allocate
// device memory (see include/simrank.h).
#include <mutex>

#include "sr_internal.h"

namespace sr {

namespace {

// Limits of the fixed scratch array.
constexpr int NA_MAX_N = 8192;           // nodes
constexpr int NA_MAX_K1 = 32;            // K + 1 terms
constexpr int NA_NT = NA_MAX_N / PT;     // 64 tiles
constexpr size_t NA_P64 = (size_t)NA_NT * 2 * NA_MAX_K1 * PT;  // doubles of the FP64 panels
constexpr size_t NA_TILES = (size_t)NA_NT * (NA_NT + 1) / 2;

// Byte offsets of the regions inside the array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_P64 = 0;
constexpr size_t OFF_P32 = align256(OFF_P64 + NA_P64 * 8);
constexpr size_t OFF_SI = align256(OFF_P32 + NA_P64 * 4);
constexpr size_t OFF_SJ = align256(OFF_SI + (size_t)NA_MAX_N * 8);
constexpr size_t OFF_SCAL = align256(OFF_SJ + (size_t)NA_MAX_N * 8);
constexpr size_t OFF_MXI = align256(OFF_SCAL + 8 * 8);
constexpr size_t OFF_META = align256(OFF_MXI + (size_t)NA_NT * 8);
constexpr size_t OFF_TILES = align256(OFF_META + (size_t)NA_NT * 8);
constexpr size_t OFF_NTILES = align256(OFF_TILES + NA_TILES * 4);
constexpr size_t OFF_CNT = align256(OFF_NTILES + 4);
constexpr size_t OFF_LEN_OLD = align256(OFF_CNT + (size_t)CNT_N * 8);
constexpr size_t OFF_LEN_NEW = align256(OFF_LEN_OLD + (size_t)NA_MAX_N * 4);
constexpr size_t OFF_SRC = align256(OFF_LEN_NEW + (size_t)NA_MAX_N * 4);
constexpr size_t NA_BYTES = align256(OFF_SRC + 4);

// The scratch array: every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// len[a] = row_ptr[a + 1] - row_ptr[a] for a < n, 0 for n <= a < n_pad;
// the source list holds the one source i.
__global__ void k_na_lengths(const int64_t* __restrict__ old_rp, const int64_t* __restrict__ new_rp,
                             int n, int n_pad, int32_t* __restrict__ len_old,
                             int32_t* __restrict__ len_new, int32_t* __restrict__ src, int i) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n_pad) {
    len_old[a] = a < n ? (int32_t)(old_rp[a + 1] - old_rp[a]) : 0;
    len_new[a] = a < n ? (int32_t)(new_rp[a + 1] - new_rp[a]) : 0;
  }
  if (a == 0) src[0] = i;
}

// Device address of the array, looked up once per device.
constexpr int NA_MAX_DEV = 64;
unsigned char* g_addr[NA_MAX_DEV] = {};
std::mutex g_addr_mu;

cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

simrank_status na_fail(simrank_status s, const std::string& m) {
  set_global_error(m);
  return s;
}

}  // namespace

}  // namespace sr

using namespace sr;

extern "C" simrank_status simrank_update_noalloc(int32_t n, int64_t ld, void* S, int32_t s_precision,
                                                 const int64_t* old_row_ptr, const int32_t* old_col,
                                                 const int64_t* new_row_ptr, const int32_t* new_col,
                                                 int32_t i, int32_t j, int32_t op, int32_t d_j,
                                                 double C, int32_t K, void* cuda_stream) {
  if (n < 1 || n > NA_MAX_N)
    return na_fail(SR_ERR_ARG, "n must be in [1, " + std::to_string(NA_MAX_N) + "]");
  if (K < 0 || K + 1 > NA_MAX_K1)
    return na_fail(SR_ERR_ARG, "K must be in [0, " + std::to_string(NA_MAX_K1 - 1) + "]");
  if (s_precision != 32 && s_precision != 64) return na_fail(SR_ERR_ARG, "s_precision must be 32 or 64");
  if (!(C > 0.0 && C < 1.0)) return na_fail(SR_ERR_ARG, "C must be in (0, 1)");
  const int n_pad = (n + PT - 1) / PT * PT;
  if (ld < n_pad || ld % PT != 0)
    return na_fail(SR_ERR_ARG, "ld must be a multiple of 128 and at least n rounded up to 128");
  if (!S || !old_row_ptr || !new_row_ptr) return na_fail(SR_ERR_ARG, "null pointer");
  if (i < 0 || j < 0 || i >= n || j >= n || i == j) return na_fail(SR_ERR_ARG, "bad edge");
  if (op != 1 && op != -1) return na_fail(SR_ERR_ARG, "op must be +1 or -1");
  if (d_j < 0 || (op < 0 && d_j < 1)) return na_fail(SR_ERR_ARG, "bad in-degree d_j");
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess)
    return na_fail(SR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nT = n_pad / PT;
  const int K1 = K + 1;
  double* P64 = (double*)(base + OFF_P64);
  float* P32 = s_precision == 32 ? (float*)(base + OFF_P32) : nullptr;
  double* sI = (double*)(base + OFF_SI);
  double* sJ = (double*)(base + OFF_SJ);
  double* scal = (double*)(base + OFF_SCAL);
  uint64_t* mXi = (uint64_t*)(base + OFF_MXI);
  uint64_t* mEta = (uint64_t*)(base + OFF_META);
  uint32_t* tiles = (uint32_t*)(base + OFF_TILES);
  int* ntiles = (int*)(base + OFF_NTILES);
  int64_t* counters = (int64_t*)(base + OFF_CNT);
  int32_t* len_old = (int32_t*)(base + OFF_LEN_OLD);
  int32_t* len_new = (int32_t*)(base + OFF_LEN_NEW);
  int32_t* src = (int32_t*)(base + OFF_SRC);
  DevAdj gin_old, gin_new;
  gin_old.start = const_cast<int64_t*>(old_row_ptr);
  gin_old.len = len_old;
  gin_old.col = const_cast<int32_t*>(old_col);
  gin_new.start = const_cast<int64_t*>(new_row_ptr);
  gin_new.len = len_new;
  gin_new.col = const_cast<int32_t*>(new_col);

  // state left by an earlier call that must start at zero
  e = cudaMemsetAsync(counters, 0, CNT_N * sizeof(int64_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ntiles, 0, sizeof(int), st);
  if (e != cudaSuccess) return na_fail(SR_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  k_na_lengths<<<(n_pad + 255) / 256, 256, 0, st>>>(old_row_ptr, new_row_ptr, n, n_pad, len_old,
                                                    len_new, src, i);
  launch_gather_rows(S, s_precision, ld, src, 1, j, n_pad, gin_old, sI, sJ, scal, st);
  launch_gamma(gin_old, sI, sJ, scal, j, 1, op, d_j, C, nT, K1, P64, P32, mXi, mEta, st);
  for (int k = 0; k < K; ++k) launch_chain_step(gin_new, k, C, nT, K1, P64, P32, mXi, mEta, st);
  launch_tile_list(mXi, mEta, nT, 1, tiles, ntiles, st);
  int num_sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  launch_s_update(S, s_precision, ld, s_precision == 64 ? (void*)P64 : (void*)P32, K1, tiles, ntiles,
                  mXi, mEta, 0, K1, 1, n, counters, s_update_grid(s_precision, num_sms), st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(SR_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return SR_OK;
}
