// knn_search_noalloc: the exact k-nearest-neighbour search of knn_search for
// callers that must not allocate device memory (see include/lnbnn.h).
//
// Every intermediate lives in one file-scope device array of fixed size.  On
// the host, the array's name denotes a host-side stand-in object, not device
// memory: host code never passes it to a kernel.  Instead, once per device and
// with that device current, its device address is looked up with
// cudaGetSymbolAddress and that address is carved into the buffers the
// existing kernels take.  Nothing here calls cudaMalloc, cudaFree or any other
// allocating routine.
#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "knn_tc.cuh"

namespace {

using namespace lnbnn;

// The fixed scratch: LNBNN_NOALLOC_SCRATCH_BYTES, reserved on a device once
// the library's device code is loaded there, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LNBNN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on the
// first call for that device (the kernels' attributes are set then too).  The
// set-up belongs to the device's primary context: after cudaDeviceReset the
// cached address is stale, and the entry point must not be used again in
// that process.
lnbnn_status scratch_on_current_device(void** addr, int* sm_count) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LNBNN_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
      cudaGetLastError();
      return LNBNN_ERR_CUDA;
    }
    if (prop.major != 10 || prop.minor != 3) return LNBNN_ERR_UNSUPPORTED;
    if (prepare_tc_kernels() != cudaSuccess) {
      cudaGetLastError();
      return LNBNN_ERR_CUDA;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LNBNN_ERR_CUDA;
    }
    g_sm_count[dev] = prop.multiProcessorCount;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *sm_count = g_sm_count[dev];
  return LNBNN_OK;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Rows of the larger operand copy (BF16, 256 bytes a row) the scratch could
// hold at all: a bound applied before any size arithmetic, so no product
// below can overflow.
constexpr int64_t kMaxRows = (int64_t)(LNBNN_NOALLOC_SCRATCH_BYTES / (kDim * 2));

// True when p is device (or managed) memory that the current device can use.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

struct Layout {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) & ~size_t(255);
    const size_t at = off;
    off += count * sizeof(T);
    return at;
  }
};

}  // namespace

extern "C" LNBNN_API lnbnn_status knn_search_noalloc(const uint8_t* ref, int64_t n_ref, const uint8_t* queries,
                                                     int64_t n_queries, int32_t k, int32_t* idx, int32_t* dist,
                                                     void* stream) {
  if (!ref || n_ref < 1 || n_queries < 0) return LNBNN_ERR_INVALID_ARG;
  if (k < 1 || k > LNBNN_MAX_K || (int64_t)k > n_ref) return LNBNN_ERR_K_RANGE;
  if (n_queries == 0) return LNBNN_OK;
  if (!queries || !idx || !dist) return LNBNN_ERR_INVALID_ARG;
  if (n_ref > kMaxRows || n_queries > kMaxRows) return LNBNN_ERR_SCRATCH_LIMIT;
  void* base = nullptr;
  int sm_count = 0;
  lnbnn_status st = scratch_on_current_device(&base, &sm_count);
  if (st != LNBNN_OK) return st;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LNBNN_ERR_CUDA;
  }
  // every array must be memory the current device reaches (not host memory,
  // not another device's)
  if (!on_device(ref, dev) || !on_device(queries, dev) || !on_device(idx, dev) || !on_device(dist, dev))
    return LNBNN_ERR_INVALID_ARG;

  // The index path's split schedule with the default model, at most 32
  // splits (which bounds the scratch the lists take).
  const int64_t n_pad = round_up(n_ref, kRefPad);
  const int64_t m_pad = round_up(n_queries, kQueryPad);
  int64_t splits = choose_splits_model(SplitModel{}, m_pad / kTcQueryTile, n_ref, sm_count, 32);
  const int64_t split_len = round_up((n_ref + splits - 1) / splits, kTcRefTile);
  splits = (n_ref + split_len - 1) / split_len;

  Layout L;
  const size_t o_err = L.take<uint32_t>(1);
  const size_t o_rbf = L.take<__nv_bfloat16>((size_t)n_pad * kDim);
  const size_t o_rext = L.take<__nv_bfloat16>((size_t)n_pad * kExt);
  const size_t o_rn = L.take<float>((size_t)n_pad);
  const size_t o_qn = L.take<int32_t>((size_t)m_pad);
  const size_t o_qbf = L.take<__nv_bfloat16>((size_t)m_pad * kDim);
  const size_t o_qext = L.take<__nv_bfloat16>((size_t)m_pad * kExt);
  const int64_t n_lists = splits * tc_lists_per_split(k);
  const size_t o_lists = L.take<uint64_t>((size_t)n_lists * m_pad * k);
  const size_t o_merged = n_lists > 1 ? L.take<uint64_t>((size_t)m_pad * k) : o_lists;
  const size_t o_rowthr = L.take<int32_t>((size_t)m_pad);  // the bound the lists of a row share
  if (L.off > (size_t)LNBNN_NOALLOC_SCRATCH_BYTES) return LNBNN_ERR_SCRATCH_LIMIT;

  char* b = static_cast<char*>(base);
  uint32_t* err = reinterpret_cast<uint32_t*>(b + o_err);
  __nv_bfloat16* ref_bf = reinterpret_cast<__nv_bfloat16*>(b + o_rbf);
  __nv_bfloat16* ref_ext = reinterpret_cast<__nv_bfloat16*>(b + o_rext);
  float* rnorm = reinterpret_cast<float*>(b + o_rn);
  int32_t* qnorm = reinterpret_cast<int32_t*>(b + o_qn);
  __nv_bfloat16* qbf = reinterpret_cast<__nv_bfloat16*>(b + o_qbf);
  __nv_bfloat16* qext = reinterpret_cast<__nv_bfloat16*>(b + o_qext);
  uint64_t* lists = reinterpret_cast<uint64_t*>(b + o_lists);
  uint64_t* merged = reinterpret_cast<uint64_t*>(b + o_merged);
  int32_t* row_thr = reinterpret_cast<int32_t*>(b + o_rowthr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  TcTensorMaps maps;
  if (!make_tc_tensor_maps(ref_bf, ref_bf, ref_ext, ref_ext, n_pad, &maps)) return LNBNN_ERR_CUDA;
  // The array keeps the previous call's contents: the error word must start at
  // zero and the rows' shared bounds above every distance; every other buffer
  // is fully written before it is read.
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess && splits > 1) e = cudaMemsetAsync(row_thr, 0x7F, sizeof(int32_t) * (size_t)m_pad, s);
  if (e == cudaSuccess) e = launch_prep_ref(ref, n_ref, n_pad, kDim, 0, ref_bf, rnorm, ref_ext, s);
  if (e == cudaSuccess) e = launch_prep_query(queries, n_queries, m_pad, kDim, 0, qnorm, qbf, qext, s);
  if (e == cudaSuccess)
    e = launch_knn_tc(maps, false, qbf, qext, n_queries, m_pad, n_ref, (int)splits, split_len, k, lists, m_pad,
                      splits > 1 ? row_thr : nullptr, err, nullptr, nullptr, TcSched{}, s);
  if (e == cudaSuccess && n_lists > 1) e = launch_merge_lists(lists, (int)n_lists, n_queries, m_pad, k, merged, s);
  if (e == cudaSuccess) e = launch_extract_knn(merged, n_queries, k, k, idx, dist, s);
  uint32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LNBNN_ERR_CUDA;
  }
  return (herr & kDevErrTimeout) ? LNBNN_ERR_TIMEOUT : LNBNN_OK;
}
