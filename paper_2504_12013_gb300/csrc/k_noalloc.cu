// Block weights c(V_i) without any device allocation.
//
// Some callers cannot allocate device memory at all: applications that hand
// the whole device to their own memory pool up front, so that any foreign
// cudaMalloc fails or fragments their budget, and latency-critical loops in
// which a cudaMalloc/cudaFree pair is ruled out because it can stall the
// device for much longer than the work itself.  They also cannot create a
// jet_ctx, whose workspace is allocated.  jet_block_weights_noalloc serves
// them: it is the block-weight pass of jet_build_pincounts with its scratch
// (per-block vertex counts and a data-error flag) held in a file-scope device
// array instead of context workspace.
//
// The array is a fixed 1.25 KiB per GPU that loads the library and stays
// resident until the process exits.  All calls share it, so two calls that
// overlap on the GPU (different streams, or different host threads on the
// same device) race on it; each call clears it before use.
#include <mutex>

#include "jet_internal.cuh"

namespace {

constexpr int kNoAllocMaxK = 256;                   // largest k the static scratch holds
constexpr int kScratchInts = kNoAllocMaxK + 64;     // counts[256], error flag at [256], padding
constexpr int kErrSlot = kNoAllocMaxK;
constexpr int kErrBadPart = 1;    // error-slot bit: a partition value outside [0, k)
constexpr int kErrBadWeight = 2;  // error-slot bit: a vertex weight below 1
constexpr int kMaxDevices = 64;

static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

std::mutex g_setup_mu;
int32_t *g_scratch_addr[kMaxDevices] = {nullptr};  // device address of the array, per device

// The block-weight kernel of k_state.cu, with its counts and error flag in `scratch`.
__global__ void k_block_weights_static(const int32_t *part, const int32_t *vwgt, int32_t n, int32_t k,
                                       int64_t *bw, int32_t *scratch) {
  __shared__ long long s_bw[kNoAllocMaxK];
  __shared__ int s_cnt[kNoAllocMaxK];
  for (int b = threadIdx.x; b < k; b += blockDim.x) { s_bw[b] = 0; s_cnt[b] = 0; }
  __syncthreads();
  int err = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int b = part[v];
    const int32_t c = vwgt[v];
    if (c < 1) {
      err |= kErrBadWeight;  // c(v) >= 1 is required, as jet_ctx_create requires it
    } else if ((unsigned)b < (unsigned)k) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&s_bw[b]), (unsigned long long)c);
      atomicAdd(&s_cnt[b], 1);
    } else {
      err |= kErrBadPart;
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < k; b += blockDim.x) {
    if (s_bw[b]) atomicAdd(reinterpret_cast<unsigned long long *>(&bw[b]), (unsigned long long)s_bw[b]);
    if (s_cnt[b]) atomicAdd(&scratch[b], s_cnt[b]);
  }
  if (err) atomicOr(&scratch[kErrSlot], err);
}

// Device address of the scratch array for the current device, looked up once
// per device with that device current.
int scratch_for_current_device(int32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    jet::set_global_error("jet_block_weights_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return JET_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    jet::set_global_error("jet_block_weights_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return JET_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      jet::set_global_error("jet_block_weights_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return JET_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<int32_t *>(p);
  }
  *out = g_scratch_addr[dev];
  return JET_OK;
}

}  // namespace

extern "C" int jet_block_weights_noalloc(const int32_t *part, const int32_t *vwgt, int32_t n, int32_t k,
                                         int64_t *block_w, int32_t *block_count, void *stream) {
  if (k < 2 || k > kNoAllocMaxK) {
    jet::set_global_error("jet_block_weights_noalloc: k = %d is outside [2, %d], the size of its static scratch",
                          k, kNoAllocMaxK);
    return JET_ERR_INVALID_ARG;
  }
  if (n < 0 || !block_w || (n > 0 && (!part || !vwgt))) {
    jet::set_global_error("jet_block_weights_noalloc: negative n or a NULL array");
    return JET_ERR_INVALID_ARG;
  }
  int32_t *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != JET_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int32_t) * kScratchInts, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(block_w, 0, sizeof(int64_t) * k, s);
  if (e == cudaSuccess && n > 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_block_weights_static<<<jet::grid_for(n, 256, sms > 0 ? sms : 1, 2), 256, 0, s>>>(part, vwgt, n, k, block_w,
                                                                                    scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && block_count)
    e = cudaMemcpyAsync(block_count, scratch, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, s);
  int32_t flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, scratch + kErrSlot, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    jet::set_global_error("jet_block_weights_noalloc: %s", cudaGetErrorString(e));
    return JET_ERR_CUDA;
  }
  if (flag & kErrBadWeight) {
    jet::set_global_error("jet_block_weights_noalloc: a vertex weight c(v) is below 1");
    return JET_ERR_DATA;
  }
  if (flag) {
    jet::set_global_error("jet_block_weights_noalloc: a partition value is outside [0, %d)", k);
    return JET_ERR_DATA;
  }
  return JET_OK;
}
