// tc_count_static: the exact count (same kernels as tc_count) for callers
// that cannot allocate device memory.
//
// Why some callers cannot allocate: a process whose device memory is owned by
// another allocator (a framework's caching allocator that has reserved the
// device, so an extra cudaMalloc fails or fragments its pool); a latency-
// critical path where cudaMalloc/cudaFree would synchronize the device and
// stall other streams; code that must stay within a memory budget declared
// up front.  tc_count needs a caller workspace and tc_ctx_create allocates;
// this entry point needs neither.
//
// Its scratch (the queue of long lists and the work cursors of the counting
// kernels) is the file-scope array below, TC_STATIC_MAX_N 4-byte slots plus
// 256 bytes (about 4 MiB).  Every GPU that loads libtc holds one copy of it
// until the process exits.  All calls on a device share that copy: calls that
// overlap on the GPU (on different streams, or from different host threads
// without ordering) race on it and their results are undefined.
#include <mutex>

#include "tc_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kCounterBytes = 256;

// counters (first kCounterBytes) followed by the queue of long lists
static __device__ __align__(256) unsigned char g_tc_static_scratch[kCounterBytes + sizeof(int32_t) * TC_STATIC_MAX_N];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};

// Once per device, with that device current: the device address of the scratch.
cudaError_t setup(int dev, void** addr, int* sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tc_static_scratch);
    if (e != cudaSuccess) return e;
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_sm_count[dev] = v > 0 ? v : 1;
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" tc_status tc_count_static(const tc_graph* g, uint64_t* total_dev, uint32_t* check_dev, tc_stream stream) {
  if (!g || !total_dev || !check_dev) return TC_ERR_INVALID_ARG;
  if (g->n < 0 || g->m < 0 || !g->offsets || (g->m > 0 && !g->cols)) return TC_ERR_INVALID_ARG;
  if (g->n > TC_STATIC_MAX_N) return TC_ERR_UNSUPPORTED;
  // the kernels read offsets as 8-byte words, add into *total_dev with a 64-bit
  // atomic and set bits of *check_dev with a 32-bit one: a misaligned pointer
  // would fault on the device, so it is refused here with nothing enqueued
  auto misaligned = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) != 0; };
  if (misaligned(g->offsets, 8) || misaligned(total_dev, 8) || misaligned(check_dev, 4) ||
      (g->cols && misaligned(g->cols, 4)))
    return TC_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TC_ERR_CUDA;
  void* scratch = nullptr;
  int sms = 0;
  if (setup(dev, &scratch, &sms) != cudaSuccess) return TC_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a context on the stack: no profiler, no allocation; device checks land in *check_dev
  tc::Ctx ctx;
  ctx.device = dev;
  ctx.sm_count = sms;
  ctx.d_err = check_dev;
  tc::CountWs w{};
  w.counters = static_cast<uint32_t*>(scratch);
  w.big_queue = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(scratch) + kCounterBytes);
  if (cudaMemsetAsync(check_dev, 0, sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s) != cudaSuccess)
    return TC_ERR_CUDA;
  tc::CountArgs a{g->n, g->m, g->offsets, g->cols, reinterpret_cast<unsigned long long*>(total_dev), nullptr,
                  nullptr, 0};
  // launch_count clears the counters at the head of the scratch before the kernels
  return tc::launch_count(&ctx, tc::MODE_COUNT, a, w, s) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
