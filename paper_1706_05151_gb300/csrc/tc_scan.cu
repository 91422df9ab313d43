// Device-wide exclusive prefix sum: out[i] = in[0] + ... + in[i-1], out[n] = total
// (n the host length, or the smaller length found at *n_dev when the stream reaches the scan).
// Used for CSR offsets (Figure 2 preprocessing builds N_v contiguously) and for
// the listing and sparsification output positions.  Three stream-ordered
// launches: per-tile sums, one block scanning the tile sums, per-tile rescan.
#include "tc_internal.cuh"

namespace tc {

namespace {

template <class T>
__device__ __forceinline__ int64_t load_or_zero(const T* in, int64_t i, int64_t n) {
  return i < n ? static_cast<int64_t>(in[i]) : 0;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ int64_t block_exclusive(int64_t x, int64_t* warp_sums, int64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t t = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < nw ? warp_sums[lane] : 0;
    int64_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t t = __shfl_up_sync(FULL, wi, d);
      if (lane >= d) wi += t;
    }
    if (lane < nw) warp_sums[lane] = wi - w;
    if (lane == nw - 1) *total = wi;
  }
  __syncthreads();
  int64_t r = warp_sums[wid] + incl - x;
  __syncthreads();
  return r;
}

// Scan length: the host bound n, or the smaller length a kernel earlier in the stream left at *n_dev.
__device__ __forceinline__ int64_t scan_len(int64_t n, const uint32_t* n_dev) {
  return n_dev ? min64(n, static_cast<int64_t>(*n_dev)) : n;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const T* __restrict__ in, int64_t n_max,
                                                            const uint32_t* n_dev, int64_t* __restrict__ sums) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t total;
  const int64_t n = scan_len(n_max, n_dev);
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  if (base >= n && base > 0) {  // past a device-side length: this tile sums to zero
    if (threadIdx.x == 0) sums[blockIdx.x] = 0;
    return;
  }
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += load_or_zero(in, base + k * kScanThreads + threadIdx.x, n);
  block_exclusive(s, warp_sums, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* sums, int64_t tiles) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t total;
  int64_t carry = 0;
  for (int64_t base = 0; base < tiles; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t x = i < tiles ? sums[i] : 0;
    int64_t e = block_exclusive(x, warp_sums, &total);
    if (i < tiles) sums[i] = carry + e;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[tiles] = carry;
}

// Padded index into the shared tile: one spare slot per kScanItems entries, so
// a thread's kScanItems consecutive int64 fall in different banks than its neighbours'.
__device__ __forceinline__ int pad(int i) { return i + i / kScanItems; }

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T* __restrict__ in, int64_t n_max,
                                                            const uint32_t* n_dev, const int64_t* __restrict__ sums,
                                                            int64_t* __restrict__ out, int64_t tiles) {
  __shared__ int64_t tile[kScanTile + kScanTile / kScanItems];
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t total;
  const int64_t n = scan_len(n_max, n_dev);
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[tiles];
  if (base >= n) return;
  // coalesced load into shared memory, then each thread owns kScanItems consecutive items
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = k * kScanThreads + threadIdx.x;
    tile[pad(idx)] = load_or_zero(in, base + idx, n);
  }
  __syncthreads();
  int64_t local[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    local[k] = s;
    s += tile[pad(threadIdx.x * kScanItems + k)];
  }
  int64_t pre = block_exclusive(s, warp_sums, &total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) tile[pad(threadIdx.x * kScanItems + k)] = pre + local[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k * kScanThreads + threadIdx.x;
    if (i < n) out[i] = tile[pad(k * kScanThreads + threadIdx.x)];
  }
}

__global__ void k_write_zero(int64_t* out) { out[0] = 0; }

template <class T>
cudaError_t scan_impl(const T* in, int64_t* out, int64_t n, const uint32_t* n_dev, ScanWs ws, cudaStream_t s) {
  if (n <= 0) {
    k_write_zero<<<1, 1, 0, s>>>(out);
    return cudaGetLastError();
  }
  const int64_t tiles = scan_tiles(n);
  k_tile_sums<T><<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(in, n, n_dev, ws.block_sums);
  k_scan_sums<<<1, 1024, 0, s>>>(ws.block_sums, tiles);
  k_tile_scan<T><<<static_cast<unsigned>(tiles), kScanThreads, 0, s>>>(in, n, n_dev, ws.block_sums, out, tiles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, ScanWs ws, cudaStream_t s,
                               const uint32_t* n_dev) {
  return scan_impl<int32_t>(in, out, n, n_dev, ws, s);
}

cudaError_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, ScanWs ws, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, nullptr, ws, s);
}

}  // namespace tc
