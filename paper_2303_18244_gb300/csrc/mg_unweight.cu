// mg_unweight.cu -- hit-or-miss unweighting on the device (mg_unweight in
// include/mg.h).
//
// The paper (Sect. 2) lists hit-or-miss unweighting among the serial steps
// that follow the matrix element in the event generator, and names it as a
// candidate to offload to the GPU.  Event i is kept when r_i * w_max < w_i
// (r_i uniform in [0, 1)); the kept indices are written in increasing order,
// so the result does not depend on the launch configuration.  Three launches: per-tile counts, one scan of
// the tile counts, then each tile ranks its kept events (warp ballots and a
// block scan) and writes them at its tile's offset.
#include <cuda_runtime.h>

#include "mg.h"

namespace {

constexpr int UW_THREADS = 256;
constexpr int UW_PER_THREAD = 8;
constexpr int UW_TILE = UW_THREADS * UW_PER_THREAD;  // events per tile

__device__ __forceinline__ bool kept(const double* __restrict__ w, const double* __restrict__ r, double w_max,
                                     long long i) {
  return r[i] * w_max < w[i];
}

// Events of tile b handled by thread t: b*TILE + j*THREADS + t (coalesced).
__global__ void __launch_bounds__(UW_THREADS)
    tile_count_kernel(const double* __restrict__ w, const double* __restrict__ r, long long n, double w_max,
                      long long* __restrict__ counts) {
  __shared__ int warp_sum[UW_THREADS / 32];
  const long long base = (long long)blockIdx.x * UW_TILE;
  int c = 0;
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
    if (i < n && kept(w, r, w_max, i)) c++;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int k = 0; k < UW_THREADS / 32; k++) s += warp_sum[k];
    counts[blockIdx.x] = s;
  }
}

// Exclusive scan of the tile counts in place (one block); total into *n_acc.
__global__ void __launch_bounds__(1024) tile_scan_kernel(long long* __restrict__ counts, long long ntiles,
                                                         long long* __restrict__ n_acc) {
  __shared__ long long part[1024];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long b0 = 0; b0 < ntiles; b0 += 1024) {
    const long long b = b0 + threadIdx.x;
    const long long v = b < ntiles ? counts[b] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 values
    for (int o = 1; o < 1024; o <<= 1) {
      const long long add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (b < ntiles) counts[b] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_acc = carry;
}

__global__ void __launch_bounds__(UW_THREADS)
    tile_write_kernel(const double* __restrict__ w, const double* __restrict__ r, long long n, double w_max,
                      const long long* __restrict__ offsets, long long* __restrict__ idx_out) {
  __shared__ int warp_tot[UW_PER_THREAD][UW_THREADS / 32];
  __shared__ long long row_base[UW_PER_THREAD];
  const long long base = (long long)blockIdx.x * UW_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool k[UW_PER_THREAD];
  int rank_in_warp[UW_PER_THREAD];
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
    k[j] = i < n && kept(w, r, w_max, i);
    const unsigned m = __ballot_sync(0xffffffffu, k[j]);
    rank_in_warp[j] = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[j][warp] = __popc(m);
  }
  __syncthreads();
  // rows j in increasing index order: row j covers events base + j*THREADS .. +THREADS-1
  if (threadIdx.x == 0) {
    long long s = offsets[blockIdx.x];
    for (int j = 0; j < UW_PER_THREAD; j++) {
      row_base[j] = s;
      for (int q = 0; q < UW_THREADS / 32; q++) {
        const int t = warp_tot[j][q];
        warp_tot[j][q] = (int)(s - row_base[j]);  // exclusive prefix within the row
        s += t;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    if (k[j]) {
      const long long i = base + j * UW_THREADS + threadIdx.x;
      idx_out[row_base[j] + warp_tot[j][warp] + rank_in_warp[j]] = i;
    }
  }
}

}  // namespace

extern "C" int mg_unweight(const double* w_dev, const double* r_dev, int64_t n, double w_max, int64_t* idx_out_dev,
                           int64_t* n_acc_dev, void* stream) {
  if (n < 0 || !(w_max > 0) || !n_acc_dev) return MG_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) return cudaMemsetAsync(n_acc_dev, 0, sizeof(int64_t), s) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
  if (!w_dev || !r_dev || !idx_out_dev) return MG_ERR_ARG;
  const long long ntiles = (n + UW_TILE - 1) / UW_TILE;
  if (ntiles > 0x7fffffffLL) return MG_ERR_ARG;
  long long* counts = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&counts), sizeof(long long) * ntiles, s) != cudaSuccess)
    return MG_ERR_NOMEM;
  tile_count_kernel<<<(unsigned)ntiles, UW_THREADS, 0, s>>>(w_dev, r_dev, n, w_max, counts);
  tile_scan_kernel<<<1, 1024, 0, s>>>(counts, ntiles, reinterpret_cast<long long*>(n_acc_dev));
  tile_write_kernel<<<(unsigned)ntiles, UW_THREADS, 0, s>>>(w_dev, r_dev, n, w_max, counts,
                                                            reinterpret_cast<long long*>(idx_out_dev));
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(counts, s);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? MG_OK : MG_ERR_CUDA;
}
