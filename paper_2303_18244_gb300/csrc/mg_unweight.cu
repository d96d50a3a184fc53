// mg_unweight.cu -- hit-or-miss unweighting on the device (mg_unweight in
// include/mg.h).
//
// The paper (Sect. 2) lists hit-or-miss unweighting among the serial steps
// that follow the matrix element in the event generator, and names it as a
// candidate to offload to the GPU.  Event i is kept when r_i * w_max < w_i
// (r_i uniform in [0, 1)); the kept indices are written in increasing order,
// so the result does not depend on the launch configuration.  Three launches:
// per tile of 2048 events, the accept bits (one warp ballot per 32 events,
// n/8 bytes in all) and their count; one scan of the tile counts; then each
// tile ranks its kept events from its bits alone and writes their indices at
// its tile's offset.  w and r are read once: 16 bytes per event, plus 8 per
// kept index.
#include <cuda_runtime.h>

#include "mg.h"

#ifndef MG_UW_PREFETCH
#define MG_UW_PREFETCH 1
#endif

namespace {

constexpr int UW_THREADS = 256;
constexpr int UW_PER_THREAD = 8;
constexpr int UW_TILE = UW_THREADS * UW_PER_THREAD;  // events per tile
constexpr int UW_WARPS = UW_THREADS / 32;
constexpr int UW_WORDS = UW_PER_THREAD * UW_WARPS;  // accept-bit words per tile

#if !MG_UW_PREFETCH
__device__ __forceinline__ bool kept(const double* __restrict__ w, const double* __restrict__ r, double w_max,
                                     long long i) {
  return r[i] * w_max < w[i];
}
#endif

// Pass 1.  Thread t of tile b takes events b*TILE + j*THREADS + t, j < PER_THREAD
// (coalesced); word j*WARPS + warp of the tile's bits holds the ballot of
// events b*TILE + j*THREADS + warp*32 + lane, so the words in order cover the
// tile in increasing index order.
__global__ void __launch_bounds__(UW_THREADS)
    tile_count_kernel(const double* __restrict__ w, const double* __restrict__ r, long long n, double w_max,
                      long long* __restrict__ counts, unsigned* __restrict__ bits) {
  __shared__ int warp_sum[UW_WARPS];
  const long long base = (long long)blockIdx.x * UW_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned* tb = bits + (long long)blockIdx.x * UW_WORDS;
  // every load of the tile issued before the first vote (MG_UW_PREFETCH=0:
  // loads interleaved with the votes)
#if MG_UW_PREFETCH
  double wv[UW_PER_THREAD], rv[UW_PER_THREAD];
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
    wv[j] = i < n ? __ldcs(w + i) : 0.0;
    rv[j] = i < n ? __ldcs(r + i) : 1.0;
  }
#endif
  int c = 0;
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
#if MG_UW_PREFETCH
    const unsigned m = __ballot_sync(0xffffffffu, i < n && rv[j] * w_max < wv[j]);
#else
    const unsigned m = __ballot_sync(0xffffffffu, i < n && kept(w, r, w_max, i));
#endif
    if (lane == 0) tb[j * UW_WARPS + warp] = m;
    c += __popc(m);  // the same in every lane of the warp
  }
  if (lane == 0) warp_sum[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int k = 0; k < UW_WARPS; k++) t += warp_sum[k];
    counts[blockIdx.x] = t;
  }
}

// Pass 2: exclusive scan of the tile counts in place (one block: each thread
// sums a contiguous run of tiles, one block scan of the run sums, each thread
// rewrites its run); the total into *n_acc.
__global__ void __launch_bounds__(1024) tile_scan_kernel(long long* __restrict__ counts, long long ntiles,
                                                         long long* __restrict__ n_acc) {
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const long long per = (ntiles + 1023) / 1024;
  const long long b0 = t * per;
  const long long b1 = b0 + per < ntiles ? b0 + per : ntiles;
  long long own = 0;
  for (long long b = b0; b < b1; b++) own += counts[b];
  part[t] = own;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
    const long long add = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  long long run = part[t] - own;
  for (long long b = b0; b < b1; b++) {
    const long long v = counts[b];
    counts[b] = run;
    run += v;
  }
  if (t == 1023) *n_acc = part[1023];
}

// Pass 3: from the tile's bits only, each kept event's rank in the tile (the
// counts of the words before its word, then the bits below its lane) and its
// index at the tile's offset.
__global__ void __launch_bounds__(UW_THREADS)
    tile_write_kernel(const unsigned* __restrict__ bits, const long long* __restrict__ offsets,
                      long long* __restrict__ idx_out) {
  static_assert(UW_WORDS == 64, "two words per lane in the word scan");
  __shared__ int word_excl[UW_WORDS];
  const long long base = (long long)blockIdx.x * UW_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned* tb = bits + (long long)blockIdx.x * UW_WORDS;
  if (warp == 0) {
    const int c0 = __popc(tb[lane]), c1 = __popc(tb[32 + lane]);
    int s0 = c0, s1 = c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a0 = __shfl_up_sync(0xffffffffu, s0, o);
      const int a1 = __shfl_up_sync(0xffffffffu, s1, o);
      if (lane >= o) {
        s0 += a0;
        s1 += a1;
      }
    }
    const int tot0 = __shfl_sync(0xffffffffu, s0, 31);
    word_excl[lane] = s0 - c0;
    word_excl[32 + lane] = tot0 + s1 - c1;
  }
  __syncthreads();
  const long long off = offsets[blockIdx.x];
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const int q = j * UW_WARPS + warp;
    const unsigned m = tb[q];
    if ((m >> lane) & 1u)
      idx_out[off + word_excl[q] + __popc(m & ((1u << lane) - 1u))] = base + j * UW_THREADS + threadIdx.x;
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
  // workspace: the tile counts (then offsets), then the accept bits
  long long* counts = nullptr;
  const size_t bytes = (size_t)ntiles * (sizeof(long long) + UW_WORDS * sizeof(unsigned));
  if (cudaMallocAsync(reinterpret_cast<void**>(&counts), bytes, s) != cudaSuccess) return MG_ERR_NOMEM;
  unsigned* bits = reinterpret_cast<unsigned*>(counts + ntiles);
  tile_count_kernel<<<(unsigned)ntiles, UW_THREADS, 0, s>>>(w_dev, r_dev, n, w_max, counts, bits);
  tile_scan_kernel<<<1, 1024, 0, s>>>(counts, ntiles, reinterpret_cast<long long*>(n_acc_dev));
  tile_write_kernel<<<(unsigned)ntiles, UW_THREADS, 0, s>>>(bits, counts, reinterpret_cast<long long*>(idx_out_dev));
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(counts, s);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? MG_OK : MG_ERR_CUDA;
}
