// mg_unweight.cu -- hit-or-miss unweighting on the device (mg_unweight in
// include/mg.h).
//
// The paper (Sect. 2) lists hit-or-miss unweighting among the serial steps
// that follow the matrix element in the event generator, and names it as a
// candidate to offload to the GPU.  Event i is kept when r_i * w_max < w_i
// (r_i uniform in [0, 1)); the kept indices are written in increasing order,
// so the result does not depend on the launch configuration.  Three launches:
// per tile of 4096 events, the accept bits (one warp ballot per 32 events,
// n/8 bytes in all) and their count; one scan of the tile counts; then each
// tile ranks its kept events from its bits alone and writes their indices at
// its tile's offset.  w and r are read once: 16 bytes per event, plus 8 per
// kept index.
#include <cuda_runtime.h>

#include "mg.h"
#include "mg_kernels.cuh"  // mbarrier and bulk-copy primitives

// MG_UW_FP32_FIRST (default 1): the decision r_i * w_max < w_i is taken in
// FP32 where the FP32 values are far enough apart to make it certain, in FP64
// otherwise (the FP64 multiply-and-compare of every event made the count pass
// FP64-bound: 82 % of the FP64 pipe on GB300, where FP64 runs at 1/64 of
// FP32); the kept set is the same bit for bit.
#ifndef MG_UW_FP32_FIRST
#define MG_UW_FP32_FIRST 1
#endif
// MG_UW_TMA: the count pass takes each full tile of 16-byte aligned w and r
// into shared memory with two bulk copies (TMA engine) instead of per-thread
// loads.
#ifndef MG_UW_TMA
#define MG_UW_TMA 0
#endif

namespace {

// MG_UW_PER_THREAD: events per thread and tile, a multiple of 4 (A/B on GB300,
// 67 M events: 4 / 8 / 16 / 24 / 32 -> 0.40 / 0.33 / 0.29 / 0.40 / 0.41 ms)
#ifndef MG_UW_PER_THREAD
#define MG_UW_PER_THREAD 16
#endif
constexpr int UW_THREADS = 256;
constexpr int UW_PER_THREAD = MG_UW_PER_THREAD;
constexpr int UW_TILE = UW_THREADS * UW_PER_THREAD;  // events per tile
constexpr int UW_WARPS = UW_THREADS / 32;
constexpr int UW_WORDS = UW_PER_THREAD * UW_WARPS;  // accept-bit words per tile

// x truncated toward zero to a normal FP32 value, built from its bits with
// integer operations (no FP64 instruction); false where x is zero, subnormal
// in FP32, beyond the FP32 range, infinite or NaN.  |x - f| < 2^-23 |x|.
__device__ __forceinline__ bool f32_trunc(double x, float& f) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffu);  // biased FP64 exponent
  if (e < 897 || e > 1150) return false;    // FP32 exponents 1..254
  f = __uint_as_float((unsigned)(b >> 32 & 0x80000000u) | ((unsigned)(e - 896) << 23) |
                      (unsigned)((b >> 29) & 0x7fffffu));
  return true;
}

// r * w_max < w, exactly as in FP64.  In FP32, p = rf * wmf carries a
// relative error below 3e-7 from the truncations and the product, and wf
// below 1.2e-7; a gap |p - wf| above 1e-6 |wf| (with p a normal FP32 value)
// therefore has the sign of r * w_max - w, which the FP64 product's rounding
// (1.1e-16) cannot change.  Closer cases, and anything outside the FP32
// normal range (zero, NaN, infinities included), take the FP64 comparison.
__device__ __forceinline__ bool kept_exact(double r, double w, double w_max, float wmf, bool wm_ok) {
#if MG_UW_FP32_FIRST
  float rf, wf;
  if (wm_ok && f32_trunc(r, rf) && f32_trunc(w, wf)) {
    const float p = rf * wmf;
    const float ap = fabsf(p);
    const float d = p - wf;
    if (ap >= 1.17549435e-38f && ap <= 3.40282347e38f && fabsf(d) > 1e-6f * fabsf(wf)) return d < 0.f;
  }
#endif
  return r * w_max < w;
}

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
  float wmf = 0.f;
  const bool wm_ok = f32_trunc(w_max, wmf);
  // every load of the tile issued before the first vote
  double wv[UW_PER_THREAD], rv[UW_PER_THREAD];
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
    wv[j] = i < n ? __ldcs(w + i) : 0.0;
    rv[j] = i < n ? __ldcs(r + i) : 1.0;
  }
  int c = 0;
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
    const unsigned m = __ballot_sync(0xffffffffu, i < n && kept_exact(rv[j], wv[j], w_max, wmf, wm_ok));
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

// Pass 1 with the tile staged by the TMA engine: one thread issues two bulk
// copies (w and r of the tile, 2 x 8 * TILE bytes) that complete on one
// mbarrier, then every thread reads its events from shared memory; events,
// bit words and counts as in tile_count_kernel.  Full tiles only, with w and
// r 16-byte aligned (checked on the host); the partial last tile takes
// per-thread loads.  A copy that does not complete within the bounded wait
// is waited for once more (bounded), so that none is left in flight, and the
// tile is then read from global memory.
constexpr size_t UW_TMA_SMEM = 128 + 2 * sizeof(double) * UW_TILE;

__global__ void __launch_bounds__(UW_THREADS)
    tile_count_tma_kernel(const double* __restrict__ w, const double* __restrict__ r, long long n, double w_max,
                          long long* __restrict__ counts, unsigned* __restrict__ bits) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int warp_sum[UW_WARPS];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  double* sw = reinterpret_cast<double*>(smem + 128);
  double* sr = sw + UW_TILE;
  const long long base = (long long)blockIdx.x * UW_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned* tb = bits + (long long)blockIdx.x * UW_WORDS;
  float wmf = 0.f;
  const bool wm_ok = f32_trunc(w_max, wmf);
  bool staged = false;
  if (base + UW_TILE <= n) {  // uniform across the CTA
    if (threadIdx.x == 0) {
      mg::mbar_init(bar, 1);
      mg::fence_mbar_init();
      mg::fence_proxy_async_smem();
      mg::mbar_arrive_expect_tx(bar, (uint32_t)(2 * sizeof(double) * UW_TILE));
      mg::bulk_g2s(sw, w + base, (uint32_t)(sizeof(double) * UW_TILE), bar);
      mg::bulk_g2s(sr, r + base, (uint32_t)(sizeof(double) * UW_TILE), bar);
    }
    __syncthreads();
    staged = __syncthreads_and(mg::mbar_wait_bounded(bar, 0, mg::WAIT_POLLS) ? 1 : 0) != 0;
    if (!staged) mg::mbar_wait_bounded(bar, 0, mg::WAIT_POLLS);
  }
  double wv[UW_PER_THREAD], rv[UW_PER_THREAD];
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const int k = j * UW_THREADS + threadIdx.x;
    const long long i = base + k;
    if (staged) {
      wv[j] = sw[k];
      rv[j] = sr[k];
    } else {
      wv[j] = i < n ? __ldcs(w + i) : 0.0;
      rv[j] = i < n ? __ldcs(r + i) : 1.0;
    }
  }
  int c = 0;
#pragma unroll
  for (int j = 0; j < UW_PER_THREAD; j++) {
    const long long i = base + j * UW_THREADS + threadIdx.x;
    const unsigned m = __ballot_sync(0xffffffffu, i < n && kept_exact(rv[j], wv[j], w_max, wmf, wm_ok));
    if (lane == 0) tb[j * UW_WARPS + warp] = m;
    c += __popc(m);
  }
  if (lane == 0) warp_sum[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int k = 0; k < UW_WARPS; k++) t += warp_sum[k];
    counts[blockIdx.x] = t;
  }
}

// Pass 2: exclusive scan of the tile counts in place, by one block, in
// passes of SCAN_T * SCAN_V tiles: thread t of warp w holds the tiles
// base + j*SCAN_T + t (j < SCAN_V; coalesced loads and stores), so the
// (j, w, lane) order is the index order.  Warp scans of each j, one scan of
// the SCAN_V * 32 warp totals in order by the first warp, the pass's total
// carried to the next; the grand total into *n_acc.
constexpr int SCAN_T = 1024, SCAN_V = 16, SCAN_W = SCAN_T / 32;

__global__ void __launch_bounds__(SCAN_T) tile_scan_kernel(long long* __restrict__ counts, long long ntiles,
                                                           long long* __restrict__ n_acc) {
  __shared__ long long wt[SCAN_V * SCAN_W];  // warp totals, then their exclusive prefixes
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  long long carry = 0;  // kept by the first warp
  for (long long base = 0; base < ntiles; base += (long long)SCAN_T * SCAN_V) {
    // tile counts are at most TILE: a warp's partial sums fit in 32 bits
    int ex[SCAN_V];
#pragma unroll
    for (int j = 0; j < SCAN_V; j++) {
      const long long b = base + (long long)j * SCAN_T + t;
      ex[j] = b < ntiles ? (int)counts[b] : 0;
    }
#pragma unroll
    for (int j = 0; j < SCAN_V; j++) {
      int x = ex[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += a;
      }
      if (lane == 31) wt[j * SCAN_W + warp] = x;
      ex[j] = x - ex[j];  // exclusive within the warp
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll 1
      for (int q = 0; q < SCAN_V * SCAN_W / 32; q++) {
        const long long own = wt[q * 32 + lane];
        long long x = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long a = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += a;
        }
        wt[q * 32 + lane] = carry + x - own;
        carry += __shfl_sync(0xffffffffu, x, 31);
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SCAN_V; j++) {
      const long long b = base + (long long)j * SCAN_T + t;
      if (b < ntiles) counts[b] = wt[j * SCAN_W + warp] + ex[j];
    }
    __syncthreads();  // wt is rewritten by the next pass
  }
  if (t == 0) *n_acc = carry;
}

// Pass 3: from the tile's bits only, each kept event's rank in the tile (the
// counts of the words before its word, then the bits below its lane) and its
// index at the tile's offset.  A tile without kept events (its offset equal
// to the next tile's, or to the total for the last tile) returns at once.
__global__ void __launch_bounds__(UW_THREADS)
    tile_write_kernel(const unsigned* __restrict__ bits, const long long* __restrict__ offsets,
                      const long long* __restrict__ n_acc, long long* __restrict__ idx_out) {
  constexpr int WPL = UW_WORDS / 32;  // words per lane in the word scan
  static_assert(UW_WORDS % 32 == 0, "whole warps of words");
  __shared__ int word_excl[UW_WORDS];
  const long long base = (long long)blockIdx.x * UW_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned* tb = bits + (long long)blockIdx.x * UW_WORDS;
  const long long off = offsets[blockIdx.x];
  const long long next = blockIdx.x + 1 < gridDim.x ? offsets[blockIdx.x + 1] : *n_acc;
  if (next == off) return;  // the same for every thread of the tile
  if (warp == 0) {
    // words q*32 + lane in index order: a warp scan per block of 32 words,
    // carried over the blocks
    int cnt[WPL];
#pragma unroll
    for (int q = 0; q < WPL; q++) cnt[q] = __popc(tb[q * 32 + lane]);
    int carry = 0;
#pragma unroll
    for (int q = 0; q < WPL; q++) {
      int sc = cnt[q];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += a;
      }
      word_excl[q * 32 + lane] = carry + sc - cnt[q];
      carry += __shfl_sync(0xffffffffu, sc, 31);
    }
  }
  __syncthreads();
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
  const bool tma = MG_UW_TMA && (reinterpret_cast<uintptr_t>(w_dev) & 15u) == 0 &&
                   (reinterpret_cast<uintptr_t>(r_dev) & 15u) == 0;
  if (tma) {
    if (cudaFuncSetAttribute(tile_count_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)UW_TMA_SMEM) != cudaSuccess) {
      cudaFreeAsync(counts, s);
      return MG_ERR_CUDA;
    }
    tile_count_tma_kernel<<<(unsigned)ntiles, UW_THREADS, UW_TMA_SMEM, s>>>(w_dev, r_dev, n, w_max, counts, bits);
  } else {
    tile_count_kernel<<<(unsigned)ntiles, UW_THREADS, 0, s>>>(w_dev, r_dev, n, w_max, counts, bits);
  }
  tile_scan_kernel<<<1, SCAN_T, 0, s>>>(counts, ntiles, reinterpret_cast<long long*>(n_acc_dev));
  tile_write_kernel<<<(unsigned)ntiles, UW_THREADS, 0, s>>>(bits, counts, reinterpret_cast<long long*>(n_acc_dev),
                                                            reinterpret_cast<long long*>(idx_out_dev));
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(counts, s);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? MG_OK : MG_ERR_CUDA;
}
