// mg_flowstore.cuh -- where a thread keeps its event's colour-flow
// accumulators (JAMPs) while the chunked helicity program runs.
//
// The chunk functions of the largest process update the flows through one
// of these stores: a pattern of amplitudes, summed in a register, is added to
// (or subtracted from) each flow of the pattern at once.
//
//   FlowsSmem<R>  the thread's column of a [flow][thread] array in shared
//                 memory (stride js), any precision;
//   FlowsTmem     two columns per flow (re, im) of the thread's lane of
//                 tensor memory (FP32), read and written with tcgen05.ld/st:
//                 it keeps 120 complex flows per event off shared memory, so
//                 that more events fit on an SM.  Warp-collective: every
//                 thread of the warp must make the same calls.
//   FlowsTmem64   the same for FP64 flows, four columns per flow.
#pragma once

#include "mg_vertices.cuh"

// MG_CHUNK_SYNC=1: the tensor-memory stores put a block barrier after each
// chunk of the helicity program, so that the CTA's warps run the same chunk's
// code together (every thread of the CTA runs the program)
#ifndef MG_CHUNK_SYNC
#define MG_CHUNK_SYNC 0
#endif

namespace mg {

template <typename R>
struct FlowsSmem {
  cx<R>* p;
  int js;
  template <int N>
  __device__ __forceinline__ void update(const int (&k)[N], const int (&sg)[N], cx<R> v) const {
#pragma unroll
    for (int i = 0; i < N; i++) {
      cx<R>& t = p[k[i] * js];
      t = sg[i] > 0 ? t + v : t - v;
    }
  }
  __device__ __forceinline__ void zero(int n) const {
    for (int c = 0; c < n; c++) p[c * js] = cx<R>{R(0), R(0)};
  }
  __device__ __forceinline__ void chunk_done() const {}
  // add v to (or, odd entries, subtract it from) the flows of list[0..n)
  __device__ __noinline__ void flush(const short* __restrict__ list, int n, cx<R> v) const {
    for (int i = 0; i < n; i++) {
      const int e = __ldg(list + i);
      cx<R>& t = p[(e >> 1) * js];
      t = (e & 1) ? t - v : t + v;
    }
  }
};

struct FlowsTmem {
  uint32_t taddr;  // lane (bits 16-31) and first column of the thread's flows
  __device__ __forceinline__ void chunk_done() const {
#ifdef __CUDA_ARCH__
    if constexpr (MG_CHUNK_SYNC != 0) __syncthreads();
#endif
  }
  template <int N>
  __device__ __forceinline__ void update(const int (&k)[N], const int (&sg)[N], cx<float> v) const {
#ifdef __CUDA_ARCH__
    __syncwarp();  // the tcgen05 accesses below are warp-collective
    uint32_t r[2 * N];
#pragma unroll
    for (int i = 0; i < N; i++)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                   : "=r"(r[2 * i]), "=r"(r[2 * i + 1])
                   : "r"(taddr + 2u * (uint32_t)k[i])
                   : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; i++) {
      const float re = __uint_as_float(r[2 * i]), im = __uint_as_float(r[2 * i + 1]);
      r[2 * i] = __float_as_uint(sg[i] > 0 ? re + v.re : re - v.re);
      r[2 * i + 1] = __float_as_uint(sg[i] > 0 ? im + v.im : im - v.im);
    }
#pragma unroll
    for (int i = 0; i < N; i++)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr + 2u * (uint32_t)k[i]),
                   "r"(r[2 * i]), "r"(r[2 * i + 1])
                   : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#endif
  }
  // add v to (odd entries: subtract it from) the flows of list[0..n), four
  // flows per batch of loads and stores (n is the same for the whole warp)
  __device__ __noinline__ void flush(const short* __restrict__ list, int n, cx<float> v) const {
#ifdef __CUDA_ARCH__
    __syncwarp();
    for (int i0 = 0; i0 < n; i0 += 4) {
      const int m = n - i0 < 4 ? n - i0 : 4;
      int e[4];
      uint32_t r[8];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        e[j] = j < m ? __ldg(list + i0 + j) : 0;
        if (j < m)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                       : "=r"(r[2 * j]), "=r"(r[2 * j + 1])
                       : "r"(taddr + 2u * (uint32_t)(e[j] >> 1))
                       : "memory");
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 4; j++) {
        if (j < m) {
          const float re = __uint_as_float(r[2 * j]), im = __uint_as_float(r[2 * j + 1]);
          const bool minus = e[j] & 1;
          r[2 * j] = __float_as_uint(minus ? re - v.re : re + v.re);
          r[2 * j + 1] = __float_as_uint(minus ? im - v.im : im + v.im);
          asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr + 2u * (uint32_t)(e[j] >> 1)),
                       "r"(r[2 * j]), "r"(r[2 * j + 1])
                       : "memory");
        }
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#endif
  }
  // zero the first n flows (2n columns, rounded up to 16)
  __device__ __forceinline__ void zero(int n) const {
#ifdef __CUDA_ARCH__
    __syncwarp();
    for (int c = 0; c < 2 * n; c += 16)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
          "%1, %1};" ::"r"(taddr + (uint32_t)c),
          "r"(0u)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#endif
  }
};

// FP64 flows in tensor memory: four columns per flow (the two 32-bit halves
// of Re, then of Im)
struct FlowsTmem64 {
  uint32_t taddr;
  __device__ __forceinline__ void chunk_done() const {
#ifdef __CUDA_ARCH__
    if constexpr (MG_CHUNK_SYNC != 0) __syncthreads();
#endif
  }
  template <int N>
  __device__ __forceinline__ void update(const int (&k)[N], const int (&sg)[N], cx<double> v) const {
#ifdef __CUDA_ARCH__
    __syncwarp();  // the tcgen05 accesses below are warp-collective
    uint32_t r[4 * N];
#pragma unroll
    for (int i = 0; i < N; i++)
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(r[4 * i]), "=r"(r[4 * i + 1]), "=r"(r[4 * i + 2]), "=r"(r[4 * i + 3])
                   : "r"(taddr + 4u * (uint32_t)k[i])
                   : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double re = __hiloint2double((int)r[4 * i + 1], (int)r[4 * i]);
      const double im = __hiloint2double((int)r[4 * i + 3], (int)r[4 * i + 2]);
      const double nre = sg[i] > 0 ? re + v.re : re - v.re;
      const double nim = sg[i] > 0 ? im + v.im : im - v.im;
      r[4 * i] = (uint32_t)__double2loint(nre);
      r[4 * i + 1] = (uint32_t)__double2hiint(nre);
      r[4 * i + 2] = (uint32_t)__double2loint(nim);
      r[4 * i + 3] = (uint32_t)__double2hiint(nim);
    }
#pragma unroll
    for (int i = 0; i < N; i++)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr + 4u * (uint32_t)k[i]),
                   "r"(r[4 * i]), "r"(r[4 * i + 1]), "r"(r[4 * i + 2]), "r"(r[4 * i + 3])
                   : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#endif
  }
  __device__ __noinline__ void flush(const short* __restrict__ list, int n, cx<double> v) const {
#ifdef __CUDA_ARCH__
    __syncwarp();
    for (int i0 = 0; i0 < n; i0 += 4) {
      const int m = n - i0 < 4 ? n - i0 : 4;
      int e[4];
      uint32_t r[16];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        e[j] = j < m ? __ldg(list + i0 + j) : 0;
        if (j < m)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(r[4 * j]), "=r"(r[4 * j + 1]), "=r"(r[4 * j + 2]), "=r"(r[4 * j + 3])
                       : "r"(taddr + 4u * (uint32_t)(e[j] >> 1))
                       : "memory");
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 4; j++) {
        if (j < m) {
          const double re = __hiloint2double((int)r[4 * j + 1], (int)r[4 * j]);
          const double im = __hiloint2double((int)r[4 * j + 3], (int)r[4 * j + 2]);
          const bool minus = e[j] & 1;
          const double nre = minus ? re - v.re : re + v.re;
          const double nim = minus ? im - v.im : im + v.im;
          asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                           taddr + 4u * (uint32_t)(e[j] >> 1)),
                       "r"((uint32_t)__double2loint(nre)), "r"((uint32_t)__double2hiint(nre)),
                       "r"((uint32_t)__double2loint(nim)), "r"((uint32_t)__double2hiint(nim))
                       : "memory");
        }
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#endif
  }
  // zero the first n flows (4n columns, rounded up to 16)
  __device__ __forceinline__ void zero(int n) const {
#ifdef __CUDA_ARCH__
    __syncwarp();
    for (int c = 0; c < 4 * n; c += 16)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
          "%1, %1};" ::"r"(taddr + (uint32_t)c),
          "r"(0u)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
#endif
  }
};

}  // namespace mg
