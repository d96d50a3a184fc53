// mg_colour_tc.cuh -- colour quadratic form on the 5th-generation tensor cores.
//
// Step A5 (paper Sect. 3: the "colour algebra" step run at reduced precision)
// for a CTA of 128 events and one helicity:
//     ME_h(e) = sum_ij Re/Im J_i(e) KNUM_ij Re/Im J_j(e)       (C = KNUM / CDEN)
// is computed as D = A . KNUM with A = [128 events x K] (K = NCOL padded to a
// multiple of 16) on the tensor cores, then a per-thread row dot J . D.
//
//   * KNUM holds small integers (|KNUM| <= 4096): exact in FP16.
//   * A = s * J split into FP16 hi + lo (hi = fp16(sJ), lo = fp16(sJ - hi)),
//     s a per-event power of two putting max|J| in [1, 2): the pair carries
//     ~22 significant bits, and D = A_hi.KNUM + A_lo.KNUM accumulates in FP32.
//   * Re and Im parts use two accumulators of N columns each in TMEM
//     (cta_group::1, M = 128: row e of D lives in TMEM lane e).
//   * One elected thread issues tcgen05.mma; completion is signalled on an
//     mbarrier through tcgen05.commit; every wait is bounded.
//
// Shared-memory operand layout: K-major, no swizzle ("interleaved" core
// matrices of 8 rows x 16 bytes).  Element (row r, k) of a tile lives at
//     (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2
// with LBO = 128 bytes (next 8 k) and SBO = (K / 8) * 128 bytes (next 8 rows).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "mg_kernels.cuh"

namespace mg {
namespace tc {

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] . B[smem]^T, kind::f16 (FP16 inputs, FP32 accumulate)
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
  // base offset 0, relative LBO mode, layout type 0 (no swizzle)
  return d;
}
// instruction descriptor, kind::f16: D FP32, A/B FP16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4)                        // D format: FP32
         | (0u << 7) | (0u << 10)         // A, B format: FP16
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

constexpr uint32_t LBO = 128;

__host__ __device__ constexpr int pad16(int n) { return ((n + 15) / 16) * 16; }

// byte offset of element (row, k) in a K-major no-swizzle tile with K columns
__host__ __device__ constexpr uint32_t tile_off(int row, int k, int K) {
  return (uint32_t)((row / 8) * (K / 8) * 128 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2);
}

}  // namespace tc

// Shared-memory layout of the tensor-core kernel.  The momenta tile is dead
// once the per-event set-up has run, so the operand tiles reuse its space.
template <class P, int NT>
struct LayoutTC {
  static constexpr int K = tc::pad16(P::NCOL);
  static constexpr int N = tc::pad16(P::NCOL);
  static constexpr size_t a_tile = size_t(NT) * K * 2;  // FP16 [NT][K]
  static constexpr size_t b_tile = size_t(N) * K * 2;   // FP16 [N][K]
  static constexpr size_t bar_bytes = 128;               // TMA bar, MMA bar, TMEM address
  static constexpr size_t stage_bytes = size_t(NT) * P::NPAR * 4 * sizeof(double);
  static constexpr size_t ops_bytes = 4 * a_tile + b_tile;
  static constexpr size_t region_bytes = stage_bytes > ops_bytes ? stage_bytes : ops_bytes;
  static constexpr size_t region_off = bar_bytes;  // no-swizzle tiles need 16-byte alignment only
  static constexpr size_t slab_off = region_off + ((region_bytes + 127) / 128) * 128;
  static constexpr size_t slab_bytes = size_t(NT) * P::NSLOT * sizeof(float);
  static constexpr size_t jamp_off = slab_off + ((slab_bytes + 127) / 128) * 128;
  static constexpr size_t jamp_bytes = size_t(NT) * P::NCOL * sizeof(cx<float>);
  static constexpr size_t base_bytes = jamp_off + ((jamp_bytes + 127) / 128) * 128;
  static constexpr uint32_t tmem_cols = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : 256;
};

// CTAs per SM the register allocation is sized for (launch bounds).  At 2 the
// straight-line gg -> t t~ g g code keeps 255 registers; 3 caps them at 168 and
// its spills halve the throughput (measured).
#ifndef MG_TC_MINB
#define MG_TC_MINB 1
#endif

// Mixed-precision |M|^2 with the tensor-core colour sum; NT = 128 events per CTA.
template <class P, int NT>
__global__ void __launch_bounds__(NT, MG_TC_MINB) sigma_tc_kernel(const double* __restrict__ mom, long long nevt,
                                                      double* __restrict__ me, const int* __restrict__ hels,
                                                      int nhel, KParams kp, const uint4* __restrict__ ctile,
                                                      unsigned* __restrict__ status) {
  static_assert(NT == 128, "one event per TMEM lane");
  using LY = LayoutTC<P, NT>;
  constexpr int K = LY::K, N = LY::N;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* tma_bar = reinterpret_cast<uint64_t*>(smem);
  uint64_t* mma_bar = reinterpret_cast<uint64_t*>(smem + 16);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 32);
  unsigned char* region = smem + LY::region_off;
  float* slab = reinterpret_cast<float*>(smem + LY::slab_off);
  cx<float>* jamp = reinterpret_cast<cx<float>*>(smem + LY::jamp_off) + threadIdx.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;

  const int nvalid =
      load_and_prepare_at<P, float, NT>(tma_bar, reinterpret_cast<double*>(region), slab, mom, nevt, kp, status);
  if (nvalid < 0) return;  // (load_and_prepare_at ends with a block barrier: the tile space is free)

  // colour matrix tile (constant), operand tiles, accumulators
  unsigned char* atile = region;                    // 4 tiles: re_hi, re_lo, im_hi, im_lo
  unsigned char* btile = region + 4 * LY::a_tile;
  for (int i = tid; i < (int)(LY::b_tile / 16); i += NT)
    reinterpret_cast<uint4*>(btile)[i] = __ldg(ctile + i);
  if (tid == 0) {
    mbar_init(mma_bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, LY::tmem_cols);
    tc::tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
  constexpr uint32_t idesc = tc::idesc_f16(128, N);
  const uint32_t a_addr = smem_u32(atile);
  const uint32_t b_addr = smem_u32(btile);
  constexpr uint32_t SBO_A = (K / 8) * 128;
  constexpr uint32_t SBO_B = (K / 8) * 128;

  double acc = 0.0;
  uint32_t phase = 0;
  bool ok = true;
#pragma unroll 1
  for (int ih = 0; ih < nhel && ok; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes<float>(slab + tid, NT, h, kp.v, jamp, NT);
    // per-event power-of-two scale, FP16 hi/lo split into the operand tiles
    float mx = 0.f;
    for (int k = 0; k < P::NCOL; k++) mx = fmaxf(mx, fmaxf(fabsf(jamp[k * NT].re), fabsf(jamp[k * NT].im)));
    const int ex = mx > 0.f ? ((int)((__float_as_uint(mx) >> 23) & 0xff) - 127) : 0;
    const float s = __uint_as_float((uint32_t)(127 - ex) << 23);  // 2^-ex
    for (int j = 0; j < K / 8; j++) {
      __align__(16) __half hr[8], lr[8], hi_[8], li[8];
      for (int q = 0; q < 8; q++) {
        const int k = 8 * j + q;
        const float xr = k < P::NCOL ? s * jamp[k * NT].re : 0.f;
        const float xi = k < P::NCOL ? s * jamp[k * NT].im : 0.f;
        hr[q] = __float2half_rn(xr);
        lr[q] = __float2half_rn(xr - __half2float(hr[q]));
        hi_[q] = __float2half_rn(xi);
        li[q] = __float2half_rn(xi - __half2float(hi_[q]));
      }
      const uint32_t off = tc::tile_off(tid, 8 * j, K);
      *reinterpret_cast<uint4*>(atile + 0 * LY::a_tile + off) = *reinterpret_cast<const uint4*>(hr);
      *reinterpret_cast<uint4*>(atile + 1 * LY::a_tile + off) = *reinterpret_cast<const uint4*>(lr);
      *reinterpret_cast<uint4*>(atile + 2 * LY::a_tile + off) = *reinterpret_cast<const uint4*>(hi_);
      *reinterpret_cast<uint4*>(atile + 3 * LY::a_tile + off) = *reinterpret_cast<const uint4*>(li);
    }
    fence_proxy_async_smem();  // generic-proxy tile writes -> visible to the tensor core
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      for (int part = 0; part < 2; part++) {  // 0: Re -> columns [0, N), 1: Im -> [N, 2N)
        const uint32_t d = tmem + part * N;
        for (int kk = 0; kk < K / 16; kk++) {
          const uint64_t bd = tc::smem_desc(b_addr + kk * 2 * tc::LBO, tc::LBO, SBO_B);
          const uint32_t hi_base = a_addr + (2 * part) * (uint32_t)LY::a_tile + kk * 2 * tc::LBO;
          const uint32_t lo_base = a_addr + (2 * part + 1) * (uint32_t)LY::a_tile + kk * 2 * tc::LBO;
          tc::mma_f16(d, tc::smem_desc(hi_base, tc::LBO, SBO_A), bd, idesc, kk > 0 ? 1u : 0u);
          tc::mma_f16(d, tc::smem_desc(lo_base, tc::LBO, SBO_A), bd, idesc, 1u);
        }
      }
      tc::mma_commit(mma_bar);
    }
    // the outcome of the bounded wait is made uniform across the CTA, so that
    // no thread can skip the warp-collective TMEM loads or a barrier alone
    if (!__syncthreads_and(mbar_wait_bounded(mma_bar, phase, WAIT_POLLS) ? 1 : 0)) {
      if (tid == 0) atomicOr(status, ST_MMA_TIMEOUT);
      ok = false;
      break;
    }
    phase ^= 1u;
    tc::fence_after_sync();
    float dsum = 0.f;
#pragma unroll
    for (int c = 0; c < N; c += 16) {
      float dr[16], di[16];
      tc::tmem_ld16(lane_base + c, dr);
      tc::tmem_ld16(lane_base + N + c, di);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; q++) {
        if (c + q < P::NCOL) {
          dsum = fmaf(jamp[(c + q) * NT].re, dr[q], dsum);
          dsum = fmaf(jamp[(c + q) * NT].im, di[q], dsum);
        }
      }
    }
    acc += (double)(dsum / s);
    tc::fence_before_sync();
    __syncthreads();  // tiles and accumulators are reused by the next helicity
  }
  if (!ok) {
    // an MMA did not signal completion: wait once more (bounded) before the
    // accumulators are released, leave the outputs unwritten
    mbar_wait_bounded(mma_bar, phase, WAIT_POLLS);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, LY::tmem_cols);
  }
  if (ok && tid < nvalid) {
    constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
    me[(long long)blockIdx.x * NT + tid] = acc * norm;
  }
}

// FP16 bit pattern of an integer, or -1 if it is not exactly representable.
inline int fp16_bits_of_int(int v) {
  if (v == 0) return 0;
  const int sgn = v < 0 ? 0x8000 : 0;
  unsigned a = (unsigned)(v < 0 ? -v : v);
  int e = 31 - __builtin_clz(a);           // a in [2^e, 2^(e+1))
  if (e > 15) return -1;
  if (e > 10 && (a & ((1u << (e - 10)) - 1u))) return -1;  // more than 11 significant bits
  const unsigned mant = e >= 10 ? (a >> (e - 10)) & 0x3FFu : (a << (10 - e)) & 0x3FFu;
  return sgn | ((e + 15) << 10) | (int)mant;
}

// FP16 image of the colour-matrix numerators in the B-operand layout.
// Returns false if a numerator is not exact in FP16.
inline bool colour_tile_host(const int* knum, int ncol, unsigned short* out /* [N*K] */) {
  const int K = tc::pad16(ncol), N = tc::pad16(ncol);
  for (int i = 0; i < N * K; i++) out[i] = 0;
  for (int n = 0; n < ncol; n++)
    for (int k = 0; k < ncol; k++) {
      const int b = fp16_bits_of_int(knum[n * ncol + k]);
      if (b < 0) return false;
      out[tc::tile_off(n, k, K) / 2] = (unsigned short)b;
    }
  return true;
}

template <class P>
int launch_sigma_tc(const LaunchArgs& a) {
  constexpr int NT = 128;
  constexpr size_t smem = LayoutTC<P, NT>::base_bytes;
  static const cudaError_t attr = set_smem_attr(sigma_tc_kernel<P, NT>, smem);
  if (attr != cudaSuccess) return -4;
  if (a.nevt <= 0) return 0;
  const long long grid = (a.nevt + NT - 1) / NT;
  sigma_tc_kernel<P, NT><<<(unsigned)grid, NT, smem, a.stream>>>(a.mom, a.nevt, a.out, a.hels, a.nhel, a.kp,
                                                                   static_cast<const uint4*>(a.ctile), a.status);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

}  // namespace mg
