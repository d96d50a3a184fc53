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

#include "mg_flowstore.cuh"
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
// With MG_TC_ALIAS the colour-flow accumulators share that space too (each
// thread moves its flows into registers before the operand tiles are
// written), which leaves the constant B tile and the slab as the only other
// regions.
#ifndef MG_TC_ALIAS
#define MG_TC_ALIAS 0
#endif
template <class P, int NT>
struct LayoutTC {
  static constexpr bool alias = MG_TC_ALIAS != 0;
  static constexpr int K = tc::pad16(P::NCOL);
  static constexpr int N = tc::pad16(P::NCOL);
  static constexpr size_t r128(size_t b) { return ((b + 127) / 128) * 128; }
  static constexpr size_t a_tile = size_t(NT) * K * 2;  // FP16 [NT][K]
  static constexpr size_t b_tile = size_t(N) * K * 2;   // FP16 [N][K]
  static constexpr size_t bar_bytes = 128;               // TMA bar, MMA bar, TMEM address
  static constexpr size_t stage_bytes = size_t(NT) * P::NPAR * 4 * sizeof(double);
  static constexpr size_t jamp_bytes = size_t(NT) * P::NCOL * sizeof(cx<float>);
  static constexpr size_t slab_bytes = size_t(NT) * slab_slots<P, float>() * sizeof(float);
  static constexpr size_t ops_bytes = 4 * a_tile + (alias ? 0 : b_tile);
  static constexpr size_t region_bytes = stage_bytes > ops_bytes
                                             ? (alias && jamp_bytes > stage_bytes ? jamp_bytes : stage_bytes)
                                             : (alias && jamp_bytes > ops_bytes ? jamp_bytes : ops_bytes);
  static constexpr size_t region_off = bar_bytes;  // no-swizzle tiles need 16-byte alignment only
  static constexpr size_t b_off = alias ? region_off + r128(region_bytes) : region_off + 4 * a_tile;
  static constexpr size_t slab_off = alias ? b_off + r128(b_tile) : region_off + r128(region_bytes);
  static constexpr size_t jamp_off = alias ? region_off : slab_off + r128(slab_bytes);
  static constexpr size_t base_bytes = alias ? slab_off + r128(slab_bytes) : jamp_off + r128(jamp_bytes);
  static constexpr uint32_t tmem_cols = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : 256;
};

// The per-helicity colour form of a CTA of 128 events, shared by the fused
// kernels.  (1) Each event's thread writes its flows, scaled by a power of two
// s = 2^-ex that puts max |J| in [1, 2), as FP16 hi + lo into the four operand
// tiles (re_hi, re_lo, im_hi, im_lo; row = event); returns s.
template <class P, int K>
__device__ __forceinline__ float colour_operands(unsigned char* atile, size_t a_tile, int row,
                                                 const float (&fr)[P::NCOL], const float (&fi)[P::NCOL]) {
  float mx = 0.f;
#pragma unroll
  for (int k = 0; k < P::NCOL; k++) mx = fmaxf(mx, fmaxf(fabsf(fr[k]), fabsf(fi[k])));
  const int ex = mx > 0.f ? ((int)((__float_as_uint(mx) >> 23) & 0xff) - 127) : 0;
  const float s = __uint_as_float((uint32_t)(127 - ex) << 23);  // 2^-ex
#pragma unroll
  for (int j = 0; j < K / 8; j++) {
    __align__(16) __half hr[8], lr[8], hi_[8], li[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int k = 8 * j + q;
      const float xr = k < P::NCOL ? s * fr[k < P::NCOL ? k : 0] : 0.f;
      const float xi = k < P::NCOL ? s * fi[k < P::NCOL ? k : 0] : 0.f;
      hr[q] = __float2half_rn(xr);
      lr[q] = __float2half_rn(xr - __half2float(hr[q]));
      hi_[q] = __float2half_rn(xi);
      li[q] = __float2half_rn(xi - __half2float(hi_[q]));
    }
    const uint32_t off = tc::tile_off(row, 8 * j, K);
    *reinterpret_cast<uint4*>(atile + 0 * a_tile + off) = *reinterpret_cast<const uint4*>(hr);
    *reinterpret_cast<uint4*>(atile + 1 * a_tile + off) = *reinterpret_cast<const uint4*>(lr);
    *reinterpret_cast<uint4*>(atile + 2 * a_tile + off) = *reinterpret_cast<const uint4*>(hi_);
    *reinterpret_cast<uint4*>(atile + 3 * a_tile + off) = *reinterpret_cast<const uint4*>(li);
  }
  return s;
}

// (2) One elected thread: D_re = (A_re_hi + A_re_lo) . KNUM into TMEM columns
// [0, N), D_im likewise into [N, 2N); completion arrives on mma_bar.
template <int K, int N>
__device__ __forceinline__ void colour_mma(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, size_t a_tile,
                                           uint64_t* mma_bar) {
  constexpr uint32_t idesc = tc::idesc_f16(128, N);
  constexpr uint32_t SBO = (K / 8) * 128;
  tc::fence_after_sync();
  for (int part = 0; part < 2; part++) {  // 0: Re -> columns [0, N), 1: Im -> [N, 2N)
    const uint32_t d = tmem + part * N;
    for (int kk = 0; kk < K / 16; kk++) {
      const uint64_t bd = tc::smem_desc(b_addr + kk * 2 * tc::LBO, tc::LBO, SBO);
      const uint32_t hi_base = a_addr + (2 * part) * (uint32_t)a_tile + kk * 2 * tc::LBO;
      const uint32_t lo_base = a_addr + (2 * part + 1) * (uint32_t)a_tile + kk * 2 * tc::LBO;
      tc::mma_f16(d, tc::smem_desc(hi_base, tc::LBO, SBO), bd, idesc, kk > 0 ? 1u : 0u);
      tc::mma_f16(d, tc::smem_desc(lo_base, tc::LBO, SBO), bd, idesc, 1u);
    }
  }
  tc::mma_commit(mma_bar);
}

// (3) Warp-collective: the event's row of D read from its TMEM lane and
// contracted with its flows, sum_k Re J_k D_re,k + Im J_k D_im,k (still
// scaled by s).
template <class P, int N>
__device__ __forceinline__ float colour_readback(uint32_t lane_base, const float (&fr)[P::NCOL],
                                                 const float (&fi)[P::NCOL]) {
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
        dsum = fmaf(fr[c + q < P::NCOL ? c + q : 0], dr[q], dsum);
        dsum = fmaf(fi[c + q < P::NCOL ? c + q : 0], di[q], dsum);
      }
    }
  }
  return dsum;
}

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
  unsigned char* btile = smem + LY::b_off;
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
  const uint32_t a_addr = smem_u32(atile);
  const uint32_t b_addr = smem_u32(btile);

  double acc = 0.0;
  uint32_t phase = 0;
  bool ok = true;
#pragma unroll 1
  for (int ih = 0; ih < nhel && ok; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes<float>(slab + tid, NT, h, kp.v, jamp, NT);
    // the event's flows into registers (their space may hold the operand tiles)
    float fr[P::NCOL], fi[P::NCOL];
#pragma unroll
    for (int k = 0; k < P::NCOL; k++) {
      fr[k] = jamp[k * NT].re;
      fi[k] = jamp[k * NT].im;
    }
    if constexpr (LY::alias) __syncthreads();
    // per-event power-of-two scale, FP16 hi/lo split into the operand tiles
    const float s = colour_operands<P, K>(atile, LY::a_tile, tid, fr, fi);
    fence_proxy_async_smem();  // generic-proxy tile writes -> visible to the tensor core
    __syncthreads();
    if (tid == 0) colour_mma<K, N>(tmem, a_addr, b_addr, LY::a_tile, mma_bar);
    // the outcome of the bounded wait is made uniform across the CTA, so that
    // no thread can skip the warp-collective TMEM loads or a barrier alone
    if (!__syncthreads_and(mbar_wait_bounded(mma_bar, phase, kp.polls) ? 1 : 0)) {
      if (tid == 0) atomicOr(status, ST_MMA_TIMEOUT);
      ok = false;
      break;
    }
    phase ^= 1u;
    tc::fence_after_sync();
    const float dsum = colour_readback<P, N>(lane_base, fr, fi);
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

// ---------------------------------------------------------------------------
// Two-phase mixed path for processes whose colour operands do not fit in
// shared memory beside the per-event state (120 flows): flows_kernel writes
// the FP32 flows of every (good helicity, event) row to a workspace in HBM;
// colour_rows_tc_kernel contracts them with the colour matrix on the tensor
// cores, batched over events x helicities, and sums the helicities per event.
// ---------------------------------------------------------------------------
// MG_ROWS_REGS (default 1): the colour kernel holds each row's flows in
// registers for the helicity (see colour_rows_tc_kernel); 0 reads them from
// the workspace where they are used.
#ifndef MG_ROWS_REGS
#define MG_ROWS_REGS 1
#endif
constexpr int ROWS_REGS = MG_ROWS_REGS;  // for the unroll counts (pragmas see no macros)
template <class P>
struct LayoutRows {
  static constexpr int K = tc::pad16(P::NCOL);
  static constexpr int N = tc::pad16(P::NCOL);
  static constexpr size_t a_tile = size_t(128) * K * 2;  // FP16 [128][K]
  static constexpr size_t b_tile = size_t(N) * K * 2;    // FP16 [N][K]
  static constexpr size_t a_off = 128;                    // MMA bar, TMEM address
  static constexpr size_t b_off = a_off + 4 * a_tile;
  static constexpr size_t base_bytes = b_off + b_tile;
  static constexpr uint32_t tmem_cols = (2 * N <= 32) ? 32 : (2 * N <= 64) ? 64 : (2 * N <= 128) ? 128 : 256;
};

// One CTA per 128 rows of events (TMEM lane = event).  Per helicity of the
// slice: the rows' flows from J (rows past nevt read as zero), a per-row
// power-of-two scale, FP16 hi/lo operand tiles, D = A K in TMEM for Re and
// Im, then sum_k J_k D_k with the FP32 flows; helicities summed in FP64 into
// me: a later slice continues the running sum stored by the one before, so
// the helicities are added in the same order however they are sliced; the
// last slice normalises.
template <class P>
__global__ void __launch_bounds__(128, 1)
    colour_rows_tc_kernel(const float2* __restrict__ J, long long ldj, long long nevt, double* __restrict__ me,
                          int nhel, int first, int last, const uint4* __restrict__ ctile,
                          unsigned* __restrict__ status, uint32_t polls) {
  using LY = LayoutRows<P>;
  constexpr int NT = 128, K = LY::K, N = LY::N;
  static_assert(2 * N <= 256, "two accumulators of N columns");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* mma_bar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
  unsigned char* atile = smem + LY::a_off;
  unsigned char* btile = smem + LY::b_off;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const long long e = (long long)blockIdx.x * NT + tid;
  const bool valid = e < nevt;

  for (int i = tid; i < (int)(LY::b_tile / 16); i += NT) reinterpret_cast<uint4*>(btile)[i] = __ldg(ctile + i);
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
  constexpr uint32_t SBO = (K / 8) * 128;

  double acc = (!first && valid) ? me[e] : 0.0;
  uint32_t phase = 0;
  bool ok = true;
#pragma unroll 1
  for (int ih = 0; ih < nhel && ok; ih++) {
    const float2* row = J + (long long)ih * P::NCOL * ldj + e;
#if MG_ROWS_REGS
    // the row's flows into registers with every load in flight at once (one
    // read of the workspace; the loads of a loop that used each value at
    // once kept only a few per thread in flight)
    float2 fv[P::NCOL];
#pragma unroll
    for (int k = 0; k < P::NCOL; k++) fv[k] = valid ? __ldcs(row + (long long)k * ldj) : make_float2(0.f, 0.f);
#define MG_ROW_FLOW(k) fv[k]
#else
#define MG_ROW_FLOW(k) row[(long long)(k) * ldj]
#endif
    float mx = 0.f;
    if (valid) {
#pragma unroll ROWS_REGS ? P::NCOL : 8
      for (int k = 0; k < P::NCOL; k++) {
        const float2 v = MG_ROW_FLOW(k);
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
    const int ex = mx > 0.f ? ((int)((__float_as_uint(mx) >> 23) & 0xff) - 127) : 0;
    const float s = __uint_as_float((uint32_t)(127 - ex) << 23);  // 2^-ex
#pragma unroll ROWS_REGS ? K / 8 : 1
    for (int j = 0; j < K / 8; j++) {
      __align__(16) __half hr[8], lr[8], hi_[8], li[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int k = 8 * j + q;
        const float2 v = (valid && k < P::NCOL) ? MG_ROW_FLOW(k < P::NCOL ? k : 0) : make_float2(0.f, 0.f);
        const float xr = s * v.x, xi = s * v.y;
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
          const uint64_t bd = tc::smem_desc(b_addr + kk * 2 * tc::LBO, tc::LBO, SBO);
          const uint32_t hi_base = a_addr + (2 * part) * (uint32_t)LY::a_tile + kk * 2 * tc::LBO;
          const uint32_t lo_base = a_addr + (2 * part + 1) * (uint32_t)LY::a_tile + kk * 2 * tc::LBO;
          tc::mma_f16(d, tc::smem_desc(hi_base, tc::LBO, SBO), bd, idesc, kk > 0 ? 1u : 0u);
          tc::mma_f16(d, tc::smem_desc(lo_base, tc::LBO, SBO), bd, idesc, 1u);
        }
      }
      tc::mma_commit(mma_bar);
    }
    // bounded wait, outcome uniform across the CTA (see sigma_tc_kernel)
    if (!__syncthreads_and(mbar_wait_bounded(mma_bar, phase, polls) ? 1 : 0)) {
      if (tid == 0) atomicOr(status, ST_MMA_TIMEOUT);
      ok = false;
      break;
    }
    phase ^= 1u;
    tc::fence_after_sync();
    float dsum = 0.f;
#pragma unroll ROWS_REGS ? N / 16 : 1
    for (int c = 0; c < N; c += 16) {
      float dr[16], di[16];
      tc::tmem_ld16(lane_base + c, dr);
      tc::tmem_ld16(lane_base + N + c, di);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; q++) {
        const int k = c + q;
        const float2 v = (valid && k < P::NCOL) ? MG_ROW_FLOW(k < P::NCOL ? k : 0) : make_float2(0.f, 0.f);
        dsum = fmaf(v.x, dr[q], dsum);
        dsum = fmaf(v.y, di[q], dsum);
      }
    }
#undef MG_ROW_FLOW
    acc += (double)(dsum / s);
    tc::fence_before_sync();
    __syncthreads();  // tiles and accumulators are reused by the next helicity
  }
  if (!ok) mbar_wait_bounded(mma_bar, phase, WAIT_POLLS);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, LY::tmem_cols);
  }
  if (ok && valid) {
    constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
    me[e] = last ? acc * norm : acc;
  }
}

// First phase with the colour flows in tensor memory (default; MG_FLOWS_TMEM=0
// selects flows_kernel): 128 events per CTA, TMEM lane = event, two columns
// per flow; shared memory holds only the momenta tile and the per-event slab,
// so that two CTAs (8 warps) fit on an SM instead of two CTAs of 64 events.
// Same output as flows_kernel; gg -> t t~ g g g mixed 1.79e5 -> 2.87e5 MEs/s.
#ifndef MG_FLOWS_TMEM
#define MG_FLOWS_TMEM 1
#endif
// MG_FLOWS_NT: events per CTA of the tensor-memory flow kernel, 128 (two
// CTAs of 4 warps per SM) or 256 (one CTA of 8 warps per SM holding all 512
// TMEM columns: warp w keeps its 32 events in lanes 32 (w mod 4) and the
// column half w / 4, so that with MG_CHUNK_SYNC all 8 warps of an SM run the
// same chunk of the helicity program together)
#ifndef MG_FLOWS_NT
#define MG_FLOWS_NT 128
#endif
template <class P, int NT_ = MG_FLOWS_NT>
struct LayoutFlowsTmem {
  static constexpr int NT = NT_;
  static_assert(NT == 128 || NT == 256, "128 TMEM lanes, one or two column halves");
  static constexpr size_t r128(size_t b) { return ((b + 127) / 128) * 128; }
  static constexpr size_t bar_bytes = 128;  // TMA bar, TMEM address
  static constexpr size_t stage_bytes = size_t(NT) * P::NPAR * 4 * sizeof(double);
  static constexpr size_t slab_bytes = size_t(NT) * slab_slots<P, float>() * sizeof(float);
  static constexpr size_t stage_off = bar_bytes;
  static constexpr size_t slab_off = stage_off + r128(stage_bytes);
  static constexpr size_t base_bytes = slab_off + r128(slab_bytes);
  static constexpr uint32_t tmem_cols = 256 * (NT / 128);
};

template <class P>
__global__ void __launch_bounds__(MG_FLOWS_NT)
    flows_tmem_kernel(const double* __restrict__ mom, long long nevt, float2* __restrict__ J, long long ldj,
                      const int* __restrict__ hels, int nhel, KParams kp, unsigned* __restrict__ status) {
  using LY = LayoutFlowsTmem<P>;
  constexpr int NT = LY::NT;
  static_assert(2 * P::NCOL <= 256, "flows fit in a column half");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* tma_bar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
  double* stage = reinterpret_cast<double*>(smem + LY::stage_off);
  float* slab = reinterpret_cast<float*>(smem + LY::slab_off);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int nvalid = load_and_prepare_at<P, float, NT>(tma_bar, stage, slab, mom, nevt, kp, status);
  if (nvalid < 0) return;
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, LY::tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const FlowsTmem fl{tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(warp >> 2) * 256u};
  const long long e = (long long)blockIdx.x * NT + tid;
  const bool in_rows = e < ldj;  // rows are padded to 128 events, the grid to NT
#pragma unroll 1
  for (int ih = 0; ih < nhel; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes_store<float>(slab + tid, NT, h, kp.v, fl);
    float2* row = J + (long long)ih * P::NCOL * ldj + e;
#pragma unroll 1
    for (int c = 0; c < 2 * P::NCOL; c += 16) {
      float v[16];
      tc::tmem_ld16(fl.taddr + (uint32_t)c, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int k = c / 2 + q;
        if (k < P::NCOL && in_rows) row[(long long)k * ldj] = make_float2(v[2 * q], v[2 * q + 1]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, LY::tmem_cols);
  }
}

// FP64 |M|^2 with the colour flows in tensor memory: 128 events per CTA,
// four TMEM columns per flow (all 512 columns for 120 flows); shared memory
// holds only the momenta tile and the FP64 slab, 4 warps per SM instead of 2.
// The colour form reads the flows back from TMEM in blocks of four.
template <class P>
struct LayoutTmem64 {
  static constexpr int NT = 128;
  static constexpr size_t r128(size_t b) { return ((b + 127) / 128) * 128; }
  static constexpr size_t bar_bytes = 128;  // TMA bar, TMEM address
  static constexpr size_t stage_bytes = size_t(NT) * P::NPAR * 4 * sizeof(double);
  static constexpr size_t slab_bytes = size_t(NT) * slab_slots<P, double>() * sizeof(double);
  static constexpr size_t stage_off = bar_bytes;
  static constexpr size_t slab_off = stage_off + r128(stage_bytes);
  static constexpr size_t base_bytes = slab_off + r128(slab_bytes);
  static constexpr uint32_t tmem_cols = 512;
};

// four FP64 flows (16 columns) from TMEM
__device__ __forceinline__ void tmem_flows4(uint32_t taddr, double re[4], double im[4]) {
  float v[16];
  tc::tmem_ld16(taddr, v);
  tc::tmem_wait_ld();
#pragma unroll
  for (int q = 0; q < 4; q++) {
    re[q] = __hiloint2double(__float_as_int(v[4 * q + 1]), __float_as_int(v[4 * q]));
    im[q] = __hiloint2double(__float_as_int(v[4 * q + 3]), __float_as_int(v[4 * q + 2]));
  }
}

// sum_ij K_ij (Re J_i Re J_j + Im J_i Im J_j) from the FP64 flows in TMEM;
// knum: K_ii on the diagonal, 2 K_ij for j > i
template <class P>
__device__ __forceinline__ double colour_tmem64(uint32_t taddr, const short* __restrict__ knum) {
  static_assert(P::NCOL % 4 == 0, "blocks of four flows");
  constexpr int NB = P::NCOL / 4;
  double acc = 0.0;
#pragma unroll 1
  for (int ib = 0; ib < NB; ib++) {
    double ri[4], ii[4], yr[4], yi[4];
    tmem_flows4(taddr + 16u * ib, ri, ii);
#pragma unroll
    for (int a = 0; a < 4; a++) {
      yr[a] = 0.0;
      yi[a] = 0.0;
#pragma unroll
      for (int b = a; b < 4; b++) {
        const double k = (double)__ldg(knum + (4 * ib + a) * P::NCOL + 4 * ib + b);
        yr[a] = ::fma(k, ri[b], yr[a]);
        yi[a] = ::fma(k, ii[b], yi[a]);
      }
    }
#pragma unroll 1
    for (int jb = ib + 1; jb < NB; jb++) {
      double rj[4], ij[4];
      tmem_flows4(taddr + 16u * jb, rj, ij);
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) {
          const double k = (double)__ldg(knum + (4 * ib + a) * P::NCOL + 4 * jb + b);
          yr[a] = ::fma(k, rj[b], yr[a]);
          yi[a] = ::fma(k, ij[b], yi[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; a++) acc = ::fma(ri[a], yr[a], ::fma(ii[a], yi[a], acc));
  }
  return acc;
}

template <class P>
__global__ void __launch_bounds__(128, 1)
    sigma_tmem64_kernel(const double* __restrict__ mom, long long nevt, double* __restrict__ me,
                        const int* __restrict__ hels, int nhel, KParams kp, unsigned* __restrict__ status) {
  using LY = LayoutTmem64<P>;
  constexpr int NT = 128;
  static_assert(4 * P::NCOL <= (int)LY::tmem_cols, "flows fit in the allocated columns");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* tma_bar = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 16);
  double* stage = reinterpret_cast<double*>(smem + LY::stage_off);
  double* slab = reinterpret_cast<double*>(smem + LY::slab_off);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int nvalid = load_and_prepare_at<P, double, NT>(tma_bar, stage, slab, mom, nevt, kp, status);
  if (nvalid < 0) return;
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, LY::tmem_cols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const FlowsTmem64 fl{tmem + ((uint32_t)(warp * 32) << 16)};
  const short* knum = P::knum_dev();
  double acc = 0.0;
#pragma unroll 1
  for (int ih = 0; ih < nhel; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes_store<double>(slab + tid, NT, h, kp.v, fl);
    acc += colour_tmem64<P>(fl.taddr, knum);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, LY::tmem_cols);
  }
  if (tid < nvalid) {
    constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
    me[(long long)blockIdx.x * NT + tid] = acc * norm;
  }
}

template <class P>
int launch_sigma_tmem64(const LaunchArgs& a) {
  constexpr size_t smem = LayoutTmem64<P>::base_bytes;
  static const cudaError_t attr = set_smem_attr(sigma_tmem64_kernel<P>, smem);
  if (attr != cudaSuccess) return -4;
  if (a.nevt <= 0) return 0;
  sigma_tmem64_kernel<P><<<(unsigned)((a.nevt + 127) / 128), 128, smem, a.stream>>>(a.mom, a.nevt, a.out, a.hels,
                                                                                     a.nhel, a.kp, a.status);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

// The two phases over slices of the good helicities, every event in each
// launch (full grids), with a stream-ordered workspace of at most
// ROWS_WORKSPACE bytes of flows (FP32 complex [slice][NCOL][events]).
constexpr size_t ROWS_WORKSPACE = size_t(1) << 30;

// Rows per event padded to 128, and the helicities of one slice: as many as
// fit ROWS_WORKSPACE (at least one, at most nhel).
inline long long rows_ld(long long nevt) { return (nevt + 127) / 128 * 128; }
inline long long rows_slice(int ncol, long long nevt, int nhel) {
  const size_t per_hel = (size_t)ncol * (size_t)rows_ld(nevt) * sizeof(float2);
  const long long hs = (long long)(ROWS_WORKSPACE / per_hel);
  return hs < 1 ? 1 : (hs > nhel ? nhel : hs);
}
// bytes one two-phase launch takes from the stream-ordered allocator
inline size_t rows_workspace_bytes(int ncol, long long nevt, int nhel) {
  if (nevt <= 0 || nhel <= 0) return 0;
  return (size_t)rows_slice(ncol, nevt, nhel) * (size_t)ncol * (size_t)rows_ld(nevt) * sizeof(float2);
}

template <class P, int NT>
int launch_sigma_rows(const LaunchArgs& a) {
  static_assert(128 % NT == 0, "flow rows are padded to 128 events");
  constexpr bool tmem_flows = MG_FLOWS_TMEM != 0;
  constexpr int NT1 = tmem_flows ? LayoutFlowsTmem<P>::NT : NT;
  constexpr size_t smem1 = tmem_flows ? LayoutFlowsTmem<P>::base_bytes : Layout<P, float, NT>::base_bytes;
  constexpr size_t smem2 = LayoutRows<P>::base_bytes;
  static const cudaError_t attr1 = [] {
    if constexpr (tmem_flows)
      return set_smem_attr(flows_tmem_kernel<P>, smem1);
    else
      return set_smem_attr(flows_kernel<P, NT>, smem1);
  }();
  static const cudaError_t attr2 = set_smem_attr(colour_rows_tc_kernel<P>, smem2);
  if (attr1 != cudaSuccess || attr2 != cudaSuccess) return -4;
  if (a.nevt <= 0 || a.nhel <= 0) return 0;
  const long long ldj = rows_ld(a.nevt);
  const long long hs = rows_slice(P::NCOL, a.nevt, a.nhel);
  float2* J = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&J), rows_workspace_bytes(P::NCOL, a.nevt, a.nhel), a.stream) !=
      cudaSuccess)
    return -4;
  if (a.marks) a.marks->mark(a.stream);
  for (int h0 = 0; h0 < a.nhel; h0 += (int)hs) {
    const int nh = a.nhel - h0 < hs ? a.nhel - h0 : (int)hs;
    if constexpr (tmem_flows)
      flows_tmem_kernel<P><<<(unsigned)((a.nevt + NT1 - 1) / NT1), NT1, smem1, a.stream>>>(
          a.mom, a.nevt, J, ldj, a.hels + h0, nh, a.kp, a.status);
    else
      flows_kernel<P, NT><<<(unsigned)((a.nevt + NT - 1) / NT), NT, smem1, a.stream>>>(
          a.mom, a.nevt, J, ldj, a.hels + h0, nh, a.kp, a.status);
    if (a.marks) a.marks->mark(a.stream);
    colour_rows_tc_kernel<P><<<(unsigned)(ldj / 128), 128, smem2, a.stream>>>(
        J, ldj, a.nevt, a.out, nh, h0 == 0, h0 + nh == a.nhel, static_cast<const uint4*>(a.ctile), a.status,
        a.kp.polls);
    if (a.marks) a.marks->mark(a.stream);
  }
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaFreeAsync(J, a.stream);
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? 0 : -4;
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
