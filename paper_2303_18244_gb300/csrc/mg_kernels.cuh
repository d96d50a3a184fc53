// mg_kernels.cuh -- kernel templates of the matrix-element hot path.
//
// One event per thread, lockstep across the warp (paper Sect. 1: data
// parallelism with lockstep processing over the events of a batch):
//   A1  the CTA's momenta tile (NT events x NPAR x 4 doubles, contiguous) is
//       copied global -> shared by the TMA engine (cp.async.bulk, completion
//       on an mbarrier with a bounded wait);
//   A2  per event, once, in FP64: external-state ingredients and every
//       propagator coefficient -g/P^2, -g/(P^2 - m^2 + i m Gamma) -- these
//       depend on the momenta only, so they are hoisted out of the helicity
//       loop and kept in a per-thread shared-memory slab [slot][thread];
//   A3-A4  per good helicity (uniform across the CTA): wavefunctions,
//       off-shell currents and amplitudes diagram by diagram, accumulated
//       into the colour flows (generated straight-line code);
//   A5  colour quadratic form J^dagger C J (FP64 FMA in the FP64 path; on
//       the tensor cores in the mixed path, see mg_colour_tc.cuh);
//   A6  helicity sum in FP64, normalised by 1/(IDEN * CDEN), one store.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_vertices.cuh"

namespace mg {

struct KParams {
  double v[8];
  uint32_t polls;  // bound of the first wait on each device barrier (the drain after a timeout uses WAIT_POLLS)
};

// status bits written by kernels
enum : unsigned { ST_TMA_TIMEOUT = 1u, ST_MMA_TIMEOUT = 2u };

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy primitives (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after max_iter polls (each poll may itself suspend
// for a short hardware-defined time).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
  for (uint32_t i = 0; i < max_iter; i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy (TMA engine), completion counted on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

constexpr uint32_t WAIT_POLLS = 1u << 22;

// ---------------------------------------------------------------------------
// shared-memory layout:
//   [mbarriers 128 B][momenta tile][per-thread slab [NSLOT][NT]][colour flows [NCOL][NT]]
// Each thread reads and writes only its own column of the slab and of the
// colour-flow accumulators, so the helicity loop needs no block barrier.
// ---------------------------------------------------------------------------
// slab slots kept per thread (the lean layout drops the external-state
// ingredients, which the FP32 code then recomputes per helicity)
template <class P, typename R>
constexpr int slab_slots() {
  return (sizeof(R) == 4 && P::LEAN_SLAB) ? P::NSLOT_LEAN : P::NSLOT;
}

template <class P, typename R, int NT>
struct Layout {
  static constexpr size_t bar_bytes = 128;
  static constexpr size_t stage_bytes = size_t(NT) * P::NPAR * 4 * sizeof(double);
  static constexpr size_t slab_bytes = size_t(NT) * slab_slots<P, R>() * sizeof(R);
  static constexpr size_t jamp_bytes = size_t(NT) * P::NCOL * sizeof(cx<R>);
  static constexpr size_t slab_off = bar_bytes;
  static constexpr size_t jamp_off = slab_off + ((slab_bytes + 127) / 128) * 128;
  // the momenta tile is staged in the colour-flow space: only prepare reads
  // it, and a block barrier separates that from the first flow update
  static constexpr size_t stage_off = jamp_off;
  static constexpr size_t union_bytes = stage_bytes > jamp_bytes ? stage_bytes : jamp_bytes;
  static constexpr size_t base_bytes = jamp_off + ((union_bytes + 127) / 128) * 128;
};

// A1 + A2: stage the tile, run the per-event set-up (arithmetic type D: FP64,
// or FP32 in the all-float mode) into the slab.  Returns the number of valid
// events in the tile, or -1 after a timed-out copy (uniformly for the whole
// CTA).
template <class P, typename R, int NT, typename D = double>
__device__ __forceinline__ int load_and_prepare_at(uint64_t* bar, double* stage, R* slab,
                                                   const double* __restrict__ mom, long long nevt,
                                                   const KParams& kp, unsigned* status) {
  const int tid = threadIdx.x;
  const long long e0 = (long long)blockIdx.x * NT;
  const long long rem = nevt - e0;
  const int nvalid = rem < NT ? (int)rem : NT;
  const uint32_t bytes = (uint32_t)nvalid * P::NPAR * 4 * sizeof(double);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(stage, mom + e0 * P::NPAR * 4, bytes, bar);
  }
  __syncthreads();
  // the outcome of the bounded wait is made uniform across the CTA
  if (!__syncthreads_and(mbar_wait_bounded(bar, 0, kp.polls) ? 1 : 0)) {
    // the copy did not complete: flag it, wait once more (bounded, full
    // length) so that no copy is left in flight into this CTA's shared
    // memory, and give up
    if (tid == 0) atomicOr(status, ST_TMA_TIMEOUT);
    mbar_wait_bounded(bar, 0, WAIT_POLLS);
    return -1;
  }
  const int le = tid < nvalid ? tid : nvalid - 1;  // ragged tail: repeat a valid event
  P::template prepare<R, D>(stage + le * P::NPAR * 4, kp.v, slab + tid, NT);
  __syncthreads();  // every thread is done with the momenta tile (its space is reused)
  return nvalid;
}

template <class P, typename R, int NT, typename D = double>
__device__ __forceinline__ int load_and_prepare(unsigned char* smem, const double* __restrict__ mom, long long nevt,
                                                const KParams& kp, unsigned* status) {
  using LY = Layout<P, R, NT>;
  return load_and_prepare_at<P, R, NT, D>(reinterpret_cast<uint64_t*>(smem),
                                       reinterpret_cast<double*>(smem + LY::stage_off),
                                       reinterpret_cast<R*>(smem + LY::slab_off), mom, nevt, kp, status);
}

// ---------------------------------------------------------------------------
// |M|^2 with the CUDA-core colour sum (FP64 path; small processes in mixed;
// the all-float mode with D = A = float: FP32 set-up and helicity sum)
// ---------------------------------------------------------------------------
template <class P, typename R, int NT, typename D = double, typename A = double>
__global__ void __launch_bounds__(NT) sigma_kernel(const double* __restrict__ mom, long long nevt,
                                                   double* __restrict__ me, const int* __restrict__ hels,
                                                   int nhel, KParams kp, unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  using LY = Layout<P, R, NT>;
  const int nvalid = load_and_prepare<P, R, NT, D>(smem, mom, nevt, kp, status);
  if (nvalid < 0) return;
  const R* ev = reinterpret_cast<const R*>(smem + LY::slab_off) + threadIdx.x;
  cx<R>* jamp = reinterpret_cast<cx<R>*>(smem + LY::jamp_off) + threadIdx.x;
  A acc = A(0);
#pragma unroll 1
  for (int ih = 0; ih < nhel; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes<R>(ev, NT, h, kp.v, jamp, NT);
    acc += (A)P::template colour_quadratic<R>(jamp, NT);
  }
  if ((int)threadIdx.x < nvalid) {
    constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
    me[(long long)blockIdx.x * NT + threadIdx.x] = (double)(acc * A(norm));
  }
}

// First phase of the two-phase mixed path (processes whose colour operands do
// not fit in shared memory next to the per-event state): the FP32 colour flows
// of every (good helicity, event) row, written to J[(ih * NCOL + k) * ldj + e]
// (e: event index within the launch, ldj >= the launch's events rounded up to
// NT; consecutive events adjacent, so the stores coalesce).  The ragged tail's
// threads repeat a valid event and write their own (padding) rows.  The
// colour quadratic form of these rows is the second phase
// (colour_rows_tc_kernel).
template <class P, int NT>
__global__ void __launch_bounds__(NT) flows_kernel(const double* __restrict__ mom, long long nevt,
                                                   float2* __restrict__ J, long long ldj,
                                                   const int* __restrict__ hels, int nhel, KParams kp,
                                                   unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  using LY = Layout<P, float, NT>;
  const int nvalid = load_and_prepare<P, float, NT>(smem, mom, nevt, kp, status);
  if (nvalid < 0) return;
  const float* ev = reinterpret_cast<const float*>(smem + LY::slab_off) + threadIdx.x;
  cx<float>* jamp = reinterpret_cast<cx<float>*>(smem + LY::jamp_off) + threadIdx.x;
  const long long e = (long long)blockIdx.x * NT + threadIdx.x;
#pragma unroll 1
  for (int ih = 0; ih < nhel; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes<float>(ev, NT, h, kp.v, jamp, NT);
    float2* row = J + (long long)ih * P::NCOL * ldj + e;
#pragma unroll 4
    for (int k = 0; k < P::NCOL; k++) row[(long long)k * ldj] = make_float2(jamp[k * NT].re, jamp[k * NT].im);
  }
}

// |M|^2 plus the event-by-event random choice of a helicity and a leading
// colour flow for unweighted events (paper Sect. 5: the last ingredient needed
// by the event files).  rnd[e] = (r_hel, r_col) in [0, 1):
//   helicity: the good helicity h_i with the smallest i whose cumulative
//             |M_h|^2 (good list order) exceeds r_hel * sum;
//   colour:   the flow k with the smallest k whose cumulative weight
//             w_k = sum_h |J_k(h)|^2 exceeds r_col * sum_k w_k.
// Colour sum on the CUDA cores in both precisions; optional per-flow weights.
template <class P, typename R, int NT>
__global__ void __launch_bounds__(NT)
    select_kernel(const double* __restrict__ mom, long long nevt, const double* __restrict__ rnd,
                  double* __restrict__ me, int* __restrict__ hel_out, int* __restrict__ col_out,
                  double* __restrict__ colw_out, const int* __restrict__ hels, int nhel, KParams kp,
                  unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  using LY = Layout<P, R, NT>;
  const int nvalid = load_and_prepare<P, R, NT>(smem, mom, nevt, kp, status);
  if (nvalid < 0) return;
  const R* ev = reinterpret_cast<const R*>(smem + LY::slab_off) + threadIdx.x;
  cx<R>* jamp = reinterpret_cast<cx<R>*>(smem + LY::jamp_off) + threadIdx.x;
  double mh[P::NHEL];
  double w[P::NCOL];
  for (int k = 0; k < P::NCOL; k++) w[k] = 0.0;
  double acc = 0.0;
#pragma unroll 1
  for (int ih = 0; ih < nhel; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes<R>(ev, NT, h, kp.v, jamp, NT);
    const double v = (double)P::template colour_quadratic<R>(jamp, NT);
    mh[ih] = v;
    acc += v;
    for (int k = 0; k < P::NCOL; k++) {
      const cx<R> j = jamp[k * NT];
      w[k] += (double)j.re * (double)j.re + (double)j.im * (double)j.im;
    }
  }
  if ((int)threadIdx.x >= nvalid) return;
  const long long e = (long long)blockIdx.x * NT + threadIdx.x;
  constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
  me[e] = acc * norm;
  const double rh = rnd[2 * e], rc = rnd[2 * e + 1];
  int sel = -1, last = 0;
  double cum = 0.0;
  const double th = rh * acc;
  for (int ih = 0; ih < nhel; ih++) {
    if (mh[ih] > 0.0) last = ih;
    cum += mh[ih];
    if (sel < 0 && cum > th && mh[ih] > 0.0) sel = ih;
  }
  hel_out[e] = __ldg(hels + (sel < 0 ? last : sel));
  double wt = 0.0;
  for (int k = 0; k < P::NCOL; k++) wt += w[k];
  const double tc = rc * wt;
  int ksel = -1, klast = 0;
  cum = 0.0;
  for (int k = 0; k < P::NCOL; k++) {
    if (w[k] > 0.0) klast = k;
    cum += w[k];
    if (ksel < 0 && cum > tc && w[k] > 0.0) ksel = k;
  }
  col_out[e] = ksel < 0 ? klast : ksel;
  if (colw_out)
    for (int k = 0; k < P::NCOL; k++) colw_out[e * P::NCOL + k] = w[k];
}

// The paper's own "mixed" mode (Sect. 3): Feynman diagrams and colour flows
// in FP64, the colour quadratic form in FP32 (colour numerators from a device
// table knum[NCOL][NCOL], upper triangle doubled), helicity sum in FP64.
template <class P, int NT>
__global__ void __launch_bounds__(NT)
    sigma_paper_kernel(const double* __restrict__ mom, long long nevt, double* __restrict__ me,
                       const int* __restrict__ hels, int nhel, KParams kp, const short* __restrict__ knum,
                       unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  using LY = Layout<P, double, NT>;
  const int nvalid = load_and_prepare<P, double, NT>(smem, mom, nevt, kp, status);
  if (nvalid < 0) return;
  const double* ev = reinterpret_cast<const double*>(smem + LY::slab_off) + threadIdx.x;
  cx<double>* jamp = reinterpret_cast<cx<double>*>(smem + LY::jamp_off) + threadIdx.x;
  double acc = 0.0;
#pragma unroll 1
  for (int ih = 0; ih < nhel; ih++) {
    const int h = __ldg(hels + ih);
    P::template amplitudes<double>(ev, NT, h, kp.v, jamp, NT);
    float q = 0.f;
#pragma unroll 1
    for (int i = 0; i < P::NCOL; i++) {
      const float jr = (float)jamp[i * NT].re, ji = (float)jamp[i * NT].im;
      float yr = 0.f, yi = 0.f;
      for (int j = i; j < P::NCOL; j++) {
        const float k = (float)__ldg(knum + i * P::NCOL + j);
        yr = fmaf(k, (float)jamp[j * NT].re, yr);
        yi = fmaf(k, (float)jamp[j * NT].im, yi);
      }
      q = fmaf(jr, yr, q);
      q = fmaf(ji, yi, q);
    }
    acc += (double)q;
  }
  if ((int)threadIdx.x < nvalid) {
    constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
    me[(long long)blockIdx.x * NT + threadIdx.x] = acc * norm;
  }
}

// Per-helicity |M_h|^2 / IDEN for every helicity, FP64 (helicity filter).
template <class P, int NT>
__global__ void __launch_bounds__(NT) helicity_kernel(const double* __restrict__ mom, long long nevt,
                                                      double* __restrict__ out, KParams kp,
                                                      unsigned* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  using LY = Layout<P, double, NT>;
  const int nvalid = load_and_prepare<P, double, NT>(smem, mom, nevt, kp, status);
  if (nvalid < 0) return;
  const double* ev = reinterpret_cast<const double*>(smem + LY::slab_off) + threadIdx.x;
  cx<double>* jamp = reinterpret_cast<cx<double>*>(smem + LY::jamp_off) + threadIdx.x;
  const long long e = (long long)blockIdx.x * NT + threadIdx.x;
  constexpr double norm = 1.0 / (P::IDEN * P::CDEN);
#pragma unroll 1
  for (int h = 0; h < P::NHEL; h++) {
    P::template amplitudes<double>(ev, NT, h, kp.v, jamp, NT);
    const double v = P::template colour_quadratic<double>(jamp, NT) * norm;
    if ((int)threadIdx.x < nvalid) out[e * P::NHEL + h] = v;
  }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
struct LaunchArgs {
  const double* mom;
  long long nevt;
  double* out;
  const int* hels;
  int nhel;
  KParams kp;
  const void* ctile;  // FP16 colour-matrix operand tile (tensor-core path)
  unsigned* status;
  cudaStream_t stream;
  // event-by-event helicity and colour choice (select kernels only)
  const double* rnd;
  int* hel_out;
  int* col_out;
  double* colw_out;
  // diagnostics (may be null): events recorded on the stream before the first
  // and after every kernel of a multi-kernel launch
  struct PhaseMarks* marks;
};

struct PhaseMarks {
  static constexpr int MAX = 257;
  cudaEvent_t ev[MAX];
  int n = 0;
  void mark(cudaStream_t s) {
    if (n < MAX) cudaEventRecord(ev[n++], s);
  }
};

template <class K>
inline cudaError_t set_smem_attr(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class P, typename R, int NT, typename D = double, typename A = double>
int launch_sigma(const LaunchArgs& a) {
  constexpr size_t smem = Layout<P, R, NT>::base_bytes;
  static const cudaError_t attr = set_smem_attr(sigma_kernel<P, R, NT, D, A>, smem);
  if (attr != cudaSuccess) return -4;
  if (a.nevt <= 0) return 0;  // attribute set-up only
  const long long grid = (a.nevt + NT - 1) / NT;
  sigma_kernel<P, R, NT, D, A><<<(unsigned)grid, NT, smem, a.stream>>>(a.mom, a.nevt, a.out, a.hels, a.nhel,
                                                                        a.kp, a.status);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <class P, typename R, int NT>
int launch_select(const LaunchArgs& a) {
  constexpr size_t smem = Layout<P, R, NT>::base_bytes;
  static const cudaError_t attr = set_smem_attr(select_kernel<P, R, NT>, smem);
  if (attr != cudaSuccess) return -4;
  if (a.nevt <= 0) return 0;
  const long long grid = (a.nevt + NT - 1) / NT;
  select_kernel<P, R, NT><<<(unsigned)grid, NT, smem, a.stream>>>(a.mom, a.nevt, a.rnd, a.out, a.hel_out, a.col_out,
                                                                   a.colw_out, a.hels, a.nhel, a.kp, a.status);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <class P, int NT>
int launch_sigma_paper(const LaunchArgs& a) {
  constexpr size_t smem = Layout<P, double, NT>::base_bytes;
  static const cudaError_t attr = set_smem_attr(sigma_paper_kernel<P, NT>, smem);
  if (attr != cudaSuccess) return -4;
  if (a.nevt <= 0) return 0;
  const long long grid = (a.nevt + NT - 1) / NT;
  sigma_paper_kernel<P, NT><<<(unsigned)grid, NT, smem, a.stream>>>(a.mom, a.nevt, a.out, a.hels, a.nhel, a.kp,
                                                                     static_cast<const short*>(a.ctile), a.status);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <class P, int NT>
int launch_helicities(const LaunchArgs& a) {
  constexpr size_t smem = Layout<P, double, NT>::base_bytes;
  static const cudaError_t attr = set_smem_attr(helicity_kernel<P, NT>, smem);
  if (attr != cudaSuccess) return -4;
  if (a.nevt <= 0) return 0;  // attribute set-up only
  const long long grid = (a.nevt + NT - 1) / NT;
  helicity_kernel<P, NT><<<(unsigned)grid, NT, smem, a.stream>>>(a.mom, a.nevt, a.out, a.kp, a.status);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

// process descriptor exported by each generated translation unit
struct ProcDesc {
  const char* name;
  const char* tag;
  int npar, nhel, ncol, ndiag, namp;
  double iden;
  int cden;
  const int* knum;  // [ncol * ncol], C = knum / cden
  int (*sigma_fp64)(const LaunchArgs&);
  int (*sigma_mixed)(const LaunchArgs&);
  int (*helicities)(const LaunchArgs&);
  int tc_k;  // > 0: the mixed path contracts colour on the tensor cores, K = N = tc_k
  int (*select_fp64)(const LaunchArgs&);
  int (*select_mixed)(const LaunchArgs&);
  int (*sigma_paper)(const LaunchArgs&);
  int (*sigma_float)(const LaunchArgs&);  // all-float mode
  int rows_mixed;  // 1: the mixed path runs in two phases through a stream-ordered HBM workspace
};

}  // namespace mg
