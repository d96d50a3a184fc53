// mg_phasespace.cu -- flat phase-space momenta generated on the device
// (mg_rambo in include/mg.h).
//
// The paper (Sect. 2) identifies the host-side random-number -> momenta step
// of the event generator as the next serial part to move to the GPU once the
// matrix elements are fast.  This kernel produces the same event stream as
// the host input module: Philox4x64-10 (Salmon et al., SC'11) with key
// (seed, 0) and counter (event, final-state slot, 0, 0), uniforms
// ((w >> 11) + 0.5) 2^-53, then RAMBO (Kleiss, Stirling, Ellis 1986) at fixed
// sqrt(s): isotropic massless momenta, conformal map to the centre-of-mass
// frame, removal of the residual 3-momentum, and the common 3-momentum scale
// that puts every final state on its mass shell.  One event per thread.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "mg.h"
#include "mg_runtime_internal.h"

namespace {

constexpr int MAX_FINAL = 5;

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; r++) {
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

__device__ __forceinline__ double to_unit(uint64_t w) {
  return ((double)(w >> 11) + 0.5) * 0x1.0p-53;
}

struct PSArgs {
  double sqrt_s;
  uint64_t seed;
  long long first_event, nevt;
  int nf;
  double mass[MAX_FINAL];
};

__global__ void __launch_bounds__(128) rambo_kernel(PSArgs a, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= a.nevt) return;
  const long long ev = a.first_event + i;
  const int nf = a.nf;
  double q[MAX_FINAL][4];
  for (int j = 0; j < nf; j++) {
    uint64_t c[4] = {(uint64_t)ev, (uint64_t)j, 0ull, 0ull};
    philox4x64_10(c, a.seed, 0ull);
    const double u0 = to_unit(c[0]), u1 = to_unit(c[1]), u2 = to_unit(c[2]), u3 = to_unit(c[3]);
    const double ct = 2.0 * u0 - 1.0;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double phi = 2.0 * 3.14159265358979323846 * u1;
    const double q0 = -log(u2 * u3);
    q[j][0] = q0;
    q[j][1] = q0 * st * cos(phi);
    q[j][2] = q0 * st * sin(phi);
    q[j][3] = q0 * ct;
  }
  double Q[4] = {0, 0, 0, 0};
  for (int j = 0; j < nf; j++)
    for (int mu = 0; mu < 4; mu++) Q[mu] += q[j][mu];
  const double M = sqrt(Q[0] * Q[0] - (Q[1] * Q[1] + Q[2] * Q[2] + Q[3] * Q[3]));
  const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  const double gam = Q[0] / M;
  const double aa = 1.0 / (1.0 + gam);
  const double x = a.sqrt_s / M;
  double p[MAX_FINAL][4];
  for (int j = 0; j < nf; j++) {
    const double bq = b[0] * q[j][1] + b[1] * q[j][2] + b[2] * q[j][3];
    p[j][0] = x * (gam * q[j][0] + bq);
    for (int k = 0; k < 3; k++) p[j][k + 1] = x * (q[j][k + 1] + b[k] * q[j][0] + aa * bq * b[k]);
  }
  // residual 3-momentum of the map removed evenly
  double R3[3] = {0, 0, 0};
  for (int j = 0; j < nf; j++)
    for (int k = 0; k < 3; k++) R3[k] += p[j][k + 1];
  for (int j = 0; j < nf; j++)
    for (int k = 0; k < 3; k++) p[j][k + 1] -= R3[k] / nf;
  // common 3-momentum scale xi onto the mass shells (Newton)
  double p3sq[MAX_FINAL], msum = 0.0;
  for (int j = 0; j < nf; j++) {
    p3sq[j] = p[j][1] * p[j][1] + p[j][2] * p[j][2] + p[j][3] * p[j][3];
    msum += a.mass[j];
  }
  double xi = sqrt(1.0 - (msum / a.sqrt_s) * (msum / a.sqrt_s));
  for (int it = 0; it < 60; it++) {
    double f = -a.sqrt_s, df = 0.0;
    for (int j = 0; j < nf; j++) {
      const double e = sqrt(a.mass[j] * a.mass[j] + xi * xi * p3sq[j]);
      f += e;
      df += xi * p3sq[j] / e;
    }
    const double step = f / df;
    xi -= step;
    if (fabs(step) <= 1e-16 * fabs(xi)) break;
  }
  double* o = out + i * (long long)(nf + 2) * 4;
  const double E = 0.5 * a.sqrt_s;
  o[0] = E; o[1] = 0.0; o[2] = 0.0; o[3] = E;
  o[4] = E; o[5] = 0.0; o[6] = 0.0; o[7] = -E;
  for (int j = 0; j < nf; j++) {
    double* t = o + 8 + 4 * j;
    t[1] = p[j][1] * xi;
    t[2] = p[j][2] * xi;
    t[3] = p[j][3] * xi;
    t[0] = sqrt(a.mass[j] * a.mass[j] + xi * xi * p3sq[j]);
  }
}

}  // namespace

extern "C" int mg_rambo(const mg_process* h, double sqrt_s, uint64_t seed, int64_t first_event, int64_t nevt,
                        double* momenta_dev, void* stream) {
  if (!h || nevt < 0 || first_event < 0 || !(sqrt_s > 0)) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!momenta_dev) return MG_ERR_ARG;
  PSArgs a{};
  a.sqrt_s = sqrt_s;
  a.seed = seed;
  a.first_event = first_event;
  a.nevt = nevt;
  a.nf = h->d->npar - 2;
  if (a.nf < 2 || a.nf > MAX_FINAL) return MG_ERR_ARG;
  // final-state masses: the top pair of g g -> t t~ (+ gluons); massless leptons
  const bool tops = std::strcmp(h->d->tag, "eemumu") != 0;
  for (int j = 0; j < a.nf; j++) a.mass[j] = (tops && j < 2) ? h->par.mt : 0.0;
  double msum = 0.0;
  for (int j = 0; j < a.nf; j++) msum += a.mass[j];
  if (msum >= sqrt_s) return MG_ERR_ARG;
  int prev = -1, dev = h->device;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  const long long grid = (nevt + 127) / 128;
  rambo_kernel<<<(unsigned)grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(a, momenta_dev);
  const cudaError_t e = cudaGetLastError();
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  return e == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
