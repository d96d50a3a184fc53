// mg_static.cu -- helicity filter that allocates no memory
// (mg_good_helicities_static in include/mg.h).
//
// The scratch of this entry point is one file-scope device array: per-event,
// per-helicity |M_h|^2 values followed by MG_STATIC_MAX_HEL reduction slots.
// Host code never dereferences the array's name (on the host it is only a
// stand-in symbol); the device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels as a plain pointer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "mg.h"
#include "mg_runtime_internal.h"

namespace {

__device__ __align__(256) double g_static_scratch[MG_STATIC_SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_addr_lock;
double* g_addr[MAX_DEVICES] = {};  // device address of g_static_scratch, per device

// max over events of |M_h|^2 / sum_h' |M_h'|^2; ratios are >= 0, so their
// IEEE bit patterns order like their values and a 64-bit atomicMax applies
__global__ void max_ratio_kernel(const double* __restrict__ v, long long nevt, int nhel,
                                 unsigned long long* __restrict__ slots) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nevt;
       e += (long long)gridDim.x * blockDim.x) {
    const double* row = v + e * nhel;
    double tot = 0.0;
    for (int k = 0; k < nhel; k++) tot += row[k];
    if (!(tot > 0.0)) continue;
    for (int k = 0; k < nhel; k++) {
      const double r = row[k] / tot;
      if (r > 0.0) atomicMax(slots + k, (unsigned long long)__double_as_longlong(r));
    }
  }
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// device address of the scratch array on device dev (looked up on first use)
double* scratch_address(int dev) {
  if (dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lk(g_addr_lock);
  if (!g_addr[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_static_scratch) != cudaSuccess) return nullptr;
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" int mg_good_helicities_static(mg_process* h, const double* momenta_dev, int64_t nevt, int* n_good_out,
                                         uint8_t* mask_host) {
  if (!h || nevt < 0) return MG_ERR_ARG;
  if (nevt > 0 && (!momenta_dev || (reinterpret_cast<uintptr_t>(momenta_dev) & 15u))) return MG_ERR_ARG;
  const int nhel = h->d->nhel;
  if (nhel > MG_STATIC_MAX_HEL) return MG_ERR_ARG;
  if (nevt > 0 && nevt > (int64_t)(MG_STATIC_SCRATCH_DOUBLES - MG_STATIC_MAX_HEL) / nhel) return MG_ERR_ARG;
  DevGuard g(h->device);
  uint8_t mask[MG_STATIC_MAX_HEL];
  for (int k = 0; k < nhel; k++) mask[k] = 1;
  if (nevt > 0) {
    double* vals = scratch_address(h->device);  // set-up: first call on this device
    if (!vals) return MG_ERR_CUDA;
    unsigned long long* slots =
        reinterpret_cast<unsigned long long*>(vals + (MG_STATIC_SCRATCH_DOUBLES - MG_STATIC_MAX_HEL));
    // the helicity list is rewritten in place below: nothing of this handle may be in flight
    if (cudaDeviceSynchronize() != cudaSuccess) return MG_ERR_CUDA;
    // the array keeps the previous call's contents: the reduction slots start at zero
    if (cudaMemsetAsync(slots, 0, sizeof(unsigned long long) * nhel, 0) != cudaSuccess) return MG_ERR_CUDA;
    mg::LaunchArgs a{};
    a.mom = momenta_dev;
    a.nevt = nevt;
    a.out = vals;
    a.kp = h->kp;
    a.status = h->d_status;
    a.stream = 0;
    if (h->d->helicities(a)) return MG_ERR_CUDA;
    const int blocks = (int)std::min<int64_t>((nevt + 255) / 256, 1024);
    max_ratio_kernel<<<blocks, 256, 0, 0>>>(vals, nevt, nhel, slots);
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
    unsigned long long res[MG_STATIC_MAX_HEL];
    if (cudaMemcpy(res, slots, sizeof(unsigned long long) * nhel, cudaMemcpyDeviceToHost) != cudaSuccess)
      return MG_ERR_CUDA;
    unsigned st = 0;
    if (cudaMemcpy(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
    if (st) {
      cudaMemset(h->d_status, 0, sizeof(unsigned));
      return MG_ERR_TIMEOUT;
    }
    bool any = false;
    for (int k = 0; k < nhel; k++) {
      double r;
      std::memcpy(&r, &res[k], sizeof(r));
      mask[k] = r > 1e-14 ? 1 : 0;
      any |= mask[k] != 0;
    }
    // no event with a positive finite |M|^2: the set says nothing, keep all
    if (!any)
      for (int k = 0; k < nhel; k++) mask[k] = 1;
  }
  int good[MG_STATIC_MAX_HEL];
  int n = 0;
  for (int k = 0; k < nhel; k++)
    if (mask[k]) good[n++] = k;
  {
    // the handle's list has room for every helicity: overwrite it in place,
    // under the lock, so that the list and its length change together
    std::lock_guard<std::mutex> lk(h->lock);
    if (cudaMemcpy(h->d_hels, good, sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess) return MG_ERR_CUDA;
    h->n_good = n;
    std::copy(mask, mask + nhel, h->mask.begin());
    h->hel_version++;
  }
  if (n_good_out) *n_good_out = n;
  if (mask_host)
    for (int k = 0; k < nhel; k++) mask_host[k] = mask[k];
  return MG_OK;
}
