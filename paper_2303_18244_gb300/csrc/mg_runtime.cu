// mg_runtime.cu -- the C ABI of include/mg.h: process handles, helicity
// filter, per-event ME launches from device or host buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "mg.h"
#include "mg_colour_tc.cuh"
#include "mg_kernels.cuh"
#include "mg_runtime_internal.h"

namespace mg {
// generated registry of the compiled processes (csrc/gen/registry.cu)
const ProcDesc* const* registry(int* n);

static const ProcDesc* find_process(const char* name) {
  int n = 0;
  const ProcDesc* const* all = registry(&n);
  for (int i = 0; i < n; i++)
    if (std::strcmp(all[i]->name, name) == 0) return all[i];
  return nullptr;
}
}  // namespace mg

using mg::KParams;
using mg::LaunchArgs;
using mg::ProcDesc;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int mg_params_default(mg_params* p) {
  if (!p) return MG_ERR_ARG;
  p->mt = 173.0;
  p->wt = 1.4915;
  p->alpha_s = 0.118;
  p->mz = 91.188;
  p->wz = 2.441404;
  p->alpha_em_inv = 132.507;
  p->gf = 1.16639e-5;
  p->precision = MG_FP64;
  p->flags = 0;
  return MG_OK;
}

// Couplings per process (standard model, G_F scheme for the electroweak sector).
static int make_kparams(const ProcDesc* d, const mg_params& p, KParams& kp) {
  std::memset(&kp, 0, sizeof(kp));
  kp.polls = mg::WAIT_POLLS;
  if (std::strcmp(d->tag, "eemumu") == 0) {
    if (!(p.alpha_em_inv > 0) || !(p.mz > 0) || !(p.wz >= 0) || !(p.gf > 0)) return MG_ERR_ARG;
    const double pi = 3.14159265358979323846;
    const double alpha = 1.0 / p.alpha_em_inv;
    const double e2 = 4.0 * pi * alpha;
    const double mz2 = p.mz * p.mz;
    const double disc = 0.25 * mz2 * mz2 - pi * alpha * mz2 / (std::sqrt(2.0) * p.gf);
    if (!(disc >= 0)) return MG_ERR_ARG;
    const double mw2 = 0.5 * mz2 + std::sqrt(disc);
    const double sw2 = 1.0 - mw2 / mz2;
    const double cw2 = 1.0 - sw2;
    kp.v[0] = e2;                                                   // photon: e^2 (Q_e Q_mu = 1)
    kp.v[1] = (p.flags & MG_PHOTON_ONLY) ? 0.0 : e2 / (sw2 * cw2);  // Z: (e / (sw cw))^2
    kp.v[2] = -0.5 + sw2;                                           // g_L = T3 - Q sw^2
    kp.v[3] = sw2;                                                  // g_R = -Q sw^2
    kp.v[4] = p.mz;
    kp.v[5] = p.wz;
  } else {
    if (!(p.alpha_s > 0) || !(p.mt > 0) || !(p.wt >= 0)) return MG_ERR_ARG;
    kp.v[0] = std::sqrt(4.0 * 3.14159265358979323846 * p.alpha_s);  // g_s
    kp.v[1] = p.mt;
    kp.v[2] = (p.flags & MG_NO_TOP_WIDTH) ? 0.0 : p.wt;
  }
  return MG_OK;
}

extern "C" int mg_process_create(const char* proc, const mg_params* p, mg_process** out) {
  if (!out) return MG_ERR_ARG;
  *out = nullptr;
  if (!proc || !p) return MG_ERR_ARG;
  const ProcDesc* d = mg::find_process(proc);
  if (!d) return MG_ERR_PROC;
  if (p->precision != MG_FP64 && p->precision != MG_MIXED && p->precision != MG_MIXED_PAPER &&
      p->precision != MG_FLOAT)
    return MG_ERR_ARG;
  KParams kp;
  int rc = make_kparams(d, *p, kp);
  if (rc) return rc;
  mg_process* h = new (std::nothrow) mg_process();
  if (!h) return MG_ERR_NOMEM;
  // a serial number that no later handle reuses, even at the same address
  // (the server keys its captured graphs by it)
  static std::atomic<uint64_t> next_serial{1};
  h->serial = next_serial.fetch_add(1);
  h->d = d;
  h->par = *p;
  h->kp = kp;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return MG_ERR_CUDA;
  }
  std::vector<int> all(d->nhel);
  for (int i = 0; i < d->nhel; i++) all[i] = i;
  h->mask.assign(d->nhel, 1);
  if (cudaMalloc(&h->d_hels, sizeof(int) * d->nhel) != cudaSuccess ||
      cudaMalloc(&h->d_status, sizeof(unsigned)) != cudaSuccess) {
    mg_process_destroy(h);
    return MG_ERR_NOMEM;
  }
  if (cudaMemcpy(h->d_hels, all.data(), sizeof(int) * d->nhel, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
    mg_process_destroy(h);
    return MG_ERR_CUDA;
  }
  h->n_good = d->nhel;
  if (p->precision == MG_MIXED && d->tc_k > 0) {
    // FP16 operand image of the colour matrix for the tensor-core colour sum
    std::vector<unsigned short> tile((size_t)d->tc_k * d->tc_k);
    if (!mg::colour_tile_host(d->knum, d->ncol, tile.data())) {
      mg_process_destroy(h);
      return MG_ERR_STATE;  // a colour numerator is not exact in FP16
    }
    if (cudaMalloc(&h->d_ctile, tile.size() * 2) != cudaSuccess) {
      mg_process_destroy(h);
      return MG_ERR_NOMEM;
    }
    if (cudaMemcpy(h->d_ctile, tile.data(), tile.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
      mg_process_destroy(h);
      return MG_ERR_CUDA;
    }
  }
  if (p->precision == MG_MIXED_PAPER) {
    // colour numerators for the FP32 colour sum: K_ii and 2 K_ij (j > i)
    std::vector<short> kt((size_t)d->ncol * d->ncol, 0);
    for (int i = 0; i < d->ncol; i++)
      for (int j = i; j < d->ncol; j++) kt[(size_t)i * d->ncol + j] = (short)(i == j ? d->knum[i * d->ncol + j]
                                                                                   : 2 * d->knum[i * d->ncol + j]);
    if (cudaMalloc(&h->d_ctile, kt.size() * sizeof(short)) != cudaSuccess) {
      mg_process_destroy(h);
      return MG_ERR_NOMEM;
    }
    if (cudaMemcpy(h->d_ctile, kt.data(), kt.size() * sizeof(short), cudaMemcpyHostToDevice) != cudaSuccess) {
      mg_process_destroy(h);
      return MG_ERR_CUDA;
    }
  }
  // one-time kernel attributes (no launch for nevt = 0), so that later calls
  // can be captured into CUDA graphs
  LaunchArgs a{};
  a.nevt = 0;
  if (d->sigma_fp64(a) || d->sigma_mixed(a) || d->helicities(a) || d->select_fp64(a) || d->select_mixed(a) ||
      d->sigma_paper(a) || d->sigma_float(a)) {
    mg_process_destroy(h);
    return MG_ERR_CUDA;
  }
  *out = h;
  return MG_OK;
}

extern "C" void mg_process_destroy(mg_process* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->d_hels);
  for (int* p : h->old_hels) cudaFree(p);
  cudaFree(h->d_status);
  cudaFree(h->d_ctile);
  cudaFree(h->d_mom);
  cudaFree(h->d_me);
  delete h;
}

extern "C" int mg_process_info(const mg_process* h, int* npar, int* n_hel, int* n_col, int* n_diag, double* iden) {
  if (!h) return MG_ERR_ARG;
  if (npar) *npar = h->d->npar;
  if (n_hel) *n_hel = h->d->nhel;
  if (n_col) *n_col = h->d->ncol;
  if (n_diag) *n_diag = h->d->ndiag;
  if (iden) *iden = h->d->iden;
  return MG_OK;
}

int mg_launch_sigma_locked(mg_process* h, const double* mom, int64_t nevt, double* me, cudaStream_t stream,
                           mg::PhaseMarks* marks) {
  LaunchArgs a{};
  a.marks = marks;
  a.mom = mom;
  a.nevt = nevt;
  a.out = me;
  a.hels = h->d_hels;
  a.nhel = h->n_good;
  a.kp = h->kp;
  a.ctile = h->d_ctile;
  a.status = h->d_status;
  a.stream = stream;
  const int rc = h->par.precision == MG_MIXED         ? h->d->sigma_mixed(a)
                 : h->par.precision == MG_MIXED_PAPER ? h->d->sigma_paper(a)
                 : h->par.precision == MG_FLOAT       ? h->d->sigma_float(a)
                                                      : h->d->sigma_fp64(a);
  return rc ? MG_ERR_CUDA : MG_OK;
}

int mg_launch_sigma(mg_process* h, const double* mom, int64_t nevt, double* me, cudaStream_t stream) {
  // the list and its length together (mg_good_helicities may replace them)
  std::lock_guard<std::mutex> lk(h->lock);
  return mg_launch_sigma_locked(h, mom, nevt, me, stream);
}

int64_t mg_workspace_bytes_locked(const mg_process* h, int64_t nevt) {
  if (h->par.precision != MG_MIXED || !h->d->rows_mixed) return 0;
  return (int64_t)mg::rows_workspace_bytes(h->d->ncol, nevt, h->n_good);
}

extern "C" int mg_sigma_workspace_bytes(mg_process* h, int64_t nevt, int64_t* bytes_out) {
  if (!h || nevt < 0 || !bytes_out) return MG_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->lock);
  *bytes_out = mg_workspace_bytes_locked(h, nevt);
  return MG_OK;
}

extern "C" int mg_sigma(mg_process* h, const double* momenta_dev, int64_t nevt, double* me_out_dev, void* stream) {
  if (!h || nevt < 0) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!momenta_dev || !me_out_dev || !aligned16(momenta_dev)) return MG_ERR_ARG;
  DeviceGuard g(h->device);
  return mg_launch_sigma(h, momenta_dev, nevt, me_out_dev, static_cast<cudaStream_t>(stream));
}

extern "C" int mg_sigma_select(mg_process* h, const double* momenta_dev, int64_t nevt, const double* rnd_dev,
                               double* me_out_dev, int* hel_out_dev, int* col_out_dev, double* colw_out_dev,
                               void* stream) {
  if (!h || nevt < 0) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!momenta_dev || !rnd_dev || !me_out_dev || !hel_out_dev || !col_out_dev || !aligned16(momenta_dev))
    return MG_ERR_ARG;
  DeviceGuard g(h->device);
  LaunchArgs a{};
  a.mom = momenta_dev;
  a.nevt = nevt;
  a.out = me_out_dev;
  a.kp = h->kp;
  a.status = h->d_status;
  a.stream = static_cast<cudaStream_t>(stream);
  a.rnd = rnd_dev;
  a.hel_out = hel_out_dev;
  a.col_out = col_out_dev;
  a.colw_out = colw_out_dev;
  // the list and its length together, up to the launch
  std::lock_guard<std::mutex> lk(h->lock);
  a.hels = h->d_hels;
  a.nhel = h->n_good;
  // the paper-style mode chooses from its FP64 amplitudes
  const bool fp32 = h->par.precision == MG_MIXED || h->par.precision == MG_FLOAT;
  const int rc = fp32 ? h->d->select_mixed(a) : h->d->select_fp64(a);
  return rc ? MG_ERR_CUDA : MG_OK;
}

extern "C" int mg_sigma_helicities(mg_process* h, const double* momenta_dev, int64_t nevt, double* out_dev,
                                   void* stream) {
  if (!h || nevt < 0) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!momenta_dev || !out_dev || !aligned16(momenta_dev)) return MG_ERR_ARG;
  DeviceGuard g(h->device);
  LaunchArgs a{};
  a.mom = momenta_dev;
  a.nevt = nevt;
  a.out = out_dev;
  a.kp = h->kp;
  a.status = h->d_status;
  a.stream = static_cast<cudaStream_t>(stream);
  return h->d->helicities(a) ? MG_ERR_CUDA : MG_OK;
}

static int read_status(mg_process* h) {
  unsigned st = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return MG_ERR_CUDA;
  if (cudaMemcpy(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return MG_ERR_CUDA;
  if (st) {
    cudaMemset(h->d_status, 0, sizeof(unsigned));
    cudaDeviceSynchronize();
    return MG_ERR_TIMEOUT;
  }
  return MG_OK;
}

extern "C" int mg_process_status(mg_process* h) {
  if (!h) return MG_ERR_ARG;
  DeviceGuard g(h->device);
  return read_status(h);
}

extern "C" int mg_good_helicities(mg_process* h, const double* momenta_dev, int64_t nevt, int* n_good_out,
                                  uint8_t* mask_host) {
  if (!h || nevt < 0) return MG_ERR_ARG;
  if (nevt > 0 && (!momenta_dev || !aligned16(momenta_dev))) return MG_ERR_ARG;
  DeviceGuard g(h->device);
  const int nhel = h->d->nhel;
  std::vector<uint8_t> mask(nhel, 1);
  if (nevt > 0) {
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(double) * nevt * nhel) != cudaSuccess) return MG_ERR_NOMEM;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaFree(tmp);
      return MG_ERR_CUDA;
    }
    int rc = mg_sigma_helicities(h, momenta_dev, nevt, tmp, s);
    std::vector<double> v;
    if (rc == MG_OK) {
      v.resize((size_t)nevt * nhel);
      if (cudaMemcpyAsync(v.data(), tmp, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        rc = MG_ERR_CUDA;
    }
    cudaStreamDestroy(s);
    cudaFree(tmp);
    if (rc == MG_OK) rc = read_status(h);
    if (rc) return rc;
    // h is kept iff max_events |M_h|^2 / sum_h' |M_h'|^2 > 1e-14
    std::vector<double> maxr(nhel, 0.0);
    for (int64_t e = 0; e < nevt; e++) {
      const double* row = v.data() + (size_t)e * nhel;
      double tot = 0.0;
      for (int k = 0; k < nhel; k++) tot += row[k];
      if (!(tot > 0.0)) continue;
      for (int k = 0; k < nhel; k++) {
        const double r = row[k] / tot;
        if (r > maxr[k]) maxr[k] = r;
      }
    }
    bool any = false;
    for (int k = 0; k < nhel; k++) {
      mask[k] = maxr[k] > 1e-14 ? 1 : 0;
      any |= mask[k] != 0;
    }
    // no event with a positive finite |M|^2: the set says nothing, keep all
    if (!any) std::fill(mask.begin(), mask.end(), 1);
  }
  std::vector<int> good;
  for (int k = 0; k < nhel; k++)
    if (mask[k]) good.push_back(k);
  {
    std::lock_guard<std::mutex> lk(h->lock);
    if (mask == h->mask) {  // unchanged: keep the list, its version and its graphs
      if (n_good_out) *n_good_out = h->n_good;
      if (mask_host) std::memcpy(mask_host, mask.data(), nhel);
      return MG_OK;
    }
  }
  int* nd = nullptr;
  if (cudaMalloc(&nd, sizeof(int) * nhel) != cudaSuccess) return MG_ERR_NOMEM;
  if (cudaMemcpy(nd, good.data(), sizeof(int) * good.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(nd);
    return MG_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lk(h->lock);
    // launches already queued, and graphs the caller captured, may still read
    // the previous list: keep it alive until the handle is destroyed
    h->old_hels.push_back(h->d_hels);
    h->d_hels = nd;
    h->n_good = (int)good.size();
    h->mask = mask;
    h->hel_version++;
  }
  if (n_good_out) *n_good_out = (int)good.size();
  if (mask_host) std::memcpy(mask_host, mask.data(), nhel);
  return MG_OK;
}

extern "C" int mg_sigma_host(mg_process* h, const double* momenta_host, int64_t nevt, double* me_out_host,
                             void* stream) {
  if (!h || nevt < 0) return MG_ERR_ARG;
  if (nevt == 0) return MG_OK;
  if (!momenta_host || !me_out_host) return MG_ERR_ARG;
  DeviceGuard g(h->device);
  std::lock_guard<std::mutex> lk(h->ws_lock);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t mbytes = sizeof(double) * (size_t)nevt * h->d->npar * 4;
  if (nevt > h->cap) {
    cudaStreamSynchronize(s);
    cudaFree(h->d_mom);
    cudaFree(h->d_me);
    h->d_mom = nullptr;
    h->d_me = nullptr;
    h->cap = 0;
    if (cudaMalloc(&h->d_mom, mbytes) != cudaSuccess || cudaMalloc(&h->d_me, sizeof(double) * nevt) != cudaSuccess)
      return MG_ERR_NOMEM;
    h->cap = nevt;
  }
  if (cudaMemcpyAsync(h->d_mom, momenta_host, mbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return MG_ERR_CUDA;
  int rc = mg_launch_sigma(h, h->d_mom, nevt, h->d_me, s);
  if (rc) return rc;
  if (cudaMemcpyAsync(me_out_host, h->d_me, sizeof(double) * nevt, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return MG_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}

extern "C" const char* mg_strerror(int code) {
  switch (code) {
    case MG_OK: return "ok";
    case MG_PENDING: return "pending";
    case MG_ERR_PROC: return "unknown process";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_NOMEM: return "out of memory or over budget";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_TIMEOUT: return "bounded wait timed out";
    case MG_ERR_STATE: return "invalid state";
    case MG_ERR_UNKNOWN_REQ: return "unknown request id";
    default: return "unknown error code";
  }
}
