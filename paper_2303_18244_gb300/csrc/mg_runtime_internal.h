// mg_runtime_internal.h -- the process handle shared by the runtime and the server.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "mg.h"
#include "mg_kernels.cuh"

struct mg_process {
  uint64_t serial = 0;              // unique per handle created in this process (never reused)
  const mg::ProcDesc* d = nullptr;
  mg_params par{};
  mg::KParams kp{};
  int device = 0;
  int* d_hels = nullptr;            // good helicity indices [n_good] (device)
  std::vector<int*> old_hels;       // superseded lists (queued launches and captured graphs may
                                    // still read them), freed at destroy
  int n_good = 0;
  unsigned hel_version = 0;         // bumped when the helicity list changes
  std::vector<uint8_t> mask;
  unsigned* d_status = nullptr;     // device status word (bounded-wait timeouts)
  void* d_ctile = nullptr;          // FP16 colour-matrix operand tile (mixed, tensor cores)
  std::mutex lock;
  // workspace of mg_sigma_host
  std::mutex ws_lock;
  double* d_mom = nullptr;
  double* d_me = nullptr;
  int64_t cap = 0;
};

// stream-ordered launch of the handle's sigma kernel (no argument checks);
// takes h->lock, so that the helicity list and its length are read together
int mg_launch_sigma(mg_process* h, const double* mom, int64_t nevt, double* me, cudaStream_t stream);
// the same with h->lock already held by the caller; marks (may be null)
// records an event before and after each kernel of a multi-kernel launch
int mg_launch_sigma_locked(mg_process* h, const double* mom, int64_t nevt, double* me, cudaStream_t stream,
                           mg::PhaseMarks* marks = nullptr);
// stream-ordered workspace bytes of one launch of nevt events (h->lock held)
int64_t mg_workspace_bytes_locked(const mg_process* h, int64_t nevt);
