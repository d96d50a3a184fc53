// mg_server.cu -- persistent request loop with continuous batching on one GPU.
//
// The paper (Sect. 2, Fig. 1) runs several host processes against one GPU and
// finds that their matrix-element launches interleave and raise the combined
// throughput.  Here one scheduler thread plays that role for many clients:
//   - requests (process handle, momenta in host or device memory, event
//     count) wait in a FIFO;
//   - a request is split into chunks of at most max_bucket events; each chunk
//     is padded up to a power-of-two shape bucket (padding repeats the chunk's
//     first event; padded results are discarded);
//   - a chunk is admitted to one of n_streams device slots when a slot is free
//     and the in-flight device bytes -- the chunk's momenta and results plus
//     the stream-ordered workspace its launch takes (the two-phase
//     g g > t t~ g g g mixed path) -- stay within mem_budget_bytes (a chunk
//     larger than the budget on its own runs when nothing else is in flight);
//   - per slot: host momenta are copied into the slot's pinned staging buffer
//     and sent with an asynchronous copy (device momenta: a device copy), the
//     padding kernel runs, the sigma launch is replayed from a CUDA graph
//     captured once per (slot, process handle, bucket, helicity list) -- the
//     handle by its serial number, never reused, so a graph is never replayed
//     for a later handle that reuses a destroyed one's address -- and the
//     results go back through pinned staging; a completion event closes it;
//   - the scheduler holds the server mutex only for queue and request
//     bookkeeping: host copies, launches and graph captures run outside it, so
//     submit and poll never wait for them, and every device copy is
//     asynchronous, so chunks on different slots overlap on the device;
//   - completions are observed by polling the slots' events; a request is done
//     when its last chunk is.
// The process constants, helicity lists and colour data stay resident in the
// process handles; slot buffers and staging are allocated at server creation.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "mg.h"
#include "mg_runtime_internal.h"

namespace {

__global__ void pad_events(double* __restrict__ mom, int row, long long n, long long bucket) {
  const long long total = (bucket - n) * row;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    mom[n * row + i] = mom[i % row];
}

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  mg_process* h = nullptr;
  const double* mom = nullptr;
  double* me = nullptr;
  bool mom_dev = false, me_dev = false;  // buffers in device memory
  int64_t nevt = 0;
  int64_t padded = 0;
  int chunks_left = 0;
  int status = MG_PENDING;
  bool done = false;
  double submit_us = 0, start_us = -1, done_us = 0;
};

struct Chunk {
  Request* req;
  int64_t off, n, bucket;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  double* d_mom = nullptr;
  double* d_me = nullptr;
  double* h_mom = nullptr;  // pinned staging of host momenta
  double* h_me = nullptr;   // pinned staging of host results
  bool busy = false;
  Chunk cur{};
  int64_t bytes = 0;
};

constexpr int MAX_NPAR = 7;

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // unregistered host memory on older runtimes: clear the error
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct mg_server {
  mg_server_cfg cfg{};
  int device = 0;
  std::vector<Slot> slots;  // touched by the scheduler thread only
  std::map<std::tuple<int, uint64_t, int64_t, unsigned>, cudaGraphExec_t> graphs;  // scheduler thread only
  int64_t inflight = 0;                                                            // scheduler thread only
  // shared with submit/poll, under m
  std::mutex m;
  std::deque<Chunk> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_id = 1;
  std::thread th;
  Clock::time_point t0 = Clock::now();

  double now_us() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }
  void run();
  int admit(int si, const Chunk& c);
  void finish_chunk(Request* r, int rc);  // under m
};

static int64_t bucket_for(const mg_server_cfg& c, int64_t n) {
  int64_t b = c.min_bucket;
  while (b < n) b <<= 1;
  return std::min(b, c.max_bucket);
}

// device bytes a chunk holds while in flight: momenta and results of its
// bucket, and the workspace of its launch
static int64_t chunk_bytes(mg_process* h, int64_t bucket) {
  int64_t ws;
  {
    std::lock_guard<std::mutex> lk(h->lock);
    ws = mg_workspace_bytes_locked(h, bucket);
  }
  return bucket * (h->d->npar * 32 + 8) + ws;
}

void mg_server::finish_chunk(Request* r, int rc) {
  if (rc != MG_OK && r->status == MG_PENDING) r->status = rc;
  if (--r->chunks_left == 0) {
    if (r->status == MG_PENDING) r->status = MG_OK;
    r->done = true;
    r->done_us = now_us();
    cv_done.notify_all();
  }
}

// Runs on the scheduler thread without the server mutex.
int mg_server::admit(int si, const Chunk& c) {
  Slot& s = slots[si];
  mg_process* h = c.req->h;
  const int row = h->d->npar * 4;
  const size_t in_bytes = sizeof(double) * c.n * row;
  const double* src = c.req->mom + c.off * row;
  if (c.req->mom_dev) {
    if (cudaMemcpyAsync(s.d_mom, src, in_bytes, cudaMemcpyDeviceToDevice, s.stream) != cudaSuccess)
      return MG_ERR_CUDA;
  } else {
    std::memcpy(s.h_mom, src, in_bytes);  // the slot is idle: its staging is free
    if (cudaMemcpyAsync(s.d_mom, s.h_mom, in_bytes, cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
      return MG_ERR_CUDA;
  }
  if (c.bucket > c.n) {
    const long long total = (c.bucket - c.n) * row;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 1024);
    pad_events<<<blocks, 256, 0, s.stream>>>(s.d_mom, row, c.n, c.bucket);
    if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  }
  if (cfg.use_graphs) {
    // the handle's lock from the helicity-list version to the launch: the
    // graph and the list it reads belong together
    std::lock_guard<std::mutex> lk(h->lock);
    auto key = std::make_tuple(si, h->serial, c.bucket, h->hel_version);
    auto it = graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it == graphs.end()) {
      // A capture fails when another thread synchronises the whole device
      // meanwhile (a device-wide wait cannot wait on a capturing stream):
      // then this chunk is launched directly and the capture is tried again
      // with the key's next chunk.
      cudaGraph_t g = nullptr;
      bool captured = cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (captured) {
        const int rc = mg_launch_sigma_locked(h, s.d_mom, c.bucket, s.d_me, s.stream);
        const cudaError_t e = cudaStreamEndCapture(s.stream, &g);
        captured = rc == MG_OK && e == cudaSuccess && g != nullptr &&
                   cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      if (captured) {
        graphs[key] = exec;
      } else {
        cudaGetLastError();  // the failed capture's error is not the chunk's
        exec = nullptr;
      }
    } else {
      exec = it->second;
    }
    if (exec) {
      if (cudaGraphLaunch(exec, s.stream) != cudaSuccess) return MG_ERR_CUDA;
    } else {
      const int rc = mg_launch_sigma_locked(h, s.d_mom, c.bucket, s.d_me, s.stream);
      if (rc) return rc;
    }
  } else {
    const int rc = mg_launch_sigma(h, s.d_mom, c.bucket, s.d_me, s.stream);
    if (rc) return rc;
  }
  const size_t out_bytes = sizeof(double) * c.n;
  if (c.req->me_dev) {
    if (cudaMemcpyAsync(c.req->me + c.off, s.d_me, out_bytes, cudaMemcpyDeviceToDevice, s.stream) != cudaSuccess)
      return MG_ERR_CUDA;
  } else if (cudaMemcpyAsync(s.h_me, s.d_me, out_bytes, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess) {
    return MG_ERR_CUDA;
  }
  if (cudaEventRecord(s.done, s.stream) != cudaSuccess) return MG_ERR_CUDA;
  return MG_OK;
}

void mg_server::run() {
  cudaSetDevice(device);
  for (;;) {
    bool progress = false;
    // completions (the slots belong to this thread; results leave the pinned
    // staging before the request is marked done)
    for (Slot& s : slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      Request* r = s.cur.req;
      if (q == cudaSuccess && !r->me_dev) std::memcpy(r->me + s.cur.off, s.h_me, sizeof(double) * s.cur.n);
      s.busy = false;
      inflight -= s.bytes;
      progress = true;
      std::lock_guard<std::mutex> lk(m);
      finish_chunk(r, q == cudaSuccess ? MG_OK : MG_ERR_CUDA);
    }
    bool stopping;
    {
      std::lock_guard<std::mutex> lk(m);
      stopping = stop;
      if (stopping) {
        // fail everything still queued, then drain the slots
        while (!queue.empty()) {
          Request* r = queue.front().req;
          queue.pop_front();
          finish_chunk(r, MG_ERR_STATE);
        }
        cv_done.notify_all();
      }
    }
    if (stopping) {
      bool any = false;
      for (Slot& s : slots) any |= s.busy;
      if (!any) break;
    }
    // admissions, FIFO: the chunk is taken off the queue under the mutex, its
    // copies and launches run without it
    for (;;) {
      int si = -1;
      for (int i = 0; i < (int)slots.size(); i++)
        if (!slots[i].busy) {
          si = i;
          break;
        }
      if (si < 0) break;
      Chunk c;
      {
        std::lock_guard<std::mutex> lk(m);
        if (queue.empty()) break;
        c = queue.front();
      }
      const int64_t need = chunk_bytes(c.req->h, c.bucket);
      if (inflight > 0 && inflight + need > cfg.mem_budget_bytes) break;
      {
        std::lock_guard<std::mutex> lk(m);
        queue.pop_front();  // only this thread pops: still the chunk read above
        if (c.req->start_us < 0) c.req->start_us = now_us();
      }
      const int rc = admit(si, c);
      progress = true;
      if (rc != MG_OK) {
        // the slot's stream may hold part of the chunk's work: wait for it
        cudaStreamSynchronize(slots[si].stream);
        std::lock_guard<std::mutex> lk(m);
        finish_chunk(c.req, rc);
        continue;
      }
      slots[si].busy = true;
      slots[si].cur = c;
      slots[si].bytes = need;
      inflight += need;
    }
    if (!progress) {
      std::unique_lock<std::mutex> lk(m);
      cv_work.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

extern "C" int mg_server_cfg_default(mg_server_cfg* cfg) {
  if (!cfg) return MG_ERR_ARG;
  cfg->n_streams = 4;
  cfg->mem_budget_bytes = int64_t(8) << 30;
  cfg->min_bucket = 256;
  cfg->max_bucket = 65536;
  cfg->use_graphs = 1;
  return MG_OK;
}

extern "C" int mg_server_create(const mg_server_cfg* cfg, mg_server** out) {
  if (!out) return MG_ERR_ARG;
  *out = nullptr;
  mg_server_cfg c;
  mg_server_cfg_default(&c);
  if (cfg) c = *cfg;
  if (c.n_streams < 1 || c.n_streams > 64 || c.min_bucket < 1 || c.max_bucket < c.min_bucket ||
      c.mem_budget_bytes <= 0)
    return MG_ERR_ARG;
  // buckets are powers of two times min_bucket
  int64_t b = c.min_bucket;
  while (b < c.max_bucket) b <<= 1;
  c.max_bucket = b;
  mg_server* s = new (std::nothrow) mg_server();
  if (!s) return MG_ERR_NOMEM;
  s->cfg = c;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return MG_ERR_CUDA;
  }
  s->slots.resize(c.n_streams);
  const size_t mom_bytes = sizeof(double) * c.max_bucket * MAX_NPAR * 4, me_bytes = sizeof(double) * c.max_bucket;
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&sl.d_mom, mom_bytes) != cudaSuccess || cudaMalloc(&sl.d_me, me_bytes) != cudaSuccess ||
        cudaMallocHost(&sl.h_mom, mom_bytes) != cudaSuccess || cudaMallocHost(&sl.h_me, me_bytes) != cudaSuccess) {
      s->stop = true;
      mg_server_destroy(s);
      return MG_ERR_NOMEM;
    }
  }
  s->th = std::thread([s] { s->run(); });
  *out = s;
  return MG_OK;
}

extern "C" int mg_server_submit(mg_server* s, mg_process* h, const double* momenta, int64_t nevt, double* me_out,
                                uint64_t* req_id) {
  if (!s || !h || !req_id || nevt < 0) return MG_ERR_ARG;
  if (nevt > 0 && (!momenta || !me_out)) return MG_ERR_ARG;
  Request* r = new (std::nothrow) Request();
  if (!r) return MG_ERR_NOMEM;
  r->h = h;
  r->mom = momenta;
  r->me = me_out;
  r->nevt = nevt;
  if (nevt > 0) {
    r->mom_dev = is_device_pointer(momenta);
    r->me_dev = is_device_pointer(me_out);
  }
  std::vector<Chunk> cs;
  for (int64_t off = 0; off < nevt; off += s->cfg.max_bucket) {
    const int64_t n = std::min(s->cfg.max_bucket, nevt - off);
    Chunk c{r, off, n, bucket_for(s->cfg, n)};
    if (chunk_bytes(h, c.bucket) > s->cfg.mem_budget_bytes) {
      delete r;
      return MG_ERR_NOMEM;  // could never be admitted
    }
    r->padded += c.bucket;
    cs.push_back(c);
  }
  std::lock_guard<std::mutex> lk(s->m);
  if (s->stop) {
    delete r;
    return MG_ERR_STATE;
  }
  r->id = s->next_id++;
  r->submit_us = s->now_us();
  r->chunks_left = (int)cs.size();
  if (cs.empty()) {
    r->status = MG_OK;
    r->done = true;
    r->start_us = r->done_us = r->submit_us;
  }
  s->reqs[r->id] = r;
  for (const Chunk& c : cs) s->queue.push_back(c);
  *req_id = r->id;
  s->cv_work.notify_one();
  return MG_OK;
}

extern "C" int mg_server_poll(mg_server* s, uint64_t req_id, int64_t timeout_us, mg_req_stats* st) {
  if (!s || timeout_us < 0) return MG_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return MG_ERR_UNKNOWN_REQ;
  Request* r = it->second;
  if (!r->done && timeout_us > 0)
    s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [r] { return r->done; });
  if (!r->done) return MG_PENDING;
  if (st) {
    st->status = r->status;
    st->submit_us = r->submit_us;
    st->start_us = r->start_us;
    st->done_us = r->done_us;
    st->latency_us = r->done_us - r->submit_us;
    st->nevt = r->nevt;
    st->padded_nevt = r->padded;
  }
  const int status = r->status;
  s->reqs.erase(it);
  delete r;
  return status;
}

extern "C" void mg_server_destroy(mg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    cudaFree(sl.d_mom);
    cudaFree(sl.d_me);
    cudaFreeHost(sl.h_mom);
    cudaFreeHost(sl.h_me);
  }
  for (auto& kv : s->reqs) delete kv.second;
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}
