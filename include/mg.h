/*
 * mg.h -- C ABI of the GB300 leading-order matrix-element library (libmg.so).
 *
 * The library computes, for a batch of phase-space points ("events"), the
 * per-event leading-order squared matrix element
 *
 *     ME = (1/IDEN) * sum_{helicities} sum_{colours} |M|^2
 *
 * from Feynman diagrams and helicity amplitudes, one event per GPU thread in
 * lockstep (paper Sect. 1: data-parallel matrix elements with lockstep
 * processing; Sect. 3: "double" and "mixed" floating-point modes; Tables 1-4:
 * throughput in matrix elements per second over an event batch, the "grid").
 * IDEN is the average over initial spins and colours times the symmetry factor
 * of identical final-state particles.
 *
 * Processes (process strings, particle order as written, initial states first):
 *   "e+ e- > mu+ mu-"     s-channel photon + Z          (2 diagrams, 16 helicities)
 *   "g g > t t~"                                        (3 diagrams, 16 helicities, 2 colour flows)
 *   "g g > t t~ g"                                      (16 diagrams, 32 helicities, 6 flows)
 *   "g g > t t~ g g"      paper Tables 1-2              (123 diagrams, 64 helicities, 24 flows)
 *   "g g > t t~ g g g"    paper Tables 3-4              (1240 diagrams, 128 helicities, 120 flows)
 *
 * Conventions shared by every entry point:
 *   - momenta: float64 array [nevt][npar][4], (E, px, py, pz) in GeV, row-major,
 *     contiguous; base address 16-byte aligned (checked; MG_ERR_ARG otherwise).
 *   - me_out: float64 array [nevt].
 *   - "_dev" pointers are CUDA device pointers on the device that was current
 *     when the handle was created; "_host" pointers are host memory (pinned
 *     memory gives asynchronous copies).
 *   - stream: a cudaStream_t passed as void*; NULL means the legacy default stream.
 *   - the caller owns every buffer it passes; a stream-ordered call only reads or
 *     writes them in stream order, so they must stay alive until the stream has
 *     reached the call.
 *   - return value: MG_OK (0) or a negative MG_ERR_* code (mg_strerror gives
 *     text).  No entry point aborts, traps or prints.
 */
#ifndef MG_H
#define MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_OK 0
#define MG_PENDING 1
#define MG_ERR_PROC (-1)     /* unknown process string                          */
#define MG_ERR_ARG (-2)      /* bad argument (NULL, negative size, misaligned)  */
#define MG_ERR_NOMEM (-3)    /* device or host allocation failed / over budget  */
#define MG_ERR_CUDA (-4)     /* a CUDA runtime call failed                      */
#define MG_ERR_TIMEOUT (-5)  /* a bounded wait ran out (poll timeout, device wait) */
#define MG_ERR_STATE (-6)    /* call not valid in the object's current state    */
#define MG_ERR_UNKNOWN_REQ (-7) /* unknown request id                           */

/* precision modes */
#define MG_FP64 0   /* every step in FP64                                        */
#define MG_MIXED 1  /* FP32 wavefunctions/amplitudes, FP64 propagator denominators,
                       FP16 hi+lo colour contraction on the tensor cores with FP32
                       accumulation, FP64 helicity sum                            */
#define MG_MIXED_PAPER 2 /* the paper's "mixed" (Sect. 3): Feynman diagrams in FP64,
                       colour algebra in FP32 on CUDA cores, FP64 helicity sum    */
#define MG_FLOAT 3  /* the paper's "float" (Sect. 3): every step in FP32, the
                       per-event set-up and propagator denominators included;
                       colour sum on CUDA cores.  mg_sigma_select in this mode
                       runs as in MG_MIXED                                        */

/* flags */
#define MG_NO_TOP_WIDTH 1   /* Gamma_t = 0 in every top propagator                 */
#define MG_PHOTON_ONLY 2    /* e+e- -> mu+mu-: drop the Z diagram                  */

typedef struct {
  double mt;           /* top mass [GeV]                       default 173.0     */
  double wt;           /* top width [GeV], every top propagator default 1.4915   */
  double alpha_s;      /* fixed strong coupling                default 0.118     */
  double mz;           /* Z mass [GeV]                         default 91.188    */
  double wz;           /* Z width [GeV]                        default 2.441404  */
  double alpha_em_inv; /* 1/alpha_em                           default 132.507   */
  double gf;           /* Fermi constant [GeV^-2]              default 1.16639e-5 */
  int precision;       /* MG_FP64, MG_MIXED, MG_MIXED_PAPER or MG_FLOAT         */
  int flags;           /* MG_NO_TOP_WIDTH | MG_PHOTON_ONLY                      */
} mg_params;

typedef struct mg_process mg_process; /* opaque; owns device-resident constants */

/* Fill *p with the defaults listed above (precision MG_FP64, flags 0). */
int mg_params_default(mg_params* p);

/* Create a process handle on the current CUDA device.  Uploads the process
 * constants (couplings, colour matrix, helicity list) to the device; every
 * helicity is active until mg_good_helicities is called.
 * proc: one of the process strings above.  Errors: MG_ERR_PROC, MG_ERR_ARG,
 * MG_ERR_NOMEM, MG_ERR_CUDA.  On error *out is set to NULL. */
int mg_process_create(const char* proc, const mg_params* p, mg_process** out);

/* Release the handle and its device memory (synchronises its own work). */
void mg_process_destroy(mg_process* h);

/* Static description of the process.  Any output pointer may be NULL. */
int mg_process_info(const mg_process* h, int* npar, int* n_hel, int* n_col, int* n_diag, double* iden);

/* Helicity filter (set-up, not per call).  Evaluates every helicity
 * combination in FP64 on nevt calibration events momenta_dev[nevt][npar][4]
 * and keeps helicity h iff max over the events of |M_h|^2 / sum_h' |M_h'|^2
 * exceeds 1e-14.  Synchronous.  n_good_out (may be NULL) receives the count;
 * mask_host (may be NULL) receives n_hel bytes, 1 = kept.  nevt = 0 restores
 * all helicities, and so does a calibration set in which no event has a
 * positive finite |M|^2 (it carries no information about the helicities).
 * Uses a temporary device buffer of nevt * n_hel doubles.  A list that differs
 * from the handle's current one is stored in a new device array; the old one
 * stays allocated until the handle is destroyed, since launches already queued
 * or CUDA graphs the caller captured may still read it (n_hel ints per
 * change). */
int mg_good_helicities(mg_process* h, const double* momenta_dev, int64_t nevt, int* n_good_out,
                       uint8_t* mask_host);

/* ME per event on the device, stream-ordered and asynchronous:
 * me_out_dev[i] for momenta_dev[i], i < nevt.  nevt = 0 is a no-op.
 * The mixed path of g g > t t~ g g g runs in two phases through a workspace
 * of at most 1 GiB taken from the stream-ordered allocator (cudaMallocAsync)
 * and released on the same stream (capturable in a CUDA graph).
 * Errors: MG_ERR_ARG (NULL handle/pointer, nevt < 0, misaligned momenta),
 * MG_ERR_CUDA (launch failure, or no memory for that workspace). */
int mg_sigma(mg_process* h, const double* momenta_dev, int64_t nevt, double* me_out_dev, void* stream);

/* Device bytes that one mg_sigma call of nevt events takes from the
 * stream-ordered allocator with the handle's current helicity list: the
 * two-phase workspace of the mixed g g > t t~ g g g path, 0 for every other
 * process and precision.  For memory planning (the serving loop's admission
 * counts it).  Errors: MG_ERR_ARG (NULL, nevt < 0). */
int mg_sigma_workspace_bytes(mg_process* h, int64_t nevt, int64_t* bytes_out);

/* Same computation from host buffers: copies momenta_host to a handle-owned
 * device workspace, launches, copies the MEs back into me_out_host and waits
 * for the stream before returning.  The workspace grows on demand (first call
 * at a new maximum size allocates). */
int mg_sigma_host(mg_process* h, const double* momenta_host, int64_t nevt, double* me_out_host, void* stream);

/* Device-side status word of the handle: 0 if every bounded device wait so far
 * completed, otherwise MG_ERR_TIMEOUT (the kernel skipped its work and left the
 * outputs unwritten).  Synchronises the device.  Clears the word. */
int mg_process_status(mg_process* h);

/* ME per event plus the event-by-event random choice of a helicity and of a
 * leading colour flow, as needed to write unweighted events (paper Sect. 5).
 * rnd_dev[nevt][2] holds uniforms (r_hel, r_col) in [0, 1):
 *   hel_out_dev[i]: the good helicity h_j (good list in increasing index
 *     order) with the smallest j whose cumulative |M_h|^2 exceeds r_hel * ME;
 *   col_out_dev[i]: the colour flow k (orderings of the gluons, lexicographic;
 *     flow k is (T^{a_s1} ... T^{a_sn}) with s1 next to the top) with the
 *     smallest k whose cumulative weight exceeds r_col * sum_k w_k, where
 *     w_k = sum over good helicities of |J_k(h)|^2;
 *   colw_out_dev (may be NULL): w[nevt][n_col].
 * me_out_dev as mg_sigma (FP64, or mixed with the colour sum on CUDA cores).
 * Stream-ordered.  Errors: MG_ERR_ARG, MG_ERR_CUDA. */
int mg_sigma_select(mg_process* h, const double* momenta_dev, int64_t nevt, const double* rnd_dev,
                    double* me_out_dev, int* hel_out_dev, int* col_out_dev, double* colw_out_dev, void* stream);

/* Per-helicity |M_h|^2 / IDEN in FP64 for every helicity (not filtered):
 * out_dev[nevt][n_hel].  Stream-ordered.  Diagnostics and helicity selection. */
int mg_sigma_helicities(mg_process* h, const double* momenta_dev, int64_t nevt, double* out_dev, void* stream);

/* Helicity filter that allocates nothing.  The paper has no counterpart: this
 * is a library-usage variant of mg_good_helicities for callers that cannot
 * call cudaMalloc -- code that runs under a fixed device-memory budget or its
 * own pool allocator, where a stray allocation fails or fragments the pool,
 * and latency-critical set-up paths that must not pay for cudaMalloc/cudaFree
 * (which may synchronise the device).  Same result as mg_good_helicities
 * (same threshold, same outputs), but its scratch (per-event, per-helicity
 * values and the per-helicity reduction) lives in one file-scope device array
 * of MG_STATIC_SCRATCH_DOUBLES doubles (8 MiB) that every GPU loading the
 * library holds until the process exits; the helicity list is rewritten in
 * place in the handle.
 *   - Limits: n_hel <= MG_STATIC_MAX_HEL and
 *     nevt * n_hel <= MG_STATIC_SCRATCH_DOUBLES - MG_STATIC_MAX_HEL
 *     (e.g. 8191 events for 128 helicities); larger requests return
 *     MG_ERR_ARG without touching the device.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the array and it keeps the last call's contents (the
 *     reduction slots are cleared at the start of each call).  Calls that
 *     overlap on the GPU -- from several host threads, or with any other use
 *     of the array -- race; serialise them.  The call synchronises the device
 *     first, so no launch of this handle may be pending in another thread.
 *   - The list is rewritten in place: a CUDA graph that the caller captured
 *     with this handle before the call must be captured again.
 *   - A calibration set in which no event has a positive finite |M|^2
 *     restores all helicities, as in mg_good_helicities.
 *   - Synchronous; runs on the legacy default stream. */
#define MG_STATIC_SCRATCH_DOUBLES (1 << 20)
#define MG_STATIC_MAX_HEL 128
int mg_good_helicities_static(mg_process* h, const double* momenta_dev, int64_t nevt, int* n_good_out,
                              uint8_t* mask_host);

/* Flat phase-space momenta generated on the device (paper Sect. 2: the
 * random-number -> momenta step of the event generator, moved to the GPU):
 * momenta_dev[nevt][npar][4] for events first_event .. first_event+nevt-1 of
 * the stream (seed), at fixed sqrt_s [GeV], for the handle's process (top
 * masses from its parameters).  Philox4x64-10 uniforms, key (seed, 0),
 * counter (event, final-state slot, 0, 0), u = ((w >> 11) + 0.5) 2^-53; RAMBO
 * massless generation, conformal map, residual 3-momentum removed, common
 * 3-momentum scale onto the mass shells; initial states (E,0,0,+-E).  The same
 * stream as the host input module to rounding of log/sin/cos.  Stream-ordered.
 * Errors: MG_ERR_ARG (nevt < 0, first_event < 0, sqrt_s below threshold, NULL). */
int mg_rambo(const mg_process* h, double sqrt_s, uint64_t seed, int64_t first_event, int64_t nevt,
             double* momenta_dev, void* stream);

/* Hit-or-miss unweighting on the device (paper Sect. 2: one of the serial
 * steps after the matrix element, named there as a candidate to offload to the
 * GPU; it turns weighted into unweighted events).  Event i of
 * w_dev[n] (weights, e.g. ME times phase-space weight) is kept when
 * r_dev[i] * w_max < w_dev[i], r_dev[n] uniforms in [0, 1); events with
 * w_i > w_max are kept (the caller may give them weight w_i / w_max).  Writes
 * the kept indices in increasing order to idx_out_dev (capacity n) and their
 * number to *n_acc_dev (device memory).  Stream-ordered; a workspace of
 * about n / 8 + n / 512 bytes (one accept bit per event and one count per
 * 4096 events) is taken from the stream-ordered allocator (cudaMallocAsync)
 * and released on the same stream.  Errors: MG_ERR_ARG (n < 0, w_max <= 0 or NaN,
 * NULL), MG_ERR_NOMEM, MG_ERR_CUDA. */
int mg_unweight(const double* w_dev, const double* r_dev, int64_t n, double w_max, int64_t* idx_out_dev,
                int64_t* n_acc_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: a persistent request loop on one GPU with continuous batching
 * (paper Sect. 2, Fig. 1: several host processes sharing one GPU).
 * Requests (process handle + batch of events) are padded up to a shape bucket
 * (powers of two from min_bucket to max_bucket events; larger requests are
 * split into max_bucket pieces) and admitted while the in-flight device memory
 * -- each piece's momenta and results plus the workspace its launch takes
 * (mg_sigma_workspace_bytes: the two-phase mixed g g > t t~ g g g path) --
 * stays within mem_budget_bytes; they run as captured CUDA graphs, one graph
 * per (stream, process, bucket, helicity list), on n_streams streams, so that
 * requests that arrive while others run overlap on the device.  Host buffers
 * travel through pinned staging buffers owned by the server, so every copy is
 * asynchronous and no copy or launch runs under the lock that submit and poll
 * take.
 * ------------------------------------------------------------------------- */
typedef struct mg_server mg_server;

typedef struct {
  int n_streams;             /* concurrent device streams          (default 4)        */
  int64_t mem_budget_bytes;  /* in-flight device memory cap     (default 8 GiB)       */
  int64_t min_bucket;        /* smallest padded batch              (default 256)      */
  int64_t max_bucket;        /* largest padded batch               (default 65536)    */
  int use_graphs;            /* 1: per-bucket CUDA graphs, 0: plain launches (default 1) */
} mg_server_cfg;

typedef struct {
  int status;          /* MG_OK, MG_PENDING or an error code                     */
  double submit_us;    /* host clock at submit  [microseconds, server epoch]     */
  double start_us;     /* host clock when the request was admitted to a stream   */
  double done_us;      /* host clock when completion was observed                */
  double latency_us;   /* done_us - submit_us                                    */
  int64_t nevt;        /* events in the request                                  */
  int64_t padded_nevt; /* events launched (bucket padding included)              */
} mg_req_stats;

int mg_server_cfg_default(mg_server_cfg* cfg);

/* Start the server (one host scheduler thread) on the current device.
 * While it captures a CUDA graph, a device-wide synchronisation from another
 * thread (cudaDeviceSynchronize, torch.cuda.synchronize) fails with
 * cudaErrorStreamCaptureUnsupported; clients that share the device with a
 * running server synchronise their own streams instead.  The server itself
 * launches a chunk whose capture failed that way directly. */
int mg_server_create(const mg_server_cfg* cfg, mg_server** out);

/* Queue a request: nevt events momenta[nevt][npar][4], results written to
 * me_out[nevt] before the request completes.  Each buffer may be in host or
 * in device memory (told apart with cudaPointerGetAttributes).  Both
 * buffers are the caller's and must stay valid until mg_server_poll has
 * returned MG_OK or an error for the request, and so must the process handle
 * h (it may be destroyed after that; the graphs the server captured for it
 * are keyed by the handle's own serial number and are not replayed for a
 * later handle).  Non-blocking.  A request whose pieces need more than the
 * memory budget each can never be admitted: MG_ERR_NOMEM at submit. */
int mg_server_submit(mg_server* s, mg_process* h, const double* momenta, int64_t nevt, double* me_out,
                     uint64_t* req_id);

/* MG_OK (done; st filled, request forgotten), MG_PENDING (timeout_us elapsed,
 * timeout_us = 0 polls once), or an error.  st may be NULL. */
int mg_server_poll(mg_server* s, uint64_t req_id, int64_t timeout_us, mg_req_stats* st);

/* Stop the scheduler; waits for in-flight work, fails queued requests with
 * MG_ERR_STATE, releases everything. */
void mg_server_destroy(mg_server* s);

const char* mg_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
