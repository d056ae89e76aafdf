/*
 * nmfa.h -- C ABI of libnmfa.so: noisy mean-field annealing (NMFA, Algorithm 1 of
 * King, Bernoudy, King, Berkley, Lanting, "Emulating the coherent Ising machine with
 * a mean-field algorithm", arXiv 1806.08422) on one NVIDIA GB300 (sm_103a).
 *
 * The method (Algorithm 1): for an Ising problem (h, J) on n spins, start every
 * spin at s_i = 0; for t = 1..t_f compute, from the old state, for every i
 *     Phi_i = (h_i + sum_j J_ij s_j) / sqrt(h_i^2 + sum_j J_ij^2) + N(0, sigma)
 *     sh_i  = -tanh(Phi_i / T_t)
 * and only then set s_i := alpha sh_i + (1 - alpha) s_i for every i; finally read
 * out the signs ~s_i = s_i / |s_i|.  The energy of a sign vector is Eq. (1),
 *     H = sum_{i<j} J_ij ~s_i ~s_j + sum_i h_i ~s_i,
 * each unordered pair counted once.
 *
 * Conventions shared by every entry point:
 *  - All calls return an int status: NMFA_OK (0) or a negative NMFA_E* code; the
 *    thread-local message of the last failure is nmfa_last_error().  On failure no
 *    output buffer is written (except where noted) and a handle stays usable.
 *  - J is symmetric with a zero diagonal (otherwise NMFA_ENOTSYM / NMFA_EDIAG);
 *    h may be NULL, meaning h = 0.  Dense J is row-major n*n float64.
 *  - A run draws R = `replicas` independent replicas r = 0..R-1.  Its Gaussian draw
 *    for (replica r, step t, spin i) is Box-Muller on Philox4x32-10 with counter
 *    (r/4, t, i, stream_id) and key (seed & 0xffffffff, seed >> 32), steps
 *    0-based; the same (seed, stream_id, r) always gives the same run, whatever
 *    else shares the GPU.
 *  - Outputs are replica-major: signs[r*n + i] in {-1, +1} (a state of exactly
 *    zero reads as +1), energy[r] = H of replica r's signs.
 *  - The caller owns every buffer it passes; the library copies what it keeps.
 *  - Every path computes in the precision it names, on the GPU, in hand-written
 *    kernels; there is no CPU fallback.  Without a usable CUDA device, calls
 *    that need one return NMFA_ECUDA.
 */
#ifndef NMFA_H_
#define NMFA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define NMFA_OK 0
#define NMFA_EINVAL (-1)       /* bad argument (size, pointer, T <= 0, alpha, sigma) */
#define NMFA_ENOTSYM (-2)      /* J is not symmetric */
#define NMFA_EDIAG (-3)        /* J has a nonzero diagonal entry */
#define NMFA_ENOMEM (-4)       /* device or host allocation failed */
#define NMFA_ECUDA (-5)        /* CUDA runtime error (message has the details) */
#define NMFA_ETIMEOUT (-6)     /* a bounded device-side wait gave up */
#define NMFA_EUNSUPPORTED (-7) /* valid input this path cannot take (size, precision) */

/* Storage and arithmetic of a problem (fixed at creation). */
typedef enum {
  NMFA_FP64 = 0,      /* FP64 CUDA-core path; coupling sums j-ascending, unfused */
  NMFA_FP32 = 1,      /* FP32 CUDA-core path, one instance per launch */
  NMFA_BF16 = 2,      /* tcgen05 tensor path: J and S in BF16, FP32 accumulation and
                         FP32 master state; J must be exactly representable in BF16 */
  NMFA_BF16_FP8J = 3  /* as NMFA_BF16 with J stored as FP8 E4M3 (exact values only;
                         half the bytes): the tensor kernel widens each staged slice to
                         BF16 in shared memory, so runs are bit-identical to NMFA_BF16
                         runs of the same J; the conversion costs time where J fits
                         in L2 (about 1.1x the step time with 256-replica tiles,
                         1.5x with 128-replica tiles, measured on GB300), so batches
                         widen problems of n <= 4096 once instead (see
                         NMFA_BATCH_FP8_IN_KERNEL) */
} nmfa_precision;

typedef struct nmfa_problem nmfa_problem; /* opaque; owns device copies of (h, J) */

/*
 * nmfa_create -- upload a dense Ising problem (Eq. (1)) and precompute in FP64 the
 * row norms d_i = sqrt(h_i^2 + sum_j J_ij^2) of Algorithm 1's field (Sec. II: the
 * root mean square of the terms acting on spin i), kept on the GPU: a kernel forms
 * them from the FP64 couplings, or, for integer tensor-path problems, creation forms
 * them on the host, where every term and the sum are exact integers and the square
 * root is correctly rounded (the same values).  A spin with d_i = 0 gets a
 * normalised field of 0.
 *   n         number of spins, 1 <= n <= 65536 (the CUDA-core paths accept less;
 *             NMFA_EUNSUPPORTED when the state does not fit on chip)
 *   h         host, n float64, or NULL for h = 0
 *   J         host, n*n float64, row-major, symmetric, zero diagonal
 *   precision an nmfa_precision value
 *   out       receives the handle (NULL on failure)
 * Checks (before any device work): n range, symmetry, diagonal, finiteness, and
 * for NMFA_BF16 / NMFA_BF16_FP8J exact representability of every J_ij in BF16 /
 * E4M3 (else NMFA_EUNSUPPORTED).
 */
int nmfa_create(int32_t n, const double* h, const double* J, int32_t precision,
                nmfa_problem** out);

/*
 * nmfa_create_csr -- the same problem given as CSR (sparse graphs, e.g. the
 * degree-3 MAX-CUT instances of Sec. III).  row_ptr has n+1 int64 entries starting
 * at 0; col/val have row_ptr[n] entries, columns strictly ascending within a row,
 * in [0, n); the pattern and values must be symmetric with no diagonal entry.
 * Coupling sums run over the stored entries in stored order.  Only NMFA_FP32 and
 * NMFA_FP64 take CSR input (others: NMFA_EUNSUPPORTED).
 */
int nmfa_create_csr(int32_t n, const double* h, const int64_t* row_ptr,
                    const int32_t* col, const double* val, int32_t precision,
                    nmfa_problem** out);

/* Frees the handle and its device memory (NULL is a no-op).  Waits for the
 * handle's runs in flight to finish first. */
void nmfa_destroy(nmfa_problem* p);

/*
 * nmfa_run -- Algorithm 1 end to end with HOST buffers: copies T to the device,
 * runs t_f annealing steps for `replicas` replicas, reads out the signs, evaluates
 * Eq. (1) on the GPU, copies the results back and returns when they are written.
 *   T              host, t_f float64 temperatures T_1..T_tf, each > 0 (Fig. 2's
 *                  schedule is an input; see the instance module for a default)
 *   t_f            number of steps, >= 0 (0 reads out the initial zero state)
 *   sigma          standard deviation of the Gaussian noise, >= 0 (Sec. II)
 *   alpha          mixing constant, 0 < alpha <= 1 (Algorithm 1's alpha-mix)
 *   replicas       R >= 1
 *   seed,stream_id select the noise stream (see the conventions above)
 *   signs_out      host, R*n int8 (may be NULL)
 *   energy_out     host, R float64 (may be NULL); exact for integer problems
 *   energy_i64_out host, R int64 or NULL; only for problems whose h and J are all
 *                  integers (else NMFA_EINVAL)
 * Not reentrant per handle: runs on one handle are serialised on the device.
 */
int nmfa_run(nmfa_problem* p, const double* T, int32_t t_f, double sigma, double alpha,
             int32_t replicas, uint64_t seed, uint32_t stream_id, int8_t* signs_out,
             double* energy_out, int64_t* energy_i64_out);

/*
 * nmfa_run_device -- as nmfa_run with DEVICE pointers, enqueued on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream) and returning without
 * synchronising.  T_dev holds t_f float64; signs_dev R*n int8, energy_dev R float64,
 * energy_i64_dev R int64; any output may be NULL.  Device-side timeouts are reported
 * by the next call on the handle or by nmfa_sync().  The handle's scratch memory
 * (grown on demand, never shrunk) is reused; consecutive runs on one handle are
 * ordered on the device even across streams.
 */
int nmfa_run_device(nmfa_problem* p, const double* T_dev, int32_t t_f, double sigma,
                    double alpha, int32_t replicas, uint64_t seed, uint32_t stream_id,
                    int8_t* signs_dev, double* energy_dev, int64_t* energy_i64_dev,
                    void* cuda_stream);

/*
 * nmfa_run_device_noalloc -- nmfa_run_device for an NMFA_BF16 or NMFA_BF16_FP8J
 * problem that allocates nothing (FP8-stored couplings are read as stored and
 * widened in the kernel, so they need no scratch).  The paper has no counterpart; this exists for callers that cannot
 * allocate device memory while they run: code inside a CUDA stream capture (an
 * allocation there is not part of the graph and may synchronise the device), a
 * framework whose memory pool owns all device memory, or a serving loop that must
 * not pay for or serialise on cudaMalloc.  The handle itself was allocated by
 * nmfa_create beforehand; this call only reuses it.
 *
 * The tensor kernel's scratch (two BF16 copies of the state, one epoch flag per
 * tile, the run plan and the per-replica energy sums) comes from a static device
 * array of 16 MiB that every GPU loading this library holds until the process
 * exits.  The rule is: the run's tensor-path workspace must fit in 16 MiB.  The
 * state alone is 4 * ceil(R/BN)*BN * ceil(n/128)*128 bytes, where BN, the run's
 * tile width, is 64 (R <= 64, or small problems), 128, or 256 (n >= 1921 when
 * 128-replica tiles would need more than one wave of the grid); the plan adds a
 * few tens of KB.  So n = 2000 takes up to R = 1792 (R = 1793 .. 1920 round up to
 * 2048 replicas, exactly 16 MiB of state, and are refused).  Larger sizes return
 * NMFA_EINVAL with nothing launched.  The flags and sums are cleared on the stream
 * before each launch; the state buffers are fully written by the kernel before
 * they are read.
 *   signs_dev  R*n int8, required (no scratch is made for signs)
 *   energy_dev, energy_i64_dev  as in nmfa_run_device (may be NULL)
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Called on a
 * capturing stream, the run (plan upload, flag reset, kernel, energy kernel) is
 * recorded into the caller's graph and neither waits for nor marks the handle's
 * completion event: the graph orders it, and nmfa_sync does not track its replays.  Every call
 * uses the same array, so calls whose kernels overlap on the GPU (different
 * streams, different handles) race and give wrong results: serialise them.
 * Returns NMFA_EUNSUPPORTED for other precisions.
 */
int nmfa_run_device_noalloc(nmfa_problem* p, const double* T_dev, int32_t t_f,
                            double sigma, double alpha, int32_t replicas, uint64_t seed,
                            uint32_t stream_id, int8_t* signs_dev, double* energy_dev,
                            int64_t* energy_i64_dev, void* cuda_stream);

/* Waits for the handle's last run and returns its device-side status
 * (NMFA_OK or NMFA_ETIMEOUT) or a CUDA error. */
int nmfa_sync(nmfa_problem* p);

/*
 * nmfa_debug_run -- test entry (not part of the stable ABI): nmfa_run_device with
 * access to the continuous state, for the single-step and trajectory parity checks.
 *   noise_sign  +1 (normal), 0 (noise off), -1 (every draw negated)
 *   s0_dev      R*n float64 initial state, or NULL for Algorithm 1's s = 0
 *   s_out_dev   R*n float64 final state s_i (before the sign readout), or NULL
 *   phi_out_dev R*n float64 Phi_i of the last step, or NULL
 * Other arguments as in nmfa_run_device.
 */
int nmfa_debug_run(nmfa_problem* p, const double* T_dev, int32_t t_f, double sigma,
                   double alpha, int32_t replicas, uint64_t seed, uint32_t stream_id,
                   int32_t noise_sign, const double* s0_dev, double* s_out_dev,
                   double* phi_out_dev, int8_t* signs_dev, double* energy_dev,
                   int64_t* energy_i64_dev, void* cuda_stream);

/*
 * Batches -- many tensor-path runs in ONE persistent launch (ragged batches of
 * instances of different sizes and replica counts).  Each job is an independent
 * Algorithm 1 run on its own NMFA_BF16 problem with its own schedule and noise
 * stream; its results are bit-identical to running it alone with nmfa_run_device
 * (the tiling of a run depends only on its own shape, and the noise counters are
 * the run's logical (replica, step, spin) indices).
 */
typedef struct {
  const double* T_dev;     /* device, t_f float64 temperatures */
  int32_t t_f;
  double sigma, alpha;
  int32_t replicas;
  uint64_t seed;
  uint32_t stream_id;
  int8_t* signs_dev;       /* device R*n int8, or NULL (batch keeps scratch) */
  double* energy_dev;      /* device R float64, or NULL */
  int64_t* energy_i64_dev; /* device R int64, or NULL (integer problems only) */
} nmfa_job;

typedef struct nmfa_batch nmfa_batch;

#define NMFA_BATCH_GRAPH 1    /* capture the batch's launches in a CUDA graph at creation */
#define NMFA_BATCH_AUTOTUNE 2 /* pick replicas per tile (64/128/256) per job by timing */
#define NMFA_BATCH_BN64 4     /* force 64 replicas per tile (results do not change) */
#define NMFA_BATCH_BN128 16   /* force 128 replicas per tile, one CTA per tile (results do not change) */
#define NMFA_BATCH_BN256 64   /* force 256 replicas per tile (results do not change) */
/* Run 128 replicas per tile as CTA pairs (two CTAs sharing one cta_group::2 MMA of
 * M = 256, each loading half of every state slice) wherever the problem allows it
 * (n rounded to 128 is a multiple of 256 and the pairs fit on the grid).  Not the
 * default: on GB300 the pairs run slower than one CTA per tile for the benchmark
 * workload.  A pair sums its odd row block's couplings in the pair's K order, so
 * results agree with one-CTA tiles to the BF16 path's rounding rather than bit for
 * bit; pair runs are still independent of what else a batch holds. */
#define NMFA_BATCH_PAIR128 32
/* FP8-stored problems (NMFA_BF16_FP8J) of n rounded to 128 up to 4096 are by default
 * widened to BF16 once, at batch creation, into a scratch copy of 2 x n_pad^2 bytes
 * held by the batch (it counts in nmfa_batch_info's workspace bytes), and run on the
 * BF16 kernel: the in-kernel widening of every staged slice costs 1.2-1.6x the step
 * time at those sizes on GB300, while the copy is at most 32 MB.  Larger FP8 problems
 * are read as stored and widened in the kernel.  With this option every FP8 problem
 * of the batch is read as stored.  Results do not change. */
#define NMFA_BATCH_FP8_IN_KERNEL 128
/* Test only: leave the first group's last row-block tile out of the plan.  Nothing
 * then publishes that tile's state, so the group's other tiles wait for a flag that
 * is never set: their bounded waits give up (within 2 s, 20 s at most),
 * nmfa_batch_sync returns NMFA_ETIMEOUT, and the device stays usable.  The failure
 * path is exercised without a GPU fault.  Needs a first job of more than 128 spins. */
#define NMFA_BATCH_DEBUG_WITHHOLD_TILE 8

/* Plans the batch (tiles of 128 spins x 64, 128 or 256 replicas; the tile pipelines of
 * one replica block are co-scheduled on the persistent grid by list scheduling),
 * allocates its workspace, uploads the plan, widens FP8-stored problems of n_pad <=
 * 4096 to BF16 (see NMFA_BATCH_FP8_IN_KERNEL) and, with NMFA_BATCH_GRAPH, captures the
 * launch sequence as a CUDA graph; it returns once that work has finished on the
 * batch's own stream.  No run starts until nmfa_batch_launch.  The
 * problems and every device buffer named in `jobs` must stay valid while the batch
 * exists; each launch overwrites the outputs. */
int nmfa_batch_create(nmfa_problem* const* problems, const nmfa_job* jobs, int32_t count,
                      int32_t options, nmfa_batch** out);
/* Enqueues one execution of the whole batch on `cuda_stream` (ordered after the
 * batch's previous execution). */
int nmfa_batch_launch(nmfa_batch* b, void* cuda_stream);
/* Waits for the last execution; NMFA_ETIMEOUT if a device-side wait gave up. */
int nmfa_batch_sync(nmfa_batch* b);
/* Re-targets the batch at other noise streams (Algorithm 1's Gaussian draws of job j
 * come from stream stream_ids[j] from the next execution on), keeping its plan and
 * workspace: a rerun of the same jobs with fresh noise needs no new batch.  Host array
 * of `count` = the batch's job count; ordered after the previous execution (the new
 * descriptors are uploaded on the batch's own stream).  NMFA_EINVAL on a count
 * mismatch; the batch is unchanged then. */
int nmfa_batch_set_stream_ids(nmfa_batch* b, const uint32_t* stream_ids, int32_t count);
/* Persistent grid size, number of replica-block groups, workspace bytes. */
int nmfa_batch_info(const nmfa_batch* b, int32_t* grid, int32_t* groups, int64_t* workspace_bytes);
void nmfa_batch_destroy(nmfa_batch* b);
/* The batch's persistent launches (one per tile variant present): for launch k,
 * bn[k] = replicas per tile (64, 128 or 256), ctas_per_mma[k] = 1, or 2 for CTA
 * pairs sharing one cta_group::2 MMA, and cluster_ctas[k] = CTAs per thread-block
 * cluster (1, or 2 for pairs).
 * Writes at most `capacity` entries; *count receives the number of launches.  Host
 * arrays; any output may be NULL. */
int nmfa_batch_plan(const nmfa_batch* b, int32_t* bn, int32_t* ctas_per_mma, int32_t* cluster_ctas,
                    int32_t capacity, int32_t* count);

/* Autotuner entry: the replicas-per-tile (64, 128 or 256) the tensor path would use for
 * `replicas` replicas of this problem, measured once per (n rounded to 128,
 * replicas) and cached for the process. */
int nmfa_autotune_bn(nmfa_problem* p, int32_t replicas, int32_t* bn);

/*
 * Serving -- a request loop on one GPU with admission by device-memory footprint,
 * continuous batching (every admitted request joins the next persistent launch as
 * soon as one of `max_inflight` launch slots frees; launches overlap on the GPU)
 * and time-to-target accounting.  A request anneals its instance with `replicas`
 * replicas; it succeeds when some replica's energy (Eq. (1)) is <= target_energy,
 * else it is rerun with the next noise stream id (attempt k uses stream k), at most
 * max_attempts runs.  Each run of a request is bit-identical to running it alone.
 * Times are seconds on the server's clock (0 = creation).
 */
typedef struct {
  int64_t memory_budget_bytes;  /* device memory admitted requests may hold (<= 0: 80% of free) */
  int32_t max_inflight;         /* concurrent launches (streams), default 2 */
  int32_t max_attempts;         /* runs per request before giving up, default 4 */
} nmfa_server_config;

typedef struct {
  int32_t n;
  const double* h;              /* host, n (or NULL); copied at submit */
  const double* J;              /* host, n*n symmetric, zero diagonal; copied at submit */
  int32_t precision;            /* NMFA_BF16 or NMFA_BF16_FP8J */
  const double* T;              /* host, t_f temperatures; copied */
  int32_t t_f;
  double sigma, alpha;
  int32_t replicas;
  uint64_t seed;
  double target_energy;
} nmfa_request;

typedef struct {
  int32_t state;        /* 0 queued, 1 admitted, 2 running, 3 done, -1 failed */
  int32_t attempts;     /* runs started */
  int32_t success;      /* 1 if the target was reached */
  int32_t error;        /* NMFA_* status of a failed request */
  double best_energy;   /* lowest energy over all runs */
  double t_submit, t_admit, t_first_start, t_done;
  double time_to_target;  /* t_done - t_submit when successful, else -1 */
  int64_t spin_updates;   /* replicas * n * t_f summed over runs */
} nmfa_result;

typedef struct nmfa_server nmfa_server;

int nmfa_server_create(const nmfa_server_config* cfg, nmfa_server** out);
/* Copies the request and queues it; returns a ticket for nmfa_server_poll. */
int nmfa_server_submit(nmfa_server* s, const nmfa_request* req, uint64_t* ticket);
/* Current state of a request; best_signs (host n int8, or NULL) gets the best
 * sign vector once the request is done. */
int nmfa_server_poll(nmfa_server* s, uint64_t ticket, nmfa_result* out, int8_t* best_signs);
/* Waits until every submitted request is done (NMFA_ETIMEOUT after timeout_s). */
int nmfa_server_drain(nmfa_server* s, double timeout_s);
/* Persistent launches so far, device memory held by admitted requests, requests not
 * finished, the most requests one launch has carried, and the launches that reused
 * the batch (plan and workspace) of their requests' previous attempt (any pointer
 * may be NULL). */
int nmfa_server_stats(nmfa_server* s, int64_t* launches, int64_t* mem_used, int32_t* outstanding,
                      int32_t* max_requests_per_launch, int64_t* batches_reused);
/* Stops the loop (waits for launches on the GPU) and frees everything. */
void nmfa_server_destroy(nmfa_server* s);

/* Problem facts: spins, precision, 1 if h and J are integer-valued, device bytes
 * held (any pointer may be NULL). */
int nmfa_problem_info(const nmfa_problem* p, int32_t* n, int32_t* precision,
                      int32_t* integer_valued, int64_t* device_bytes);

/* Profiling: when enabled, each run records CUDA events around its annealing
 * kernel(s) on the run's stream; nmfa_last_kernel_ms() then waits for the last run
 * and returns the annealing-kernel time in milliseconds (energy kernel excluded). */
int nmfa_profile_enable(nmfa_problem* p, int32_t on);
int nmfa_last_kernel_ms(nmfa_problem* p, float* ms);

/* Tuning of the CUDA-core paths: replicas held by one CTA of the replica-resident
 * kernels (0 = automatic, else 1, 2, 4 or 8).  Results do not depend on it, with one
 * exception: a nonzero value also sends FP32 dense problems that would take the tiled
 * kernel (n >= 256, or n > 128 with more than 512 replicas) to the replica-resident
 * one, whose coupling sums round in another order (the results agree within the FP32
 * path's tolerance); that kernel needs the state of n spins to fit in shared memory. */
int nmfa_tune_replicas_per_cta(nmfa_problem* p, int32_t replicas_per_cta);

/* nmfa_debug_withhold_arrival -- test entry (not part of the stable ABI), for
 * testing failure detection without a GPU fault: on the FP32 tiled path (dense FP32
 * problems of n >= 256, and n > 128 with more than 512 replicas) the first CTA of
 * the following runs of `p` does not arrive at the grid barrier that closes step
 * `step` (-1: off, the default).  The other CTAs' bounded waits then give up (after
 * about 2 s), nmfa_sync reports NMFA_ETIMEOUT, and the next run is unaffected.
 * Returns NMFA_EINVAL for a NULL handle or step < -1. */
int nmfa_debug_withhold_arrival(nmfa_problem* p, int32_t step);

/* Measured CUDA-core arithmetic peaks of the current device, the denominators of
 * the CUDA-core paths' rooflines: out[0] = FP32 FMA throughput, out[1] = FP64 FMA
 * throughput, both in TFLOP/s (2 flops per FMA), out[2] = tanh.approx.f32 throughput
 * of the MUFU in Tops/s; from dependent-chain loops on every SM (eight chains per
 * thread, 1024 threads per CTA, two CTAs per SM), the best of three timed launches
 * each on `cuda_stream` (NULL: the legacy default stream).  `out` is host memory of
 * 3 doubles.  Synchronous; takes a few tens of ms.
 * Returns NMFA_EINVAL for a NULL `out`, NMFA_ECUDA on a CUDA error. */
int nmfa_measure_alu_peaks(double* out, void* cuda_stream);

/* Number of kernels this library has launched in this process so far. */
uint64_t nmfa_launch_count(void);

/* Thread-local description of the last failure ("" if none). */
const char* nmfa_last_error(void);

/* Library version string. */
const char* nmfa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NMFA_H_ */
