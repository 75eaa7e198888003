/*
 * sk.h -- C ABI of the B300 spectral-kurtosis RFI detector.
 *
 * Method: Taylor et al., "Spectral Kurtosis Based RFI Mitigation for CHIME"
 * (arXiv:1808.10365).  Notation: M samples per input per estimate (the
 * paper's n), N inputs (receivers), N_eff the inputs with non-zero power in
 * a frame.  A frame is one estimate: M time samples of all N inputs of one
 * frequency channel.
 *
 * Input bytes: one complex sample per byte, 4+4-bit offset binary, real part
 * in the high nibble and imaginary part in the low nibble, each value
 * v + 8 with v in [-8, 7] (the generator never writes -8; the library decodes
 * it as -8).
 *
 * Layouts:
 *   SK_LAYOUT_TIME_MAJOR  uint8 [frame][t = 0..M-1][input = 0..N-1]
 *   SK_LAYOUT_INPUT_MAJOR uint8 [frame][input][t]
 * Several frequencies of the same (N, M) are simply more frames.
 *
 * Ownership: the caller owns every buffer and CUDA stream it passes.  A plan
 * owns its threshold tables and device copies of them.  No C++ exception or
 * abort crosses this interface: every call returns an sk_status_t and
 * sk_last_error() gives a message for the calling thread's last failure.
 * Calls taking a stream enqueue work and return without synchronising
 * unless stated otherwise.
 *
 * Environment (read once per process; none changes results, only speed):
 *   SK_AUTOTUNE_CACHE    launch configuration cache file, read at each plan
 *                        creation (lines "N M layout rows grid path team_log2
 *                        prefetch batch_path", see sk_launch_config_t; older
 *                        "N M layout rows grid" lines are still read)
 *   SK_WARP_SLICE=0      one-item launches: team path (one barrier per frame)
 *                        instead of the warp-slice path (time-major, N a multiple
 *                        of 8 from 256 to 4096)
 *                        and the slot-ring combine (input-major teams of >= 2 warps)
 *   SK_ROW_BALANCE=0     warp-slice launches hand out whole frames instead of
 *                        equal row ranges (no plan scratch)
 *   SK_TAIL_FOLD=0       time-major N = 256 W + 8 k (k of 1..min(4, W), where that
 *                        adds a team per CTA): teams of W + 1 warps instead of W
 *                        warps that also read the k groups of 8 columns past the
 *                        last whole 256-column slice
 *   SK_IMAJOR_GROUPED=0  input-major: per-input path instead of the grouped one
 *   SK_IMAJOR_PREFETCH=0 input-major grouped path without the L2 prefetch
 *   SK_IMAJOR_LANES      input-major per-input path: lanes per input (2, 4, 8)
 *   SK_SERVER_ZEROCOPY=0 server: upload each batch instead of zero-copy reads
 *   SK_SERVER_INFLIGHT   server: launches in flight (1..8, default 2)
 *   SK_SERVER_TRACE=1    server: per-launch stage times on destroy
 *   SK_SERVER_SPLIT=0    server: no per-frame row split for small batches
 *   SK_SERVER_INJECT_FAULT=k  server (tests): launch k fails on the host, before
 *                        any CUDA call, as a failed launch would; its tickets and
 *                        the queued ones complete with SK_ERR_CUDA
 *   SK_DEBUG_SHRINK_INPUT=k   debug build only (tests): the bounds checks take every
 *                        input as k bytes shorter than it is, so that its last
 *                        loads fail their checks and the plan reports it
 * The Python binding loads the debug build of this library (every kernel load
 * and store checked, a failed check skipped and reported as SK_ERR_CUDA by the
 * plan's next call) instead of the release build when SK_DEBUG_LIBRARY=1.
 */
#ifndef SK_H
#define SK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SK_OK = 0,
    SK_ERR_INVALID_ARG = 1, /* null pointer, size out of range, misaligned */
    SK_ERR_UNSUPPORTED = 2, /* valid request the library does not serve    */
    SK_ERR_OOM = 3,         /* device or host allocation failed            */
    SK_ERR_CUDA = 4,        /* a CUDA runtime call failed                  */
    SK_ERR_BUSY = 5,        /* admission refused: ring full or over budget */
    SK_ERR_TIMEOUT = 6,     /* a bounded wait ran out                      */
    SK_ERR_NOT_READY = 7,   /* result not yet available                    */
    SK_ERR_CLOSED = 8       /* stream or server already closed             */
} sk_status_t;

typedef enum {
    SK_LAYOUT_TIME_MAJOR = 0,
    SK_LAYOUT_INPUT_MAJOR = 1
} sk_layout_t;

/* sk_params_t.flags */
#define SK_RUNNING_OFFSET 0x1u /* served streams: per-input power state sets the
                                  digitisation offset of the threshold centre */
#define SK_THRESH_PEARSON3 0x2u /* false-alarm thresholds for small M*N_eff (Sec.
                                  3.2): SK~ modelled as a Pearson type III with
                                  mean 1+delta, variance 4/m, skewness 10/sqrt(m),
                                  m = M*N_eff; each tail at probability Phi(-a)
                                  (Wilson-Hilferty gamma quantile).  Tends to
                                  the symmetric interval as m grows. */
#define SK_RUNNING_MU 0x4u      /* served streams: normalise each input by its
                                  running power mu_i = P_i / (2^6 M) from the
                                  state instead of the frame's S1_i / M, and use
                                  Eq. avgSK (first line) with n' = M N_eff and
                                  S1bar = sum S1_i/mu_i, S2bar = sum S2_i/mu_i^2,
                                  rescaled by Eq. final (first line); flagged
                                  in double against the symmetric interval.
                                  Unlike the per-frame normalisation it also
                                  reacts to power steps.  Keeps the state like
                                  SK_RUNNING_OFFSET. */

#define SK_MAX_INPUTS 4096
#define SK_MAX_TIME 4096
#define SK_OFFSET_BUCKETS 4096 /* power buckets of the running-offset table */
#define SK_STATE_SHIFT 6       /* leaky-integrator gain 2^-6 of the state   */

typedef struct {
    int32_t n_inputs;   /* N, 1..SK_MAX_INPUTS                              */
    int32_t n_time;     /* M (the paper's n), 2..SK_MAX_TIME                */
    int32_t layout;     /* sk_layout_t                                      */
    uint32_t flags;     /* SK_RUNNING_OFFSET | SK_THRESH_PEARSON3 | SK_RUNNING_MU */
    double n_sigma;     /* a: flag outside centre +- a*sqrt(4/(M N_eff))    */
    double mean_offset; /* static delta added to the centre 1 (App. B)     */
    /* optional host table [SK_OFFSET_BUCKETS] of per-input offsets in Q
       units for SK_RUNNING_OFFSET; NULL builds it from the App. B model */
    const int64_t *offset_table;
} sk_params_t;

typedef struct sk_plan_s *sk_plan_t;
typedef struct sk_batch_s *sk_batch_t;
typedef struct sk_server_s *sk_server_t;
typedef void *sk_cuda_stream_t; /* a cudaStream_t; NULL = legacy default */
typedef int32_t sk_stream_id;
typedef int64_t sk_ticket_t;

/* ---------------------------------------------------------------- plans */

/*
 * Validate params and build the plan for one (N, M, layout): integer
 * thresholds on Q for N_eff = 1..N (Sec. 3.2: outside mean +- a*sqrt(var),
 * var = 4/(M N_eff) from the moments below Eq. final; mean 1 + delta, App.
 * B), the fp32 scale (M+1)/((M-1) N_eff) of Eq. final, and, with
 * SK_RUNNING_OFFSET, the offset table.  Copies them to `device`.  The launch
 * configuration (sk_launch_config_t) comes from the autotune cache file named
 * by the environment variable SK_AUTOTUNE_CACHE when it has an entry for
 * (N, M, layout), else from the built-in defaults.
 * Errors: INVALID_ARG (null, N or M out of range, bad layout, n_sigma < 0),
 * CUDA, OOM.  *out is NULL on error.
 */
sk_status_t sk_plan_create(const sk_params_t *params, int device,
                           sk_plan_t *out);
sk_status_t sk_plan_destroy(sk_plan_t plan);

/* Host copies of the threshold tables, N+1 entries each (entry 0 unused). */
sk_status_t sk_plan_thresholds(sk_plan_t plan, int64_t *t_lo, int64_t *t_hi);
/* Host copy of the offset table (SK_OFFSET_BUCKETS entries). */
sk_status_t sk_plan_offset_table(sk_plan_t plan, int64_t *e);

/*
 * Tile choice of the fused kernel for this plan: rows_per_batch (8 or 16)
 * rows of 8 bytes each thread keeps in flight per register batch, and
 * grid_ctas (0 = one CTA per SM) for the plain launches.  Results do not
 * depend on either (exact integer combination); only speed does.  The rows
 * and grid of sk_launch_config_t (below), which carries the rest of the
 * configuration.  Not to be called while another thread issues launches of
 * the same plan.  INVALID_ARG for other values.
 */
sk_status_t sk_plan_set_tiles(sk_plan_t plan, int32_t rows_per_batch,
                              int32_t grid_ctas);
sk_status_t sk_plan_get_tiles(sk_plan_t plan, int32_t *rows_per_batch,
                              int32_t *grid_ctas);

/*
 * Read paths of the fused kernel.  Requested (sk_launch_config_t.path,
 * .batch_path): AUTO lets the library choose by shape; TEAM takes the team
 * path (the threads of a frame meet at one barrier per frame); WARP_SLICE
 * has the warps of a frame combine through a ring of shared-memory slots
 * (whole frames per team); ROW_BALANCED adds equal row ranges over the grid
 * through the plan's scratch.  A path the shape cannot take (or the launch:
 * a captured launch has no row balancing) falls back to the one it can.
 * STREAM reads frames in aligned 16-byte chunks.  Time-major (N / gcd(N, 16) <=
 * 512): each frame as one run, a group of lanes per frame whose byte positions
 * keep their inputs from chunk to chunk -- the path of frames of few inputs and of
 * the general shapes, any M.  Input-major, the path of lengths M without a fast
 * path: up to M = 192 a launch stages blocks of 32 inputs per warp in shared
 * memory and each lane adds its own input; longer inputs take 2, 4 or 8 lanes per
 * input over the chunks that cover it, the neighbours' bytes masked.  Batched
 * items the library would put on it take batch classes of their own.  Asked for
 * on a time-major shape with no unit of at most 512 lanes, a launch takes the
 * path the library would choose.
 * Reported (sk_launch_config_t.last_path) besides those: GENERAL (any N and
 * M, either layout) and PER_INPUT (input-major lengths of the per-input path).
 */
typedef enum {
    SK_PATH_AUTO = 0,
    SK_PATH_TEAM = 1,
    SK_PATH_WARP_SLICE = 2,
    SK_PATH_ROW_BALANCED = 3,
    SK_PATH_GENERAL = 4,
    SK_PATH_PER_INPUT = 5,
    SK_PATH_STREAM = 6
} sk_path_t;

/*
 * Launch configuration of a plan, the space the autotuner searches.  None of
 * it changes results (the combination over inputs and rows is exact integer
 * arithmetic), only speed.
 *   rows       rows of 8 bytes per register batch of the time-major vector
 *              paths: 16 (needs M % 32 == 0) or 8; the warp-slice paths run
 *              32-row turns on 16 and, only where M = 16 mod 32, 16-row
 *              turns on 8
 *   grid_ctas  CTAs of a one-item launch (0: one per SM)
 *   path       sk_path_t requested for one-item launches (0..3 or 6)
 *   team_log2  input-major layout: threads per frame as a power of two,
 *              5..8 (5..9 on the per-input path); set 0 for the plan's own
 *              choice (about 2 KB of frame per thread); get returns the size
 *              in use (0 for plans without an input-major fast path)
 *   prefetch   0: the L2 prefetch of the read paths, 1: none
 *   batch_path sk_path_t requested for this plan's items in sk_batch_create:
 *              time-major N = 2048 items take the warp-slice class for
 *              WARP_SLICE or ROW_BALANCED, the team class for TEAM, and by
 *              their M for AUTO (warp slices at M <= 128)
 *   last_path  (get only) the path the plan's latest one-item launch took
 *              (0 before any)
 */
typedef struct {
    int32_t rows;
    int32_t grid_ctas;
    int32_t path;
    int32_t team_log2;
    int32_t prefetch;
    int32_t batch_path;
    int32_t last_path;
} sk_launch_config_t;

/* Set the plan's launch configuration (last_path is ignored).  INVALID_ARG
 * for values outside the ranges above.  Like sk_plan_set_tiles, not to be
 * called while another thread issues launches of the same plan. */
sk_status_t sk_plan_set_config(sk_plan_t plan, const sk_launch_config_t *cfg);
sk_status_t sk_plan_get_config(sk_plan_t plan, sk_launch_config_t *cfg);

/*
 * Raw statistics of n_frames frames at d_in (device, 16-byte aligned,
 * n_frames*M*N bytes).  Per frame f and input i (Eq. 1 / Eq. singlesums):
 *   S1[f][i] = sum_t |x|^2, S2[f][i] = sum_t |x|^4        (int32, exact)
 * per frame (Eqs. discreteMean, normedSum2, final; SK~ = Avg(SK^_i)):
 *   Q[f]   = sum_{i: S1_i > 0} rint(2^32 * fp32(M S2_i - S1_i^2) / fp32(S1_i^2))
 *            (M S2_i - S1_i^2 formed exactly in int64; one fp32 divide)
 *   neff[f]= #{i : S1_i > 0}
 *   sk[f]  = fp32(Q) * 2^-32 * fp32((M+1)/((M-1) neff))   (NaN if neff = 0)
 * Every output pointer may be NULL (not written); S1 and S2 go together and
 * must be 16-byte aligned.  Device pointers only.
 * Errors: INVALID_ARG (null plan or d_in, misaligned pointer, n_frames < 0),
 * CUDA (launch failure), TIMEOUT (a bounded wait inside an earlier launch of
 * this plan ran out: that launch's outputs are void; reported once, by the
 * plan's next call, which then runs normally -- every call that takes a plan
 * reports it the same way).
 */
sk_status_t sk_compute(sk_plan_t plan, const uint8_t *d_in, int64_t n_frames,
                       int32_t *d_s1, int32_t *d_s2, int64_t *d_q,
                       float *d_sk, int32_t *d_neff, sk_cuda_stream_t stream);

/*
 * Input sharding: the inputs of one frequency split over several devices.  Each
 * device holds its own inputs' bytes as a contiguous array of n_frames frames
 * (its own N and M, in a plan of its own), and sk_compute gives its per-frame Q
 * and neff.  The per-input terms of Eq. final do not depend on the other
 * inputs, so the frame's Q and N_eff are the exact int64 / int32 sums of the
 * shards' values; once they are summed (one all-reduce of 12 bytes a frame),
 * sk_finish forms SK and the mask with the plan of the whole array (its N is
 * the total).  The result is bit-identical to sk_flag on the whole array.
 * d_q [n_frames] int64 and d_neff [n_frames] int32 are required, d_sk may be
 * NULL, d_mask is required.  A neff outside 0..N gives mask 1 and SK NaN.
 * Errors: INVALID_ARG, UNSUPPORTED (plans with SK_RUNNING_OFFSET or
 * SK_RUNNING_MU: their state belongs to served streams), CUDA.
 */
sk_status_t sk_finish(sk_plan_t plan, const int64_t *d_q, const int32_t *d_neff,
                      int64_t n_frames, float *d_sk, uint8_t *d_mask,
                      sk_cuda_stream_t stream);

/*
 * Scratch of the device calls (sk_compute, sk_flag, sk_compute_inputs and
 * the chunks of sk_flag_host).  Time-major plans with N a multiple of 8 from
 * 256 to 4096 and M % 16 == 0, and input-major plans of M = 128, 256 or 4096, give
 * every team of the launch an equal share of rows; frames cut between teams
 * are combined in a scratch of the plan (about 5 MB time-major, a few KB
 * input-major) that every launch leaves zero.  The first such call that is
 * not being captured into a graph allocates it; a call that cannot allocate
 * it, or is being captured, hands out whole frames instead (same results).
 * Calls of one plan on two streams take turns on the scratch: the later one
 * waits, on the device, for the earlier one.  SK_ROW_BALANCE=0 turns it off.
 */

/*
 * Fused compute + threshold: mask[f] = 1 when Q lies above T_hi[neff] or
 * below T_lo[neff] (SK~ strictly outside the centre +- a*sigma interval,
 * Sec. 3.2) or neff = 0.  d_sk may be NULL.  Same rules as sk_compute.
 */
sk_status_t sk_flag(sk_plan_t plan, const uint8_t *d_in, int64_t n_frames,
                    float *d_sk, uint8_t *d_mask, sk_cuda_stream_t stream);

/*
 * Per-input (independent) estimates, the "Independent SK^ Estimates" variant
 * of Sec. 2.2.3: for every frame f and input i,
 *   sk_in[f][i]   = fp32(r_i) * fp32((M+1)/(M-1)) = SK^_i of Eq. originalSK,
 *                   NaN when S1_i = 0;
 *   mask_in[f][i] = 1 when rint(2^32 r_i) lies outside [T_lo[1], T_hi[1]]
 *                   (the one-input interval centre +- a*2/sqrt(M)) or S1_i = 0.
 * The average of SK^_i over inputs is SK~ (Eq. final).  d_sk_in is
 * [n_frames][N] float (required), d_mask_in [n_frames][N] uint8 (may be NULL);
 * d_sk and d_mask per frame as in sk_flag (may be NULL).
 */
sk_status_t sk_compute_inputs(sk_plan_t plan, const uint8_t *d_in,
                              int64_t n_frames, float *d_sk_in,
                              uint8_t *d_mask_in, float *d_sk, uint8_t *d_mask,
                              sk_cuda_stream_t stream);

/*
 * sk_flag on HOST buffers: h_in (n_frames*M*N bytes), h_sk (may be NULL) and
 * h_mask are host memory (page-locked for full copy speed).  The plan
 * stages chunks through device buffers it owns, overlapping the host-to-
 * device copy of one chunk with the kernel on the previous one.  Returns
 * after the results are in h_sk/h_mask (synchronous).  Calls on one plan
 * are serialised.
 */
sk_status_t sk_flag_host(sk_plan_t plan, const uint8_t *h_in, int64_t n_frames,
                         float *h_sk, uint8_t *h_mask, sk_cuda_stream_t stream);

/*
 * sk_flag_host without any device allocation (the paper has no counterpart;
 * this is an interface for callers that cannot allocate).  Some callers must
 * not call cudaMalloc after start-up: their device memory belongs to another
 * allocator, or an allocation could stall a real-time loop.  This call stages
 * the bytes through a fixed array built into the library instead of the
 * buffers sk_flag_host allocates, so it allocates nothing (the plan itself is
 * made beforehand with sk_plan_create).  One call takes at most
 * SK_NOALLOC_MAX_BYTES input bytes (n_frames*M*N) and SK_NOALLOC_MAX_FRAMES
 * frames; larger requests get INVALID_ARG and must be split.  The array
 * (about 16.3 MiB) is set up when sk_plan_create makes a plan on the device:
 * the plan looks up its device address, which loads the part of the library
 * holding it, and the device keeps it until the process exits.  So create the
 * plan before handing the device's memory to another allocator; if that
 * set-up failed, the first call on the device retries it and reports its
 * error.  Calls on one device share the array: this process serialises them
 * and each returns after its results are in h_sk/h_mask, but other work that
 * overlaps a call on the GPU would race.  Like sk_flag_host, the call returns
 * the plan's pending fault (SK_ERR_TIMEOUT) if a bounded wait inside its own
 * launch gave up.
 */
#define SK_NOALLOC_MAX_BYTES (16 * 1024 * 1024)
#define SK_NOALLOC_MAX_FRAMES 65536
sk_status_t sk_flag_host_noalloc(sk_plan_t plan, const uint8_t *h_in,
                                 int64_t n_frames, float *h_sk, uint8_t *h_mask,
                                 sk_cuda_stream_t stream);

/* ------------------------------------------------------ batched launch */

typedef struct {
    sk_plan_t plan;      /* its N, M and thresholds                     */
    const uint8_t *d_in; /* n_frames frames, 16-byte aligned            */
    int64_t n_frames;
    float *d_sk;         /* may be NULL                                 */
    uint8_t *d_mask;     /* may be NULL (not both)                      */
} sk_batch_item_t;

/*
 * One persistent launch over many (N, M) items (frequencies of different
 * array sizes and integration lengths).  Builds a static schedule that
 * gives every CTA an equal share of bytes and captures the launch in a CUDA
 * graph on first run.  Items (buffers, plans) must stay valid until
 * destroy.
 */
sk_status_t sk_batch_create(const sk_batch_item_t *items, int32_t n_items,
                            int device, sk_batch_t *out);
sk_status_t sk_batch_run(sk_batch_t batch, sk_cuda_stream_t stream);
/* Kernel launches one sk_batch_run replays: one persistent launch per
 * non-empty kernel class of the batch's items (0 if no item has frames). */
sk_status_t sk_batch_launches(sk_batch_t batch, int32_t *launches);
sk_status_t sk_batch_destroy(sk_batch_t batch);

/* ------------------------------------------------------------ serving */

/*
 * A continuous-batching server on one device.  Streams (one array of N
 * inputs each, different N allowed) submit frames as they arrive into one
 * shared, arrival-ordered ring of page-locked host memory; a launcher thread
 * takes the ready frames (at most one per stream with running state, so its
 * state advances in frame order) and launches one batched kernel over them
 * while the previous launch is still on the GPU.  The kernel reads the frames
 * from the host ring directly (zero copy); SK_SERVER_ZEROCOPY=0 selects a
 * device mirror of the ring with one upload per batch instead.  The ring is
 * half of hbm_budget_bytes (at most 4 GiB); a stream is admitted while its
 * ring share (ring_frames frames) fits the ring, its device state and
 * tables fit the rest of the budget, and they fit the device's free memory
 * at the time of sk_stream_open (cudaMemGetInfo) less a headroom of
 * 256 MiB kept for the launches: admission follows the lesser of the
 * caller's budget and the memory really free.  SK_SERVER_INFLIGHT (1..8, default 2)
 * sets how many launches may be in flight; SK_SERVER_TRACE=1 prints per-launch
 * timing averages when the server is destroyed.
 */
sk_status_t sk_server_create(int device, size_t hbm_budget_bytes,
                             sk_server_t *out);
sk_status_t sk_server_destroy(sk_server_t server);
/* BUSY if the ring and state would exceed the remaining budget.  Either
 * layout; input-major frames take the kernel's general (byte-load) path. */
sk_status_t sk_stream_open(sk_server_t server, const sk_params_t *params,
                           int32_t ring_frames, sk_stream_id *out);
/*
 * Queue one frame (M*N bytes of host memory, copied before return) with its
 * index in the stream.  BUSY if the stream's ring is full.  *ticket
 * identifies the result.
 */
sk_status_t sk_stream_submit(sk_server_t server, sk_stream_id stream,
                             const uint8_t *frame, int64_t frame_index,
                             sk_ticket_t *ticket);
/*
 * Queue one frame by reference: no copy.  frame (16-byte aligned) is device
 * memory of the server's device, or page-locked host memory the device can
 * read (mapped); the kernel reads it where it is, so it must stay unchanged
 * until the ticket completes.  INVALID_ARG for pageable host memory.  Frames
 * passed either way may be mixed in one stream; they are processed in
 * submission order.  Host frames are best kept in page-locked buffers pinned
 * once and reused: on the B300 machines measured, serving from pools pinned just
 * before the run gave multi-millisecond p99 latency episodes in every run,
 * while pools pinned earlier and warmed by a short replay held p99 near
 * 0.22 ms.
 */
sk_status_t sk_stream_submit_ref(sk_server_t server, sk_stream_id stream,
                                 const uint8_t *frame, int64_t frame_index,
                                 sk_ticket_t *ticket);
/*
 * Wait up to timeout_us (< 0: no limit) for a ticket; fills *sk and *mask
 * (either may be NULL) and releases the ticket.  TIMEOUT if not done in
 * time, INVALID_ARG for an unknown or already collected ticket.
 */
sk_status_t sk_ticket_wait(sk_server_t server, sk_ticket_t ticket,
                           int64_t timeout_us, float *sk, uint8_t *mask);
/* Block until every submitted frame of the stream has its result. */
sk_status_t sk_stream_drain(sk_server_t server, sk_stream_id stream,
                            int64_t timeout_us);
/*
 * Checkpoint of a stream's running state: an initialised flag followed by
 * the per-input power P_i (uint32); *len is in/out (bytes).  Set restores
 * it; both need the stream drained.
 */
sk_status_t sk_stream_get_state(sk_server_t server, sk_stream_id stream,
                                void *buf, size_t *len);
sk_status_t sk_stream_set_state(sk_server_t server, sk_stream_id stream,
                                const void *buf, size_t len);
sk_status_t sk_stream_close(sk_server_t server, sk_stream_id stream);

typedef struct {
    int64_t frames_done;
    int64_t frames_flagged;
    int64_t launches;
    int64_t rejected;       /* BUSY answers to submit and open           */
    double latency_p50_us;  /* submit -> result host-visible              */
    double latency_p99_us;
    size_t hbm_in_use;
} sk_server_stats_t;
sk_status_t sk_server_stats(sk_server_t server, sk_server_stats_t *out);

/* Counters of one open stream: frames retired, of which flagged; submits
 * refused with SK_ERR_BUSY; frames outstanding; submit-to-result latency over
 * its last 16384 frames.  INVALID_ARG for an unknown or closed stream. */
typedef struct {
    int64_t frames_done;
    int64_t frames_flagged;
    int64_t rejected;
    int32_t outstanding;
    int32_t pad;
    double latency_p50_us;
    double latency_p99_us;
} sk_stream_stats_t;
sk_status_t sk_stream_stats(sk_server_t server, sk_stream_id stream,
                            sk_stream_stats_t *out);

/*
 * Load generator for a server (measurement, not part of the method): replays
 * pools of frames into open streams from `threads` submitter threads.  Stream
 * j submits frames_per_stream frames, frame k due at k*cadence_s plus an
 * exponential jitter of mean jitter_mean_s (seeded), or as fast as admission
 * allows when paced = 0; frame k is pool entry k % pool_frames[j] of
 * frames[j] (host memory, pool_frames[j] * M * N bytes).  A BUSY answer makes
 * the submitter wait for its stream's oldest result and retry.  Latencies are
 * the server's submit-to-result times over this replay only.
 */
typedef struct {
    int32_t n_streams;
    int32_t threads;
    const sk_stream_id *streams;
    const uint8_t *const *frames;
    const int32_t *pool_frames;
    int64_t frames_per_stream;
    double cadence_s;
    double jitter_mean_s;
    int32_t paced;
    int32_t by_reference;  /* submit with sk_stream_submit_ref (the pools must
                              then be device-readable, e.g. page-locked) */
    uint64_t seed;
} sk_replay_t;
typedef struct {
    double wall_s;
    int64_t frames;
    int64_t launches;
    int64_t busy_retries;
    double bytes;
    double latency_p50_us;
    double latency_p99_us;
    double submit_p50_us;
    double submit_p99_us;
} sk_replay_result_t;
sk_status_t sk_server_replay(sk_server_t server, const sk_replay_t *replay,
                             sk_replay_result_t *out);

/* --------------------------------------------------------------- misc */

/*
 * Mean offset delta of SK~ from 1 for 4+4-bit data whose components had rms
 * sigma before rounding and clipping to [-7, 7] (App. B), from the level
 * probabilities of the quantised Gaussian: delta = m4/(2 m2^2) - 3/2.
 */
sk_status_t sk_digitisation_offset(double sigma, double *delta);

/*
 * Self-test on `device` of the exact conversions the kernels use instead of
 * the int64 <-> fp32 conversion instructions (the input term of Eqs.
 * discreteMean and normedSum2 with M S2 - S1^2 exact in int64 and one fp32
 * divide): each is compared bit for bit with CUDA's conversion intrinsics on
 * every non-negative fp32 below 2^62, on every halfway case below 2^43 and its
 * neighbours, on hashed samples of int64 values and of (S1, S2, M), and on the
 * fp32 square of every S1 from 1 to 2^19.
 * *n_checked gets the number of cases, *n_bad the mismatches (0 expected).
 * Takes about a second.  Errors: INVALID_ARG (NULL output), CUDA.
 */
sk_status_t sk_selftest_conversions(int device, int64_t *n_checked, int64_t *n_bad);

/*
 * Self-test of the one bounded wait inside the kernels (the paper has no
 * failure model; this exercises the library's own error path).  Warps of a
 * frame's team combine their parts through a ring of slots in shared memory,
 * and a warp that runs a whole ring ahead waits for its slot to be freed, for
 * at most a bounded number of 64 ns polls, then sets the plan's error word and
 * returns.  This entry launches one warp of a two-warp team (1 CTA, on the
 * plan's device and `stream`) whose slot is held by a frame that never
 * completes, with a bound of spin_limit polls (1 .. 2^22), so the wait runs
 * out and the kernel returns.  It synchronises the stream and sets *gave_up to
 * 1 if the kernel raised the plan's error word (it does not consume it): the
 * plan's next call then returns SK_ERR_TIMEOUT.  The kernel writes nothing
 * else and allocates nothing.  Errors: INVALID_ARG (null plan or output,
 * spin_limit out of range), CUDA.
 */
sk_status_t sk_selftest_slot_wait(sk_plan_t plan, int32_t spin_limit, int32_t *gave_up,
                                  sk_cuda_stream_t stream);

/* Message for the calling thread's last failed call ("" if none). */
const char *sk_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SK_H */
