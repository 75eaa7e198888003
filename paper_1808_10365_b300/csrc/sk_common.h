// Host-side shared declarations of the library (plan object, error helpers,
// launch helpers).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sk.h"
#include "sk_device.cuh"

namespace sk {

sk_status_t set_error(sk_status_t s, const char *fmt, ...);
sk_status_t cuda_error(cudaError_t e, const char *what);

// Kernel launch over one item with a contiguous frame range per CTA, or over
// a prebuilt chunk schedule (items/chunks/cta_chunks on the device).  Given its
// plan, a time-major launch of the warp-slice shapes balances rows over the
// grid through the plan's scratch (allocated on first use when may_alloc).
sk_status_t launch_single(const Item &it, int rows, bool served, int device, cudaStream_t st,
                          int grid_cap = 0, sk_plan_t plan = nullptr, bool may_alloc = true);
// tile: 0 = 16 rows x 2 batches (M % 32 == 0), 1 = 8 x 2 (M % 16 == 0);
// nclass: batched launches, the kernel for items of batch_class nclass; served
// launches, 0 = teams on different frames, 1 = one frame per CTA with its rows
// split over the CTA's teams
sk_status_t launch_schedule(const Item *d_items, const Chunk *d_chunks,
                            const int32_t *d_cta_chunks, int grid, int tile, bool served,
                            int device, cudaStream_t st, int nclass = 0);
// Kernel class of a batched item: 2 for time-major fast-path items of N = 2048,
// 1 for N = 256, 4..9 for input-major items on the grouped path with M = 128,
// 256, ..., 4096 and 10 for M = 64, 0 for the rest (runtime row stride or the
// general path).
// sk_batch_create moves class-2 items with a tensor map to class 3 (the
// warp-slice path).
int batch_class(const Item &it);
// Time-major shapes of the warp-slice path (N a multiple of 8 from 256 to 4096,
// M % 16 == 0: 32-row turns, or 16-row turns when M = 16 mod 32), unless
// SK_WARP_SLICE=0.
bool warp_slice_shape(int N, int M);
// Tensor map of a time-major input for the warp-slice path's prefetch: rows of N
// bytes (N % 16 == 0), boxes of 32 rows x 256 bytes.  False if none can be made.
bool encode_input_map(const uint8_t *in, int N, int64_t rows, CUtensorMap *out);
// Stream path (time-major frames of few inputs, sk_path_stream.cuh): its launch
// shape for (N, M) (false if no unit of at most 512 lanes fits), whether a launch of
// the item takes it when the plan asks for no path, and the launch.
struct StreamShape;
bool stream_shape(int N, int M, StreamShape *out);
bool stream_auto(const Item &it);
sk_status_t launch_stream(const Item &it, const StreamShape &sh, int device, cudaStream_t st,
                          int grid_cap);
// Input-major frames of any M (run_imajor_chunks in sk_path_stream.cuh): the launch.
sk_status_t launch_imajor_chunks(const Item &it, int device, cudaStream_t st, int grid_cap);
// Dynamic shared memory attributes of the stream and chunk kernels on `device` (once).
sk_status_t stream_kernel_attrs(int device);
// Batched launches of the stream and chunk paths (sk_batch_create / sk_batch_run): the
// class of an item (0: time-major stream path, 1..3: input-major chunk path with 2, 4
// or 8 lanes per input, 4: input-major staged blocks (M <= 192); -1: a fused-kernel
// class), the frames one CTA takes per round (the schedule's unit), and the launch of
// one class over its schedule.  d_shapes holds each item's stream shape (used by
// class 0).
constexpr int kStreamClasses = 5;
constexpr int kStagedClass = 4;
int stream_batch_class(const Item &it, StreamShape *sh);
int64_t stream_batch_round(const Item &it, const StreamShape &sh, int cls);
sk_status_t launch_stream_schedule(int cls, const Item *d_items, const StreamShape *d_shapes,
                                   const Chunk *d_chunks, const int32_t *d_cta, int grid,
                                   int device, cudaStream_t st);
// SK_ERR_TIMEOUT once if a bounded wait in an earlier launch of the plan gave up.
sk_status_t pending_fault(sk_plan_t plan, const char *who);
// Set-up of sk_flag_host_noalloc on `device` (current): looks up the device
// address of its fixed staging array, which loads the module holding it.
void noalloc_prepare(int device);
constexpr int kBatchClasses = 11;
constexpr int kWarpSliceClass = 3;
constexpr int kFirstImajorClass = 4;
int pick_tile(int rows, bool all_m32);
int imajor_lanes(int M);
int imajor_shape(int M);
sk_status_t ensure_kernel_attrs(int device);
int sm_count(int device);

// Static byte-balanced schedule of the items listed in `sel` over `grid` CTAs;
// chunk item indices refer to `items`.  imajor: rounds follow the input-major
// kernel's team size; rounds: frames per round of each item (the stream classes).
void build_schedule(const std::vector<Item> &items, const std::vector<int32_t> &sel, int grid,
                    std::vector<Chunk> &chunks, std::vector<int32_t> &cta, bool imajor = false,
                    const std::vector<int64_t> *rounds = nullptr);

// One chunk per one-frame item, round-robin over at most grid_max CTAs (the
// served launch that splits each frame's rows over a CTA); returns the grid.
int build_split_schedule(int n_items, int grid_max, std::vector<Chunk> &chunks,
                         std::vector<int32_t> &cta);

// Schedule for a batch of one-frame items; reorders items, returns the grid.
int build_item_schedule(std::vector<Item> &items, int grid_max, std::vector<Chunk> &chunks,
                        std::vector<int32_t> &cta, std::vector<int32_t> &perm);

// App. B digitisation model, host double precision.
double digitisation_delta(double sigma);
double sigma_of_power(double mu);
void build_offset_table(int32_t M, int64_t *e);

// Scoped NVTX range (plan creation, launches, batch replay, served launches), seen
// by profilers that trace NVTX (ncu --nvtx); a function-pointer test otherwise.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Scoped switch of the current device.
struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

}  // namespace sk

struct sk_plan_s {
    sk_params_t p;
    int device = 0;
    int team_log2 = 0;         // vector and general paths (8 inputs per thread)
    int imajor_team_log2 = 0;  // input-major kernel
    bool fast = false;
    bool imajor = false;  // input-major fast path applies
    bool ragged = false;  // time-major N % 8 != 0, M % 16 == 0: ragged balanced path
    bool mr = false;      // time-major N % 8 == 0, M % 16 != 0: partial last turn
    int rows = 16;      // register batch rows of the fast path
    int grid_ctas = 0;  // 0: one CTA per SM
    // launch configuration (sk_launch_config_t): requested read path of one-item
    // launches and of batched items, input-major team size override (0: none),
    // L2 prefetch off; the path the latest one-item launch took
    int path = SK_PATH_AUTO;
    int batch_path = SK_PATH_AUTO;
    int team_override = 0;
    bool prefetch_off = false;
    std::atomic<int> last_path{0};
    std::vector<int64_t> t_lo, t_hi, etab;
    std::vector<float> c_tab;
    int64_t *d_t_lo = nullptr, *d_t_hi = nullptr, *d_e = nullptr;
    float *d_c = nullptr;
    // a word in mapped host memory that a kernel sets when a bounded wait gives up
    int32_t *h_err = nullptr, *d_err = nullptr;
    // scratch of the row-balanced launch (zero between launches); rb_ev follows its
    // last launch, on stream rb_last, so that a launch on another stream waits
    std::mutex rb_mu;
    int32_t *rb = nullptr;
    size_t rb_bytes = 0;
    bool rb_failed = false, rb_used = false;
    cudaEvent_t rb_ev = nullptr;
    cudaStream_t rb_last = nullptr;
    // staging for sk_flag_host
    std::mutex host_mu;
    uint8_t *d_stage[2] = {nullptr, nullptr};
    float *d_sk_stage[2] = {nullptr, nullptr};
    uint8_t *d_mask_stage[2] = {nullptr, nullptr};
    int64_t stage_frames = 0;
    cudaStream_t s_copy = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    cudaEvent_t ev_used[2] = {nullptr, nullptr};

    sk::Item item(const uint8_t *in, int64_t n_frames) const;
};
