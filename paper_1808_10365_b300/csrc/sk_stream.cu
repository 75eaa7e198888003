// Kernels and launches of the stream path (time-major frames of few inputs) and of the
// chunk path (input-major frames of any M), one-item and batched, with the host-side
// choice of their launch shapes.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "sk_common.h"
#include "sk_path_stream.cuh"

namespace sk {

__global__ void __launch_bounds__(kStreamThreads, 1) sk_stream_kernel(Item it, StreamShape sh)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ long long red_q[kStreamWarps];
    __shared__ int red_c[kStreamWarps];
    const uint32_t lb = build_table(dyn_smem);
    // the table sits on a 64 KiB boundary (lb holds it and the lane's offset);
    // the partial sums follow it, inside the kStreamSmem bytes of the launch
    const uint32_t part_sh = (lb & ~0xFFFFu) + (uint32_t)kLutBytes;
    int32_t *part = reinterpret_cast<int32_t *>(
        dyn_smem + (part_sh - (uint32_t)__cvta_generic_to_shared(dyn_smem)));
    const int64_t F = it.n_frames;
    const int64_t G = gridDim.x;
    const int64_t fb = F * (int64_t)blockIdx.x / G;
    const int64_t fe = F * ((int64_t)blockIdx.x + 1) / G;
    run_stream(it, sh, fb, fe, lb, part, red_q, red_c);
}

// Input-major frames of any M (run_imajor_chunks): a contiguous frame range per CTA,
// teams of W warps per frame.
template <int G>
__global__ void __launch_bounds__(kThreads, 1) sk_imajor_chunk_kernel(Item it, int W)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ long long red_q[kThreads / 32];
    __shared__ int red_c[kThreads / 32];
    __shared__ ChunkMasks cm;
    init_chunk_masks(cm);  // ordered before use by build_table's barrier
    const uint32_t lb = build_table(dyn_smem);
    const int64_t F = it.n_frames;
    const int64_t NB = gridDim.x;
    const int64_t fb = F * (int64_t)blockIdx.x / NB;
    const int64_t fe = F * ((int64_t)blockIdx.x + 1) / NB;
    run_imajor_chunks<G>(it, W, fb, fe, lb, cm, red_q, red_c);
}

// Input-major frames of M <= kStageMaxM: each warp's blocks of 32 inputs staged in
// its own buffer past the table (run_imajor_staged).
template <int CH, bool VEC, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1) sk_imajor_staged_kernel(Item it, int W)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ long long red_q[kThreads / 32];
    __shared__ int red_c[kThreads / 32];
    const uint32_t lb = build_table(dyn_smem);
    const uint32_t stage_sh = (lb & ~0xFFFFu) + (uint32_t)kLutBytes +
                              (threadIdx.x >> 5) * (uint32_t)stage_warp_bytes(it.M);
    uint8_t *buf = dyn_smem + (stage_sh - (uint32_t)__cvta_generic_to_shared(dyn_smem));
    const int64_t F = it.n_frames;
    const int64_t NB = gridDim.x;
    const int64_t fb = F * (int64_t)blockIdx.x / NB;
    const int64_t fe = F * ((int64_t)blockIdx.x + 1) / NB;
    run_imajor_staged<CH, VEC, SPLIT>(it, W, fb, fe, lb, buf, red_q, red_c);
}

// Batched launches: one persistent grid walks a chunk schedule (item, frame range)
// of items of the class, each with its own launch shape; the CTA's threads meet at
// one barrier between chunks (the slots and the per-warp sums are reused).
__global__ void __launch_bounds__(kStreamThreads, 1)
    sk_stream_batch_kernel(const Item *__restrict__ items, const StreamShape *__restrict__ shapes,
                           const Chunk *__restrict__ chunks, const int32_t *__restrict__ cta)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ long long red_q[kStreamWarps];
    __shared__ int red_c[kStreamWarps];
    const uint32_t lb = build_table(dyn_smem);
    const uint32_t part_sh = (lb & ~0xFFFFu) + (uint32_t)kLutBytes;
    int32_t *part = reinterpret_cast<int32_t *>(
        dyn_smem + (part_sh - (uint32_t)__cvta_generic_to_shared(dyn_smem)));
    // each chunk's item and shape staged in shared memory: its fields are read in the
    // frame loop, and copies in registers spilled
    __shared__ Item s_it;
    __shared__ StreamShape s_sh;
    const int32_t c0 = cta[blockIdx.x], c1 = cta[blockIdx.x + 1];
    for (int32_t c = c0; c < c1; ++c) {
        const Chunk ch = chunks[c];
        __syncthreads();  // the previous chunk is done with the slots and the staged item
        if (threadIdx.x == 0) {
            s_it = items[ch.item];
            s_sh = shapes[ch.item];
        }
        __syncthreads();
        run_stream(s_it, s_sh, ch.f_begin, ch.f_end, lb, part, red_q, red_c);
    }
}

template <int G>
__global__ void __launch_bounds__(kThreads, 1)
    sk_imajor_chunk_batch_kernel(const Item *__restrict__ items, const Chunk *__restrict__ chunks,
                                 const int32_t *__restrict__ cta)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ long long red_q[kThreads / 32];
    __shared__ int red_c[kThreads / 32];
    __shared__ ChunkMasks cm;
    init_chunk_masks(cm);
    const uint32_t lb = build_table(dyn_smem);
    __shared__ Item s_it;  // each chunk's item, staged as in sk_stream_batch_kernel
    const int32_t c0 = cta[blockIdx.x], c1 = cta[blockIdx.x + 1];
    for (int32_t c = c0; c < c1; ++c) {
        const Chunk ch = chunks[c];
        __syncthreads();
        if (threadIdx.x == 0)
            s_it = items[ch.item];
        __syncthreads();
        run_imajor_chunks<G>(s_it, imajor_chunk_team(s_it.N), ch.f_begin, ch.f_end, lb, cm,
                             red_q, red_c);
    }
}

// Batched staged blocks: the chunks' items have their own M (at most kStageMaxM), so
// one kernel takes every M with the largest register set, 4-byte words and whole-block
// loads without end checks; each item's buffers follow its M.
__global__ void __launch_bounds__(kThreads, 1)
    sk_imajor_staged_batch_kernel(const Item *__restrict__ items,
                                  const Chunk *__restrict__ chunks,
                                  const int32_t *__restrict__ cta)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ long long red_q[kThreads / 32];
    __shared__ int red_c[kThreads / 32];
    const uint32_t lb = build_table(dyn_smem);
    __shared__ Item s_it;  // each chunk's item, staged as in sk_stream_batch_kernel
    const int32_t c0 = cta[blockIdx.x], c1 = cta[blockIdx.x + 1];
    for (int32_t c = c0; c < c1; ++c) {
        const Chunk ch = chunks[c];
        __syncthreads();  // the previous chunk is done with the buffers and the item
        if (threadIdx.x == 0)
            s_it = items[ch.item];
        __syncthreads();
        const uint32_t stage_sh = (lb & ~0xFFFFu) + (uint32_t)kLutBytes +
                                  (threadIdx.x >> 5) * (uint32_t)stage_warp_bytes(s_it.M);
        uint8_t *buf = dyn_smem + (stage_sh - (uint32_t)__cvta_generic_to_shared(dyn_smem));
        run_imajor_staged<13, false, true>(s_it, imajor_staged_team(s_it.N), ch.f_begin,
                                           ch.f_end, lb, buf, red_q, red_c);
    }
}

typedef void (*KernelFnI)(Item, int);
static const KernelFnI kChunkFns[3] = {sk_imajor_chunk_kernel<2>, sk_imajor_chunk_kernel<4>,
                                       sk_imajor_chunk_kernel<8>};
typedef void (*KernelFnB)(const Item *, const Chunk *, const int32_t *);
static const KernelFnB kChunkBatchFns[3] = {sk_imajor_chunk_batch_kernel<2>,
                                            sk_imajor_chunk_batch_kernel<4>,
                                            sk_imajor_chunk_batch_kernel<8>};

// Staged kernels by whole-block loads without end checks (SPLIT), 4-byte words or
// 16-byte pieces (M % 16 == 0), and chunks a lane (4: M <= 62, 8: M <= 127, 13: M <= 192).
#define SK_STAGED3(S, V)                                                               \
    {sk_imajor_staged_kernel<4, V, S>, sk_imajor_staged_kernel<8, V, S>,               \
     sk_imajor_staged_kernel<13, V, S>}
static const KernelFnI kStagedFns[2][2][3] = {{SK_STAGED3(false, false), SK_STAGED3(false, true)},
                                              {SK_STAGED3(true, false), SK_STAGED3(true, true)}};
#undef SK_STAGED3
static_assert(stage_lane_chunks(62) <= 4 && stage_lane_chunks(127) <= 8 &&
                  stage_lane_chunks(kStageMaxM) <= 13,
              "chunks a lane of the staged kernels");
constexpr int kStagedSmemMax = kDynSmem + kStreamWarps * stage_warp_bytes(kStageMaxM);
static_assert(kStreamWarps == kThreads / 32, "warps of the staged kernels");

// Staged input-major kernels unless SK_IMAJOR_STAGED=0 (then the chunk kernels take
// every M; for comparisons).
static bool staged_on()
{
    static const bool v = [] {
        const char *e = getenv("SK_IMAJOR_STAGED");
        return !(e && e[0] == '0');
    }();
    return v;
}

// The dynamic shared memory of the stream and chunk kernels, once per device (plan
// creation sets it, before any stream capture; the launches check it again).
sk_status_t stream_kernel_attrs(int device)
{
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lk(mu);
    for (int d : done)
        if (d == device)
            return SK_OK;
    cudaError_t e = cudaFuncSetAttribute((const void *)sk_stream_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kStreamSmem);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = cudaFuncSetAttribute((const void *)kChunkFns[k],
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)sk_stream_batch_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = cudaFuncSetAttribute((const void *)kChunkBatchFns[k],
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
    for (int k = 0; k < 12 && e == cudaSuccess; ++k)
        e = cudaFuncSetAttribute((const void *)kStagedFns[k / 6][(k / 3) % 2][k % 3],
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)sk_imajor_staged_batch_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
    if (e != cudaSuccess)
        return cuda_error(e, "cudaFuncSetAttribute (stream and chunk paths)");
    done.push_back(device);
    return SK_OK;
}

sk_status_t launch_imajor_chunks(const Item &it, int device, cudaStream_t st, int grid_cap)
{
    if (it.n_frames == 0)
        return SK_OK;
    const bool staged = it.M <= kStageMaxM && staged_on();
    const int W = staged ? imajor_staged_team(it.N) : imajor_chunk_team(it.N);
    const int64_t teams = (kThreads / 32) / W;
    const int64_t gmax = grid_cap > 0 ? grid_cap : sm_count(device);
    int64_t g = std::min<int64_t>(gmax, (it.n_frames + teams - 1) / teams);
    if (g < 1)
        g = 1;
    sk_status_t s = stream_kernel_attrs(device);
    if (s != SK_OK)
        return s;
    if (staged) {
        const int ch = stage_lane_chunks(it.M);
        // whole blocks without end checks pay everywhere measured but on small arrays
        // with a partial last block (A/B, 3 GB launches: N = 2048, M = 100 0.555 ->
        // 0.607, M = 48 0.496 -> 0.558, M = 33 0.330 -> 0.381; N = 200, M = 100 0.556
        // -> 0.598; N = 64, M = 48 0.482 -> 0.516; N = 100, M = 100 0.480 -> 0.412)
        const bool split = it.N % 32 == 0 || it.N >= 128;
        const KernelFnI fn =
            kStagedFns[split][it.M % 16 == 0][ch <= 4 ? 0 : (ch <= 8 ? 1 : 2)];
        const int smem = kDynSmem + kStreamWarps * stage_warp_bytes(it.M);
        // the L2 look-ahead pays on long inputs and costs on short ones (A/B, 3 GB
        // launches: M = 127 0.419 -> 0.448, M = 176 0.501 -> 0.577; M = 100 0.511 ->
        // 0.504, M = 48 0.454 -> 0.408, M = 33 0.319 -> 0.280)
        Item run = it;
        if (it.M < 112)
            run.prefetch = 0;
        fn<<<(unsigned)g, kThreads, smem, st>>>(run, W);
    } else {
        const int G = imajor_chunk_lanes(it.M);
        const KernelFnI fn = kChunkFns[G == 2 ? 0 : (G == 4 ? 1 : 2)];
        fn<<<(unsigned)g, kThreads, kDynSmem, st>>>(it, W);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "sk input-major chunk kernel launch");
    return SK_OK;
}

static int gcd_int(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Lanes per frame override (SK_STREAM_LANES, a multiple of N / gcd(N, 16) up to
// 512), for launch-shape sweeps; 0 = the library's choice.
static int forced_lanes()
{
    static const int v = [] {
        const char *e = getenv("SK_STREAM_LANES");
        return e ? atoi(e) : 0;
    }();
    return v;
}

// Warp instructions per frame of a launch shape, a model of the two parts of the
// path: the chunk loop (one load, 16 PRMT, 16 LDS and 8 IADD3 a pass of a warp) and
// the combine (the slots' stores, R loads and adds per input, about 30 for the
// term, the sums; named barriers cost units of several warps about 40 a warp).
static double stream_cost(int N, int M, const StreamShape &c)
{
    const double fb = (double)M * N;
    const double P = std::ceil(fb / (16.0 * c.s));
    const int R = 16 * c.s / N;
    if (c.W == 1) {
        const double rounds = std::ceil((double)N / c.s);
        return (P * 41.0 + 8.0 + rounds * (4.0 * R + 30.0) + 20.0) / c.per_warp;
    }
    const double rounds = std::ceil((double)N / (32.0 * c.W));
    return c.W * (P * 41.0 + 8.0 + rounds * (4.0 * R + 30.0) + 15.0 + 80.0);
}

bool stream_shape(int N, int M, StreamShape *out)
{
    if (N < 1 || M < 1)
        return false;
    const int g = N / gcd_int(N, 16);  // lanes whose 16-byte chunks span whole rows
    if (g > 512)
        return false;
    StreamShape best;
    memset(&best, 0, sizeof best);
    double best_cost = 0.0;
    bool have = false;
    const int want = forced_lanes();
    for (int s = g; s <= 512; s += g) {
        if (s < 8)
            continue;
        StreamShape c;
        c.s = s;
        if (s <= 32) {
            c.W = 1;
            c.per_warp = 32 / s;
            c.units = kStreamWarps * c.per_warp;
        } else {
            c.W = (s + 31) / 32;
            c.per_warp = 0;
            c.units = kStreamWarps / c.W;
        }
        if (c.units < 1)
            continue;
        if (want > 0) {
            if (s == want) {
                *out = c;
                return true;
            }
            continue;
        }
        const double cost = stream_cost(N, M, c);
        if (!have || cost < best_cost) {
            best = c;
            best_cost = cost;
            have = true;
        }
    }
    if (!have)
        return false;
    *out = best;
    return true;
}

// Where a plan that asks for no path takes the stream path, measured against the
// path the shape had before (B300, 3 GB launches, fraction of measured copy bandwidth):
//   general-path shapes (time-major N % 8 != 0 and M % 16 != 0), any N: N = 100,
//   M = 100: 0.25 -> 0.56; N = 120: 0.31 -> 0.69; N = 260: 0.17 -> 0.46; N = 300:
//   0.19 -> 0.43; N = 500: 0.31 -> 0.61; N = 1500: 0.23 -> 0.53; N = 2044: 0.30 ->
//   0.58 (M = 100)
//   below N = 256 also N % 8 == 0 with M % 16 != 0 (N = 64, M = 100: 0.30 -> 0.74),
//   ragged N (N = 100, M = 256: 0.39 -> 0.69) and the team path below N = 64 (N = 8:
//   0.28 -> 0.69, N = 16: 0.45 -> 0.81, N = 24: 0.49 -> 0.59-0.63, M = 256); from
//   N = 64 the team path keeps up (N = 64: 0.85, N = 128: 0.99), and from N = 256 the
//   warp-slice paths (N = 300, M = 48 on the ragged path: 0.47 against 0.37)
// except frames that are not a multiple of 16 bytes on units of several warps
// (N = 99, M = 101: 0.19 against 0.23 on the general path).
bool stream_auto(const Item &it)
{
    if (it.layout != 0)
        return false;
    StreamShape sh;
    if (!stream_shape(it.N, it.M, &sh))
        return false;
    const bool clean = ((int64_t)it.M * it.N) % 16 == 0;
    if (!clean && sh.W != 1)
        return false;
    if (it.fast == 0)
        return true;
    if (it.N >= 256)
        return false;
    return !(it.fast == 1 && it.N >= 64);
}

sk_status_t launch_stream(const Item &it, const StreamShape &sh, int device, cudaStream_t st,
                          int grid_cap)
{
    if (it.n_frames == 0)
        return SK_OK;
    sk_status_t s = stream_kernel_attrs(device);
    if (s != SK_OK)
        return s;
    const int64_t gmax = grid_cap > 0 ? grid_cap : sm_count(device);
    int64_t g = std::min<int64_t>(gmax, (it.n_frames + sh.units - 1) / sh.units);
    if (g < 1)
        g = 1;
    // the look-ahead L2 prefetch pays on units of several warps (N = 250, M = 200:
    // 0.639 against 0.597 of measured copy bandwidth) and costs on one-warp units
    // (N = 100, M = 100: 0.536 against 0.548; N = 8, 16, 120: 2-3 %)
    Item run = it;
    if (sh.W == 1)
        run.prefetch = 0;
    sk_stream_kernel<<<(unsigned)g, kStreamThreads, kStreamSmem, st>>>(run, sh);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "sk stream kernel launch");
    return SK_OK;
}

int stream_batch_class(const Item &it, StreamShape *sh)
{
    if (it.layout == 1) {
        if (it.fast == 2)
            return -1;
        if (it.M <= kStageMaxM && staged_on())
            return kStagedClass;
        const int G = imajor_chunk_lanes(it.M);
        return G == 2 ? 1 : (G == 4 ? 2 : 3);
    }
    if (!stream_auto(it) || !stream_shape(it.N, it.M, sh))
        return -1;
    return 0;
}

int64_t stream_batch_round(const Item &it, const StreamShape &sh, int cls)
{
    if (cls == kStagedClass)
        return (kThreads / 32) / imajor_staged_team(it.N);
    return cls == 0 ? sh.units : (kThreads / 32) / imajor_chunk_team(it.N);
}

sk_status_t launch_stream_schedule(int cls, const Item *d_items, const StreamShape *d_shapes,
                                   const Chunk *d_chunks, const int32_t *d_cta, int grid,
                                   int device, cudaStream_t st)
{
    if (grid <= 0)
        return SK_OK;
    NvtxRange nv("sk batched stream launch");
    sk_status_t s = stream_kernel_attrs(device);
    if (s != SK_OK)
        return s;
    if (cls == 0)
        sk_stream_batch_kernel<<<(unsigned)grid, kStreamThreads, kStreamSmem, st>>>(
            d_items, d_shapes, d_chunks, d_cta);
    else if (cls == kStagedClass)
        sk_imajor_staged_batch_kernel<<<(unsigned)grid, kThreads, kStagedSmemMax, st>>>(
            d_items, d_chunks, d_cta);
    else
        kChunkBatchFns[cls - 1]<<<(unsigned)grid, kThreads, kDynSmem, st>>>(d_items, d_chunks,
                                                                          d_cta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "sk batched stream kernel launch");
    return SK_OK;
}

}  // namespace sk
