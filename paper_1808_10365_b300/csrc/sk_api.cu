// Plans, the plain launches (sk_compute, sk_flag, sk_flag_host) and the
// host-side tables: integer thresholds on Q (Sec. 3.2), the fp32 scale of
// Eq. final and the App. B digitisation offset.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "sk_common.h"
#include "sk_path_general.cuh"
#include "sk_path_input.cuh"
#include "sk_path_stream.cuh"
#include "sk_path_time.cuh"

namespace sk {

static thread_local std::string g_err;

sk_status_t set_error(sk_status_t s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

sk_status_t cuda_error(cudaError_t e, const char *what)
{
    return set_error(SK_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int sm_count(int device)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return n;
}

// Register pipelines of the fast path: (rows per batch, batches in the ring).
// Tile 0: 16 x 2 (needs M % 32 == 0), tile 1: 8 x 2 (M % 16 == 0).  NC fixes
// the row stride N at compile time (0: read it from the item); a kernel is only
// launched with NC > 0 for items of that N, and any other item takes the
// general path.  MODE selects the one work layout a kernel handles, so that
// each instantiation holds a single copy of the pipeline:
//   0  one item, a contiguous frame range per CTA (sk_compute, sk_flag)
//   1  chunk list of frame ranges (batched launch)
//   2  chunk list of one-frame items, teams on different items (served batch)
//   3  chunk list of one-frame items, one item per CTA at a time, its rows split
//      over the CTA's teams (served batch smaller than the GPU: more loads in
//      flight per frame)
//   5  one item on warp slices with a folded tail (Item::wtail), a partial last turn
//      (Item::fast = 4) or ragged N (Item::fast = 3, balanced rows): kernels of their
//      own, so that the extra state stays out of the register allocation of the
//      mode-0 kernels
template <int R, int S, bool SRV, int NC, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    sk_fused_kernel(const Item *__restrict__ items, const Chunk *__restrict__ chunks,
                    const int32_t *__restrict__ cta_chunks, Item single,
                    const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ TeamSmem ts;
    if (MODE == 0 || MODE == 5)
        init_wi_slots(ts);  // ordered before first use by build_table's barrier
    const uint32_t lb = build_table(dyn_smem);
    int parity = 0;
    if constexpr (MODE == 5 && (R * S == 32 || R * S == 16) && !SRV) {
        const int64_t F = single.n_frames;
        const int64_t G = gridDim.x;
        const int64_t fb = F * (int64_t)blockIdx.x / G;
        const int64_t fe = F * ((int64_t)blockIdx.x + 1) / G;
        if (single.fast == 4) {
            // M not a multiple of 16 (N a multiple of 8): whole-frame warp slices whose
            // last 16-row turn is partial
            if constexpr (R * S == 16)
                run_fast_wi<R, S, NC, false, true>(single, fb, fe, lb, ts, &tmap);
        } else if (single.fast == 3) {
            // ragged N (not a multiple of 8), balanced rows: one loop per N mod 8
            if constexpr (R * S == 16 && NC == 0) {
                switch (single.N & 7) {
                case 1: run_fast_rag<1>(single, lb, ts); break;
                case 2: run_fast_rag<2>(single, lb, ts); break;
                case 3: run_fast_rag<3>(single, lb, ts); break;
                case 4: run_fast_rag<4>(single, lb, ts); break;
                case 5: run_fast_rag<5>(single, lb, ts); break;
                case 6: run_fast_rag<6>(single, lb, ts); break;
                default: run_fast_rag<7>(single, lb, ts); break;
                }
            }
        } else if constexpr (NC == 0) {
            // a folded tail (N not a compiled multiple of 256)
            if (single.rb)
                run_fast_rb<R, S, NC, true>(single, lb, ts, &tmap);
            else
                run_fast_wi<R, S, NC, true>(single, fb, fe, lb, ts, &tmap);
        }
        return;
    }
    if (MODE == 0) {
        const int64_t F = single.n_frames;
        const int64_t G = gridDim.x;
        const int64_t fb = F * (int64_t)blockIdx.x / G;
        const int64_t fe = F * ((int64_t)blockIdx.x + 1) / G;
        const bool fast =
            single.fast == 1 && single.M % (R * S) == 0 && (NC == 0 || single.N == NC);
        if constexpr ((R * S == 32 || R * S == 16) && !SRV) {
            if (fast && single.wi) {
                if (single.rb)
                    run_fast_rb<R, S, NC>(single, lb, ts, &tmap);
                else
                    run_fast_wi<R, S, NC>(single, fb, fe, lb, ts, &tmap);
                return;
            }
        }
        if (fast)
            run_fast<R, S, SRV, NC>(single, fb, fe, lb, ts, parity);
        else
            run_general<SRV, !SRV, 8>(single, fb, fe, lb, ts, parity);
        return;
    }
    const int32_t c0 = cta_chunks[blockIdx.x], c1 = cta_chunks[blockIdx.x + 1];
    for (int32_t c = c0; c < c1; ++c) {
        const Chunk ch = chunks[c];
        __syncthreads();
        if (MODE == 1) {
            const Item it = items[ch.item];
            const bool fast = it.fast == 1 && it.M % (R * S) == 0 && (NC == 0 || it.N == NC);
            if (fast)
                run_fast<R, S, SRV, NC>(it, ch.f_begin, ch.f_end, lb, ts, parity);
            else
                run_general<SRV>(it, ch.f_begin, ch.f_end, lb, ts, parity);
        } else if (MODE == 4) {
            // batched items on the warp-slice path (each with its input's tensor map
            // in device memory), a fresh slot ring per chunk
            if constexpr (R * S == 32 && !SRV && NC >= 512) {
                // by reference: a copy of the item would hold its fields in registers
                // through the loop
                const Item &it = items[ch.item];
                init_wi_slots(ts);
                if ((threadIdx.x & 31) == 0)
                    tensormap_acquire(it.tmap);
                __syncthreads();
                run_fast_wi<R, S, NC>(it, ch.f_begin, ch.f_end, lb, ts, it.tmap);
            }
        } else if (MODE == 3) {
            const Item it = items[ch.item];
            const int tl = it.team_log2;
            const int team_idx = threadIdx.x >> tl;
            const int lit = threadIdx.x & ((1 << tl) - 1);
            const int col0 = lit * kVec;
            if (it.fast == 1 && it.M % (R * S) == 0 && (NC == 0 || it.N == NC)) {
                // teams 0..P-1 take equal shares of the ring iterations; teams 1..P-1
                // leave their partial sums in the dynamic shared memory beside the
                // table, and team 0 adds them and runs the epilogue
                const int nit = it.M / (R * S);
                const int T = kThreads >> tl;
                const int P = T < nit ? T : nit;
                int32_t s1[kVec], s2[kVec];
#pragma unroll
                for (int k = 0; k < kVec; ++k) {
                    s1[k] = 0;
                    s2[k] = 0;
                }
                if (team_idx < P && col0 < it.N) {
                    const int i0 = nit * team_idx / P, i1 = nit * (team_idx + 1) / P;
                    run_rows<R, S, NC>(it, 0, i0 * S, i1 * S, col0, lb, s1, s2);
                }
                if (P > 1) {
                    // the larger free piece of the dynamic shared memory: below or
                    // above the 64 KiB-aligned table, at least 32 KiB either way
                    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(dyn_smem);
                    const uint32_t below = (lb & ~0xFFFFu) - raw;
                    int32_t *part = (int32_t *)(below >= kLutBytes / 2
                                                    ? dyn_smem
                                                    : dyn_smem + below + kLutBytes);
                    const int team = 1 << tl;
                    int32_t *mine = part + ((team_idx - 1) * team + lit) * (2 * kVec);
                    if (team_idx >= 1 && team_idx < P && col0 < it.N) {
#pragma unroll
                        for (int k = 0; k < kVec; ++k) {
                            mine[k] = s1[k];
                            mine[kVec + k] = s2[k];
                        }
                    }
                    __syncthreads();
                    if (team_idx == 0 && col0 < it.N) {
                        for (int t = 1; t < P; ++t) {
                            const int32_t *o = part + ((t - 1) * team + lit) * (2 * kVec);
#pragma unroll
                            for (int k = 0; k < kVec; ++k) {
                                s1[k] += o[k];
                                s2[k] += o[kVec + k];
                            }
                        }
                    }
                }
                if (team_idx == 0) {
                    frame_epilogue<SRV>(it, 0, true, col0, lit, 0, parity, s1, s2, ts);
                    parity ^= 1;
                }
            } else if (team_idx == 0) {
                run_general<SRV>(it, 0, 1, lb, ts, parity, true);  // toggles parity
            }
        } else {
            // one frame per item, teams on different items; every item of the
            // chunk has the same shape, so all teams take the same path the same
            // number of times
            const Item it0 = items[ch.f_begin];
            const int tl = it0.team_log2;
            const int64_t T = kThreads >> tl;
            const int64_t team_idx = threadIdx.x >> tl;
            const bool fast = it0.fast == 1 && it0.M % (R * S) == 0 && (NC == 0 || it0.N == NC);
            for (int64_t base = ch.f_begin; base < ch.f_end; base += T) {
                const int64_t idx = base + team_idx;
                const bool v = idx < ch.f_end;
                const Item it = items[v ? idx : ch.f_begin];
                if (fast)
                    run_fast<R, S, SRV, NC>(it, 0, v ? 1 : 0, lb, ts, parity, true);
                else
                    run_general<SRV>(it, 0, v ? 1 : 0, lb, ts, parity, true);
            }
        }
    }
}

// Input-major fast paths.  G lanes per input; CH > 0 selects the grouped path
// for M = 16 G CH (PF: L2 prefetch of the next group), CH = 0 the per-input
// path for any M that 16 G divides.  MODE 0: one item, a contiguous frame range
// per CTA; MODE 1 (grouped path only): a chunk list of a batched launch whose
// items all have this M.  Served launches take input-major items through the
// general path.
template <int G, int CH, bool PF, int MODE = 0, int SPLIT = 1>
__global__ void __launch_bounds__(kThreads, 1)
    sk_imajor_kernel(const Item *__restrict__ items, const Chunk *__restrict__ chunks,
                     const int32_t *__restrict__ cta_chunks, Item single,
                     const __grid_constant__ CUtensorMap tmap)
{
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    __shared__ TeamSmem ts;
    if (MODE == 0)
        init_wi_slots(ts);  // ordered before first use by build_table's barrier
    const uint32_t lb = build_table(dyn_smem);
    int parity = 0;
    if constexpr (MODE == 1) {
        static_assert(CH > 0, "batched input-major launches use the grouped path");
        const int32_t c0 = cta_chunks[blockIdx.x], c1 = cta_chunks[blockIdx.x + 1];
        for (int32_t c = c0; c < c1; ++c) {
            const Chunk ch = chunks[c];
            __syncthreads();
            const Item it = items[ch.item];
            Item im = it;
            im.team_log2 = it.imajor_team_log2;
            im.wi = 0;
            if (it.fast == 2 && it.M == 16 * G * CH * SPLIT && im.team_log2 >= 5)
                run_imajor_grouped<G, CH, PF, SPLIT>(im, ch.f_begin, ch.f_end, lb, ts, parity);
            else
                run_general<false, false>(it, ch.f_begin, ch.f_end, lb, ts, parity);
        }
        return;
    }
    const int64_t F = single.n_frames;
    const int64_t Gd = gridDim.x;
    const int64_t fb = F * (int64_t)blockIdx.x / Gd;
    const int64_t fe = F * ((int64_t)blockIdx.x + 1) / Gd;
    Item im = single;  // the same item with the input-major team size
    im.team_log2 = single.imajor_team_log2;
    if constexpr (CH > 0) {
        if (single.fast == 2 && single.M == 16 * G * CH * SPLIT && im.team_log2 >= 5) {
            // balanced rows only where they pay: at M = 512 .. 2048 the path's
            // registers spill (measured 12 % slower than whole frames)
            if constexpr (CH <= 2 || SPLIT == 8) {
                if (single.rb) {
                    run_imajor_rb<G, CH, PF, SPLIT>(im, lb, ts);
                    return;
                }
            }
            run_imajor_grouped<G, CH, PF, SPLIT>(im, fb, fe, lb, ts, parity);
        } else
            run_general<false, false>(single, fb, fe, lb, ts, parity);
    } else {
        if (single.fast == 2 && single.M % (16 * G) == 0 && im.team_log2 >= 5)
            run_imajor<G, 8>(im, fb, fe, lb, ts, parity);
        else
            run_general<false, false>(single, fb, fe, lb, ts, parity);
    }
}

using KernelFn = void (*)(const Item *, const Chunk *, const int32_t *, Item,
                          const CUtensorMap);

// one-item launches: [tile][0 -> runtime N, 1 -> N = 256, 2 -> N = 2048]
static const KernelFn kSingle[2][3] = {
    {sk_fused_kernel<16, 2, false, 0, 0>, sk_fused_kernel<16, 2, false, 256, 0>,
     sk_fused_kernel<16, 2, false, 2048, 0>},
    {sk_fused_kernel<8, 2, false, 0, 0>, sk_fused_kernel<8, 2, false, 256, 0>,
     sk_fused_kernel<8, 2, false, 2048, 0>}};
// one-item launches with a folded tail ([tile], runtime N), a partial last turn
// (8-row tile, [0 -> runtime N, 1 -> N = 256, 2 -> N = 2048]) or ragged N on balanced
// rows (kPartial[0])
static const KernelFn kTail[2] = {sk_fused_kernel<16, 2, false, 0, 5>,
                                  sk_fused_kernel<8, 2, false, 0, 5>};
static const KernelFn kPartial[3] = {sk_fused_kernel<8, 2, false, 0, 5>,
                                     sk_fused_kernel<8, 2, false, 256, 5>,
                                     sk_fused_kernel<8, 2, false, 2048, 5>};
// batched launches: [tile][0 -> runtime N, 1 -> N = 256, 2 -> N = 2048] (the row
// stride as a load immediate is worth 7-12 % here too; one kernel holding the
// three pipelines spills, so a batch launches once per class)
static const KernelFn kBatched[2][3] = {
    {sk_fused_kernel<16, 2, false, 0, 1>, sk_fused_kernel<16, 2, false, 256, 1>,
     sk_fused_kernel<16, 2, false, 2048, 1>},
    {sk_fused_kernel<8, 2, false, 0, 1>, sk_fused_kernel<8, 2, false, 256, 1>,
     sk_fused_kernel<8, 2, false, 2048, 1>}};
// batched time-major N = 2048 items on the warp-slice path
static const KernelFn kBatchedWi = sk_fused_kernel<16, 2, false, 2048, 4>;
static const KernelFn kServed[2] = {sk_fused_kernel<16, 2, true, 0, 2>,
                                    sk_fused_kernel<8, 2, true, 0, 2>};
static const KernelFn kServedSplit[2] = {sk_fused_kernel<16, 2, true, 0, 3>,
                                         sk_fused_kernel<8, 2, true, 0, 3>};
// input-major: per-input path G = 2, 4, 8; grouped path G = 8 for M = 128,
// 256, 512 (CH = 1, 2, 4) and 1024, 2048, 4096 (CH = 4 on SPLIT = 2, 4, 8
// sub-inputs), and G = 4 for M = 64 (CH = 1), without and with the L2 prefetch
constexpr int kImajorShapes = 7;
constexpr int kImajorGroupedNoPf = 3, kImajorGroupedPf = 3 + kImajorShapes;
static const KernelFn kImajor[3 + 2 * kImajorShapes] = {
    sk_imajor_kernel<2, 0, false>,          sk_imajor_kernel<4, 0, false>,
    sk_imajor_kernel<8, 0, false>,          sk_imajor_kernel<8, 1, false>,
    sk_imajor_kernel<8, 2, false>,          sk_imajor_kernel<8, 4, false>,
    sk_imajor_kernel<8, 4, false, 0, 2>,    sk_imajor_kernel<8, 4, false, 0, 4>,
    sk_imajor_kernel<8, 4, false, 0, 8>,    sk_imajor_kernel<4, 1, false>,
    sk_imajor_kernel<8, 1, true>,           sk_imajor_kernel<8, 2, true>,
    sk_imajor_kernel<8, 4, true>,           sk_imajor_kernel<8, 4, true, 0, 2>,
    sk_imajor_kernel<8, 4, true, 0, 4>,     sk_imajor_kernel<8, 4, true, 0, 8>,
    sk_imajor_kernel<4, 1, true>};

// Lanes per input on the per-input input-major path: 4 up to M = 512, 8 above
// (measured best on B300), or SK_IMAJOR_LANES (2, 4 or 8); reduced while 16 G
// does not divide M.
int imajor_lanes(int M)
{
    static const int forced = [] {
        const char *v = getenv("SK_IMAJOR_LANES");
        const int x = v ? atoi(v) : 0;
        return (x == 2 || x == 4 || x == 8) ? x : 0;
    }();
    int g = forced ? forced : (M <= 512 ? 4 : 8);
    while (g > 2 && M % (16 * g) != 0)
        g /= 2;
    return g;
}

// Shape index of M on the grouped input-major path: 0..5 for M = 128, 256, 512,
// 1024, 2048, 4096 (groups of 8 inputs on 8 lanes), 6 for M = 64 (groups of 4 on
// 4 lanes), else -1 (the per-input path).  SK_IMAJOR_GROUPED=0 turns the grouped
// path off.
int imajor_shape(int M)
{
    static const bool off = [] {
        const char *v = getenv("SK_IMAJOR_GROUPED");
        return v && atoi(v) == 0;
    }();
    if (off)
        return -1;
    for (int sh = 0; sh < 6; ++sh)
        if (M == (128 << sh))
            return sh;
    return M == 64 ? 6 : -1;
}


static bool imajor_prefetch()
{
    static const bool on = [] {
        const char *v = getenv("SK_IMAJOR_PREFETCH");
        return !(v && atoi(v) == 0);
    }();
    return on;
}

// batched input-major launches: grouped path per M shape (batch classes
// kFirstImajorClass + shape index)
static const KernelFn kImajorBatched[kImajorShapes] = {
    sk_imajor_kernel<8, 1, true, 1>,    sk_imajor_kernel<8, 2, true, 1>,
    sk_imajor_kernel<8, 4, true, 1>,    sk_imajor_kernel<8, 4, true, 1, 2>,
    sk_imajor_kernel<8, 4, true, 1, 4>, sk_imajor_kernel<8, 4, true, 1, 8>,
    sk_imajor_kernel<4, 1, true, 1>};
static_assert(kFirstImajorClass + kImajorShapes == kBatchClasses, "batch classes");

static KernelFn imajor_kernel(int M, bool prefetch)
{
    const int sh = imajor_shape(M);
    if (sh >= 0)
        return kImajor[(prefetch && imajor_prefetch() ? kImajorGroupedPf : kImajorGroupedNoPf) +
                       sh];
    const int g = imajor_lanes(M);
    return kImajor[g == 2 ? 0 : (g == 4 ? 1 : 2)];
}

// Tile for a requested rows-per-batch and whether every M is a multiple of 32.
int pick_tile(int rows, bool all_m32)
{
    if (!all_m32 || rows == 8)
        return 1;
    return 0;
}

sk_status_t ensure_kernel_attrs(int device)
{
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> g(mu);
    for (int d : done)
        if (d == device)
            return SK_OK;
    std::vector<KernelFn> fns;
    for (KernelFn f : kImajor)
        fns.push_back(f);
    for (KernelFn f : kImajorBatched)
        fns.push_back(f);
    fns.push_back(kBatchedWi);
    for (int t = 0; t < 2; ++t) {
        fns.push_back(kServed[t]);
        fns.push_back(kServedSplit[t]);
        for (int j = 0; j < 3; ++j) {
            fns.push_back(kSingle[t][j]);
            fns.push_back(kBatched[t][j]);
            if (t == 0)
                fns.push_back(kPartial[j]);
        }
    }
    fns.push_back(kTail[0]);
    for (KernelFn f : fns) {
        cudaError_t e = cudaFuncSetAttribute((const void *)f,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kDynSmem);
        if (e != cudaSuccess)
            return cuda_error(e, "cudaFuncSetAttribute");
    }
    done.push_back(device);
    return SK_OK;
}

// Shapes of the warp-slice path: N a multiple of 8 from 256 to 4096, a team of
// ceil(N/256) warps (one at N = 256), each warp a 256-column slice.
// SK_WARP_SLICE=0 turns it off.
static bool warp_slice_on()
{
    static const bool off = [] {
        const char *v = getenv("SK_WARP_SLICE");
        return v && atoi(v) == 0;
    }();
    return !off;
}

bool warp_slice_shape(int N, int M)
{
    return warp_slice_on() && N >= 256 && N % 8 == 0 && N <= 4096 && M % 16 == 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of a time-major input for the warp-slice path's prefetch: rows of N
// bytes (N % 16 == 0: the map's row stride must be a multiple of 16), boxes of 32
// rows x 256 bytes.  False if no map can be made.
bool encode_input_map(const uint8_t *in, int N, int64_t rows, CUtensorMap *out)
{
    static const EncodeTiledFn encode = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (EncodeTiledFn)f;
    }();
    if (!encode || rows <= 0 || rows > 0x7FFFFFFFLL || ((uintptr_t)in & 15u) || N % 16 != 0)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)N};
    const cuuint32_t box[2] = {256, 32};
    const cuuint32_t es[2] = {1, 1};
    return encode(out, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)in, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Folded tail of the warp slices (Item::wtail), on unless SK_TAIL_FOLD=0.
static bool tail_fold_on()
{
    static const bool off = [] {
        const char *v = getenv("SK_TAIL_FOLD");
        return v && atoi(v) == 0;
    }();
    return !off;
}

static bool row_balance_on()
{
    static const bool off = [] {
        const char *v = getenv("SK_ROW_BALANCE");
        return v && atoi(v) == 0;
    }();
    return !off;
}

// The plan's scratch for a row-balanced launch of `need` bytes on stream st, or
// nullptr (the launch then hands out whole frames).  Called with plan->rb_mu held.
// Not while st is being captured; a launch on another stream than the last one
// waits for that one, since launches share the scratch.
static int32_t *rb_acquire(sk_plan_t plan, cudaStream_t st, size_t need, bool may_alloc)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cs != cudaStreamCaptureStatusNone)
        return nullptr;
    if (plan->rb_bytes < need) {
        if (!may_alloc || plan->rb_failed)
            return nullptr;
        cudaFree(plan->rb);  // waits for the launches that used it
        plan->rb = nullptr;
        plan->rb_bytes = 0;
        plan->rb_used = false;
        if ((!plan->rb_ev &&
             cudaEventCreateWithFlags(&plan->rb_ev, cudaEventDisableTiming) != cudaSuccess) ||
            cudaMalloc(&plan->rb, need) != cudaSuccess ||
            cudaMemsetAsync(plan->rb, 0, need, st) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(plan->rb);
            plan->rb = nullptr;
            plan->rb_failed = true;  // whole frames from now on
            return nullptr;
        }
        plan->rb_bytes = need;
    }
    if (plan->rb_used && plan->rb_last != st &&
        cudaStreamWaitEvent(st, plan->rb_ev, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return plan->rb;
}

sk_status_t launch_single(const Item &it, int rows, bool served, int device, cudaStream_t st,
                          int grid_cap, sk_plan_t plan, bool may_alloc)
{
    if (it.n_frames == 0)
        return SK_OK;
    NvtxRange nv("sk launch");
    sk_status_t s = ensure_kernel_attrs(device);
    if (s != SK_OK)
        return s;
    if (served)
        return set_error(SK_ERR_UNSUPPORTED, "served items go through launch_schedule");
    const int64_t T = kThreads >> (it.fast == 2 ? it.imajor_team_log2 : it.team_log2);
    const int64_t gmax = grid_cap > 0 ? grid_cap : sm_count(device);
    const int nci = it.N == 256 ? 1 : (it.N == 2048 ? 2 : 0);
    // ragged N takes its balanced path on the 8-row tile (16-row turns)
    const int tile = it.fast == 3 ? 1 : pick_tile(rows, it.M % 32 == 0);
    // the plan's requested path and prefetch (autotuned launch configuration); the stream
    // path asked for where the shape has none is the library's own choice
    int req = plan ? plan->path : SK_PATH_AUTO;
    StreamShape ssh;
    if (req == SK_PATH_STREAM && it.layout == 0 && !stream_shape(it.N, it.M, &ssh))
        req = SK_PATH_AUTO;
    const bool pf_off = plan && plan->prefetch_off;
    // time-major frames of few inputs: the stream path, requested or by shape
    if (it.layout == 0 && (req == SK_PATH_STREAM || (req == SK_PATH_AUTO && stream_auto(it))) &&
        stream_shape(it.N, it.M, &ssh)) {
        Item run = it;
        if (pf_off)
            run.prefetch = 0;
        if (plan)
            plan->last_path.store(SK_PATH_STREAM, std::memory_order_relaxed);
        return launch_stream(run, ssh, device, st, grid_cap);
    }
    // input-major frames without a fast path (M % 32 != 0 outside the grouped lengths):
    // the chunk path, requested or by shape
    if (it.layout == 1 && (req == SK_PATH_STREAM || (req == SK_PATH_AUTO && it.fast != 2))) {
        if (plan)
            plan->last_path.store(SK_PATH_STREAM, std::memory_order_relaxed);
        return launch_imajor_chunks(it, device, st, grid_cap);
    }
    KernelFn fn = kSingle[tile][nci];
    if (it.fast == 2)
        fn = imajor_kernel(it.M, !pf_off);
    Item run = it;
    if (pf_off)
        run.prefetch = 0;
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof tmap);
    // warp-slice path: 1 with the tensor map of the prefetch, 2 without one (N % 16
    // != 0; measured faster than a map of row pairs, whose prefetch slowed N = 1000
    // from 6.0 to 4.2 TB/s; or the prefetch turned off), 0 not taken (or the map
    // failed)
    run.wi = 0;
    // one-warp teams (N = 256) have no barrier to remove: there the warp-slice path
    // pays only when too few frames to occupy the grid would leave most warps idle
    // (64 frames: 16 against 30 us); with more it measured 1-15 % slower
    const bool ws_n256 = it.N > 256 || it.n_frames * 4 < (int64_t)gmax * (kThreads / 32);
    const bool want_ws = req == SK_PATH_AUTO
                             ? ws_n256
                             : (req == SK_PATH_WARP_SLICE || req == SK_PATH_ROW_BALANCED);
    // 16-row turns on the 8-row tile only where 32-row turns do not fit (M = 16
    // mod 32): an 8-row tile requested for M % 32 == 0 keeps the team path
    const bool ws_tile = tile == 0 || it.M % 32 != 0;
    if (it.fast == 1 && ws_tile && warp_slice_shape(it.N, it.M) && want_ws)
        run.wi = (it.N % 16 != 0 || pf_off)
                     ? 2
                     : (encode_input_map(it.in, it.N, it.n_frames * it.M, &tmap) ? 1 : 0);
    // M not a multiple of 16: whole-frame warp slices on the 8-row tile, the last turn
    // of a frame partial (otherwise the general path, at a third of the rate: two
    // loads, a shift and a mask a row)
    const bool ws_mr = it.fast == 4 && tile == 1 && warp_slice_on() &&
                       it.N >= 256 && it.N <= 4096 && req != SK_PATH_TEAM;
    if (ws_mr)
        run.wi = (it.N % 16 != 0 || pf_off)
                     ? 2
                     : (encode_input_map(it.in, it.N, it.n_frames * it.M, &tmap) ? 1 : 2);
    // input-major teams of two or more warps combine through the same slot ring
    if (it.fast == 2 && warp_slice_on() && it.imajor_team_log2 >= 6 && req != SK_PATH_TEAM)
        run.wi = 1;
    // N = 256 W + 8 NT with NT of 1..min(4, W): teams of W warps, the NT groups of 8
    // columns past the last whole slice read row-per-lane by them, one group a warp
    // (a warp of its own would cost as much as a whole slice for NT busy lanes).
    // Folded only where that adds a team per CTA (W = 1..5 and 8; at W = 9, N = 2312,
    // it measured 2 % slower), and without the tensor map's L2 prefetch, which
    // slowed folded shapes (N = 2064: 5.18 TB/s without it, 4.05 with it).
    run.wtail = 0;
    if (run.wi && it.fast == 1 && !ws_mr && tail_fold_on() && it.N > 256 &&
        (it.N & 255) != 0 && (it.N & 255) <= 8 * kMaxTail &&
        (it.N & 255) / 8 <= it.N / 256 &&
        (kThreads / 32) / (it.N / 256) > (kThreads / 32) / (it.N / 256 + 1)) {
        run.wtail = (it.N & 255) / 8;
        run.wi = 2;
    }
    if (run.wtail)
        fn = kTail[tile];
    else if (ws_mr)
        fn = kPartial[nci];
    // ragged N: warp slices without a tensor map, given balanced rows (below)
    const bool tm_ws = it.fast == 1 || it.fast == 3 || it.fast == 4;
    if (it.fast == 3 && warp_slice_on() && it.M % 16 == 0 &&
        (req == SK_PATH_AUTO || req == SK_PATH_ROW_BALANCED))
        run.wi = 2;
    // teams per CTA: 16 / ceil(N/256) on the warp-slice paths
    const int64_t Wl = run.wtail ? it.N / 256 : (it.N + 255) / 256;  // warps per frame
    const int64_t Tl = (run.wi && tm_ws) ? (kThreads / 32) / Wl : T;
    // frames per team decide the grid, unless rows are balanced over the grid
    int64_t g = std::min<int64_t>(gmax, (it.n_frames + Tl - 1) / Tl);
    std::unique_lock<std::mutex> lk;
    bool rb = false;
    // time-major: 32-row turns, scratch for partial sums of cut frames; grouped
    // input-major (sub-inputs of a frame a multiple of the team): group rows of
    // team*M bytes, scratch for Q and N_eff of cut frames
    int64_t units = 0;
    size_t need = 0;
    if (run.wi && tm_ws && !ws_mr) {
        units = it.n_frames * (it.M / (tile == 0 ? 32 : 16));
        const int64_t K = std::max<int64_t>(1, std::min<int64_t>(gmax, units / Tl)) * Tl;
        need = (size_t)K * it.N * 8 + (size_t)((K * Wl + 1) & ~(int64_t)1) * 4 + (size_t)K * 16;
    } else if (run.wi && it.fast == 2 && imajor_shape(it.M) >= 0 &&
               (it.M <= 256 || it.M == 4096)) {
        const int64_t split = it.M >= 1024 ? it.M / 512 : 1;
        if ((it.N * split) % (kThreads / T) == 0 &&
            it.n_frames * (it.N * split / (kThreads / T)) < (int64_t)1 << 31) {
            units = it.n_frames * (it.N * split / (kThreads / T));
            need = (size_t)std::max<int64_t>(1, std::min<int64_t>(gmax, units / T)) * T * 16;
        }
    }
    if (units > 0 && plan && row_balance_on() &&
        (req == SK_PATH_AUTO || req == SK_PATH_ROW_BALANCED)) {
        const int64_t grb = std::max<int64_t>(1, std::min<int64_t>(gmax, units / Tl));
        lk = std::unique_lock<std::mutex>(plan->rb_mu);
        run.rb = rb_acquire(plan, st, need, may_alloc);
        if (run.rb) {
            rb = true;
            g = grb;
        } else {
            lk.unlock();
        }
    }
    if (it.fast == 3 && !rb) {
        // ragged N without balanced rows: the general path, whole frames per team
        run.wi = 0;
        g = std::min<int64_t>(gmax, (it.n_frames + T - 1) / T);
    } else if (it.fast == 3) {
        fn = kPartial[0];  // the ragged balanced path (mode 5, 8-row tile, runtime N)
        // its whole-row L2 prefetch pays on long frames of teams of up to 8 warps
        // (N = 2047: +2 % at M = 128, +7 % at 256, +11 % at 1024) and costs elsewhere
        // (M = 64 or 48: -7 to -12 %; 9 or 16 warps: -2 to -4 %)
        if (!(it.M >= 256 && it.N <= 2048))
            run.prefetch = 0;
    }
    if (g < 1)
        g = 1;
#ifdef SK_DEBUG
    // slots of the row-balancing scratch: one per team of the grid
    run.dbg_rb_slots = rb ? g * (tm_ws ? Tl : T) : 0;
#endif
    if (plan) {
        // the path the kernel takes for this item (sk_fused_kernel, sk_imajor_kernel)
        int taken = SK_PATH_GENERAL;
        const bool grouped = imajor_shape(it.M) >= 0;
        if ((it.fast == 1 && it.M % (tile == 0 ? 32 : 16) == 0) ||
            (it.fast == 2 && grouped && it.imajor_team_log2 >= 5))
            taken = run.wi ? (rb ? SK_PATH_ROW_BALANCED : SK_PATH_WARP_SLICE) : SK_PATH_TEAM;
        else if (ws_mr)
            taken = SK_PATH_WARP_SLICE;
        else if (it.fast == 3 && rb)
            taken = SK_PATH_ROW_BALANCED;
        else if (it.fast == 2 && !grouped && it.imajor_team_log2 >= 5)
            taken = SK_PATH_PER_INPUT;
        plan->last_path.store(taken, std::memory_order_relaxed);
    }
    fn<<<(unsigned)g, kThreads, kDynSmem, st>>>(nullptr, nullptr, nullptr, run, tmap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "sk kernel launch");
    if (rb) {
        plan->rb_used = true;
        plan->rb_last = st;
        if ((e = cudaEventRecord(plan->rb_ev, st)) != cudaSuccess) {
            plan->rb_failed = true;  // no later launch uses the scratch
            return cuda_error(e, "sk scratch event");
        }
    }
    return SK_OK;
}

int batch_class(const Item &it)
{
    if (it.fast == 1)
        return it.N == 256 ? 1 : (it.N == 2048 ? 2 : 0);
    if (it.fast == 2) {
        const int sh = imajor_shape(it.M);
        return sh >= 0 ? kFirstImajorClass + sh : 0;
    }
    return 0;
}

sk_status_t launch_schedule(const Item *d_items, const Chunk *d_chunks,
                            const int32_t *d_cta_chunks, int grid, int tile, bool served,
                            int device, cudaStream_t st, int nclass)
{
    if (grid <= 0)
        return SK_OK;
    NvtxRange nv(served ? "sk served launch" : "sk batched launch");
    sk_status_t s = ensure_kernel_attrs(device);
    if (s != SK_OK)
        return s;
    Item dummy;
    memset(&dummy, 0, sizeof dummy);
    CUtensorMap no_map;
    memset(&no_map, 0, sizeof no_map);
    KernelFn fn = served ? (nclass == 1 ? kServedSplit[tile] : kServed[tile])
                         : (nclass < kWarpSliceClass
                                ? kBatched[tile][nclass]
                                : (nclass == kWarpSliceClass
                                       ? kBatchedWi
                                       : kImajorBatched[nclass - kFirstImajorClass]));
    fn<<<(unsigned)grid, kThreads, kDynSmem, st>>>(d_items, d_chunks, d_cta_chunks, dummy,
                                                   no_map);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "sk batched kernel launch");
    return SK_OK;
}

// ---------------------------------------------------------------------------
// App. B digitisation model (host).  A component v = clip(round(sigma g), -7, 7):
// P(v = k) from normal tail probabilities; m2 = E v^2, m4 = E v^4;
// delta = m4 / (2 m2^2) - 3/2 (offset of SK~ from 1 for large M).
// ---------------------------------------------------------------------------

static void quantised_moments(double sigma, double *m2, double *m4)
{
    const int L = 7;
    const double s2 = sigma * std::sqrt(2.0);
    double a2 = 0.0, a4 = 0.0;
    for (int k = 1; k <= L; ++k) {
        // Pr(sigma g > k - 1/2) - Pr(sigma g > k + 1/2); the top level takes the tail
        double upper_in = 0.5 * std::erfc((k - 0.5) / s2);
        double upper_out = (k == L) ? 0.0 : 0.5 * std::erfc((k + 0.5) / s2);
        double pk = upper_in - upper_out;
        double k2 = (double)k * (double)k;
        a2 += 2.0 * pk * k2;  // levels +k and -k
        a4 += 2.0 * pk * k2 * k2;
    }
    *m2 = a2;
    *m4 = a4;
}

double digitisation_delta(double sigma)
{
    double m2, m4;
    quantised_moments(sigma, &m2, &m4);
    return m4 / (2.0 * m2 * m2) - 1.5;
}

double sigma_of_power(double mu)
{
    double a = std::log(1e-3), b = std::log(1e3);
    for (int i = 0; i < 200; ++i) {
        double c = 0.5 * (a + b);
        double m2, m4;
        quantised_moments(std::exp(c), &m2, &m4);
        if (2.0 * m2 < mu)
            a = c;
        else
            b = c;
    }
    return std::exp(0.5 * (a + b));
}

void build_offset_table(int32_t M, int64_t *e)
{
    for (int b = 0; b < kOffsetBuckets; ++b) {
        double mu = ((double)b + 0.5) * 128.0 / (double)kOffsetBuckets;
        double d = digitisation_delta(sigma_of_power(mu));
        double x = d * 4294967296.0 * (double)(M - 1) / (double)(M + 1);
        e[b] = (int64_t)std::llrint(x);
    }
}

static int ceil_log2(int64_t v)
{
    int l = 0;
    while ((int64_t(1) << l) < v)
        ++l;
    return l;
}

// Autotune cache: lines "N M layout rows grid path team_log2 prefetch batch_path"
// (sk_launch_config_t; grid 0 = one CTA per SM), or the older "N M layout rows
// grid" (the rest AUTO / default).  The last valid line for (N, M, layout) wins.
struct CachedConfig {
    int rows = 16, grid = 0, path = SK_PATH_AUTO, team_log2 = 0, prefetch = 0,
        batch_path = SK_PATH_AUTO;
};

static bool config_valid(const CachedConfig &c)
{
    return (c.rows == 8 || c.rows == 16) && c.grid >= 0 && c.grid <= 65535 && c.path >= 0 &&
           (c.path <= SK_PATH_ROW_BALANCED || c.path == SK_PATH_STREAM) && (c.team_log2 == 0 ||
                                              (c.team_log2 >= 5 && c.team_log2 <= 9)) &&
           (c.prefetch == 0 || c.prefetch == 1) && c.batch_path >= 0 &&
           c.batch_path <= SK_PATH_ROW_BALANCED;
}

static bool cached_config(int32_t N, int32_t M, int32_t layout, CachedConfig *out)
{
    const char *path = getenv("SK_AUTOTUNE_CACHE");
    if (!path || !*path)
        return false;
    FILE *f = fopen(path, "r");
    if (!f)
        return false;
    bool found = false;
    char line[256];
    while (fgets(line, sizeof line, f)) {
        int n, m, l;
        CachedConfig c;
        const int k = sscanf(line, "%d %d %d %d %d %d %d %d %d", &n, &m, &l, &c.rows, &c.grid,
                             &c.path, &c.team_log2, &c.prefetch, &c.batch_path);
        if ((k == 5 || k == 9) && n == N && m == M && l == layout && config_valid(c)) {
            if (k == 5)
                c.path = c.team_log2 = c.prefetch = c.batch_path = 0;
            *out = c;
            found = true;
        }
    }
    fclose(f);
    return found;
}

// Valid input-major team size override for a plan (grouped path 5..8, per-input
// path 5..9).
static bool team_override_ok(const sk_plan_s *pl, int t)
{
    if (t == 0)
        return true;
    if (!pl->imajor)
        return false;
    return t >= 5 && t <= (imajor_shape(pl->p.n_time) >= 0 ? 8 : 9);
}

}  // namespace sk

using namespace sk;

sk::Item sk_plan_s::item(const uint8_t *in, int64_t n_frames) const
{
    Item it;
    memset(&it, 0, sizeof it);
    it.in = in;
    it.n_frames = n_frames;
    it.M = p.n_time;
    it.N = p.n_inputs;
    it.layout = p.layout;
    it.team_log2 = team_log2;
    it.imajor_team_log2 = team_override ? team_override : imajor_team_log2;
    it.t_lo = d_t_lo;
    it.t_hi = d_t_hi;
    it.c_tab = d_c;
    it.e_tab = d_e;
    it.fast = fast ? 1 : (imajor ? 2 : (ragged ? 3 : (mr ? 4 : 0)));
    it.prefetch = 1;
    it.running_mu = (p.flags & SK_RUNNING_MU) ? 1 : 0;
    it.n_sigma = p.n_sigma;
    it.mean_offset = p.mean_offset;
    it.wi = 0;
    it.wtail = 0;
    it.err = d_err;
    it.tmap = nullptr;
    it.rb = nullptr;
#ifdef SK_DEBUG
    // SK_DEBUG_SHRINK_INPUT=k (debug builds, tests): the checks take the input as
    // k bytes shorter than it is, so that the last bytes' loads fail their check
    static const int64_t shrink = [] {
        const char *v = getenv("SK_DEBUG_SHRINK_INPUT");
        return v ? (int64_t)atoll(v) : (int64_t)0;
    }();
    it.dbg_in_bytes = n_frames * (int64_t)p.n_time * p.n_inputs - shrink;
    it.dbg_rb_slots = 0;
#endif
    return it;
}

extern "C" const char *sk_last_error(void) { return sk::g_err.c_str(); }

extern "C" sk_status_t sk_digitisation_offset(double sigma, double *delta)
{
    if (!delta || !(sigma > 0.0) || !std::isfinite(sigma))
        return set_error(SK_ERR_INVALID_ARG, "sk_digitisation_offset: sigma must be > 0");
    *delta = digitisation_delta(sigma);
    return SK_OK;
}

static void free_plan_device(sk_plan_s *pl)
{
    if (pl->h_err)
        cudaFreeHost(pl->h_err);
    cudaFree(pl->d_t_lo);
    cudaFree(pl->d_t_hi);
    cudaFree(pl->d_c);
    cudaFree(pl->d_e);
    for (int b = 0; b < 2; ++b) {
        cudaFree(pl->d_stage[b]);
        cudaFree(pl->d_sk_stage[b]);
        cudaFree(pl->d_mask_stage[b]);
        if (pl->ev_copied[b])
            cudaEventDestroy(pl->ev_copied[b]);
        if (pl->ev_used[b])
            cudaEventDestroy(pl->ev_used[b]);
    }
    if (pl->s_copy)
        cudaStreamDestroy(pl->s_copy);
    cudaFree(pl->rb);
    if (pl->rb_ev)
        cudaEventDestroy(pl->rb_ev);
}

extern "C" sk_status_t sk_plan_create(const sk_params_t *params, int device, sk_plan_t *out)
{
    if (!out)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_create: out is NULL");
    *out = nullptr;
    if (!params)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_create: params is NULL");
    const sk_params_t &p = *params;
    if (p.n_inputs < 1 || p.n_inputs > SK_MAX_INPUTS)
        return set_error(SK_ERR_INVALID_ARG, "n_inputs %d outside 1..%d", p.n_inputs,
                         SK_MAX_INPUTS);
    if (p.n_time < 2 || p.n_time > SK_MAX_TIME)
        return set_error(SK_ERR_INVALID_ARG, "n_time %d outside 2..%d", p.n_time, SK_MAX_TIME);
    if (p.layout != SK_LAYOUT_TIME_MAJOR && p.layout != SK_LAYOUT_INPUT_MAJOR)
        return set_error(SK_ERR_INVALID_ARG, "layout %d unknown", p.layout);
    if (!(p.n_sigma >= 0.0) || !std::isfinite(p.n_sigma) || !std::isfinite(p.mean_offset))
        return set_error(SK_ERR_INVALID_ARG, "n_sigma must be finite and >= 0, mean_offset finite");
    if (p.flags & ~(SK_RUNNING_OFFSET | SK_THRESH_PEARSON3 | SK_RUNNING_MU))
        return set_error(SK_ERR_INVALID_ARG, "unknown flags 0x%x", p.flags);
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess)
        return cuda_error(ce, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev)
        return set_error(SK_ERR_INVALID_ARG, "device %d not present", device);
    NvtxRange nv("sk_plan_create");

    sk_plan_s *pl = new (std::nothrow) sk_plan_s();
    if (!pl)
        return set_error(SK_ERR_OOM, "host allocation");
    pl->p = p;
    pl->p.offset_table = nullptr;
    pl->device = device;
    const int32_t N = p.n_inputs, M = p.n_time;
    pl->team_log2 = ceil_log2((N + kVec - 1) / kVec);
    pl->fast = (p.layout == SK_LAYOUT_TIME_MAJOR) && (N % kVec == 0) && (M % kFlushRows == 0);
    // time-major N not a multiple of 8: the ragged balanced path (16-row turns)
    pl->ragged = (p.layout == SK_LAYOUT_TIME_MAJOR) && (N % kVec != 0) && (M % 16 == 0);
    pl->mr = (p.layout == SK_LAYOUT_TIME_MAJOR) && (N % kVec == 0) && (M % 16 != 0);
    const int gl = imajor_lanes(M);
    const bool grouped = imajor_shape(M) >= 0;
    pl->imajor = (p.layout == SK_LAYOUT_INPUT_MAJOR) && (grouped || M % (16 * gl) == 0);
    if (pl->imajor) {
        // grouped: about 2 KB of the frame per team thread, 32..256 threads (a
        // sweep over N in {256, 1024, 2048}, M in {128, 256, 512} on B300: fewer
        // team barriers per byte than one thread per input, and two or more
        // frames in flight per CTA); per-input: segments of gl lanes, about 8
        // inputs per segment, 32..512 threads
        const int tl = grouped ? ceil_log2(((int64_t)N * M + 2047) / 2048)
                               : ceil_log2(((int64_t)N * gl + 7) / 8);
        const int tmax = grouped ? 8 : 9;
        pl->imajor_team_log2 = tl < 5 ? 5 : (tl > tmax ? tmax : tl);
    }
    pl->rows = 16;
    pl->grid_ctas = 0;
    CachedConfig cc;
    if (cached_config(N, M, p.layout, &cc)) {
        pl->rows = cc.rows;
        pl->grid_ctas = cc.grid;
        pl->path = cc.path;
        pl->team_override = team_override_ok(pl, cc.team_log2) ? cc.team_log2 : 0;
        pl->prefetch_off = cc.prefetch == 1;
        pl->batch_path = cc.batch_path;
    }

    // thresholds on Q, one pair per N_eff (Sec. 3.2); order of operations fixed
    pl->t_lo.assign(N + 1, 0);
    pl->t_hi.assign(N + 1, 0);
    pl->c_tab.assign(N + 1, 0.0f);
    const double centre = 1.0 + p.mean_offset;
    const double a = p.n_sigma;
    const bool pearson = (p.flags & SK_THRESH_PEARSON3) != 0;
    for (int32_t ne = 1; ne <= N; ++ne) {
        const double m = (double)((int64_t)M * ne);
        double v_hi, v_lo;
        if (pearson) {
            // shifted gamma: shape k = 4/skew^2 = m/25, scale 10/m, location
            // centre - 0.4; quantile k (1 - 1/(9k) + z/(3 sqrt k))^3, z = +-a
            const double k = m / 25.0;
            const double b_hi = 1.0 - 1.0 / (9.0 * k) + a / (3.0 * std::sqrt(k));
            const double b_lo = 1.0 - 1.0 / (9.0 * k) - a / (3.0 * std::sqrt(k));
            v_hi = (centre - 0.4) + 0.4 * (b_hi * b_hi * b_hi);
            v_lo = (centre - 0.4) + 0.4 * (b_lo * b_lo * b_lo);
        } else {
            const double s = 2.0 / std::sqrt(m);
            v_hi = centre + a * s;
            v_lo = centre - a * s;
        }
        const double x_hi = v_hi * (double)(M - 1) * (double)ne * 4294967296.0 / (double)(M + 1);
        const double x_lo = v_lo * (double)(M - 1) * (double)ne * 4294967296.0 / (double)(M + 1);
        pl->t_hi[ne] = (int64_t)std::floor(x_hi);
        pl->t_lo[ne] = (int64_t)std::ceil(x_lo);
        pl->c_tab[ne] = (float)((double)(M + 1) / ((double)(M - 1) * (double)ne));
    }
    pl->etab.assign(kOffsetBuckets, 0);
    if (p.flags & (SK_RUNNING_OFFSET | SK_RUNNING_MU)) {
        if (p.offset_table)
            memcpy(pl->etab.data(), p.offset_table, sizeof(int64_t) * kOffsetBuckets);
        else
            build_offset_table(M, pl->etab.data());
    }

    sk_status_t st = SK_OK;
    {
        DeviceGuard dg(device);
        size_t tb = sizeof(int64_t) * (N + 1);
        if (cudaMalloc(&pl->d_t_lo, tb) != cudaSuccess ||
            cudaMalloc(&pl->d_t_hi, tb) != cudaSuccess ||
            cudaMalloc(&pl->d_c, sizeof(float) * (N + 1)) != cudaSuccess ||
            cudaMalloc(&pl->d_e, sizeof(int64_t) * kOffsetBuckets) != cudaSuccess ||
            cudaHostAlloc(&pl->h_err, sizeof(int32_t), cudaHostAllocMapped) != cudaSuccess) {
            st = set_error(SK_ERR_OOM, "device allocation of plan tables");
        } else if (cudaHostGetDevicePointer((void **)&pl->d_err, pl->h_err, 0) != cudaSuccess) {
            st = set_error(SK_ERR_CUDA, "mapping of the plan's error word");
        } else if (cudaMemcpy(pl->d_t_lo, pl->t_lo.data(), tb, cudaMemcpyHostToDevice) !=
                       cudaSuccess ||
                   cudaMemcpy(pl->d_t_hi, pl->t_hi.data(), tb, cudaMemcpyHostToDevice) !=
                       cudaSuccess ||
                   cudaMemcpy(pl->d_c, pl->c_tab.data(), sizeof(float) * (N + 1),
                              cudaMemcpyHostToDevice) != cudaSuccess ||
                   cudaMemcpy(pl->d_e, pl->etab.data(), sizeof(int64_t) * kOffsetBuckets,
                              cudaMemcpyHostToDevice) != cudaSuccess) {
            st = set_error(SK_ERR_CUDA, "copy of plan tables");
        } else {
            *pl->h_err = 0;
            st = ensure_kernel_attrs(device);
            if (st == SK_OK)
                st = stream_kernel_attrs(device);
            if (st == SK_OK)
                noalloc_prepare(device);
        }
        if (st != SK_OK)
            free_plan_device(pl);
    }
    if (st != SK_OK) {
        delete pl;
        return st;
    }
    *out = pl;
    return SK_OK;
}

extern "C" sk_status_t sk_plan_destroy(sk_plan_t plan)
{
    if (!plan)
        return SK_OK;
    {
        DeviceGuard dg(plan->device);
        free_plan_device(plan);
    }
    delete plan;
    return SK_OK;
}

extern "C" sk_status_t sk_plan_thresholds(sk_plan_t plan, int64_t *t_lo, int64_t *t_hi)
{
    if (!plan || !t_lo || !t_hi)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_thresholds: null argument");
    memcpy(t_lo, plan->t_lo.data(), sizeof(int64_t) * plan->t_lo.size());
    memcpy(t_hi, plan->t_hi.data(), sizeof(int64_t) * plan->t_hi.size());
    return SK_OK;
}

extern "C" sk_status_t sk_plan_offset_table(sk_plan_t plan, int64_t *e)
{
    if (!plan || !e)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_offset_table: null argument");
    memcpy(e, plan->etab.data(), sizeof(int64_t) * plan->etab.size());
    return SK_OK;
}

extern "C" sk_status_t sk_plan_set_tiles(sk_plan_t plan, int32_t rows, int32_t grid_ctas)
{
    if (!plan)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_set_tiles: plan is NULL");
    if ((rows != 8 && rows != 16) || grid_ctas < 0 || grid_ctas > 65535)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_set_tiles: rows 8 or 16, grid >= 0");
    plan->rows = rows;
    plan->grid_ctas = grid_ctas;
    return SK_OK;
}

extern "C" sk_status_t sk_plan_get_tiles(sk_plan_t plan, int32_t *rows, int32_t *grid_ctas)
{
    if (!plan || !rows || !grid_ctas)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_get_tiles: null argument");
    *rows = plan->rows;
    *grid_ctas = plan->grid_ctas;
    return SK_OK;
}

extern "C" sk_status_t sk_plan_set_config(sk_plan_t plan, const sk_launch_config_t *cfg)
{
    if (!plan || !cfg)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_set_config: null argument");
    CachedConfig c;
    c.rows = cfg->rows;
    c.grid = cfg->grid_ctas;
    c.path = cfg->path;
    c.team_log2 = cfg->team_log2;
    c.prefetch = cfg->prefetch;
    c.batch_path = cfg->batch_path;
    if (!config_valid(c) || !team_override_ok(plan, c.team_log2))
        return set_error(SK_ERR_INVALID_ARG,
                         "sk_plan_set_config: rows 8 or 16, grid 0..65535, path 0..3 or 6, "
                         "batch_path 0..3, team_log2 0 or 5..8 (5..9 on the per-input path; input-major "
                         "plans only), prefetch 0 or 1");
    plan->rows = c.rows;
    plan->grid_ctas = c.grid;
    plan->path = c.path;
    plan->team_override = c.team_log2;
    plan->prefetch_off = c.prefetch == 1;
    plan->batch_path = c.batch_path;
    return SK_OK;
}

extern "C" sk_status_t sk_plan_get_config(sk_plan_t plan, sk_launch_config_t *cfg)
{
    if (!plan || !cfg)
        return set_error(SK_ERR_INVALID_ARG, "sk_plan_get_config: null argument");
    cfg->rows = plan->rows;
    cfg->grid_ctas = plan->grid_ctas;
    cfg->path = plan->path;
    cfg->team_log2 = plan->imajor ? (plan->team_override ? plan->team_override
                                                         : plan->imajor_team_log2)
                                  : 0;
    cfg->prefetch = plan->prefetch_off ? 1 : 0;
    cfg->batch_path = plan->batch_path;
    cfg->last_path = plan->last_path.load(std::memory_order_relaxed);
    return SK_OK;
}

// A bounded wait inside an earlier launch of this plan gave up (its results are
// void): report it once, as SK_ERR_TIMEOUT, on the next call.
sk_status_t sk::pending_fault(sk_plan_t plan, const char *who)
{
    const int32_t err = plan->h_err ? *reinterpret_cast<volatile int32_t *>(plan->h_err) : 0;
    if (err) {
        *plan->h_err = 0;
        if (err == kErrBounds)
            return set_error(SK_ERR_CUDA, "%s: a bounds check inside an earlier launch failed "
                                          "(debug build); the access was skipped and that "
                                          "launch's results are void", who);
        return set_error(SK_ERR_TIMEOUT, "%s: a bounded wait inside an earlier launch "
                                         "ran out; that launch's results are void", who);
    }
    return SK_OK;
}

static sk_status_t check_call(sk_plan_t plan, const void *d_in, int64_t n_frames,
                              const char *who)
{
    if (!plan)
        return set_error(SK_ERR_INVALID_ARG, "%s: plan is NULL", who);
    if (sk_status_t f = pending_fault(plan, who))
        return f;
    if (n_frames < 0)
        return set_error(SK_ERR_INVALID_ARG, "%s: n_frames < 0", who);
    if (n_frames > 0 && !d_in)
        return set_error(SK_ERR_INVALID_ARG, "%s: input is NULL", who);
    if (((uintptr_t)d_in & 15u) != 0)
        return set_error(SK_ERR_INVALID_ARG, "%s: input not 16-byte aligned", who);
    return SK_OK;
}

extern "C" sk_status_t sk_compute(sk_plan_t plan, const uint8_t *d_in, int64_t n_frames,
                                  int32_t *d_s1, int32_t *d_s2, int64_t *d_q, float *d_sk,
                                  int32_t *d_neff, sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_compute");
    sk_status_t s = check_call(plan, d_in, n_frames, "sk_compute");
    if (s != SK_OK)
        return s;
    if ((d_s1 == nullptr) != (d_s2 == nullptr))
        return set_error(SK_ERR_INVALID_ARG, "sk_compute: give both S1 and S2 or neither");
    if (((uintptr_t)d_s1 & 15u) || ((uintptr_t)d_s2 & 15u))
        return set_error(SK_ERR_INVALID_ARG, "sk_compute: S1/S2 not 16-byte aligned");
    Item it = plan->item(d_in, n_frames);
    it.s1 = d_s1;
    it.s2 = d_s2;
    it.q = d_q;
    it.sk = d_sk;
    it.neff = d_neff;
    DeviceGuard dg(plan->device);
    return launch_single(it, plan->rows, false, plan->device, (cudaStream_t)stream,
                         plan->grid_ctas, plan);
}

extern "C" sk_status_t sk_flag(sk_plan_t plan, const uint8_t *d_in, int64_t n_frames,
                               float *d_sk, uint8_t *d_mask, sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_flag");
    sk_status_t s = check_call(plan, d_in, n_frames, "sk_flag");
    if (s != SK_OK)
        return s;
    if (!d_mask && n_frames > 0)
        return set_error(SK_ERR_INVALID_ARG, "sk_flag: mask is NULL");
    Item it = plan->item(d_in, n_frames);
    it.sk = d_sk;
    it.mask = d_mask;
    DeviceGuard dg(plan->device);
    return launch_single(it, plan->rows, false, plan->device, (cudaStream_t)stream,
                         plan->grid_ctas, plan);
}

namespace sk {

// Per frame: SK and the mask from a frame's Q and N_eff summed over input shards
// (write_frame: Sec. 3.2 test against the plan's integer thresholds, Eq. final).
// An N_eff outside 0..N cannot come from shards of this plan's inputs: mask 1,
// SK NaN.
__global__ void finish_kernel(const int64_t *__restrict__ q, const int32_t *__restrict__ neff,
                              int64_t n_frames, Item it)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_frames;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t C = neff[f];
        if (C < 0 || C > it.N) {
            if (it.sk)
                it.sk[f] = __int_as_float(0x7FC00000);
            if (it.mask)
                it.mask[f] = 1;
            continue;
        }
        write_frame(it, f, q[f], C);
    }
}

}  // namespace sk

extern "C" sk_status_t sk_finish(sk_plan_t plan, const int64_t *d_q, const int32_t *d_neff,
                                 int64_t n_frames, float *d_sk, uint8_t *d_mask,
                                 sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_finish");
    if (!plan)
        return set_error(SK_ERR_INVALID_ARG, "sk_finish: plan is NULL");
    if (sk_status_t f = pending_fault(plan, "sk_finish"))
        return f;
    if (n_frames < 0)
        return set_error(SK_ERR_INVALID_ARG, "sk_finish: n_frames < 0");
    if (n_frames > 0 && (!d_q || !d_neff || !d_mask))
        return set_error(SK_ERR_INVALID_ARG, "sk_finish: q, neff and mask are required");
    if (plan->p.flags & (SK_RUNNING_OFFSET | SK_RUNNING_MU))
        return set_error(SK_ERR_UNSUPPORTED,
                         "sk_finish: running state belongs to served streams, not to shards");
    if (n_frames == 0)
        return SK_OK;
    Item it = plan->item(nullptr, n_frames);
    it.sk = d_sk;
    it.mask = d_mask;
    DeviceGuard dg(plan->device);
    const int64_t blocks =
        std::min<int64_t>((n_frames + 255) / 256, (int64_t)sm_count(plan->device) * 8);
    finish_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(d_q, d_neff, n_frames, it);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "sk_finish launch");
    return SK_OK;
}

extern "C" sk_status_t sk_compute_inputs(sk_plan_t plan, const uint8_t *d_in,
                                         int64_t n_frames, float *d_sk_in, uint8_t *d_mask_in,
                                         float *d_sk, uint8_t *d_mask, sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_compute_inputs");
    sk_status_t s = check_call(plan, d_in, n_frames, "sk_compute_inputs");
    if (s != SK_OK)
        return s;
    if (!d_sk_in && n_frames > 0)
        return set_error(SK_ERR_INVALID_ARG, "sk_compute_inputs: sk_in is NULL");
    Item it = plan->item(d_in, n_frames);
    it.sk_in = d_sk_in;
    it.mask_in = d_mask_in;
    it.sk = d_sk;
    it.mask = d_mask;
    DeviceGuard dg(plan->device);
    return launch_single(it, plan->rows, false, plan->device, (cudaStream_t)stream,
                         plan->grid_ctas, plan);
}

// Host-buffer path: chunks of stage_frames frames alternate between two device
// staging buffers.  Chunk c's upload (plan's copy stream) overlaps chunk c-1's
// kernel (caller's stream); an event per buffer keeps an upload from
// overwriting a buffer whose kernel and download have not finished.
static sk_status_t ensure_staging(sk_plan_s *pl)
{
    if (pl->stage_frames > 0)
        return SK_OK;
    const int64_t fb = (int64_t)pl->p.n_time * pl->p.n_inputs;
    int64_t frames = ((int64_t)64 << 20) / fb;
    if (frames < 1)
        frames = 1;
    for (int b = 0; b < 2; ++b) {
        if (cudaMalloc(&pl->d_stage[b], (size_t)(frames * fb)) != cudaSuccess ||
            cudaMalloc(&pl->d_sk_stage[b], sizeof(float) * frames) != cudaSuccess ||
            cudaMalloc(&pl->d_mask_stage[b], (size_t)frames) != cudaSuccess)
            return set_error(SK_ERR_OOM, "staging buffers");
        if (cudaEventCreateWithFlags(&pl->ev_copied[b], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_used[b], cudaEventDisableTiming) != cudaSuccess)
            return set_error(SK_ERR_CUDA, "staging events");
    }
    if (cudaStreamCreateWithFlags(&pl->s_copy, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(SK_ERR_CUDA, "staging stream");
    pl->stage_frames = frames;
    return SK_OK;
}

extern "C" sk_status_t sk_flag_host(sk_plan_t plan, const uint8_t *h_in, int64_t n_frames,
                                    float *h_sk, uint8_t *h_mask, sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_flag_host");
    if (!plan)
        return set_error(SK_ERR_INVALID_ARG, "sk_flag_host: plan is NULL");
    if (sk_status_t f = pending_fault(plan, "sk_flag_host"))
        return f;
    if (n_frames < 0 || (n_frames > 0 && (!h_in || !h_mask)))
        return set_error(SK_ERR_INVALID_ARG, "sk_flag_host: bad arguments");
    if (n_frames == 0)
        return SK_OK;
    std::lock_guard<std::mutex> g(plan->host_mu);
    DeviceGuard dg(plan->device);
    cudaStream_t st = (cudaStream_t)stream;
    sk_status_t s = ensure_staging(plan);
    const int64_t fb = (int64_t)plan->p.n_time * plan->p.n_inputs;
    for (int64_t f0 = 0, c = 0; s == SK_OK && f0 < n_frames; f0 += plan->stage_frames, ++c) {
        const int b = (int)(c & 1);
        const int64_t nf = std::min(plan->stage_frames, n_frames - f0);
        cudaError_t e = cudaStreamWaitEvent(plan->s_copy, plan->ev_used[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(plan->d_stage[b], h_in + f0 * fb, (size_t)(nf * fb),
                                cudaMemcpyHostToDevice, plan->s_copy);
        if (e == cudaSuccess)
            e = cudaEventRecord(plan->ev_copied[b], plan->s_copy);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(st, plan->ev_copied[b], 0);
        if (e != cudaSuccess) {
            s = cuda_error(e, "sk_flag_host upload");
            break;
        }
        Item it = plan->item(plan->d_stage[b], nf);
        it.sk = h_sk ? plan->d_sk_stage[b] : nullptr;
        it.mask = plan->d_mask_stage[b];
        s = launch_single(it, plan->rows, false, plan->device, st, plan->grid_ctas, plan);
        if (s != SK_OK)
            break;
        e = cudaMemcpyAsync(h_mask + f0, plan->d_mask_stage[b], (size_t)nf,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && h_sk)
            e = cudaMemcpyAsync(h_sk + f0, plan->d_sk_stage[b], sizeof(float) * nf,
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaEventRecord(plan->ev_used[b], st);
        if (e != cudaSuccess)
            s = cuda_error(e, "sk_flag_host download");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (s == SK_OK && e != cudaSuccess)
        s = cuda_error(e, "sk_flag_host synchronize");
    // the launches are complete: a bounded wait of their own that gave up voids them
    if (s == SK_OK)
        s = pending_fault(plan, "sk_flag_host");
    return s;
}
