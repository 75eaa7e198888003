// Batched persistent launch: one grid of one CTA per SM walks a static,
// byte-balanced schedule of (item, frame range) chunks that mixes items of
// different M (integration lengths 128..1024).  Items are split by kernel class
// (time-major N = 2048 and N = 256 with the row stride compiled in, input-major
// items by M on the grouped input-major path, time-major items of the stream path,
// input-major items of the chunk path by lanes per input, and the rest), and each
// non-empty class is one such launch; the launches are captured once into a CUDA
// graph and replayed.
#include <algorithm>
#include <cstring>
#include <new>

#include "sk_common.h"
#include "sk_path_stream.cuh"

struct sk_batch_s {
    int device = 0;
    int grid = 0;
    std::vector<sk::Item> items;
    std::vector<sk::Chunk> chunks;  // all classes, concatenated
    std::vector<int32_t> cta;       // per class: grid + 1 offsets into chunks
    int tile[sk::kBatchClasses] = {};   // kernel tile (see launch_schedule)
    bool used[sk::kBatchClasses] = {};
    sk::Item *d_items = nullptr;
    sk::Chunk *d_chunks = nullptr;
    int32_t *d_cta = nullptr;
    CUtensorMap *d_maps = nullptr;  // tensor maps of the warp-slice items' inputs
    // stream classes (time-major stream path, input-major chunk path by lanes per
    // input): used flags and each item's stream shape, on the host and the device
    bool sused[sk::kStreamClasses] = {};
    std::vector<sk::StreamShape> shapes;
    sk::StreamShape *d_shapes = nullptr;
    std::vector<sk_plan_t> plans;   // the items' plans, each once
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace sk {

// Static schedule.  An item with team size t has T = kThreads / t teams per
// CTA, so its frames go in rounds of T (one frame per team).  Rounds are laid
// end to end and cut into `grid` pieces of equal bytes: a round with c bytes
// before it and b bytes of its own goes to CTA floor((c + b/2) / (total/grid)).
// Consecutive rounds of one item on one CTA merge into one chunk.
void build_schedule(const std::vector<Item> &items, const std::vector<int32_t> &sel, int grid,
                    std::vector<Chunk> &chunks, std::vector<int32_t> &cta, bool imajor,
                    const std::vector<int64_t> *rounds)
{
    double total = 0.0;
    for (int32_t k : sel)
        total += (double)items[k].n_frames * items[k].M * items[k].N;
    chunks.clear();
    cta.assign(grid + 1, 0);
    if (total <= 0.0 || grid <= 0)
        return;
    const double target = total / grid;
    std::vector<std::vector<Chunk>> per(grid);
    double cum = 0.0;
    for (int32_t k : sel) {
        const Item &it = items[k];
        const int64_t T = rounds ? (*rounds)[k]
                                 : kThreads >> (imajor ? it.imajor_team_log2 : it.team_log2);
        const double fbytes = (double)it.M * it.N;
        for (int64_t f0 = 0; f0 < it.n_frames; f0 += T) {
            const int64_t f1 = std::min(f0 + T, it.n_frames);
            const double b = fbytes * (double)(f1 - f0);
            int c = (int)((cum + 0.5 * b) / target);
            c = std::max(0, std::min(grid - 1, c));
            cum += b;
            std::vector<Chunk> &v = per[c];
            if (!v.empty() && v.back().item == k && v.back().f_end == f0) {
                v.back().f_end = f1;
            } else {
                Chunk ch;
                ch.item = k;
                ch.kind = 0;
                ch.f_begin = f0;
                ch.f_end = f1;
                v.push_back(ch);
            }
        }
    }
    for (int c = 0; c < grid; ++c) {
        cta[c] = (int32_t)chunks.size();
        chunks.insert(chunks.end(), per[c].begin(), per[c].end());
    }
    cta[grid] = (int32_t)chunks.size();
}

// Schedule for items of one frame each (a served batch): items of one shape
// (team size, N, M, layout) are grouped, up to T per chunk so that every team
// of a CTA takes one; chunks go round-robin to at most `grid_max` CTAs.  The
// items are reordered in place (their outputs are addressed through their own
// pointers, so order does not matter); perm[k] = original index of item k.
int build_item_schedule(std::vector<Item> &items, int grid_max, std::vector<Chunk> &chunks,
                        std::vector<int32_t> &cta, std::vector<int32_t> &perm)
{
    const int n = (int)items.size();
    perm.resize(n);
    for (int k = 0; k < n; ++k)
        perm[k] = k;
    auto key = [&](int k) {
        const Item &it = items[k];
        return std::make_tuple(it.team_log2, it.N, it.M, it.layout);
    };
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return key(a) < key(b); });
    std::vector<Item> sorted(n);
    for (int k = 0; k < n; ++k)
        sorted[k] = items[perm[k]];
    items.swap(sorted);
    std::vector<Chunk> all;
    for (int k = 0; k < n;) {
        const int64_t T = kThreads >> items[k].team_log2;
        int e = k + 1;
        while (e < n && e - k < T && items[e].team_log2 == items[k].team_log2 &&
               items[e].N == items[k].N && items[e].M == items[k].M &&
               items[e].layout == items[k].layout)
            ++e;
        Chunk ch;
        ch.item = k;
        ch.kind = 1;
        ch.f_begin = k;
        ch.f_end = e;
        all.push_back(ch);
        k = e;
    }
    const int grid = std::max(1, std::min(grid_max, (int)all.size()));
    std::vector<std::vector<Chunk>> per(grid);
    for (size_t c = 0; c < all.size(); ++c)
        per[c % grid].push_back(all[c]);
    chunks.clear();
    cta.assign(grid + 1, 0);
    for (int c = 0; c < grid; ++c) {
        cta[c] = (int32_t)chunks.size();
        chunks.insert(chunks.end(), per[c].begin(), per[c].end());
    }
    cta[grid] = (int32_t)chunks.size();
    return grid;
}

int build_split_schedule(int n_items, int grid_max, std::vector<Chunk> &chunks,
                         std::vector<int32_t> &cta)
{
    const int grid = std::max(1, std::min(grid_max, n_items));
    std::vector<std::vector<Chunk>> per(grid);
    for (int k = 0; k < n_items; ++k) {
        Chunk ch;
        ch.item = k;
        ch.kind = 1;
        ch.f_begin = k;
        ch.f_end = k + 1;
        per[k % grid].push_back(ch);
    }
    chunks.clear();
    cta.assign(grid + 1, 0);
    for (int c = 0; c < grid; ++c) {
        cta[c] = (int32_t)chunks.size();
        chunks.insert(chunks.end(), per[c].begin(), per[c].end());
    }
    cta[grid] = (int32_t)chunks.size();
    return grid;
}

}  // namespace sk

using namespace sk;

static void free_batch(sk_batch_s *b)
{
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    cudaFree(b->d_items);
    cudaFree(b->d_chunks);
    cudaFree(b->d_cta);
    cudaFree(b->d_maps);
    cudaFree(b->d_shapes);
}

extern "C" sk_status_t sk_batch_create(const sk_batch_item_t *items, int32_t n_items,
                                       int device, sk_batch_t *out)
{
    NvtxRange nv("sk_batch_create");
    if (!out)
        return set_error(SK_ERR_INVALID_ARG, "sk_batch_create: out is NULL");
    *out = nullptr;
    if (!items || n_items <= 0)
        return set_error(SK_ERR_INVALID_ARG, "sk_batch_create: no items");
    sk_batch_s *b = new (std::nothrow) sk_batch_s();
    if (!b)
        return set_error(SK_ERR_OOM, "host allocation");
    b->device = device;
    int rows[kBatchClasses] = {};
    bool all_m32[kBatchClasses];
    std::fill(all_m32, all_m32 + kBatchClasses, true);
    std::vector<int32_t> sel[kBatchClasses];
    std::vector<int32_t> ssel[kStreamClasses];
    std::vector<int64_t> srounds(n_items, 1);
    b->shapes.assign(n_items, StreamShape{});
    std::vector<CUtensorMap> maps;
    std::vector<int32_t> map_of;
    for (int32_t k = 0; k < n_items; ++k) {
        const sk_batch_item_t &bi = items[k];
        if (!bi.plan || bi.n_frames < 0 || (bi.n_frames > 0 && !bi.d_in) ||
            ((uintptr_t)bi.d_in & 15u) || (bi.n_frames > 0 && !bi.d_mask && !bi.d_sk)) {
            delete b;
            return set_error(SK_ERR_INVALID_ARG, "sk_batch_create: bad item %d", k);
        }
        if (bi.plan->device != device) {
            delete b;
            return set_error(SK_ERR_INVALID_ARG, "sk_batch_create: item %d on another device",
                             k);
        }
        Item it = bi.plan->item(bi.d_in, bi.n_frames);
        it.sk = bi.d_sk;
        it.mask = bi.d_mask;
        if (std::find(b->plans.begin(), b->plans.end(), bi.plan) == b->plans.end())
            b->plans.push_back(bi.plan);
        // items without a fused-kernel fast path that the stream or chunk path takes
        // (as a one-item launch of the plan would, when it asks for no path)
        StreamShape ssh;
        memset(&ssh, 0, sizeof ssh);
        const int sc = bi.plan->batch_path == SK_PATH_AUTO ? stream_batch_class(it, &ssh) : -1;
        if (sc >= 0) {
            if (sc == 0 && ssh.W == 1)
                it.prefetch = 0;  // the look-ahead prefetch pays only on multi-warp units
            if (sc == kStagedClass && it.M < 112)
                it.prefetch = 0;  // and on the staged blocks only from M = 112
            b->shapes[k] = ssh;
            srounds[k] = stream_batch_round(it, ssh, sc);
            b->items.push_back(it);
            map_of.push_back(-1);
            ssel[sc].push_back(k);
            continue;
        }
        int c = batch_class(it);
        // time-major N = 2048 items on 16-row tiles take the warp-slice path when
        // the plan's batch path asks for it, or by default at M <= 128 (measured
        // 5-6 % faster there; at M = 256 and 1024 the team path was 1.5 % and 8 %
        // faster in a batch): each gets a tensor map of its input, in device
        // memory, for the per-warp prefetch
        const int bp = bi.plan->batch_path;
        const bool want_ws = bp == SK_PATH_AUTO ? it.M <= 128 : bp != SK_PATH_TEAM;
        CUtensorMap m;
        if (c == 2 && bi.plan->rows == 16 && it.M % 32 == 0 && want_ws &&
            it.n_frames > 0 && warp_slice_shape(it.N, it.M) &&
            encode_input_map(it.in, it.N, it.n_frames * it.M, &m)) {
            c = kWarpSliceClass;
            map_of.push_back((int32_t)maps.size());
            maps.push_back(m);
        } else {
            map_of.push_back(-1);
        }
        b->items.push_back(it);
        sel[c].push_back(k);
        rows[c] = std::max(rows[c], bi.plan->rows);
        all_m32[c] = all_m32[c] && (bi.plan->p.n_time % 32 == 0);
    }
    b->grid = sm_count(device);
    for (int c = 0; c < kBatchClasses; ++c) {
        b->tile[c] = pick_tile(rows[c] == 8 ? 8 : 16, all_m32[c]);
        std::vector<Chunk> ch;
        std::vector<int32_t> cta;
        build_schedule(b->items, sel[c], b->grid, ch, cta, c >= kFirstImajorClass);
        b->used[c] = !ch.empty();
        const int32_t base = (int32_t)b->chunks.size();
        for (int32_t &x : cta)
            x += base;
        b->chunks.insert(b->chunks.end(), ch.begin(), ch.end());
        b->cta.insert(b->cta.end(), cta.begin(), cta.end());
    }
    for (int c = 0; c < kStreamClasses; ++c) {
        std::vector<Chunk> ch;
        std::vector<int32_t> cta;
        build_schedule(b->items, ssel[c], b->grid, ch, cta, false, &srounds);
        b->sused[c] = !ch.empty();
        const int32_t base = (int32_t)b->chunks.size();
        for (int32_t &x : cta)
            x += base;
        b->chunks.insert(b->chunks.end(), ch.begin(), ch.end());
        b->cta.insert(b->cta.end(), cta.begin(), cta.end());
    }
    bool any_stream = false;
    for (int c = 0; c < kStreamClasses; ++c)
        any_stream = any_stream || b->sused[c];
    sk_status_t s = SK_OK;
    {
        DeviceGuard dg(device);
        if (!maps.empty()) {
            if (cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * maps.size()) != cudaSuccess ||
                cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                           cudaMemcpyHostToDevice) != cudaSuccess) {
                s = set_error(SK_ERR_OOM, "batch tensor maps");
            } else {
                for (size_t k = 0; k < b->items.size(); ++k)
                    if (map_of[k] >= 0) {
                        b->items[k].wi = 1;
                        b->items[k].tmap = b->d_maps + map_of[k];
                    }
            }
        }
        size_t ni = sizeof(Item) * b->items.size();
        size_t nc = sizeof(Chunk) * std::max<size_t>(1, b->chunks.size());
        size_t nt = sizeof(int32_t) * b->cta.size();
        if (s != SK_OK) {
            // no room for the tensor maps
        } else if (cudaMalloc(&b->d_items, ni) != cudaSuccess ||
                   cudaMalloc(&b->d_chunks, nc) != cudaSuccess ||
                   cudaMalloc(&b->d_cta, nt) != cudaSuccess) {
            s = set_error(SK_ERR_OOM, "batch schedule");
        } else if (cudaMemcpy(b->d_items, b->items.data(), ni, cudaMemcpyHostToDevice) !=
                       cudaSuccess ||
                   (!b->chunks.empty() &&
                    cudaMemcpy(b->d_chunks, b->chunks.data(), sizeof(Chunk) * b->chunks.size(),
                               cudaMemcpyHostToDevice) != cudaSuccess) ||
                   cudaMemcpy(b->d_cta, b->cta.data(), nt, cudaMemcpyHostToDevice) !=
                       cudaSuccess) {
            s = set_error(SK_ERR_CUDA, "batch schedule upload");
        } else if (any_stream &&
                   (cudaMalloc(&b->d_shapes, sizeof(StreamShape) * b->shapes.size()) !=
                        cudaSuccess ||
                    cudaMemcpy(b->d_shapes, b->shapes.data(),
                               sizeof(StreamShape) * b->shapes.size(),
                               cudaMemcpyHostToDevice) != cudaSuccess)) {
            s = set_error(SK_ERR_OOM, "batch stream shapes");
        } else {
            s = ensure_kernel_attrs(device);
            if (s == SK_OK)
                s = stream_kernel_attrs(device);
        }
        if (s != SK_OK)
            free_batch(b);
    }
    if (s != SK_OK) {
        delete b;
        return s;
    }
    *out = b;
    return SK_OK;
}

extern "C" sk_status_t sk_batch_run(sk_batch_t b, sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_batch_run");
    if (!b)
        return set_error(SK_ERR_INVALID_ARG, "sk_batch_run: batch is NULL");
    DeviceGuard dg(b->device);
    sk_status_t s = SK_OK;
    // a bounded wait of an earlier run that gave up voids that run's results
    for (sk_plan_t p : b->plans)
        if ((s = pending_fault(p, "sk_batch_run")) != SK_OK)
            return s;
    if (b->chunks.empty())
        return SK_OK;  // no frames in any item
    if (!b->exec) {
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            return cuda_error(e, "sk_batch_run capture stream");
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int c = 0; c < kBatchClasses && s == SK_OK; ++c)
                if (b->used[c])
                    s = launch_schedule(b->d_items, b->d_chunks, b->d_cta + c * (b->grid + 1),
                                        b->grid, b->tile[c], false, b->device, cs, c);
            for (int c = 0; c < kStreamClasses && s == SK_OK; ++c)
                if (b->sused[c])
                    s = launch_stream_schedule(c, b->d_items, b->d_shapes, b->d_chunks,
                                               b->d_cta + (kBatchClasses + c) * (b->grid + 1),
                                               b->grid, b->device, cs);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (s == SK_OK && e2 == cudaSuccess) {
                b->graph = g;
                e = cudaGraphInstantiate(&b->exec, g, 0);
            } else {
                if (g)
                    cudaGraphDestroy(g);
                e = e2;
            }
        }
        cudaStreamDestroy(cs);
        if (s == SK_OK && e != cudaSuccess)
            s = cuda_error(e, "sk_batch_run graph capture");
    }
    if (s == SK_OK) {
        cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
        if (e != cudaSuccess)
            s = cuda_error(e, "cudaGraphLaunch");
    }
    return s;
}

extern "C" sk_status_t sk_batch_launches(sk_batch_t b, int32_t *launches)
{
    if (!b || !launches)
        return set_error(SK_ERR_INVALID_ARG, "sk_batch_launches: null argument");
    int32_t n = 0;
    if (!b->chunks.empty())
        for (int c = 0; c < kBatchClasses; ++c)
            n += b->used[c] ? 1 : 0;
    if (!b->chunks.empty())
        for (int c = 0; c < kStreamClasses; ++c)
            n += b->sused[c] ? 1 : 0;
    *launches = n;
    return SK_OK;
}

extern "C" sk_status_t sk_batch_destroy(sk_batch_t b)
{
    if (!b)
        return SK_OK;
    {
        DeviceGuard dg(b->device);
        free_batch(b);
    }
    delete b;
    return SK_OK;
}
