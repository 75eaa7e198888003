// Continuous-batching serving loop.
//
// All streams share one arrival-ordered frame ring of page-locked host memory.
// sk_stream_submit reserves the
// next bytes of the ring, copies the frame there and marks it ready.  A
// launcher thread takes the ready prefix of the ring -- stopping before a
// second frame of a stream with running state, so each stream's state is
// updated in frame order -- and launches it as one batch: one copy of the work
// list, one kernel over every frame in it, one copy of the results back.  With
// two launches in flight, the next batch is prepared while the current one
// runs, and frames that arrive meanwhile join the batch after it.
// A completion thread retires launches in order: it hands sk and mask to the
// tickets, frees the ring bytes and records submit-to-result latency.
//
// Frames reach the GPU in one of two ways.  By default (zero copy) the ring is
// page-locked host memory mapped into the device address space and the kernel
// reads each frame straight from it, so the PCIe transfer overlaps the
// reduction instead of preceding it.  With SK_SERVER_ZEROCOPY=0 the ring has a
// device mirror and each batch is one contiguous host-to-device copy before its
// kernel.  The ring is sized to half of the server's budget (at most 4 GiB);
// streams are admitted while their ring share (ring_frames frames) fits the
// ring and their device state and tables fit both the other half of the budget
// and the device's memory free at sk_stream_open, less a headroom.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <unordered_map>
#if defined(__SSE2__)
#include <emmintrin.h>
#endif

#include "sk_common.h"

using namespace sk;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kLaunchSlots = 8;  // at most this many launches in flight
constexpr int kMaxBatch = 1024;        // frames per launch
constexpr uint64_t kAlign = 256;       // ring placement granularity
constexpr size_t kMaxRing = (size_t)4 << 30;
// device memory kept free beside admitted streams (kernel local memory, driver
// bookkeeping): a stream is refused if its state and tables would leave less
constexpr size_t kHbmHeadroom = (size_t)256 << 20;

struct StreamRec {
    sk_stream_id id = -1;
    sk_plan_t plan = nullptr;
    int32_t N = 0, M = 0;
    int64_t fbytes = 0;
    int32_t ring_frames = 0;     // frames it may have outstanding
    uint32_t *d_state = nullptr; // [N]
    bool stateful = false;
    bool initialised = false;
    size_t share = 0;            // ring bytes reserved
    size_t small = 0;            // state + tables bytes
    int32_t outstanding = 0;     // submitted, not yet retired
    bool closing = false;
    // per-stream counters (sk_stream_stats)
    int64_t frames_done = 0, frames_flagged = 0, rejected = 0;
    std::vector<double> lat_us;  // last kStreamLatKeep submit-to-result times
    size_t lat_next = 0;
};

static constexpr size_t kStreamLatKeep = 1 << 14;

struct Frame {
    StreamRec *stream;
    uint64_t off;   // monotonic ring offset
    uint64_t size;  // bytes reserved (aligned); 0 for a frame passed by reference
    sk_ticket_t ticket;
    bool ready;
    bool first;     // the stream's first frame with running state (set at launch)
    const uint8_t *ref;  // device address of a frame passed by reference, else null
};

struct TicketRec {
    bool done = false;
    sk_status_t status = SK_OK;
    float sk = 0.0f;
    uint8_t mask = 0;
    Clock::time_point t_submit;
};

struct Launch {
    bool busy = false;
    int n = 0;
    uint64_t end = 0;  // ring offset after its last frame
    std::vector<sk_ticket_t> tickets;
    std::vector<StreamRec *> streams;
    // work block: items | chunks | cta (one copy); result block: sk | mask
    uint8_t *h_work = nullptr, *d_work = nullptr;
    uint8_t *h_res = nullptr, *d_res = nullptr;
    // zero copy: device addresses of the mapped h_work and h_res, which the kernel
    // then reads and writes directly (no work-list upload, no result download)
    uint8_t *h_work_dev = nullptr, *h_res_dev = nullptr;
    cudaEvent_t uploaded = nullptr, done = nullptr;
    // tracing (SK_SERVER_TRACE=1): timing events and host times of one launch
    cudaEvent_t t_copy0 = nullptr, t_copy1 = nullptr, t_k0 = nullptr, t_k1 = nullptr;
    Clock::time_point t_issue, t_issued;
    uint64_t bytes = 0;
    bool failed = false;  // this launch failed to issue (its tickets get the fault)
};

size_t round16(size_t v) { return (v + 15) / 16 * 16; }

// Work block of one launch, packed: cta offsets | chunks | items.
size_t work_bytes(int sms)
{
    return round16(sizeof(int32_t) * (sms + 1)) + round16(sizeof(Chunk) * (kMaxBatch + sms + 1)) +
           sizeof(Item) * kMaxBatch;
}

}  // namespace

struct sk_server_s {
    int device = 0;
    int sms = 0;
    size_t budget = 0;
    size_t ring_cap = 0;
    size_t ring_reserved = 0;  // sum of stream shares
    size_t small_in_use = 0;   // sum of stream state + tables
    uint8_t *h_ring = nullptr, *d_ring = nullptr;
    uint8_t *h_ring_dev = nullptr;  // device address of h_ring (zero-copy mode)
    bool zero_copy = true;          // kernel reads frames from the host ring directly
    uint64_t head = 0, tail = 0;  // monotonic byte offsets
    std::mutex mu;
    std::condition_variable cv_work, cv_flight, cv_done;
    bool stop = false;
    std::map<sk_stream_id, std::unique_ptr<StreamRec>> streams;
    std::deque<Frame> fifo;  // submitted, not launched
    std::unordered_map<sk_ticket_t, TicketRec> tickets;
    sk_stream_id next_stream = 1;
    sk_ticket_t next_ticket = 1;
    Launch slots[kLaunchSlots];
    int nslots = 2;  // launches allowed in flight (SK_SERVER_INFLIGHT, 1..8)
    std::deque<int> flight;
    cudaStream_t s_copy = nullptr, s_compute = nullptr;
    std::thread launcher, completer;
    int64_t frames_done = 0, frames_flagged = 0, launches = 0, rejected = 0;
    std::vector<double> lat_us;
    size_t lat_next = 0;
    sk_status_t fault = SK_OK;
    std::string fault_msg;
    int64_t inject_at = 0;  // SK_SERVER_INJECT_FAULT: the launch that fails on the host
    bool split = true;      // SK_SERVER_SPLIT: small batches split each frame over a CTA
    bool trace = false;
    double tr_n = 0, tr_frames = 0, tr_bytes = 0, tr_host_issue = 0, tr_host_total = 0,
           tr_copy = 0, tr_kernel = 0, tr_copy_to_kernel_end = 0;
    // the slowest launches: max kernel time, host issue and issue->retire, and the
    // launches whose kernel or issue->retire took over 500 us (SK_SERVER_TRACE)
    double tr_kernel_max = 0, tr_issue_max = 0, tr_total_max = 0, tr_slow_kernel = 0,
           tr_slow_total = 0;
};

static constexpr size_t kLatKeep = 1 << 20;

static void record_latency(sk_server_s *s, double us)
{
    if (s->lat_us.size() < kLatKeep)
        s->lat_us.push_back(us);
    else
        s->lat_us[s->lat_next++ % kLatKeep] = us;
}

static void set_fault(sk_server_s *s, sk_status_t st, const char *msg)
{
    if (s->fault == SK_OK) {
        s->fault = st;
        s->fault_msg = msg;
    }
}

// Issue one batch (the lock is NOT held; `frames` were taken off the fifo).
static void issue_batch(sk_server_s *s, Launch &L, const std::vector<Frame> &frames,
                        int64_t launch_no)
{
    NvtxRange nv("sk_server issue_batch");
    if (s->inject_at > 0 && launch_no == s->inject_at) {
        // host-side fault injection for tests: this launch fails before any CUDA call
        std::lock_guard<std::mutex> g(s->mu);
        set_fault(s, SK_ERR_CUDA, "injected launch failure (SK_SERVER_INJECT_FAULT)");
        L.failed = true;
        return;
    }
    const int n = (int)frames.size();
    std::vector<Item> items(n);
    uint8_t *res = s->zero_copy ? L.h_res_dev : L.d_res;
    float *d_sk = (float *)res;
    uint8_t *d_mask = res + sizeof(float) * n;
    bool all_m32 = true;
    for (int k = 0; k < n; ++k) {
        const Frame &f = frames[k];
        StreamRec *r = f.stream;
        Item it = r->plan->item(
            f.ref ? f.ref : (s->zero_copy ? s->h_ring_dev : s->d_ring) + (f.off % s->ring_cap),
            1);
        if (s->zero_copy)
            it.prefetch = 0;
        it.sk = d_sk + k;
        it.mask = d_mask + k;
        if (r->stateful) {
            it.state = r->d_state;
            it.state_init = f.first ? 1 : 0;
        }
        all_m32 = all_m32 && (it.M % 32 == 0);
        items[k] = it;
    }
    std::vector<Chunk> chunks;
    std::vector<int32_t> cta;
    std::vector<int32_t> perm;
    // a batch smaller than the GPU gives each frame a CTA of its own, its rows
    // split over the CTA's teams; a larger one packs one frame per team
    const bool split = s->split && n <= s->sms;
    int grid;
    if (split) {
        perm.resize(n);
        for (int k = 0; k < n; ++k)
            perm[k] = k;
        grid = build_split_schedule(n, s->sms, chunks, cta);
    } else {
        grid = build_item_schedule(items, s->sms, chunks, cta, perm);
    }
    // result slot k now belongs to the frame items[k] came from
    {
        std::vector<sk_ticket_t> tk(n);
        std::vector<StreamRec *> sr(n);
        for (int k = 0; k < n; ++k) {
            tk[k] = L.tickets[perm[k]];
            sr[k] = L.streams[perm[k]];
            items[k].sk = d_sk + k;
            items[k].mask = d_mask + k;
        }
        L.tickets.swap(tk);
        L.streams.swap(sr);
    }
    const size_t o_chunks = round16(sizeof(int32_t) * cta.size());
    const size_t o_items = o_chunks + round16(sizeof(Chunk) * chunks.size());
    const size_t used = o_items + sizeof(Item) * n;
    memcpy(L.h_work, cta.data(), sizeof(int32_t) * cta.size());
    memcpy(L.h_work + o_chunks, chunks.data(), sizeof(Chunk) * chunks.size());
    memcpy(L.h_work + o_items, items.data(), sizeof(Item) * n);
    // frames in the ring: one contiguous range, split at the wrap point (frames
    // passed by reference are read where they are)
    uint64_t a = 0, b = 0;
    for (const Frame &f : frames)
        if (!f.ref) {
            if (b == 0)
                a = f.off;
            b = f.off + f.size;
        }
    cudaError_t e = cudaSuccess;
    if (s->trace)
        e = cudaEventRecord(L.t_copy0, s->s_copy);
    L.bytes = b - a;
    // the work list goes first on the copy stream: a copy queued on the compute
    // stream would wait on the copy engine behind the next batch's frames.  With
    // zero copy the kernel reads it from the mapped host buffer instead.
    if (e == cudaSuccess && !s->zero_copy)
        e = cudaMemcpyAsync(L.d_work, L.h_work, used, cudaMemcpyHostToDevice, s->s_copy);
    uint64_t pos = s->zero_copy ? b : a;
    while (pos < b && e == cudaSuccess) {
        const uint64_t ra = pos % s->ring_cap;
        const uint64_t len = std::min<uint64_t>(b - pos, s->ring_cap - ra);
        e = cudaMemcpyAsync(s->d_ring + ra, s->h_ring + ra, len, cudaMemcpyHostToDevice,
                            s->s_copy);
        pos += len;
    }
    if (e == cudaSuccess && !s->zero_copy)
        e = cudaEventRecord(L.uploaded, s->s_copy);
    if (e == cudaSuccess && s->trace)
        e = cudaEventRecord(L.t_copy1, s->s_copy);
    if (e == cudaSuccess && !s->zero_copy)
        e = cudaStreamWaitEvent(s->s_compute, L.uploaded, 0);
    if (e == cudaSuccess && s->trace)
        e = cudaEventRecord(L.t_k0, s->s_compute);
    sk_status_t st = SK_OK;
    uint8_t *work = s->zero_copy ? L.h_work_dev : L.d_work;
    if (e == cudaSuccess)
        st = launch_schedule((const Item *)(work + o_items),
                             (const Chunk *)(work + o_chunks), (const int32_t *)work,
                             grid, pick_tile(16, all_m32), true, s->device, s->s_compute,
                             split ? 1 : 0);
    if (e == cudaSuccess && st == SK_OK && s->trace)
        e = cudaEventRecord(L.t_k1, s->s_compute);
    if (e == cudaSuccess && st == SK_OK && !s->zero_copy)
        e = cudaMemcpyAsync(L.h_res, L.d_res, (sizeof(float) + 1) * (size_t)n,
                            cudaMemcpyDeviceToHost, s->s_compute);
    if (e == cudaSuccess && st == SK_OK)
        e = cudaEventRecord(L.done, s->s_compute);
    if (e != cudaSuccess || st != SK_OK) {
        std::lock_guard<std::mutex> g(s->mu);
        set_fault(s, e != cudaSuccess ? SK_ERR_CUDA : st,
                  e != cudaSuccess ? cudaGetErrorString(e) : "batch launch failed");
        L.failed = true;
    }
}

static void launcher_main(sk_server_s *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        int slot = -1;
        for (int i = 0; i < s->nslots; ++i)
            if (!s->slots[i].busy) {
                slot = i;
                break;
            }
        const bool ready = !s->fifo.empty() && s->fifo.front().ready;
        if (s->stop)
            return;
        if (s->fault != SK_OK && !s->fifo.empty()) {
            // nothing launches after a fault: the queued frames' tickets complete
            // with the fault status instead of waiting for ever
            for (const Frame &f : s->fifo) {
                auto t = s->tickets.find(f.ticket);
                if (t != s->tickets.end()) {
                    t->second.done = true;
                    t->second.status = s->fault;
                }
                f.stream->outstanding -= 1;
            }
            s->fifo.clear();
            s->cv_done.notify_all();
            continue;
        }
        if (slot < 0 || !ready || s->fault != SK_OK) {
            s->cv_work.wait(lk);
            continue;
        }
        // ready prefix, at most one frame per stream with running state
        std::vector<Frame> batch;
        std::vector<StreamRec *> seen;
        while (!s->fifo.empty() && (int)batch.size() < kMaxBatch) {
            const Frame &f = s->fifo.front();
            if (!f.ready)
                break;
            if (f.stream->stateful &&
                std::find(seen.begin(), seen.end(), f.stream) != seen.end())
                break;
            batch.push_back(f);
            if (f.stream->stateful) {
                seen.push_back(f.stream);
                batch.back().first = !f.stream->initialised;
                f.stream->initialised = true;
            }
            s->fifo.pop_front();
        }
        Launch &L = s->slots[slot];
        L.busy = true;
        L.n = (int)batch.size();
        L.end = 0;
        for (const Frame &f : batch)
            if (!f.ref)
                L.end = f.off + f.size;
        L.tickets.clear();
        L.streams.clear();
        for (const Frame &f : batch) {
            L.tickets.push_back(f.ticket);
            L.streams.push_back(f.stream);
        }
        s->launches += 1;
        const int64_t launch_no = s->launches;
        L.failed = false;
        lk.unlock();
        L.t_issue = Clock::now();
        issue_batch(s, L, batch, launch_no);
        L.t_issued = Clock::now();
        lk.lock();
        s->flight.push_back(slot);
        s->cv_flight.notify_one();
    }
}

static void completer_main(sk_server_s *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        while (s->flight.empty() && !s->stop)
            s->cv_flight.wait(lk);
        if (s->flight.empty())
            return;
        const int idx = s->flight.front();
        Launch &L = s->slots[idx];
        lk.unlock();
        cudaError_t e = cudaEventSynchronize(L.done);
        const Clock::time_point now = Clock::now();
        lk.lock();
        s->flight.pop_front();
        if (e != cudaSuccess)
            set_fault(s, SK_ERR_CUDA, cudaGetErrorString(e));
        // a launch that completed keeps its results even when a later launch has
        // failed since; a launch that failed itself gets the server's fault
        const sk_status_t lst = (e != cudaSuccess || L.failed) ? s->fault : SK_OK;
        const float *h_sk = (const float *)L.h_res;
        const uint8_t *h_mask = L.h_res + sizeof(float) * L.n;
        for (int k = 0; k < L.n; ++k) {
            auto t = s->tickets.find(L.tickets[k]);
            if (t != s->tickets.end()) {
                t->second.done = true;
                t->second.status = lst;
                t->second.sk = h_sk[k];
                t->second.mask = h_mask[k];
                const double us =
                    std::chrono::duration<double, std::micro>(now - t->second.t_submit).count();
                record_latency(s, us);
                StreamRec *r = L.streams[k];
                if (r->lat_us.size() < kStreamLatKeep)
                    r->lat_us.push_back(us);
                else
                    r->lat_us[r->lat_next++ % kStreamLatKeep] = us;
            }
            if (lst == SK_OK) {  // a failed launch has no results to count
                s->frames_done += 1;
                s->frames_flagged += h_mask[k] ? 1 : 0;
                L.streams[k]->frames_done += 1;
                L.streams[k]->frames_flagged += h_mask[k] ? 1 : 0;
            }
            L.streams[k]->outstanding -= 1;
        }
        s->tail = std::max(s->tail, L.end);
        if (s->trace && e == cudaSuccess) {
            float c = 0, k = 0, ck = 0;
            cudaEventElapsedTime(&c, L.t_copy0, L.t_copy1);
            cudaEventElapsedTime(&k, L.t_k0, L.t_k1);
            cudaEventElapsedTime(&ck, L.t_copy0, L.t_k1);
            s->tr_n += 1;
            s->tr_frames += L.n;
            s->tr_bytes += (double)L.bytes;
            s->tr_copy += c * 1e3;
            s->tr_kernel += k * 1e3;
            s->tr_copy_to_kernel_end += ck * 1e3;
            const double hi = std::chrono::duration<double, std::micro>(L.t_issued - L.t_issue).count();
            const double ht = std::chrono::duration<double, std::micro>(now - L.t_issue).count();
            s->tr_host_issue += hi;
            s->tr_host_total += ht;
            s->tr_kernel_max = std::max(s->tr_kernel_max, (double)k * 1e3);
            s->tr_issue_max = std::max(s->tr_issue_max, hi);
            s->tr_total_max = std::max(s->tr_total_max, ht);
            s->tr_slow_kernel += k * 1e3 > 500.0 ? 1 : 0;
            s->tr_slow_total += ht > 500.0 ? 1 : 0;
        }
        L.busy = false;
        L.n = 0;
        s->cv_done.notify_all();
        s->cv_work.notify_one();
    }
}

static void free_launch(Launch &L)
{
    cudaFreeHost(L.h_work);
    cudaFreeHost(L.h_res);
    cudaFree(L.d_work);
    cudaFree(L.d_res);
    if (L.uploaded)
        cudaEventDestroy(L.uploaded);
    if (L.done)
        cudaEventDestroy(L.done);
    for (cudaEvent_t ev : {L.t_copy0, L.t_copy1, L.t_k0, L.t_k1})
        if (ev)
            cudaEventDestroy(ev);
}

static void free_stream(StreamRec *r)
{
    cudaFree(r->d_state);
    sk_plan_destroy(r->plan);
}

extern "C" sk_status_t sk_server_create(int device, size_t hbm_budget_bytes, sk_server_t *out)
{
    if (!out)
        return set_error(SK_ERR_INVALID_ARG, "sk_server_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return set_error(SK_ERR_INVALID_ARG, "sk_server_create: device %d not present", device);
    if (hbm_budget_bytes < ((size_t)2 << 20))
        return set_error(SK_ERR_INVALID_ARG, "sk_server_create: budget below 2 MiB");
    sk_server_s *s = new (std::nothrow) sk_server_s();
    if (!s)
        return set_error(SK_ERR_OOM, "host allocation");
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->ring_cap = std::min(kMaxRing, hbm_budget_bytes / 2) / kAlign * kAlign;
    s->sms = sm_count(device);
    if (const char *v = getenv("SK_SERVER_ZEROCOPY"))
        s->zero_copy = atoi(v) != 0;
    if (const char *v = getenv("SK_SERVER_TRACE"))
        s->trace = atoi(v) != 0;
    if (const char *v = getenv("SK_SERVER_INFLIGHT")) {
        const int k = atoi(v);
        if (k >= 1 && k <= kLaunchSlots)
            s->nslots = k;
    }
    if (const char *v = getenv("SK_SERVER_INJECT_FAULT"))
        s->inject_at = atoll(v);
    if (const char *v = getenv("SK_SERVER_SPLIT"))
        s->split = atoi(v) != 0;
    sk_status_t st = SK_OK;
    {
        DeviceGuard dg(device);
        if (cudaHostAlloc(&s->h_ring, s->ring_cap, cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess ||
            (!s->zero_copy && cudaMalloc(&s->d_ring, s->ring_cap) != cudaSuccess))
            st = set_error(SK_ERR_OOM, "server frame ring (%zu bytes)", s->ring_cap);
        else if (s->zero_copy &&
                 cudaHostGetDevicePointer((void **)&s->h_ring_dev, s->h_ring, 0) != cudaSuccess)
            st = set_error(SK_ERR_CUDA, "server frame ring mapping");
        const size_t wb = work_bytes(s->sms), rb = sizeof(float) * kMaxBatch + kMaxBatch;
        for (int i = 0; i < s->nslots && st == SK_OK; ++i) {
            Launch &L = s->slots[i];
            if (cudaHostAlloc(&L.h_work, wb, cudaHostAllocMapped) != cudaSuccess ||
                cudaHostAlloc(&L.h_res, rb, cudaHostAllocMapped) != cudaSuccess ||
                cudaMalloc(&L.d_work, wb) != cudaSuccess || cudaMalloc(&L.d_res, rb) != cudaSuccess)
                st = set_error(SK_ERR_OOM, "server launch buffers");
            else if (cudaHostGetDevicePointer((void **)&L.h_work_dev, L.h_work, 0) !=
                         cudaSuccess ||
                     cudaHostGetDevicePointer((void **)&L.h_res_dev, L.h_res, 0) != cudaSuccess)
                st = set_error(SK_ERR_CUDA, "server launch buffer mapping");
            else if (cudaEventCreateWithFlags(&L.uploaded, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess)
                st = set_error(SK_ERR_CUDA, "server events");
            else if (s->trace && (cudaEventCreate(&L.t_copy0) != cudaSuccess ||
                                  cudaEventCreate(&L.t_copy1) != cudaSuccess ||
                                  cudaEventCreate(&L.t_k0) != cudaSuccess ||
                                  cudaEventCreate(&L.t_k1) != cudaSuccess))
                st = set_error(SK_ERR_CUDA, "server trace events");
        }
        if (st == SK_OK &&
            (cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
             cudaStreamCreateWithFlags(&s->s_compute, cudaStreamNonBlocking) != cudaSuccess))
            st = set_error(SK_ERR_CUDA, "server streams");
        if (st == SK_OK)
            st = ensure_kernel_attrs(device);
        if (st != SK_OK) {
            for (auto &L : s->slots)
                free_launch(L);
            cudaFreeHost(s->h_ring);
            cudaFree(s->d_ring);
            if (s->s_copy)
                cudaStreamDestroy(s->s_copy);
            if (s->s_compute)
                cudaStreamDestroy(s->s_compute);
        }
    }
    if (st != SK_OK) {
        delete s;
        return st;
    }
    s->launcher = std::thread(launcher_main, s);
    s->completer = std::thread(completer_main, s);
    *out = s;
    return SK_OK;
}

extern "C" sk_status_t sk_server_destroy(sk_server_t s)
{
    if (!s)
        return SK_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_flight.notify_all();
    s->launcher.join();
    s->completer.join();
    if (s->trace && s->tr_n > 0)
        fprintf(stderr,
                "sk_server trace: %.0f launches, %.2f frames and %.0f KB each; host issue %.1f us, "
                "issue->retire %.1f us, upload %.1f us (%.1f GB/s), kernel %.1f us, "
                "upload start->kernel end %.1f us\n",
                s->tr_n, s->tr_frames / s->tr_n, s->tr_bytes / s->tr_n / 1024.0,
                s->tr_host_issue / s->tr_n, s->tr_host_total / s->tr_n, s->tr_copy / s->tr_n,
                s->tr_bytes / (s->tr_copy * 1e3 + 1e-9), s->tr_kernel / s->tr_n,
                s->tr_copy_to_kernel_end / s->tr_n);
    if (s->trace && s->tr_n > 0)
        fprintf(stderr,
                "sk_server trace: slowest kernel %.0f us, host issue %.0f us, issue->retire "
                "%.0f us; launches over 500 us: %.0f kernels, %.0f issue->retire\n",
                s->tr_kernel_max, s->tr_issue_max, s->tr_total_max, s->tr_slow_kernel,
                s->tr_slow_total);
    {
        DeviceGuard dg(s->device);
        cudaStreamSynchronize(s->s_compute);
        cudaStreamSynchronize(s->s_copy);
        for (auto &kv : s->streams)
            free_stream(kv.second.get());
        for (auto &L : s->slots)
            free_launch(L);
        cudaFreeHost(s->h_ring);
        cudaFree(s->d_ring);
        cudaStreamDestroy(s->s_copy);
        cudaStreamDestroy(s->s_compute);
    }
    delete s;
    return SK_OK;
}

static uint64_t frame_span(int64_t fbytes) { return ((uint64_t)fbytes + kAlign - 1) / kAlign * kAlign; }

// Copy a frame into the ring with streaming (non-temporal) stores.  The CPU never
// reads the ring again; lines that are not left dirty in its caches reach the
// GPU's zero-copy reads without being snooped back first.  Measured on B300 with
// 32 real-time streams: submit 68 -> 51 us, kernel time per batch 89 -> 72 us.
static void copy_to_ring(uint8_t *dst, const uint8_t *src, size_t n)
{
    size_t k = 0;
#if defined(__SSE2__)
    if (((uintptr_t)dst & 15u) == 0) {
        for (; k + 64 <= n; k += 64) {
            const __m128i a = _mm_loadu_si128((const __m128i *)(src + k));
            const __m128i b = _mm_loadu_si128((const __m128i *)(src + k + 16));
            const __m128i c = _mm_loadu_si128((const __m128i *)(src + k + 32));
            const __m128i d = _mm_loadu_si128((const __m128i *)(src + k + 48));
            _mm_stream_si128((__m128i *)(dst + k), a);
            _mm_stream_si128((__m128i *)(dst + k + 16), b);
            _mm_stream_si128((__m128i *)(dst + k + 32), c);
            _mm_stream_si128((__m128i *)(dst + k + 48), d);
        }
        _mm_sfence();  // the stores are visible before the frame is marked ready
    }
#endif
    if (k < n)
        memcpy(dst + k, src + k, n - k);
}

extern "C" sk_status_t sk_stream_open(sk_server_t s, const sk_params_t *params,
                                      int32_t ring_frames, sk_stream_id *out)
{
    if (!s || !params || !out)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_open: null argument");
    *out = -1;
    if (ring_frames < 1 || ring_frames > 65536)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_open: ring_frames outside 1..65536");
    if (params->layout != SK_LAYOUT_TIME_MAJOR && params->layout != SK_LAYOUT_INPUT_MAJOR)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_open: unknown layout %d", params->layout);
    if (params->n_inputs < 1 || params->n_inputs > SK_MAX_INPUTS || params->n_time < 2 ||
        params->n_time > SK_MAX_TIME)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_open: N or M out of range");
    const int64_t fbytes = (int64_t)params->n_time * params->n_inputs;
    const size_t share = (size_t)frame_span(fbytes) * ring_frames;
    const size_t small = sizeof(uint32_t) * params->n_inputs +
                         sizeof(int64_t) * (2 * (params->n_inputs + 1) + SK_OFFSET_BUCKETS) +
                         sizeof(float) * (params->n_inputs + 1);
    // the device's real free memory, less a headroom for the launches (kernel
    // local memory, driver bookkeeping): admission takes the lesser of it and the
    // caller's budget
    size_t dev_free = SIZE_MAX, dev_total = 0;
    {
        DeviceGuard dg(s->device);
        if (cudaMemGetInfo(&dev_free, &dev_total) != cudaSuccess) {
            cudaGetLastError();
            dev_free = SIZE_MAX;
        }
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (dev_free < kHbmHeadroom || small > dev_free - kHbmHeadroom) {
            s->rejected += 1;
            return set_error(SK_ERR_BUSY,
                             "sk_stream_open: the device has %zu bytes free; the stream needs "
                             "%zu beside a headroom of %zu",
                             dev_free, small, kHbmHeadroom);
        }
        if (s->ring_reserved + share > s->ring_cap ||
            s->small_in_use + small > s->budget - s->ring_cap) {
            s->rejected += 1;
            return set_error(SK_ERR_BUSY, "sk_stream_open: no room (ring share %zu of %zu free)",
                             share, s->ring_cap - s->ring_reserved);
        }
        s->ring_reserved += share;
        s->small_in_use += small;
    }
    auto r = std::make_unique<StreamRec>();
    sk_status_t st = sk_plan_create(params, s->device, &r->plan);
    if (st == SK_OK) {
        DeviceGuard dg(s->device);
        r->N = params->n_inputs;
        r->M = params->n_time;
        r->fbytes = fbytes;
        r->ring_frames = ring_frames;
        r->stateful = (params->flags & (SK_RUNNING_OFFSET | SK_RUNNING_MU)) != 0;
        r->share = share;
        r->small = small;
        if (cudaMalloc(&r->d_state, sizeof(uint32_t) * r->N) != cudaSuccess)
            st = set_error(SK_ERR_OOM, "sk_stream_open: state allocation");
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (st != SK_OK) {
        s->ring_reserved -= share;
        s->small_in_use -= small;
        if (r->plan)
            free_stream(r.get());
        return st;
    }
    r->id = s->next_stream++;
    *out = r->id;
    s->streams[r->id] = std::move(r);
    return SK_OK;
}

extern "C" sk_status_t sk_stream_submit(sk_server_t s, sk_stream_id id, const uint8_t *frame,
                                        int64_t frame_index, sk_ticket_t *ticket)
{
    if (!s || !frame || !ticket)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_submit: null argument");
    (void)frame_index;
    const Clock::time_point t0 = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->fault != SK_OK)
        return set_error(s->fault, "server fault: %s", s->fault_msg.c_str());
    auto it = s->streams.find(id);
    if (it == s->streams.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_submit: unknown stream %d", id);
    StreamRec *r = it->second.get();
    if (r->closing)
        return set_error(SK_ERR_CLOSED, "sk_stream_submit: stream %d closing", id);
    if (r->outstanding >= r->ring_frames) {
        s->rejected += 1;
        r->rejected += 1;
        return set_error(SK_ERR_BUSY, "sk_stream_submit: stream %d has %d frames outstanding",
                         id, r->outstanding);
    }
    const uint64_t size = frame_span(r->fbytes);
    uint64_t off = s->head;
    if (off % s->ring_cap + size > s->ring_cap)  // do not straddle the wrap point
        off = (off / s->ring_cap + 1) * s->ring_cap;
    if (off + size - s->tail > s->ring_cap) {
        s->rejected += 1;
        r->rejected += 1;
        return set_error(SK_ERR_BUSY, "sk_stream_submit: frame ring full");
    }
    s->head = off + size;
    r->outstanding += 1;
    const sk_ticket_t t = s->next_ticket++;
    TicketRec tr;
    tr.t_submit = t0;
    s->tickets.emplace(t, tr);
    s->fifo.push_back(Frame{r, off, size, t, false, false, nullptr});
    uint8_t *dst = s->h_ring + off % s->ring_cap;
    const int64_t fb = r->fbytes;
    lk.unlock();
    copy_to_ring(dst, frame, (size_t)fb);  // the reserved bytes are ours until retired
    lk.lock();
    for (auto f = s->fifo.rbegin(); f != s->fifo.rend(); ++f)
        if (f->ticket == t) {
            f->ready = true;
            break;
        }
    *ticket = t;
    lk.unlock();
    s->cv_work.notify_one();
    return SK_OK;
}

extern "C" sk_status_t sk_stream_submit_ref(sk_server_t s, sk_stream_id id, const uint8_t *frame,
                                            int64_t frame_index, sk_ticket_t *ticket)
{
    if (!s || !frame || !ticket)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_submit_ref: null argument");
    (void)frame_index;
    if ((uintptr_t)frame & 15u)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_submit_ref: frame not 16-byte aligned");
    // the kernel reads the frame where it is: device memory of the server's
    // device, or page-locked host memory mapped into its address space
    cudaPointerAttributes pa;
    const uint8_t *dev = nullptr;
    {
        DeviceGuard dg(s->device);
        // a thread that has made no CUDA call yet has no current context until
        // cudaSetDevice (which makes the device's primary context current)
        cudaSetDevice(s->device);
        if (cudaPointerGetAttributes(&pa, frame) == cudaSuccess) {
            if ((pa.type == cudaMemoryTypeDevice && pa.device == s->device) ||
                pa.type == cudaMemoryTypeManaged || pa.type == cudaMemoryTypeHost)
                dev = (const uint8_t *)pa.devicePointer;
        } else {
            cudaGetLastError();  // clear the error a foreign pointer leaves behind
        }
    }
    if (!dev)
        return set_error(SK_ERR_INVALID_ARG,
                         "sk_stream_submit_ref: frame is neither device memory nor "
                         "page-locked host memory the device can read");
    const Clock::time_point t0 = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->fault != SK_OK)
        return set_error(s->fault, "server fault: %s", s->fault_msg.c_str());
    auto it = s->streams.find(id);
    if (it == s->streams.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_submit_ref: unknown stream %d", id);
    StreamRec *r = it->second.get();
    if (r->closing)
        return set_error(SK_ERR_CLOSED, "sk_stream_submit_ref: stream %d closing", id);
    if (r->outstanding >= r->ring_frames) {
        s->rejected += 1;
        r->rejected += 1;
        return set_error(SK_ERR_BUSY, "sk_stream_submit_ref: stream %d has %d frames outstanding",
                         id, r->outstanding);
    }
    r->outstanding += 1;
    const sk_ticket_t t = s->next_ticket++;
    TicketRec tr;
    tr.t_submit = t0;
    s->tickets.emplace(t, tr);
    s->fifo.push_back(Frame{r, 0, 0, t, true, false, dev});
    *ticket = t;
    lk.unlock();
    s->cv_work.notify_one();
    return SK_OK;
}

extern "C" sk_status_t sk_ticket_wait(sk_server_t s, sk_ticket_t ticket, int64_t timeout_us,
                                      float *sk, uint8_t *mask)
{
    if (!s)
        return set_error(SK_ERR_INVALID_ARG, "sk_ticket_wait: server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->tickets.find(ticket) == s->tickets.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_ticket_wait: unknown ticket %lld",
                         (long long)ticket);
    auto ready = [&] {
        auto t = s->tickets.find(ticket);
        return t == s->tickets.end() || t->second.done;
    };
    if (timeout_us < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return set_error(SK_ERR_TIMEOUT, "sk_ticket_wait: ticket %lld not done",
                         (long long)ticket);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_ticket_wait: ticket gone");
    const TicketRec tr = it->second;
    s->tickets.erase(it);
    if (tr.status != SK_OK)
        return set_error(tr.status, "server fault: %s", s->fault_msg.c_str());
    if (sk)
        *sk = tr.sk;
    if (mask)
        *mask = tr.mask;
    return SK_OK;
}

static bool stream_idle(sk_server_s *s, sk_stream_id id)
{
    auto it = s->streams.find(id);
    return it == s->streams.end() || it->second->outstanding == 0;
}

extern "C" sk_status_t sk_stream_drain(sk_server_t s, sk_stream_id id, int64_t timeout_us)
{
    if (!s)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_drain: server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->streams.find(id) == s->streams.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_drain: unknown stream %d", id);
    auto ready = [&] { return stream_idle(s, id) || s->fault != SK_OK; };
    if (timeout_us < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return set_error(SK_ERR_TIMEOUT, "sk_stream_drain: stream %d busy", id);
    if (s->fault != SK_OK)
        return set_error(s->fault, "server fault: %s", s->fault_msg.c_str());
    return SK_OK;
}

extern "C" sk_status_t sk_stream_get_state(sk_server_t s, sk_stream_id id, void *buf,
                                           size_t *len)
{
    if (!s || !len)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_get_state: null argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->streams.find(id);
    if (it == s->streams.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_get_state: unknown stream %d", id);
    StreamRec *r = it->second.get();
    const size_t need = sizeof(uint32_t) * (2 + (size_t)r->N);
    if (!buf) {
        *len = need;
        return SK_OK;
    }
    if (*len < need)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_get_state: need %zu bytes", need);
    if (r->outstanding != 0)
        return set_error(SK_ERR_BUSY, "sk_stream_get_state: stream %d not drained", id);
    uint32_t *u = (uint32_t *)buf;
    u[0] = r->initialised ? 1u : 0u;
    u[1] = (uint32_t)r->N;
    DeviceGuard dg(s->device);
    cudaError_t e = cudaMemcpy(u + 2, r->d_state, sizeof(uint32_t) * r->N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_error(e, "sk_stream_get_state");
    *len = need;
    return SK_OK;
}

extern "C" sk_status_t sk_stream_set_state(sk_server_t s, sk_stream_id id, const void *buf,
                                           size_t len)
{
    if (!s || !buf)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_set_state: null argument");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->streams.find(id);
    if (it == s->streams.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_set_state: unknown stream %d", id);
    StreamRec *r = it->second.get();
    const uint32_t *u = (const uint32_t *)buf;
    if (len != sizeof(uint32_t) * (2 + (size_t)r->N) || u[1] != (uint32_t)r->N || u[0] > 1)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_set_state: state of another shape");
    if (r->outstanding != 0)
        return set_error(SK_ERR_BUSY, "sk_stream_set_state: stream %d not drained", id);
    DeviceGuard dg(s->device);
    cudaError_t e = cudaMemcpy(r->d_state, u + 2, sizeof(uint32_t) * r->N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_error(e, "sk_stream_set_state");
    r->initialised = u[0] != 0;
    return SK_OK;
}

extern "C" sk_status_t sk_stream_close(sk_server_t s, sk_stream_id id)
{
    if (!s)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_close: server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->streams.find(id);
    if (it == s->streams.end())
        return set_error(SK_ERR_CLOSED, "sk_stream_close: unknown or closed stream %d", id);
    it->second->closing = true;
    // launches in flight reference its state: wait for them (bounded)
    bool idle = s->cv_done.wait_for(lk, std::chrono::seconds(30),
                                    [&] { return stream_idle(s, id) || s->fault != SK_OK; });
    if (!idle)
        return set_error(SK_ERR_TIMEOUT, "sk_stream_close: stream %d still busy", id);
    std::unique_ptr<StreamRec> r = std::move(s->streams[id]);
    s->streams.erase(id);
    s->ring_reserved -= r->share;
    s->small_in_use -= r->small;
    lk.unlock();
    DeviceGuard dg(s->device);
    cudaStreamSynchronize(s->s_compute);
    free_stream(r.get());
    return SK_OK;
}

extern "C" sk_status_t sk_server_stats(sk_server_t s, sk_server_stats_t *out)
{
    if (!s || !out)
        return set_error(SK_ERR_INVALID_ARG, "sk_server_stats: null argument");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> g(s->mu);
        out->frames_done = s->frames_done;
        out->frames_flagged = s->frames_flagged;
        out->launches = s->launches;
        out->rejected = s->rejected;
        out->hbm_in_use = s->ring_cap + s->small_in_use;
        lat = s->lat_us;
    }
    out->latency_p50_us = 0.0;
    out->latency_p99_us = 0.0;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        out->latency_p50_us = lat[(size_t)(0.50 * (lat.size() - 1))];
        out->latency_p99_us = lat[(size_t)(0.99 * (lat.size() - 1))];
    }
    return SK_OK;
}

extern "C" sk_status_t sk_stream_stats(sk_server_t s, sk_stream_id id, sk_stream_stats_t *out)
{
    if (!s || !out)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_stats: null argument");
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->streams.find(id);
        if (it == s->streams.end())
            return set_error(SK_ERR_INVALID_ARG, "sk_stream_stats: unknown stream %d", id);
        const StreamRec *r = it->second.get();
        memset(out, 0, sizeof *out);
        out->frames_done = r->frames_done;
        out->frames_flagged = r->frames_flagged;
        out->rejected = r->rejected;
        out->outstanding = r->outstanding;
        lat = r->lat_us;
    }
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        out->latency_p50_us = lat[(size_t)(0.50 * (lat.size() - 1))];
        out->latency_p99_us = lat[(size_t)(0.99 * (lat.size() - 1))];
    }
    return SK_OK;
}

// ---------------------------------------------------------------------------
// Load generator: replays frames into open streams from several submitter
// threads, paced at a cadence with exponential jitter or flat out.
// ---------------------------------------------------------------------------
#include <random>

extern "C" sk_status_t sk_server_replay(sk_server_t s, const sk_replay_t *rp,
                                        sk_replay_result_t *out)
{
    if (!s || !rp || !out || rp->n_streams <= 0 || !rp->streams || !rp->frames ||
        !rp->pool_frames || rp->frames_per_stream < 0 || rp->threads <= 0 ||
        rp->threads > 256 || !(rp->cadence_s >= 0.0))
        return set_error(SK_ERR_INVALID_ARG, "sk_server_replay: bad arguments");
    std::vector<int64_t> fbytes(rp->n_streams);
    {
        std::lock_guard<std::mutex> g(s->mu);
        for (int j = 0; j < rp->n_streams; ++j) {
            auto it = s->streams.find(rp->streams[j]);
            if (it == s->streams.end() || rp->pool_frames[j] <= 0 || !rp->frames[j])
                return set_error(SK_ERR_INVALID_ARG, "sk_server_replay: stream %d", j);
            fbytes[j] = it->second->fbytes;
        }
        s->lat_us.clear();
        s->lat_next = 0;
    }
    sk_server_stats_t before;
    sk_server_stats(s, &before);
    const int nt = rp->threads;
    std::vector<std::vector<double>> sub_us(nt);
    std::vector<int64_t> retries(nt, 0);
    std::vector<sk_status_t> status(nt, SK_OK);
    std::vector<std::string> message(nt);
    const Clock::time_point t0 = Clock::now();
    auto worker = [&](int w) {
        std::mt19937_64 rng(rp->seed * 1000003ull + (uint64_t)w);
        std::exponential_distribution<double> jit(rp->jitter_mean_s > 0 ? 1.0 / rp->jitter_mean_s
                                                                         : 1.0);
        struct Ev {
            double t;
            int j;
            int64_t k;
        };
        std::vector<Ev> sched;
        for (int j = w; j < rp->n_streams; j += nt)
            for (int64_t k = 0; k < rp->frames_per_stream; ++k)
                sched.push_back(Ev{k * rp->cadence_s + (rp->jitter_mean_s > 0 ? jit(rng) : 0.0),
                                   j, k});
        std::sort(sched.begin(), sched.end(), [](const Ev &a, const Ev &b) { return a.t < b.t; });
        std::vector<std::deque<sk_ticket_t>> pend(rp->n_streams);
        for (const Ev &e : sched) {
            if (rp->paced)
                while (std::chrono::duration<double>(Clock::now() - t0).count() < e.t) {
                }
            const uint8_t *fr = rp->frames[e.j] + (e.k % rp->pool_frames[e.j]) * fbytes[e.j];
            for (;;) {
                sk_ticket_t t;
                const Clock::time_point a = Clock::now();
                sk_status_t st = rp->by_reference
                                     ? sk_stream_submit_ref(s, rp->streams[e.j], fr, e.k, &t)
                                     : sk_stream_submit(s, rp->streams[e.j], fr, e.k, &t);
                sub_us[w].push_back(std::chrono::duration<double, std::micro>(Clock::now() - a).count());
                if (st == SK_OK) {
                    pend[e.j].push_back(t);
                    break;
                }
                if (st != SK_ERR_BUSY || pend[e.j].empty()) {
                    status[w] = st;
                    message[w] = sk_last_error();  // the message is per thread
                    return;
                }
                retries[w] += 1;
                sk_ticket_wait(s, pend[e.j].front(), -1, nullptr, nullptr);
                pend[e.j].pop_front();
            }
            // collect results lazily, keeping at most half of a small window open
            while (pend[e.j].size() > 8) {
                sk_ticket_wait(s, pend[e.j].front(), -1, nullptr, nullptr);
                pend[e.j].pop_front();
            }
        }
        for (auto &q : pend)
            for (sk_ticket_t t : q)
                sk_ticket_wait(s, t, -1, nullptr, nullptr);
    };
    std::vector<std::thread> th;
    for (int w = 0; w < nt; ++w)
        th.emplace_back(worker, w);
    for (auto &t : th)
        t.join();
    const double wall = std::chrono::duration<double>(Clock::now() - t0).count();
    for (int w = 0; w < nt; ++w)
        if (status[w] != SK_OK)
            return set_error(status[w], "sk_server_replay: submit failed: %s",
                             message[w].c_str());
    sk_server_stats_t after;
    sk_server_stats(s, &after);
    std::vector<double> all;
    for (auto &v : sub_us)
        all.insert(all.end(), v.begin(), v.end());
    std::sort(all.begin(), all.end());
    memset(out, 0, sizeof *out);
    out->wall_s = wall;
    out->frames = after.frames_done - before.frames_done;
    out->launches = after.launches - before.launches;
    for (int64_t r : retries)
        out->busy_retries += r;
    double bytes = 0.0;
    for (int j = 0; j < rp->n_streams; ++j)
        bytes += (double)fbytes[j] * (double)rp->frames_per_stream;
    out->bytes = bytes;
    out->latency_p50_us = after.latency_p50_us;
    out->latency_p99_us = after.latency_p99_us;
    if (!all.empty()) {
        out->submit_p50_us = all[all.size() / 2];
        out->submit_p99_us = all[(size_t)(0.99 * (all.size() - 1))];
    }
    return SK_OK;
}
