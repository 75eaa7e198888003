// Continuous-batching serving loop.
//
// Streams are arrays (N inputs, M samples per frame) that submit frames as they
// arrive.  sk_stream_submit copies the frame into the stream's page-locked
// staging ring and queues it.  A launcher thread forms a batch from whatever is
// queued -- the oldest frame of every stream that has one -- uploads those
// frames into the streams' device rings (copy stream), and launches the fused
// kernel over the batch (compute stream), without waiting for earlier batches:
// up to kLaunchSlots batches are in flight, so frames that arrive while a batch
// runs are admitted and launched behind it.  A completion thread waits for each
// batch in launch order, hands sk and mask to the tickets and frees the ring
// slots.  One frame per stream per batch plus in-order launches on one compute
// stream keep each stream's running power state (SK_RUNNING_OFFSET) updated in
// frame order.  Device memory per stream is admitted against the server's HBM
// budget.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <unordered_map>

#include "sk_common.h"

using namespace sk;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kLaunchSlots = 4;
constexpr int kMaxBatch = 1024;  // frames per launch

struct Pending {
    int32_t slot;
    sk_ticket_t ticket;
};

struct StreamRec {
    sk_stream_id id = -1;
    sk_plan_t plan = nullptr;
    int32_t N = 0, M = 0;
    int64_t fbytes = 0;
    int32_t ring = 0;
    uint8_t *h_stage = nullptr;  // pinned [ring][fbytes]
    uint8_t *d_ring = nullptr;   // [ring][fbytes]
    uint32_t *d_state = nullptr; // [N] when SK_RUNNING_OFFSET
    bool stateful = false;
    bool initialised = false;    // state holds a stream history
    size_t hbm = 0;
    int32_t next_slot = 0;
    int32_t used = 0;            // queued + in flight
    int64_t in_flight = 0;
    std::deque<Pending> queue;
    bool closing = false;
};

struct TicketRec {
    sk_stream_id stream;
    bool done = false;
    sk_status_t status = SK_OK;
    float sk = 0.0f;
    uint8_t mask = 0;
    Clock::time_point t_submit;
};

struct LaunchSlot {
    bool busy = false;
    int n = 0;
    int tile = 0;
    std::vector<sk_ticket_t> tickets;
    std::vector<sk_stream_id> streams;
    // pinned host mirrors and device copies of the work list and results
    Item *h_items = nullptr;
    Chunk *h_chunks = nullptr;
    int32_t *h_cta = nullptr;
    float *h_sk = nullptr;
    uint8_t *h_mask = nullptr;
    Item *d_items = nullptr;
    Chunk *d_chunks = nullptr;
    int32_t *d_cta = nullptr;
    float *d_sk = nullptr;
    uint8_t *d_mask = nullptr;
    int max_chunks = 0;
    cudaEvent_t uploaded = nullptr;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct sk_server_s {
    int device = 0;
    int sms = 0;
    size_t budget = 0;
    size_t in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // launcher: queued frames or a free slot
    std::condition_variable cv_flight; // completion thread: a launch in flight
    std::condition_variable cv_done;   // waiters: a ticket finished
    bool stop = false;
    std::map<sk_stream_id, std::unique_ptr<StreamRec>> streams;
    std::unordered_map<sk_ticket_t, TicketRec> tickets;
    sk_stream_id next_stream = 1;
    sk_ticket_t next_ticket = 1;
    size_t rr = 0;  // round-robin start among streams
    LaunchSlot slots[kLaunchSlots];
    std::deque<int> flight;  // launch slots in launch order
    cudaStream_t s_copy = nullptr, s_compute = nullptr;
    std::thread launcher, completer;
    // statistics
    int64_t frames_done = 0, frames_flagged = 0, launches = 0, rejected = 0;
    std::vector<double> lat_us;
    size_t lat_next = 0;
    sk_status_t fault = SK_OK;
    std::string fault_msg;
};

static constexpr size_t kLatKeep = 1 << 20;

static void record_latency(sk_server_s *s, double us)
{
    if (s->lat_us.size() < kLatKeep)
        s->lat_us.push_back(us);
    else
        s->lat_us[s->lat_next++ % kLatKeep] = us;
}

// Build and launch one batch from the queues (called with the lock held; the
// CUDA calls are asynchronous).  Returns false when nothing was launched.
static bool launch_batch(sk_server_s *s, int slot_idx)
{
    LaunchSlot &L = s->slots[slot_idx];
    L.tickets.clear();
    L.streams.clear();
    std::vector<Item> items;
    std::vector<StreamRec *> recs;
    std::vector<int32_t> ring_slots;
    const size_t ns = s->streams.size();
    if (ns == 0)
        return false;
    std::vector<StreamRec *> order;
    for (auto &kv : s->streams)
        order.push_back(kv.second.get());
    for (size_t j = 0; j < ns && (int)items.size() < kMaxBatch; ++j) {
        StreamRec *r = order[(s->rr + j) % ns];
        if (r->queue.empty())
            continue;
        Pending pd = r->queue.front();
        r->queue.pop_front();
        Item it = r->plan->item(r->d_ring + (int64_t)pd.slot * r->fbytes, 1);
        const int k = (int)items.size();
        it.sk = L.d_sk + k;
        it.mask = L.d_mask + k;
        if (r->stateful) {
            it.state = r->d_state;
            it.state_init = r->initialised ? 0 : 1;
            r->initialised = true;
        }
        items.push_back(it);
        recs.push_back(r);
        ring_slots.push_back(pd.slot);
        L.tickets.push_back(pd.ticket);
        L.streams.push_back(r->id);
        r->in_flight += 1;
    }
    s->rr = (s->rr + 1) % ns;
    if (items.empty())
        return false;
    bool all_m32 = true;
    for (const Item &it : items)
        all_m32 = all_m32 && (it.M % 32 == 0);
    L.tile = pick_tile(16, all_m32);
    // schedule over at most one CTA per frame-round, at most one per SM
    int rounds = 0;
    for (const Item &it : items)
        rounds += 1;
    const int grid = std::min(s->sms, rounds);
    std::vector<Chunk> chunks;
    std::vector<int32_t> cta;
    build_schedule(items, grid, chunks, cta);
    L.n = (int)items.size();
    memcpy(L.h_items, items.data(), sizeof(Item) * items.size());
    memcpy(L.h_chunks, chunks.data(), sizeof(Chunk) * chunks.size());
    memcpy(L.h_cta, cta.data(), sizeof(int32_t) * cta.size());
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < items.size() && e == cudaSuccess; ++k) {
        StreamRec *r = recs[k];
        e = cudaMemcpyAsync(r->d_ring + (int64_t)ring_slots[k] * r->fbytes,
                            r->h_stage + (int64_t)ring_slots[k] * r->fbytes, (size_t)r->fbytes,
                            cudaMemcpyHostToDevice, s->s_copy);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(L.uploaded, s->s_copy);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(s->s_compute, L.uploaded, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.d_items, L.h_items, sizeof(Item) * items.size(),
                            cudaMemcpyHostToDevice, s->s_compute);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.d_chunks, L.h_chunks, sizeof(Chunk) * chunks.size(),
                            cudaMemcpyHostToDevice, s->s_compute);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.d_cta, L.h_cta, sizeof(int32_t) * cta.size(),
                            cudaMemcpyHostToDevice, s->s_compute);
    sk_status_t st = SK_OK;
    if (e == cudaSuccess)
        st = launch_schedule(L.d_items, L.d_chunks, L.d_cta, grid, L.tile, true, s->device,
                             s->s_compute);
    if (e == cudaSuccess && st == SK_OK)
        e = cudaMemcpyAsync(L.h_sk, L.d_sk, sizeof(float) * items.size(), cudaMemcpyDeviceToHost,
                            s->s_compute);
    if (e == cudaSuccess && st == SK_OK)
        e = cudaMemcpyAsync(L.h_mask, L.d_mask, items.size(), cudaMemcpyDeviceToHost,
                            s->s_compute);
    if (e == cudaSuccess && st == SK_OK)
        e = cudaEventRecord(L.done, s->s_compute);
    if (e != cudaSuccess || st != SK_OK) {
        s->fault = e != cudaSuccess ? SK_ERR_CUDA : st;
        s->fault_msg = e != cudaSuccess ? cudaGetErrorString(e) : "launch failed";
    }
    L.busy = true;
    s->launches += 1;
    s->flight.push_back(slot_idx);
    return true;
}

static void launcher_main(sk_server_s *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        int free_slot = -1;
        for (int i = 0; i < kLaunchSlots; ++i)
            if (!s->slots[i].busy) {
                free_slot = i;
                break;
            }
        bool any = false;
        for (auto &kv : s->streams)
            if (!kv.second->queue.empty()) {
                any = true;
                break;
            }
        if (free_slot < 0 || !any || s->fault != SK_OK) {
            s->cv_work.wait(lk);
            continue;
        }
        if (launch_batch(s, free_slot))
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
        if (s->flight.empty() && s->stop)
            return;
        const int idx = s->flight.front();
        LaunchSlot &L = s->slots[idx];
        lk.unlock();
        cudaError_t e = cudaEventSynchronize(L.done);
        const Clock::time_point now = Clock::now();
        lk.lock();
        s->flight.pop_front();
        if (e != cudaSuccess && s->fault == SK_OK) {
            s->fault = SK_ERR_CUDA;
            s->fault_msg = cudaGetErrorString(e);
        }
        for (int k = 0; k < L.n; ++k) {
            auto t = s->tickets.find(L.tickets[k]);
            if (t != s->tickets.end()) {
                t->second.done = true;
                t->second.status = s->fault;
                t->second.sk = L.h_sk[k];
                t->second.mask = L.h_mask[k];
                record_latency(s, std::chrono::duration<double, std::micro>(
                                      now - t->second.t_submit).count());
            }
            s->frames_done += 1;
            s->frames_flagged += L.h_mask[k] ? 1 : 0;
            auto r = s->streams.find(L.streams[k]);
            if (r != s->streams.end()) {
                r->second->in_flight -= 1;
                r->second->used -= 1;
            }
        }
        L.busy = false;
        L.n = 0;
        s->cv_done.notify_all();
        s->cv_work.notify_one();
    }
}

static void free_slot_buffers(LaunchSlot &L)
{
    cudaFreeHost(L.h_items);
    cudaFreeHost(L.h_chunks);
    cudaFreeHost(L.h_cta);
    cudaFreeHost(L.h_sk);
    cudaFreeHost(L.h_mask);
    cudaFree(L.d_items);
    cudaFree(L.d_chunks);
    cudaFree(L.d_cta);
    cudaFree(L.d_sk);
    cudaFree(L.d_mask);
    if (L.uploaded)
        cudaEventDestroy(L.uploaded);
    if (L.done)
        cudaEventDestroy(L.done);
}

static void free_stream(StreamRec *r)
{
    cudaFreeHost(r->h_stage);
    cudaFree(r->d_ring);
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
    sk_server_s *s = new (std::nothrow) sk_server_s();
    if (!s)
        return set_error(SK_ERR_OOM, "host allocation");
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->sms = sm_count(device);
    sk_status_t st = SK_OK;
    {
        DeviceGuard dg(device);
        const int max_chunks = kMaxBatch + s->sms + 1;
        for (int i = 0; i < kLaunchSlots && st == SK_OK; ++i) {
            LaunchSlot &L = s->slots[i];
            L.max_chunks = max_chunks;
            if (cudaHostAlloc(&L.h_items, sizeof(Item) * kMaxBatch, 0) != cudaSuccess ||
                cudaHostAlloc(&L.h_chunks, sizeof(Chunk) * max_chunks, 0) != cudaSuccess ||
                cudaHostAlloc(&L.h_cta, sizeof(int32_t) * (s->sms + 1), 0) != cudaSuccess ||
                cudaHostAlloc(&L.h_sk, sizeof(float) * kMaxBatch, 0) != cudaSuccess ||
                cudaHostAlloc(&L.h_mask, kMaxBatch, 0) != cudaSuccess ||
                cudaMalloc(&L.d_items, sizeof(Item) * kMaxBatch) != cudaSuccess ||
                cudaMalloc(&L.d_chunks, sizeof(Chunk) * max_chunks) != cudaSuccess ||
                cudaMalloc(&L.d_cta, sizeof(int32_t) * (s->sms + 1)) != cudaSuccess ||
                cudaMalloc(&L.d_sk, sizeof(float) * kMaxBatch) != cudaSuccess ||
                cudaMalloc(&L.d_mask, kMaxBatch) != cudaSuccess)
                st = set_error(SK_ERR_OOM, "server launch buffers");
            else if (cudaEventCreateWithFlags(&L.uploaded, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess)
                st = set_error(SK_ERR_CUDA, "server events");
        }
        if (st == SK_OK &&
            (cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
             cudaStreamCreateWithFlags(&s->s_compute, cudaStreamNonBlocking) != cudaSuccess))
            st = set_error(SK_ERR_CUDA, "server streams");
        if (st == SK_OK)
            st = ensure_kernel_attrs(device);
        if (st != SK_OK) {
            for (auto &L : s->slots)
                free_slot_buffers(L);
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
    {
        DeviceGuard dg(s->device);
        cudaStreamSynchronize(s->s_compute);
        cudaStreamSynchronize(s->s_copy);
        for (auto &kv : s->streams)
            free_stream(kv.second.get());
        for (auto &L : s->slots)
            free_slot_buffers(L);
        cudaStreamDestroy(s->s_copy);
        cudaStreamDestroy(s->s_compute);
    }
    delete s;
    return SK_OK;
}

extern "C" sk_status_t sk_stream_open(sk_server_t s, const sk_params_t *params,
                                      int32_t ring_frames, sk_stream_id *out)
{
    if (!s || !params || !out)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_open: null argument");
    *out = -1;
    if (ring_frames < 1 || ring_frames > 65536)
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_open: ring_frames outside 1..65536");
    if (params->layout != SK_LAYOUT_TIME_MAJOR)
        return set_error(SK_ERR_UNSUPPORTED, "sk_stream_open: served streams are time-major");
    const int64_t fbytes = (int64_t)params->n_time * params->n_inputs;
    const size_t need = (size_t)fbytes * ring_frames + sizeof(uint32_t) * params->n_inputs +
                        sizeof(int64_t) * (2 * (params->n_inputs + 1) + SK_OFFSET_BUCKETS) +
                        sizeof(float) * (params->n_inputs + 1);
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->in_use + need > s->budget) {
            s->rejected += 1;
            return set_error(SK_ERR_BUSY, "sk_stream_open: %zu bytes over the HBM budget",
                             s->in_use + need - s->budget);
        }
        s->in_use += need;  // reserve
    }
    auto r = std::make_unique<StreamRec>();
    sk_status_t st = sk_plan_create(params, s->device, &r->plan);
    if (st == SK_OK) {
        DeviceGuard dg(s->device);
        r->N = params->n_inputs;
        r->M = params->n_time;
        r->fbytes = fbytes;
        r->ring = ring_frames;
        r->stateful = (params->flags & SK_RUNNING_OFFSET) != 0;
        r->hbm = need;
        if (cudaHostAlloc(&r->h_stage, (size_t)fbytes * ring_frames, 0) != cudaSuccess ||
            cudaMalloc(&r->d_ring, (size_t)fbytes * ring_frames) != cudaSuccess ||
            cudaMalloc(&r->d_state, sizeof(uint32_t) * r->N) != cudaSuccess)
            st = set_error(SK_ERR_OOM, "sk_stream_open: ring or state allocation");
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (st != SK_OK) {
        s->in_use -= need;
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
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->fault != SK_OK)
        return set_error(s->fault, "server fault: %s", s->fault_msg.c_str());
    auto it = s->streams.find(id);
    if (it == s->streams.end())
        return set_error(SK_ERR_INVALID_ARG, "sk_stream_submit: unknown stream %d", id);
    StreamRec *r = it->second.get();
    if (r->closing)
        return set_error(SK_ERR_CLOSED, "sk_stream_submit: stream %d closing", id);
    if (r->used >= r->ring) {
        s->rejected += 1;
        return set_error(SK_ERR_BUSY, "sk_stream_submit: ring of stream %d full", id);
    }
    const int32_t slot = r->next_slot;
    r->next_slot = (r->next_slot + 1) % r->ring;
    r->used += 1;
    const sk_ticket_t t = s->next_ticket++;
    TicketRec tr;
    tr.stream = id;
    tr.t_submit = Clock::now();
    s->tickets.emplace(t, tr);
    // the slot is ours until its launch completes: copy outside the lock
    uint8_t *dst = r->h_stage + (int64_t)slot * r->fbytes;
    const int64_t fb = r->fbytes;
    lk.unlock();
    memcpy(dst, frame, (size_t)fb);
    lk.lock();
    auto it2 = s->streams.find(id);
    if (it2 == s->streams.end())
        return set_error(SK_ERR_CLOSED, "sk_stream_submit: stream %d closed", id);
    it2->second->queue.push_back(Pending{slot, t});
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
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end())
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
    it = s->tickets.find(ticket);
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
    return it == s->streams.end() || it->second->used == 0;
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
    if (r->used != 0)
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
    if (r->used != 0)
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
    // in-flight launches reference the ring and state: wait for them (bounded)
    bool idle = s->cv_done.wait_for(lk, std::chrono::seconds(30),
                                    [&] { return stream_idle(s, id) || s->fault != SK_OK; });
    if (!idle)
        return set_error(SK_ERR_TIMEOUT, "sk_stream_close: stream %d still busy", id);
    std::unique_ptr<StreamRec> r = std::move(s->streams[id]);
    s->streams.erase(id);
    s->in_use -= r->hbm;
    // drop its uncollected tickets of frames never launched
    for (const Pending &p : r->queue)
        s->tickets.erase(p.ticket);
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
        out->hbm_in_use = s->in_use;
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
