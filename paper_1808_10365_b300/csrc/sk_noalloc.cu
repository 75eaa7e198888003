// sk_flag_host_noalloc: the host-buffer flagging call without any device
// allocation.  sk_flag_host stages the caller's bytes through device buffers
// that the plan allocates on first use; this variant stages them through one
// fixed array compiled into the library instead.
//
// Who needs it: callers that must not call cudaMalloc once they are running --
// a process whose device memory is all handed out by another allocator (a
// framework's caching pool that reserved the HBM), or a real-time loop where an
// allocation could synchronise the device and miss a deadline.  Such callers
// create their plan at start-up and then use only this call.
//
// The array is a file-scope __device__ variable: every GPU on which the module
// holding it is loaded keeps it (SK_NOALLOC_MAX_BYTES + 5 * SK_NOALLOC_MAX_FRAMES
// bytes) until the process exits.  Host code cannot use the array's name as a
// device address (on the host it names a stand-in), so its device address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current.  The look-up is part of set-up: sk_plan_create does it for the
// plan's device (noalloc_prepare), because with lazy module loading it is the
// look-up that loads this file's module and so takes the array's memory from
// the driver.  A plan created before the device's memory is handed to another
// allocator therefore leaves nothing for this call to allocate.  If that
// look-up failed at plan creation, the first call on the device retries it and
// reports its error.  All calls on a device share the array and each call leaves
// its data there; nothing in it has to start at zero, because the kernel writes
// every output it reads back.  Calls from this process are serialised per device
// (the call synchronises its stream before returning); work issued elsewhere
// that overlaps on the GPU with a call would race on the array.
#include <mutex>

#include "sk_common.h"

using namespace sk;

namespace {

constexpr size_t kInBytes = (size_t)SK_NOALLOC_MAX_BYTES;
constexpr size_t kSkOff = kInBytes;
constexpr size_t kMaskOff = kSkOff + sizeof(float) * (size_t)SK_NOALLOC_MAX_FRAMES;
constexpr size_t kTotal = kMaskOff + (size_t)SK_NOALLOC_MAX_FRAMES;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kTotal];

constexpr int kMaxDevices = 64;
std::mutex g_dev_mu[kMaxDevices];
uint8_t *g_dev_ptr[kMaxDevices] = {};

// Device address of the array on `device` (current); looked up once.  Called
// with g_dev_mu[device] held.
sk_status_t scratch_address(int device, uint8_t **out)
{
    if (!g_dev_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_error(e, "sk_flag_host_noalloc: cudaGetSymbolAddress");
        g_dev_ptr[device] = (uint8_t *)p;
    }
    *out = g_dev_ptr[device];
    return SK_OK;
}

}  // namespace

// Set-up at plan creation (device current): the array's address on `device`,
// which loads the module that holds it.  A failure here is left for the first
// sk_flag_host_noalloc call on the device to report.
void sk::noalloc_prepare(int device)
{
    if (device < 0 || device >= kMaxDevices)
        return;
    std::lock_guard<std::mutex> g(g_dev_mu[device]);
    uint8_t *p = nullptr;
    if (scratch_address(device, &p) != SK_OK)
        cudaGetLastError();
}

extern "C" sk_status_t sk_flag_host_noalloc(sk_plan_t plan, const uint8_t *h_in,
                                            int64_t n_frames, float *h_sk, uint8_t *h_mask,
                                            sk_cuda_stream_t stream)
{
    NvtxRange nv("sk_flag_host_noalloc");
    if (!plan)
        return set_error(SK_ERR_INVALID_ARG, "sk_flag_host_noalloc: plan is NULL");
    if (sk_status_t f = pending_fault(plan, "sk_flag_host_noalloc"))
        return f;
    if (n_frames < 0 || (n_frames > 0 && (!h_in || !h_mask)))
        return set_error(SK_ERR_INVALID_ARG, "sk_flag_host_noalloc: bad arguments");
    if (n_frames == 0)
        return SK_OK;
    const int64_t fbytes = (int64_t)plan->p.n_time * plan->p.n_inputs;
    if (n_frames > (int64_t)SK_NOALLOC_MAX_FRAMES || n_frames * fbytes > (int64_t)kInBytes)
        return set_error(SK_ERR_INVALID_ARG,
                         "sk_flag_host_noalloc: %lld frames of %lld bytes exceed the fixed "
                         "staging area (%lld bytes, %d frames); split the call",
                         (long long)n_frames, (long long)fbytes, (long long)kInBytes,
                         SK_NOALLOC_MAX_FRAMES);
    if (plan->device < 0 || plan->device >= kMaxDevices)
        return set_error(SK_ERR_UNSUPPORTED, "sk_flag_host_noalloc: device %d", plan->device);
    std::lock_guard<std::mutex> g(g_dev_mu[plan->device]);
    DeviceGuard dg(plan->device);
    uint8_t *base = nullptr;
    sk_status_t s = scratch_address(plan->device, &base);
    if (s != SK_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    float *d_sk = (float *)(base + kSkOff);
    uint8_t *d_mask = base + kMaskOff;
    cudaError_t e = cudaMemcpyAsync(base, h_in, (size_t)(n_frames * fbytes),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return cuda_error(e, "sk_flag_host_noalloc: upload");
    Item it = plan->item(base, n_frames);
    it.sk = h_sk ? d_sk : nullptr;
    it.mask = d_mask;
    // the plan's row-balancing scratch only if an earlier call allocated it
    s = launch_single(it, plan->rows, false, plan->device, st, plan->grid_ctas, plan, false);
    if (s != SK_OK)
        return s;
    e = cudaMemcpyAsync(h_mask, d_mask, (size_t)n_frames, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && h_sk)
        e = cudaMemcpyAsync(h_sk, d_sk, sizeof(float) * (size_t)n_frames,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_error(e, "sk_flag_host_noalloc: download");
    // the launch is complete: a bounded wait of its own that gave up voids it
    return pending_fault(plan, "sk_flag_host_noalloc");
}
