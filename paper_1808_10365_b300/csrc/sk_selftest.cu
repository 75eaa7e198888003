// Self-test of the exact conversions the kernels' epilogue uses in place of
// CUDA's int64 <-> fp32 conversion instructions (u43_to_f32_rn, f32_to_i64_rn,
// and the input term built on them): each is compared, bit for bit, with the
// conversion intrinsics it replaces (__ll2float_rn, __float2ll_rn).
//   fp32 -> int64: every non-negative fp32 below 2^62 (the whole domain).
//   int64 -> fp32: every x below 2^25; every value with 25 significant bits
//     below 2^43 (the halfway cases of round-to-nearest-even) and its two
//     neighbours; a hashed sample of 2^28 values below 2^43.
//   input term (Eqs. discreteMean, normedSum2): a hashed sample of 2^26 valid
//     (S1, S2, M) with M from 2 to 4096 and 0 < S1 <= 128 M, S1^2 <= M S2 <= 128 M S1.
//   fp32(S1^2) from an exact fp32 S1 and one multiply: every S1 from 1 to 2^19.
//
// And a self-test of the bounded slot wait of the warp-slice combine
// (wi_commit): one warp of a two-warp team commits frame counter 0 into a slot
// still held by the frame a ring back, which never completes.
#include "sk_common.h"

namespace sk {

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void check_f32_to_i64(uint32_t n, unsigned long long *bad)
{
    unsigned long long nb = 0;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x) {
        const float y = __uint_as_float(b);
        nb += f32_to_i64_rn(y) != __float2ll_rn(y);
    }
    if (nb)
        atomicAdd(bad, nb);
}

// Index space: [0, 2^25) all x; then 19 exponents x 2^23 odd 25-bit mantissas,
// each with its neighbours -1, 0, +1 (3 values); then 2^28 hashed values.
constexpr uint64_t kSmall = 1ull << 25;
constexpr uint64_t kTies = 19ull * (1ull << 23) * 3;
constexpr uint64_t kHashed = 1ull << 28;

__device__ __forceinline__ int64_t u43_case(uint64_t i)
{
    if (i < kSmall)
        return (int64_t)i;
    i -= kSmall;
    if (i < kTies) {
        const uint64_t k = i / 3, d = i % 3;
        const uint64_t e = 25 + k / (1ull << 23);              // 25 .. 43
        const uint64_t t = (1ull << 24) | ((k % (1ull << 23)) << 1) | 1ull;  // odd, 25 bits
        const int64_t x = (int64_t)(t << (e - 25));
        return x + (int64_t)d - 1;
    }
    i -= kTies;
    return (int64_t)(mix64(i) & ((1ull << 43) - 1));
}

__global__ void check_u43_to_f32(uint64_t n, unsigned long long *bad)
{
    unsigned long long nb = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t x = u43_case(i);
        if (x < 0 || x >= (1ll << 43))
            continue;
        nb += __float_as_uint(u43_to_f32_rn(x)) != __float_as_uint(__ll2float_rn(x));
    }
    if (nb)
        atomicAdd(bad, nb);
}

// fp32(S1^2) as the epilogue forms it (an exact fp32 S1, one IEEE multiply) against
// CUDA's conversion of the exact integer S1^2, for every S1 from 1 to 2^19 (the
// largest S1: 4096 samples of power 128)
__global__ void check_square(uint32_t n, unsigned long long *bad)
{
    unsigned long long nb = 0;
    for (uint32_t s1 = 1 + blockIdx.x * blockDim.x + threadIdx.x; s1 <= n;
         s1 += gridDim.x * blockDim.x) {
        const float fs1 = __fsub_rn(__uint_as_float(0x4B000000u | s1), 8388608.0f);
        nb += __float_as_uint(__fmul_rn(fs1, fs1)) !=
              __float_as_uint(__ll2float_rn((int64_t)s1 * (int64_t)s1));
    }
    if (nb)
        atomicAdd(bad, nb);
}

__global__ void check_input_term(uint64_t n, unsigned long long *bad)
{
    unsigned long long nb = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t h = mix64(i ^ 0x5EC7E57ull);
        const int32_t M = 2 + (int32_t)(h % 4095);
        const int32_t s1 = 1 + (int32_t)((h >> 12) % (uint64_t)(128 * M));
        // S2 between S1^2/M (all samples equal) and 128 S1 (every sample 128)
        const int64_t lo = ((int64_t)s1 * s1 + M - 1) / M;
        const int64_t hi = 128ll * s1;
        const int32_t s2 = (int32_t)(lo + (int64_t)((h >> 32) % (uint64_t)(hi - lo + 1)));
        float ra = 0.0f, rb = 0.0f;
        int64_t qa = 0, qb = 0;
        const bool ha = input_term_alu(s1, s2, M, ra, qa);
        const bool hb = input_term(s1, s2, M, rb, qb);
        nb += ha != hb || __float_as_uint(ra) != __float_as_uint(rb) || qa != qb;
    }
    if (nb)
        atomicAdd(bad, nb);
}

}  // namespace

}  // namespace sk

extern "C" sk_status_t sk_selftest_conversions(int device, int64_t *n_checked, int64_t *n_bad)
{
    using namespace sk;
    if (!n_checked || !n_bad)
        return set_error(SK_ERR_INVALID_ARG, "sk_selftest_conversions: NULL output");
    DeviceGuard dg(device);
    unsigned long long *d_bad = nullptr;
    cudaError_t e = cudaMalloc(&d_bad, 3 * sizeof(unsigned long long));
    if (e != cudaSuccess)
        return cuda_error(e, "sk_selftest_conversions allocation");
    const uint32_t n_f32 = 0x5E800000u;  // bits of 2^62
    const uint64_t n_u43 = kSmall + kTies + kHashed;
    const uint64_t n_term = 1ull << 26;
    const uint32_t n_square = 1u << 19;
    const int grid = sm_count(device) * 8;
    unsigned long long h_bad[3] = {0, 0, 0};
    if ((e = cudaMemset(d_bad, 0, sizeof h_bad)) == cudaSuccess) {
        check_f32_to_i64<<<grid, 256>>>(n_f32, d_bad);
        check_u43_to_f32<<<grid, 256>>>(n_u43, d_bad + 1);
        check_input_term<<<grid, 256>>>(n_term, d_bad + 2);
        check_square<<<grid, 256>>>(n_square, d_bad + 2);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpy(h_bad, d_bad, sizeof h_bad, cudaMemcpyDeviceToHost);
    }
    cudaFree(d_bad);
    if (e != cudaSuccess)
        return cuda_error(e, "sk_selftest_conversions");
    *n_checked = (int64_t)n_f32 + (int64_t)n_u43 + (int64_t)n_term + (int64_t)n_square;
    *n_bad = (int64_t)(h_bad[0] + h_bad[1] + h_bad[2]);
    return SK_OK;
}

namespace sk {

namespace {

// One warp (the first of a team of W = 2) commits its part of frame counter 0.
// Slot 0 is initialised as held by counter -kWiSlots (its tag is kWiSlots, not
// 0), the state a ring turn behind a slow warp leaves; nobody frees it, so the
// wait gives up after spin_limit polls and raises it.err.  The part is added
// into the slot afterwards, as on the real path, but the second warp never
// arrives, so no frame is written.
__global__ void slot_wait_kernel(Item it, int spin_limit)
{
    __shared__ WiSlot slots[kWiSlots];
    if (threadIdx.x < kWiSlots) {
        slots[threadIdx.x].q = 0ull;
        slots[threadIdx.x].cnt = 0;
        slots[threadIdx.x].arrive = 0;
        slots[threadIdx.x].tag = (unsigned)(threadIdx.x + kWiSlots);
    }
    __syncwarp();
    if (threadIdx.x == 0)
        wi_commit(it, slots, 0, 2, 0, 0, 0, spin_limit);
    __syncwarp();
}

}  // namespace

}  // namespace sk

extern "C" sk_status_t sk_selftest_slot_wait(sk_plan_t plan, int32_t spin_limit,
                                             int32_t *gave_up, sk_cuda_stream_t stream)
{
    using namespace sk;
    if (!plan || !gave_up)
        return set_error(SK_ERR_INVALID_ARG, "sk_selftest_slot_wait: null argument");
    if (spin_limit < 1 || spin_limit > kWiSpinLimit)
        return set_error(SK_ERR_INVALID_ARG, "sk_selftest_slot_wait: spin_limit %d outside 1..%d",
                         spin_limit, kWiSpinLimit);
    DeviceGuard dg(plan->device);
    const int32_t before = *reinterpret_cast<volatile int32_t *>(plan->h_err);
    Item it = plan->item(nullptr, 1);
    cudaStream_t st = (cudaStream_t)stream;
    slot_wait_kernel<<<1, 32, 0, st>>>(it, spin_limit);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_error(e, "sk_selftest_slot_wait");
    *gave_up = (!before && *reinterpret_cast<volatile int32_t *>(plan->h_err)) ? 1 : 0;
    return SK_OK;
}
