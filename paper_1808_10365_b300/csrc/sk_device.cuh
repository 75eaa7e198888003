// Device code of the fused spectral-kurtosis kernel (sm_103a).
//
// One pass over the packed bytes computes, per frame of M samples x N inputs:
//   a1 unpack    re = (b >> 4) - 8, im = (b & 15) - 8     (4+4-bit offset binary)
//   a2 power     p = re^2 + im^2                          (Sec. 2.2.3 table)
//   a3 sums      S1_i = sum p, S2_i = sum p^2  exact int32 (Eq. 1, Eq. singlesums)
//   a4 normalise r_i = (M S2_i - S1_i^2) / S1_i^2, numerator and denominator exact
//                in int64, one fp32 divide                  (Eqs. discreteMean, normedSum2)
//   a5 combine   Q = sum_i rint(2^32 r_i) (int64, order independent), N_eff
//   a6 SK~       (M+1)/((M-1) N_eff) * Q 2^-32 in fp32     (Eq. final: SK~ = Avg(SK^_i))
//   a7 flag      Q outside [T_lo, T_hi][N_eff]             (Sec. 3.2, App. B offset)
//   a8 served    per-input power state shifts the thresholds by its digitisation offset
//
// Sample path.  a1-a3 cost one byte of HBM per sample, so they must run in about
// three instructions per byte to keep up with HBM.  Each sample is:
//   PRMT  builds a shared-memory address from the byte itself:
//         [lane*4 | byte << 8 | table base]  (table base 64 KiB aligned),
//   LDS   reads the packed value p^2 | p << 19 from a 256-entry table replicated
//         once per lane (entry b of lane L sits in bank L: conflict free),
//   IADD  accumulates it.
// Sixteen samples fit the packed 32-bit accumulator (16 p^2 <= 2^18 < 2^19,
// 16 p <= 2^11), after which it is split into the exact S1 and S2.
#pragma once

#include <cuda.h>  // CUtensorMap (the 2D tensor prefetch of the warp-slice path)
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace sk {

constexpr int kThreads = 512;               // one CTA per SM
constexpr int kVec = 8;                     // inputs per thread: one 8-byte load per row
constexpr int kFlushRows = 16;              // rows per packed accumulator
constexpr int kLutRow = 256;                // bytes per table entry (32 lanes x 4 B used)
constexpr int kLutBytes = 256 * kLutRow;    // 64 KiB
constexpr int kDynSmem = 2 * kLutBytes;     // room to put the table on a 64 KiB boundary
constexpr int kSlots = kThreads / 32;       // partial-sum slots per parity
constexpr int kPackShift = 19;
constexpr uint32_t kPackMask = (1u << kPackShift) - 1u;
constexpr int kOffsetBuckets = 4096;
constexpr int kStateShift = 6;

// Output and table pointers of one work item: frames of one (N, M).
struct Item {
    const uint8_t *in;       // [n_frames][M][N] time-major or [n_frames][N][M]
    int64_t n_frames;
    int32_t M, N;
    int32_t layout;          // 0 time-major, 1 input-major
    int32_t team_log2;       // threads per frame = 1 << team_log2 (vector and general paths)
    int32_t imajor_team_log2;  // threads per frame on the input-major kernel
    float *sk;
    uint8_t *mask;
    int64_t *q;
    int32_t *neff;
    int32_t *s1;
    int32_t *s2;
    const int64_t *t_lo;     // [N+1]
    const int64_t *t_hi;     // [N+1]
    const float *c_tab;      // [N+1]: fp32((M+1)/((M-1) n))
    uint32_t *state;         // served: per-input power P_i [N], or null
    const int64_t *e_tab;    // served: offset per power bucket [kOffsetBuckets]
    int32_t state_init;      // served: 1 on the stream's first frame
    int32_t fast;            // 1: time-major vector path, 2: input-major path, 3: time-major
                             // ragged N (balanced rows, else general), 4: time-major
                             // M % 16 != 0 (warp slices with a partial last turn, else
                             // general), 0: general
    float *sk_in;            // per-input SK^_i [n_frames][N] (Eq. originalSK), or null
    uint8_t *mask_in;        // per-input flag at the N_eff = 1 thresholds, or null
    int32_t prefetch;        // 1: input in device memory, L2 bulk prefetch allowed
    int32_t running_mu;      // served: normalise by the running power in the state
    double n_sigma;          // running-mu decision (double domain)
    double mean_offset;
    int32_t wi;              // nonzero: the warps of a frame combine through the slot ring
                             // (time-major: warp-slice path, 1 with the tensor map for
                             // the L2 prefetch, 2 without, when N % 16 != 0)
    int32_t wtail;           // time-major warp slices: groups of 8 columns past the last
                             // whole 256-column slice read row-per-lane by the team's
                             // warps (1..4), or 0: the partial slice is a warp of its own
    int32_t *err;            // mapped host word: set when a bounded wait gives up
    const CUtensorMap *tmap;  // batched time-major items: the input's map in device memory
    int32_t *rb;              // row-balanced warp-slice launch: the plan's zeroed scratch
#ifdef SK_DEBUG
    int64_t dbg_in_bytes;     // debug builds: bytes of `in` the kernel may read
    int64_t dbg_rb_slots;     // debug builds: slots of the row-balancing scratch
#endif
};

// Debug builds (-DSK_DEBUG) check every global load and every output store of
// the kernels against the item's buffers before making it: an access outside
// them is skipped (a load gives bytes without power) and sets the plan's error
// word to kErrBounds, which the plan's next call reports.  No trap: the launch
// runs to its end.  Release builds compile the checks to nothing.
constexpr int32_t kErrBounds = 2;
#ifdef SK_DEBUG
__device__ __forceinline__ bool dbg_fail(const Item &it)
{
    if (it.err)
        atomicExch(it.err, kErrBounds);
    return false;
}
// [p, p + bytes) inside the item's input
__device__ __forceinline__ bool dbg_in(const Item &it, const void *p, int64_t bytes)
{
    const uint8_t *b = (const uint8_t *)p;
    return (b >= it.in && bytes >= 0 && b + bytes <= it.in + it.dbg_in_bytes) ? true
                                                                              : dbg_fail(it);
}
// frame f of the item's per-frame outputs, and input i of its per-input ones
__device__ __forceinline__ bool dbg_out(const Item &it, int64_t f, int64_t i = 0)
{
    return (f >= 0 && f < it.n_frames && i >= 0 && i < it.N) ? true : dbg_fail(it);
}
__device__ __forceinline__ bool dbg_slot(const Item &it, int64_t slot)
{
    return (slot >= 0 && slot < it.dbg_rb_slots) ? true : dbg_fail(it);
}
#define SK_DBG_IN(it, p, bytes) ::sk::dbg_in((it), (p), (int64_t)(bytes))
#define SK_DBG_OUT(it, f) ::sk::dbg_out((it), (int64_t)(f))
#define SK_DBG_OUT_IN(it, f, i) ::sk::dbg_out((it), (int64_t)(f), (int64_t)(i))
#define SK_DBG_SLOT(it, s) ::sk::dbg_slot((it), (int64_t)(s))
#else
#define SK_DBG_IN(it, p, bytes) true
#define SK_DBG_OUT(it, f) true
#define SK_DBG_OUT_IN(it, f, i) true
#define SK_DBG_SLOT(it, s) true
#endif

// Work of one CTA.  kind 0: frames [f_begin, f_end) of item `item`, the CTA's
// teams striding through them.  kind 1: items [f_begin, f_end), one frame each
// and all of one shape (N, M, layout), each team taking its own items.
struct Chunk {
    int32_t item;
    int32_t kind;
    int64_t f_begin;
    int64_t f_end;
};

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// volatile: the load must never be hoisted or speculated past the bounds test
// that guards it (callers only issue it for rows inside the frame).
__device__ __forceinline__ uint2 ldg_stream(const uint8_t *p)
{
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v2.u32 {%0, %1}, [%2];"
        : "=r"(v.x), "=r"(v.y)
        : "l"(p));
    return v;
}

// One 16-byte chunk, streamed like ldg_stream (p 16-byte aligned).
__device__ __forceinline__ uint4 ldg_stream16(const uint8_t *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Same load at base + OFF with OFF a compile-time immediate of the instruction.
template <int OFF>
__device__ __forceinline__ uint2 ldg_stream_at(const uint8_t *base)
{
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v2.u32 {%0, %1}, [%2+%3];"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(base), "n"(OFF));
    return v;
}

// Rows 0..R-1 of a batch whose row stride NC is known at compile time.
template <int NC, int... Rs>
__device__ __forceinline__ void load_rows_imm(uint2 *b, const uint8_t *base,
                                              std::integer_sequence<int, Rs...>)
{
    ((b[Rs] = ldg_stream_at<Rs * NC>(base)), ...);
}

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of
// 16); a hint only, results never depend on it.
__device__ __forceinline__ void prefetch_l2(const uint8_t *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Packed table value for byte b: p^2 in bits 0..18, p in bits 19..31.
__device__ __forceinline__ uint32_t packed_power(uint32_t b)
{
    int32_t re = (int32_t)(b >> 4) - 8;
    int32_t im = (int32_t)(b & 15u) - 8;
    uint32_t p = (uint32_t)(re * re + im * im);
    return (p << kPackShift) | (p * p);
}

// Fill the lane-replicated table; returns this thread's lane base address.
__device__ __forceinline__ uint32_t build_table(uint8_t *dyn_smem)
{
    uint32_t raw = (uint32_t)__cvta_generic_to_shared(dyn_smem);
    uint32_t base = (raw + 0xFFFFu) & ~0xFFFFu;
    for (int idx = threadIdx.x; idx < 256 * 32; idx += blockDim.x) {
        uint32_t b = (uint32_t)idx >> 5, lane = (uint32_t)idx & 31u;
        uint32_t addr = base + b * kLutRow + lane * 4u;
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(packed_power(b)) : "memory");
    }
    __syncthreads();
    // The lane base goes through a volatile shared load issued after the
    // barrier, so no table read that depends on it can move above the barrier.
    uint32_t probe;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(probe) : "r"(base) : "memory");
    uint32_t lane = threadIdx.x & 31u;
    return (base + (probe & 0u)) | (lane << 2);
}

// Accumulate one row (8 inputs, bytes in w) into the packed accumulators.
// PRMT selector 0x76k4: byte0 = lane*4, byte1 = byte k of the data word,
// bytes 2-3 = table base.
__device__ __forceinline__ void accum_row(uint2 w, uint32_t lb, uint32_t (&acc)[kVec])
{
    acc[0] += lds_u32(prmt(w.x, lb, 0x7604u));
    acc[1] += lds_u32(prmt(w.x, lb, 0x7614u));
    acc[2] += lds_u32(prmt(w.x, lb, 0x7624u));
    acc[3] += lds_u32(prmt(w.x, lb, 0x7634u));
    acc[4] += lds_u32(prmt(w.y, lb, 0x7604u));
    acc[5] += lds_u32(prmt(w.y, lb, 0x7614u));
    acc[6] += lds_u32(prmt(w.y, lb, 0x7624u));
    acc[7] += lds_u32(prmt(w.y, lb, 0x7634u));
}

// Two rows at once: both table values of an input go into one three-input add.
__device__ __forceinline__ void accum_pair(uint2 w0, uint2 w1, uint32_t lb, uint32_t (&acc)[kVec])
{
    acc[0] += lds_u32(prmt(w0.x, lb, 0x7604u)) + lds_u32(prmt(w1.x, lb, 0x7604u));
    acc[1] += lds_u32(prmt(w0.x, lb, 0x7614u)) + lds_u32(prmt(w1.x, lb, 0x7614u));
    acc[2] += lds_u32(prmt(w0.x, lb, 0x7624u)) + lds_u32(prmt(w1.x, lb, 0x7624u));
    acc[3] += lds_u32(prmt(w0.x, lb, 0x7634u)) + lds_u32(prmt(w1.x, lb, 0x7634u));
    acc[4] += lds_u32(prmt(w0.y, lb, 0x7604u)) + lds_u32(prmt(w1.y, lb, 0x7604u));
    acc[5] += lds_u32(prmt(w0.y, lb, 0x7614u)) + lds_u32(prmt(w1.y, lb, 0x7614u));
    acc[6] += lds_u32(prmt(w0.y, lb, 0x7624u)) + lds_u32(prmt(w1.y, lb, 0x7624u));
    acc[7] += lds_u32(prmt(w0.y, lb, 0x7634u)) + lds_u32(prmt(w1.y, lb, 0x7634u));
}

// Packed accumulator of 16 rows into the exact sums: S1 takes the high field
// (acc >> 19), and s2 takes the whole packed word, so that until finish_s2 it
// holds S2 + 2^19 S1 modulo 2^32 (one add per input instead of a mask and an add).
__device__ __forceinline__ void flush(uint32_t (&acc)[kVec], int32_t (&s1)[kVec],
                                      int32_t (&s2)[kVec])
{
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
        s1[k] += (int32_t)(acc[k] >> kPackShift);
        s2[k] = (int32_t)((uint32_t)s2[k] + acc[k]);
        acc[k] = 0u;
    }
}

// The exact S2 from flush's running sum: S2 = (S2 + 2^19 S1) - 2^19 S1 modulo 2^32,
// exact because 0 <= S2 < 2^32 (S2 <= 4096 * 128^2 = 2^26).  Once per frame part,
// after its last flush.
__device__ __forceinline__ void finish_s2(const int32_t (&s1)[kVec], int32_t (&s2)[kVec])
{
#pragma unroll
    for (int k = 0; k < kVec; ++k)
        s2[k] = (int32_t)((uint32_t)s2[k] - ((uint32_t)s1[k] << kPackShift));
}

// r_i scaled to 2^32 fixed point: D_i = M S2_i - S1_i^2 and S1_i^2 exact in
// int64, converted with round-to-nearest, one IEEE fp32 division, exact
// scaling by 2^32, round-to-nearest-even to int64.  Returns false (and leaves
// r, qi alone) for an input without power.
__device__ __forceinline__ bool input_term(int32_t s1, int32_t s2, int32_t M, float &r,
                                           int64_t &qi)
{
    if (s1 <= 0)
        return false;
    int64_t den = (int64_t)s1 * (int64_t)s1;
    int64_t d = (int64_t)M * (int64_t)s2 - den;
    r = __fdiv_rn(__ll2float_rn(d), __ll2float_rn(den));
    qi = __float2ll_rn(__fmul_rn(r, 4294967296.0f));
    return true;
}

// Exact conversions on the ALU and FMA pipes (the int64 <-> fp32 conversion
// instructions run on the FP64 pipe, which this GPU has little of).
//
// fp32 nearest to 0 <= x < 2^43: x = h 2^20 + l with h, l < 2^23 both exact in
// fp32 (formed by OR-ing them into the mantissa of 2^23 and subtracting 2^23);
// fmaf forms h 2^20 + l exactly and rounds once, so the result is x rounded to
// nearest even.
__device__ __forceinline__ float u43_to_f32_rn(int64_t x)
{
    const uint32_t h = (uint32_t)((uint64_t)x >> 20);
    const uint32_t l = (uint32_t)x & 0xFFFFFu;
    const float fh = __fsub_rn(__uint_as_float(0x4B000000u | h), 8388608.0f);
    const float fl = __fsub_rn(__uint_as_float(0x4B000000u | l), 8388608.0f);
    return __fmaf_rn(fh, 1048576.0f, fl);
}

// Nearest integer (ties to even) to a non-negative fp32 y < 2^62: below 2^23 by
// adding and removing 2^23 (the fp32 addition rounds to an integer), above it y
// already is an integer, its mantissa shifted by its exponent.
__device__ __forceinline__ int64_t f32_to_i64_rn(float y)
{
    const uint32_t bits = __float_as_uint(y);
    if (y < 8388608.0f)
        return (int64_t)(__float_as_uint(__fadd_rn(y, 8388608.0f)) - 0x4B000000u);
    const uint32_t m = (bits & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)(bits >> 23) - 150;  // exponent - 127 - 23 >= 0
    return (int64_t)((uint64_t)m << sh);
}

#ifndef SK_EPILOGUE_ALU
#define SK_EPILOGUE_ALU 1
#endif

// input_term with the conversions above (bit-identical results).
__device__ __forceinline__ bool input_term_alu(int32_t s1, int32_t s2, int32_t M, float &r,
                                               int64_t &qi)
{
    if (s1 <= 0)
        return false;
    int64_t den = (int64_t)s1 * (int64_t)s1;
    int64_t d = (int64_t)M * (int64_t)s2 - den;
    // fp32(S1^2): S1 < 2^23 is exact in fp32 (OR-ed into the mantissa of 2^23, less
    // 2^23), and one IEEE multiply rounds the exact product S1^2 once -- the same
    // value as converting the exact integer, in two instructions fewer than that
    const float fs1 = __fsub_rn(__uint_as_float(0x4B000000u | (uint32_t)s1), 8388608.0f);
    r = __fdiv_rn(u43_to_f32_rn(d), __fmul_rn(fs1, fs1));
    qi = f32_to_i64_rn(__fmul_rn(r, 4294967296.0f));
    return true;
}

// Per-frame accumulators of the warp-slice path: each team has a ring of kWiSlots
// slots; slot j holds the sums of the team's frame with counter `tag`.
constexpr int kWiSlots = 4;
constexpr int kMaxTail = 4;  // folded 8-column groups of the warp slices (Item::wtail)
struct WiSlot {
    unsigned long long q;
    int cnt;
    int arrive;
    unsigned tag;
    int pad;
};

struct TeamSmem {
    long long q[2][kSlots];
    long long e[2][kSlots];
    long long ra[2][kSlots];
    long long rb[2][kSlots];
    int cnt[2][kSlots];
    int rn[2][kSlots];
    WiSlot wi[kThreads / 32][kWiSlots];  // warp-slice paths: up to 16 teams (of one warp)
};

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p)
{
    return *reinterpret_cast<const volatile unsigned *>(p);
}

// Slots of the warp-slice combine before first use: slot j expects frame counter j.
__device__ __forceinline__ void init_wi_slots(TeamSmem &ts)
{
    for (int i = threadIdx.x; i < (kThreads / 32) * kWiSlots; i += blockDim.x) {
        WiSlot &sl = ts.wi[i / kWiSlots][i % kWiSlots];
        sl.q = 0ull;
        sl.cnt = 0;
        sl.arrive = 0;
        sl.tag = (unsigned)(i % kWiSlots);
    }
}

// The outputs of one frame from its Q and N_eff = C: the mask (Sec. 3.2 test of Q
// against the integer thresholds of C), SK (Eq. final), Q and N_eff.
__device__ __forceinline__ void write_frame(const Item &it, int64_t frame, int64_t Q, int32_t C)
{
    if (!SK_DBG_OUT(it, frame))
        return;
    uint8_t m = 1;
    if (C > 0)
        m = (Q > it.t_hi[C] || Q < it.t_lo[C]) ? 1 : 0;
    if (it.sk) {
        float skv = __int_as_float(0x7FC00000);
        if (C > 0)
            skv = __fmul_rn(__fmul_rn(__ll2float_rn(Q), 0x1p-32f), it.c_tab[C]);
        it.sk[frame] = skv;
    }
    if (it.mask)
        it.mask[frame] = m;
    if (it.q)
        it.q[frame] = Q;
    if (it.neff)
        it.neff[frame] = C;
}

// Lane 0 of a warp adds the warp's part (q, cnt) of the team's frame with counter
// kk (the frame's index `frame`) into the team's slot for it; the warp that arrives
// last of the team's W writes the frame's outputs (Sec. 3.2 test on Q against the
// integer thresholds of N_eff = cnt, SK of Eq. final) and frees the slot for frame
// counter kk + kWiSlots.  The wait for the slot is bounded: past spin_limit polls
// (64 ns apart; the default is about a quarter of a second) the warp sets the
// plan's error word and goes on, and the launch's results are void.
constexpr int kWiSpinLimit = 1 << 22;
__device__ __forceinline__ void wi_commit(const Item &it, WiSlot *slots, int64_t kk, int W,
                                          int64_t frame, int64_t q, int32_t cnt,
                                          int spin_limit = kWiSpinLimit)
{
    WiSlot &sl = slots[kk % kWiSlots];
    // the slot is this frame's once the frame kWiSlots back is done
    for (int spins = 0; ld_volatile_u32(&sl.tag) != (unsigned)kk; ++spins) {
        if (spins >= spin_limit) {
            atomicExch(it.err, 1);
            break;
        }
        __nanosleep(64);
    }
    atomicAdd(&sl.q, (unsigned long long)q);
    atomicAdd(&sl.cnt, cnt);
    __threadfence_block();
    if (atomicAdd(&sl.arrive, 1) == W - 1) {
        __threadfence_block();
        write_frame(it, frame, (int64_t)atomicAdd(&sl.q, 0ull), atomicAdd(&sl.cnt, 0));
        sl.q = 0ull;
        sl.cnt = 0;
        sl.arrive = 0;
        __threadfence_block();
        *reinterpret_cast<volatile unsigned *>(&sl.tag) = (unsigned)(kk + kWiSlots);
    }
}

// Sum of the running-mu terms (A, B, n) over the team, every thread gets them.
// Called by every thread of a served kernel whatever its item's flags, so that
// teams sharing a warp take the same shuffles.
__device__ __forceinline__ void team_sum_rmu(int64_t &a, int64_t &b, int32_t &n, int team_log2,
                                            int team_idx, int parity, TeamSmem &ts)
{
    const int team = 1 << team_log2;
    const int w = team < 32 ? team : 32;
    for (int o = w >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    }
    if (team > 32) {
        const int nw = team >> 5;
        const int slot0 = team_idx * nw;
        const int wit = (threadIdx.x >> 5) - slot0;
        if ((threadIdx.x & 31) == 0) {
            ts.ra[parity][slot0 + wit] = a;
            ts.rb[parity][slot0 + wit] = b;
            ts.rn[parity][slot0 + wit] = n;
        }
        named_sync(1 + team_idx, team);
        a = 0;
        b = 0;
        n = 0;
        for (int j = 0; j < nw; ++j) {
            a += ts.ra[parity][slot0 + j];
            b += ts.rb[parity][slot0 + j];
            n += ts.rn[parity][slot0 + j];
        }
    }
}

// Sum (q, cnt, e) over the team's threads; every thread of the team gets the
// totals.  Teams of up to 32 threads stay inside a warp; larger teams go
// through double-buffered shared slots and one named barrier per frame.
__device__ __forceinline__ void team_sum(int64_t &q, int32_t &cnt, int64_t &e, int team_log2,
                                        int team_idx, int parity, TeamSmem &ts, bool with_e)
{
    const int team = 1 << team_log2;
    const int w = team < 32 ? team : 32;
    for (int o = w >> 1; o > 0; o >>= 1) {
        q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        if (with_e)
            e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    }
    if (team > 32) {
        const int nw = team >> 5;
        const int slot0 = team_idx * nw;
        const int wit = (threadIdx.x >> 5) - slot0;
        if ((threadIdx.x & 31) == 0) {
            ts.q[parity][slot0 + wit] = q;
            ts.cnt[parity][slot0 + wit] = cnt;
            if (with_e)
                ts.e[parity][slot0 + wit] = e;
        }
        named_sync(1 + team_idx, team);
        q = 0;
        cnt = 0;
        e = 0;
        for (int j = 0; j < nw; ++j) {
            q += ts.q[parity][slot0 + j];
            cnt += ts.cnt[parity][slot0 + j];
            if (with_e)
                e += ts.e[parity][slot0 + j];
        }
    }
}

__device__ __forceinline__ int64_t bucket_of(uint32_t P, int32_t M)
{
    uint64_t b = ((uint64_t)P * (uint64_t)kOffsetBuckets) /
                 ((uint64_t)(1u << kStateShift) * (uint64_t)M * 128ull);
    return b < (uint64_t)(kOffsetBuckets - 1) ? (int64_t)b : (int64_t)(kOffsetBuckets - 1);
}

// Per-frame epilogue: terms, team sum, outputs (leader), served state.
template <bool SERVED>
__device__ __forceinline__ void frame_epilogue(const Item &it, int64_t frame, bool fvalid,
                                               int col0, int lit, int team_idx, int parity,
                                               int32_t (&s1)[kVec], int32_t (&s2)[kVec],
                                               TeamSmem &ts)
{
    const bool mine = fvalid && col0 < it.N;
    const bool stateful = SERVED && it.state != nullptr;
    int64_t q = 0, e = 0, ra = 0, rb = 0;
    int32_t rn = 0;
    int32_t cnt = 0;
    uint32_t P[kVec];
    if (mine) {
#pragma unroll
        for (int k = 0; k < kVec; ++k) {
            if (col0 + k < it.N) {
                float r = 0.0f;
                int64_t qi = 0;
                const bool has = SK_EPILOGUE_ALU ? input_term_alu(s1[k], s2[k], it.M, r, qi)
                                                 : input_term(s1[k], s2[k], it.M, r, qi);
                if (has) {
                    q += qi;
                    cnt += 1;
                }
                if (it.sk_in && SK_DBG_OUT_IN(it, frame, col0 + k)) {
                    // single-receiver estimate SK^_i = (M+1)/(M-1) r_i and its own
                    // flag against the one-input thresholds (Sec. 2.2.3, independent
                    // estimates)
                    const int64_t o = frame * it.N + col0 + k;
                    it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1]) : __int_as_float(0x7FC00000);
                    if (it.mask_in)
                        it.mask_in[o] = has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                }
            }
        }
        if (it.s1 && SK_DBG_OUT_IN(it, frame, col0)) {
            int32_t *o1 = it.s1 + frame * it.N + col0;
            int32_t *o2 = it.s2 + frame * it.N + col0;
#pragma unroll
            for (int k = 0; k < kVec; ++k)
                if (col0 + k < it.N) {
                    o1[k] = s1[k];
                    o2[k] = s2[k];
                }
        }
        if (stateful) {
            const int64_t sc = (int64_t)(1 << kStateShift) * it.M;
#pragma unroll
            for (int k = 0; k < kVec; ++k) {
                P[k] = 0;
                if (col0 + k < it.N) {
                    uint32_t pk = it.state_init ? ((uint32_t)s1[k] << kStateShift)
                                                : it.state[col0 + k];
                    P[k] = pk;
                    if (s1[k] > 0)
                        e += it.e_tab[bucket_of(pk, it.M)];
                    if (it.running_mu && s1[k] > 0 && pk > 0) {
                        // a = S1 / mu, b = S2 / mu^2 with mu = P / (2^k M): exact
                        // integer numerators and denominators, one fp32 divide each
                        const float fa = __fdiv_rn(__ll2float_rn((int64_t)s1[k] * sc),
                                                   __ll2float_rn((int64_t)pk));
                        const float fb =
                            __fdiv_rn(__ll2float_rn((int64_t)s2[k] * sc * sc),
                                      __ll2float_rn((int64_t)pk * (int64_t)pk));
                        ra += __float2ll_rn(__fmul_rn(fa, 16777216.0f));
                        rb += __float2ll_rn(__fmul_rn(fb, 16777216.0f));
                        rn += 1;
                    }
                }
            }
        }
    }
    team_sum(q, cnt, e, it.team_log2, team_idx, parity, ts, SERVED);
    if (SERVED)
        team_sum_rmu(ra, rb, rn, it.team_log2, team_idx, parity, ts);
    uint8_t m = 1;
    float sk_rmu = __int_as_float(0x7FC00000);
    if (SERVED && it.running_mu && stateful) {
        // Eq. (avgSK) first line over n' = M N_eff samples, rescaled by Eq. (final)
        // first line; flagged against the symmetric interval around 1 + delta
        if (rn > 0 && ra > 0) {
            const double mp = (double)((int64_t)it.M * rn);
            const double af = __dmul_rn(__ll2double_rn(ra), 0x1p-24);
            const double bf = __dmul_rn(__ll2double_rn(rb), 0x1p-24);
            const double t1 = __ddiv_rn(__dadd_rn(mp, 1.0), __dsub_rn(mp, 1.0));
            const double t2 = __dsub_rn(__ddiv_rn(__dmul_rn(mp, bf), __dmul_rn(af, af)), 1.0);
            const double skh = __dmul_rn(t1, t2);
            const double sc2 = __ddiv_rn(__dmul_rn(__dsub_rn(mp, 1.0), (double)(it.M + 1)),
                                         __dmul_rn(__dadd_rn(mp, 1.0), (double)(it.M - 1)));
            const double skd = __dmul_rn(sc2, skh);
            const double cen = __dadd_rn(
                __dadd_rn(1.0, it.mean_offset),
                __ddiv_rn(__dmul_rn(__ll2double_rn(e), (double)(it.M + 1)),
                          __dmul_rn(__dmul_rn((double)(it.M - 1), (double)rn), 4294967296.0)));
            const double half = __ddiv_rn(__dmul_rn(it.n_sigma, 2.0), __dsqrt_rn(mp));
            m = (skd > __dadd_rn(cen, half) || skd < __dsub_rn(cen, half)) ? 1 : 0;
            sk_rmu = __double2float_rn(skd);
        }
    } else if (cnt > 0) {
        int64_t lo = it.t_lo[cnt] + (stateful ? e : 0);
        int64_t hi = it.t_hi[cnt] + (stateful ? e : 0);
        m = (q > hi || q < lo) ? 1 : 0;
    }
    if (fvalid && lit == 0 && SK_DBG_OUT(it, frame)) {
        if (it.sk) {
            float skv = __int_as_float(0x7FC00000);
            if (SERVED && it.running_mu && stateful)
                skv = sk_rmu;
            else if (cnt > 0)
                skv = __fmul_rn(__fmul_rn(__ll2float_rn(q), 0x1p-32f), it.c_tab[cnt]);
            it.sk[frame] = skv;
        }
        if (it.mask)
            it.mask[frame] = m;
        if (it.q)
            it.q[frame] = q;
        if (it.neff)
            it.neff[frame] = cnt;
    }
    if (stateful && mine) {
#pragma unroll
        for (int k = 0; k < kVec; ++k) {
            if (col0 + k < it.N) {
                uint32_t pk = P[k];
                if (!m)
                    pk = pk - (pk >> kStateShift) + (uint32_t)s1[k];
                if (!m || it.state_init)
                    it.state[col0 + k] = pk;
            }
        }
    }
}

}  // namespace sk
