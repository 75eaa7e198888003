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
constexpr int kImajorG = 8;                 // lanes per input on the input-major path

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
    int32_t fast;            // 1: time-major vector path, 2: input-major path, 0: general
    float *sk_in;            // per-input SK^_i [n_frames][N] (Eq. originalSK), or null
    uint8_t *mask_in;        // per-input flag at the N_eff = 1 thresholds, or null
    int32_t prefetch;        // 1: input in device memory, L2 bulk prefetch allowed
    int32_t running_mu;      // served: normalise by the running power in the state
    double n_sigma;          // running-mu decision (double domain)
    double mean_offset;
};

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

__device__ __forceinline__ void flush(uint32_t (&acc)[kVec], int32_t (&s1)[kVec],
                                      int32_t (&s2)[kVec])
{
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
        s1[k] += (int32_t)(acc[k] >> kPackShift);
        s2[k] += (int32_t)(acc[k] & kPackMask);
        acc[k] = 0u;
    }
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
    r = __fdiv_rn(u43_to_f32_rn(d), u43_to_f32_rn(den));
    qi = f32_to_i64_rn(__fmul_rn(r, 4294967296.0f));
    return true;
}

struct TeamSmem {
    long long q[2][kSlots];
    long long e[2][kSlots];
    long long ra[2][kSlots];
    long long rb[2][kSlots];
    int cnt[2][kSlots];
    int rn[2][kSlots];
};

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
                if (it.sk_in) {
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
        if (it.s1) {
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
    if (fvalid && lit == 0) {
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

// Fast path: time-major, N % 8 == 0, M % (R*S) == 0, 8-byte aligned rows.
// Every load stays inside rows 0..M-1 of a frame below f_end.  Rows stream
// through a ring of S register batches of R rows: batch g is loaded right after
// batch g-S has been consumed, so each load has S-1 batches of work to hide
// behind, and the first S batches of the team's next frame are in flight while
// the current frame's epilogue runs.  A thread whose frame or columns are out of
// range issues no loads and skips the accumulation.
// NC > 0 fixes the row stride N at compile time (row offsets become load
// immediates); NC = 0 reads it from the item.
// one = true: the team takes frame f_begin alone (f_end is f_begin + 1, or
// f_begin when it has nothing to do) -- teams of a CTA then work on different
// items; otherwise the CTA's teams stride through [f_begin, f_end).
template <int R, int S, bool SERVED, int NC, bool PF = true, int PD = 1>
__device__ __forceinline__ void run_fast(const Item &it, int64_t f_begin, int64_t f_end,
                                         uint32_t lb, TeamSmem &ts, int &parity,
                                         bool one = false)
{
    static_assert(R == 8 || R == 16, "rows per batch");
    static_assert((R * S) % kFlushRows == 0, "flush cadence");
    const int team_log2 = it.team_log2;
    const int T = kThreads >> team_log2;
    const int team_idx = threadIdx.x >> team_log2;
    const int lit = threadIdx.x & ((1 << team_log2) - 1);
    const int col0 = lit * kVec;
    const bool col_ok = col0 < it.N;
    const int64_t N = NC > 0 ? (int64_t)NC : (int64_t)it.N;
    const int64_t fbytes = (int64_t)it.M * N;
    const int nb = it.M / R;
    const int64_t fstride = one ? 1 : T;
    const int64_t kmax = one ? 1 : (f_end - f_begin + T - 1) / T;

    uint2 buf[S][R];
    int64_t frame = one ? f_begin : f_begin + team_idx;
    bool ok = col_ok && frame < f_end;
    const uint8_t *fp = it.in + frame * fbytes + col0;
    if (ok) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            if constexpr (NC > 0) {
                load_rows_imm<NC>(buf[j], fp + (int64_t)j * R * NC,
                                  std::make_integer_sequence<int, R>{});
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    buf[j][r] = ldg_stream(fp + (int64_t)(j * R + r) * N);
            }
        }
    }

    for (int64_t k = 0; k < kmax; ++k) {
        const bool fvalid = frame < f_end;
        const int64_t nframe = frame + fstride;
        const bool nok = col_ok && nframe < f_end;
        const uint8_t *nfp = it.in + nframe * fbytes + col0;
        uint32_t acc[kVec];
        int32_t s1[kVec], s2[kVec];
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            acc[j] = 0u;
            s1[j] = 0;
            s2[j] = 0;
        }
        for (int jb = 0; jb < nb; jb += S) {
            if (PF && it.prefetch && lit == 0) {
                // the S batches a later iteration will load, in this frame or,
                // past its end, in the team's next frame
                // PD iterations ahead: batches jb+(PD+1)S .. jb+(PD+2)S-1
                const uint8_t *pp = nullptr;
                const int ba = jb + (PD + 1) * S;
                if (ba < nb) {
                    if (ok)
                        pp = fp + (int64_t)ba * R * N;
                } else {
                    const int b0 = ba - nb;
                    if (nok && b0 + S <= nb)
                        pp = nfp + (int64_t)b0 * R * N - col0;
                }
                if (pp) {
                    const uint32_t total = (uint32_t)(S * R) * (uint32_t)N;
                    for (uint32_t o = 0; o < total; o += 32768u)
                        prefetch_l2(pp + o, total - o < 32768u ? total - o : 32768u);
                }
            }
            const bool same_frame = jb + S < nb;
            const uint8_t *pn = same_frame ? fp + (int64_t)(jb + S) * R * N : nfp;
            const bool lok = same_frame ? ok : nok;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                if (ok) {
#pragma unroll
                    for (int r = 0; r < R; r += 2)
                        accum_pair(buf[j][r], buf[j][r + 1], lb, acc);
                    if (((j + 1) * R) % kFlushRows == 0)
                        flush(acc, s1, s2);
                }
                if (lok) {
                    if constexpr (NC > 0) {
                        load_rows_imm<NC>(buf[j], pn + (int64_t)j * R * NC,
                                          std::make_integer_sequence<int, R>{});
                    } else {
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            buf[j][r] = ldg_stream(pn + (int64_t)(j * R + r) * N);
                    }
                }
            }
        }
        frame_epilogue<SERVED>(it, frame, fvalid, col0, lit, team_idx, parity, s1, s2, ts);
        parity ^= 1;
        frame = nframe;
        fp = nfp;
        ok = nok;
    }
}

__device__ __forceinline__ uint4 ldg_stream16(const uint8_t *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// 16 samples of one input (one 16-byte chunk) into one packed accumulator.
__device__ __forceinline__ uint32_t accum16(uint4 w, uint32_t lb)
{
    uint32_t a = 0u;
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        a += lds_u32(prmt(ww[h], lb, 0x7604u)) + lds_u32(prmt(ww[h], lb, 0x7614u));
        a += lds_u32(prmt(ww[h], lb, 0x7624u)) + lds_u32(prmt(ww[h], lb, 0x7634u));
    }
    return a;
}

// Input-major fast path: layout [frame][input][t], M % (16 G) == 0, team of at
// least 32 threads.  A segment of G lanes owns one input at a time: lane j reads
// the 16-byte chunks j, j+G, j+2G, ... of that input's M bytes, so one warp
// instruction reads 32/G runs of 16 G contiguous bytes.  Each chunk (16 samples)
// fills one packed accumulator, which is split into exact S1, S2 at once.  After
// an input's last chunk the segment adds S1 and S2 over its G lanes with
// log2(G) shuffles and its lane 0 forms the input's term.  The lane's chunks of
// successive inputs, and of the team's next frame, form one flat sequence that
// streams through two register batches of KB chunks; a frame's sequence is padded
// to a multiple of KB so that frame ends fall on batch boundaries.
template <int G, int KB>
__device__ __forceinline__ void run_imajor(const Item &it, int64_t f_begin, int64_t f_end,
                                           uint32_t lb, TeamSmem &ts, int &parity)
{
    const int team_log2 = it.team_log2;
    const int T = kThreads >> team_log2;
    const int team_idx = threadIdx.x >> team_log2;
    const int lit = threadIdx.x & ((1 << team_log2) - 1);
    const int nseg = (1 << team_log2) / G;
    const int seg = lit / G, j = lit % G;
    const int N = it.N, M = it.M;
    const int C = M / (16 * G);                 // chunks per lane per input
    const int K = (N + nseg - 1) / nseg;        // inputs per segment
    const int per = ((K * C + KB - 1) / KB) * KB;  // padded flat chunks per frame
    const int nbat = per / KB;
    const int64_t fbytes = (int64_t)M * N;
    const int64_t kmax = (f_end - f_begin + T - 1) / T;

    // load cursor: frame, input slot k, chunk c, flat position g
    int64_t lf = f_begin + team_idx;
    int lk = 0, lc = 0, lg = 0;
    auto load_batch = [&](uint4 (&buf)[KB]) {
#pragma unroll
        for (int u = 0; u < KB; ++u) {
            const int i = seg + lk * nseg;
            if (lf < f_end && lk < K && i < N)
                buf[u] = ldg_stream16(it.in + lf * fbytes + (int64_t)i * M +
                                      (int64_t)(j + lc * G) * 16);
            if (++lc == C) {
                lc = 0;
                ++lk;
            }
        }
        // frame ends fall on batch boundaries (per is a multiple of KB)
        lg += KB;
        if (lg >= per) {
            lg = 0;
            lk = 0;
            lc = 0;
            lf += T;
        }
    };

    uint4 A[KB], B[KB];
    load_batch(A);
    int64_t frame = f_begin + team_idx;
    for (int64_t kk = 0; kk < kmax; ++kk) {
        const bool fvalid = frame < f_end;
        int64_t q = 0, e = 0;
        int32_t cnt = 0;
        int32_t s1 = 0, s2 = 0;
        int pk = 0, pc = 0;  // process cursor inside the frame
        for (int b = 0; b < nbat; b += 2) {
            const bool has_b = b + 1 < nbat;
            if (has_b)
                load_batch(B);
            // process A then B; the same code for both buffers
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && !has_b)
                    break;
                uint4 (&buf)[KB] = half == 0 ? A : B;
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    const int i = seg + pk * nseg;
                    const bool live = fvalid && pk < K && i < N;
                    if (live) {
                        const uint32_t a = accum16(buf[u], lb);
                        s1 += (int32_t)(a >> kPackShift);
                        s2 += (int32_t)(a & kPackMask);
                    }
                    if (++pc == C) {
                        // input done: combine the segment's lanes (all lanes of a
                        // warp reach this point together)
                        pc = 0;
#pragma unroll
                        for (int o = 1; o < G; o <<= 1) {
                            s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
                            s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
                        }
                        if (live && j == 0) {
                            float r = 0.0f;
                            int64_t qi = 0;
                            const bool has = input_term(s1, s2, M, r, qi);
                            if (has) {
                                q += qi;
                                cnt += 1;
                            }
                            const int64_t o = frame * N + i;
                            if (it.s1) {
                                it.s1[o] = s1;
                                it.s2[o] = s2;
                            }
                            if (it.sk_in) {
                                it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1])
                                                  : __int_as_float(0x7FC00000);
                                if (it.mask_in)
                                    it.mask_in[o] =
                                        has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                            }
                        }
                        s1 = 0;
                        s2 = 0;
                        ++pk;
                    }
                }
                if (half == 0)
                    load_batch(A);
            }
        }
        team_sum(q, cnt, e, team_log2, team_idx, parity, ts, false);
        if (fvalid && lit == 0) {
            uint8_t m = 1;
            if (cnt > 0)
                m = (q > it.t_hi[cnt] || q < it.t_lo[cnt]) ? 1 : 0;
            if (it.sk) {
                float skv = __int_as_float(0x7FC00000);
                if (cnt > 0)
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
        parity ^= 1;
        frame += T;
    }
}

// 16-byte streaming load at base + OFF, OFF an immediate of the instruction.
template <int OFF>
__device__ __forceinline__ uint4 ldg_stream16_at(const uint8_t *base)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4+%5];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(base), "n"(OFF));
    return v;
}

// Batch nb of a group on the grouped input-major path: chunk t of the batch is
// the group's chunk g = nb KB + t, i.e. chunk g % CH of input g / CH; all offsets
// are load immediates.
template <int M, int G, int CH, int KB, int nb, int... Ts>
__device__ __forceinline__ void load_group_imm(uint4 *buf, const uint8_t *base,
                                               std::integer_sequence<int, Ts...>)
{
    ((buf[Ts] = ldg_stream16_at<((nb * KB + Ts) / CH) * M + ((nb * KB + Ts) % CH) * G * 16>(
          base)),
     ...);
}

template <int M, int G, int CH, int KB, int nb>
__device__ __forceinline__ void load_group_batch(uint4 (&buf)[KB], const uint8_t *base, int live)
{
    if (live == G) {
        load_group_imm<M, G, CH, KB, nb>(buf, base, std::make_integer_sequence<int, KB>{});
    } else {
#pragma unroll
        for (int t = 0; t < KB; ++t) {
            const int g = nb * KB + t;
            buf[t] = g / CH < live ? ldg_stream16(base + (g / CH) * M + (g % CH) * G * 16)
                                   : make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// Batches nb .. NB-1 of a group: load the following batch into nxt (the group's
// next one, or batch 0 of the next group), then add cur into the sums.
template <int M, int G, int CH, int NB, int KB, int nb>
__device__ __forceinline__ void group_batches(uint4 (&cur)[KB], uint4 (&nxt)[KB],
                                              const uint8_t *cur_base, int cur_live,
                                              const uint8_t *nxt_base, int nxt_live,
                                              uint32_t lb, int32_t (&s1)[G], int32_t (&s2)[G])
{
    if constexpr (nb < NB) {
        if constexpr (nb + 1 < NB)
            load_group_batch<M, G, CH, KB, nb + 1>(nxt, cur_base, cur_live);
        else
            load_group_batch<M, G, CH, KB, 0>(nxt, nxt_base, nxt_live);
#pragma unroll
        for (int t = 0; t < KB; ++t) {
            const uint32_t a = accum16(cur[t], lb);
            s1[(nb * KB + t) / CH] += (int32_t)(a >> kPackShift);
            s2[(nb * KB + t) / CH] += (int32_t)(a & kPackMask);
        }
        group_batches<M, G, CH, NB, KB, nb + 1>(nxt, cur, cur_base, cur_live, nxt_base, nxt_live,
                                                lb, s1, s2);
    }
}

// Input-major path with grouped inputs: layout [frame][input][t] with
// M = 16 G CH.  A segment of G lanes owns a group of G consecutive inputs; lane
// j reads the 16-byte chunks j, j+G, ..., j+(CH-1)G of each of them (one warp
// instruction reads 32/G whole 128-byte lines when G = 8), every offset inside
// the group a load immediate.  Each lane keeps S1, S2 for all G inputs of the
// group; a reduce-scatter over the segment's lanes (G-1 shuffle pairs) leaves
// input u's totals in lane u, so all lanes form an input term at once.  The
// segment's groups are (k nseg + seg) G .. + G-1 for k = 0, 1, ...; a frame is
// NG = ceil(N / team) groups per segment (team = threads per frame, which the
// plan sets to about one per 2 KB of frame).  Inputs longer than 512 samples are
// read as SPLIT sub-inputs of 512 (measured: the 512-sample shape streams at
// 6.2 TB/s, the 1024-sample one at 4.4).  The group streams through two
// register batches of KB chunks (NB batches per group, NB even, so every group
// starts in batch A); with PF the next group's bytes are requested into L2 while
// this one is read.
template <int G, int CH, bool PF, int SPLIT = 1>
__device__ __forceinline__ void run_imajor_grouped(const Item &it, int64_t f_begin,
                                                   int64_t f_end, uint32_t lb, TeamSmem &ts,
                                                   int &parity)
{
    // SPLIT > 1: each input is read as SPLIT consecutive sub-inputs of M / SPLIT
    // bytes (the layout is the same bytes), whose sums are added after the
    // reduce-scatter; M here is the sub-input length
    static_assert(SPLIT >= 1 && G % SPLIT == 0, "sub-inputs of one input share a group");
    constexpr int M = 16 * G * CH;
    constexpr int NB = (G * CH / 8) < 2 ? 2 : G * CH / 8;  // batches per group
    constexpr int KB = G * CH / NB;                       // chunks per batch
    static_assert(KB * NB == G * CH && NB % 2 == 0, "batch shape");
    const int team_log2 = it.team_log2;
    const int team = 1 << team_log2;
    const int T = kThreads >> team_log2;
    const int team_idx = threadIdx.x >> team_log2;
    const int lit = threadIdx.x & (team - 1);
    const int nseg = team / G;
    const int seg = lit / G, j = lit % G;
    const int N = it.N;
    const int NS = N * SPLIT;  // sub-inputs per frame
    const int NG = (NS + team - 1) / team;
    const int64_t fbytes = (int64_t)M * NS;
    const int64_t kmax = (f_end - f_begin + T - 1) / T;

    // sub-inputs of group (frame f, k) that this segment may read: 0..G
    auto live_of = [&](int64_t f, int k) -> int {
        const int i0 = (k * nseg + seg) * G;
        const int r = NS - i0;
        return (f < f_end) ? (r < 0 ? 0 : (r > G ? G : r)) : 0;
    };
    auto base_of = [&](int64_t f, int k) -> const uint8_t * {
        return it.in + f * fbytes + (int64_t)((k * nseg + seg) * G) * M + j * 16;
    };
    uint4 A[KB], B[KB];
    int64_t frame = f_begin + team_idx;
    const uint8_t *cur_base = base_of(frame, 0);
    int cur_live = live_of(frame, 0);
    load_group_batch<M, G, CH, KB, 0>(A, cur_base, cur_live);
    for (int64_t kk = 0; kk < kmax; ++kk) {
        const bool fvalid = frame < f_end;
        int64_t q = 0, e = 0;
        int32_t cnt = 0;
        for (int k = 0; k < NG; ++k) {
            // the group after this one: next k, else the team's next frame
            const int64_t nf = (k + 1 < NG) ? frame : frame + T;
            const int nk = (k + 1 < NG) ? k + 1 : 0;
            const uint8_t *nxt_base = base_of(nf, nk);
            const int nxt_live = live_of(nf, nk);
            if (PF && nxt_live > 0 && j == 0)
                prefetch_l2(nxt_base, (uint32_t)(nxt_live * M));
            int32_t s1[G], s2[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                s1[u] = 0;
                s2[u] = 0;
            }
            group_batches<M, G, CH, NB, KB, 0>(A, B, cur_base, cur_live, nxt_base, nxt_live, lb,
                                               s1, s2);
            // reduce-scatter: lane j ends with input j's sums in s1[0], s2[0]
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) {
                const bool up = (j & o) != 0;
#pragma unroll
                for (int t = 0; t < o; ++t) {
                    const int32_t send1 = up ? s1[t] : s1[t + o];
                    const int32_t send2 = up ? s2[t] : s2[t + o];
                    const int32_t keep1 = up ? s1[t + o] : s1[t];
                    const int32_t keep2 = up ? s2[t + o] : s2[t];
                    s1[t] = keep1 + __shfl_xor_sync(0xFFFFFFFFu, send1, o);
                    s2[t] = keep2 + __shfl_xor_sync(0xFFFFFFFFu, send2, o);
                }
            }
            // an input's sub-inputs sit in lanes j .. j + SPLIT - 1 (j % SPLIT == 0)
#pragma unroll
            for (int o = 1; o < SPLIT; o <<= 1) {
                s1[0] += __shfl_xor_sync(0xFFFFFFFFu, s1[0], o);
                s2[0] += __shfl_xor_sync(0xFFFFFFFFu, s2[0], o);
            }
            if (j < cur_live && j % SPLIT == 0) {
                const int i = ((k * nseg + seg) * G + j) / SPLIT;
                float r = 0.0f;
                int64_t qi = 0;
                const bool has = SK_EPILOGUE_ALU
                                     ? input_term_alu(s1[0], s2[0], M * SPLIT, r, qi)
                                     : input_term(s1[0], s2[0], M * SPLIT, r, qi);
                if (has) {
                    q += qi;
                    cnt += 1;
                }
                const int64_t o = frame * N + i;
                if (it.s1) {
                    it.s1[o] = s1[0];
                    it.s2[o] = s2[0];
                }
                if (it.sk_in) {
                    it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1]) : __int_as_float(0x7FC00000);
                    if (it.mask_in)
                        it.mask_in[o] =
                            has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                }
            }
            cur_base = nxt_base;
            cur_live = nxt_live;
        }
        team_sum(q, cnt, e, team_log2, team_idx, parity, ts, false);
        if (fvalid && lit == 0) {
            uint8_t m = 1;
            if (cnt > 0)
                m = (q > it.t_hi[cnt] || q < it.t_lo[cnt]) ? 1 : 0;
            if (it.sk) {
                float skv = __int_as_float(0x7FC00000);
                if (cnt > 0)
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
        parity ^= 1;
        frame += T;
    }
}

// General path: any N (<= 4096), any M >= 2, either layout; the same table,
// terms and epilogue.  With ALIGNED, time-major rows go through aligned 8-byte
// loads and a shift; otherwise (and for input-major) through byte loads with
// bounds checks.  Serves the sizes the fast paths do not take.  Served and
// input-major kernels leave ALIGNED off: its registers would spill in them.
template <bool SERVED, bool ALIGNED = !SERVED>
__device__ __forceinline__ void run_general(const Item &it, int64_t f_begin, int64_t f_end,
                                            uint32_t lb, TeamSmem &ts, int &parity,
                                            bool one = false)
{
    const int team_log2 = it.team_log2;
    const int T = kThreads >> team_log2;
    const int team_idx = threadIdx.x >> team_log2;
    const int lit = threadIdx.x & ((1 << team_log2) - 1);
    const int col0 = lit * kVec;
    const int64_t N = it.N;
    const int M = it.M;
    const int64_t fbytes = (int64_t)M * N;
    const int64_t fstride = one ? 1 : T;
    const int64_t kmax = one ? 1 : (f_end - f_begin + T - 1) / T;
    int64_t frame = one ? f_begin : f_begin + team_idx;
    for (int64_t k = 0; k < kmax; ++k) {
        const bool fvalid = frame < f_end;
        uint32_t acc[kVec];
        int32_t s1[kVec], s2[kVec];
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            acc[j] = 0u;
            s1[j] = 0;
            s2[j] = 0;
        }
        if (ALIGNED && fvalid && col0 < N && it.layout == 0) {
            // time-major, any N: the thread's 8 bytes of row t start at an address
            // with the same offset d modulo 8 for every lane (col0 is a multiple of
            // 8), so two aligned 8-byte loads and a shift give them; bytes past
            // column N become 0x88 (no power).  A row whose 16-byte window would
            // leave the item's bytes falls back to byte loads.
            const uint8_t *fb = it.in + frame * fbytes;
            const uint8_t *lo_lim = it.in;
            const uint8_t *hi_lim = it.in + it.n_frames * fbytes;
            const int keep = (int)(N - col0 < kVec ? N - col0 : kVec);  // bytes of ours
            const uint64_t kmask = keep == kVec ? ~0ull : ((1ull << (8 * keep)) - 1ull);
            const uint64_t fill = 0x8888888888888888ull & ~kmask;
            constexpr int RB = 4;  // rows per load batch
            for (int t0 = 0; t0 < M; t0 += RB) {
                uint64_t lo[RB], hi[RB];
                int sh[RB];
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    lo[r] = hi[r] = 0x8888888888888888ull;
                    sh[r] = 0;
                    const int t = t0 + r;
                    if (t < M) {
                        const uint8_t *a = fb + (int64_t)t * N + col0;
                        const int d = (int)((uintptr_t)a & 7u);
                        const uint8_t *w = a - d;
                        sh[r] = d;
                        if (w >= lo_lim && w + 16 <= hi_lim) {
                            lo[r] = __ldg((const unsigned long long *)w);
                            hi[r] = __ldg((const unsigned long long *)(w + 8));
                        } else {
                            uint64_t v = 0;
                            for (int j = 0; j < keep; ++j)
                                v |= (uint64_t)a[j] << (8 * j);
                            lo[r] = v;  // already aligned to the thread's columns
                            sh[r] = -1;
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int t = t0 + r;
                    if (t >= M)
                        break;
                    uint64_t v = lo[r];
                    if (sh[r] > 0)
                        v = (lo[r] >> (8 * sh[r])) | (hi[r] << (64 - 8 * sh[r]));
                    v = (v & kmask) | fill;
                    accum_row(make_uint2((uint32_t)v, (uint32_t)(v >> 32)), lb, acc);
                    if ((t & (kFlushRows - 1)) == kFlushRows - 1)
                        flush(acc, s1, s2);
                }
            }
            flush(acc, s1, s2);
        } else if (fvalid && col0 < N) {
            const uint8_t *fb = it.in + frame * fbytes;
            for (int t = 0; t < M; ++t) {
                uint32_t w0 = 0x88888888u, w1 = 0x88888888u;
#pragma unroll
                for (int j = 0; j < kVec; ++j) {
                    const int64_t c = col0 + j;
                    if (c < N) {
                        uint32_t b = it.layout == 0 ? fb[(int64_t)t * N + c] : fb[c * M + t];
                        const uint32_t sh = 8u * (uint32_t)(j & 3);
                        if (j < 4)
                            w0 = (w0 & ~(0xFFu << sh)) | (b << sh);
                        else
                            w1 = (w1 & ~(0xFFu << sh)) | (b << sh);
                    }
                }
                accum_row(make_uint2(w0, w1), lb, acc);
                if ((t & (kFlushRows - 1)) == kFlushRows - 1)
                    flush(acc, s1, s2);
            }
            flush(acc, s1, s2);
        }
        frame_epilogue<SERVED>(it, frame, fvalid, col0, lit, team_idx, parity, s1, s2, ts);
        parity ^= 1;
        frame += fstride;
    }
}

}  // namespace sk
