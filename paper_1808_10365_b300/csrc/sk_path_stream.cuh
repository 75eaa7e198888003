// Stream path of the fused kernel: time-major frames of few inputs (small N, any
// M), each frame read as one flat run of bytes in aligned 16-byte chunks.
//
// A time-major frame is M rows of N bytes, fbytes = M N contiguous bytes, and
// byte o of the frame belongs to input o mod N.  A unit of s lanes reads the
// frame's 16-byte chunks round robin: lane u takes chunks u, u + s, u + 2s, ...
// With d the frame's offset from a 16-byte boundary, byte j of lane u's chunk of
// pass p is frame byte 16 (u + s p) + j - d.  When 16 s is a multiple of N that
// byte belongs to input (16 u + j - d) mod N in every pass: each lane keeps one
// packed accumulator per byte position of its chunks for the whole frame, and
// the table path of the other read paths applies unchanged (PRMT + LDS + half an
// IADD3 a sample, one 16-byte load a chunk), whatever N and M are.  After the
// frame the unit's 16 s partial sums go to shared memory, and input i adds the
// R = 16 s / N of them that hold its samples: slots x + r N, r < R, with
// x = (i + d) mod N.  The sums are exact integers, so the order is free.
//
// A unit is either part of one warp (s <= 32: 32 / s units a warp, lanes past the
// last unit idle) or W = ceil(s / 32) warps (s > 32, one named barrier per frame
// step).  s is a multiple of N / gcd(N, 16), at least 8 so that a unit's pass
// reads at least 128 contiguous bytes, chosen on the host by a model of the
// instructions a frame costs.  The slots are written once per frame, lane u's 16
// values as four 16-byte pieces rotated by u / 2, so that each group of 8 lanes
// of a store covers all 32 banks; the units of one warp start 8 words apart
// (modulo 32).
#pragma once

#include "sk_device.cuh"

namespace sk {

// Launch shape of the stream path, chosen on the host (stream_shape).
struct StreamShape {
    int32_t s;         // lanes per frame, a multiple of N / gcd(N, 16)
    int32_t W;         // warps per unit: 1 (several units a warp) or ceil(s / 32)
    int32_t per_warp;  // units per warp when W == 1
    int32_t units;     // units (frames in flight) per CTA
};

constexpr int kStreamThreads = 512;             // 16 warps a CTA, one CTA per SM
constexpr int kStreamWarps = kStreamThreads / 32;
constexpr int kStreamBatch = 8;                  // passes per register batch (loads in flight)
constexpr int kStreamLead = 2 * kStreamBatch;    // L2 prefetch distance, in passes
// slots: 16 s x 8 B per unit, plus 8 words per unit (at most 64 units) of skew
constexpr int kStreamPartBytes = kStreamWarps * 32 * 16 * 8 + 64 * 32;
constexpr int kStreamSmem = kDynSmem + kStreamPartBytes;
constexpr uint32_t kNoPower = 0x88888888u;       // bytes that decode to 0 + 0i

// The 16 bytes at p (16-byte aligned) with every byte outside the frame [lo, hi)
// replaced by 0x88 (no power).  Only bytes of the frame are read, so the chunks
// that stick out of the frame (and of the input buffer, at its two ends) never
// touch memory outside it.
__device__ __forceinline__ uint4 load_clipped(const Item &it, const uint8_t *p, const uint8_t *lo,
                                              const uint8_t *hi)
{
    if (p >= lo && p + 16 <= hi)
        return SK_DBG_IN(it, p, 16) ? ldg_stream16(p) : make_uint4(kNoPower, kNoPower, kNoPower,
                                                                   kNoPower);
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t x = kNoPower;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint8_t *q = p + 4 * k + b;
            if (q >= lo && q < hi && SK_DBG_IN(it, q, 1))
                x = (x & ~(0xFFu << (8 * b))) | ((uint32_t)__ldg(q) << (8 * b));
        }
        w[k] = x;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// One chunk of one lane into its 16 packed accumulators (byte j of the chunk
// into accumulator j).
__device__ __forceinline__ void accum_chunk(uint4 a, uint32_t lb, uint32_t (&acc)[16])
{
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc[4 * k + j] += lds_u32(prmt(wa[k], lb, 0x7604u | ((uint32_t)j << 4)));
}

// Two chunks of one lane (same byte positions, two passes): one three-input add
// per position.
__device__ __forceinline__ void accum_chunk_pair(uint4 a, uint4 b, uint32_t lb,
                                                 uint32_t (&acc)[16])
{
    const uint32_t wa[4] = {a.x, a.y, a.z, a.w};
    const uint32_t wb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t sel = 0x7604u | ((uint32_t)j << 4);  // byte j of the data word
            acc[4 * k + j] += lds_u32(prmt(wa[k], lb, sel)) + lds_u32(prmt(wb[k], lb, sel));
        }
}

// Packed accumulators (at most 16 samples each) into the exact sums: S1 takes the
// high field, s2 the whole word, so that s2 holds S2 + 2^19 S1 modulo 2^32 until
// the frame ends (as in flush()).
__device__ __forceinline__ void flush16(uint32_t (&acc)[16], int32_t (&s1)[16],
                                        int32_t (&s2)[16])
{
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        s1[j] += (int32_t)(acc[j] >> kPackShift);
        s2[j] = (int32_t)((uint32_t)s2[j] + acc[j]);
        acc[j] = 0u;
    }
}

// Word of slot x (lane x / 16, position x % 16) in a unit's slot array: lane u's
// piece q (positions 4q .. 4q + 3) sits at piece (q + u / 2) mod 4 of its 16 words.
__device__ __forceinline__ int slot_word(int x)
{
    const int u = x >> 4, q = (x >> 2) & 3;
    return (u << 4) | ((((q + (u >> 1)) & 3)) << 2) | (x & 3);
}

// L2 prefetch of passes [q, q + n) of a unit whose frame starts at fa, limited to
// the frame's own 16-byte blocks (a hint: results never depend on it).
__device__ __forceinline__ void prefetch_passes(const uint8_t *fa, int32_t fbytes, int32_t pbytes,
                                                int32_t q, int32_t n)
{
    const uintptr_t a0 = (uintptr_t)fa & ~(uintptr_t)15u;
    uintptr_t b = a0 + (uintptr_t)q * (uintptr_t)pbytes;
    uintptr_t e = b + (uintptr_t)n * (uintptr_t)pbytes;
    const uintptr_t lo = ((uintptr_t)fa + 15u) & ~(uintptr_t)15u;
    const uintptr_t hi = ((uintptr_t)fa + (uintptr_t)fbytes) & ~(uintptr_t)15u;
    b = b < lo ? lo : b;
    e = e > hi ? hi : e;
    if (e > b)
        prefetch_l2((const uint8_t *)b, (uint32_t)(e - b));
}

// Passes [q, q + kStreamBatch) of the unit's run of frames (this frame, P passes,
// then its next one, nfa, or none) into L2, kStreamLead passes ahead of the reads.
__device__ __forceinline__ void prefetch_ahead(const uint8_t *fa, const uint8_t *nfa, int32_t P,
                                               int32_t fbytes, int32_t pbytes, int32_t q)
{
    if (q < P)
        prefetch_passes(fa, fbytes, pbytes, q, kStreamBatch);
    if (nfa && q + kStreamBatch > P)
        prefetch_passes(nfa, fbytes, pbytes, q > P ? q - P : 0,
                        q > P ? kStreamBatch : q + kStreamBatch - P);
}

// Frames [f_begin, f_end) of the item on the stream path (kStreamThreads threads).
// part: the CTA's slot area (kStreamPartBytes of shared memory, 16-byte aligned);
// red_q, red_c: one entry per warp.
__device__ __forceinline__ void run_stream(const Item &it, const StreamShape &sh, int64_t f_begin,
                                           int64_t f_end, uint32_t lb, int32_t *part,
                                           long long *red_q, int *red_c)
{
    const int s = sh.s;
    const int N = it.N;
    const int M = it.M;
    const int32_t fbytes = M * N;  // <= 2^24 (M, N <= 4096): frame offsets fit 32 bits
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int unit, u, tsz;
    bool active, in_unit;
    if (sh.W == 1) {
        const int sub = lane / s;
        u = lane - sub * s;
        unit = warp * sh.per_warp + sub;
        in_unit = sub < sh.per_warp;
        active = in_unit;
        tsz = s;
    } else {
        const int team = warp / sh.W;
        u = (int)threadIdx.x - team * 32 * sh.W;
        unit = team;
        in_unit = team < sh.units;
        active = in_unit && u < s;
        tsz = 32 * sh.W;
        if (!in_unit)
            return;  // whole warps past the last team: no barrier of theirs is waited on
    }
    // the unit's S1 slots (16 s words) and S2 slots; with several units a warp each
    // unit's area is 8 words longer, so that neighbours start 8 words apart modulo 32
    // and their combine reads fall in different banks
    int32_t *const ps1 = part + unit * (32 * s + (sh.W == 1 ? 8 : 0));
    int32_t *const ps2 = ps1 + 16 * s;
    const int R = (16 * s) / N;
    const int64_t nunits = sh.units;
    const int64_t rounds = (f_end - f_begin + nunits - 1) / nunits;
    // A pass of the unit reads pbytes = 16 s bytes.  With the frame d bytes past a
    // 16-byte boundary its chunks cover span = fbytes + d bytes: passes p < Pe hold
    // whole chunks of the frame in every lane (but for lane 0's chunk of pass 0 when
    // d > 0), and at most one more pass, P = Pe or Pe + 1, ends past the frame.
    const int32_t pbytes = 16 * s;
    const int32_t pe0 = fbytes / pbytes;             // Pe at d = 0
    const int32_t rem0 = fbytes - pe0 * pbytes;
    // The next frame's first batch of chunks, loaded before this frame's combine so
    // that its loads are in flight while the combine runs (pre: v holds it).
    uint4 v[kStreamBatch];
    bool pre = false;
    for (int64_t k = 0; k < rounds; ++k) {
        const int64_t frame = f_begin + k * nunits + unit;
        const bool fvalid = in_unit && frame < f_end;
        const bool rd = active && fvalid;
        const uint8_t *fa = it.in + (fvalid ? frame : f_begin) * (int64_t)fbytes;
        const int d = (int)((uintptr_t)fa & 15u);
        const uint8_t *lp = fa - d + 16 * u;  // the lane's chunk of pass 0
        const int32_t span = fbytes + d;
        const int32_t nch = (span + 15) >> 4;  // chunks covering the frame
        const int32_t Pe = pe0 + (rem0 + d >= pbytes ? 1 : 0);
        const int32_t P = Pe + ((span - Pe * pbytes) != 0 ? 1 : 0);
        // L2 prefetch kStreamLead passes ahead of the reads, by the unit's lane 0:
        // a bounded amount in flight (units x kStreamLead passes a CTA)
        const bool pf = it.prefetch && rd && u == 0;
        const uint8_t *nfa = frame + nunits < f_end ? fa + nunits * (int64_t)fbytes : nullptr;
        if (pf && k == 0)
            prefetch_ahead(fa, nfa, P, fbytes, pbytes, 0);
        if (pf && k == 0)
            prefetch_ahead(fa, nfa, P, fbytes, pbytes, kStreamBatch);
        uint32_t acc[16];
        int32_t s1[16], s2[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            acc[j] = 0u;
            s1[j] = 0;
            s2[j] = 0;
        }
        const uint4 none = make_uint4(kNoPower, kNoPower, kNoPower, kNoPower);
        int32_t p = 0;
        int held = 0;  // samples in each packed accumulator since the last flush
        if (d > 0) {
            // pass 0: lane 0's chunk starts d bytes before the frame
            accum_chunk(rd && u < nch ? load_clipped(it, lp, fa, fa + fbytes) : none, lb, acc);
            p = 1;
            held = 1;
        }
        for (; p + kStreamBatch <= Pe; p += kStreamBatch) {
            // whole chunks of the frame: no checks, kStreamBatch loads in flight
            if (pf)
                prefetch_ahead(fa, nfa, P, fbytes, pbytes, p + kStreamLead);
            if (!pre) {
#pragma unroll
                for (int r = 0; r < kStreamBatch; ++r) {
                    const uint8_t *q = lp + (p + r) * pbytes;
                    v[r] = (rd && SK_DBG_IN(it, q, 16)) ? ldg_stream16(q) : none;
                }
            }
            pre = false;
            if (held > 16 - kStreamBatch) {
                flush16(acc, s1, s2);
                held = 0;
            }
#pragma unroll
            for (int r = 0; r < kStreamBatch; r += 2)
                accum_chunk_pair(v[r], v[r + 1], lb, acc);
            held += kStreamBatch;
        }
        for (; p + 2 <= Pe; p += 2) {
            const uint8_t *q = lp + p * pbytes;
            const uint4 a = (rd && SK_DBG_IN(it, q, 16)) ? ldg_stream16(q) : none;
            const uint4 b = (rd && SK_DBG_IN(it, q + pbytes, 16)) ? ldg_stream16(q + pbytes) : none;
            if (held > 14) {
                flush16(acc, s1, s2);
                held = 0;
            }
            accum_chunk_pair(a, b, lb, acc);
            held += 2;
        }
        if (p < Pe) {
            const uint8_t *q = lp + p * pbytes;
            const uint4 a = (rd && SK_DBG_IN(it, q, 16)) ? ldg_stream16(q) : none;
            if (held > 15) {
                flush16(acc, s1, s2);
                held = 0;
            }
            accum_chunk(a, lb, acc);
            held += 1;
            ++p;
        }
        for (; p < P; ++p) {
            // the pass that ends past the frame (its chunks clipped to the frame)
            const int32_t c = u + s * p;
            const uint4 a = (rd && c < nch) ? load_clipped(it, lp + p * pbytes, fa, fa + fbytes)
                                            : none;
            if (held > 15) {
                flush16(acc, s1, s2);
                held = 0;
            }
            accum_chunk(a, lb, acc);
            held += 1;
        }
        flush16(acc, s1, s2);
        if (rd) {
            // the lane's 16 slots as four rotated 16-byte pieces
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int w = 16 * u + 4 * ((q + (u >> 1)) & 3);
                *reinterpret_cast<int4 *>(ps1 + w) =
                    make_int4(s1[4 * q], s1[4 * q + 1], s1[4 * q + 2], s1[4 * q + 3]);
                *reinterpret_cast<int4 *>(ps2 + w) =
                    make_int4(s2[4 * q], s2[4 * q + 1], s2[4 * q + 2], s2[4 * q + 3]);
            }
        }
        {
            // the next round's frame: when it starts on a 16-byte boundary with a whole
            // first batch, its first kStreamBatch passes are loaded now (the same loads
            // its batch loop would issue: same lane, addresses and predicate)
            const int64_t nf = frame + nunits;
            const bool nvalid = in_unit && nf < f_end;
            const uint8_t *na = it.in + (nvalid ? nf : f_begin) * (int64_t)fbytes;
            const int nd = (int)((uintptr_t)na & 15u);
            const int32_t npe = pe0 + (rem0 + nd >= pbytes ? 1 : 0);
            if (k + 1 < rounds && nd == 0 && npe >= kStreamBatch) {
                const bool nrd = active && nvalid;
                const uint8_t *nlp = na + 16 * u;
#pragma unroll
                for (int r = 0; r < kStreamBatch; ++r) {
                    const uint8_t *q = nlp + r * pbytes;
                    v[r] = (nrd && SK_DBG_IN(it, q, 16)) ? ldg_stream16(q) : none;
                }
                pre = true;
            }
        }
        if (sh.W == 1)
            __syncwarp();
        else
            named_sync(1 + unit, 32 * sh.W);
        // inputs of the frame over the unit's threads: the R slots of each, its term
        int64_t q = 0;
        int32_t cnt = 0;
        if (fvalid) {
            int dn = d;
            while (dn >= N)
                dn -= N;
            for (int i = u; i < N; i += tsz) {
                int x = i + dn;
                if (x >= N)
                    x -= N;
                int32_t a1 = 0;
                uint32_t a2 = 0;
                for (int r = 0; r < R; ++r, x += N) {
                    const int w = slot_word(x);
                    a1 += ps1[w];
                    a2 += (uint32_t)ps2[w];
                }
                // exact S2 from the slots' S2 + 2^19 S1 (0 <= S2 < 2^32)
                a2 -= (uint32_t)a1 << kPackShift;
                float rr = 0.0f;
                int64_t qi = 0;
                const bool has = SK_EPILOGUE_ALU ? input_term_alu(a1, (int32_t)a2, M, rr, qi)
                                                 : input_term(a1, (int32_t)a2, M, rr, qi);
                if (has) {
                    q += qi;
                    cnt += 1;
                }
                const int64_t o = frame * N + i;
                if (it.s1 && SK_DBG_OUT_IN(it, frame, i)) {
                    it.s1[o] = a1;
                    it.s2[o] = (int32_t)a2;
                }
                if (it.sk_in && SK_DBG_OUT_IN(it, frame, i)) {
                    // single-receiver estimate and its flag at the one-input thresholds
                    it.sk_in[o] = has ? __fmul_rn(rr, it.c_tab[1]) : __int_as_float(0x7FC00000);
                    if (it.mask_in)
                        it.mask_in[o] =
                            has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                }
            }
        }
        if (sh.W == 1) {
            // sum over the unit's s lanes: segmented shuffles, lane u = 0 ends with it
            for (int o = 1; o < s; o <<= 1) {
                const long long qo = __shfl_down_sync(0xFFFFFFFFu, (long long)q, o);
                const int co = __shfl_down_sync(0xFFFFFFFFu, cnt, o);
                if (u + o < s) {
                    q += qo;
                    cnt += co;
                }
            }
            if (fvalid && u == 0)
                write_frame(it, frame, q, cnt);
            __syncwarp();  // the slots are free for the next frame
        } else {
            for (int o = 16; o > 0; o >>= 1) {
                q += __shfl_xor_sync(0xFFFFFFFFu, (long long)q, o);
                cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
            }
            if (lane == 0) {
                red_q[warp] = q;
                red_c[warp] = cnt;
            }
            named_sync(1 + unit, 32 * sh.W);
            if (fvalid && u == 0) {
                int64_t tq = 0;
                int32_t tc = 0;
                for (int w = 0; w < sh.W; ++w) {
                    tq += red_q[unit * sh.W + w];
                    tc += red_c[unit * sh.W + w];
                }
                write_frame(it, frame, tq, tc);
            }
        }
    }
}


// ---------------------------------------------------------------------------
// Input-major frames of any M ([frame][input][t]: input i's M samples are the
// bytes [i M, i M + M) of its frame).  G lanes per input (8 for inputs of six or
// more chunks, 4 for three to five, else 2) read the aligned 16-byte chunks that
// cover it (lane g: chunks g, g + G, ...), so that one warp load reads 32 / G
// neighbouring inputs' bytes as one run.  Every chunk goes through
// a byte mask (two entries of small shared tables: the input's first chunk drops the
// bytes before it, its last the bytes after it, the others keep all 16), which
// replaces the neighbours' bytes by 0x88 (no power) without a branch.  A lane holds
// G inputs (i0 + (32 / G) r + j, r < G, j = lane / G); after the chunks a
// reduce-scatter over the G lanes of an input group leaves each lane with the
// totals of one input, and all 32 lanes form a term.  A team of W warps takes a
// frame (warp w: input blocks of 32 at w, w + W, ...) and combines Q and N_eff
// through shared memory and one named barrier when W > 1.
// ---------------------------------------------------------------------------

// Byte mask of the bytes [kl, kh) of word w of a 16-byte chunk (0 <= kl <= kh <= 16).
__device__ __forceinline__ uint32_t chunk_word_mask(int kl, int kh, int w)
{
    const int a = max(kl - 4 * w, 0);
    const int b = min(kh - 4 * w, 4);
    if (b <= a)
        return 0u;
    const uint32_t hi = b >= 4 ? 0xFFFFFFFFu : ((1u << (8 * b)) - 1u);
    return hi & ~((1u << (8 * a)) - 1u);
}

// Mask tables: head[k] keeps bytes k..15, tail[k] keeps bytes 0..k-1 (k = 0..16).
struct ChunkMasks {
    uint4 head[17];
    uint4 tail[17];
};

__device__ __forceinline__ void init_chunk_masks(ChunkMasks &cm)
{
    for (int k = threadIdx.x; k < 17; k += blockDim.x) {
        cm.head[k] = make_uint4(chunk_word_mask(k, 16, 0), chunk_word_mask(k, 16, 1),
                                chunk_word_mask(k, 16, 2), chunk_word_mask(k, 16, 3));
        cm.tail[k] = make_uint4(chunk_word_mask(0, k, 0), chunk_word_mask(0, k, 1),
                                chunk_word_mask(0, k, 2), chunk_word_mask(0, k, 3));
    }
}

// One chunk of one input into its exact sums: the 16 samples through the table into
// a packed accumulator, then split (S1 the high field, s2 the packed word: S2 +
// 2^19 S1 modulo 2^32 until finished).
__device__ __forceinline__ void imc_add(uint4 a, uint32_t lb, int32_t &s1, int32_t &s2)
{
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
    uint32_t acc = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        acc += lds_u32(prmt(w[k], lb, 0x7604u)) + lds_u32(prmt(w[k], lb, 0x7614u)) +
               lds_u32(prmt(w[k], lb, 0x7624u)) + lds_u32(prmt(w[k], lb, 0x7634u));
    s1 += (int32_t)(acc >> kPackShift);
    s2 = (int32_t)((uint32_t)s2 + acc);
}

// load_clipped kept out of line: only a chunk past the end of the item's bytes takes
// it (the last input of the last frame), and inlined it would cost the loop registers.
static __device__ __noinline__ uint4 load_clipped_tail(const Item &it, const uint8_t *p,
                                                const uint8_t *lo, const uint8_t *hi)
{
    return load_clipped(it, p, lo, hi);
}

__device__ __forceinline__ uint32_t keep_bytes(uint32_t v, uint32_t m)
{
    return (v & m) | (kNoPower & ~m);
}

// Warps per frame of the input-major chunk path: about four blocks of 32 inputs a
// warp, a power of two from 1 to 16.
__host__ __device__ __forceinline__ int imajor_chunk_team(int N)
{
    const int blocks = (N + 31) / 32;
    int W = 1;
    while (W < 16 && blocks >= 8 * W)
        W *= 2;
    return W;
}

// Lanes per input of the chunk path by the chunks an input spans (A/B on B300, 3 GB
// launches: M = 48, 4 chunks: 2 lanes 0.28, 8 lanes 0.19, 4 lanes 0.31; M = 100, 8
// chunks: 2 lanes 0.27-0.32, 8 lanes 0.32-0.34).
__host__ __device__ __forceinline__ int imajor_chunk_lanes(int M)
{
    const int cmax = (M + 30) >> 4;
    return cmax >= 6 ? 8 : (cmax >= 3 ? 4 : 2);
}

// Frames [f_begin, f_end) of an input-major item, G lanes per input (2, 4 or 8) and G
// inputs a lane, teams of W warps per frame.  red_q, red_c: one entry per warp.
template <int G>
__device__ __forceinline__ void run_imajor_chunks(const Item &it, int W, int64_t f_begin,
                                                  int64_t f_end, uint32_t lb,
                                                  const ChunkMasks &cm, long long *red_q,
                                                  int *red_c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int team = warp / W, wt = warp - team * W;
    const int teams = (int)(blockDim.x >> 5) / W;
    if (team >= teams)
        return;  // whole warps past the last team
    static_assert(G == 2 || G == 4 || G == 8, "lanes per input");
    constexpr int IPW = 32 / G;  // inputs a warp load covers
    const int g = lane & (G - 1), j = lane / G;
    const int N = it.N, M = it.M;
    const int64_t fbytes = (int64_t)M * N;
    const uint8_t *end = it.in + it.n_frames * fbytes;
    const int kmax = (((M + 30) >> 4) + G - 1) / G;  // chunk iterations per input and lane
    // M % 16 == 0: every input starts and ends on a 16-byte boundary (the item's bytes
    // start on one), so no chunk holds a neighbour's bytes and none is masked
    const bool whole = (M & 15) == 0;
    const int64_t rounds = (f_end - f_begin + teams - 1) / teams;
    const uint4 none = make_uint4(kNoPower, kNoPower, kNoPower, kNoPower);
    for (int64_t k = 0; k < rounds; ++k) {
        const int64_t frame = f_begin + k * teams + team;
        const bool fvalid = frame < f_end;
        const uint8_t *fa = it.in + (fvalid ? frame : f_begin) * fbytes;
        int64_t q = 0;
        int32_t cnt = 0;
        for (int i0 = 32 * wt; fvalid && i0 < N; i0 += 32 * W) {
            int32_t s1[G], s2[G];
#pragma unroll
            for (int r = 0; r < G; ++r) {
                s1[r] = 0;
                s2[r] = 0;
            }
            for (int kb = 0; kb < kmax; ++kb) {
                const int c = g + G * kb;  // the lane's chunk of each of its inputs
                uint4 v[G];
#pragma unroll
                for (int r = 0; r < G; ++r) {
                    const int i = i0 + IPW * r + j;
                    const uint8_t *lo = fa + (int64_t)(i < N ? i : 0) * M;
                    const uint8_t *p =
                        (const uint8_t *)((uintptr_t)lo & ~(uintptr_t)15u) + 16 * c;
                    const int nci = (int)(((uintptr_t)lo & 15u) + M + 15) >> 4;
                    v[r] = none;
                    if (i < N && c < nci) {
                        if (p + 16 <= end)
                            v[r] = SK_DBG_IN(it, p, 16) ? ldg_stream16(p) : none;
                        else
                            v[r] = load_clipped_tail(it, p, lo, lo + M);  // the item's last bytes
                    }
                }
                if (!whole) {
#pragma unroll
                    for (int r = 0; r < G; ++r) {
                        const int i = i0 + IPW * r + j;
                        const uint8_t *lo = fa + (int64_t)(i < N ? i : 0) * M;
                        const int nci = (int)(((uintptr_t)lo & 15u) + M + 15) >> 4;
                        const int kl = c == 0 ? (int)((uintptr_t)lo & 15u) : 0;
                        const int kh =
                            c == nci - 1 ? (int)(((uintptr_t)lo + M - 1) & 15u) + 1 : 16;
                        const uint4 mh = cm.head[kl], mt = cm.tail[kh];
                        v[r].x = keep_bytes(v[r].x, mh.x & mt.x);
                        v[r].y = keep_bytes(v[r].y, mh.y & mt.y);
                        v[r].z = keep_bytes(v[r].z, mh.z & mt.z);
                        v[r].w = keep_bytes(v[r].w, mh.w & mt.w);
                    }
                }
#pragma unroll
                for (int r = 0; r < G; ++r)
                    imc_add(v[r], lb, s1[r], s2[r]);
            }
            // reduce-scatter over the G lanes of each input group: lane g keeps input r = g
#pragma unroll
            for (int h = G / 2; h >= 1; h /= 2) {
                const bool up = (g & h) != 0;
#pragma unroll
                for (int t = 0; t < h; ++t) {
                    const int32_t k1 = up ? s1[t + h] : s1[t], o1 = up ? s1[t] : s1[t + h];
                    const int32_t k2 = up ? s2[t + h] : s2[t], o2 = up ? s2[t] : s2[t + h];
                    s1[t] = k1 + __shfl_xor_sync(0xFFFFFFFFu, o1, h);
                    s2[t] = (int32_t)((uint32_t)k2 +
                                      (uint32_t)__shfl_xor_sync(0xFFFFFFFFu, o2, h));
                }
            }
            const int32_t a1 = s1[0];
            const uint32_t a2 = (uint32_t)s2[0] - ((uint32_t)a1 << kPackShift);  // exact S2
            const int i = i0 + IPW * g + j;
            if (i < N) {
                float rr = 0.0f;
                int64_t qi = 0;
                const bool has = SK_EPILOGUE_ALU ? input_term_alu(a1, (int32_t)a2, M, rr, qi)
                                                 : input_term(a1, (int32_t)a2, M, rr, qi);
                if (has) {
                    q += qi;
                    cnt += 1;
                }
                const int64_t o = frame * N + i;
                if (it.s1 && SK_DBG_OUT_IN(it, frame, i)) {
                    it.s1[o] = a1;
                    it.s2[o] = (int32_t)a2;
                }
                if (it.sk_in && SK_DBG_OUT_IN(it, frame, i)) {
                    it.sk_in[o] = has ? __fmul_rn(rr, it.c_tab[1]) : __int_as_float(0x7FC00000);
                    if (it.mask_in)
                        it.mask_in[o] =
                            has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            q += __shfl_xor_sync(0xFFFFFFFFu, (long long)q, o);
            cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        }
        if (W == 1) {
            if (fvalid && lane == 0)
                write_frame(it, frame, q, cnt);
        } else {
            if (lane == 0) {
                red_q[warp] = q;
                red_c[warp] = cnt;
            }
            named_sync(1 + team, 32 * W);
            if (fvalid && wt == 0 && lane == 0) {
                int64_t tq = 0;
                int32_t tc = 0;
                for (int w = 0; w < W; ++w) {
                    tq += red_q[team * W + w];
                    tc += red_c[team * W + w];
                }
                write_frame(it, frame, tq, tc);
            }
            named_sync(1 + team, 32 * W);  // red_* free for the next frame
        }
    }
}

// ---------------------------------------------------------------------------
// Input-major frames of short inputs (M <= kStageMaxM), staged per warp.  A warp
// takes blocks of 32 consecutive inputs of a frame: it reads the aligned 16-byte
// chunks that cover the block's 32·M contiguous bytes, writes them to its own
// shared buffer, and lane r then adds input i0 + r's M bytes from there, as 4-byte
// words (a funnel shift when the input starts off a word boundary; the bytes past
// M in its last word become 0x88, no power) or, when M % 16 == 0, as 16-byte
// pieces.  A lane's sums are its input's: no byte masks and no exchange between
// lanes.  The next block's chunks are loaded into registers before the current
// block is added, so they are in flight meanwhile; with it.prefetch, lane 0 also
// asks L2 for the block after that.  The warp's own __syncwarp orders its buffer's
// writes and reads.  Frames go to teams of W warps (about eight blocks a warp,
// imajor_staged_team), each warp taking the blocks wt, wt + W, ... of its team's
// frame; the team combines Q and N_eff as on the chunk path.
// ---------------------------------------------------------------------------
constexpr int kStageMaxM = 192;

// Warps per frame of the staged blocks: about eight blocks of 32 inputs a warp, a
// power of two from 1 to 16 (A/B, 3 GB launches, N = 2048: M = 100 0.561 -> 0.612,
// M = 48 0.485 -> 0.559 against the chunk path's four; half the team combines).
__host__ __device__ __forceinline__ int imajor_staged_team(int N)
{
    const int blocks = (N + 31) / 32;
    int W = 1;
    while (W < 16 && blocks >= 16 * W)
        W *= 2;
    return W;
}

// Bytes of one warp's buffer: a block's chunks (at most 32·M + 30 bytes) and the
// word read after an input's last, rounded to 16.
__host__ __device__ constexpr int stage_warp_bytes(int M)
{
    return (32 * M + 32 + 15) / 16 * 16;
}

// Chunks a lane loads per block: a block of 32 inputs starting at any offset
// covers at most ceil((15 + 32·M) / 16) chunks.
__host__ __device__ constexpr int stage_lane_chunks(int M)
{
    return ((15 + 32 * M + 15) / 16 + 31) / 32;
}

// The four samples of word w through the lane's table into one packed sum.
__device__ __forceinline__ uint32_t lut_word(uint32_t w, uint32_t lb)
{
    return lds_u32(prmt(w, lb, 0x7604u)) + lds_u32(prmt(w, lb, 0x7614u)) +
           lds_u32(prmt(w, lb, 0x7624u)) + lds_u32(prmt(w, lb, 0x7634u));
}

// Input r's M samples from the staged block: 4-byte words from byte o of the buffer
// (SHIFT: o need not be a multiple of 4; each word then joins two with a funnel
// shift), the bytes past M in the last word as 0x88.  a1 += S1, a2 += S2 + 2^19 S1.
template <bool SHIFT>
__device__ __forceinline__ void staged_words(const uint32_t *buf32, int o, int M, uint32_t lb,
                                             int32_t &a1, uint32_t &a2)
{
    const int nw = (M + 3) >> 2;      // words of the input
    const int nwf = (M >> 4) << 2;    // words of its whole 16-sample groups
    const int qw = o >> 2;
    const uint32_t sh = 8u * (uint32_t)(o & 3);
    uint32_t cur = SHIFT ? buf32[qw] : 0u;
    auto word = [&](int kw) {
        if (!SHIFT)
            return buf32[qw + kw];
        const uint32_t nxt = buf32[qw + kw + 1];
        const uint32_t w = __funnelshift_r(cur, nxt, sh);
        cur = nxt;
        return w;
    };
    int kw = 0;
    for (; kw < nwf; kw += 4) {
        uint32_t acc = 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            acc += lut_word(word(kw + u), lb);
        a1 += (int32_t)(acc >> kPackShift);
        a2 += acc;
    }
    if (kw < nw) {  // the last M % 16 samples (at most 4 words)
        uint32_t acc = 0u;
        for (; kw < nw; ++kw) {
            uint32_t w = word(kw);
            const int left = M - 4 * kw;  // samples from this word on
            if (left < 4)
                w = keep_bytes(w, (1u << (8 * left)) - 1u);
            acc += lut_word(w, lb);
        }
        a1 += (int32_t)(acc >> kPackShift);
        a2 += acc;
    }
}

// Frames [f_begin, f_end) of an input-major item with M <= kStageMaxM; CH >=
// stage_lane_chunks(M); VEC: M % 16 == 0 (16-byte pieces; every block starts on a
// 16-byte boundary); SPLIT: whole blocks load without end checks.  buf: the warp's buffer of stage_warp_bytes(M) bytes.
template <int CH, bool VEC, bool SPLIT>
__device__ __forceinline__ void run_imajor_staged(const Item &it, int W, int64_t f_begin,
                                                  int64_t f_end, uint32_t lb, uint8_t *buf,
                                                  long long *red_q, int *red_c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int team = warp / W, wt = warp - team * W;
    const int teams = (int)(blockDim.x >> 5) / W;
    if (team >= teams)
        return;  // whole warps past the last team
    const int N = it.N, M = it.M;
    const int64_t fbytes = (int64_t)M * N;
    const uint8_t *end = it.in + it.n_frames * fbytes;
    const int nblk = (N + 31) >> 5;
    const int per = wt < nblk ? (nblk - wt + W - 1) / W : 0;  // the warp's blocks a frame
    const int64_t rounds = (f_end - f_begin + teams - 1) / teams;
    const uint4 none = make_uint4(kNoPower, kNoPower, kNoPower, kNoPower);
    uint4 *buf4 = reinterpret_cast<uint4 *>(buf);
    const uint32_t *buf32 = reinterpret_cast<const uint32_t *>(buf);
    uint4 v[CH];
    // the chunks of block b of `frame` into v (chunk lane + 32c of the block)
    auto load_block = [&](int64_t frame, int b) {
        const int i0 = 32 * b;
        const int nb = min(32, N - i0);
        const int64_t start = frame * fbytes + (int64_t)i0 * M;
        const uint8_t *a0 = it.in + (start & ~(int64_t)15);  // the input is 16-byte aligned
        const int nch = (int)(((start & 15) + (int64_t)nb * M + 15) >> 4);
        if (SPLIT && nb == 32 && a0 + 16 * (int64_t)nch <= end) {
            // a whole block inside the item: no end checks, no fill of unused chunks
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const uint8_t *p = a0 + 16 * (lane + 32 * c);
                if (lane + 32 * c < nch)
                    v[c] = SK_DBG_IN(it, p, 16) ? ldg_stream16(p) : none;
            }
        } else {
            // a frame's last, partial block, the item's last block, or every block
            // without SPLIT
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int ci = lane + 32 * c;
                const uint8_t *p = a0 + 16 * ci;
                v[c] = none;
                if (ci < nch)
                    v[c] = p + 16 <= end ? (SK_DBG_IN(it, p, 16) ? ldg_stream16(p) : none)
                                         : load_clipped_tail(it, p, it.in, end);
            }
        }
    };
    if (per > 0 && f_begin + team < f_end)
        load_block(f_begin + team, wt);
    for (int64_t k = 0; k < rounds; ++k) {
        const int64_t frame = f_begin + k * teams + team;
        const bool fvalid = frame < f_end;
        int64_t q = 0;
        int32_t cnt = 0;
        for (int jb = 0; fvalid && jb < per; ++jb) {
            const int b = wt + jb * W;
            const int i0 = 32 * b;
            const int nb = min(32, N - i0);
            const int64_t start = frame * fbytes + (int64_t)i0 * M;
            const int s = (int)(start & 15);
            const int nch = (s + nb * M + 15) >> 4;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (lane + 32 * c < nch)
                    buf4[lane + 32 * c] = v[c];
            __syncwarp();
            // the warp's next block (this frame's, else the team's next frame's first)
            if (jb + 1 < per)
                load_block(frame, b + W);
            else if (frame + teams < f_end)
                load_block(frame + teams, wt);
            if (it.prefetch && lane == 0) {  // the block after that into L2
                int64_t pf = frame;
                int pj = jb + 2;
                if (pj >= per) {
                    pf = frame + teams;
                    pj -= per;
                }
                if (pj < per && pf < f_end) {
                    const int pi0 = 32 * (wt + pj * W);
                    const int pnb = min(32, N - pi0);
                    const int64_t ps = pf * fbytes + (int64_t)pi0 * M;
                    const uint8_t *pa = it.in + (ps & ~(int64_t)15);
                    int64_t bytes = (((ps & 15) + (int64_t)pnb * M + 15) >> 4) << 4;
                    if (pa + bytes > end)
                        bytes = (end - pa) & ~(int64_t)15;
                    if (bytes > 0)
                        prefetch_l2(pa, (uint32_t)bytes);
                }
            }
            int32_t a1 = 0;
            uint32_t a2 = 0u;  // S2 + 2^19 S1 modulo 2^32 until finished
            const int o = s + lane * M;  // the lane's first byte in the buffer
            if (VEC) {
                for (int t = 0; t < M; t += 16) {
                    const uint4 w = buf4[(o + t) >> 4];
                    const uint32_t acc = lut_word(w.x, lb) + lut_word(w.y, lb) +
                                         lut_word(w.z, lb) + lut_word(w.w, lb);
                    a1 += (int32_t)(acc >> kPackShift);
                    a2 += acc;
                }
            } else if (((s | M) & 3) == 0) {
                staged_words<false>(buf32, o, M, lb, a1, a2);  // every input starts on a word
            } else {
                staged_words<true>(buf32, o, M, lb, a1, a2);
            }
            __syncwarp();  // the buffer is read before the next block is written
            a2 -= (uint32_t)a1 << kPackShift;  // exact S2
            const int i = i0 + lane;
            if (lane < nb) {
                float rr = 0.0f;
                int64_t qi = 0;
                const bool has = SK_EPILOGUE_ALU ? input_term_alu(a1, (int32_t)a2, M, rr, qi)
                                                 : input_term(a1, (int32_t)a2, M, rr, qi);
                if (has) {
                    q += qi;
                    cnt += 1;
                }
                const int64_t oi = frame * N + i;
                if (it.s1 && SK_DBG_OUT_IN(it, frame, i)) {
                    it.s1[oi] = a1;
                    it.s2[oi] = (int32_t)a2;
                }
                if (it.sk_in && SK_DBG_OUT_IN(it, frame, i)) {
                    it.sk_in[oi] = has ? __fmul_rn(rr, it.c_tab[1]) : __int_as_float(0x7FC00000);
                    if (it.mask_in)
                        it.mask_in[oi] =
                            has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                }
            }
        }
        for (int sft = 16; sft > 0; sft >>= 1) {
            q += __shfl_xor_sync(0xFFFFFFFFu, (long long)q, sft);
            cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, sft);
        }
        if (W == 1) {
            if (fvalid && lane == 0)
                write_frame(it, frame, q, cnt);
        } else {
            if (lane == 0) {
                red_q[warp] = q;
                red_c[warp] = cnt;
            }
            named_sync(1 + team, 32 * W);
            if (fvalid && wt == 0 && lane == 0) {
                int64_t tq = 0;
                int32_t tc = 0;
                for (int w = 0; w < W; ++w) {
                    tq += red_q[team * W + w];
                    tc += red_c[team * W + w];
                }
                write_frame(it, frame, tq, tc);
            }
            named_sync(1 + team, 32 * W);  // red_* free for the next frame
        }
    }
}

}  // namespace sk
