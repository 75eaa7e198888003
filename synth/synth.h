/*
 * Seeded synthetic channelised-voltage generator: the one module that the
 * oracle and the CUDA path both take their inputs from.  It holds none of the
 * detector's arithmetic; it only draws 4+4-bit complex samples.
 *
 * Sample model (the data characteristics of the paper's App. B simulation and
 * of the CHIME correlator input, Sec. 3.1):
 *   v = clip(round(s + sigma_i * g), -7, 7),  g ~ N(0,1),
 * independently for the real and imaginary part, where s is the RFI
 * contribution to that component (0 on clean samples).  The byte is
 *   ((v_re + 8) << 4) | (v_im + 8)            (offset binary, real high).
 *
 * Drawing v: the host tabulates, per input and per component, the 14
 * thresholds c_k = floor(2^32 * P(v <= k)), k = -7..6, of the quantised
 * distribution (see synth_thresholds in synth_cpu.c).  One uniform 32-bit
 * word u then gives v = -7 + #{k : u >= c_k}.  This uses integer operations
 * only, so the CPU build (gcc) and the GPU build (nvcc) of this header emit
 * the same bytes for the same seed.
 *
 * Uniform words come from the counter-based generator Philox4x32-10 of
 * Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As Easy as 1, 2,
 * 3" (SC'11), written here from its published definition.  Counters are
 * (global frame, time, input pair, stream tag), so any frame can be
 * regenerated on its own.
 */
#ifndef SYNTH_H
#define SYNTH_H

#include <stdint.h>

#ifdef __CUDACC__
#define SYN_HD __host__ __device__ __forceinline__
#else
#define SYN_HD static inline
#endif

#define SYN_NTHR 14 /* thresholds between the 15 levels -7..7 */

/* stream tags: the fourth counter word separates independent draws */
#define SYN_TAG_NOISE 0x4E4F4953u
#define SYN_TAG_SIGMA 0x5349474Du
#define SYN_TAG_PHASE 0x50484153u
#define SYN_TAG_PERM 0x5045524Du
#define SYN_TAG_AMP 0x414D504Cu

/* Philox4x32 round constants (multipliers and Weyl key increments) */
#define SYN_PHILOX_M0 0xD2511F53u
#define SYN_PHILOX_M1 0xCD9E8D57u
#define SYN_PHILOX_W0 0x9E3779B9u
#define SYN_PHILOX_W1 0xBB67AE85u

SYN_HD void syn_mulhilo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: out = bijection of ctr under key (k0, k1). */
SYN_HD void syn_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                       uint32_t k0, uint32_t k1, uint32_t out[4])
{
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        if (r > 0) {
            k0 += SYN_PHILOX_W0;
            k1 += SYN_PHILOX_W1;
        }
        syn_mulhilo(SYN_PHILOX_M0, c0, &hi0, &lo0);
        syn_mulhilo(SYN_PHILOX_M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Offset-binary nibble (v + 8, v in -7..7) for uniform word u. */
SYN_HD uint32_t syn_nibble(uint32_t u, const uint32_t *thr)
{
    uint32_t n = 1; /* v = -7 */
#pragma unroll
    for (int k = 0; k < SYN_NTHR; ++k)
        n += (u >= thr[k]) ? 1u : 0u;
    return n;
}

/*
 * Per-frame RFI descriptor.  slot < 0: clean frame.  Otherwise the frame's
 * samples with (t % period) < on_len use the shifted thresholds of RFI table
 * `slot` (a CW tone has period 1, on_len 1; a pulse of duty d has
 * on_len = d * period).
 */
typedef struct {
    int32_t slot;
    int32_t period;
    int32_t on_len;
    int32_t pad;
} syn_frame_t;

/*
 * The two bytes of inputs (2*ip, 2*ip+1) at (global frame g, time t).
 * thr_clean: [N][14] (same table for real and imaginary part).
 * thr_rfi:   [n_slots][N][2][14] (real table, then imaginary table).
 */
SYN_HD void syn_pair(uint32_t k0, uint32_t k1, uint32_t g, uint32_t t,
                     uint32_t ip, int32_t N, const uint32_t *thr_clean,
                     const syn_frame_t *fr, const uint32_t *thr_rfi,
                     uint8_t out[2])
{
    uint32_t u[4];
    syn_philox(g, t, ip, SYN_TAG_NOISE, k0, k1, u);
    int on = 0;
    if (fr->slot >= 0)
        on = ((int32_t)(t % (uint32_t)fr->period) < fr->on_len);
    for (int h = 0; h < 2; ++h) {
        int32_t i = (int32_t)(2 * ip) + h;
        if (i >= N) {
            out[h] = 0x88;
            continue;
        }
        const uint32_t *tr, *ti;
        if (on) {
            const uint32_t *base =
                thr_rfi + ((int64_t)fr->slot * N + i) * (2 * SYN_NTHR);
            tr = base;
            ti = base + SYN_NTHR;
        } else {
            tr = thr_clean + (int64_t)i * SYN_NTHR;
            ti = tr;
        }
        uint32_t re = syn_nibble(u[2 * h], tr);
        uint32_t im = syn_nibble(u[2 * h + 1], ti);
        out[h] = (uint8_t)((re << 4) | im);
    }
}

#endif /* SYNTH_H */
