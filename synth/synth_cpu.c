/*
 * Host side of the synthetic generator: per-input noise levels, RFI phases,
 * quantisation threshold tables, and a CPU byte generator that emits the same
 * bytes as the GPU one (synth_gpu.cu) because both run synth.h.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "synth.h"

#define TWO32 4294967296.0

static void key_of(uint64_t seed, uint32_t *k0, uint32_t *k1)
{
    *k0 = (uint32_t)seed;
    *k1 = (uint32_t)(seed >> 32);
}

/* One Philox4x32-10 block (exported for the known-answer test). */
void synth_philox_block(const uint32_t ctr[4], const uint32_t key[2],
                        uint32_t out[4])
{
    syn_philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1], out);
}

/* out[j] = (u + 0.5) / 2^32 with u the first word of Philox(a, b, j, tag). */
void synth_u01(uint64_t seed, uint32_t tag, uint32_t a, uint32_t b, int64_t n,
               double *out)
{
    uint32_t k0, k1, r[4];
    key_of(seed, &k0, &k1);
    for (int64_t j = 0; j < n; ++j) {
        syn_philox(a, b, (uint32_t)j, tag, k0, k1, r);
        out[j] = ((double)r[0] + 0.5) / TWO32;
    }
}

/* Per-input noise level sigma_i ~ U[lo, hi]. */
void synth_sigmas(uint64_t seed, int32_t N, double lo, double hi, double *out)
{
    uint32_t k0, k1, r[4];
    key_of(seed, &k0, &k1);
    for (int32_t i = 0; i < N; ++i) {
        syn_philox((uint32_t)i, 0, 0, SYN_TAG_SIGMA, k0, k1, r);
        out[i] = lo + (hi - lo) * (((double)r[0] + 0.5) / TWO32);
    }
}

/* RFI phase of input i in global frame g, uniform on [0, 2pi). */
static double phase_of(uint32_t k0, uint32_t k1, uint32_t g, uint32_t i)
{
    uint32_t r[4];
    syn_philox(g, i, 0, SYN_TAG_PHASE, k0, k1, r);
    return 2.0 * M_PI * (((double)r[0] + 0.5) / TWO32);
}

void synth_phases(uint64_t seed, uint32_t g, int32_t N, double *out)
{
    uint32_t k0, k1;
    key_of(seed, &k0, &k1);
    for (int32_t i = 0; i < N; ++i)
        out[i] = phase_of(k0, k1, g, (uint32_t)i);
}

/*
 * c_k = floor(2^32 * P(v <= k)), k = -7..6, for v = clip(round(shift +
 * sigma*g), -7, 7):  P(v <= k) = Phi((k + 0.5 - shift) / sigma).
 */
void synth_thresholds(double sigma, double shift, uint32_t out[SYN_NTHR])
{
    for (int j = 0; j < SYN_NTHR; ++j) {
        double k = (double)(j - 7);
        double z = (k + 0.5 - shift) / sigma;
        double p = 0.5 * erfc(-z / sqrt(2.0));
        double c = floor(p * TWO32);
        if (c < 0.0)
            c = 0.0;
        if (c > TWO32 - 1.0)
            c = TWO32 - 1.0;
        out[j] = (uint32_t)c;
    }
}

void synth_clean_tables(int32_t N, const double *sigma, uint32_t *out)
{
    for (int32_t i = 0; i < N; ++i)
        synth_thresholds(sigma[i], 0.0, out + (int64_t)i * SYN_NTHR);
}

/*
 * Shifted tables for RFI slots: slot r sits in global frame slot_frame[r]
 * with amplitude slot_amp[r]; input i gets the constant phasor
 * A * exp(j * phi_{g,i}), i.e. shift A cos(phi) on the real part and
 * A sin(phi) on the imaginary part.  out: [n_slots][N][2][14].
 */
void synth_rfi_tables(uint64_t seed, int32_t N, const double *sigma,
                      int32_t n_slots, const int64_t *slot_frame,
                      const double *slot_amp, uint32_t *out)
{
    uint32_t k0, k1;
    key_of(seed, &k0, &k1);
#pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < n_slots; ++r) {
        for (int32_t i = 0; i < N; ++i) {
            double phi = phase_of(k0, k1, (uint32_t)slot_frame[r], (uint32_t)i);
            double a = slot_amp[r];
            uint32_t *base = out + ((int64_t)r * N + i) * (2 * SYN_NTHR);
            synth_thresholds(sigma[i], a * cos(phi), base);
            synth_thresholds(sigma[i], a * sin(phi), base + SYN_NTHR);
        }
    }
}

/*
 * Bytes of frames frame0 .. frame0+n_frames-1 of a dataset.
 * layout 0: [frame][t][input] (time-major); 1: [frame][input][t].
 * frames: descriptor per generated frame (index 0 = frame0).
 */
void synth_generate_cpu(uint8_t *out, int64_t n_frames, int64_t frame0,
                        int32_t M, int32_t N, int32_t layout, uint64_t seed,
                        const uint32_t *thr_clean, const syn_frame_t *frames,
                        const uint32_t *thr_rfi)
{
    uint32_t k0, k1;
    key_of(seed, &k0, &k1);
    int32_t npair = (N + 1) / 2;
    int64_t fbytes = (int64_t)M * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t f = 0; f < n_frames; ++f) {
        uint32_t g = (uint32_t)(frame0 + f);
        uint8_t *fo = out + f * fbytes;
        for (int32_t t = 0; t < M; ++t) {
            for (int32_t ip = 0; ip < npair; ++ip) {
                uint8_t b[2];
                syn_pair(k0, k1, g, (uint32_t)t, (uint32_t)ip, N, thr_clean,
                         &frames[f], thr_rfi, b);
                for (int h = 0; h < 2; ++h) {
                    int32_t i = 2 * ip + h;
                    if (i >= N)
                        break;
                    if (layout == 0)
                        fo[(int64_t)t * N + i] = b[h];
                    else
                        fo[(int64_t)i * M + t] = b[h];
                }
            }
        }
    }
}
