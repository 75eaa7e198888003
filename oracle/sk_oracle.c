/*
 * ORACLE -- test infrastructure only.  Plain, slow CPU statement of the
 * multi-receiver spectral-kurtosis estimator of Taylor et al., "Spectral
 * Kurtosis Based RFI Mitigation for CHIME" (arXiv:1808.10365).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may call it; the
 * product library never links or loads it, and it shares no code with it.
 *
 * Notation: M samples per input per estimate (the paper's n), N inputs.
 * Bytes are 4+4-bit offset binary: real = high nibble - 8, imag = low nibble
 * - 8 (the data format of the paper's App. B simulation).
 *
 * Functions and the passages they follow:
 *   oracle_power_sums  -- Eq. 1 / Eq. (singlesums): S1 = sum |x|^2,
 *                         S2 = sum |x|^4 per input, exact integers; |x|^2 is
 *                         re*re + im*im (Sec. 2.2.3, "Calculating Power").
 *   oracle_sk_f64      -- Eqs. (discreteMean), (normedSum1), (normedSum2)
 *                         and (final), evaluated in that order in fp64.
 *   oracle_sk_spec     -- the same estimator with the per-input normalised
 *                         term r_i = n*S2_i/S1_i^2 - 1 (Eq. normedSimplifiedSum2
 *                         and Eq. final, third line: SK~ = Avg(SK^_i),
 *                         SK^_i = (n+1)/(n-1) r_i), taken in the precision the
 *                         CUDA path declares: D_i = n*S2_i - S1_i^2 exact in
 *                         int64, one IEEE fp32 division, r_i scaled by 2^32
 *                         and rounded to an int64, exact int64 sum over inputs,
 *                         fp32 final scaling.  This fixes every rounding so
 *                         that Q and the mask can be compared bit for bit.
 * Inputs with S1_i = 0 (no power) are left out and N_eff counts the rest; the
 * paper divides by mu_i without a guard (Eq. normedSum2).
 * Built with -ffp-contract=off: no fused multiply-add anywhere.
 */
#include <math.h>
#include <stdint.h>

static inline uint8_t byte_at(const uint8_t *x, int64_t f, int32_t t, int32_t i,
                              int32_t M, int32_t N, int32_t layout)
{
    int64_t base = f * (int64_t)M * N;
    if (layout == 0)
        return x[base + (int64_t)t * N + i];
    return x[base + (int64_t)i * M + t];
}

/* S1[f][i], S2[f][i] for every frame f and input i. */
void oracle_power_sums(const uint8_t *x, int64_t n_frames, int32_t M, int32_t N,
                       int32_t layout, int64_t *S1, int64_t *S2)
{
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < n_frames; ++f) {
        for (int32_t i = 0; i < N; ++i) {
            int64_t s1 = 0, s2 = 0;
            for (int32_t t = 0; t < M; ++t) {
                uint8_t b = byte_at(x, f, t, i, M, N, layout);
                int64_t re = (int64_t)(b >> 4) - 8;
                int64_t im = (int64_t)(b & 15) - 8;
                int64_t p = re * re + im * im; /* |x|^2 */
                s1 += p;
                s2 += p * p; /* |x|^4 */
            }
            S1[f * N + i] = s1;
            S2[f * N + i] = s2;
        }
    }
}

/*
 * fp64, in the paper's order: mu_i = S1_i / n; S1bar = sum S1_i / mu_i;
 * S2bar = sum S2_i / mu_i^2; SK~ = (n+1)/(n-1) * (S2bar / (n N) - 1).
 * s1bar receives S1bar (= n N_eff up to rounding, Eq. normedSum1).
 */
void oracle_sk_f64(const int64_t *S1, const int64_t *S2, int64_t n_frames,
                   int32_t M, int32_t N, double *sk, double *s1bar,
                   int32_t *neff)
{
    const double n = (double)M;
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < n_frames; ++f) {
        double sb1 = 0.0, sb2 = 0.0;
        int32_t ne = 0;
        for (int32_t i = 0; i < N; ++i) {
            int64_t s1 = S1[f * N + i];
            if (s1 <= 0)
                continue;
            double mu = (double)s1 / n;
            sb1 += (double)s1 / mu;
            sb2 += (double)S2[f * N + i] / (mu * mu);
            ne += 1;
        }
        if (ne > 0)
            sk[f] = (n + 1.0) / (n - 1.0) * (sb2 / (n * (double)ne) - 1.0);
        else
            sk[f] = NAN;
        if (s1bar)
            s1bar[f] = sb1;
        if (neff)
            neff[f] = ne;
    }
}

/*
 * Kernel-precision statement (see header).  Q[f] = sum_i rint(2^32 r_i),
 * r_i = fp32(D_i) / fp32(S1_i^2); sk[f] = fp32(Q) * 2^-32 * c,
 * c = fp32((n+1) / ((n-1) N_eff)) from a double division.
 */
void oracle_sk_spec(const int64_t *S1, const int64_t *S2, int64_t n_frames,
                    int32_t M, int32_t N, int64_t *Q, int32_t *neff, float *sk)
{
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < n_frames; ++f) {
        int64_t q_sum = 0;
        int32_t ne = 0;
        for (int32_t i = 0; i < N; ++i) {
            int64_t s1 = S1[f * N + i];
            if (s1 <= 0)
                continue;
            int64_t d = (int64_t)M * S2[f * N + i] - s1 * s1;
            int64_t den = s1 * s1;
            float r = (float)d / (float)den;
            long long q = llrintf(r * 4294967296.0f);
            q_sum += (int64_t)q;
            ne += 1;
        }
        Q[f] = q_sum;
        neff[f] = ne;
        if (ne > 0) {
            float c = (float)((double)(M + 1) / ((double)(M - 1) * (double)ne));
            float qf = (float)q_sum;
            sk[f] = (qf * 0x1p-32f) * c;
        } else {
            sk[f] = NAN;
        }
    }
}

/*
 * Per-input terms in the kernel precision: q[j] = rint(2^32 r_j) with r_j as
 * in oracle_sk_spec, and sk1[j] = fp32(r_j) * fp32((n+1)/(n-1)), the single-
 * receiver SK^_j of Eq. originalSK; valid[j] = 0 (q = 0, sk1 = NaN) when
 * S1_j = 0.
 */
void oracle_terms_spec(const int64_t *S1, const int64_t *S2, int64_t count, int32_t M,
                       int64_t *q, float *sk1, uint8_t *valid)
{
    const float c1 = (float)((double)(M + 1) / ((double)(M - 1) * 1.0));
    for (int64_t j = 0; j < count; ++j) {
        int64_t s1 = S1[j];
        if (s1 <= 0) {
            q[j] = 0;
            sk1[j] = NAN;
            valid[j] = 0;
            continue;
        }
        int64_t d = (int64_t)M * S2[j] - s1 * s1;
        float r = (float)d / (float)(s1 * s1);
        q[j] = (int64_t)llrintf(r * 4294967296.0f);
        sk1[j] = r * c1;
        valid[j] = 1;
    }
}

/* Per-input single-receiver SK^_i (Eq. originalSK) in fp64; NaN if S1_i = 0. */
void oracle_sk_single_f64(const int64_t *S1, const int64_t *S2, int64_t count,
                          int32_t M, double *out)
{
    const double n = (double)M;
    for (int64_t j = 0; j < count; ++j) {
        if (S1[j] <= 0) {
            out[j] = NAN;
            continue;
        }
        double s1 = (double)S1[j];
        out[j] = (n + 1.0) / (n - 1.0) * (n * (double)S2[j] / (s1 * s1) - 1.0);
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the parallel loops that follow (timing only; results do not
 * depend on it: every sum is exact integer arithmetic or per-frame). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
