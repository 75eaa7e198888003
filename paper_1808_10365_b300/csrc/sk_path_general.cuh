// General path of the fused kernel: any N and M, either layout.
#pragma once

#include "sk_device.cuh"

namespace sk {

// General path: any N (<= 4096), any M >= 2, either layout; the same table,
// terms and epilogue.  With ALIGNED, time-major rows go through aligned 8-byte
// loads and a shift; otherwise (and for input-major) through byte loads with
// bounds checks.  Serves the sizes the fast paths do not take.  Served and
// input-major kernels leave ALIGNED off: its registers would spill in them.
template <bool SERVED, bool ALIGNED = !SERVED, int RB = 4>
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
            // RB rows per load batch: 8 in one-item launches (two loads of 8 bytes a
            // row, 16 in flight: 12-17 % faster on N = 2047, M = 100 or 33, N = 3001,
            // N = 99, M = 101 than 4), 4 in the batched kernels, where 8 spills
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
                        if (w >= lo_lim && w + 16 <= hi_lim && SK_DBG_IN(it, w, 16)) {
                            lo[r] = __ldg((const unsigned long long *)w);
                            hi[r] = __ldg((const unsigned long long *)(w + 8));
                        } else {
                            uint64_t v = 0x8888888888888888ull;
                            if (SK_DBG_IN(it, a, keep)) {
                                v = 0;
                                for (int j = 0; j < keep; ++j)
                                    v |= (uint64_t)a[j] << (8 * j);
                            }
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
                        const uint8_t *pb = fb + (it.layout == 0 ? (int64_t)t * N + c : c * M + t);
                        const uint32_t b = SK_DBG_IN(it, pb, 1) ? *pb : 0x88u;
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
        finish_s2(s1, s2);
        frame_epilogue<SERVED>(it, frame, fvalid, col0, lit, team_idx, parity, s1, s2, ts);
        parity ^= 1;
        frame += fstride;
    }
}

}  // namespace sk
