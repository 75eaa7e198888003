// Time-major vector path of the fused kernel: rows of 8-byte vectors through a
// register ring, table lookups and the frame epilogue of sk_device.cuh.
#pragma once

#include "sk_device.cuh"

namespace sk {

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

// Rows [b0 R, b1 R) of one frame for this thread's 8 columns, added into exact
// s1, s2 (b1 - b0 a multiple of S).  The same ring of S register batches of R
// rows as run_fast, without the frame epilogue: a frame whose rows are shared
// by several teams sums their partial S1, S2 before its epilogue.
template <int R, int S, int NC>
__device__ __forceinline__ void run_rows(const Item &it, int64_t frame, int b0, int b1,
                                         int col0, uint32_t lb, int32_t (&s1)[kVec],
                                         int32_t (&s2)[kVec])
{
    static_assert((R * S) % kFlushRows == 0, "flush cadence");
    const int64_t N = NC > 0 ? (int64_t)NC : (int64_t)it.N;
    const uint8_t *fp = it.in + frame * (int64_t)it.M * N + col0;
    uint2 buf[S][R];
    uint32_t acc[kVec];
#pragma unroll
    for (int k = 0; k < kVec; ++k)
        acc[k] = 0u;
    auto load = [&](uint2 (&b)[R], int batch) {
        const uint8_t *p = fp + (int64_t)batch * R * N;
        if constexpr (NC > 0) {
            load_rows_imm<NC>(b, p, std::make_integer_sequence<int, R>{});
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                b[r] = ldg_stream(p + (int64_t)r * N);
        }
    };
#pragma unroll
    for (int j = 0; j < S; ++j)
        if (b0 + j < b1)
            load(buf[j], b0 + j);
    for (int jb = b0; jb < b1; jb += S) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
#pragma unroll
            for (int r = 0; r < R; r += 2)
                accum_pair(buf[j][r], buf[j][r + 1], lb, acc);
            if (((j + 1) * R) % kFlushRows == 0)
                flush(acc, s1, s2);
            if (jb + S + j < b1)
                load(buf[j], jb + S + j);
        }
    }
}

}  // namespace sk
