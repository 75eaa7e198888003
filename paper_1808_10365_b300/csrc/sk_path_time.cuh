// Time-major vector path of the fused kernel: rows of 8-byte vectors through a
// register ring, table lookups and the frame epilogue of sk_device.cuh.
#pragma once

#include "sk_device.cuh"

namespace sk {

// R rows of bytes 0x88 (re = im = 0): no power, so they add nothing to the sums.
template <int R>
__device__ __forceinline__ void fill_zero_power_rows(uint2 (&b)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r)
        b[r] = make_uint2(0x88888888u, 0x88888888u);
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
            if (!SK_DBG_IN(it, fp + (int64_t)j * R * N, (R - 1) * N + 8)) {
                fill_zero_power_rows<R>(buf[j]);
            } else if constexpr (NC > 0) {
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
                    if (!SK_DBG_IN(it, pn + (int64_t)j * R * N, (R - 1) * N + 8)) {
                        fill_zero_power_rows<R>(buf[j]);
                    } else if constexpr (NC > 0) {
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
        finish_s2(s1, s2);
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
        if (!SK_DBG_IN(it, p, (R - 1) * N + 8)) {
            fill_zero_power_rows<R>(b);
            return;
        }
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
    finish_s2(s1, s2);
}

// L2 prefetch of a box of the input through its tensor map (rows y .. y+31 of
// columns x .. x+255 for the warp-slice path); a hint, results never depend on it.
__device__ __forceinline__ void prefetch_box(const CUtensorMap *tm, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(x), "r"(y)
                 : "memory");
}

// L2 prefetch of whole rows [r0, r0 + nr) of the input (row stride N bytes) by bulk
// prefetches of at most 32 KB: the ragged path issues one per team and turn where the
// host allows it (Item::prefetch; N = 2047, M = 256: +7 %; on the aligned warp-slice
// paths without a tensor map, N = 1000 or a folded tail, it measured 19-30 % slower).
// The range is widened to 16-byte boundaries and cut at the input's last whole 16
// bytes; a hint, results never depend on it.
__device__ __forceinline__ void prefetch_rows(const Item &it, int64_t r0, int64_t nr, int64_t N)
{
    const int64_t total = (it.n_frames * (int64_t)it.M * N) & ~(int64_t)15;
    int64_t b = (r0 * N) & ~(int64_t)15;
    int64_t e = ((r0 + nr) * N + 15) & ~(int64_t)15;
    if (e > total)
        e = total;
    for (; b < e; b += 32768)
        prefetch_l2(it.in + b, (uint32_t)(e - b < 32768 ? e - b : 32768));
}

// Orders a tensor map in device memory, written by a host copy before the launch,
// before this thread's first use of it through the tensor-map proxy.
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *tm)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(tm))
                 : "memory");
}

// Register batches of a lane past the last input: bytes 0x88 (re = im = 0) have
// no power, so the lane's sums stay zero and its inputs count for nothing.

template <int S, int R>
__device__ __forceinline__ void fill_zero_power(uint2 (&buf)[S][R])
{
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
        for (int r = 0; r < R; ++r)
            buf[j][r] = make_uint2(0x88888888u, 0x88888888u);
}

// The input terms (Eq. normedSum2 per input) of one lane's 8 inputs of a frame,
// with the per-input outputs the item asks for (S1, S2, SK_i and its one-input
// flag), and the sum over the warp of their fixed-point q_i and count.  A lane
// past the last input (its sums zero) adds nothing and writes nothing.
// PART: the lane may hold columns past N (ragged N), whose sums are not inputs'
// and are left out.
// q0, cnt0: a lane's terms of other inputs (a folded tail's), added before the sum
// over the warp.
template <bool PART = false>
__device__ __forceinline__ void slice_terms(const Item &it, int64_t frame, int col0, int M,
                                            const int32_t (&s1)[kVec],
                                            const int32_t (&s2)[kVec], int64_t &q,
                                            int32_t &cnt, int64_t q0 = 0, int32_t cnt0 = 0)
{
    q = q0;
    cnt = cnt0;
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
        if (PART && col0 + k >= it.N)
            continue;
        float r = 0.0f;
        int64_t qi = 0;
        const bool has = SK_EPILOGUE_ALU ? input_term_alu(s1[k], s2[k], M, r, qi)
                                         : input_term(s1[k], s2[k], M, r, qi);
        if (has) {
            q += qi;
            cnt += 1;
        }
        if (it.sk_in && col0 < it.N && SK_DBG_OUT_IN(it, frame, col0 + k)) {
            const int64_t o = frame * it.N + col0 + k;
            it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1]) : __int_as_float(0x7FC00000);
            if (it.mask_in)
                it.mask_in[o] = has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
        }
    }
    if (it.s1 && col0 < it.N && SK_DBG_OUT_IN(it, frame, col0)) {
        int32_t *o1 = it.s1 + frame * it.N + col0;
        int32_t *o2 = it.s2 + frame * it.N + col0;
#pragma unroll
        for (int k = 0; k < kVec; ++k) {
            if (PART && col0 + k >= it.N)
                break;
            o1[k] = s1[k];
            o2[k] = s2[k];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    }
}

// Folded tail of the warp slices (Item::wtail = NT): with N = 256 W + 8 NT and
// NT <= W, a team is W warps instead of W + 1, since a warp with NT busy lanes
// costs as much as a whole slice (and at W = 8 leaves a CTA's 16 warps short of a
// second team).  Group g of the NT groups of 8 columns past the last whole slice
// falls, for frame f, to warp (f + g) mod W of the team (on the row-balanced path
// the same warp in every team that shares the frame).  Inside the turn loop that
// warp loads, one turn ahead, the group's 8-byte word of each of the turn's rows
// (lane l: row l of the turn), so that no load latency is left for the frame's
// end; its sectors are shared with the slice loads of the same and the next row.
// tail_turn adds one turn: the lane's 8 table values go through 3 reduce-scatter
// steps over lane bits 4, 3 and 2, after which lane l holds input (l >> 2) & 7 of
// the group summed over 8 rows (packed, at most 8 rows: the fields cannot carry),
// added exactly into ts1, ts2.  Lanes that differ in bits 0 and 1 hold the input's
// other rows.
__device__ __forceinline__ void tail_turn(uint2 w, uint32_t lb, int32_t &ts1, int32_t &ts2)
{
    const int lane = threadIdx.x & 31;
    uint32_t v[kVec];
    v[0] = lds_u32(prmt(w.x, lb, 0x7604u));
    v[1] = lds_u32(prmt(w.x, lb, 0x7614u));
    v[2] = lds_u32(prmt(w.x, lb, 0x7624u));
    v[3] = lds_u32(prmt(w.x, lb, 0x7634u));
    v[4] = lds_u32(prmt(w.y, lb, 0x7604u));
    v[5] = lds_u32(prmt(w.y, lb, 0x7614u));
    v[6] = lds_u32(prmt(w.y, lb, 0x7624u));
    v[7] = lds_u32(prmt(w.y, lb, 0x7634u));
    // lane bit 4 keeps inputs 4..7 (set) or 0..3 and sends the other half
    const bool b4 = lane & 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t keep = b4 ? v[k + 4] : v[k], send = b4 ? v[k] : v[k + 4];
        v[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
    }
    const bool b3 = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const uint32_t keep = b3 ? v[k + 2] : v[k], send = b3 ? v[k] : v[k + 2];
        v[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
    }
    const bool b2 = lane & 4;
    const uint32_t keep = b2 ? v[1] : v[0], send = b2 ? v[0] : v[1];
    const uint32_t t = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
    ts1 += (int32_t)(t >> kPackShift);
    ts2 += (int32_t)(t & ((1u << kPackShift) - 1u));
}

// The folded group's input (l >> 2) & 7 at the end of a frame (part): its sums over
// the lanes that share it, into every one of them.
__device__ __forceinline__ void tail_reduce(int32_t &ts1, int32_t &ts2)
{
    ts1 += __shfl_xor_sync(0xFFFFFFFFu, ts1, 2);
    ts2 += __shfl_xor_sync(0xFFFFFFFFu, ts2, 2);
    ts1 += __shfl_xor_sync(0xFFFFFFFFu, ts1, 1);
    ts2 += __shfl_xor_sync(0xFFFFFFFFu, ts2, 1);
}

// Lanes l with l % 4 == 0 form the term of input col + l / 4 (Eq. normedSum2) from
// its totals, with the per-input outputs the item asks for, into q and cnt (which
// slice_terms then sums over the warp with the slice's terms).
__device__ __forceinline__ void tail_lane_term(const Item &it, int64_t frame, int col, int M,
                                               int32_t ts1, int32_t ts2, int64_t &q,
                                               int32_t &cnt)
{
    const int lane = threadIdx.x & 31;
    if ((lane & 3) != 0)
        return;
    const int c = col + (lane >> 2);
    float r = 0.0f;
    int64_t qi = 0;
    const bool has = SK_EPILOGUE_ALU ? input_term_alu(ts1, ts2, M, r, qi)
                                     : input_term(ts1, ts2, M, r, qi);
    if (has) {
        q += qi;
        cnt += 1;
    }
    if (SK_DBG_OUT_IN(it, frame, c)) {
        const int64_t o = frame * it.N + c;
        if (it.sk_in) {
            it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1]) : __int_as_float(0x7FC00000);
            if (it.mask_in)
                it.mask_in[o] = has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
        }
        if (it.s1) {
            it.s1[o] = ts1;
            it.s2[o] = ts2;
        }
    }
}

// Warp-slice path: one-item launches and batched items with a tensor map,
// time-major, N a multiple of 8 from 256 to 4096, 16 x 2 tiles (8 x 2 for
// M = 16 mod 32: 16-row turns, the 32-row prefetch box every other turn).  The team of a
// frame is ceil(N/256) warps (floor(N/256) with a folded tail, above), each owning a
// 256-column slice of the team's frames and running on its own: no barrier per frame.  Lane 0 of each warp asks L2 for
// the rows the warp will load two ring turns ahead with one 2D tensor prefetch
// (32 rows x 256 bytes) through the input's tensor map (a kernel parameter of a
// one-item launch, or the item's map in device memory; none when N % 16 != 0).  After a frame, the warp adds its
// slice's Q and N_eff into the team's slot for that frame (shared-memory
// atomics); the warp that arrives last forms the frame's mask and SK and frees
// the slot.  A team's slots form a ring of kWiSlots frames; a warp that gets
// that far ahead of a slow one waits, bounded, for its slot.
template <int R, int S, int NC, bool TAIL = false, bool MR = false>
__device__ __forceinline__ void run_fast_wi(const Item &it, int64_t f_begin, int64_t f_end,
                                            uint32_t lb, TeamSmem &ts, const CUtensorMap *tmap)
{
    static_assert(R * S == 32 || R * S == 16, "ring turns of 32 or 16 rows");
    // one 32-row prefetch box per 32 rows: every turn, or every other 16-row turn
    constexpr int BB = 32 / R;             // batches per box
    constexpr int PER = 32 / (R * S);      // turns per box
    const int M = it.M;
    const int64_t N = NC > 0 ? (int64_t)NC : (int64_t)it.N;
    // teams of W warps, one 256-column slice each (the last one partial when 256
    // does not divide N, unless the columns past the whole slices are folded);
    // the CTA's last 16 - T W warps have nothing to do
    // TAIL: NT = Item::wtail groups of 8 columns folded (NT <= W), read inside the
    // turn loop by one warp of the team per group and frame (tail_turn)
    constexpr int RS = R * S;  // rows per turn
    const int NT = TAIL ? it.wtail : 0;
    const int W = NT ? (int)(N >> 8) : (int)((N + 255) >> 8);
    const int T = (kThreads / 32) / W;
    const int warp = threadIdx.x >> 5;
    const int team_idx = warp / W;
    if (team_idx >= T)
        return;
    const int lane = threadIdx.x & 31;
    const int c = warp - team_idx * W;  // the warp's slice
    const int xs = c * 256;             // its first column
    const int col0 = xs + lane * kVec;
    // lanes past N read nothing (none when N is a compiled multiple of 256)
    const bool col_ok = (NC > 0 && NC % 256 == 0) || col0 < N;
    // no tensor map when N is not a multiple of 16 (the map's row stride must
    // be) or the plan turned the prefetch off: those launches stream without it
    const bool pf = it.wi != 2;
    // the first row of a prefetch box; MR: kept inside the input (a frame's padded last
    // turn puts boxes past its rows)
    auto box_row = [&](int64_t y) -> int {
        if constexpr (MR) {
            const int64_t last = it.n_frames * M - 32;
            return (int)(y < last ? y : (last > 0 ? last : 0));
        }
        return (int)y;
    };
    const int64_t fbytes = (int64_t)M * N;
    // MR: M not a multiple of the turn; a frame is ceil(M / RS) turns, the last one
    // partial (rows past M read nothing and have no power)
    const int nb = MR ? (M + RS - 1) / RS * S : M / R;
    const int64_t kmax = (f_end - f_begin + T - 1) / T;
    WiSlot *slots = ts.wi[team_idx];
    const uint8_t *const in = it.in;

    uint2 buf[S][R];
    if (!col_ok)
        fill_zero_power(buf);
    int64_t frame = f_begin + team_idx;
    bool ok = frame < f_end;
    const uint8_t *fp = in + frame * fbytes + col0;
    // R rows from p, the frame's rows row0.., row stride N (a load immediate when
    // NC > 0)
    auto load = [&](uint2 (&b)[R], const uint8_t *p, int row0) {
        if constexpr (MR) {
            const int left = M - row0;
            if (left < R) {
                // the frame's last rows: loads below M only
                const bool in = left > 0 && SK_DBG_IN(it, p, (int64_t)(left - 1) * N + 8);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    b[r] = (in && r < left) ? ldg_stream(p + (int64_t)r * N)
                                            : make_uint2(0x88888888u, 0x88888888u);
                return;
            }
        }
        if (!SK_DBG_IN(it, p, (R - 1) * N + 8)) {
            fill_zero_power_rows<R>(b);
            return;
        }
        if constexpr (NC > 0) {
            load_rows_imm<NC>(b, p, std::make_integer_sequence<int, R>{});
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                b[r] = ldg_stream(p + (int64_t)r * N);
        }
    };
    if (ok && col_ok) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            load(buf[j], fp + (int64_t)j * R * N, j * R);
    }
    // folded tail: the first column of this warp's group of frame f, or -1
    auto tail_col = [&](int64_t f) -> int {
        const int gt = (c - (int)(f % W) + W) % W;
        return gt < NT ? 256 * W + 8 * gt : -1;
    };
    // the group's word of row `lane` of the turn whose first row's byte col0 is at
    // t0p (rows past the turn: no power)
    auto tail_load = [&](const uint8_t *t0p, int tc) -> uint2 {
        const uint8_t *p = t0p + (tc - col0) + (int64_t)lane * N;
        return (lane < RS && SK_DBG_IN(it, p, 8)) ? ldg_stream(p)
                                                  : make_uint2(0x88888888u, 0x88888888u);
    };
    [[maybe_unused]] int tcc = -1;   // this warp's group of the current frame
    [[maybe_unused]] uint2 wt = make_uint2(0x88888888u, 0x88888888u);
    [[maybe_unused]] int32_t ts1 = 0, ts2 = 0;
    if constexpr (TAIL) {
        tcc = ok ? tail_col(frame) : -1;
        if (tcc >= 0)
            wt = tail_load(fp, tcc);
    }
    for (int64_t kk = 0; kk < kmax; ++kk) {
        const int64_t nframe = frame + T;
        const bool nok = nframe < f_end;
        const uint8_t *nfp = in + nframe * fbytes + col0;
        uint32_t acc[kVec];
        int32_t s1[kVec], s2[kVec];
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            acc[j] = 0u;
            s1[j] = 0;
            s2[j] = 0;
        }
        for (int jb = 0; jb < nb; jb += S) {
            if (lane == 0 && pf && (jb / S) % PER == 0) {
                const int ba = jb + 2 * BB;  // two boxes (64 rows) ahead
                if (ba < nb) {
                    if (ok)
                        prefetch_box(tmap, xs, box_row(frame * M + ba * R));
                } else if (nok && ba - nb + BB <= nb) {
                    prefetch_box(tmap, xs, box_row(nframe * M + (ba - nb) * R));
                }
            }
            const bool same_frame = jb + S < nb;
            const uint8_t *pn = same_frame ? fp + (int64_t)(jb + S) * R * N : nfp;
            const bool lok = same_frame ? ok : nok;
            if constexpr (TAIL) {
                // this turn's word, then the next turn's (in flight over this turn;
                // past the frame's last turn, the group of the team's next frame)
                if (tcc >= 0)
                    tail_turn(wt, lb, ts1, ts2);
                const int ntc = same_frame ? tcc : (nok ? tail_col(nframe) : -1);
                wt = ntc >= 0 ? tail_load(pn, ntc) : make_uint2(0x88888888u, 0x88888888u);
            }
#pragma unroll
            for (int j = 0; j < S; ++j) {
                if (ok) {
                    // MR: a batch wholly past the frame's last row adds nothing
                    if (!MR || (jb + j) * R < M) {
#pragma unroll
                        for (int r = 0; r < R; r += 2)
                            accum_pair(buf[j][r], buf[j][r + 1], lb, acc);
                    }
                    if (((j + 1) * R) % kFlushRows == 0)
                        flush(acc, s1, s2);
                }
                if (lok && col_ok)
                    load(buf[j], pn + (int64_t)j * R * N, (same_frame ? jb + S + j : j) * R);
            }
        }
        if (ok) {
            // the slice's terms and per-input outputs, summed over the warp
            finish_s2(s1, s2);
            int64_t q = 0, q0 = 0;
            int32_t cnt = 0, c0 = 0;
            if constexpr (TAIL) {
                if (tcc >= 0) {
                    tail_reduce(ts1, ts2);
                    tail_lane_term(it, frame, tcc, M, ts1, ts2, q0, c0);
                }
            }
            slice_terms(it, frame, col0, M, s1, s2, q, cnt, q0, c0);
            if (lane == 0)
                wi_commit(it, slots, kk, W, frame, q, cnt);
            __syncwarp();
        }
        if constexpr (TAIL) {
            ts1 = 0;
            ts2 = 0;
            tcc = nok ? tail_col(nframe) : -1;
        }
        frame = nframe;
        fp = nfp;
        ok = nok;
    }
}

// Row-balanced warp-slice path (one-item time-major launches of the warp-slice
// shapes, given the plan's scratch).  The input is one sequence of F*M rows (a
// frame is a block of M consecutive rows), cut into TT = F*M/RS ring turns of RS
// rows (RS = R*S: 32, or 16 on the 8-row tile for M = 16 mod 32).  Team k of the grid's K teams takes the turns [TT*k/K, TT*(k+1)/K), so
// teams differ by at most one turn whatever F is, and each of its warps runs its
// 256-column slice of those rows.  A frame that lies inside the range goes through
// the team's slot ring as on the warp-slice path.  A frame that a range boundary
// cuts is shared with the neighbouring team(s): each part adds its S1, S2 into the
// frame's slot in the scratch (device memory), the warp that completes a column's
// rows forms that column's terms, and the warp that completes the last column
// writes the frame.  Whoever reads a scratch word back leaves it zero, so the
// scratch is all zero before and after every launch.  Scratch layout for K teams
// of W warps: uint64 S2:S1[K][N], int32 turns[K][W] (padded to an even count),
// uint64 Q[K], int32 cnt[K], int32 arrive[K]; the slot of a cut frame is the
// index of the first team boundary inside it.
template <int R, int S, int NC, bool TAIL = false>
__device__ __forceinline__ void run_fast_rb(const Item &it, uint32_t lb, TeamSmem &ts,
                                            const CUtensorMap *tmap)
{
    static_assert(R * S == 32 || R * S == 16, "one turn per ring revolution");
    constexpr int RS = R * S;         // rows per turn: 32, or 16 for M = 16 mod 32
    constexpr int PER = 32 / RS;      // turns per 32-row prefetch box
    const int M = it.M;
    const int64_t N = NC > 0 ? (int64_t)NC : (int64_t)it.N;
    // teams of W warps (256-column slices, the last one partial when 256 does not
    // divide N, unless the columns past the whole slices are folded); the CTA's
    // last 16 - T W warps have nothing to do
    // TAIL: NT = Item::wtail groups of 8 columns folded (NT <= W), read inside the
    // turn loop by one warp of the team per group and frame (tail_turn)
    const int NT = TAIL ? it.wtail : 0;
    const int W = NT ? (int)(N >> 8) : (int)((N + 255) >> 8);
    const int T = (kThreads / 32) / W;
    const int warp = threadIdx.x >> 5;
    const int team_idx = warp / W;
    if (team_idx >= T)
        return;
    const int lane = threadIdx.x & 31;
    const int c = warp - team_idx * W;
    const int xs = c * 256;
    const int col0 = xs + lane * kVec;
    // lanes past N read and add nothing (none when N is a compiled multiple of 256)
    const bool col_ok = (NC > 0 && NC % 256 == 0) || col0 < N;
    // no tensor map when N is not a multiple of 16 (the map's row stride must
    // be) or the plan turned the prefetch off: those launches stream without it
    const bool pf = it.wi != 2;
    const int64_t tpf = M / RS;  // turns per frame
    const int64_t TT = it.n_frames * tpf;
    const int64_t K = (int64_t)gridDim.x * T;
    const int64_t kt = (int64_t)blockIdx.x * T + team_idx;
    const int64_t t0 = TT * kt / K, t1 = TT * (kt + 1) / K;
    unsigned long long *const ps = reinterpret_cast<unsigned long long *>(it.rb);
    int32_t *const pturn = reinterpret_cast<int32_t *>(ps + K * N);
    // the turn counters padded to an even count keep the 64-bit words aligned
    unsigned long long *const pq =
        reinterpret_cast<unsigned long long *>(pturn + ((K * W + 1) & ~(int64_t)1));
    int32_t *const pcnt = reinterpret_cast<int32_t *>(pq + K);
    int32_t *const parr = pcnt + K;
    WiSlot *slots = ts.wi[team_idx];
    const uint8_t *const in = it.in + col0;

    // R rows from p, row stride N (a load immediate when NC > 0)
    auto load = [&](uint2 (&b)[R], const uint8_t *p) {
        if (!SK_DBG_IN(it, p, (R - 1) * N + 8)) {
            fill_zero_power_rows<R>(b);
            return;
        }
        if constexpr (NC > 0) {
            load_rows_imm<NC>(b, p, std::make_integer_sequence<int, R>{});
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                b[r] = ldg_stream(p + (int64_t)r * N);
        }
    };
    uint2 buf[S][R];
    if (!col_ok)
        fill_zero_power(buf);
    if (t0 < t1 && col_ok) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            load(buf[j], in + (t0 * RS + j * R) * N);
    }
    uint32_t acc[kVec];
    int32_t s1[kVec], s2[kVec];
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
        acc[j] = 0u;
        s1[j] = 0;
        s2[j] = 0;
    }
    int64_t kk = 0;               // whole frames this team has committed
    int64_t frame = t0 / tpf;     // the current turn's frame ...
    int gf = (int)(t0 - frame * tpf);  // ... and turn in it (counters: no division per turn)
    int gf0 = gf;                 // first turn of the current frame part

    // folded tail: the first column of this warp's group of a frame f with
    // f mod W = fw, or -1
    auto tail_col = [&](int fw) -> int {
        const int gt = c >= fw ? c - fw : c - fw + W;
        return gt < NT ? 256 * W + 8 * gt : -1;
    };
    // the group's word of row `lane` of the turn whose first row's byte col0 is at
    // t0p (rows past the turn: no power)
    auto tail_load = [&](const uint8_t *t0p, int tc) -> uint2 {
        const uint8_t *p = t0p + (tc - col0) + (int64_t)lane * N;
        return (lane < RS && SK_DBG_IN(it, p, 8)) ? ldg_stream(p)
                                                  : make_uint2(0x88888888u, 0x88888888u);
    };
    [[maybe_unused]] int fw = 0;     // the current frame mod W (a counter)
    [[maybe_unused]] int tcc = -1;   // this warp's group of the current frame
    [[maybe_unused]] uint2 wt = make_uint2(0x88888888u, 0x88888888u);
    [[maybe_unused]] int32_t ts1 = 0, ts2 = 0;
    if constexpr (TAIL) {
        fw = (int)(frame % W);
        tcc = tail_col(fw);
        if (t0 < t1 && tcc >= 0)
            wt = tail_load(in + t0 * RS * N, tcc);
    }
    for (int64_t g = t0; g < t1; ++g) {
        if (lane == 0 && pf && g % PER == 0 && g + 2 * PER < t1)
            prefetch_box(tmap, xs, (int)((g + 2 * PER) * RS));  // 64 rows ahead
        const bool more = g + 1 < t1;
        const uint8_t *pn = in + (g + 1) * RS * N;
        [[maybe_unused]] int tcn = -1;  // the group of the next turn's frame
        if constexpr (TAIL) {
            // the next turn's word first, then this turn's
            tcn = gf + 1 == (int)tpf ? tail_col(fw + 1 == W ? 0 : fw + 1) : tcc;
            const uint2 wn = (more && tcn >= 0) ? tail_load(pn, tcn)
                                                : make_uint2(0x88888888u, 0x88888888u);
            if (tcc >= 0)
                tail_turn(wt, lb, ts1, ts2);
            wt = wn;
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
#pragma unroll
            for (int r = 0; r < R; r += 2)
                accum_pair(buf[j][r], buf[j][r + 1], lb, acc);
            if (((j + 1) * R) % kFlushRows == 0)
                flush(acc, s1, s2);
            if (more && col_ok)
                load(buf[j], pn + (int64_t)j * R * N);
        }
        ++gf;
        const bool fend = gf == (int)tpf;
        if (!fend && more)
            continue;
        finish_s2(s1, s2);
        if constexpr (TAIL) {
            if (tcc >= 0)
                tail_reduce(ts1, ts2);
        }
        if (fend && gf0 == 0) {
            // a whole frame: the slice's part goes into the team's slot ring
            int64_t q = 0, q0 = 0;
            int32_t cnt = 0, c0 = 0;
            if constexpr (TAIL) {
                if (tcc >= 0)
                    tail_lane_term(it, frame, tcc, M, ts1, ts2, q0, c0);
            }
            slice_terms(it, frame, col0, M, s1, s2, q, cnt, q0, c0);
            if (lane == 0)
                wi_commit(it, slots, kk, W, frame, q, cnt);
            __syncwarp();
            ++kk;
        } else {
            // part of a cut frame: add the column's sums into the frame's slot, S2 in
            // the high and S1 in the low half of one word per input (S1 <= 2^19 and
            // S2 <= 2^26 for M <= 4096, so the halves never carry into each other)
            const int64_t slot = ((frame * tpf + 1) * K + TT - 1) / TT;
            unsigned long long *sp = ps + slot * N + col0;
            if (col_ok && SK_DBG_SLOT(it, slot)) {
#pragma unroll
                for (int k = 0; k < kVec; ++k)
                    atomicAdd(sp + k,
                              ((unsigned long long)(uint32_t)s2[k] << 32) | (uint32_t)s1[k]);
            }
            // this warp's folded group of the part's rows goes into the same slot
            // (lane 4j: input j), counted with the warp's own column below
            if constexpr (TAIL) {
                if (tcc >= 0 && (lane & 3) == 0 && SK_DBG_SLOT(it, slot))
                    atomicAdd(ps + slot * N + tcc + (lane >> 2),
                              ((unsigned long long)(uint32_t)ts2 << 32) | (uint32_t)ts1);
            }
            __syncwarp();
            int fin = 0;
            if (lane == 0) {
                // one fence for the warp: it orders the lanes' adds, which the
                // __syncwarp put before it, ahead of the count
                __threadfence();
                const int part = gf - gf0;
                fin = atomicAdd(pturn + slot * W + c, part) + part == (int)tpf;
                if (fin)
                    __threadfence();
            }
            fin = __shfl_sync(0xFFFFFFFFu, fin, 0);
            if (fin) {
                // this warp completed the column: its totals, and the slot words zero
                // (the __syncwarp orders the lanes' reads after lane 0's fence)
                __syncwarp();
                if (col_ok) {
#pragma unroll
                    for (int k = 0; k < kVec; ++k) {
                        const unsigned long long v = atomicExch(sp + k, 0ull);
                        s1[k] = (int32_t)(uint32_t)v;
                        s2[k] = (int32_t)(v >> 32);
                    }
                }
                int64_t q = 0, q0 = 0;
                int32_t cnt = 0, c0 = 0;
                if constexpr (TAIL) {
                    // the column's folded group: its totals (lane 4j: input j) and terms
                    if (tcc >= 0 && (lane & 3) == 0) {
                        const unsigned long long v =
                            atomicExch(ps + slot * N + tcc + (lane >> 2), 0ull);
                        tail_lane_term(it, frame, tcc, M, (int32_t)(uint32_t)v,
                                       (int32_t)(v >> 32), q0, c0);
                    }
                }
                slice_terms(it, frame, col0, M, s1, s2, q, cnt, q0, c0);
                if (lane == 0) {
                    atomicExch(pturn + slot * W + c, 0);
                    atomicAdd(pq + slot, (unsigned long long)q);
                    atomicAdd(pcnt + slot, cnt);
                    __threadfence();
                    if (atomicAdd(parr + slot, 1) == W - 1) {
                        // the last column: the frame's outputs
                        __threadfence();
                        const int64_t Q = (int64_t)atomicExch(pq + slot, 0ull);
                        const int32_t C = atomicExch(pcnt + slot, 0);
                        atomicExch(parr + slot, 0);
                        write_frame(it, frame, Q, C);
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            acc[j] = 0u;
            s1[j] = 0;
            s2[j] = 0;
        }
        if constexpr (TAIL) {
            ts1 = 0;
            ts2 = 0;
            tcc = tcn;
            if (fend)
                fw = fw + 1 == W ? 0 : fw + 1;
        }
        if (fend) {
            gf = 0;
            ++frame;
        }
        gf0 = gf;
    }
}

// Ragged N (time-major, N % 8 != 0, M % 16 == 0; one-item launches given the
// plan's scratch): the row-balanced warp-slice path above, for rows that are not
// 8-byte aligned.  A lane's 8 bytes of row t start at a = in + t N + col0; `in`
// is 16-byte aligned and col0 a multiple of 8, so a lies D = (t N) mod 8 bytes
// past an 8-byte boundary, and over 16-row turns and 8-row batches D depends
// only on the row r within its batch: D = (r NR) mod 8 with NR = N mod 8, a
// template parameter, so every row's D is a compile-time constant.  A row takes
// the aligned word at a - D and, when its bytes reach past it, the next one;
// a funnel shift of each 32-bit half puts the 8 bytes in place (no shift when
// D = 0, a swap when D = 4).  Both words start inside the row's own bytes, so no
// load leaves the input; the last lane's bytes past column N (the next row's, or
// beyond the input's end inside the same aligned word) are left out of the terms.
// Rows go through L1 (ld.global.nc), where a warp's two words of a row share
// lines.  Cut frames combine as on run_fast_rb, for the lane's columns below N.
template <int NR>
__device__ __forceinline__ void run_fast_rag(const Item &it, uint32_t lb, TeamSmem &ts)
{
    static_assert(NR >= 1 && NR <= 7, "N mod 8");
    constexpr int R = 8, S = 2, RS = R * S;
    const int M = it.M;
    const int64_t N = it.N;
    const int W = (int)((N + 255) >> 8);
    const int T = (kThreads / 32) / W;
    const int warp = threadIdx.x >> 5;
    const int team_idx = warp / W;
    if (team_idx >= T)
        return;
    const int lane = threadIdx.x & 31;
    const int c = warp - team_idx * W;
    const int col0 = c * 256 + lane * kVec;
    const bool col_ok = col0 < N;
    const int keep = col_ok ? (N - col0 < kVec ? (int)(N - col0) : kVec) : 0;  // bytes of ours
    const int64_t tpf = M / RS;  // turns per frame
    const int64_t TT = it.n_frames * tpf;
    const int64_t K = (int64_t)gridDim.x * T;
    const int64_t kt = (int64_t)blockIdx.x * T + team_idx;
    const int64_t t0 = TT * kt / K, t1 = TT * (kt + 1) / K;
    unsigned long long *const ps = reinterpret_cast<unsigned long long *>(it.rb);
    int32_t *const pturn = reinterpret_cast<int32_t *>(ps + K * N);
    unsigned long long *const pq =
        reinterpret_cast<unsigned long long *>(pturn + ((K * W + 1) & ~(int64_t)1));
    int32_t *const pcnt = reinterpret_cast<int32_t *>(pq + K);
    int32_t *const parr = pcnt + K;
    WiSlot *slots = ts.wi[team_idx];
    const uint8_t *const in = it.in + col0;

    // the aligned word(s) of R rows from p (row stride N)
    auto load = [&](uint2 (&lo)[R], uint2 (&hi)[R], const uint8_t *p) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int D = (r * NR) & 7;
            const uint8_t *a = p + (int64_t)r * N;
            if (!SK_DBG_IN(it, a, keep)) {
                lo[r] = hi[r] = make_uint2(0x88888888u, 0x88888888u);
                continue;
            }
            const uint2 *w = reinterpret_cast<const uint2 *>(a - D);
            lo[r] = __ldg(w);
            if (D > 0 && D + keep > kVec)
                hi[r] = __ldg(w + 1);
        }
    };
    // the lane's 8 bytes of a row from its aligned words
    auto place = [](const uint2 &lo, const uint2 &hi, int D) -> uint2 {
        const int sh = 8 * (D & 3);
        if (D == 0)
            return lo;
        if (D < 4)
            return make_uint2(__funnelshift_r(lo.x, lo.y, sh), __funnelshift_r(lo.y, hi.x, sh));
        if (D == 4)
            return make_uint2(lo.y, hi.x);
        return make_uint2(__funnelshift_r(lo.y, hi.x, sh), __funnelshift_r(hi.x, hi.y, sh));
    };
    uint2 lo[S][R], hi[S][R];
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
        for (int r = 0; r < R; ++r)
            lo[j][r] = hi[j][r] = make_uint2(0x88888888u, 0x88888888u);
    if (t0 < t1 && col_ok) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            load(lo[j], hi[j], in + (t0 * RS + j * R) * N);
    }
    uint32_t acc[kVec];
    int32_t s1[kVec], s2[kVec];
#pragma unroll
    for (int j = 0; j < kVec; ++j) {
        acc[j] = 0u;
        s1[j] = 0;
        s2[j] = 0;
    }
    int64_t kk = 0;
    int64_t frame = t0 / tpf;
    int gf = (int)(t0 - frame * tpf);
    int gf0 = gf;
    // no tensor map (N % 8 != 0): the team's first warp asks L2 for whole rows two
    // turns ahead
    const bool pfr = it.prefetch != 0;
    for (int64_t g = t0; g < t1; ++g) {
        if (pfr && c == 0 && lane == 0 && g + 2 < t1)
            prefetch_rows(it, (g + 2) * RS, RS, N);
        const bool more = g + 1 < t1;
        const uint8_t *pn = in + (g + 1) * RS * N;
#pragma unroll
        for (int j = 0; j < S; ++j) {
#pragma unroll
            for (int r = 0; r < R; r += 2)
                accum_pair(place(lo[j][r], hi[j][r], (r * NR) & 7),
                           place(lo[j][r + 1], hi[j][r + 1], ((r + 1) * NR) & 7), lb, acc);
            if (((j + 1) * R) % kFlushRows == 0)
                flush(acc, s1, s2);
            if (more && col_ok)
                load(lo[j], hi[j], pn + (int64_t)j * R * N);
        }
        ++gf;
        const bool fend = gf == (int)tpf;
        if (!fend && more)
            continue;
        finish_s2(s1, s2);
        if (fend && gf0 == 0) {
            int64_t q;
            int32_t cnt;
            slice_terms<true>(it, frame, col0, M, s1, s2, q, cnt);
            if (lane == 0)
                wi_commit(it, slots, kk, W, frame, q, cnt);
            __syncwarp();
            ++kk;
        } else {
            const int64_t slot = ((frame * tpf + 1) * K + TT - 1) / TT;
            unsigned long long *sp = ps + slot * N + col0;
            if (col_ok && SK_DBG_SLOT(it, slot)) {
#pragma unroll
                for (int k = 0; k < kVec; ++k)
                    if (k < keep)
                        atomicAdd(sp + k,
                                  ((unsigned long long)(uint32_t)s2[k] << 32) | (uint32_t)s1[k]);
            }
            __syncwarp();
            int fin = 0;
            if (lane == 0) {
                __threadfence();
                const int part = gf - gf0;
                fin = atomicAdd(pturn + slot * W + c, part) + part == (int)tpf;
                if (fin)
                    __threadfence();
            }
            fin = __shfl_sync(0xFFFFFFFFu, fin, 0);
            if (fin) {
                __syncwarp();
#pragma unroll
                for (int k = 0; k < kVec; ++k) {
                    s1[k] = 0;
                    s2[k] = 0;
                    if (k < keep) {
                        const unsigned long long v = atomicExch(sp + k, 0ull);
                        s1[k] = (int32_t)(uint32_t)v;
                        s2[k] = (int32_t)(v >> 32);
                    }
                }
                int64_t q;
                int32_t cnt;
                slice_terms<true>(it, frame, col0, M, s1, s2, q, cnt);
                if (lane == 0) {
                    atomicExch(pturn + slot * W + c, 0);
                    atomicAdd(pq + slot, (unsigned long long)q);
                    atomicAdd(pcnt + slot, cnt);
                    __threadfence();
                    if (atomicAdd(parr + slot, 1) == W - 1) {
                        __threadfence();
                        const int64_t Q = (int64_t)atomicExch(pq + slot, 0ull);
                        const int32_t C = atomicExch(pcnt + slot, 0);
                        atomicExch(parr + slot, 0);
                        write_frame(it, frame, Q, C);
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            acc[j] = 0u;
            s1[j] = 0;
            s2[j] = 0;
        }
        if (fend) {
            gf = 0;
            ++frame;
        }
        gf0 = gf;
    }
}

}  // namespace sk
