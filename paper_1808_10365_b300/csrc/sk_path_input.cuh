// Input-major paths of the fused kernel: the grouped path (8 lanes per group of
// 8 inputs, reduce-scatter) and the per-input path for the other lengths.
#pragma once

#include "sk_device.cuh"

namespace sk {

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
            if (lf < f_end && lk < K && i < N) {
                const uint8_t *a = it.in + lf * fbytes + (int64_t)i * M + (int64_t)(j + lc * G) * 16;
                buf[u] = SK_DBG_IN(it, a, 16) ? ldg_stream16(a)
                                              : make_uint4(0x88888888u, 0x88888888u,
                                                           0x88888888u, 0x88888888u);
            }
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
                            if (it.s1 && SK_DBG_OUT_IN(it, frame, i)) {
                                it.s1[o] = s1;
                                it.s2[o] = s2;
                            }
                            if (it.sk_in && SK_DBG_OUT_IN(it, frame, i)) {
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
        if (fvalid && lit == 0 && SK_DBG_OUT(it, frame)) {
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

// Inputs between consecutive members of a segment's group.  Groups of 8 inputs on
// 8 lanes (M >= 128) are 8 consecutive inputs: a segment reads whole 128-byte
// lines.  Groups of 4 on 4 lanes (M = 64) are strided by 8 inputs: the 8 segments
// of a warp share the warp's 32 consecutive inputs, segment s taking inputs s,
// s + 8, s + 16 and s + 24, so that each warp load instruction reads 512
// contiguous bytes (4 whole lines) instead of 8 runs of 64 bytes.
// Both need teams of at least one warp (team_log2 >= 5, which the host keeps on
// the grouped paths) and, when strided, whole inputs (SPLIT = 1).
template <int G>
__host__ __device__ constexpr int group_stride()
{
    return G == 4 ? 8 : 1;
}

// First (sub-)input of the group of segment seg (of nseg per team) in group row k
// of a frame (team inputs a group row).
template <int G>
__device__ __forceinline__ int group_first(int k, int nseg, int seg)
{
    if constexpr (group_stride<G>() == 1)
        return (k * nseg + seg) * G;
    else
        return k * nseg * G + (seg >> 3) * (8 * G) + (seg & 7);
}

// Members of a group below NS (sub-)inputs, 0..G.
template <int G>
__device__ __forceinline__ int group_live(int first, int NS)
{
    constexpr int IST = group_stride<G>();
    const int r = NS - first;
    if constexpr (IST == 1)
        return r < 0 ? 0 : (r > G ? G : r);
    const int n = r <= 0 ? 0 : (r + IST - 1) / IST;
    return n > G ? G : n;
}

// Batch nb of a group on the grouped input-major path: chunk t of the batch is
// the group's chunk g = nb KB + t, i.e. chunk g % CH of its member g / CH; all
// offsets are load immediates.
template <int M, int G, int CH, int KB, int nb, int... Ts>
__device__ __forceinline__ void load_group_imm(uint4 *buf, const uint8_t *base,
                                               std::integer_sequence<int, Ts...>)
{
    constexpr int IST = group_stride<G>();
    ((buf[Ts] = ldg_stream16_at<((nb * KB + Ts) / CH) * IST * M +
                                ((nb * KB + Ts) % CH) * G * 16>(base)),
     ...);
}

template <int M, int G, int CH, int KB, int nb>
__device__ __forceinline__ void load_group_batch(uint4 (&buf)[KB], const uint8_t *base, int live)
{
    if (live == G) {
        load_group_imm<M, G, CH, KB, nb>(buf, base, std::make_integer_sequence<int, KB>{});
    } else {
        constexpr int IST = group_stride<G>();
#pragma unroll
        for (int t = 0; t < KB; ++t) {
            const int g = nb * KB + t;
            buf[t] = g / CH < live
                         ? ldg_stream16(base + (g / CH) * IST * M + (g % CH) * G * 16)
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

// The sums of a segment's group once its chunks are read (the balanced path; the
// grouped path spells the same steps out, which ptxas allocates with fewer
// spills in the batched kernels): a reduce-scatter over
// the G lanes leaves input j's S1, S2 in lane j (the sub-inputs of an input are
// added), and lane j adds its input's term (Eq. normedSum2) to q, cnt and writes
// the per-input outputs the item asks for.  i0 is the group's first sub-input in
// the frame (its members group_stride apart), M the sub-input length.
template <int G, int SPLIT>
__device__ __forceinline__ void group_terms(const Item &it, int32_t (&s1)[G], int32_t (&s2)[G],
                                            int j, int live, int64_t frame, int i0, int M,
                                            int64_t &q, int32_t &cnt)
{
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
    if (j < live && j % SPLIT == 0) {
        const int i = (i0 + j * group_stride<G>()) / SPLIT;
        float r = 0.0f;
        int64_t qi = 0;
        const bool has = SK_EPILOGUE_ALU ? input_term_alu(s1[0], s2[0], M * SPLIT, r, qi)
                                         : input_term(s1[0], s2[0], M * SPLIT, r, qi);
        if (has) {
            q += qi;
            cnt += 1;
        }
        const int64_t o = frame * it.N + i;
        if (it.s1 && SK_DBG_OUT_IN(it, frame, i)) {
            it.s1[o] = s1[0];
            it.s2[o] = s2[0];
        }
        if (it.sk_in && SK_DBG_OUT_IN(it, frame, i)) {
            it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1]) : __int_as_float(0x7FC00000);
            if (it.mask_in)
                it.mask_in[o] = has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
        }
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
    static_assert(group_stride<G>() == 1 || SPLIT == 1, "strided groups hold whole inputs");
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
    // teams of two or more warps in a single-item launch combine a frame's warps
    // through the team's slot ring instead of a barrier per frame
    const bool wi = it.wi && team >= 64;

    constexpr int IST = group_stride<G>();  // inputs between a group's members
    // sub-inputs of group (frame f, k) that this segment may read: 0..G
    auto live_of = [&](int64_t f, int k) -> int {
        return (f < f_end) ? group_live<G>(group_first<G>(k, nseg, seg), NS) : 0;
    };
    auto base_of = [&](int64_t f, int k) -> const uint8_t * {
        return it.in + f * fbytes + (int64_t)group_first<G>(k, nseg, seg) * M + j * 16;
    };
    // debug builds: a group whose chunks would leave the input is not read
    auto dbg_live = [&](const uint8_t *base, int live) -> int {
        return (live > 0 && !SK_DBG_IN(it, base, (int64_t)(live - 1) * IST * M +
                                                     (CH - 1) * G * 16 + 16))
                   ? 0
                   : live;
    };
    uint4 A[KB], B[KB];
    int64_t frame = f_begin + team_idx;
    const uint8_t *cur_base = base_of(frame, 0);
    int cur_live = dbg_live(cur_base, live_of(frame, 0));
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
            const int nxt_live = dbg_live(nxt_base, live_of(nf, nk));
            if constexpr (PF) {
                if (IST == 1 && nxt_live > 0 && j == 0) {
                    prefetch_l2(nxt_base, (uint32_t)(nxt_live * M));
                } else if (IST > 1 && j == 0 && (seg & 7) == 0 && nf < f_end) {
                    // strided groups: the warp's first segment asks for the warp's
                    // contiguous block of 8 G inputs
                    const int r = NS - group_first<G>(nk, nseg, seg);
                    if (r > 0)
                        prefetch_l2(nxt_base, (uint32_t)((r < 8 * G ? r : 8 * G) * M));
                }
            }
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
                const int i = (group_first<G>(k, nseg, seg) + j * IST) / SPLIT;
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
                if (it.s1 && SK_DBG_OUT_IN(it, frame, i)) {
                    it.s1[o] = s1[0];
                    it.s2[o] = s2[0];
                }
                if (it.sk_in && SK_DBG_OUT_IN(it, frame, i)) {
                    it.sk_in[o] = has ? __fmul_rn(r, it.c_tab[1]) : __int_as_float(0x7FC00000);
                    if (it.mask_in)
                        it.mask_in[o] =
                            has ? ((qi > it.t_hi[1] || qi < it.t_lo[1]) ? 1 : 0) : 1;
                }
            }
            cur_base = nxt_base;
            cur_live = nxt_live;
        }
        if (wi) {
            // warp-slice combine: the warp's part goes into the team's slot, no barrier
            if (fvalid) {
                for (int o = 16; o > 0; o >>= 1) {
                    q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
                    cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
                }
                if ((lit & 31) == 0)
                    wi_commit(it, ts.wi[team_idx], kk, team >> 5, frame, q, cnt);
                __syncwarp();
            }
            frame += T;
            continue;
        }
        team_sum(q, cnt, e, team_log2, team_idx, parity, ts, false);
        if (fvalid && lit == 0 && SK_DBG_OUT(it, frame)) {
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

// The grouped input-major path with rows balanced over the grid (one-item
// launches given the plan's scratch, teams of two or more warps whose sub-inputs
// divide a frame's).  A group row is one group per segment of a team, team*M
// consecutive bytes, and the input is one sequence of TT = F*NG group rows (NG
// per frame).  Team k of the grid's K teams takes the group rows
// [TT*k/K, TT*(k+1)/K), and each of its warps runs its segments' groups of those
// rows.  A group holds whole inputs, so a frame that a range boundary cuts needs
// only its Q and N_eff combined: every warp adds its part into the frame's slot in
// the scratch and counts its group rows, and the warp that brings the count to NG
// times the team's warps writes the frame and zeroes the slot.  Frames inside the
// range go through the team's slot ring.  Scratch layout for K teams: uint64 Q[K],
// int32 cnt[K], int32 rows[K]; the slot of a cut frame is the index of the first
// team boundary inside it.
template <int G, int CH, bool PF, int SPLIT = 1>
__device__ __forceinline__ void run_imajor_rb(const Item &it, uint32_t lb, TeamSmem &ts)
{
    static_assert(SPLIT >= 1 && G % SPLIT == 0, "sub-inputs of one input share a group");
    static_assert(group_stride<G>() == 1 || SPLIT == 1, "strided groups hold whole inputs");
    constexpr int M = 16 * G * CH;
    constexpr int NB = (G * CH / 8) < 2 ? 2 : G * CH / 8;  // batches per group
    constexpr int KB = G * CH / NB;                       // chunks per batch
    static_assert(KB * NB == G * CH && NB % 2 == 0, "batch shape");
    // 32-bit counters (the host keeps TT below 2^31): fewer live registers beside
    // the two register batches
    const int team_log2 = it.team_log2;
    const int team = 1 << team_log2;
    const int T = kThreads >> team_log2;
    const int team_idx = threadIdx.x >> team_log2;
    const int lit = threadIdx.x & (team - 1);
    const int nseg = team / G;
    const int seg = lit / G, j = lit % G;
    const int NG = it.N * SPLIT / team;  // group rows per frame
    const int TT = (int)it.n_frames * NG;
    const int K = (int)gridDim.x * T;
    const int kt = (int)blockIdx.x * T + team_idx;
    const int u0 = (int)((int64_t)TT * kt / K), u1 = (int)((int64_t)TT * (kt + 1) / K);
    const int64_t step = (int64_t)team * M;  // bytes per group row
    constexpr int IST = group_stride<G>();  // inputs between a group's members
    const uint8_t *cur =
        it.in + (int64_t)u0 * step + (int64_t)group_first<G>(0, nseg, seg) * M + j * 16;

    // debug builds: a group row whose chunks would leave the input is not read
    [[maybe_unused]] const int64_t gext =
        (int64_t)(G - 1) * IST * M + (CH - 1) * G * 16 + 16;
    uint4 A[KB], B[KB];
    if (u0 < u1)
        load_group_batch<M, G, CH, KB, 0>(A, cur, SK_DBG_IN(it, cur, gext) ? G : 0);
    int64_t q = 0;
    int32_t cnt = 0;
    int frame = u0 / NG, ku = u0 % NG;  // the group row's frame and row in it
    int ku0 = ku;                       // first row of the current frame part
    int kk = 0;                         // whole frames this team has committed
    for (int u = u0; u < u1; ++u) {
        const bool more = u + 1 < u1;
        const uint8_t *nxt = more ? cur + step : cur;
        // the next group row's bytes: the segment's group, or with strided groups
        // the warp's block of 8 G inputs (from its first segment)
        if (PF && more && j == 0 && (IST == 1 || (seg & 7) == 0))
            prefetch_l2(nxt, (uint32_t)((IST == 1 ? G : 8 * G) * M));
        int32_t s1[G], s2[G];
#pragma unroll
        for (int t = 0; t < G; ++t) {
            s1[t] = 0;
            s2[t] = 0;
        }
        group_batches<M, G, CH, NB, KB, 0>(A, B, cur, G, nxt,
                                           (more && SK_DBG_IN(it, nxt, gext)) ? G : 0, lb, s1,
                                           s2);
        group_terms<G, SPLIT>(it, s1, s2, j, G, frame, group_first<G>(ku, nseg, seg), M, q,
                              cnt);
        cur = nxt;
        ++ku;
        const bool fend = ku == NG;
        if (!fend && more)
            continue;
        for (int o = 16; o > 0; o >>= 1) {
            q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
            cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        }
        const int W = team >> 5;
        if (fend && ku0 == 0) {
            if ((lit & 31) == 0)
                wi_commit(it, ts.wi[team_idx], kk, W, frame, q, cnt);
            ++kk;
        } else if ((lit & 31) == 0) {
            // part of a cut frame: the warp's Q, N_eff and group rows into the slot
            unsigned long long *pq = reinterpret_cast<unsigned long long *>(it.rb);
            int32_t *pcnt = reinterpret_cast<int32_t *>(pq + K);
            int32_t *prow = pcnt + K;
            const int64_t slot = (((int64_t)frame * NG + 1) * K + TT - 1) / TT;
            if (SK_DBG_SLOT(it, slot)) {
                atomicAdd(pq + slot, (unsigned long long)q);
                atomicAdd(pcnt + slot, cnt);
                __threadfence();
                const int part = ku - ku0;
                if (atomicAdd(prow + slot, part) + part == NG * W) {
                    __threadfence();
                    const int64_t Q = (int64_t)atomicExch(pq + slot, 0ull);
                    const int32_t C = atomicExch(pcnt + slot, 0);
                    atomicExch(prow + slot, 0);
                    write_frame(it, frame, Q, C);
                }
            }
        }
        __syncwarp();
        q = 0;
        cnt = 0;
        if (fend) {
            ku = 0;
            ++frame;
        }
        ku0 = ku;
    }
}

}  // namespace sk
