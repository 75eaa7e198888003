"""The continuous-batching server: results equal the oracle alone and in the
mix, the running per-input power state follows the oracle's served path,
checkpoint/resume continues identically, admission refuses what does not fit,
and a full ring answers BUSY.  Failures are made on the host."""

import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402
from oracle import digitisation as dg  # noqa: E402
from oracle import served  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _stream_data(k, N, M, T):
    s = synth.sub_seed(3, k)
    ds = synth.Dataset(n_frames=T, M=M, N=N, seed=s, rfi=synth.rfi_plan(s, T, 0.1, 0.05))
    return ds, ds.generate_cpu()


def _run_streams(server, specs, datas, interleave=True, ring=8, stateful=True, tables=None):
    """Submit every stream's frames (interleaved across streams, or one stream
    after another) and collect (sk, mask) per stream in frame order."""
    ids = []
    for (N, M), (ds, x), e in zip(specs, datas, tables):
        ids.append(sk.sk_stream_open(server, N, M, ring_frames=ring, n_sigma=3.0,
                                     flags=sk.SK_RUNNING_OFFSET if stateful else 0,
                                     offset_table=e))
    out = [([], []) for _ in specs]
    order = []
    T = max(x.shape[0] for _, x in datas)
    if interleave:
        for f in range(T):
            for j, (_, x) in enumerate(datas):
                if f < x.shape[0]:
                    order.append((j, f))
    else:
        for j, (_, x) in enumerate(datas):
            order += [(j, f) for f in range(x.shape[0])]
    pending = [[] for _ in specs]
    for j, f in order:
        x = datas[j][1]
        while True:
            try:
                t = sk.sk_stream_submit(server, ids[j], x[f], f)
                break
            except sk.SkError as e:
                assert e.status == sk.SK_ERR_BUSY
                skv, m = sk.sk_ticket_wait(server, pending[j].pop(0))
                out[j][0].append(skv)
                out[j][1].append(m)
        pending[j].append(t)
    for j in range(len(specs)):
        for t in pending[j]:
            skv, m = sk.sk_ticket_wait(server, t)
            out[j][0].append(skv)
            out[j][1].append(m)
    for i in ids:
        sk.sk_stream_close(server, i)
    return [(np.array(a, dtype=np.float32), np.array(b, dtype=np.uint8)) for a, b in out]


@pytest.mark.parametrize("split", ["1", "0"])
def test_served_results_match_oracle_alone_and_in_mix(split, monkeypatch):
    """Both served launch shapes: small batches with each frame's rows split over a
    CTA (default) and teams on different frames (SK_SERVER_SPLIT=0)."""
    _need_gpu()
    monkeypatch.setenv("SK_SERVER_SPLIT", split)
    specs = [(2048, 256), (256, 256), (256, 256), (2048, 256), (512, 128)]
    T = 30
    datas = [_stream_data(k, N, M, T) for k, (N, M) in enumerate(specs)]
    tables = [dg.offset_table(M) for (_, M) in specs]
    wants = [served.served_flags(x, M, N, e) for (N, M), (_, x), e in zip(specs, datas, tables)]
    server = sk.sk_server_create(0, 8 << 30)
    try:
        mix = _run_streams(server, specs, datas, True, tables=tables)
        alone = [_run_streams(server, [s], [d], False, tables=[e])[0]
                 for s, d, e in zip(specs, datas, tables)]
        st = sk.sk_server_stats(server)
    finally:
        sk.sk_server_destroy(server)
    for w, m, a in zip(wants, mix, alone):
        assert np.array_equal(m[1], w["mask"])
        assert np.array_equal(m[0].view(np.uint32), w["sk"].view(np.uint32))
        assert np.array_equal(a[0].view(np.uint32), m[0].view(np.uint32))
        assert np.array_equal(a[1], m[1])
    assert st["frames_done"] == 2 * len(specs) * T
    assert st["latency_p99_us"] >= st["latency_p50_us"] > 0


def test_stateless_stream_matches_plain_flag():
    _need_gpu()
    N, M, T = 256, 256, 20
    ds, x = _stream_data(9, N, M, T)
    delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
    want = oracle.flag(x, M, N, 3.0, delta)
    server = sk.sk_server_create(0, 1 << 30)
    try:
        sid = sk.sk_stream_open(server, N, M, ring_frames=4, n_sigma=3.0, mean_offset=delta)
        tickets = []
        got = []
        for f in range(T):
            while True:
                try:
                    tickets.append(sk.sk_stream_submit(server, sid, x[f], f))
                    break
                except sk.SkError as e:
                    assert e.status == sk.SK_ERR_BUSY
                    got.append(sk.sk_ticket_wait(server, tickets.pop(0)))
        got += [sk.sk_ticket_wait(server, t) for t in tickets]
        sk.sk_stream_close(server, sid)
    finally:
        sk.sk_server_destroy(server)
    assert np.array_equal(np.array([m for _, m in got], dtype=np.uint8), want["mask"])
    assert np.array_equal(np.array([s for s, _ in got], dtype=np.float32).view(np.uint32),
                          want["sk"].view(np.uint32))


@pytest.mark.parametrize("N,M", [(2048, 128), (256, 256), (100, 64), (37, 50), (2048, 48),
                                 (4096, 1024)])
def test_input_major_stream_matches_time_major_stream(N, M):
    """The same frames served as [input][t] and as [t][input] give identical results,
    and the time-major stream matches the served-state oracle."""
    _need_gpu()
    T = 24
    ds, x = _stream_data(21, N, M, T)
    xi = np.ascontiguousarray(x.reshape(T, M, N).transpose(0, 2, 1).reshape(T, -1))
    e = dg.offset_table(M)
    want = served.served_flags(x, M, N, e)
    server = sk.sk_server_create(0, 2 << 30)
    try:
        ids = [sk.sk_stream_open(server, N, M, ring_frames=T, flags=sk.SK_RUNNING_OFFSET,
                                 offset_table=e, layout=lay) for lay in (0, 1)]
        tickets = [[sk.sk_stream_submit(server, i, d[f], f) for f in range(T)]
                   for i, d in zip(ids, (x, xi))]
        got = [[sk.sk_ticket_wait(server, t, 10_000_000) for t in ts] for ts in tickets]
        for i in ids:
            sk.sk_stream_close(server, i)
    finally:
        sk.sk_server_destroy(server)
    sk_t = np.array([a for a, _ in got[0]], dtype=np.float32)
    sk_i = np.array([a for a, _ in got[1]], dtype=np.float32)
    assert np.array_equal(np.array([m for _, m in got[0]], dtype=np.uint8), want["mask"])
    assert np.array_equal(sk_t.view(np.uint32), want["sk"].view(np.uint32))
    assert np.array_equal(sk_i.view(np.uint32), sk_t.view(np.uint32))
    assert [m for _, m in got[1]] == [m for _, m in got[0]]


@pytest.mark.parametrize("M", [64, 256, 1024])
def test_plan_offset_table_matches_oracle_model(M):
    """A running-offset plan without a caller table builds e[] from its own App. B model;
    it must equal the oracle's table (entries may differ by one where rounding of
    delta * 2^32 (M-1)/(M+1) falls on the other side of a half)."""
    _need_gpu()
    plan = sk.sk_plan_create(256, M, flags=sk.SK_RUNNING_OFFSET)
    try:
        e = sk.sk_plan_offset_table(plan)
    finally:
        sk.sk_plan_destroy(plan)
    want = dg.offset_table(M)
    d = np.abs(e - want)
    assert d.max() <= 1 and (d == 0).mean() > 0.99


def test_checkpoint_resume_continues_identically():
    _need_gpu()
    N, M, T = 512, 256, 24
    ds, x = _stream_data(11, N, M, T)
    e = dg.offset_table(M)
    want = served.served_flags(x, M, N, e)
    server = sk.sk_server_create(0, 1 << 30)
    try:
        a = sk.sk_stream_open(server, N, M, ring_frames=4, flags=sk.SK_RUNNING_OFFSET,
                              offset_table=e)
        first = []
        for f in range(10):
            t = sk.sk_stream_submit(server, a, x[f], f)
            first.append(sk.sk_ticket_wait(server, t))
        sk.sk_stream_drain(server, a)
        state = sk.sk_stream_get_state(server, a)
        sk.sk_stream_close(server, a)
        b = sk.sk_stream_open(server, N, M, ring_frames=4, flags=sk.SK_RUNNING_OFFSET,
                              offset_table=e)
        sk.sk_stream_set_state(server, b, state)
        second = []
        for f in range(10, T):
            t = sk.sk_stream_submit(server, b, x[f], f)
            second.append(sk.sk_ticket_wait(server, t))
        sk.sk_stream_drain(server, b)
        final = sk.sk_stream_get_state(server, b)
        sk.sk_stream_close(server, b)
    finally:
        sk.sk_server_destroy(server)
    got = np.array([m for _, m in first + second], dtype=np.uint8)
    assert np.array_equal(got, want["mask"])
    P = np.frombuffer(final, dtype=np.uint32)[2:]
    assert np.array_equal(P.astype(np.int64), want["P"])


def test_admission_budget_and_ring_full():
    _need_gpu()
    N, M = 2048, 256
    fb = N * M
    server = sk.sk_server_create(0, 10 * fb)
    try:
        a = sk.sk_stream_open(server, N, M, ring_frames=4)
        with pytest.raises(sk.SkError) as e:
            sk.sk_stream_open(server, N, M, ring_frames=8)
        assert e.value.status == sk.SK_ERR_BUSY
        frame = np.full(fb, 0x99, dtype=np.uint8)
        # fill the ring faster than it drains, host-side: BUSY must come back
        busy = 0
        tickets = []
        for f in range(200):
            try:
                tickets.append(sk.sk_stream_submit(server, a, frame, f))
            except sk.SkError as err:
                assert err.status == sk.SK_ERR_BUSY
                busy += 1
                sk.sk_ticket_wait(server, tickets.pop(0))
        for t in tickets:
            sk.sk_ticket_wait(server, t)
        with pytest.raises(sk.SkError) as e:
            sk.sk_ticket_wait(server, 10 ** 9, 0)
        assert e.value.status == sk.SK_ERR_INVALID_ARG
        sk.sk_stream_close(server, a)
        # its ring share is returned: a second stream of the same share fits now
        b = sk.sk_stream_open(server, N, M, ring_frames=4)
        sk.sk_stream_close(server, b)
        st = sk.sk_server_stats(server)
        assert st["rejected"] >= 1 + busy
    finally:
        sk.sk_server_destroy(server)


def test_admission_by_device_free_memory():
    """Admission takes the lesser of the caller's budget and the device's real free
    memory (cudaMemGetInfo at each sk_stream_open, less the server's 256 MiB headroom):
    with a budget far above the device, a stream is refused while other allocations
    hold the device's memory, and admitted once they are released."""
    _need_gpu()
    N, M = 2048, 256
    server = sk.sk_server_create(0, 1 << 40)
    hold = []
    try:
        a = sk.sk_stream_open(server, N, M, ring_frames=4)
        # hold device memory until less than the headroom is free (plain allocations)
        step = 1 << 30
        while True:
            free = torch.cuda.mem_get_info()[0]
            if free < (160 << 20):
                break
            want = min(step, free - (96 << 20))
            if want < (8 << 20):
                break
            try:
                hold.append(torch.empty(want, dtype=torch.uint8, device="cuda:0"))
            except RuntimeError:
                step //= 4
                if step < (8 << 20):
                    break
        assert torch.cuda.mem_get_info()[0] < (256 << 20)
        with pytest.raises(sk.SkError) as e:
            sk.sk_stream_open(server, N, M, ring_frames=4)
        assert e.value.status == sk.SK_ERR_BUSY
        assert "free" in e.value.message
        hold.clear()
        torch.cuda.empty_cache()
        b = sk.sk_stream_open(server, N, M, ring_frames=4)
        # the admitted streams still serve frames
        frame = np.full(N * M, 0x99, dtype=np.uint8)
        for sid in (a, b):
            t = sk.sk_stream_submit(server, sid, frame, 0)
            sk.sk_ticket_wait(server, t)
        sk.sk_stream_close(server, a)
        sk.sk_stream_close(server, b)
        assert sk.sk_server_stats(server)["rejected"] >= 1
    finally:
        hold.clear()
        torch.cuda.empty_cache()
        sk.sk_server_destroy(server)


def test_ticket_timeout_and_concurrent_submitters():
    _need_gpu()
    N, M, T = 256, 256, 40
    server = sk.sk_server_create(0, 1 << 30)
    errors = []
    try:
        datas = [_stream_data(20 + k, N, M, T) for k in range(4)]
        wants = [oracle.flag(x, M, N, 3.0, 0.0)["mask"] for _, x in datas]
        results = [None] * 4

        def worker(k):
            try:
                sid = sk.sk_stream_open(server, N, M, ring_frames=6)
                out = []
                for f in range(T):
                    t = sk.sk_stream_submit(server, sid, datas[k][1][f], f)
                    out.append(sk.sk_ticket_wait(server, t, 10_000_000)[1])
                sk.sk_stream_close(server, sid)
                results[k] = np.array(out, dtype=np.uint8)
            except Exception as ex:  # noqa: BLE001
                errors.append(ex)

        th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join(120)
        assert not errors, errors
        for r, w in zip(results, wants):
            assert np.array_equal(r, w)
        # a wait with a zero limit on a ticket whose frame cannot have run yet times out
        sid = sk.sk_stream_open(server, N, M, ring_frames=2)
        t0 = time.time()
        t = sk.sk_stream_submit(server, sid, datas[0][1][0], 0)
        try:
            sk.sk_ticket_wait(server, t, 0)          # done already, or times out
        except sk.SkError as e:
            assert e.status == sk.SK_ERR_TIMEOUT
            sk.sk_ticket_wait(server, t, 10_000_000)  # a timed-out ticket stays valid
        assert time.time() - t0 < 30
        sk.sk_stream_close(server, sid)
    finally:
        sk.sk_server_destroy(server)


def test_ring_wraps_many_times_with_changing_data():
    """A small ring reused many times over: every result must belong to the frame
    just submitted (no stale bytes from an earlier pass over the ring)."""
    _need_gpu()
    N, M, T = 2048, 256, 48
    ds, x = _stream_data(31, N, M, T)
    e = dg.offset_table(M)
    want = served.served_flags(x, M, N, e)
    server = sk.sk_server_create(0, 8 * N * M)   # ring = 4 frames
    try:
        sid = sk.sk_stream_open(server, N, M, ring_frames=3, flags=sk.SK_RUNNING_OFFSET,
                                offset_table=e)
        got_sk, got_m, pend = [], [], []
        for f in range(T):
            while True:
                try:
                    pend.append(sk.sk_stream_submit(server, sid, x[f], f))
                    break
                except sk.SkError as err:
                    assert err.status == sk.SK_ERR_BUSY
                    a, b = sk.sk_ticket_wait(server, pend.pop(0))
                    got_sk.append(a)
                    got_m.append(b)
        for t in pend:
            a, b = sk.sk_ticket_wait(server, t)
            got_sk.append(a)
            got_m.append(b)
        sk.sk_stream_close(server, sid)
    finally:
        sk.sk_server_destroy(server)
    assert np.array_equal(np.array(got_m, dtype=np.uint8), want["mask"])
    assert np.array_equal(np.array(got_sk, dtype=np.float32).view(np.uint32),
                          want["sk"].view(np.uint32))


def test_running_mu_streams_match_oracle():
    """SK_RUNNING_MU: frames normalised by the running power of each input; SK and
    masks equal the oracle's running-mu statement, including a power step."""
    _need_gpu()
    M, N, T = 256, 128, 24
    sig = np.full(N, 1.6)
    ds1 = synth.Dataset(n_frames=T, M=M, N=N, seed=41, sigma=sig,
                        rfi=[synth.RFI(9, "cw", 3.0)])
    sig2 = sig.copy()
    sig2[: N // 2] *= np.sqrt(2.0)
    ds2 = synth.Dataset(n_frames=4, M=M, N=N, seed=42, sigma=sig2)
    x = np.concatenate([ds1.generate_cpu(), ds2.generate_cpu()])
    e = dg.offset_table(M)
    want = served.served_flags(x, M, N, e, running_mu=True)
    server = sk.sk_server_create(0, 1 << 30)
    try:
        sid = sk.sk_stream_open(server, N, M, ring_frames=4, flags=sk.SK_RUNNING_MU,
                                offset_table=e)
        got = [sk.sk_ticket_wait(server, sk.sk_stream_submit(server, sid, x[f], f))
               for f in range(x.shape[0])]
        sk.sk_stream_drain(server, sid)
        P = np.frombuffer(sk.sk_stream_get_state(server, sid), dtype=np.uint32)[2:]
        sk.sk_stream_close(server, sid)
    finally:
        sk.sk_server_destroy(server)
    assert np.array_equal(np.array([m for _, m in got], dtype=np.uint8), want["mask"])
    assert np.array_equal(np.array([v for v, _ in got], dtype=np.float32).view(np.uint32),
                          want["sk"].astype(np.float32).view(np.uint32))
    assert np.array_equal(P.astype(np.int64), want["P"])
    assert want["mask"][9] == 1 and want["mask"][T] == 1


def test_close_and_destroy_with_work_outstanding():
    """Closing a stream waits for its frames; submits to a closed or unknown stream are
    refused; a server destroyed with tickets still uncollected shuts down cleanly."""
    _need_gpu()
    N, M = 256, 256
    ds, x = _stream_data(50, N, M, 12)
    server = sk.sk_server_create(0, 1 << 30)
    sid = sk.sk_stream_open(server, N, M, ring_frames=8, flags=sk.SK_RUNNING_OFFSET)
    tickets = [sk.sk_stream_submit(server, sid, x[f], f) for f in range(8)]
    sk.sk_stream_close(server, sid)                  # waits for the 8 frames
    for t in tickets:                                # their results are still collectable
        skv, m = sk.sk_ticket_wait(server, t, 5_000_000)
        assert m in (0, 1)
    for bad in (sid, 12345):
        with pytest.raises(sk.SkError) as e:
            sk.sk_stream_submit(server, bad, x[0], 0)
        assert e.value.status == sk.SK_ERR_INVALID_ARG
    with pytest.raises(sk.SkError) as e:
        sk.sk_stream_close(server, sid)
    assert e.value.status == sk.SK_ERR_CLOSED
    sid2 = sk.sk_stream_open(server, N, M, ring_frames=8)
    for f in range(6):
        sk.sk_stream_submit(server, sid2, x[f], f)   # never collected
    sk.sk_server_destroy(server)
    # the device is still usable afterwards
    plan = sk.sk_plan_create(N, M)
    d = torch.from_numpy(x[:2].reshape(-1)).to("cuda")
    mask = torch.empty(2, dtype=torch.uint8, device="cuda")
    sk.sk_flag(plan, d, 2, None, mask)
    torch.cuda.synchronize()
    sk.sk_plan_destroy(plan)


def test_injected_launch_failure_fails_tickets_and_device_stays_usable(monkeypatch):
    """Failure detection with the fault made on the host: SK_SERVER_INJECT_FAULT=3 makes
    the third launch fail before any CUDA call.  The frames launched before it complete;
    its frame, the frames queued behind it and later submits report SK_ERR_CUDA instead
    of waiting; the server shuts down; a fresh plan then runs on the same device."""
    _need_gpu()
    N, M, T = 256, 256, 12
    ds, x = _stream_data(33, N, M, T)
    monkeypatch.setenv("SK_SERVER_INJECT_FAULT", "3")
    server = sk.sk_server_create(0, 1 << 30)
    monkeypatch.delenv("SK_SERVER_INJECT_FAULT")
    ok, failed = 0, 0
    try:
        sid = sk.sk_stream_open(server, N, M, ring_frames=T, flags=sk.SK_RUNNING_OFFSET)
        tickets = []
        for f in range(T):
            try:
                tickets.append(sk.sk_stream_submit(server, sid, x[f], f))
            except sk.SkError as e:
                assert e.status == sk.SK_ERR_CUDA
                failed += 1
        for t in tickets:
            try:
                sk.sk_ticket_wait(server, t, 5_000_000)
                ok += 1
            except sk.SkError as e:
                assert e.status == sk.SK_ERR_CUDA, e
                assert "injected" in e.message
                failed += 1
        assert ok == 2 and failed == T - 2
        with pytest.raises(sk.SkError) as e:
            sk.sk_stream_submit(server, sid, x[0], T)
        assert e.value.status == sk.SK_ERR_CUDA
        assert sk.sk_server_stats(server)["frames_done"] == 2   # failed frames not counted
    finally:
        sk.sk_server_destroy(server)
    # the device still runs a fresh plan
    want = oracle.flag(x[:4], M, N)
    plan = sk.sk_plan_create(N, M)
    try:
        d = torch.from_numpy(x[:4].reshape(-1)).to("cuda")
        mask = torch.empty(4, dtype=torch.uint8, device="cuda")
        skv = torch.empty(4, dtype=torch.float32, device="cuda")
        sk.sk_flag(plan, d, 4, skv, mask)
        torch.cuda.synchronize()
    finally:
        sk.sk_plan_destroy(plan)
    assert np.array_equal(mask.cpu().numpy(), want["mask"])


def test_stream_stats_count_frames_flags_and_rejections():
    """sk_stream_stats: frames retired and flagged per stream, BUSY refusals, and
    submit-to-result percentiles; a second stream's counters stay separate."""
    _need_gpu()
    N, M, T = 256, 256, 24
    ds, x = _stream_data(7, N, M, T)
    server = sk.sk_server_create(0, 1 << 30)
    try:
        a = sk.sk_stream_open(server, N, M, ring_frames=1, flags=sk.SK_RUNNING_OFFSET)
        b = sk.sk_stream_open(server, N, M, ring_frames=8)
        masks, busy, pending = [], 0, []
        for f in range(T):
            while True:
                try:
                    pending.append(sk.sk_stream_submit(server, a, x[f], f))
                    break
                except sk.SkError as e:
                    assert e.status == sk.SK_ERR_BUSY
                    busy += 1
                    masks.append(sk.sk_ticket_wait(server, pending.pop(0))[1])
        masks += [sk.sk_ticket_wait(server, t)[1] for t in pending]
        for t in [sk.sk_stream_submit(server, b, x[f], f) for f in range(3)]:
            sk.sk_ticket_wait(server, t)
        sa, sb = sk.sk_stream_stats(server, a), sk.sk_stream_stats(server, b)
        assert sa["frames_done"] == T and sa["frames_flagged"] == sum(masks)
        assert sa["rejected"] == busy and sa["outstanding"] == 0
        assert 0 < sa["latency_p50_us"] <= sa["latency_p99_us"]
        assert sb["frames_done"] == 3 and sb["rejected"] == 0
        sk.sk_stream_close(server, b)
        with pytest.raises(sk.SkError):
            sk.sk_stream_stats(server, b)
    finally:
        sk.sk_server_destroy(server)


def test_submit_by_reference_mixed_with_copies():
    """sk_stream_submit_ref reads frames where they are -- device memory, or page-locked
    host memory -- and mixes in one stream with copied frames: the results follow the
    served oracle frame by frame.  Pageable or misaligned frames are refused."""
    _need_gpu()
    N, M, T = 2048, 256, 12
    ds, x = _stream_data(17, N, M, T)
    e = dg.offset_table(M)
    want = served.served_flags(x, M, N, e)
    d_x = torch.from_numpy(x).to("cuda")
    p_x = torch.from_numpy(x).pin_memory()
    server = sk.sk_server_create(0, 1 << 30)
    try:
        sid = sk.sk_stream_open(server, N, M, ring_frames=T, flags=sk.SK_RUNNING_OFFSET,
                                offset_table=e)
        tickets = []
        for f in range(T):
            if f % 3 == 0:
                tickets.append(sk.sk_stream_submit_ref(server, sid, d_x[f], f))
            elif f % 3 == 1:
                tickets.append(sk.sk_stream_submit_ref(server, sid, p_x[f], f))
            else:
                tickets.append(sk.sk_stream_submit(server, sid, x[f], f))
        got = [sk.sk_ticket_wait(server, t, 10_000_000) for t in tickets]
        for bad in (x[0].ctypes.data, d_x.data_ptr() + 8):
            with pytest.raises(sk.SkError) as err:
                sk.sk_stream_submit_ref(server, sid, bad, T)
            assert err.value.status == sk.SK_ERR_INVALID_ARG
        sk.sk_stream_close(server, sid)
    finally:
        sk.sk_server_destroy(server)
    assert np.array_equal(np.array([m for _, m in got], dtype=np.uint8), want["mask"])
    assert np.array_equal(np.array([v for v, _ in got], dtype=np.float32).view(np.uint32),
                          want["sk"].view(np.uint32))


def test_randomised_streams_against_the_oracle():
    """Seeded stress of the server's bookkeeping: streams of different N, M and flags,
    frames copied or passed by reference (device or page-locked memory), submitted in
    a random interleaving against small rings (BUSY and ring wrap-around), one stream
    closed and another opened half way.  Every result equals the served oracle's."""
    _need_gpu()
    rng = np.random.default_rng(2026)
    shapes = [(2048, 256), (37, 64), (256, 256), (512, 128), (2048, 64), (100, 256)]
    flag_of = [sk.SK_RUNNING_OFFSET, 0, sk.SK_RUNNING_MU, sk.SK_RUNNING_OFFSET, 0,
               sk.SK_RUNNING_OFFSET]
    T = 15
    datas, wants, tables = [], [], []
    for k, ((N, M), fl) in enumerate(zip(shapes, flag_of)):
        ds, x = _stream_data(100 + k, N, M, T)
        e = dg.offset_table(M)
        if fl:
            w = served.served_flags(x, M, N, e, running_mu=bool(fl & sk.SK_RUNNING_MU))
        else:
            w = oracle.flag(x, M, N, 3.0, 0.0)
        datas.append((x, torch.from_numpy(x).to("cuda"), torch.from_numpy(x).pin_memory()))
        wants.append(w)
        tables.append(e)
    server = sk.sk_server_create(0, 64 << 20)      # a 32 MiB ring: it wraps
    try:
        sids = {}
        opened = list(range(5))                    # the sixth opens half way
        for k in opened:
            N, M = shapes[k]
            sids[k] = sk.sk_stream_open(server, N, M, ring_frames=int(rng.integers(2, 5)),
                                        flags=flag_of[k], offset_table=tables[k])
        nxt = {k: 0 for k in range(6)}
        pend = {k: [] for k in range(6)}
        got = {k: [] for k in range(6)}
        closed = set()

        def collect(k):
            got[k].append(sk.sk_ticket_wait(server, pend[k].pop(0), 10_000_000))

        while any(nxt[k] < T for k in sids if k not in closed):
            live = [k for k in sids if k not in closed and nxt[k] < T]
            k = int(rng.choice(live))
            f = nxt[k]
            x, dx, px = datas[k]
            how = int(rng.integers(0, 3))
            try:
                if how == 0:
                    t = sk.sk_stream_submit(server, sids[k], x[f], f)
                elif how == 1:
                    t = sk.sk_stream_submit_ref(server, sids[k], dx[f], f)
                else:
                    t = sk.sk_stream_submit_ref(server, sids[k], px[f], f)
            except sk.SkError as e:
                assert e.status == sk.SK_ERR_BUSY
                if pend[k]:
                    collect(k)
                continue
            pend[k].append(t)
            nxt[k] += 1
            if k == 1 and nxt[k] == T:             # finish and close stream 1 ...
                while pend[k]:
                    collect(k)
                sk.sk_stream_close(server, sids[k])
                closed.add(k)
                N, M = shapes[5]                    # ... and open stream 5 instead
                sids[5] = sk.sk_stream_open(server, N, M, ring_frames=3, flags=flag_of[5],
                                            offset_table=tables[5])
        for k in sids:
            while pend[k]:
                collect(k)
    finally:
        sk.sk_server_destroy(server)
    for k in range(6):
        skv = np.array([v for v, _ in got[k]], dtype=np.float32)
        m = np.array([b for _, b in got[k]], dtype=np.uint8)
        assert np.array_equal(m, wants[k]["mask"]), k
        assert np.array_equal(skv.view(np.uint32), wants[k]["sk"].view(np.uint32)), k
