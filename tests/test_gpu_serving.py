"""Serving through hz_submit / hz_poll: frames from several streams, submitted
concurrently, batched by the scheduler; every result must equal the result
of the same frames processed alone (in order, same per-stream airlight
chain), and match the FP64 oracle within 1 LSB."""
import threading

import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, oracle_params, torch, u8_diff

pytestmark = pytest.mark.gpu

STREAMS = [(320, 240, 0), (200, 150, 0), (256, 192, 2)]  # (W, H, flags: 2 = guided)
NF = 5


def _frames(W, H, seed):
    return hazegen.make_sequence(W, H, NF, seed=seed, period=NF)


def _serve(m, ctx, seqs, host_io=True):
    sids = [m.hz_open_stream(ctx, W, H, fl) for (W, H, fl) in STREAMS]
    outs, tickets = [], [[] for _ in STREAMS]
    ins = []
    for k, seq in enumerate(seqs):
        if host_io:
            ins.append(torch.from_numpy(seq).pin_memory())
            outs.append(torch.zeros_like(ins[-1]).pin_memory())
        else:
            ins.append(torch.from_numpy(seq).cuda())
            outs.append(torch.zeros_like(ins[-1]))

    def submitter(k):
        for f in range(NF):
            tickets[k].append(m.hz_submit(ctx, sids[k], ins[k][f], outs[k][f],
                                          m.HZ_IO_HOST if host_io else 0))

    th = [threading.Thread(target=submitter, args=(k,)) for k in range(len(STREAMS))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    infos = [[None] * NF for _ in STREAMS]
    for k in range(len(STREAMS)):
        for f in range(NF):
            st, info = m.hz_poll(ctx, tickets[k][f], -1)
            assert st == m.HZ_OK
            infos[k][f] = info.as_dict()
    torch.cuda.synchronize()
    return sids, [o.cpu().numpy() for o in outs], infos, tickets


@pytest.mark.parametrize("host_io", [True, False])
def test_served_results_equal_alone(host_io):
    kw = dict(airlight_ema=0.9, gf_radius=8)
    seqs = [_frames(W, H, 40 + k) for k, (W, H, _) in enumerate(STREAMS)]
    with context(**kw) as (m, ctx):
        sids, outs, infos, tickets = _serve(m, ctx, seqs, host_io)
        st = m.hz_get_server_stats(ctx)
        assert st.frames_done == NF * len(STREAMS)
        assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
        # collected tickets are gone
        with pytest.raises(m.HzError):
            m.hz_poll(ctx, tickets[0][0], 0)
        with pytest.raises(m.HzError):
            m.hz_poll(ctx, 10 ** 9, 0)
    # the same frames alone, one batch call per frame, on a fresh context
    with context(**kw) as (m, ctx):
        sids2 = [m.hz_open_stream(ctx, W, H, fl) for (W, H, fl) in STREAMS]
        for k, (W, H, fl) in enumerate(STREAMS):
            for f in range(NF):
                a = torch.from_numpy(seqs[k][f]).cuda()
                b = torch.empty_like(a)
                info = m.hz_dehaze_batch(ctx, [a], [b], stream_ids=[sids2[k]], guided=[bool(fl & 2)],
                                         want_info=True)[0]
                np.testing.assert_array_equal(outs[k][f], b.cpu().numpy())
                assert infos[k][f]["A"] == list(info.A)
    # and every stream against the oracle's sequence (the guided stream in
    # image mode, its airlight smoothed across frames like the others)
    for k, (W, H, fl) in enumerate(STREAMS):
        ref = _oracle_stream(seqs[k], oracle_params(**kw), bool(fl & 2))
        for f in range(NF):
            mx, exact = u8_diff(outs[k][f], ref[f].out)
            assert mx <= 1 and exact > 0.99
            assert infos[k][f]["T"] == ref[f].T and infos[k][f]["cut_index"] == ref[f].cut_index
            assert infos[k][f]["S"] == [int(v) for v in ref[f].S]


def _oracle_stream(seq, prm, guided):
    res, A_prev = [], None
    for I in seq:
        r = O.dehaze_frame(I, prm, A_prev=A_prev, guided=guided)
        res.append(r)
        A_prev = r.A
    return res


def test_served_fp16_guided_stream_matches_oracle():
    """A served guided stream with FP16 planes (the 4K serving form) against
    the oracle's image mode: selection bit-exact, output within the FP16
    bound of the image-mode tests."""
    from tests.test_gpu_image import FP16_MAX_LSB, FP16_EXACT_MIN
    kw = dict(airlight_ema=0.9, gf_radius=12, precision="fp16")
    W, H = 384, 216
    seq = _frames(W, H, 61)
    with context(**kw) as (m, ctx):
        sid = m.hz_open_stream(ctx, W, H, m.HZ_GUIDED)
        a = torch.from_numpy(seq).pin_memory()
        b = torch.zeros_like(a).pin_memory()
        tickets = [m.hz_submit(ctx, sid, a[f], b[f], m.HZ_IO_HOST) for f in range(NF)]
        infos = []
        for t in tickets:
            st, info = m.hz_poll(ctx, t, -1)
            assert st == m.HZ_OK
            infos.append(info.as_dict())
        out = b.numpy().copy()
    ref = _oracle_stream(seq, oracle_params(**kw), True)
    for f in range(NF):
        assert infos[f]["T"] == ref[f].T and infos[f]["cut_index"] == ref[f].cut_index
        mx, exact = u8_diff(out[f], ref[f].out)
        assert mx <= FP16_MAX_LSB and exact > FP16_EXACT_MIN, (mx, exact)


def test_admission_by_memory_budget():
    m = pytest.importorskip("paper_2512_16609_gb300")
    from tests.gpu_util import hzp
    m = hzp()
    ctx = m.hz_create(m.params(), 0, 64 << 20)  # 64 MiB budget
    try:
        sid = m.hz_open_stream(ctx, 640, 480)
        with pytest.raises(m.HzError) as e:
            m.hz_open_stream(ctx, 3840, 2160, m.HZ_GUIDED)
        assert e.value.status == m.HZ_EBUSY
        m.hz_close_stream(ctx, sid)
        with pytest.raises(m.HzError):
            m.hz_close_stream(ctx, sid)
    finally:
        m.hz_destroy(ctx)


def test_poll_timeout_and_state_roundtrip():
    with context(airlight_ema=0.5) as (m, ctx):
        W, H = 160, 120
        sid = m.hz_open_stream(ctx, W, H)
        seq = _frames(W, H, 7)
        a = torch.from_numpy(seq).cuda()
        b = torch.empty_like(a)
        t0 = m.hz_submit(ctx, sid, a[0], b[0])
        st, _ = m.hz_poll(ctx, t0, -1)
        assert st == m.HZ_OK
        state = m.hz_stream_get_state(ctx, sid)
        assert len(state) == m.HZ_STREAM_STATE_BYTES
        t1 = m.hz_submit(ctx, sid, a[1], b[1])
        st, _ = m.hz_poll(ctx, t1, 2_000_000)
        assert st == m.HZ_OK
        m.hz_stream_set_state(ctx, sid, state)  # rewind to after frame 0
        t2 = m.hz_submit(ctx, sid, a[1], b[2])
        assert m.hz_poll(ctx, t2, -1)[0] == m.HZ_OK
        torch.cuda.synchronize()
        assert torch.equal(b[1], b[2])


def test_served_batches_overlap_on_the_device():
    """Continuous batching overlaps work on the device: with frames of six
    1080p streams submitted faster than they are processed, later batches'
    input copies or compute start (timed CUDA events) before earlier
    batches' outputs are back; every result still equals the frame
    processed alone."""
    W, H, NS, NFR = 1920, 1080, 6, 6
    seqs = [hazegen.make_sequence(W, H, NFR, seed=90 + k, period=NFR) for k in range(NS)]
    with context(airlight_ema=0.9) as (m, ctx):
        sids = [m.hz_open_stream(ctx, W, H) for _ in range(NS)]
        ins = [torch.from_numpy(s).pin_memory() for s in seqs]
        outs = [torch.zeros_like(x).pin_memory() for x in ins]
        tickets = []
        for f in range(NFR):
            for k in range(NS):
                tickets.append(m.hz_submit(ctx, sids[k], ins[k][f], outs[k][f], m.HZ_IO_HOST))
        for t in tickets:
            assert m.hz_poll(ctx, t, -1)[0] == m.HZ_OK
        st = m.hz_get_server_stats(ctx)
        assert st.frames_done == NS * NFR
        assert st.batches < NS * NFR          # frames were batched
        assert st.overlapped_batches >= 1, (st.batches, st.overlapped_batches)
        # alone: the same frames through the video call, stream by stream
        for k in (0, NS - 1):
            a = torch.from_numpy(seqs[k]).cuda()
            b = torch.empty_like(a)
            m.hz_dehaze_video(ctx, a, b)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(outs[k].numpy(), b.cpu().numpy())
