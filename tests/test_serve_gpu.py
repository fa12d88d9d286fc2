"""Continuous-batching server (hb_server_*): every frame's result is the same alone and in
a mixed batch, admission follows the memory budget, full streams push back, batches form
under load."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1706_07263_gb300 import Context, HbError, Server, build, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
GRID = dict(n0=64, n1=64, lo0=0.0, hi0=150.0, lo1=0.0, hi1=100.0, sigma_l=0.02)
LAM = 1e-3
# (width, height, levels): mixed sizes and levels, ragged sizes included
STREAMS = [(160, 120, 2), (320, 240, 3), (200, 150, 4), (96, 80, 0), (250, 130, 1), (640, 480, 3)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _frames(A, w, h, n, seed):
    return [synth.make_frame(seed + k, h, w, A, 6, max(3.0, w / 30), max(6.0, w / 8), 0.01, "u8").rgb
            for k in range(n)]


def _alone(A, frame, levels):
    h, w, _ = frame.shape
    with Context(A, GRID, levels, LAM, w, h, "u8") as ctx:
        f = torch.from_numpy(frame).to(DEV)
        thb = torch.empty((h, w), dtype=torch.float32, device=DEV)
        so2 = torch.empty_like(thb)
        ctx.estimate(f, thb, so2)
        torch.cuda.synchronize()
        return thb.cpu().numpy(), so2.cpu().numpy()


def _collect(srv, n, timeout_s=30.0):
    out = {}
    t0 = time.time()
    while len(out) < n and time.time() - t0 < timeout_s:
        for r in srv.poll(64, wait_us=2000):
            out[r["tag"]] = (r["thb"].copy(), r["so2"].copy(), r["latency_ms"], r["stream"])
            srv.release(r["stream"], r["slot"])
    return out


def test_each_result_is_the_same_alone_and_in_the_mix():
    A = synth.make_mixing(3).A
    frames = {}
    with Server(A, GRID, LAM, max_batch=16, batch_lowpass_pixels=400_000) as srv:
        sids = [srv.open_stream(w, h, lv, slots=4) for (w, h, lv) in STREAMS]
        srv.pause(True)                          # let a burst queue up, then batch it
        tag = 0
        for k in range(3):                      # three rounds of one frame per stream, back to back
            for sid, (w, h, lv) in zip(sids, STREAMS):
                fr = _frames(A, w, h, 1, 1000 * sid + 17 * k)[0]
                frames[tag] = (fr, lv)
                assert srv.submit(sid, fr, tag)
                tag += 1
        srv.pause(False)
        got = _collect(srv, tag)
        stats = srv.stats()
    assert len(got) == tag
    assert stats["frames"] == tag and stats["max_batch_frames"] == 16     # 18 frames: batches of 16 and 2
    for t, (fr, lv) in frames.items():
        thb_a, so2_a = _alone(A, fr, lv)
        thb_m, so2_m, _, _ = got[t]
        rel = np.abs(thb_m - thb_a) / np.maximum(np.abs(thb_a), 1.0)
        assert rel.max() <= 1e-4, (t, rel.max())
        mask = thb_a >= 1.0
        assert np.abs(so2_m - so2_a)[mask].max(initial=0.0) <= 1e-3
    # and one mixed-batch result against the FP64 oracle
    fr, lv = frames[5]
    ref = oracle.estimate(fr, A, GRID, lv, LAM)
    rel = np.abs(got[5][0] - ref["thb"]) / np.maximum(np.abs(ref["thb"]), 1.0)
    assert rel.max() <= 1e-4


def test_admission_follows_the_budget():
    A = synth.make_mixing(4).A
    slot_bytes = 640 * 480 * 3 + 2 * 640 * 480 * 4
    with Server(A, GRID, LAM, max_batch=4, batch_lowpass_pixels=50_000) as probe:
        scratch = probe.stats()["bytes_in_use"]          # the batches' scratch, before any stream
    assert scratch >= 50_000 * (16 + 8 + 4 * 3 * 8 + 4)
    budget = scratch + 3 * 2 * slot_bytes + 1000          # room for three 2-slot streams
    with Server(A, GRID, LAM, budget_bytes=budget, max_batch=4, batch_lowpass_pixels=50_000) as srv:
        ids = [srv.open_stream(640, 480, 3, slots=2) for _ in range(3)]
        with pytest.raises(HbError) as e:
            srv.open_stream(640, 480, 3, slots=2)
        assert e.value.status == 5                       # HB_ERR_BUDGET
        used = srv.stats()["bytes_in_use"]
        assert used <= budget
        srv.close_stream(ids[1])
        assert srv.stats()["bytes_in_use"] == used - 2 * slot_bytes
        srv.open_stream(640, 480, 3, slots=2)            # fits again
        with pytest.raises(HbError) as e:
            srv.open_stream(4096, 4096, 1, slots=1)      # low pass larger than a batch
        assert e.value.status == 2


def test_full_stream_pushes_back_until_released():
    A = synth.make_mixing(5).A
    fr = _frames(A, 128, 96, 1, 3)[0]
    with Server(A, GRID, LAM, max_batch=4, batch_lowpass_pixels=100_000) as srv:
        sid = srv.open_stream(128, 96, 2, slots=1)
        assert srv.submit(sid, fr, 1)
        assert not srv.submit(sid, fr, 2)                # the only slot is busy
        got = []
        t0 = time.time()
        while not got and time.time() - t0 < 10:
            got = srv.poll(4, wait_us=5000)
        assert len(got) == 1 and got[0]["tag"] == 1
        assert not srv.submit(sid, fr, 3)                # completed but not released yet
        srv.release(sid, got[0]["slot"])
        assert srv.submit(sid, fr, 4)
        _collect(srv, 1)


def test_sequential_mode_runs_one_frame_per_batch():
    A = synth.make_mixing(6).A
    with Server(A, GRID, LAM, max_batch=1, batch_lowpass_pixels=100_000, sequential=True) as srv:
        sid = srv.open_stream(160, 120, 2, slots=8)
        for k, fr in enumerate(_frames(A, 160, 120, 6, 9)):
            assert srv.submit(sid, fr, k)
        got = _collect(srv, 6)
        st = srv.stats()
    assert len(got) == 6 and st["batches"] == 6 and st["max_batch_frames"] == 1


def test_drain_waits_for_every_frame_and_times_out_while_held():
    A = synth.make_mixing(7).A
    frames = _frames(A, 200, 150, 3, 21)
    with Server(A, GRID, LAM, max_batch=4, batch_lowpass_pixels=100_000) as srv:
        sid = srv.open_stream(200, 150, 2, slots=4)
        srv.drain(0)                                      # nothing submitted: idle at once
        srv.pause(True)
        for k, fr in enumerate(frames):
            assert srv.submit(sid, fr, k)
        t0 = time.time()
        with pytest.raises(HbError) as e:
            srv.drain(20)                                 # held frames cannot complete
        assert e.value.status == 6                        # HB_ERR_TIMEOUT
        assert 0.015 <= time.time() - t0 < 5.0
        assert srv.stats()["queued"] == 3                 # the timeout left every frame queued
        srv.pause(False)
        srv.drain(10_000)
        assert srv.stats()["queued"] == 0
        got = srv.poll(8, wait_us=0)                      # all three ready without waiting
        assert sorted(r["tag"] for r in got) == [0, 1, 2]
        for r in got:
            srv.release(r["stream"], r["slot"])
