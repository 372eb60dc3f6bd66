"""Streaming server (GPU): continuous batching, admission by device memory,
running averages, in-order delivery, overflow and bounded waits.

Every streamed result must equal, bit for bit, what ``cg_process`` gives for
the same frame through a separate plan with the same options (the kernels
are deterministic per frame, whatever the batch), whether the stream runs
alone or mixed with other instrument streams.  Faults are made on the host
(a throttled or held scheduler, an injected launch failure); no GPU fault is
provoked.
"""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2307_12988_gb300 as cg
import synth
from tests import workloads

pytestmark = pytest.mark.gpu

GEOMS = {"paper_rate": (synth.PAPER_RATE, dict(snr_db=30.0, center_amp_hz=20e6)),
         "wide": (synth.WIDE, dict(snr_db=30.0, center_amp_hz=20e6)),
         "serve4096": (synth.SERVE_4096, dict(snr_db=30.0, center_amp_hz=20e6))}


def _frames(name, n):
    g, kw = GEOMS[name]
    st = synth.make_stream(g, synth.BASE_SEED + 700 + list(GEOMS).index(name))
    return synth.frames(st, n, **kw)["frames"]


def _plan(name):
    w = workloads.workload(name)
    return cg.Plan(*workloads.plan_args(w))


def _expected(name, frames):
    with _plan(name) as p:
        o = p.process(torch.from_numpy(frames).cuda())
        torch.cuda.synchronize()
        return {k: o[k].cpu().numpy() for k in ("amps", "params", "rss", "iters", "status")}


def _produce(stream, frames, chunk, seq0=1000, pace_s=0.0):
    n = frames.shape[0]
    for s in range(0, n, chunk):
        while True:
            st = stream.push(frames[s:s + chunk], seq0 + s)
            if st == 0:
                break
            time.sleep(1e-4)    # ring full: the consumer catches up
        if pace_s:
            time.sleep(pace_s)


def _consume(stream, n, timeout=60.0):
    recs, amps = [], []
    got, t_end = 0, time.time() + timeout
    while got < n and time.time() < t_end:
        r, a, _ = stream.poll(cap=4096, timeout_s=0.2, want_amps=True)
        if len(r):
            recs.append(r)
            amps.append(a)
            got += len(r)
    return np.concatenate(recs), np.concatenate(amps)


def _check_equal(recs, amps, exp, seq0=1000):
    n = exp["params"].shape[0]
    assert recs.shape[0] == n
    assert np.array_equal(recs["seq"], seq0 + np.arange(n, dtype=np.uint64))
    assert np.array_equal(recs["params"], exp["params"])
    assert np.array_equal(recs["rss"], exp["rss"])
    assert np.array_equal(recs["iters"], exp["iters"])
    assert np.array_equal(recs["status"], exp["status"])
    assert np.array_equal(amps, exp["amps"])
    assert np.all(recs["t_done"] >= recs["t_arrival"])


def _run_stream(server, name, frames, batch, window=1000, chunk=700):
    plan = _plan(name)
    s = cg.Stream(server, plan, ring_bytes=frames.shape[1] * 2 * 4 * batch, batch_frames=batch,
                  max_delay_s=1e-3, avg_window=window)
    out = {}
    prod = threading.Thread(target=_produce, args=(s, frames, chunk))
    prod.start()
    out["recs"], out["amps"] = _consume(s, frames.shape[0])
    prod.join()
    out["stats"] = s.stats()
    out["window"] = s.window()
    s.close()
    plan.close()
    return out


def test_stream_alone_matches_process_and_averages():
    name = "paper_rate"
    frames = _frames(name, 5000)
    exp = _expected(name, frames)
    with cg.Server(1 << 30) as srv:
        out = _run_stream(srv, name, frames, batch=1024, window=1000)
    _check_equal(out["recs"], out["amps"], exp)
    st = out["stats"]
    # (a push that found the ring full was retried; its frames count as dropped once)
    assert st["frames_done"] == 5000 and st["frames_polled"] == 5000 and st["frames_pushed"] == 5000
    assert 0 < st["latency_p50_s"] <= st["latency_p99_s"] <= st["latency_max_s"] * 1.0101
    assert st["admitted"] == 1 and st["batches"] >= 5
    # the last complete window: frames 4000..4999; FP64 means of y and params
    win = out["window"]
    assert win["index"] == 4
    sel = slice(4000, 5000)
    ok = (exp["status"][sel] & 3) == 0
    assert win["count"] == int(ok.sum())
    w = workloads.workload(name)
    inv_ref = (1.0 / w["ref"]).astype(np.float32).astype(np.float64)
    y = exp["amps"][sel][ok].astype(np.float64) * inv_ref
    assert np.allclose(win["mean_y"], y.mean(axis=0), rtol=1e-12, atol=0)
    assert np.allclose(win["mean_params"], exp["params"][sel][ok].astype(np.float64).mean(axis=0),
                       rtol=1e-12, atol=1e-9)
    # and the mean spectrum against the oracle's readout of the same frames
    bins = oracle.tooth_bins(w["geom"].sample_rate, w["geom"].frame_len, w["geom"].tooth_freqs)
    _, y_or = oracle.readout(frames[sel][ok], bins, w["ref"])
    assert np.max(np.abs(win["mean_y"] - y_or.mean(axis=0))) <= 1e-5


def test_three_instruments_in_the_mix_equal_alone():
    sizes = {"paper_rate": 6000, "wide": 2500, "serve4096": 2000}
    batches = {"paper_rate": 1024, "wide": 512, "serve4096": 256}
    frames = {k: _frames(k, n) for k, n in sizes.items()}
    alone = {}
    with cg.Server(1 << 30) as srv:
        for k in sizes:
            alone[k] = _run_stream(srv, k, frames[k], batches[k])
    mixed = {}
    with cg.Server(1 << 30) as srv:
        threads = [threading.Thread(target=lambda k=k: mixed.__setitem__(k, _run_stream(srv, k, frames[k],
                                                                                        batches[k])))
                   for k in sizes]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    for k in sizes:
        a, m = alone[k], mixed[k]
        assert np.array_equal(a["recs"]["params"], m["recs"]["params"]), k
        assert np.array_equal(a["recs"]["status"], m["recs"]["status"]), k
        assert np.array_equal(a["recs"]["iters"], m["recs"]["iters"]), k
        assert np.array_equal(a["amps"], m["amps"]), k
        exp = _expected(k, frames[k])
        _check_equal(m["recs"], m["amps"], exp)


def test_admission_waits_for_device_memory():
    name = "paper_rate"
    frames = _frames(name, 2000)
    exp = _expected(name, frames)
    batch = 512
    per_buffer = batch * (2 * 1100 + 4 * 99 + 24)
    with cg.Server(2 * per_buffer + per_buffer // 2) as srv:       # room for one stream only
        pa, pb = _plan(name), _plan(name)
        sa = cg.Stream(srv, pa, ring_bytes=1100 * 2 * 8 * batch, batch_frames=batch)
        time.sleep(0.05)
        sb = cg.Stream(srv, pb, ring_bytes=1100 * 2 * 8 * batch, batch_frames=batch)
        assert sb.push(frames, 1000) == 0
        r, _, status = sb.poll(timeout_s=0.3)
        assert len(r) == 0 and status == 6                            # CG_ERR_TIMEOUT: not admitted
        assert sa.stats()["admitted"] == 1 and sb.stats()["admitted"] == 0
        sa.close()                                                    # memory returns to the budget
        recs, amps = _consume(sb, 2000)
        _check_equal(recs, amps, exp)
        assert sb.stats()["admitted"] == 1
        sb.close()
        pa.close()
        pb.close()


def test_overflow_when_the_consumer_stalls_then_recovers():
    name = "paper_rate"
    frames = _frames(name, 4096)
    batch = 256
    with cg.Server(1 << 30) as srv, _plan(name) as plan:
        s = cg.Stream(srv, plan, ring_bytes=1100 * 2 * 4 * batch, batch_frames=batch)
        codes = [s.push(frames[i:i + 256], 1000 + i) for i in range(0, 4096, 256)]
        assert 5 in codes                                             # CG_ERR_OVERFLOW
        st = s.stats()
        assert st["frames_dropped"] > 0 and st["frames_pushed"] + st["frames_dropped"] == 4096
        assert s.flush(10.0) == 0
        recs, _, _ = s.poll(cap=8192, timeout_s=1.0)
        assert len(recs) == st["frames_pushed"]
        assert s.push(frames[:256], 99999) == 0                      # room again
        s.close()


def test_held_pipeline_times_out_then_delivers():
    name = "paper_rate"
    frames = _frames(name, 1000)
    exp = _expected(name, frames)
    with cg.Server(1 << 30) as srv, _plan(name) as plan:
        s = cg.Stream(srv, plan, ring_bytes=1100 * 2 * 8 * 512, batch_frames=512)
        srv.inject(cg.INJECT_HOLD, 1)
        assert s.push(frames, 1000) == 0
        assert s.flush(0.3) == 6                                      # CG_ERR_TIMEOUT
        r, _, status = s.poll(timeout_s=0.2)
        assert len(r) == 0 and status == 6
        srv.inject(cg.INJECT_HOLD, 0)
        recs, amps = _consume(s, 1000)
        _check_equal(recs, amps, exp)
        s.close()


def test_injected_launch_failure_puts_the_stream_in_error():
    name = "paper_rate"
    frames = _frames(name, 600)
    with cg.Server(1 << 30) as srv, _plan(name) as plan:
        s = cg.Stream(srv, plan, ring_bytes=1100 * 2 * 8 * 256, batch_frames=256)
        srv.inject(cg.INJECT_FAIL_LAUNCH, 1)
        assert s.push(frames, 0) == 0
        with pytest.raises(cg.CgError, match="CG_ERR_CUDA"):
            for _ in range(50):
                s.poll(timeout_s=0.1)
        with pytest.raises(cg.CgError, match="CG_ERR_CUDA"):
            s.push(frames, 600)
        s.close()


def test_stream_argument_errors():
    with cg.Server(1 << 20) as srv, _plan("paper_rate") as plan:
        with pytest.raises(cg.CgError, match="ring_bytes"):
            cg.Stream(srv, plan, ring_bytes=1100 * 2 * 100, batch_frames=256)
        with pytest.raises(cg.CgError, match="budget"):
            cg.Stream(srv, plan, ring_bytes=1 << 26, batch_frames=4096)
        with pytest.raises(cg.CgError, match="batch_frames"):
            cg.Stream(srv, plan, ring_bytes=1 << 26, batch_frames=0)
