"""Served request stream: continuous batching, admission by deadline and memory, and results that
do not depend on the co-runners.  Every served request is compared element by element with the
CPU oracle (FP64 sum of Eq. dynamicandstatic, quantised in FP64: int16 within 1 LSB) and with its
standalone render (bit for bit: alone and in the mix give the same samples)."""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def awg(awglib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return awglib


def _request(seed, fs, K, chunk, n_chunks, n_chirps):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.02 * fs, 0.45 * fs, K)
    a = np.full(K, 1.0 / K)
    th = rng.uniform(0, 2 * np.pi, K)
    chirps = []
    for t in rng.choice(K, size=min(n_chirps, K), replace=False):
        chirps.append(dict(tone=int(t), f_start=float(f[t]), f_end=float(rng.uniform(0.02 * fs, 0.45 * fs)),
                           duration=float(rng.integers(3000, 60000)) / fs, profile=int(rng.integers(0, 2)),
                           start_sample=int(rng.integers(0, 5000))))
    return f, a, th, chirps, chunk, n_chunks


def _standalone(awg, fs, req, engine=0):
    f, a, th, chirps, chunk, n_chunks = req
    s = awg.Synth(fs)
    s.set_tones(f, a, th)
    s.set_chirp_list(chirps)
    s.set_static_engine(engine)
    out = torch.empty(chunk * n_chunks, dtype=torch.int16, device="cuda")
    for c in range(n_chunks):
        s.render(chunk, out[c * chunk:])
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle_codes(oracle, fs, req):
    """The oracle's int16 codes for the whole request (its chunks back to back from sample 0; chirp
    start samples are relative to the request's first sample; full scale sum |A|)."""
    f, a, th, chirps, chunk, n_chunks = req
    w = oracle.make_waveform(fs, f, a, th, chirps)
    return oracle.quantize(oracle.render(w, 0, chunk * n_chunks, nthreads=NTHREADS), w.full_scale())


def _check_against_oracle(oracle, fs, req, got):
    q_ref = _oracle_codes(oracle, fs, req)
    dq = np.abs(got.astype(np.int32) - q_ref.astype(np.int32))
    assert got.shape == q_ref.shape
    assert dq.max() <= 1, (int(dq.max()), int(np.argmax(dq)))
    return float(np.mean(dq == 0))


def test_results_same_alone_and_in_the_mix(awg, oracle):
    fs = 20e6     # long playback periods: every request is admitted
    reqs = [_request(i, fs, K, chunk, 4, nc) for i, (K, chunk, nc) in
            enumerate([(50, 1 << 16, 10), (700, 1 << 17, 40), (3000, 1 << 16, 100), (129, 70000, 5),
                       (1500, 1 << 18, 0), (64, 1 << 16, 64), (960, 99999, 30), (5000, 1 << 17, 100)])]
    srv = awg.Server(fs, 8 << 30, 64)
    ids = []
    for i, r in enumerate(reqs):
        f, a, th, chirps, chunk, n_chunks = r
        ids.append(srv.submit(f, a, th, chunk, n_chunks, chirps))
        if i == 3:
            time.sleep(0.004)    # the rest arrive while the first ones are running
    srv.drain(60000)
    st = srv.stats()
    assert st["admitted"] == len(reqs) and st["completed"] == len(reqs)
    for rid, r in zip(ids, reqs):
        state, done = srv.poll(rid)
        assert state == awg.binding.REQ_DONE and done == r[5]
        got = srv.read(rid, r[4] * r[5])
        assert np.array_equal(got, _standalone(awg, fs, r)), rid
        _check_against_oracle(oracle, fs, r, got)
        srv.release(rid)
    srv.close()


def test_two_split_sizes_in_one_round_match_the_oracle(awg, oracle):
    """A 16-tone request (tone split 1) with 1.6 ms chunks starts first and keeps rounds short
    (a third of its period); a 10,000-tone request (split 16) arriving while it plays has its
    2^20-sample chunk cut into five tile pieces, issued over more than one period of the short
    request, so a piece shares a round with a short chunk: such a round launches the batched
    render once per split size.  Both requests' samples equal the oracle's within 1 LSB and their
    standalone renders bit for bit."""
    fs = 20e6
    reqs = [_request(22, fs, 16, 1 << 15, 48, 16), _request(21, fs, 10000, 1 << 20, 1, 100)]
    srv = awg.Server(fs, 8 << 30, 64)
    ids = []
    for r in reqs:
        ids.append(srv.submit(r[0], r[1], r[2], r[4], r[5], r[3]))
        time.sleep(0.002)
    srv.drain(60000)
    st = srv.stats()
    assert st["admitted"] == 2 and st["completed"] == 2, st
    assert st["max_batch"] >= 2, st          # a round held pieces of both requests
    for rid, r in zip(ids, reqs):
        got = srv.read(rid, r[4] * r[5])
        assert np.array_equal(got, _standalone(awg, fs, r)), rid
        _check_against_oracle(oracle, fs, r, got)
        srv.release(rid)
    srv.close()


def test_served_requests_on_the_tensor_core_engine(awg, oracle):
    """Requests of at least 1000 tones have their static tones summed by the split-precision GEMM
    (FP16 hi + lo), only their chirping tones through the batched render; a request without chirps
    is written by the GEMM alone.  Each equals a standalone render with the same engine bit for bit
    and the oracle within 1 LSB; a small request in the same rounds stays on the direct path."""
    fs = 20e6
    reqs = [_request(31, fs, 3000, 1 << 17, 3, 60), _request(32, fs, 200, 1 << 16, 4, 20),
            _request(33, fs, 1200, 1 << 17, 2, 0)]
    srv = awg.Server(fs, 8 << 30, 64)
    srv.set_static_engine(awg.STATIC_GEMM_FP16, 1000)
    assert srv.stats()["est_engine_throughput"] > srv.stats()["est_throughput"]
    ids = [srv.submit(r[0], r[1], r[2], r[4], r[5], r[3]) for r in reqs]
    srv.drain(60000)
    st = srv.stats()
    assert st["completed"] == 3, st
    for rid, r in zip(ids, reqs):
        got = srv.read(rid, r[4] * r[5])
        engine = awg.STATIC_GEMM_FP16 if len(r[0]) >= 1000 else awg.STATIC_DIRECT
        assert np.array_equal(got, _standalone(awg, fs, r, engine)), rid
        _check_against_oracle(oracle, fs, r, got)
        srv.release(rid)
    srv.close()


def test_admission_rejects_what_cannot_meet_its_deadline(awg):
    fs = 280e6    # 10,000 tones at 280 MS/s with 2^16-sample chunks (234 us) cannot keep up
    srv = awg.Server(fs, 8 << 30, 64)
    f, a, th, chirps, chunk, n = _request(1, fs, 10000, 1 << 16, 4, 0)
    rid = srv.submit(f, a, th, chunk, n, chirps)
    f2, a2, th2, c2, chunk2, n2 = _request(2, fs, 100, 1 << 20, 2, 3)
    rid2 = srv.submit(f2, a2, th2, chunk2, n2, c2)
    srv.drain(60000)
    assert srv.poll(rid)[0] == awg.binding.REQ_REJECTED
    assert srv.poll(rid2)[0] == awg.binding.REQ_DONE
    st = srv.stats()
    assert st["rejected_deadline"] >= 1 and st["deadline_misses"] == 0
    srv.close()


def test_admission_by_memory(awg):
    fs = 20e6
    srv = awg.Server(fs, 1 << 20, 8)       # 1 MiB budget: a 2^18 x 8 chunk output does not fit
    f, a, th, chirps, chunk, n = _request(3, fs, 50, 1 << 18, 8, 0)
    rid = srv.submit(f, a, th, chunk, n, chirps)
    srv.drain(30000)
    assert srv.poll(rid)[0] == awg.binding.REQ_REJECTED
    assert srv.stats()["rejected_memory"] == 1
    srv.close()


def test_chunks_cut_into_tile_pieces_match_standalone(awg, oracle):
    """At 280 MS/s a 2^16-sample chunk plays for 234 us, so rounds stay short and the 2^20-sample
    chunks of a 1500-tone request are rendered in many tile-aligned pieces; the samples still equal
    a standalone render of each request."""
    fs = 280e6
    reqs = [_request(11, fs, 40, 1 << 16, 64, 5), _request(12, fs, 1500, 1 << 20, 2, 50)]   # 15 ms, 7.5 ms
    srv = awg.Server(fs, 8 << 30, 64)
    ids = [srv.submit(r[0], r[1], r[2], r[4], r[5], r[3]) for r in reqs]
    srv.drain(60000)
    st = srv.stats()
    assert st["completed"] == 2, st
    pieces = round(st["mean_batch"] * st["rounds"])
    assert pieces >= 64 + 2 + 6, st      # the 2^20 chunks were cut into pieces
    assert st["max_batch"] >= 2, st      # the short request's chunks joined rounds of the long one
    for rid, r in zip(ids, reqs):
        got = srv.read(rid, r[4] * r[5])
        assert np.array_equal(got, _standalone(awg, fs, r)), rid
        _check_against_oracle(oracle, fs, r, got)
        srv.release(rid)
    srv.close()


@pytest.mark.parametrize("depth", [2, 3])
def test_start_up_chunks_fill_the_buffer_before_playback(awg, depth):
    """The timing model of a served request: its first `depth` chunks are the start-up, released
    when its set-up is done; playback starts (t_play) when they are all complete; every later
    chunk c is due at t_play + c period and released `depth` periods earlier, never before t_play,
    so each streamed chunk has the whole look-ahead.  Read from the exported chunk traces of one
    request on an otherwise idle server."""
    fs, chunk, n_chunks = 20e6, 1 << 16, 7
    period = chunk / fs
    f, a, th, chirps, _, _ = _request(31, fs, 200, chunk, n_chunks, 20)
    srv = awg.Server(fs, 8 << 30, 64)
    srv.set_prefetch(depth)
    rid = srv.submit(f, a, th, chunk, n_chunks, chirps)
    srv.drain(60000)
    tr = srv.trace_chunks()
    tr = np.sort(tr[tr["id"] == rid], order="chunk")
    assert list(tr["chunk"]) == list(range(n_chunks))
    start, streamed = tr[:depth], tr[depth:]
    t_ready = start["release"][0]
    assert np.all(start["release"] == t_ready)
    assert np.allclose(start["due"], t_ready + period * (np.arange(depth) + 1), rtol=0, atol=1e-9)
    assert not np.any(start["late"])
    t_play = float(np.max(start["done"]))
    c = streamed["chunk"].astype(np.float64)
    assert np.allclose(streamed["due"], t_play + c * period, rtol=0, atol=1e-9)
    assert np.allclose(streamed["release"], t_play + (c - depth) * period, rtol=0, atol=1e-9)
    assert np.all(streamed["release"] >= t_play - 1e-12)
    assert not np.any(streamed["late"]) and np.all(streamed["done"] <= streamed["due"])
    assert srv.stats()["deadline_misses"] == 0
    srv.release(rid)
    srv.close()
