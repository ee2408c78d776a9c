"""Streaming driver: feeds a Ring chunk by chunk, scheduling each chunk's chirps just before it is
rendered (a tone may chirp many times; each new chirp folds the tone's previous one)."""
from __future__ import annotations

import time


def run_stream(synth, ring, chirps, n_chunks: int, stream=None, prefill: int = 2, capture=None,
               push_timeout_ms: int = 10000, finish_timeout_ms: int = 120000, producer_delay_s: float = 0.0):
    """Render n_chunks chunks through `ring` while its sink plays them in real time.

    chirps: dicts (tone, f_start, f_end, duration, profile, start_sample).  Before chunk c is
    pushed, every chirp starting before the chunk's end is handed to the synthesiser.
    producer_delay_s: extra host delay before each push (to provoke underruns in tests).
    Returns the ring statistics (dict) plus the producer's wall time."""
    import numpy as np
    order = sorted(chirps, key=lambda c: c.get("start_sample", 0))
    # each chunk's batch as arrays, built before playback starts: the loop below only hands them to
    # the library
    batches = []
    nxt = 0
    for c in range(n_chunks):
        end = (c + 1) * ring.chunk
        first = nxt
        while nxt < len(order) and order[nxt].get("start_sample", 0) < end:
            nxt += 1
        b = order[first:nxt]
        batches.append(None if not b else (
            np.array([x["tone"] for x in b], dtype=np.int32), np.array([x["f_start"] for x in b], dtype=np.float64),
            np.array([x["f_end"] for x in b], dtype=np.float64), np.array([x["duration"] for x in b], dtype=np.float64),
            np.array([x["profile"] for x in b], dtype=np.int32),
            np.array([x.get("start_sample", 0) for x in b], dtype=np.int64)))
    ring.start(prefill, n_chunks, capture)
    t0 = time.perf_counter()
    for c in range(n_chunks):
        if batches[c] is not None:
            synth.set_chirps(*batches[c])
        if producer_delay_s:
            time.sleep(producer_delay_s)
        ring.push(stream, push_timeout_ms)
    produce_s = time.perf_counter() - t0
    stats = ring.finish(finish_timeout_ms)
    stats["produce_s"] = produce_s
    return stats
