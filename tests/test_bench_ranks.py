"""The multi-rank (replicas) logic of bench.py on CPU: two gloo ranks, each with its own step time;
the reported time is the maximum over ranks, the same on every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [12.5, 30.25]
    out[rank] = bench.max_over_ranks(times[rank], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_step_time_is_max_over_two_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        assert dict(out) == {0: 30.25, 1: 30.25}


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.0, None, "cpu") == 7.0


def test_parity_report_of_the_oracle_window(oracle):
    """bench.py's parity line: the oracle window against a record, exact and with one sample off."""
    import bench
    from paper_2403_15582_gb300 import workloads as wl
    wk = wl.static_100(seed=0, n_samples=1 << 14)
    w = oracle.make_waveform(wk.fs, wk.freq_hz, wk.amp, wk.phase_rad, wk.chirps, grid_log2=wk.grid_log2)
    rec = oracle.quantize(oracle.render(w, 0, wk.n_samples), w.full_scale())
    par = {}
    bench.oracle_window_rate(wk, 0.05, record=rec, parity=par)
    assert par["samples"] > 0 and par["from_sample"] == wk.n_samples // 2
    assert par["max_lsb"] == 0 and par["exact_fraction"] == 1.0
    rec[par["from_sample"] + 3] += 2
    par2 = {}
    bench.oracle_window_rate(wk, 0.05, record=rec, parity=par2)
    assert par2["max_lsb"] == 2 and par2["exact_fraction"] == 1.0 - 1.0 / par2["samples"]
