"""The paper's parallel algorithms (Sec. 4.2 copy, Sec. 4.3 ring) as the
package's distributed driver runs them, on two gloo ranks on the CPU with
each rank's local system answered by the FP64 oracle
(tests/_oracle_engine.py): the copy algorithm repeats the one-rank oracle
integration bit for bit, the ring algorithm to the rounding of its split sums."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, algorithm, N, t_end, out):
    import torch.distributed as dist
    sys.path[:0] = [ROOT, TESTS]
    import oracle
    from _oracle_engine import OracleEngine
    from paper_0709_4552_gb300 import distributed as D, inputs
    oracle.build()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    comm = D.Comm("cpu")
    eps, eta, dt_min, dt_max = 1 / 64, 0.01, 2.0 ** -22, t_end
    m, x, v = inputs.plummer(N, 31, "salpeter")
    if algorithm == "copy":
        eng = OracleEngine(m, x, v, eps, eta, dt_min, dt_max)
        eng.initial_forces_and_dt()
        steps = D.integrate(eng, comm, t_end, "copy", N=N)
        lo, hi = 0, N
    else:
        lo, hi = D.share(N, ws, rank)
        eng = OracleEngine(m[lo:hi], x[lo:hi], v[lo:hi], eps, eta, dt_min, dt_max)
        D.ring_initialize(eng, comm, lo)
        steps = D.integrate(eng, comm, t_end, "ring", base=lo)
    out[rank] = dict(lo=lo, hi=hi, steps=steps, x=eng.x.copy(), v=eng.v.copy(), t=eng.t.copy(), dt=eng.dt.copy(),
                     a=eng.a.copy())
    dist.barrier()
    dist.destroy_process_group()


def _run(algorithm, N=96, t_end=2.0 ** -4, ws=2):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(ws, _free_port(), algorithm, N, t_end, out), nprocs=ws, join=True,
                       start_method="spawn")
    return dict(out)


def _reference(N=96, t_end=2.0 ** -4):
    sys.path[:0] = [ROOT, TESTS]
    import oracle
    from paper_0709_4552_gb300 import inputs
    m, x, v = inputs.plummer(N, 31, "salpeter")
    return oracle.hermite_run(m, x, v, 1 / 64, 0.01, 2.0 ** -22, t_end, t_end)


def test_share_covers_every_index():
    sys.path.insert(0, ROOT)
    from paper_0709_4552_gb300.distributed import share
    for N in (1, 7, 96, 1001):
        for p in (1, 2, 3, 8):
            cuts = [share(N, p, r) for r in range(p)]
            assert cuts[0][0] == 0 and cuts[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
            assert max(h - l for l, h in cuts) - min(h - l for l, h in cuts) <= 1


def test_copy_algorithm_repeats_one_rank_bit_for_bit(orc):
    ref = _reference()
    out = _run("copy")
    for r in (0, 1):   # every rank ends with the whole system, identical to one rank
        for k in ("x", "v", "a", "t", "dt"):
            assert np.array_equal(out[r][k], ref[k]), (r, k)
    assert out[0]["steps"] == out[1]["steps"] == ref["block_steps"]


def test_ring_algorithm_matches_one_rank(orc):
    ref = _reference()
    out = _run("ring")
    x = np.concatenate([out[r]["x"] for r in (0, 1)])
    dt = np.concatenate([out[r]["dt"] for r in (0, 1)])
    t = np.concatenate([out[r]["t"] for r in (0, 1)])
    assert out[0]["steps"] == out[1]["steps"] == ref["block_steps"]
    assert np.array_equal(t, ref["t"]) and np.array_equal(dt, ref["dt"])
    assert np.abs(x - ref["x"]).max() < 1e-12


def test_fence_orders_streams_only_where_needed():
    # _fence: nothing for host tensors or an engine on torch's current stream,
    # a device synchronisation for an engine on a stream of its own
    from types import SimpleNamespace
    from paper_0709_4552_gb300 import distributed as D

    calls = []
    cur = SimpleNamespace(cuda_stream=1234)
    fake_torch = SimpleNamespace(cuda=SimpleNamespace(current_stream=lambda dev: cur,
                                                      synchronize=lambda dev: calls.append(dev)))

    def comm(kind):
        return SimpleNamespace(device=SimpleNamespace(type=kind), torch=fake_torch)

    D._fence(SimpleNamespace(stream_handle=None), comm("cpu"))
    D._fence(SimpleNamespace(stream_handle=1234), comm("cuda"))
    assert calls == []
    D._fence(SimpleNamespace(stream_handle=None), comm("cuda"))
    D._fence(SimpleNamespace(stream_handle=99), comm("cuda"))
    D._fence(SimpleNamespace(), comm("cuda"))
    assert len(calls) == 3
