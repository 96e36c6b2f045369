"""The copy (Sec. 4.2) and ring (Sec. 4.3) algorithms with each rank's local
system a CUDA context driven through the C ABI: two ranks, both on cuda:0,
exchanging host buffers over gloo (the kernels of the two ranks never wait on
each other; the host collectives do the waiting).  FP64: the copy algorithm
repeats a one-rank run with one j-split bit for bit, and the two-rank ring a
one-rank run with two j-splits at the same boundary; mixed: both follow the
one-rank run within the mixed path's reach and the oracle pins the forces.
One rank on NCCL runs the device data path (CUDA tensors, device pointers)
and repeats the one-rank run bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_0709_4552_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EPS, ETA = 1 / 256, 0.01


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, algorithm, prec, N, t_end, nsplit, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_0709_4552_gb300 import distributed as D, nbody as nb
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    comm = D.Comm("cpu")
    m, x, v = inputs.plummer(N, 77, "salpeter")
    if algorithm == "copy":
        lo, hi = 0, N
    else:
        lo, hi = D.share(N, ws, rank)
    s = nb.NBody(hi - lo, prec, 0)
    s.set_params(EPS, ETA, 2.0 ** -22, t_end)
    if nsplit:
        s.set_tuning(n_split=nsplit)
    s.set_j_particles(0, m[lo:hi], x[lo:hi], v[lo:hi])
    if algorithm == "copy":
        s.initial_forces_and_dt()
        steps = D.integrate(s, comm, t_end, "copy", N=N)
    else:
        D.ring_initialize(s, comm, lo)
        steps = D.integrate(s, comm, t_end, "ring", base=lo)
    st = s.get_particles(0, hi - lo)
    s.close()
    out[rank] = dict(lo=lo, hi=hi, steps=steps, **{k: st[k] for k in ("x", "v", "a", "jerk", "pot", "t", "dt")})
    dist.barrier()
    dist.destroy_process_group()


def _run(algorithm, prec, N, t_end, nsplit):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(2, _free_port(), algorithm, prec, N, t_end, nsplit, out), nprocs=2,
                       join=True, start_method="spawn")
    return dict(out)


def _one_rank(nb, prec, N, t_end, nsplit):
    m, x, v = inputs.plummer(N, 77, "salpeter")
    with nb.NBody(N, prec, 0) as s:
        s.set_params(EPS, ETA, 2.0 ** -22, t_end)
        if nsplit:
            s.set_tuning(n_split=nsplit)
        s.set_j_particles(0, m, x, v)
        s.initial_forces_and_dt()
        c0 = s.get_counters()
        s.integrate(t_end)
        steps = s.get_counters()["block_steps"] - c0["block_steps"]
        return s.get_particles(0, N), steps


def _joined(out, key):
    return np.concatenate([out[r][key] for r in sorted(out)])


def _oracle_run(N, t_end):
    m, x, v = inputs.plummer(N, 77, "salpeter")
    return oracle.hermite_run(m, x, v, EPS, ETA, 2.0 ** -22, t_end, t_end, compensated=True)


def _energy_drift(N, st):
    m, x, v = inputs.plummer(N, 77, "salpeter")
    E0 = sum(oracle.energy(m, x, v, EPS))
    return abs(sum(oracle.energy(m, st["x"], st["v"], EPS)) - E0) / abs(E0)


def test_copy_fp64_bit_for_bit(nbl):
    N, t_end = 1000, 2.0 ** -4
    ref, steps = _one_rank(nbl, nbl.NB_FP64, N, t_end, 1)
    out = _run("copy", nbl.NB_FP64, N, t_end, 1)
    for r in (0, 1):
        assert out[r]["steps"] == steps
        for k in ("x", "v", "a", "jerk", "pot", "t", "dt"):
            assert np.array_equal(out[r][k], ref[k]), (r, k)
    orc = _oracle_run(N, t_end)
    assert np.array_equal(out[0]["dt"], orc["dt"]) and np.abs(out[0]["x"] - orc["x"]).max() < 1e-11


def test_ring_fp64_bit_for_bit(nbl):
    # N/2 a multiple of the FP64 j-tile (64): the one-rank run's two j-splits
    # meet where the ring's two shares do
    N, t_end = 1024, 2.0 ** -4
    ref, steps = _one_rank(nbl, nbl.NB_FP64, N, t_end, 2)
    out = _run("ring", nbl.NB_FP64, N, t_end, 1)
    assert out[0]["steps"] == out[1]["steps"] == steps
    for k in ("x", "v", "a", "jerk", "pot", "t", "dt"):
        assert np.array_equal(_joined(out, k), ref[k]), k
    orc = _oracle_run(N, t_end)
    assert np.array_equal(_joined(out, "dt"), orc["dt"]) and np.abs(_joined(out, "x") - orc["x"]).max() < 1e-11


@pytest.mark.parametrize("algorithm", ["copy", "ring"])
def test_mixed_follows_one_rank_and_oracle(nbl, algorithm):
    N, t_end = 3000, 2.0 ** -5
    ref, steps = _one_rank(nbl, nbl.NB_MIXED, N, t_end, 0)
    out = _run(algorithm, nbl.NB_MIXED, N, t_end, 0)
    if algorithm == "copy":
        got = {k: out[0][k] for k in ("x", "v", "a", "jerk", "pot", "t", "dt")}
        for k in got:
            assert np.array_equal(out[1][k], got[k]), k   # the copies stay identical
    else:
        got = {k: _joined(out, k) for k in ("x", "v", "a", "jerk", "pot", "t", "dt")}
    assert np.all(got["t"] == t_end)
    assert abs(out[0]["steps"] - steps) <= 0.05 * steps
    assert np.mean(got["dt"] == ref["dt"]) > 0.95
    assert np.abs(got["x"] - ref["x"]).max() < 1e-5
    # energy drift within 2x the oracle's own over the same integration
    orc = _oracle_run(N, t_end)
    assert _energy_drift(N, got) <= 2 * _energy_drift(N, orc) + 1e-9


def _nccl_main(rank, port, algorithm, same_stream, out):
    # one rank on NCCL: the blocks travel as CUDA tensors and the context reads
    # and writes device pointers (the multi-GPU data path, at p = 1), on
    # torch's current stream or on a stream of its own (fenced)
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_0709_4552_gb300 import distributed as D, nbody as nb
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1)
    comm = D.Comm("cuda:0")
    N, t_end = 1024, 2.0 ** -5
    m, x, v = inputs.plummer(N, 77, "salpeter")
    s = nb.NBody(N, nb.NB_FP64, 0, stream=torch.cuda.current_stream() if same_stream else None)
    s.set_params(EPS, ETA, 2.0 ** -22, t_end)
    s.set_tuning(n_split=1)
    s.set_j_particles(0, m, x, v)
    if algorithm == "copy":
        s.initial_forces_and_dt()
        steps = D.integrate(s, comm, t_end, "copy", N=N)
    else:
        D.ring_initialize(s, comm, 0)
        steps = D.integrate(s, comm, t_end, "ring", base=0)
    torch.cuda.synchronize()
    st = s.get_particles(0, N)
    s.close()
    out[0] = dict(steps=steps, **{k: st[k] for k in ("x", "v", "a", "t", "dt")})
    dist.destroy_process_group()


@pytest.mark.parametrize("algorithm,same_stream", [("copy", False), ("ring", False), ("ring", True)])
def test_nccl_device_path_single_rank(nbl, algorithm, same_stream):
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_nccl_available():
        pytest.skip("no NCCL")
    N, t_end = 1024, 2.0 ** -5
    ref, steps = _one_rank(nbl, nbl.NB_FP64, N, t_end, 1)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_nccl_main, args=(_free_port(), algorithm, same_stream, out), nprocs=1, join=True, start_method="spawn")
    got = out[0]
    assert got["steps"] == steps
    for k in ("x", "v", "a", "t", "dt"):
        assert np.array_equal(got[k], ref[k]), k
