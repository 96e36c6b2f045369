"""The paper's two parallel algorithms for the block-step loop, one rank per
GPU over ``torch.distributed`` (NCCL on GPUs, gloo on host buffers).

Copy algorithm (Sec. 4.2): every rank holds all N particles.  Each block step
every rank selects the same block (identical copies give identical choices),
predicts all N, computes the forces on -- and corrects -- only the active
particles of its own share of the indices, [lo_r, hi_r), and then the ranks
exchange the corrected particles: an all-gather of the block sizes and an
all-gather of the particles (the paper's MPI_Allgather + MPI_Allgatherv), after
which every copy is again identical.  Per step each rank computes n/p of the
block against all N (Eq. for t_force = tau_force N n/p).

Ring algorithm (Sec. 4.3): each rank holds only its N/p particles.  The ranks
agree on the next block time with an all-reduce (minimum), each predicts its
own particles, and the active block of every rank -- predicted positions and
velocities, global indices and running force sums -- travels around the ring
in p shifts: at every rank it visits, that rank adds the forces of its own
particles on it (nb_forces_on), then passes it on (a send-receive pair).
After p shifts each block is home with the forces of all N and its rank
corrects it (nb_set_forces + nb_correct).  Per step each rank computes
n/p x N/p interactions p times.

A rank's local system (the "engine") is a :class:`paper_0709_4552_gb300.nbody.NBody`
context driven through the C ABI; all arithmetic of a step runs in its CUDA
kernels.  This module only moves data between ranks and orders the calls.
Blocks travel as tensors on the communicator's device: CUDA tensors with
NCCL (the engine then reads and writes device pointers), host tensors with
gloo.  No TMA multicast or NVLink multicast is used anywhere.  On device
pointers the engine's calls are asynchronous on the engine's stream while
torch's tensor operations and NCCL's collectives are ordered on torch's
current stream; an engine created on that stream
(``NBody(..., stream=torch.cuda.current_stream())``) needs nothing more,
any other engine is fenced with a device synchronisation wherever a tensor
passes between the two (:func:`_fence`).

Determinism: on the FP64 path the copy algorithm sums every force over all N
in the same j order as one rank, so with one j-split per force call (the
tuning ``n_split=1`` on every context) a p-rank run repeats a one-rank run
bit for bit.  The ring algorithm adds p partial sums in ring order; for p = 2
that equals a one-rank run with two j-splits at the same boundary (the
split-j reduction adds the same two partials), otherwise it differs in the
last bits.
"""
from __future__ import annotations

import numpy as np

_KEYS = ("x", "v", "a", "jerk", "pot", "t", "dt")
_WIDTH = dict(x=3, v=3, a=3, jerk=3, pot=1, t=1, dt=1)


def share(N, p, r):
    """[lo, hi) of rank r's share of N indices (sizes differ by at most one)."""
    return (N * r) // p, (N * (r + 1)) // p


class Comm:
    """The collectives the two algorithms use, on ``torch.distributed``."""

    def __init__(self, device="cpu", group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.device = torch.device(device)
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def tensor(self, a, dtype=None):
        t = self.torch.as_tensor(a, dtype=dtype)
        return t.to(self.device)

    def allreduce_min(self, x):
        t = self.tensor([float(x)], self.torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return float(t.item())

    def allreduce_sum_int(self, x):
        t = self.tensor([int(x)], self.torch.int64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return int(t.item())

    def allgatherv(self, rows):
        """All-gather of [n_r, w] float64 row blocks of different lengths:
        the sizes first (MPI_Allgather), then the rows padded to the largest
        block (MPI_Allgatherv); returns the blocks in rank order."""
        torch = self.torch
        counts = [self.tensor([0], torch.int64) for _ in range(self.size)]
        self.dist.all_gather(counts, self.tensor([rows.shape[0]], torch.int64), group=self.group)
        counts = [int(c.item()) for c in counts]
        w = rows.shape[1]
        cap = max(max(counts), 1)
        pad = torch.zeros((cap, w), dtype=torch.float64, device=self.device)
        pad[: rows.shape[0]] = rows
        out = [torch.empty((cap, w), dtype=torch.float64, device=self.device) for _ in range(self.size)]
        self.dist.all_gather(out, pad, group=self.group)
        return [o[:c] for o, c in zip(out, counts)]

    def shift(self, rows):
        """One ring shift: send the block to rank r - 1, receive the block of
        rank r + 1 (sizes first, then the rows; MPI_Sendrecv)."""
        torch, dist = self.torch, self.dist
        if self.size == 1:
            return rows
        dst, src = (self.rank - 1) % self.size, (self.rank + 1) % self.size
        n_in = self.tensor([0], torch.int64)
        ops = [dist.P2POp(dist.isend, self.tensor([rows.shape[0]], torch.int64), dst, self.group),
               dist.P2POp(dist.irecv, n_in, src, self.group)]
        for q in dist.batch_isend_irecv(ops):
            q.wait()
        got = torch.empty((int(n_in.item()), rows.shape[1]), dtype=torch.float64, device=self.device)
        ops = []
        if rows.shape[0]:
            ops.append(dist.P2POp(dist.isend, rows.contiguous(), dst, self.group))
        if got.shape[0]:
            ops.append(dist.P2POp(dist.irecv, got, src, self.group))
        if ops:
            for q in dist.batch_isend_irecv(ops):
                q.wait()
        return got


def _fence(engine, comm):
    """Orders the engine's kernels against torch's work on CUDA tensors at a
    hand-off: nothing when the engine works on torch's current stream (or the
    tensors live on the host, where the engine's calls synchronise), else a
    synchronisation of the device (both directions at once)."""
    if comm.device.type != "cuda":
        return
    h = getattr(engine, "stream_handle", None)
    if h is not None and h == comm.torch.cuda.current_stream(comm.device).cuda_stream:
        return
    comm.torch.cuda.synchronize(comm.device)


def _index(comm, idx):
    return comm.tensor(np.ascontiguousarray(idx, dtype=np.int32), comm.torch.int32)


def copy_step(engine, comm, lo, hi):
    """One block step of the copy algorithm (Sec. 4.2); returns (t, n) of the
    whole block.  ``engine`` holds all N particles; this rank owns [lo, hi)."""
    torch = comm.torch
    t, n, idx = engine.next_block()
    engine.predict(t)
    mine = idx[(idx >= lo) & (idx < hi)]
    k = len(mine)
    dmine = _index(comm, mine)
    f = [torch.empty((k, 3), dtype=torch.float64, device=comm.device) for _ in range(2)]
    f.append(torch.empty(k, dtype=torch.float64, device=comm.device))
    # the corrected block of this rank: index + x v a jerk pot t dt (18 columns)
    out = {key: torch.empty((k,) if _WIDTH[key] == 1 else (k, 3), dtype=torch.float64, device=comm.device)
           for key in _KEYS}
    _fence(engine, comm)
    if k:
        engine.compute_forces(dmine, *f)
        engine.correct(dmine, t)
        engine.get_particles_idx(dmine, out=out)
    _fence(engine, comm)
    rows = torch.cat([dmine.to(torch.float64)[:, None]] + [out[key].reshape(k, _WIDTH[key]) for key in _KEYS],
                     dim=1)
    blocks = comm.allgatherv(rows)
    others = [b for r, b in enumerate(blocks) if r != comm.rank and b.shape[0]]
    if others:
        rows = torch.cat(others)   # shares in rank order: ascending indices
        oidx = rows[:, 0].to(torch.int32).contiguous()
        vals, c0 = {}, 1
        for key in _KEYS:
            w = _WIDTH[key]
            vals[key] = rows[:, c0:c0 + w].reshape(-1) if w == 1 else rows[:, c0:c0 + w].contiguous()
            vals[key] = vals[key].contiguous()
            c0 += w
        _fence(engine, comm)
        engine.set_particles_idx(oidx, vals)
        _fence(engine, comm)
    return t, n


def ring_step(engine, comm, base):
    """One block step of the ring algorithm (Sec. 4.3); returns (t, n) of the
    whole block.  ``engine`` holds this rank's particles, global indices
    base + [0, N_r)."""
    torch = comm.torch
    t_loc, n_loc, idx = engine.next_block()
    t = comm.allreduce_min(t_loc)
    mine = idx if t_loc == t else idx[:0]
    n_all = comm.allreduce_sum_int(len(mine))
    engine.predict(t)
    k = len(mine)
    dmine = _index(comm, mine)
    # the travelling block: xp vp (6) | global index (1) | acc jerk pot sums (7)
    block = torch.zeros((k, 14), dtype=torch.float64, device=comm.device)
    if k:
        xp = torch.empty((k, 3), dtype=torch.float64, device=comm.device)
        vp = torch.empty_like(xp)
        _fence(engine, comm)
        engine.get_predicted(dmine, xp, vp)
        _fence(engine, comm)
        block[:, 0:3] = xp
        block[:, 3:6] = vp
        block[:, 6] = dmine.to(torch.float64) + base
    for _ in range(comm.size):
        m = block.shape[0]
        if m:
            xi, vi = block[:, 0:3].contiguous(), block[:, 3:6].contiguous()
            gid = block[:, 6].to(torch.int64).contiguous()
            acc, jerk = block[:, 7:10].contiguous(), block[:, 10:13].contiguous()
            pot = block[:, 13].contiguous()
            _fence(engine, comm)
            engine.forces_on(xi, vi, gid, base, acc, jerk, pot, accumulate=True)
            _fence(engine, comm)
            block[:, 7:10], block[:, 10:13], block[:, 13] = acc, jerk, pot
        block = comm.shift(block)
    if k:
        fa, fj, fp = block[:, 7:10].contiguous(), block[:, 10:13].contiguous(), block[:, 13].contiguous()
        _fence(engine, comm)
        engine.set_forces(dmine, fa, fj, fp)
        engine.correct(dmine, t)
        _fence(engine, comm)
    return t, n_all


def ring_initialize(engine, comm, base):
    """Sec. 4.1 step 1 under the ring algorithm: every rank's particles make
    one full circuit (all of them active at t = 0, positions as set), summing
    the forces of all N, and each rank then takes its initial steps
    (nb_set_initial_forces).  The copy algorithm needs no pass of its own:
    every rank holds all N (nb_initial_forces_and_dt)."""
    torch = comm.torch
    N_r = engine.get_n()
    engine.predict(0.0)
    own = _index(comm, np.arange(N_r, dtype=np.int32))
    xp = torch.empty((N_r, 3), dtype=torch.float64, device=comm.device)
    vp = torch.empty_like(xp)
    _fence(engine, comm)
    engine.get_predicted(own, xp, vp)
    _fence(engine, comm)
    block = torch.zeros((N_r, 14), dtype=torch.float64, device=comm.device)
    block[:, 0:3], block[:, 3:6] = xp, vp
    block[:, 6] = own.to(torch.float64) + base
    for _ in range(comm.size):
        if block.shape[0]:
            acc, jerk = block[:, 7:10].contiguous(), block[:, 10:13].contiguous()
            pot = block[:, 13].contiguous()
            xi, vi, gid = block[:, 0:3].contiguous(), block[:, 3:6].contiguous(), block[:, 6].to(torch.int64).contiguous()
            _fence(engine, comm)
            engine.forces_on(xi, vi, gid, base, acc, jerk, pot, accumulate=True)
            _fence(engine, comm)
            block[:, 7:10], block[:, 10:13], block[:, 13] = acc, jerk, pot
        block = comm.shift(block)
    fa, fj, fp = block[:, 7:10].contiguous(), block[:, 10:13].contiguous(), block[:, 13].contiguous()
    _fence(engine, comm)
    engine.set_initial_forces(fa, fj, fp)
    _fence(engine, comm)


def integrate(engine, comm, t_end, algorithm, N=None, base=0, max_steps=None):
    """Block steps until every particle has reached t_end (Sec. 4.1 step 6)
    with the copy or the ring algorithm; returns the number of block steps.
    copy: ``N`` is the particle count every rank holds; ring: ``base`` is
    this rank's first global index."""
    if algorithm == "copy":
        lo, hi = share(N, comm.size, comm.rank)
        step = lambda: copy_step(engine, comm, lo, hi)
        peek = lambda: engine.next_block(want_indices=False)[0]
    elif algorithm == "ring":
        step = lambda: ring_step(engine, comm, base)
        peek = lambda: comm.allreduce_min(engine.next_block(want_indices=False)[0])
    else:
        raise ValueError(f"unknown algorithm {algorithm!r}")
    steps = 0
    while peek() <= t_end:
        step()
        steps += 1
        if max_steps is not None and steps >= max_steps:
            break
    return steps
