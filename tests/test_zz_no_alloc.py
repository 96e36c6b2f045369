"""The allocation-free force entry point, nb_forces_fp64_noalloc.

It exists for callers that cannot let a library allocate device memory
(applications that own all device memory through their own pool, and
latency-critical loops where an allocation could stall or fail mid-run).
Checked here through the C ABI against the FP64 oracle (compensated sums,
the bound of every FP64 parity test) and against the existing context-based
entry point (nb_compute_forces, FP64), on calls in a row that reuse the
library's fixed scratch array: with NULL outputs, on a stream of the
caller's, and without softening.  Collected last so that a stop at the first
failure has run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_0709_4552_gb300 import inputs
from _util import gpu_forces, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _fp64_close(got, want):
    assert rel_vec(got[0], want[0]).max() <= FP64_TOL
    assert rel_vec(got[1], want[1]).max() <= FP64_TOL
    assert rel_scalar(got[2], want[2]).max() <= FP64_TOL


def test_noalloc_matches_oracle_and_context_entry_point(nbl):
    torch = pytest.importorskip("torch")
    N, eps = 5003, 1.0 / 256
    m, x, v = inputs.plummer(N, 301, "salpeter")
    md, xd, vd = _dev(torch, m), _dev(torch, x), _dev(torch, v)
    # calls in a row with different active blocks (each reuses the scratch
    # the previous one left behind), then the first block again
    for n, seed in ((1700, 302), (37, 303), (1700, 302)):
        idx = inputs.sample_indices(N, n, seed).astype(np.int32)
        ref = oracle.forces(m, x, v, eps, idx=idx.astype(np.int64), compensated=True)
        ctx = gpu_forces(nbl, nbl.NB_FP64, m, x, v, eps, idx)
        acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty_like(acc)
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nbl.nb_forces_fp64_noalloc(md, xd, vd, eps, _dev(torch, idx), acc, jerk, pot)
        torch.cuda.synchronize()
        got = (acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy())
        _fp64_close(got, ref)
        _fp64_close(got, ctx)


def test_noalloc_null_outputs_on_a_caller_stream(nbl):
    # only the acceleration is wanted (jerk and pot NULL), enqueued on a
    # non-default stream; the result equals a full call on the default stream
    torch = pytest.importorskip("torch")
    N, eps, n = 3001, 1.0 / 512, 900
    m, x, v = inputs.plummer(N, 311)
    idx = _dev(torch, inputs.sample_indices(N, n, 312).astype(np.int32))
    md, xd, vd = _dev(torch, m), _dev(torch, x), _dev(torch, v)
    full = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
    full.append(torch.empty(n, dtype=torch.float64, device="cuda"))
    nbl.nb_forces_fp64_noalloc(md, xd, vd, eps, idx, *full)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        nbl.nb_forces_fp64_noalloc(md, xd, vd, eps, idx, acc, None, None, stream=side)
    side.synchronize()
    assert torch.equal(acc, full[0])


def test_noalloc_unsoftened(nbl):
    # eps = 0: the self pair is excluded by index; distinct particles only
    torch = pytest.importorskip("torch")
    N = 1200
    m, x, v = inputs.plummer(N, 321)
    assert len(np.unique(x, axis=0)) == N
    idx = inputs.sample_indices(N, 333, 322).astype(np.int32)
    ref = oracle.forces(m, x, v, 0.0, idx=idx.astype(np.int64), compensated=True)
    out = [torch.empty((333, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
    out.append(torch.empty(333, dtype=torch.float64, device="cuda"))
    nbl.nb_forces_fp64_noalloc(_dev(torch, m), _dev(torch, x), _dev(torch, v), 0.0, _dev(torch, idx), *out)
    torch.cuda.synchronize()
    _fp64_close([o.cpu().numpy() for o in out], ref)


def test_noalloc_rejects_blocks_beyond_its_scratch(nbl):
    torch = pytest.importorskip("torch")
    L = nbl.lib()
    n = (1 << 19) + 1  # NB_NOALLOC_MAX_ACTIVE + 1
    buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    code = L.nb_forces_fp64_noalloc(n, p, p, p, 0.01, idx.data_ptr(), n, p, p, p, None)
    assert code == nbl.NB_EINVAL
