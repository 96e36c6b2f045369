"""The allocation-free force entry point, nb_forces_fp64_noalloc.

It exists for callers that cannot let a library allocate device memory
(applications that own all device memory through their own pool, and
latency-critical loops where an allocation could stall or fail mid-run).
Checked here through the C ABI against the existing context-based entry point
(nb_compute_forces, FP64), within the FP64 tolerance of the other parity
tests, on two calls in a row that reuse the library's fixed scratch array.
Collected last so that a stop at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_0709_4552_gb300 import inputs
from _util import gpu_forces, rel_scalar, rel_vec

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def test_noalloc_matches_context_entry_point(nbl):
    torch = pytest.importorskip("torch")
    N, eps = 5003, 1.0 / 256
    m, x, v = inputs.plummer(N, 301, "salpeter")
    md, xd, vd = _dev(torch, m), _dev(torch, x), _dev(torch, v)
    # two calls in a row with different active blocks (the second reuses the
    # scratch the first left behind), then the first block again
    for n, seed in ((1700, 302), (37, 303), (1700, 302)):
        idx = inputs.sample_indices(N, n, seed).astype(np.int32)
        a_ref, j_ref, p_ref = gpu_forces(nbl, nbl.NB_FP64, m, x, v, eps, idx)
        acc = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        jerk = torch.empty_like(acc)
        pot = torch.empty(n, dtype=torch.float64, device="cuda")
        nbl.nb_forces_fp64_noalloc(md, xd, vd, eps, _dev(torch, idx), acc, jerk, pot)
        torch.cuda.synchronize()
        assert rel_vec(acc.cpu().numpy(), a_ref).max() <= FP64_TOL
        assert rel_vec(jerk.cpu().numpy(), j_ref).max() <= FP64_TOL
        assert rel_scalar(pot.cpu().numpy(), p_ref).max() <= FP64_TOL


def test_noalloc_rejects_blocks_beyond_its_scratch(nbl):
    torch = pytest.importorskip("torch")
    L = nbl.lib()
    n = (1 << 19) + 1  # NB_NOALLOC_MAX_ACTIVE + 1
    buf = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    code = L.nb_forces_fp64_noalloc(n, p, p, p, 0.01, idx.data_ptr(), n, p, p, p, None)
    assert code == nbl.NB_EINVAL
