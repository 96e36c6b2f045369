"""One rank's local system for the distributed driver
(paper_0709_4552_gb300.distributed), answered by the FP64 oracle: test
infrastructure that lets the copy and ring algorithms' partitioning and
exchange run on CPU gloo ranks.  Its block step is the oracle's own
(orc_hermite_run's order: predict all, plain left-to-right sums over j,
corrector, Aarseth step, block rule), so the copy algorithm over it repeats
oracle.hermite_run bit for bit."""
import numpy as np

import oracle


def _np(a):
    return a.numpy() if hasattr(a, "numpy") else np.asarray(a)


class OracleEngine:
    def __init__(self, m, x, v, eps, eta, dt_min, dt_max):
        self.m = np.array(m, dtype=np.float64)
        self.x = np.array(x, dtype=np.float64)
        self.v = np.array(v, dtype=np.float64)
        N = len(self.m)
        self.a, self.jk = np.zeros((N, 3)), np.zeros((N, 3))
        self.pot, self.t, self.dt = np.zeros(N), np.zeros(N), np.zeros(N)
        self.eps, self.eta, self.dt_min, self.dt_max = eps, eta, dt_min, dt_max
        self.xp = self.vp = None
        self.f = None

    def get_n(self):
        return len(self.m)

    def initial_forces_and_dt(self):
        a, j, p = oracle.forces(self.m, self.x, self.v, self.eps)
        self.set_initial_forces(a, j, p)

    def set_initial_forces(self, acc, jerk, pot):
        self.a, self.jk, self.pot = _np(acc).copy(), _np(jerk).copy(), _np(pot).copy()
        self.t[:] = 0.0
        self.dt = np.array([oracle.initial_dt(self.a[i], self.jk[i], self.eta, self.dt_min, self.dt_max)
                            for i in range(len(self.m))])

    def next_block(self, want_indices=True):
        due = self.t + self.dt
        t = due.min()
        idx = np.nonzero(due == t)[0].astype(np.int32)
        return float(t), len(idx), (idx if want_indices else None)

    def predict(self, t):
        self.xp, self.vp = oracle.predict(self.x, self.v, self.a, self.jk, self.t, t)

    def compute_forces(self, idx, acc, jerk, pot):
        i = _np(idx).astype(np.int64)
        a, j, p = oracle.forces(self.m, self.xp, self.vp, self.eps, idx=i)
        self.f = (i, a, j, p)
        _np(acc)[...], _np(jerk)[...], _np(pot)[...] = a, j, p

    def set_forces(self, idx, acc, jerk, pot):
        self.f = (_np(idx).astype(np.int64), _np(acc).copy(), _np(jerk).copy(), _np(pot).copy())

    def correct(self, idx, t):
        i, a1, j1, p1 = self.f
        assert np.array_equal(i, _np(idx))
        h = t - self.t[i]
        x1, v1, a2, a3 = oracle.correct(self.x[i], self.v[i], self.a[i], self.jk[i], self.xp[i], self.vp[i],
                                        a1, j1, h)
        self.x[i], self.v[i], self.a[i], self.jk[i], self.pot[i] = x1, v1, a1, j1, p1
        for k, q in enumerate(i):
            crit = oracle.aarseth_dt(a1[k], j1[k], a2[k], a3[k], self.eta)
            self.dt[q] = oracle.block_dt(crit, self.dt[q], t, self.dt_min, self.dt_max)[0]
        self.t[i] = t

    def _state(self):
        return dict(x=self.x, v=self.v, a=self.a, jerk=self.jk, pot=self.pot, t=self.t, dt=self.dt, m=self.m)

    def get_particles_idx(self, idx, out):
        i = _np(idx).astype(np.int64)
        st = self._state()
        for k, dst in out.items():
            _np(dst)[...] = st[k][i]
        return out

    def set_particles_idx(self, idx, values):
        i = _np(idx).astype(np.int64)
        st = self._state()
        for k, src in values.items():
            st[k][i] = _np(src).reshape(st[k][i].shape)

    def get_predicted(self, idx, xp, vp):
        i = _np(idx).astype(np.int64)
        _np(xp)[...], _np(vp)[...] = self.xp[i], self.vp[i]

    def forces_on(self, xi, vi, gid, base, acc, jerk, pot, accumulate=True):
        xi, vi, gid = _np(xi), _np(vi), _np(gid)
        N = len(self.m)
        local = gid - base
        here = (local >= 0) & (local < N)
        # particles held here are i by index (their prediction is this rank's);
        # the others join as massless particles after the local ones
        away = np.nonzero(~here)[0]
        m = np.concatenate([self.m, np.zeros(len(away))])
        x = np.concatenate([self.xp, xi[away]])
        v = np.concatenate([self.vp, vi[away]])
        idx = np.where(here, local, 0).astype(np.int64)
        idx[away] = N + np.arange(len(away))
        a, j, p = oracle.forces(m, x, v, self.eps, idx=idx)
        for dst, val in ((acc, a), (jerk, j), (pot, p)):
            d = _np(dst)
            d[...] = d + val if accumulate else val
