"""Starting subspaces for the block LOBPCG eigen path: the layout of the
low-order plane-wave coefficients that a warm start supplies.

A displacement eigenvector u of a cell with truncation M has n = 2N
coefficients, index I*N + a with component I in {x, y} and plane wave
a = (alpha + M)(2M + 1) + (beta + M) (the index map of Sec. IV.A).  A warm
start gives only the waves |alpha|, |beta| <= Mp (Mp <= M), in the same
component-major order with the index map of truncation Mp; the library sets
the others to zero.
"""
from __future__ import annotations

import numpy as np


def low_order_index(M: int, Mp: int) -> np.ndarray:
    """Positions, in a length-2N vector of truncation M, of the 2 (2Mp+1)^2
    coefficients of a truncation-Mp vector (component-major)."""
    if not 0 <= Mp <= M:
        raise ValueError("need 0 <= Mp <= M")
    r = np.arange(-Mp, Mp + 1)
    al = np.repeat(r, 2 * Mp + 1)
    be = np.tile(r, 2 * Mp + 1)
    a = (al + M) * (2 * M + 1) + (be + M)
    N = (2 * M + 1) ** 2
    return np.concatenate([a, N + a])


def truncate(U: np.ndarray, M: int, Mp: int) -> np.ndarray:
    """(..., 2N) coefficient vectors of truncation M -> (..., 2 (2Mp+1)^2)."""
    return np.ascontiguousarray(U[..., low_order_index(M, Mp)])


# ------------------------------------------------------------------ network inputs
class CellPack:
    """The network's per-cell inputs in the library's layout: 64 x 64 phase
    maps, concatenated (lam | mu | rho) tables with offsets, phase counts and
    lattice flags."""

    def __init__(self, cell_list):
        for c in cell_list:
            if c.P != 64:
                raise ValueError("the warm-start network takes 64 x 64 cells")
        self.n = len(cell_list)
        self.phase = np.ascontiguousarray(np.stack([c.phase for c in cell_list]), np.uint16)
        tabs, offs, o = [], [], 0
        for c in cell_list:
            offs.append(o)
            tabs += [c.lam, c.mu, c.rho]
            o += 3 * len(c.lam)
        self.table = np.ascontiguousarray(np.concatenate(tabs), np.float64)
        self.toff = np.array(offs, np.int64)
        self.nph = np.array([len(c.lam) for c in cell_list], np.int32)
        self.hexflag = np.array([1 if c.lattice == "hex" else 0 for c in cell_list], np.int32)

    def subset(self, idx):
        """Inputs of the cells idx (a new pack sharing nothing)."""
        sub = CellPack.__new__(CellPack)
        idx = np.asarray(idx)
        sub.n = len(idx)
        sub.phase = np.ascontiguousarray(self.phase[idx])
        tabs, offs, o = [], [], 0
        for i in idx:
            t = self.table[self.toff[i]:self.toff[i] + 3 * self.nph[i]]
            offs.append(o)
            tabs.append(t)
            o += len(t)
        sub.table = np.ascontiguousarray(np.concatenate(tabs))
        sub.toff = np.array(offs, np.int64)
        sub.nph = np.ascontiguousarray(self.nph[idx])
        sub.hexflag = np.ascontiguousarray(self.hexflag[idx])
        return sub


def init_params(nvec: int, Mp: int, seed: int) -> np.ndarray:
    """He-normal weights (fan-in), zero biases; the last layer scaled by 1/4.
    The random numbers come from numpy's seeded generator."""
    from . import binding as bs   # noqa: F401  (layout is fixed by the library)
    rng = np.random.default_rng(seed)
    parts = []
    conv = [(3, 16), (16, 32), (32, 32), (32, 32)]
    for ci, co in conv:
        parts.append(rng.standard_normal(co * ci * 9) * np.sqrt(2.0 / (ci * 9)))
        parts.append(np.zeros(co))
    out = nvec * 2 * (2 * Mp + 1) ** 2 * 2
    dims = [(512 + 7, 512), (512, 512), (512, out)]
    for l, (di, do) in enumerate(dims):
        sc = np.sqrt(2.0 / di) * (0.25 if l == 2 else 1.0)
        parts.append(rng.standard_normal(do * di) * sc)
        parts.append(np.zeros(do))
    return np.ascontiguousarray(np.concatenate(parts), np.float32)


class WarmStartNet:
    """Handle of the library's network (bs_cnn_*)."""

    def __init__(self, nvec=12, Mp=3, max_cells=256, max_samples=1024, seed=0):
        from . import binding as bs
        self.bs, self.nvec, self.Mp = bs, nvec, Mp
        self.L = 2 * (2 * Mp + 1) ** 2
        self.h = bs.bs_cnn_create(nvec, Mp, max_cells, max_samples)
        self.max_cells, self.max_samples = max_cells, max_samples
        self.set_params(init_params(nvec, Mp, seed))

    def close(self):
        if self.h is not None:
            self.bs.bs_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        return self.bs.bs_cnn_num_params(self.h)

    def set_params(self, p):
        self.bs.bs_cnn_set_params(self.h, np.ascontiguousarray(p, np.float32))

    def params(self):
        p = np.empty(self.num_params(), np.float32)
        self.bs.bs_cnn_get_params(self.h, p, None)
        return p

    def grads(self):
        g = np.empty(self.num_params(), np.float32)
        self.bs.bs_cnn_get_params(self.h, None, g)
        return g

    def predict(self, pack: CellPack, Q: np.ndarray) -> np.ndarray:
        """Q (cells, kper, 2) -> starting vectors (cells, kper, nvec, L) complex64."""
        C, kper = Q.shape[0], Q.shape[1]
        out = np.empty((C, kper, self.nvec, self.L), np.complex64)
        step = max(1, min(self.max_cells, self.max_samples // kper))
        for c0 in range(0, C, step):
            idx = np.arange(c0, min(C, c0 + step))
            sub = pack.subset(idx)
            Qs = np.ascontiguousarray(Q[idx].reshape(-1, 2), np.float64)
            raw = np.empty((len(idx) * kper, self.nvec * self.L * 2), np.float32)
            self.bs.bs_cnn_forward(self.h, sub.phase, sub.table, sub.toff, sub.nph, sub.hexflag,
                                   Qs, kper, raw)
            out[idx] = raw.view(np.complex64).reshape(len(idx), kper, self.nvec, self.L)
        return out

    def train_step(self, pack: CellPack, Q: np.ndarray, V: np.ndarray, lr: float):
        """Q (cells, kper, 2), V (cells, kper, nb, L) complex64: per-sample losses."""
        C, kper = Q.shape[0], Q.shape[1]
        loss = np.empty(C * kper, np.float32)
        self.bs.bs_cnn_train_step(self.h, pack.phase, pack.table, pack.toff, pack.nph,
                                  pack.hexflag, np.ascontiguousarray(Q.reshape(-1, 2), np.float64),
                                  kper, np.ascontiguousarray(V.reshape(C * kper, V.shape[2], -1),
                                                             np.complex64), lr, loss)
        return loss


# ------------------------------------------------------------------ data and training
def solve_batch(cell_list, M_list, Q, nbands, solver, start=None, Mp=3, vectors=False,
                graph=False):
    """One ragged batch through bs_batch_*: omega (cells, nk, nbands), status,
    LOBPCG iterations, fallback flags and (optional) low-order eigenvectors."""
    from . import binding as bs
    args = [(c.h1, c.h2, np.ascontiguousarray(c.phase, np.uint16), c.lam.copy(), c.mu.copy(),
             c.rho.copy(), M, bs.BS_PREC_MIXED) for c, M in zip(cell_list, M_list)]
    C, nk = Q.shape[0], Q.shape[1]
    b = bs.bs_batch_create(args, nk, nbands)
    try:
        bs.bs_batch_set_solver(b, solver)
        if start is not None:
            bs.bs_batch_set_start(b, np.ascontiguousarray(start, np.complex64), Mp)
        if vectors:
            bs.bs_batch_set_vectors(b, Mp)
        if graph:
            bs.bs_batch_set_graph(b, True)
        w = np.empty((C, nk, nbands))
        st = np.empty((C, nk), np.int32)
        bs.bs_batch_solve(b, np.ascontiguousarray(Q, np.float64), w, st)
        it, fb = bs.bs_batch_stats(b, C * nk)
        vec = None
        if vectors:
            vec = np.empty((C, nk, nbands, 2 * (2 * Mp + 1) ** 2), np.complex64)
            bs.bs_batch_vectors(b, vec)
    finally:
        bs.bs_batch_destroy(b)
    return w, st, it.reshape(C, nk), fb.reshape(C, nk), vec


def train(net: WarmStartNet, pack: CellPack, Q: np.ndarray, V: np.ndarray, epochs: int,
          cells_per_step: int, lr: float, seed: int = 0, log=None):
    """Adam on minibatches of cells (all of a cell's kper samples together).
    Q (cells, kper, 2), V (cells, kper, nb, L).  Returns the mean loss per epoch."""
    rng = np.random.default_rng(seed)
    C = Q.shape[0]
    hist = []
    for ep in range(epochs):
        order = rng.permutation(C)
        tot, cnt = 0.0, 0
        for s0 in range(0, C - cells_per_step + 1, cells_per_step):
            idx = np.sort(order[s0:s0 + cells_per_step])
            loss = net.train_step(pack.subset(idx), Q[idx], V[idx], lr)
            tot += float(loss.sum())
            cnt += loss.size
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist
