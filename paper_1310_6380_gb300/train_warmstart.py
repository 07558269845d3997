"""Train the warm-start network on bands the method itself computes.

    python -m paper_1310_6380_gb300.train_warmstart --cells 50000 --out <file.npz>

Training cells are the ragged-batch style cells with seeds 10^6 + i (lattice,
geometry and phase count as there), solved with truncation M = 5 for the
targets: the network predicts only the waves |alpha|, |beta| <= 3, whose
coefficients the larger truncations of the evaluation cells change little.
Each cell contributes `kper` wavevectors drawn uniformly from its 30-point
IBZ path.  The targets are the low-order coefficients of the lowest 10
eigenvectors from the batch solver (dense mixed path, bs_batch_set_vectors);
entries that fell back to the FP64 solve carry no vectors and are left out.  Training is
Adam on minibatches of cells with every kernel in the library (bs_cnn_*).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

from . import cells
from . import warmstart as ws

MP, NVEC, NB, M_TRAIN = 3, 12, 10, 5


def _make(i):
    c = cells.config4_train_cell(i)
    return c["cell"], c["Q"]


def generate_cells(n, procs):
    """Training cells, built in a spawn pool (the generator is pure Python)."""
    if procs <= 1:
        return [_make(i) for i in range(n)]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_make, range(n), chunksize=64)


def make_targets(cell_list, paths, kper, seed, chunk, log):
    """(Q (C, kper, 2), V (C, kper, NB, L), keep mask (C, kper)) from batch solves."""
    from . import binding as bs
    rng = np.random.default_rng(seed)
    C = len(cell_list)
    pick = np.stack([rng.choice(len(p), kper, replace=False) for p in paths])
    Q = np.stack([paths[c][pick[c]] for c in range(C)])
    L = 2 * (2 * MP + 1) ** 2
    V = np.empty((C, kper, NB, L), np.complex64)
    keep = np.zeros((C, kper), bool)
    for c0 in range(0, C, chunk):
        sl = slice(c0, min(C, c0 + chunk))
        t0 = time.time()
        w, st, it, fb, vec = ws.solve_batch(cell_list[sl], [M_TRAIN] * (sl.stop - sl.start),
                                            np.ascontiguousarray(Q[sl]), NB, bs.BS_SOLVER_DENSE,
                                            Mp=MP, vectors=True)
        V[sl] = vec
        keep[sl] = (fb == 0) & np.isfinite(vec).all(axis=(2, 3))
        log(f"targets {sl.stop}/{C}: {time.time() - t0:.1f} s, fallbacks {int(fb.sum())}")
    return Q, V, keep


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cells", type=int, default=50000)
    ap.add_argument("--kper", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch-cells", type=int, default=64)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--chunk", type=int, default=4096, help="cells per batch solve")
    ap.add_argument("--procs", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)

    def log(msg):
        print(msg, file=sys.stderr, flush=True)

    t0 = time.time()
    made = generate_cells(a.cells, a.procs)
    cell_list = [m[0] for m in made]
    paths = [m[1] for m in made]
    log(f"{a.cells} cells generated in {time.time() - t0:.1f} s")
    t1 = time.time()
    Q, V, keep = make_targets(cell_list, paths, a.kper, a.seed, a.chunk, log)
    t_data = time.time() - t1
    # drop cells with any sample missing (keeps the kper-per-cell layout)
    good = keep.all(axis=1)
    pack = ws.CellPack([cell_list[i] for i in np.flatnonzero(good)])
    Q, V = Q[good], V[good]
    log(f"training samples: {int(good.sum())} cells x {a.kper} k")
    net = ws.WarmStartNet(NVEC, MP, max_cells=a.batch_cells, max_samples=a.batch_cells * a.kper,
                          seed=a.seed)
    t2 = time.time()
    hist = ws.train(net, pack, Q, V, a.epochs, a.batch_cells, a.lr, seed=a.seed + 1, log=log)
    t_train = time.time() - t2
    p = net.params()
    meta = dict(cells=int(good.sum()), kper=a.kper, epochs=a.epochs, lr=a.lr,
                batch_cells=a.batch_cells, M_train=M_TRAIN, Mp=MP, nvec=NVEC, nb=NB,
                loss_per_epoch=hist, seconds_targets=t_data, seconds_training=t_train,
                seeds="1e6 + i")
    np.savez_compressed(a.out, params=p, meta=json.dumps(meta))
    log(json.dumps(meta))
    net.close()


if __name__ == "__main__":
    main()
