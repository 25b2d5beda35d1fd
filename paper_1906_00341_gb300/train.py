"""Training driver of the density-proposal network.

Not in the paper.  The network (libdsd: dsd_model_*) maps the 64 graph
statistics of dsd_graph_features to log(1 + rho'), where rho' should be a
lower bound of the density of the densest level set S* that CoreApp reports
(the level sets R_k of the (k,Psi)-core decomposition, Def. 6; densest level
as in Pruning1 of Sec. 5.1).  Labels come from the plain CUDA path
(dsd_core_app); the loss is the pinball loss at quantile q = 0.05, so that
about 95% of the proposals fall at or below the label; Adam, batch 256.

A proposal that overshoots only costs time: dsd_core_app_seeded tests it
exactly and falls back to the full decomposition.

The training set mixes two families of generated graphs (graphgen): small
ones of many shapes (train_graph: ER, Chung-Lu, planted blocks; n <= 200,000)
and large ones shaped like the evaluation workload (train_large_graph:
Chung-Lu plus planted blocks, n 100,000 .. 2,000,000), all with seeds never
used for evaluation.

Usage (one GPU):
    python -m paper_1906_00341_gb300.train --graphs 19000 --large 1000 --out proposal_h3.npz

Checkpoints are .npz files holding the flat float32 state (parameters, Adam
moments, step) with a header: format version, parameter count, clique size,
and the SHA-256 of the state bytes, checked on load.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import _lib
from . import graphgen as gg

FORMAT = 1
DEFAULT_CHECKPOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_h3.npz")


# ------------------------------------------------------------------ labels

def label_graph(n, src, dst, h):
    """(features [64] float32, label log1p(rho(S*)), densest (mu, size), m)."""
    with _lib.Graph.from_edges(n, src, dst) as g:
        f = g.features(h)
        r = g.core_app(h, sets=False)
        mu, size = r["densest_mu"], r["densest_size"]
        rho = mu / size if size else 0.0
        return f, math.log1p(rho), (mu, size), g.m


def _gen(i):
    return gg.train_graph(i)


def _gen_large(i):
    return gg.train_large_graph(i)


def make_dataset(count, start=0, workers=8, log=print, large=False):
    """Generate training graphs start .. start+count-1 (of the small family,
    or with large=True of the large one) on host processes and label them
    on the GPU.  Returns a dict of arrays."""
    X = np.zeros((count, _lib.NFEAT), np.float32)
    y = np.zeros(count, np.float32)
    mus = np.zeros(count, np.uint64)
    sizes = np.zeros(count, np.uint32)
    ns = np.zeros(count, np.uint32)
    ms = np.zeros(count, np.uint64)
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        gen = _gen_large if large else _gen
        for j, (n, s, d, h) in enumerate(pool.imap(gen, range(start, start + count),
                                                   1 if large else 16)):
            f, lab, (mu, size), m = label_graph(n, s, d, h)
            X[j], y[j], mus[j], sizes[j], ns[j], ms[j] = f, lab, mu, size, n, m
            if log and ((j + 1) % 1000 == 0 or (large and (j + 1) % 100 == 0)):
                log("labelled %d/%d graphs (%.1f s)" % (j + 1, count, time.time() - t0))
    return dict(X=X, y=y, mu=mus, size=sizes, n=ns, m=ms,
                index=np.arange(start, start + count, dtype=np.int64))


# -------------------------------------------------------------- training

def train(X, y, epochs=30, batch=256, q=0.05, lr=1e-3, seed=0, val_frac=0.1, log=print,
          model=None):
    """Adam on the pinball loss; returns (model, history)."""
    rng = np.random.default_rng(seed)
    N = len(y)
    perm = rng.permutation(N)
    nval = int(N * val_frac)
    val, tr = perm[:nval], perm[nval:]
    M = model or _lib.Model(seed=seed)
    hist = []
    for ep in range(epochs):
        rng.shuffle(tr)
        losses = []
        # cosine decay of the learning rate over the run
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / max(epochs, 1)))
        for a in range(0, len(tr), batch):
            idx = tr[a:a + batch]
            if len(idx) == 0:
                continue
            losses.append(M.train_step(X[idx], y[idx], q, lr_ep))
        rec = dict(epoch=ep, train_loss=float(np.mean(losses)) if losses else 0.0)
        if nval:
            pred = predict(M, X[val])
            rec["val_loss"] = float(np.mean((y[val] - pred) * (q - (y[val] < pred))))
            rec["val_below"] = float(np.mean(pred <= y[val]))
        hist.append(rec)
        if log:
            log(json.dumps(rec))
    return M, hist


def predict(M, X):
    out = [M.forward(X[a:a + 1024]) for a in range(0, len(X), 1024)]
    return np.concatenate(out) if out else np.zeros(0, np.float32)


# ------------------------------------------------------------ checkpoints

def save_checkpoint(M, path, h=3, meta=None, with_optimizer=True):
    """Write M's state; without the optimizer, the Adam moments and step
    are stored as zeros (a smaller file for inference)."""
    st = M.state()
    if not with_optimizer:
        st[M.count:] = 0
    digest = hashlib.sha256(st.tobytes()).hexdigest()
    header = dict(format=FORMAT, params=int(M.count), h=int(h), sha256=digest, meta=meta or {})
    np.savez_compressed(path, state=st, header=np.array(json.dumps(header)))
    return digest


def load_checkpoint(path, stream=None):
    """A Model with the checkpoint's state (raises on a corrupt or foreign file)."""
    with np.load(path, allow_pickle=False) as z:
        st = z["state"].astype(np.float32)
        header = json.loads(str(z["header"]))
    if header.get("format") != FORMAT:
        raise ValueError("unknown checkpoint format %r" % header.get("format"))
    M = _lib.Model(seed=0, stream=stream)
    if header.get("params") != M.count or st.size != 3 * M.count + 1:
        raise ValueError("checkpoint holds %s parameters, the network has %d"
                         % (header.get("params"), M.count))
    if hashlib.sha256(st.tobytes()).hexdigest() != header.get("sha256"):
        raise ValueError("checkpoint state does not match its SHA-256")
    M.set_state(st)
    M.header = header
    return M


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--graphs", type=int, default=19000, help="small training graphs")
    ap.add_argument("--large", type=int, default=1000,
                    help="large training graphs (the evaluation workload's shape)")
    ap.add_argument("--large-workers", type=int, default=16)
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--q", type=float, default=0.05)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--dataset", default=None, help="reuse or write labelled data (.npz)")
    ap.add_argument("--out", default=DEFAULT_CHECKPOINT)
    ap.add_argument("--no-optimizer-state", action="store_true",
                    help="store the parameters only")
    a = ap.parse_args(argv)
    _lib.load()
    t0 = time.time()
    if a.dataset and os.path.exists(a.dataset):
        with np.load(a.dataset) as z:
            data = {k: z[k] for k in z.files}
    else:
        data = make_dataset(a.graphs, a.start, a.workers)
        if a.large:
            big = make_dataset(a.large, 0, a.large_workers, large=True)
            big["index"] = -1 - big["index"]          # large graph i is stored as -1 - i
            data = {k: np.concatenate([data[k], big[k]]) for k in data}
        if a.dataset:
            np.savez_compressed(a.dataset, **data)
    t1 = time.time()
    M, hist = train(data["X"], data["y"], a.epochs, a.batch, a.q, a.lr, a.seed)
    t2 = time.time()
    meta = dict(graphs=int(len(data["y"])), large=int(np.sum(data["index"] < 0)),
                start=int(a.start), epochs=a.epochs, batch=a.batch,
                q=a.q, lr=a.lr, seed=a.seed, label_s=round(t1 - t0, 1),
                train_s=round(t2 - t1, 1), final=hist[-1] if hist else {})
    digest = save_checkpoint(M, a.out, 3, meta, with_optimizer=not a.no_optimizer_state)
    print(json.dumps(dict(checkpoint=a.out, sha256=digest, **meta)))


if __name__ == "__main__":
    main()
