"""Learned work estimator: data collection, training and use.

The plain method logs, for every root, the number of Bron-Kerbosch calls of
its first-level subtree (mce_run's per-root tree nodes). A small network,
16 -> 64 -> 64 -> 1 with BF16 weights and FP32 accumulation, learns log2 of
that count from 16 root features (mce_root_features). Its prediction orders
the roots (heaviest first, MCE_ORDER_PRIORITY); the results never change.
Every arithmetic step -- features, forward, backward, Adam -- runs in the
library's kernels; this module only moves tensors between those calls.

    python -m paper_2212_01473_gb300.learn train [--out FILE]
    python -m paper_2212_01473_gb300.learn eval  [--model FILE]

Training data: the Erdos-Renyi (n=2000, m=20000) and Chung-Lu (n=10^6)
workload families regenerated with seeds 10-73; evaluation: seeds 100-103.
"""
import argparse
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import engine as E

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "work_model.json")
TRAIN_SEEDS = range(10, 74)
EVAL_SEEDS = range(100, 104)
FAMILIES = ("er_2000", "chunglu_1m")


def _gen(family, seed):
    sys.path.insert(0, os.path.dirname(HERE))
    import gen
    return gen.workload(family, seed=seed)


def collect(g, light_keep=10000, seed=0):
    """(features [k,16] CUDA float32, labels [k] CUDA float32 = log2 tree nodes)
    for the graph's roots: every root with |P0| > 32 plus `light_keep` others."""
    import torch
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    h = E.mce_create(rp, col)
    try:
        feat = E.mce_root_features(h)
        nodes = torch.zeros(max(g.n, 1), dtype=torch.int64, device="cuda")
        o = E.mce_default_opts()
        o.root_nodes = nodes.data_ptr()
        E.mce_run(h, o)
        torch.cuda.synchronize()
    finally:
        E.mce_destroy(h)
    nodes = nodes[: g.n]
    label = torch.log2(nodes.clamp(min=1).double()).float()
    p0 = feat[:, 2]  # log2(1 + |P0|)
    heavy = torch.nonzero(p0 > np.log2(33.0)).flatten()
    light = torch.nonzero(p0 <= np.log2(33.0)).flatten()
    if len(light) > light_keep:
        gen_ = torch.Generator(device="cpu").manual_seed(seed)
        light = light[torch.randperm(len(light), generator=gen_)[:light_keep].cuda()]
    sel = torch.cat([heavy, light])
    return feat[sel].contiguous(), label[sel].contiguous()


def init_params(mean, std, seed=0):
    """He-uniform weights, zero biases, the given standardisation."""
    rs = np.random.default_rng(seed)
    p = np.zeros(E.MCE_MODEL_PARAMS, np.float32)
    F, H = 16, 64
    off = 0
    for fan_in, fan_out in ((F, H), (H, H), (H, 1)):
        lim = np.sqrt(6.0 / fan_in)
        p[off:off + fan_in * fan_out] = rs.uniform(-lim, lim, fan_in * fan_out)
        off += fan_in * fan_out + fan_out
    p[-32:-16] = mean
    p[-16:] = np.maximum(std, 1e-3)
    return p


def gather(families=FAMILIES, seeds=TRAIN_SEEDS, threads=8, log=print):
    import torch
    feats, labels = [], []
    jobs = [(f, s) for s in seeds for f in families]
    with ThreadPoolExecutor(threads) as ex:
        futs = [ex.submit(_gen, f, s) for f, s in jobs]
        for (f, s), fut in zip(jobs, futs):
            x, y = collect(fut.result(), seed=s)
            feats.append(x)
            labels.append(y)
            log("collected %s seed %d: %d roots" % (f, s, len(y)))
    return torch.cat(feats), torch.cat(labels)


def train(feat, label, epochs=4, batch=4096, lr=2e-3, seed=0, log=print):
    """Adam on the library's gradient kernel; returns (model, history)."""
    import torch
    x = feat.double()
    mean = x.mean(0).cpu().numpy()
    std = x.std(0).cpu().numpy()
    model = E.Model(init_params(mean, std, seed))
    n = len(label)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        losses = []
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            losses.append(model.train_step(feat[idx].contiguous(), label[idx].contiguous(), lr,
                                           want_loss=(i // batch) % 64 == 0))
        lr *= 0.5
        ls = [v for v in losses if v is not None]
        hist.append(float(np.mean(ls)))
        log("epoch %d: mean sampled loss %.4f" % (ep, hist[-1]))
    return model, hist


def spearman(a, b):
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    return float(np.corrcoef(ra, rb)[0, 1])


def save(model, path, meta):
    with open(path, "w") as f:
        json.dump({"params": [float(v) for v in model.params()], "meta": meta}, f)


def load(path=DEFAULT_MODEL):
    with open(path) as f:
        d = json.load(f)
    return E.Model(np.array(d["params"], np.float32)), d.get("meta", {})


def priority(model, h, min_p=33):
    """Predicted log2 subtree size per root (CUDA float32 [n], by input id);
    roots with fewer than min_p later neighbours are not scored (-1)."""
    return E.mce_predict_priority(h, model, min_p)


def evaluate(model, families=FAMILIES, seeds=EVAL_SEEDS, repeats=3, log=print):
    """Held-out error, rank correlation, and traversal time with plain,
    learned and true-label root orders (all with the default worker list)."""
    import torch
    rows = []
    for fam in families:
        for s in seeds:
            g = _gen(fam, s)
            rp = torch.from_numpy(g.row_ptr).cuda()
            col = torch.from_numpy(g.col).cuda()
            h = E.mce_create(rp, col)
            nodes = torch.zeros(max(g.n, 1), dtype=torch.int64, device="cuda")
            o = E.mce_default_opts()
            o.root_nodes = nodes.data_ptr()
            base = E.mce_run(h, o)
            truth = torch.log2(nodes[: g.n].clamp(min=1).double()).float().contiguous()
            full = model.predict(E.mce_root_features(h))  # every root, for the accuracy figures
            pred = priority(model, h)                     # what the ordering uses
            torch.cuda.synchronize()
            # the priority pass itself (features + network for the scored roots)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            priority(model, h)
            e1.record()
            e1.synchronize()
            ms_priority = e0.elapsed_time(e1)
            _, rank, _ = E.mce_get_order(h)
            t, p = truth.cpu().numpy(), full.cpu().numpy()
            heavy = t > 1.0
            row = {"family": fam, "seed": s, "mse": float(np.mean((p - t) ** 2)),
                   "spearman": spearman(p, t), "spearman_nontrivial": spearman(p[heavy], t[heavy]) if heavy.sum() > 2 else None,
                   "spearman_rank_nontrivial": spearman(rank[heavy], t[heavy]) if heavy.sum() > 2 else None,
                   "ms_priority": ms_priority}
            for name, pr in (("plain", None), ("learned", pred), ("true", truth)):
                ms = []
                for _ in range(repeats):
                    o = E.mce_default_opts()
                    if pr is not None:
                        o.order = E.MCE_ORDER_PRIORITY
                        o.root_priority = pr.data_ptr()
                    r = E.mce_run(h, o)
                    assert (r.count, r.hash) == (base.count, base.hash)
                    ms.append(r.ms_traverse)
                row["ms_" + name] = float(np.median(ms))
            E.mce_destroy(h)
            rows.append(row)
            log(json.dumps(row))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval", "reeval"])
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--model", default=DEFAULT_MODEL)
    ap.add_argument("--epochs", type=int, default=4)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.init()
    if args.cmd == "train":
        t0 = time.time()
        feat, label = gather()
        t1 = time.time()
        model, hist = train(feat, label, epochs=args.epochs)
        t2 = time.time()
        rows = evaluate(model)
        meta = {"train": "seeds %d-%d of %s" % (TRAIN_SEEDS[0], TRAIN_SEEDS[-1], ", ".join(FAMILIES)),
                "samples": int(len(label)), "epochs": args.epochs, "loss_history": hist,
                "collect_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 2), "eval": rows}
        save(model, args.out, meta)
        print(json.dumps({"saved": args.out, "samples": int(len(label)), "train_s": round(t2 - t1, 2)}))
    elif args.cmd == "reeval":
        # the held-out evaluation again, with the current engine, stored in the model file
        model, meta = load(args.model)
        meta["eval"] = evaluate(model)
        meta["eval_note"] = "held-out seeds re-evaluated with the current traversal kernel"
        save(model, args.out, meta)
    else:
        model, meta = load(args.model)
        evaluate(model)


if __name__ == "__main__":
    main()
