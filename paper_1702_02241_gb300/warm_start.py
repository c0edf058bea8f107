"""Training and evaluation driver of the learned warm start (argument marshalling and
bookkeeping only: instance generation, the solves, the features/targets, the network's
training steps and inference all run in the library's CUDA kernels through its C ABI).

Protocol (the planted training/held-out workloads):
* Training instances: m x n = 4096 x 256, planted rank r ~ U{1..10}, factor rank
  k = min(16, r + d) with d ~ U{1..6}, outlier rate ~ U[0.02, 0.08] with +-U[1, 5], noise
  1e-3, generated on the device (rpca_gen_planted, Philox4x32-10; instance i of a seed).
  lam_S = 1 / sqrt(max(m, n)), lam_L = lam_S (sqrt(m) + sqrt(n)).
* Sample of an instance: the sketch start (rpca_init_sketch), the plain solve from it to the
  certificate, then rpca_ws_sample: features of the sketch spectrum and the targets w*.
* Training: Adam, batches of 256, a cosine-decayed step size, the samples reshuffled every
  epoch (on the host; each epoch's order is uploaded once).
* Evaluation: held-out instances solved from the sketch start, the learned start and the
  random start; iterations and time-to-certificate (wall time of rpca_solve) per start.
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np
import torch

from . import gen, rpca
from .engine import ld_for

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS_PATH = os.path.join(HERE, "ws_params_planted4096x256.npy")
FEAT, OUT = 40, 16


def default_model(stream=None):
    """The model trained by this module's protocol (5000 planted 4096 x 256 instances), as a
    library handle for rpca_set_warm_start (release it with rpca_ws_destroy)."""
    return rpca.rpca_ws_create(np.load(PARAMS_PATH), stream)


def init_params(seed=0):
    """He-normal hidden layers, a small output layer, zero biases (w = 1/2 at the start)."""
    g = np.random.default_rng(seed)
    nparam = rpca.rpca_ws_nparam()
    th = np.zeros(nparam, np.float32)
    o = 0
    for rows, cols, std in ((256, FEAT, math.sqrt(2.0 / FEAT)), (256, 256, math.sqrt(2.0 / 256)),
                            (OUT, 256, 0.01)):
        th[o:o + rows * cols] = std * g.standard_normal(rows * cols)
        o += rows * cols + rows  # weights, then the biases (zero)
    assert o == nparam
    return th


def instance_params(count, seed, m=4096, n=256):
    """Host-side draws of the instances' shape parameters (rank, k, outlier rate)."""
    g = np.random.default_rng(seed)
    ranks = g.integers(1, 11, size=count)
    ks = np.minimum(16, ranks + g.integers(1, 7, size=count))
    ps = g.uniform(0.02, 0.08, size=count)
    return [dict(m=m, n=n, rank=int(r), k=int(k), p=float(p)) for r, k, p in zip(ranks, ks, ps)]


def lambdas(m, n):
    lam_S = 1.0 / math.sqrt(max(m, n))
    return lam_S * (math.sqrt(m) + math.sqrt(n)), lam_S


def _opts(init, max_iter=3000, cert_every=10, x_dtype=None):
    o = rpca.rpca_default_options()
    o.init = init
    o.max_iter = max_iter
    o.cert_every = cert_every
    if x_dtype is not None:
        o.x_dtype = x_dtype
        o.refine_fp32 = 1
    return o


def _factors(m, n, k):
    return (torch.zeros((k, m), dtype=torch.float32, device="cuda"),
            torch.zeros((k, n), dtype=torch.float32, device="cuda"))


def generate(spec, seed, instance):
    m, n = spec["m"], spec["n"]
    ld = ld_for(m)
    X = torch.empty((n, ld), dtype=torch.float32, device="cuda")
    rpca.rpca_gen_planted(m, n, spec["rank"], spec["p"], 1e-3, seed, instance, X, ld)
    return X, ld


def make_samples(specs, seed):
    """Features, targets and ranks (device tensors) of solved training instances."""
    N = len(specs)
    x = torch.zeros((N, FEAT), dtype=torch.float32, device="cuda")
    t = torch.zeros((N, OUT), dtype=torch.float32, device="cuda")
    K = torch.tensor([s["k"] for s in specs], dtype=torch.int32, device="cuda")
    iters = []
    for i, s in enumerate(specs):
        X, ld = generate(s, seed, i)
        lam_L, lam_S = lambdas(s["m"], s["n"])
        ctx = rpca.rpca_create(s["m"], s["n"], X, ld, None, 0, s["k"], lam_L, lam_S, _opts(rpca.RPCA_INIT_USER))
        Us, Vs = _factors(s["m"], s["n"], s["k"])
        rpca.rpca_init_sketch(ctx, None, Us, Vs)
        U, V = Us.clone(), Vs.clone()
        r = rpca.rpca_solve(ctx, U, V)
        iters.append(r.iters)
        rpca.rpca_ws_sample(ctx, Us, Vs, U, V, x[i], t[i])
        rpca.rpca_destroy(ctx)
    torch.cuda.synchronize()
    return x.cpu().numpy(), t.cpu().numpy(), K.cpu().numpy(), iters


def train(x, t, K, epochs=300, batch=256, lr=2e-3, seed=0, log=None):
    """Trains a fresh model on the samples (host arrays x: N x 40, t: N x 16, K: N); returns
    (model handle, [(epoch, loss of its first batch)])."""
    w = rpca.rpca_ws_create(init_params(seed))
    N = x.shape[0]
    batch = min(batch, N)
    g = np.random.default_rng(seed + 1)
    per_epoch = max(1, N // batch)
    steps = epochs * per_epoch
    step = 0
    losses = []
    for ep in range(epochs):
        perm = g.permutation(N)
        xs = torch.from_numpy(np.ascontiguousarray(x[perm])).cuda()
        ts = torch.from_numpy(np.ascontiguousarray(t[perm])).cuda()
        ks = torch.from_numpy(np.ascontiguousarray(K[perm])).cuda()
        for q in range(per_epoch):
            b0 = q * batch
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * step / steps))
            want = q == 0 and (ep % 10 == 0 or ep == epochs - 1)
            loss = rpca.rpca_ws_train_step(w, rpca.offset(xs, b0 * FEAT), rpca.offset(ts, b0 * OUT),
                                           rpca.offset(ks, b0), batch, cur, want_loss=want)
            if want:
                losses.append((ep, loss))
                if log:
                    log(f"epoch {ep} loss {loss:.5f}")
            step += 1
    return w, losses


def predict(w, x):
    """Network outputs (host N x 16) for host features x (N x 40)."""
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    out = torch.zeros((x.shape[0], OUT), dtype=torch.float32, device="cuda")
    rpca.rpca_ws_predict(w, xd, x.shape[0], out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def evaluate(w, specs, seed, starts=("sketch", "learned", "random")):
    """Per start: iterations, time-to-certificate (s), certified count, learned-start use."""
    kinds = {"sketch": rpca.RPCA_INIT_SKETCH, "learned": rpca.RPCA_INIT_LEARNED, "random": rpca.RPCA_INIT_RANDOM}
    res = {s: {"iters": [], "seconds": [], "ok": 0, "used": 0, "F": []} for s in starts}
    for i, s in enumerate(specs):
        X, ld = generate(s, seed, i) if "X" not in s else (s["X"], s["ld"])
        lam_L, lam_S = (s["lam_L"], s["lam_S"]) if "lam_L" in s else lambdas(s["m"], s["n"])
        for st in starts:
            ctx = rpca.rpca_create(s["m"], s["n"], X, ld, None, 0, s["k"], lam_L, lam_S, _opts(kinds[st]))
            if st == "learned":
                rpca.rpca_set_warm_start(ctx, w)
            U, V = _factors(s["m"], s["n"], s["k"])
            r = rpca.rpca_solve(ctx, U, V)
            torch.cuda.synchronize()
            d = res[st]
            d["iters"].append(r.iters)
            d["seconds"].append(r.seconds)
            d["F"].append(r.F)
            d["ok"] += int(r.status == rpca.RPCA_OK)
            d["used"] += int(r.init_used == rpca.RPCA_INIT_LEARNED)
            rpca.rpca_destroy(ctx)
    return res


def evaluate_batch(w, specs, seed, reps=2):
    """The held-out instances solved as one batch (rpca_solve_batch), from the sketch starts and
    from the learned starts: wall time per batch (best of reps), iterations, certified count."""
    Xs, lds = zip(*[generate(s, seed, i) for i, s in enumerate(specs)])
    lams = [lambdas(s["m"], s["n"]) for s in specs]
    out = {}
    for name, kind in (("sketch", rpca.RPCA_INIT_SKETCH), ("learned", rpca.RPCA_INIT_LEARNED)):
        b = rpca.rpca_create_batch(list(Xs), [(s["m"], ld) for s, ld in zip(specs, lds)], [s["k"] for s in specs],
                                   [l[0] for l in lams], [l[1] for l in lams], _opts(kind))
        if kind == rpca.RPCA_INIT_LEARNED:
            for i in range(len(specs)):
                rpca.rpca_set_warm_start(rpca.rpca_batch_context(b, i), w)
        best = None
        for _ in range(reps):
            Us, Vs = zip(*[_factors(s["m"], s["n"], s["k"]) for s in specs])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, res = rpca.rpca_solve_batch(b, list(Us), list(Vs))
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if best is None or dt < best[0]:
                best = (dt, sum(r.iters for r in res), sum(r.status == rpca.RPCA_OK for r in res),
                        sum(r.init_used == rpca.RPCA_INIT_LEARNED for r in res))
        out[name] = {"batch_seconds": best[0], "iters": best[1], "certified": best[2], "learned_start_kept": best[3],
                     "count": len(specs)}
        rpca.rpca_destroy_batch(b)
    return out


def evaluate_combined(w, specs, seed, reps=2):
    """The end-to-end comparison on instances whose rank the narrow storage supports (k <= 8):
    the plain float32 solver one instance after another from the sketch start, against the
    batched form from the learned starts in float32 and with X stored in bfloat16 (float32
    refinement to the same certificate).  Wall time for the whole set (best of reps), total
    iterations, certified count (the float32 certificate at cert_tol 1e-4 in every form)."""
    specs = [s for s in specs if s["k"] <= 8]
    Xs, lds = zip(*[generate(s, seed, i) for i, s in enumerate(specs)])
    lams = [lambdas(s["m"], s["n"]) for s in specs]
    out = {"count": len(specs)}
    best = None
    for _ in range(reps):
        ctxs = [rpca.rpca_create(s["m"], s["n"], X, ld, None, 0, s["k"], l[0], l[1], _opts(rpca.RPCA_INIT_SKETCH))
                for s, X, ld, l in zip(specs, Xs, lds, lams)]
        fac = [_factors(s["m"], s["n"], s["k"]) for s in specs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = [rpca.rpca_solve(c, U, V) for c, (U, V) in zip(ctxs, fac)]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for c in ctxs:
            rpca.rpca_destroy(c)
        if best is None or dt < best[0]:
            best = (dt, sum(r.iters for r in res), sum(r.status == rpca.RPCA_OK for r in res))
    out["plain_f32_one_by_one"] = {"seconds": best[0], "iters": best[1], "certified": best[2]}
    for name, xd in (("learned_batched_f32", None), ("learned_batched_bf16", rpca.RPCA_BF16)):
        b = rpca.rpca_create_batch(list(Xs), [(s["m"], ld) for s, ld in zip(specs, lds)], [s["k"] for s in specs],
                                   [l[0] for l in lams], [l[1] for l in lams],
                                   _opts(rpca.RPCA_INIT_LEARNED, x_dtype=xd))
        for i in range(len(specs)):
            rpca.rpca_set_warm_start(rpca.rpca_batch_context(b, i), w)
        best = None
        for _ in range(reps):
            Us, Vs = zip(*[_factors(s["m"], s["n"], s["k"]) for s in specs])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, res = rpca.rpca_solve_batch(b, list(Us), list(Vs))
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if best is None or dt < best[0]:
                best = (dt, sum(r.iters for r in res), sum(r.status == rpca.RPCA_OK for r in res))
        out[name] = {"seconds": best[0], "iters": best[1], "certified": best[2]}
        rpca.rpca_destroy_batch(b)
    return out


def summary(res):
    out = {}
    for st, d in res.items():
        out[st] = {"mean_iters": float(np.mean(d["iters"])), "median_iters": float(np.median(d["iters"])),
                   "mean_seconds": float(np.mean(d["seconds"])), "median_seconds": float(np.median(d["seconds"])),
                   "certified": d["ok"], "count": len(d["iters"]), "learned_start_kept": d["used"]}
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start")
    ap.add_argument("--train", type=int, default=5000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--video", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed", type=int, default=20170207)
    ap.add_argument("--out", default=PARAMS_PATH)
    ap.add_argument("--json", default=None)
    ap.add_argument("--load", action="store_true", help="evaluate the saved parameters instead of training")
    ap.add_argument("--combined", type=int, default=0,
                    help="draw this many held-out instances and compare, on those with k <= 8, the plain float32 "
                         "solver one by one with the learned + batched form in float32 and in bfloat16")
    ap.add_argument("--batch-eval", type=int, default=0,
                    help="also solve this many held-out instances as one batch, sketch vs learned starts")
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)  # noqa: E731
    losses = []
    if a.load:
        w = rpca.rpca_ws_create(np.load(a.out))
    else:
        t0 = time.time()
        specs = instance_params(a.train, a.seed)
        x, t, K, it_train = make_samples(specs, a.seed)
        log(f"training set: {a.train} instances in {time.time() - t0:.1f} s, "
            f"mean sketch iterations {np.mean(it_train):.1f}")
        t1 = time.time()
        w, losses = train(x, t, K, epochs=a.epochs, seed=a.seed, log=log)
        log(f"training: {time.time() - t1:.1f} s")
        th, _ = rpca.rpca_ws_get_params(w)
        np.save(a.out, th)
    held = instance_params(a.heldout, a.seed + 1)
    res = summary(evaluate(w, held, a.seed + 1))
    log("held-out 4096x256: " + json.dumps(res))
    out = {"train": a.train, "epochs": a.epochs, "final_loss": losses[-1][1] if losses else None,
           "heldout_4096x256": res}
    if a.combined:
        rc = evaluate_combined(w, instance_params(a.combined, a.seed + 3), a.seed + 3)
        log("combined form on held-out instances with k <= 8: " + json.dumps(rc))
        out["combined_k_le_8"] = rc
    if a.batch_eval:
        rb = evaluate_batch(w, instance_params(a.batch_eval, a.seed + 2), a.seed + 2)
        log(f"held-out batch of {a.batch_eval}: " + json.dumps(rb))
        out["heldout_batch"] = rb
    if a.video:
        vids = []
        for i in range(a.video):
            inst = gen.video(h=240, w=320, n=500, rank=3, k=5, seed=1000 + i)
            Xd = torch.from_numpy(np.ascontiguousarray(inst.X.T)).cuda()
            vids.append(dict(m=inst.m, n=inst.n, k=inst.k, X=Xd, ld=inst.m, lam_L=inst.lam_L, lam_S=inst.lam_S))
        resv = summary(evaluate(w, vids, 0))
        log("held-out video 76800x500: " + json.dumps(resv))
        out["heldout_video_76800x500"] = resv
    if a.json:
        with open(a.json, "w") as f:
            json.dump(out, f, indent=1)
    rpca.rpca_ws_destroy(w)
    return 0


if __name__ == "__main__":
    sys.exit(main())
