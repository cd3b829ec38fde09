"""Train the learned selector on solves the library itself times, and save
the weights the package ships (selector_weights.npz).

    python -m paper_2406_16499_gb300.train_selector [--lse 1000] [--gls 1000]
        [--seed 7] [--out paper_2406_16499_gb300/selector_weights.npz]
        [--timings selector_weights_timings.npz]

For every training problem (LSE and GLS problems with kappa_2 log-uniform in
[1, 1e12], random xLATM1 patterns) the six classes {BF16, FP32, FP64}
factorization x {classical IR, GMRES-IR} are solved without escalation and
timed with the library's CUDA events (refinement capped at 20 steps and
200 GMRES iterations per step, so that hopeless classes stop early); the
label is the fastest class that converged (ties within 3 % go to the higher
precision, then to classical IR; GMRES-IR must beat classical IR at the
same precision by 25 %).  The features and class times are saved beside the
weights (<out>_timings.npz), so that the labels can be changed and the
network retrained without timing the solves again.  The 16 features come from the library's
feature kernel, the network is trained with its forward / backward / Adam
kernels.  Needs a GPU.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2406_16499_gb300 import inputs as I  # noqa: E402
from paper_2406_16499_gb300 import mpir  # noqa: E402
from paper_2406_16499_gb300 import selector as SEL  # noqa: E402

CAPS = dict(maxit=20, inner_maxit=200)


def collect(h, lse, gls, seed, log=None):
    """Features, per-class times and convergence flags of `lse` LSE and `gls`
    GLS training problems."""
    X, T, OK, kinds = [], [], [], []
    t0 = time.time()
    probs = [("lse", P) for P in I.selector_lse_problems(seed, lse)]
    probs += [("gls", G) for G in I.selector_gls_problems(seed + 1, gls)]
    for k, (kind, P) in enumerate(probs):
        if kind == "lse":
            times, ok = SEL.time_lse_classes(h, P, **CAPS)
            f = SEL.lse_features(h, P)
        else:
            times, ok = SEL.time_gls_classes(h, P, **CAPS)
            f = SEL.gls_features(h, P)
        X.append(f)
        T.append(times)
        OK.append(ok)
        kinds.append(kind)
        if log and (k + 1) % 200 == 0:
            log("%d / %d problems timed (%.0f s)" % (k + 1, len(probs), time.time() - t0))
    return np.array(X, np.float32), np.array(T, np.float64), np.array(OK, bool), kinds


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--lse", type=int, default=1000)
    ap.add_argument("--gls", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--out", default=os.path.join(HERE, "selector_weights.npz"))
    ap.add_argument("--timings", default=None,
                    help="reuse the features and class times saved by an earlier run (skips the timed solves)")
    a = ap.parse_args(argv)
    stem = os.path.splitext(a.out)[0]
    h = mpir.Handle()
    try:
        if a.timings:
            z = np.load(a.timings)
            X, T, OK, kinds = z["X"], z["times"], z["ok"], [str(k) for k in z["kinds"]]
        else:
            X, T, OK, kinds = collect(h, a.lse, a.gls, a.seed, log=lambda s: print(s, flush=True))
            np.savez(stem + "_timings.npz", X=X, times=T, ok=OK, kinds=np.array(kinds))
        y = np.array([SEL.label(t, o) for t, o in zip(T, OK)], np.int32)
        keep = y >= 0
        kinds = [k for k, q in zip(kinds, keep) if q]
        X, y = X[keep], y[keep]
        sel, losses = SEL.train(h, X, y, steps=a.steps, lr=3e-3)
        pred = np.argmax(sel.predict(h, X), axis=1)
    finally:
        h.close()
    sel.save(a.out)
    summary = {"problems_labelled": int(len(y)), "lse": kinds.count("lse"), "gls": kinds.count("gls"),
               "training_solves": 6 * int(len(T)), "label_histogram": np.bincount(y, minlength=6).tolist(),
               "final_loss": float(losses[-1][1]) if losses else None,
               "train_accuracy": float((pred == y).mean()), "classes": [list(c) for c in SEL.CLASSES]}
    with open(stem + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
