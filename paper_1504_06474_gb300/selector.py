"""Learned variant and tile-shape selector (not in the paper).

The library has several ways to compute the same y = A x: the speculative
segmented sum at four tile lengths, the exact-store variant, two warp counts,
and the row-parallel kernels.  Which is fastest depends on the row structure.
This module

* measures it: ``autotune`` times every class on a matrix on the GPU
  (CUDA events, L2 flushed before each run, median of a few runs);
* describes a matrix by 16 statistics of its row pointers, computed on the
  GPU by ``ssspmv_features`` (no pass over the entries);
* learns the map: a perceptron 16 -> 64 -> 64 -> K predicts log2 of every
  class's time, trained on the GPU by the library's own FP32 forward,
  backward and Adam kernels (``ssspmv_mlp_*``);
* chooses: the class of least predicted time (``ssspmv_mlp_select``); with no
  model, or non-finite features, the plain speculative kernel (class 0, the
  library's defaults) is the fallback.

The choice never changes the arithmetic of a class, only which class runs.

    python -m paper_1504_06474_gb300.selector --train 2000 --test 200 --out DIR

generates the seeded training and held-out matrices, measures every class,
trains, and writes ``DIR/selector_weights.json`` and ``DIR/selector_report.json``
(held-out regret against the measured optimum and speedup over the fixed
default).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import ssspmv as C

F, H1, H2 = 16, 64, 64

# (name, opts fields).  Class 0 is the fixed default: all library defaults.
CLASSES = [
    ("speculative W15 (default)", dict()),
    ("speculative W21", dict(W=21, variant=C.VARIANT_SPECULATIVE)),
    ("speculative W27", dict(W=27, variant=C.VARIANT_SPECULATIVE)),
    ("speculative W31", dict(W=31, variant=C.VARIANT_SPECULATIVE)),
    ("exact W15", dict(W=15, variant=C.VARIANT_EXACT)),
    ("exact W27", dict(W=27, variant=C.VARIANT_EXACT)),
    ("speculative W15, all warps", dict(W=15, variant=C.VARIANT_SPECULATIVE, block_warps=32)),
    ("speculative W15, 17 warps per block", dict(W=15, variant=C.VARIANT_SPECULATIVE,
                                                 block_warps=17)),
    ("rows, lanes by mean length", dict(W=0, variant=C.VARIANT_ROWS)),
    ("rows, one lane per row", dict(W=1, variant=C.VARIANT_ROWS)),
]
K = len(CLASSES)


def class_opts(k: int, timer=None):
    return C.make_opts(timer=timer, **CLASSES[k][1])


# ---------------------------------------------------------------------------
# features and timing on the GPU

def device_features(rp, m: int, n: int, nnz: int, stream=None):
    """The 16 features of a device row_ptr, as a device float32 tensor."""
    import torch
    f = torch.empty(F, dtype=torch.float32, device=rp.device)
    scratch = torch.empty(C.ssspmv_features_scratch_bytes(), dtype=torch.uint8, device=rp.device)
    C.check(C.ssspmv_features(m, n, nnz, rp, f, scratch, stream), "ssspmv_features")
    return f


@dataclass
class DeviceMatrix:
    m: int
    n: int
    nnz: int
    rp: object
    col: object
    val: object
    x: object
    y: object


def to_device(A, x, dev) -> DeviceMatrix:
    import torch
    return DeviceMatrix(A.m, A.n, A.nnz, torch.as_tensor(A.row_ptr, device=dev),
                        torch.as_tensor(A.col, device=dev), torch.as_tensor(A.val, device=dev),
                        torch.as_tensor(x, device=dev),
                        torch.empty(A.m, dtype=torch.float64, device=dev))


class Timer:
    """Times library calls on one stream: L2 flushed (512 MB written, then read)
    before each run, CUDA events around the call only."""

    def __init__(self, dev):
        import torch
        self.torch = torch
        self.dev = dev
        self.flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        self.sink = torch.empty(1, dtype=torch.int64, device=dev)
        self.ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)

    def workspace(self, nbytes: int):
        if self.ws.numel() < nbytes:
            self.ws = self.torch.empty(nbytes + (nbytes >> 2), dtype=self.torch.uint8,
                                       device=self.dev)
        return self.ws

    def time_ms(self, fn, reps: int) -> float:
        torch = self.torch
        s = torch.cuda.current_stream(self.dev)
        out = []
        for _ in range(reps):
            self.flush.fill_(1)
            torch.sum(self.flush.view(torch.int64), 0, keepdim=True, out=self.sink)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.median(out))


def autotune(Ad: DeviceMatrix, timer: Timer, reps: int = 3) -> np.ndarray:
    """Median time (ms) of every class on this matrix."""
    times = np.empty(K)
    for k in range(K):
        o = class_opts(k)
        ws = timer.workspace(max(256, C.ssspmv_workspace_bytes(Ad.m, Ad.nnz, 8, o)))

        def call():
            C.check(C.ssspmv_csr_f64(Ad.m, Ad.n, Ad.nnz, Ad.rp, Ad.col, Ad.val, Ad.x, Ad.y, opts=o,
                                     workspace=ws), "class %d" % k)
        call()  # warm-up (first launch of a kernel, attributes)
        times[k] = timer.time_ms(call, reps)
    return times


def tune_batched(count: int, desc, total_nnz: int, dev, reps: int = 3):
    """The autotuner for a batch (ssspmv_csr_batched_f32): times every
    compiled tile shape with speculative and exact stores on this batch and
    returns (opts fields of the fastest, {name: ms})."""
    import torch
    timer = Timer(dev)
    cands = {}
    for W in C.ssspmv_supported_w():
        for variant in (C.VARIANT_SPECULATIVE, C.VARIANT_EXACT):
            cands["W%d %s" % (W, "exact" if variant == C.VARIANT_EXACT else "speculative")] = \
                dict(W=W, variant=variant)
    need = max(C.ssspmv_batched_workspace_bytes(count, total_nnz, 4, C.make_opts(**kw))
               for kw in cands.values())
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    times = {}
    for name, kw in cands.items():
        o = C.make_opts(**kw)

        def call():
            C.check(C.ssspmv_csr_batched_f32(count, desc, total_nnz, opts=o, workspace=ws),
                    "ssspmv_csr_batched_f32")
        call()
        times[name] = timer.time_ms(call, reps)
    best = min(times, key=times.get)
    return cands[best], times


# ---------------------------------------------------------------------------
# the seeded training set: six families, m log-uniform

FAMILIES = ("banded", "stencil", "rmat", "blockdiag", "uniform", "longrows", "rmatlong")


def dataset_specs(count: int, seed: int, m_lo: int = 10_000, m_hi: int = 8_000_000,
                  max_nnz: int = 120_000_000):
    """(family, m, parameter, seed) per matrix; m log-uniform in [m_lo, m_hi]
    and lowered where the family's nnz would pass max_nnz."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        fam = FAMILIES[int(rng.integers(0, len(FAMILIES)))]
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        if fam == "banded":
            par = int(rng.integers(1, 65))
            m = min(m, max_nnz // (2 * par + 1))
        elif fam == "stencil":
            par = 27
            m = min(m, max_nnz // 27)
        elif fam == "rmat":
            par = int(rng.integers(4, 17))            # edge factor
            m = min(m, max_nnz // par)
        elif fam == "blockdiag":
            par = int(rng.integers(32, 257))          # largest block
            m = min(m, max_nnz // par)
        elif fam == "uniform":
            par = int(rng.integers(2, 41))            # longest row
            m = min(m, max_nnz // par)
        elif fam == "longrows":
            par = int(rng.integers(1, 9))             # number of long rows
        else:
            # R-MAT over 2^ceil(log2 m) rows with one injected row of a quarter
            # of them (the power-law benchmark graph's shape)
            par = int(rng.integers(4, 17))            # edge factor
            m = min(m, max_nnz // (par + 1))
        out.append((fam, max(m, 64), par, seed * 1_000_003 + i))
    return out


def make_matrix(spec):
    import synth
    fam, m, par, s = spec
    if fam == "banded":
        A = synth.banded(m, par, s)
    elif fam == "stencil":
        k = max(2, int(round(m ** (1.0 / 3.0))))
        A = synth.stencil27(k, k, k, seed=s)
    elif fam == "rmat":
        A = synth.rmat_clipped(m, par, s)
    elif fam == "blockdiag":
        A = synth.blockdiag(m, 32, par, s)
    elif fam == "uniform":
        A = synth.range_rows(m, 0, par, s)
    elif fam == "longrows":
        A = synth.long_rows(m, par, min(m, 2_000_000), s)
    else:
        scale = max(6, int(math.ceil(math.log2(m))))
        A = synth.rmat(scale, par, seed=s, inject_len=min(1 << (scale - 2), 1_000_000))
    return A, synth.sym_vector(A.n, seed=s)


def collect(specs, dev, reps: int = 3, log=None):
    """Features (from the GPU kernel) and per-class times (ms) of every matrix."""
    timer = Timer(dev)
    X = np.empty((len(specs), F), np.float32)
    T = np.empty((len(specs), K))
    for i, sp in enumerate(specs):
        A, x = make_matrix(sp)
        Ad = to_device(A, x, dev)
        X[i] = device_features(Ad.rp, A.m, A.n, A.nnz).cpu().numpy()
        T[i] = autotune(Ad, timer, reps)
        if log and (i % 50 == 0 or i == len(specs) - 1):
            log("%d/%d %s m=%d nnz=%d best=%s" % (i + 1, len(specs), sp[0], A.m, A.nnz,
                                                  CLASSES[int(np.argmin(T[i]))][0]))
        del Ad
    return X, T


# ---------------------------------------------------------------------------
# training and selection with the library's kernels

def init_params(T_train: np.ndarray, seed: int = 0) -> np.ndarray:
    """He-normal hidden weights, zero biases, output bias = the mean target."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.normal(0, math.sqrt(2.0 / F), (H1, F))
    W2 = rng.normal(0, math.sqrt(2.0 / H1), (H2, H1))
    W3 = rng.normal(0, math.sqrt(1.0 / H2), (K, H2)) * 0.1
    b3 = np.nanmean(T_train, axis=0)
    return np.concatenate([W1.ravel(), np.zeros(H1), W2.ravel(), np.zeros(H2), W3.ravel(),
                           b3]).astype(np.float32)


def targets(times_ms: np.ndarray) -> np.ndarray:
    """What the network predicts: log2 of each class's time in microseconds."""
    return np.log2(np.maximum(times_ms, 1e-4) * 1e3).astype(np.float32)


def train(X: np.ndarray, T: np.ndarray, dev, steps: int = 4000, lr: float = 3e-3,
          weight_decay: float = 1e-4, seed: int = 0, log=None) -> np.ndarray:
    import torch
    B = X.shape[0]
    n = C.ssspmv_mlp_param_count(F, H1, H2, K)
    p = torch.as_tensor(init_params(T, seed), device=dev)
    assert p.numel() == n
    Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device=dev)
    Td = torch.as_tensor(np.ascontiguousarray(T, np.float32), device=dev)
    scratch = torch.empty(C.ssspmv_mlp_scratch_floats(B, F, H1, H2, K), dtype=torch.float32,
                          device=dev)
    g = torch.empty_like(p)
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    for t in range(1, steps + 1):
        C.check(C.ssspmv_mlp_backward(p, Xd, Td, B, F, H1, H2, K, scratch, g, loss),
                "ssspmv_mlp_backward")
        C.check(C.ssspmv_mlp_adam(p, g, m1, m2, n, lr, 0.9, 0.999, 1e-8, weight_decay, t),
                "ssspmv_mlp_adam")
        if log and (t % 1000 == 0 or t == 1):
            log("step %d loss %.5f" % (t, float(loss.item())))
    return p.cpu().numpy()


def select(params: np.ndarray, X: np.ndarray, dev) -> np.ndarray:
    """Class per row of X; class 0 (the default) where a feature is not finite."""
    import torch
    B = X.shape[0]
    p = torch.as_tensor(np.ascontiguousarray(params, np.float32), device=dev)
    Xd = torch.as_tensor(np.nan_to_num(np.ascontiguousarray(X, np.float32)), device=dev)
    scratch = torch.empty(C.ssspmv_mlp_scratch_floats(B, F, H1, H2, K), dtype=torch.float32,
                          device=dev)
    cls = torch.empty(B, dtype=torch.int32, device=dev)
    C.check(C.ssspmv_mlp_select(p, Xd, B, F, H1, H2, K, scratch, cls), "ssspmv_mlp_select")
    out = cls.cpu().numpy()
    out[~np.all(np.isfinite(X), axis=1)] = 0
    return out


def evaluate(choice: np.ndarray, times_ms: np.ndarray) -> dict:
    """Regret of the choices against the measured optimum, and speedup over
    the fixed default (class 0), both from the measured times."""
    idx = np.arange(times_ms.shape[0])
    t_sel = times_ms[idx, choice]
    t_best = times_ms.min(axis=1)
    t_def = times_ms[:, 0]
    regret = t_sel / t_best - 1.0
    return {"matrices": int(len(choice)),
            "mean_regret": float(regret.mean()),
            "median_regret": float(np.median(regret)),
            "optimum_hit_rate": float(np.mean(t_sel <= t_best * (1 + 1e-9))),
            "default_mean_regret": float((t_def / t_best - 1.0).mean()),
            "geomean_speedup_vs_default": float(np.exp(np.mean(np.log(t_def / t_sel)))),
            "geomean_speedup_oracle_choice_vs_default": float(np.exp(np.mean(np.log(t_def / t_best)))),
            "total_time_ratio_default_over_selected": float(t_def.sum() / t_sel.sum())}


def save(params: np.ndarray, path: str, meta: dict):
    with open(path, "w") as f:
        json.dump({"dims": [F, H1, H2, K], "classes": [c[0] for c in CLASSES],
                   "params": [float(v) for v in params], **meta}, f)


def load(path: str) -> np.ndarray:
    with open(path) as f:
        d = json.load(f)
    if d["dims"] != [F, H1, H2, K]:
        raise ValueError("selector weights for dims %s, expected %s" % (d["dims"], [F, H1, H2, K]))
    return np.asarray(d["params"], np.float32)


DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")


def load_default():
    """The weights trained by this module's command line on 2,000 generated
    matrices (shipped with the package), or None if absent."""
    try:
        return load(DEFAULT_WEIGHTS)
    except (OSError, ValueError, KeyError):
        return None


def choose_opts(rp, m: int, n: int, nnz: int, params=None, timer=None):
    """opts for ssspmv_csr_f64 on this matrix: the selector's class, or the
    defaults when there is no model."""
    if params is None:
        return class_opts(0, timer)
    f = device_features(rp, m, n, nnz).cpu().numpy()[None, :]
    k = int(select(params, f, rp.device)[0])
    return class_opts(k, timer)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--m-hi", type=int, default=8_000_000)
    ap.add_argument("--out", default=".")
    args = ap.parse_args(argv)
    import torch
    from . import _build
    _build.build()
    dev = torch.device("cuda:0")
    os.makedirs(args.out, exist_ok=True)
    t0 = time.time()
    log = lambda s: print("[%7.1fs] %s" % (time.time() - t0, s), flush=True)
    tr = dataset_specs(args.train, seed=1000, m_hi=args.m_hi)
    te = dataset_specs(args.test, seed=5000, m_hi=args.m_hi)
    Xtr, Ttr = collect(tr, dev, args.reps, log)
    Xte, Tte = collect(te, dev, args.reps, log)
    np.savez(os.path.join(args.out, "selector_data.npz"), Xtr=Xtr, Ttr=Ttr, Xte=Xte, Tte=Tte)
    params = train(Xtr, targets(Ttr), dev, steps=args.steps, log=log)
    rep = {"train": evaluate(select(params, Xtr, dev), Ttr),
           "held_out": evaluate(select(params, Xte, dev), Tte),
           "classes": [c[0] for c in CLASSES],
           "best_class_counts_held_out": np.bincount(Tte.argmin(axis=1), minlength=K).tolist(),
           "chosen_class_counts_held_out": np.bincount(select(params, Xte, dev), minlength=K).tolist(),
           "train_matrices": args.train, "held_out_matrices": args.test,
           "m_range": [10_000, args.m_hi], "reps": args.reps, "steps": args.steps,
           "seconds": round(time.time() - t0, 1)}
    save(params, os.path.join(args.out, "selector_weights.json"),
         {"trained_on": "%d seeded matrices, families %s" % (args.train, ", ".join(FAMILIES))})
    with open(os.path.join(args.out, "selector_report.json"), "w") as f:
        json.dump(rep, f, indent=1)
    log(json.dumps(rep["held_out"]))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
