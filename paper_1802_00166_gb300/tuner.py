"""Exhaustive autotuner and learned tile picker.

The paper characterises both schedules over a sweep of tile sizes and keeps
the mean of three runs per size (Sec. 5.1.5).  Here the same exploration is
the autotuner (every candidate timed on the GPU by the library's
``pcot_autotune``), its records train a small MLP cost model whose forward,
backward and Adam steps are the library's CUDA kernels, and ``pcot_pick``
runs the model to choose a candidate without timing all of them.

This module only orchestrates: it builds candidate lists and problem
lists, allocates device memory with PyTorch and calls the C ABI.

Command line (needs a GPU):
    python -m paper_1802_00166_gb300.tuner train --out DIR [--problems2d N --problems3d N]
        collects records, trains the picker, evaluates the regret on held-out
        problems and writes DIR/picker.npz, DIR/records.npz, DIR/report.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

import paper_1802_00166_gb300 as pcot

HEAT2D = [0.5, 0.125, 0.125, 0.125, 0.125]
JAC3D = [0.4] + [0.1] * 6
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


# ------------------------------------------------------------- candidates --

def candidates(dims, dtype, periodic):
    """(schedule, tile-parameter dict) pairs explored for a problem: the
    library's own candidate list (pcot_candidates), the one pcot_pick and
    PCOT_AUTO choose among."""
    coeffs = {1: [1 / 3] * 3, 2: HEAT2D, 3: JAC3D}[dims]
    h = pcot.pcot_create(dims, 1, coeffs, pcot.PCOT_PERIODIC if periodic else pcot.PCOT_DIRICHLET)
    try:
        return _trim(pcot.pcot_candidates(h, dtype), dims)
    finally:
        pcot.pcot_destroy(h)


def _trim(cands, dims):
    """Tile-parameter dicts in the short form the records use: only the
    fields a schedule sets."""
    out = []
    for sched, p in cands:
        if sched == pcot.PCOT_SWEEP:
            out.append((sched, dict()))
            continue
        d = dict(tile=tuple(p["tile"][:dims]), time_depth=p["time_depth"])
        if sched == pcot.PCOT_COT:
            d["cot_threshold"] = tuple(p["cot_threshold"][:dims + 1])
        out.append((sched, d))
    return out


def default_candidate(dims, dtype):
    """The method without the model: one fixed mid-range tile shape."""
    if dims == 2:
        return (pcot.PCOT_SLT, dict(tile=(0, 0), time_depth=4 if dtype == pcot.PCOT_F32 else 1))
    if dims == 3:
        return (pcot.PCOT_SLT, dict(tile=(64, 0, 0), time_depth=2))
    return (pcot.PCOT_SLT, dict(tile=(32,), time_depth=16))


# --------------------------------------------------------------- problems --

def problem_set(seed, n2d, n3d, n2d_f64=0):
    """Seeded Heat-2D (zero Dirichlet ring, sides log-uniform in [1024, 8192],
    T uniform in [64, 512]) and periodic Jacobi-3D (sides log-uniform in
    [128, 512], T uniform in [16, 128]) problems in FP32, and optionally
    Heat-2D problems in FP64 exact mode (sides log-uniform in [512, 2048],
    T uniform in [16, 128]; the FP64 pipe makes them slow to tune)."""
    import seeded_inputs as si
    u = si.uniform01(seed, 2 * (n2d + n3d + n2d_f64))
    probs = []
    for i in range(n2d):
        side = int(round(1024 * 8 ** u[2 * i]))
        T = 64 + min(int(u[2 * i + 1] * 449), 448)
        probs.append(dict(dims=2, sizes=(side, side), T=T, periodic=False))
    for j in range(n3d):
        i = n2d + j
        side = int(round(128 * 4 ** u[2 * i]))
        side -= side % 8
        T = 16 + min(int(u[2 * i + 1] * 113), 112)
        probs.append(dict(dims=3, sizes=(side, side, side), T=T, periodic=True))
    for j in range(n2d_f64):
        i = n2d + n3d + j
        side = int(round(512 * 4 ** u[2 * i]))
        T = 16 + min(int(u[2 * i + 1] * 113), 112)
        probs.append(dict(dims=2, sizes=(side, side), T=T, periodic=False, dtype=pcot.PCOT_F64_EXACT))
    return probs


def padded_layout(sizes, periodic, elem=4):
    shape = tuple(n if periodic else n + 2 for n in sizes)
    step = 32
    inner = ((shape[-1] + step - 1) // step) * step
    strides = [1] * len(shape)
    acc = inner
    for a in range(len(shape) - 2, -1, -1):
        strides[a] = acc
        acc *= shape[a]
    span = sum((shape[a] - 1) * strides[a] for a in range(len(shape))) + 1
    return shape, strides, span


def modelled_bytes(sizes, T, schedule, k, elem=4):
    """Algorithmic HBM traffic: one read and one write of the grid per pass;
    a pass is one step for the sweep and k steps for the tiled schedules."""
    passes = T if schedule == pcot.PCOT_SWEEP else math.ceil(T / max(1, k))
    return 2.0 * passes * float(np.prod(sizes)) * elem


# ------------------------------------------------------------- autotuner --

def tune_problem(prob, dtype=pcot.PCOT_F32, reps=2, cands=None, stream=None):
    """Time every candidate of one problem; returns (cands, ms list, features)."""
    import torch
    dims, sizes, T, periodic = prob["dims"], prob["sizes"], prob["T"], prob["periodic"]
    coeffs = {2: HEAT2D, 3: JAC3D, 1: [1 / 3] * 3}[dims]
    h = pcot.pcot_create(dims, 1, coeffs, pcot.PCOT_PERIODIC if periodic else pcot.PCOT_DIRICHLET)
    try:
        cands = cands if cands is not None else candidates(dims, dtype, periodic)
        shape, strides, span = padded_layout(sizes, periodic)
        tdt = torch.float32 if dtype == pcot.PCOT_F32 else torch.float64
        grid = torch.rand(span, dtype=tdt, device="cuda")
        need = 0
        for sched, p in cands:
            try:
                need = max(need, pcot.pcot_workspace_bytes(h, sizes, strides, T, dtype, sched,
                                                           pcot.tile_params(**p) if p else None))
            except pcot.PcotError:
                pass
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        params = [pcot.tile_params(**p) for _, p in cands]
        ms = pcot.pcot_autotune(h, grid, ws, need, sizes, strides, T, dtype, [s for s, _ in cands], params,
                                reps=reps, stream=stream)
        feats = []
        for (sched, p) in cands:
            try:
                feats.append(pcot.pcot_features(h, sizes, T, dtype, sched, pcot.tile_params(**p) if p else None))
            except pcot.PcotError:
                feats.append(np.zeros(12, dtype=np.float32))
        del grid, ws
        return cands, ms, np.stack(feats)
    finally:
        pcot.pcot_destroy(h)


def batch_candidates():
    """Tile shapes explored for a batched launch (one shape for every grid of
    the launch): the persistent-order depths and tile heights of the 2-D set."""
    return [dict(tile=(H, 112), time_depth=k, cot_threshold=(2, 256, 256)) for k in (4, 6, 8)
            for H in (64, 80, 96, 128)]


def tune_batched(h, grids, sizes, strides, Ts, dtype, stream, cands=None, reps=2):
    """The exhaustive autotuner applied to a batch: every candidate shape is
    timed on the batch itself (one warm-up launch, then `reps` launches between
    CUDA events).  Returns (best candidate, [(candidate, ms per launch)])."""
    import torch
    cands = cands or batch_candidates()
    results = []
    for c in cands:
        params = [pcot.tile_params(**c)] * len(Ts)
        try:
            nb = pcot.pcot_batch_workspace_bytes(h, sizes, strides, Ts, dtype, params)
        except pcot.PcotError:
            continue
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        done = torch.zeros(len(Ts) + 1, dtype=torch.int64, device="cuda")
        b = pcot.pcot_batch_create(h, grids, sizes, strides, Ts, dtype, params, ws, nb, done, stream)
        try:
            pcot.pcot_batch_launch(b, stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                pcot.pcot_batch_launch(b, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            st = pcot.pcot_check(h, stream)
        finally:
            pcot.pcot_batch_destroy(b)
        if st != pcot.PCOT_OK:
            raise pcot.PcotError(st, "tune_batched")
        results.append((c, e0.elapsed_time(e1) / reps))
    if not results:
        raise ValueError("tune_batched: no candidate fits this batch")
    return min(results, key=lambda r: r[1])[0], results


# Largest slowdown the second target distinguishes: candidates more than 3x
# slower than a problem's fastest are all "far off", and the loss spends its
# capacity on ranking the candidates that compete for the pick.
SLOWDOWN_CAP = math.log(3.0)


def records_for(prob, cands, ms, feats, dtype=pcot.PCOT_F32):
    """Training rows of one tuned problem: the candidate's features and two
    measured targets, log milliseconds and the log slowdown against the
    problem's fastest candidate (capped).  The picker chooses by the second:
    it carries no per-problem scale, so the network's error goes into the
    order of a problem's candidates, which is what a pick needs."""
    rows_x, rows_y = [], []
    valid = [t for t in ms if t > 0]
    if not valid:
        return rows_x, rows_y
    best = min(valid)
    for (sched, p), t, f in zip(cands, ms, feats):
        if t <= 0:
            continue
        rows_x.append(f)
        rows_y.append([math.log(t), min(math.log(t / best), SLOWDOWN_CAP)])
    return rows_x, rows_y


# ------------------------------------------------------------ the picker --

class Picker:
    """Trained MLP weights plus the feature and target normalisation."""

    def __init__(self, params, feat_mean, feat_std, targ_mean, targ_std):
        self.params = np.asarray(params, dtype=np.float32)
        self.feat_mean = np.asarray(feat_mean, dtype=np.float32)
        self.feat_std = np.asarray(feat_std, dtype=np.float32)
        self.targ_mean = np.asarray(targ_mean, dtype=np.float32)
        self.targ_std = np.asarray(targ_std, dtype=np.float32)
        self._dev = None

    def save(self, path):
        np.savez(path, params=self.params, feat_mean=self.feat_mean, feat_std=self.feat_std,
                 targ_mean=self.targ_mean, targ_std=self.targ_std)

    @classmethod
    def load(cls, path=None):
        path = path or os.path.join(DATA_DIR, "picker.npz")
        z = np.load(path)
        return cls(z["params"], z["feat_mean"], z["feat_std"], z["targ_mean"], z["targ_std"])

    def device_params(self):
        import torch
        if self._dev is None:
            self._dev = torch.from_numpy(self.params.copy()).cuda()
        return self._dev

    def pick(self, h, sizes, T, dtype, cands, stream=None):
        import torch
        n = len(cands)
        scratch = torch.empty(n * 14 * 4 + 512, dtype=torch.uint8, device="cuda")
        params = [pcot.tile_params(**p) for _, p in cands]
        return pcot.pcot_pick_among(h, sizes, T, dtype, self.device_params(), self.feat_mean, self.feat_std,
                              [s for s, _ in cands], params, scratch, stream)

    def predict(self, x_norm):
        """Normalised targets for normalised features (forward kernel)."""
        import torch
        x = torch.from_numpy(np.ascontiguousarray(x_norm, dtype=np.float32)).cuda()
        y = torch.empty((x.shape[0], 2), dtype=torch.float32, device="cuda")
        pcot.pcot_mlp_forward(self.device_params(), x, x.shape[0], y)
        return y.cpu().numpy()


def init_params(seed=11):
    """He-uniform weights, zero biases (float32), seeded."""
    import seeded_inputs as si
    layers = (12, 64, 64, 64, 2)
    u = si.uniform01(seed, sum(layers[i] * layers[i + 1] for i in range(4)))
    out, o = [], 0
    for i in range(4):
        fi, fo = layers[i], layers[i + 1]
        lim = math.sqrt(6.0 / fi)
        out.append(((2 * u[o:o + fi * fo] - 1) * lim).astype(np.float32))
        o += fi * fo
        out.append(np.zeros(fo, dtype=np.float32))
    return np.concatenate(out)


def train(x, y, steps=4000, batch=256, lr=2e-3, seed=11, log_every=500):
    """Train on (features, targets) with the library's grad and Adam kernels."""
    import torch
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    fm, fs = x.mean(0), x.std(0)
    fs[fs < 1e-6] = 1.0
    tm, ts = y.mean(0), y.std(0)
    ts[ts < 1e-6] = 1.0
    xd = torch.from_numpy((x - fm) / fs).cuda()
    yd = torch.from_numpy((y - tm) / ts).cuda()
    n = pcot.pcot_mlp_param_count()
    P = torch.from_numpy(init_params(seed)).cuda()
    G = torch.zeros(n, dtype=torch.float32, device="cuda")
    M = torch.zeros_like(G)
    V = torch.zeros_like(G)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    sb = pcot.pcot_mlp_scratch_bytes(batch)
    scratch = torch.empty(sb, dtype=torch.uint8, device="cuda")
    gen = np.random.default_rng(seed)
    N = xd.shape[0]
    hist = []
    for step in range(1, steps + 1):
        idx = torch.from_numpy(gen.integers(0, N, size=batch)).cuda()
        xb = xd.index_select(0, idx).contiguous()
        yb = yd.index_select(0, idx).contiguous()
        pcot.pcot_mlp_grad(P, xb, yb, batch, G, loss, scratch, sb)
        lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / steps))
        pcot.pcot_mlp_adam(P, G, M, V, n, step, lr_t)
        if step % log_every == 0 or step == 1:
            hist.append((step, float(loss.item())))
    return Picker(P.cpu().numpy(), fm, fs, tm, ts), hist


def evaluate(picker, probs, dtype=pcot.PCOT_F32, reps=2):
    """Regret of the picker, of the fixed default and of a random pick."""
    rows = []
    rng = np.random.default_rng(5)
    for prob in probs:
        dt = prob.get("dtype", dtype)
        cands, ms, feats = tune_problem(prob, dt, reps)
        valid = [i for i, t in enumerate(ms) if t > 0]
        best = min(ms[i] for i in valid)
        coeffs = {2: HEAT2D, 3: JAC3D}[prob["dims"]]
        h = pcot.pcot_create(prob["dims"], 1, coeffs,
                             pcot.PCOT_PERIODIC if prob["periodic"] else pcot.PCOT_DIRICHLET)
        try:
            i_pick = picker.pick(h, prob["sizes"], prob["T"], dt, cands)
        finally:
            pcot.pcot_destroy(h)
        dflt = default_candidate(prob["dims"], dt)
        i_def = next((i for i, c in enumerate(cands) if c[0] == dflt[0] and c[1] == dflt[1]), valid[0])
        i_rand = int(rng.choice(valid))
        rows.append(dict(prob=prob, best_ms=best, pick_ms=ms[i_pick], default_ms=ms[i_def], random_ms=ms[i_rand],
                         pick=cands[i_pick], best=cands[int(np.argmin([t if t > 0 else 1e30 for t in ms]))]))
    pick = np.array([r["pick_ms"] / r["best_ms"] - 1 for r in rows])
    dflt = np.array([r["default_ms"] / r["best_ms"] - 1 for r in rows])
    rand = np.array([r["random_ms"] / r["best_ms"] - 1 for r in rows])
    tot = sum(r["pick_ms"] for r in rows) / sum(r["best_ms"] for r in rows) - 1
    summary = dict(n=len(rows), regret_mean=float(pick.mean()), regret_median=float(np.median(pick)),
                   regret_max=float(pick.max()), regret_time_weighted=float(tot),
                   frac_within_10pct=float((pick <= 0.10).mean()),
                   default_regret_mean=float(dflt.mean()), random_regret_mean=float(rand.mean()))
    return summary, rows


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", default=DATA_DIR)
    t.add_argument("--problems2d", type=int, default=250)
    t.add_argument("--problems3d", type=int, default=120)
    t.add_argument("--heldout2d", type=int, default=32)
    t.add_argument("--heldout3d", type=int, default=32)
    t.add_argument("--problems2d-f64", type=int, default=40)
    t.add_argument("--steps", type=int, default=10000)
    args = ap.parse_args()
    from paper_1802_00166_gb300 import build
    build.build()
    os.makedirs(args.out, exist_ok=True)
    t0 = time.time()
    X, Y, meta = [], [], []
    for pi, prob in enumerate(problem_set(4, args.problems2d, args.problems3d, args.problems2d_f64)):
        dt = prob.get("dtype", pcot.PCOT_F32)
        cands, ms, feats = tune_problem(prob, dt)
        rx, ry = records_for(prob, cands, ms, feats, dt)
        X += rx
        Y += ry
        meta.append(dict(prob=prob, best_ms=min(v for v in ms if v > 0)))
    t_collect = time.time() - t0
    X = np.array(X, dtype=np.float32)
    Y = np.array(Y, dtype=np.float32)
    np.savez_compressed(os.path.join(args.out, "records.npz"), x=X, y=Y)
    picker, hist = train(X, Y, steps=args.steps)
    picker.save(os.path.join(args.out, "picker.npz"))
    held = problem_set(5, args.heldout2d, args.heldout3d)
    summary, rows = evaluate(picker, held, reps=3)
    report = dict(records=int(X.shape[0]), problems=len(meta), collect_seconds=t_collect, loss_history=hist,
                  heldout=summary, rows=[dict(sizes=r["prob"]["sizes"], T=r["prob"]["T"], best_ms=r["best_ms"],
                                              pick_ms=r["pick_ms"], default_ms=r["default_ms"],
                                              random_ms=r["random_ms"]) for r in rows])
    with open(os.path.join(args.out, "report.json"), "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(dict(records=report["records"], heldout=summary)))


if __name__ == "__main__":
    main()
