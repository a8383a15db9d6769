"""The learned surrogate: a BF16 MLP trained on the batch simulator's outputs.

Inputs (10, padded to 16): mesh side, injection period, private / shared /
remote address fractions, write fraction, private working set (KB), L2 policy
one-hot (interleaved, LSPD-local, LSPD-migrate).  Outputs (3, padded to 16):
log mean L2 access latency, deflections per flit, accepted flits per node per
cycle -- each computed from a simulation's counters (mean L2 access latency =
l2lat_sum / l2lat_cnt, deflections / ejected flits, ejected / (tiles x cycles)).
Network: 16 -> 256 -> 256 -> 256 -> 256 -> 16, GELU,
trained with AdamW on the standardised outputs by the library's own tensor-core
forward / backward kernels (include/mlp.h); torch only holds the buffers.

The exact simulator is both the training-data source and the reference the
surrogate is scored against: the relative error of each output against fresh
simulations is reported with epsilon floors in the denominators (0.01
deflections/flit, 1e-3 flits/node/cycle; latency on its natural scale).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import inputs as I
from . import noc

DIMS = (16, 256, 256, 256, 256, 16)
N_IN, N_OUT = 10, 3
OUT_NAMES = ("log_l2_latency", "deflections_per_flit", "accepted_per_node_cycle")
EPS_FLOOR = (None, 0.01, 1e-3)


class Shape(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("dims", C.c_int32 * 9)]


def _mlp_lib():
    L = noc.lib()
    if not getattr(L, "_mlp_sigs", False):
        vp, i32, sz = C.c_void_p, C.c_int, C.c_size_t
        f = C.c_float
        for name, res, args in (
            ("mlp_param_count", sz, [C.POINTER(Shape)]),
            ("mlp_workspace_bytes", sz, [C.POINTER(Shape), i32]),
            ("mlp_forward", i32, [C.POINTER(Shape), vp, vp, i32, vp, vp, vp]),
            ("mlp_backward", i32, [C.POINTER(Shape), vp, vp, i32, vp, vp, vp, vp]),
            ("mlp_mse", i32, [vp, vp, i32, i32, i32, vp, vp, vp]),
            ("mlp_adamw", i32, [sz, vp, vp, vp, vp, vp, f, f, f, f, f, i32, vp]),
            ("mlp_to_bf16", i32, [vp, vp, sz, vp]),
            ("mlp_set_gemm_path", i32, [i32]),
            ("mlp_gemm_status", i32, []),
            ("mlp_packed_bytes", sz, [C.POINTER(Shape)]),
            ("mlp_pack", i32, [C.POINTER(Shape), vp, vp, vp]),
            ("mlp_infer", i32, [C.POINTER(Shape), vp, vp, i32, vp, vp]),
        ):
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        L._mlp_sigs = True
    return L


def set_gemm_path(path: int) -> int:
    """0: tcgen05 tensor cores where they apply (default), 1: mma.sync for
    every GEMM; returns the previous setting."""
    return _mlp_lib().mlp_set_gemm_path(path)


def gemm_status() -> int:
    """0, or MLP_ERR_TIMEOUT if a tcgen05 GEMM gave up waiting for its MMAs."""
    return _mlp_lib().mlp_gemm_status()


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


def _p(t):
    return C.c_void_p(t.data_ptr())


class MLP:
    """Parameters, AdamW state and workspaces on the current CUDA device."""

    def __init__(self, dims=DIMS, seed=0, max_batch=4096):
        import torch
        self.torch = torch
        self.dims = tuple(dims)
        self.shape = Shape()
        self.shape.n_layers = len(dims) - 1
        for i, d in enumerate(dims):
            self.shape.dims[i] = d
        L = _mlp_lib()
        self.n = L.mlp_param_count(C.byref(self.shape))
        g = torch.Generator().manual_seed(seed)
        parts = []
        for l in range(len(dims) - 1):
            k, n = dims[l], dims[l + 1]
            bound = math.sqrt(6.0 / k) if l < len(dims) - 2 else math.sqrt(1.0 / k)
            parts.append((torch.rand(n * k, generator=g, dtype=torch.float64) * 2 - 1) * bound)
            parts.append(torch.zeros(n, dtype=torch.float64))
        self.params = torch.cat(parts).float().cuda()
        assert self.params.numel() == self.n
        self.params_bf16 = torch.empty(self.n, dtype=torch.bfloat16, device="cuda")
        self.grads = torch.zeros(self.n, dtype=torch.float32, device="cuda")
        self.m = torch.zeros_like(self.grads)
        self.v = torch.zeros_like(self.grads)
        self.step = 0
        self.max_batch = max_batch
        self.ws = torch.empty(L.mlp_workspace_bytes(C.byref(self.shape), max_batch) + 256,
                              dtype=torch.uint8, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        nb = L.mlp_packed_bytes(C.byref(self.shape))
        self.packed = torch.empty(nb + 16, dtype=torch.uint8, device="cuda") if nb else None
        self._packed_step = None               # parameter version the image holds
        self.sync_bf16()

    def _stream(self):
        return C.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _ws(self):
        p = self.ws.data_ptr()
        return C.c_void_p(p + (-p) % 256)

    def sync_bf16(self):
        _ok(_mlp_lib().mlp_to_bf16(_p(self.params), _p(self.params_bf16), self.n, self._stream()),
            "mlp_to_bf16")
        self._packed_step = None

    def _packed(self):
        p = self.packed.data_ptr()
        return C.c_void_p(p + (-p) % 16)

    def infer(self, xb, out=None):
        """The whole network in one fused tcgen05 kernel (mlp_infer): xb BF16
        [B, dims[0]] with B a multiple of 128 -> FP32 [B, dims[-1]] (into `out`
        if given), equal to forward() on the tensor-core path."""
        B = xb.shape[0]
        if self.packed is None or B < 128 or B % 128 or xb.dtype != self.torch.bfloat16:
            raise ValueError("mlp_infer takes BF16 batches of a multiple of 128 rows of a packable shape")
        if self._packed_step != self.step:
            _ok(_mlp_lib().mlp_pack(C.byref(self.shape), _p(self.params_bf16), self._packed(),
                                    self._stream()), "mlp_pack")
            self._packed_step = self.step
        y = out if out is not None else self.torch.empty(B, self.dims[-1], dtype=self.torch.float32,
                                                         device="cuda")
        _ok(_mlp_lib().mlp_infer(C.byref(self.shape), self._packed(), _p(xb), B, _p(y),
                                 self._stream()), "mlp_infer")
        return y

    def load_params(self, flat):
        self.params.copy_(self.torch.as_tensor(flat, dtype=self.torch.float32))
        self.sync_bf16()

    def forward(self, xb):
        """xb: BF16 [B, dims[0]] CUDA tensor -> FP32 [B, dims[-1]]."""
        B = xb.shape[0]
        assert B <= self.max_batch and xb.dtype == self.torch.bfloat16
        y = self.torch.empty(B, self.dims[-1], dtype=self.torch.float32, device="cuda")
        _ok(_mlp_lib().mlp_forward(C.byref(self.shape), _p(self.params_bf16), _p(xb), B, _p(y),
                                   self._ws(), self._stream()), "mlp_forward")
        return y

    def backward(self, xb, dy):
        _ok(_mlp_lib().mlp_backward(C.byref(self.shape), _p(self.params_bf16), _p(xb),
                                    xb.shape[0], _p(dy), _p(self.grads), self._ws(),
                                    self._stream()), "mlp_backward")
        return self.grads

    def mse(self, y, t, used):
        dy = self.torch.empty_like(y)
        _ok(_mlp_lib().mlp_mse(_p(y), _p(t), y.shape[0], y.shape[1], used, _p(self.loss), _p(dy),
                               self._stream()), "mlp_mse")
        return self.loss, dy

    def adamw(self, lr, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
        self.step += 1
        _ok(_mlp_lib().mlp_adamw(self.n, _p(self.params), _p(self.params_bf16), _p(self.grads),
                                 _p(self.m), _p(self.v), lr, b1, b2, eps, wd, self.step,
                                 self._stream()), "mlp_adamw")

    def train_step(self, xb, tb, lr):
        y = self.forward(xb)
        loss, dy = self.mse(y, tb, N_OUT)
        self.backward(xb, dy)
        self.adamw(lr)
        return loss


# ----------------------------------------------------------------- data
def features(design: dict) -> np.ndarray:
    d = design
    f = np.zeros(DIMS[0], dtype=np.float32)
    f[0] = d["side"] / 128.0
    f[1] = d["period"] / 40.0
    f[2], f[3], f[4] = d["priv"], d["shared"], d["remote"]
    f[5] = d["write"]
    f[6] = d["ws_kb"] / 64.0
    f[7 + d["policy"]] = 1.0
    return f


def targets(stats: dict, tiles: int) -> np.ndarray:
    """(log mean L2 access latency, deflections per flit, accepted throughput)."""
    lat = stats["l2lat_sum"] / max(stats["l2lat_cnt"], 1)
    defl = stats["deflections"] / max(stats["ejected"], 1)
    acc = stats["ejected"] / (tiles * max(stats["cycle"], 1))
    return np.array([math.log(max(lat, 1e-9)), defl, acc], dtype=np.float64)


def simulate(designs_params, cycles):
    """Exact outputs of design points through the batch engine, in the
    autotuner's layout for each kernel-variant group."""
    b = noc.Batch([{k: v for k, v in p.items() if k != "design"} for p in designs_params], cycles,
                  collect_hash=False)
    b.run()
    ys = np.stack([targets(b.stats(i), p["mesh_w"] * p["mesh_h"])
                   for i, p in enumerate(designs_params)])
    b.close()
    return ys


def make_dataset(n, cycles, seed=0, **kw):
    pts = I.batch_design_points(n, seed=seed, **kw)
    X = np.stack([features(p["design"]) for p in pts])
    Y = simulate(pts, cycles)
    return X, Y, pts


def relative_errors(pred, true):
    """Per-output relative error, |pred - true| / max(|true|, floor) with floors
    0.01 deflections/flit and 1e-3 flits/node/cycle; latency is compared on its
    natural (not log) scale."""
    err = np.empty_like(true)
    lp, lt = np.exp(pred[:, 0]), np.exp(true[:, 0])
    err[:, 0] = np.abs(lp - lt) / np.abs(lt)
    for j in (1, 2):
        err[:, j] = np.abs(pred[:, j] - true[:, j]) / np.maximum(np.abs(true[:, j]), EPS_FLOOR[j])
    return err


class Surrogate:
    """Standardisation + MLP + training loop."""

    def __init__(self, seed=0, max_batch=4096):
        self.net = MLP(seed=seed, max_batch=max_batch)
        self.torch = self.net.torch
        self.mu = np.zeros(N_OUT)
        self.sd = np.ones(N_OUT)

    def _x(self, X):
        return self.torch.as_tensor(X, dtype=self.torch.float32).cuda().to(self.torch.bfloat16)

    def fit(self, X, Y, epochs=200, batch=1024, lr=2e-3, seed=0, verbose=False):
        torch = self.torch
        self.mu = Y.mean(axis=0)
        self.sd = Y.std(axis=0) + 1e-12
        T = np.zeros((len(Y), DIMS[-1]), dtype=np.float32)
        T[:, :N_OUT] = (Y - self.mu) / self.sd
        xs = self._x(X)
        ts = torch.as_tensor(T).cuda()
        g = torch.Generator(device="cuda").manual_seed(seed)
        n = len(X)
        steps = 0
        total = epochs * max(1, n // batch)
        for ep in range(epochs):
            perm = torch.randperm(n, device="cuda", generator=g)
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                frac = steps / max(total, 1)
                cur = lr * 0.5 * (1 + math.cos(math.pi * frac))     # cosine decay
                loss = self.net.train_step(xs[idx].contiguous(), ts[idx].contiguous(), cur)
                steps += 1
            if verbose and (ep % max(1, epochs // 10) == 0 or ep == epochs - 1):
                print(f"  epoch {ep}: loss {float(loss.item()):.5f}", flush=True)
        return float(loss.item())

    def predict(self, X):
        """Network outputs for design-point features X, through the fused
        inference kernel (each chunk padded to a multiple of 128 rows)."""
        out = []
        for s in range(0, len(X), self.net.max_batch):
            chunk = X[s:s + self.net.max_batch]
            n = len(chunk)
            if self.net.packed is not None:
                pad = (-n) % 128
                xb = self._x(np.concatenate([chunk, np.repeat(chunk[-1:], pad, axis=0)]) if pad else chunk)
                y = self.net.infer(xb)[:n]
            else:
                y = self.net.forward(self._x(chunk))
            out.append(y[:, :N_OUT].double().cpu().numpy())
        Z = np.concatenate(out)
        return Z * self.sd + self.mu


# ----------------------------------------------------------------- screening
def screen(pred, true, k, top_frac=0.01, objective=0, minimise=True, random_draws=200, seed=0):
    """Design-space screening with the network: of a candidate pool whose
    exact outputs `true` are known, pick the k candidates the network ranks
    best on output `objective` (the ones the exact simulator would then run)
    and report the recall of the pool's true best top_frac, against k picks
    at random (the same simulator budget), averaged over random_draws draws.
    Returns (network recall, mean random recall, the true top indices)."""
    n = len(true)
    m = max(1, int(round(top_frac * n)))
    sign = 1.0 if minimise else -1.0
    best = set(np.argsort(sign * true[:, objective], kind="stable")[:m].tolist())
    picks = np.argsort(sign * pred[:, objective], kind="stable")[:k]
    recall = len(best & set(picks.tolist())) / m
    rng = np.random.default_rng(seed)
    rnd = np.mean([len(best & set(rng.choice(n, size=k, replace=False).tolist())) / m
                   for _ in range(random_draws)])
    return recall, float(rnd), sorted(best)


def evaluate(train=2_000, holdout=500, cycles=20_000, seeds=(0,), epochs=400, batch=256, lr=2e-3,
             data_seed=11, screen_k=None, log=None):
    """Simulate train + holdout design points of the batch workload with the
    batch engine, train one network per seed on the first `train`, and score
    each on the held-out points: per-output mean relative error (S-3
    definitions, relative_errors) and, with the held-out points as a
    candidate pool, the screening recall of the best 1% by mean L2 access
    latency when the network picks screen_k of them (default 5%).  Returns a
    dict of the per-seed results and the simulation / training times."""
    import time
    pts = I.batch_design_points(train + holdout, seed=data_seed)
    X = np.stack([features(p["design"]) for p in pts])
    a = time.perf_counter()
    Y = simulate(pts, cycles)
    sim_s = time.perf_counter() - a
    k = screen_k or max(1, holdout // 20)
    runs = []
    for sd in seeds:
        model = Surrogate(seed=sd, max_batch=4096)
        a = time.perf_counter()
        model.fit(X[:train], Y[:train], epochs=epochs, batch=batch, lr=lr, seed=sd)
        train_s = time.perf_counter() - a
        pred = model.predict(X[train:])
        mre = relative_errors(pred, Y[train:]).mean(axis=0)
        rec, rnd, _ = screen(pred, Y[train:], k, objective=0, seed=sd)
        runs.append({"seed": sd, "mre": dict(zip(OUT_NAMES, map(float, mre))),
                     "screen_recall": rec, "random_recall": rnd, "train_s": train_s})
        if log:
            log(f"seed {sd}: MRE {mre}, screening recall {rec:.2f} (random {rnd:.3f})")
    return {"train": train, "holdout": holdout, "cycles": cycles, "screen_k": k,
            "simulate_s": sim_s, "runs": runs}


# ----------------------------------------------------------------- full run
def run(points=50_000, holdout=5_000, cycles=20_000, chunk=2_000, epochs=300, batch=1024,
        lr=2e-3, data_path=None, seed=0, log=print, from_data=None, time_points=2_000):
    """Simulate `points` design points with the batch engine, train on all but
    `holdout`, score the held-out ones against their exact simulations, and time
    batch-4096 inference against the batched simulator.  With `from_data`, the
    design points' exact outputs come from a dataset this function saved
    before (same points, seed and cycles), and the simulator's rate is timed on
    the first `time_points` of them."""
    import json
    import time

    import torch

    t0 = time.perf_counter()
    Xs, Ys = [], []
    pts_all = I.batch_design_points(points, seed=seed)
    sim_s = 0.0
    if from_data:
        z = np.load(from_data)
        if int(z["cycles"]) != cycles or int(z["seed"]) != seed or len(z["X"]) != points:
            raise ValueError(f"{from_data} holds other design points")
        X, Y = z["X"], z["Y"]
        n = min(time_points, points)
        a = time.perf_counter()
        Yt = simulate(pts_all[:n], cycles)
        sim_s = (time.perf_counter() - a) * points / n     # the rate, scaled to all points
        if not np.array_equal(Yt, Y[:n]):
            raise ValueError("the simulator no longer reproduces the saved outputs")
        log(f"loaded {points} design points; simulator timed on {n} ({sim_s * n / points:.0f} s)")
    else:
        for s in range(0, points, chunk):
            pts = pts_all[s:s + chunk]
            a = time.perf_counter()
            Ys.append(simulate(pts, cycles))
            sim_s += time.perf_counter() - a
            Xs.append(np.stack([features(p["design"]) for p in pts]))
            log(f"simulated {min(s + chunk, points)}/{points} design points ({sim_s:.0f} s)")
        X, Y = np.concatenate(Xs), np.concatenate(Ys)
    if data_path:
        np.savez_compressed(data_path, X=X, Y=Y, cycles=cycles, seed=seed)
    ntr = points - holdout
    model = Surrogate(seed=seed, max_batch=4096)
    a = time.perf_counter()
    loss = model.fit(X[:ntr], Y[:ntr], epochs=epochs, batch=batch, lr=lr)
    train_s = time.perf_counter() - a
    err = relative_errors(model.predict(X[ntr:]), Y[ntr:])
    mre = err.mean(axis=0)
    # inference throughput at batch 4096 (device time, CUDA events)
    xb = model._x(np.tile(X[:4096], (max(1, 4096 // min(4096, len(X))), 1))[:4096])
    for _ in range(5):
        model.net.forward(xb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    e0.record()
    for _ in range(reps):
        model.net.forward(xb)
    e1.record()
    torch.cuda.synchronize()
    inf_pts_s = reps * 4096 / (e0.elapsed_time(e1) / 1e3)
    sim_pts_s = points / sim_s
    res = {"points": points, "holdout": holdout, "cycles": cycles, "train_loss": loss,
           "train_s": train_s, "simulate_s": sim_s, "mre": dict(zip(OUT_NAMES, map(float, mre))),
           "mre_max": float(mre.max()), "p90_rel_err": dict(zip(OUT_NAMES, map(float, np.quantile(err, 0.9, axis=0)))),
           "inference_points_per_s": inf_pts_s, "simulator_points_per_s": sim_pts_s,
           "speedup": inf_pts_s / sim_pts_s, "epochs": epochs, "batch": batch, "lr": lr,
           "wall_s": time.perf_counter() - t0}
    log(json.dumps(res))
    return res, model


if __name__ == "__main__":
    import argparse
    import json
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ap = argparse.ArgumentParser(description="simulate, train and score the surrogate")
    ap.add_argument("--points", type=int, default=50_000)
    ap.add_argument("--holdout", type=int, default=5_000)
    ap.add_argument("--cycles", type=int, default=20_000)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--data", default=None, help="save the simulated dataset (.npz)")
    ap.add_argument("--from-data", default=None,
                    help="reuse a saved dataset; time the simulator on --time-points of it")
    ap.add_argument("--time-points", type=int, default=2_000)
    ap.add_argument("--out", default=None, help="write the result JSON here")
    ap.add_argument("--gemm-path", type=int, default=0,
                    help="0: tcgen05 where it applies (default), 1: mma.sync for every GEMM")
    a = ap.parse_args()
    from paper_1508_03235_b300 import surrogate as S
    S.set_gemm_path(a.gemm_path)
    res, _ = S.run(points=a.points, holdout=a.holdout, cycles=a.cycles, epochs=a.epochs,
                   data_path=a.data, log=lambda m: print(m, flush=True), from_data=a.from_data,
                   time_points=a.time_points)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
