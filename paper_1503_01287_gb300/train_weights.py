"""Trains the learned-weights network on convergence factors measured by the
AMG solver itself, on the GPU, with the library's own network kernels.

    python -m paper_1503_01287_gb300.train_weights --problems 2000 \
        --out paper_1503_01287_gb300/weights/mlp_theta.npy

Data.  Seeded problems with n^3 cubes, n uniform in 8..16: even indices are
mixed displacement-pressure elasticity (nu = 0.5 - 10^U[-4, -1.3], vertices
jittered by U[0, 0.2] h), odd indices pure-displacement elasticity (nu in
U[0.2, 0.45], side lengths U[1, 4] per axis, N(0, 1) traction).  Each problem
is set up once (FP32 cycle; flexible CG or FGMRES(300)) and solved to 1e-8
with the plain weights and with `--candidates` random changes of one level:
a level l drawn among the non-coarsest levels and a random (ws, wc, wp) from
the box of the selection grid for that level, the other levels plain.  A
solve's convergence factor is rho = (||r_k|| / ||r_0||)^(1/k).  One training
sample is
  input  = the 13 statistics of level l and the level below (amg_level_features),
           ws, wc, log2 wp
  target = log10(rho_candidate / rho_plain), clipped to [-1, 1]
(wp and its input are 1 and 0 for the SPD problems).  Each problem also gives
one plain sample (level 0, candidate (1, 1, 0), target 0), so the plain method
is the yardstick of every problem's samples.

Training.  Adam with the amg_mlp_* kernels (BF16 products, FP32 accumulation)
on the mean squared error of the targets (--loss mse) or on a listwise ranking
loss of each problem's candidates (--loss rank: the loss gradient per sample is
formed on the host and back-propagated by amg_mlp_backward), full batch, problems split 90 / 10 into
training and validation sets, learning rate divided by 10 over the last third;
the parameters with the lowest validation selection regret are kept (per
validation problem: how much worse the measured candidate the network ranks
first is than the best measured one), since the selection uses the network's
argmin, not its values.  They (float32,
AMG_MLP_NPARAM) are written to --out, the measured dataset next to it as
.data.npz (retrain with --data) and a summary (data, losses, timings) as .json.

Problems are generated by a process pool started with `spawn` before the
first CUDA call, a chunk ahead of the GPU measurements.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

SEED0 = 20_000
RESTART = 300
MAXIT = 400


def problem_spec(i: int, seed0: int = SEED0) -> dict:
    rng = np.random.default_rng(seed0 + i)
    n = int(rng.integers(8, 17))
    if i % 2 == 0:
        return {"kind": "mixed", "n": n, "nu": float(0.5 - 10.0 ** rng.uniform(-4.0, -1.3)),
                "jitter": float(rng.uniform(0.0, 0.2)), "seed": seed0 + i}
    return {"kind": "elasticity", "n": n, "nu": float(rng.uniform(0.2, 0.45)),
            "lengths": tuple(float(v) for v in rng.uniform(1.0, 4.0, 3)), "seed": seed0 + i}


def make_problem(spec: dict):
    from fem_inputs import problems as fp
    if spec["kind"] == "mixed":
        return fp.mixed_elasticity_family(spec["n"], [spec["nu"]], seed=spec["seed"],
                                          jitter=spec["jitter"])[0]
    return fp.elasticity_problem(spec["n"], seed=spec["seed"], nu=spec["nu"],
                                 lengths=spec["lengths"], traction="gaussian")


def candidate_box(rng: np.random.Generator, saddle: bool):
    from . import binding as B
    ws = rng.uniform(*B.WS_RANGE)
    wc = rng.uniform(*B.WC_RANGE)
    lp = rng.uniform(*B.WP_LOG2_RANGE) if saddle else 0.0
    return ws, wc, lp


def _rho(st) -> float:
    if st.iterations <= 0:
        return 0.0
    r = st.rel_residual
    if not np.isfinite(r) or r <= 0.0:
        return 10.0
    return float(r ** (1.0 / st.iterations))


# setup options of the measurements: the per-operation cycle (the one-launch
# sweep variants only change the speed, not the iteration)
MEASURE_OPTS = dict(cluster_from=0, cycle_kernel=1, gs_cluster=0, gs_flow=0, gs_stream=0)


def measure(prob, n_cand: int, rng: np.random.Generator, torch):
    """([features per sample], [(level, ws, wc, lp, target, iterations, ms)],
    plain (rho, iterations, ms)): one plain sample, then n_cand one-level changes."""
    from . import binding as B
    saddle = prob.kind in ("mixed", "stokes")
    h = B.setup_problem(prob, B.default_options(precision=1, gmres_restart=RESTART,
                                                max_iterations=MAXIT, **MEASURE_OPTS))
    nl = h.n_levels
    lf = [h.level_features(l) for l in range(nl - 1)]
    b = torch.from_numpy(prob.rhs()).cuda()
    x = torch.zeros_like(b)

    def run(w):
        h.set_level_weights(w)
        x.zero_()
        try:
            st = h.solve(b, x, 1e-8, device_ptrs=True)
        except B.AmgError:
            return 10.0, MAXIT, float("nan")
        return _rho(st), st.iterations, st.solve_ms

    plain_w = np.ones((nl, 3))
    rho_p, it_p, ms_p = run(plain_w)
    feats = [lf[0]]
    rows = [(0, 1.0, 1.0, 0.0, 0.0, it_p, ms_p)]
    for _ in range(n_cand):
        l = int(rng.integers(0, nl - 1))
        ws, wc, lp = candidate_box(rng, saddle)
        w = plain_w.copy()
        w[l] = (ws, wc, 2.0 ** lp)
        rho, it, ms = run(w)
        t = float(np.clip(np.log10(max(rho, 1e-12) / rho_p), -1.0, 1.0))
        feats.append(lf[l])
        rows.append((l, ws, wc, lp, t, it, ms))
    h.free()
    return feats, rows, (rho_p, it_p, ms_p)


def selection_regret(y: np.ndarray, T: np.ndarray, owner: np.ndarray) -> float:
    """Mean over problems of T[argmin_k y_k] - min_k T_k over each problem's measured
    candidates: how much slower the network's pick converges than the best measured
    one (log10 of the factor ratio).  This is what the selection needs from the
    network (its argmin), unlike the mean squared error over all candidates."""
    order = np.argsort(owner, kind="stable")
    o, yy, tt = owner[order], y[order], T[order]
    starts = np.flatnonzero(np.r_[True, o[1:] != o[:-1]])
    ends = np.r_[starts[1:], len(o)]
    reg = [tt[a + int(np.argmin(yy[a:b]))] - tt[a:b].min() for a, b in zip(starts, ends)]
    return float(np.mean(reg)) if reg else 0.0


RANK_TAU = 0.01   # softmax temperature of the listwise ranking loss (log10 factor units)


def rank_loss_grad(y: np.ndarray, T: np.ndarray, groups: int, tau: float = RANK_TAU):
    """Listwise ranking loss over each problem's measured candidates (rows of the
    (groups, k) reshapes of y and T): L = -mean_p sum_k q_pk log p_pk with
    q = softmax(-T / tau) (the measured order) and p = softmax(-y / tau) (the
    network's), so the candidate the network ranks first is pushed towards the one
    that measured best.  Returns (L, dL/dy)."""
    yy = y.reshape(groups, -1) / -tau
    tt = T.reshape(groups, -1) / -tau
    yy = yy - yy.max(axis=1, keepdims=True)
    tt = tt - tt.max(axis=1, keepdims=True)
    lp = yy - np.log(np.exp(yy).sum(axis=1, keepdims=True))
    q = np.exp(tt) / np.exp(tt).sum(axis=1, keepdims=True)
    loss = float(-(q * lp).sum(axis=1).mean())
    d = (q - np.exp(lp)) / tau / groups
    return loss, d.reshape(-1)


def train(X: np.ndarray, T: np.ndarray, train_idx, val_idx, steps: int, lr: float, seed: int,
          torch, owner: np.ndarray | None = None, loss_kind: str = "mse"):
    from . import binding as B
    rng = np.random.default_rng(seed)
    # He-scaled normal initialisation, zero biases (W1, b1, W2, b2, W3, b3)
    th = np.concatenate([rng.standard_normal(64 * 16) * np.sqrt(2 / 16), np.zeros(64),
                         rng.standard_normal(64 * 64) * np.sqrt(2 / 64), np.zeros(64),
                         rng.standard_normal(64) * np.sqrt(1 / 64), np.zeros(1)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa
    theta = dev(th)
    g = torch.zeros(B.MLP_NPARAM, device="cuda")
    m, v = torch.zeros_like(g), torch.zeros_like(g)
    loss = torch.zeros(1, device="cuda")
    Xt, Tt, Xv, Tv = dev(X[train_idx]), dev(T[train_idx]), dev(X[val_idx]), dev(T[val_idx])
    hist = []
    best, best_val = theta.clone(), float("inf")
    yv = torch.zeros(max(len(val_idx), 1), device="cuda")
    Tv_h = T[val_idx]
    ov = owner[val_idx] if owner is not None else None
    t0 = time.time()
    rank = loss_kind == "rank"
    if rank:
        # every problem contributes the same number of consecutive rows
        ot = owner[train_idx]
        per = int(np.sum(ot == ot[0]))
        assert len(ot) % per == 0 and np.all(ot.reshape(-1, per) == ot[::per, None])
        groups = len(ot) // per
        Th = T[train_idx].astype(np.float64)
        yt = torch.zeros(len(train_idx), device="cuda")
        dyt = torch.zeros(len(train_idx), device="cuda")
    for step in range(1, steps + 1):
        # learning rate: constant, then divided by 10 over the last third
        lr_k = lr if step <= 2 * steps // 3 else lr * 0.1
        if rank:
            B.mlp_forward(theta, Xt, yt)
            lval, d = rank_loss_grad(yt.cpu().numpy().astype(np.float64), Th, groups)
            dyt.copy_(torch.from_numpy(d.astype(np.float32)))
            B.mlp_backward(theta, Xt, dyt, g)
            loss.fill_(lval)
        else:
            B.mlp_gradient(theta, Xt, Tt, g, loss)
        B.mlp_adam(theta, g, m, v, step, lr_k)
        if step % 100 == 0 or step == steps:
            B.mlp_forward(theta, Xv, yv)
            vl = float(((yv[:len(val_idx)] - Tv) ** 2).mean().item()) if len(val_idx) else 0.0
            # keep the parameters whose argmin over each validation problem's measured
            # candidates is best (selection regret); the MSE without problem ids
            crit = (selection_regret(yv[:len(val_idx)].cpu().numpy(), Tv_h, ov)
                    if ov is not None and len(val_idx) else vl)
            if crit < best_val:
                best_val = crit
                best.copy_(theta)
            if step % 500 == 0 or step == steps:
                hist.append({"step": step, "train_mse": loss.item(), "val_mse": vl,
                             "val_regret": crit if ov is not None else None})
    torch.cuda.synchronize()
    hist.append({"kept": "lowest validation selection regret" if owner is not None
                 else "lowest validation error", "value": best_val})
    return best.cpu().numpy(), hist, time.time() - t0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--problems", type=int, default=1200)
    ap.add_argument("--candidates", type=int, default=6)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "weights",
                                                  "mlp_theta.npy"))
    ap.add_argument("--loss", default="mse", choices=["mse", "rank"],
                    help="mse: fit the measured targets; rank: listwise ranking of each "
                         "problem's candidates (back-propagated with amg_mlp_backward)")
    ap.add_argument("--data", default=None,
                    help="train on a dataset written by an earlier run (<out>.data.npz) "
                         "instead of measuring one")
    args = ap.parse_args(argv)
    if args.data:
        return train_only(args)

    specs = [problem_spec(i) for i in range(args.problems)]
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(args.workers)          # before the first CUDA call
    import torch
    from . import binding as B
    B.load_library()
    rng = np.random.default_rng(7)
    feats, rows, plain, owner = [], [], [], []
    t0 = time.time()
    chunks = [specs[k:k + args.chunk] for k in range(0, len(specs), args.chunk)]
    pending = pool.map_async(make_problem, chunks[0]) if chunks else None
    gen_wait = 0.0
    for ci in range(len(chunks)):
        tw = time.time()
        probs = pending.get()
        gen_wait += time.time() - tw
        pending = pool.map_async(make_problem, chunks[ci + 1]) if ci + 1 < len(chunks) else None
        for k, prob in enumerate(probs):
            fs, r, p = measure(prob, args.candidates, rng, torch)
            pi = ci * args.chunk + k
            for f, row in zip(fs, r):
                feats.append(f)
                rows.append(row)
                owner.append(pi)
            plain.append(p)
        del probs
        print(f"chunk {ci + 1}/{len(chunks)}: {len(plain)} problems, "
              f"{time.time() - t0:.0f} s", flush=True)
    pool.close()
    pool.join()
    measure_s = time.time() - t0

    F = np.array(feats)
    R = np.array(rows)          # level, ws, wc, lp, target, iterations, ms
    X = np.concatenate([F, R[:, 1:4]], axis=1).astype(np.float32)
    T = R[:, 4].astype(np.float32)
    owner = np.array(owner)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(os.path.splitext(args.out)[0] + ".data.npz", X=X, T=T, owner=owner, rows=R,
             plain=np.array(plain))
    perm = np.random.default_rng(11).permutation(len(plain))
    val_p = set(perm[:max(1, len(plain) // 10)].tolist())
    val_idx = np.array([i for i in range(len(T)) if owner[i] in val_p], dtype=np.int64)
    train_idx = np.array([i for i in range(len(T)) if owner[i] not in val_p], dtype=np.int64)
    theta, hist, train_s = train(X, T, train_idx, val_idx, args.steps, args.lr, 3, torch, owner,
                                 args.loss)

    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, theta.astype(np.float32))
    Pl = np.array(plain)
    summary = {
        "problems": args.problems, "candidates_per_problem": args.candidates,
        "samples": int(len(T)), "train_samples": int(len(train_idx)),
        "val_samples": int(len(val_idx)), "seed0": SEED0, "steps": args.steps, "lr": args.lr,
        "target_mean": float(T.mean()), "target_std": float(T.std()),
        "share_candidates_better_than_plain": float(np.mean(R[R[:, 4] != 0.0, 4] < 0.0))
        if np.any(R[:, 4] != 0.0) else 0.0,
        "share_better_by_level": {int(l): float(np.mean(R[(R[:, 0] == l) & (R[:, 4] != 0.0), 4]
                                                        < 0.0))
                                  for l in np.unique(R[1:, 0])},
        "plain_iterations_mean": float(Pl[:, 1].mean()),
        "history": hist, "measure_s": measure_s, "generation_wait_s": gen_wait,
        "train_s": train_s,
    }
    with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k != "history"}), flush=True)
    print(json.dumps(hist[-1]), flush=True)


def train_only(args):
    """Retrain on a saved dataset (seconds on the GPU)."""
    import torch
    from . import binding as B
    B.load_library()
    d = np.load(args.data)
    X, T, owner = d["X"], d["T"], d["owner"]
    nprob = int(owner.max()) + 1
    perm = np.random.default_rng(11).permutation(nprob)
    val_p = np.zeros(nprob, dtype=bool)
    val_p[perm[:max(1, nprob // 10)]] = True
    val_idx = np.nonzero(val_p[owner])[0]
    train_idx = np.nonzero(~val_p[owner])[0]
    theta, hist, train_s = train(X, T, train_idx, val_idx, args.steps, args.lr, 3, torch, owner,
                                 args.loss)
    np.save(args.out, theta.astype(np.float32))
    summary = {"data": os.path.basename(args.data), "loss": args.loss, "samples": int(len(T)),
               "train_samples": int(len(train_idx)), "val_samples": int(len(val_idx)),
               "steps": args.steps, "lr": args.lr, "target_mean": float(T.mean()),
               "target_std": float(T.std()), "history": hist, "train_s": train_s}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps(hist[-1]), flush=True)


if __name__ == "__main__":
    main()
