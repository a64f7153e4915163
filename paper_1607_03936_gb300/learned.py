"""Train and evaluate the learned pressure-Poisson correction (orchestration only).

Every numerical step runs in libwbfbt.so: the solver generates the training pairs
(wbfbt_learned_sample: features of a random residual and its V-cycle correction for
K_r = B D_w^-1 B^T), the U-Net trains with the library's BF16 tensor-core forward and
backward kernels and Adam, and the evaluation runs FGMRES with the net attached and the
V-cycle as fallback.

  python -m paper_1607_03936_gb300.learned train --out net.bin
  python -m paper_1607_03936_gb300.learned evaluate --ckpt net.bin
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import build as _build
from . import inputs

_build.build()
from . import wbfbt as wb  # noqa: E402


def problem_draw(seed: int):
    """Seeded multi-sinker problem of the training family: 8-48 sinkers, DR log-uniform [1e4, 1e8]."""
    u = inputs.uniform01(seed * 7919 + 17, 2)
    ns = 8 + int(u[0] * 41)
    dr = 10.0 ** (4.0 + 4.0 * u[1])
    return inputs.sinker_centres(seed, ns), dr


def smooth_pressure(n: int, np_: int, seed: int) -> np.ndarray:
    """A smooth random pressure field on the element grid as P_{k-1} coefficients [n^3][Np]:
    a sum of cosines of wave numbers 0..3 per axis, the constant mode taking the value at the
    element centre and the three linear modes its derivatives times h/2."""
    rng = np.random.default_rng(seed)
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    val = np.zeros_like(X)
    gx, gy, gz = np.zeros_like(X), np.zeros_like(X), np.zeros_like(X)
    for kz in range(4):
        for ky in range(4):
            for kx in range(4):
                if kx + ky + kz == 0:
                    continue
                a = rng.standard_normal() / (kx * kx + ky * ky + kz * kz)
                cx, cy, cz = np.cos(np.pi * kx * X), np.cos(np.pi * ky * Y), np.cos(np.pi * kz * Z)
                val += a * cx * cy * cz
                gx += -a * np.pi * kx * np.sin(np.pi * kx * X) * cy * cz
                gy += -a * np.pi * ky * cx * np.sin(np.pi * ky * Y) * cz
                gz += -a * np.pi * kz * cx * cy * np.sin(np.pi * kz * Z)
    out = np.zeros((n ** 3, np_))
    h = 1.0 / n
    out[:, 0] = val.ravel()
    if np_ >= 4:
        out[:, 1], out[:, 2], out[:, 3] = gx.ravel() * h / 2, gy.ravel() * h / 2, gz.ravel() * h / 2
    return out.ravel()


def make_pairs(n: int, k: int, n_fields: int, per_field: int, seed0: int, omega=0.1, delta=200.0,
               smooth_fraction: float = 0.0):
    """(x [P][n^3][1+Np], y [P][n^3][Np]) device tensors from n_fields viscosity fields.

    A fraction of the residuals is r = K_w z for a smooth random pressure z (the low-frequency
    residuals FGMRES feeds the preconditioner late in a solve), the rest standard normal.
    """
    xs, ys = [], []
    solver = None
    for f in range(n_fields):
        centres, dr = problem_draw(seed0 + f)
        mu, _ = wb.sinker_setup(n, k, centres, omega, delta, dr)
        if solver is None:
            solver = wb.Solver(n, k, mu, precision=wb.MIXED)
        else:
            solver.setup(mu)
        for j in range(per_field):
            sd = 1_000_003 * (seed0 + f) + j
            if j < int(round(smooth_fraction * per_field)):
                z = torch.tensor(smooth_pressure(n, solver.np, sd), device="cuda")
                r = solver.apply_Kw(1, z) if solver.precision == wb.F64 else \
                    solver.apply_Kw(1, z.float()).double()
            else:
                r = torch.tensor(inputs.normal_vector(sd, solver.n_p), device="cuda")
            r = r.view(-1, solver.np)
            r[:, 0] -= r[:, 0].mean()                         # mean-free (constant mode)
            x, y = solver.learned_sample(1, r.reshape(-1).contiguous())
            xs.append(x)
            ys.append(y)
    solver.close()
    return torch.stack(xs), torch.stack(ys)


def train(n=32, k=2, n_fields=100, per_field=20, epochs=20, batch=4, lr=1e-3, seed=1000, init_seed=7,
          smooth_fraction=0.0, log=print):
    t0 = time.time()
    x, y = make_pairs(n, k, n_fields, per_field, seed, smooth_fraction=smooth_fraction)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    npe = k * (k + 1) * (k + 2) // 6
    net = wb.Net(1 + npe, npe, n, max_batch=batch)
    net.set_params(torch.tensor(inputs.unet_init_params(init_seed, 1 + npe, npe), device="cuda"))
    P = x.shape[0]
    steps = epochs * (P // batch)
    order_rng = np.random.default_rng(seed + 12345)
    t1 = time.time()
    step, hist = 0, []
    for ep in range(epochs):
        perm = order_rng.permutation(P)
        losses = []
        for b in range(P // batch):
            idx = torch.tensor(perm[b * batch:(b + 1) * batch], device="cuda")
            loss, _ = net.loss_grad(x[idx], y[idx], want_grad=False)
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / steps))   # cosine decay
            net.adam_step(max(lr_t, 1e-5))
            losses.append(loss)
            step += 1
        hist.append(float(np.mean(losses)))
        log(json.dumps({"epoch": ep, "loss": hist[-1], "elapsed_s": round(time.time() - t1, 2)}))
    torch.cuda.synchronize()
    return net, {"pairs": P, "data_s": t_data, "train_s": time.time() - t1, "steps": steps, "loss_hist": hist}


def evaluate(net, n=32, k=2, seeds=range(5000, 5020), omega=0.1, delta=200.0, accept_ratio=1.0, log=print):
    """FGMRES with and without the net on held-out problems (mixed precision)."""
    rows = []
    for s in seeds:
        centres, dr = problem_draw(s)
        mu, f = wb.sinker_setup(n, k, centres, omega, delta, dr)
        res = {"seed": s, "sinkers": len(centres), "dr": dr}
        sols = {}
        for tag in ("vcycle", "learned"):
            solver = wb.Solver(n, k, mu, precision=wb.MIXED)
            if tag == "learned":
                solver.attach_net(net, 2, accept_ratio)
            solver.solve(f)                                    # warm-up
            torch.cuda.synchronize()
            t0 = time.time()
            u, p, r = solver.solve(f)
            torch.cuda.synchronize()
            res[tag] = {"iters": r.iters, "rel_res": r.rel_res, "solve_s": round(time.time() - t0, 4)}
            if tag == "learned":
                a, rj = solver.learned_stats()
                res[tag]["accepted"], res[tag]["rejected"] = a, rj
            sols[tag] = (u.clone(), p.clone())
            solver.close()
        res["u_diff"] = float((torch.linalg.norm(sols["learned"][0] - sols["vcycle"][0]) /
                               torch.linalg.norm(sols["vcycle"][0])).item())
        rows.append(res)
        log(json.dumps(res))
    return rows


def profile(n=32, k=2, batch=1):
    """Three warm-up forwards, then one forward and one loss/gradient pass of the U-Net inside the
    NVTX range "prof" (for ncu --nvtx --nvtx-include prof/); prints the timed forward."""
    npe = k * (k + 1) * (k + 2) // 6
    net = wb.Net(1 + npe, npe, n, max_batch=batch)
    net.set_params(torch.tensor(inputs.unet_init_params(7, 1 + npe, npe), device="cuda"))
    g = torch.Generator("cuda").manual_seed(0)
    x = torch.randn(batch, n ** 3, 1 + npe, device="cuda", generator=g)
    t = torch.randn(batch, n ** 3, npe, device="cuda", generator=g)
    for _ in range(3):
        net.forward(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        net.forward(x)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("prof")
    net.forward(x)
    net.loss_grad(x, t)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"unet_forward_us": e0.elapsed_time(e1) * 100.0, "n": n, "batch": batch,
                      "params": wb.Net.num_params(1 + npe, npe)}))


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    pr = sub.add_parser("profile")
    pr.add_argument("--n", type=int, default=32)
    t = sub.add_parser("train")
    t.add_argument("--n", type=int, default=32)
    t.add_argument("--fields", type=int, default=100)
    t.add_argument("--per-field", type=int, default=20)
    t.add_argument("--epochs", type=int, default=20)
    t.add_argument("--batch", type=int, default=4)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--out", required=True)
    t.add_argument("--evaluate", type=int, default=0, help="held-out seeds to evaluate after training")
    t.add_argument("--accept", type=float, default=1.0, help="keep a learned step if it leaves < accept x ||r||")
    t.add_argument("--smooth", type=float, default=0.0, help="fraction of smooth (K_w z) residuals")
    e = sub.add_parser("evaluate")
    e.add_argument("--ckpt", required=True)
    e.add_argument("--n", type=int, default=32)
    e.add_argument("--seeds", type=int, default=20)
    e.add_argument("--accept", type=float, default=1.0)
    a = ap.parse_args()
    if a.cmd == "profile":
        profile(n=a.n)
    elif a.cmd == "train":
        net, info = train(n=a.n, n_fields=a.fields, per_field=a.per_field, epochs=a.epochs, batch=a.batch, lr=a.lr,
                          smooth_fraction=a.smooth)
        net.save(a.out)
        print(json.dumps({"train": info}))
        if a.evaluate:
            evaluate(net, n=a.n, seeds=range(5000, 5000 + a.evaluate), accept_ratio=a.accept)
    else:
        net = wb.Net(5, 4, a.n)
        net.load(a.ckpt)
        evaluate(net, n=a.n, seeds=range(5000, 5000 + a.seeds), accept_ratio=a.accept)


if __name__ == "__main__":
    main()
