"""Learned coarse correction: training data, training and held-out evaluation,
driven through the C ABI (every step runs in libnh's kernels).

    python -m paper_2204_01722_b300.learned [--n 64 --p 3 --train 20 --test 5]

Recipe (the defaults): Q_p on an n^3 unit cube with seeded spherical
inclusions (volume fraction 0.3, radius 2-6 elements, stiffness contrast 1e3),
x = 0 clamped, x = 1 pushed along x.  For every training layout the solver is
first run to a deformed state (1% compression), then for a few right-hand sides
(N(0,1) and smooth seeded fields) nh_mg_collect records (network input,
target) pairs along the FCG + V-cycle iterations of J x = b.  The network
(3 levels, 16/32/64 channels, BF16 weights and activations, FP32 accumulation)
is trained by Adam on the mean relative squared error.  Evaluation solves the
held-out layouts (load-stepped compression to 5%) with the chosen solver
(mixed precision) with and without the learned stage, and with plain FP64 p-MG.
"""
import argparse
import json
import sys
import time

import numpy as np

from . import inputs, nh


def problem(ctx, n, p, seed, vf=0.3, rmin=2.0, rmax=6.0, contrast=1e3):
    import torch
    V = inputs.box_vertices(n, n, n)
    sp, nn, nd = nh.nh_space_box(ctx, n, n, n, V, p, p + 1)
    N = p * n + 1
    mask = inputs.uniaxial_mask((N, N, N))
    nh.nh_space_set_dirichlet(ctx, sp, mask)
    E = inputs.inclusion_modulus(n, n, n, seed=seed, vf=vf, rmin=rmin, rmax=rmax, contrast=contrast)
    op = nh.nh_op_create(ctx, sp, 0.3, E)
    g1 = torch.from_numpy(inputs.uniaxial_bc((N, N, N), 1.0)).cuda()
    X = nh.nh_space_coords(ctx, sp, nn)
    return dict(space=sp, op=op, g1=g1, nd=nd, mask=mask, X=X)


def close(pb, mg=None):
    if mg:
        nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(pb["op"])
    nh.nh_space_destroy(pb["space"])


def collect(ctx, stream, n, p, seeds, delta_state=0.01, rhs=3, pairs=8, mixed=1):
    import torch
    Nv = n + 1
    F, T = [], []
    for s in seeds:
        pb = problem(ctx, n, p, s)
        mg = nh.nh_mg_create(ctx, pb["op"], nh.nh_mg_default_opts(ctx, pb["op"], mixed=mixed, load_steps=1))
        u = torch.zeros(pb["nd"], dtype=torch.float64, device="cuda")
        nh.nh_solve(ctx, mg, pb["g1"] * delta_state, u, check=False)
        nh.nh_qdata_setup(ctx, pb["op"], u)
        nh.nh_mg_setup(ctx, mg)
        for j in range(rhs):
            if j % 2 == 0:
                b = inputs.normal_vector(pb["nd"], seed=1000 * s + j)
            else:
                b = inputs.smooth_field(pb["X"], 1.0, seed=1000 * s + j).ravel()
            b[pb["mask"]] = 0.0
            f = torch.zeros((pairs, 4, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
            t = torch.zeros((pairs, 3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
            k = nh.nh_mg_collect(ctx, mg, torch.from_numpy(b).cuda(), pairs, f, t)
            F.append(f[:k])
            T.append(t[:k])
        close(pb, mg)
    stream.synchronize()
    return torch.cat(F).contiguous(), torch.cat(T).contiguous()


def train(ctx, net, feats, tgts, epochs=20, lr=1e-3, batch=4, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    m = feats.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(m)).cuda()
        tot, cnt = 0.0, 0
        for i in range(0, m - batch + 1, batch):
            idx = perm[i:i + batch]
            x = feats.index_select(0, idx).contiguous()
            t = tgts.index_select(0, idx).contiguous()
            tot += nh.nh_net_train_step(ctx, net, batch, x, t, lr) * batch
            cnt += batch
        hist.append(tot / max(cnt, 1))
    return hist


def evaluate(ctx, stream, n, p, seeds, delta=0.05, steps=5, nets=(("plain_fp64", 0, None),)):
    import torch
    rows = []
    for s in seeds:
        pb = problem(ctx, n, p, s)
        for name, mixed, net in nets:
            mg = nh.nh_mg_create(ctx, pb["op"], nh.nh_mg_default_opts(ctx, pb["op"], mixed=mixed, load_steps=steps))
            if net:
                nh.nh_mg_set_learned(ctx, mg, net)
            u = torch.zeros(pb["nd"], dtype=torch.float64, device="cuda")
            rep = nh.nh_solve(ctx, mg, pb["g1"] * delta, u, check=False)
            stream.synchronize()
            d = rep.as_dict()
            d.update(layout=s, solver=name)
            rows.append(d)
            nh.nh_mg_destroy(mg)
        close(pb)
    return rows


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--train", type=int, default=20)
    ap.add_argument("--test", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--rhs", type=int, default=3)
    ap.add_argument("--pairs", type=int, default=8)
    ap.add_argument("--channels", default="16,32,64")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    stream = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(stream):
        ctx = nh.nh_create(0, stream.cuda_stream)
        t0 = time.perf_counter()
        feats, tgts = collect(ctx, stream, a.n, a.p, range(1, a.train + 1), rhs=a.rhs, pairs=a.pairs)
        res["pairs"] = int(feats.shape[0])
        res["collect_s"] = time.perf_counter() - t0
        ch = [int(c) for c in a.channels.split(",")]
        net = nh.nh_net_create(ctx, a.n + 1, len(ch), ch, bf16=True, seed=7)
        t0 = time.perf_counter()
        res["loss"] = train(ctx, net, feats, tgts, epochs=a.epochs, lr=a.lr)
        stream.synchronize()
        res["train_s"] = time.perf_counter() - t0
        del feats, tgts
        rows = evaluate(ctx, stream, a.n, a.p, range(101, 101 + a.test),
                        nets=(("plain_fp64", 0, None), ("mixed", 1, None), ("mixed_learned", 1, net)))
        res["eval"] = rows
        for name in ("plain_fp64", "mixed", "mixed_learned"):
            sel = [r for r in rows if r["solver"] == name]
            res[name] = {k: float(np.mean([r[k] for r in sel])) for k in
                         ("seconds", "krylov_its", "newton_its", "vcycles", "coarse_its", "learned_accepted",
                          "learned_rejected")}
            res[name]["converged"] = all(r["status"] == 0 for r in sel)
        nh.nh_net_destroy(net)
        nh.nh_destroy(ctx)
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    sys.exit(main())
