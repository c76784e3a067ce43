"""Learned coarse correction: training data, training and held-out evaluation,
driven through the C ABI (every step runs in libnh's kernels).

    python -m paper_2204_01722_b300.learned [--n 64 --p 3 --train 20 --test 5]

Recipe (the defaults): Q_p on an n^3 unit cube with seeded spherical
inclusions (volume fraction 0.3, radius 2-6 elements, stiffness contrast 1e3),
x = 0 clamped, x = 1 pushed along x.  For every layout the state is first
solved to 1% compression (L-BFGS with the mixed-precision V-cycle and the
geometric coarse multigrid).  At that state the p-multigrid hierarchy
p -> 2 -> 1 uses the fixed coarse solve (``coarse_fixed`` Chebyshev-Jacobi
steps on the assembled Q1 level), and for a few right-hand sides (N(0,1) and
smooth seeded fields) nh_mg_collect records, at every coarsest solve along the
FCG + V-cycle iterations of J x = b, the residual r1 that fixed solve leaves
and its exact correction A_c^-1 r1.  The network (4 levels, 16/32/48/64
channels, BF16 weights and activations, FP32 accumulation) is trained by Adam
on the mean relative squared error; its predictions then span the learned
coarse space (learned_mode 4).  Held-out layouts: the tangent system at 1%
compression with an N(0,1) right-hand side is solved to ||r|| <= 1e-8 ||b|| by
plain FP64 p-MG (Jacobi-PCG coarse solve to 1e-3, the paper's), the
mixed-precision V-cycle with the fixed coarse solve, the same with a coarse
space built without the network and with the learned coarse space (each size
in --vectors), and the mixed-precision V-cycle with the geometric coarse
multigrid; setup and solve are timed apart (median after a warm-up).
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
    return dict(space=sp, op=op, g1=g1, nd=nd, mask=mask, X=X, n=n, p=p)


def close(pb, mg=None):
    if mg:
        nh.nh_mg_destroy(mg)
    nh.nh_op_destroy(pb["op"])
    nh.nh_space_destroy(pb["space"])


def solve_state(ctx, pb, delta):
    """Displacement at `delta` compression (one load step), by the chosen solver."""
    import torch
    o = nh.nh_mg_default_opts(ctx, pb["op"], mixed=1, fp64_kind=1, coarse_rediscretize=1, nonlinear=1,
                              coarse_solver=1, load_steps=1)
    mg = nh.nh_mg_create(ctx, pb["op"], o)
    u = torch.zeros(pb["nd"], dtype=torch.float64, device="cuda")
    rep = nh.nh_solve(ctx, mg, pb["g1"] * delta, u, check=False)
    nh.nh_mg_destroy(mg)
    nh.nh_qdata_setup(ctx, pb["op"], u)
    return u, rep


def rhs_vectors(pb, seed, k):
    out = []
    for j in range(k):
        if j % 2 == 0:
            b = inputs.normal_vector(pb["nd"], seed=1000 * seed + j)
        else:
            b = inputs.smooth_field(pb["X"], 1.0, seed=1000 * seed + j).ravel()
        b[pb["mask"]] = 0.0
        out.append(b)
    return out


VARIANTS = ("plain_fp64", "mixed_fixed", "mixed_fixed_space", "mixed_fixed_learned", "mixed_fixed_exact",
            "mixed_geometric")


def variant_opts(ctx, pb, name, coarse_fixed, vectors=32):
    kw = dict(plain_fp64=dict(),
              mixed_fixed=dict(mixed=1, coarse_fixed=coarse_fixed, learned_mode=3),
              mixed_fixed_space=dict(mixed=1, coarse_fixed=coarse_fixed, learned_mode=4, learned_vectors=vectors),
              mixed_fixed_learned=dict(mixed=1, coarse_fixed=coarse_fixed, learned_mode=4, learned_vectors=vectors),
              mixed_fixed_exact=dict(mixed=1, coarse_fixed=coarse_fixed, learned_mode=4, learned_vectors=vectors,
                                     learned_accept=1),
              mixed_geometric=dict(mixed=1, coarse_solver=1))[name]
    return nh.nh_mg_default_opts(ctx, pb["op"], **kw)


def collect(ctx, stream, pb, seed, coarse_fixed, rhs=3, pairs=16):
    """(network input, target) pairs of the post-correction at the current state."""
    import torch
    Nv = pb["n"] + 1
    mg = nh.nh_mg_create(ctx, pb["op"], variant_opts(ctx, pb, "mixed_fixed", coarse_fixed))
    nh.nh_mg_setup(ctx, mg)
    F, T = [], []
    for b in rhs_vectors(pb, seed, rhs):
        f = torch.zeros((pairs, 4, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
        t = torch.zeros((pairs, 3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
        k = nh.nh_mg_collect(ctx, mg, torch.from_numpy(b).cuda(), pairs, f, t)
        F.append(f[:k])
        T.append(t[:k])
    nh.nh_mg_destroy(mg)
    stream.synchronize()
    return torch.cat(F), torch.cat(T)


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


def validation_loss(ctx, net, feats, tgts):
    """Mean relative squared error on held-out pairs (forward only)."""
    import torch
    Nv = feats.shape[-1]
    y = torch.empty((3, Nv, Nv, Nv), dtype=torch.float32, device="cuda")
    errs = []
    for i in range(feats.shape[0]):
        nh.nh_net_forward(ctx, net, feats[i].contiguous(), y)
        t = tgts[i]
        errs.append(float(((y - t) ** 2).sum() / (t ** 2).sum()))
    return float(np.mean(errs)) if errs else float("nan")


def linear_eval(ctx, stream, pb, seed, net, coarse_fixed, vectors=(32,), rtol=1e-8, maxit=2000, repeats=1,
                exact=False):
    """Tangent solve J x = b at the current state, per solver variant: setup
    (diagonals, Lanczos, coarse level, coarse space) and solve timed apart, each
    the median over `repeats` runs after one discarded warm-up."""
    import torch
    b = torch.from_numpy(rhs_vectors(pb, 10 ** 6 + seed, 1)[0]).cuda()
    rows = []
    runs = [(name, k) for name in VARIANTS if name != "mixed_fixed_exact" or exact
            for k in (vectors if "space" in name or "learned" in name or "exact" in name else (0,))]
    for name, k in runs:
        mg = nh.nh_mg_create(ctx, pb["op"], variant_opts(ctx, pb, name, coarse_fixed, k))
        if name == "mixed_fixed_learned":
            nh.nh_mg_set_learned(ctx, mg, net)
        t_setup, t_solve, rep = [], [], None
        for _ in range(repeats + 1):
            stream.synchronize()
            t0 = time.perf_counter()
            nh.nh_mg_setup(ctx, mg)
            stream.synchronize()
            t1 = time.perf_counter()
            x = torch.zeros(pb["nd"], dtype=torch.float64, device="cuda")
            rep = nh.nh_linear_solve(ctx, mg, b, x, rtol=rtol, maxit=maxit, norm=1, check=False)
            stream.synchronize()
            t_setup.append(t1 - t0)
            t_solve.append(time.perf_counter() - t1)
        d = rep.as_dict()
        d.update(layout=seed, solver=name if k in (0, vectors[0]) else f"{name}_{k}",
                 t_setup=float(np.median(t_setup[1:])),
                 seconds=float(np.median(t_solve[1:])))
        d["total"] = d["t_setup"] + d["seconds"]
        rows.append(d)
        nh.nh_mg_destroy(mg)
    return rows


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--train", type=int, default=20)
    ap.add_argument("--test", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--rhs", type=int, default=3)
    ap.add_argument("--pairs", type=int, default=16)
    ap.add_argument("--coarse-fixed", type=int, default=30)
    ap.add_argument("--channels", default="16,32,48,64")
    ap.add_argument("--delta", type=float, default=0.01)
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--vectors", default="32")
    ap.add_argument("--exact-space", action="store_true",
                    help="also evaluate the coarse space of exact coarse errors (what a perfect network would give)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    stream = torch.cuda.Stream()
    res = dict(n=a.n, p=a.p, train_layouts=a.train, test_layouts=a.test, coarse_fixed=a.coarse_fixed,
               channels=a.channels, delta=a.delta)
    with torch.cuda.stream(stream):
        ctx = nh.nh_create(0, stream.cuda_stream)
        t0 = time.perf_counter()
        F, T = [], []
        for s in range(1, a.train + 1):
            pb = problem(ctx, a.n, a.p, s)
            solve_state(ctx, pb, a.delta)
            f, t = collect(ctx, stream, pb, s, a.coarse_fixed, rhs=a.rhs, pairs=a.pairs)
            F.append(f)
            T.append(t)
            close(pb)
        feats, tgts = torch.cat(F).contiguous(), torch.cat(T).contiguous()
        del F, T
        res["pairs"] = int(feats.shape[0])
        res["collect_s"] = time.perf_counter() - t0
        ch = [int(c) for c in a.channels.split(",")]
        net = nh.nh_net_create(ctx, a.n + 1, len(ch), ch, bf16=True, seed=7)
        t0 = time.perf_counter()
        res["loss"] = train(ctx, net, feats, tgts, epochs=a.epochs, lr=a.lr)
        stream.synchronize()
        res["train_s"] = time.perf_counter() - t0
        print(json.dumps(dict(pairs=res["pairs"], collect_s=res["collect_s"], train_s=res["train_s"],
                              loss=res["loss"])), flush=True)
        del feats, tgts
        rows, vloss = [], []
        for s in range(101, 101 + a.test):
            pb = problem(ctx, a.n, a.p, s)
            _, rep = solve_state(ctx, pb, a.delta)
            f, t = collect(ctx, stream, pb, s, a.coarse_fixed, rhs=1, pairs=a.pairs)
            vloss.append(validation_loss(ctx, net, f, t))
            del f, t
            rows += linear_eval(ctx, stream, pb, s, net, a.coarse_fixed, [int(v) for v in a.vectors.split(",")],
                                repeats=a.repeats, exact=a.exact_space)
            close(pb)
            if a.out:   # partial results after every held-out layout
                with open(a.out, "w") as f:
                    f.write(json.dumps(dict(res, eval=rows, heldout_loss=vloss)) + "\n")
        res["heldout_loss"] = vloss
        res["eval"] = rows
        for name in sorted({r["solver"] for r in rows}):
            sel = [r for r in rows if r["solver"] == name]
            res[name] = {k: float(np.mean([r[k] for r in sel])) for k in
                         ("seconds", "t_setup", "total", "krylov_its", "vcycles", "coarse_its", "rel_residual")}
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
