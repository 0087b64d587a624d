"""Learned warm start for lb_steady: a small 3D convolutional encoder-decoder that maps a
porous medium (its fluid and forced-cluster masks) to an estimate of the steady LB state
(velocity and density) driven by a unit body force, used only as the starting state of
lb_steady. The plain LB still runs to the same residual, so it alone decides convergence; a
poor estimate costs steps, never accuracy. The paper solves the LB from rest; this is a
GB300-side acceleration of that solve.

The density matters as much as the velocity: restarted from f^eq(rho = 1, u*) with the
exact steady velocity u*, the LB of a 128^3 porous medium needs as many steps as from rest
(its slow modes are the pressure field's), while f^eq(rho*, u*) converges about five times
faster. The network therefore predicts (rho - 1) / F as a fourth output.

Network (2.35 M parameters): U-Net style, periodic 3x3x3 convolutions, ReLU, three 2x average
poolings and three nearest upsamplings with additive skips, 32 / 64 / 96 / 128 channels:
    e0a 16->32, e0b 32->32 | pool | e1a 32->64, e1b 64->64 | pool | e2a 64->96, e2b 96->96 |
    pool | b0 96->128, b1 128->128 | up | d2a 128->96 (+ e2b), d2b 96->96 | up |
    d1a 96->64 (+ e1b), d1b 64->64 | up | d0a 64->32 (+ e0b), d0b 32->32 | out 32->16
(receptive field about 120 nodes; a version with two poolings, 56 nodes, predicted the flow
with twice the error and saved fewer LB steps).
Inputs: channel 0 = fluid, 1 = in the largest connected fluid cluster (where the body force
acts); outputs: channels 0..2 = u / (|F| s_u) along the network axes, the force along the
first, channel 3 = (rho - 1) / (|F| s_rho); the warm start shifts the density to mean 1 over
the cluster (the LB conserves its mass). Every operation runs in the library's kernels (include/surrogate.h): BF16 activations
and weights, FP32 accumulation on the tensor cores, FP32 master weights and Adam. PyTorch only
allocates device memory.

Training data: seeded random-sphere media (Boolean model, porosity and radius drawn per
medium) solved by this library's lb_steady to residual 1e-7 under a force along x; the
weights file records the data recipe, the output scale s_u and the training log.

    python -m paper_1303_2470_gb300.surrogate train --out weights.npz
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import media

LAYERS = [  # name, input channels, output channels, ReLU
    ("e0a", 16, 32, True), ("e0b", 32, 32, True),
    ("e1a", 32, 64, True), ("e1b", 64, 64, True),
    ("e2a", 64, 96, True), ("e2b", 96, 96, True),
    ("b0", 96, 128, True), ("b1", 128, 128, True),
    ("d2a", 128, 96, True), ("d2b", 96, 96, True),
    ("d1a", 96, 64, True), ("d1b", 64, 64, True),
    ("d0a", 64, 32, True), ("d0b", 32, 32, True),
    ("out", 32, 16, False),
]
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_weights.npz")
F_TRAIN = 1e-5  # body force of the training solves (Stokes-linear regime: u scales with F)


def _torch():
    import torch
    return torch


class Surrogate:
    """Parameters (FP32 master, BF16 copies in forward and transposed order) and the
    forward / backward passes. All tensors live on the current CUDA device."""

    def __init__(self, params=None, seed=0, s_u=1.0, s_rho=1.0):
        torch = _torch()
        from . import mp
        self.mp = mp
        self.s_u = float(s_u)
        self.s_rho = float(s_rho)
        dev = torch.device("cuda")
        rng = np.random.default_rng(seed)
        self.p = {}
        for name, cin, cout, _ in LAYERS:
            if params is not None:
                W = np.asarray(params[name + ".W"], dtype=np.float32)
                b = np.asarray(params[name + ".b"], dtype=np.float32)
            else:
                fan = 27 * (2 if name == "e0a" else cin)    # the input has two live channels
                W = (rng.standard_normal((27, cin, cout)) * np.sqrt(2.0 / fan)).astype(np.float32)
                if name == "out":
                    W *= 0.1
                b = np.zeros(cout, dtype=np.float32)
            t = {
                "W": torch.as_tensor(W).to(dev).contiguous(),
                "b": torch.as_tensor(b).to(dev).contiguous(),
                "Wf": torch.empty((27, cout, cin), dtype=torch.bfloat16, device=dev),
                "Wb": torch.empty((27, cin, cout), dtype=torch.bfloat16, device=dev),
                "gW": torch.zeros((27, cin, cout), dtype=torch.float32, device=dev),
                "gb": torch.zeros(cout, dtype=torch.float32, device=dev),
                "mW": torch.zeros((27, cin, cout), dtype=torch.float32, device=dev),
                "vW": torch.zeros((27, cin, cout), dtype=torch.float32, device=dev),
                "mb": torch.zeros(cout, dtype=torch.float32, device=dev),
                "vb": torch.zeros(cout, dtype=torch.float32, device=dev),
                "cin": cin, "cout": cout,
            }
            self.p[name] = t
            # BF16 copies from the master weights: an Adam call with zero rate and gradient
            mp.sg_adam(t["W"], t["gW"], t["mW"], t["vW"], t["W"].numel(), 0.0, 0.9, 0.999, 1e-8, 1,
                       t["Wf"], t["Wb"], cin, cout)

    def n_params(self):
        return sum(t["W"].numel() + t["b"].numel() for t in self.p.values())

    # ---------------------------------------------------------------------------------
    def _conv(self, name, x, B, dims, out_f32=False):
        torch = _torch()
        t = self.p[name]
        D, H, W = dims
        relu = dict((l[0], l[3]) for l in LAYERS)[name]
        if out_f32:
            y = torch.empty((B, D * H * W, t["cout"]), dtype=torch.float32, device=x.device)
            self.mp.sg_conv3d(x, t["Wf"], t["b"], None, y, B, D, H, W, t["cin"], t["cout"], 1, relu)
        else:
            y = torch.empty((B, D * H * W, t["cout"]), dtype=torch.bfloat16, device=x.device)
            self.mp.sg_conv3d(x, t["Wf"], t["b"], y, None, B, D, H, W, t["cin"], t["cout"], 1, relu)
        return y

    def forward(self, x0, B, dims, keep=False):
        """x0 BF16 [B][V][16]; dims = (D, H, W) of the network box (multiples of 8).
        Returns (y FP32 [B][V][16], saved activations or None)."""
        torch = _torch()
        mp = self.mp
        D, H, W = dims
        l0, l1, l2, l3 = (D, H, W), (D // 2, H // 2, W // 2), (D // 4, H // 4, W // 4), (D // 8, H // 8, W // 8)
        dev = x0.device

        def new(level, C):
            d = level[0] * level[1] * level[2]
            return torch.empty((B, d, C), dtype=torch.bfloat16, device=dev)

        a = {}
        a["x0"] = x0
        a["a0"] = self._conv("e0a", x0, B, l0)
        a["s0"] = self._conv("e0b", a["a0"], B, l0)
        a["p0"] = new(l1, 32)
        mp.sg_pool2(a["s0"], a["p0"], B, *l0, 32)
        a["a1"] = self._conv("e1a", a["p0"], B, l1)
        a["s1"] = self._conv("e1b", a["a1"], B, l1)
        a["p1"] = new(l2, 64)
        mp.sg_pool2(a["s1"], a["p1"], B, *l1, 64)
        a["a2"] = self._conv("e2a", a["p1"], B, l2)
        a["s2"] = self._conv("e2b", a["a2"], B, l2)
        a["p2"] = new(l3, 96)
        mp.sg_pool2(a["s2"], a["p2"], B, *l2, 96)
        a["a3"] = self._conv("b0", a["p2"], B, l3)
        a["c3"] = self._conv("b1", a["a3"], B, l3)
        a["u2"] = new(l2, 128)
        mp.sg_up2(a["c3"], a["u2"], B, *l3, 128)
        a["d2"] = self._conv("d2a", a["u2"], B, l2)
        a["h2"] = new(l2, 96)
        mp.sg_add(a["d2"], a["s2"], a["h2"], a["h2"].numel())
        a["e2"] = self._conv("d2b", a["h2"], B, l2)
        a["u1"] = new(l1, 96)
        mp.sg_up2(a["e2"], a["u1"], B, *l2, 96)
        a["d1"] = self._conv("d1a", a["u1"], B, l1)
        a["h1"] = new(l1, 64)
        mp.sg_add(a["d1"], a["s1"], a["h1"], a["h1"].numel())
        a["e1"] = self._conv("d1b", a["h1"], B, l1)
        a["u0"] = new(l0, 64)
        mp.sg_up2(a["e1"], a["u0"], B, *l1, 64)
        a["d0"] = self._conv("d0a", a["u0"], B, l0)
        a["h0"] = new(l0, 32)
        mp.sg_add(a["d0"], a["s0"], a["h0"], a["h0"].numel())
        a["e0"] = self._conv("d0b", a["h0"], B, l0)
        y = self._conv("out", a["e0"], B, l0, out_f32=True)
        return y, (a if keep else None)

    def _back(self, name, x, g, B, dims, need_input_grad=True):
        """Accumulate the weight and bias gradients of layer `name` (input x, output gradient
        g already masked by its ReLU) and return the input gradient."""
        torch = _torch()
        t = self.p[name]
        self.mp.sg_conv3d_wgrad(x, g, t["gW"], t["gb"], B, *dims, t["cin"], t["cout"])
        if not need_input_grad:
            return None
        gx = torch.empty((B, x.shape[1], t["cin"]), dtype=torch.bfloat16, device=x.device)
        self.mp.sg_conv3d(g, t["Wb"], None, gx, None, B, *dims, t["cout"], t["cin"], -1, False)
        return gx

    def backward(self, a, gy, B, dims):
        """gy BF16 [B][V][16] (from sg_mse); accumulates every layer's gradients."""
        torch = _torch()
        mp = self.mp
        D, H, W = dims
        l0, l1, l2, l3 = (D, H, W), (D // 2, H // 2, W // 2), (D // 4, H // 4, W // 4), (D // 8, H // 8, W // 8)

        def relu_g(act, g):
            mp.sg_relu_grad(act, g, g.numel())
            return g

        def up_g(g, act, C, coarse):
            out = torch.empty((B, act.shape[1], C), dtype=torch.bfloat16, device=gy.device)
            mp.sg_up2_grad(g, out, B, *coarse, C)
            return out

        g = self._back("out", a["e0"], gy, B, l0)
        g = self._back("d0b", a["h0"], relu_g(a["e0"], g), B, l0)
        g_s0 = g.clone()
        g = self._back("d0a", a["u0"], relu_g(a["d0"], g), B, l0)
        g = self._back("d1b", a["h1"], relu_g(a["e1"], up_g(g, a["e1"], 64, l1)), B, l1)
        g_s1 = g.clone()
        g = self._back("d1a", a["u1"], relu_g(a["d1"], g), B, l1)
        g = self._back("d2b", a["h2"], relu_g(a["e2"], up_g(g, a["e2"], 96, l2)), B, l2)
        g_s2 = g.clone()
        g = self._back("d2a", a["u2"], relu_g(a["d2"], g), B, l2)
        g = self._back("b1", a["a3"], relu_g(a["c3"], up_g(g, a["c3"], 128, l3)), B, l3)
        g = self._back("b0", a["p2"], relu_g(a["a3"], g), B, l3)
        for lvl, gs, act_s, pin, C, fine in ((2, g_s2, "s2", "a2", 96, l2), (1, g_s1, "s1", "a1", 64, l1),
                                             (0, g_s0, "s0", "a0", 32, l0)):
            gp = torch.empty_like(gs)
            mp.sg_pool2_grad(g, gp, B, *fine, C)
            mp.sg_add(gs, gp, gs, gs.numel())
            names = {2: ("e2b", "e2a"), 1: ("e1b", "e1a"), 0: ("e0b", "e0a")}[lvl]
            below = {2: "p1", 1: "p0", 0: "x0"}[lvl]
            g = self._back(names[0], a[pin], relu_g(a[act_s], gs), B, fine)
            g = self._back(names[1], a[below], relu_g(a[pin], g), B, fine, need_input_grad=lvl > 0)

    def zero_grad(self):
        for t in self.p.values():
            t["gW"].zero_()
            t["gb"].zero_()

    def adam(self, lr, step, b1=0.9, b2=0.999, eps=1e-8):
        for t in self.p.values():
            self.mp.sg_adam(t["W"], t["gW"], t["mW"], t["vW"], t["W"].numel(), lr, b1, b2, eps, step,
                            t["Wf"], t["Wb"], t["cin"], t["cout"])
            self.mp.sg_adam(t["b"], t["gb"], t["mb"], t["vb"], t["b"].numel(), lr, b1, b2, eps, step)

    def state(self):
        out = {}
        for name, t in self.p.items():
            out[name + ".W"] = t["W"].cpu().numpy()
            out[name + ".b"] = t["b"].cpu().numpy()
        return out

    # ---------------------------------------------------------------------------------
    def predict(self, cls_dev, shape, force, u_out, rho_out=None):
        """Add the estimated steady flow for body force `force` to u_out (FP32 SoA [3][N],
        device) and, when given, the density deviation to rho_out (FP32 [N]), on the forced
        cluster only. cls_dev: device u8 node classes of mp_classify (shape (nz, ny, nx)).
        Each nonzero force component is one network pass with the box read along that axis;
        the estimate is linear in the force (Stokes regime)."""
        torch = _torch()
        nz, ny, nx = shape
        for axis, F in enumerate(force):
            if F == 0.0:
                continue
            P, Q, R = [(nx, ny, nz), (ny, nx, nz), (nz, nx, ny)][axis]
            if P % 8 or Q % 8 or R % 8:
                raise ValueError("the surrogate needs every box dimension to be a multiple of 8")
            x0 = torch.empty((1, P * Q * R, 16), dtype=torch.bfloat16, device=u_out.device)
            self.mp.sg_pack_input(cls_dev, x0, nx, ny, nz, axis)
            y, _ = self.forward(x0, 1, (R, Q, P))
            self.mp.sg_unpack_output(y, 16, cls_dev, u_out, rho_out, nx, ny, nz, axis, F * self.s_u, F * self.s_rho)
            del x0, y
        # raises if a bounded wait inside a tensor-core convolution gave up
        self.mp.sg_check(torch.cuda.current_stream(u_out.device))


def load(path=WEIGHTS):
    """The trained surrogate (weights file written by `train`)."""
    z = np.load(path, allow_pickle=False)
    meta = json.loads(str(z["meta"]))
    return Surrogate(params={k: z[k] for k in z.files if k != "meta"}, s_u=meta["s_u"], s_rho=meta["s_rho"]), meta


def warm_start(solid, force, model=None):
    """Estimated steady state for lb_steady's u_init and rho_init: (u FP32 SoA [3][N], rho
    FP32 [N]) device tensors; rho is 1 outside the forced cluster and has mean 1 on it."""
    torch = _torch()
    from . import mp
    model = model or load()[0]
    cls, _ = mp.mp_classify(solid)
    cls_dev = torch.as_tensor(cls).cuda()
    u = torch.zeros((3,) + tuple(solid.shape), dtype=torch.float32, device="cuda")
    rho = torch.ones(tuple(solid.shape), dtype=torch.float32, device="cuda")
    model.predict(cls_dev, solid.shape, force, u, rho)
    return u, rho


# -------------------------------------------------------------------------------------
def make_dataset(n, size, seed0, radii=(4, 8), porosity=(0.3, 0.6), log=print):
    """n seeded media of size^3 with their LB steady states (u, rho) under F_TRAIN along x
    (device tensors)."""
    torch = _torch()
    from . import mp
    rng = np.random.default_rng(seed0)
    xs, us, rhos, info = [], [], [], []
    t0 = time.time()
    for i in range(n):
        phi = float(rng.uniform(*porosity))
        R = int(rng.integers(radii[0], radii[1] + 1))
        solid, _ = media.random_spheres((size, size, size), R, phi, seed=seed0 + i)
        cls, (nf, _, ncl) = mp.mp_classify(solid)
        sd = torch.as_tensor(solid).cuda()
        u = torch.zeros((3, size, size, size), dtype=torch.float32, device="cuda")
        rho = torch.zeros((size, size, size), dtype=torch.float32, device="cuda")
        steps, res, conv = mp.lb_steady(sd, (F_TRAIN, 0.0, 0.0), u, tol=1e-7, max_steps=100_000, check_every=100,
                                        rho_out=rho)
        x0 = torch.empty((size ** 3, 16), dtype=torch.bfloat16, device="cuda")
        mp.sg_pack_input(torch.as_tensor(cls).cuda(), x0, size, size, size, 0)
        xs.append(x0)
        us.append(u)
        rhos.append(rho)
        info.append({"seed": seed0 + i, "porosity": phi, "radius": R, "lb_steps": int(steps),
                     "converged": bool(conv), "n_fluid": int(nf), "n_cluster": int(ncl)})
        if (i + 1) % 64 == 0:
            log(f"dataset {i + 1}/{n}, {time.time() - t0:.1f} s")
    return xs, us, rhos, info


def train(out, n_train=512, size=64, batch=4, iters=3000, lr=1e-3, seed=1000, n_val=16, val_seed=90_000, log=print,
          init=None):
    """Generates the dataset and trains; `init`: a weights file to start from (fine-tuning:
    its output scales are kept, so that its targets keep their meaning)."""
    torch = _torch()
    from . import mp
    xs, us, rhos, info = make_dataset(n_train, size, seed, log=log)
    xv, uv, rv, _ = make_dataset(n_val, size, val_seed, log=log)      # held-out media
    meta0 = None
    if init is not None:
        model, meta0 = load(init)
        s_u, s_rho = model.s_u, model.s_rho
    else:
        # output scales: RMS of u/F and of (rho - 1)/F over the forced fluid (targets O(1))
        su, sr, cnt = 0.0, 0.0, 0
        for x0, u, r in zip(xs, us, rhos):
            m = x0[:, 1].float().view(size, size, size) > 0.5
            su += float((u.pow(2).sum(0)[m]).sum()) / F_TRAIN ** 2
            sr += float(((r - 1.0).pow(2)[m]).sum()) / F_TRAIN ** 2
            cnt += int(m.sum())
        s_u = float(np.sqrt(su / (3 * cnt)))
        s_rho = float(np.sqrt(sr / cnt))

    def targets(flows, dens):
        out = []
        for u, r in zip(flows, dens):
            t = torch.empty((size ** 3, 4), dtype=torch.float32, device="cuda")
            mp.sg_pack_target(u, r, t, size, size, size, 0, 1.0 / (F_TRAIN * s_u), 1.0 / (F_TRAIN * s_rho))
            out.append(t)
        return out
    ts, tv = targets(us, rhos), targets(uv, rv)
    del us, uv, rhos, rv
    if init is None:
        model = Surrogate(seed=seed, s_u=s_u, s_rho=s_rho)
    rng = np.random.default_rng(seed + 1)
    V = size ** 3
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    gy = torch.empty((batch, V, 16), dtype=torch.bfloat16, device="cuda")
    hist, vhist = [], []
    gv = torch.empty((1, V, 16), dtype=torch.bfloat16, device="cuda")

    def val_loss():
        tot = 0.0
        for x, t in zip(xv, tv):
            xb1 = x.unsqueeze(0)
            y1, _ = model.forward(xb1, 1, (size, size, size))
            loss.zero_()
            mp.sg_mse(y1, 16, t.unsqueeze(0), 4, xb1, gv, loss, 1, V, float(x[:, 0].float().sum()))
            tot += float(loss.item())
        return tot / len(xv)
    t0 = time.time()
    for it in range(1, iters + 1):
        idx = rng.choice(n_train, size=batch, replace=False)
        xb = torch.stack([xs[i] for i in idx])
        tb = torch.stack([ts[i] for i in idx])
        nfl = float(xb[:, :, 0].float().sum())
        y, acts = model.forward(xb, batch, (size, size, size), keep=True)
        loss.zero_()
        mp.sg_mse(y, 16, tb, 4, xb, gy, loss, batch, V, nfl)
        model.zero_grad()
        model.backward(acts, gy, batch, (size, size, size))
        rate = lr * 0.5 * (1.0 + np.cos(np.pi * (it - 1) / iters))     # cosine decay
        model.adam(rate, it)
        if it % 50 == 0 or it == 1:
            hist.append((it, float(loss.item())))
            log(f"iter {it} loss {hist[-1][1]:.5f} ({time.time() - t0:.1f} s)")
        if it % 500 == 0 or it == iters:
            vhist.append((it, val_loss()))
            log(f"iter {it} held-out loss {vhist[-1][1]:.5f}")
    meta = {"s_u": s_u, "s_rho": s_rho, "size": size, "n_train": n_train, "batch": batch, "iters": iters, "lr": lr,
            "seed": seed, "force": F_TRAIN, "radii": [4, 8], "porosity": [0.3, 0.6], "lb_tol": 1e-7,
            "loss_history": hist, "val_history": vhist, "n_val": n_val, "val_seed": val_seed,
            "train_seconds": time.time() - t0, "n_params": model.n_params(),
            "dataset_lb_steps_mean": float(np.mean([d["lb_steps"] for d in info]))}
    if meta0 is not None:
        # the runs this one continues, oldest first
        meta["previous"] = meta0.get("previous", []) + [{k: v for k, v in meta0.items()
                                                          if k not in ("loss_history", "val_history", "previous")}]
    np.savez(out, meta=json.dumps(meta), **model.state())
    return model, meta


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train", help="generate the LB dataset and train the surrogate")
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--n-train", type=int, default=512)
    tr.add_argument("--size", type=int, default=64)
    tr.add_argument("--batch", type=int, default=4)
    tr.add_argument("--iters", type=int, default=3000)
    tr.add_argument("--lr", type=float, default=1e-3)
    tr.add_argument("--seed", type=int, default=1000)
    tr.add_argument("--init", default=None, help="weights file to fine-tune from (keeps its output scales)")
    args = ap.parse_args()
    from . import build
    build.build()
    if args.cmd == "train":
        _, meta = train(args.out, args.n_train, args.size, args.batch, args.iters, args.lr, args.seed,
                        log=lambda s: print(s, flush=True), init=args.init)
        print(json.dumps({k: v for k, v in meta.items() if k not in ("loss_history", "val_history")}))
        print("held-out loss", meta["val_history"])


if __name__ == "__main__":
    main()
