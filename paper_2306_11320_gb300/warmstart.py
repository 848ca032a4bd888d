"""Learned warm start for the steady heated microchannel (the paper has no network;
this is an addition to its method).

A 4-level BF16 U-Net (include/tpfnet.h kernels, paper_2306_11320_gb300.unet) maps
maps of the channel's parameters to its steady fields (phi, u_x, u_y, p, T), each
predicted as its (normalised) departure from the cold start: the flat-interface,
quiescent, conduction state the lattice would otherwise start from.  The lattice then
starts from the predicted fields and runs to the same steady-state residual.

Instances follow the heated two-layer microchannel of Sec. 4.1 at 512 x 128: wall
temperatures T_h + T_0 cos(2 pi k x / L) below and T_c above, layer-height ratio
h / H, conductivity ratio lambda_r.  Each instance is drawn from lambda_r ~ U[0.1, 10],
h / H ~ U[0.5, 2], k ~ U{1, 2, 3, 4} with a seeded generator.

Warm start (everything after the host-side parameter maps and cold-start fields runs
in the library's kernels): parameter maps -> bf16 NHWC input (tpfnet_pack) -> U-Net
forward -> de-normalised planes plus the cold start (tpfnet_unpack) -> phi
re-thresholded to the tanh profile about its predicted zero contour, shifted to the
cold start's sum of phi (tpflbm_project_phi) -> equilibrium populations (tpflbm_init;
tpflbm_init_forced, which takes half of the forcing sources off, is an option that
helped only from exact fields).
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
import time

import numpy as np

from . import workloads as WL

NX, NY = 512, 128
T_H, T_C, T_0 = 20.0, 10.0, 4.0
DT_SCALE = T_H - T_C              # temperature scale of the residual
# steps between residual evaluations; r is the mean change per step over that window,
# and its float32 noise floor falls as 1/K (5e-10 to 1.5e-8 at K = 1000 on these
# channels): at 4000 it stays below the 1e-8 tolerance for the weakest flows
RESID_K = 4000
OUT_FIELDS = ("phi", "ux", "uy", "p", "T")
C_IN = 4
CHANNELS = (32, 64, 128, 256)
INIT_FORCED = 0                   # warm start populations: plain equilibria (measured best)


# ------------------------------------------------------------------ instances

def sample_instances(n, seed):
    """n parameter draws (lambda_r, h/H, k) of the heated microchannel."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(dict(lam_r=float(rng.uniform(0.1, 10.0)), hr=float(rng.uniform(0.5, 2.0)),
                        k=int(rng.integers(1, 5))))
    return out


def channel(inst, nx=NX, ny=NY):
    """(params, cold-start fields, meta) of one instance."""
    return WL.microchannel(nx=nx, ny=ny, lam_r=inst["lam_r"], k=inst["k"],
                           h_frac=inst["hr"] / (1.0 + inst["hr"]), T_h=T_H, T_c=T_C, T_0=T_0)


def features(inst, nx=NX, ny=NY):
    """The network's input maps (C_IN, ny, nx) float32: the cold-start phase field,
    log10 of the local conductivity relative to the heavy layer's, the bottom-wall
    temperature modulation cos(2 pi k x / L) and the height coordinate in [-1, 1]."""
    _, f, _ = channel(inst, nx, ny)
    phi = f["phi"]
    lam = inst["lam_r"] + (1.0 - inst["lam_r"]) * 0.5 * (1.0 + np.clip(phi, -1, 1))
    x = np.arange(nx) + 0.0
    y = np.arange(ny) + 0.5
    mod = np.broadcast_to(np.cos(2 * math.pi * inst["k"] * x / nx)[None, :], (ny, nx))
    yc = np.broadcast_to((2.0 * y / ny - 1.0)[:, None], (ny, nx))
    return np.stack([phi, np.log10(lam), mod, yc]).astype(np.float32)


def cold_base(inst, nx=NX, ny=NY):
    """(5, ny, nx) float32 planes of the cold start in OUT_FIELDS order: the base the
    network's outputs are departures from."""
    _, f, _ = channel(inst, nx, ny)
    return np.stack([f[n] for n in OUT_FIELDS]).astype(np.float32)


def cold_mass(inst, nx=NX, ny=NY):
    """FP64 sum of phi of the cold start (conserved by the Allen-Cahn LBE)."""
    _, f, _ = channel(inst, nx, ny)
    return float(f["phi"].astype(np.float32).astype(np.float64).sum())


# ------------------------------------------------------------ normalisation

class Normalizer:
    """out_c = (field_c - cold_c - shift_c) / scale_c for the network's output
    channels (cold_c: the cold-start field)."""

    def __init__(self, scale, shift):
        self.scale = np.asarray(scale, dtype=np.float64)
        self.shift = np.asarray(shift, dtype=np.float64)

    @classmethod
    def fit(cls, fields, bases):
        """Mean and standard deviation of each field's departure from the cold start."""
        scale, shift = [], []
        for c, n in enumerate(OUT_FIELDS):
            v = np.stack([f[n].astype(np.float64) - b[c] for f, b in zip(fields, bases)])
            shift.append(float(v.mean()))
            scale.append(float(v.std()) or 1.0)
        return cls(scale, shift)

    def to_dict(self):
        return dict(scale=self.scale.tolist(), shift=self.shift.tolist())


# ------------------------------------------------------------ data generation

def generate(instances, max_steps, tol, batch_size=64, log=print):
    """Run cold starts of the instances to steady state with the batch engine.

    Returns (fields, steps): the fields at the end of the run (dict of float32
    arrays per instance) and, per instance, the first multiple of RESID_K steps at
    which max(r_u, r_T) < tol (None if never)."""
    from .tpflbm import Batch

    # a batch runs until its slowest member converges: group the instances by wall
    # wavenumber (the k = 1 channels take the longest), then restore the given order
    order = sorted(range(len(instances)), key=lambda j: (instances[j]["k"], instances[j]["lam_r"]))
    fields_o, steps_o = [None] * len(instances), [None] * len(instances)
    for s in range(0, len(order), batch_size):
        idx = order[s:s + batch_size]
        chunk = [instances[j] for j in idx]
        cases = [channel(i) for i in chunk]
        b = Batch([(NX, NY, p) for p, _, _ in cases])
        for k, (_, f, _) in enumerate(cases):
            b.init(k, **{n: v.astype(np.float32) for n, v in f.items()})
        b.tune(steps=10)
        b.residual(DT_SCALE)
        first = [None] * len(chunk)
        t0 = time.time()
        while b.t < max_steps and any(v is None for v in first):
            b.step(RESID_K)
            r = b.residual(DT_SCALE)
            rr = np.maximum(r[:, 0], r[:, 1])
            for k in range(len(chunk)):
                if first[k] is None and rr[k] < tol:
                    first[k] = b.t
        for k, j in enumerate(idx):
            fields_o[j] = b.fields(k)
            steps_o[j] = first[k]
        log("generated %d/%d (t = %d, %.1f s, converged %d)" % (s + len(chunk), len(instances), b.t,
                                                                 time.time() - t0, sum(v is not None for v in first)))
        b.close()
    return fields_o, steps_o


# ------------------------------------------------------------------ network

def _lib_ptr(t):
    return C.c_void_p(t.data_ptr())


def pack_inputs(net, maps):
    """(N, C_IN, ny, nx) float32 CUDA maps -> (N, ny, nx, 32) bf16 network input."""
    t = net.torch
    N, c, ny, nx = maps.shape
    x = t.zeros((N, ny, nx, net.cinp), dtype=t.bfloat16, device="cuda")
    s = C.c_void_p(net.stream.cuda_stream)
    for n in range(N):
        rc = net.lib.tpfnet_pack(_lib_ptr(maps[n]), None, ny * nx, c, ny * nx, None, None,
                                 C.c_void_p(x.data_ptr() + n * ny * nx * net.cinp * 2), net.cinp, 1, s)
        if rc != 0:
            raise RuntimeError("tpfnet_pack failed (%d)" % rc)
    return x


def pack_targets(net, fields, insts, norm):
    """list of field dicts -> (N, ny, nx, 5) float32 normalised targets (on the GPU)."""
    t = net.torch
    N = len(fields)
    y = t.empty((N, NY, NX, len(OUT_FIELDS)), dtype=t.float32, device="cuda")
    scale = (C.c_float * 5)(*[1.0 / v for v in norm.scale])
    shift = (C.c_float * 5)(*[-m / v for m, v in zip(norm.shift, norm.scale)])
    s = C.c_void_p(net.stream.cuda_stream)
    for n, (f, inst) in enumerate(zip(fields, insts)):
        planes = t.from_numpy(np.stack([f[k] for k in OUT_FIELDS]).astype(np.float32)).cuda()
        base = t.from_numpy(cold_base(inst)).cuda()
        rc = net.lib.tpfnet_pack(_lib_ptr(planes), _lib_ptr(base), NY * NX, 5, NY * NX, scale, shift,
                                 C.c_void_p(y.data_ptr() + n * NY * NX * 5 * 4), 5, 0, s)
        if rc != 0:
            raise RuntimeError("tpfnet_pack failed (%d)" % rc)
    return y


def make_net(seed=0, stream=None):
    from .unet import UNet

    return UNet(C_IN, len(OUT_FIELDS), CHANNELS, seed=seed, stream=stream)


def train(net, X, Y, epochs, batch=4, lr=1e-3, lr_final=1e-4, seed=0, max_seconds=None, log=print):
    """Adam on minibatches of (X, Y) (GPU tensors); cosine learning-rate decay over
    `epochs` (fewer when max_seconds runs out first).  Returns the per-epoch mean
    losses."""
    rng = np.random.default_rng(seed)
    N = X.shape[0]
    hist = []
    total = epochs * ((N + batch - 1) // batch)
    it = 0
    t0 = time.time()
    for ep in range(epochs):
        if max_seconds is not None and time.time() - t0 > max_seconds:
            log("training stopped by the time limit after %d epochs" % ep)
            break
        order = rng.permutation(N)
        losses = []
        for s in range(0, N - batch + 1, batch):
            idx = net.torch.from_numpy(order[s:s + batch]).cuda()
            prog = it / total
            if max_seconds:
                prog = max(prog, (time.time() - t0) / max_seconds)
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * min(prog, 1.0)))
            losses.append(net.train_step(X.index_select(0, idx), Y.index_select(0, idx), lr=a))
            it += 1
        hist.append(float(np.mean(losses)))
        if ep % 10 == 0 or ep == epochs - 1:
            log("epoch %d loss %.4e" % (ep, hist[-1]))
    return hist


def _bf16_bits(a):
    """float32 array -> uint16 bit patterns of its round-to-nearest-even bfloat16."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def _from_bf16_bits(b):
    return (b.astype(np.uint32) << 16).view(np.float32)


def save(path, net, norm, meta=None):
    """Store the network: the 3x3 weights as bfloat16 (the precision the convolutions
    use), the 1x1 head and every bias in float32, and the normaliser."""
    arrs = {}
    for k, v in net.state_dict().items():
        if k.endswith(".W") and not k.startswith("head"):
            arrs[k + ":bf16"] = _bf16_bits(v)
        else:
            arrs[k] = v
    arrs["__norm__"] = np.array(json.dumps(dict(norm.to_dict(), meta=meta or {})))
    np.savez_compressed(path, **arrs)


def load(path, stream=None):
    d = np.load(path, allow_pickle=False)
    info = json.loads(str(d["__norm__"]))
    net = make_net(stream=stream)
    state = {}
    for k in d.files:
        if k == "__norm__":
            continue
        state[k[:-5] if k.endswith(":bf16") else k] = _from_bf16_bits(d[k]) if k.endswith(":bf16") else d[k]
    net.load_state_dict(state)
    return net, Normalizer(info["scale"], info["shift"]), info.get("meta", {})


# ---------------------------------------------------------------- warm start

def predict(net, norm, insts):
    """Network prediction of the steady fields: (N, 5, ny, nx) float32 CUDA planes."""
    t = net.torch
    maps = t.from_numpy(np.stack([features(i) for i in insts])).cuda()
    base = t.from_numpy(np.stack([cold_base(i) for i in insts])).cuda()
    x = pack_inputs(net, maps)
    out = net.forward(x)
    N = len(insts)
    planes = t.empty((N, len(OUT_FIELDS), NY, NX), dtype=t.float32, device="cuda")
    scale = (C.c_float * 5)(*norm.scale)
    shift = (C.c_float * 5)(*norm.shift)
    s = C.c_void_p(net.stream.cuda_stream)
    for n in range(N):
        rc = net.lib.tpfnet_unpack(C.c_void_p(out.data_ptr() + n * NY * NX * 5 * 4), NY * NX, 5, scale, shift,
                                   _lib_ptr(base[n]), _lib_ptr(planes[n]), NY * NX, s)
        if rc != 0:
            raise RuntimeError("tpfnet_unpack failed (%d)" % rc)
    return planes


def warm_init(lat, net, norm, inst, forced=INIT_FORCED):
    """Initialise lattice `lat` from the network's prediction for `inst` (`forced`: the
    half-source selection of tpflbm_init_forced, 0 for plain equilibria)."""
    planes = predict(net, norm, [inst])[0]
    phi, got = lat.project_phi(planes[0], cold_mass(inst), mode=1)
    lat.init(phi=phi, ux=planes[1], uy=planes[2], p=planes[3], T=planes[4], forced=forced)
    return got


def time_to_steady(lat, tol, max_steps):
    """Step until max(r_u, r_T) < tol (checked every RESID_K steps).  Returns
    (steps or None, seconds from the call to convergence)."""
    torch = lat.torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.residual(DT_SCALE)
    while lat.t < max_steps:
        lat.step(RESID_K)
        ru, rT, _ = lat.residual(DT_SCALE)
        if max(ru, rT) < tol:
            return lat.t, time.perf_counter() - t0
    return None, time.perf_counter() - t0


def compare(net, norm, insts, tols=(1e-7, 1e-8), max_steps=800_000, log=print, forced=INIT_FORCED):
    """Cold versus warm start of each instance, on its own lattice and stream.
    Returns a list of dicts with steps and wall seconds to each tolerance."""
    import torch

    from .tpflbm import Lattice

    stream = torch.cuda.Stream()
    res = []
    for i, inst in enumerate(insts):
        p, f, _ = channel(inst)
        row = dict(inst)
        for mode in ("cold", "warm"):
            lat = Lattice(NX, NY, p, stream=stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                if mode == "cold":
                    lat.init(**{n: v.astype(np.float32) for n, v in f.items()})
                else:
                    net.stream = stream
                    warm_init(lat, net, norm, inst, forced)
            torch.cuda.synchronize()
            t_init = time.perf_counter() - t0
            row[mode + "_init_s"] = t_init
            # seconds from the start of the initialisation; a run that does not reach a
            # tolerance within max_steps records steps None and the seconds to max_steps
            elapsed = t_init
            for tol in sorted(tols, reverse=True):
                if lat.t < max_steps:
                    steps, sec = time_to_steady(lat, tol, max_steps)
                    elapsed += sec
                else:
                    steps = None
                row["%s_steps_%g" % (mode, tol)] = steps
                row["%s_s_%g" % (mode, tol)] = elapsed
            row[mode + "_final"] = lat.fields()
            lat.close()
        a, b = row["cold_final"], row["warm_final"]
        row["final_rel_l2"] = {n: float(np.linalg.norm(a[n].astype(np.float64) - b[n]) /
                                        max(np.linalg.norm(a[n].astype(np.float64)), 1e-300))
                               for n in ("phi", "ux", "uy", "T")}
        del row["cold_final"], row["warm_final"]
        log(json.dumps({k: v for k, v in row.items()}))
        res.append(row)
    return res


def summarize(rows, tols):
    """Speed-ups of the warm start.  Per instance: cold / warm time and steps where both
    converged.  Aggregate: total cold time / total warm time over all instances, a run
    that never converged counted at its time to max_steps (so the aggregate is a
    lower bound when the cold start is the one that did not converge)."""
    out = {}
    for tol in tols:
        key = "%g" % tol
        both = [r for r in rows if r.get("cold_steps_" + key) and r.get("warm_steps_" + key)]
        ratios = [r["cold_s_" + key] / r["warm_s_" + key] for r in both]
        sratios = [r["cold_steps_" + key] / r["warm_steps_" + key] for r in both]
        out["speedup_time_" + key] = dict(
            median=float(np.median(ratios)) if ratios else None,
            geomean=float(np.exp(np.mean(np.log(ratios)))) if ratios else None, n=len(ratios))
        out["speedup_steps_" + key] = dict(median=float(np.median(sratios)) if sratios else None, n=len(sratios))
        cold = sum(r["cold_s_" + key] for r in rows)
        warm = sum(r["warm_s_" + key] for r in rows)
        out["aggregate_" + key] = dict(
            cold_s=cold, warm_s=warm, ratio=cold / warm if warm > 0 else None,
            cold_unconverged=sum(r.get("cold_steps_" + key) is None for r in rows),
            warm_unconverged=sum(r.get("warm_steps_" + key) is None for r in rows))
    out["final_rel_l2_max"] = {n: max(r["final_rel_l2"][n] for r in rows) for n in ("phi", "ux", "uy", "T")}
    return out


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "warmstart_unet.npz")


def held_out(meta, n=None):
    """The held-out instances of a trained network (drawn with its training set)."""
    insts = sample_instances(meta["train"] + meta["test"], meta["seed"])[meta["train"]:]
    return insts if n is None else insts[:n]


# --------------------------------------------------------------------- driver

def main(argv=None):
    """Generate steady states, train the network, save it, and compare cold and warm
    starts on held-out instances.  Prints one JSON summary line at the end."""
    import argparse

    import torch

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=128)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--gen-steps", type=int, default=400_000)
    ap.add_argument("--gen-tol", type=float, default=1e-8)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--train-seconds", type=float, default=None)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--max-steps", type=int, default=800_000)
    ap.add_argument("--out", default=None, help="where to save the trained network (.npz)")
    ap.add_argument("--weights", default=None, help="skip generation and training: load this network")
    ap.add_argument("--json", default=None)
    ap.add_argument("--init-forced", type=int, default=INIT_FORCED,
                    help="warm start populations: 0 equilibria, 1/2/3 less half of the f/g/both sources")
    a = ap.parse_args(argv)

    def log(msg):
        print(msg, flush=True)

    insts = sample_instances(a.train + a.test, a.seed)
    train_i, test_i = insts[:a.train], insts[a.train:]
    summary = dict(train=a.train, test=a.test, seed=a.seed)
    if a.weights:
        net, norm, meta = load(a.weights)
        summary["weights"] = meta
    else:
        t0 = time.time()
        fields, steps = generate(train_i, a.gen_steps, a.gen_tol, log=log)
        summary["gen_seconds"] = time.time() - t0
        summary["gen_converged"] = int(sum(v is not None for v in steps))
        norm = Normalizer.fit(fields, [cold_base(i) for i in train_i])
        net = make_net(seed=a.seed)
        maps = torch.from_numpy(np.stack([features(i) for i in train_i])).cuda()
        X = pack_inputs(net, maps)
        Y = pack_targets(net, fields, train_i, norm)
        del maps
        t0 = time.time()
        hist = train(net, X, Y, a.epochs, batch=a.batch, lr=a.lr, seed=a.seed, max_seconds=a.train_seconds, log=log)
        torch.cuda.synchronize()
        summary["train_seconds"] = time.time() - t0
        summary["epochs"] = len(hist)
        summary["loss_first_last"] = [hist[0], hist[-1]]
        meta = dict(train=a.train, test=a.test, seed=a.seed, epochs=len(hist), gen_steps=a.gen_steps,
                    gen_tol=a.gen_tol, loss=hist[-1], channels=list(CHANNELS), c_in=C_IN, out=list(OUT_FIELDS))
        if a.out:
            save(a.out, net, norm, meta)
        del X, Y
    res = compare(net, norm, test_i, max_steps=a.max_steps, log=log, forced=a.init_forced)
    summary["init_forced"] = a.init_forced
    summary.update(summarize(res, (1e-7, 1e-8)))
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(dict(summary=summary, rows=res), fh, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
