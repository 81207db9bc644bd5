"""Train the BF16 MLP surrogate of the chemistry step on the GPU.

Data: states sampled from the quasi-DNS state distribution (synth.states.flamelet_samples),
advanced over dt by the FP64 GPU integrator (chem_advance); features and targets
(chem_train_features), statistics (chem_column_stats) and normalisation (chem_train_normalize)
run in libchem kernels; the network is trained by chem_mlp_forward / chem_mlp_backward /
chem_mlp_adam_step (tcgen05 GEMMs).  torch only holds device buffers, shuffles indices and
gathers batches.

    python -m paper_2312_13513_gb300.train --out model.chemsur --states 4194304 --epochs 40
    python -m torch.distributed.run --nproc-per-node N -m paper_2312_13513_gb300.train --out ...
        (data-parallel: each rank takes 1/N of every global batch, one NCCL all-reduce of the
        gradients per step; --checkpoint / --resume save and continue the trainer state; --graph
        replays one captured step per batch on a single GPU)
"""
from __future__ import annotations

import argparse
import ctypes
import os
import struct
import time

import numpy as np

from . import Mechanism, _lib, _ptr, _stream_ptr, advance, check

PAD = 128


class Trainer:
    """chem_mlp_trainer_*: n_in -> hidden... -> n_out GELU network with Adam (hidden defaults to the
    single network's 512 x 4; the per-species networks use 1600, 800, 400)."""

    def __init__(self, n_in, n_out, batch, W=None, b=None, seed=0, hidden=(512, 512, 512, 512)):
        L = _lib.load()
        self.n_in, self.n_out, self.batch = n_in, n_out, batch
        self.hidden = [int(h) for h in hidden]
        nl = len(self.hidden) + 1
        hid = (ctypes.c_int * len(self.hidden))(*self.hidden)
        h = ctypes.c_void_p()
        if W is not None:
            self._w = [np.ascontiguousarray(w, np.float32) for w in W]
            self._b = [np.ascontiguousarray(x, np.float32) for x in b]
            Wp = (ctypes.c_void_p * nl)(*[w.ctypes.data for w in self._w])
            bp = (ctypes.c_void_p * nl)(*[x.ctypes.data for x in self._b])
            check(L.chem_mlp_trainer_create_layers(n_in, n_out, len(self.hidden), hid, batch, Wp, bp, seed,
                                                   ctypes.byref(h)))
        else:
            check(L.chem_mlp_trainer_create_layers(n_in, n_out, len(self.hidden), hid, batch, None, None, seed,
                                                   ctypes.byref(h)))
        self.handle = h

    def forward(self, X, out=None, stream=None):
        # the backward pass reads X again (weight gradient of the first layer): keep it alive
        self._x = X
        check(_lib.load().chem_mlp_forward(self.handle, _ptr(X), _ptr(out), _stream_ptr(stream)))

    def backward(self, target, loss=None, stream=None):
        check(_lib.load().chem_mlp_backward(self.handle, _ptr(target), _ptr(loss), _stream_ptr(stream)))

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        check(_lib.load().chem_mlp_adam_step(self.handle, ctypes.c_float(lr), ctypes.c_float(beta1),
                                             ctypes.c_float(beta2), ctypes.c_float(eps),
                                             _stream_ptr(stream)))

    def adam_dev(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """Adam with the learning rate read from the one-element FP32 device tensor lr when the
        update runs (chem_mlp_adam_step_dev: capturable in a CUDA graph)."""
        check(_lib.load().chem_mlp_adam_step_dev(self.handle, _ptr(lr), ctypes.c_float(beta1),
                                                 ctypes.c_float(beta2), ctypes.c_float(eps),
                                                 _stream_ptr(stream)))

    @property
    def step(self):
        """Adam steps taken (restored by load)."""
        v = ctypes.c_int64(0)
        check(_lib.load().chem_mlp_trainer_step(self.handle, ctypes.byref(v)))
        return int(v.value)

    def save(self, path):
        """Checkpoint: master weights, Adam moments and step counter (chem_mlp_trainer_save)."""
        check(_lib.load().chem_mlp_trainer_save(self.handle, os.fsencode(path)))

    def load(self, path):
        """Resume from a checkpoint of a network of the same shape (chem_mlp_trainer_load)."""
        check(_lib.load().chem_mlp_trainer_load(self.handle, os.fsencode(path)))

    def grad_count(self):
        v = ctypes.c_int64(0)
        check(_lib.load().chem_mlp_grad_count(self.handle, ctypes.byref(v)))
        return int(v.value)

    def pack_grads(self, flat, stream=None):
        """The last gradients into a flat FP32 device tensor (layout of parallel.flatten_grads)."""
        check(_lib.load().chem_mlp_grad_pack(self.handle, _ptr(flat), _stream_ptr(stream)))

    def unpack_grads(self, flat, scale=1.0, stream=None):
        """scale * flat becomes the gradient of the next Adam step."""
        check(_lib.load().chem_mlp_grad_unpack(self.handle, _ptr(flat), ctypes.c_float(scale),
                                               _stream_ptr(stream)))

    def allreduce_grads(self, group=None, stream=None):
        """Data-parallel step: the mean over the ranks of their gradients, in place (pack, one
        all-reduce of the flat buffer, unpack scaled by 1 / ranks)."""
        import torch
        from .parallel import allreduce_sum_
        if getattr(self, "_flat", None) is None:
            self._flat = torch.empty(self.grad_count(), dtype=torch.float32, device="cuda")
        self.pack_grads(self._flat, stream)
        world = allreduce_sum_(self._flat, group)
        if world > 1:
            self.unpack_grads(self._flat, 1.0 / world, stream)
        return world

    def get(self, which=0):
        dims = [self.n_in] + self.hidden + [self.n_out]
        nl = len(dims) - 1
        W = [np.zeros((dims[i + 1], dims[i]), np.float32) for i in range(nl)]
        b = [np.zeros(dims[i + 1], np.float32) for i in range(nl)]
        Wp = (ctypes.c_void_p * nl)(*[w.ctypes.data for w in W])
        bp = (ctypes.c_void_p * nl)(*[x.ctypes.data for x in b])
        check(_lib.load().chem_mlp_trainer_get(self.handle, which, Wp, bp))
        return W, b

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().chem_mlp_trainer_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def column_stats(A):
    """mean, std, min, max per column of a [n x c] FP32 device tensor (chem_column_stats)."""
    import torch
    n, c = A.shape
    st = torch.zeros(4 * c, dtype=torch.float64, device=A.device)
    check(_lib.load().chem_column_stats(_ptr(A), n, c, _ptr(st), _stream_ptr(None)))
    s = st.cpu().numpy().reshape(4, c)
    mean = s[0] / n
    var = np.maximum(s[1] / n - mean * mean, 0.0)
    return mean, np.sqrt(var), s[2], s[3]


def make_dataset(mech, dm, n, dt, seed, rtol=1e-6, atol=1e-10, stats=None, front_fraction=0.5):
    """States (flamelet samples) advanced by the GPU integrator -> normalised X, target.

    X rows are the compensated split [x_hi | x_lo | x_hi | 0] of the z-scored features.  A species
    whose increment is zero in every sample (an inert one) gets y_std = 0 in the stats: the
    model then leaves it unchanged, and its training target is the constant 0."""
    import torch
    from synth.states import flamelet_samples, load_table
    f = flamelet_samples(load_table("h2_flamelet.npz"), n, seed, front_fraction=front_fraction)
    dev = torch.device("cuda")
    T0 = torch.tensor(f["T"], device=dev)
    p = torch.tensor(f["p"], device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(f["Y"]), device=dev)
    T1, Y1 = T0.clone(), Y0.clone()
    advance(dm, T1, p, Y1, dt, rtol, atol)
    ns = mech.ns
    nin = ns + 2
    x = torch.empty((n, nin), dtype=torch.float32, device=dev)
    t = torch.empty((n, ns), dtype=torch.float32, device=dev)
    check(_lib.load().chem_train_features(_ptr(T0), _ptr(p), _ptr(Y0), _ptr(Y1), n, n, ns, _ptr(x),
                                          _ptr(t), _stream_ptr(None)))
    if stats is None:
        xm, xs, xlo, xhi = column_stats(x)
        tm, ts, tlo, thi = column_stats(t)
        # a constant feature (ln p at fixed pressure) has a rounding-noise deviation: scale 1
        xs = np.where(xs > 1e-6 * np.maximum(1.0, np.abs(xm)), xs, 1.0)
        inert = (tlo == 0.0) & (thi == 0.0)
        ts = np.where(inert, 0.0, np.where(ts > 1e-12, ts, 1.0))
        stats = {"x_mean": xm, "x_std": xs, "y_mean": np.where(inert, 0.0, tm), "y_std": ts,
                 "box_lo": xlo, "box_hi": xhi}
    X = torch.empty((n, PAD), dtype=torch.bfloat16, device=dev)
    Tn = torch.empty((n, ns), dtype=torch.float32, device=dev)
    f32 = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev)
    # an inert species' target is 0: normalise it with scale 1
    sx, sxs, sy = f32(stats["x_mean"]), f32(stats["x_std"]), f32(stats["y_mean"])
    sys_ = f32(np.where(np.asarray(stats["y_std"]) > 0.0, stats["y_std"], 1.0))
    check(_lib.load().chem_train_normalize(_ptr(x), n, nin, _ptr(sx), _ptr(sxs), _ptr(X), PAD, _ptr(t), ns,
                                           _ptr(sy), _ptr(sys_), _ptr(Tn), _stream_ptr(None)))
    torch.cuda.synchronize()
    return {"X": X, "T": Tn, "stats": stats, "state0": (T0, p, Y0), "state1": (T1, Y1)}


def epoch_order(n, seed, epoch):
    """The sample order of one epoch, a function of (seed, epoch) alone: a resumed or a
    data-parallel run visits the same batches as one uninterrupted single-rank run."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed) * 1000003 + int(epoch))
    return torch.randperm(n, device="cuda", generator=g)


def cosine_lr(step, total, lr, lr_final):
    """Cosine learning-rate decay from lr to lr_final over total steps."""
    frac = step / max(1, total - 1)
    return lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * frac))


def train(mech, n_states=1 << 22, epochs=40, batch=4096, lr=3e-4, lr_final=1e-5, dt=5e-7, seed=7,
          log=print, time_budget_s=None, front_fraction=0.5, data=None, checkpoint=None, resume=None,
          group=None, max_steps=None, graph=False):
    """Train the single 4 x 512 network.  checkpoint: a file rewritten at the end of every epoch
    (and at max_steps) with the trainer state; resume: such a file to continue from (its Adam step
    counter gives the epoch and batch to continue at).  group: a torch.distributed process group
    for data-parallel training -- every rank builds the same data set, takes its equal share of
    each global batch and averages the gradients with one all-reduce before Adam; the statistics
    are rank 0's.  max_steps: stop after that many steps in total (for tests).  graph: on one rank,
    capture the step (batch gather, forward, backward, Adam with the rate from a device buffer)
    once in a CUDA graph and replay it per batch; the results are bitwise those of the direct
    calls, without the per-kernel launch cost."""
    import torch
    rank, world = 0, 1
    if group is not None or (torch.distributed.is_available() and torch.distributed.is_initialized()):
        import torch.distributed as dist
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    dm = Mechanism(mech)
    t0 = time.time()
    if data is None and world == 1:
        data = make_dataset(mech, dm, n_states, dt, seed, front_fraction=front_fraction)
    elif data is None:
        # every rank builds the same states; the normalisation statistics are rank 0's
        import torch.distributed as dist
        box = [None]
        if rank == 0:
            data = make_dataset(mech, dm, n_states, dt, seed, front_fraction=front_fraction)
            box = [data["stats"]]
        dist.broadcast_object_list(box, src=0, group=group)
        if rank != 0:
            data = make_dataset(mech, dm, n_states, dt, seed, stats=box[0], front_fraction=front_fraction)
    log(f"dataset: {data['X'].shape[0]} states in {time.time() - t0:.1f} s")
    ns = mech.ns
    if batch % (128 * world):
        raise ValueError(f"global batch {batch} must split into {world} shares of a multiple of 128")
    tr = Trainer(ns + 2, ns, batch // world, seed=seed)
    if resume is not None:
        tr.load(resume)
    X, Tt = data["X"], data["T"]
    n = X.shape[0]
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    if max_steps is not None:
        total_run = min(total, int(max_steps))
    else:
        total_run = total
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    history = []
    step = tr.step
    t1 = time.time()
    from .parallel import batch_share
    replay = None
    if graph and world == 1 and step < total_run:
        replay = _captured_step(tr, X, Tt, batch, loss)
    while step < total_run:
        ep, i0 = divmod(step, steps_per_epoch)
        perm = epoch_order(n, seed, ep)
        acc = 0.0
        for i in range(i0, steps_per_epoch):
            idx = batch_share(perm[i * batch:(i + 1) * batch], rank, world)
            if replay is not None:
                replay(idx, cosine_lr(step, total, lr, lr_final))
            else:
                xb = X.index_select(0, idx)
                yb = Tt.index_select(0, idx)
                tr.forward(xb)
                tr.backward(yb, loss)
                if world > 1:
                    tr.allreduce_grads(group)
                tr.adam(cosine_lr(step, total, lr, lr_final))
            step += 1
            if i % 64 == 0:
                acc = float(loss.item())
            if step >= total_run:
                break
        history.append(acc)
        if checkpoint is not None and rank == 0:
            tr.save(checkpoint)
        log(f"epoch {ep + 1}/{epochs}: loss {acc:.4e}  ({time.time() - t1:.1f} s)")
        if time_budget_s is not None and time.time() - t1 > time_budget_s:
            log("time budget reached")
            break
    W, b = tr.get(0)
    params = dict(data["stats"])
    params.update({"W": W, "b": b, "dt": dt, "history": history, "steps": step})
    return params


def _captured_step(tr, X, Tt, batch, loss):
    """One training step captured in a CUDA graph: gather the batch rows named by a static index
    buffer, forward, backward, Adam with the rate from a static device buffer.  Returns
    replay(idx, lr), which writes idx and lr into the buffers and replays the graph on the current
    stream.  The capture runs nothing: the trainer's state is untouched until the first replay."""
    import torch
    idx_buf = torch.zeros(batch, dtype=torch.int64, device="cuda")
    lr_buf = torch.zeros(1, dtype=torch.float32, device="cuda")
    xb = torch.empty((batch, X.shape[1]), dtype=X.dtype, device="cuda")
    yb = torch.empty((batch, Tt.shape[1]), dtype=Tt.dtype, device="cuda")
    # one direct forward + backward first (it writes activations and gradients only, which the
    # first replay overwrites): the kernels' one-time host set-up then happens outside the capture
    torch.index_select(X, 0, idx_buf, out=xb)
    torch.index_select(Tt, 0, idx_buf, out=yb)
    tr.forward(xb)
    tr.backward(yb, loss)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        s = torch.cuda.current_stream()
        torch.index_select(X, 0, idx_buf, out=xb)
        torch.index_select(Tt, 0, idx_buf, out=yb)
        tr.forward(xb, stream=s)
        tr.backward(yb, loss, stream=s)
        tr.adam_dev(lr_buf, stream=s)

    def replay(idx, lr):
        idx_buf.copy_(idx, non_blocking=True)
        lr_buf.fill_(float(lr))
        g.replay()

    replay.graph = g
    return replay


PER_SPECIES_HIDDEN = (1600, 800, 400)


def networked_species(y_std):
    """Species that get a network of their own (§2: none for inert species).  The training
    statistics give y_std = 0 exactly to a species whose increment over dt is zero in every state,
    which is what an inert species (one that no reaction produces or consumes) shows."""
    return [k for k in range(len(y_std)) if float(y_std[k]) > 0.0]


def train_per_species(mech, n_states=1 << 21, epochs=20, batch=4096, lr=3e-4, lr_final=1e-5, dt=5e-7,
                      seed=7, log=print, time_budget_s=None, front_fraction=0.5, hidden=PER_SPECIES_HIDDEN,
                      data=None):
    """The paper's per-species variant (§2): one n_in -> 1600 -> 800 -> 400 -> 1 GELU network per
    species with a nonzero increment (inert species get none), each trained on its own column of
    the same normalised targets, on the same data, features and statistics as the single network.
    The networks train in lockstep (one Adam step of each per batch)."""
    import torch
    dm = Mechanism(mech)
    t0 = time.time()
    if data is None:
        data = make_dataset(mech, dm, n_states, dt, seed, front_fraction=front_fraction)
    log(f"dataset: {data['X'].shape[0]} states in {time.time() - t0:.1f} s")
    ns = mech.ns
    species = networked_species(data["stats"]["y_std"])
    trainers = {k: Trainer(ns + 2, 1, batch, seed=seed + 17 * k, hidden=hidden) for k in species}
    X, Tt = data["X"], data["T"]
    n = X.shape[0]
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    loss = {k: torch.zeros(1, dtype=torch.float64, device="cuda") for k in species}
    history = []
    step = 0
    t1 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda")
        acc = 0.0
        for i in range(steps_per_epoch):
            idx = perm[i * batch:(i + 1) * batch]
            xb = X.index_select(0, idx)
            yb = Tt.index_select(0, idx)
            frac = step / max(1, total - 1)
            lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * frac))
            for k in species:
                tr = trainers[k]
                tr.forward(xb)
                tr.backward(yb[:, k].contiguous(), loss[k])
                tr.adam(lr_t)
            step += 1
            if i % 64 == 0:
                acc = float(sum(float(loss[k].item()) for k in species) / len(species))
        history.append(acc)
        log(f"epoch {ep + 1}/{epochs}: mean loss over {len(species)} networks {acc:.4e}  "
            f"({time.time() - t1:.1f} s)")
        if time_budget_s is not None and time.time() - t1 > time_budget_s:
            log("time budget reached")
            break
    params = dict(data["stats"])
    params.update({"hidden": list(hidden), "dt": dt, "history": history, "nets": {}})
    for k in species:
        W, b = trainers[k].get(0)
        params["nets"][k] = {"W": W, "b": b}
        trainers[k].close()
    return params


def save_model_per_species(params, path):
    """CHEMSUR2 file: magic, int32 ns, int32 h1, h2, h3, float64 dt, int32 nnet, int32 species[nnet],
    then float32 W1, b1, W2, b2, W3, b3, W4, b4 of each network and the statistics."""
    ns = len(params["y_std"])
    species = sorted(int(k) for k in params["nets"])
    with open(path, "wb") as f:
        f.write(b"CHEMSUR2")
        f.write(struct.pack("<iiiidi", ns, *[int(h) for h in params["hidden"]], float(params["dt"]), len(species)))
        f.write(np.asarray(species, np.int32).tobytes())
        for k in species:
            net = params["nets"][k]
            for l in range(4):
                f.write(np.ascontiguousarray(net["W"][l], np.float32).tobytes())
                f.write(np.ascontiguousarray(net["b"][l], np.float32).tobytes())
        for key in ("x_mean", "x_std", "y_mean", "y_std", "box_lo", "box_hi"):
            f.write(np.ascontiguousarray(params[key], np.float32).tobytes())


def save_model(params, path):
    """CHEMSUR1 file: magic, int32 ns, int32 hidden, float64 dt, then float32 arrays."""
    W, b = params["W"], params["b"]
    ns = W[4].shape[0]
    with open(path, "wb") as f:
        f.write(b"CHEMSUR1")
        f.write(struct.pack("<iid", ns, W[0].shape[0], float(params["dt"])))
        for l in range(5):
            f.write(np.ascontiguousarray(W[l], np.float32).tobytes())
            f.write(np.ascontiguousarray(b[l], np.float32).tobytes())
        for k in ("x_mean", "x_std", "y_mean", "y_std", "box_lo", "box_hi"):
            f.write(np.ascontiguousarray(params[k], np.float32).tobytes())


def load_model_params(path):
    with open(path, "rb") as f:
        raw = f.read()
    assert raw[:8] == b"CHEMSUR1"
    ns, hid, dt = struct.unpack("<iid", raw[8:24])
    nin = ns + 2
    off = 24

    def take(count, shape):
        nonlocal off
        a = np.frombuffer(raw, np.float32, count, off).reshape(shape).copy()
        off += 4 * count
        return a

    dims = [nin, hid, hid, hid, hid, ns]
    W, b = [], []
    for l in range(5):
        W.append(take(dims[l + 1] * dims[l], (dims[l + 1], dims[l])))
        b.append(take(dims[l + 1], (dims[l + 1],)))
    out = {"W": W, "b": b, "dt": dt}
    for k, c in (("x_mean", nin), ("x_std", nin), ("y_mean", ns), ("y_std", ns), ("box_lo", nin),
                 ("box_hi", nin)):
        out[k] = take(c, (c,))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--states", type=int, default=1 << 22)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--lr-final", type=float, default=1e-5)
    ap.add_argument("--front-fraction", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--budget", type=float, default=None, help="training time budget (s)")
    ap.add_argument("--log", default=None, help="also write the training log to this file")
    ap.add_argument("--checkpoint", default=None, help="trainer state file rewritten every epoch")
    ap.add_argument("--resume", default=None, help="continue from this trainer state file")
    ap.add_argument("--graph", action="store_true",
                    help="replay one captured CUDA graph per batch (one GPU; bitwise the direct steps)")
    args = ap.parse_args()
    from synth.mechanism import h2_mechanism
    import torch
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        # data-parallel training, one process per GPU (torchrun): NCCL all-reduce of the gradients
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lines = []

    def log(msg):
        if rank == 0:
            print(msg, flush=True)
            lines.append(msg)

    log(f"train: states {args.states} epochs {args.epochs} batch {args.batch} lr {args.lr} -> "
        f"{args.lr_final} (cosine) front_fraction {args.front_fraction} seed {args.seed}")
    params = train(h2_mechanism(), args.states, args.epochs, args.batch, args.lr, args.lr_final,
                   seed=args.seed, log=log, time_budget_s=args.budget,
                   front_fraction=args.front_fraction, checkpoint=args.checkpoint, resume=args.resume,
                   graph=args.graph)
    if rank == 0:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        save_model(params, args.out)
        log(f"saved {args.out}")
        if args.log:
            with open(args.log, "w") as f:
                f.write("\n".join(lines) + "\n")
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
