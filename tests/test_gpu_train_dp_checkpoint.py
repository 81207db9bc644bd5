"""GPU tests of data-parallel training and of checkpoint / resume (training with Adam, §2).

* The library's flat gradient layout is the one parallel.flatten_grads defines.
* Two trainers standing for two ranks, each on half of a global batch, whose gradients are
  summed (the all-reduce) and scaled by 1/2, take the step a single trainer takes on the whole
  batch, and stay identical to each other.
* A run checkpointed after some steps and resumed in a fresh trainer continues bitwise like the
  uninterrupted run, through the C ABI and through train()'s epoch bookkeeping.
"""
import filecmp

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp  # noqa: E402
from paper_2312_13513_gb300 import parallel  # noqa: E402

pytestmark = pytest.mark.gpu


def _problem(seed, B, nin=11, nout=9):
    rng = np.random.default_rng(seed)
    dims = [nin, 512, 512, 512, 512, nout]
    W = [np.float32(rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i])) for i in range(5)]
    b = [np.float32(0.1 * rng.standard_normal(dims[i + 1])) for i in range(5)]
    X = omlp.bf16_round(rng.standard_normal((B, nin)))
    T = rng.standard_normal((B, nout))
    return W, b, X, T


def _dev(X, T):
    from paper_2312_13513_gb300.train import PAD
    Xd = torch.zeros((X.shape[0], PAD), dtype=torch.bfloat16, device="cuda")
    Xd[:, :X.shape[1]] = torch.tensor(X, dtype=torch.float32).to(torch.bfloat16)
    return Xd, torch.tensor(T, dtype=torch.float32, device="cuda")


def test_pack_layout_is_the_flat_layout():
    from paper_2312_13513_gb300.train import Trainer
    W, b, X, T = _problem(1, 256)
    tr = Trainer(11, 9, 256, W=W, b=b)
    Xd, Td = _dev(X, T)
    tr.forward(Xd)
    tr.backward(Td)
    flat = torch.empty(tr.grad_count(), dtype=torch.float32, device="cuda")
    tr.pack_grads(flat)
    dW, db = tr.get(1)
    assert tr.grad_count() == (11 * 512 + 3 * 512 * 512 + 512 * 9) + (4 * 512 + 9)
    assert np.array_equal(flat.cpu().numpy(), parallel.flatten_grads(dW, db))
    # unpack with a scale writes scale * flat back as the gradients
    tr.unpack_grads(flat, 0.25)
    dW2, db2 = tr.get(1)
    assert all(np.array_equal(a, np.float32(0.25) * c) for a, c in zip(dW2 + db2, dW + db))


def test_two_ranks_on_half_batches_take_the_single_rank_step(tmp_path):
    """Each step starts the single trainer from the ranks' state (a checkpoint of rank a), so each
    step's comparison sees the same weights and moments on both sides."""
    from paper_2312_13513_gb300.train import Trainer
    W, b, X, T = _problem(2, 512)
    ra = Trainer(11, 9, 256, W=W, b=b)
    rb = Trainer(11, 9, 256, W=W, b=b)
    one = Trainer(11, 9, 512, W=W, b=b)
    lr = 1e-3
    for step in range(3):
        Xs = X if step == 0 else omlp.bf16_round(np.random.default_rng(10 + step).standard_normal(X.shape))
        Xd, Td = _dev(Xs, T)
        ra.forward(Xd[:256]); ra.backward(Td[:256])
        rb.forward(Xd[256:]); rb.backward(Td[256:])
        fa = torch.empty(ra.grad_count(), dtype=torch.float32, device="cuda")
        fb = torch.empty_like(fa)
        ra.pack_grads(fa); rb.pack_grads(fb)
        s = fa + fb                          # what the all-reduce (sum) delivers to both ranks
        ra.unpack_grads(s, 0.5); rb.unpack_grads(s, 0.5)
        one.forward(Xd); one.backward(Td)
        gA = parallel.flatten_grads(*ra.get(1)).astype(np.float64)
        g1 = parallel.flatten_grads(*one.get(1)).astype(np.float64)
        # the mean of the two halves' means is the mean over the batch, up to FP32 summation order
        assert np.max(np.abs(gA - g1)) <= 1e-5 * np.max(np.abs(g1)), step
        ra.adam(lr); rb.adam(lr); one.adam(lr)
        wA = parallel.flatten_grads(*ra.get(0))
        wB = parallel.flatten_grads(*rb.get(0))
        w1 = parallel.flatten_grads(*one.get(0)).astype(np.float64)
        assert np.array_equal(wA, wB), step              # the replicas stay identical
        # Adam divides by |g|: where g sits at rounding level its update can differ by up to lr;
        # elsewhere the two steps agree to FP32 rounding
        big = np.abs(g1) > 1e-3 * np.max(np.abs(g1))
        assert np.max(np.abs(wA.astype(np.float64) - w1)[big]) <= 1e-6, step
        assert np.max(np.abs(wA.astype(np.float64) - w1)) <= 2.0 * lr, step
        ck = str(tmp_path / f"ranks_after_{step}.chemtrn")
        ra.save(ck)
        one.load(ck)


def test_checkpoint_resume_is_bitwise_the_uninterrupted_run(tmp_path):
    from paper_2312_13513_gb300.train import Trainer
    W, b, X, T = _problem(3, 2048)
    Xd, Td = _dev(X, T)
    batches = [(Xd[i * 256:(i + 1) * 256], Td[i * 256:(i + 1) * 256]) for i in range(8)]
    lrs = [1e-3 * (0.9 ** k) for k in range(8)]

    def run(tr, ks):
        for k in ks:
            tr.forward(batches[k][0]); tr.backward(batches[k][1]); tr.adam(lrs[k])

    full = Trainer(11, 9, 256, W=W, b=b)
    run(full, range(8))
    first = Trainer(11, 9, 256, W=W, b=b)
    run(first, range(5))
    ck = str(tmp_path / "after5.chemtrn")
    first.save(ck)
    resumed = Trainer(11, 9, 256, seed=99)       # other initial weights: the file overrides them
    resumed.load(ck)
    assert resumed.step == 5
    run(resumed, range(5, 8))
    a, c = str(tmp_path / "full.chemtrn"), str(tmp_path / "resumed.chemtrn")
    full.save(a); resumed.save(c)
    assert resumed.step == full.step == 8
    assert filecmp.cmp(a, c, shallow=False)     # weights, both moments and the step, bitwise
    # a file of another shape is refused and leaves the trainer as it was
    other = Trainer(11, 8, 256, seed=1)
    from paper_2312_13513_gb300 import ChemError
    with pytest.raises(ChemError):
        other.load(ck)
    assert other.step == 0


def test_train_resume_continues_the_epoch_schedule(tmp_path, h2):
    """train(): stop after 5 steps with a checkpoint, resume to 12 steps; the same weights as 12
    uninterrupted steps (per-epoch sample order and learning rate follow from the step count)."""
    from paper_2312_13513_gb300 import Mechanism
    from paper_2312_13513_gb300 import train as trn
    dm = Mechanism(h2)
    data = trn.make_dataset(h2, dm, 4096, 5e-7, seed=3)
    quiet = lambda *a: None
    ref = trn.train(h2, epochs=3, batch=512, data=data, seed=3, log=quiet, max_steps=12)
    ck = str(tmp_path / "ck.chemtrn")
    part = trn.train(h2, epochs=3, batch=512, data=data, seed=3, log=quiet, max_steps=5, checkpoint=ck)
    assert part["steps"] == 5
    rest = trn.train(h2, epochs=3, batch=512, data=data, seed=3, log=quiet, max_steps=12, resume=ck)
    assert rest["steps"] == 12 == ref["steps"]
    for x, y in zip(rest["W"] + rest["b"], ref["W"] + ref["b"]):
        assert np.array_equal(x, y)


def test_captured_training_step_is_bitwise_the_direct_step(tmp_path, h2):
    """train(graph=True) replays one captured step (gather, forward, backward, Adam with the rate
    and the step counter in device memory): the same weights as the direct calls, bitwise, also
    when it resumes a run that the direct path checkpointed."""
    from paper_2312_13513_gb300 import Mechanism
    from paper_2312_13513_gb300 import train as trn
    dm = Mechanism(h2)
    data = trn.make_dataset(h2, dm, 4096, 5e-7, seed=4)
    quiet = lambda *a: None
    ref = trn.train(h2, epochs=3, batch=512, data=data, seed=4, log=quiet, max_steps=20)
    cap = trn.train(h2, epochs=3, batch=512, data=data, seed=4, log=quiet, max_steps=20, graph=True)
    assert cap["steps"] == ref["steps"] == 20
    for x, y in zip(cap["W"] + cap["b"], ref["W"] + ref["b"]):
        assert np.array_equal(x, y)
    ck = str(tmp_path / "ck.chemtrn")
    trn.train(h2, epochs=3, batch=512, data=data, seed=4, log=quiet, max_steps=7, checkpoint=ck)
    rest = trn.train(h2, epochs=3, batch=512, data=data, seed=4, log=quiet, max_steps=20, resume=ck, graph=True)
    assert rest["steps"] == 20
    for x, y in zip(rest["W"] + rest["b"], ref["W"] + ref["b"]):
        assert np.array_equal(x, y)
