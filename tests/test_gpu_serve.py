"""Serving loop and batched advances on the GPU."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2312_13513_gb300 as cg  # noqa: E402
from paper_2312_13513_gb300 import serve  # noqa: E402
from oracle import surrogate as osur  # noqa: E402
from synth.states import les_field, load_table, quasi_dns_field  # noqa: E402

from gpu_common import to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


def _h2_state(n, seed):
    f = quasi_dns_field(load_table("h2_flamelet.npz"), n=n, seed=seed)
    return f["T"], f["p"], f["Y"]


def _identity_model(dm, mech, T, p, Y, dt=5e-7):
    x = osur.features(T, p, Y)
    rng = np.random.default_rng(0)
    nin = mech.ns + 2
    dims = [nin, 512, 512, 512, 512, mech.ns]
    W = [rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]) for i in range(5)]
    b = [np.zeros(dims[i + 1]) for i in range(5)]
    W[4] = np.zeros_like(W[4])
    sd = x.std(axis=0)
    prm = {"W": W, "b": b, "dt": dt, "x_mean": x.mean(axis=0),
           "x_std": np.where(sd > 1e-6 * np.maximum(1, np.abs(x.mean(axis=0))), sd, 1.0),
           "y_mean": np.zeros(mech.ns), "y_std": np.ones(mech.ns),
           "box_lo": x.min(axis=0) - 1.0, "box_hi": x.max(axis=0) + 1.0}
    return cg.Surrogate(dm, prm)


def test_batch_equals_individual_launches(h2):
    dm = cg.Mechanism(h2)
    segs, ref = [], []
    for i, (n, dt, rtol) in enumerate(((3000, 5e-7, 1e-6), (1234, 1e-6, 1e-7), (77, 2e-7, 1e-6))):
        T, p, Y = _h2_state(n, 100 + i)
        a = to_dev(T, p, Y)
        b = to_dev(T, p, Y)
        cg.advance(dm, b[0], b[1], b[2], dt, rtol)
        segs.append({"T": a[0], "p": a[1], "Y": a[2], "dt": dt, "rtol": rtol})
        ref.append(b)
    serve.advance_batch(dm, segs)
    torch.cuda.synchronize()
    for s, r in zip(segs, ref):
        assert torch.equal(s["T"], r[0]) and torch.equal(s["Y"], r[2])


def _fresh(states):
    return [tuple(x.clone() for x in s) for s in states]


def test_same_result_alone_and_in_the_mix(h2, ch4):
    dm_h2, dm_ch4 = cg.Mechanism(h2), cg.Mechanism(ch4)
    base = [_h2_state(n, 200 + i) for i, n in enumerate((20000, 5000, 50000, 12000))]
    f = les_field(load_table("ch4_flamelet.npz"), n=3000, seed=9)
    base_ch4 = (f["T"], f["p"], f["Y"])
    model = _identity_model(dm_h2, h2, *base[0])
    dev = [to_dev(*s) for s in base] + [to_dev(*base_ch4)]
    mechs = [dm_h2] * 4 + [dm_ch4]
    routes = [serve.ROUTE_SURROGATE, serve.ROUTE_FP64, serve.ROUTE_FP64, serve.ROUTE_SURROGATE, serve.ROUTE_FP64]

    def run(which):
        states = _fresh(dev)
        srv = serve.Server(8 << 30, n_streams=4)
        ids = [srv.register(mechs[i], *states[i], model=model if i < 4 else None) for i in range(5)]
        reqs = [srv.submit(ids[i], routes[i], 5e-7) for i in which]
        for r in reqs:
            srv.wait(r, 120.0)
        st = srv.stats()
        srv.close()
        return states, st

    alone = {}
    for i in range(5):
        states, _ = run([i])
        alone[i] = states[i]
    mixed, st = run(range(5))
    assert st["completed"] == 5 and st["failed"] == 0
    assert st["max_concurrent"] >= 2          # launches overlapped on the device
    for i in range(5):
        assert torch.equal(mixed[i][0], alone[i][0]) and torch.equal(mixed[i][2], alone[i][2]), i


def test_small_budget_forces_queueing(h2):
    dm = cg.Mechanism(h2)
    states = [to_dev(*_h2_state(20000, 300 + i)) for i in range(4)]
    model = _identity_model(dm, h2, *[s.cpu().numpy() for s in states[0]])
    resident = sum(s[0].numel() * (h2.ns + 2) * 8 for s in states)
    # a surrogate request's workspace: gathered state copy, route, network output, box flag, fallback index
    one_request = 20000 * ((h2.ns + 2) * 8 + 1 + h2.ns * 4 + 1 + 4) + 4096
    srv = serve.Server(resident + one_request + 1000, n_streams=4)
    ids = [srv.register(dm, *s, model=model) for s in states]
    reqs = [srv.submit(i, serve.ROUTE_SURROGATE, 5e-7) for i in ids]
    for r in reqs:
        srv.wait(r, 60.0)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 4 and st["max_concurrent"] == 1


def test_never_admissible_request_is_rejected(h2):
    dm = cg.Mechanism(h2)
    s = to_dev(*_h2_state(20000, 400))
    model = _identity_model(dm, h2, *[x.cpu().numpy() for x in s])
    resident = 20000 * (h2.ns + 2) * 8
    srv = serve.Server(resident + 10000, n_streams=2)
    sid = srv.register(dm, *s, model=model)
    with pytest.raises(cg.ChemError) as e:
        srv.submit(sid, serve.ROUTE_SURROGATE, 5e-7)
    assert e.value.code == -4
    rid = srv.submit(sid, serve.ROUTE_FP64, 5e-7)       # the FP64 route fits
    srv.wait(rid, 60.0)
    srv.close()


def test_wait_times_out_and_poll_does_not_block(h2):
    dm = cg.Mechanism(h2)
    s = to_dev(*_h2_state(1 << 20, 500))
    srv = serve.Server(8 << 30)
    sid = srv.register(dm, *s)
    rid = srv.submit(sid, serve.ROUTE_FP64, 5e-7)
    t0 = time.time()
    state, lat = srv.poll(rid)
    assert time.time() - t0 < 0.05 and state in (serve.QUEUED, serve.RUNNING)
    with pytest.raises(cg.ChemError) as e:
        srv.wait(rid, 1e-4)
    assert e.value.code == -5
    srv.wait(rid, 120.0)
    state, lat = srv.poll(rid)
    assert state == serve.DONE and lat > 0.0
    srv.close()


def test_failed_request_does_not_poison_others(h2):
    dm = cg.Mechanism(h2)
    a = to_dev(*_h2_state(5000, 600))
    b = to_dev(*_h2_state(5000, 601))
    model = _identity_model(dm, h2, *[x.cpu().numpy() for x in a], dt=1e-6)   # trained for 1e-6
    srv = serve.Server(8 << 30)
    sa = srv.register(dm, *a, model=model)
    sb = srv.register(dm, *b)
    bad = srv.submit(sa, serve.ROUTE_SURROGATE, 5e-7)     # wrong dt: fails at launch
    good = srv.submit(sb, serve.ROUTE_FP64, 5e-7)
    srv.wait(good, 60.0)
    with pytest.raises(cg.ChemError):
        srv.wait(bad, 60.0)
    assert srv.poll(bad)[0] == serve.FAILED and srv.poll(good)[0] == serve.DONE
    again = srv.submit(sa, serve.ROUTE_FP64, 5e-7)
    srv.wait(again, 60.0)
    st = srv.stats()
    srv.close()
    assert st["failed"] == 1 and st["completed"] == 2


def test_time_sliced_job_equals_single_launch(ch4):
    """An FP64 job run as many short slices gives bitwise the result of one launch."""
    dm = cg.Mechanism(ch4)
    f = les_field(load_table("ch4_flamelet.npz"), n=6000, seed=31)
    a = to_dev(f["T"], f["p"], f["Y"])
    b = to_dev(f["T"], f["p"], f["Y"])
    cg.advance(dm, b[0], b[1], b[2], 1e-6)
    srv = serve.Server(8 << 30, slice_ms=2.0)
    sid = srv.register(dm, *a)
    srv.wait(srv.submit(sid, serve.ROUTE_FP64, 1e-6), 120.0)
    st = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    assert st["slices"] > 1
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2])


def test_small_request_is_not_stuck_behind_a_long_fp64_job(h2, ch4):
    """A long CH4 FP64 job runs in time slices; a small H2 surrogate request submitted after it
    completes while the job is still running."""
    dm_h2, dm_ch4 = cg.Mechanism(h2), cg.Mechanism(ch4)
    f = les_field(load_table("ch4_flamelet.npz"), n=65536, seed=32)
    big = to_dev(f["T"], f["p"], f["Y"])
    small = to_dev(*_h2_state(20000, 33))
    model = _identity_model(dm_h2, h2, *[x.cpu().numpy() for x in small])
    srv = serve.Server(8 << 30, slice_ms=10.0)
    s_big = srv.register(dm_ch4, *big)
    s_small = srv.register(dm_h2, *small, model=model)
    r_big = srv.submit(s_big, serve.ROUTE_FP64, 1e-6)
    time.sleep(0.02)
    r_small = srv.submit(s_small, serve.ROUTE_SURROGATE, 5e-7)
    srv.wait(r_small, 60.0)
    state_big, _ = srv.poll(r_big)
    srv.wait(r_big, 120.0)
    lat_small = srv.poll(r_small)[1]
    lat_big = srv.poll(r_big)[1]
    srv.close()
    assert state_big in (serve.QUEUED, serve.RUNNING), "the long job finished before the small request"
    assert lat_small < 0.5 * lat_big, (lat_small, lat_big)


def test_surrogate_batch_equals_individual_passes(h2):
    """Several states in one gathered surrogate pass give bitwise the results and routes of one
    chem_surrogate_advance per state (out-of-box cells take the FP64 fallback in both)."""
    dm = cg.Mechanism(h2)
    base = [_h2_state(n, 700 + i) for i, n in enumerate((5000, 129, 20000, 1))]
    model = _identity_model(dm, h2, *base[2])
    segs, ref = [], []
    for i, (T, p, Y) in enumerate(base):
        T = T.copy()
        T[::11] = 2600.0                          # outside the training box: FP64 fallback
        a = to_dev(T, p, Y)
        b = to_dev(T, p, Y)
        ra = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
        rb = torch.full((T.size,), -1, dtype=torch.int8, device="cuda")
        cg.surrogate_advance(model, b[0], b[1], b[2], 5e-7, route=rb)
        segs.append({"T": a[0], "p": a[1], "Y": a[2], "dt": 5e-7, "route": ra})
        ref.append((b, rb))
    serve.surrogate_advance_batch(model, segs)
    torch.cuda.synchronize()
    for s_, (b, rb) in zip(segs, ref):
        assert torch.equal(s_["T"], b[0]) and torch.equal(s_["Y"], b[2])
        assert torch.equal(s_["route"], rb) and int(rb.sum()) >= 1


def test_surrogate_batch_of_more_segments_than_one_pass_takes(h2):
    """40 states (more than the 32 segments of one pass): consecutive passes, same results as one
    call per state, an empty segment included."""
    dm = cg.Mechanism(h2)
    base = _h2_state(40 * 301, 800)
    model = _identity_model(dm, h2, *base)
    segs, ref = [], []
    for i in range(40):
        n = 0 if i == 7 else 301
        T, p, Y = (a[..., i * 301:i * 301 + n] for a in base)
        a = to_dev(T, p, Y)
        b = to_dev(T, p, Y)
        if n:
            cg.surrogate_advance(model, b[0], b[1], b[2], 5e-7)
        segs.append({"T": a[0], "p": a[1], "Y": a[2], "dt": 5e-7})
        ref.append(b)
    serve.surrogate_advance_batch(model, segs)
    torch.cuda.synchronize()
    for s_, b in zip(segs, ref):
        assert torch.equal(s_["T"], b[0]) and torch.equal(s_["Y"], b[2])


def test_fp64_requests_join_a_running_sliced_job(ch4):
    """FP64 requests of a mechanism whose time-sliced job is running join that job at its next
    slice boundary (no new launch) and give bitwise the result of their own launch."""
    dm = cg.Mechanism(ch4)
    f = les_field(load_table("ch4_flamelet.npz"), n=30000, seed=41)
    big = to_dev(f["T"], f["p"], f["Y"])
    smalls = []
    for i in range(3):
        g = les_field(load_table("ch4_flamelet.npz"), n=300 + 57 * i, seed=42 + i)
        smalls.append((g["T"], g["p"], g["Y"]))
    srv = serve.Server(8 << 30, n_streams=2, slice_ms=2.0)
    sid_big = srv.register(dm, *big)
    dev_small = [to_dev(*x) for x in smalls]
    sids = [srv.register(dm, *x) for x in dev_small]
    r_big = srv.submit(sid_big, serve.ROUTE_FP64, 1e-6)
    time.sleep(0.05)
    assert srv.poll(r_big)[0] == serve.RUNNING
    reqs = [srv.submit(s_, serve.ROUTE_FP64, 1e-6) for s_ in sids]
    for r in reqs + [r_big]:
        srv.wait(r, 120.0)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 4 and st["failed"] == 0
    assert st["joined"] >= 1 and st["launches"] <= 3
    for (T, p, Y), d in zip(smalls, dev_small):
        r = to_dev(T, p, Y)
        cg.advance(dm, r[0], r[1], r[2], 1e-6)
        torch.cuda.synchronize()
        assert torch.equal(d[0], r[0]) and torch.equal(d[2], r[2])
    rb = to_dev(f["T"], f["p"], f["Y"])
    cg.advance(dm, rb[0], rb[1], rb[2], 1e-6)
    torch.cuda.synchronize()
    assert torch.equal(big[0], rb[0]) and torch.equal(big[2], rb[2])


def test_surrogate_pass_ends_a_long_fp64_slice_early(h2, ch4):
    """With 500 ms FP64 slices, a surrogate request submitted while a long CH4 job runs completes
    in far less than a slice: issuing its pass ends the running slice (after its 2 ms minimum),
    and the job continues in later slices with bitwise the result of one launch."""
    dm_h2, dm_ch4 = cg.Mechanism(h2), cg.Mechanism(ch4)
    f = les_field(load_table("ch4_flamelet.npz"), n=262144, seed=35)
    big = to_dev(f["T"], f["p"], f["Y"])
    small = to_dev(*_h2_state(20000, 36))
    model = _identity_model(dm_h2, h2, *[x.cpu().numpy() for x in small])
    srv = serve.Server(8 << 30, slice_ms=500.0)
    s_big = srv.register(dm_ch4, *big)
    s_small = srv.register(dm_h2, *small, model=model)
    r_big = srv.submit(s_big, serve.ROUTE_FP64, 1e-6)
    time.sleep(0.05)
    assert srv.poll(r_big)[0] == serve.RUNNING
    r_small = srv.submit(s_small, serve.ROUTE_SURROGATE, 5e-7)
    srv.wait(r_small, 60.0)
    lat_small = srv.poll(r_small)[1]
    state_big = srv.poll(r_big)[0]
    srv.wait(r_big, 120.0)
    st = srv.stats()
    srv.close()
    assert state_big == serve.RUNNING, "the long job finished before the small request"
    assert lat_small < 0.15, lat_small          # a whole 500 ms slice would be waited out otherwise
    assert st["slices"] >= 2 and st["failed"] == 0
    ref = to_dev(f["T"], f["p"], f["Y"])
    cg.advance(dm_ch4, ref[0], ref[1], ref[2], 1e-6)
    torch.cuda.synchronize()
    assert torch.equal(big[0], ref[0]) and torch.equal(big[2], ref[2])
