"""GPU tests of the continuous-batching request loop: results equal to the
direct calls, identical alone and in a mix, admission by budget, timeouts,
cancellation and argument errors (all failures made on the host)."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import FP32_TOL, GRAD_TOL, grad_err, odet, ovol, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


@pytest.fixture(scope="module")
def vols(drr):
    rng = np.random.default_rng(70)
    a = inputs.ellipsoid_phantom((40, 48, 56), (1.2, 1.0, 1.1), seed=71)
    hu = inputs.ct_phantom_hu((30, 64, 64), (1.3, 1.3, 3.0), seed=72)
    c = rng.uniform(0, 0.03, (24, 20, 28)).astype(np.float32)
    return {
        "a": (a, (1.2, 1.0, 1.1), drr.Volume(a, (1.2, 1.0, 1.1))),
        "hu": (hu, (1.3, 1.3, 3.0), drr.Volume(hu, (1.3, 1.3, 3.0), hu=True, storage="bf16")),
        "c": (c, (0.9, 1.4, 1.0), drr.Volume(c, (0.9, 1.4, 1.0), storage="f16")),
    }


def _direct(drr, vol, det, poses_np, g_np=None):
    poses = torch.from_numpy(poses_np).cuda()
    if g_np is None:
        return drr.render(vol, det, poses).cpu().numpy(), None
    E, J = drr.render(vol, det, poses, jacobian=True)
    G = drr.render_backward(vol, det, poses, torch.from_numpy(g_np).cuda())
    return E.cpu().numpy(), G.cpu().numpy()


def _mix(vols, seed, n):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        key = ["a", "hu", "c"][i % 3]
        H, W = int(rng.integers(9, 70)), int(rng.integers(9, 70))
        det = inputs.Detector(300.0, H, W, float(rng.uniform(1.0, 2.5)), float(rng.uniform(1.0, 2.5)))
        B = int(rng.integers(1, 4))
        poses = inputs.random_poses(B, seed=seed * 100 + i)
        g = inputs.upstream_grad((B, H, W), seed=seed * 100 + i) if rng.uniform() < 0.5 else None
        reqs.append((key, det, poses, g))
    return reqs


@pytest.mark.parametrize("graph", [True, False])
def test_server_matches_direct_calls(drr, vols, graph):
    srv = drr.Server(device_budget=64 << 20, use_cuda_graph=graph)
    reqs = _mix(vols, seed=1, n=12)
    tickets = [srv.submit(vols[k][2], det, p, g) for (k, det, p, g) in reqs]
    for (k, det, p, g), t in zip(reqs, tickets):
        E, G = t.wait(20000)
        E_d, G_d = _direct(drr, vols[k][2], det, p, g)
        if g is None:
            np.testing.assert_array_equal(E, E_d)  # the same forward walk
        else:
            np.testing.assert_array_equal(G, G_d)  # same re-trace, same per-tile partials and order
            E_j, _ = drr.render(vols[k][2], det, torch.from_numpy(p).cuda(), jacobian=True)
            np.testing.assert_array_equal(E, E_j.cpu().numpy())
    st = srv.stats()
    assert st["completed"] == 12 and st["failed"] == 0 and st["pending"] == 0
    srv.close()


def test_server_results_match_oracle(drr, vols):
    srv = drr.Server(device_budget=64 << 20)
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 33, 47, 1.7, 1.6)
    poses = inputs.random_poses(2, seed=73)
    g = inputs.upstream_grad((2, 33, 47), seed=74)
    E, G = srv.submit(vol, det, poses, g).wait(20000)
    E_ref = oracle.render(ovol(data, sp), odet(det), poses)
    G_ref = oracle.pose_grad(ovol(data, sp), odet(det), poses, g.astype(np.float64))
    assert rel_err(E, E_ref).max() < FP32_TOL
    assert grad_err(G, G_ref).max() < GRAD_TOL
    srv.close()


def test_alone_and_in_mix_are_identical(drr, vols):
    probe = ("hu", inputs.Detector(300.0, 40, 52, 1.8, 1.8), inputs.random_poses(3, seed=75),
             inputs.upstream_grad((3, 40, 52), seed=76))
    srv = drr.Server(device_budget=128 << 20, max_inflight=16)
    E1, G1 = srv.submit(vols[probe[0]][2], probe[1], probe[2], probe[3]).wait(20000)
    # the same request in the middle of a stream of others (several ticks, mixed volumes)
    mix = _mix(vols, seed=2, n=30)
    tickets = [srv.submit(vols[k][2], d, p, g) for (k, d, p, g) in mix[:15]]
    tp = srv.submit(vols[probe[0]][2], probe[1], probe[2], probe[3])
    tickets += [srv.submit(vols[k][2], d, p, g) for (k, d, p, g) in mix[15:]]
    E2, G2 = tp.wait(20000)
    for t in tickets:
        t.wait(20000)
    np.testing.assert_array_equal(E1, E2)
    np.testing.assert_array_equal(G1, G2)
    assert srv.stats()["ticks"] >= 2
    srv.close()


def test_admission_by_budget(drr, vols):
    # a budget that holds one 64x64 request at a time: the others queue and still complete
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 64, 64, 1.5, 1.5)
    srv = drr.Server(device_budget=40 << 10, host_budget=40 << 10)
    tickets = [srv.submit(vol, det, inputs.random_poses(2, seed=80 + i)) for i in range(6)]
    outs = [t.wait(20000)[0] for t in tickets]
    st = srv.stats()
    assert st["completed"] == 6 and st["ticks"] >= 3  # never more than one request per tick fits
    E_d, _ = _direct(drr, vol, det, inputs.random_poses(2, seed=85))
    np.testing.assert_array_equal(outs[5], E_d)
    # a request larger than the whole budget is refused up front
    with pytest.raises(drr.DrrError) as ei:
        srv.submit(vol, inputs.Detector(300.0, 200, 200, 0.5, 0.5), inputs.random_poses(4, seed=1))
    assert ei.value.status == 2  # DRR_ERR_OOM
    srv.close()


def test_timeout_cancel_and_busy_volume(drr, vols):
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 64, 64, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)  # admit nothing: every request below stays queued
    tickets = [srv.submit(vol, det, inputs.random_poses(2, seed=90 + i)) for i in range(8)]
    last = tickets[-1]
    with pytest.raises(drr.DrrError) as ei:
        last.wait(0)
    assert ei.value.status == 4  # DRR_ERR_TIMEOUT, the ticket stays valid
    # a volume referenced by queued requests cannot be destroyed
    with pytest.raises(drr.DrrError) as ei:
        vol.close()
    assert ei.value.status == 5  # DRR_ERR_BUSY
    last.cancel()
    with pytest.raises(drr.DrrError) as ei:
        last.wait(1000)
    assert ei.value.status == 8  # DRR_ERR_CANCELLED
    srv.pause(False)
    for t in tickets[:-1]:
        t.wait(60000)
    st = srv.stats()
    assert st["cancelled"] == 1 and st["completed"] == 7
    with pytest.raises(drr.DrrError) as ei:
        tickets[0].cancel()  # finished and released
    assert ei.value.status == 6
    srv.close()


def test_malformed_requests(drr, vols):
    data, sp, vol = vols["a"]
    srv = drr.Server(device_budget=16 << 20)
    with pytest.raises(drr.DrrError):
        srv.submit(vol, inputs.Detector(300.0, 0, 10, 1.0, 1.0), inputs.random_poses(1, seed=1))
    with pytest.raises(drr.DrrError):
        srv.submit(vol, inputs.Detector(-3.0, 10, 10, 1.0, 1.0), inputs.random_poses(1, seed=1))
    with pytest.raises(drr.DrrError):
        srv.submit(vol, inputs.Detector(300.0, 10, 10, 1.0, 1.0), np.zeros((0, 6), np.float32))
    t = srv.submit(vol, inputs.Detector(300.0, 10, 10, 1.0, 1.0), inputs.random_poses(1, seed=1))
    t.wait(20000)
    with pytest.raises(drr.DrrError) as ei:
        t.wait(0)  # released
    assert ei.value.status == 6  # DRR_ERR_NOT_FOUND
    srv.close()


def test_destroy_with_queued_requests(drr, vols):
    data, sp, vol = vols["c"]
    det = inputs.Detector(300.0, 64, 64, 1.5, 1.5)
    srv = drr.Server(device_budget=40 << 10, host_budget=40 << 10)
    tickets = [srv.submit(vol, det, inputs.random_poses(2, seed=100 + i)) for i in range(10)]
    srv.close()  # drains what runs, cancels what waits
    assert True


def test_backlog_is_split_between_two_ticks(drr, vols):
    # A backlog of small requests: no tick takes more than 1/tick_depth of the
    # request slots, so that the next ticks can be formed while one runs;
    # results are those of the direct calls.
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 24, 20, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20, max_inflight=16)
    srv.pause(True)
    poses = [inputs.random_poses(1, seed=300 + i) for i in range(40)]
    tickets = [srv.submit(vol, det, p) for p in poses]
    srv.pause(False)
    outs = [t.wait(20000)[0] for t in tickets]
    per_tick = {}
    for t in tickets:
        per_tick[t.result.tick] = per_tick.get(t.result.tick, 0) + 1
    assert max(per_tick.values()) <= 8 and len(per_tick) >= 5, per_tick
    for i in (0, 17, 39):
        np.testing.assert_array_equal(outs[i], _direct(drr, vol, det, poses[i])[0])
    srv.close()


def test_device_status_word_fails_only_its_request(drr, vols):
    # The status path end to end without a bad table: the host uploads one
    # request's status word with a bit already set, the kernels leave it, the
    # word comes back with the tick's results, and that request (only) ends
    # with DRR_ERR_DEVICE; a clean mix leaves every word at zero (all other
    # serving tests complete with DRR_OK).
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 20, 24, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)
    poses = [inputs.random_poses(1, seed=400 + i) for i in range(5)]
    g = inputs.upstream_grad((1, 20, 24), seed=401)
    tickets = [srv.submit(vol, det, p, g if i % 2 else None) for i, p in enumerate(poses)]
    tickets[2].inject_device_status(1)
    assert [t.poll() for t in tickets] == ["queued"] * 5
    srv.pause(False)
    for i, t in enumerate(tickets):
        if i == 2:
            with pytest.raises(drr.DrrError) as ei:
                t.wait(20000)
            assert ei.value.status == 7  # DRR_ERR_DEVICE
            assert "status word" in str(ei.value)
        else:
            E, G = t.wait(20000)
            E_d, G_d = _direct(drr, vol, det, poses[i], g if i % 2 else None)
            np.testing.assert_array_equal(E, E_d)
            if i % 2:
                np.testing.assert_array_equal(G, G_d)
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 4
    # admitted requests can no longer be flagged from the host
    t = srv.submit(vol, det, poses[0])
    t.wait(20000)
    with pytest.raises(drr.DrrError) as ei:
        t.poll()
    assert ei.value.status == 6  # released by wait
    srv.close()


def test_poll_reports_queued_running_done(drr, vols):
    data, sp, vol = vols["hu"]
    det = inputs.Detector(300.0, 64, 64, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)
    t = srv.submit(vol, det, inputs.random_poses(2, seed=410))
    assert t.poll() == "queued"
    srv.pause(False)
    import time
    deadline = time.time() + 20
    while t.poll() != "done" and time.time() < deadline:
        time.sleep(0.001)
    assert t.poll() == "done"
    t.wait(0)
    srv.close()


def test_destroy_while_threads_wait(drr, vols):
    # drr_server_destroy returns only after threads blocked in drr_server_wait
    # have left it: each waiter gets its request's result or a cancellation
    import threading
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 48, 48, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)
    tickets = [srv.submit(vol, det, inputs.random_poses(1, seed=420 + i)) for i in range(6)]
    codes = []

    def waiter(t):
        try:
            t.wait(-1)
            codes.append(0)
        except drr.DrrError as e:
            codes.append(e.status)

    threads = [threading.Thread(target=waiter, args=(t,)) for t in tickets]
    for th in threads:
        th.start()
    import time
    time.sleep(0.5)  # the waiter threads are inside drr_server_wait by then
    srv.close()
    for th in threads:
        th.join(timeout=30)
        assert not th.is_alive()
    assert sorted(codes) == [8] * 6  # all were queued (paused): cancelled


def test_two_threads_wait_on_one_ticket(drr, vols):
    # both waiters get the request's result; the ticket is released once, by
    # the last of them, and a later wait finds it gone
    import threading
    import time
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 40, 40, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)
    t = srv.submit(vol, det, inputs.random_poses(2, seed=430))
    codes = []

    def waiter():
        try:
            t.wait(-1)
            codes.append(0)
        except drr.DrrError as e:
            codes.append(e.status)

    threads = [threading.Thread(target=waiter) for _ in range(2)]
    for th in threads:
        th.start()
    time.sleep(0.5)  # the waiter threads are inside drr_server_wait by then
    srv.pause(False)
    for th in threads:
        th.join(timeout=30)
        assert not th.is_alive()
    assert codes == [0, 0]
    ref, _ = _direct(drr, vol, det, inputs.random_poses(2, seed=430))
    assert np.array_equal(t.out, ref)
    with pytest.raises(drr.DrrError) as ei:
        t.wait(0)
    assert ei.value.status == 6  # DRR_ERR_NOT_FOUND: released
    srv.close()


def _registration_direct(drr, vol, det, poses_np, fixed_np, eps=1e-8):
    poses = torch.from_numpy(poses_np).cuda()
    E, J = drr.render(vol, det, poses, jacobian=True)
    loss, g = drr.zncc(E, torch.from_numpy(fixed_np).cuda(), eps=eps)
    G = drr.render_backward(vol, det, poses, g, jac=J)
    return E.cpu().numpy(), G.cpu().numpy(), loss.cpu().numpy()


def test_registration_step_requests(drr, vols):
    # registration steps (fixed images in, -ZNCC and its pose gradient out) served in the
    # same ticks as renders and gradient requests: every result is the direct calls' bits,
    # and the loss and gradient match the oracle's render -> ZNCC -> pose gradient
    data, sp, vol = vols["hu"]
    det = inputs.Detector(300.0, 37, 41, 1.6, 1.7)
    truth = inputs.random_poses(3, seed=440)
    fixed = drr.render(vol, det, torch.from_numpy(truth).cuda()).cpu().numpy()
    moving = truth + inputs.pose_offsets(3, seed=441, max_angle_deg=5, max_trans_mm=5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)  # everything below lands in one tick
    t_reg = srv.submit(vol, det, moving, fixed=fixed)
    t_reg1 = srv.submit(vol, det, moving[:1], fixed=fixed[:1], eps=1e-6)
    g = inputs.upstream_grad((2, 37, 41), seed=442)
    t_grad = srv.submit(vol, det, moving[:2], g)
    t_ren = srv.submit(vol, det, moving)
    srv.pause(False)
    E, G, L = t_reg.wait(20000)
    E1, G1, L1 = t_reg1.wait(20000)
    Eg, Gg = t_grad.wait(20000)
    Er, _ = t_ren.wait(20000)
    assert t_reg.result.tick == t_grad.result.tick == t_ren.result.tick
    E_d, G_d, L_d = _registration_direct(drr, vol, det, moving.astype(np.float32), fixed)
    np.testing.assert_array_equal(E, E_d)
    np.testing.assert_array_equal(G, G_d)
    np.testing.assert_array_equal(L, L_d)
    E_d1, G_d1, L_d1 = _registration_direct(drr, vol, det, moving[:1].astype(np.float32), fixed[:1], eps=1e-6)
    np.testing.assert_array_equal(G1, G_d1)
    np.testing.assert_array_equal(L1, L_d1)
    Eg_d, Gg_d = _direct(drr, vol, det, moving[:2].astype(np.float32), g)
    np.testing.assert_array_equal(Gg, Gg_d)
    np.testing.assert_array_equal(Er, _direct(drr, vol, det, moving.astype(np.float32))[0])
    # against the oracle (which renders its own fixed images) on the BF16-stored volume
    ov = ovol(oracle.round_bf16(oracle.hu_to_mu(data, inputs.MU_WATER).astype(np.float32)), sp)
    F_ref = oracle.render(ov, odet(det), truth)
    E_ref = oracle.render(ov, odet(det), moving.astype(np.float32))
    np.testing.assert_allclose(L, oracle.zncc_loss(E_ref, F_ref, 1e-8), atol=1e-5)
    G_ref = oracle.pose_grad(ov, odet(det), moving.astype(np.float32), oracle.zncc_loss_grad(E_ref, F_ref, 1e-8))
    assert grad_err(G, G_ref).max() < GRAD_TOL
    # argument errors: both kinds of gradient at once; the comparison server
    with pytest.raises(drr.DrrError):
        srv.submit(vol, det, moving[:2], g, fixed=fixed[:2])
    srv.close()
    plain = drr.Server(device_budget=64 << 20, plain_fp32_baseline=True)
    with pytest.raises(drr.DrrError):
        plain.submit(vol, det, moving, fixed=fixed)
    plain.close()


def test_spin_polling_server_gives_the_same_bits(drr, vols):
    # a server that polls a lone tick's completion (spin_poll_us) returns the same results
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 40, 44, 1.5, 1.5)
    g = inputs.upstream_grad((2, 40, 44), seed=451)
    P = inputs.random_poses(2, seed=450)
    out = []
    for spin in (0, 500):
        srv = drr.Server(device_budget=64 << 20, spin_poll_us=spin)
        out.append([srv.submit(vol, det, P, g).wait(20000) for _ in range(3)])
        srv.close()
    for (E0, G0), (E1, G1) in zip(out[0], out[1]):
        np.testing.assert_array_equal(E0, E1)
        np.testing.assert_array_equal(G0, G1)


def test_caller_result_buffers(drr, vols):
    # a request may name the array that receives its DRR; it gets the same bits as a
    # fresh one, and a mis-shaped or mistyped array is refused before submission
    data, sp, vol = vols["c"]
    det = inputs.Detector(300.0, 21, 26, 1.5, 1.5)
    P = inputs.random_poses(2, seed=460)
    with drr.Server(device_budget=64 << 20) as srv:
        mine = np.full((2, 21, 26), -7.0, np.float32)
        E1, _ = srv.submit(vol, det, P, out=mine).wait(20000)
        E2, _ = srv.submit(vol, det, P).wait(20000)
        assert E1 is mine
        np.testing.assert_array_equal(mine, E2)
        for bad in (np.zeros((2, 21, 25), np.float32), np.zeros((2, 21, 26), np.float64),
                    np.zeros((2, 26, 21), np.float32).transpose(0, 2, 1)):
            with pytest.raises(ValueError):
                srv.submit(vol, det, P, out=bad)
    assert not srv.h.value  # closed on leaving the block


def test_dropped_ticket_keeps_its_buffers_alive(drr, vols):
    # a ticket dropped before its request ran: the server object keeps the request's
    # buffers (and volume) until the server is closed, so the loop never writes into
    # freed memory
    import gc
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 30, 30, 1.5, 1.5)
    srv = drr.Server(device_budget=64 << 20)
    srv.pause(True)
    t = srv.submit(vol, det, inputs.random_poses(1, seed=470), inputs.upstream_grad((1, 30, 30), seed=471))
    tid = t.id
    del t
    gc.collect()
    srv.pause(False)
    E, _ = srv.submit(vol, det, inputs.random_poses(1, seed=472)).wait(20000)
    assert np.isfinite(E).all()
    assert tid in srv._live
    srv.close()
    assert not srv._live


def test_tick_work_cap_bounds_each_tick(drr, vols):
    # a cap of about two requests' work per tick: a backlog of equal requests goes
    # into ticks of at most two, a request larger than the cap alone, and every
    # result is the direct call's
    data, sp, vol = vols["a"]
    det = inputs.Detector(300.0, 24, 20, 1.5, 1.5)
    work = 24 * 20 * (40 + 48 + 56)  # ray-planes of a one-pose render
    srv = drr.Server(device_budget=64 << 20, max_inflight=32, max_tick_work=2 * work)
    srv.pause(True)
    poses = [inputs.random_poses(1, seed=430 + i) for i in range(12)]
    tickets = [srv.submit(vol, det, p) for p in poses]
    big = srv.submit(vol, det, inputs.random_poses(3, seed=443))  # 3x the work of one: alone
    srv.pause(False)
    outs = [t.wait(20000)[0] for t in tickets]
    E_big = big.wait(20000)[0]
    per_tick = {}
    for t in tickets + [big]:
        per_tick[t.result.tick] = per_tick.get(t.result.tick, 0) + 1
    assert max(per_tick.values()) <= 2, per_tick
    assert per_tick[big.result.tick] == 1
    for i in (0, 5, 11):
        np.testing.assert_array_equal(outs[i], _direct(drr, vol, det, poses[i])[0])
    np.testing.assert_array_equal(E_big, _direct(drr, vol, det, inputs.random_poses(3, seed=443))[0])
    srv.close()


def test_plain_fp32_comparison_server(drr, vols):
    # the comparison server (one request per tick, plain FP32 walk, central
    # differences on it): its DRR is the plain walk's, bit for bit, and its
    # gradient the central differences of plain renders at the same 13 poses
    data, sp, vol = vols["hu"]
    det = inputs.Detector(300.0, 33, 29, 1.5, 1.7)
    srv = drr.Server(device_budget=64 << 20, plain_fp32_baseline=True)
    P = inputs.random_poses(2, seed=450)
    g = inputs.upstream_grad((2, 33, 29), seed=451)
    t_r = srv.submit(vol, det, P)
    t_g = srv.submit(vol, det, P, g)
    E_r, _ = t_r.wait(20000)
    E_g, G = t_g.wait(20000)
    assert t_r.result.tick != t_g.result.tick  # one request per tick
    E_plain = drr.render_plain_fp32(vol, det, torch.from_numpy(P).cuda()).cpu().numpy()
    np.testing.assert_array_equal(E_r, E_plain)
    np.testing.assert_array_equal(E_g, E_plain)
    h = np.array([1e-3] * 3 + [1e-2] * 3, np.float32)
    G_ref = np.zeros((2, 6))
    for k in range(6):
        Pp, Pm = P.copy(), P.copy()
        Pp[:, k] += h[k]
        Pm[:, k] -= h[k]
        Ep = drr.render_plain_fp32(vol, det, torch.from_numpy(Pp).cuda()).cpu().numpy().astype(np.float64)
        Em = drr.render_plain_fp32(vol, det, torch.from_numpy(Pm).cuda()).cpu().numpy().astype(np.float64)
        G_ref[:, k] = np.sum(g * (Ep - Em), axis=(1, 2)) / (2.0 * np.float64(h[k]))
    scale = np.abs(G_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(G - G_ref) <= 1e-4 * scale), (G, G_ref)
    srv.close()
