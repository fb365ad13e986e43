"""Packed multi-lattice solves and the continuous-batching server (GPU).

* a packed solve over lattices of different sizes gives, for each lattice,
  exactly (bit for bit) the result of that lattice solved alone;
* a served request gives the same solution alone and in a mix of
  concurrent requests (bitwise: per-request reductions never mix);
* admission never exceeds the HBM budget; rejection paths report
  LQCD_ENOMEM / LQCD_EBUSY / LQCD_EINVAL / LQCD_ENOTREADY."""
import time

import numpy as np
import pytest

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(8, 8, 8, 8), (4, 6, 8, 10), (6, 6, 6, 6), (12, 12, 12, 12)]


def test_packed_equals_solo(gpu, orc):
    shifts = [inputs.log_shifts(15), [1e-3, 0.1], inputs.log_shifts(5, 1e-4, 10.0), [0.01]]
    masses = [0.01, 0.05, 0.02, 0.1]
    ctxs, bs, solo = [], [], []
    for k, d in enumerate(SIZES):
        c = gpu.Context(d)
        c.links_upload(inputs.random_links(d, seed=100 + k))
        b = inputs.gaussian_field(d, k=k)
        x, _ = c.mscg_solve(masses[k], shifts[k], 1e-10, b)
        ctxs.append(c)
        bs.append(b)
        solo.append(x)
    xs, infos = gpu.mscg_solve_packed(ctxs, masses, shifts, [1e-10] * 4, bs)
    for k, d in enumerate(SIZES):
        assert np.array_equal(xs[k], solo[k]), f"lattice {d}"
        assert max(infos[k]["true_resid"]) <= 1e-10
        U = inputs.random_links(d, seed=100 + k)
        assert orc.true_residual(d, U, masses[k], shifts[k][0], bs[k], xs[k][0]) <= 1e-10
    for c in ctxs:
        c.close()


def test_packed_maximum_job_count(gpu):
    """64 lattices, the most one packed launch takes (the finaliser's job
    mask has 64 bits): each result equals its lattice solved alone, bit for
    bit; a 65th lattice is rejected before any launch."""
    shifts = [1e-3, 0.1]
    ctxs, bs, solo = [], [], []
    try:
        for k in range(65):
            d = (6, 6, 6, 6) if k % 4 == 0 else (4, 4, 4, 4)  # 3 tiles or 1, both ragged
            c = gpu.Context(d)
            ctxs.append(c)
            c.links_upload(inputs.random_links(d, seed=300 + k))
            b = inputs.gaussian_field(d, k=k)
            bs.append(b)
            if k < 64:
                solo.append(c.mscg_solve(0.05, shifts, 1e-10, b)[0])
        xs, infos = gpu.mscg_solve_packed(ctxs[:64], [0.05] * 64, [shifts] * 64, [1e-10] * 64, bs[:64])
        for k in range(64):
            assert np.array_equal(xs[k], solo[k]), f"lattice {k}"
            assert max(infos[k]["true_resid"]) <= 1e-10
        with pytest.raises(gpu.LqcdError) as e:
            gpu.mscg_solve_packed(ctxs, [0.05] * 65, [shifts] * 65, [1e-10] * 65, bs)
        assert e.value.status == gpu.LQCD_EINVAL
    finally:
        for c in ctxs:
            c.close()


def _wait(srv, ticket, fid, n, timeout=120):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = srv.poll(ticket, fid, n)
        if r is not None:
            return r
        time.sleep(0.002)
    raise TimeoutError


def test_served_request_alone_equals_in_mix(gpu, orc):
    with gpu.Server(8 << 30, max_slots=8, max_queue=64) as srv:
        fids = [srv.register_field(d, inputs.random_links(d, seed=200 + k)) for k, d in enumerate(SIZES)]
        target = (fids[0], 0.01, inputs.log_shifts(8), 1e-10, inputs.gaussian_field(SIZES[0], k=7))
        t = srv.submit(*target)
        x_alone, info_alone = _wait(srv, t, fids[0], 8)
        # the same request among others arriving before and after it
        others = []
        rng = np.random.default_rng(3)
        for k in range(6):
            f = int(rng.integers(0, len(fids)))
            n = int(rng.integers(1, 9))
            others.append((srv.submit(fids[f], 0.02, inputs.log_shifts(n, 1e-4, 1.0), 1e-8,
                                      inputs.gaussian_field(SIZES[f], k=20 + k)), f, n))
            if k == 2:
                t2 = srv.submit(*target)
        x_mix, info_mix = _wait(srv, t2, fids[0], 8)
        for tk, f, n in others:
            x, info = _wait(srv, tk, fids[f], n)
            assert max(info["true_resid"]) <= 1e-8
        srv.drain(60)
        st = srv.stats()
    assert np.array_equal(x_alone, x_mix)
    assert info_alone["iters"] == info_mix["iters"]
    U = inputs.random_links(SIZES[0], seed=200)
    for i, s in enumerate(inputs.log_shifts(8)):
        assert orc.true_residual(SIZES[0], U, 0.01, s, target[4], x_mix[i]) <= 1e-10
    assert st["completed"] == 8 and st["p99_latency"] >= st["p50_latency"] > 0
    assert st["hbm_in_use"] <= st["hbm_budget"]


@pytest.mark.parametrize("fp64_until", [3e-4, 0.0])
def test_served_mixed_request_alone_equals_in_mix_and_solo(gpu, orc, fp64_until):
    """Mixed-precision serving (FP32 12-real links, FP64 phase down to
    fp64_until, reliable updates, refinement): a request gives the same
    solution alone, in a mix of FP32 requests, and as a solo mixed solve."""
    with gpu.Server(8 << 30, max_slots=8, max_queue=64) as srv:
        srv.set_opts(prec=gpu.PREC_FP32, recon=12, fp64_until=fp64_until)
        fids = [srv.register_field(d, inputs.random_links(d, seed=300 + k)) for k, d in enumerate(SIZES)]
        target = (fids[0], 0.01, inputs.log_shifts(8), 1e-10, inputs.gaussian_field(SIZES[0], k=9))
        x_alone, info_alone = _wait(srv, srv.submit(*target), fids[0], 8)
        others = []
        rng = np.random.default_rng(5)
        for k in range(6):
            f = int(rng.integers(0, len(fids)))
            n = int(rng.integers(1, 9))
            others.append((srv.submit(fids[f], 0.02, inputs.log_shifts(n, 1e-4, 1.0), 1e-9,
                                      inputs.gaussian_field(SIZES[f], k=40 + k)), f, n))
            if k == 2:
                t2 = srv.submit(*target)
        x_mix, info_mix = _wait(srv, t2, fids[0], 8)
        for tk, f, n in others:
            x, info = _wait(srv, tk, fids[f], n)
            assert max(info["true_resid"]) <= 1e-9
        srv.drain(60)
        with pytest.raises(gpu.LqcdError) as e:  # FP16 requests are not served
            srv.set_opts(prec=gpu.PREC_FP16)
        assert e.value.status == gpu.LQCD_EINVAL
    assert np.array_equal(x_alone, x_mix)
    assert info_alone["reliable_updates"] == info_mix["reliable_updates"] > 0
    U = inputs.random_links(SIZES[0], seed=300)
    with gpu.Context(SIZES[0], prec=gpu.PREC_FP32, recon=12, fp64_until=fp64_until) as c:
        c.links_upload(U)
        x_solo, _ = c.mscg_solve(0.01, inputs.log_shifts(8), 1e-10, target[4])
    assert np.array_equal(x_alone, x_solo)
    for i, s in enumerate(inputs.log_shifts(8)):
        assert orc.true_residual(SIZES[0], U, 0.01, s, target[4], x_mix[i]) <= 1e-10


def test_set_opts_busy_while_requests_run(gpu):
    d = (8, 8, 8, 8)
    with gpu.Server(1 << 30, max_slots=2, max_queue=16) as srv:
        fid = srv.register_field(d, inputs.random_links(d))
        ts = [srv.submit(fid, 0.01, inputs.log_shifts(8), 1e-10, inputs.gaussian_field(d, k=k)) for k in range(4)]
        with pytest.raises(gpu.LqcdError) as e:
            srv.set_opts(prec=gpu.PREC_FP32)
        assert e.value.status == gpu.LQCD_EBUSY
        for t in ts:
            _wait(srv, t, fid, 8)
        srv.drain(60)
        srv.set_opts(prec=gpu.PREC_FP32)


def test_admission_respects_budget(gpu):
    d = (8, 8, 8, 8)
    with gpu.Server(64 << 20, max_slots=8, max_queue=64) as srv:
        fid = srv.register_field(d, inputs.random_links(d))
        tickets = [srv.submit(fid, 0.05, [1e-3, 0.1, 1.0], 1e-9, inputs.gaussian_field(d, k=k)) for k in range(10)]
        peak = 0
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            st = srv.stats()
            peak = max(peak, st["hbm_in_use"])
            assert st["hbm_in_use"] <= st["hbm_budget"]
            for t in tickets:
                if t not in done:
                    r = srv.poll(t, fid, 3)
                    if r is not None:
                        done[t] = r
        assert len(done) == len(tickets)
        for x, info in done.values():
            assert max(info["true_resid"]) <= 1e-9


def test_rejections(gpu):
    d = (4, 4, 4, 4)
    with gpu.Server(16 << 20, max_slots=1, max_queue=2) as srv:
        with pytest.raises(gpu.LqcdError) as e:  # 12^4 links in every storage format exceed 16 MB
            srv.register_field((12, 12, 12, 12), inputs.random_links((12, 12, 12, 12)))
        assert e.value.status == gpu.LQCD_ENOMEM
        fid = srv.register_field(d, inputs.random_links(d))
        b = inputs.gaussian_field(d)
        with pytest.raises(gpu.LqcdError) as e:
            srv.submit(fid, 0.1, [-1.0], 1e-8, b)
        assert e.value.status == gpu.LQCD_EINVAL
        with pytest.raises(gpu.LqcdError) as e:
            srv.submit(99, 0.1, [0.0], 1e-8, b)
        assert e.value.status == gpu.LQCD_EINVAL
        with pytest.raises(gpu.LqcdError) as e:
            srv.poll(12345, fid, 1)
        assert e.value.status == gpu.LQCD_EINVAL
        got_busy = False
        tickets = []
        for k in range(50):
            try:
                tickets.append(srv.submit(fid, 0.01, inputs.log_shifts(8), 1e-10, b))
            except gpu.LqcdError as ex:
                assert ex.status == gpu.LQCD_EBUSY
                got_busy = True
                break
        assert got_busy
        srv.drain(120)
        for t in tickets:
            assert srv.poll(t, fid, 8) is not None
