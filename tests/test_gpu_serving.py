"""Continuous-batching server: every result is the same alone and in the mix,
equal to the direct API, within its tolerance's bound of the oracle's exact
posterior mean, unaffected by cancelled requests, and admission respects the
HBM budget."""
import time

import numpy as np
import pytest
import torch

import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _requests():
    reqs = []
    for i, (n, d, kern, tol, prec) in enumerate([
            (1500, 3, wl.RBF, 1e-2, ap.AP_FP32), (5000, 7, wl.MATERN52, 1e-4, ap.AP_BF16_REFINE),
            (2048, 20, wl.RBF, 1e-4, ap.AP_FP32), (9000, 12, wl.MATERN52, 1e-2, ap.AP_BF16_REFINE),
            (1024, 5, wl.MATERN52, 1e-4, ap.AP_FP32), (6000, 16, wl.RBF, 1e-2, ap.AP_BF16_REFINE)]):
        req = wl.Request(i, 0.0, n, d, kern, wl.log_uniform(np.random.default_rng(30 + i), 0.3, 3.0, d).astype(np.float32),
                         1.0, 0.05, tol, prec == ap.AP_BF16_REFINE, 40_000 + i)
        X, y, Xt = wl.request_data(req, m_test=256)
        reqs.append((req, X, y, Xt, prec))
    return reqs


def _submit(srv, req, X, y, Xt, prec):
    h = ap.Hyper(req.kernel, req.lengthscale, req.outputscale, req.noise, 0.1)
    return srv.submit(X, y, Xt, h, block=min(req.n, 1024), tol=req.tol, max_epochs=60, precision=prec,
                      refine_every=4)


def test_results_same_alone_and_in_mix():
    reqs = _requests()
    solo = []
    srv = ap.ApServer(hbm_budget=40 * GB, slots=1)
    for r in reqs:
        rid = _submit(srv, *r)
        res = srv.wait(rid)
        assert res["done"] and res["status"] in (ap.AP_OK, ap.AP_ERR_NOT_CONVERGED)
        solo.append(srv.mean(rid).copy())
    srv.close()
    srv = ap.ApServer(hbm_budget=40 * GB, slots=4)
    ids = [_submit(srv, *r) for r in reqs]
    for rid, ref in zip(ids, solo):
        res = srv.wait(rid)
        assert res["done"]
        got = srv.mean(rid)
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
    srv.close()


def test_server_matches_direct_api():
    req, X, y, Xt, prec = _requests()[1]
    srv = ap.ApServer(hbm_budget=40 * GB, slots=2)
    rid = _submit(srv, req, X, y, Xt, prec)
    srv.wait(rid)
    got = srv.mean(rid).copy()
    srv.close()
    dev = "cuda:0"
    h = ap.Hyper(req.kernel, req.lengthscale, req.outputscale, req.noise, 0.1)
    ctx = ap.ap_create(torch.from_numpy(X).to(dev), h,
                       ap.ap_opts_default(block=min(req.n, 1024), tol=req.tol, stop=ap.AP_STOP_MAX_REL, min_epochs=1,
                                          max_epochs=60, precision=prec, refine_every=4))
    yd = torch.from_numpy(y - np.float32(0.1)).to(dev)
    _, W, _, _ = ap.ap_solve(ctx, yd)
    mu = ap.ap_predict_mean(ctx, W[:, 0].contiguous(), torch.from_numpy(Xt).to(dev)).cpu().numpy()
    assert np.abs(got - mu).max() <= 1e-5 * max(1.0, np.abs(mu).max())


def test_admission_by_budget_serialises_when_only_one_fits():
    reqs = _requests()[3:5]
    sizes = []
    srv = ap.ApServer(hbm_budget=64 * GB, slots=2)
    for r in reqs:
        rid = _submit(srv, *r)
        sizes.append(srv.wait(rid)["reserved_bytes"])
    srv.close()
    budget = max(sizes) + min(sizes) // 2  # both never fit at once
    srv = ap.ApServer(hbm_budget=budget, slots=2)
    ids = [_submit(srv, *r) for r in reqs]
    res = [srv.wait(i) for i in ids]
    srv.close()
    # the second request starts only after the first has finished
    assert res[1]["queue_s"] >= res[0]["latency_s"] - 1e-3
    srv = ap.ApServer(hbm_budget=1 << 20, slots=1)
    with pytest.raises(ap.ApError) as e:
        _submit(srv, *reqs[0])
    assert e.value.status == ap.AP_ERR_NOMEM
    srv.close()


def _oracle_requests():
    # sizes the FP64 dense solve finishes in seconds; both forms, both tolerances
    out = []
    for i, (n, d, kern, tol, prec) in enumerate([
            (1500, 3, wl.RBF, 1e-2, ap.AP_FP32), (3000, 7, wl.MATERN52, 1e-4, ap.AP_BF16_REFINE),
            (2048, 12, wl.RBF, 1e-4, ap.AP_FP32), (4000, 5, wl.MATERN52, 1e-2, ap.AP_BF16_REFINE),
            (1024, 16, wl.MATERN52, 1e-4, ap.AP_FP32), (2500, 9, wl.RBF, 1e-4, ap.AP_BF16_REFINE)]):
        req = wl.Request(i, 0.0, n, d, kern, wl.log_uniform(np.random.default_rng(60 + i), 0.3, 3.0, d).astype(np.float32),
                         1.0, 0.05, tol, prec == ap.AP_BF16_REFINE, 50_000 + i)
        X, y, Xt = wl.request_data(req, m_test=256)
        out.append((req, X, y, Xt, prec))
    return out


def _submit_to_tol(srv, req, X, y, Xt, prec):
    h = ap.Hyper(req.kernel, req.lengthscale, req.outputscale, req.noise, 0.1)
    return srv.submit(X, y, Xt, h, block=min(req.n, 1024), tol=req.tol, max_epochs=100000, precision=prec,
                      refine_every=4)


def test_every_request_meets_its_tolerance_against_the_oracle():
    """Each request runs to its tolerance, and its posterior mean is within the
    bound its certified residual implies of the oracle's exact posterior mean
    (Sec. 2): mu_gpu - mu* = s k(x*, X) K_hat^{-1} r, so
    |mu_gpu,t - mu*_t| <= ||s k(x*_t, X)||_2 ||r||_2 / sigma^2 + the FP32 product
    error of the mean; ||r|| <= (rel_res + e_rec) ||y - mu|| with e_rec the error
    of the recompute that certified rel_res: 2e-5 || K_hat |w*| + |y - mu| || /
    ||y - mu|| for the plain FP32 one, 2^-23 + 1e-9 || K_hat |w*| + |y - mu| || /
    ||y - mu|| for the compensated one (the tolerances of the residual parity
    tests)."""
    import oracle
    reqs = _oracle_requests()
    srv = ap.ApServer(hbm_budget=40 * GB, slots=3)
    ids = [_submit_to_tol(srv, *r) for r in reqs]
    for rid, (req, X, y, Xt, prec) in zip(ids, reqs):
        res = srv.wait(rid)
        assert res["done"] and res["status"] == ap.AP_OK, (req, res)
        assert res["rel_res"] <= req.tol
        h = oracle.Hyper(req.kernel, req.lengthscale, req.outputscale, req.noise, 0.1)
        X64, b = X.astype(np.float64), y.astype(np.float64) - np.float64(np.float32(0.1))
        w = oracle.dense_solve(h, X64, b)
        mu = oracle.predict_mean(h, X64, w, Xt.astype(np.float64))
        Ks = oracle.gram(h, Xt.astype(np.float64), X64, noise=False)
        Kw = -oracle.residual_rows(h, X64, np.zeros_like(b), np.abs(w))[:, 0]
        mag = np.linalg.norm(Kw + np.abs(b)) / np.linalg.norm(b)
        e_rec = 2.0 ** -23 + 1e-9 * mag if res["compensated"] else 2e-5 * mag
        r_norm = (res["rel_res"] + e_rec) * np.linalg.norm(b)
        bound = np.linalg.norm(Ks, axis=1) * r_norm / req.noise + 2e-5 * (np.abs(Ks) @ np.abs(w) + 0.1)
        got = srv.mean(rid).astype(np.float64)
        assert np.all(np.abs(got - mu) <= bound), (req.n, np.max(np.abs(got - mu) / bound))
        print(f"request n={req.n} d={req.d} tol={req.tol:g} prec={prec}: epochs {res['epochs']}, "
              f"compensated {res['compensated']}, max |mu - mu*| / bound {np.max(np.abs(got - mu) / bound):.3f}")
    srv.close()


def test_cancelled_requests_leave_the_others_unchanged():
    reqs = _oracle_requests()[:2]
    solo = []
    srv = ap.ApServer(hbm_budget=40 * GB, slots=1)
    for r in reqs:
        rid = _submit_to_tol(srv, *r)
        assert srv.wait(rid)["status"] == ap.AP_OK
        solo.append(srv.mean(rid).copy())
    srv.close()
    # a long request (its tolerance is out of reach) holds the only slot until
    # it is cancelled while running; a queued request is cancelled before it starts
    lreq = wl.Request(9, 0.0, 20000, 3, wl.MATERN52, np.array([1.0, 2.0, 1.5], np.float32), 1.0, 0.01, 1e-9,
                      False, 59_000)
    LX, Ly, LXt = wl.request_data(lreq, m_test=256)
    srv = ap.ApServer(hbm_budget=40 * GB, slots=1)
    lid = srv.submit(LX, Ly, LXt, ap.Hyper(lreq.kernel, lreq.lengthscale, 1.0, 0.01, 0.0), block=1024, tol=1e-9,
                     max_epochs=1_000_000)
    ids = [_submit_to_tol(srv, *r) for r in reqs]
    qid = _submit_to_tol(srv, *reqs[0])
    deadline = time.time() + 60
    while not srv.poll(lid)["started"] and time.time() < deadline:
        time.sleep(0.01)
    time.sleep(0.5)
    srv.cancel(qid)
    srv.cancel(lid)
    res_l = srv.wait(lid)
    assert res_l["status"] == ap.AP_ERR_CANCELLED and res_l["started"]
    res_q = srv.wait(qid)
    assert res_q["status"] == ap.AP_ERR_CANCELLED and not res_q["started"]
    for rid, ref in zip(ids, solo):
        res = srv.wait(rid)
        assert res["status"] == ap.AP_OK
        assert np.abs(srv.mean(rid) - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())
    srv.close()
