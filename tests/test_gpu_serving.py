"""Continuous-batching server: every result is the same alone and in the mix,
equal to the direct API, and admission respects the HBM budget."""
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
