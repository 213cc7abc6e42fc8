"""Serving loop: continuous batching of CP-ALS requests under an HBM budget.

* every result is the same, bit for bit, when its request runs alone (one slot)
  and when it runs mixed with others (four slots, all submitted at once);
* a served result equals a direct device CP-ALS run on the same inputs and
  agrees with the FP64 CP-ALS reference;
* admission respects the budget (a budget for one request at a time still
  serves them all), and a request larger than the whole budget fails alone
  with DEINSUM_ERR_OOM while the others are served.
"""
import numpy as np
import pytest

import oracle
from paper_2206_08301_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_08301_gb300 as dz  # noqa: E402

GB = 1 << 30


def _request(seed, dims, rank, sweeps=3, noise=1e-2):
    cpf = [inputs.factor_normal(seed, m, d, rank, stream_base=inputs.STREAM_CP).astype(np.float32)
           for m, d in enumerate(dims)]
    ini = [inputs.factor_normal(seed, m, d, rank, stream_base=inputs.STREAM_INIT).astype(np.float32)
           for m, d in enumerate(dims)]
    return dict(dims=dims, rank=rank, sweeps=sweeps, seed=seed, cp_factors=cpf, init_factors=ini, noise=noise)


REQS = [_request(100 + k, d, r) for k, (d, r) in enumerate(
    [((96, 80, 72), 8), ((64, 130, 100), 16), ((200, 64, 96), 32), ((128, 128, 128), 24), ((70, 90, 110), 64),
     ((150, 66, 75), 12)])]


def _serve(slots, budget=8 * GB, reqs=REQS):
    srv = dz.Server(budget, slots)
    ids = [srv.submit(want_factors=True, **q) for q in reqs]
    out = {}
    while len(out) < len(ids):
        srv.poll()
        for i in ids:
            if i not in out:
                r = srv.take(i)
                if r is not None:
                    out[i] = r
    srv.close()
    return [out[i] for i in ids]


def test_results_identical_alone_and_in_the_mix():
    alone = _serve(1)
    mixed = _serve(4)
    for a, b in zip(alone, mixed):
        assert a["status"] == 0 and b["status"] == 0
        np.testing.assert_array_equal(a["fits"], b["fits"])
        np.testing.assert_array_equal(a["lambda"], b["lambda"])
        for fa, fb in zip(a["factors"], b["factors"]):
            np.testing.assert_array_equal(fa, fb)


def test_served_result_matches_direct_run_and_oracle():
    q = REQS[2]
    (res,) = _serve(2, reqs=[q])
    X = inputs.tensor_cp_f32(q["seed"], q["dims"], q["cp_factors"], q["noise"])
    F = [torch.from_numpy(f.copy()).cuda() for f in q["init_factors"]]
    lam, fits = dz.CPALS(q["dims"], q["rank"]).run(torch.from_numpy(X).cuda(), F, q["sweeps"])
    np.testing.assert_array_equal(fits.cpu().numpy(), res["fits"])
    for m in range(3):
        np.testing.assert_array_equal(F[m].cpu().numpy(), res["factors"][m])
    ref_f, ref_lam, ref_fits = oracle.cpals(X, [f.astype(np.float64) for f in q["init_factors"]], q["sweeps"])
    assert abs(res["fit"] - ref_fits[-1]) <= 1e-4
    for m in range(3):
        assert oracle.rel_error(res["factors"][m], ref_f[m]) <= 1e-3
        assert oracle.max_elem_error(res["factors"][m], ref_f[m]) <= 1e-2


def test_budget_admission_and_oversize_request():
    # ~60 MB: roughly one of these requests at a time
    small = [_request(300 + k, (100, 100, 100), 8, sweeps=2) for k in range(4)]
    res = _serve(4, budget=60 << 20, reqs=small)
    assert all(r["status"] == 0 for r in res)
    # admission was serialised by the budget: no two requests overlapped
    spans = sorted((r["admit"], r["done"]) for r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-3
    big = _request(400, (512, 512, 512), 8, sweeps=1)   # X alone is 512 MB
    res = _serve(2, budget=256 << 20, reqs=[small[0], big, small[1]])
    assert res[0]["status"] == 0 and res[2]["status"] == 0
    assert res[1]["status"] == 6   # DEINSUM_ERR_OOM
