"""The learned cost model's kernels against the double-precision reference network, its
training, and the learned census schedule (exact counts, better cost prediction)."""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import costmodel_ref as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_6308_gb300 import _build
    _build.build()
    import paper_1209_6308_gb300 as m
    m.load()
    return m


def _dataset(n=3000, seed=0):
    rng = np.random.default_rng(seed)
    X = np.stack([rng.gamma(2.0, 1.5, n), rng.gamma(2.0, 1.5, n), rng.gamma(3.0, 1.2, n), rng.gamma(6.0, 1.5, n)], 1)
    T = 5.0 + 0.8 * X[:, 2] + 0.3 * X[:, 3] + 0.2 * np.sin(X[:, 0]) + rng.normal(0, 0.05, n)
    return X.astype(np.float32), T.astype(np.float32)


def _device(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda()


def test_gpu_gradient_matches_reference(tc):
    X, T = _dataset()
    c = tc.tc_costmodel_create(3)
    try:
        mean, std, tm = X.mean(0), X.std(0), float(T.mean())
        tc.tc_costmodel_set_norm(c, mean, std, tm, 1.0)
        rng = np.random.default_rng(5)
        p = rng.normal(0, 0.3, tc.tc_costmodel_num_params()).astype(np.float32)
        tc.tc_costmodel_set_params(c, p)
        g_gpu, loss_gpu = tc.tc_costmodel_grad(c, _device(X), _device(T), len(T))
        p16 = p.astype(np.float16).astype(np.float64)     # the forward pass uses FP16 weights
        loss_ref, g_ref = ref.loss_and_grad(p16, X.astype(np.float64), T.astype(np.float64),
                                            mean.astype(np.float64), std.astype(np.float64), tm)
        assert abs(loss_gpu - loss_ref) <= 1e-3 * abs(loss_ref) + 1e-5
        scale = np.abs(g_ref).max()
        assert np.max(np.abs(g_gpu - g_ref)) <= 2e-3 * scale, np.max(np.abs(g_gpu - g_ref)) / scale
    finally:
        tc.tc_costmodel_destroy(c)


def test_gpu_prediction_matches_reference(tc):
    import torch
    X, T = _dataset(500, 1)
    c = tc.tc_costmodel_create(4)
    try:
        mean, std, tm = X.mean(0), X.std(0), float(T.mean())
        tc.tc_costmodel_set_norm(c, mean, std, tm, 1.0)
        out = torch.empty(len(T), dtype=torch.float32, device="cuda")
        tc.tc_costmodel_predict(c, _device(X), len(T), out)
        torch.cuda.synchronize()
        p16 = tc.tc_costmodel_get_params(c).astype(np.float16).astype(np.float64)
        y, _ = ref.forward(p16, X.astype(np.float64), mean, std, tm)
        np.testing.assert_allclose(np.log(out.cpu().numpy()), y + tm, rtol=0, atol=2e-3)
    finally:
        tc.tc_costmodel_destroy(c)


def test_training_reduces_loss(tc):
    X, T = _dataset(4000, 2)
    c = tc.tc_costmodel_create(7)
    try:
        dx, dt = _device(X), _device(T)
        tc.tc_costmodel_fit_norm(c, dx, dt, len(T), 1.0)
        before = tc.tc_costmodel_train(c, dx, dt, len(T), 0, 3e-3)
        after = tc.tc_costmodel_train(c, dx, dt, len(T), 400, 3e-3)
        assert after < 0.2 * before, (before, after)
    finally:
        tc.tc_costmodel_destroy(c)


def test_features_of_a_small_graph(tc):
    import torch
    s = np.array([0, 1, 2, 0], np.uint32)
    d = np.array([1, 0, 0, 3], np.uint32)
    with tc.Graph.from_arcs(5, s, d) as g:
        _, adj, perm = tc.tc_graph_export_csr(g.handle)
        feat = torch.empty(5 * 4, dtype=torch.float32, device="cuda")
        tc.tc_graph_features(g.handle, feat)
        torch.cuda.synchronize()
        f = feat.cpu().numpy().reshape(5, 4)
    # vertex 0 (old id): out {1, 3}, in {1, 2}, neighbours {1, 2, 3} with degrees 1, 1, 1
    x = perm[0]
    np.testing.assert_allclose(f[x], np.log1p([2, 2, 3, 3]), rtol=1e-6)


def test_learned_schedule_is_exact_and_predicts_cost_better(tc):
    import torch
    from paper_1209_6308_gb300 import learned
    model, info = learned.train_cost_model(scales=(14, 15, 16), seeds=(41, 42, 43), steps=400)
    try:
        assert info["samples"] > 100 and info["loss_final"] < info["loss_initial"]
        n, s, d = graphgen.rmat(15, 16, 0.2, 77)               # held-out graph
        want = oracle.census_bm_parallel(n, s, d)              # the oracle, not the plain GPU schedule
        with tc.Graph.from_arcs(n, s, d, options=learned.PLAIN) as g:
            learned.attach(model, g)
            assert g.census(options=learned.LEARNED) == want
            assert g.census(options=dict(learned.LEARNED, chunk_entries=512, item_work=4096)) == want
            q = learned.prediction_quality(model, g)
        assert q["vertices"] > 50
        assert q["rms_log_err_model"] < q["rms_log_err_degree"], q
    finally:
        tc.tc_costmodel_destroy(model)


def test_learned_schedule_keeps_the_work_balance(tc):
    """The plain schedule (items cut by exact pair work) is the fallback and the yardstick: on a
    held-out graph the learned schedule of the triangle form must give the oracle's counts and
    a makespan, from the per-CTA timestamps of the profiled census, no worse than the plain
    one's beyond timing noise; both must keep the CTAs busy most of the makespan."""
    from paper_1209_6308_gb300 import learned
    tri = {"algo": tc.TC_ALGO_TRIANGLE}
    model, info = learned.train_cost_model(scales=(14, 15, 16), seeds=(51, 52, 53), steps=300, options=tri)
    try:
        n, s, d = graphgen.rmat(17, 16, 0.2, 78)                # held-out graph
        want = oracle.census_bm_parallel(n, s, d)
        with tc.Graph.from_arcs(n, s, d, options=tri) as g:
            learned.attach(model, g)
            lrn = dict(tri, schedule=tc.TC_SCHED_LEARNED)
            assert g.census(options=lrn) == want
            bp = learned.balance(g, tri)
            bl = learned.balance(g, lrn)
        assert bl["ctas"] == bp["ctas"] > 0
        assert bl["makespan_ms"] <= 1.25 * bp["makespan_ms"] + 0.05, (bp, bl)
        assert bp["mean_busy_frac"] > 0.5 and bl["mean_busy_frac"] > 0.5, (bp, bl)
    finally:
        tc.tc_costmodel_destroy(model)
