"""The learned sketch and the pruned join.

* forward pass and gradients of the GPU network against the FP64 reference
  (oracle/mlp.py, itself pinned by finite differences);
* training lowers the loss;
* with pruning disabled (eps_sketch = -2) the pruned join returns exactly the
  plain join's result;
* on clustered data, the sketch trained and calibrated in the library
  (ejoin_sketch_train, through the C ABI alone) keeps recall >= 0.995 of the
  exact join (calibrated for 0.999 on held-out rows), as does the same recipe
  orchestrated from Python over the primitive calls, within 0.005 of it; it
  never emits a pair the exact join does not, keeps under 8 % of the tile
  pairs, under a quarter of what the untrained network keeps, and the
  library's sampled recall estimate is within 0.02 of the recall.
"""
import numpy as np
import pytest

import ejoin_inputs as inputs
import oracle
from oracle import mlp as mlp_ref
from parity_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402
from paper_2312_01476_gb300 import ejoin as E  # noqa: E402
import sketch_reference as L  # noqa: E402


def _tiny(seed=0, n=300, d=48, hid=32):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32) * 3.0
    flat = inputs.sketch_init_params(d, hid, 64, seed)
    flat[hid * d:hid * d + hid] = rng.standard_normal(hid).astype(np.float32) * 0.1
    return X, flat


def test_forward_matches_fp64_reference():
    X, flat = _tiny(1)
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        sk = E.Sketch(ctx, X.shape[1], 32, 64)
        sk.set_params(flat)
        S = sk.forward(torch.from_numpy(X).cuda()).cpu().numpy()
        params = sk.unflatten(flat.astype(np.float64))
        sk.close()
    Xu = X.astype(np.float64) / np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True)
    ref = mlp_ref.forward(params, Xu)["s"]
    assert np.abs(S - ref).max() < 2e-5


@pytest.mark.parametrize("n,d,hid", [(300, 48, 32), (5000, 768, 256), (1300, 100, 64)])
def test_tensor_core_forward_matches_fp64_reference(n, d, hid):
    # the TF32 forward the pruned join uses: sketches and sketch cosines within a few 1e-3 of FP64
    rng = np.random.default_rng(n)
    X = (rng.standard_normal((n, d)) * 2.0).astype(np.float32)
    flat = inputs.sketch_init_params(d, hid, 64, 7)
    flat[hid * d:hid * d + hid] = rng.standard_normal(hid).astype(np.float32) * 0.1
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        sk = E.Sketch(ctx, d, hid, 64)
        sk.set_params(flat)
        Xd = torch.from_numpy(X).cuda()
        St = sk.forward_tc(Xd).cpu().numpy()
        params = sk.unflatten(flat.astype(np.float64))
        sk.close()
    Xu = X.astype(np.float64) / np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True)
    ref = mlp_ref.forward(params, Xu)["s"]
    err = np.abs(St - ref)
    # TF32 products: about 1e-3 relative on z; a row of small |z| magnifies it in the normalised sketch
    assert np.median(err) < 1e-3 and np.quantile(err, 0.999) < 5e-3 and err.max() < 3e-2, (np.median(err),
                                                                                          err.max())
    p = rng.integers(0, n, 2000)
    q = rng.integers(0, n, 2000)
    cerr = np.abs(np.sum(St[p] * St[q], 1) - np.sum(ref[p] * ref[q], 1))
    assert np.quantile(cerr, 0.999) < 3e-3 and cerr.max() < 3e-2, cerr.max()


def test_gradients_match_fp64_reference():
    X, flat = _tiny(2)
    rng = np.random.default_rng(5)
    B = 70
    p = rng.integers(0, X.shape[0], B).astype(np.int32)
    q = rng.integers(0, X.shape[0], B).astype(np.int32)
    t = rng.uniform(-1, 1, B).astype(np.float32)
    w = rng.uniform(0.5, 2.0, B).astype(np.float32)
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        sk = E.Sketch(ctx, X.shape[1], 32, 64)
        sk.set_params(flat)
        Xd = torch.from_numpy(X).cuda()
        inv = E.ejoin_row_inv_norm(ctx, Xd)
        g, loss = sk.grad(Xd, inv, *(torch.from_numpy(a).cuda() for a in (p, q, t, w)))
        g = g.cpu().numpy()
        params = sk.unflatten(flat.astype(np.float64))
        sk.close()
    Xu = X.astype(np.float64) / np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True)
    # the reference takes rows by index: pair k = (p_k, q_k) of Xu
    ref = mlp_ref.backward(params, Xu, p, q, t.astype(np.float64), w.astype(np.float64))
    ref_loss = mlp_ref.loss(params, Xu, p, q, t, w)
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss))
    flat_ref = np.concatenate([ref["W1"].ravel(), ref["b1"], ref["W2"].ravel(), ref["b2"]])
    err = np.abs(g - flat_ref).max() / np.abs(flat_ref).max()
    assert err < 1e-4, err


def test_training_lowers_the_loss():
    rng = np.random.default_rng(9)
    d = 64
    centres = inputs.sphere_centres(40, d, 77)
    X = inputs.clustered(3000, d, centres, 0.3, 78, threads=1)
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        Xd = torch.from_numpy(X).cuda()
        sk = E.Sketch(ctx, d, 64, 64)
        sk.set_params(inputs.sketch_init_params(d, 64, 64, 3))
        p, q, t, w = L.labelled_pairs(ctx, Xd, 0.8, 40000, seed=1)
        inv = E.ejoin_row_inv_norm(ctx, Xd)
        _, l0 = sk.grad(Xd, inv, p, q, t, w)
        L.train(sk, Xd, p, q, t, w, epochs=4, batch=8192, lr=3e-3)
        _, l1 = sk.grad(Xd, inv, p, q, t, w)
        # the library's own training from its seeded initialisation, on the same rows
        eps_sk, rep = E.ejoin_sketch_train(sk, Xd, Xd, 0.8, n_pairs=40000, epochs=4, batch=8192, lr=3e-3, seed=1,
                                           init=True)
        _, l2 = sk.grad(Xd, inv, p, q, t, w)
        sk.close()
    assert l1 < 0.5 * l0, (l0, l1)
    assert rep["loss_last"] < 0.5 * rep["loss_first"], rep
    assert l2 < 0.5 * l0, (l0, l2)
    assert rep["labelled_join"] + rep["labelled_random"] == 40000
    assert -1.0 <= eps_sk <= 1.0


def test_pruning_disabled_equals_plain_join():
    X, flat = _tiny(4, n=2000, d=96, hid=64)
    S = np.random.default_rng(6).standard_normal((1500, 96)).astype(np.float32)
    S[:100] = X[:100] + 0.3 * np.random.default_rng(7).standard_normal((100, 96)).astype(np.float32)
    eps = 0.3
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        sk = E.Sketch(ctx, 96, 64, 64)
        sk.set_params(inputs.sketch_init_params(96, 64, 64, 4))
        Xd, Sd = torch.from_numpy(X).cuda(), torch.from_numpy(S).cuda()
        res, st = E.ejoin_threshold_pruned(ctx, sk, Xd, Sd, eps, -2.0)
        got = set(zip(res.i.cpu().numpy().tolist(), res.j.cpu().numpy().tolist()))
        assert st["tiles_kept"] == st["tiles_total"]
        plain = pkg.ejoin_threshold(ctx, Xd, Sd, eps)
        want = set(zip(plain.i.cpu().numpy().tolist(), plain.j.cpu().numpy().tolist()))
        sk.close()
    assert got == want and len(got) > 100
    oi, oj, os_ = oracle.join(X, S, eps)
    gi = np.array([a for a, b in sorted(got)], dtype=np.uint32)
    gj = np.array([b for a, b in sorted(got)], dtype=np.uint32)
    sims = dict(zip(zip(res.i.cpu().numpy().tolist(), res.j.cpu().numpy().tolist()), res.sim.cpu().numpy().tolist()))
    compare(X, S, eps, gi, gj, np.array([sims[(a, b)] for a, b in zip(gi, gj)]), oi, oj, os_)


def test_pruned_self_join_equals_plain_join():
    # self-join: the pruned path lists only tile pairs on or above the block diagonal and mirrors the
    # pairs; with nothing pruned it must return the plain join's set (every (i, i), both orders)
    X, flat = _tiny(5, n=2300, d=96, hid=64)
    X[1200:1500] = X[:300] + np.float32(0.3) * np.random.default_rng(8).standard_normal((300, 96)).astype(np.float32)
    eps = 0.3
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        sk = E.Sketch(ctx, 96, 64, 64)
        sk.set_params(inputs.sketch_init_params(96, 64, 64, 5))
        Xd = torch.from_numpy(X).cuda()
        res, st = E.ejoin_threshold_pruned(ctx, sk, Xd, Xd, eps, -2.0)
        got = dict(zip(zip(res.i.cpu().numpy().tolist(), res.j.cpu().numpy().tolist()), res.sim.cpu().numpy().tolist()))
        plain = pkg.ejoin_threshold(ctx, Xd, Xd, eps)
        want = set(zip(plain.i.cpu().numpy().tolist(), plain.j.cpu().numpy().tolist()))
        sk.close()
    assert len(got) == res.count and set(got) == want
    assert all((j, i) in got and got[(j, i)] == got[(i, j)] for (i, j) in got)
    assert all((i, i) in got for i in range(len(X)))
    oi, oj, os_ = oracle.join(X, X, eps)
    keys = sorted(got)
    compare(X, X, eps, np.array([a for a, b in keys], dtype=np.uint32), np.array([b for a, b in keys], dtype=np.uint32),
            np.array([got[k] for k in keys]), oi, oj, os_)


def test_trained_sketch_prunes_with_recall():
    d, eps, theta = 128, 0.8, 0.3
    centres = inputs.sphere_centres(120, d, 1234)  # ~200 rows per cluster, as in the 4M-row workload
    X = inputs.clustered(24000, d, centres, theta, 1235, threads=4)   # the join's input (self-join)
    Xtr = inputs.clustered(6000, d, centres, theta, 1236, threads=4)  # held out: training labels
    Xcal = inputs.clustered(6000, d, centres, theta, 1237, threads=4)  # held out: calibration
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        Xd, Xtrd, Xcald = (torch.from_numpy(a).cuda() for a in (X, Xtr, Xcal))
        plain = pkg.ejoin_threshold(ctx, Xd, Xd, eps)
        exact = set(zip(plain.i.cpu().numpy().tolist(), plain.j.cpu().numpy().tolist()))
        kept, recalls = {}, {}
        # "library": trained and calibrated by ejoin_sketch_train through the C ABI alone; "python": the
        # same recipe orchestrated over the primitive calls (sketch_reference); "untrained": calibration only
        for name in ("library", "python", "untrained"):
            sk = E.Sketch(ctx, d, 128, 64)
            sk.set_params(inputs.sketch_init_params(d, 128, 64, 11))
            if name == "library":
                eps_sk, rep = E.ejoin_sketch_train(sk, Xtrd, Xcald, eps, n_pairs=200000, epochs=6, batch=16384,
                                                   lr=3e-3, recall=0.999, seed=2, init=False)
                assert rep["labelled_join"] > 1000 and rep["loss_last"] < rep["loss_first"], rep
                assert rep["calibration_matches"] > 1000
            else:
                if name == "python":
                    p, q, t, w = L.labelled_pairs(ctx, Xtrd, eps, 200000, seed=2)
                    L.train(sk, Xtrd, p, q, t, w, epochs=6, batch=16384, lr=3e-3)
                eps_sk = L.calibrate(sk, ctx, Xcald, eps, recall=0.999)
            res, st = E.ejoin_threshold_pruned(ctx, sk, Xd, Xd, eps, eps_sk, recall_est=True)
            got = set(zip(res.i.cpu().numpy().tolist(), res.j.cpu().numpy().tolist()))
            assert got <= exact
            recalls[name] = len(got) / len(exact)
            kept[name] = st["tiles_kept"] / st["tiles_total"]
            # the library's estimate from 2048 sampled rows against the recall over all rows
            assert abs(st["recall_est"] - recalls[name]) <= 0.02, (name, st["recall_est"], recalls[name])
            assert st["recall_sample_rows"] == 2048 and st["recall_sample_matches"] > 0
            print(name, "eps_sketch", eps_sk, "recall", recalls[name], "estimate", st["recall_est"],
                  "kept", kept[name])
            sk.close()
    assert recalls["library"] >= 0.995 and recalls["python"] >= 0.995, recalls
    assert abs(recalls["library"] - recalls["python"]) <= 0.005, recalls
    # 120 clusters of ~200 rows: a tile pair can hold matches only when both tiles share a
    # cluster, a few percent of all pairs; the untrained network cannot separate them
    assert kept["library"] < 0.08 and kept["python"] < 0.08, kept
    assert kept["library"] < 0.25 * kept["untrained"], kept


def test_pair_sims_beyond_one_grid_of_rows():
    # 2.2M pairs -> 4.4M gathered rows: more than 65,535 row blocks of the GEMM grid
    rng = np.random.default_rng(21)
    X = rng.standard_normal((5000, 32)).astype(np.float32)
    n = 2_200_000
    p = rng.integers(0, 5000, n).astype(np.int32)
    q = rng.integers(0, 5000, n).astype(np.int32)
    with pkg.Ctx(device=0, prec="bf16") as ctx:
        sk = E.Sketch(ctx, 32, 16, 64)
        flat = inputs.sketch_init_params(32, 16, 64, 5)
        sk.set_params(flat)
        Xd = torch.from_numpy(X).cuda()
        inv = E.ejoin_row_inv_norm(ctx, Xd)
        got = sk.pair_sims(Xd, inv, torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda()).cpu().numpy()
        S = sk.forward(Xd).cpu().numpy()
        sk.close()
    want = np.sum(S[p] * S[q], axis=1)
    assert np.abs(got - want).max() < 1e-5
