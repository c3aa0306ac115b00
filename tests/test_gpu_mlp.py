"""The learned detection threshold on the GPU, against the oracle
(oracle/mlp.py and the FP64 GEMM oracle).

* forward pass and gradient of the project's kernels vs the float64 oracle;
* training (minibatch Adam) vs the oracle's training;
* the features and residual ratios the GEMM epilogue writes for training;
* the network as evaluated inside the epilogue vs the oracle's forward pass;
* what a network trained on the method's own residuals gains over the fixed
  analytic threshold: on coherent and on zero-mean inputs alike, detection of
  faults below the analytic threshold (whose checksum-growth term keeps
  coherent inputs free of false alarms at a wide margin), with no false
  alarm from either -- judged against the injected positions.
"""
import numpy as np
import pytest

import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
U = 2.0 ** -24
TDM, TDN = 125, 252  # bf16 data tile with checksums (ftgemm_tc_tile)


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


@pytest.fixture()
def handle(ft):
    h = ft.Handle(0)
    yield h
    h.close()


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _theta(seed, scale=0.3):
    return synth.normal((omlp.N_PARAMS,), seed).astype(np.float64) * scale


def test_forward_matches_oracle(ft, handle):
    th = _theta(300)
    X = synth.uniform((2000, 5), 301).astype(np.float64)
    y = handle.mlp_forward(_dev(X), _dev(th)).cpu().numpy().astype(np.float64)
    want, _ = omlp.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(y, want, rtol=1e-5, atol=1e-5)


def test_gradient_matches_oracle_and_repeats(ft, handle):
    th = _theta(302)
    X = synth.uniform((3000, 5), 303).astype(np.float32).astype(np.float64)
    t = synth.normal((3000,), 304).astype(np.float32).astype(np.float64)
    th32 = th.astype(np.float32).astype(np.float64)
    L, g = handle.mlp_grad(_dev(X), _dev(t), _dev(th32))
    Lo, go = omlp.grad(th32, X, t)
    g = g.cpu().numpy().astype(np.float64)
    assert L == pytest.approx(Lo, rel=1e-5)
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()
    # fixed-order reduction: the same gradient bit for bit
    _, g2 = handle.mlp_grad(_dev(X), _dev(t), _dev(th32))
    assert np.array_equal(g, g2.cpu().numpy().astype(np.float64))


def test_training_tracks_oracle(ft, handle):
    X = synth.uniform((512, 5), 305).astype(np.float32).astype(np.float64)
    t = (0.3 * X[:, 0] - 0.2 * X[:, 1] + 0.5).astype(np.float32).astype(np.float64)
    th0 = _theta(306, 0.2).astype(np.float32).astype(np.float64)
    dth = _dev(th0)
    lr, epochs, batch = 1e-3, 3, 64
    losses = handle.mlp_train(_dev(X), _dev(t), dth, epochs, batch, lr)
    th_o, lo = omlp.train(th0, X, t, epochs, batch, lr)
    per_epoch = [np.mean(lo[e * 8:(e + 1) * 8]) for e in range(epochs)]
    np.testing.assert_allclose(losses, per_epoch, rtol=2e-3)
    # each Adam step moves a parameter by at most about lr: a sign flip of a
    # tiny gradient component in fp32 costs at most 2 lr per step
    assert np.abs(dth.cpu().numpy().astype(np.float64) - th_o).max() <= 2 * lr * epochs * 8


def _bf16(orc, x):
    return orc.round_bf16(x).astype(np.float32)


def _inputs(orc, kind, M, N, K, seed):
    if kind == "normal":
        A, B = synth.normal((M, K), seed), synth.normal((K, N), seed + 1)
    elif kind.startswith("shift"):  # N(mu, 1): partly coherent
        mu = float(kind[5:])
        A, B = synth.normal((M, K), seed) + mu, synth.normal((K, N), seed + 1) + mu
    elif kind == "positive":  # U(0, 1): fully coherent
        A = (synth.uniform((M, K), seed) + 1) / 2
        B = (synth.uniform((K, N), seed + 1) + 1) / 2
    return _bf16(orc, A), _bf16(orc, B)


def _oracle_features(A, B, K):
    """The 5 features of every tile, computed in float64 from the operands."""
    M, N = A.shape[0], B.shape[1]
    tm, tn = -(-M // TDM), -(-N // TDN)
    co_a = [omlp.coherence(A[i * TDM:(i + 1) * TDM], axis=0) for i in range(tm)]
    co_b = [omlp.coherence(B[:, j * TDN:(j + 1) * TDN], axis=1) for j in range(tn)]
    out = []
    for i in range(tm):
        for j in range(tn):
            rows, cols = min(TDM, M - i * TDM), min(TDN, N - j * TDN)
            out.append(omlp.features(K, rows, cols, co_a[i], co_b[j], "bf16"))
    return np.array(out)


def _run(ft, handle, A, B, faults=None, sink=True):
    """TILE-level bf16 GEMM through the library; returns (C, report, lam_needed, features)."""
    import torch
    M, K = A.shape
    N = B.shape[1]
    tiles = -(-M // TDM) * -(-N // TDN)
    lam = torch.zeros(tiles, device="cuda")
    feat = torch.zeros(tiles * 5, device="cuda")
    if sink:
        handle.set_residual_sink(lam, feat)
    dC = torch.zeros(M, N, device="cuda")
    rep = handle.gemm(_dev(A).to(torch.bfloat16), _dev(B).to(torch.bfloat16), dC, level=ft.FT_TILE,
                      dtype=ft.BF16, inject=faults)
    torch.cuda.synchronize()
    handle.set_residual_sink(None)
    return dC, rep, lam.cpu().numpy().astype(np.float64), feat.cpu().numpy().reshape(-1, 5).astype(np.float64)


def _analytic_tau(A64, B64, i, j, tm_, tn_, lam=32.0, mu=8.0):
    """The analytic row and column thresholds of element (i, j) after the
    whole K: lam*u*norms + mu*u*sqrt(K)*|checksum|, the checksums from the
    exact product."""
    K = A64.shape[1]
    I = slice(tm_ * TDM, (tm_ + 1) * TDM)
    J = slice(tn_ * TDN, (tn_ + 1) * TDN)
    c_r = A64[i] @ B64[:, J].sum(1)
    c_c = A64[I].sum(0) @ B64[:, j]
    row = lam * U * np.linalg.norm(A64[i]) * np.linalg.norm(B64[:, J]) + mu * U * np.sqrt(K) * abs(c_r)
    col = lam * U * np.linalg.norm(A64[I]) * np.linalg.norm(B64[:, j]) + mu * U * np.sqrt(K) * abs(c_c)
    return row, col


def test_epilogue_features_and_residual_ratios(ft, handle, orc):
    """The sink's features equal the oracle's.  On coherent inputs a tile's
    lambda_needed (the residual in units of the norm term) exceeds the
    analytic lambda of 32 -- the norm term alone would raise false alarms --
    and the checksum-growth term keeps every tile free of them."""
    M, N, K = 600, 1000, 4096
    A, B = _inputs(orc, "positive", M, N, K, 310)
    _, rep, lam, feat = _run(ft, handle, A, B)
    np.testing.assert_allclose(feat, _oracle_features(A, B, K), rtol=1e-5, atol=1e-6)
    assert np.all(np.isfinite(lam)) and np.all(lam >= 0)
    assert np.all(lam > 32.0)
    assert rep.detected == 0


def test_epilogue_network_matches_oracle_forward(ft, handle, orc):
    """With the learned threshold on, the tau of a fault record is
    lambda_t * u * (||A_i|| ||B_J||_F + ||A_I||_F ||B_j||) with lambda_t =
    scale * 2^f(x_t) and f the oracle's network."""
    M, N, K = 360, 496, 1024
    A, B = _inputs(orc, "normal", M, N, K, 320)
    th = _theta(321, 0.2).astype(np.float32)
    scale = 64.0  # with a small network output, about the analytic lambda: no false alarms
    handle.set_threshold(1, scale, th)
    faults = [(1, 1, 0, 7, 11, 50.0), (2, 0, 0, 100, 200, -40.0)]
    _, rep, _, feat = _run(ft, handle, A, B, faults=faults)
    handle.set_threshold(0)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    nA, nB = np.linalg.norm(A64, axis=1), np.linalg.norm(B64, axis=0)
    tn = -(-N // TDN)
    assert len(rep.records) == 2
    for r in rep.records:
        tm_, tn_ = r["tile_m"], r["tile_n"]
        x = feat[tm_ * tn + tn_]
        y, _ = omlp.forward(th.astype(np.float64), x[None, :])
        lam_t = scale * 2.0 ** y[0]
        I = slice(tm_ * TDM, (tm_ + 1) * TDM)
        J = slice(tn_ * TDN, (tn_ + 1) * TDN)
        tau = lam_t * U * (nA[r["row"]] * np.linalg.norm(B64[:, J]) + np.linalg.norm(A64[I]) * nB[r["col"]])
        assert r["tau"] == pytest.approx(tau, rel=1e-4)


def _collect(ft, handle, orc, specs):
    Xs, ts = [], []
    for q, (kind, M, N, K) in enumerate(specs):
        A, B = _inputs(orc, kind, M, N, K, 400 + 10 * q)
        _, _, lam, feat = _run(ft, handle, A, B)
        Xs.append(feat)
        ts.append(np.log2(np.maximum(lam, 2.0 ** -6)))
    return np.vstack(Xs), np.concatenate(ts)


def test_learned_threshold_gains_over_analytic(ft, handle, orc):
    import torch
    kinds = ["normal", "shift0.25", "shift1", "shift3", "positive"]
    specs = [(k, M, M, K) for k in kinds for K in (128, 512, 2048, 8192) for M in (800, 1600)]
    X, t = _collect(ft, handle, orc, specs)
    # train on the GPU with the project's kernels
    th = torch.from_numpy((synth.normal((omlp.N_PARAMS,), 330) * 0.2).astype(np.float32)).cuda()
    order = np.argsort(synth.uniform((len(t),), 331))
    Xd, td = _dev(X[order]), _dev(t[order])
    losses = handle.mlp_train(Xd, td, th, epochs=300, batch=256, lr=3e-3)
    assert losses[-1] < 0.25 * losses[0]
    y = handle.mlp_forward(Xd, th).cpu().numpy().astype(np.float64)
    margin = float(np.max(t[order] - y)) + 1.0  # calibrated on the training tiles, then x2
    handle.set_threshold(1, 2.0 ** margin, th.cpu().numpy())

    # (1) coherent inputs: no false alarm from either threshold; faults put
    #     at 1.25x the larger of their learned row / column thresholds lie
    #     below the analytic threshold on both sides: missed by the analytic
    #     threshold, located and corrected by the learned one.  Whole tiles
    #     only: on a ragged edge tile a dozen columns wide the learned lambda
    #     is the larger of the two
    M, N = 12 * TDM, 6 * TDN
    K = 4096
    A, B = _inputs(orc, "positive", M, N, K, 500)
    _, rep_mlp, _, _ = _run(ft, handle, A, B, sink=False)
    handle.set_threshold(0)
    _, rep_ana, _, _ = _run(ft, handle, A, B, sink=False)
    assert rep_ana.detected == 0 and rep_mlp.detected == 0
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    nA, nB = np.linalg.norm(A64, axis=1), np.linalg.norm(B64, axis=0)
    tiles_m, tiles_n = -(-M // TDM), -(-N // TDN)
    y_tiles, _ = omlp.forward(th.cpu().numpy().astype(np.float64), _oracle_features(A, B, K))
    lam_t = 2.0 ** margin * 2.0 ** y_tiles
    pos = synth.fault_positions(synth.workload_seed("tc_square", 91), 12, tiles_m, tiles_n, K // 64, TDM, TDN, M, N, K // 64)
    faults, ratio = [], []
    for (tm_, tn_, ks, r, c) in pos:
        i, j = tm_ * TDM + r, tn_ * TDN + c
        I = slice(tm_ * TDM, (tm_ + 1) * TDM)
        J = slice(tn_ * TDN, (tn_ + 1) * TDN)
        lt = lam_t[tm_ * tiles_n + tn_]
        delta = 1.25 * lt * U * max(nA[i] * np.linalg.norm(B64[:, J]), np.linalg.norm(A64[I]) * nB[j])
        ratio.append(delta / min(_analytic_tau(A64, B64, i, j, tm_, tn_)))
        faults.append((tm_, tn_, ks, r, c, float(delta)))
    print(f"coherent tiles: learned lambda median {np.median(lam_t):.3g}; "
          f"fault / analytic-threshold ratio: max {max(ratio):.3g}")
    assert max(ratio) < 1.0  # every planted fault sits below the analytic threshold
    _, rep_ana, _, _ = _run(ft, handle, A, B, faults=faults, sink=False)
    handle.set_threshold(1, 2.0 ** margin, th.cpu().numpy())
    _, rep_mlp, _, _ = _run(ft, handle, A, B, faults=faults, sink=False)
    assert rep_ana.detected == 0
    injected = sorted((tm_ * TDM + r, tn_ * TDN + c) for (tm_, tn_, ks, r, c, d) in faults)
    assert sorted((r["row"], r["col"]) for r in rep_mlp.records) == injected
    assert rep_mlp.corrected == len(faults)
    handle.set_threshold(0)

    M = N = 1500
    # (2) zero-mean inputs: each fault is put at 1.25x the larger of its
    #     learned row / column thresholds (the oracle's network on the tile's
    #     features); the gain is that this lies below the analytic threshold
    #     on both sides: missed by the analytic threshold, located by the
    #     learned one
    K = 2048
    A, B = _inputs(orc, "normal", M, N, K, 510)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    nA, nB = np.linalg.norm(A64, axis=1), np.linalg.norm(B64, axis=0)
    tiles_m, tiles_n = -(-M // TDM), -(-N // TDN)
    x_tiles = _oracle_features(A, B, K)
    y_tiles, _ = omlp.forward(th.cpu().numpy().astype(np.float64), x_tiles)
    lam_t = 2.0 ** margin * 2.0 ** y_tiles
    pos = synth.fault_positions(synth.workload_seed("tc_square", 90), 12, tiles_m, tiles_n, 32, TDM, TDN, M, N, 32)
    faults, gain = [], []
    for (tm_, tn_, ks, r, c) in pos:
        I = slice(tm_ * TDM, (tm_ + 1) * TDM)
        J = slice(tn_ * TDN, (tn_ + 1) * TDN)
        i, j = tm_ * TDM + r, tn_ * TDN + c
        row_t, col_t = nA[i] * np.linalg.norm(B64[:, J]), np.linalg.norm(A64[I]) * nB[j]
        lt = lam_t[tm_ * tiles_n + tn_]
        delta = 1.25 * lt * U * max(row_t, col_t)
        gain.append(min(_analytic_tau(A64, B64, i, j, tm_, tn_)) / delta)
        faults.append((tm_, tn_, ks, r, c, float(delta)))
    print(f"learned lambda on zero-mean tiles: median {np.median(lam_t):.3g}; analytic 32; "
          f"fault / analytic-threshold ratio: max {1 / min(gain):.3g}")
    assert min(gain) > 1.0  # every planted fault sits below the analytic threshold
    _, rep_ana, _, _ = _run(ft, handle, A, B, faults=faults, sink=False)
    handle.set_threshold(1, 2.0 ** margin, th.cpu().numpy())
    C, rep_mlp, _, _ = _run(ft, handle, A, B, faults=faults, sink=False)
    handle.set_threshold(0)
    assert rep_ana.detected == 0
    injected = sorted((tm_ * TDM + r, tn_ * TDN + c) for (tm_, tn_, ks, r, c, d) in faults)
    assert sorted((r["row"], r["col"]) for r in rep_mlp.records) == injected
    assert rep_mlp.corrected == len(faults)
    # and C is the fault-free product within the fp32 bound
    ref = orc.gemm_ref(A, B)
    bound = 2 * K * U * (np.abs(A64) @ np.abs(B64))
    assert np.all(np.abs(C.cpu().numpy().astype(np.float64) - ref) <= bound)
