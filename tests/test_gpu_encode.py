"""The encoding pass on its own (ftgemm_encode, Eq. 1-2): e^T A per block of
m_u rows, B e per block of n_u columns, row norms of A and column norms of B,
against the oracle.  Integer inputs make every sum exact, so the block sums
must match bit for bit and the norms to the rounding of one square root."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ft():
    import torch
    import paper_2305_01024_gb300 as ft
    assert torch.cuda.is_available()
    ft.lib()
    return ft


def _encode(ft, h, A, B, m_u, n_u, lda=None):
    import torch
    M, K = A.shape
    N = B.shape[1]
    if lda is None:
        dA = torch.from_numpy(A).cuda()
    else:  # a row-strided view: A inside a wider buffer
        buf = torch.zeros(M, lda, dtype=torch.float32, device="cuda")
        buf[:, :K] = torch.from_numpy(A).cuda()
        dA = buf[:, :K]
    dB = torch.from_numpy(B).cuda()
    V = torch.empty(-(-M // m_u), K, device="cuda")
    W = torch.empty(-(-N // n_u), K, device="cuda")
    nA, nB = torch.empty(M, device="cuda"), torch.empty(N, device="cuda")
    h.encode(dA, dB, m_u, n_u, V, W, nA, nB)
    torch.cuda.synchronize()
    return V.cpu().numpy(), W.cpu().numpy(), nA.cpu().numpy(), nB.cpu().numpy()


@pytest.mark.parametrize("shape,m_u,n_u,lda", [((300, 260, 520), 128, 64, None),
                                              ((5, 7, 13), 2, 1024, None),
                                              ((1000, 33, 777), 1024, 2, None),
                                              ((130, 140, 250), 64, 128, 257)])
def test_encode_integers_exact(ft, orc, shape, m_u, n_u, lda):
    M, N, K = shape
    A = synth.integers((M, K), 700 + M)
    B = synth.integers((K, N), 701 + N)
    h = ft.Handle(0)
    V, W, nA, nB = _encode(ft, h, A, B, m_u, n_u, lda)
    h.close()
    Vo, Wo, nAo, nBo = orc.encode(A, B, m_u, n_u)
    assert np.array_equal(V, Vo) and np.array_equal(W, Wo)
    np.testing.assert_array_max_ulp(nA, nAo.astype(np.float32), maxulp=1)
    np.testing.assert_array_max_ulp(nB, nBo.astype(np.float32), maxulp=1)


def test_encode_float_inputs(ft, orc):
    M, N, K = 640, 384, 2048
    A = synth.normal((M, K), 711)
    B = synth.normal((K, N), 712)
    h = ft.Handle(0)
    V, W, nA, nB = _encode(ft, h, A, B, 128, 128)
    h.close()
    Vo, Wo, nAo, nBo = orc.encode(A, B, 128, 128)
    # fp32 sums of 128 terms against fp64: within 128 u of the sum of |terms|
    absA = np.add.reduceat(np.abs(A.astype(np.float64)), np.arange(0, M, 128), axis=0)
    absB = np.add.reduceat(np.abs(B.astype(np.float64)), np.arange(0, N, 128), axis=1).T
    u = 2.0 ** -24
    assert np.all(np.abs(V - Vo) <= 128 * u * absA)
    assert np.all(np.abs(W - Wo) <= 128 * u * absB)
    assert np.allclose(nA, nAo, rtol=4 * K * u, atol=0) and np.allclose(nB, nBo, rtol=4 * K * u, atol=0)
