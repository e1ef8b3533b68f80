"""GPU parity of the orthogonalisation steps (Sec. 4, Alg. 3(c): block classical Gram-Schmidt and
CholQR2; the Gram of s-step CG's basis) through the C ABI, against FP64 NumPy products of the same
FP32 (or FP64) data copied to the host.

The stated precision of every Gram product in an FP32 basis: FP32 sums of at most 32 terms per
lane, a fixed FP32 tree of at most eight levels over lanes or row groups, FP64 beyond, so per
entry |G^ - G| <= (40 u32 + m u64) (|X|^T |Y|) with m the FP64 additions (at most n / 1024 +
the partials).  The tests use that bound, with m taken generously."""
import numpy as np
import pytest

from tests.gpu_util import U32, U64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    from paper_2309_02228_gb300 import build
    build.build()
    import paper_2309_02228_gb300 as mod
    torch.cuda.set_device(0)
    return mod


def gram_bound(n):
    """Entrywise bound factor on |G^ - G| / (|X|^T |Y|) for an FP32 basis of n rows."""
    return 40 * U32 + (n / 1024 + 4096) * U64


def _blocks(n, K, seed, kind, dtype=np.float32):
    rng = np.random.default_rng(seed)
    if kind == "positive":          # no cancellation: the accumulation error is all there is
        return (0.5 + 0.5 * rng.random((K, n))).astype(dtype)
    return (2 * rng.random((K, n)) - 1).astype(dtype)      # mixed signs


def _check_gram(G, X, Y, bound):
    X64 = X.astype(np.float64)
    Y64 = Y.astype(np.float64)
    ref = X64 @ Y64.T                                    # K x S, FP64 of the exact FP32 values
    den = np.abs(X64) @ np.abs(Y64).T
    err = np.abs(G - ref) / den
    assert np.all(np.isfinite(err))
    assert float(err.max()) <= bound, float(err.max())
    return float(err.max())


@pytest.mark.parametrize("kind", ["positive", "mixed"])
@pytest.mark.parametrize("K,S", [(49, 8), (17, 4), (145, 16), (1, 1)])
def test_gram_fp32_bound(m, kind, K, S):
    """C = V^T W of the block Gram-Schmidt at the c4 size (n = 128^3 = 2,097,152 rows) and a
    ragged n; every entry within the stated bound relative to |V|^T |W|."""
    import torch
    for n in (2_097_152, 100_003):
        X = _blocks(n, K, 1, kind)
        Y = _blocks(n, S, 2, kind)
        G = m.mpk_gram(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()).cpu().numpy()
        _check_gram(G, X, Y, gram_bound(n))


def test_gram_fp64_and_leading_dimension(m):
    """FP64 blocks sum in FP64 throughout; a leading dimension above n (the solver's padded
    columns) reads only the first n rows."""
    import torch
    n, ld, K, S = 300_001, 300_032, 33, 8
    X = _blocks(ld, K, 3, "mixed", np.float64)
    Y = _blocks(ld, S, 4, "mixed", np.float64)
    G = m.mpk_gram(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), n=n).cpu().numpy()
    _check_gram(G, X[:, :n], Y[:, :n], 64 * U64 + (n / 1024 + 4096) * U64)


@pytest.mark.parametrize("S", [8, 12])
def test_block_update_and_fused_gram(m, S):
    """W <- (W - Q C) Rinv against the FP64 evaluation of the same FP32 data, and the Gram of
    the new W (fused into the update for S <= 8) against the FP64 product of the new W."""
    import torch
    n, K1 = 1_000_003, 17
    rng = np.random.default_rng(5)
    Q = _blocks(n, K1, 6, "mixed")
    W = _blocks(n, S, 7, "mixed")
    C = rng.standard_normal((K1, S)) * 0.1
    R = np.triu(rng.standard_normal((S, S)) * 0.1) + np.eye(S)
    Rinv = np.linalg.inv(R)
    Wd = torch.from_numpy(W.copy()).cuda()
    G = m.mpk_block_update(torch.from_numpy(Q).cuda(), Wd, torch.from_numpy(C), torch.from_numpy(Rinv))
    Wn = Wd.cpu().numpy()
    # the kernel works in FP32 with C and Rinv rounded to FP32
    C32 = C.astype(np.float32).astype(np.float64)
    R32 = np.triu(Rinv.astype(np.float32).astype(np.float64))
    ref = (W.astype(np.float64).T - Q.astype(np.float64).T @ C32) @ R32          # n x S
    den = (np.abs(W.astype(np.float64).T) + np.abs(Q.astype(np.float64).T) @ np.abs(C32)) @ np.abs(R32)
    err = np.abs(Wn.T - ref) / den
    assert float(err.max()) <= (K1 + S + 2) * U32, float(err.max())
    _check_gram(G.cpu().numpy(), Wn, Wn, gram_bound(n))
    # K1 = 0: the normalisation step of CholQR alone (W R^-1)
    Wd2 = torch.from_numpy(W.copy()).cuda()
    G2 = m.mpk_block_update(None, Wd2, None, torch.from_numpy(Rinv))
    W2 = Wd2.cpu().numpy()
    ref2 = W.astype(np.float64).T @ R32
    den2 = np.abs(W.astype(np.float64).T) @ np.abs(R32)
    assert float((np.abs(W2.T - ref2) / den2).max()) <= (S + 2) * U32
    _check_gram(G2.cpu().numpy(), W2, W2, gram_bound(n))


@pytest.mark.parametrize("K,S", [(41, 8), (9, 8), (3, 4), (70, 16)])
@pytest.mark.parametrize("n", [100_003, 257, 2_097_157])
def test_staged_path_ragged_rows(m, K, S, n):
    """FP32 columns padded to a 16-byte multiple (the solver's basis layout) take the staged
    kernels, whose last row block is rounded up and filled with zeros by the copy engine: the
    Gram of a ragged n against the FP64 product, and the block update (with its fused Gram)
    against the FP64 evaluation; rows past n of the output columns stay untouched."""
    import torch
    ld = (n + 31) // 32 * 32
    rng = np.random.default_rng(K * 7 + S)
    Xf = np.zeros((K, ld), np.float32)
    Yf = np.zeros((S, ld), np.float32)
    Xf[:, :n] = _blocks(n, K, 11, "mixed")
    Yf[:, :n] = _blocks(n, S, 12, "mixed")
    Xf[:, n:] = 7.0            # padding rows hold garbage the kernels must not read as data
    Yf[:, n:] = -3.0
    G = m.mpk_gram(torch.from_numpy(Xf).cuda(), torch.from_numpy(Yf).cuda(), n=n).cpu().numpy()
    _check_gram(G, Xf[:, :n], Yf[:, :n], gram_bound(n))
    C = rng.standard_normal((K, S)) * 0.1
    R = np.triu(rng.standard_normal((S, S)) * 0.1) + np.eye(S)
    Rinv = np.linalg.inv(R)
    Wd = torch.from_numpy(Yf.copy()).cuda()
    G2 = m.mpk_block_update(torch.from_numpy(Xf).cuda(), Wd, torch.from_numpy(C), torch.from_numpy(Rinv), n=n,
                            gram=S <= 8)
    Wn = Wd.cpu().numpy()
    assert np.array_equal(Wn[:, n:], Yf[:, n:])
    C32 = C.astype(np.float32).astype(np.float64)
    R32 = np.triu(Rinv.astype(np.float32).astype(np.float64))
    W64, Q64 = Yf[:, :n].astype(np.float64).T, Xf[:, :n].astype(np.float64).T
    ref = (W64 - Q64 @ C32) @ R32
    den = (np.abs(W64) + np.abs(Q64) @ np.abs(C32)) @ np.abs(R32)
    assert float((np.abs(Wn[:, :n].T - ref) / den).max()) <= (K + S + 2) * U32
    if S <= 8:
        _check_gram(G2.cpu().numpy(), Wn[:, :n], Wn[:, :n], gram_bound(n))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("s,n", [(8, 1_000_000), (3, 257), (15, 300_001), (1, 99_999), (10, 200_003), (12, 168 * 1001)])
def test_gram_pairs(m, dtype, s, n):
    """The CG basis Gram over the 2s + 2 storage columns in pair order, ragged n included."""
    import torch
    ldv = (n + 31) // 32 * 32
    M = 2 * s + 2
    rng = np.random.default_rng(s * 1000 + n % 997)
    cols = (2 * rng.random((M, n)) - 1).astype(dtype)        # storage column c = 2k + q
    Y = np.zeros((s + 1, ldv, 2), dtype=dtype)
    for c in range(M):
        Y[c // 2, :n, c % 2] = cols[c]
    G = m.mpk_gram_pairs(torch.from_numpy(Y.reshape(-1)).cuda(), s, n, ldv).cpu().numpy()
    bound = gram_bound(n) if dtype == np.float32 else 64 * U64 + (n / 1024 + 4096) * U64
    _check_gram(G, cols, cols, bound)
    assert np.array_equal(G, G.T)


def test_invalid_arguments(m):
    import torch
    X = torch.zeros((2, 64), device="cuda")
    with pytest.raises(m.MpkError):
        m.mpk_gram(X, torch.zeros((17, 64), device="cuda"))            # S > 16
    with pytest.raises(m.MpkError):
        m.mpk_gram_pairs(torch.zeros(3 * 2 * 65, device="cuda"), 2, 64, 65)   # FP32 ldv odd
