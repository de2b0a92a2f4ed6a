"""Parity of the single-instance entry points (te_embed, te_knn_maxnorm, te_range_count)
with the CPU oracle, through the C ABI: coordinates, kNN radii, neighbour lists and counts
must be bit-exact. Sizes span several shared-memory tiles (256 references) with ragged tails,
the supported joint dimensions (exact kernels) and other D (padded kernels), tie-heavy
integer data and the degenerate cases (N = k + 1, empty marginal groups, duplicates)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu


def _soa(points_aos: np.ndarray):
    """AoS [N][D] -> device SoA [D][ld] with ld a multiple of 4 (padding filled with junk)."""
    N, D = points_aos.shape
    ld = ((N + 3) // 4) * 4 + 4
    buf = np.full((D, ld), 12345.0, np.float32)
    buf[:, :N] = points_aos.T
    return torch.from_numpy(buf).cuda(), ld


def _points(kind, N, D, seed):
    rng = np.random.default_rng(seed)
    if kind == "gauss":
        return rng.standard_normal((N, D)).astype(np.float32)
    if kind == "int":  # few distinct values: many exact ties
        return rng.integers(0, 5, size=(N, D)).astype(np.float32)
    if kind == "dup":  # heavy duplication of whole points
        base = rng.standard_normal((max(2, N // 7), D)).astype(np.float32)
        return base[rng.integers(0, base.shape[0], size=N)]
    raise ValueError(kind)


# ---------------------------------------------------------------- embedding
@pytest.mark.parametrize("d,tau,u,t_start,W,perm", [
    (1, 1, 1, 1, 1, False), (2, 1, 5, 10, 5, False), (3, 2, 5, 9, 3, True),
    (5, 1, 5, 9, 3, True), (4, 3, 7, 30, 2, True), (7, 2, 2, 40, 4, False)])
def test_embed_bit_exact(te_handle, d, tau, u, t_start, W, perm):
    rng = np.random.default_rng(3)
    R, T = 37, 60
    src = rng.standard_normal((R, T)).astype(np.float32)
    tgt = rng.standard_normal((R, T)).astype(np.float32)
    p = rng.permutation(R).astype(np.int32) if perm else None
    ref = oracle.embed(src, tgt, d, tau, u, t_start, W, p)
    pts, N, D, ld = te.te_embed(te_handle, torch.from_numpy(src).cuda(), torch.from_numpy(tgt).cuda(),
                                d, tau, u, t_start, W, None if p is None else torch.from_numpy(p).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pts[:, :N].cpu().numpy().T, ref)


def test_embed_range_error(te_handle):
    src = torch.zeros((4, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(te.TEError, match="TE_ERANGE"):
        te.te_embed(te_handle, src, src, 2, 3, 5, 6, 1)
    with pytest.raises(te.TEError, match="TE_ERANGE"):
        te.te_embed(te_handle, src, src, 1, 1, 1, 18, 3)


def test_embed_bad_perm_is_flagged(te_handle):
    src = torch.zeros((4, 20), dtype=torch.float32, device="cuda")
    perm = torch.tensor([0, 1, 2, 9], dtype=torch.int32, device="cuda")
    te.te_embed(te_handle, src, src, 1, 1, 1, 5, 2, perm)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_sync_status(te_handle)
    te.te_sync_status(te_handle)  # the flag was cleared


# ---------------------------------------------------------------- kNN radii
KNN_CASES = []
for D in (3, 5, 7, 9, 11):          # exact-dimension kernels
    for N in (5, 17, 257, 1030):
        KNN_CASES.append(("gauss", N, D, 4))
for D in (1, 2, 4, 6, 8, 12, 17, 32):  # padded kernels
    KNN_CASES.append(("gauss", 300, D, 4))
for k in (1, 2, 5, 8, 16):
    KNN_CASES.append(("gauss", 600, 7, k))
    KNN_CASES.append(("int", 300, 5, k))
KNN_CASES += [("int", 1500, 7, 4), ("dup", 513, 7, 4), ("dup", 200, 4, 3), ("gauss", 5, 7, 4),
              ("gauss", 2, 3, 1), ("int", 2600, 11, 4)]


@pytest.mark.parametrize("kind,N,D,k", KNN_CASES)
def test_knn_eps_bit_exact(te_handle, kind, N, D, k):
    P = _points(kind, N, D, N * 31 + D * 7 + k)
    ref = oracle.knn(P, k)
    dev, ld = _soa(P)
    eps = te.te_knn_maxnorm(te_handle, dev, N, D, ld, k)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(eps.cpu().numpy(), ref)


@pytest.mark.parametrize("kind,N,D,k", [("int", 200, 3, 4), ("int", 300, 7, 1), ("dup", 257, 5, 6),
                                        ("int", 40, 2, 16), ("gauss", 700, 9, 4), ("int", 6, 3, 5)])
def test_knn_neighbour_lists(te_handle, kind, N, D, k):
    P = _points(kind, N, D, 17 + N + k)
    ref_eps, ref_nn = oracle.knn(P, k, want_nn=True)
    dev, ld = _soa(P)
    eps, nn = te.te_knn_maxnorm(te_handle, dev, N, D, ld, k, want_nn=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(eps.cpu().numpy(), ref_eps)
    np.testing.assert_array_equal(nn.cpu().numpy(), ref_nn)


def test_knn_argument_errors(te_handle):
    dev, ld = _soa(_points("gauss", 10, 3, 1))
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_knn_maxnorm(te_handle, dev, 10, 3, ld, 10)   # k = N
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_knn_maxnorm(te_handle, dev, 10, 3, ld, 17)   # k > 16
    wide = torch.zeros((33, ld), dtype=torch.float32, device="cuda")
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_knn_maxnorm(te_handle, wide, 10, 33, ld, 4)  # D > 32
    with pytest.raises(ValueError, match="points"):        # the binding: 3 x ld floats for D = 5
        te.te_knn_maxnorm(te_handle, dev, 10, 5, ld, 4)
    with pytest.raises(ValueError, match="eps"):
        te.te_knn_maxnorm(te_handle, dev, 10, 3, ld, 4, eps=torch.zeros(9, dtype=torch.float32, device="cuda"))
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_knn_maxnorm(te_handle, dev, 10, 3, 6, 4)     # ld not a multiple of 4


# ---------------------------------------------------------------- range counts
COUNT_CASES = []
for d in (1, 2, 3, 4, 5):
    for N in (9, 257, 1111):
        COUNT_CASES.append(("gauss", N, d, d, 4))
COUNT_CASES += [("int", 800, 3, 3, 4), ("dup", 600, 2, 2, 4), ("gauss", 300, 0, 2, 4),
                ("gauss", 300, 2, 0, 4), ("int", 300, 1, 3, 2), ("gauss", 500, 6, 6, 4),
                ("gauss", 257, 3, 12, 8), ("int", 97, 0, 0, 3)]


@pytest.mark.parametrize("kind,N,dy,dx,k", COUNT_CASES)
def test_range_count_bit_exact(te_handle, kind, N, dy, dx, k):
    D = 1 + dy + dx
    P = _points(kind, N, D, 1000 + N + 10 * dy + dx)
    eps = oracle.knn(P, k)
    ref = oracle.range_count(P, dy, dx, eps)
    dev, ld = _soa(P)
    g = te.te_range_count(te_handle, dev, N, dy, dx, ld, torch.from_numpy(eps).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g.cpu().numpy(), ref)


def test_knn_then_count_pipeline_matches_oracle_te(te_handle):
    rng = np.random.default_rng(5)
    src = rng.standard_normal((150, 80)).astype(np.float32)
    tgt = rng.standard_normal((150, 80)).astype(np.float32)
    ref_te, ref_eps, ref_c = oracle.te_points(oracle.embed(src, tgt, 3, 2, 4, 20, 6), 3, 3, 4)
    pts, N, D, ld = te.te_embed(te_handle, torch.from_numpy(src).cuda(), torch.from_numpy(tgt).cuda(),
                                3, 2, 4, 20, 6)
    eps = te.te_knn_maxnorm(te_handle, pts, N, D, ld, 4)
    c = te.te_range_count(te_handle, pts, N, 3, 3, ld, eps)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(eps.cpu().numpy(), ref_eps)
    np.testing.assert_array_equal(c.cpu().numpy(), ref_c)
