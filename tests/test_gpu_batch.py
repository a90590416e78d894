"""GPU tests of the batched path (arrow_batch_spmm): many matrices, one launch per kernel class.

Each matrix of a batch must give exactly the bits of arrow_spmm on it alone (same row
arithmetic, fixed order), in eager mode and replayed from a CUDA graph, and must match the
FP64 oracle within the 16-bit tolerance (normwise 2e-2) or the FP32 one (1e-5 * iters).
"""
import numpy as np
import pytest

import workloads as w
from oracle import spmm as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def arrow():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_19364_gb300 import build
    build.build()
    import paper_2402_19364_gb300 as pkg
    return pkg


def _rgg_batch(count, seed, lo=1000, hi=20000):
    sizes = w.log_uniform_sizes(count, lo, hi, seed)
    rng = np.random.default_rng(seed)
    ks = rng.choice([8, 16, 32, 64], count)
    mats = [w.rgg(int(n), seed=seed * 1000 + i) for i, n in enumerate(sizes)]
    return mats, [int(k) for k in ks]


def test_batch_equals_single_rgg_fp16(arrow):
    mats, ks = _rgg_batch(12, 7)
    ms = [arrow.ArrowMatrix(A, int(np.ceil(np.sqrt(A.n))), value_dtype="f16") for A in mats]
    Xs = [torch.from_numpy(w.features(A.n, k, seed=i)).to("cuda", torch.float16) for i, (A, k) in enumerate(zip(mats, ks))]
    B = arrow.ArrowBatch(ms)
    iters = 10
    Ys = B.spmm(Xs, iters)
    Yg = B.spmm(Xs, iters, graph=True)
    Yg2 = B.spmm(Xs, iters, graph=True)                  # replay
    torch.cuda.synchronize()
    assert B.status() == 0
    for A, M, X, Y, G, G2, k in zip(mats, ms, Xs, Ys, Yg, Yg2, ks):
        ref = M.spmm(X, iters)
        torch.cuda.synchronize()
        assert torch.equal(Y, ref) and torch.equal(G, ref) and torch.equal(G2, ref)
        R = S.iterate(A, X.float().cpu().numpy().astype(np.float64), iters)
        Yn = Y.float().cpu().numpy().astype(np.float64)
        assert np.max(np.linalg.norm(Yn - R, axis=0) / np.linalg.norm(R, axis=0)) <= 2e-2


def test_batch_mixed_families_split_rows_fp32(arrow):
    # grid, power-law (split head rows), random-geometric and an empty matrix in one batch
    mats = [w.grid3d(14, seed=2), w.rmat_gcn(11, 16, seed=4), w.rgg(3000, seed=9),
            w.Csr(100, np.zeros(101, np.int64), np.zeros(0, np.int32), np.zeros(0))]
    bs = [64, 64, 55, 8]
    ks = [16, 32, 8, 4]
    ms = [arrow.ArrowMatrix(A, b, long_row=16, segment=64) for A, b in zip(mats, bs)]
    assert ms[1].stats()["segments"] > 0
    Xs = [torch.from_numpy(w.features(A.n, k, seed=3 + i)).cuda() for i, (A, k) in enumerate(zip(mats, ks))]
    B = arrow.ArrowBatch(ms)
    iters = 5
    Ys = B.spmm(Xs, iters, graph=True)
    torch.cuda.synchronize()
    for A, M, X, Y in zip(mats, ms, Xs, Ys):
        assert torch.equal(Y, M.spmm(X, iters))
        R = S.iterate(A, X.cpu().numpy().astype(np.float64), iters)
        if A.nnz:
            Yn = Y.cpu().numpy().astype(np.float64)
            assert np.max(np.max(np.abs(Yn - R), axis=0) / np.max(np.abs(R), axis=0)) <= 1e-5 * iters
        else:
            assert torch.count_nonzero(Y).item() == 0


def test_batch_argument_errors(arrow):
    A = w.grid2d_64()
    M = arrow.ArrowMatrix(A, 64)
    B = arrow.ArrowBatch([M])
    with pytest.raises(arrow.ArrowError):
        B.spmm([torch.zeros(A.n, 12, device="cuda")], 1)            # k / V not a power of two
    Mh = arrow.ArrowMatrix(A, 64, host_only=True)
    with pytest.raises(arrow.ArrowError):
        arrow.ArrowBatch([Mh])                                       # not uploaded
    Mc = M.copy("bf16")
    with pytest.raises(arrow.ArrowError):
        arrow.ArrowBatch([M, Mc])                                    # mixed value dtypes


def test_handle_copy_same_structure(arrow):
    A = w.rmat_gcn(10, 16, seed=3)
    M = arrow.ArrowMatrix(A, 32)
    C = M.copy("f16")
    assert C.num_levels == M.num_levels
    for i in range(M.num_levels):
        assert np.array_equal(C.level_perm(i), M.level_perm(i))
    X = torch.from_numpy(w.features(A.n, 16, seed=1)).cuda()
    Yf = M.spmm(X, 3)
    Yh = C.spmm(X.half(), 3).float()
    assert torch.linalg.vector_norm(Yh - Yf) / torch.linalg.vector_norm(Yf) < 2e-2


def test_tunings_give_same_bits_and_autotune_keeps_one(arrow):
    # the row arithmetic does not depend on the tiling; the FP64 norm sums are grouped by
    # CTA, so with the rescale the results agree within the FP32 tolerance instead
    A = w.grid3d(40, seed=5)
    M = arrow.ArrowMatrix(A, 512)
    X = torch.from_numpy(w.features(A.n, 16, seed=2)).cuda()
    ref = M.spmm(X, 5)
    ref_r = M.spmm(X, 5, rescale=True)
    for tr, tn, c, co in ((128, 1024, 2, 40), (512, 4096, 3, 100), (256, 2048, 1, 30)):
        M.set_tuning(tr, tn, c, co)
        assert torch.equal(M.spmm(X, 5), ref)
        Yr = M.spmm(X, 5, rescale=True)
        assert float(((Yr - ref_r).abs().max(0).values / ref_r.abs().max(0).values).max()) <= 5e-5
    best, ms = M.autotune(X, 5, rescale=True)
    assert ms > 0 and best == M.tuning
    assert torch.equal(M.spmm(X, 5), ref)


def test_batch_autotune(arrow):
    mats, ks = _rgg_batch(6, 3)
    ms = [arrow.ArrowMatrix(A, int(np.ceil(np.sqrt(A.n))), value_dtype="f16") for A in mats]
    Xs = [torch.from_numpy(w.features(A.n, k, seed=i)).to("cuda", torch.float16) for i, (A, k) in enumerate(zip(mats, ks))]
    B = arrow.ArrowBatch(ms)
    ref = [y.clone() for y in B.spmm(Xs, 4, graph=True)]
    best, t = B.autotune(Xs, 4)
    assert t > 0 and all(m.tuning == best for m in ms)
    for y, r in zip(B.spmm(Xs, 4, graph=True), ref):
        assert torch.equal(y, r)


def test_member_retuned_after_batch_creation(arrow):
    # re-tiling a member handle changes its tile count and frees its old tile table; the
    # batch must notice on its next call and rebuild its work-unit tables and descriptors
    mats, ks = _rgg_batch(5, 21)
    ms = [arrow.ArrowMatrix(A, int(np.ceil(np.sqrt(A.n))), value_dtype="f16") for A in mats]
    Xs = [torch.from_numpy(w.features(A.n, k, seed=i)).to("cuda", torch.float16) for i, (A, k) in enumerate(zip(mats, ks))]
    B = arrow.ArrowBatch(ms)
    ref = [y.clone() for y in B.spmm(Xs, 3, graph=True)]
    for shape in ((512, 4096, 3, 97), (128, 1024, 2, 40)):
        for M in ms:
            M.set_tuning(*shape)
        for graph in (False, True):
            Ys = B.spmm(Xs, 3, graph=graph)
            torch.cuda.synchronize()
            assert B.status() == 0
            assert all(torch.equal(y, r) for y, r in zip(Ys, ref))
