"""GPU tests of the continuous-batching server (arrow_server_*).

Requests from three matrix families, with different widths and iteration counts, arrive
while others are on the GPU.  Each result must equal, bit for bit, the same request run
alone through arrow_spmm (the per-row arithmetic does not depend on what shares a launch),
and must match the FP64 oracle within the BF16 tolerance (normwise 2e-2).  A small memory
budget forces admission to wait; the peak use must stay within it.
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


@pytest.fixture(scope="module")
def pool(arrow):
    mats = [w.grid3d(18, seed=1), w.rmat_gcn(11, 16, seed=2), w.rgg(4000, seed=3), w.grid_stencil((50, 41), seed=4)]
    bs = [64, 64, 64, 41]
    hs = [arrow.ArrowMatrix(A, b, value_dtype="bf16", long_row=32, segment=128) for A, b in zip(mats, bs)]
    assert hs[1].stats()["segments"] > 0
    return mats, hs


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(0, 4)), int(rng.choice([16, 32, 64, 128])), int(rng.integers(0, 13))) for _ in range(count)]


def test_mix_equals_alone(arrow, pool):
    mats, hs = pool
    reqs = _requests(40, 11)
    srv = arrow.ArrowServer(hbm_budget=1 << 30, max_active=16, x_dtype="bf16")
    gen = torch.Generator(device="cuda").manual_seed(5)
    Xs, Ys, ids = [], [], []
    for i, (m, k, it) in enumerate(reqs):
        X = torch.randn(mats[m].n, k, device="cuda", generator=gen).bfloat16()
        Y = torch.full_like(X, float("nan"))
        Xs.append(X)
        Ys.append(Y)
        ids.append(srv.submit(hs[m], X, Y, it))
        if i % 7 == 6:                                   # requests arrive while others run
            for _ in range(3):
                srv.step()
    srv.drain()
    done = dict(srv.poll())
    assert sorted(done) == sorted(ids)
    assert all(v >= 0 for v in done.values())
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["active"] == 0 and st["queued"] == 0 and st["status"] == 0
    torch.cuda.synchronize()
    for (m, k, it), X, Y in zip(reqs, Xs, Ys):
        alone = hs[m].spmm(X, it)
        torch.cuda.synchronize()
        assert torch.equal(Y, alone), (m, k, it)
    for (m, k, it), X, Y in list(zip(reqs, Xs, Ys))[:6]:
        if it == 0:
            continue
        R = S.iterate(mats[m], X.float().cpu().numpy().astype(np.float64), it)
        Yn = Y.float().cpu().numpy().astype(np.float64)
        assert np.max(np.linalg.norm(Yn - R, axis=0) / np.linalg.norm(R, axis=0)) <= 2e-2


def test_admission_by_memory_budget(arrow, pool):
    mats, hs = pool
    reqs = [(m, 64, 5) for m in (0, 1, 2, 3, 0, 1, 2, 3)]
    per = [2 * ((mats[m].n * 64 * 2 + 255) // 256 * 256) for m, _, _ in reqs]
    budget = int(max(per) * 2.2 + (1 << 20))            # about two requests at a time
    srv = arrow.ArrowServer(hbm_budget=budget, max_active=64, x_dtype="bf16")
    Xs, Ys = [], []
    for m, k, it in reqs:
        X = torch.randn(mats[m].n, k, device="cuda").bfloat16()
        Y = torch.empty_like(X)
        Xs.append(X)
        Ys.append(Y)
        srv.submit(hs[m], X, Y, it)
    seen_active = 0
    while srv.stats()["queued"] or srv.stats()["active"]:
        seen_active = max(seen_active, srv.step())
    srv.drain()
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["peak_bytes"] <= budget and seen_active < len(reqs)
    for (m, k, it), X, Y in zip(reqs, Xs, Ys):
        assert torch.equal(Y, hs[m].spmm(X, it))


def test_server_argument_errors(arrow, pool):
    mats, hs = pool
    srv = arrow.ArrowServer(hbm_budget=1 << 20, max_active=4, x_dtype="bf16")
    X = torch.zeros(mats[0].n, 12, device="cuda").bfloat16()
    with pytest.raises(arrow.ArrowError):
        srv.submit(hs[0], X, X.clone(), 3)                              # k = 12: not V * 2^j
    big = torch.zeros(mats[0].n, 128, device="cuda").bfloat16()
    with pytest.raises(arrow.ArrowError):
        srv.submit(hs[0], big, big.clone(), 3)                          # larger than the whole budget
    Mf = arrow.ArrowMatrix(mats[3], 41)                                 # f32 values
    X3 = torch.zeros(mats[3].n, 16, device="cuda").bfloat16()
    srv.submit(hs[3], X3, X3.clone(), 1)
    with pytest.raises(arrow.ArrowError):
        srv.submit(Mf, X3, X3.clone(), 1)                               # mixed value dtypes
    srv.drain()
