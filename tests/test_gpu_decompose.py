"""GPU steps of LA-Decompose (ARROW_DEVICE_DECOMPOSE) against the host decomposer.

The degrees, the edges of G_i' with their keys, the minimum spanning forest (Boruvka) and
the split by the arrow shape run on the GPU; the head choice and the tree layout stay on
the host.  The spanning forest is unique (distinct keys) and every other step is a fixed
function of its inputs, so the decomposition must equal the host path's bit for bit:
every level's permutation, CSR (columns and values), active rows, nnz, and the fused row
program; and the host path is bit-exact with the oracle (tests/test_abi_host.py), so the
device path is too.  A product through the device-decomposed handle is checked against the
oracle as well.
"""
import numpy as np
import pytest

import workloads as w
from oracle import decompose as D
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


def _star(n=300):
    rows = np.r_[np.zeros(n - 1, np.int64), np.arange(1, n), np.arange(n)]
    cols = np.r_[np.arange(1, n), np.zeros(n - 1, np.int64), np.arange(n)]
    rp, ci = w._csr_from_pairs(n, rows, cols)
    return w.Csr(n, rp, ci, np.linspace(0.5, 1.5, ci.size))


CASES = {
    "grid2d_64": (lambda: w.grid2d_64(), 64, {}),
    "grid3d_40": (lambda: w.grid3d(40, seed=3), 400, {}),
    "rmat14_split": (lambda: w.rmat_gcn(14, 16, seed=5), 256, {"long_row": 32, "segment": 64}),
    "rgg": (lambda: w.rgg(20000, seed=7), 142, {}),
    "nonsym": (lambda: w.random_csr(3000, 0.002, 8), 16, {}),
    "star": (lambda: _star(), 2, {}),
    "empty": (lambda: w.Csr(100, np.zeros(101, np.int64), np.zeros(0, np.int32), np.zeros(0)), 8, {}),
    "b_ge_n": (lambda: w.random_csr(50, 0.1, 1, symmetric=True, diag=True), 64, {}),
}


def _same_decomposition(Mh, Md):
    assert Mh.num_levels == Md.num_levels
    for i in range(Mh.num_levels):
        assert np.array_equal(Mh.level_perm(i), Md.level_perm(i))
        assert Mh.level_info(i) == Md.level_info(i)
        a, b = Mh.level_csr(i), Md.level_csr(i)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    ph, pd = Mh.program(), Md.program()
    for key in ph:
        assert np.array_equal(np.asarray(ph[key]), np.asarray(pd[key])), key


@pytest.mark.parametrize("pred", ["block", "band"])
@pytest.mark.parametrize("case", list(CASES))
def test_device_decomposition_equals_host(arrow, case, pred):
    make, b, kw = CASES[case]
    A = make()
    for seed in (0, 12345):
        Mh = arrow.ArrowMatrix(A, b, seed=seed, predicate=pred, host_only=True, **kw)
        Md = arrow.ArrowMatrix(A, b, seed=seed, predicate=pred, device_decompose=True, **kw)
        _same_decomposition(Mh, Md)
        Mh.close()
        Md.close()


def test_device_decomposition_matches_oracle_and_computes(arrow):
    A = w.rmat_gcn(11, 16, seed=2)
    Md = arrow.ArrowMatrix(A, 64, seed=7, device_decompose=True, long_row=16, segment=32)
    L = D.la_decompose(A, 64, seed=7)
    assert Md.num_levels == len(L)
    for i, lv in enumerate(L):
        assert np.array_equal(Md.level_perm(i), lv.perm)
    X = w.features(A.n, 32, seed=3)
    Y = Md.spmm(torch.from_numpy(X).cuda(), 4).cpu().numpy().astype(np.float64)
    R = S.iterate(A, X, 4)
    assert float(np.max(np.max(np.abs(Y - R), axis=0) / np.max(np.abs(R), axis=0))) <= 4e-5


def test_device_decomposition_argument_errors(arrow):
    from paper_2402_19364_gb300 import _native
    with pytest.raises(arrow.ArrowError) as e:
        arrow.ArrowMatrix(w.grid2d_64(), 64, host_only=True, device_decompose=True)
    assert e.value.code == _native.ARROW_EINVAL
