"""GPU parity: arrow_spmm (through the C-ABI) against the FP64 oracle.

Tolerances (stated per dtype, the accuracy bar of the arrow-SpMM workloads):
  * FP32 values and features: max over columns j of
        ||y_j - y_ref,j||_inf / ||y_ref,j||_inf  <=  1e-5 * iters
  * BF16 / FP16 storage, FP32 accumulation: max_j ||y_j - y_ref,j||_2 / ||y_ref,j||_2 <= 2e-2
The oracle is the plain FP64 product iterated (Eq. 1 is an identity), run on
the same seeded inputs; no expected value comes from the GPU.
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


TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def err_inf(Y, R):
    return float(np.max(np.max(np.abs(Y - R), axis=0) / np.max(np.abs(R), axis=0)))


def err_2(Y, R):
    return float(np.max(np.linalg.norm(Y - R, axis=0) / np.linalg.norm(R, axis=0)))


def run(arrow, A, b, X, iters, dt="f32", vdt=None, rescale=False, **kw):
    M = arrow.ArrowMatrix(A, b, value_dtype=vdt or dt, **kw)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to("cuda", TORCH_DT[dt])
    Y = M.spmm(Xd, iters, rescale=rescale)
    torch.cuda.synchronize()
    return M, Xd, Y.float().cpu().numpy().astype(np.float64)


def test_grid2d_64_fp32_ten_iterations(arrow):
    # 2D 64x64 grid, 5-point stencil, U(0.5,1.5) row-normalised f32, b = 64, X 4096x16 N(0,1), 10 iterations
    A = w.grid2d_64(seed=1)
    X = w.features(A.n, 16, seed=2)
    M, _, Y = run(arrow, A, 64, X, 10)
    assert M.num_levels >= 2
    assert err_inf(Y, S.iterate(A, X, 10)) <= 1e-5 * 10


def test_grid3d_rescale_fp64_norms(arrow):
    # 3D 7-point grid with the per-iteration FP64 column-norm rescale (scaled-down 400^3 workload)
    A = w.grid3d(24, seed=3)
    X = w.features(A.n, 16, seed=4)
    _, _, Y = run(arrow, A, 96, X, 20, rescale=True)
    R = S.iterate(A, X, 20, rescale=True)
    assert err_inf(Y, R) <= 1e-5 * 20
    assert np.allclose(np.linalg.norm(Y, axis=0), 1.0, atol=1e-5)


@pytest.mark.parametrize("dt,k", [("f32", 4), ("f32", 8), ("f32", 16), ("f32", 32), ("f32", 64), ("f32", 128),
                                  ("f32", 256), ("bf16", 8), ("bf16", 16), ("bf16", 64), ("bf16", 128),
                                  ("bf16", 512), ("f16", 8), ("f16", 32), ("f16", 256)])
def test_power_law_split_rows_all_widths(arrow, dt, k):
    # R-MAT GCN matrix; long_row / segment small so head rows and many band rows are split
    A = w.rmat_gcn(11, 16, seed=5)
    X = w.features(A.n, k, seed=6)
    iters = 4
    M, _, Y = run(arrow, A, 64, X, iters, dt=dt, long_row=16, segment=32)
    assert M.stats()["segments"] > 0
    R = S.iterate(A, X, iters)
    if dt == "f32":
        assert err_inf(Y, R) <= 1e-5 * iters
    else:
        assert err_2(Y, R) <= 2e-2


def test_bf16_values_against_fp32_and_fp64(arrow):
    # power-law workload: BF16 A and X with FP32 accumulation vs the FP32 path and the FP64 oracle
    A = w.rmat_gcn(13, 16, seed=5)
    X = w.features(A.n, 128, seed=6)
    iters = 8
    R = S.iterate(A, X, iters)
    _, _, Yb = run(arrow, A, 256, X, iters, dt="bf16")
    _, _, Yf = run(arrow, A, 256, X, iters, dt="f32")
    assert err_inf(Yf, R) <= 1e-5 * iters
    assert err_2(Yb, R) <= 2e-2
    assert err_2(Yb, Yf) <= 2e-2
    # bf16 features with f32 values
    _, _, Ym = run(arrow, A, 256, X, iters, dt="bf16", vdt="f32")
    assert err_2(Ym, R) <= 2e-2


@pytest.mark.parametrize("k", [8, 16, 32, 64])
def test_rgg_fp16(arrow, k):
    A = w.rgg(6000, seed=7)
    b = int(np.ceil(np.sqrt(A.n)))
    X = w.features(A.n, k, seed=8)
    _, _, Y = run(arrow, A, b, X, 10, dt="f16")
    assert err_2(Y, S.iterate(A, X, 10)) <= 2e-2


@pytest.mark.parametrize("case", ["grid2d", "grid3d_rescale", "rmat_split_bf16", "rgg_f16"])
def test_band_predicate_device_path(arrow, case):
    """The band predicate of Section 1 (|p - q| <= b) on the device, against the oracle, and
    against the block predicate's result on the same inputs (both are A X)."""
    if case == "grid2d":
        A, b, X, it, dt, kw, rs = w.grid2d_64(seed=1), 64, w.features(4096, 16, seed=2), 10, "f32", {}, False
    elif case == "grid3d_rescale":
        A = w.grid3d(24, seed=3)
        b, X, it, dt, kw, rs = 96, w.features(A.n, 16, seed=4), 20, "f32", {}, True
    elif case == "rmat_split_bf16":
        A = w.rmat_gcn(12, 16, seed=5)
        b, X, it, dt, kw, rs = 64, w.features(A.n, 64, seed=6), 4, "bf16", {"long_row": 16, "segment": 64}, False
    else:
        A = w.rgg(6000, seed=7)
        b, X, it, dt, kw, rs = 78, w.features(A.n, 32, seed=8), 10, "f16", {}, False
    Mb, _, Yb = run(arrow, A, b, X, it, dt=dt, rescale=rs, predicate="band", **kw)
    Mk, _, Yk = run(arrow, A, b, X, it, dt=dt, rescale=rs, **kw)
    R = S.iterate(A, X, it, rescale=rs)
    if dt == "f32":
        assert err_inf(Yb, R) <= 1e-5 * it
        assert err_inf(Yb, Yk) <= 2e-5 * it
    else:
        assert err_2(Yb, R) <= 2e-2
    # every entry lands in one level of the band decomposition
    assert sum(Mb.level_info(i)[1] for i in range(Mb.num_levels)) == A.nnz
    Mb2 = arrow.ArrowMatrix(A, b, value_dtype=dt, predicate="band", **kw)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to("cuda", TORCH_DT[dt])
    assert torch.equal(Mb.spmm(Xd, it, rescale=rs), Mb2.spmm(Xd, it, rescale=rs))   # fixed order


@pytest.mark.parametrize("dt,k,relu,rownorm,rescale", [
    ("f32", 16, True, False, False), ("f32", 16, False, True, False), ("f32", 32, True, True, True),
    ("f32", 128, True, True, False), ("bf16", 64, True, False, False), ("bf16", 256, False, True, True),
    ("f16", 8, True, True, False)])
def test_sigma_epilogues(arrow, dt, k, relu, rownorm, rescale):
    """sigma = colnorm(rownorm(relu(.))) fused into the row stores, on a grid and on a power-law
    matrix whose hub rows are split (their rows are written by the combine kernel)."""
    iters = 5
    for A, b, kw in ((w.grid_stencil((45, 38), seed=9), 45, {}),
                     (w.rmat_gcn(11, 16, seed=5), 64, {"long_row": 16, "segment": 32})):
        X = w.features(A.n, k, seed=k)
        M = arrow.ArrowMatrix(A, b, value_dtype=dt, **kw)
        Xd = torch.from_numpy(X).to("cuda", TORCH_DT[dt])
        Y = M.spmm(Xd, iters, relu=relu, rownorm=rownorm, rescale=rescale)
        torch.cuda.synchronize()
        Y = Y.float().cpu().numpy().astype(np.float64)
        R = S.iterate(A, X, iters, rescale=rescale, rectify=relu, rownorm=rownorm)
        if dt == "f32":
            assert err_inf(Y, R) <= 1e-5 * iters
        else:
            assert err_2(Y, R) <= 2e-2
        if relu and not rownorm:
            assert float(Y.min()) >= 0.0
        if rownorm and not rescale:
            nrm = np.linalg.norm(Y, axis=1)
            assert np.allclose(nrm[nrm > 0], 1.0, atol=1e-5 if dt == "f32" else 1e-2)


def test_sigma_rownorm_needs_one_team_per_row(arrow):
    from paper_2402_19364_gb300 import _native
    M = arrow.ArrowMatrix(w.grid2d_64(), 64)
    with pytest.raises(arrow.ArrowError) as e:
        M.spmm(torch.zeros(4096, 256, device="cuda"), 1, rownorm=True)   # 64 vectors of 16 B: two chunks
    assert e.value.code == _native.ARROW_EINVAL
    Y = M.spmm(torch.zeros(4096, 256, device="cuda"), 1, relu=True)    # the rectifier works per element
    assert torch.count_nonzero(Y).item() == 0


@pytest.mark.parametrize("dt,k,rescale", [("f32", 16, True), ("bf16", 128, False), ("f16", 32, False)])
def test_folded_permute_in_keeps_the_bits(arrow, dt, k, rescale):
    """The permute-in folded into the first iteration changes where the first step reads X
    from, not the arithmetic: results are bit-identical to the plain path and match the
    oracle; the caller's X is only read, and X and Y may still alias."""
    A = w.rmat_gcn(13, 16, seed=5)
    X = w.features(A.n, k, seed=3)
    M = arrow.ArrowMatrix(A, 128, value_dtype=dt, long_row=32, segment=128)
    Xd = torch.from_numpy(X).to("cuda", TORCH_DT[dt])
    t = M.tuning
    M.set_tuning(t["tile_rows"], t["tile_nnz"], t["ctas_per_sm"], t["carveout"], 0)
    ref = M.spmm(Xd, 6, rescale=rescale)
    M.set_tuning(t["tile_rows"], t["tile_nnz"], t["ctas_per_sm"], t["carveout"], 1)
    for iters in (6, 1):
        Xa = Xd.clone()
        Y = M.spmm(Xa, iters, rescale=rescale)
        torch.cuda.synchronize()
        assert torch.equal(Xa, Xd)                              # the caller's X is only read
        if iters == 6:
            assert torch.equal(Y, ref)
        M.spmm(Xa, iters, rescale=rescale, out=Xa)             # X and Y may alias with the fold
        assert torch.equal(Xa, Y)
    R = S.iterate(A, X, 6, rescale=rescale)
    Yn = ref.float().cpu().numpy().astype(np.float64)
    assert (err_inf(Yn, R) <= 6e-5) if dt == "f32" else (err_2(Yn, R) <= 2e-2)


@pytest.mark.parametrize("case", ["grid2d_f32", "rmat_split_bf16", "rgg_f16_k8", "grid_sigma_f32"])
def test_one_launch_path(arrow, case):
    """fused_small = 1: the whole call as one cooperative launch.  Without the rescale it gives
    the multi-launch path's bits (same row, segment and combine arithmetic); with it, the FP64
    column sums are grouped by its CTAs, so it agrees within the FP32 bar; both match the oracle."""
    kw, sig = {}, {}
    if case == "grid2d_f32":
        A, b, k, dt, it = w.grid2d_64(seed=1), 64, 16, "f32", 10
    elif case == "rmat_split_bf16":
        A, b, k, dt, it = w.rmat_gcn(12, 16, seed=5), 64, 128, "bf16", 5
        kw = {"long_row": 16, "segment": 48}
    elif case == "rgg_f16_k8":
        A = w.rgg(6000, seed=7)
        b, k, dt, it = int(np.ceil(np.sqrt(A.n))), 8, "f16", 10
    else:
        A, b, k, dt, it = w.grid_stencil((45, 38), seed=9), 45, 32, "f32", 6
        sig = {"relu": True, "rownorm": True}
    X = w.features(A.n, k, seed=11)
    M = arrow.ArrowMatrix(A, b, value_dtype=dt, **kw)
    if kw:
        assert M.stats()["segments"] > 0
    Xd = torch.from_numpy(X).to("cuda", TORCH_DT[dt])
    t = M.tuning
    for rescale in (False, True):
        M.set_tuning(t["tile_rows"], t["tile_nnz"], t["ctas_per_sm"], t["carveout"], 0, 0)
        ref = M.spmm(Xd, it, rescale=rescale, **sig)
        M.set_tuning(t["tile_rows"], t["tile_nnz"], t["ctas_per_sm"], t["carveout"], 0, 1)
        Y = M.spmm(Xd, it, rescale=rescale, **sig, profile=True)
        torch.cuda.synchronize()
        assert M.profile_get(arrow.ARROW_K_FUSED)[1] == 1          # the one-launch path ran
        assert M.profile_get(arrow.ARROW_K_ROWS)[1] == 0
        assert M.status() == 0
        Yn = Y.float().cpu().numpy().astype(np.float64)
        R = S.iterate(A, X, it, rescale=rescale, rectify=bool(sig), rownorm=bool(sig))
        if not rescale:
            assert torch.equal(Y, ref)
        if dt == "f32":
            assert err_inf(Yn, R) <= 1e-5 * it
            assert err_inf(Yn, ref.cpu().numpy().astype(np.float64)) <= 2e-5 * it
        else:
            assert err_2(Yn, R) <= 2e-2
        Xa = Xd.clone()
        M.spmm(Xa, it, rescale=rescale, out=Xa, **sig)               # X and Y may alias
        assert torch.equal(Xa, Y)


def test_iters_zero_alias_and_determinism(arrow):
    A = w.grid_stencil((37, 29), seed=9)            # ragged: n = 1073 is not a multiple of b
    X = w.features(A.n, 32, seed=10)
    M = arrow.ArrowMatrix(A, 16)
    Xd = torch.from_numpy(X).cuda()
    Y0 = M.spmm(Xd, 0)
    assert torch.equal(Y0, Xd)
    Y1 = M.spmm(Xd, 7)
    Y2 = M.spmm(Xd, 7)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)                       # fixed accumulation order: bit-identical
    Xa = Xd.clone()
    M.spmm(Xa, 7, out=Xa)                            # X and Y may alias
    assert torch.equal(Xa, Y1)
    ws = torch.empty(M.workspace_size(32, "f32"), dtype=torch.uint8, device="cuda")
    Y3 = M.spmm_ws(Xd, 7, ws)
    torch.cuda.synchronize()
    assert torch.equal(Y3, Y1)
    assert err_inf(Y1.cpu().numpy().astype(np.float64), S.iterate(A, X, 7)) <= 7e-5


def test_empty_and_single_level(arrow):
    n = 640
    A0 = w.Csr(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    M = arrow.ArrowMatrix(A0, 8)
    Xd = torch.randn(n, 16, device="cuda")
    assert torch.count_nonzero(M.spmm(Xd, 3)).item() == 0
    A = w.random_csr(300, 0.02, 3, symmetric=True, diag=True)
    X = w.features(A.n, 16, seed=1)
    M, _, Y = run(arrow, A, 512, X, 5)               # b >= n: one level, all rows are head rows
    assert M.num_levels == 1
    assert err_inf(Y, S.iterate(A, X, 5)) <= 5e-5


def test_nonsymmetric_matrix(arrow):
    A = w.random_csr(2000, 0.002, 11)
    X = w.features(A.n, 16, seed=3)
    _, _, Y = run(arrow, A, 32, X, 3)
    assert err_inf(Y, S.iterate(A, X, 3)) <= 3e-5


def test_argument_errors(arrow):
    from paper_2402_19364_gb300 import _native
    M = arrow.ArrowMatrix(w.grid2d_64(), 64)
    with pytest.raises(arrow.ArrowError) as e:
        M.spmm(torch.zeros(4096, 12, device="cuda"), 1)       # 3 vectors of 16 B: not a power of two
    assert e.value.code == _native.ARROW_EINVAL
    M.spmm(torch.zeros(4096, 16, device="cuda", dtype=torch.bfloat16), 1)   # f32 values, bf16 X: allowed
    Mb = arrow.ArrowMatrix(w.grid2d_64(), 64, value_dtype="bf16")
    with pytest.raises(arrow.ArrowError) as e:
        Mb.spmm(torch.zeros(4096, 16, device="cuda"), 1)      # bf16 values need 16-bit features
    assert e.value.code == _native.ARROW_EINVAL
    big = torch.zeros(4096 * 16 + 1, device="cuda")
    L = _native.lib()
    rc = L.arrow_spmm(M._h, _native.ctypes.c_void_p(big.data_ptr() + 4), 16, 1,
                      _native.ctypes.c_void_p(big.data_ptr()), 0, 0, None)
    assert rc == _native.ARROW_EINVAL                          # misaligned X


def test_profile_events(arrow):
    A = w.grid3d(20)
    M = arrow.ArrowMatrix(A, 64)
    Xd = torch.randn(A.n, 16, device="cuda")
    M.spmm(Xd, 5, rescale=True, profile=True)
    ms, cnt = M.profile_get(arrow.ARROW_K_ROWS)
    assert cnt == 5 and ms > 0
    assert M.profile_get(arrow.ARROW_K_NORM)[1] == 5
    assert M.profile_get(arrow.ARROW_K_PERMUTE)[1] == 2
    assert M.profile_get(arrow.ARROW_K_ROWS)[1] == 0           # read once, then forgotten


def test_status_word_and_bounded_wait_selftest(arrow):
    import ctypes
    import time
    from paper_2402_19364_gb300 import _native
    A = w.grid3d(16)
    M = arrow.ArrowMatrix(A, 64)
    M.spmm(torch.randn(A.n, 16, device="cuda"), 3)
    assert M.status() == 0                                     # no wait ran out
    st = ctypes.c_int32(-1)
    t0 = time.time()
    _native.check(_native.lib().arrow_selftest_timeout(50_000_000, ctypes.byref(st)))
    assert st.value == 1 and time.time() - t0 < 5.0            # gave up after ~50 ms, reported it
    # the one-launch path's grid barrier: one block never arrives, the other 15 give up
    gave = ctypes.c_int32(-1)
    t0 = time.time()
    _native.check(_native.lib().arrow_selftest_grid_timeout(50_000_000, 16, ctypes.byref(gave)))
    assert gave.value == 15 and time.time() - t0 < 5.0
    Y = M.spmm(torch.ones(A.n, 16, device="cuda"), 2)          # context still usable
    assert torch.allclose(Y, torch.ones_like(Y), atol=1e-5)


def test_saved_handle_gives_same_bits(arrow, tmp_path):
    A = w.rmat_gcn(11, 16, seed=2)
    M = arrow.ArrowMatrix(A, 64, long_row=32)
    M.save(tmp_path / "a.arw")
    L = arrow.ArrowMatrix.load(tmp_path / "a.arw")
    Xh = w.features(A.n, 32, seed=5)
    X = torch.from_numpy(Xh).cuda()
    YL = L.spmm(X, 4)
    assert torch.equal(M.spmm(X, 4), YL)
    # the loaded handle against the oracle, not only against the handle it was saved from
    R = S.iterate(A, Xh, 4)
    assert err_inf(YL.cpu().numpy().astype(np.float64), R) <= 1e-5 * 4
    Lb = arrow.ArrowMatrix.load(tmp_path / "a.arw", value_dtype="bf16")
    Yb = Lb.spmm(X.bfloat16(), 4).float()
    assert err_2(Yb.cpu().numpy().astype(np.float64), R) <= 2e-2
    Yf = M.spmm(X, 4)
    assert float(torch.linalg.vector_norm(Yb - Yf) / torch.linalg.vector_norm(Yf)) < 2e-2


def test_device_arguments(arrow):
    """The upload goes to opts.device and leaves the caller's current device as it was; an
    ordinal with no GPU is an error and gives no handle; calls on a handle whose device is
    not current return ARROW_EINVAL and launch nothing (that last part needs two GPUs)."""
    from paper_2402_19364_gb300 import _native
    A = w.grid2d_64(seed=1)
    X = w.features(A.n, 16, seed=2)
    cur = torch.cuda.current_device()
    M = arrow.ArrowMatrix(A, 64, device=cur)
    assert torch.cuda.current_device() == cur
    Y = M.spmm(torch.from_numpy(X).cuda(), 3).cpu().numpy().astype(np.float64)
    assert err_inf(Y, S.iterate(A, X, 3)) <= 3e-5
    with pytest.raises(arrow.ArrowError) as e:
        arrow.ArrowMatrix(A, 64, device=torch.cuda.device_count())
    assert e.value.code in (_native.ARROW_ECUDA, _native.ARROW_EINVAL)
    assert torch.cuda.current_device() == cur
    if torch.cuda.device_count() < 2:
        return
    other = (cur + 1) % torch.cuda.device_count()
    M1 = arrow.ArrowMatrix(A, 64, device=other)
    assert torch.cuda.current_device() == cur
    with torch.cuda.device(other):
        X1 = torch.from_numpy(X).cuda()
        Y1 = torch.empty_like(X1)
    L = _native.lib()
    for fn in (L.arrow_spmm, L.arrow_spmm_static):
        rc = fn(M1._h, _native.ctypes.c_void_p(X1.data_ptr()), 16, 2, _native.ctypes.c_void_p(Y1.data_ptr()),
                _native.ARROW_F32, 0, None)
        assert rc == _native.ARROW_EINVAL
        assert b"current" in L.arrow_last_error()


# ---- full-size workloads (the launch configuration bench.py times) -----------------------

def _sample_rows(n, count, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.r_[0, n - 1, rng.integers(0, n, count)])


def _oracle_columns(A, X, cols, iters, rescale=False):
    """Every row of the columns `cols` of the oracle's result.  The columns of X_{t+1} =
    sigma(A X_t) are independent (A acts on each column alone and the rescale divides each
    column by its own norm), so the multi-core FP64 oracle run on those columns of X gives
    exactly those columns of the full result."""
    from oracle import cspmm as C
    return C.iterate(A, np.ascontiguousarray(X[:, cols], dtype=np.float64), iters, rescale=rescale)


def test_full_size_grid3d_400(arrow):
    """3D 400^3 7-point grid (n = 64M, nnz = 447.04M), b = 4096, k = 16 f32, 20 iterations.

    Every row of four columns is compared with the multi-core FP64 oracle, with and without
    the rescale; sampled rows are also computed by the oracle one by one (dependency cone of
    20 hops); with the rescale on, the column of ones must stay constant and every column has
    unit norm.
    """
    A = w.grid3d(400, seed=3)
    assert A.n == 64_000_000 and A.nnz == 447_040_000
    M = arrow.ArrowMatrix(A, 4096)
    X = w.features(A.n, 16, seed=4)
    X[:, 0] = 1.0
    Xd = torch.from_numpy(X).cuda()
    Y = M.spmm(Xd, 20)
    rows = _sample_rows(A.n, 48, 1)
    Ys = Y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    R = S.iterate_rows(A, X, 20, rows)
    assert np.max(np.abs(Ys - R)) <= 1e-5 * 20 * np.max(np.abs(R))
    assert np.max(np.abs(Ys[:, 0] - 1.0)) <= 1e-5 * 20            # A row-normalised: A^t 1 = 1
    Yr = M.spmm(Xd, 20, rescale=True)
    nrm = torch.linalg.vector_norm(Yr.double(), dim=0).cpu().numpy()
    assert np.allclose(nrm, 1.0, atol=1e-5)
    c0 = Yr[:, 0].double()
    assert float((c0 * np.sqrt(A.n) - 1.0).abs().max()) <= 1e-5 * 20
    # the rescaled result is A^20 X times one factor per column: fit it, compare the rows
    Yrs = Yr[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    c = np.sum(Yrs * R, axis=0) / np.sum(R * R, axis=0)
    assert err_inf(Yrs, R * c) <= 1e-5 * 20
    # every row of four columns against the oracle (FP32 bar: 1e-5 * iters, inf-norm per column)
    cols = [0, 3, 9, 14]
    ci = torch.tensor(cols, device="cuda")
    Yc = Y.index_select(1, ci).cpu().numpy().astype(np.float64)
    Yrc = Yr.index_select(1, ci).cpu().numpy().astype(np.float64)
    del Y, Yr
    assert err_inf(Yc, _oracle_columns(A, X, cols, 20)) <= 1e-5 * 20
    assert err_inf(Yrc, _oracle_columns(A, X, cols, 20, rescale=True)) <= 1e-5 * 20


def test_full_size_rmat23_gcn_bf16(arrow):
    """R-MAT scale 23 (n = 8.39M), symmetrised, self-loops, GCN-normalised; b = 8192; k = 128;
    8 iterations in BF16 storage with FP32 accumulation and in FP32.

    Every row of eight columns (the d^{1/2} column and seven others) is compared with the
    multi-core FP64 oracle: within 1e-5 * iters (inf-norm, relative) in FP32 and 2e-2
    (normwise) in BF16.  A . d^{1/2} = d^{1/2} holds for the GCN normalisation at any size, so
    the column set to d^{1/2} must also come back unchanged; on all 128 columns the two paths
    agree normwise within 2e-2.
    """
    A = w.rmat_gcn(23, 16, seed=5)
    assert A.n == 1 << 23
    M16 = arrow.ArrowMatrix(A, 8192, value_dtype="bf16")
    M32 = M16.copy("f32")
    assert M16.stats()["long_rows"] > 0
    X = w.features(A.n, 128, seed=6)
    d = np.sqrt(np.diff(A.rowptr).astype(np.float64))
    X[:, 0] = d
    cols = [0, 1, 17, 42, 63, 64, 101, 127]
    Xf = torch.from_numpy(X).cuda()
    Xc = np.ascontiguousarray(X[:, cols])
    del X
    iters = 8
    Yf = M32.spmm(Xf, iters)
    Yb = M16.spmm(Xf.bfloat16(), iters).float()
    dd = torch.from_numpy(d).cuda()
    assert float((Yf[:, 0].double() - dd).abs().max() / dd.max()) <= 1e-5 * iters
    assert float(torch.linalg.vector_norm(Yb[:, 0].double() - dd) / torch.linalg.vector_norm(dd)) <= 2e-2
    rel = torch.linalg.vector_norm(Yb - Yf, dim=0) / torch.linalg.vector_norm(Yf, dim=0)
    assert float(rel.max()) <= 2e-2
    ci = torch.tensor(cols, device="cuda")
    Yfc = Yf.index_select(1, ci).cpu().numpy().astype(np.float64)
    Ybc = Yb.index_select(1, ci).cpu().numpy().astype(np.float64)
    del Yf, Yb, Xf
    R = _oracle_columns(A, Xc, list(range(len(cols))), iters)
    assert err_inf(Yfc, R) <= 1e-5 * iters
    assert err_2(Ybc, R) <= 2e-2
