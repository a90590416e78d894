"""GPU test of arrow_spmm_static, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc: plugins inside a framework that owns all device memory
through its own allocator, and serving loops that forbid allocation after start-up (cudaMalloc
and cudaFree synchronise the device).  arrow_spmm_static keeps its scratch in a fixed 64 MiB
device array of the library instead.  This file is collected last so that, should it fail, a run stopping at
the first failure has already run every other test.  It checks, through the C-ABI, that two
calls in a row give the result of arrow_spmm within the FP32 tolerance of the parity tests
(max over columns of ||y - y_ref||_inf / ||y_ref||_inf <= 1e-5 * iters), and that a
problem too large for the array is refused, and that calls after the first leave the device's
free memory unchanged.
"""
import ctypes

import numpy as np
import pytest

import workloads as w

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


def _rel_inf(Y, R):
    Y = Y.double().cpu().numpy()
    R = R.double().cpu().numpy()
    return float(np.max(np.max(np.abs(Y - R), axis=0) / np.max(np.abs(R), axis=0)))


@pytest.mark.parametrize("rescale", [False, True])
def test_static_scratch_matches_arrow_spmm(arrow, rescale):
    from paper_2402_19364_gb300 import _native
    L = _native.lib()
    A = w.rmat_gcn(12, 16, seed=5)                    # power law: split rows use the scratch too
    M = arrow.ArrowMatrix(A, 128, long_row=16, segment=64)
    iters = 6
    flags = _native.ARROW_RESCALE if rescale else 0
    for k in (16, 64):
        X = torch.from_numpy(w.features(A.n, k, seed=k)).cuda()
        ref = M.spmm(X, iters, rescale=rescale)
        for _ in range(2):                            # two calls in a row share the array
            Y = torch.full_like(X, float("nan"))
            stream = torch.cuda.current_stream()
            _native.check(L.arrow_spmm_static(M._h, ctypes.c_void_p(X.data_ptr()), k, iters,
                                              ctypes.c_void_p(Y.data_ptr()), _native.ARROW_F32, flags,
                                              ctypes.c_void_p(stream.cuda_stream)))
            torch.cuda.synchronize()
            assert _rel_inf(Y, ref) <= 1e-5 * iters


def test_static_scratch_allocates_nothing(arrow):
    """After a first call (which looks the array's address up), further calls leave the
    device's free memory exactly as it was: the scratch is the library's fixed array."""
    from paper_2402_19364_gb300 import _native
    L = _native.lib()
    A = w.rmat_gcn(12, 16, seed=5)
    M = arrow.ArrowMatrix(A, 128, long_row=16, segment=64)
    X = torch.from_numpy(w.features(A.n, 32, seed=1)).cuda()
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()

    def call():
        _native.check(L.arrow_spmm_static(M._h, ctypes.c_void_p(X.data_ptr()), 32, 4, ctypes.c_void_p(Y.data_ptr()),
                                          _native.ARROW_F32, _native.ARROW_RESCALE,
                                          ctypes.c_void_p(stream.cuda_stream)))

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_one_launch_path(arrow):
    """The one-launch path (tuning fused_small) through the static scratch: the same bits as
    arrow_spmm on that path, two calls in a row."""
    from paper_2402_19364_gb300 import _native
    L = _native.lib()
    A = w.grid2d_64(seed=1)
    M = arrow.ArrowMatrix(A, 64)
    t = M.tuning
    M.set_tuning(t["tile_rows"], t["tile_nnz"], t["ctas_per_sm"], t["carveout"], 0, 1)
    X = torch.from_numpy(w.features(A.n, 16, seed=2)).cuda()
    ref = M.spmm(X, 10, rescale=True)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        _native.check(L.arrow_spmm_static(M._h, ctypes.c_void_p(X.data_ptr()), 16, 10, ctypes.c_void_p(Y.data_ptr()),
                                          _native.ARROW_F32, _native.ARROW_RESCALE,
                                          ctypes.c_void_p(stream.cuda_stream)))
        torch.cuda.synchronize()
        assert torch.equal(Y, ref)


def test_static_scratch_refuses_large_problems(arrow):
    from paper_2402_19364_gb300 import _native
    L = _native.lib()
    A = w.grid3d(100)                                 # 1M rows x 16 f32: 128 MB of scratch
    M = arrow.ArrowMatrix(A, 4096)
    X = torch.zeros(A.n, 16, device="cuda")
    Y = torch.zeros_like(X)
    rc = L.arrow_spmm_static(M._h, ctypes.c_void_p(X.data_ptr()), 16, 2, ctypes.c_void_p(Y.data_ptr()),
                             _native.ARROW_F32, 0, None)
    assert rc == _native.ARROW_EINVAL
    assert b"static" in L.arrow_last_error()
