"""Host-side tests of the C-ABI library (no GPU): exports, error codes, decomposer parity.

The library's C++ decomposer and the oracle share no code; they must agree
bit-exactly on permutations, per-level CSR structure, values, active rows and
nonzero counts (both follow the same reading of LA-Decompose).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as w
from oracle import decompose as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def arrow():
    from paper_2402_19364_gb300 import build
    build.build()
    import paper_2402_19364_gb300 as pkg
    return pkg


def test_library_exports_every_declared_symbol(arrow):
    from paper_2402_19364_gb300 import _native
    with open(os.path.join(ROOT, "include", "arrow.h")) as f:
        hdr = f.read()
    declared = set(re.findall(r"\b(arrow_[a-z_0-9]+)\s*\(", hdr))
    assert "arrow_spmm" in declared and "arrow_decompose" in declared
    lib = ctypes.CDLL(str(_native.LIB_PATH))
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(_native.SIGNATURES), declared - set(_native.SIGNATURES)


def _parity(arrow, A, b, seed=0, **kw):
    M = arrow.ArrowMatrix(A, b, seed=seed, host_only=True, **kw)
    L = D.la_decompose(A, b, seed=seed)
    assert M.num_levels == len(L)
    for i, lv in enumerate(L):
        assert np.array_equal(M.level_perm(i), lv.perm)
        rp, ci, vv = M.level_csr(i)
        assert np.array_equal(rp, lv.rowptr)
        assert np.array_equal(ci, lv.colidx)
        assert np.array_equal(vv, lv.values)
        assert M.level_info(i) == (lv.n_active, lv.nnz)
        sh = M.level_shape(i)
        assert (sh["head_nnz"], sh["band_nnz"], sh["tiles"]) == D.level_shape(lv)
        assert (sh["n_active"], sh["nnz"]) == (lv.n_active, lv.nnz)
    return M


@pytest.mark.parametrize("case", ["grid2d_64", "grid3d_24", "rmat12", "rgg", "nonsym", "star", "b_ge_n"])
def test_decomposer_matches_oracle(arrow, case):
    if case == "grid2d_64":
        M = _parity(arrow, w.grid2d_64(), 64)                       # 2D 64x64, b = 64
        assert M.num_levels >= 2
    elif case == "grid3d_24":
        _parity(arrow, w.grid3d(24), 96, seed=3)                   # 3D 7-point, scaled down
    elif case == "rmat12":
        _parity(arrow, w.rmat_gcn(12, 16, seed=5), 128, seed=5)     # power law, GCN-normalised
    elif case == "rgg":
        A = w.rgg(3000, seed=7)
        _parity(arrow, A, int(np.ceil(np.sqrt(A.n))), seed=7)      # random geometric, b = ceil(sqrt n)
    elif case == "nonsym":
        _parity(arrow, w.random_csr(400, 0.01, 8), 4, seed=2)
    elif case == "star":
        n = 300
        rows = np.r_[np.zeros(n - 1, np.int64), np.arange(1, n)]
        cols = np.r_[np.arange(1, n), np.zeros(n - 1, np.int64)]
        rp, ci = w._csr_from_pairs(n, rows, cols)
        _parity(arrow, w.Csr(n, rp, ci, np.linspace(1, 2, ci.size)), 2)
    else:
        M = _parity(arrow, w.random_csr(50, 0.1, 1, symmetric=True, diag=True), 64)
        assert M.num_levels == 1


def test_decomposer_thread_count_invariant(arrow):
    A = w.grid3d(40)
    ms = [arrow.ArrowMatrix(A, 512, seed=9, host_only=True, nthreads=t) for t in (1, 3, 8)]
    for i in range(ms[0].num_levels):
        p = ms[0].level_perm(i)
        for m in ms[1:]:
            assert m.num_levels == ms[0].num_levels
            assert np.array_equal(m.level_perm(i), p)
            assert m.level_info(i) == ms[0].level_info(i)


def test_empty_and_degenerate_inputs(arrow):
    M = arrow.ArrowMatrix(w.Csr(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)), 2, host_only=True)
    assert M.num_levels == 0
    M = arrow.ArrowMatrix(w.Csr(5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0)), 2, host_only=True)
    assert M.num_levels == 0 and M.stats()["nnz"] == 0


def _bad(arrow, A, b, **kw):
    with pytest.raises(arrow.ArrowError) as e:
        arrow.ArrowMatrix(A, b, host_only=True, **kw)
    return e.value


def test_invalid_inputs_rejected(arrow):
    from paper_2402_19364_gb300 import _native
    A = w.grid2d_64()
    assert _bad(arrow, A, 1).code == _native.ARROW_EINVAL                     # b < 2 (Section 4.1)
    bad = w.Csr(A.n, A.rowptr.copy(), A.colidx.copy(), A.values)
    bad.colidx[5] = A.n                                                      # column out of range
    assert _bad(arrow, bad, 8).code == _native.ARROW_EINVAL
    bad = w.Csr(A.n, A.rowptr.copy(), A.colidx.copy(), A.values)
    bad.colidx[1], bad.colidx[2] = bad.colidx[2], bad.colidx[1]              # unsorted row
    assert _bad(arrow, bad, 8).code == _native.ARROW_EINVAL
    bad = w.Csr(A.n, A.rowptr.copy(), A.colidx, A.values)
    bad.rowptr[10] = bad.rowptr[12]                                          # non-monotone rowptr
    assert _bad(arrow, bad, 8).code == _native.ARROW_EINVAL
    assert "strictly increasing" in _bad(arrow, w.Csr(3, np.array([0, 2, 2, 2]), np.array([1, 1], np.int32),
                                                      np.ones(2)), 2).args[0]
    assert _bad(arrow, A, 8, max_levels=1).code == _native.ARROW_EINVAL      # level cap
    # size limits of the int32 indices: n and nnz below 2^31, checked before any array is read
    import ctypes
    L = _native.lib()
    o = _native.ArrowOpts()
    L.arrow_opts_default(ctypes.byref(o))
    o.flags = _native.ARROW_HOST_ONLY
    h = ctypes.c_void_p()
    for n, nnz in ((1 << 31, 0), (4, 1 << 31), (-1, 0), (4, -1)):
        csr = _native.ArrowCsr(n, nnz, None, None, None)
        assert L.arrow_decompose(ctypes.byref(csr), 8, ctypes.byref(o), ctypes.byref(h)) == _native.ARROW_EINVAL
        assert not h.value
        t = ctypes.c_int64()
        assert L.arrow_count_tiles(ctypes.byref(csr), 8, ctypes.byref(t)) == _native.ARROW_EINVAL


def test_state_errors_without_gpu(arrow):
    from paper_2402_19364_gb300 import _native
    M = arrow.ArrowMatrix(w.grid2d_64(), 64, host_only=True)
    L = _native.lib()
    rc = L.arrow_spmm(M._h, ctypes.c_void_p(16), 16, 1, ctypes.c_void_p(16), 0, 0, None)
    assert rc == _native.ARROW_ESTATE                                        # not uploaded
    sz = ctypes.c_size_t()
    assert L.arrow_workspace_size(M._h, 16, 0, 0, ctypes.byref(sz)) == _native.ARROW_ESTATE
    L.arrow_free(None)                                                       # NULL-safe
    assert L.arrow_level_info(M._h, 99, None, None) == _native.ARROW_EINVAL


def test_band_predicate_matches_oracle(arrow):
    A = w.grid_stencil((20, 20), seed=4)
    M = arrow.ArrowMatrix(A, 5, seed=1, host_only=True, predicate="band")
    L = D.la_decompose(A, 5, seed=1, predicate=D.pred_band)
    assert M.num_levels == len(L)
    for i, lv in enumerate(L):
        assert np.array_equal(M.level_perm(i), lv.perm)
        assert M.level_info(i) == (lv.n_active, lv.nnz)
        sh = M.level_shape(i)
        assert (sh["head_nnz"], sh["band_nnz"], sh["tiles"]) == D.level_shape(lv)


def test_count_tiles_and_structure_report(arrow):
    cases = [(w.grid2d_64(), 64), (w.grid_stencil((13, 13), seed=2), 13), (w.rmat_gcn(10, 16, seed=5), 32),
             (w.random_csr(300, 0.02, 3), 7), (w.grid3d(12), 144)]
    for A, b in cases:
        for bb in (b, 1, 5, A.n, 10 * A.n):
            assert arrow.count_tiles(A, bb) == D.count_tiles(A, bb)
    assert arrow.count_tiles(w.grid_stencil((13, 13), seed=2), 13) == 3 * 13 - 2
    A = w.grid2d_64()
    M = arrow.ArrowMatrix(A, 64, host_only=True)
    rep = M.structure_report()
    assert len(rep["levels"]) == M.num_levels
    assert sum(lv["nnz"] for lv in rep["levels"]) == A.nnz
    assert rep["tiles"] == sum(D.level_shape(lv)[2] for lv in D.la_decompose(A, 64))
    with pytest.raises(arrow.ArrowError):
        arrow.count_tiles(A, 0)
    with pytest.raises(arrow.ArrowError):
        M.level_shape(M.num_levels)
    bad = w.Csr(A.n, A.rowptr, A.colidx[::-1].copy(), A.values)          # columns not increasing
    with pytest.raises(arrow.ArrowError):
        arrow.count_tiles(bad, 8)


def test_fused_program_stats(arrow):
    A = w.rmat_gcn(12, 16, seed=5)
    M = arrow.ArrowMatrix(A, 128, host_only=True, long_row=32, segment=64)
    s = M.stats()
    deg = np.diff(A.rowptr)
    assert s["long_rows"] == int((deg > 32).sum())
    assert s["segments"] == int(np.sum((deg[deg > 32] + 63) // 64))
    assert s["tiles"] >= (A.n + 255) // 256                  # at most 256 rows per tile


def test_save_load_roundtrip_and_corruption(arrow, tmp_path):
    from paper_2402_19364_gb300 import _native
    A = w.rmat_gcn(11, 16, seed=4)
    M = arrow.ArrowMatrix(A, 64, seed=3, host_only=True, long_row=16)
    p = tmp_path / "m.arw"
    M.save(p)
    L2 = arrow.ArrowMatrix.load(p, host_only=True)
    assert L2.num_levels == M.num_levels and L2.stats()["segments"] == M.stats()["segments"]
    for i in range(M.num_levels):
        assert np.array_equal(L2.level_perm(i), M.level_perm(i))
        assert L2.level_info(i) == M.level_info(i)
        for x, y in zip(L2.level_csr(i), M.level_csr(i)):
            assert np.array_equal(x, y)
    raw = bytearray(p.read_bytes())
    raw[len(raw) // 2] ^= 0xFF                                   # flip a byte: checksum fails
    bad = tmp_path / "bad.arw"
    bad.write_bytes(bytes(raw))
    with pytest.raises(arrow.ArrowError) as e:
        arrow.ArrowMatrix.load(bad, host_only=True)
    assert e.value.code == _native.ARROW_EINVAL
    short = tmp_path / "short.arw"
    short.write_bytes(p.read_bytes()[:1000])                      # truncated
    with pytest.raises(arrow.ArrowError):
        arrow.ArrowMatrix.load(short, host_only=True)
    with pytest.raises(arrow.ArrowError):
        arrow.ArrowMatrix.load(tmp_path / "missing.arw", host_only=True)


def test_tuning_retiles_and_validates(arrow):
    A = w.grid3d(30)
    M = arrow.ArrowMatrix(A, 256, host_only=True)
    t = M.tuning
    assert (t["tile_rows"], t["tile_nnz"], t["ctas_per_sm"], t["carveout"]) == (256, 2048, 4, 70)
    n_default = M.stats()["tiles"]
    M.set_tuning(128, 1024, 2, 50)
    assert M.tuning["tile_rows"] == 128 and M.stats()["tiles"] > n_default
    assert M.stats()["tiles"] >= (A.n + 127) // 128
    for bad in ((16, 1024, 2, 50), (128, 512, 2, 50), (128, 1024, 5, 50), (128, 1024, 2, 101), (4096, 1024, 2, 50)):
        with pytest.raises(arrow.ArrowError):
            M.set_tuning(*bad)
    assert M.tuning["tile_rows"] == 128                      # unchanged after rejected values


def test_structure_report_cli(arrow, capsys):
    from paper_2402_19364_gb300 import report
    report.main(["--workload", "grid2d", "--size", "24", "--b", "24", "--predicate", "both"])
    import json
    out = json.loads(capsys.readouterr().out)
    A = w.grid_stencil((24, 24), seed=3)
    assert out["n"] == A.n and out["nnz"] == A.nnz and len(out["reports"]) == 2
    for r, pred in zip(out["reports"], (D.pred_block, D.pred_band)):
        L = D.la_decompose(A, 24, seed=3, predicate=pred)
        assert [(lv["head_nnz"], lv["band_nnz"], lv["tiles"]) for lv in r["levels"]] == [D.level_shape(x) for x in L]
        assert r["tiles_input_order"] == D.count_tiles(A, 24) == 3 * 24 - 2


def test_closed_matrix_guard(arrow):
    # batches hold raw handle pointers: the binding refuses a batch call once a member is closed
    A = w.grid2d_64()
    Ms = [arrow.ArrowMatrix(A, 64, host_only=True) for _ in range(2)]
    arrow._check_open(Ms, "test")
    Ms[1].close()
    with pytest.raises(arrow.ArrowError) as ei:
        arrow._check_open(Ms, "arrow_batch_spmm")
    assert ei.value.code == -5
    Ms[0].close()


def test_injected_host_allocation_failure(arrow, monkeypatch):
    # a failed host allocation in the middle of LA-Decompose surfaces as ARROW_ENOMEM with no
    # handle returned, and the next decomposition is unaffected
    from paper_2402_19364_gb300 import _native
    A = w.grid2d_64()
    for level in (0, 1, 2):
        monkeypatch.setenv("ARROW_INJECT_HOST_ALLOC_FAILURE", str(level))
        for _ in range(20):
            with pytest.raises(arrow.ArrowError) as ei:
                arrow.ArrowMatrix(A, 64, host_only=True)
            assert ei.value.code == _native.ARROW_ENOMEM and "allocation" in str(ei.value)
    monkeypatch.setenv("ARROW_INJECT_HOST_ALLOC_FAILURE", "99")     # past the last level: no failure
    M = arrow.ArrowMatrix(A, 64, host_only=True)
    monkeypatch.delenv("ARROW_INJECT_HOST_ALLOC_FAILURE")
    ref = D.la_decompose(A, 64)
    assert M.num_levels == len(ref) and np.array_equal(M.level_perm(0), ref[0].perm)
