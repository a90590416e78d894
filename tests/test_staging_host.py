"""CPU check of the rows kernel's tile staging arithmetic on real tile tables (no GPU).

For every tile of a handle's program, under several tunings, the byte ranges that the bulk
copies move are recomputed the way the staging code does (16-byte aligned supersets of the
tile's row pointers, columns and values) and checked to fit the shared-memory regions of the
tile layout and to stay inside the device arrays, which are padded by 64 bytes; the reads
the kernel then makes at the misaligned offsets (r0 & 3, e0 & 3, e0 & (16/s - 1)) must stay
inside the staged ranges.
"""
import numpy as np
import pytest

import workloads as w

PAD = 64   # bytes every device array is padded by


@pytest.fixture(scope="module")
def arrow():
    from paper_2402_19364_gb300 import build
    build.build()
    import paper_2402_19364_gb300 as pkg
    return pkg


def _layout(tile_rows, tile_nnz):
    rp = ((tile_rows + 1 + 6) * 4 + 15) // 16 * 16
    col = ((tile_nnz + 8) * 4 + 15) // 16 * 16
    buf = (rp + 2 * col + 127) // 128 * 128
    return rp, col, buf


@pytest.mark.parametrize("tuning", [(256, 2048), (128, 1024), (384, 3072), (512, 4096), (2048, 8192), (32, 1024)])
def test_staged_ranges_fit(arrow, tuning):
    mats = [(w.grid3d(16), 256, {}), (w.rmat_gcn(10, 16, seed=4), 32, {"long_row": 16, "segment": 64}),
            (w.rgg(5000, seed=3), 71, {}), (w.grid_stencil((37, 29), seed=1), 37, {})]
    for A, b, kw in mats:
        M = arrow.ArrowMatrix(A, b, host_only=True, **kw)
        M.set_tuning(tuning[0], tuning[1], 3, 70)
        pg = M.program()
        rp_bytes, col_bytes, buf = _layout(*tuning)
        n, n_short = A.n, pg["col"].size
        tr, te = pg["tile_row"].astype(np.int64), pg["tile_ent"].astype(np.int64)
        for s in (4, 2):                                   # value bytes: f32, 16-bit
            ve = 16 // s
            for t in range(tr.size - 1):
                r0, r1, e0, e1 = tr[t], tr[t + 1], te[t], te[t + 1]
                ra, rb = r0 & ~3, (r1 + 1 + 3) & ~3
                ca, cb = e0 & ~3, (e1 + 3) & ~3
                va, vb = e0 & ~(ve - 1), (e1 + ve - 1) & ~(ve - 1)
                brp, bcol, bval = (rb - ra) * 4, (cb - ca) * 4, (vb - va) * s
                # the staged regions fit the buffer's layout
                assert brp <= rp_bytes and bcol <= col_bytes and bval <= buf - rp_bytes - col_bytes
                # every copy is 16-byte sized and starts 16-byte aligned in the source
                assert brp % 16 == 0 and bcol % 16 == 0 and bval % 16 == 0
                assert (ra * 4) % 16 == 0 and (ca * 4) % 16 == 0 and (va * s) % 16 == 0
                # the sources stay inside the padded device arrays
                assert rb * 4 <= (n + 1) * 4 + PAD and cb * 4 <= n_short * 4 + PAD and vb * s <= n_short * s + PAD
                # the kernel's reads at the misaligned offsets stay inside what was staged
                assert (r0 - ra) + (r1 - r0) < rb - ra                 # srp[0 .. nrows]
                if e1 > e0:
                    assert (e0 - ca) + (e1 - e0) <= cb - ca           # scol[0 .. e1-e0)
                    assert (e0 - va) + (e1 - e0) <= vb - va           # sval[0 .. e1-e0)
        M.close()


def test_oversized_tile_rejected(arrow):
    # two staging buffers of a 2048-row / 16384-entry tile do not fit 227 KB of shared memory
    M = arrow.ArrowMatrix(w.grid2d_64(), 64, host_only=True)
    with pytest.raises(arrow.ArrowError):
        M.set_tuning(2048, 16384, 3, 70)
