"""CPU checks of bench.py's helpers: the Table 1 fixture reader, the symmetry
images used to compare a found sequence with Table 1's, and the work unit of
the roofline accounting."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_table1_rows_read_the_fixture():
    rows = bench.table1_rows()
    assert len(rows) == 17
    assert rows[171][0] == 1669 and rows[247][0] == 3259 and rows[247][2] == 13.0


def test_symmetry_images_keep_energy_and_skew_symmetry(oracle_mod):
    import paper_2210_15962_gb300 as m
    for L, (E, _, _, hx) in bench.table1_rows().items():
        s = m.from_hex(hx, L)
        imgs = bench.symmetry_orbit(s)
        assert len(imgs) == 8 and any(np.array_equal(i, s) for i in imgs)
        D = (L + 1) // 2
        for i in imgs:
            assert oracle_mod.energy(i) == E
            assert np.array_equal(oracle_mod.skew_expand(i[:D], L), i)  # still skew-symmetric
        assert len({i.tobytes() for i in imgs}) >= 4


def test_roofline_unit_counts_the_lags_of_each_space():
    # 4 LOP3 per 32 lags and digit plane: (L-1)/2 even lags of a skew sequence, L-1 lags in the full space
    assert bench.core_alu_ops_per_eval(121, 5.0) == 4.0 * 5.0 * 60 / 32
    assert bench.core_alu_ops_per_eval(121, 5.0, full=True) == 4.0 * 5.0 * 120 / 32
